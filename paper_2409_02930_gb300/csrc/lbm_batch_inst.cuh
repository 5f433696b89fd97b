// Instantiates the batched-form kernels for one precision; the including file
// defines LBM_REAL and LBM_BATCH_OPS_NAME.
#include "lbm_batch.cuh"

namespace lbm {
namespace {

template <class R, int D, int M, bool EN>
struct BatchLaunch {
  static constexpr int kTiles[3] = {64, 128, 256};
  static int tile(int v) { return kTiles[v / 2]; }
  template <int TB>
  static int occ() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch<R, D, M, EN, TB, false>, TB, 0) != cudaSuccess) a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<R, D, M, EN, TB, true>, TB, 0) != cudaSuccess) b = 1;
    return a < b ? (a > 0 ? a : 1) : (b > 0 ? b : 1);
  }
  static int occupancy(int v) {
    switch (v / 2) {
      case 0: return occ<64>();
      case 1: return occ<128>();
      default: return occ<256>();
    }
  }
  template <int TB>
  static void run(const BatchArgs<R>& b, int grid, int collide, cudaStream_t s) {
    if (collide) k_batch<R, D, M, EN, TB, true><<<grid, TB, 0, s>>>(b);
    else k_batch<R, D, M, EN, TB, false><<<grid, TB, 0, s>>>(b);
  }
  static void pass(const BatchArgs<R>& b, int v, int grid, int collide, cudaStream_t s) {
    switch (v / 2) {
      case 0: run<64>(b, grid, collide, s); break;
      case 1: run<128>(b, grid, collide, s); break;
      default: run<256>(b, grid, collide, s); break;
    }
  }
  static BatchOps<R> ops() { return BatchOps<R>{tile, occupancy, pass, 6}; }
};

}  // namespace

bool LBM_BATCH_OPS_NAME(int M, int energy, BatchOps<LBM_REAL>* out) {
  if (M == 2 && !energy) { *out = BatchLaunch<LBM_REAL, 2, 2, false>::ops(); return true; }
  if (M == 3 && energy) { *out = BatchLaunch<LBM_REAL, 2, 3, true>::ops(); return true; }
  return false;
}

}  // namespace lbm
