// Instantiates the batched-form kernels for one precision; the including file
// defines LBM_REAL and LBM_BATCH_OPS_NAME.
#include "lbm_batch.cuh"

namespace lbm {
namespace {

template <class R, int D, int M, bool EN>
struct BatchLaunch {
  // variant v: tile length kTiles[(v % 6) / 2]; grid mode v % 2; v >= 6 stages populations in shared memory
  static constexpr int kTiles[3] = {64, 128, 256};
  static int tile(int v) { return kTiles[(v % 6) / 2]; }
  template <int TB>
  static constexpr size_t smem() { return sizeof(R) * (size_t)n_pops<R, D, M, EN>() * TB; }
  template <int TB>
  static int occ(bool staged) {
    int a = 0, b = 0;
    cudaError_t e1, e2;
    if (staged) {
      e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_staged<R, D, M, EN, TB, false>, TB, smem<TB>());
      e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_staged<R, D, M, EN, TB, true>, TB, smem<TB>());
    } else {
      e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch<R, D, M, EN, TB, false>, TB, 0);
      e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<R, D, M, EN, TB, true>, TB, 0);
    }
    if (e1 != cudaSuccess) a = 1;
    if (e2 != cudaSuccess) b = 1;
    return a < b ? (a > 0 ? a : 1) : (b > 0 ? b : 1);
  }
  static int occupancy(int v) {
    const bool staged = v >= 6;
    switch ((v % 6) / 2) {
      case 0: return occ<64>(staged);
      case 1: return occ<128>(staged);
      default: return occ<256>(staged);
    }
  }
  template <int TB>
  static void run(const BatchArgs<R>& b, int grid, int collide, bool staged, cudaStream_t s) {
    if (staged) {
      constexpr size_t sm = smem<TB>();
      if (sm > 48 * 1024) {
        static bool done = false;
        if (!done) {
          cudaFuncSetAttribute(k_batch_staged<R, D, M, EN, TB, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          cudaFuncSetAttribute(k_batch_staged<R, D, M, EN, TB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
          done = true;
        }
      }
      if (collide) k_batch_staged<R, D, M, EN, TB, true><<<grid, TB, sm, s>>>(b);
      else k_batch_staged<R, D, M, EN, TB, false><<<grid, TB, sm, s>>>(b);
    } else {
      if (collide) k_batch<R, D, M, EN, TB, true><<<grid, TB, 0, s>>>(b);
      else k_batch<R, D, M, EN, TB, false><<<grid, TB, 0, s>>>(b);
    }
  }
  static void pass(const BatchArgs<R>& b, int v, int grid, int collide, cudaStream_t s) {
    const bool staged = v >= 6;
    switch ((v % 6) / 2) {
      case 0: run<64>(b, grid, collide, staged, s); break;
      case 1: run<128>(b, grid, collide, staged, s); break;
      default: run<256>(b, grid, collide, staged, s); break;
    }
  }
  static BatchOps<R> ops() { return BatchOps<R>{tile, occupancy, pass, 12}; }
};

}  // namespace

bool LBM_BATCH_OPS_NAME(int M, int energy, BatchOps<LBM_REAL>* out) {
  if (M == 2 && !energy) { *out = BatchLaunch<LBM_REAL, 2, 2, false>::ops(); return true; }
  if (M == 3 && energy) { *out = BatchLaunch<LBM_REAL, 2, 3, true>::ops(); return true; }
  return false;
}

}  // namespace lbm
