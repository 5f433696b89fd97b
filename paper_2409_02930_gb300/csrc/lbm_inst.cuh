// Instantiates the step kernels for one (precision, dimension); the including
// file defines LBM_REAL, LBM_DIM and LBM_OPS_NAME.
#include "lbm_fused.cuh"
#include "lbm_kernels.cuh"
#include "lbm_ops.h"

namespace lbm {
namespace {

// tile shapes (TX, TY, SEG) of the fused kernel tried by the autotuner
template <int D> struct Tiles;
template <> struct Tiles<2> {
  static constexpr int n = 4;
  static constexpr int tx[n] = {32, 64, 32, 128};
  static constexpr int ty[n] = {1, 1, 1, 1};
  static constexpr int seg[n] = {8, 8, 16, 4};
};
template <> struct Tiles<3> {
  static constexpr int n = 3;
  static constexpr int tx[n] = {32, 32, 32};
  static constexpr int ty[n] = {4, 8, 4};
  static constexpr int seg[n] = {16, 16, 8};
};

template <class R, int D, int M, bool EN>
struct Launch {
  static int grid(int N) { return (N + 255) / 256; }
  static void macro(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    k_macro<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a);
  }
  static void collide(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    k_collide<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a);
  }
  template <int TX, int TY, int SEG>
  static int fused_tile(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    constexpr size_t smem = fused_smem_bytes<R, D, M, EN, TX, TY>();
    auto kern = k_fused<R, D, M, EN, TX, TY, SEG>;
    static bool configured = false;
    if (!configured) {
      if (smem > 48 * 1024 &&
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
      configured = true;
    }
    dim3 g((p.nx + TX - 1) / TX, D == 3 ? (p.ny + TY - 1) / TY : (p.ny + SEG - 1) / SEG,
           D == 3 ? (p.nz + SEG - 1) / SEG : 1);
    kern<<<g, TX * TY, smem, s>>>(p, it, a);
    return 0;
  }
  static int fused(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, int v, cudaStream_t s) {
    using T = Tiles<D>;
    switch (v) {
      case 0: return fused_tile<T::tx[0], T::ty[0], T::seg[0]>(p, it, a, s);
      case 1: return fused_tile<T::tx[1], T::ty[1], T::seg[1]>(p, it, a, s);
      case 2: return fused_tile<T::tx[2], T::ty[2], T::seg[2]>(p, it, a, s);
      case 3:
        if constexpr (T::n > 3) return fused_tile<T::tx[3 % T::n], T::ty[3 % T::n], T::seg[3 % T::n]>(p, it, a, s);
        return -1;
      default: return -1;
    }
  }
  static void init(const Params<R>& p, const double* X, const double* T, const double* P, const double* U,
                   double cvel, double RU, R* dst, const R* phi, cudaStream_t s) {
    k_init<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, X, T, P, U, cvel, RU, dst, phi);
  }
  static void moments(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, int which, double cvel,
                      double* out, cudaStream_t s) {
    k_moments<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a, which, cvel, out);
  }
  static Ops<R> ops() { return Ops<R>{macro, collide, fused, Tiles<D>::n, init, moments}; }
};

}  // namespace

bool LBM_OPS_NAME(int M, int energy, Ops<LBM_REAL>* out) {
  switch (M * 2 + (energy ? 1 : 0)) {
    case 4: *out = Launch<LBM_REAL, LBM_DIM, 2, false>::ops(); return true;
    case 5: *out = Launch<LBM_REAL, LBM_DIM, 2, true>::ops(); return true;
    case 6: *out = Launch<LBM_REAL, LBM_DIM, 3, false>::ops(); return true;
    case 7: *out = Launch<LBM_REAL, LBM_DIM, 3, true>::ops(); return true;
    case 12: *out = Launch<LBM_REAL, LBM_DIM, 6, false>::ops(); return true;
    case 13: *out = Launch<LBM_REAL, LBM_DIM, 6, true>::ops(); return true;
    default: return false;
  }
}

}  // namespace lbm
