// Instantiates the step kernels for one (precision, dimension); the including
// file defines LBM_REAL, LBM_DIM and LBM_OPS_NAME.
#include "lbm_kernels.cuh"
#include "lbm_ops.h"

namespace lbm {
namespace {

template <class R, int D, int M, bool EN>
struct Launch {
  static int grid(int N) { return (N + 255) / 256; }
  static void macro(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    k_macro<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a);
  }
  static void collide(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    k_collide<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a);
  }
  static void init(const Params<R>& p, const double* X, const double* T, const double* P, const double* U,
                   double cvel, double RU, R* dst, const R* phi, cudaStream_t s) {
    k_init<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, X, T, P, U, cvel, RU, dst, phi);
  }
  static void moments(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, int which, double cvel,
                      double* out, cudaStream_t s) {
    k_moments<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a, which, cvel, out);
  }
  static Ops<R> ops() { return Ops<R>{macro, collide, init, moments}; }
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
