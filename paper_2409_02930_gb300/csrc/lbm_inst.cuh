// Instantiates the step kernels for one (precision, dimension); the including
// file defines LBM_REAL, LBM_DIM and LBM_OPS_NAME.
#include "lbm_fused.cuh"
#include "lbm_kernels.cuh"
#include "lbm_march2d.cuh"
#include "lbm_ops.h"
#include "lbm_staged.cuh"
#include "lbm_surface.cuh"

namespace lbm {
namespace {

constexpr size_t kMaxSmem = 227 * 1024;

template <class Kern>
int configure(Kern kern, size_t smem, bool& done) {
  if (smem > kMaxSmem) return -1;
  if (!done) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    done = true;
  }
  return 0;
}

template <class R, int D, int M, bool EN>
struct Launch {
  static int grid(int N) { return (N + 255) / 256; }
  static void macro(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    k_macro<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a);
  }
  static void collide(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    k_collide<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a);
  }
  // fused step, shared-memory halo ring, tile TX x TY marching SEG planes
  template <int TX, int TY, int SEG>
  static int fused_tile(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    constexpr size_t smem = fused_smem_bytes<R, D, M, EN, TX, TY>();
    auto kern = k_fused<R, D, M, EN, TX, TY, SEG>;
    static bool done = false;
    if (configure(kern, smem, done)) return -1;
    dim3 g((p.nx + TX - 1) / TX, D == 3 ? (p.ny + TY - 1) / TY : (p.ny + SEG - 1) / SEG,
           D == 3 ? (p.nz + SEG - 1) / SEG : 1);
    kern<<<g, TX * TY, smem, s>>>(p, it, a);
    return 0;
  }
  // pipelined 2-D step (cp.async staging), TX columns marching SEG rows
  template <int TX, int SEG, int MINB, int PD>
  static int march2d(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    if constexpr (D != 2) {
      return -1;
    } else {
      constexpr size_t smem = march2d_smem_bytes<R, M, EN, TX, PD>();
      if constexpr (smem > kMaxSmem) {
        return -1;
      } else {
        // the reservoir-column path is compiled in only when a face is a reservoir
        const bool inlet = p.bc_lo == BC_INLET || p.bc_hi == BC_INLET;
        auto kern = inlet ? k_march2d<R, M, EN, TX, SEG, MINB, PD, true> : k_march2d<R, M, EN, TX, SEG, MINB, PD, false>;
        static bool done[2] = {false, false};
        if (configure(kern, smem, done[inlet ? 1 : 0])) return -1;
        dim3 g((p.nx + TX - 3) / (TX - 2), (p.ny + SEG - 1) / SEG, 1);
        kern<<<g, TX, smem, s>>>(p, it, a, TmaMaps{});
        return 0;
      }
    }
  }
  // the same march with each row staged by bulk tensor copies (TMA); lattices
  // whose rows are not a multiple of 16 bytes take the cp.async form
  template <int TX, int SEG, int MINB, int PD>
  static int march2d_tma(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    if constexpr (D != 2) {
      return -1;
    } else {
      using LB = RowBoxLayout<R, M, EN, TX, PD>;
      constexpr size_t smem = LB::bytes();
      if constexpr (smem > kMaxSmem) {
        return -1;
      } else {
        TmaMaps tm;
        if (!encode_row_maps<R>(tm, a.src, a.phi, EN ? nullptr : a.Tfix, p.nx, p.ny, Lat<D>::Q, LB::NL, LB::W))
          return march2d<TX, SEG, MINB, PD>(p, it, a, s);
        const bool inlet = p.bc_lo == BC_INLET || p.bc_hi == BC_INLET;
        auto kern = inlet ? k_march2d<R, M, EN, TX, SEG, MINB, PD, true, true>
                          : k_march2d<R, M, EN, TX, SEG, MINB, PD, false, true>;
        static bool done[2] = {false, false};
        if (configure(kern, smem, done[inlet ? 1 : 0])) return -1;
        dim3 g((p.nx + TX - 3) / (TX - 2), (p.ny + SEG - 1) / SEG, 1);
        kern<<<g, TX, smem, s>>>(p, it, a, tm);
        return 0;
      }
    }
  }
  // two-pass form whose node update stages each node's pulled populations in shared memory
  template <int TB>
  static int staged(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    constexpr size_t smem = sizeof(R) * (size_t)n_pops<R, D, M, EN>() * TB;
    if constexpr (smem > kMaxSmem) {
      return -1;
    } else {
      auto kern = k_collide_staged<R, D, M, EN, TB>;
      auto kmac = k_macro_staged<R, D, M, EN, TB>;
      static bool done = false, done_mac = false;
      if (configure(kern, smem, done) || configure(kmac, smem, done_mac)) return -1;
      kmac<<<(p.N + TB - 1) / TB, TB, smem, s>>>(p, it, a);
      kern<<<(p.N + TB - 1) / TB, TB, smem, s>>>(p, it, a);
      return 0;
    }
  }
  // the staged form with the gradient inputs computed once per node in a pass
  // of their own (3-D; the macro buffer holds them after the macro fields)
  template <int TB>
  static int staged_grad(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, cudaStream_t s) {
    constexpr size_t smem = sizeof(R) * (size_t)n_pops<R, D, M, EN>() * TB;
    if constexpr (D != 3 || smem > kMaxSmem) {
      return -1;
    } else {
      auto kern = k_collide_staged_g<R, D, M, EN, TB>;
      auto kmac = k_macro_staged<R, D, M, EN, TB>;
      static bool done = false, done_mac = false;
      if (configure(kern, smem, done) || configure(kmac, smem, done_mac)) return -1;
      kmac<<<(p.N + TB - 1) / TB, TB, smem, s>>>(p, it, a);
      k_grad<R, D, M, EN><<<(p.N + 255) / 256, 256, 0, s>>>(p, a);
      kern<<<(p.N + TB - 1) / TB, TB, smem, s>>>(p, it, a);
      return 0;
    }
  }
  static int fused(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, int v, cudaStream_t s) {
    if constexpr (D == 2) {
      switch (v) {
        case 0: return march2d<64, 8, 1, 1>(p, it, a, s);
        case 1: return march2d<64, 8, 1, 2>(p, it, a, s);
        case 2: return march2d<32, 8, 1, 1>(p, it, a, s);
        case 3: return march2d<128, 4, 1, 1>(p, it, a, s);
        case 4: return march2d<64, 16, 1, 1>(p, it, a, s);
        case 5: return fused_tile<32, 1, 8>(p, it, a, s);
        case 6: return staged<64>(p, it, a, s);
        case 7: return staged<128>(p, it, a, s);
        case 8: return march2d_tma<32, 8, 1, 1>(p, it, a, s);
        case 9: return march2d_tma<64, 8, 1, 1>(p, it, a, s);
        default: return -1;
      }
    } else {
      switch (v) {
        case 0: return fused_tile<32, 4, 16>(p, it, a, s);
        case 1: return fused_tile<32, 8, 16>(p, it, a, s);
        case 2: return fused_tile<32, 4, 8>(p, it, a, s);
        case 3: return staged<64>(p, it, a, s);
        case 4: return staged<32>(p, it, a, s);
        case 5: return staged_grad<64>(p, it, a, s);
        default: return -1;
      }
    }
  }
  static constexpr int n_variants = (D == 2) ? 10 : 6;
  static void init(const Params<R>& p, const double* X, const double* T, const double* P, const double* U,
                   double cvel, double RU, R* dst, const R* phi, cudaStream_t s) {
    k_init<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, X, T, P, U, cvel, RU, dst, phi);
  }
  static void moments(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, int which, double cvel,
                      double* out, cudaStream_t s) {
    k_moments<R, D, M, EN><<<grid(p.N), 256, 0, s>>>(p, it, a, which, cvel, out);
  }
  static constexpr bool has_react = (D == 3 && M == 6 && EN);
  static void react_macro(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, const ReactArgs& ra,
                          cudaStream_t s) {
    if constexpr (has_react) k_macro_react<R, D, M, EN><<<(p.N + 127) / 128, 128, 0, s>>>(p, it, a, ra);
  }
  static void react_collide(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, const ReactArgs& ra,
                            cudaStream_t s) {
    if constexpr (has_react) {
      // node populations staged in shared memory (TB x 216 values per block)
      constexpr int TB = sizeof(R) == 4 ? 64 : 32;
      constexpr size_t smem = sizeof(R) * (size_t)n_pops<R, D, M, EN>() * TB;
      auto kern = k_collide_react_staged<R, D, M, EN, TB>;
      static bool done = false;
      if (configure(kern, smem, done)) {
        k_collide_react<R, D, M, EN><<<(p.N + 127) / 128, 128, 0, s>>>(p, it, a, ra);
        return;
      }
      kern<<<(p.N + TB - 1) / TB, TB, smem, s>>>(p, it, a, ra);
    }
  }
  static Ops<R> ops() {
    return Ops<R>{macro, collide, fused, n_variants, init, moments, has_react ? react_macro : nullptr,
                  has_react ? react_collide : nullptr};
  }
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
