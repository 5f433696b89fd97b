// Instantiates the adjoint kernels for one precision; the including file
// defines LBM_REAL and LBM_ADJ_OPS_NAME.
#include "lbm_adjoint.cuh"

namespace lbm {
namespace {

// dual lanes of the node-update evaluations: fewer lanes spill less (with
// populations seeded, FP32 took 1.65 ms per adjoint step of the 256x256 slab
// with 2 lanes and 2.87 ms with 4); with the moments seeded, 4 lanes in FP64
// push the node code past the register file into a 13 KB stack frame
template <class B> constexpr int kLanesOf() { return 2; }
constexpr int kLanesSmall = 8;   // dual lanes of the macro-field and reservoir-ghost evaluations

template <class To, class From>
void params_cast(const Params<From>& s, Params<To>& d) {
  d.nx = s.nx; d.ny = s.ny; d.nz = s.nz; d.N = s.N;
  d.bc_lo = s.bc_lo; d.bc_hi = s.bc_hi; d.knudsen = s.knudsen;
  d.RU = To(s.RU);
  for (int a = 0; a < MMAX; ++a) {
    d.m[a] = To(s.m[a]); d.Ra[a] = To(s.Ra[a]); d.muref[a] = To(s.muref[a]);
    d.cvR[a] = To(s.cvR[a]); d.U0[a] = To(s.U0[a]); d.knc[a] = To(s.knc[a]);
    for (int b = 0; b < MMAX; ++b) d.invDmm[a][b] = To(s.invDmm[a][b]);
    d.rho_in[0][a] = To(s.rho_in[0][a]); d.rho_in[1][a] = To(s.rho_in[1][a]);
  }
  d.mu_exp = To(s.mu_exp); d.inv_Pr = To(s.inv_Pr); d.bulk_ratio = To(s.bulk_ratio);
  d.T_thermo = To(s.T_thermo); d.inv_T_ref = To(s.inv_T_ref); d.Pref = To(s.Pref);
  d.T_in[0] = To(s.T_in[0]); d.T_in[1] = To(s.T_in[1]);
  d.kappa_thr = To(s.kappa_thr);
}

template <class B, int D, int M, bool EN>
struct AdjLaunch {
  static constexpr int K = kLanesOf<B>(), KS = kLanesSmall;
  template <int KK>
  static AdjParams<B, KK> make(const Params<B>& p) {
    AdjParams<B, KK> ap;
    params_cast(p, ap.pz);
    ap.pz.N = 1;                 // node-local evaluation into a local array
    ap.pk = ap.pz;
    for (int a = 0; a < MMAX; ++a) ap.pk.knc[a].d[0] = p.knc[a];
    return ap;
  }
  static int grid(int n, int b) { return (n + b - 1) / b; }
  static int collide(const Params<B>& p, const InletTables<B>& it, const AdjArgs<B>& a, cudaStream_t s) {
    k_adj_collide<B, D, M, EN, K><<<grid(p.N, 128), 128, 0, s>>>(p, it, a, make<K>(p));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
  }
  static int macro(const Params<B>& p, const InletTables<B>& it, const AdjArgs<B>& a, cudaStream_t s) {
    k_adj_macro<B, D, M, EN, KS><<<grid(p.N, 128), 128, 0, s>>>(p, it, a, make<KS>(p));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
  }
  static int ghost(const Params<B>& p, const InletTables<B>& it, const AdjArgs<B>& a, cudaStream_t s) {
    k_adj_ghost<B, D, M, EN, KS><<<grid(p.ny * p.nz, 128), 128, 0, s>>>(p, it, a, make<KS>(p));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
  }
  static void stream(const Params<B>& p, const AdjArgs<B>& a, cudaStream_t s) {
    k_adj_stream<B, D, M, EN><<<grid(p.N, 256), 256, 0, s>>>(p, a);
  }
  static void seed_flux(const Params<B>& p, const AdjArgs<B>& a, int species, int axis, int xo, double w,
                        cudaStream_t s) {
    k_adj_seed_flux<B, D, M, EN><<<grid(p.N, 256), 256, 0, s>>>(p, a, species, axis, xo, (B)w);
  }
  static void init(const Params<B>& p, const double* X, const double* T, const double* P, const double* U,
                   double cvel, double RU, const AdjArgs<B>& a, cudaStream_t s) {
    k_adj_init<B, D, M, EN><<<grid(p.N, 128), 128, 0, s>>>(p, X, T, P, U, cvel, RU, a);
  }
  static AdjOps<B> ops() { return AdjOps<B>{collide, macro, ghost, stream, seed_flux, init, n_grad<D, M, EN>()}; }
};

}  // namespace

bool LBM_ADJ_OPS_NAME(int D, int M, int energy, AdjOps<LBM_REAL>* out) {
  if (D != 2) return false;
  if (M == 2 && !energy) { *out = AdjLaunch<LBM_REAL, 2, 2, false>::ops(); return true; }
  if (M == 3 && energy) { *out = AdjLaunch<LBM_REAL, 2, 3, true>::ops(); return true; }
  return false;
}

}  // namespace lbm
