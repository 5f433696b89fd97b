// Host side of the C ABI declared in include/lbm.h: configuration checks,
// lattice-unit conversion, device allocation and the per-step launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_ctx.h"

namespace {

const double R_UNIV_SI = 8.314462618;   // J/(mol K)
const double PI_SI = 3.14159265358979323846;

thread_local std::string g_create_error;

}  // namespace



namespace {

int fail(lbm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

size_t real_size(const lbm_ctx* c) { return c->precision == LBM_FP64 ? 8 : 4; }

template <class R>
void convert_params(const lbm::Params<double>& d, lbm::Params<R>& r) {
  r.nx = d.nx; r.ny = d.ny; r.nz = d.nz; r.N = d.N;
  r.bc_lo = d.bc_lo; r.bc_hi = d.bc_hi; r.knudsen = d.knudsen;
  r.RU = (R)d.RU;
  for (int a = 0; a < lbm::MMAX; ++a) {
    r.m[a] = (R)d.m[a]; r.Ra[a] = (R)d.Ra[a]; r.muref[a] = (R)d.muref[a];
    r.cvR[a] = (R)d.cvR[a]; r.U0[a] = (R)d.U0[a]; r.knc[a] = (R)d.knc[a];
    for (int b = 0; b < lbm::MMAX; ++b) r.invDmm[a][b] = (R)d.invDmm[a][b];
    r.rho_in[0][a] = (R)d.rho_in[0][a]; r.rho_in[1][a] = (R)d.rho_in[1][a];
  }
  r.mu_exp = (R)d.mu_exp; r.inv_Pr = (R)d.inv_Pr; r.bulk_ratio = (R)d.bulk_ratio;
  r.T_thermo = (R)d.T_thermo; r.inv_T_ref = (R)d.inv_T_ref; r.Pref = (R)d.Pref;
  r.T_in[0] = (R)d.T_in[0]; r.T_in[1] = (R)d.T_in[1];
  r.kappa_thr = (R)d.kappa_thr;
  r.wait_limit = d.wait_limit;
}

template <class R>
void convert_inlet(const lbm::InletTables<double>& d, lbm::InletTables<R>& r) {
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < lbm::MMAX; ++a) r.rho[s][a] = (R)d.rho[s][a];
    r.rho_sum[s] = (R)d.rho_sum[s]; r.Rmix[s] = (R)d.Rmix[s]; r.Umix[s] = (R)d.Umix[s]; r.T[s] = (R)d.T[s];
  }
}

// Checks of the configuration itself; with fields, also the per-node input
// arrays (porosity, X_init, T_init, P_init) that lbm_create reads.
constexpr int kDefaultWaitLimit = 1 << 22;

int validate(const lbm_config* c, bool fields = true) {
  if (!c) return fail(nullptr, LBM_ERR_ARG, "null config");
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return fail(nullptr, LBM_ERR_ARG, "lattice dimensions must be >= 1");
  if ((double)c->nx * c->ny * c->nz > 2.0e9) return fail(nullptr, LBM_ERR_ARG, "lattice too large");
  if (c->M != 2 && c->M != 3 && c->M != 6) return fail(nullptr, LBM_ERR_ARG, "M must be 2, 3 or 6");
  for (int s = 0; s < 2; ++s) {
    int bc = s ? c->bc_hi : c->bc_lo;
    if (bc < 0 || bc > 2) return fail(nullptr, LBM_ERR_ARG, "unknown boundary condition");
    if (bc == LBM_BC_INLET && c->nx < 3) return fail(nullptr, LBM_ERR_ARG, "inlet faces need nx >= 3");
    if (bc != LBM_BC_PERIODIC && c->nx < 2) return fail(nullptr, LBM_ERR_ARG, "walls need nx >= 2");
  }
  if ((c->bc_lo == LBM_BC_PERIODIC) != (c->bc_hi == LBM_BC_PERIODIC))
    return fail(nullptr, LBM_ERR_ARG, "x faces must be both periodic or both non-periodic");
  if (c->precision != LBM_FP64 && c->precision != LBM_FP32) return fail(nullptr, LBM_ERR_ARG, "unknown precision");
  if (!(c->dx > 0) || !(c->theta_max > 0) || !(c->theta_max < 1) || !(c->T_scale > 0) || !(c->T_ref > 0) ||
      !(c->P_ref > 0) || !(c->Pr > 0))
    return fail(nullptr, LBM_ERR_ARG, "dx, theta_max in (0,1), T_scale, T_ref, P_ref and Pr must be positive");
  if (c->knudsen && (!(c->pore_radius > 0) || !(c->tortuosity > 0)))
    return fail(nullptr, LBM_ERR_ARG, "Knudsen diffusion needs a positive pore radius and tortuosity");
  if (!c->molar_mass || !c->D_ref || !c->mu_ref || !c->cv_factor || !c->U0)
    return fail(nullptr, LBM_ERR_ARG, "missing input array");
  if (fields && (!c->porosity || !c->X_init || !c->T_init || !c->P_init))
    return fail(nullptr, LBM_ERR_ARG, "missing input array");
  for (int a = 0; a < c->M; ++a) {
    if (!(c->molar_mass[a] > 0) || !(c->mu_ref[a] >= 0) || !(c->cv_factor[a] > 0))
      return fail(nullptr, LBM_ERR_ARG, "molar masses and heat capacities must be positive");
    for (int b = 0; b < c->M; ++b)
      if (a != b && !(c->D_ref[a * c->M + b] > 0))
        return fail(nullptr, LBM_ERR_ARG, "binary diffusivities must be positive");
  }
  size_t N = fields ? (size_t)c->nx * c->ny * c->nz : 0;
  for (size_t n = 0; n < N; ++n) {
    if (!(c->porosity[n] > 0) || !(c->porosity[n] <= 1)) return fail(nullptr, LBM_ERR_ARG, "porosity outside (0, 1]");
    if (!(c->T_init[n] > 0) || !(c->P_init[n] > 0)) return fail(nullptr, LBM_ERR_ARG, "non-positive T or P");
  }
  if (c->bc_lo == LBM_BC_INLET || c->bc_hi == LBM_BC_INLET) {
    if (!c->X_in_lo || !c->X_in_hi || !(c->T_in_lo > 0) || !(c->T_in_hi > 0) || !(c->P_in_lo > 0) ||
        !(c->P_in_hi > 0))
      return fail(nullptr, LBM_ERR_ARG, "inlet faces need reservoir composition, T and P");
  }
  if (c->S < 0 || c->S > lbm::SMAX || c->R < 0 || c->R > lbm::RMAX)
    return fail(nullptr, LBM_ERR_ARG, "surface mechanism too large (S <= 12, R <= 32)");
  if (c->S > 0) {
    if (c->R < 1 || !c->nu_gas || !c->nu_surf || !c->A_pre || !c->Ea || !c->surf_cv_factor || !c->surf_U0 ||
        !c->Xs_init || !(c->gamma > 0) || !(c->a_s > 0))
      return fail(nullptr, LBM_ERR_ARG, "incomplete surface mechanism");
    if (!c->energy) return fail(nullptr, LBM_ERR_ARG, "a surface mechanism needs the energy lattice");
    if (c->edge && (!c->n_el || !(c->l_tpb > 0) || !(c->beta_ct >= 0) || !(c->resistivity >= 0)))
      return fail(nullptr, LBM_ERR_ARG, "TPB steps need electron counts, a positive TPB length and beta >= 0");
  }
  return LBM_OK;
}

}  // namespace

namespace lbm {
// configuration checks of lbm_create without its per-node input arrays
int validate_config(const lbm_config* c) { return validate(c, false); }

// Lattice-unit parameters of a validated configuration.
void make_params(const lbm_config* c, Params<double>& p, InletTables<double>& it, double& dt, double& cvel) {
  const int M = c->M;
  const int knudsen = c->knudsen ? 1 : 0;
  // lattice units: max_a R_a T_scale dt^2/dx^2 = theta_max
  double mmin = 1e300;
  for (int a = 0; a < M; ++a) mmin = std::fmin(mmin, c->molar_mass[a]);
  dt = c->dx * std::sqrt(c->theta_max * mmin / (R_UNIV_SI * c->T_scale));
  cvel = c->dx / dt;
  const double c2 = cvel * cvel;
  std::memset(&p, 0, sizeof(p));
  p.nx = c->nx; p.ny = c->ny; p.nz = c->nz; p.N = c->nx * c->ny * c->nz;
  p.bc_lo = c->bc_lo; p.bc_hi = c->bc_hi; p.knudsen = knudsen;
  p.RU = R_UNIV_SI / c2;
  const double d0 = 2.0 * c->pore_radius / c->dx;
  for (int a = 0; a < M; ++a) p.m[a] = c->molar_mass[a];
  for (int a = 0; a < M; ++a) {
    p.Ra[a] = p.RU / p.m[a];
    p.muref[a] = c->mu_ref[a] / (cvel * c->dx);
    p.cvR[a] = c->cv_factor[a] * p.Ra[a];
    p.U0[a] = c->U0[a] / c2;
    for (int b = 0; b < M; ++b)
      p.invDmm[a][b] = (a == b) ? 0.0 : 1.0 / ((c->D_ref[a * M + b] / (cvel * c->dx)) * p.m[a] * p.m[b]);
    // D^k = (phi/tortuosity)(d0/3) sqrt(8 R_U T/(pi m_a)); 1/tau^k = R_U T/(D^k m_a)
    if (knudsen)
      p.knc[a] = 3.0 * c->tortuosity * p.RU / (d0 * p.m[a] * std::sqrt(8.0 * p.RU / (PI_SI * p.m[a])));
  }
  p.mu_exp = c->mu_exp;
  p.inv_Pr = 1.0 / c->Pr;
  p.bulk_ratio = c->bulk_ratio;
  p.T_thermo = c->T_thermo;
  p.inv_T_ref = 1.0 / c->T_ref;
  p.Pref = c->P_ref / c2;
  p.kappa_thr = c->kappa_threshold > 0 ? c->kappa_threshold : 1e3;
  p.wait_limit = kDefaultWaitLimit;
  std::memset(&it, 0, sizeof(it));
  const double* Xin[2] = {c->X_in_lo, c->X_in_hi};
  const double Tin[2] = {c->T_in_lo, c->T_in_hi}, Pin[2] = {c->P_in_lo, c->P_in_hi};
  for (int s = 0; s < 2; ++s) {
    if (!Xin[s] || !(Tin[s] > 0)) continue;
    double rho = 0.0, inv_m = 0.0, U = 0.0;
    for (int a = 0; a < M; ++a) {
      it.rho[s][a] = Pin[s] * Xin[s][a] * p.m[a] / (R_UNIV_SI * Tin[s]);
      rho += it.rho[s][a];
    }
    for (int a = 0; a < M; ++a) {
      inv_m += (it.rho[s][a] / rho) / p.m[a];
      U += (it.rho[s][a] / rho) * (p.U0[a] + p.cvR[a] * (Tin[s] - p.T_thermo));
    }
    it.rho_sum[s] = rho;
    it.Rmix[s] = p.RU * inv_m;
    it.Umix[s] = U;
    it.T[s] = Tin[s];
    p.T_in[s] = Tin[s];
    for (int a = 0; a < M; ++a) p.rho_in[s][a] = it.rho[s][a];
  }
}

}  // namespace lbm

// Device state of a surface mechanism: coverages, per-node sources and the
// mechanism table in SI units (the surface source works in FP64).
static int setup_surface(lbm_ctx* x, const lbm_config* c) {
  const bool have = (x->precision == LBM_FP64) ? (x->od.react_macro != nullptr) : (x->of.react_macro != nullptr);
  if (!have) return fail(nullptr, LBM_ERR_ARG, "surface mechanisms need D3Q27 with M = 6 and the energy lattice");
  const size_t N = x->N;
  lbm::MechDev h;
  std::memset(&h, 0, sizeof(h));
  h.M = c->M;
  h.S = c->S;
  h.R = c->R;
  for (int k = 0; k < c->R; ++k) {
    int nr = 0;
    for (int a = 0; a < c->M + c->S; ++a) {
      const double v = a < c->M ? c->nu_gas[k * c->M + a] : c->nu_surf[k * c->S + (a - c->M)];
      if (a < c->M) h.nu_g[k][a] = v;
      else h.nu_s[k][a - c->M] = v;
      h.nu_all[k][a] = v;
      if (v != 0) {
        if (h.npart[k] >= 8) return fail(nullptr, LBM_ERR_ARG, "at most 8 species take part in one surface step");
        h.pidx[k][h.npart[k]] = a;
        h.pnu[k][h.npart[k]] = v;
        h.npart[k]++;
        h.sr_k[a][h.nsr[a]] = k;
        h.sr_nuf[a][h.nsr[a]] = (float)v;
        h.sr_nud[a][h.nsr[a]] = v;
        h.nsr[a]++;
      }
      if (v < 0) {
        // mass-action reactant with an integer order
        const double ord = -v;
        if (nr >= 4 || ord != (double)(int)ord) return fail(nullptr, LBM_ERR_ARG, "reactant orders must be integers, at most 4 reactants");
        h.ridx[k][nr] = a;
        h.rord[k][nr] = (int)ord;
        ++nr;
      }
    }
    h.nre[k] = nr;
    h.A[k] = c->A_pre[k];
    h.Ea[k] = c->Ea[k];
    h.edge[k] = c->edge ? (c->edge[k] != 0) : 0;
    h.nel[k] = c->edge ? c->n_el[k] : 0.0;
    if (h.edge[k])
      for (int a = 0; a < c->M; ++a)
        if (c->nu_gas[k * c->M + a] != 0) return fail(nullptr, LBM_ERR_ARG, "a TPB step involves adsorbates only");
  }
  if (c->edge) {
    h.l_tpb = c->l_tpb;
    h.beta_ct = c->beta_ct;
    h.resist = c->resistivity;
    h.dphi = c->dphi;
  }
  h.dx = c->dx;
  h.gamma = c->gamma;
  h.a_s = c->a_s;
  for (int q = 0; q < c->S; ++q) {
    h.cvs[q] = c->surf_cv_factor[q];
    h.Us0[q] = c->surf_U0[q];
  }
  for (int a = 0; a < c->M; ++a) h.m[a] = c->molar_mass[a];
  h.T_thermo = c->T_thermo;
  h.dt = x->dt;
  h.cvel2 = x->cvel * x->cvel;
  cudaError_t e = cudaMalloc(&x->mech, sizeof(lbm::MechDev));
  if (e == cudaSuccess) e = cudaMalloc(&x->Xs[0], (size_t)c->S * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&x->Xs[1], (size_t)c->S * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&x->rsrc, (size_t)(c->M + 2) * N * sizeof(double));
  if (e != cudaSuccess) return fail(nullptr, LBM_ERR_ALLOC, "surface state allocation failed");
  std::vector<double> xs((size_t)c->S * N);
  for (int q = 0; q < c->S; ++q)
    for (size_t n = 0; n < N; ++n) xs[(size_t)q * N + n] = c->Xs_init[q];
  e = cudaMemcpy(x->mech, &h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(x->Xs[0], xs.data(), xs.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "surface state upload");
  x->xs_cur = 0;
  return LBM_OK;
}

extern "C" {

int lbm_create(lbm_ctx** out, const lbm_config* c) {
  if (!out) return fail(nullptr, LBM_ERR_ARG, "null output pointer");
  *out = nullptr;
  int rc = validate(c);
  if (rc) return rc;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1) return fail(nullptr, LBM_ERR_CUDA, "no CUDA device");

  lbm_ctx* x = new (std::nothrow) lbm_ctx();
  if (!x) return fail(nullptr, LBM_ERR_ALLOC, "host allocation failed");
  x->nx = c->nx; x->ny = c->ny; x->nz = c->nz;
  x->N = c->nx * c->ny * c->nz;
  x->D = c->nz > 1 ? 3 : 2;
  x->Q = x->D == 3 ? 27 : 9;
  x->M = c->M;
  x->energy = c->energy ? 1 : 0;
  x->knudsen = c->knudsen ? 1 : 0;
  x->L = c->M + 1 + x->energy;
  x->precision = c->precision;
  x->S = c->S;
  x->stream = (cudaStream_t)c->stream;
  x->cur = 0;
  // default form: in 3-D the staged form with a gradient pass; in 2-D the TMA row march
  // where it fills the GPU (one 32-column block per 8 rows: 1152 blocks at
  // 512 x 512) and no x face is a reservoir (reservoir columns take a
  // global-memory path that sets the march's pace), else the two-pass form
  const bool reservoir = c->bc_lo == LBM_BC_INLET || c->bc_hi == LBM_BC_INLET;
  x->variant = c->nz > 1 ? 5 : ((!reservoir && x->N >= (1 << 18)) ? 8 : -1);

  bool ok = (x->precision == LBM_FP64)
                ? (x->D == 2 ? lbm::get_ops_f64_2d(x->M, x->energy, &x->od) : lbm::get_ops_f64_3d(x->M, x->energy, &x->od))
                : (x->D == 2 ? lbm::get_ops_f32_2d(x->M, x->energy, &x->of) : lbm::get_ops_f32_3d(x->M, x->energy, &x->of));
  if (!ok) { delete x; return fail(nullptr, LBM_ERR_ARG, "no kernel for this (M, energy)"); }

  lbm::make_params(c, x->pd, x->itd, x->dt, x->cvel);
  const int M = x->M;
  convert_params(x->pd, x->pf);
  convert_inlet(x->itd, x->itf);

  // ---- device state ---------------------------------------------------------
  const size_t N = x->N;
  const size_t rs = real_size(x);
  const size_t pop_bytes = (size_t)x->L * x->Q * N * rs;
  void* ptrs[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // macro scratch: u, Pi, Y_a, and in 3-D the gradient inputs of the staged
  // form with a gradient pass (1 + D + M D more fields)
  const size_t mac_fields = (size_t)(2 * x->D + M) + (x->D == 3 ? (size_t)(1 + x->D + M * x->D) : 0);
  size_t sizes[6] = {pop_bytes, pop_bytes, N * rs, N * rs, mac_fields * N * rs, 64};
  for (int k = 0; k < 6; ++k) {
    e = cudaMalloc(&ptrs[k], sizes[k]);
    if (e != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaFree(ptrs[j]);
      delete x;
      return fail(nullptr, LBM_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  x->pops[0] = ptrs[0]; x->pops[1] = ptrs[1]; x->phi = ptrs[2]; x->Tfix = ptrs[3]; x->mac = ptrs[4];
  x->status = (int*)ptrs[5];
  x->scratch_out = nullptr;
  x->scratch_bytes = 0;

  // upload static fields in the working precision
  std::vector<char> hbuf(N * rs);
  auto upload = [&](void* dst, const double* src) -> cudaError_t {
    if (rs == 8) std::memcpy(hbuf.data(), src, N * 8);
    else for (size_t n = 0; n < N; ++n) ((float*)hbuf.data())[n] = (float)src[n];
    return cudaMemcpy(dst, hbuf.data(), N * rs, cudaMemcpyHostToDevice);
  };
  if ((e = upload(x->phi, c->porosity)) != cudaSuccess || (e = upload(x->Tfix, c->T_init)) != cudaSuccess ||
      (e = cudaMemset(x->status, 0, 64)) != cudaSuccess) {
    lbm_destroy(x);
    return cuda_fail(nullptr, e, "upload");
  }
  // initial fields -> temporary device copies -> equilibrium populations
  double *dX = nullptr, *dT = nullptr, *dP = nullptr, *dU = nullptr;
  size_t nb = N * sizeof(double);
  e = cudaMalloc(&dX, nb * M);
  if (e == cudaSuccess) e = cudaMalloc(&dT, nb);
  if (e == cudaSuccess) e = cudaMalloc(&dP, nb);
  if (e == cudaSuccess && c->U_init) e = cudaMalloc(&dU, nb * 3);
  if (e == cudaSuccess) e = cudaMemcpy(dX, c->X_init, nb * M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dT, c->T_init, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dP, c->P_init, nb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && c->U_init) e = cudaMemcpy(dU, c->U_init, nb * 3, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (x->precision == LBM_FP64)
      x->od.init(x->pd, dX, dT, dP, dU, x->cvel, R_UNIV_SI, (double*)x->pops[0], (const double*)x->phi, x->stream);
    else
      x->of.init(x->pf, dX, dT, dP, dU, x->cvel, R_UNIV_SI, (float*)x->pops[0], (const float*)x->phi, x->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  // the initial fields stay on the device (lbm_adjoint restarts from them)
  x->init_X = dX;
  x->init_T = dT;
  x->init_P = dP;
  x->init_U = dU;
  x->tortuosity = c->tortuosity;
  x->pore_radius = c->pore_radius;
  if (e != cudaSuccess) {
    lbm_destroy(x);
    return cuda_fail(nullptr, e, "initialisation");
  }
  if (x->S > 0) {
    int rc2 = setup_surface(x, c);
    if (rc2 != LBM_OK) {
      lbm_destroy(x);
      return rc2;
    }
  }
  *out = x;
  return LBM_OK;
}

}  // extern "C"

// Builds the device case table of a batched context.
template <class R>
static cudaError_t upload_cases(lbm_ctx* x, const std::vector<lbm::Params<R>>& ps,
                                const std::vector<lbm::InletTables<R>>& its) {
  std::vector<lbm::CaseDev<R>> h(x->n_cases);
  const long long mac_fields = 2 * x->D + x->M;
  for (int c = 0; c < x->n_cases; ++c) {
    h[c].p = ps[c];
    h[c].it = its[c];
    h[c].node_off = x->case_node_off[c];
    h[c].pop_off = x->case_node_off[c] * x->L * x->Q;
    h[c].mac_off = x->case_node_off[c] * mac_fields;
  }
  cudaError_t e = cudaMalloc(&x->cases_dev, h.size() * sizeof(h[0]));
  if (e == cudaSuccess) e = cudaMemcpy(x->cases_dev, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice);
  return e;
}

extern "C" {

int lbm_create_batch(lbm_ctx** out, int n_cases, const lbm_config* cfgs) {
  if (!out) return fail(nullptr, LBM_ERR_ARG, "null output pointer");
  *out = nullptr;
  if (n_cases < 1 || !cfgs) return fail(nullptr, LBM_ERR_ARG, "a batch needs at least one case");
  for (int c = 0; c < n_cases; ++c) {
    int rc = validate(&cfgs[c]);
    if (rc) return fail(nullptr, rc, "case " + std::to_string(c) + ": " + g_create_error);
    const lbm_config& k = cfgs[c];
    if (k.nz != 1 || k.S != 0) return fail(nullptr, LBM_ERR_ARG, "batched cases are 2-D and without surface mechanism");
    if (k.M != cfgs[0].M || (k.energy != 0) != (cfgs[0].energy != 0) || k.precision != cfgs[0].precision)
      return fail(nullptr, LBM_ERR_ARG, "batched cases must share M, the energy flag and the precision");
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1) return fail(nullptr, LBM_ERR_CUDA, "no CUDA device");
  lbm_ctx* x = new (std::nothrow) lbm_ctx();
  if (!x) return fail(nullptr, LBM_ERR_ALLOC, "host allocation failed");
  const lbm_config& c0 = cfgs[0];
  x->D = 2;
  x->Q = 9;
  x->nz = 1;
  x->M = c0.M;
  x->energy = c0.energy ? 1 : 0;
  x->L = x->M + 1 + x->energy;
  x->precision = c0.precision;
  x->stream = (cudaStream_t)c0.stream;
  x->n_cases = n_cases;
  x->variant = 2;
  bool ok = (x->precision == LBM_FP64)
                ? lbm::get_ops_f64_2d(x->M, x->energy, &x->od) && lbm::get_batch_ops_f64(x->M, x->energy, &x->bd)
                : lbm::get_ops_f32_2d(x->M, x->energy, &x->of) && lbm::get_batch_ops_f32(x->M, x->energy, &x->bf);
  if (!ok) {
    delete x;
    return fail(nullptr, LBM_ERR_ARG, "batched cases need (M, energy) = (2, off) or (3, on)");
  }
  long long off = 0;
  x->case_pd.resize(n_cases);
  x->case_pf.resize(n_cases);
  x->case_itd.resize(n_cases);
  x->case_itf.resize(n_cases);
  for (int c = 0; c < n_cases; ++c) {
    double dt = 0, cvel = 0;
    lbm::make_params(&cfgs[c], x->case_pd[c], x->case_itd[c], dt, cvel);
    convert_params(x->case_pd[c], x->case_pf[c]);
    convert_inlet(x->case_itd[c], x->case_itf[c]);
    x->case_dt.push_back(dt);
    x->case_cvel.push_back(cvel);
    x->case_N.push_back(cfgs[c].nx * cfgs[c].ny);
    x->case_nx.push_back(cfgs[c].nx);
    x->case_ny.push_back(cfgs[c].ny);
    x->case_node_off.push_back(off);
    off += (long long)cfgs[c].nx * cfgs[c].ny;
  }
  if (off > 2000000000LL) {
    delete x;
    return fail(nullptr, LBM_ERR_ARG, "batch too large");
  }
  x->N = (int)off;
  x->nx = c0.nx;
  x->ny = c0.ny;
  x->dt = x->case_dt[0];
  x->cvel = x->case_cvel[0];
  const size_t N = x->N, rs = real_size(x);
  const size_t pop_bytes = (size_t)x->L * x->Q * N * rs;
  void** slots[6] = {&x->pops[0], &x->pops[1], &x->phi, &x->Tfix, &x->mac, (void**)&x->status};
  const size_t sizes[6] = {pop_bytes, pop_bytes, N * rs, N * rs, (size_t)(2 * x->D + x->M) * N * rs, 64};
  for (int k = 0; k < 6; ++k) {
    e = cudaMalloc(slots[k], sizes[k]);
    if (e != cudaSuccess) {
      lbm_destroy(x);
      return fail(nullptr, LBM_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  // static fields, concatenated over cases in the working precision
  std::vector<double> phi_all(N), T_all(N);
  for (int c = 0; c < n_cases; ++c) {
    std::memcpy(&phi_all[x->case_node_off[c]], cfgs[c].porosity, x->case_N[c] * sizeof(double));
    std::memcpy(&T_all[x->case_node_off[c]], cfgs[c].T_init, x->case_N[c] * sizeof(double));
  }
  std::vector<char> hbuf(N * rs);
  auto upload = [&](void* dst, const double* src) -> cudaError_t {
    if (rs == 8) std::memcpy(hbuf.data(), src, N * 8);
    else for (size_t n = 0; n < N; ++n) ((float*)hbuf.data())[n] = (float)src[n];
    return cudaMemcpy(dst, hbuf.data(), N * rs, cudaMemcpyHostToDevice);
  };
  e = upload(x->phi, phi_all.data());
  if (e == cudaSuccess) e = upload(x->Tfix, T_all.data());
  if (e == cudaSuccess) e = cudaMemset(x->status, 0, 64);
  // per-case equilibrium initialisation with the case's own parameters
  for (int c = 0; c < n_cases && e == cudaSuccess; ++c) {
    const lbm_config& k = cfgs[c];
    const size_t Nc = x->case_N[c], nb = Nc * sizeof(double);
    const size_t o = (size_t)x->case_node_off[c];
    double *dX = nullptr, *dT = nullptr, *dP = nullptr, *dU = nullptr;
    e = cudaMalloc(&dX, nb * x->M);
    if (e == cudaSuccess) e = cudaMalloc(&dT, nb);
    if (e == cudaSuccess) e = cudaMalloc(&dP, nb);
    if (e == cudaSuccess && k.U_init) e = cudaMalloc(&dU, nb * 3);
    if (e == cudaSuccess) e = cudaMemcpy(dX, k.X_init, nb * x->M, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dT, k.T_init, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dP, k.P_init, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && k.U_init) e = cudaMemcpy(dU, k.U_init, nb * 3, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      if (x->precision == LBM_FP64)
        x->od.init(x->case_pd[c], dX, dT, dP, dU, x->case_cvel[c], R_UNIV_SI,
                   (double*)x->pops[0] + o * x->L * x->Q, (const double*)x->phi + o, x->stream);
      else
        x->of.init(x->case_pf[c], dX, dT, dP, dU, x->case_cvel[c], R_UNIV_SI,
                   (float*)x->pops[0] + o * x->L * x->Q, (const float*)x->phi + o, x->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
    cudaFree(dX); cudaFree(dT); cudaFree(dP); if (dU) cudaFree(dU);
  }
  // case table and the work lists of node tiles
  if (e == cudaSuccess)
    e = x->precision == LBM_FP64 ? upload_cases(x, x->case_pd, x->case_itd) : upload_cases(x, x->case_pf, x->case_itf);
  const int tl[3] = {64, 128, 256};
  for (int t = 0; t < 3 && e == cudaSuccess; ++t) {
    std::vector<int2> tiles;
    for (int c = 0; c < n_cases; ++c)
      for (int n0 = 0; n0 < x->case_N[c]; n0 += tl[t]) tiles.push_back(make_int2(c, n0));
    x->ntiles[t] = (int)tiles.size();
    e = cudaMalloc(&x->tiles_dev[t], tiles.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(x->tiles_dev[t], tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice);
  }
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&x->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    lbm_destroy(x);
    return cuda_fail(nullptr, e, "batch initialisation");
  }
  *out = x;
  return LBM_OK;
}

static int read_status(lbm_ctx* x) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, x->status, sizeof(int), cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_fail(x, e, "status read");
  if (st & 1) return fail(x, LBM_ERR_NUMERIC, "non-finite or non-positive density or temperature");
  if (st & lbm::kStatusTimeout) return fail(x, LBM_ERR_TIMEOUT, "a bounded device wait gave up");
  return LBM_OK;
}

}  // extern "C"

// Records a start/stop event pair around one launch when timing is on.
template <class F>
static void timed(lbm_ctx* x, int kind, F&& launch) {
  const size_t kMaxLaunches = 65536;
  if (!x->timing || x->ev_used >= kMaxLaunches) {
    launch();
    return;
  }
  if (x->ev.size() < 2 * (x->ev_used + 1)) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      launch();
      return;
    }
    x->ev.push_back(a);
    x->ev.push_back(b);
    x->ev_kind.push_back(kind);
  }
  x->ev_kind[x->ev_used] = kind;
  cudaEventRecord(x->ev[2 * x->ev_used], x->stream);
  launch();
  cudaEventRecord(x->ev[2 * x->ev_used + 1], x->stream);
  x->ev_used++;
}

// One time step with the context's kernel form: variant < 0 is the two-pass
// form, variant >= 0 the fused kernel with that tile shape.
template <class R>
static int launch_step(lbm_ctx* x, const lbm::Ops<R>& ops, const lbm::Params<R>& p, const lbm::InletTables<R>& it) {
  lbm::StepArgs<R> a{(const R*)x->pops[x->cur], (R*)x->pops[1 - x->cur], (const R*)x->phi, (const R*)x->Tfix,
                     (R*)x->mac, x->status};
  int rc = 0;
  if (x->variant < 0) {
    timed(x, 0, [&] { ops.macro(p, it, a, x->stream); });
    timed(x, 1, [&] { ops.collide(p, it, a, x->stream); });
  } else {
    timed(x, 1, [&] { rc = ops.fused(p, it, a, x->variant, x->stream); });
  }
  return rc;
}

// Reactive step: macro fields and surface source, then the node update with
// the reaction sources (two-pass form).
template <class R>
static void launch_react(lbm_ctx* x, const lbm::Ops<R>& ops, const lbm::Params<R>& p,
                         const lbm::InletTables<R>& it) {
  lbm::StepArgs<R> a{(const R*)x->pops[x->cur], (R*)x->pops[1 - x->cur], (const R*)x->phi, (const R*)x->Tfix,
                     (R*)x->mac, x->status};
  lbm::ReactArgs ra{x->mech, x->Xs[x->xs_cur], x->Xs[1 - x->xs_cur], x->rsrc};
  timed(x, 0, [&] { ops.react_macro(p, it, a, ra, x->stream); });
  timed(x, 1, [&] { ops.react_collide(p, it, a, ra, x->stream); });
  x->xs_cur = 1 - x->xs_cur;
}

// ---------------------------------------------------------------------------
// Batched form
// ---------------------------------------------------------------------------
constexpr int kGraphSteps = 50;    // even: a replay returns to the same ping-pong buffer

template <class R>
static lbm::BatchArgs<R> batch_args(lbm_ctx* x, int cur) {
  const int t = (x->variant % 6) / 2;
  return lbm::BatchArgs<R>{(const lbm::CaseDev<R>*)x->cases_dev, x->tiles_dev[t], x->ntiles[t],
                           (const R*)x->pops[cur], (R*)x->pops[1 - cur], (const R*)x->phi, (const R*)x->Tfix,
                           (R*)x->mac, x->status};
}

template <class R>
static int batch_grid(lbm_ctx* x, const lbm::BatchOps<R>& ops) {
  const int nt = x->ntiles[(x->variant % 6) / 2];
  if (x->variant % 2) return nt;
  const int g = x->sm_count * ops.occupancy(x->variant);
  return g < nt ? g : nt;
}

template <class R>
static void batch_launch(lbm_ctx* x, const lbm::BatchOps<R>& ops, int cur, cudaStream_t s) {
  const lbm::BatchArgs<R> a = batch_args<R>(x, cur);
  const int grid = batch_grid(x, ops);
  ops.pass(a, x->variant, grid, 0, s);
  ops.pass(a, x->variant, grid, 1, s);
}

static void drop_graphs(lbm_ctx* x) {
  for (int k = 0; k < 2; ++k)
    if (x->gexec[k]) {
      cudaGraphExecDestroy(x->gexec[k]);
      x->gexec[k] = nullptr;
    }
}

// Captures kGraphSteps steps starting from buffer `cur` with the current variant.
template <class R>
static cudaError_t batch_capture(lbm_ctx* x, const lbm::BatchOps<R>& ops, int cur) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int s = 0; s < kGraphSteps; ++s) batch_launch(x, ops, (cur + s) & 1, x->cap_stream);
  e = cudaStreamEndCapture(x->cap_stream, &g);
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&x->gexec[cur], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) x->gexec[cur] = nullptr;
  x->gvariant[cur] = x->variant;
  return e;
}

// n steps of every case: whole graphs of kGraphSteps steps, then single steps.
// With timing on, every kernel is launched (and timed) directly instead.
template <class R>
static int batch_steps(lbm_ctx* x, const lbm::BatchOps<R>& ops, int n) {
  if (!x->timing) {
    while (n >= kGraphSteps) {
      if (!x->gexec[x->cur] || x->gvariant[x->cur] != x->variant) {
        if (x->gexec[x->cur]) {
          cudaGraphExecDestroy(x->gexec[x->cur]);
          x->gexec[x->cur] = nullptr;
        }
        cudaError_t e = batch_capture(x, ops, x->cur);
        if (e != cudaSuccess) return cuda_fail(x, e, "graph capture");
      }
      cudaError_t e = cudaGraphLaunch(x->gexec[x->cur], x->stream);
      if (e != cudaSuccess) return cuda_fail(x, e, "graph launch");
      n -= kGraphSteps;
    }
  }
  for (; n > 0; --n) {
    const lbm::BatchArgs<R> a = batch_args<R>(x, x->cur);
    const int grid = batch_grid(x, ops);
    timed(x, 0, [&] { ops.pass(a, x->variant, grid, 0, x->stream); });
    timed(x, 1, [&] { ops.pass(a, x->variant, grid, 1, x->stream); });
    x->cur = 1 - x->cur;
  }
  return LBM_OK;
}

static int step_once(lbm_ctx* x) {
  if (x->n_cases > 0)
    return x->precision == LBM_FP64 ? batch_steps(x, x->bd, 1) : batch_steps(x, x->bf, 1);
  if (x->S > 0) {
    if (x->precision == LBM_FP64) launch_react(x, x->od, x->pd, x->itd);
    else launch_react(x, x->of, x->pf, x->itf);
    x->cur = 1 - x->cur;
    return LBM_OK;
  }
  int rc = (x->precision == LBM_FP64) ? launch_step(x, x->od, x->pd, x->itd) : launch_step(x, x->of, x->pf, x->itf);
  if (rc < 0) return fail(x, LBM_ERR_CUDA, "fused kernel configuration failed");
  x->cur = 1 - x->cur;
  return LBM_OK;
}

// gather (get) / scatter of the x columns [x0, x0 + ncols) of rows of nx values
namespace {
template <class T>
__global__ void k_columns(T* __restrict__ pops, T* __restrict__ buf, long long rows, int nx, int x0, int ncols,
                          int get) {
  const long long total = rows * ncols;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / ncols;
    const int c = (int)(i - r * ncols);
    T* p = pops + r * nx + x0 + c;
    if (get) buf[i] = *p;
    else *p = buf[i];
  }
}
}  // namespace

// Single lattice without a surface mechanism: kGraphSteps steps from buffer
// `cur` captured on the private capture stream into one graph (small lattices
// are bound by the launch rate; the replay removes the per-launch host cost).
static cudaError_t single_capture(lbm_ctx* x, int cur) {
  cudaError_t e = cudaSuccess;
  if (!x->cap_stream) e = cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaStream_t keep = x->stream;
  const int cur0 = x->cur;
  x->stream = x->cap_stream;
  x->cur = cur;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    int rc = LBM_OK;
    for (int s = 0; s < kGraphSteps && rc == LBM_OK; ++s) rc = step_once(x);
    cudaError_t e2 = cudaStreamEndCapture(x->cap_stream, &g);
    e = (rc != LBM_OK) ? cudaErrorInvalidValue : e2;
  }
  x->stream = keep;
  x->cur = cur0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&x->gexec[cur], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) x->gexec[cur] = nullptr;
  x->gvariant[cur] = x->variant;
  return e;
}

extern "C" {

int lbm_step(lbm_ctx* x, int n_steps) {
  if (!x) return LBM_ERR_ARG;
  if (n_steps < 0) return fail(x, LBM_ERR_ARG, "negative step count");
  if (x->n_cases > 0) {
    int rc = x->precision == LBM_FP64 ? batch_steps(x, x->bd, n_steps) : batch_steps(x, x->bf, n_steps);
    if (rc) return rc;
    x->steps_done += n_steps;
    n_steps = 0;
  }
  if (x->S == 0 && !x->timing && n_steps > kGraphSteps) {
    // one plain step first (it configures the kernels), then whole graphs of
    // kGraphSteps steps (an even count: a replay ends on the buffer it began on)
    int rc = step_once(x);
    if (rc) return rc;
    ++x->steps_done;
    --n_steps;
    while (n_steps >= kGraphSteps) {
      if (!x->gexec[x->cur] || x->gvariant[x->cur] != x->variant) {
        if (x->gexec[x->cur]) {
          cudaGraphExecDestroy(x->gexec[x->cur]);
          x->gexec[x->cur] = nullptr;
        }
        cudaError_t e = single_capture(x, x->cur);
        if (e != cudaSuccess) return cuda_fail(x, e, "graph capture");
      }
      cudaError_t e = cudaGraphLaunch(x->gexec[x->cur], x->stream);
      if (e != cudaSuccess) return cuda_fail(x, e, "graph launch");
      n_steps -= kGraphSteps;
      x->steps_done += kGraphSteps;
    }
  }
  for (int s = 0; s < n_steps; ++s) {
    int rc = step_once(x);
    if (rc) return rc;
    ++x->steps_done;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(x, e, "step launch");
  return LBM_OK;
}

int lbm_variant_count(const lbm_ctx* x) {
  if (!x) return LBM_ERR_ARG;
  if (x->n_cases > 0) return x->precision == LBM_FP64 ? x->bd.n_variants : x->bf.n_variants;
  return x->precision == LBM_FP64 ? x->od.n_variants : x->of.n_variants;
}

int lbm_set_variant(lbm_ctx* x, int variant) {
  if (!x) return LBM_ERR_ARG;
  if (variant < (x->n_cases > 0 ? 0 : -1) || variant >= lbm_variant_count(x))
    return fail(x, LBM_ERR_ARG, "unknown kernel variant");
  x->variant = variant;
  return LBM_OK;
}

int lbm_get_variant(const lbm_ctx* x) { return x ? x->variant : LBM_ERR_ARG; }

int lbm_autotune(lbm_ctx* x, int steps, int* best) {
  if (!x || steps < 1) return LBM_ERR_ARG;
  const size_t bytes = lbm_population_bytes(x);
  void* save = nullptr;
  cudaError_t e = cudaMalloc(&save, bytes);
  if (e != cudaSuccess) return fail(x, LBM_ERR_ALLOC, "autotune scratch allocation failed");
  e = cudaMemcpyAsync(save, x->pops[x->cur], bytes, cudaMemcpyDeviceToDevice, x->stream);
  const int cur0 = x->cur, var0 = x->variant;
  const int timing0 = x->timing;
  x->timing = 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best_ms = 1e30f;
  int best_v = var0;
  const int nv = lbm_variant_count(x);
  for (int v = (x->n_cases > 0 ? 0 : -1); v < nv && e == cudaSuccess; ++v) {
    x->variant = v;
    if (step_once(x) != LBM_OK) continue;           // warm-up (also configures the kernel)
    cudaEventRecord(t0, x->stream);
    int rc = 0;
    for (int s = 0; s < steps && rc == 0; ++s) rc = step_once(x);
    cudaEventRecord(t1, x->stream);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (rc == 0 && e == cudaSuccess && cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best_v = v;
    }
    e = cudaGetLastError();
  }
  // restore the state and keep the fastest form
  x->cur = cur0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(x->pops[x->cur], save, bytes, cudaMemcpyDeviceToDevice, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  cudaFree(save);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  x->timing = timing0;
  x->variant = best_v;
  if (best) *best = best_v;
  if (e != cudaSuccess) return cuda_fail(x, e, "autotune");
  return LBM_OK;
}

int lbm_set_timing(lbm_ctx* x, int enable) {
  if (!x) return LBM_ERR_ARG;
  x->timing = enable ? 1 : 0;
  x->ev_used = 0;
  return LBM_OK;
}

int lbm_get_timing(lbm_ctx* x, double* ms, long long* launches) {
  if (!x || !ms || !launches) return LBM_ERR_ARG;
  if (!x->timing) return fail(x, LBM_ERR_STATE, "timing is off");
  cudaError_t e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_fail(x, e, "timing sync");
  for (int k = 0; k < 3; ++k) { ms[k] = 0.0; launches[k] = 0; }
  for (size_t i = 0; i < x->ev_used; ++i) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, x->ev[2 * i], x->ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(x, e, "event time");
    int k = x->ev_kind[i];
    ms[k] += t;
    launches[k] += 1;
  }
  return LBM_OK;
}

int lbm_moments(lbm_ctx* x, int which, void* out, size_t bytes, int out_on_device) {
  if (!x || !out) return LBM_ERR_ARG;
  const size_t N = x->N, M = x->M, D = x->D;
  size_t count;
  switch (which) {
    case LBM_MOM_RHO_A: count = M * N; break;
    case LBM_MOM_J_A: case LBM_MOM_V_A: case LBM_MOM_N_A: count = M * D * N; break;
    case LBM_MOM_RHO: case LBM_MOM_T: case LBM_MOM_P: case LBM_MOM_RHO_S: count = N; break;
    case LBM_MOM_U: count = D * N; break;
    case LBM_MOM_CURRENT: {
      // the surface-source pass of the next step, run on the current state
      // into the scratch it owns (sources, macro fields, next coverages)
      count = N;
      if (bytes < count * sizeof(double)) return fail(x, LBM_ERR_ARG, "output buffer too small");
      cudaError_t e2 = cudaSuccess;
      if (x->S == 0 || x->n_cases > 0) {
        std::vector<double> zero(N, 0.0);
        e2 = cudaMemcpyAsync(out, zero.data(), count * sizeof(double),
                             out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, x->stream);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(x->stream);
        return e2 == cudaSuccess ? LBM_OK : cuda_fail(x, e2, "current copy");
      }
      lbm::ReactArgs ra{x->mech, x->Xs[x->xs_cur], x->Xs[1 - x->xs_cur], x->rsrc};
      if (x->precision == LBM_FP64) {
        lbm::StepArgs<double> a{(const double*)x->pops[x->cur], nullptr, (const double*)x->phi,
                                (const double*)x->Tfix, (double*)x->mac, x->status};
        x->od.react_macro(x->pd, x->itd, a, ra, x->stream);
      } else {
        lbm::StepArgs<float> a{(const float*)x->pops[x->cur], nullptr, (const float*)x->phi,
                               (const float*)x->Tfix, (float*)x->mac, x->status};
        x->of.react_macro(x->pf, x->itf, a, ra, x->stream);
      }
      e2 = cudaGetLastError();
      if (e2 == cudaSuccess)
        e2 = cudaMemcpyAsync(out, x->rsrc + (size_t)(M + 1) * N, count * sizeof(double),
                             out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, x->stream);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(x->stream);
      return e2 == cudaSuccess ? LBM_OK : cuda_fail(x, e2, "current");
    }
    case LBM_MOM_XS: {
      count = (size_t)x->S * N;
      if (bytes < count * sizeof(double)) return fail(x, LBM_ERR_ARG, "output buffer too small");
      if (count == 0) return LBM_OK;
      cudaError_t e2 = cudaMemcpyAsync(out, x->Xs[x->xs_cur], count * sizeof(double),
                                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, x->stream);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(x->stream);
      return e2 == cudaSuccess ? LBM_OK : cuda_fail(x, e2, "coverage copy");
    }
    default: return fail(x, LBM_ERR_ARG, "unknown moment selector");
  }
  const size_t need = count * sizeof(double);
  if (bytes < need) return fail(x, LBM_ERR_ARG, "output buffer too small");
  if (count == 0) return LBM_OK;
  double* dout = (double*)out;
  cudaError_t e;
  if (which == LBM_MOM_XS && x->n_cases > 0) return fail(x, LBM_ERR_ARG, "batched cases have no surface");
  if (!out_on_device) {
    if (x->scratch_bytes < need) {
      if (x->scratch_out) cudaFree(x->scratch_out);
      x->scratch_out = nullptr;
      x->scratch_bytes = 0;
      e = cudaMalloc(&x->scratch_out, need);
      if (e != cudaSuccess) return fail(x, LBM_ERR_ALLOC, "moment scratch allocation failed");
      x->scratch_bytes = need;
    }
    dout = x->scratch_out;
  }
  if (x->n_cases > 0) {
    // each case writes its own single-lattice layout at its offset
    const size_t per_node = count / N;
    const size_t mac_fields = 2 * x->D + x->M;
    for (int c = 0; c < x->n_cases; ++c) {
      const size_t off = (size_t)x->case_node_off[c];
      const size_t pop_off = off * x->L * x->Q;
      if (x->precision == LBM_FP64) {
        lbm::StepArgs<double> a{(const double*)x->pops[x->cur] + pop_off, nullptr, (const double*)x->phi + off,
                                (const double*)x->Tfix + off, (double*)x->mac + off * mac_fields, x->status};
        x->od.moments(x->case_pd[c], x->case_itd[c], a, which, x->case_cvel[c], dout + off * per_node, x->stream);
      } else {
        lbm::StepArgs<float> a{(const float*)x->pops[x->cur] + pop_off, nullptr, (const float*)x->phi + off,
                               (const float*)x->Tfix + off, (float*)x->mac + off * mac_fields, x->status};
        x->of.moments(x->case_pf[c], x->case_itf[c], a, which, x->case_cvel[c], dout + off * per_node, x->stream);
      }
    }
  } else if (x->precision == LBM_FP64) {
    lbm::StepArgs<double> a{(const double*)x->pops[x->cur], nullptr, (const double*)x->phi, (const double*)x->Tfix,
                            (double*)x->mac, x->status};
    x->od.moments(x->pd, x->itd, a, which, x->cvel, dout, x->stream);
  } else {
    lbm::StepArgs<float> a{(const float*)x->pops[x->cur], nullptr, (const float*)x->phi, (const float*)x->Tfix,
                           (float*)x->mac, x->status};
    x->of.moments(x->pf, x->itf, a, which, x->cvel, dout, x->stream);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(x, e, "moments launch");
  if (!out_on_device) {
    e = cudaMemcpyAsync(out, dout, need, cudaMemcpyDeviceToHost, x->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
    if (e != cudaSuccess) return cuda_fail(x, e, "moments copy");
  }
  return LBM_OK;
}

size_t lbm_population_bytes(const lbm_ctx* x) {
  return x ? (size_t)x->L * x->Q * x->N * real_size(x) : 0;
}

int lbm_get_populations(lbm_ctx* x, void* buf, size_t bytes, int on_device) {
  if (!x || !buf) return LBM_ERR_ARG;
  if (bytes != lbm_population_bytes(x)) return fail(x, LBM_ERR_ARG, "population buffer size mismatch");
  cudaError_t e = cudaMemcpyAsync(buf, x->pops[x->cur], bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(x, e, "population copy");
}

int lbm_set_populations(lbm_ctx* x, const void* buf, size_t bytes, int on_device) {
  if (!x || !buf) return LBM_ERR_ARG;
  if (bytes != lbm_population_bytes(x)) return fail(x, LBM_ERR_ARG, "population buffer size mismatch");
  cudaError_t e = cudaMemcpyAsync(x->pops[x->cur], buf, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(x, e, "population copy");
}

// x columns [x0, x0 + ncols) of the stored populations <-> a packed buffer
// [L][Q][nz][ny][ncols]: L Q nz ny rows of ncols values.  Device buffers take
// a gather / scatter kernel (rows of a few values are far below what a
// pitched DMA copy moves efficiently), host buffers one pitched copy.
static int column_copy(lbm_ctx* x, int x0, int ncols, void* buf, size_t bytes, int on_device, bool get) {
  if (!x || !buf) return LBM_ERR_ARG;
  if (x->n_cases > 0) return fail(x, LBM_ERR_STATE, "column copies: single lattices only");
  if (ncols < 1 || x0 < 0 || x0 + ncols > x->nx) return fail(x, LBM_ERR_ARG, "column range outside the lattice");
  const size_t rs = real_size(x);
  const size_t rows = (size_t)x->L * x->Q * x->ny * x->nz;
  if (bytes != rows * ncols * rs) return fail(x, LBM_ERR_ARG, "column buffer size mismatch");
  cudaError_t e = cudaSuccess;
  if (on_device) {
    const long long total = (long long)rows * ncols;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (rs == 8)
      k_columns<double><<<grid, 256, 0, x->stream>>>(static_cast<double*>(x->pops[x->cur]), static_cast<double*>(buf),
                                                     (long long)rows, x->nx, x0, ncols, get ? 1 : 0);
    else
      k_columns<float><<<grid, 256, 0, x->stream>>>(static_cast<float*>(x->pops[x->cur]), static_cast<float*>(buf),
                                                    (long long)rows, x->nx, x0, ncols, get ? 1 : 0);
    e = cudaGetLastError();
  } else {
    char* pops = static_cast<char*>(x->pops[x->cur]) + (size_t)x0 * rs;
    const size_t width = (size_t)ncols * rs, pitch = (size_t)x->nx * rs;
    e = get ? cudaMemcpy2DAsync(buf, width, pops, pitch, width, rows, cudaMemcpyDeviceToHost, x->stream)
            : cudaMemcpy2DAsync(pops, pitch, buf, width, width, rows, cudaMemcpyHostToDevice, x->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  }
  return e == cudaSuccess ? LBM_OK : cuda_fail(x, e, "column copy");
}

int lbm_get_columns(lbm_ctx* x, int x0, int ncols, void* buf, size_t bytes, int on_device) {
  return column_copy(x, x0, ncols, buf, bytes, on_device, true);
}

int lbm_set_columns(lbm_ctx* x, int x0, int ncols, const void* buf, size_t bytes, int on_device) {
  return column_copy(x, x0, ncols, const_cast<void*>(buf), bytes, on_device, false);
}

// checkpoint image: 128-byte header, populations, coverages
namespace {
constexpr size_t kImageHeader = 128;
constexpr long long kImageVersion = 1;
size_t coverage_bytes(const lbm_ctx* x) { return x->S > 0 ? (size_t)x->S * x->N * sizeof(double) : 0; }
void image_header(const lbm_ctx* x, long long* h /* [10] */) {
  h[0] = kImageVersion; h[1] = x->precision; h[2] = x->D; h[3] = x->N; h[4] = x->L; h[5] = x->Q;
  h[6] = x->S; h[7] = x->steps_done; h[8] = (long long)lbm_population_bytes(x); h[9] = (long long)coverage_bytes(x);
}
}  // namespace

int lbm_save(lbm_ctx* x, void* buf, size_t* bytes) {
  if (!x || !bytes) return LBM_ERR_ARG;
  const size_t pb = lbm_population_bytes(x), cb = coverage_bytes(x);
  const size_t need = kImageHeader + pb + cb;
  if (!buf) {
    *bytes = need;
    return LBM_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return fail(x, LBM_ERR_ARG, "checkpoint buffer too small");
  }
  unsigned char* out = static_cast<unsigned char*>(buf);
  std::memset(out, 0, kImageHeader);
  std::memcpy(out, "LBMSTATE", 8);
  long long h[10];
  image_header(x, h);
  std::memcpy(out + 8, h, sizeof(h));
  cudaError_t e = cudaMemcpyAsync(out + kImageHeader, x->pops[x->cur], pb, cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess && cb)
    e = cudaMemcpyAsync(out + kImageHeader + pb, x->Xs[x->xs_cur], cb, cudaMemcpyDeviceToHost, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_fail(x, e, "checkpoint copy");
  *bytes = need;
  return LBM_OK;
}

int lbm_load(lbm_ctx* x, const void* buf, size_t bytes) {
  if (!x || !buf) return LBM_ERR_ARG;
  const size_t pb = lbm_population_bytes(x), cb = coverage_bytes(x);
  if (bytes != kImageHeader + pb + cb) return fail(x, LBM_ERR_ARG, "checkpoint image size does not match the context");
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  if (std::memcmp(in, "LBMSTATE", 8) != 0) return fail(x, LBM_ERR_ARG, "not a checkpoint image");
  long long h[10], mine[10];
  std::memcpy(h, in + 8, sizeof(h));
  image_header(x, mine);
  for (int k = 0; k < 10; ++k)
    if (k != 7 && h[k] != mine[k]) return fail(x, LBM_ERR_ARG, "checkpoint image does not match the context");
  cudaError_t e = cudaMemcpyAsync(x->pops[x->cur], in + kImageHeader, pb, cudaMemcpyHostToDevice, x->stream);
  if (e == cudaSuccess && cb)
    e = cudaMemcpyAsync(x->Xs[x->xs_cur], in + kImageHeader + pb, cb, cudaMemcpyHostToDevice, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  if (e != cudaSuccess) return cuda_fail(x, e, "checkpoint copy");
  x->steps_done = h[7];
  return LBM_OK;
}

static void release_streaming(lbm_ctx* x) {
  if (x->d2h) cudaStreamSynchronize(x->d2h);
  if (x->h2d) cudaStreamSynchronize(x->h2d);
  for (int k = 0; k < 4; ++k)
    if (x->hslot[k]) cudaFree(x->hslot[k]), x->hslot[k] = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (x->ev_in[k]) cudaEventDestroy(x->ev_in[k]), x->ev_in[k] = nullptr;
    if (x->ev_done[k]) cudaEventDestroy(x->ev_done[k]), x->ev_done[k] = nullptr;
    if (x->ev_free[k]) cudaEventDestroy(x->ev_free[k]), x->ev_free[k] = nullptr;
    x->free_recorded[k] = false;
  }
  if (x->h2d) cudaStreamDestroy(x->h2d), x->h2d = nullptr;
  if (x->d2h) cudaStreamDestroy(x->d2h), x->d2h = nullptr;
}

int lbm_step_host(lbm_ctx* x, const void* in_host, void* out_host, int n_steps) {
  if (!x) return LBM_ERR_ARG;
  if (!in_host || !out_host || n_steps < 0) return fail(x, LBM_ERR_ARG, "lbm_step_host: null buffer or negative step count");
  if (x->n_cases > 0 || x->S > 0)
    return fail(x, LBM_ERR_STATE, "lbm_step_host: single lattices without a surface mechanism only");
  const size_t pb = lbm_population_bytes(x);
  cudaError_t e = cudaSuccess;
  if (!x->h2d) {
    e = cudaStreamCreateWithFlags(&x->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x->d2h, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&x->ev_in[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->ev_done[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x->ev_free[k], cudaEventDisableTiming);
    }
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaMalloc(&x->hslot[k], pb);
    if (e != cudaSuccess) {
      release_streaming(x);
      return fail(x, LBM_ERR_ALLOC, std::string("lbm_step_host: stream or slot allocation failed: ") +
                                        cudaGetErrorString(e));
    }
  }
  const int P = (int)(x->hcall & 1);
  void* sa = x->hslot[2 * P];
  void* sb = x->hslot[2 * P + 1];
  // upload once the download of the pair's previous call has finished
  if (x->free_recorded[P]) e = cudaStreamWaitEvent(x->h2d, x->ev_free[P], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sa, in_host, pb, cudaMemcpyHostToDevice, x->h2d);
  if (e == cudaSuccess) e = cudaEventRecord(x->ev_in[P], x->h2d);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(x->stream, x->ev_in[P], 0);
  if (e != cudaSuccess) return cuda_fail(x, e, "lbm_step_host upload");
  // the steps ping-pong between the pair's slots on the context's stream
  void* keep0 = x->pops[0];
  void* keep1 = x->pops[1];
  const int keep_cur = x->cur;
  x->pops[0] = sa;
  x->pops[1] = sb;
  x->cur = 0;
  int rc = LBM_OK;
  for (int s = 0; s < n_steps && rc == LBM_OK; ++s) rc = step_once(x);
  void* result = x->pops[x->cur];
  x->pops[0] = keep0;
  x->pops[1] = keep1;
  x->cur = keep_cur;
  if (rc != LBM_OK) return rc;
  e = cudaEventRecord(x->ev_done[P], x->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(x->d2h, x->ev_done[P], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, result, pb, cudaMemcpyDeviceToHost, x->d2h);
  if (e == cudaSuccess) e = cudaEventRecord(x->ev_free[P], x->d2h);
  if (e != cudaSuccess) return cuda_fail(x, e, "lbm_step_host download");
  x->free_recorded[P] = true;
  ++x->hcall;
  return LBM_OK;
}

int lbm_set_wait_limit(lbm_ctx* x, int probes) {
  if (!x) return LBM_ERR_ARG;
  if (probes < 0) return fail(x, LBM_ERR_ARG, "negative wait limit");
  x->pd.wait_limit = probes;
  x->pf.wait_limit = probes;
  drop_graphs(x);                    // captured launches carry the old parameters
  return LBM_OK;
}

int lbm_set_potential(lbm_ctx* x, const double* field, double uniform) {
  if (!x) return LBM_ERR_ARG;
  if (x->S == 0 || x->n_cases > 0) return fail(x, LBM_ERR_STATE, "no surface mechanism");
  cudaError_t e = cudaSuccess;
  const double* dev = nullptr;
  if (field) {
    if (!x->dphi_dev) e = cudaMalloc(&x->dphi_dev, (size_t)x->N * sizeof(double));
    if (e != cudaSuccess) return fail(x, LBM_ERR_ALLOC, "potential field allocation failed");
    e = cudaMemcpyAsync(x->dphi_dev, field, (size_t)x->N * sizeof(double), cudaMemcpyHostToDevice, x->stream);
    dev = x->dphi_dev;
  }
  char* m = reinterpret_cast<char*>(x->mech);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m + offsetof(lbm::MechDev, dphi), &uniform, sizeof(double), cudaMemcpyHostToDevice, x->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m + offsetof(lbm::MechDev, dphi_field), &dev, sizeof(dev), cudaMemcpyHostToDevice, x->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
  return e == cudaSuccess ? LBM_OK : cuda_fail(x, e, "potential upload");
}

int lbm_sync(lbm_ctx* x) {
  if (!x) return LBM_ERR_ARG;
  if (x->h2d) {
    cudaError_t e = cudaStreamSynchronize(x->h2d);
    if (e == cudaSuccess) e = cudaStreamSynchronize(x->d2h);
    if (e != cudaSuccess) return cuda_fail(x, e, "copy stream synchronisation");
  }
  return read_status(x);
}

int lbm_case_info(const lbm_ctx* x, int c, double* out6) {
  if (!x || !out6) return LBM_ERR_ARG;
  if (x->n_cases == 0) {
    if (c != 0) return LBM_ERR_ARG;
    out6[0] = x->dt; out6[1] = x->cvel; out6[2] = x->N; out6[3] = x->nx; out6[4] = x->ny; out6[5] = 0;
    return LBM_OK;
  }
  if (c < 0 || c >= x->n_cases) return LBM_ERR_ARG;
  out6[0] = x->case_dt[c];
  out6[1] = x->case_cvel[c];
  out6[2] = x->case_N[c];
  out6[3] = x->case_nx[c];
  out6[4] = x->case_ny[c];
  out6[5] = (double)(x->case_node_off[c] * x->L * x->Q);
  return LBM_OK;
}

int lbm_info(const lbm_ctx* x, double* out5) {
  if (!x || !out5) return LBM_ERR_ARG;
  out5[0] = x->dt;
  out5[1] = x->cvel;
  out5[2] = x->L;
  out5[3] = x->Q;
  out5[4] = x->D;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* x) {
  if (!x) return;
  cudaStreamSynchronize(x->stream);
  release_streaming(x);
  void* bufs[16] = {x->pops[0], x->pops[1], x->phi, x->Tfix, x->mac, x->status, x->scratch_out,
                   x->Xs[0], x->Xs[1], x->rsrc, x->mech, x->init_X, x->init_T, x->init_P, x->init_U,
                   x->dphi_dev};
  for (void* b : bufs)
    if (b) cudaFree(b);
  drop_graphs(x);
  if (x->cases_dev) cudaFree(x->cases_dev);
  for (int t = 0; t < 3; ++t)
    if (x->tiles_dev[t]) cudaFree(x->tiles_dev[t]);
  if (x->cap_stream) cudaStreamDestroy(x->cap_stream);
  for (cudaEvent_t ev : x->ev) cudaEventDestroy(ev);
  delete x;
}

const char* lbm_last_error(const lbm_ctx* x) {
  return x ? x->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
