// Heterogeneous surface source on the GPU (Sec. 4, Sec. 4.2) and the
// reactive two-pass step that applies it.
//
// Per node and step: mass-action rates with Arrhenius constants, backward
// Euler in the reaction extents over the physical time step solved by
// Newton's method (analytic sparse Jacobian, Gaussian elimination with
// partial pivoting, steps shortened so that no concentration crosses zero).
// Rates, residual and extents are FP64 whatever the population precision;
// the Jacobian is FP64 on the FP64 path and FP32 on the FP32 path, and is
// reused across iterations (iterative refinement to the same FP64 root).  Then the gas mass production
// (Eq. 68, Eq. 69), the new coverages
// (Eq. 70, Eq. 71 with the TPB edge
// steps), the volumetric current (Eq. 74) and the change of the
// fluid internal energy: the unified internal energy of fluid and adsorbed
// phases (Eq. 80, Eq. 85) gains the ohmic heat
// and loses the electric power of the current (Sec. 4.2).
#pragma once

#include "lbm_compact.cuh"

namespace lbm {

constexpr double R_UNIV_DEV = 8.314462618;    // J/(mol K)

// Mechanism and unit data of a reactive context (device memory, read-only).
// Species are indexed 0..M-1 (gas, mol/m^3 of fluid) then M..M+S-1 (surface,
// mol/m^2); reactant lists hold the integer mass-action orders.
struct MechDev {
  int M, S, R;
  double nu_g[RMAX][MMAX];
  double nu_s[RMAX][SMAX];
  double nu_all[RMAX][MMAX + SMAX];
  int npart[RMAX];                   // species taking part in each step (nonzero stoichiometry)
  int pidx[RMAX][8];
  double pnu[RMAX][8];
  int nsr[MMAX + SMAX];               // steps in which each species takes part
  int sr_k[MMAX + SMAX][RMAX];
  float sr_nuf[MMAX + SMAX][RMAX];
  double sr_nud[MMAX + SMAX][RMAX];
  int nre[RMAX];                     // reactants of each step
  int ridx[RMAX][4];
  int rord[RMAX][4];
  double A[RMAX], Ea[RMAX];
  double gamma, a_s;
  double cvs[SMAX], Us0[SMAX];       // molar C_v / R_U and molar U at T_thermo of the adsorbates
  double m[MMAX];                    // gas molar masses
  double T_thermo;
  double dt;                         // physical time step [s]
  double cvel2;                      // (dx/dt)^2 [m^2/s^2]
  // electrochemistry: TPB (edge) steps run as surface steps whose extent is
  // counted per unit surface (the per-length extent times l_tpb/a_s), so
  // their constants carry the factor l_tpb/a_s and the potential factor
  int edge[RMAX];
  double nel[RMAX];                  // electrons released per step
  double l_tpb, beta_ct, resist, dphi, dx;
  const double* dphi_field;          // per-node potential difference [N] (null: dphi everywhere)
};

constexpr double FARADAY_DEV = 96485.33212;   // C/mol

// stoichiometric coefficient of species i in its q-th step, in the Jacobian's precision
template <class RK> __device__ __forceinline__ RK sr_nu(const MechDev& mc, int i, int q);
template <> __device__ __forceinline__ float sr_nu<float>(const MechDev& mc, int i, int q) { return mc.sr_nuf[i][q]; }
template <> __device__ __forceinline__ double sr_nu<double>(const MechDev& mc, int i, int q) { return mc.sr_nud[i][q]; }

__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  for (int k = 0; k < n; ++k) r *= x;
  return r;
}

// Surface source of one node.  rho_a in kg/m^3 of fluid, T in K; returns
// rhodot[a] (kg/m^3 of porous medium per step), the new coverages and dU
// (fluid internal energy change per unit volume, lattice units).
//
// Mixed precision (iterative refinement): concentrations, rates, the
// residual F = xi - dt r(xi) and the extents are FP64; the Newton systems are
// solved in FP32 (RK = float) or FP64 (RK = double) through the species-space
// matrix K = I - V U of the Woodbury identity (NS x NS instead of R x R),
// whose factors are reused across iterations (simplified Newton) until the
// contraction of the steps slows down or a step is shortened, when they are
// rebuilt at the current iterate.  The FP64 residual fixes the root, so every variant
// converges to the same FP64 solution.
template <int M, class RK>
__device__ void surface_source_dev(const MechDev& mc, double T, const double* rho_a, double phi, const double* Xs0,
                                   double* rhodot, double* Xs1, double& dU, double& current, double dphi,
                                   int* status) {
  const int S = mc.S, Rn = mc.R, NS = M + mc.S;
  double c0[MMAX + SMAX], kr[RMAX], xi[RMAX];
  for (int a = 0; a < M; ++a) c0[a] = rho_a[a] / mc.m[a];
  for (int s = 0; s < S; ++s) c0[M + s] = mc.gamma * Xs0[s];
  for (int k = 0; k < Rn; ++k) {
    kr[k] = mc.A[k] * exp(-mc.Ea[k] / (R_UNIV_DEV * T));
    // TPB step: rate per unit TPB length, extent counted per unit surface
    if (mc.edge[k])
      kr[k] *= (mc.l_tpb / mc.a_s) * exp(mc.beta_ct * mc.nel[k] * FARADAY_DEV * dphi / (R_UNIV_DEV * T));
    xi[k] = 0.0;
  }
  const double scale = mc.a_s / phi;     // gas concentration change per extent
  // J = I - U V with U = dt dr/dc (R x NS, the reactants of each step) and
  // V = diag(scale) nu^T (NS x R); by the Woodbury identity
  // J^-1 b = b + U K^-1 V b with K = I - V U (NS x NS), whose LU factors and U
  // are kept while the iteration reuses them.
  constexpr int NSX = MMAX + SMAX;
  RK LU[NSX][NSX];
  RK uk[RMAX][4];
  int swp[NSX];
  bool refresh = true, converged = false;
  double prev = 0.0;
  for (int it = 0; it < 40; ++it) {
    double c[MMAX + SMAX], r[RMAX];
    // c = c0 + (scaled) nu^T xi, over the few species of each step
    double d[MMAX + SMAX];
    for (int i = 0; i < NS; ++i) d[i] = 0.0;
    for (int k = 0; k < Rn; ++k)
      for (int j = 0; j < mc.npart[k]; ++j) d[mc.pidx[k][j]] += mc.pnu[k][j] * xi[k];
    for (int i = 0; i < NS; ++i) c[i] = c0[i] + (i < M ? scale : 1.0) * d[i];
    for (int k = 0; k < Rn; ++k) {
      double v = kr[k];
      for (int j = 0; j < mc.nre[k]; ++j) v *= ipow(fmax(c[mc.ridx[k][j]], 0.0), mc.rord[k][j]);
      r[k] = v;
    }
    if (refresh) {
      // U entries dt r_k ord / c_j of the reactants j of each step, and K = I - V U
      for (int i = 0; i < NS; ++i)
        for (int j = 0; j < NS; ++j) LU[i][j] = (i == j) ? RK(1) : RK(0);
      for (int k = 0; k < Rn; ++k)
        for (int j = 0; j < mc.nre[k]; ++j) {
          const int jj = mc.ridx[k][j];
          const RK u = c[jj] > 0.0 ? RK(mc.dt * r[k] * mc.rord[k][j] / c[jj]) : RK(0);
          uk[k][j] = u;
          for (int q = 0; q < mc.npart[k]; ++q) {
            const int i = mc.pidx[k][q];
            LU[i][jj] -= RK((i < M ? scale : 1.0) * mc.pnu[k][q]) * u;
          }
        }
      // LU factors of K with partial pivoting (row swaps recorded in swp)
      for (int cc = 0; cc < NS; ++cc) {
        int pv = cc;
        for (int k = cc + 1; k < NS; ++k)
          if (fabs(LU[k][cc]) > fabs(LU[pv][cc])) pv = k;
        swp[cc] = pv;
        if (pv != cc)
          for (int l = 0; l < NS; ++l) {
            RK t = LU[cc][l];
            LU[cc][l] = LU[pv][l];
            LU[pv][l] = t;
          }
        const RK inv = RK(1) / LU[cc][cc];
        for (int k = cc + 1; k < NS; ++k) {
          const RK f = LU[k][cc] * inv;
          LU[k][cc] = f;
          for (int l = cc + 1; l < NS; ++l) LU[k][l] -= f * LU[cc][l];
        }
      }
      refresh = false;
    }
    // solve J dxi = -F:  w = V b, K z = w, dxi = b + U z
    RK b[RMAX], w[NSX];
    for (int k = 0; k < Rn; ++k) b[k] = RK(-(xi[k] - mc.dt * r[k]));
    for (int i = 0; i < NS; ++i) w[i] = RK(0);
    for (int k = 0; k < Rn; ++k)
      for (int q = 0; q < mc.npart[k]; ++q) {
        const int i = mc.pidx[k][q];
        w[i] += RK((i < M ? scale : 1.0) * mc.pnu[k][q]) * b[k];
      }
    for (int cc = 0; cc < NS; ++cc)
      if (swp[cc] != cc) {
        RK t = w[cc];
        w[cc] = w[swp[cc]];
        w[swp[cc]] = t;
      }
    for (int k = 1; k < NS; ++k)
      for (int l = 0; l < k; ++l) w[k] -= LU[k][l] * w[l];
    for (int k = NS - 1; k >= 0; --k) {
      RK s2 = w[k];
      for (int l = k + 1; l < NS; ++l) s2 -= LU[k][l] * w[l];
      w[k] = s2 / LU[k][k];
    }
    double dxi[RMAX];
    for (int k = 0; k < Rn; ++k) {
      RK x = b[k];
      for (int j = 0; j < mc.nre[k]; ++j) x += uk[k][j] * w[mc.ridx[k][j]];
      dxi[k] = (double)x;
    }
    // steps that would take a non-negative concentration below zero are shortened
    double alpha = 1.0;
    {
      double dd[MMAX + SMAX];
      for (int i = 0; i < NS; ++i) dd[i] = 0.0;
      for (int k = 0; k < Rn; ++k)
        for (int j = 0; j < mc.npart[k]; ++j) dd[mc.pidx[k][j]] += mc.pnu[k][j] * dxi[k];
      for (int i = 0; i < NS; ++i) {
        const double di = dd[i] * (i < M ? scale : 1.0);
        if (c[i] >= 0.0 && c[i] + di < 0.0) alpha = fmin(alpha, 0.9 * c[i] / (-di));
      }
    }
    double dmax = 0.0, xmax = 0.0;
    for (int k = 0; k < Rn; ++k) {
      xi[k] += alpha * dxi[k];
      dmax = fmax(dmax, fabs(alpha * dxi[k]));
      xmax = fmax(xmax, fabs(xi[k]));
    }
    if (alpha == 1.0 && dmax <= 1e-14 * (xmax + 1e-300)) {
      converged = true;
      break;
    }
    // rebuild the Jacobian when a step was shortened or the steps stop contracting fast
    refresh = (alpha < 1.0) || (it > 0 && dmax > 0.25 * prev);
    prev = dmax;
  }
  if (!converged) flag(status, 4);
  // moles produced per unit surface, nu^T xi, over the few species of each step
  double dn_all[MMAX + SMAX];
  for (int i = 0; i < NS; ++i) dn_all[i] = 0.0;
  for (int k = 0; k < Rn; ++k)
    for (int j = 0; j < mc.npart[k]; ++j) dn_all[mc.pidx[k][j]] += mc.pnu[k][j] * xi[k];
  for (int a = 0; a < M; ++a) rhodot[a] = mc.a_s * mc.m[a] * dn_all[a];
  double dUs = 0.0;
  for (int s = 0; s < S; ++s) {
    const double dn = dn_all[M + s];
    Xs1[s] = Xs0[s] + dn / mc.gamma;
    const double Us = mc.Us0[s] + mc.cvs[s] * R_UNIV_DEV * (T - mc.T_thermo);
    dUs += mc.a_s * dn * Us;
  }
  // volumetric current: F a_s (electrons per unit surface) per second, the
  // same as F l_tpb (electrons per TPB length) per second
  double ne = 0.0;
  for (int k = 0; k < Rn; ++k)
    if (mc.edge[k]) ne += mc.nel[k] * xi[k];
  current = FARADAY_DEV * mc.a_s * ne / mc.dt;
  // ohmic heat stays in the fluid, electric power leaves (Sec. 4.2)
  double Usrc = 0.0;
  if (mc.l_tpb > 0.0)
    Usrc = ((mc.a_s / mc.l_tpb) * current * current * mc.resist * mc.dx - fabs(dphi) * current) * mc.dt;
  dU = (-dUs + Usrc) / mc.cvel2;
}

// Arguments of the reactive passes.
struct ReactArgs {
  const MechDev* mech;
  const double* Xs_in;     // [S][N]
  double* Xs_out;          // [S][N]
  double* src;             // [M + 2][N]: rhodot_a, then dU, then the volumetric current
};

// Pass 1: macro fields (as k_macro) plus the surface source of the node.
template <class R, int D, int M, bool EN>
__global__ void __launch_bounds__(128) k_macro_react(Params<R> p, InletTables<R> it, StepArgs<R> a, ReactArgs ra) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  macro_node<R, D, M, EN>(p, it, a, n);
  // the surface source needs the streamed species densities and temperature
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Site<R, D> st;
  st.init(p, x, y, z);
  Ghost<R, D> gh;
  gh.side = -1;
  if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
  Moments<R, D, M, EN, false> mo;
  moments_rt<R, D, M, EN, false>(p, it, a.src, st, gh, mo);
  State<R, D, M> s;
  s.template from_moments<EN, false>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
  const MechDev& mc = *ra.mech;
  double rho[MMAX], Xs0[SMAX], Xs1[SMAX], rd[MMAX], dU = 0.0, cur = 0.0;
  for (int k = 0; k < M; ++k) rho[k] = (double)s.rho_a[k];
  for (int k = 0; k < mc.S; ++k) Xs0[k] = ra.Xs_in[(size_t)k * p.N + n];
  const double dphi_n = mc.dphi_field ? mc.dphi_field[n] : mc.dphi;
  surface_source_dev<M, R>(mc, (double)s.T, rho, (double)s.phi, Xs0, rd, Xs1, dU, cur, dphi_n, a.status);
  for (int k = 0; k < M; ++k) ra.src[(size_t)k * p.N + n] = rd[k];
  ra.src[(size_t)M * p.N + n] = dU;
  ra.src[(size_t)(M + 1) * p.N + n] = cur;
  for (int k = 0; k < mc.S; ++k) ra.Xs_out[(size_t)k * p.N + n] = Xs1[k];
}

// Pass 2: node update with the reaction sources.
template <class R, int D, int M, bool EN>
__global__ void __launch_bounds__(128) k_collide_react(Params<R> p, InletTables<R> it, StepArgs<R> a, ReactArgs ra) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Site<R, D> st;
  st.init(p, x, y, z);
  Ghost<R, D> gh;
  gh.side = -1;
  if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
  Moments<R, D, M, EN, true> mo;
  moments_rt<R, D, M, EN, true>(p, it, a.src, st, gh, mo);
  State<R, D, M> s;
  s.template from_moments<EN, true>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
  Grad<R, D, M, EN> gr;
  const R* __restrict__ mac = a.mac;
  const int N = p.N;
  gr.compute(p, x, y, z, [&](int k, int nb) { return mac[(size_t)k * N + nb]; });
  NodeSource<R> src;
  for (int k = 0; k < M; ++k) src.rhodot[k] = (R)ra.src[(size_t)k * N + n];
  src.dU = (R)ra.src[(size_t)M * N + n];
  GlobalPull<R, D, M, EN> pf{p, it, a.src, st, gh};
  collide_gen<R, D, M, EN, GlobalPull<R, D, M, EN>, true>(p, pf, n, mo, s, gr, a.dst, a.status, &src);
}

}  // namespace lbm
