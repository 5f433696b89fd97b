// Kernels of the fused stream-and-collide step.  Included by the per-precision
// / per-dimension translation units, which instantiate them.
#pragma once

#include "lbm_node.cuh"

namespace lbm {

// Arguments shared by the step kernels (device pointers).
template <class R>
struct StepArgs {
  const R* __restrict__ src;     // post-collision populations of the previous step
  R* __restrict__ dst;           // new post-collision populations
  const R* __restrict__ phi;     // porosity [N]
  const R* __restrict__ Tfix;    // fixed temperature [N] (isothermal lattices)
  R* __restrict__ mac;           // macro fields for the gradients [2D+M][N]
  int* status;                   // bit 0: non-finite / non-positive density, bit 1: FP64 solve used,
                                 // bit 2: surface Newton not converged, bit 3: a bounded wait gave up
};

constexpr int kStatusTimeout = 8;   // status bit 3: a bounded device wait gave up

LBM_HD void flag(int* status, int bit) {
#ifdef __CUDA_ARCH__
  atomicOr(status, bit);
#else
  *status |= bit;
#endif
}

template <class R, int D>
LBM_HD void node_xyz(const Params<R>& p, int n, int& x, int& y, int& z) {
  x = n % p.nx;
  int r = n / p.nx;
  y = r % p.ny;
  z = (D == 3) ? r / p.ny : 0;
}

// ---------------------------------------------------------------------------
// Pass 1 (two-pass form): macroscopic fields needed by the neighbours'
// gradients -- u, Pi_alpha of Eq. 45 and Y_a (Eq. 59).
// ---------------------------------------------------------------------------
template <class R, int D, int M, bool EN>
LBM_HD void macro_node(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, int n) {
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Puller<R, D, M, EN> pl;
  pl.setup(p, it, a.src, a.phi, x, y, z);
  Moments<R, D, M, EN, false> mo;
  mo.compute(pl);
  State<R, D, M> s;
  s.template from_moments<EN, false>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    a.mac[(size_t)b * p.N + n] = s.u[b];
    a.mac[(size_t)(D + b) * p.N + n] = s.Pi(b);
  }
  if (EN) {
#pragma unroll
    for (int k = 0; k < M; ++k) a.mac[(size_t)(2 * D + k) * p.N + n] = s.Y[k];
  }
}

template <class R, int D, int M, bool EN>
__global__ void __launch_bounds__(256) k_macro(Params<R> p, InletTables<R> it, StepArgs<R> a) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < p.N) macro_node<R, D, M, EN>(p, it, a, n);
}

// Gradient inputs at node (x, y, z) from the neighbours' macro fields
// (isotropic stencil; zero-gradient copy across non-periodic x faces).
template <class R, int D, int M, bool EN>
struct Grad {
  R divu, dPi[D], dY[M][D];
  template <class Fetch>
  LBM_HD void compute(const Params<R>& p, int x, int y, int z, Fetch&& fetch) {
    constexpr int Q = Lat<D>::Q;
    divu = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      dPi[b] = R(0);
#pragma unroll
      for (int k = 0; k < M; ++k) dY[k][b] = R(0);
    }
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if (csq_of<D>(I) == 0) return;
      const R w = grad_w<R, D>(I);
      int sx = x + c_of<D>(I, 0);
      if (sx < 0) sx = (p.bc_lo == BC_PERIODIC) ? sx + p.nx : 0;
      if (sx >= p.nx) sx = (p.bc_hi == BC_PERIODIC) ? sx - p.nx : p.nx - 1;
      int sy = wrapi(y + c_of<D>(I, 1), p.ny);
      int sz = (D == 3) ? wrapi(z + c_of<D>(I, 2), p.nz) : 0;
      int nb = sx + p.nx * (sy + p.ny * sz);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int cb = c_of<D>(I, b);
        if (cb == 0) continue;
        const R wc = w * R(cb);
        divu += wc * fetch(b, nb);
        dPi[b] += wc * fetch(D + b, nb);
        if (EN) {
#pragma unroll
          for (int k = 0; k < M; ++k) dY[k][b] += wc * fetch(2 * D + k, nb);
        }
      }
    });
  }
};

// Collision of one node (a4-a9) given its streamed populations (through the
// puller), its state and the gradient inputs.  Writes the new populations.
template <class R, int D, int M, bool EN>
LBM_HD void collide_and_store(const Params<R>& p, const Puller<R, D, M, EN>& pl,
                                                  const Moments<R, D, M, EN, true>& mo, const State<R, D, M>& s,
                                                  const Grad<R, D, M, EN>& gr, R* __restrict__ dst, int n,
                                                  int* status) {
  constexpr int Q = Lat<D>::Q;
  constexpr int REST = (Q - 1) / 2;   // index of c = 0
  const int N = p.N;
  if (!(s.rho_s > R(0)) || !(s.rho_f > R(0)) || !finite_<R>(s.T)) flag(status, 1);

  Transport<R, D, M> tr;
  tr.compute(p, s, &mo.ja[0][0], mo.sabs);
  if (tr.used_fp64) flag(status, 2);

  const R phi = s.phi;
  const R inv_phi = R(1) / phi;
  R w[D];
#pragma unroll
  for (int b = 0; b < D; ++b) w[b] = s.u[b] * inv_phi;

  // ---- species (Eq. 21 with Eq. 25) -------
  {
    R E[M][D][3], S[M][D][3], K[M][3], pr[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      R RaT = p.Ra[a] * s.T;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        psi3<R>(w[b], w[b] * w[b] + RaT, E[a][b]);                  // Eq. 15
        R xs = (s.u[b] + tr.V[a][b]) * inv_phi;                      // Eq. 28 over phi
        psi3<R>(xs, xs * xs + RaT, S[a][b]);                         // Eq. 16
      }
      psi3<R>(R(0), RaT, K[a]);                                      // Eq. 18
      pr[a] = phi * s.rho_a[a];
    }
    // The rest population is written last as the remainder of the streamed
    // zeroth moment, so that rounding cannot bias the conserved masses.
    R acc[M];
#pragma unroll
    for (int a = 0; a < M; ++a) acc[a] = R(0);
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if (I == REST) return;
      R feq[M], fst[M], fk[M];
#pragma unroll
      for (int a = 0; a < M; ++a) {
        R e = pr[a], st = pr[a], k = pr[a];
#pragma unroll
        for (int b = 0; b < D; ++b) {
          const int c = c_of<D>(I, b) + 1;
          e *= E[a][b][c];
          st *= S[a][b][c];
          k *= K[a][c];
        }
        feq[a] = e;
        fst[a] = st;
        fk[a] = k;
      }
#pragma unroll
      for (int a = 0; a < M; ++a) {
        R F = R(0);
#pragma unroll
        for (int b = 0; b < M; ++b)
          if (b != a) F += tr.inv_tau_ab[a][b] * (feq[b] - fst[b]);
        F = s.Y[a] * F + tr.inv_tauk[a] * (fst[a] - fk[a]);
        R f = pl.template get<I>(a);
        R out = f + R(2) * tr.beta[a] * (feq[a] - f) + (tr.beta[a] - R(1)) * F;
        acc[a] += out;
        dst[(size_t)(a * Q + I) * N + n] = out;
      }
    });
#pragma unroll
    for (int a = 0; a < M; ++a) dst[(size_t)(a * Q + REST) * N + n] = mo.sa[a] - acc[a];
  }

  // ---- transport of the mixture (Eq. 65, Eq. 67) --------------------------
  R mu = R(0);
  {
    R pw = pow_<R>(s.T * p.inv_T_ref, p.mu_exp);
#pragma unroll
    for (int a = 0; a < M; ++a) mu += s.X[a] * p.muref[a];
    mu *= pw;
  }
  const R omega = R(1) / (R(0.5) + mu / s.P);
  const R omega1 = R(1) / (R(0.5) + mu * p.inv_Pr / s.P);
  const R bulk = -p.bulk_ratio * mu + mu * (R(2) / R(D) - (EN ? s.Rg / s.cv : R(0)));

  // ---- momentum lattice (Eq. 42, Eq. 44, Eq. 45, Eq. 48) ----
  {
    R FX[D][3];
    const R irf = R(1) / (phi * s.rho_f);
    R kdrag = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) kdrag += s.rho_a[a] * tr.inv_tauk[a];
    const R inv_drag = R(1) / (R(1) + R(0.5) * kdrag / s.rho_f);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      // component velocity u* + (V_a - Vbar): diffusion velocities taken
      // relative to the species' mass average, the mixture velocity at the
      // middle of the step (trapezoidal drag of the mixture; reading R8)
      R Vbar = R(0);
#pragma unroll
      for (int a = 0; a < M; ++a) Vbar += s.Y[a] * tr.V[a][b];
      R Fk = R(0);
#pragma unroll
      for (int a = 0; a < M; ++a) Fk -= s.rho_a[a] * (s.u[b] + tr.V[a][b] - Vbar) * tr.inv_tauk[a];
      Fk *= inv_drag;
      R uex = s.u[b] + Fk / (omega * s.rho_f);
      R Pex = s.Rg * s.T + w[b] * w[b] + bulk * gr.divu * irf +
              (R(2) - omega) / (R(2) * omega) * irf * gr.dPi[b];
      psi3<R>(uex * inv_phi, Pex, FX[b]);
    }
    const R pref = phi * s.rho_f;
    R acc = R(0);
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if (I == REST) return;
      R fex = pref;
#pragma unroll
      for (int b = 0; b < D; ++b) fex *= FX[b][c_of<D>(I, b) + 1];
      R f = pl.template get<I>(M);
      R out = f + omega * (fex - f);
      acc += out;
      dst[(size_t)(M * Q + I) * N + n] = out;
    });
    dst[(size_t)(M * Q + REST) * N + n] = mo.sf - acc;
  }

  // ---- energy lattice (Eq. 43 with Eq. 54, multiplied through by omega - omega1)
  if (EN) {
    R U = R(0), Ha[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      R Ua = p.U0[a] + p.cvR[a] * (s.T - p.T_thermo);
      Ha[a] = Ua + p.Ra[a] * s.T;
      U += s.Y[a] * Ua;
    }
    const R RT = s.Rg * s.T;
    const R H = U + RT;
    R w2 = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) w2 += w[b] * w[b];
    GeqFactors<R, D> G;
    G.init(phi, s.rho_f, s.u, RT, U);
    R Dq[D];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      R qeq = (H + R(0.5) * w2) * s.rho_f * s.u[b];                    // Eq. 52
      R uP = R(0);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R Peq = s.rho_f * s.u[b] * w[c] + (b == c ? phi * s.rho_f * RT : R(0));   // Eq. 49
        uP += w[c] * (mo.Pt[b][c] - Peq);
      }
      R Vbar = R(0);
#pragma unroll
      for (int a = 0; a < M; ++a) Vbar += s.Y[a] * tr.V[a][b];
      R sV = R(0), sdY = R(0);
#pragma unroll
      for (int a = 0; a < M; ++a) {
        sV += Ha[a] * s.Y[a] * (tr.V[a][b] - Vbar);
        sdY += Ha[a] * gr.dY[a][b];
      }
      // (omega - omega1) (q* - q^eq) with q^diff, q^corr, q^ex of Eq. 55
      Dq[b] = (omega - omega1) * (mo.q[b] - uP - qeq) + omega1 * s.rho_f * sV +
              R(0.5) * (R(2) - omega1) * s.P * phi * sdY + s.u[b] * omega * bulk * gr.divu * inv_phi -
              R(0.5) * (omega - omega1) * w[b] * gr.dPi[b];
    }
    R acc = R(0);
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if (I == REST) return;
      R geq = G.template value<I>();
      R g = pl.template get<I>(M + 1);
      R out = g + omega * (geq - g);
      if (csq_of<D>(I) == 1) {
#pragma unroll
        for (int b = 0; b < D; ++b)
          if (c_of<D>(I, b) != 0) out += R(0.5) * R(c_of<D>(I, b)) * Dq[b];
      }
      acc += out;
      dst[(size_t)((M + 1) * Q + I) * N + n] = out;
    });
    dst[(size_t)((M + 1) * Q + REST) * N + n] = mo.sg - acc;
  }
}

// ---------------------------------------------------------------------------
// Pass 2 (two-pass form): full node update reading the neighbours' macro
// fields from global memory.
// ---------------------------------------------------------------------------
template <class R, int D, int M, bool EN>
LBM_HD void collide_node(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a, int n) {
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Puller<R, D, M, EN> pl;
  pl.setup(p, it, a.src, a.phi, x, y, z);
  Moments<R, D, M, EN, true> mo;
  mo.compute(pl);
  State<R, D, M> s;
  s.template from_moments<EN, true>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
  Grad<R, D, M, EN> gr;
  const R* __restrict__ mac = a.mac;
  const int N = p.N;
  gr.compute(p, x, y, z, [&](int k, int nb) { return mac[(size_t)k * N + nb]; });
  collide_and_store<R, D, M, EN>(p, pl, mo, s, gr, a.dst, n, a.status);
}

template <class R, int D, int M, bool EN>
__global__ void __launch_bounds__(256) k_collide(Params<R> p, InletTables<R> it, StepArgs<R> a) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < p.N) collide_node<R, D, M, EN>(p, it, a, n);
}

// ---------------------------------------------------------------------------
// Initial populations: equilibria of the initial fields (Eq. 15, Eq. 44
// without extension, Eq. 51).
// ---------------------------------------------------------------------------
// Initial populations of node n: equilibria of the initial fields (Eq. 15,
// Eq. 44 without extension, Eq. 51).  R is the computing type, PR the
// parameter type; store(l, i, value).
template <class R, int D, int M, bool EN, class PR, class Store>
LBM_HD void init_node(const PR& p, const double* __restrict__ X, const double* __restrict__ T0,
                      const double* __restrict__ P0, const double* __restrict__ U0v, double cvel, double RU_si,
                      int n, int N, R phi, Store&& store) {
  constexpr int Q = Lat<D>::Q;
  R T = (R)T0[n];
  R rho_a[M], rho = R(0), inv_m = R(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    // rho_a = P X_a m_a / (R_U T)  (Dalton and the ideal-gas law, Sec. 2.1)
    rho_a[a] = (R)(P0[n] * X[(size_t)a * N + n] * (double)p.m[a] / (RU_si * T0[n]));
    rho += rho_a[a];
  }
#pragma unroll
  for (int a = 0; a < M; ++a) inv_m += (rho_a[a] / rho) / R(p.m[a]);
  R Rg = R(p.RU) * inv_m;
  R u[D], w[D];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    u[b] = U0v ? (R)(U0v[(size_t)b * N + n] / cvel) : R(0);
    w[b] = u[b] / phi;
  }
#pragma unroll
  for (int a = 0; a < M; ++a) {
    R F[D][3];
#pragma unroll
    for (int b = 0; b < D; ++b) psi3<R>(w[b], w[b] * w[b] + R(p.Ra[a]) * T, F[b]);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R v = phi * rho_a[a];
#pragma unroll
      for (int b = 0; b < D; ++b) v *= F[b][c_of<D>(i, b) + 1];
      store(a, i, v);
    }
  }
  {
    R F[D][3];
#pragma unroll
    for (int b = 0; b < D; ++b) psi3<R>(w[b], w[b] * w[b] + Rg * T, F[b]);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R v = phi * rho;
#pragma unroll
      for (int b = 0; b < D; ++b) v *= F[b][c_of<D>(i, b) + 1];
      store(M, i, v);
    }
  }
  if (EN) {
    R U = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) U += (rho_a[a] / rho) * (R(p.U0[a]) + R(p.cvR[a]) * (T - R(p.T_thermo)));
    GeqFactors<R, D> G;
    G.init(phi, rho, u, Rg * T, U);
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      store(M + 1, I, G.template value<I>());
    });
  }
}

template <class R, int D, int M, bool EN>
__global__ void __launch_bounds__(256) k_init(Params<R> p, const double* __restrict__ X, const double* __restrict__ T0,
                                             const double* __restrict__ P0, const double* __restrict__ U0v,
                                             double cvel, double RU_si, R* __restrict__ dst,
                                             const R* __restrict__ phiA) {
  constexpr int Q = Lat<D>::Q;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int N = p.N;
  init_node<R, D, M, EN>(p, X, T0, P0, U0v, cvel, RU_si, n, N, phiA[n],
                         [&](int l, int i, R v) { dst[(size_t)(l * Q + i) * N + n] = v; });
}

// ---------------------------------------------------------------------------
// Macroscopic fields of the current state for lbm_moments.
// ---------------------------------------------------------------------------
template <class R, int D, int M, bool EN>
__global__ void __launch_bounds__(256) k_moments(Params<R> p, InletTables<R> it, StepArgs<R> a, int which,
                                                double cvel, double* __restrict__ out) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int N = p.N;
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Puller<R, D, M, EN> pl;
  pl.setup(p, it, a.src, a.phi, x, y, z);
  Moments<R, D, M, EN, true> mo;
  mo.compute(pl);
  State<R, D, M> s;
  s.template from_moments<EN, true>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
  switch (which) {
    case 0:
      for (int k = 0; k < M; ++k) out[(size_t)k * N + n] = (double)s.rho_a[k];
      break;
    case 1:
      for (int k = 0; k < M; ++k)
        for (int b = 0; b < D; ++b) out[((size_t)k * D + b) * N + n] = (double)mo.ja[k][b];
      break;
    case 2: out[n] = (double)s.rho_f; break;
    case 3:
      for (int b = 0; b < D; ++b) out[(size_t)b * N + n] = (double)s.u[b];
      break;
    case 4: out[n] = (double)s.T; break;
    case 5: out[n] = (double)s.P * cvel * cvel; break;
    case 6:
    case 7: {
      Transport<R, D, M> tr;
      tr.compute(p, s, &mo.ja[0][0], mo.sabs);
      for (int k = 0; k < M; ++k)
        for (int b = 0; b < D; ++b) {
          double v = (double)tr.V[k][b];
          if (which == 7) v = (double)s.rho_a[k] * ((double)s.u[b] + v) * cvel / (double)p.m[k];
          out[((size_t)k * D + b) * N + n] = v;
        }
      break;
    }
    case 9: out[n] = (double)s.rho_s; break;
    default: break;
  }
}

}  // namespace lbm
