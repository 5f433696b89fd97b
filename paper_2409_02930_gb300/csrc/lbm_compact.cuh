// Compact per-node code: runtime loops over the discrete velocities with the
// per-axis product-form factors selected by c in {-1, 0, 1}.  The arithmetic
// is the one of lbm_kernels.cuh (same equations, same order of the
// conservation-preserving rest-population remainder); only the code shape
// differs, so that the fused kernel fits the instruction cache and keeps the
// register count low enough for several resident blocks per SM.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <class R>
LBM_HD R sel3(const R (&v)[3], int c) {
  return c < 0 ? v[0] : (c == 0 ? v[1] : v[2]);
}

// Iterate over the discrete velocities: runtime loops over c_z and c_y, the
// c_x loop unrolled.  f(i, cx, cy, cz).
template <int D, bool UNROLL = false, class F>
LBM_HD void for_each_dir(F&& f) {
  if constexpr (UNROLL) {
    // same order, every direction a compile-time constant
    Unroll<0, Lat<D>::Q>::run([&](auto ic) {
      constexpr int i = decltype(ic)::value;
      f(i, c_of<D>(i, 0), c_of<D>(i, 1), c_of<D>(i, 2));
    });
    return;
  }
  const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
#pragma unroll 1
  for (int cz = zlo; cz <= zhi; ++cz) {
#pragma unroll 1
    for (int cy = -1; cy <= 1; ++cy) {
#pragma unroll
      for (int cx = -1; cx <= 1; ++cx) {
        const int i = (cx + 1) + 3 * (cy + 1) + ((D == 3) ? 9 * (cz + 1) : 0);
        f(i, cx, cy, cz);
      }
    }
  }
}

// Source of the streamed population i at node (x, y, z) (pull with the
// boundary rules).  Returns the source node index, or -1 - n for bounce-back
// at this node, or SRC_GHOST for a reservoir ghost.
template <class R, int D>
struct Site {
  int x, y, z, n;
  int nx, ny, nz, bc_lo, bc_hi;
  LBM_HD void init(const Params<R>& p, int x_, int y_, int z_) {
    x = x_; y = y_; z = z_;
    nx = p.nx; ny = p.ny; nz = p.nz; bc_lo = p.bc_lo; bc_hi = p.bc_hi;
    n = x + nx * (y + ny * z);
  }
  LBM_HD int source(int cx, int cy, int cz) const {
    int sy = wrapi(y - cy, ny);
    int sz = (D == 3) ? wrapi(z - cz, nz) : 0;
    int sx = x - cx;
    if (sx < 0 || sx >= nx) {
      int bc = sx < 0 ? bc_lo : bc_hi;
      if (bc == BC_PERIODIC) sx = wrapi(sx, nx);
      else if (bc == BC_BOUNCEBACK) return -1 - n;
      else return SRC_GHOST;
    }
    return sx + nx * (sy + ny * sz);
  }
  LBM_HD bool has_ghost() const {
    return (x == 0 && bc_lo == BC_INLET) || (x == nx - 1 && bc_hi == BC_INLET);
  }
};

// Streamed value of lattice l, direction i, with the source already resolved.
template <class R, int D, int M, bool EN>
LBM_HD R pull_rt(const Params<R>& p, const InletTables<R>& it, const R* __restrict__ src, const Ghost<R, D>& gh,
                 int n, int s, int l, int i, int cx, int cy, int cz) {
  constexpr int Q = Lat<D>::Q;
  const size_t N = p.N;
  if (s >= 0) return src[(size_t)(l * Q + i) * N + s];
  if (s != SRC_GHOST) return src[(size_t)(l * Q + (Q - 1 - i)) * N + (-1 - s)];
  // reservoir equilibrium (Eq. 15 / Eq. 44 / Eq. 51 at the reservoir state)
  const int sd = gh.side;
  const R phi = gh.phi;
  const R T = it.T[sd];
  const int cc[3] = {cx, cy, cz};
  if (l < M || l == M) {
    const R RT = (l < M) ? p.Ra[l] * T : it.Rmix[sd] * T;
    R v = phi * ((l < M) ? it.rho[sd][l] : it.rho_sum[sd]);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      R w = gh.u[b] / phi;
      v *= psi<R>(cc[b], w, w * w + RT);
    }
    return v;
  }
  GeqFactors<R, D> G;
  G.init(phi, it.rho_sum[sd], gh.u, it.Rmix[sd] * T, it.Umix[sd]);
  R prod = R(1), s2 = R(0);
#pragma unroll
  for (int b = 0; b < D; ++b) prod *= sel3(G.P1[b], cc[b]);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    R t = sel3(G.P2[b], cc[b]);
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (a != b) t *= sel3(G.P1[a], cc[a]);
    s2 += t;
  }
  return G.pref_U * prod + G.pref * s2;
}

// velocity of the node adjacent to a reservoir face (all its sources inside)
template <class R, int D, int M>
LBM_HD void ghost_velocity(const Params<R>& p, const R* __restrict__ src, const R* __restrict__ phiA, int x, int y,
                           int z, Ghost<R, D>& gh) {
  constexpr int Q = Lat<D>::Q;
  gh.side = (x == 0 && p.bc_lo == BC_INLET) ? 0 : 1;
  const int xa = gh.side == 0 ? 1 : p.nx - 2;
  Site<R, D> sa;
  sa.init(p, xa, y, z);
  R s0 = R(0), j[D];
#pragma unroll
  for (int b = 0; b < D; ++b) j[b] = R(0);
  for_each_dir<D>([&](int i, int cx, int cy, int cz) {
    R f = src[(size_t)(M * Q + i) * p.N + sa.source(cx, cy, cz)];
    s0 += f;
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int b = 0; b < D; ++b) j[b] += R(cc[b]) * f;
  });
  R rho_f = s0 / phiA[sa.n];
#pragma unroll
  for (int b = 0; b < D; ++b) gh.u[b] = j[b] / rho_f;
  gh.phi = phiA[x + p.nx * (y + p.ny * z)];
}

// Streamed values from global memory with the boundary rules: the handle of
// a direction is its resolved source (see Site::source).
template <class R, int D, int M, bool EN>
struct GlobalPull {
  const Params<R>& p;
  const InletTables<R>& it;
  const R* __restrict__ src;
  const Site<R, D>& st;
  const Ghost<R, D>& gh;
  static constexpr bool kUnroll = false;
  LBM_HD int prep(int cx, int cy, int cz) const { return st.source(cx, cy, cz); }
  LBM_HD R get(int h, int l, int i, int cx, int cy, int cz) const {
    return pull_rt<R, D, M, EN>(p, it, src, gh, st.n, h, l, i, cx, cy, cz);
  }
};

// Moments of the streamed populations (runtime loop form), from any puller.
template <class R, int D, int M, bool EN, bool FULL, class PullF>
LBM_HD void moments_gen(const PullF& pf, Moments<R, D, M, EN, FULL>& mo) {
#pragma unroll
  for (int a = 0; a < M; ++a) {
    mo.sa[a] = R(0);
    mo.sabs[a] = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) mo.ja[a][b] = R(0);
  }
  mo.sf = R(0);
  mo.sg = R(0);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    mo.jf[b] = R(0);
    mo.q[b] = R(0);
#pragma unroll
    for (int c = 0; c < D; ++c) mo.Pt[b][c] = R(0);
  }
  for_each_dir<D, PullF::kUnroll>([&](int i, int cx, int cy, int cz) {
    const int h = pf.prep(cx, cy, cz);
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int a = 0; a < M; ++a) {
      R f = pf.get(h, a, i, cx, cy, cz);
      mo.sa[a] += f;
      if (FULL && ScalarTraits<R>::single) mo.sabs[a] += fabs(f);
      if (FULL) {
#pragma unroll
        for (int b = 0; b < D; ++b) mo.ja[a][b] += R(cc[b]) * f;
      }
    }
    R f = pf.get(h, M, i, cx, cy, cz);
    mo.sf += f;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      mo.jf[b] += R(cc[b]) * f;
      if (FULL && EN) {
#pragma unroll
        for (int c = 0; c < D; ++c) mo.Pt[b][c] += R(cc[b] * cc[c]) * f;
      }
    }
    if (EN) {
      R g = pf.get(h, M + 1, i, cx, cy, cz);
      mo.sg += g;
      if (FULL) {
#pragma unroll
        for (int b = 0; b < D; ++b) mo.q[b] += R(cc[b]) * g;
      }
    }
  });
}

template <class R, int D, int M, bool EN, bool FULL>
LBM_HD void moments_rt(const Params<R>& p, const InletTables<R>& it, const R* __restrict__ src, const Site<R, D>& st,
                       const Ghost<R, D>& gh, Moments<R, D, M, EN, FULL>& mo) {
  GlobalPull<R, D, M, EN> pf{p, it, src, st, gh};
  moments_gen<R, D, M, EN, FULL>(pf, mo);
}

// Heterogeneous-reaction sources of one node for one step (Sec. 4.2): gas
// mass production rhodot_a dt per unit volume of porous medium
// (Eq. 68) and the change of the fluid internal energy
// per unit volume (Eq. 85), in lattice energy units.
template <class R>
struct NodeSource {
  R rhodot[MMAX];
  R dU;
};

// Collision and store of one node (runtime loop form of collide_and_store).
// With SRC the reaction sources are added: Eq. 89 to the species,
// Eq. 87 to the momentum lattice and Eq. 88 to the energy lattice.
// With COEF, coef[l] receives the derivative of every non-rest post-collision
// population of lattice l with respect to its own streamed population at
// fixed moments (1 - 2 beta_a for the species, 1 - omega for the momentum and
// energy lattices): the adjoint needs it, the step does not.
template <class R, int D, int M, bool EN, class PullF, bool SRC = false, bool COEF = false>
LBM_HD void collide_gen(const Params<R>& p, const PullF& pf, int n, const Moments<R, D, M, EN, true>& mo,
                        const State<R, D, M>& s, const Grad<R, D, M, EN>& gr, R* __restrict__ dst, int* status,
                        const NodeSource<R>* srcv = nullptr, R* coef = nullptr) {
  constexpr int Q = Lat<D>::Q;
  constexpr int REST = (Q - 1) / 2;
  const size_t N = p.N;
  if (!(s.rho_s > R(0)) || !(s.rho_f > R(0)) || !finite_<R>(s.T)) flag(status, 1);

  Transport<R, D, M> tr;
  tr.compute(p, s, &mo.ja[0][0], mo.sabs);
  if (tr.used_fp64) flag(status, 2);

  const R phi = s.phi;
  const R inv_phi = R(1) / phi;
  R w[D];
#pragma unroll
  for (int b = 0; b < D; ++b) w[b] = s.u[b] * inv_phi;

  // mixture transport (Eq. 65, Eq. 67)
  R mu = R(0);
  {
    R pw = pow_<R>(s.T * p.inv_T_ref, p.mu_exp);
#pragma unroll
    for (int a = 0; a < M; ++a) mu += s.X[a] * p.muref[a];
    mu *= pw;
  }
  const R omega = R(1) / (R(0.5) + mu / s.P);
  const R omega1 = R(1) / (R(0.5) + mu * p.inv_Pr / s.P);
  if constexpr (COEF) {
#pragma unroll
    for (int a = 0; a < M; ++a) coef[a] = R(1) - R(2) * tr.beta[a];
    coef[M] = R(1) - omega;
    if (EN) coef[M + 1] = R(1) - omega;
  }
  const R bulk = -p.bulk_ratio * mu + mu * (R(2) / R(D) - (EN ? s.Rg / s.cv : R(0)));

  // per-axis factors of the species equilibria, quasi-equilibria and
  // Knudsen states (Eq. 15, Eq. 16 with Eq. 28, Eq. 18)
  R E[M][D][3], S[M][D][3], K[M][3], pr[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    R RaT = p.Ra[a] * s.T;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      psi3<R>(w[b], w[b] * w[b] + RaT, E[a][b]);
      R xs = (s.u[b] + tr.V[a][b]) * inv_phi;
      psi3<R>(xs, xs * xs + RaT, S[a][b]);
    }
    psi3<R>(R(0), RaT, K[a]);
    pr[a] = phi * s.rho_a[a];
  }
  // momentum lattice factors (Eq. 44, Eq. 45, reading of u^ex)
  R FX[D][3];
  {
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
      R Pex = s.Rg * s.T + w[b] * w[b] + bulk * gr.divu * irf + (R(2) - omega) / (R(2) * omega) * irf * gr.dPi[b];
      psi3<R>(uex * inv_phi, Pex, FX[b]);
    }
  }
  const R pref_f = phi * s.rho_f;
  // post-collision density (Eq. 78) and the Eq. 87 factor
  R rho_pc = s.rho_f, kpc = R(0);
  if (SRC) {
    R sum_rd = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) sum_rd += srcv->rhodot[a];
    rho_pc = s.rho_f + sum_rd * inv_phi;
    kpc = rho_pc / s.rho_f - R(1);
  }
  // energy lattice (Eq. 43 with Eq. 54, multiplied through by omega - omega1)
  GeqFactors<R, D> G, G2;
  R Dq[D];
  R g_src_total = R(0);
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
    G.init(phi, s.rho_f, s.u, RT, U);
    if (SRC) {
      // source distribution with the post-reaction density and internal energy (Eq. 86)
      const R U_pc = (phi * s.rho_f * U + srcv->dU) / (phi * rho_pc);
      G2.init(phi, rho_pc, s.u, RT, U_pc);
      g_src_total = phi * rho_pc * (U_pc + R(0.5) * w2) - phi * s.rho_f * (U + R(0.5) * w2);
    }
#pragma unroll
    for (int b = 0; b < D; ++b) {
      R qeq = (H + R(0.5) * w2) * s.rho_f * s.u[b];
      R uP = R(0);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        R Peq = s.rho_f * s.u[b] * w[c] + (b == c ? phi * s.rho_f * RT : R(0));
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
      Dq[b] = (omega - omega1) * (mo.q[b] - uP - qeq) + omega1 * s.rho_f * sV +
              R(0.5) * (R(2) - omega1) * s.P * phi * sdY + s.u[b] * omega * bulk * gr.divu * inv_phi -
              R(0.5) * (omega - omega1) * w[b] * gr.dPi[b];
    }
  }

  R acc[M + 2];
#pragma unroll
  for (int l = 0; l < M + 2; ++l) acc[l] = R(0);
  for_each_dir<D, PullF::kUnroll>([&](int i, int cx, int cy, int cz) {
    if (i == REST) return;
    const int h = pf.prep(cx, cy, cz);
    // species (Eq. 21, Eq. 25)
    R feq[M], fst[M], fk[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      R e = pr[a] * E[a][0][cx + 1], sv = pr[a] * S[a][0][cx + 1], k = pr[a] * K[a][cx + 1];
      if (D >= 2) {
        e *= sel3(E[a][1], cy);
        sv *= sel3(S[a][1], cy);
        k *= sel3(K[a], cy);
      }
      if (D == 3) {
        e *= sel3(E[a][D - 1], cz);
        sv *= sel3(S[a][D - 1], cz);
        k *= sel3(K[a], cz);
      }
      feq[a] = e;
      fst[a] = sv;
      fk[a] = k;
    }
#pragma unroll
    for (int a = 0; a < M; ++a) {
      R F = R(0);
#pragma unroll
      for (int b = 0; b < M; ++b)
        if (b != a) F += tr.inv_tau_ab[a][b] * (feq[b] - fst[b]);
      F = s.Y[a] * F + tr.inv_tauk[a] * (fst[a] - fk[a]);
      R f = pf.get(h, a, i, cx, cy, cz);
      R out = f + R(2) * tr.beta[a] * (feq[a] - f) + (tr.beta[a] - R(1)) * F;
      if (SRC) {
        R shape = E[a][0][cx + 1];
        if (D >= 2) shape *= sel3(E[a][1], cy);
        if (D == 3) shape *= sel3(E[a][D - 1], cz);
        out += srcv->rhodot[a] * shape;                  // Eq. 89, R^r = fdot^r dt
      }
      acc[a] += out;
      dst[(size_t)(a * Q + i) * N + n] = out;
    }
    // momentum (Eq. 42)
    {
      R fex = pref_f * FX[0][cx + 1];
      if (D >= 2) fex *= sel3(FX[1], cy);
      if (D == 3) fex *= sel3(FX[D - 1], cz);
      R f = pf.get(h, M, i, cx, cy, cz);
      R out = f + omega * (fex - f);
      if (SRC) out += kpc * fex;                          // Eq. 87
      acc[M] += out;
      dst[(size_t)(M * Q + i) * N + n] = out;
    }
    // energy (Eq. 43, Eq. 51, Eq. 54)
    if (EN) {
      const int cc[3] = {cx, cy, cz};
      R prod = R(1), s2 = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) prod *= sel3(G.P1[b], cc[b]);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        R t = sel3(G.P2[b], cc[b]);
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2)
          if (a2 != b) t *= sel3(G.P1[a2], cc[a2]);
        s2 += t;
      }
      R geq = G.pref_U * prod + G.pref * s2;
      R g = pf.get(h, M + 1, i, cx, cy, cz);
      R out = g + omega * (geq - g);
      if (SRC) {                                          // Eq. 88
        R prod2 = R(1), s22 = R(0);
#pragma unroll
        for (int b = 0; b < D; ++b) prod2 *= sel3(G2.P1[b], cc[b]);
#pragma unroll
        for (int b = 0; b < D; ++b) {
          R t2 = sel3(G2.P2[b], cc[b]);
#pragma unroll
          for (int a2 = 0; a2 < D; ++a2)
            if (a2 != b) t2 *= sel3(G2.P1[a2], cc[a2]);
          s22 += t2;
        }
        out += (G2.pref_U * prod2 + G2.pref * s22) - geq;
      }
      const int c2 = cx * cx + cy * cy + cz * cz;
      if (c2 == 1) {
        R dq = R(0);
#pragma unroll
        for (int b = 0; b < D; ++b) dq += R(cc[b]) * Dq[b];
        out += R(0.5) * dq;
      }
      acc[M + 1] += out;
      dst[(size_t)((M + 1) * Q + i) * N + n] = out;
    }
  });
  // rest populations as remainders of the streamed zeroth moments
#pragma unroll
  for (int a = 0; a < M; ++a)
    dst[(size_t)(a * Q + REST) * N + n] = mo.sa[a] + (SRC ? srcv->rhodot[a] : R(0)) - acc[a];
  dst[(size_t)(M * Q + REST) * N + n] = mo.sf + (SRC ? phi * (rho_pc - s.rho_f) : R(0)) - acc[M];
  if (EN) dst[(size_t)((M + 1) * Q + REST) * N + n] = mo.sg + g_src_total - acc[M + 1];
}

template <class R, int D, int M, bool EN>
LBM_HD void collide_rt(const Params<R>& p, const InletTables<R>& it, const R* __restrict__ src, const Site<R, D>& st,
                       const Ghost<R, D>& gh, const Moments<R, D, M, EN, true>& mo, const State<R, D, M>& s,
                       const Grad<R, D, M, EN>& gr, R* __restrict__ dst, int* status) {
  GlobalPull<R, D, M, EN> pf{p, it, src, st, gh};
  collide_gen<R, D, M, EN>(p, pf, st.n, mo, s, gr, dst, status);
}

}  // namespace lbm
