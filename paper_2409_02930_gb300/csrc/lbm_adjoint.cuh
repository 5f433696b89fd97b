// Adjoint (reverse-mode) step kernels: given the adjoint lambda^{n+1} of
// the post-collision populations after step n, they return lambda^n and
// accumulate dJ/dphi (porosity field) and dJ/dlambda, where lambda scales
// every Knudsen coefficient 1/tau^k_a (pore radius and tortuosity enter the
// step only through tortuosity / pore radius, Eq. 26 with the Knudsen
// diffusivity of Sec. 5.1).
//
// The step f^{n+1} = C(S f^n) is differentiated in its own structure:
//   streamed populations P(x)   = pull of f^n with the boundary rules (a1)
//   macro fields     m(x)        = u, Pi, Y_a of P(x) and phi(x)       (a2, a3)
//   gradients        G(x)        = isotropic stencil of m              (a5)
//   node update      f^{n+1}(x)  = collide(P(x), phi(x), G(x), lambda) (a4, a6-a9)
// k_adj_collide forms lambda^{n+1}(x)^T dC for all inputs of the node
// update, K directions per evaluation of the node code in dual numbers;
// k_adj_macro transposes the stencil and the macro fields; k_adj_ghost
// carries the reservoir ghosts' dependence on the adjacent node's velocity;
// k_adj_stream transposes the pull.  k_adj_init adds the dependence of the
// initial equilibria on the porosity.
#pragma once

#include "lbm_compact.cuh"
#include "lbm_dual.cuh"

namespace lbm {

template <int D, int M, bool EN>
LBM_HD constexpr int n_grad() { return 1 + D + (EN ? M * D : 0); }
template <int D, int M, bool EN>
LBM_HD constexpr int n_lat() { return M + 1 + (EN ? 1 : 0); }

// Node-local parameters in dual form (N = 1): pz carries no derivative, pk
// seeds d(1/tau^k_a)/dlambda = 1/tau^k_a in lane 0.
template <class B, int K>
struct AdjParams {
  Params<Dual<B, K>> pz;
  Params<Dual<B, K>> pk;
};

template <class B>
struct AdjArgs {
  const B* f;         // f^n [L][Q][N]
  const B* mac;       // macro fields of f^n [2D+M][N]
  const B* phi;       // [N]
  const B* Tfix;      // [N]
  const B* lam1;      // adjoint of f^{n+1} [L][Q][N]
  B* Pbar;            // adjoint of the streamed populations of step n [L][Q][N]
  B* Gbar;            // adjoint of the gradient inputs [NG][N]
  double* phibar;     // dJ/dphi accumulator [N]
  double* kbar;       // dJ/dlambda accumulator per node [N]
  B* lam0;            // adjoint of f^n [L][Q][N]
  int* status;
};

// Streamed populations of node n (base type) with the boundary rules.
template <class B, int D, int M, bool EN>
LBM_HD void pull_node(const Params<B>& p, const InletTables<B>& it, const B* f, const B* phi, int x, int y, int z,
                      B* P) {
  constexpr int Q = Lat<D>::Q, L = n_lat<D, M, EN>();
  Site<B, D> st;
  st.init(p, x, y, z);
  Ghost<B, D> gh;
  gh.side = -1;
  if (st.has_ghost()) ghost_velocity<B, D, M>(p, f, phi, x, y, z, gh);
  for_each_dir<D>([&](int i, int cx, int cy, int cz) {
    const int h = st.source(cx, cy, cz);
#pragma unroll
    for (int l = 0; l < L; ++l) P[l * Q + i] = pull_rt<B, D, M, EN>(p, it, f, gh, st.n, h, l, i, cx, cy, cz);
  });
}

// Streamed populations of the node as dual numbers with zero derivative: the
// node update's dependence on them is split into the moments (seeded) and
// the direct relaxation term (coefficient returned by collide_gen).
template <class B, int K, int D, int M, bool EN>
struct PlainPull {
  const B* P;
  static constexpr bool kUnroll = false;
  LBM_HD int prep(int, int, int) const { return 0; }
  LBM_HD Dual<B, K> get(int, int l, int i, int, int, int) const { return Dual<B, K>(P[l * Lat<D>::Q + i]); }
};

// Moments seeded in the dual lanes [first, first + K) of a running index
// (sa, ja, sf, jf, Pt, sg, q in that order).
template <class B, int K, int D, int M, bool EN>
LBM_HD void seed_moments(const Moments<B, D, M, EN, true>& m0, int first, Moments<Dual<B, K>, D, M, EN, true>& mo) {
  using T = Dual<B, K>;
  int idx = 0;
  auto put = [&](T& dst, B v) {
    dst = T(v);
    const int lane = idx - first;
    if (lane >= 0 && lane < K) dst.d[lane] = B(1);
    ++idx;
  };
#pragma unroll
  for (int a = 0; a < M; ++a) put(mo.sa[a], m0.sa[a]);
#pragma unroll
  for (int a = 0; a < M; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) put(mo.ja[a][b], m0.ja[a][b]);
  put(mo.sf, m0.sf);
#pragma unroll
  for (int b = 0; b < D; ++b) put(mo.jf[b], m0.jf[b]);
#pragma unroll
  for (int b = 0; b < D; ++b)
#pragma unroll
    for (int c = 0; c < D; ++c) put(mo.Pt[b][c], m0.Pt[b][c]);
  put(mo.sg, m0.sg);
#pragma unroll
  for (int b = 0; b < D; ++b) put(mo.q[b], m0.q[b]);
#pragma unroll
  for (int a = 0; a < M; ++a) mo.sabs[a] = T(m0.sabs[a]);     // a resolution test only: no derivative
}

template <int D, int M>
LBM_HD constexpr int n_mom() { return M + M * D + 1 + D + D * D + 1 + D; }

// Base-type puller over the node's streamed populations.
template <class B, int D>
struct BasePull {
  const B* P;
  static constexpr bool kUnroll = false;
  LBM_HD int prep(int, int, int) const { return 0; }
  LBM_HD B get(int, int l, int i, int, int, int) const { return P[l * Lat<D>::Q + i]; }
};

// Node update: lambda^{n+1}(x)^T dC / d(lambda, phi(x), G(x), P(x)).  The
// populations enter the node update through the moments and through the
// direct relaxation term: dC_{l,i}/dP_{l,j} = coef_l delta_ij for i, j not
// the rest velocity, and the rest population (a conservation remainder)
// carries -coef_l.  Dual evaluations seed lambda, phi, the gradient inputs
// and the moments; the populations' adjoint follows from the moments'
// transpose plus the direct term.
template <class B, int D, int M, bool EN, int K>
__global__ void __launch_bounds__(128) k_adj_collide(Params<B> p, InletTables<B> it, AdjArgs<B> a,
                                                     const __grid_constant__ AdjParams<B, K> ap) {
  using T = Dual<B, K>;
  constexpr int Q = Lat<D>::Q, L = n_lat<D, M, EN>(), LQ = L * Q, NG = n_grad<D, M, EN>();
  constexpr int NM = n_mom<D, M>();
  constexpr int ND = 2 + NG + NM;     // directions: lambda, phi, gradients, moments
  constexpr int REST = (Q - 1) / 2;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int N = p.N;
  int x, y, z;
  node_xyz<B, D>(p, n, x, y, z);
  B P[LQ];
  pull_node<B, D, M, EN>(p, it, a.f, a.phi, x, y, z, P);
  Moments<B, D, M, EN, true> m0;
  moments_gen<B, D, M, EN, true>(BasePull<B, D>{P}, m0);
  Grad<B, D, M, EN> g0;
  const B* __restrict__ mac = a.mac;
  g0.compute(p, x, y, z, [&](int k, int nb) { return mac[(size_t)k * N + nb]; });
  const B phin = a.phi[n];
  const B Tf = EN ? B(0) : a.Tfix[n];
  B lam[LQ];
#pragma unroll
  for (int j = 0; j < LQ; ++j) lam[j] = a.lam1[(size_t)j * N + n];
  double pb_phi = 0.0, pb_k = 0.0;
  B mbar[NM], coef[L];
#pragma unroll 1
  for (int c0 = 0; c0 < ND; c0 += K) {
    T phid(phin);
    if (1 - c0 >= 0 && 1 - c0 < K) phid.d[1 - c0] = B(1);
    Grad<T, D, M, EN> gd;
    auto seed = [&](T& dst, B v, int g) {
      dst = T(v);
      const int dir = 2 + g - c0;
      if (dir >= 0 && dir < K) dst.d[dir] = B(1);
    };
    seed(gd.divu, g0.divu, 0);
#pragma unroll
    for (int b = 0; b < D; ++b) seed(gd.dPi[b], g0.dPi[b], 1 + b);
#pragma unroll
    for (int k = 0; k < M; ++k)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        if (EN) seed(gd.dY[k][b], g0.dY[k][b], 1 + D + k * D + b);
        else gd.dY[k][b] = T(B(0));
      }
    const Params<T>& pp = (c0 == 0) ? ap.pk : ap.pz;      // lambda is direction 0
    Moments<T, D, M, EN, true> mo;
    seed_moments<B, K, D, M, EN>(m0, c0 - 2 - NG, mo);
    PlainPull<B, K, D, M, EN> pf{P};
    State<T, D, M> s;
    s.template from_moments<EN, true>(pp, mo, phid, T(Tf));
    T out[LQ], cf[L];
    collide_gen<T, D, M, EN, PlainPull<B, K, D, M, EN>, false, true>(pp, pf, 0, mo, s, gd, out, a.status, nullptr, cf);
#pragma unroll
    for (int l = 0; l < L; ++l) coef[l] = cf[l].v;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int dir = c0 + k;
      if (dir >= ND) break;
      B acc = B(0);
#pragma unroll
      for (int j = 0; j < LQ; ++j) acc += lam[j] * out[j].d[k];
      if (dir == 0) pb_k += (double)acc;
      else if (dir == 1) pb_phi += (double)acc;
      else if (dir < 2 + NG) a.Gbar[(size_t)(dir - 2) * N + n] = acc;
      else mbar[dir - 2 - NG] = acc;
    }
  }
  // populations: moments' transpose plus the direct relaxation term
  const B* mb_sa = mbar;
  const B* mb_ja = mbar + M;
  const B mb_sf = mbar[M + M * D];
  const B* mb_jf = mbar + M + M * D + 1;
  const B* mb_Pt = mbar + M + M * D + 1 + D;
  const B mb_sg = mbar[M + M * D + 1 + D + D * D];
  const B* mb_q = mbar + M + M * D + 1 + D + D * D + 1;
  for_each_dir<D>([&](int i, int cx, int cy, int cz) {
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int l = 0; l < L; ++l) {
      B v;
      if (l < M) {
        v = mb_sa[l];
#pragma unroll
        for (int b = 0; b < D; ++b) v += B(cc[b]) * mb_ja[l * D + b];
      } else if (l == M) {
        v = mb_sf;
#pragma unroll
        for (int b = 0; b < D; ++b) {
          v += B(cc[b]) * mb_jf[b];
#pragma unroll
          for (int c = 0; c < D; ++c) v += B(cc[b] * cc[c]) * mb_Pt[b * D + c];
        }
      } else {
        v = mb_sg;
#pragma unroll
        for (int b = 0; b < D; ++b) v += B(cc[b]) * mb_q[b];
      }
      if (i != REST) v += (lam[l * Q + i] - lam[l * Q + REST]) * coef[l];
      a.Pbar[(size_t)(l * Q + i) * N + n] = v;
    }
  });
  a.phibar[n] += pb_phi;
  a.kbar[n] += pb_k;
}

// Macro fields and gradient stencil: Pbar(x) += (dm/dP)^T mbar(x), with
// mbar(x) = sum over the nodes y whose stencil reads x of the stencil weight
// times Gbar(y); phibar(x) += (dm/dphi)^T mbar(x).
template <class B, int D, int M, bool EN, int K>
__global__ void __launch_bounds__(128) k_adj_macro(Params<B> p, InletTables<B> it, AdjArgs<B> a,
                                                   const __grid_constant__ AdjParams<B, K> ap) {
  using T = Dual<B, K>;
  constexpr int Q = Lat<D>::Q, L = n_lat<D, M, EN>(), LQ = L * Q;
  constexpr int NMAC = 2 * D + (EN ? M : 0);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int N = p.N;
  int x, y, z;
  node_xyz<B, D>(p, n, x, y, z);
  // ---- transpose of the stencil (same neighbour rule as Grad::compute) ----
  B mb[NMAC];
#pragma unroll
  for (int k = 0; k < NMAC; ++k) mb[k] = B(0);
  int cand[27];
  int nc = 0;
  const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
  for (int oz = zlo; oz <= zhi; ++oz)
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        int sx = x + ox;
        if (sx < 0 || sx >= p.nx) {
          if (p.bc_lo != BC_PERIODIC) continue;
          sx = wrapi(sx, p.nx);
        }
        const int sy = wrapi(y + oy, p.ny);
        const int sz = (D == 3) ? wrapi(z + oz, p.nz) : 0;
        const int m = sx + p.nx * (sy + p.ny * sz);
        bool seen = false;
        for (int q = 0; q < nc; ++q) seen |= (cand[q] == m);
        if (!seen) cand[nc++] = m;
      }
  for (int q = 0; q < nc; ++q) {
    const int m = cand[q];
    int mx, my, mz;
    node_xyz<B, D>(p, m, mx, my, mz);
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      if (csq_of<D>(I) == 0) return;
      int sx = mx + c_of<D>(I, 0);
      if (sx < 0) sx = (p.bc_lo == BC_PERIODIC) ? sx + p.nx : 0;
      if (sx >= p.nx) sx = (p.bc_hi == BC_PERIODIC) ? sx - p.nx : p.nx - 1;
      const int sy = wrapi(my + c_of<D>(I, 1), p.ny);
      const int sz = (D == 3) ? wrapi(mz + c_of<D>(I, 2), p.nz) : 0;
      if (sx + p.nx * (sy + p.ny * sz) != n) return;
      const B w = grad_w<B, D>(I);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int cb = c_of<D>(I, b);
        if (cb == 0) continue;
        const B wc = w * B(cb);
        mb[b] += wc * a.Gbar[(size_t)0 * N + m];
        mb[D + b] += wc * a.Gbar[(size_t)(1 + b) * N + m];
        if (EN) {
#pragma unroll
          for (int k = 0; k < M; ++k) mb[2 * D + k] += wc * a.Gbar[(size_t)(1 + D + k * D + b) * N + m];
        }
      }
    });
  }
  // ---- macro fields of the streamed populations ----------------------------
  B P[LQ];
  pull_node<B, D, M, EN>(p, it, a.f, a.phi, x, y, z, P);
  B sa[M], sf = B(0), jf[D], sg = B(0);
#pragma unroll
  for (int k = 0; k < M; ++k) sa[k] = B(0);
#pragma unroll
  for (int b = 0; b < D; ++b) jf[b] = B(0);
  for_each_dir<D>([&](int i, int cx, int cy, int cz) {
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int k = 0; k < M; ++k) sa[k] += P[k * Q + i];
    sf += P[M * Q + i];
#pragma unroll
    for (int b = 0; b < D; ++b) jf[b] += B(cc[b]) * P[M * Q + i];
    if (EN) sg += P[(M + 1) * Q + i];
  });
  // directions: sa (M), sf, jf (D), sg (EN), phi
  constexpr int NDM = M + 1 + D + (EN ? 1 : 0) + 1;
  B bar[NDM];
  const B Tf = EN ? B(0) : a.Tfix[n];
#pragma unroll 1
  for (int c0 = 0; c0 < NDM; c0 += K) {
    auto seeded = [&](B v, int dir) {
      T t(v);
      if (dir - c0 >= 0 && dir - c0 < K) t.d[dir - c0] = B(1);
      return t;
    };
    Moments<T, D, M, EN, false> mo;
#pragma unroll
    for (int k = 0; k < M; ++k) mo.sa[k] = seeded(sa[k], k);
    mo.sf = seeded(sf, M);
#pragma unroll
    for (int b = 0; b < D; ++b) mo.jf[b] = seeded(jf[b], M + 1 + b);
    mo.sg = EN ? seeded(sg, M + 1 + D) : T(B(0));
    const T phid = seeded(a.phi[n], NDM - 1);
    State<T, D, M> s;
    s.template from_moments<EN, false>(ap.pz, mo, phid, T(Tf));
    T m[NMAC];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      m[b] = s.u[b];
      m[D + b] = s.Pi(b);
    }
    if (EN) {
#pragma unroll
      for (int k = 0; k < M; ++k) m[2 * D + k] = s.Y[k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (c0 + k >= NDM) break;
      B acc = B(0);
#pragma unroll
      for (int q = 0; q < NMAC; ++q) acc += mb[q] * m[q].d[k];
      bar[c0 + k] = acc;
    }
  }
  // d(moments)/dP: species sums, momentum-lattice mass and momentum, energy sum
  for_each_dir<D>([&](int i, int cx, int cy, int cz) {
    const int cc[3] = {cx, cy, cz};
#pragma unroll
    for (int k = 0; k < M; ++k) a.Pbar[(size_t)(k * Q + i) * N + n] += bar[k];
    B v = bar[M];
#pragma unroll
    for (int b = 0; b < D; ++b) v += B(cc[b]) * bar[M + 1 + b];
    a.Pbar[(size_t)(M * Q + i) * N + n] += v;
    if (EN) a.Pbar[(size_t)((M + 1) * Q + i) * N + n] += bar[M + 1 + D];
  });
  a.phibar[n] += (double)bar[NDM - 1];
}

// Reservoir ghosts: the missing populations of a face node are equilibria
// moving with u = j / (sum f / phi) of the adjacent node's streamed momentum
// populations.  One thread per (y, z) handles both faces in turn.
template <class B, int D, int M, bool EN, int K>
__global__ void __launch_bounds__(128) k_adj_ghost(Params<B> p, InletTables<B> it, AdjArgs<B> a,
                                                   const __grid_constant__ AdjParams<B, K> ap) {
  using T = Dual<B, K>;
  constexpr int Q = Lat<D>::Q, L = n_lat<D, M, EN>();
  static_assert(D + 3 <= K, "ghost directions exceed the dual lanes");
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.ny * p.nz) return;
  const int N = p.N;
  const int y = t % p.ny, z = t / p.ny;
  InletTables<T> itd;
  for (int s = 0; s < 2; ++s) {
    for (int k = 0; k < MMAX; ++k) itd.rho[s][k] = T(it.rho[s][k]);
    itd.rho_sum[s] = T(it.rho_sum[s]);
    itd.Rmix[s] = T(it.Rmix[s]);
    itd.Umix[s] = T(it.Umix[s]);
    itd.T[s] = T(it.T[s]);
  }
  for (int side = 0; side < 2; ++side) {
    if ((side == 0 ? p.bc_lo : p.bc_hi) != BC_INLET) continue;
    const int xb = side == 0 ? 0 : p.nx - 1;
    const int xa = side == 0 ? 1 : p.nx - 2;
    const int nb = xb + p.nx * (y + p.ny * z), na = xa + p.nx * (y + p.ny * z);
    Site<B, D> sa;
    sa.init(p, xa, y, z);
    B s0 = B(0), j[D];
#pragma unroll
    for (int b = 0; b < D; ++b) j[b] = B(0);
    for_each_dir<D>([&](int i, int cx, int cy, int cz) {
      const B f = a.f[(size_t)(M * Q + i) * N + sa.source(cx, cy, cz)];
      const int cc[3] = {cx, cy, cz};
      s0 += f;
#pragma unroll
      for (int b = 0; b < D; ++b) j[b] += B(cc[b]) * f;
    });
    // directions: s0, j (D), phi(xa), phi(face)
    auto seeded = [&](B v, int dir) {
      T r(v);
      r.d[dir] = B(1);
      return r;
    };
    const T s0d = seeded(s0, 0);
    T jd[D];
#pragma unroll
    for (int b = 0; b < D; ++b) jd[b] = seeded(j[b], 1 + b);
    const T pha = seeded(a.phi[na], D + 1);
    Ghost<T, D> gh;
    gh.side = side;
    const T rho_f = s0d / pha;
#pragma unroll
    for (int b = 0; b < D; ++b) gh.u[b] = jd[b] / rho_f;
    gh.phi = seeded(a.phi[nb], D + 2);
    Site<B, D> sb;
    sb.init(p, xb, y, z);
    B acc[D + 3];
#pragma unroll
    for (int k = 0; k < D + 3; ++k) acc[k] = B(0);
    for_each_dir<D>([&](int i, int cx, int cy, int cz) {
      if (sb.source(cx, cy, cz) != SRC_GHOST) return;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        const T g = pull_rt<T, D, M, EN>(ap.pz, itd, (const T*)nullptr, gh, nb, SRC_GHOST, l, i, cx, cy, cz);
        const B pb = a.Pbar[(size_t)(l * Q + i) * N + nb];
#pragma unroll
        for (int k = 0; k < D + 3; ++k) acc[k] += pb * g.d[k];
      }
    });
    for_each_dir<D>([&](int i, int cx, int cy, int cz) {
      const int cc[3] = {cx, cy, cz};
      B v = acc[0];
#pragma unroll
      for (int b = 0; b < D; ++b) v += B(cc[b]) * acc[1 + b];
      a.Pbar[(size_t)(M * Q + i) * N + na] += v;
    });
    a.phibar[na] += (double)acc[D + 1];
    a.phibar[nb] += (double)acc[D + 2];
  }
}

// Transpose of the pull: lambda^n_j(z) is the adjoint of every streamed
// population that copied f^n_j(z).
template <class B, int D, int M, bool EN>
__global__ void __launch_bounds__(256) k_adj_stream(Params<B> p, AdjArgs<B> a) {
  constexpr int Q = Lat<D>::Q, L = n_lat<D, M, EN>();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int N = p.N;
  int x, y, z;
  node_xyz<B, D>(p, n, x, y, z);
  for (int j = 0; j < Q; ++j) {
    const int cx = c_of<D>(j, 0), cy = c_of<D>(j, 1), cz = c_of<D>(j, 2);
    int tx = x + cx;
    int tgt = -1, lane = j;
    if (tx < 0 || tx >= p.nx) {
      const int bc = tx < 0 ? p.bc_lo : p.bc_hi;
      if (bc == BC_PERIODIC) tx = wrapi(tx, p.nx);
      else if (bc == BC_BOUNCEBACK) {
        tgt = n;                       // pulled back by this node in the opposite direction
        lane = opp_of<D>(j);
      } else {
        tgt = -2;                      // leaves through a reservoir face
      }
    }
    if (tgt == -1) tgt = tx + p.nx * (wrapi(y + cy, p.ny) + p.ny * ((D == 3) ? wrapi(z + cz, p.nz) : 0));
#pragma unroll
    for (int l = 0; l < L; ++l)
      a.lam0[(size_t)(l * Q + j) * N + n] = tgt >= 0 ? a.Pbar[(size_t)(l * Q + lane) * N + tgt] : B(0);
  }
}

// Objective: J = w * sum over the nodes of plane x = xo of the species-a
// momentum along `axis` of the streamed populations (the flux moment j_a of
// the state); seeds Pbar with its gradient.
template <class B, int D, int M, bool EN>
__global__ void k_adj_seed_flux(Params<B> p, AdjArgs<B> a, int species, int axis, int xo, B w) {
  constexpr int Q = Lat<D>::Q, L = n_lat<D, M, EN>();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int N = p.N;
  const bool on = (n % p.nx) == xo;
  for (int l = 0; l < L; ++l)
    for (int i = 0; i < Q; ++i)
      a.Pbar[(size_t)(l * Q + i) * N + n] = (on && l == species) ? w * B(c_of<D>(i, axis)) : B(0);
}

// Initial equilibria: phibar(x) += lambda^0(x)^T df^0(x)/dphi(x).
template <class B, int D, int M, bool EN>
__global__ void __launch_bounds__(128) k_adj_init(Params<B> p, const double* __restrict__ X,
                                                  const double* __restrict__ T0, const double* __restrict__ P0,
                                                  const double* __restrict__ U0v, double cvel, double RU_si,
                                                  AdjArgs<B> a) {
  using T = Dual<B, 1>;
  constexpr int Q = Lat<D>::Q;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  const int N = p.N;
  T phid(a.phi[n]);
  phid.d[0] = B(1);
  double acc = 0.0;
  init_node<T, D, M, EN>(p, X, T0, P0, U0v, cvel, RU_si, n, N, phid, [&](int l, int i, const T& v) {
    acc += (double)a.lam0[(size_t)(l * Q + i) * N + n] * (double)v.d[0];
  });
  a.phibar[n] += acc;
}

// Launch table of the adjoint kernels for one (precision, D, M, energy).
template <class B>
struct AdjOps {
  int (*collide)(const Params<B>&, const InletTables<B>&, const AdjArgs<B>&, cudaStream_t);
  int (*macro)(const Params<B>&, const InletTables<B>&, const AdjArgs<B>&, cudaStream_t);
  int (*ghost)(const Params<B>&, const InletTables<B>&, const AdjArgs<B>&, cudaStream_t);
  void (*stream)(const Params<B>&, const AdjArgs<B>&, cudaStream_t);
  void (*seed_flux)(const Params<B>&, const AdjArgs<B>&, int species, int axis, int xo, double w, cudaStream_t);
  void (*init)(const Params<B>&, const double*, const double*, const double*, const double*, double, double,
               const AdjArgs<B>&, cudaStream_t);
  int n_grad;
};

bool get_adj_ops_f32(int D, int M, int energy, AdjOps<float>* out);
bool get_adj_ops_f64(int D, int M, int energy, AdjOps<double>* out);

}  // namespace lbm
