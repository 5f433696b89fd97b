// Per-node stream / moments / collide building blocks, shared by the kernels.
#pragma once

#include <type_traits>

#include "lbm_device.cuh"

namespace lbm {

constexpr int BC_PERIODIC = 0;
constexpr int BC_INLET = 1;
constexpr int BC_BOUNCEBACK = 2;
constexpr int SRC_GHOST = -0x7fffffff;

// Ghost state of a reservoir face: reservoir density, temperature and
// composition from the configuration, velocity of the adjacent interior node
// of the same step (reading of the "simplified flux" condition of Sec. 5.1,
// replacing only the missing populations).
template <class R, int D>
struct Ghost {
  int side;        // 0: x = 0 face, 1: x = nx-1 face
  R phi;
  R u[D];
};

template <class R>
struct InletTables {
  R rho[2][MMAX];   // species densities of the reservoirs
  R rho_sum[2];
  R Rmix[2];        // mixture gas constant
  R Umix[2];        // mixture specific internal energy at T_in
  R T[2];
};

// Streamed populations of one node: pull f(x - c_i) with the boundary rules.
template <class R, int D, int M, bool EN>
struct Puller {
  static constexpr int Q = Lat<D>::Q;
  const R* __restrict__ src;
  int N;
  int n;
  int sidx[Q];        // >= 0 source node; < 0 && != SRC_GHOST: bounce-back at -1-sidx
  Ghost<R, D> gh;
  const InletTables<R>* it;
  const Params<R>* p;

  LBM_HD void setup(const Params<R>& P, const InletTables<R>& IT, const R* __restrict__ s,
                                        const R* __restrict__ phiA, int x, int y, int z) {
    p = &P;
    it = &IT;
    src = s;
    N = P.N;
    n = x + P.nx * (y + P.ny * z);
    gh.side = -1;
    bool need_ghost = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = c_of<D>(i, 0), cy = c_of<D>(i, 1), cz = c_of<D>(i, 2);
      int sx = x - cx;
      int sy = wrapi(y - cy, P.ny);
      int sz = (D == 3) ? wrapi(z - cz, P.nz) : 0;
      int code;
      if (sx < 0 || sx >= P.nx) {
        int bc = sx < 0 ? P.bc_lo : P.bc_hi;
        if (bc == BC_PERIODIC) {
          code = wrapi(sx, P.nx) + P.nx * (sy + P.ny * sz);
        } else if (bc == BC_BOUNCEBACK) {
          code = -1 - n;
        } else {
          code = SRC_GHOST;
          need_ghost = true;
          gh.side = sx < 0 ? 0 : 1;
        }
      } else {
        code = sx + P.nx * (sy + P.ny * sz);
      }
      sidx[i] = code;
    }
    if (need_ghost) {
      // velocity of the adjacent interior node: its sources are all inside
      int xa = gh.side == 0 ? 1 : P.nx - 2;
      int na = xa + P.nx * (y + P.ny * z);
      R s0 = R(0), j[D];
#pragma unroll
      for (int a = 0; a < D; ++a) j[a] = R(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int cx = c_of<D>(i, 0), cy = c_of<D>(i, 1), cz = c_of<D>(i, 2);
        int sx = xa - cx;
        int sy = wrapi(y - cy, P.ny);
        int sz = (D == 3) ? wrapi(z - cz, P.nz) : 0;
        R f = s[(size_t)(M * Q + i) * N + sx + P.nx * (sy + P.ny * sz)];
        s0 += f;
#pragma unroll
        for (int a = 0; a < D; ++a) j[a] += f * R(c_of<D>(i, a));
      }
      R rho_f = s0 / phiA[na];
#pragma unroll
      for (int a = 0; a < D; ++a) gh.u[a] = j[a] / rho_f;
      gh.phi = phiA[n];
    }
  }

  // equilibrium population of lattice l, direction I, at the reservoir state
  template <int I>
  LBM_HD R ghost(int l) const {
    const int sd = gh.side;
    const R phi = gh.phi;
    R T = it->T[sd];
    if (l < M) {
      R RaT = p->Ra[l] * T;
      R v = phi * it->rho[sd][l];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        R w = gh.u[a] / phi;
        v *= psi<R>(c_of<D>(I, a), w, w * w + RaT);
      }
      return v;
    }
    R RT = it->Rmix[sd] * T;
    if (l == M) {
      R v = phi * it->rho_sum[sd];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        R w = gh.u[a] / phi;
        v *= psi<R>(c_of<D>(I, a), w, w * w + RT);
      }
      return v;
    }
    GeqFactors<R, D> G;
    G.init(phi, it->rho_sum[sd], gh.u, RT, it->Umix[sd]);
    return G.template value<I>();
  }

  template <int I>
  LBM_HD R get(int l) const {
    int s = sidx[I];
    if (s >= 0) return src[(size_t)(l * Q + I) * N + s];
    if (s != SRC_GHOST) return src[(size_t)(l * Q + opp_of<D>(I)) * N + (-1 - s)];
    return ghost<I>(l);
  }
};

// Moments of the streamed populations (Eq. 4, Eq. 5,
// Eq. 37, Eq. 38, Eq. 39, q, P).
template <class R, int D, int M, bool EN, bool FULL>
struct Moments {
  R sa[M], ja[M][D];
  R sabs[M];              // sum_i |f_ai| (FP32 full moments only): resolution of rho_a
  R sf, jf[D];
  R Pt[D][D];
  R sg, q[D];

  template <class PullT>
  LBM_HD void compute(const PullT& pl) {
    constexpr int Q = Lat<D>::Q;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      sa[a] = R(0);
      sabs[a] = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) ja[a][b] = R(0);
    }
    sf = R(0);
    sg = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      jf[b] = R(0);
      q[b] = R(0);
#pragma unroll
      for (int c = 0; c < D; ++c) Pt[b][c] = R(0);
    }
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
#pragma unroll
      for (int a = 0; a < M; ++a) {
        R f = pl.template get<I>(a);
        sa[a] += f;
        if (FULL && ScalarTraits<R>::single) sabs[a] += fabs(f);
        if (FULL) {
#pragma unroll
          for (int b = 0; b < D; ++b)
            if (c_of<D>(I, b) != 0) ja[a][b] += R(c_of<D>(I, b)) * f;
        }
      }
      R f = pl.template get<I>(M);
      sf += f;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        if (c_of<D>(I, b) != 0) jf[b] += R(c_of<D>(I, b)) * f;
        if (FULL && EN) {
#pragma unroll
          for (int c = 0; c < D; ++c)
            if (c_of<D>(I, b) * c_of<D>(I, c) != 0) Pt[b][c] += R(c_of<D>(I, b) * c_of<D>(I, c)) * f;
        }
      }
      if (EN) {
        R g = pl.template get<I>(M + 1);
        sg += g;
        if (FULL) {
#pragma unroll
          for (int b = 0; b < D; ++b)
            if (c_of<D>(I, b) != 0) q[b] += R(c_of<D>(I, b)) * g;
        }
      }
    });
  }
};

// Composition, velocity, temperature and pressure of one node.
template <class R, int D, int M>
struct State {
  R phi, rho_a[M], rho_s, Y[M], X[M], m_mix, Rg, rho_f, u[D], T, P, cv;

  template <bool EN, bool FULL>
  LBM_HD void from_moments(const Params<R>& p, const Moments<R, D, M, EN, FULL>& mo,
                                               R phi_, R Tfixed) {
    phi = phi_;
    R inv_phi = R(1) / phi;
    rho_s = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      rho_a[a] = mo.sa[a] * inv_phi;          // Eq. 4
      rho_s += rho_a[a];                      // Eq. 1
    }
    R inv_rs = R(1) / rho_s;
    R inv_m = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      Y[a] = rho_a[a] * inv_rs;
      inv_m += Y[a] / p.m[a];
    }
    m_mix = R(1) / inv_m;
#pragma unroll
    for (int a = 0; a < M; ++a) X[a] = m_mix * Y[a] / p.m[a];
    Rg = p.RU * inv_m;                        // R = R_U / m
    rho_f = mo.sf * inv_phi;                  // Eq. 37
#pragma unroll
    for (int b = 0; b < D; ++b) u[b] = mo.jf[b] / rho_f;
    cv = R(0);
#pragma unroll
    for (int a = 0; a < M; ++a) cv += Y[a] * p.cvR[a];
    if (EN) {
      // Eq. 41 with constant C_v and u^2/(2 phi^2)
      R E = mo.sg / (phi * rho_f);
      R w2 = R(0), U0m = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) w2 += u[b] * u[b];
      w2 *= inv_phi * inv_phi;
#pragma unroll
      for (int a = 0; a < M; ++a) U0m += Y[a] * p.U0[a];
      T = p.T_thermo + (E - R(0.5) * w2 - U0m) / cv;
    } else {
      T = Tfixed;
    }
    P = rho_f * Rg * T;                       // Eq. 3
  }

  // Pi_alpha = rho u_alpha (1 - 3RT) - rho u_alpha^3 / phi^2 (Eq. 45)
  LBM_HD R Pi(int b) const {
    R w = u[b] / phi;
    return rho_f * u[b] * (R(1) - R(3) * Rg * T) - rho_f * u[b] * w * w;
  }
};

// Transport coefficients (Eq. 23, Eq. 24, Eq. 22, Eq. 26) and the
// diffusion-velocity solve (Eq. 29).
template <class R, int D, int M>
struct Transport {
  R inv_tau_ab[M][M];
  R inv_tau[M], beta[M], inv_tauk[M];
  R V[M][D];
  int used_fp64;

  LBM_HD void compute(const Params<R>& p, const State<R, D, M>& s,
                                          const R* ja /* [M][D] */, const R* sabs /* [M] */) {
    // D_ab = D_ref (T/T_ref)^1.5 (P_ref/P);  1/tau_ab = m R_U T / (D_ab m_a m_b)
    R tr = s.T * p.inv_T_ref;
    R C = s.m_mix * p.RU * s.T * s.P / (p.Pref * tr * sqrt_<R>(tr));
#pragma unroll
    for (int a = 0; a < M; ++a) {
      R acc = R(0);
#pragma unroll
      for (int b = 0; b < M; ++b) {
        inv_tau_ab[a][b] = C * p.invDmm[a][b];
        acc += s.Y[b] * inv_tau_ab[a][b];
      }
      inv_tau[a] = acc;
      beta[a] = acc / (R(2) + acc);           // dt/(2 tau + dt) with dt = 1
      inv_tauk[a] = p.knudsen ? p.knc[a] * sqrt_<R>(s.T) / s.phi : R(0);
    }
    // A V = u_a - u - u/(2tau^k_a), A_aa = 1 + 1/(2tau_a) + 1/(2tau^k_a),
    // A_ab = -Y_b/(2 tau_ab): the trapezoidal rule on the Knudsen relaxation
    // toward the resting f^k acts on the component velocity u + V_a, which
    // adds -u/(2tau^k_a) to the right-hand side (reading R27)
    R A[M][M], B[M][D];
    R amax = R(0), dmin = R(1e30);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      R rs = R(0);
#pragma unroll
      for (int b = 0; b < M; ++b) {
        A[a][b] = (a == b) ? (R(1) + R(0.5) * inv_tau[a] + R(0.5) * inv_tauk[a])
                           : (R(-0.5) * s.Y[b] * inv_tau_ab[a][b]);
        rs += fabs(A[a][b]);
      }
      amax = rs > amax ? rs : amax;
      R d = R(1) + R(0.5) * inv_tauk[a];
      dmin = d < dmin ? d : dmin;
      // trace species move with the mixture: below 1e-14 of the mixture
      // density (the oracle's bound) and, in FP32, where the species density
      // is not resolved by its populations.  Where the streamed populations
      // of a species cancel (sum |f_ai| > 1e4 rho_a: a trace tail crossed by
      // weakly relaxed non-equilibrium populations), FP32 leaves j_a / rho_a
      // to rounding noise, which the quasi-equilibrium then amplifies.
      bool tiny = s.rho_a[a] < R(1e-14) * s.rho_s;
      if (ScalarTraits<R>::single) tiny = tiny || !(sabs[a] <= R(1e4) * s.phi * s.rho_a[a]);
#pragma unroll
      for (int b = 0; b < D; ++b)
        B[a][b] = (tiny ? R(0) : (ja[a * D + b] / s.rho_a[a] - s.u[b])) - R(0.5) * inv_tauk[a] * s.u[b];
    }
    used_fp64 = 0;
    bool fp64_solve = false;
    if constexpr (std::is_same<R, float>::value) fp64_solve = amax > p.kappa_thr * dmin;
    if (fp64_solve) {
      if constexpr (std::is_same<R, float>::value) {
      // condition bound above the threshold: assemble and solve in double
      // from the single-precision moments (the relaxation rates and the
      // right-hand side's differences of velocities formed in double)
      double Ad[M][M], Bd[M][D];
      const double Td = (double)s.T;
      const double trd = Td * (double)p.inv_T_ref;
      const double Cd = (double)s.m_mix * (double)p.RU * Td * (double)s.P / ((double)p.Pref * trd * sqrt(trd));
      double itk[M];
#pragma unroll
      for (int a = 0; a < M; ++a)
        itk[a] = p.knudsen ? (double)p.knc[a] * sqrt(Td) / (double)s.phi : 0.0;
#pragma unroll
      for (int a = 0; a < M; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < M; ++b) acc += (double)s.Y[b] * Cd * (double)p.invDmm[a][b];
#pragma unroll
        for (int b = 0; b < M; ++b)
          Ad[a][b] = (a == b) ? 1.0 + 0.5 * acc + 0.5 * itk[a] : -0.5 * (double)s.Y[b] * Cd * (double)p.invDmm[a][b];
        bool tiny = s.rho_a[a] < R(1e-14) * s.rho_s || !(sabs[a] <= R(1e4) * s.phi * s.rho_a[a]);
#pragma unroll
        for (int b = 0; b < D; ++b)
          Bd[a][b] = (tiny ? 0.0 : ((double)ja[a * D + b] / (double)s.rho_a[a] - (double)s.u[b])) -
                     0.5 * itk[a] * (double)s.u[b];
      }
      gauss<double>(Ad, Bd);
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) V[a][b] = (R)Bd[a][b];
      used_fp64 = 1;
      }
    } else {
      gauss<R>(A, B);
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) V[a][b] = B[a][b];
    }
  }

  // Gaussian elimination without pivoting: the matrix is strictly row
  // diagonally dominant (margin 1 + dt/2tau^k), so no pivoting is needed.
  template <class T>
  LBM_HD static void gauss(T (&A)[M][M], T (&B)[M][D]) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      T inv = T(1) / A[k][k];
#pragma unroll
      for (int r = k + 1; r < M; ++r) {
        T f = A[r][k] * inv;
#pragma unroll
        for (int c = k + 1; c < M; ++c) A[r][c] -= f * A[k][c];
#pragma unroll
        for (int c = 0; c < D; ++c) B[r][c] -= f * B[k][c];
      }
    }
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
      T inv = T(1) / A[k][k];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        T s = B[k][c];
#pragma unroll
        for (int j = k + 1; j < M; ++j) s -= A[k][j] * B[j][c];
        B[k][c] = s * inv;
      }
    }
  }
};

// Isotropic gradient weights 3 w_i (c_s^2 = 1/3) of the standard lattice.
template <class R, int D>
LBM_HD constexpr R grad_w(int i) {
  return R(3) * ((c_of<D>(i, 0) == 0 ? R(2) / R(3) : R(1) / R(6)) * (c_of<D>(i, 1) == 0 ? R(2) / R(3) : R(1) / R(6)) *
                 (D == 3 ? (c_of<D>(i, 2) == 0 ? R(2) / R(3) : R(1) / R(6)) : R(1)));
}

}  // namespace lbm
