// Device-side physics of the mean-field porous-media LBM step (sm_103a).
//
// Every per-node quantity follows Sawant & Karlin, arXiv 2409.02930:
//   species lattices      Sec. 2.2-2.3 (Eq. 15, Eq. 16, Eq. 18,
//                         Eq. 21, Eq. 22,
//                         Eq. 23, Eq. 24, Eq. 25, Eq. 26,
//                         Eq. 28, Eq. 29)
//   momentum lattice      Sec. 3.2 (Eq. 42, Eq. 44, Eq. 45, Eq. 47,
//                         Eq. 48)
//   energy lattice        Sec. 3.3 (Eq. 43, Eq. 51, Eq. 54,
//                         Eq. 55, Eq. 58, Eq. 59,
//                         Eq. 60)
//   transport             Eq. 65, Eq. 67; Knudsen diffusivity of Sec. 5.1
// The readings taken where the paper is ambiguous are the library's
// documented ones (dimensional tau_ab and tau^k; porosity-weighted
// quasi-equilibrium and energy operator; u^ex = u + dt F^k/(omega rho);
// rho of the momentum lattice in every Sec. 3 quantity; component
// velocities u + V_b in F^k; mass-average-free V in q^diff).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

// Per-node functions are host+device so that the exact kernel arithmetic can
// also be exercised by host-side debugging harnesses.
#define LBM_HD __host__ __device__ __forceinline__

namespace lbm {

constexpr int MMAX = 6;
constexpr int SMAX = 12;
constexpr int RMAX = 32;

// Lattice-unit parameters, computed on the host once per context.
template <class R>
struct Params {
  int nx, ny, nz, N;
  int bc_lo, bc_hi;
  int knudsen;
  R RU;                       // universal gas constant, lattice units per kelvin
  R m[MMAX];                  // molar masses [kg/mol]
  R Ra[MMAX];                 // R_a = R_U / m_a
  R invDmm[MMAX][MMAX];       // 1 / (D_ab,ref m_a m_b), zero on the diagonal
  R muref[MMAX];
  R mu_exp, inv_Pr, bulk_ratio, T_thermo, inv_T_ref, Pref;
  R cvR[MMAX];                // C_v,a = cv_factor_a R_a
  R U0[MMAX];
  R knc[MMAX];                // 1/tau^k_a = knc_a sqrt(T) / phi
  R rho_in[2][MMAX];          // reservoir densities [kg/m^3]
  R T_in[2];
  R kappa_thr;
  int wait_limit;             // probes per bounded device wait of the row-staged forms
};

// ---------------------------------------------------------------------------
// velocity set helpers (c_i of Eq. 10; i = (cx+1) + 3(cy+1) + 9(cz+1))
// ---------------------------------------------------------------------------
template <int D> struct Lat { static constexpr int Q = (D == 3) ? 27 : 9; };

__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }
template <int D> __host__ __device__ constexpr int c_of(int i, int a) {
  return a == 0 ? cx_of(i) : (a == 1 ? cy_of(i) : (D == 3 ? cz_of(i) : 0));
}
template <int D> __host__ __device__ constexpr int opp_of(int i) {
  return (D == 3) ? (26 - i) : (8 - i);
}
template <int D> __host__ __device__ constexpr int csq_of(int i) {
  return c_of<D>(i, 0) * c_of<D>(i, 0) + c_of<D>(i, 1) * c_of<D>(i, 1) + c_of<D>(i, 2) * c_of<D>(i, 2);
}

// Product-form factor Psi_c(xi, P) (Eq. 11, Eq. 12, Eq. 13).
template <class R>
LBM_HD R psi(int c, R xi, R P) {
  return c == 0 ? (R(1) - P) : R(0.5) * (R(c) * xi + P);
}

// the three per-axis factors for c = -1, 0, +1 (index c+1)
template <class R>
LBM_HD void psi3(R xi, R P, R out[3]) {
  out[0] = R(0.5) * (P - xi);
  out[1] = R(1) - P;
  out[2] = R(0.5) * (P + xi);
}

// single-precision storage and arithmetic (dual numbers inherit it from their base)
template <class R> struct ScalarTraits { static constexpr bool single = sizeof(R) == 4; };

// square root and power per scalar type (specialised for dual numbers too)
template <class R> struct MathOps;
template <> struct MathOps<float> {
  static LBM_HD float sqrt(float v) { return sqrtf(v); }
  static LBM_HD float pow(float a, float b) { return powf(a, b); }
};
template <> struct MathOps<double> {
  static LBM_HD double sqrt(double v) { return ::sqrt(v); }
  static LBM_HD double pow(double a, double b) { return ::pow(a, b); }
};
template <class R> LBM_HD R sqrt_(R v) { return MathOps<R>::sqrt(v); }
template <class R> LBM_HD R pow_(R a, R b) { return MathOps<R>::pow(a, b); }
template <class R> LBM_HD bool finite_(R v) { return v == v && v - v == v - v; }

LBM_HD int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// ---------------------------------------------------------------------------
// Energy equilibrium (Eq. 51) in closed form.  The operator O_alpha of
// Eq. 50 acts in w = u/phi; on the generating function
// E = U + sum_beta w_beta^2/2 it gives, per axis,
//   O 1 = w, O^2 1 = RT + w^2                         (the factors P1)
//   O (w^2/2) = RT w + w^3/2, O^2 (w^2/2) = RT^2 + 5/2 RT w^2 + w^4/2
// so g^eq_i = phi rho [ U Prod_a P1_a + sum_b P2_b Prod_{a != b} P1_a ].
// ---------------------------------------------------------------------------
template <class R, int D>
struct GeqFactors {
  R P1[3][3], P2[3][3];
  R pref_U, pref;  // phi rho U, phi rho
  LBM_HD void init(R phi, R rho, const R* u, R RT, R U) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      R w = u[a] / phi;
      R w2 = w * w;
      psi3<R>(w, RT + w2, P1[a]);
      R O = RT * w + R(0.5) * w2 * w;
      R O2 = RT * RT + R(2.5) * RT * w2 + R(0.5) * w2 * w2;
      P2[a][0] = R(0.5) * (O2 - O);
      P2[a][1] = R(0.5) * w2 - O2;
      P2[a][2] = R(0.5) * (O2 + O);
    }
    pref = phi * rho;
    pref_U = pref * U;
  }
  template <int I>
  LBM_HD R value() const {
    R prod = R(1);
#pragma unroll
    for (int a = 0; a < D; ++a) prod *= P1[a][c_of<D>(I, a) + 1];
    R s = R(0);
#pragma unroll
    for (int b = 0; b < D; ++b) {
      R t = P2[b][c_of<D>(I, b) + 1];
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a != b) t *= P1[a][c_of<D>(I, a) + 1];
      s += t;
    }
    return pref_U * prod + pref * s;
  }
};

// compile-time loop helper
template <int I, int N>
struct Unroll {
  template <class F>
  LBM_HD static void run(F&& f) {
    f(std::integral_constant<int, I>{});
    Unroll<I + 1, N>::run(f);
  }
};
template <int N>
struct Unroll<N, N> {
  template <class F>
  LBM_HD static void run(F&&) {}
};

}  // namespace lbm
