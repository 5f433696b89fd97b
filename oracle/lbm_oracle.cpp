// Plain FP64 CPU oracle of the mean-field lattice Boltzmann step for reactive
// mixtures in homogenised porous media (Sawant & Karlin, arXiv 2409.02930).
//
// TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
// leg of the benchmark load this file.  It shares no code, header, table or
// helper with the CUDA library; the two only see the same physical inputs.
//
// The oracle is deliberately slow and literal: every per-node quantity is
// computed from the paper's equations in the paper's order, in double
// precision, with plain loops over nodes, populations and species.  Where the
// paper is ambiguous the reading taken is stated at the point of use (the
// readings are numbered R1..R21 as in the design notes).
//
// Units: lattice units (length dx, time dt) for velocities, temperatures R*T,
// diffusivities, viscosities and pressures; densities stay in kg/m^3 (every
// lattice equation is homogeneous in the density).  Temperatures are kept in
// kelvin and R_a is stored per kelvin.

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// ---------------------------------------------------------------------------
// Scalar type.  The plain build computes in double.  Built with
// -DORACLE_DUAL=K every quantity also carries K directional derivatives
// (forward-mode dual numbers): the value part repeats the plain build's
// operations one for one and each derivative part applies the chain rule of
// the operation, so the derivative parts after n steps are exact
// Jacobian-vector products of the whole time loop with respect to the seeded
// inputs (porosity field, pore radius, tortuosity, pre-exponential factors).
// ---------------------------------------------------------------------------
inline double rmax(double a, double b) { return (a < b) ? b : a; }
inline double rmin(double a, double b) { return (b < a) ? b : a; }
#ifndef ORACLE_DUAL
typedef double real;
inline double comp(double x, int) { return x; }
inline double r_sqrt(double x) { return std::sqrt(x); }
inline double r_exp(double x) { return std::exp(x); }
inline double r_pow(double x, double p) { return std::pow(x, p); }
inline double r_fabs(double x) { return std::fabs(x); }
#else
const int NT = ORACLE_DUAL;
struct real {
  double v;
  double d[NT];
  real() : v(0.0) { for (int k = 0; k < NT; ++k) d[k] = 0.0; }
  real(double x) : v(x) { for (int k = 0; k < NT; ++k) d[k] = 0.0; }
  real(int x) : real((double)x) {}
  real& operator+=(const real& b) { v += b.v; for (int k = 0; k < NT; ++k) d[k] += b.d[k]; return *this; }
  real& operator-=(const real& b) { v -= b.v; for (int k = 0; k < NT; ++k) d[k] -= b.d[k]; return *this; }
  real& operator*=(const real& b) {            // (uv)' = u'v + uv'
    for (int k = 0; k < NT; ++k) d[k] = d[k] * b.v + v * b.d[k];
    v *= b.v;
    return *this;
  }
  real& operator/=(const real& b) {            // (u/v)' = (u' - (u/v) v')/v
    const double q = v / b.v;
    for (int k = 0; k < NT; ++k) d[k] = (d[k] - q * b.d[k]) / b.v;
    v = q;
    return *this;
  }
};
inline real operator+(real a, const real& b) { return a += b; }
inline real operator-(real a, const real& b) { return a -= b; }
inline real operator*(real a, const real& b) { return a *= b; }
inline real operator/(real a, const real& b) { return a /= b; }
inline real operator-(const real& a) { real r; r.v = -a.v; for (int k = 0; k < NT; ++k) r.d[k] = -a.d[k]; return r; }
inline bool operator<(const real& a, const real& b) { return a.v < b.v; }
inline bool operator>(const real& a, const real& b) { return a.v > b.v; }
inline bool operator<=(const real& a, const real& b) { return a.v <= b.v; }
inline bool operator>=(const real& a, const real& b) { return a.v >= b.v; }
inline bool operator==(const real& a, const real& b) { return a.v == b.v; }
inline bool operator!=(const real& a, const real& b) { return a.v != b.v; }
inline double comp(const real& x, int lane) { return lane < 0 ? x.v : x.d[lane]; }
inline real chain(const real& x, double fx, double dfx) {
  real r;
  r.v = fx;
  for (int k = 0; k < NT; ++k) r.d[k] = dfx * x.d[k];
  return r;
}
inline real r_sqrt(const real& x) { const double s = std::sqrt(x.v); return chain(x, s, 0.5 / s); }
inline real r_exp(const real& x) { const double e = std::exp(x.v); return chain(x, e, e); }
inline real r_pow(const real& x, double p) {
  return chain(x, std::pow(x.v, p), p == 0.0 ? 0.0 : p * std::pow(x.v, p - 1.0));
}
inline real r_fabs(const real& x) { return x.v < 0 ? -x : x; }
inline real rmax(const real& a, const real& b) { return (a < b) ? b : a; }
inline real rmin(const real& a, const real& b) { return (b < a) ? b : a; }
#endif

// Stored populations.  The plain build keeps them in double.  Built with
// -DORACLE_STORE_F32 every stored population (the initial equilibria and the
// output of every collision) is rounded to single precision while all the
// arithmetic stays in double: the error that single-precision storage alone
// imposes on a lattice, the floor any single-precision implementation sits
// on (a measuring build of the test infrastructure, not a second method).
#ifdef ORACLE_STORE_F32
inline real stored(const real& v) { return (double)(float)v; }
#else
inline real stored(const real& v) { return v; }
#endif

namespace {

const double R_UNIV = 8.314462618;      // J/(mol K)
const double PI_D = 3.14159265358979323846;
const int MMAX = 8;
const int QMAX = 27;
const int SMAX = 12;
const int RMAX = 32;

// ---------------------------------------------------------------------------
// velocity set (Sec. 2.2, Eq. 10): c_i in {-1,0,1}^D, D = 2 or 3.
// ordering i = (cx+1) + 3 (cy+1) + 9 (cz+1).
// ---------------------------------------------------------------------------
struct Lattice {
  int D, Q;
  int c[QMAX][3];
  int opp[QMAX];
};

Lattice make_lattice(int D) {
  Lattice L;
  L.D = D;
  L.Q = (D == 3) ? 27 : 9;
  for (int i = 0; i < L.Q; ++i) {
    L.c[i][0] = i % 3 - 1;
    L.c[i][1] = (i / 3) % 3 - 1;
    L.c[i][2] = (D == 3) ? (i / 9) - 1 : 0;
  }
  for (int i = 0; i < L.Q; ++i)
    for (int j = 0; j < L.Q; ++j)
      if (L.c[j][0] == -L.c[i][0] && L.c[j][1] == -L.c[i][1] && L.c[j][2] == -L.c[i][2]) L.opp[i] = j;
  return L;
}

// ---------------------------------------------------------------------------
// Product form, Sec. 2.2: Eq. 11, Eq. 12, Eq. 13 and Eq. 14.
// ---------------------------------------------------------------------------
real psi(int c, real xi, real P) {
  if (c == 0) return 1.0 - P;
  if (c == 1) return 0.5 * (xi + P);
  return 0.5 * (-xi + P);
}

void product_form(const Lattice& L, const real* xi, const real* P, real* out) {
  for (int i = 0; i < L.Q; ++i) {
    real v = 1.0;
    for (int a = 0; a < L.D; ++a) v *= psi(L.c[i][a], xi[a], P[a]);
    out[i] = v;
  }
}

// Lattice weights used by the isotropic gradient (reading R9): the textbook
// D2Q9 / D3Q27 weights 4/9,1/9,1/36 and 8/27,2/27,1/54,1/216, i.e. the
// per-axis factors 2/3 (c=0) and 1/6 (c=+-1) multiplied over the axes.
double lattice_weight(const Lattice& L, int i) {
  double w = 1.0;
  for (int a = 0; a < L.D; ++a) w *= (L.c[i][a] == 0) ? (2.0 / 3.0) : (1.0 / 6.0);
  return w;
}

// ---------------------------------------------------------------------------
// Polynomials in one velocity component w, used to apply the operators
// O_alpha of Eq. 50 literally (Sec. 3.3).
// ---------------------------------------------------------------------------
const int PDEG = 10;
struct Poly { real a[PDEG + 1]; };

Poly poly_zero() { Poly p; for (int k = 0; k <= PDEG; ++k) p.a[k] = 0.0; return p; }

// O A = RT dA/dw + w A   (Eq. 50; reading R4: w = u/phi)
Poly poly_apply_O(const Poly& A, real RT) {
  Poly r = poly_zero();
  for (int k = 1; k <= PDEG; ++k) r.a[k - 1] += RT * k * A.a[k];
  for (int k = 0; k < PDEG; ++k) r.a[k + 1] += A.a[k];
  return r;
}

real poly_eval(const Poly& p, real w) {
  real s = 0.0;
  for (int k = PDEG; k >= 0; --k) s = s * w + p.a[k];
  return s;
}

// Psi_c(O, O^2) applied to the one-axis function h(w), evaluated at w:
// c = 0: h - O^2 h ; c = +-1: (+-O h + O^2 h)/2  (Eq. 11..Eq. 13 with
// xi -> O and P -> O^2, as Eq. 51 prescribes).
real psi_operator(int c, const Poly& h, real RT, real w) {
  Poly o1 = poly_apply_O(h, RT);
  Poly o2 = poly_apply_O(o1, RT);
  real h0 = poly_eval(h, w), v1 = poly_eval(o1, w), v2 = poly_eval(o2, w);
  if (c == 0) return h0 - v2;
  if (c == 1) return 0.5 * (v1 + v2);
  return 0.5 * (-v1 + v2);
}

// g^eq_i = phi rho Prod_alpha Psi_{c_i alpha}(O_alpha, O_alpha^2) E   (Eq. 51)
// with the generating function E = U + sum_beta w_beta^2 / 2 (Eq. 40),
// w = u/phi (reading R4).  E is a sum of separable terms (a constant and one
// quadratic per axis); the product of one-axis operators acts on each term
// axis by axis.
void energy_equilibrium(const Lattice& L, real phi, real rho, const real* u, real RT,
                        real U, real* out) {
  real w[3];
  for (int a = 0; a < L.D; ++a) w[a] = u[a] / phi;
  Poly one = poly_zero(); one.a[0] = 1.0;
  Poly half_w2 = poly_zero(); half_w2.a[2] = 0.5;
  for (int i = 0; i < L.Q; ++i) {
    // term U * 1
    real t = U;
    for (int a = 0; a < L.D; ++a) t *= psi_operator(L.c[i][a], one, RT, w[a]);
    real s = t;
    // terms w_beta^2/2
    for (int b = 0; b < L.D; ++b) {
      real tb = 1.0;
      for (int a = 0; a < L.D; ++a)
        tb *= psi_operator(L.c[i][a], (a == b) ? half_w2 : one, RT, w[a]);
      s += tb;
    }
    out[i] = phi * rho * s;
  }
}

// ---------------------------------------------------------------------------
// Householder QR solve of a small dense system, as the paper does for the
// diffusion-velocity system (Sec. 2.3, after Eq. 30).
// A is n x n row-major, b has nrhs columns (b[k*nrhs + r]).
// ---------------------------------------------------------------------------
void householder_qr_solve(int n, const real* Ain, int nrhs, const real* bin, real* x) {
  real A[MMAX * MMAX], B[MMAX * 3];
  for (int k = 0; k < n * n; ++k) A[k] = Ain[k];
  for (int k = 0; k < n * nrhs; ++k) B[k] = bin[k];
  for (int j = 0; j < n; ++j) {
    real norm = 0.0;
    for (int i = j; i < n; ++i) norm += A[i * n + j] * A[i * n + j];
    norm = r_sqrt(norm);
    if (norm == 0.0) continue;
    real alpha = (A[j * n + j] > 0) ? -norm : norm;
    real v[MMAX];
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int i = j; i < n; ++i) v[i] = A[i * n + j];
    v[j] -= alpha;
    real vv = 0.0;
    for (int i = j; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int k = j; k < n; ++k) {
      real s = 0.0;
      for (int i = j; i < n; ++i) s += v[i] * A[i * n + k];
      s = 2.0 * s / vv;
      for (int i = j; i < n; ++i) A[i * n + k] -= s * v[i];
    }
    for (int r = 0; r < nrhs; ++r) {
      real s = 0.0;
      for (int i = j; i < n; ++i) s += v[i] * B[i * nrhs + r];
      s = 2.0 * s / vv;
      for (int i = j; i < n; ++i) B[i * nrhs + r] -= s * v[i];
    }
  }
  for (int r = 0; r < nrhs; ++r)
    for (int i = n - 1; i >= 0; --i) {
      real s = B[i * nrhs + r];
      for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * x[k * nrhs + r];
      x[i * nrhs + r] = s / A[i * n + i];
    }
}

}  // namespace

// ===========================================================================
// Configuration (physical inputs; mirrors oracle/__init__.py's ctypes struct)
// ===========================================================================
extern "C" {

struct oc_config {
  int nx, ny, nz;
  int bc_lo, bc_hi;          // 0 periodic, 1 inlet reservoir, 2 bounce-back
  int M;
  int energy, knudsen;
  int nthreads;              // OpenMP threads (0: default)
  double dx, theta_max, T_scale, T_ref, P_ref;
  double mu_exp, Pr, bulk_ratio, T_thermo, tortuosity, pore_radius;
  const double* molar_mass;  // [M]
  const double* D_ref;       // [M*M]
  const double* mu_ref;      // [M]
  const double* cv_factor;   // [M]
  const double* U0;          // [M]
  const double* porosity;    // [N]
  const double* X_init;      // [M*N]
  const double* T_init;      // [N]
  const double* P_init;      // [N]
  const double* X_in_lo;     // [M]
  const double* X_in_hi;     // [M]
  double T_in_lo, T_in_hi, P_in_lo, P_in_hi;
  // surface mechanism (S == 0: none)
  int S, R;
  const double* nu_gas;      // [R*M]
  const double* nu_surf;     // [R*S]
  const double* A_pre;       // [R]
  const double* Ea;          // [R]
  double gamma, a_s;
  const double* surf_molar_mass;  // [S]
  const double* surf_cv_factor;   // [S]
  const double* surf_U0;          // [S] J/mol
  const double* gas_U0_molar;     // [M] J/mol
  const double* Xs_init;          // [S]
  const double* U_init;           // [3*N] initial velocity [m/s] (null: at rest)
  // electrochemistry (Sec. 4): triple-phase-boundary (edge) steps
  const int* edge;                // [R] 1: the step runs on the TPB edge (null: none)
  const double* n_el;             // [R] electrons produced by the step
  double l_tpb;                   // TPB length per volume of porous medium [1/m^2]
  double beta_ct;                 // charge-transfer symmetry factor
  double resistivity;             // electrolyte resistivity Omega [Ohm m]
  double dphi;                    // Phi_electrode - Phi_electrolyte [V]
};

}  // extern "C"

namespace {

// Per-node macroscopic state of the streamed populations (Sec. 2.1, 3.1).
struct Macro {
  real phi;
  real rho_a[MMAX], j_a[MMAX][3];     // Eq. 4, Eq. 5
  real rho_f, j_f[3], u[3];           // Eq. 37, Eq. 38
  real Pt[3][3];                      // P = sum f c c
  real sum_g, q[3];                   // Eq. 39, q = sum g c
  real rho_s, Y[MMAX], X[MMAX], m_mix, R, T, P;
  real Pi[3];                         // rho u (1 - 3RT) - rho u^3/phi^2 (Eq. 45)
};

struct Oracle {
  oc_config cfg;
  Lattice L;
  int N, M, Q, D, nl;                   // nl = number of lattices
  int energy, knudsen;
  // lattice units
  real dt, cvel;                      // physical time step [s], dx/dt [m/s]
  real RU;                            // R_U in lattice units per kelvin (kg/mol/K)
  real m[MMAX], Dref[MMAX][MMAX], muref[MMAX], cvf[MMAX], U0[MMAX];
  real Pref, d0, tort;                  // d0 = 2 r_p / dx; tortuosity
  real rho_in[2][MMAX], T_in[2];
  // mechanism
  int S, Rn;
  double nu_g[RMAX][MMAX], nu_s[RMAX][SMAX], Ea[RMAX];
  real Apre[RMAX];                  // pre-exponential factors (dual build: seedable)
  real gamma, a_s, ms[SMAX], cvs[SMAX], Us0[SMAX], Ug0[MMAX];
  int edge[RMAX];
  double nel[RMAX], l_tpb, beta_ct, resist, dphi;
  std::vector<double> dphi_node;      // per-node Phi_electrode - Phi_electrolyte (empty: dphi everywhere)
  // state
  std::vector<real> pops, pulled, phi, Tfix, Xs, Xs_new;
  std::vector<Macro> mac;
  // diagnostics of the last collision
  std::vector<real> dg_V, dg_Fk, dg_omega, dg_omega1, dg_T, dg_P, dg_rhodot, dg_kappa, dg_current;
  long steps_done;
  // initial fields (kept to rebuild the initial populations)
  std::vector<double> X0, T0, P0, U0i, Xs_init0;
};

inline size_t PIDX(const Oracle& o, int l, int i, int n) { return ((size_t)l * o.Q + i) * o.N + n; }

void node_coords(const Oracle& o, int n, int& x, int& y, int& z) {
  x = n % o.cfg.nx;
  y = (n / o.cfg.nx) % o.cfg.ny;
  z = n / (o.cfg.nx * o.cfg.ny);
}

int node_index(const Oracle& o, int x, int y, int z) { return x + o.cfg.nx * (y + o.cfg.ny * z); }

int wrap(int v, int n) { return ((v % n) + n) % n; }

// ---------------------------------------------------------------------------
// Thermodynamics (Sec. 2.1 nomenclature, Sec. 3.1 Eq. 33..Eq. 36).
// ---------------------------------------------------------------------------
real R_species(const Oracle& o, int a) { return o.RU / o.m[a]; }            // R_a = R_U / m_a
real U_species(const Oracle& o, int a, real T) {                          // Eq. 33
  return o.U0[a] + o.cvf[a] * R_species(o, a) * (T - o.cfg.T_thermo);
}

// Species equilibrium (Eq. 15), quasi-equilibrium (Eq. 16 with the
// parameterisation Eq. 28) and Knudsen quasi-equilibrium (Eq. 18):
// phi rho_a Prod Psi(xi, P) with the per-axis parameters given.
void species_form(const Oracle& o, real phi, real rho_a, const real* xi, real RaT, real* out) {
  real P[3];
  for (int al = 0; al < o.D; ++al) P[al] = xi[al] * xi[al] + RaT;
  real pf[QMAX];
  product_form(o.L, xi, P, pf);
  for (int i = 0; i < o.Q; ++i) out[i] = phi * rho_a * pf[i];
}

// Macroscopic state from populations at one node (a2 + a3).
void compute_macro(const Oracle& o, const real* fpop /* [nl][Q] */, real phi, real Tfixed, Macro& m) {
  const Lattice& L = o.L;
  m.phi = phi;
  for (int a = 0; a < o.M; ++a) {
    real s = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < o.Q; ++i) {
      real f = fpop[a * o.Q + i];
      s += f;
      for (int al = 0; al < 3; ++al) j[al] += f * L.c[i][al];
    }
    m.rho_a[a] = s / phi;                               // Eq. 4
    for (int al = 0; al < 3; ++al) m.j_a[a][al] = j[al]; // Eq. 5
  }
  {
    const real* f = fpop + o.M * o.Q;
    real s = 0.0, j[3] = {0, 0, 0}, P[3][3] = {{0}};
    for (int i = 0; i < o.Q; ++i) {
      s += f[i];
      for (int al = 0; al < 3; ++al) {
        j[al] += f[i] * L.c[i][al];
        for (int be = 0; be < 3; ++be) P[al][be] += f[i] * L.c[i][al] * L.c[i][be];
      }
    }
    m.rho_f = s / phi;                                  // Eq. 37
    for (int al = 0; al < 3; ++al) { m.j_f[al] = j[al]; m.u[al] = j[al] / m.rho_f; }
    for (int al = 0; al < 3; ++al) for (int be = 0; be < 3; ++be) m.Pt[al][be] = P[al][be];
  }
  m.sum_g = 0.0;
  m.q[0] = m.q[1] = m.q[2] = 0.0;
  if (o.energy) {
    const real* g = fpop + (o.M + 1) * o.Q;
    for (int i = 0; i < o.Q; ++i) {
      m.sum_g += g[i];
      for (int al = 0; al < 3; ++al) m.q[al] += g[i] * L.c[i][al];
    }
  }
  // composition (Sec. 2.1): rho = sum rho_a, Y_a, 1/m = sum Y_a/m_a, X_a
  m.rho_s = 0.0;
  for (int a = 0; a < o.M; ++a) m.rho_s += m.rho_a[a];
  real inv_m = 0.0;
  for (int a = 0; a < o.M; ++a) { m.Y[a] = m.rho_a[a] / m.rho_s; inv_m += m.Y[a] / o.m[a]; }
  m.m_mix = 1.0 / inv_m;
  for (int a = 0; a < o.M; ++a) m.X[a] = m.m_mix * m.Y[a] / o.m[a];
  m.R = o.RU / m.m_mix;                                 // R = R_U / m
  // temperature (Eq. 41 with u^2/(2 phi^2), reading R5; constant C_v)
  if (o.energy) {
    real E = m.sum_g / (phi * m.rho_f);               // Eq. 40 with the momentum lattice's rho (reading R7)
    real w2 = 0.0;
    for (int al = 0; al < o.D; ++al) w2 += (m.u[al] / phi) * (m.u[al] / phi);
    real cv = 0.0, U0m = 0.0;
    for (int a = 0; a < o.M; ++a) {
      cv += m.Y[a] * o.cvf[a] * R_species(o, a);
      U0m += m.Y[a] * o.U0[a];
    }
    // sum_a Y_a [U0_a + Cv_a (T - T_thermo)] = E - w^2/2
    m.T = o.cfg.T_thermo + (E - 0.5 * w2 - U0m) / cv;
  } else {
    m.T = Tfixed;
  }
  m.P = m.rho_f * m.R * m.T;                            // Eq. 3 with rho of Eq. 37 (reading R7)
  for (int al = 0; al < 3; ++al) {
    real w = m.u[al] / phi;
    m.Pi[al] = m.rho_f * m.u[al] * (1.0 - 3.0 * m.R * m.T) - m.rho_f * m.u[al] * w * w;
  }
}

// ---------------------------------------------------------------------------
// Surface source (a10): mass-action kinetics, backward Euler in the reaction
// extents over one time step by Newton iteration (readings R15, R16).
// Returns gas mass production rates rhodot_f[a] (kg/m^3 per lattice time,
// Eq. 68 / Eq. 69) and the new coverages.
// ---------------------------------------------------------------------------
void surface_source(const Oracle& o, const Macro& m, const real* Xs0, real* rhodot_f,
                    real* Xs1, real& dU_fluid_volumetric, real& current, double dphi);

// ---------------------------------------------------------------------------
// One node's collision (a4 .. a9).  fin: streamed populations [nl][Q];
// fout: post-collision populations.  Gradient inputs come from neighbours.
// ---------------------------------------------------------------------------
struct Grad {
  real divu;              // d_beta u_beta
  real dPi[3];            // d_alpha Pi_alpha (no sum)
  real dY[MMAX][3];       // d_alpha Y_a
};

void collide_node(const Oracle& o, int n, const Macro& m, const Grad& gr, const real* fin,
                  real* fout, const real* Xs0, real* Xs1) {
  const Lattice& L = o.L;
  const int M = o.M, Q = o.Q, D = o.D;
  const real phi = m.phi, T = m.T, P = m.P;

  // --- transport coefficients (a4) ----------------------------------------
  // synthetic binary diffusivities (reading R13): D_ab(T,P) = Dref (T/Tref)^1.5 (Pref/P)
  real tau_ab[MMAX][MMAX];
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      if (a == b) { tau_ab[a][b] = 0.0; continue; }
      real Dab = o.Dref[a][b] * r_pow(T / o.cfg.T_ref, 1.5) * (o.Pref / P);
      // Eq. 23 read dimensionally (reading R1): tau_ab = D_ab m_a m_b / (m R_U T)
      tau_ab[a][b] = Dab * o.m[a] * o.m[b] / (m.m_mix * o.RU * T);
    }
  real inv_tau[MMAX], inv_tauk[MMAX], beta[MMAX];
  for (int a = 0; a < M; ++a) {
    real s = 0.0;                                      // Eq. 24
    for (int b = 0; b < M; ++b) if (b != a) s += m.Y[b] / tau_ab[a][b];
    inv_tau[a] = s;
    // Eq. 22: beta = dt/(2 tau + dt), written as (1/tau)/(2 + 1/tau) so that
    // a species with no partner (1/tau = 0) gets beta = 0 (reading R11)
    beta[a] = inv_tau[a] / (2.0 + inv_tau[a]);
    if (o.knudsen) {
      // Knudsen diffusivity (Sec. 5.1): D^k = (phi/tortuosity)(d0/3) sqrt(8 R_U T/(pi m_a))
      real Dk = (phi / o.tort) * (o.d0 / 3.0) * r_sqrt(8.0 * o.RU * T / (PI_D * o.m[a]));
      // Eq. 26 read dimensionally (reading R1): tau^k = D^k m_a / (R_U T)
      real tk = Dk * o.m[a] / (o.RU * T);
      inv_tauk[a] = 1.0 / tk;
    } else {
      inv_tauk[a] = 0.0;
    }
  }

  // --- component velocities and the diffusion-velocity solve (a6) ---------
  real ua[MMAX][3];
  for (int a = 0; a < M; ++a)
    for (int al = 0; al < 3; ++al)
      ua[a][al] = (m.rho_a[a] < 1e-14 * m.rho_s) ? m.u[al] : m.j_a[a][al] / m.rho_a[a];   // R11
  // Eq. 29 with the Knudsen part taken on the component velocity
  // (reading R27): the trapezoidal rule of Sec. 2.3 applied to the Knudsen
  // relaxation (f*_a - f^k_a)/tau^k_a, whose f^k rests (Eq. 18), acts on
  // u + V_a, not on V_a alone, which adds -(dt/2tau^k_a) u to the printed
  // right-hand side (the printed system is the u = 0 case).
  real A[MMAX * MMAX], rhs[MMAX * 3], V[MMAX * 3];
  for (int a = 0; a < M; ++a) {
    for (int b = 0; b < M; ++b) {
      if (a == b) A[a * M + b] = 1.0 + 0.5 * inv_tau[a] + 0.5 * inv_tauk[a];   // Eq. 29
      else A[a * M + b] = -0.5 * m.Y[b] / tau_ab[a][b];
    }
    for (int al = 0; al < 3; ++al)
      rhs[a * 3 + al] = (al < D) ? (ua[a][al] - m.u[al] - 0.5 * inv_tauk[a] * m.u[al]) : 0.0;
  }
  householder_qr_solve(M, A, 3, rhs, V);
  // condition bound (reading R12): ||A||_inf * ||A^-1||_inf <= max row sum / min(1 + dt/2tau^k)
  {
    real amax = 0.0, dmin = 1e300;
    for (int a = 0; a < M; ++a) {
      real rs = 0.0;
      for (int b = 0; b < M; ++b) rs += r_fabs(A[a * M + b]);
      if (rs > amax) amax = rs;
      real d = 1.0 + 0.5 * inv_tauk[a];
      if (d < dmin) dmin = d;
    }
    const_cast<Oracle&>(o).dg_kappa[n] = amax / dmin;
  }
  for (int a = 0; a < M; ++a)
    for (int al = 0; al < 3; ++al) const_cast<Oracle&>(o).dg_V[((size_t)a * 3 + al) * o.N + n] = V[a * 3 + al];

  // --- surface source (a10), zero without a mechanism ----------------------
  real rhodot[MMAX];
  for (int a = 0; a < M; ++a) rhodot[a] = 0.0;
  real dU_src = 0.0;
  real Iv = 0.0;
  // potential difference Phi_electrode - Phi_electrolyte at this node
  const double dphi_n = o.dphi_node.empty() ? o.dphi : o.dphi_node[n];
  if (o.S > 0) surface_source(o, m, Xs0, rhodot, Xs1, dU_src, Iv, dphi_n);
  const_cast<Oracle&>(o).dg_current[n] = Iv;
  for (int a = 0; a < M; ++a) const_cast<Oracle&>(o).dg_rhodot[(size_t)a * o.N + n] = rhodot[a];

  // --- species collision (a7): Eq. 21 ----------
  real feq[MMAX][QMAX], fst[MMAX][QMAX], fk[MMAX][QMAX], fr[MMAX][QMAX];
  for (int a = 0; a < M; ++a) {
    real RaT = R_species(o, a) * T;
    real xi_eq[3], xi_st[3], xi_k[3] = {0, 0, 0};
    for (int al = 0; al < 3; ++al) {
      xi_eq[al] = m.u[al] / phi;                         // Eq. 15
      xi_st[al] = (m.u[al] + V[a * 3 + al]) / phi;       // Eq. 28 with phi (reading R2)
    }
    species_form(o, phi, m.rho_a[a], xi_eq, RaT, feq[a]);
    species_form(o, phi, m.rho_a[a], xi_st, RaT, fst[a]);
    species_form(o, phi, m.rho_a[a], xi_k, RaT, fk[a]);  // Eq. 18
    // reaction source populations (Eq. 89): rhodot Prod Psi(u/phi, ...)
    real pf[QMAX], Pp[3];
    for (int al = 0; al < D; ++al) Pp[al] = xi_eq[al] * xi_eq[al] + RaT;
    product_form(L, xi_eq, Pp, pf);
    for (int i = 0; i < Q; ++i) fr[a][i] = rhodot[a] * pf[i];
  }
  for (int a = 0; a < M; ++a) {
    for (int i = 0; i < Q; ++i) {
      real F = 0.0;                                    // Eq. 25
      for (int b = 0; b < M; ++b) if (b != a) F += (1.0 / tau_ab[a][b]) * (feq[b][i] - fst[b][i]);
      F *= m.Y[a];
      F += inv_tauk[a] * (fst[a][i] - fk[a][i]);
      real f = fin[a * Q + i];
      // R^r ~ fdot^r dt (Eq. 32), dt = 1
      fout[a * Q + i] = f + 2.0 * beta[a] * (feq[a][i] - f) + (beta[a] - 1.0) * F + fr[a][i];
    }
  }

  // --- momentum lattice (a8): Eq. 42 / Eq. 87 ---------------------------
  // net Knudsen force Eq. 48 with P X_b / D^k_b = rho_b / tau^k_b
  // and the component velocity u_b = u* + (V_b - Vbar) (reading R8): the
  // mixture velocity plus the diffusion velocity taken relative to the
  // species' mass average Vbar = sum_c Y_c V_c, whose mass-weighted sum
  // vanishes as Eq. 6 requires.  The mixture velocity u* is the
  // momentum lattice's, at the middle of the step (u* = u + dt F^k/(2 rho)):
  // the trapezoidal rule of Sec. 2.3 applied to the drag of the mixture, so
  //   F^k = -sum_b rho_b (u + V_b - Vbar)/tau^k_b / (1 + (dt/2) sum_b (rho_b/rho)/tau^k_b).
  real Fk[3] = {0, 0, 0};
  real kdrag = 0.0;
  for (int b = 0; b < M; ++b) kdrag += (m.rho_a[b] / m.rho_f) * inv_tauk[b];
  for (int al = 0; al < D; ++al) {
    real Vbar = 0.0;
    for (int c = 0; c < M; ++c) Vbar += m.Y[c] * V[c * 3 + al];
    for (int b = 0; b < M; ++b) Fk[al] -= m.rho_a[b] * (m.u[al] + V[b * 3 + al] - Vbar) * inv_tauk[b];
    Fk[al] /= 1.0 + 0.5 * kdrag;
  }
  for (int al = 0; al < 3; ++al) const_cast<Oracle&>(o).dg_Fk[(size_t)al * o.N + n] = Fk[al];
  // viscosity (reading R13): mu = sum_a X_a mu_a(T), mu_a = mu_ref,a (T/Tref)^mu_exp
  real mu = 0.0;
  for (int a = 0; a < M; ++a) mu += m.X[a] * o.muref[a] * r_pow(T / o.cfg.T_ref, o.cfg.mu_exp);
  real omega = 1.0 / (0.5 + mu / P);                   // Eq. 65 with dt = 1
  real omega1 = 1.0 / (0.5 + mu / (o.cfg.Pr * P));     // Eq. 67 with lambda = mu C_p / Pr
  real vs = o.cfg.bulk_ratio * mu;                      // bulk viscosity
  const_cast<Oracle&>(o).dg_omega[n] = omega;
  const_cast<Oracle&>(o).dg_omega1[n] = omega1;
  real cv_mix = 0.0;
  for (int a = 0; a < M; ++a) cv_mix += m.Y[a] * o.cvf[a] * R_species(o, a);
  // bulk-viscosity bracket of Eq. 45; isothermal lattices have no energy
  // equation, so the R/C_v part (from dT/dt) is absent there.
  real bulk = -vs + mu * (2.0 / D - (o.energy ? m.R / cv_mix : 0.0));
  real uex[3], xi_ex[3], Pex[3];
  for (int al = 0; al < 3; ++al) uex[al] = m.u[al] + Fk[al] / (omega * m.rho_f);   // reading R3
  for (int al = 0; al < D; ++al) {
    real Peq = m.R * T + (m.u[al] / phi) * (m.u[al] / phi);                      // Eq. 47
    Pex[al] = Peq + bulk * gr.divu / (phi * m.rho_f)
              + ((2.0 - omega) / (2.0 * phi * m.rho_f * omega)) * gr.dPi[al];      // Eq. 45
    xi_ex[al] = uex[al] / phi;
  }
  real pfx[QMAX];
  product_form(L, xi_ex, Pex, pfx);
  // post-collision mixture density (Eq. 78): phi rho_pc = phi rho + sum rhodot dt
  real sum_rd = 0.0;
  for (int a = 0; a < M; ++a) sum_rd += rhodot[a];
  real rho_pc = m.rho_f + sum_rd / phi;
  for (int i = 0; i < Q; ++i) {
    real fex = phi * m.rho_f * pfx[i];                                          // Eq. 44
    real f = fin[M * Q + i];
    fout[M * Q + i] = f + omega * (fex - f) + (rho_pc / m.rho_f * fex - fex);     // Eq. 87
  }

  // --- energy lattice (a9): Eq. 43 / Eq. 88 -----------------------------
  if (o.energy) {
    real U = 0.0, H = 0.0, Ha[MMAX];
    for (int a = 0; a < M; ++a) {
      real Ua = U_species(o, a, T);
      Ha[a] = Ua + R_species(o, a) * T;                  // H_a = U_a + R_a T (Mayer)
      U += m.Y[a] * Ua;                                  // Eq. 35
      H += m.Y[a] * Ha[a];                               // Eq. 36
    }
    real geq[QMAX];
    energy_equilibrium(L, phi, m.rho_f, m.u, m.R * T, U, geq);
    real w2 = 0.0;
    for (int al = 0; al < D; ++al) w2 += (m.u[al] / phi) * (m.u[al] / phi);
    real qeq[3] = {0, 0, 0};
    for (int al = 0; al < D; ++al) qeq[al] = (H + 0.5 * w2) * m.rho_f * m.u[al];   // Eq. 52
    // equilibrium pressure tensor of the momentum lattice (Eq. 49, reading R6)
    real Peq[3][3];
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be)
        Peq[al][be] = phi * m.rho_f * (m.u[al] / phi) * (m.u[be] / phi) + (al == be ? phi * m.rho_f * m.R * T : 0.0);
    real qdiff[3] = {0, 0, 0}, qcorr[3] = {0, 0, 0}, qex[3] = {0, 0, 0}, qst[3] = {0, 0, 0};
    for (int al = 0; al < D; ++al) {
      // diffusion velocities relative to the mass average: Eq. 6 with
      // u_a = u + V_a implies sum_a rho_a V_a = 0, which the discrete system
      // Eq. 29 satisfies only up to the weak-coupling drift (reading R22)
      real Vbar = 0.0;
      for (int a = 0; a < M; ++a) Vbar += m.Y[a] * V[a * 3 + al];
      real sV = 0.0, sdY = 0.0;
      for (int a = 0; a < M; ++a) { sV += Ha[a] * m.Y[a] * (V[a * 3 + al] - Vbar); sdY += Ha[a] * gr.dY[a][al]; }
      qdiff[al] = (omega1 / (omega - omega1)) * m.rho_f * sV;                      // Eq. 58
      qcorr[al] = 0.5 * ((omega1 - 2.0) / (omega1 - omega)) * P * phi * sdY;        // Eq. 59
      qex[al] = m.u[al] * (omega / (omega - omega1)) * bulk * gr.divu / phi
                - 0.5 * (m.u[al] / phi) * gr.dPi[al];                                // Eq. 60
      real uP = 0.0;
      for (int be = 0; be < D; ++be) uP += (m.u[be] / phi) * (m.Pt[al][be] - Peq[al][be]);
      qst[al] = m.q[al] - uP + qdiff[al] + qcorr[al] + qex[al];                     // Eq. 55
    }
    // source distribution (Eq. 86): same equilibrium with the
    // post-reaction density and internal energy (zero change without reactions)
    real gsrc[QMAX];
    bool have_src = (o.S > 0);
    if (have_src) {
      real U_pc = (phi * m.rho_f * U + dU_src) / (phi * rho_pc);
      energy_equilibrium(L, phi, rho_pc, m.u, m.R * T, U_pc, gsrc);
    }
    const real* g = fin + (M + 1) * Q;
    for (int i = 0; i < Q; ++i) {
      int c2 = 0;
      for (int al = 0; al < D; ++al) c2 += L.c[i][al] * L.c[i][al];
      real gst = geq[i];                                                           // Eq. 54
      if (c2 == 1)
        for (int al = 0; al < D; ++al) gst += 0.5 * L.c[i][al] * (qst[al] - qeq[al]);
      real src = have_src ? (gsrc[i] - geq[i]) : 0.0;
      fout[(M + 1) * Q + i] = g[i] + omega1 * (geq[i] - g[i]) + (omega - omega1) * (gst - g[i]) + src;
    }
  }
}

// ---------------------------------------------------------------------------
// Inlet reservoir ghost populations (reading R10): equilibria at the
// prescribed composition, pressure and temperature, moving with the velocity
// of the adjacent interior node of the same step.
// ---------------------------------------------------------------------------
void inlet_ghost(const Oracle& o, int side, real phi, const real* u, real* ghost /* [nl][Q] */) {
  const int M = o.M, Q = o.Q;
  real T = o.T_in[side];
  real rho = 0.0;
  for (int a = 0; a < M; ++a) rho += o.rho_in[side][a];
  real inv_m = 0.0;
  for (int a = 0; a < M; ++a) inv_m += (o.rho_in[side][a] / rho) / o.m[a];
  real R = o.RU * inv_m;
  real xi[3];
  for (int al = 0; al < 3; ++al) xi[al] = u[al] / phi;
  for (int a = 0; a < M; ++a) species_form(o, phi, o.rho_in[side][a], xi, R_species(o, a) * T, ghost + a * Q);
  species_form(o, phi, rho, xi, R * T, ghost + M * Q);
  if (o.energy) {
    real U = 0.0;
    for (int a = 0; a < M; ++a) U += (o.rho_in[side][a] / rho) * U_species(o, a, T);
    energy_equilibrium(o.L, phi, rho, u, R * T, U, ghost + (M + 1) * Q);
  }
}

// Pull streaming (a1) with boundary conditions into o.pulled.
void stream(Oracle& o) {
  const Lattice& L = o.L;
  const int nx = o.cfg.nx, ny = o.cfg.ny, nz = o.cfg.nz, Q = o.Q, nl = o.nl;
  std::vector<char> missing((size_t)Q * o.N, 0);
#pragma omp parallel for schedule(static)
  for (int n = 0; n < o.N; ++n) {
    int x, y, z;
    node_coords(o, n, x, y, z);
    for (int i = 0; i < Q; ++i) {
      int sx = x - L.c[i][0], sy = wrap(y - L.c[i][1], ny), sz = wrap(z - L.c[i][2], nz);
      int side = -1;
      if (sx < 0) { if (o.cfg.bc_lo == 0) sx = wrap(sx, nx); else side = 0; }
      if (sx >= nx) { if (o.cfg.bc_hi == 0) sx = wrap(sx, nx); else side = 1; }
      if (side < 0) {
        int s = node_index(o, sx, sy, sz);
        for (int l = 0; l < nl; ++l) o.pulled[PIDX(o, l, i, n)] = o.pops[PIDX(o, l, i, s)];
      } else {
        int bc = (side == 0) ? o.cfg.bc_lo : o.cfg.bc_hi;
        if (bc == 2) {   // bounce-back: the node's own opposite post-collision population
          for (int l = 0; l < nl; ++l) o.pulled[PIDX(o, l, i, n)] = o.pops[PIDX(o, l, L.opp[i], n)];
        } else {
          missing[(size_t)i * o.N + n] = 1;
        }
      }
    }
  }
  // inlet ghosts need the adjacent interior node's velocity (its sources are all inside)
  for (int side = 0; side < 2; ++side) {
    int bc = side == 0 ? o.cfg.bc_lo : o.cfg.bc_hi;
    if (bc != 1) continue;
    int xb = side == 0 ? 0 : nx - 1;
    int xa = side == 0 ? 1 : nx - 2;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y) {
        int nb = node_index(o, xb, y, z), na = node_index(o, xa, y, z);
        real js = 0.0, jf[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          real f = o.pulled[PIDX(o, o.M, i, na)];
          js += f;
          for (int al = 0; al < 3; ++al) jf[al] += f * L.c[i][al];
        }
        real rho_f = js / o.phi[na];
        real u[3] = {jf[0] / rho_f, jf[1] / rho_f, jf[2] / rho_f};
        real ghost[(MMAX + 2) * QMAX];
        inlet_ghost(o, side, o.phi[nb], u, ghost);
        for (int i = 0; i < Q; ++i)
          if (missing[(size_t)i * o.N + nb])
            for (int l = 0; l < nl; ++l) o.pulled[PIDX(o, l, i, nb)] = ghost[l * Q + i];
      }
  }
}

void compute_all_macro(Oracle& o) {
#pragma omp parallel for schedule(static)
  for (int n = 0; n < o.N; ++n) {
    real f[(MMAX + 2) * QMAX];
    for (int l = 0; l < o.nl; ++l)
      for (int i = 0; i < o.Q; ++i) f[l * o.Q + i] = o.pulled[PIDX(o, l, i, n)];
    compute_macro(o, f, o.phi[n], o.Tfix[n], o.mac[n]);
  }
}

// Isotropic lattice gradient (Sec. 3.3 after Eq. 60; reading R9):
// d_alpha A(x) = (1/c_s^2) sum_i w_i c_i,alpha A(x + c_i), c_s^2 = 1/3.
// Outside a non-periodic x face the neighbour value is the boundary node's
// own value (zero-gradient ghost, reading R10).
void gradients(const Oracle& o, int n, Grad& gr) {
  const Lattice& L = o.L;
  int x, y, z;
  node_coords(o, n, x, y, z);
  gr.divu = 0.0;
  for (int al = 0; al < 3; ++al) gr.dPi[al] = 0.0;
  for (int a = 0; a < MMAX; ++a) for (int al = 0; al < 3; ++al) gr.dY[a][al] = 0.0;
  for (int i = 0; i < L.Q; ++i) {
    int sx = x + L.c[i][0];
    if (sx < 0) sx = (o.cfg.bc_lo == 0) ? wrap(sx, o.cfg.nx) : 0;
    if (sx >= o.cfg.nx) sx = (o.cfg.bc_hi == 0) ? wrap(sx, o.cfg.nx) : o.cfg.nx - 1;
    int sy = wrap(y + L.c[i][1], o.cfg.ny), sz = wrap(z + L.c[i][2], o.cfg.nz);
    const Macro& mn = o.mac[node_index(o, sx, sy, sz)];
    real w = 3.0 * lattice_weight(L, i);
    for (int al = 0; al < L.D; ++al) {
      if (L.c[i][al] == 0) continue;
      gr.divu += w * L.c[i][al] * mn.u[al];
      gr.dPi[al] += w * L.c[i][al] * mn.Pi[al];
      for (int a = 0; a < o.M; ++a) gr.dY[a][al] += w * L.c[i][al] * mn.Y[a];
    }
  }
}

// ---------------------------------------------------------------------------
// Surface chemistry.
// ---------------------------------------------------------------------------
// Rates of progress r_k [mol m^-2 s^-1] by mass action with Arrhenius
// constants k = A exp(-Ea/(R_U T)) (reading R15).  c_gas in mol/m^3 (fluid),
// theta = surface concentration Gamma X^(s) in mol/m^2.
// Edge (triple-phase-boundary) steps, Sec. 4: their rates are per unit TPB
// length [mol m^-1 s^-1], and a step that releases n electrons has its
// constant raised by exp(beta n F (Phi_electrode - Phi_electrolyte)/(R_U T))
// (charge transfer with symmetry factor beta; reading R29).
const double FARADAY = 96485.33212;     // C/mol

void mass_action_rates(const Oracle& o, real T, const real* cg, const real* cs, real* r, double dphi) {
  for (int k = 0; k < o.Rn; ++k) {
    real kr = o.Apre[k] * r_exp(-o.Ea[k] / (R_UNIV * T));
    if (o.edge[k]) kr *= r_exp(o.beta_ct * o.nel[k] * FARADAY * dphi / (R_UNIV * T));
    real v = kr;
    for (int a = 0; a < o.M; ++a)
      if (o.nu_g[k][a] < 0) v *= r_pow(rmax(cg[a], 0.0), -o.nu_g[k][a]);
    for (int s = 0; s < o.S; ++s)
      if (o.nu_s[k][s] < 0) v *= r_pow(rmax(cs[s], 0.0), -o.nu_s[k][s]);
    r[k] = v;
  }
}

// Backward Euler in the extents xi_k [mol/m^2] over the physical step dt:
// xi = dt * r(c_gas0 + (a_s/phi) nu_g^T xi, theta0 + nu_s^T xi), solved by
// Newton with a finite-difference-free analytic Jacobian of mass action.
void surface_source(const Oracle& o, const Macro& m, const real* Xs0, real* rhodot_f,
                    real* Xs1, real& dU_fluid_volumetric, real& current, double dphi) {
  const int M = o.M, S = o.S, Rn = o.Rn;
  const real T = m.T;
  const real dtp = o.dt;                        // physical seconds
  real cg0[MMAX], cs0[SMAX];
  for (int a = 0; a < M; ++a) cg0[a] = m.rho_a[a] / o.m[a];                 // mol/m^3 of fluid
  for (int s = 0; s < S; ++s) cs0[s] = o.gamma * Xs0[s];                    // Eq. 70
  real xi[RMAX];
  for (int k = 0; k < Rn; ++k) xi[k] = 0.0;
  real scale = o.a_s / m.phi;                   // surface area per fluid volume
  // surface concentration change per extent: 1 for a surface step, l_TPB/a^(s)
  // for an edge step (Eq. 71), whose extent is per TPB length
  real es[RMAX];
  for (int k = 0; k < Rn; ++k) es[k] = o.edge[k] ? o.l_tpb / o.a_s : 1.0;
  for (int it = 0; it < 30; ++it) {
    real cg[MMAX], cs[SMAX];
    for (int a = 0; a < M; ++a) { cg[a] = cg0[a]; for (int k = 0; k < Rn; ++k) cg[a] += scale * o.nu_g[k][a] * xi[k]; }
    for (int s = 0; s < S; ++s) { cs[s] = cs0[s]; for (int k = 0; k < Rn; ++k) cs[s] += o.nu_s[k][s] * es[k] * xi[k]; }
    real r[RMAX];
    mass_action_rates(o, T, cg, cs, r, dphi);
    real Fv[RMAX], J[RMAX * RMAX];
    for (int k = 0; k < Rn; ++k) Fv[k] = xi[k] - dtp * r[k];
    // Jacobian: dF_k/dxi_l = delta_kl - dt * dr_k/dxi_l
    for (int k = 0; k < Rn; ++k)
      for (int l = 0; l < Rn; ++l) {
        real d = 0.0;
        for (int a = 0; a < M; ++a)
          if (o.nu_g[k][a] < 0 && cg[a] > 0) d += r[k] * (-o.nu_g[k][a]) / cg[a] * scale * o.nu_g[l][a];
        for (int s = 0; s < S; ++s)
          if (o.nu_s[k][s] < 0 && cs[s] > 0) d += r[k] * (-o.nu_s[k][s]) / cs[s] * o.nu_s[l][s] * es[l];
        J[k * Rn + l] = (k == l ? 1.0 : 0.0) - dtp * d;
      }
    // Gaussian elimination with partial pivoting on J dxi = -F
    real Ab[RMAX * (RMAX + 1)];
    for (int k = 0; k < Rn; ++k) {
      for (int l = 0; l < Rn; ++l) Ab[k * (Rn + 1) + l] = J[k * Rn + l];
      Ab[k * (Rn + 1) + Rn] = -Fv[k];
    }
    for (int c = 0; c < Rn; ++c) {
      int p = c;
      for (int k = c + 1; k < Rn; ++k) if (r_fabs(Ab[k * (Rn + 1) + c]) > r_fabs(Ab[p * (Rn + 1) + c])) p = k;
      if (p != c) for (int l = 0; l <= Rn; ++l) std::swap(Ab[c * (Rn + 1) + l], Ab[p * (Rn + 1) + l]);
      for (int k = c + 1; k < Rn; ++k) {
        real f = Ab[k * (Rn + 1) + c] / Ab[c * (Rn + 1) + c];
        for (int l = c; l <= Rn; ++l) Ab[k * (Rn + 1) + l] -= f * Ab[c * (Rn + 1) + l];
      }
    }
    real dxi[RMAX];
    for (int k = Rn - 1; k >= 0; --k) {
      real s = Ab[k * (Rn + 1) + Rn];
      for (int l = k + 1; l < Rn; ++l) s -= Ab[k * (Rn + 1) + l] * dxi[l];
      dxi[k] = s / Ab[k * (Rn + 1) + k];
    }
    // positivity-preserving damping: the backward-Euler solution of mass
    // action keeps every concentration >= 0, so a Newton step that would take
    // a non-negative concentration below zero is shortened (to 9/10 of the
    // distance to zero)
    real alpha = 1.0;
    for (int a = 0; a < M; ++a) {
      real d = 0.0;
      for (int k = 0; k < Rn; ++k) d += scale * o.nu_g[k][a] * dxi[k];
      if (cg[a] >= 0.0 && cg[a] + d < 0.0) alpha = rmin(alpha, 0.9 * cg[a] / (-d));
    }
    for (int s = 0; s < S; ++s) {
      real d = 0.0;
      for (int k = 0; k < Rn; ++k) d += o.nu_s[k][s] * es[k] * dxi[k];
      if (cs[s] >= 0.0 && cs[s] + d < 0.0) alpha = rmin(alpha, 0.9 * cs[s] / (-d));
    }
    real dmax = 0.0, xmax = 0.0;
    for (int k = 0; k < Rn; ++k) {
      xi[k] += alpha * dxi[k];
      dmax = rmax(dmax, r_fabs(alpha * dxi[k]));
      xmax = rmax(xmax, r_fabs(xi[k]));
    }
    if (alpha == 1.0 && dmax <= 1e-14 * (xmax + 1e-300)) break;
  }
  // gas production per unit volume of porous medium over dt (Eq. 68,
  // Eq. 69), converted to kg/m^3 per lattice time step
  for (int a = 0; a < M; ++a) {
    real dn = 0.0;
    for (int k = 0; k < Rn; ++k) dn += o.nu_g[k][a] * xi[k];
    rhodot_f[a] = o.a_s * o.m[a] * dn;            // [kg/m^3 of REV] per step
  }
  for (int s = 0; s < S; ++s) {
    real dn = 0.0;
    for (int k = 0; k < Rn; ++k) dn += o.nu_s[k][s] * es[k] * xi[k];
    Xs1[s] = Xs0[s] + dn / o.gamma;               // Eq. 71 (surface and edge terms)
  }
  // volumetric current (Eq. 74): I = F l_TPB (electrons per TPB length per second)
  real ne = 0.0;
  for (int k = 0; k < Rn; ++k)
    if (o.edge[k]) ne += o.nel[k] * xi[k];
  current = FARADAY * o.l_tpb * ne / dtp;         // A per m^3 of porous medium
  // Unified internal energy (Eq. 80, Eq. 85): at
  // fixed temperature the fluid gains what the adsorbed phase loses; molar
  // internal energies U_s(T) = U0_s + cv_s R_U (T - T_thermo).
  real dUs = 0.0;
  for (int s = 0; s < S; ++s) {
    real Us = o.Us0[s] + o.cvs[s] * R_UNIV * (T - o.cfg.T_thermo);
    real dn = 0.0;
    for (int k = 0; k < Rn; ++k) dn += o.nu_s[k][s] * es[k] * xi[k];
    dUs += o.a_s * dn * Us;                       // J/m^3 of REV
  }
  // electric power leaves, ohmic heat stays (Sec. 4.2, reading R28):
  // P_elec = |Phi_electrode - Phi_electrolyte| I, P_Omega = (a^(s)/l_TPB) I^2 Omega dx,
  // source over the step (P_Omega - P_elec) dt
  real U_source = 0.0;
  if (o.l_tpb > 0.0) {
    const real P_elec = std::fabs(dphi) * current;
    const real P_ohm = (o.a_s / o.l_tpb) * current * current * o.resist * o.cfg.dx;
    U_source = (P_ohm - P_elec) * dtp;
  }
  dU_fluid_volumetric = (-dUs + U_source) / (o.cvel * o.cvel); // lattice energy units (J/kg -> (dx/dt)^2)
}

}  // namespace

// ===========================================================================
// C API used by oracle/__init__.py
// ===========================================================================
namespace {

// Initial populations: equilibria of the initial macroscopic fields.
void init_populations(Oracle* o) {
  const int N = o->N;
  for (int n = 0; n < N; ++n) {
    real T = o->T0[n], P = o->P0[n], ph = o->phi[n];
    real rho_a[MMAX], rho = 0.0;
    for (int a = 0; a < o->M; ++a) {
      rho_a[a] = P * o->X0[(size_t)a * N + n] * o->m[a] / (R_UNIV * T);
      rho += rho_a[a];
    }
    real inv_m = 0.0;
    for (int a = 0; a < o->M; ++a) inv_m += (rho_a[a] / rho) / o->m[a];
    real R = o->RU * inv_m;
    real u[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
    if (!o->U0i.empty())
      for (int al = 0; al < o->D; ++al) u[al] = o->U0i[(size_t)al * N + n] / o->cvel;
    for (int al = 0; al < 3; ++al) xi[al] = u[al] / ph;
    real f[QMAX];
    for (int a = 0; a < o->M; ++a) {
      species_form(*o, ph, rho_a[a], xi, R_species(*o, a) * T, f);
      for (int i = 0; i < o->Q; ++i) o->pops[PIDX(*o, a, i, n)] = stored(f[i]);
    }
    species_form(*o, ph, rho, xi, R * T, f);
    for (int i = 0; i < o->Q; ++i) o->pops[PIDX(*o, o->M, i, n)] = stored(f[i]);
    if (o->energy) {
      real U = 0.0;
      for (int a = 0; a < o->M; ++a) U += (rho_a[a] / rho) * U_species(*o, a, T);
      energy_equilibrium(o->L, ph, rho, u, R * T, U, f);
      for (int i = 0; i < o->Q; ++i) o->pops[PIDX(*o, o->M + 1, i, n)] = stored(f[i]);
    }
  }
}

// One node's collision with its gradients, from the streamed populations.
void collide_at(Oracle* o, int n, real* fout) {
  Grad gr;
  gradients(*o, n, gr);
  real fin[(MMAX + 2) * QMAX];
  for (int l = 0; l < o->nl; ++l)
    for (int i = 0; i < o->Q; ++i) fin[l * o->Q + i] = o->pulled[PIDX(*o, l, i, n)];
  real xs0[SMAX], xs1[SMAX];
  for (int s = 0; s < o->S; ++s) xs0[s] = o->Xs[(size_t)s * o->N + n];
  collide_node(*o, n, o->mac[n], gr, fin, fout, xs0, xs1);
  for (int s = 0; s < o->S; ++s) o->Xs_new[(size_t)s * o->N + n] = xs1[s];
}

// Macroscopic fields of the current state (value, or derivative `lane`).
void moments_lane(Oracle* o, int which, int lane, double* out) {
  const int N = o->N, M = o->M, D = o->D;
  if (which == 8) {
    for (size_t k = 0; k < (size_t)o->S * N; ++k) out[k] = comp(o->Xs[k], lane);
    return;
  }
  stream(*o);
  compute_all_macro(*o);
  if (which == 6 || which == 7 || which == 10) {
    // the diffusion velocities and the current need the collision's transport
    // coefficients and surface source;
    // run the collision into a scratch buffer and read its diagnostics
    std::vector<real> keep_xs = o->Xs_new;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; ++n) {
      real fout[(MMAX + 2) * QMAX];
      collide_at(o, n, fout);
    }
    o->Xs_new = keep_xs;
  }
  for (int n = 0; n < N; ++n) {
    const Macro& m = o->mac[n];
    switch (which) {
      case 0: for (int a = 0; a < M; ++a) out[(size_t)a * N + n] = comp(m.rho_a[a], lane); break;
      case 1: for (int a = 0; a < M; ++a) for (int al = 0; al < D; ++al)
                out[((size_t)a * D + al) * N + n] = comp(m.j_a[a][al], lane); break;
      case 2: out[n] = comp(m.rho_f, lane); break;
      case 3: for (int al = 0; al < D; ++al) out[(size_t)al * N + n] = comp(m.u[al], lane); break;
      case 4: out[n] = comp(m.T, lane); break;
      case 5: out[n] = comp(m.P * o->cvel * o->cvel, lane); break;
      case 6: for (int a = 0; a < M; ++a) for (int al = 0; al < D; ++al)
                out[((size_t)a * D + al) * N + n] = comp(o->dg_V[((size_t)a * 3 + al) * N + n], lane); break;
      case 7: for (int a = 0; a < M; ++a) for (int al = 0; al < D; ++al)
                out[((size_t)a * D + al) * N + n] =
                    comp(m.rho_a[a] * (m.u[al] + o->dg_V[((size_t)a * 3 + al) * N + n]) * o->cvel / o->m[a], lane);
              break;
      case 9: out[n] = comp(m.rho_s, lane); break;
      case 10: out[n] = comp(o->dg_current[n], lane); break;
      default: break;
    }
  }
}

}  // namespace

extern "C" {

void* oc_create(const oc_config* c) {
  if (c->M < 1 || c->M > MMAX) return nullptr;
  if (c->S > SMAX || c->R > RMAX) return nullptr;
  Oracle* o = new Oracle();
  o->cfg = *c;
  o->D = (c->nz > 1) ? 3 : 2;
  o->L = make_lattice(o->D);
  o->Q = o->L.Q;
  o->M = c->M;
  o->N = c->nx * c->ny * c->nz;
  o->energy = c->energy;
  o->knudsen = c->knudsen;
  o->nl = c->M + 1 + (c->energy ? 1 : 0);
#ifdef _OPENMP
  if (c->nthreads > 0) omp_set_num_threads(c->nthreads);
#endif
  // lattice scaling (reading R14): max_a R_a T_scale dt^2/dx^2 = theta_max
  double mmin = 1e300;
  for (int a = 0; a < o->M; ++a) mmin = rmin(mmin, c->molar_mass[a]);
  const double dt = c->dx * std::sqrt(c->theta_max * mmin / (R_UNIV * c->T_scale));
  const double cvel = c->dx / dt;
  const double c2 = cvel * cvel;
  o->dt = dt;
  o->cvel = cvel;
  o->RU = R_UNIV / c2;
  for (int a = 0; a < o->M; ++a) {
    o->m[a] = c->molar_mass[a];
    o->muref[a] = c->mu_ref[a] / (cvel * c->dx);          // mu dt/dx^2
    o->cvf[a] = c->cv_factor[a];
    o->U0[a] = c->U0[a] / c2;
    for (int b = 0; b < o->M; ++b) o->Dref[a][b] = c->D_ref[a * o->M + b] / (cvel * c->dx);
  }
  o->Pref = c->P_ref / c2;
  o->d0 = 2.0 * c->pore_radius / c->dx;
  o->tort = c->tortuosity;
  const double* Xin[2] = {c->X_in_lo, c->X_in_hi};
  double Tin[2] = {c->T_in_lo, c->T_in_hi}, Pin[2] = {c->P_in_lo, c->P_in_hi};
  for (int s = 0; s < 2; ++s) {
    o->T_in[s] = Tin[s];
    // rho_a = P X_a m_a / (R_U T)  (Dalton + ideal gas, Sec. 2.1), kg/m^3
    for (int a = 0; a < o->M; ++a) o->rho_in[s][a] = Pin[s] * Xin[s][a] * c->molar_mass[a] / (R_UNIV * Tin[s]);
  }
  o->S = c->S;
  o->Rn = c->R;
  if (o->S > 0) {
    for (int k = 0; k < o->Rn; ++k) {
      for (int a = 0; a < o->M; ++a) o->nu_g[k][a] = c->nu_gas[k * o->M + a];
      for (int s = 0; s < o->S; ++s) o->nu_s[k][s] = c->nu_surf[k * o->S + s];
      o->Apre[k] = c->A_pre[k];
      o->Ea[k] = c->Ea[k];
      o->edge[k] = c->edge ? c->edge[k] : 0;
      o->nel[k] = c->n_el ? c->n_el[k] : 0.0;
    }
    o->l_tpb = c->l_tpb;
    o->beta_ct = c->beta_ct;
    o->resist = c->resistivity;
    o->dphi = c->dphi;
    o->gamma = c->gamma;
    o->a_s = c->a_s;
    for (int s = 0; s < o->S; ++s) {
      o->ms[s] = c->surf_molar_mass[s];
      o->cvs[s] = c->surf_cv_factor[s];
      o->Us0[s] = c->surf_U0[s];
    }
    for (int a = 0; a < o->M; ++a) o->Ug0[a] = c->gas_U0_molar[a];
  }
  const size_t N = o->N;
  size_t NP = (size_t)o->nl * o->Q * N;
  o->pops.assign(NP, 0.0);
  o->pulled.assign(NP, 0.0);
  o->phi.assign(c->porosity, c->porosity + N);
  o->Tfix.assign(c->T_init, c->T_init + N);
  o->mac.resize(N);
  o->dg_V.assign((size_t)MMAX * 3 * N, 0.0);
  o->dg_Fk.assign((size_t)3 * N, 0.0);
  o->dg_omega.assign(N, 0.0);
  o->dg_omega1.assign(N, 0.0);
  o->dg_kappa.assign(N, 0.0);
  o->dg_rhodot.assign((size_t)MMAX * N, 0.0);
  o->dg_current.assign(N, 0.0);
  if (o->S > 0) {
    o->Xs.assign((size_t)o->S * N, 0.0);
    for (int s = 0; s < o->S; ++s)
      for (size_t n = 0; n < N; ++n) o->Xs[(size_t)s * N + n] = c->Xs_init[s];
    o->Xs_new = o->Xs;
  }
  if (o->S > 0) o->Xs_init0.assign(c->Xs_init, c->Xs_init + o->S);
  o->X0.assign(c->X_init, c->X_init + (size_t)o->M * N);
  o->T0.assign(c->T_init, c->T_init + N);
  o->P0.assign(c->P_init, c->P_init + N);
  if (c->U_init) o->U0i.assign(c->U_init, c->U_init + (size_t)3 * N);
  init_populations(o);
  o->steps_done = 0;
  return o;
}

void oc_destroy(void* h) { delete (Oracle*)h; }

int oc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Number of derivative lanes of this build (0: the plain FP64 build).
int oc_lanes(void) {
#ifdef ORACLE_DUAL
  return NT;
#else
  return 0;
#endif
}

void oc_info(void* h, double* out) {
  Oracle* o = (Oracle*)h;
  out[0] = comp(o->dt, -1);
  out[1] = comp(o->cvel, -1);
  out[2] = comp(o->RU, -1);
  out[3] = o->nl;
  out[4] = o->Q;
  out[5] = o->D;
}

// One time step: stream (a1), macroscopic fields (a2, a3), gradients (a5),
// collision (a4, a6-a10) and store (a11).
void oc_step(void* h, int nsteps) {
  Oracle* o = (Oracle*)h;
  for (int s = 0; s < nsteps; ++s) {
    stream(*o);
    compute_all_macro(*o);
#pragma omp parallel for schedule(static)
    for (int n = 0; n < o->N; ++n) {
      real fout[(MMAX + 2) * QMAX];
      collide_at(o, n, fout);
      for (int l = 0; l < o->nl; ++l)
        for (int i = 0; i < o->Q; ++i) o->pops[PIDX(*o, l, i, n)] = stored(fout[l * o->Q + i]);
    }
    if (o->S > 0) o->Xs.swap(o->Xs_new);
    o->steps_done++;
  }
}

// Stored populations (lane < 0: values; lane k: derivative k).
void oc_get_pops_lane(void* h, int lane, double* out) {
  Oracle* o = (Oracle*)h;
  for (size_t k = 0; k < o->pops.size(); ++k) out[k] = comp(o->pops[k], lane);
}

void oc_get_pops(void* h, double* out) { oc_get_pops_lane(h, -1, out); }

// Replaces the populations (derivative parts set to zero).
void oc_set_pops(void* h, const double* in) {
  Oracle* o = (Oracle*)h;
  for (size_t k = 0; k < o->pops.size(); ++k) o->pops[k] = in[k];
}

// Streamed (pre-collision) populations of the last step.
void oc_get_pulled(void* h, double* out) {
  Oracle* o = (Oracle*)h;
  for (size_t k = 0; k < o->pulled.size(); ++k) out[k] = comp(o->pulled[k], -1);
}

// Diagnostics of the last collision: which = 0 V[M][3], 1 Fk[3], 2 omega,
// 3 omega1, 4 kappa bound, 5 rhodot[M]; node-major blocks of N.
void oc_get_diag(void* h, int which, double* out) {
  Oracle* o = (Oracle*)h;
  const std::vector<real>* v = nullptr;
  size_t cnt = 0;
  switch (which) {
    case 0: v = &o->dg_V; cnt = (size_t)o->M * 3 * o->N; break;
    case 1: v = &o->dg_Fk; cnt = (size_t)3 * o->N; break;
    case 2: v = &o->dg_omega; cnt = o->N; break;
    case 3: v = &o->dg_omega1; cnt = o->N; break;
    case 4: v = &o->dg_kappa; cnt = o->N; break;
    case 5: v = &o->dg_rhodot; cnt = (size_t)o->M * o->N; break;
    case 6: v = &o->dg_current; cnt = o->N; break;
    default: return;
  }
  for (size_t k = 0; k < cnt; ++k) out[k] = comp((*v)[k], -1);
}

// Macroscopic fields of the current state: the populations are streamed (with
// the boundary conditions) and their moments taken, exactly as the next step
// would see them; the stored populations are not changed.
// which: 0 rho_a [M][N] (kg/m^3), 1 j_a [M][D][N] (lattice), 2 rho (momentum
// lattice) [N], 3 u [D][N] (lattice), 4 T [N] (K), 5 P [N] (Pa),
// 6 V_a [M][D][N] (lattice), 7 N_a [M][D][N] (mol m^-2 s^-1), 8 X_s [S][N],
// 9 rho_s = sum rho_a [N].
void oc_moments(void* h, int which, double* out) { moments_lane((Oracle*)h, which, -1, out); }

// Derivative `lane` of the same fields (dual build; lane < oc_lanes()).
void oc_moments_lane(void* h, int which, int lane, double* out) { moments_lane((Oracle*)h, which, lane, out); }

// Seeds the derivative lanes (dual build): dphi [lanes][N] (null: zero),
// dpore [lanes] and dtort [lanes] (null: zero) are the directions of the
// porosity field, pore radius [m] and tortuosity; the populations are reset
// to the initial equilibria, whose derivatives follow from the porosity.
// Potential difference Phi_electrode - Phi_electrolyte of the TPB steps: per
// node (field of N values) or, with field == NULL, the same everywhere.
void oc_set_potential(void* h, const double* field, double uniform) {
  Oracle* o = (Oracle*)h;
  o->dphi = uniform;
  if (field) o->dphi_node.assign(field, field + o->N);
  else o->dphi_node.clear();
}

void oc_set_tangents(void* h, const double* dphi, const double* dpore, const double* dtort, const double* dA) {
  Oracle* o = (Oracle*)h;
#ifdef ORACLE_DUAL
  for (int n = 0; n < o->N; ++n)
    for (int k = 0; k < NT; ++k) o->phi[n].d[k] = dphi ? dphi[(size_t)k * o->N + n] : 0.0;
  for (int k = 0; k < NT; ++k) {
    o->d0.d[k] = dpore ? 2.0 * dpore[k] / o->cfg.dx : 0.0;
    o->tort.d[k] = dtort ? dtort[k] : 0.0;
  }
  // directions of the pre-exponential factors A_r [lane][reaction]
  for (int r = 0; r < o->Rn; ++r)
    for (int k = 0; k < NT; ++k) o->Apre[r].d[k] = dA ? dA[(size_t)k * o->Rn + r] : 0.0;
#else
  (void)dphi; (void)dpore; (void)dtort; (void)dA;
#endif
  init_populations(o);
  for (int s = 0; s < o->S; ++s)
    for (int n = 0; n < o->N; ++n) o->Xs[(size_t)s * o->N + n] = o->Xs_init0[s];
  o->steps_done = 0;
}

// ---- single-node helpers for the pin tests --------------------------------
void oc_product_form(int D, const double* xi, const double* P, double* out) {
  Lattice L = make_lattice(D);
  real x[3], p[3], r[QMAX];
  for (int a = 0; a < 3; ++a) { x[a] = xi[a < D ? a : 0]; p[a] = P[a < D ? a : 0]; }
  product_form(L, x, p, r);
  for (int i = 0; i < L.Q; ++i) out[i] = comp(r[i], -1);
}

void oc_energy_equilibrium(int D, double phi, double rho, const double* u, double RT, double U, double* out) {
  Lattice L = make_lattice(D);
  real uu[3] = {u[0], u[1], u[2]}, r[QMAX];
  energy_equilibrium(L, phi, rho, uu, RT, U, r);
  for (int i = 0; i < L.Q; ++i) out[i] = comp(r[i], -1);
}

void oc_qr_solve(int n, const double* A, int nrhs, const double* b, double* x) {
  real Ar[MMAX * MMAX], br[MMAX * 3], xr[MMAX * 3];
  for (int k = 0; k < n * n; ++k) Ar[k] = A[k];
  for (int k = 0; k < n * nrhs; ++k) br[k] = b[k];
  householder_qr_solve(n, Ar, nrhs, br, xr);
  for (int k = 0; k < n * nrhs; ++k) x[k] = comp(xr[k], -1);
}

void oc_lattice(int D, int* c, double* w) {
  Lattice L = make_lattice(D);
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c[i * 3 + a] = L.c[i][a];
    w[i] = lattice_weight(L, i);
  }
}

}  // extern "C"
