/*
 * lbm.h -- C ABI of the GB300 library for the mean-field lattice Boltzmann
 * step of reactive gas mixtures in homogenised porous media
 * (N. Sawant and I. V. Karlin, "Mean field lattice Boltzmann model for
 * reactive mixtures in porous media", arXiv 2409.02930).
 *
 * One call of lbm_step advances every node by one fused stream-and-collide
 * time step: the M species lattices (Sec. 2.3, Eq. 21
 * with the dusty-gas relaxation Eq. 25 and the diffusion-velocity system
 * Eq. 29), the mixture momentum lattice (Sec. 3.2, Eq. 42 with the
 * extended equilibrium Eq. 44 and the net Knudsen force
 * Eq. 48), the mixture energy lattice (Sec. 3.3, Eq. 43 with
 * Eq. 51 and Eq. 54) and, when a surface mechanism is given, the
 * heterogeneous-reaction sources of Sec. 4.2 (Eq. 78, Eq. 87,
 * Eq. 88, Eq. 89).
 *
 * Conventions
 *   - All functions return LBM_OK (0) or a negative status code; no C++
 *     exception crosses this boundary.  lbm_last_error() describes the last
 *     failure of a context (or of lbm_create when ctx is NULL).
 *   - The library owns every device buffer it allocates; the caller owns
 *     every buffer it passes in.  Host arrays in lbm_config are read during
 *     lbm_create only and may be freed afterwards.
 *   - Work is issued on the stream given in lbm_config (NULL: the legacy
 *     default stream) and is asynchronous unless stated otherwise.
 *   - Node order is n = x + nx*(y + ny*z), x fastest.  Populations are stored
 *     structure-of-arrays [lattice][i][n]; lattice 0..M-1 are the species,
 *     M the momentum lattice, M+1 the energy lattice (when on).  Velocity i
 *     has c = (i%3-1, (i/3)%3-1, i/9-1) (D3Q27) or (i%3-1, i/3-1, 0) (D2Q9).
 *   - Internally velocities, temperatures R*T, diffusivities and pressures are
 *     in lattice units (dx, dt); densities stay in kg/m^3.  dt is fixed so
 *     that the lightest species has R_a T_scale dt^2/dx^2 = theta_max.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK            0
#define LBM_ERR_ARG      -1   /* invalid argument or configuration */
#define LBM_ERR_ALLOC    -2   /* device or host allocation failed */
#define LBM_ERR_NUMERIC  -3   /* non-finite or negative density seen by a kernel */
#define LBM_ERR_TIMEOUT  -4   /* a bounded device wait gave up */
#define LBM_ERR_STATE    -5   /* call not valid in the context's state */
#define LBM_ERR_CUDA     -6   /* a CUDA runtime call failed */

/* boundary conditions of the two x faces (y and z are periodic) */
#define LBM_BC_PERIODIC   0
#define LBM_BC_INLET      1   /* reservoir: missing populations replaced by equilibria */
#define LBM_BC_BOUNCEBACK 2   /* missing populations reflected (no flux, no slip) */

/* precision of storage and relaxation */
#define LBM_FP64 0
#define LBM_FP32 1            /* FP32 storage and arithmetic; the diffusion-velocity
                                 solve switches to FP64 where its condition bound
                                 exceeds kappa_threshold */

/* moment selectors for lbm_moments (layout [component][n]) */
#define LBM_MOM_RHO_A 0       /* species densities rho_a, [M][N], kg/m^3 (Eq. 4) */
#define LBM_MOM_J_A   1       /* species momenta sum_i f_ai c_i, [M][D][N], lattice units (Eq. 5) */
#define LBM_MOM_RHO   2       /* mixture density of the momentum lattice, [N], kg/m^3 (Eq. 37) */
#define LBM_MOM_U     3       /* mixture velocity, [D][N], lattice units (Eq. 38) */
#define LBM_MOM_T     4       /* temperature, [N], K (Eq. 41) */
#define LBM_MOM_P     5       /* pressure, [N], Pa (Eq. 3) */
#define LBM_MOM_V_A   6       /* diffusion velocities V_a, [M][D][N], lattice units (Eq. 29) */
#define LBM_MOM_N_A   7       /* molar fluxes rho_a (u + V_a)/m_a, [M][D][N], mol m^-2 s^-1 */
#define LBM_MOM_XS    8       /* surface coverages X^(s), [S][N] (Eq. 70) */
#define LBM_MOM_RHO_S 9       /* sum_a rho_a, [N], kg/m^3 (Eq. 1) */
#define LBM_MOM_CURRENT 10    /* volumetric current of the TPB steps, [N], A per m^3 of porous medium
                                 (Eq. 74; zero without edge steps) */

typedef struct lbm_ctx lbm_ctx;

/*
 * Physical description of one lattice.  Arrays are host pointers, double
 * precision, SI units unless stated; N = nx*ny*nz.
 */
typedef struct lbm_config {
  int nx, ny, nz;              /* nz == 1: D2Q9, nz > 1: D3Q27 */
  int bc_lo, bc_hi;            /* LBM_BC_* of the x = 0 and x = nx-1 faces */
  int M;                       /* gas species: 2, 3 or 6 */
  int energy;                  /* 1: energy lattice on; 0: isothermal at T_init */
  int knudsen;                 /* 1: Knudsen diffusion on */
  int precision;               /* LBM_FP64 or LBM_FP32 */
  double dx;                   /* lattice spacing [m] */
  double theta_max;            /* lattice temperature of the lightest species at T_scale */
  double T_scale;              /* [K] */
  double T_ref, P_ref;         /* reference state of D_ref and mu_ref [K], [Pa] */
  double mu_exp;               /* mu_a = mu_ref,a (T/T_ref)^mu_exp */
  double Pr;                   /* Prandtl number: lambda = mu C_p / Pr */
  double bulk_ratio;           /* bulk viscosity / shear viscosity */
  double T_thermo;             /* reference temperature of U0 [K] */
  double tortuosity;
  double pore_radius;          /* [m]; Knudsen diameter d0 = 2 pore_radius */
  double kappa_threshold;      /* LBM_FP32: FP64 solve above this bound (<= 0: 1e3) */
  const double* molar_mass;    /* [M] kg/mol */
  const double* D_ref;         /* [M*M] binary diffusivities at (T_ref, P_ref) [m^2/s] */
  const double* mu_ref;        /* [M] Pa s at T_ref */
  const double* cv_factor;     /* [M] C_v,a / R_a */
  const double* U0;            /* [M] specific internal energy at T_thermo [J/kg] */
  const double* porosity;      /* [N] in (0, 1] */
  const double* X_init;        /* [M*N] initial mole fractions */
  const double* T_init;        /* [N] initial (isothermal: fixed) temperature [K] */
  const double* P_init;        /* [N] initial pressure [Pa] */
  const double* U_init;        /* [3*N] initial velocity [m/s], or NULL for rest */
  const double* X_in_lo;       /* [M] reservoir composition at x = 0 (LBM_BC_INLET) */
  const double* X_in_hi;       /* [M] reservoir composition at x = nx-1 */
  double T_in_lo, T_in_hi, P_in_lo, P_in_hi;
  /* surface mechanism (Sec. 4): S == 0 for none */
  int S, R;                    /* surface species (<= 12), reactions (<= 32); every step has
                                  integer reactant orders, at most 4 reactants and at most 8
                                  species with nonzero stoichiometry (else LBM_ERR_ARG) */
  const double* nu_gas;        /* [R*M] signed stoichiometry, gas */
  const double* nu_surf;       /* [R*S] signed stoichiometry, surface */
  const double* A_pre;         /* [R] Arrhenius prefactors (SI for the order) */
  const double* Ea;            /* [R] activation energies [J/mol] */
  double gamma;                /* site density [mol/m^2] */
  double a_s;                  /* specific surface area [1/m] */
  const double* surf_cv_factor;/* [S] molar C_v / R_U of the adsorbates */
  const double* surf_U0;       /* [S] molar internal energy at T_thermo [J/mol] */
  const double* Xs_init;       /* [S] initial coverages */
  void* stream;                /* cudaStream_t for all work of the context */
  /* electrochemistry (Sec. 4): steps on the triple-phase boundary (TPB), an
   * edge whose length per volume of porous medium is l_tpb.  An edge step's
   * rate is per unit TPB length, involves adsorbates only, changes the
   * coverages by nu l_tpb/(a_s Gamma) per extent (Eq. 71)
   * and releases n_el electrons; its constant carries the factor
   * exp(beta_ct n_el F dphi/(R_U T)).  The volumetric current is
   * F l_tpb (electrons per TPB length and second) (Eq. 74); the
   * fluid energy gains the ohmic heat (a_s/l_tpb) I^2 resistivity dx and
   * loses the electric power |dphi| I (Sec. 4.2).  edge == NULL: no edge
   * steps (the fields below are then not read). */
  const int* edge;             /* [R] 1 for a TPB step, 0 for a surface step */
  const double* n_el;          /* [R] electrons released by each step */
  double l_tpb;                /* TPB length per volume [1/m^2] */
  double beta_ct;              /* charge-transfer symmetry factor */
  double resistivity;          /* electrolyte resistivity [Ohm m] */
  double dphi;                 /* Phi_electrode - Phi_electrolyte [V] */
} lbm_config;

/*
 * lbm_create -- validate cfg, allocate device state and set every population
 * to the equilibrium of the initial fields (Eq. 15, Eq. 44 without
 * extension, Eq. 51).  On success *out holds a new context.
 * Errors: LBM_ERR_ARG (dimensions < 1, inlet face with nx < 3, M outside
 * {2, 3, 6}, porosity outside (0, 1], non-positive mass, temperature, pressure,
 * dx or theta_max), LBM_ERR_ALLOC, LBM_ERR_CUDA (no device).
 */
int lbm_create(lbm_ctx** out, const lbm_config* cfg);

/*
 * lbm_create_batch -- one context holding n_cases independent D2Q9 lattices
 * (for instance the binary counter-diffusion capillaries of Sec. 5.1 at many
 * lengths, pressures and pore radii).  cfgs[c] describes case c exactly as
 * lbm_create would (each case gets its own lattice scaling from its dx,
 * theta_max and T_scale); every case must have nz = 1, no surface mechanism
 * and the same M, energy flag and precision, with (M, energy) = (2, off) or
 * (3, on); the stream of cfgs[0] is used.  The cases are stepped together:
 * each lbm_step launches two persistent kernels (macro-field pass, node
 * update) over one work list of node tiles of all cases, replayed from a
 * CUDA graph of 50 steps.  Variants 0..11 select the tile length (64, 128,
 * 256 nodes for (v % 6)/2 = 0, 1, 2), the grid (v even: one block per
 * resident slot of every SM, looping over a contiguous range of tiles; v odd:
 * one block per tile) and, for v >= 6, the staging of every node's pulled
 * populations in shared memory; lbm_autotune picks among them.  Per-node outputs
 * (lbm_moments, populations) are the concatenation over cases, in case
 * order, of each case's single-lattice layout.  Errors as lbm_create, plus
 * LBM_ERR_ARG for n_cases < 1 or cases of different kinds.
 */
int lbm_create_batch(lbm_ctx** out, int n_cases, const lbm_config* cfgs);

/*
 * lbm_case_info -- for case c of a batched context (c = 0 for a single
 * lattice): dt [s], dx/dt [m/s], nodes N_c, nx, ny and the element offset of
 * its populations into out[0..5].  Errors: LBM_ERR_ARG for c out of range.
 */
int lbm_case_info(const lbm_ctx* ctx, int c, double* out6);

/*
 * lbm_step -- advance n_steps time steps (pull streaming with the boundary
 * conditions, moments, isotropic gradients, diffusion-velocity solve,
 * species / momentum / energy collisions and surface source), asynchronously
 * on the context's stream.  Returns the status recorded by kernels of earlier
 * steps (LBM_ERR_NUMERIC if a non-finite density was seen) or LBM_OK.
 */
int lbm_step(lbm_ctx* ctx, int n_steps);

/*
 * lbm_moments -- macroscopic fields of the current state, as the next step
 * would see them (streamed populations, boundary conditions applied); the
 * state is not changed.  out is caller-owned, bytes its size; out_on_device
 * says whether out is a device pointer.  Values are written as double
 * (layouts per LBM_MOM_*).  The call synchronises the stream when out is a
 * host pointer.  Errors: LBM_ERR_ARG (unknown selector, buffer too small).
 */
int lbm_moments(lbm_ctx* ctx, int which, void* out, size_t bytes, int out_on_device);

/*
 * lbm_get_populations / lbm_set_populations -- copy the stored populations
 * (post-collision state, [L][Q][N] in the context's precision: 8 bytes per
 * value for LBM_FP64, 4 for LBM_FP32) to / from a caller buffer (host when
 * on_device == 0).  Synchronous.  Errors: LBM_ERR_ARG when bytes differs
 * from lbm_population_bytes().
 */
size_t lbm_population_bytes(const lbm_ctx* ctx);
int lbm_get_populations(lbm_ctx* ctx, void* buf, size_t bytes, int on_device);
int lbm_set_populations(lbm_ctx* ctx, const void* buf, size_t bytes, int on_device);

/*
 * lbm_get_columns / lbm_set_columns -- copy the stored populations of the x
 * columns [x0, x0 + ncols) to / from a packed caller buffer laid out
 * [L][Q][nz][ny][ncols] in the context's precision: the halo of an x-slab
 * decomposition, where a node's update reads the previous step's
 * populations up to two columns away (the pull, then the isotropic
 * gradient stencil of the moments used after Eq. 59 and Eq. 60), so two
 * columns cross each slab boundary.
 * bytes = L Q nz ny ncols times the value size.  Device buffers
 * (on_device != 0) are copied asynchronously on the context's stream, in
 * order with its steps; host buffers synchronously.  Single lattices only.
 * Errors: LBM_ERR_ARG (null buffer, x0 < 0, ncols < 1, x0 + ncols > nx, size
 * mismatch), LBM_ERR_STATE (batch context), LBM_ERR_CUDA.
 */
int lbm_get_columns(lbm_ctx* ctx, int x0, int ncols, void* buf, size_t bytes, int on_device);
int lbm_set_columns(lbm_ctx* ctx, int x0, int ncols, const void* buf, size_t bytes, int on_device);

/*
 * lbm_save / lbm_load -- checkpoint and resume the evolving state of a
 * context (single lattice or batch): the stored populations [L][Q][N] in the
 * context's precision, the surface coverages [S][N] (FP64) when it has a
 * surface mechanism, and the number of steps taken.  The image is a 128-byte
 * header (the 8 bytes "LBMSTATE", then int64 fields: format version 1,
 * precision, D, N, L, Q, S, steps taken, population bytes, coverage bytes)
 * followed by the populations and the coverages.  Static fields (porosity,
 * tortuosity, pore radius, mechanism, boundary conditions) are not saved:
 * load into a context created from the same configuration.
 *
 * lbm_save: buf is a caller-owned host buffer of *bytes bytes; on return
 * *bytes holds the image size.  buf == NULL only queries the size.
 * Errors: LBM_ERR_ARG when bytes is NULL or the buffer is too small (*bytes
 * then holds the size needed).
 * lbm_load: buf is a host buffer holding an image of `bytes` bytes.  Errors:
 * LBM_ERR_ARG when the header does not match the context (magic, version,
 * precision, D, N, L, Q or S differ) or bytes is not the image size; the
 * state is unchanged then.  Both calls are synchronous.
 */
int lbm_save(lbm_ctx* ctx, void* buf, size_t* bytes);
int lbm_load(lbm_ctx* ctx, const void* buf, size_t bytes);

/*
 * lbm_step_host -- streaming form for states that live in host memory: copies
 * the state in_host ([L][Q][N] populations in the context's precision, the
 * layout of lbm_get_populations) to the device, advances it n_steps with the
 * context's kernel form and parameters, and copies the result to out_host.
 * The context's own state (lbm_step, lbm_get_populations) is not touched.
 * Asynchronous: the call only enqueues.  The upload runs on an upload
 * stream, the steps on the context's stream and the download on a download
 * stream; alternate calls use two different pairs of device state slots, so
 * the upload of one call overlaps the steps and the download of the one
 * before.  in_host must stay unmodified, and out_host must not be read,
 * until lbm_sync returns (which waits for every stream of the context).  Use
 * page-locked host memory for the copies to overlap.  The first call
 * allocates four state slots.  Errors: LBM_ERR_ARG (null buffers, n_steps <
 * 0), LBM_ERR_STATE (batched contexts and lattices with a surface mechanism,
 * whose state is more than the populations), LBM_ERR_ALLOC, LBM_ERR_CUDA.
 */
int lbm_step_host(lbm_ctx* ctx, const void* in_host, void* out_host, int n_steps);

/* lbm_sync -- wait for the context's stream; returns the device status:
 * LBM_ERR_NUMERIC once a step met a non-finite or non-positive density or
 * temperature, LBM_ERR_TIMEOUT once a bounded device wait gave up (the status
 * is kept until the context is destroyed). */
int lbm_sync(lbm_ctx* ctx);

/*
 * lbm_set_potential -- the potential difference Phi_electrode -
 * Phi_electrolyte [V] seen by the TPB steps (Sec. 4, Sec. 4.1): field is a
 * host array of N values, one per node, or NULL for `uniform` everywhere.
 * The electrode phase has one potential (Eq. 75) while the
 * electrolyte potential varies along the cell (Eq. 77), so a
 * driver of the membrane-electrode assembly sets the field between steps.
 * Synchronous.  Errors: LBM_ERR_STATE (no surface mechanism), LBM_ERR_ALLOC.
 */
int lbm_set_potential(lbm_ctx* ctx, const double* field, double uniform);

/*
 * lbm_set_wait_limit -- the bound of the device waits of the kernel forms
 * that stage lattice rows with bulk tensor copies: the number of mbarrier
 * probes a wait makes before it gives up (default 4194304).  The paper has
 * no counterpart; the setting exists to exercise the timeout path.  A wait
 * that gives up records LBM_ERR_TIMEOUT in the status word, the block stops
 * stepping and first drains the copies it has in flight (those waits keep
 * their own fixed bound), so no block ends with a copy outstanding; the
 * step's output is then not a valid state.  With a limit of 0 every staged
 * row wait gives up at once.  Errors: LBM_ERR_ARG (probes < 0).
 */
int lbm_set_wait_limit(lbm_ctx* ctx, int probes);

/* lbm_info -- dt [s], dx/dt [m/s], lattices L, velocities Q, dimension D into out[0..4]. */
int lbm_info(const lbm_ctx* ctx, double* out5);

/*
 * lbm_set_timing / lbm_get_timing -- kernel timing with CUDA events recorded
 * on the context's stream around every kernel that lbm_step launches.
 * lbm_set_timing(ctx, 1) clears and starts recording (at most 65536 launches
 * are kept); lbm_get_timing synchronises the stream and returns, per kernel
 * kind (0: macro-field pass, 1: collide / fused step, 2: reserved), the summed
 * device milliseconds and the launch counts.  Errors: LBM_ERR_STATE when
 * timing is off.
 */
int lbm_set_timing(lbm_ctx* ctx, int enable);
int lbm_get_timing(lbm_ctx* ctx, double* ms_by_kind /* [3] */, long long* launches_by_kind /* [3] */);

/*
 * Kernel forms.  Variant -1 is the two-pass form (a macro-field pass writes
 * u, Pi and Y_a to a device buffer, then the node update reads it); variants
 * 0 .. lbm_variant_count()-1 are single-launch or staged forms with
 * different tile shapes.  D2Q9: 0-4 the pipelined row march with per-thread
 * asynchronous copies, 5 a fused halo tile, 6-7 the staged two-pass form,
 * 8-9 the row march staged by bulk tensor copies (TMA; on lattices whose
 * rows are not a multiple of 16 bytes they run the per-thread-copy march of
 * the same tile shape, variants 2 and 0).
 * D3Q27: 0-2 fused halo tiles, 3-4 the staged two-pass form, 5 the staged
 * form with the gradient inputs computed in a pass of their own.  Every form
 * computes the same step (the gradient stencil is summed in different
 * orders, so the forms agree to rounding).  New contexts use variant 5 in
 * 3-D and, in 2-D, variant 8 on lattices of at least 2^18 nodes without a
 * reservoir face, else the two-pass form; batches use variant 2.  The adjoint's
 * forward and recompute steps use the context's form.  lbm_autotune times
 * every form for `steps` steps on the
 * current state, restores the state, selects the fastest form and writes its
 * index to *best (may be NULL).  Errors: LBM_ERR_ARG (unknown variant,
 * steps < 1), LBM_ERR_ALLOC.
 */
int lbm_variant_count(const lbm_ctx* ctx);
int lbm_set_variant(lbm_ctx* ctx, int variant);
int lbm_get_variant(const lbm_ctx* ctx);
int lbm_autotune(lbm_ctx* ctx, int steps, int* best);

/*
 * Objective of lbm_adjoint: J = weight * sum over the nodes of the plane
 * x = plane of the species-`species` momentum along `axis` of the streamed
 * populations of the final state (the flux moment LBM_MOM_J_A, lattice
 * units; with plane next to an outlet face this is the outlet flux of that
 * species).  kind must be LBM_OBJ_PLANE_FLUX.
 */
#define LBM_OBJ_PLANE_FLUX 0
typedef struct {
  int kind;
  int species;
  int axis;
  int plane;
  double weight;
} lbm_objective;

/*
 * lbm_adjoint -- gradient of an objective of the state after n_steps steps
 * from the configured initial state, by the discrete adjoint of the step
 * (reverse-mode differentiation of every stage: pull with the boundary
 * rules, macro fields, isotropic gradients, node update, initial
 * equilibria).  The forward run keeps a checkpoint every ckpt_every steps;
 * the reverse sweep recomputes the states of one segment at a time from its
 * checkpoint.  Device memory: (n_steps/ckpt_every + ckpt_every + 3) copies of
 * the populations, allocated for the call and freed before it returns.
 * Outputs (host pointers, each may be NULL): *J, dJ_dphi [N] (derivative
 * with respect to the porosity of every node), *dJ_dpore (pore radius, per
 * metre) and *dJ_dtort (tortuosity); pore radius and tortuosity enter the
 * step through their ratio (the Knudsen diffusivity of Sec. 5.1), so
 * r_p dJ/dr_p = -tau dJ/dtau.  On return the context holds the final state
 * of the forward run.  Supported: single 2-D lattices without a surface
 * mechanism, (M, energy) = (2, off) or (3, on).  Errors: LBM_ERR_ARG
 * (unsupported context, bad objective, n_steps < 0, ckpt_every < 1),
 * LBM_ERR_ALLOC, LBM_ERR_NUMERIC (non-finite state during the forward run).
 */
int lbm_adjoint(lbm_ctx* ctx, const lbm_objective* obj, int n_steps, int ckpt_every, double* J,
                double* dJ_dphi, double* dJ_dpore, double* dJ_dtort);

/*
 * lbm_step_noalloc -- one time step that allocates nothing.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * device memory while they run, such as a host framework that owns all
 * device memory through its own pool allocator, or a time-critical loop in
 * which cudaMalloc / cudaFree would synchronise the device.
 *
 * The caller owns the state: pops_in and pops_out are distinct device
 * buffers of L*Q*N values ([lattice][i][n], the layout of
 * lbm_get_populations, the precision of cfg->precision), porosity and
 * T_fixed are device arrays of N values in that precision (T_fixed is the
 * temperature of isothermal lattices and is not read when cfg->energy is
 * on).  cfg supplies the physical parameters (its host arrays molar_mass,
 * D_ref, mu_ref, cv_factor, U0 and the reservoir fields are read; porosity,
 * X_init, T_init, P_init are not) and the stream.  The step is the two-pass
 * form on a D2Q9 lattice (nz == 1, M = 2 or 3, no surface mechanism), issued
 * on cfg->stream.
 *
 * Its scratch (the macro fields of the first pass and a status word) lives
 * in one fixed array compiled into the library, lbm_noalloc_scratch_limit()
 * bytes of macro fields: (4 + M) * N * (8 or 4) bytes must fit, otherwise the
 * call returns LBM_ERR_ARG.  Every GPU that loads the library holds this
 * array until the process exits.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it for the rest of the process; make that first call before any
 * stream capture, and do not call again after resetting the device
 * (cudaDeviceReset unloads the array, so the kept address is stale).  All
 * calls share the array and it keeps the last call's contents, so calls whose
 * work overlaps on the GPU race.  The status word is cleared at every call;
 * the call then waits for the step to finish on cfg->stream and reports it.
 * The configuration is checked as lbm_create checks it (without the per-node
 * input arrays, which this call does not read).
 * Errors: LBM_ERR_ARG (invalid arguments, unsupported shape -- nz != 1, M
 * other than 2 or 3, a surface mechanism -- or a lattice too large),
 * LBM_ERR_NUMERIC (the step met a non-finite or non-positive state),
 * LBM_ERR_CUDA (address look-up, launch or the wait failed).
 */
int lbm_step_noalloc(const lbm_config* cfg, const void* pops_in, void* pops_out, const void* porosity,
                     const void* T_fixed);
size_t lbm_noalloc_scratch_limit(void);

/* lbm_destroy -- free the context (synchronises its stream first). NULL is a no-op. */
void lbm_destroy(lbm_ctx* ctx);

/* lbm_last_error -- message of the last failure (ctx may be NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
