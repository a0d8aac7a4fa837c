/*
 * lbm.h -- C ABI of the B300 (sm_103a) double-distribution lattice Boltzmann
 * library: consistent body force and heat source for compressible flows of
 * generic fluids (arxiv 2609.28679).
 *
 * One call of lbm_step advances every population of a simulation by one time
 * step of the paper's scheme (Sec. II.E, Fig. "Structure of the algorithm"):
 *   moments with the half-force/half-source shifts (Eqs. def_h, def_u, def_E),
 *   force F = rho*a + Korteweg kappa rho grad lap rho (Eqs. force_decomposition,
 *   korteweg_force) and heat source Q, temperature from the equation of state
 *   (Eq. TdependsongenericEOS), closure scalars theta = P/rho, alpha, gamma
 *   (Eqs. theta, corr_bulk, corr_heat_source), shifted states u*, theta*, T*,
 *   q^c and the Galilean correction Phi (Eqs. sh_vel_1, sh_temp_1, sh_T_1,
 *   qc_1, correction), product-form equilibria f^eq, f*, g^eq, g* (Eqs. LBMeq,
 *   LBMstar, LBMeqG, LBMgstar), collision with beta = 1/(2 tau + 1)
 *   (Eqs. beta, LBM_f, LBM_g, lambda = dt) and streaming.
 *
 * Units: lattice units, dt = dx = c = 1, varsigma^2 = 1/3 (Eq. cs).
 * Lattices: dim = 3 is the paper's D3Q27 (Eq. D3Q27c); dim = 2 its product
 * restriction D2Q9.  Population i has base-3 digits (d_x, d_y, d_z) with digit
 * 0, 1, 2 meaning c = 0, +1, -1.
 *
 * Conventions shared by every call:
 *  - Host-visible fields are float64, cell index k = x + nx*(y + ny*z);
 *    scalars are [N], vectors [dim][N] (component-major).  For a batch handle
 *    the fields of simulation s follow those of simulation s-1 (rho and T by
 *    N_s, u by dim*N_s).
 *  - Pointers are host pointers when on_device == 0, device pointers of the
 *    library's device otherwise.  The caller owns every buffer it passes; the
 *    library owns the populations and its work arrays, which callers never see
 *    except through lbm_populations.
 *  - Device memory comes from PyTorch's CUDA caching allocator (libc10_cuda);
 *    it must be initialised (torch.cuda.init(), which the Python binding does)
 *    before lbm_create.  Work is enqueued on the handle's stream (default: the
 *    current PyTorch stream of the device at lbm_create; see lbm_set_stream).
 *  - Every function returns LBM_OK (0) or a negative LBM_E_* code and keeps a
 *    message retrievable with lbm_last_error.  Calls that copy to host memory
 *    synchronise the handle's stream; lbm_step only enqueues.
 *  - A handle is not safe to use from several threads at once.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_E_INVALID (-1)     /* bad argument or struct field            */
#define LBM_E_NOMEM (-2)       /* device allocation failed                */
#define LBM_E_CUDA (-3)        /* a CUDA runtime call or launch failed    */
#define LBM_E_UNSUPPORTED (-4) /* valid but not built (e.g. form/lattice) */
#define LBM_E_STATE (-5)       /* call out of order (e.g. step before init) */

/* population storage */
#define LBM_F64 0  /* float64 populations, float64 arithmetic                   */
#define LBM_F32 1  /* float32 populations, float32 arithmetic                   */
#define LBM_BF16 2 /* bfloat16 of f_i - f_i^ref, float32 arithmetic            */
#define LBM_F16 3  /* float16 of f_i - f_i^ref, float32 arithmetic             */

/* equations of state */
#define LBM_IDEAL 0 /* P = rho R T (Eq. idealEOS)                                 */
#define LBM_VDW 1   /* P = rho R T/(1 - b rho) - a rho^2 (Eq. vdw_eos)             */
#define LBM_PR 2    /* Peng-Robinson, Soave alpha(T), constant ideal-part c_v    */

/* temperature inversion T(rho, e) for Peng-Robinson */
#define LBM_T_NEWTON 0 /* Newton's method, warm-started from the previous T         */
#define LBM_T_MLP 1    /* learned T(rho, e) (lbm_mlp_load) with Newton fallback      */

/* derivative in the Galilean correction Phi (Eq. correction) */
#define LBM_PHI_UPWIND 0  /* 3rd-order upwind-biased: (2 X+1 + 3 X0 - 6 X-1 + X-2)/6 for u >= 0, mirrored */
#define LBM_PHI_CENTRAL 1 /* 2-point central                                     */

/* kernel variants (lbm_set_kernel) */
#define LBM_KERNEL_AUTO 0  /* the library's choice (autotuned when a cache entry exists) */
#define LBM_KERNEL_SPLIT 1 /* moments, macroscopic, collide-stream: three passes         */
#define LBM_KERNEL_FUSED 2 /* one pass per step, shared-memory halo tiles                */
#define LBM_KERNEL_ZMARCH 3 /* D3Q27: macroscopic pass + z-marching collide-stream pass   */
#define LBM_KERNEL_ZGATHER 4 /* D3Q27: macroscopic pass + column-march collide-stream pass with
                                staged pulls and gathered moments (32-/16-bit storage)      */
#define LBM_KERNEL_YMARCH 5  /* D2Q9: one pass per step, CTAs marching up x strips with row
                                rings (32-/16-bit storage, no learned temperature)          */

typedef struct lbm_ctx *lbm_handle;

typedef struct {
    int dim;        /* 2 -> D2Q9, 3 -> D3Q27                                   */
    int nx, ny, nz; /* cells; nz = 1 when dim = 2                             */
    int zwalls;     /* 0: periodic in z; 1: half-way bounce-back at both z faces (dim 3);
                       2: non-equilibrium-extrapolation walls on the cells z = 0 and z = nz - 1
                       (dim 3, nz >= 4; wall state from lbm_set_walls / lbm_set_face; split kernels,
                       and the z-march with 32- or 64-bit storage on tiles 30x14 and 30x6) */
    int storage;    /* LBM_F64 | LBM_F32 | LBM_BF16 | LBM_F16                  */
    int phi_scheme; /* LBM_PHI_UPWIND | LBM_PHI_CENTRAL                        */
} lbm_lattice;

typedef struct {
    int kind;           /* LBM_IDEAL | LBM_VDW | LBM_PR                          */
    double R, cv;       /* gas constant; constant (ideal-part) specific heat    */
    double a, b;        /* attraction, co-volume (vdW, PR); PR: if a == 0 they
                           follow from (Tc, Pc): a = 0.45724 R^2 Tc^2/Pc,
                           b = 0.07780 R Tc/Pc                                  */
    double Tc, Pc;      /* PR critical temperature and pressure                 */
    double omega;       /* PR acentric factor                                    */
    double kappa;       /* Korteweg capillarity coefficient (0: no F_K)         */
    double eta_over_mu; /* bulk / shear viscosity (Eq. corr_bulk)                */
    double k_over_mu;   /* thermal conductivity / shear viscosity (Eq. qc_1)    */
    int t_solver;       /* LBM_T_NEWTON | LBM_T_MLP                              */
    double mu;          /* shear viscosity of the paper's tau = mu / P (Sec. II.C):
                           > 0: tau and beta (Eq. beta) per cell from the cell's
                           pressure, one tau for f and g (tau_f, tau_g unused);
                           0: constant tau_f, tau_g                              */
    int isothermal;     /* 1: the g equation is not solved, as in the paper's
                           isothermal tests (Sec. III.A): every cell keeps the
                           temperature lbm_init gave it, e = e(rho, T), and the
                           g populations and the energy invariant are left
                           undefined; needs no heat source and t_solver
                           LBM_T_NEWTON; not for lbm_step_static.  0: full model */
} lbm_eos;

typedef struct {
    double accel[3]; /* body acceleration a: F_B = rho a (Eq. force_decomposition) */
    double friction; /* duct friction k = f_D / (2 D_h) >= 0 (Fanno flow, Sec. III.A): F_f = -k rho |u| u
                        joins F and its work returns as heat, Q_f = -F_f.u; u = (sum c f + F/2)/rho is
                        solved with F_f exactly, u = 2 w / (1 + sqrt(1 + 2 k |w|)), w the velocity without
                        F_f.  Split kernels, and the z-march when the lattice has zwalls = 2. */
    double throttle_K;     /* Darcy throttle (throttling process, Sec. III.B): F_t = -K phi(z) rho u with */
    double throttle_sigma; /* phi = exp(-((z - (nz-1)/2)/sigma)^2), dim 3, and its heat Q_t = -F_t.u; solved
                              with F_f: u = 2 w / (a + sqrt(a^2 + 2 k |w|)), a = 1 + K phi/2.  Kernels
                              as for friction; K >= 0, sigma > 0 when K > 0. */
    const double *field;   /* optional per-cell body force F_B(x) added to rho a (Eq. force_decomposition):
                              device memory, float64 [dim][N] over this simulation's N cells, x fastest;
                              owned by the caller, read at every step (it may change between steps) and
                              kept alive while the handle steps; NULL for none.  Split kernels. */
} lbm_force;

typedef struct {
    double q;         /* volumetric heat source Q                                 */
    int zmask_lo;     /* Q acts on cells with zmask_lo <= z < zmask_hi ...        */
    int zmask_hi;     /* ... and everywhere when zmask_hi <= 0                    */
    const double *field; /* optional per-cell heat source Q(x) added to the above: device memory,
                            float64 [N] of this simulation, owned by the caller, read at every step;
                            NULL for none.  Split kernels. */
} lbm_heat;

/* Create one simulation.  tau_f, tau_g are the paper's relaxation time tau of
 * f and g (beta = 1/(2 tau + 1), Eq. beta; tau > 0), used when eos->mu is 0
 * (eos->mu > 0: tau = mu / P per cell instead).  force and heat may be
 * NULL (no body force / no heat source).  Allocates 2 x 2 x Q x N populations
 * of the storage type plus work arrays.  Errors: LBM_E_INVALID (dim not 2/3,
 * sizes < 1, nz != 1 in 2-D, walls in 2-D, kind/storage/scheme out of range,
 * tau <= 0, b*rho limits are not checked), LBM_E_NOMEM, LBM_E_CUDA. */
int lbm_create(const lbm_lattice *lattice, const lbm_eos *eos, double tau_f, double tau_g,
               const lbm_force *force, const lbm_heat *heat, lbm_handle *out);

/* Create nsim independent simulations stepped together (one launch per step
 * for all of them).  Arrays of nsim entries; every lattice must share dim and
 * storage; force/heat may be NULL (none for all) or arrays of nsim. */
int lbm_create_batch(int nsim, const lbm_lattice *lattices, const lbm_eos *eos, const double *tau_f,
                     const double *tau_g, const lbm_force *force, const lbm_heat *heat, lbm_handle *out);

void lbm_destroy(lbm_handle h);

/* Use `stream` (a cudaStream_t) for all later work of h; NULL selects the
 * legacy default stream. */
int lbm_set_stream(lbm_handle h, void *stream);

/* Replace the body acceleration a (F_B = rho a, Eq. force_decomposition) of
 * every simulation of h from the next step on, for forcing that varies in
 * time (the pulsatile flows of Sec. III.A use a cos(omega t)).  accel: 3
 * doubles (host); a 2-D lattice ignores accel[2].  The update is enqueued on
 * h's stream ahead of later steps; captured step graphs read it too.
 * Errors: LBM_E_INVALID (NULL, non-finite values), LBM_E_CUDA. */
int lbm_set_force(lbm_handle h, const double *accel);

/* Wall state of the non-equilibrium-extrapolation walls (zwalls = 2), the
 * wall treatment of the thermal Couette flow (App. B), for every simulation
 * of h that has them.  The walls lie on the boundary cells z = 0 (u_lo, T_lo)
 * and z = nz - 1 (u_hi, T_hi).  Each step, after the macroscopic pass, a
 * boundary cell B with neighbour N (z = 1, nz - 2) is rebuilt as
 *   f_B = f^eq(rho_B, u_W, theta(rho_B, T_W)) + f_N - f^eq(rho_N, u_N, theta_N)
 * and g_B alike, then collides like any cell.  rho_B: wall_rho 1 takes
 * rho_N as the text states; wall_rho 0 solves P(rho_B, T_W) = P(rho_N, T_N)
 * by eight Newton steps from rho_N, which is rho_N wherever T_W = T_N and
 * keeps mass from leaking through a wall whose temperature differs from its
 * neighbour's; wall_rho 2 solves P(rho_B, T_W) = 2 P_N - P_NN (NN two cells
 * inside), the same where the pressure is uniform, and also tight under a
 * force normal to the wall (a hydrostatic pressure gradient).  Stencils past a wall use the
 * linear extrapolation through the boundary cell, 2 v(z_B) - v(2 z_B - z).
 * u_lo, u_hi: 3 doubles (host); T_lo, T_hi > 0.  Stepping a handle with such
 * walls before this call fails with LBM_E_STATE.  The split kernels run
 * them, and the z-march with 32- or 64-bit storage on its 30x14 and 30x6
 * tiles (the default then); lbm_set_kernel answers LBM_E_UNSUPPORTED for
 * the fused kernels and other z-march tiles.  Errors:
 * LBM_E_INVALID (NULL, non-finite, T <= 0, wall_rho not 0, 1 or 2), LBM_E_STATE
 * (no such walls in h), LBM_E_CUDA. */
int lbm_set_walls(lbm_handle h, const double *u_lo, double T_lo, const double *u_hi, double T_hi, int wall_rho);

/* Boundary kinds of one z face with zwalls = 2 (the ends of the 1-D duct of
 * Sec. III.A; the duct runs as a 1 x 1 x nz column of D3Q27, whose
 * populations summed over c_x, c_y follow the 1-D product form exactly). */
#define LBM_FACE_INLET_TOTAL 1   /* subsonic inlet: total pressure P and temperature T (ideal gas); u of the neighbour */
#define LBM_FACE_INLET_STATIC 2  /* supersonic inlet: static P, T and the velocity u */
#define LBM_FACE_OUTLET_P 3      /* subsonic outlet: static P; T and the mass flux rho u of the neighbour */
#define LBM_FACE_OUTLET_EXTRAP 4 /* supersonic outlet: rho, u, T of the neighbour */
#define LBM_FACE_INLET_PT 5      /* inlet at fixed static P and T (throttling); u of the neighbour */

/* Make face 0 (z = 0) or 1 (z = nz - 1) of every simulation of h that has
 * zwalls = 2 an open duct end of the given kind.  The boundary cell is
 * rebuilt each step as for lbm_set_walls: f_B = f^eq(rho_B, u_B, theta_B) +
 * f_N - f^eq(N), g alike, with the boundary state (rho_B, u_B, T_B) of the
 * kind: INLET_TOTAL T_B = T - |u_N|^2/(2 c_p), P_B = P (T_B/T)^(c_p/R),
 * u_B = u_N; INLET_STATIC P, T and u as given; OUTLET_P P as given, T_N and
 * u_B = u_N rho_N / rho_B; OUTLET_EXTRAP rho_N, u_N, T_N; INLET_PT P and T as
 * given, u_N.  rho_B meets the
 * pressure at T_B by eight Newton steps from rho_N.  u: 3 doubles (host;
 * read for INLET_STATIC only, may be NULL otherwise); T > 0 for the inlets;
 * P > 0 for all but OUTLET_EXTRAP.  A face set here replaces the wall that
 * lbm_set_walls put there; each face must be set (here or by lbm_set_walls)
 * before h steps.  Errors: LBM_E_INVALID (face, kind, values), LBM_E_STATE
 * (no such walls in h), LBM_E_UNSUPPORTED (INLET_TOTAL with a non-ideal
 * equation of state), LBM_E_CUDA. */
int lbm_set_face(lbm_handle h, int face, int kind, const double *u, double T, double P);

/* Initial state (flowchart, first box): f = f^eq(rho, u, theta), g = g^eq with
 * theta = P(rho,T)/rho and e = e(rho,T).  rho [N], u [dim][N] and T [N]
 * float64, N the total cells of the handle (simulations concatenated, u per
 * simulation as dim planes of its cells); on_device 0: host memory (pinned
 * memory is copied by DMA, pageable memory through the driver's staging),
 * 1: device memory.  From host memory, handles of 2 M cells or more copy in
 * up to eight runs of cells on a copy stream of their own, each run set up
 * on h's stream while the next one crosses the link (with, on the kernels
 * that carry moments between steps, those of the new state).  The caller keeps
 * ownership; the call synchronises, so the buffers may be reused on return.  For 16-bit storage the per-direction
 * offsets f^ref, g^ref are the rest equilibria at the mean rho and mean T of
 * each simulation.  Errors: LBM_E_INVALID for a NULL field or for rho <= 0,
 * T <= 0 or NaN in any cell (checked on the device for 32- and 64-bit
 * storage); after any error the handle must be initialised again before it
 * steps (LBM_E_STATE); LBM_E_NOMEM, LBM_E_CUDA. */
int lbm_init(lbm_handle h, const double *rho, const double *u, const double *T, int on_device);

/* lbm_init with float32 fields (same layout, ownership, checks and errors).
 * For float32 and 16-bit storage nothing is lost: the state is formed in
 * float32 from the fields either way; half the bytes cross the host link. */
int lbm_init_f32(lbm_handle h, const float *rho, const float *u, const float *T, int on_device);

/* Advance every simulation of h by n >= 0 time steps (enqueue only). */
int lbm_step(lbm_handle h, int n);

/* Macroscopic fields of the current state: rho (Eq. def_h), the physical
 * velocity u = (sum c f + F/2)/rho (Eq. def_u) and T from the EoS.  Any of the
 * three pointers may be NULL.  Layout and on_device as lbm_init; to host
 * memory, handles of 2 M cells or more copy run by run as the runs are
 * evaluated.  Synchronises. */
int lbm_moments(lbm_handle h, double *rho, double *u, double *T, int on_device);

/* lbm_moments into float32 fields (same layout; for float32 and 16-bit
 * storage the values are exactly those lbm_moments returns as float64). */
int lbm_moments_f32(lbm_handle h, float *rho, float *u, float *T, int on_device);

/* The current populations as float64 [Q][N] (f) and [Q][N] (g), decoded from
 * the storage type (offset added back).  For tests and diagnostics. */
int lbm_populations(lbm_handle h, double *f, double *g, int on_device);

/* Totals of the current state, per simulation, 2*dim + 3 doubles each:
 *   [ sum rho, sum rho u (dim), sum rho E, sum F (dim), sum (u.F + Q) ]
 * with rho u, rho E the half-force moments (Eqs. def_u, def_E).  Reduced in
 * float64 (warp shuffles, then a fixed-order pass over the block partials).
 * Host pointer; synchronises. */
int lbm_invariants(lbm_handle h, double *out);

/* Diagnostic counters accumulated since lbm_init, summed over simulations:
 *   out[0] cells with a non-finite rho, u or T seen by a step
 *   out[1] cells with theta = P/rho <= 0 seen by a step
 *   out[2] Newton solves that hit the iteration cap
 *   out[3] cells whose learned temperature failed the residual test (Newton fallback)
 * Host pointer; synchronises. */
int lbm_diagnostics(lbm_handle h, long long out[4]);

/* Kernel selection: variant LBM_KERNEL_AUTO / SPLIT / FUSED / ZMARCH /
 * ZGATHER / YMARCH; tx, ty, tz the tile of the fused variant, or for ZMARCH
 * (3-D only) the xy tile and the number of z planes each CTA marches through
 * (0: default); ZGATHER has the xy tile 30 x 14 (tx, ty 0 or 30, 14) and
 * takes tz as its number of planes; YMARCH (2-D only) has strips of 124
 * columns (every simulation with the central Phi) or 122, tx 0 or that width,
 * and takes ty as the rows each CTA marches through (0: the row count that
 * lets the device's resident CTAs take the strips' ranges in the fewest
 * rounds of (rows + pipeline fill), at least 32; also the automatic choice
 * for 2-D lattices of 4 M cells and more).  Errors:
 * LBM_E_INVALID for a tile the variant cannot run, LBM_E_UNSUPPORTED for a
 * lattice or boundary set it does not run. */
int lbm_set_kernel(lbm_handle h, int variant, int tx, int ty, int tz);

/* n eager time steps (no graphs) with CUDA events recorded on h's stream
 * between the passes of every step; on return (synchronised) ms_per_pass
 * holds the mean device time per step of pass 1, 2, 3 and of the whole step:
 *   z-march variants: macroscopic pass, boundary-cell rebuild (0 without
 *                     extrapolated faces), collide-stream pass;
 *   fused:            0, 0, the one-pass step;
 *   split:            moments, macroscopic pass (and boundary cells), collide-stream.
 * The carried moments (after lbm_init or a kernel change) are prepared
 * before the first recorded step, outside its passes.  Errors as lbm_step. */
int lbm_step_timed(lbm_handle h, int n, double ms_per_pass[4]);

/* The float64 fused multiply-add rate of the current device (TFLOP/s, 2
 * FLOP per FMA): eight independent chains per thread, four full waves of
 * CTAs, best of three timed launches after a warm-up (ms: that launch's
 * duration, may be NULL).  Measurement infrastructure for the arithmetic
 * bound of the float64 forms; allocates nothing; synchronises `stream`
 * (NULL: the legacy default stream).  Errors: LBM_E_INVALID, LBM_E_CUDA. */
int lbm_fp64_peak(double *tflops, double *ms, void *stream);

/* Replay lbm_step's time steps as CUDA graphs of `steps_per_graph` steps (an
 * even number >= 2; 0 turns graphs off).  lbm_step(h, n) then runs one eager
 * step, n-1 steps as whole graphs and the remainder eagerly.  The graph is
 * captured on the first such call and kept until the kernel or stream
 * changes.  Needs a created stream (lbm_set_stream), not the legacy default
 * stream: LBM_E_STATE otherwise. */
int lbm_set_graph(lbm_handle h, int steps_per_graph);

/* Autotuner: time trial_steps steps (after 2 warm-up steps) of the split path
 * and of every built fused and z-march tile that runs this lattice, storage,
 * equation of state and boundary set, select the fastest, and restore the state as it was (populations,
 * Newton guess and diagnostic counters; the step count does not advance).
 * Outputs (any may be NULL): the chosen variant and tile, its ms per step.
 * Synchronises; allocates one snapshot of the populations for the duration
 * of the call. */
int lbm_autotune(lbm_handle h, int trial_steps, int *variant, int *tx, int *ty, int *tz, double *ms_per_step);

/* The variant and tile that lbm_step uses now. */
int lbm_get_kernel(lbm_handle h, int *variant, int *tx, int *ty, int *tz);

/* One time step of float64 populations owned by the caller, allocating
 * nothing.  The paper has no counterpart: this is a variant of the library's
 * three-pass step for callers that cannot allocate device memory when they
 * step.  The handle path takes its memory from PyTorch's caching allocator at
 * lbm_create; hosts that give each library a fixed device-memory budget up
 * front, programs that link this library without PyTorch, and time-critical
 * loops that must not call cudaMalloc or cudaFree (which waits for the whole
 * device) cannot use it.  This call keeps its work arrays in one fixed-size
 * static device array (room for 65536 cells, about 11.5 MB, held on every GPU
 * that loads the library until the process exits) and passes the simulation
 * constants to the device as a kernel argument: no allocation, no copy from
 * host memory.
 *
 * f_in, g_in: pre-collision populations [Q][N] (device, float64, the layout
 * of lbm_populations); f_out, g_out: the pre-collision populations of the
 * next step (device, must not overlap the inputs).  lattice->storage must be
 * LBM_F64.  Peng-Robinson's Newton iteration starts from the critical
 * temperature Tc in every cell (no temperature is carried between calls).
 * Work is enqueued on `stream` (NULL: the legacy default stream); the call
 * does not synchronise.
 *
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array: calls whose kernels overlap on the GPU (other
 * streams, other threads) race and corrupt each other -- serialise them.
 * Nothing carries over between calls: each one rewrites what it reads.
 * Errors: LBM_E_INVALID (NULL pointers, what lbm_create rejects, more than
 * 65536 cells, overlapping inputs and outputs), LBM_E_UNSUPPORTED (storage
 * other than float64, extrapolated walls, friction, throttles, force or heat
 * fields, t_solver other than LBM_T_NEWTON, the isothermal mode, which needs
 * the temperature a handle carries), LBM_E_CUDA; lbm_last_error(NULL)
 * describes the failure. */
int lbm_step_static(const lbm_lattice *lattice, const lbm_eos *eos, double tau_f, double tau_g,
                    const lbm_force *force, const lbm_heat *heat, const double *f_in, const double *g_in,
                    double *f_out, double *g_out, void *stream);

/* Learned temperature inversion T(rho, e) for Peng-Robinson (the form that
 * stands in for the per-cell Newton solve, falling back to Newton).  Network
 * 2 -> 64 -> 64 -> 1 with tanh hidden units; the 64 x 64 layer runs on the
 * tensor cores in bfloat16 with float32 accumulation.  Parameters are
 * lbm_mlp_nparams() floats:
 *   [c_rho, s_rho, c_e, s_e, c_T, s_T | W1 (64x2) | b1 (64) | W2 (64x64, [out][in]) | b2 (64) | W3 (64) | b3]
 * with inputs ((log rho - c_rho)/s_rho, (e - c_e)/s_e) and T_hat = c_T + s_T y. */
int lbm_mlp_nparams(void);

/* Train on nsamples samples drawn on the GPU: rho log-uniform over
 * [box[0], box[1]], T uniform over [box[2], box[3]] * Tc, e = e(rho, T), and
 * the target T re-solved from (rho, e) by float64 Newton.  `steps` Adam steps
 * (lr; beta 0.9/0.999) of minibatches of `batch` samples (counter-based
 * sampling with `seed`).  params (host, float32) is read as the start point,
 * or first initialised when init != 0 (normalisation from the box and the
 * samples' e range, weights uniform in +-1/sqrt(fan_in)); it receives the
 * trained network.  loss_hist (host, `steps` doubles) may be NULL.  eos must
 * be Peng-Robinson.  Synchronises `stream`. */
int lbm_mlp_train(const lbm_eos *eos, const double box[4], long long nsamples, int steps, int batch, double lr,
                  unsigned long long seed, int init, float *params, double *loss_hist, void *stream);

/* Loss (mean of (y - t)^2/2 over the n samples, t = (T - c_T)/s_T) and its
 * gradient with respect to the parameters (normalisation entries 0), from
 * the training kernel, for the host arrays rho, e, T of n samples. */
int lbm_mlp_grad(const float *params, const double *rho, const double *e, const double *T, long long n,
                 float *grad, double *loss);

/* T_hat for n (rho, e) pairs (host arrays) through the in-step inference routine. */
int lbm_mlp_predict(const float *params, const double *rho, const double *e, long long n, double *T_out);

/* Attach learned-inversion parameters (host, lbm_mlp_nparams() floats) to h:
 * simulations with eos kind LBM_PR and t_solver LBM_T_MLP then start each
 * cell's Newton solve from the network's T_hat and accept it when the first
 * Newton correction meets the tolerance (diagnostics[3] counts the cells
 * that needed more).  Without loaded parameters they use the previous step's
 * T.  The fused kernel runs the learned start for float32 storage; other
 * storages step through the split path. */
int lbm_mlp_load(lbm_handle h, const float *params);

/* Message of the last failing call on h (or of the last failing lbm_create*
 * or lbm_step_static when h is NULL).  Valid until the next call on h. */
const char *lbm_last_error(lbm_handle h);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
