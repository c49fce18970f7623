/*
 * dvbm.h -- C ABI of the GB300 double-distribution quasi-equilibrium DVBM
 * time step (libdvbm.so).
 *
 * Model (Strässle, Hosseini & Karlin, double-distribution quasi-equilibrium
 * approach): f (density/momentum) and g (internal non-translational energy,
 * split II, Sec. II.B.3 Eq. energy_eq_1) populations on the D2Q25
 * Gauss--Hermite lattice (App. G), fourth-order Grad--Hermite equilibria for f
 * and second-order for g (Sec. II.D.2-3), quasi-equilibria from the Table I
 * moment sets, two-rate relaxation (Eqs. new_collision_fi/gi) with
 * tau_1, tau_2 from mu and Pr (Sec. II.C), explicit Euler finite-volume update
 * with NND reconstruction and the generalized limiter (Sec. III.A.1-2,
 * Eq. finalDiscretePDE).
 *
 * Conventions for every entry point:
 *  - Every function returns a dvbm_status and never aborts or throws.  On a
 *    non-OK status a message is available from dvbm_last_error(ctx) (or
 *    dvbm_last_error(NULL) for failures of dvbm_create on the calling thread).
 *  - Macroscopic fields are row-major [Ny][Nx] double arrays (x fastest), cell
 *    centres x_j = (j + 1/2) Lx/Nx, y_k = (k + 1/2) Ly/Ny.  The caller owns
 *    every field buffer; the library owns the population buffers.
 *  - on_device = 1: pointers are device pointers on the context's device; the
 *    copies are stream-ordered on the context's stream.  on_device = 0: host
 *    pointers; the call synchronises the stream before returning.
 *  - A context is not thread-safe; calls on one context must be serialised.
 *  - GPU work is issued on the CUDA stream given at creation (NULL = legacy
 *    default stream).
 */
#ifndef DVBM_H
#define DVBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dvbm_ctx dvbm_ctx; /* opaque, owned by the library */

typedef enum {
  DVBM_OK = 0,
  DVBM_EINVAL = 1,    /* invalid argument (null pointer, bad size or parameter) */
  DVBM_ENOMEM = 2,    /* device allocation failed */
  DVBM_ECUDA = 3,     /* a CUDA runtime call failed */
  DVBM_EUNSTABLE = 4, /* a cell reached rho <= 0, T <= 0 or a non-finite value */
  DVBM_ETIMEOUT = 5,  /* the stream did not finish within opts.timeout_s; the
                         work queued on it stays queued and runs on, and a
                         later call waits for it again (see timeout_s) */
  DVBM_ESTATE = 6     /* call not valid in the context's current state */
} dvbm_status;

/* Lattice / energy split (Sec. II.D.3, App. G): D2Q25 with the internal
 * non-translational energy split (II; N_f = 4, N_g = 2; 50 planes) or D2Q16
 * with the total energy split (I; E = sum g, N_f = 3, N_g = 2, Table I split-I
 * quasi-equilibria; 32 planes; FP64 storage only, no adjoint). */
typedef enum { DVBM_D2Q25_SPLIT_II = 0, DVBM_D2Q16_SPLIT_I = 1 } dvbm_lattice;

/* Population storage.  FP64: populations as doubles.  FP32DEV: populations
 * stored as float deviations from w_i rho0 (f) and w_i rho0 (C_v - R) T0 (g);
 * moments, temperature and the collision coefficients are evaluated in
 * double, the Grad expansion of the collision target at FP64-or-better
 * precision (block fixed point, as for FP64 storage), advection in float on
 * the deviations. */
typedef enum { DVBM_FP64 = 0, DVBM_FP32DEV = 1 } dvbm_storage;

/* Boundary kinds (Sec. III.A.3, Sec. III.E).  PERIODIC: wrap (must be set on
 * both sides of an axis).  ZEROGRAD: zero-gradient ("von Neumann") ghost
 * cells copying the boundary cell.  WALL: isothermal no-slip wall on the
 * boundary face by ghost node + non-equilibrium extrapolation,
 * rho_G = rho_B, u_G = 2 u_W - u_B, T_G = 2 T_W - T_B,
 * f_G = f^eq(G) + (f_B - f^eq(B)) (same for g); ghost k mirrors interior
 * cell k, k = 1, 2. */
typedef enum { DVBM_BC_PERIODIC = 0, DVBM_BC_ZEROGRAD = 1, DVBM_BC_WALL = 2, DVBM_BC_EXTERNAL = 3 } dvbm_bc_kind;
/* EXTERNAL (y sides only): the context holds one band of rows of a grid
 * decomposed along y into slabs.  The scheme's stencil reaches two cells
 * along each axis (Sec. III.A.2, Eq. finalDiscretePDE), so before every step
 * the two ghost rows of an EXTERNAL side must be supplied with
 * dvbm_halo_unpack: the neighbouring slab's two boundary rows of the same
 * time level, taken from it with dvbm_halo_pack.  dvbm_step then advances one
 * step per call (n <= 1) and refuses (ESTATE) while a halo is stale.  An
 * EXTERNAL side counts as non-periodic for the pairing rule. */

typedef struct {
  int kind;         /* dvbm_bc_kind */
  double u_wall[2]; /* WALL: wall velocity */
  double T_wall;    /* WALL: wall temperature */
} dvbm_bc;

/* Sides of the bcs[4] array passed to dvbm_create. */
enum { DVBM_XLO = 0, DVBM_XHI = 1, DVBM_YLO = 2, DVBM_YHI = 3 };

typedef struct {
  double Lx, Ly;     /* domain size (default 1, Ny/Nx * Lx) */
  double R;          /* specific gas constant (default 1, Sec. III.A.3) */
  double T_ref;      /* lattice reference temperature (default 1, App. G) */
  double rho0, T0;   /* FP32DEV reference state (default 1, 1) */
  double beta;       /* limiter parameter in [1, 2] (default 1.2, Sec. III.A.3) */
  double cfl;        /* CFL number of the time-step rule (default 0.01) */
  double dt;         /* > 0: fixed time step overriding the CFL rule */
  int check_every;   /* dvbm_step checks the instability flag every k steps
                        (default 0: once at the end of each dvbm_step call;
                        < 0: never) */
  double timeout_s;  /* limit, in seconds, on every host wait for the stream
                        (default 600 s; <= 0 selects the default): the
                        instability checks, dvbm_init, dvbm_moments and
                        dvbm_totals with host outputs, dvbm_get_state /
                        dvbm_set_state, dvbm_adjoint, dvbm_adjoint_finish.
                        dvbm_create does not wait for the stream; dvbm_destroy
                        waits without a limit (below).  The stream is drained
                        under this limit before any copy into or out of
                        pageable host memory (such a copy would otherwise
                        block the calling thread without a limit).  A device
                        temporary that queued work may still use after an
                        ETIMEOUT is freed by dvbm_destroy, which synchronises
                        the stream first. */
} dvbm_opts;

/* Fill *opts with the defaults listed above (Lx = 1, Ly = 0 meaning
 * Ny/Nx * Lx).  Returns DVBM_EINVAL for a null pointer. */
dvbm_status dvbm_default_opts(dvbm_opts* opts);

/* Create a context: validate parameters, allocate two population buffers
 * (2 x 50 planes of (Ny + 4) x pitch values, ghost layers included) on the
 * current CUDA device.  Pr > 0; 1 < gamma <= 2 (split II needs
 * C_v >= R D/2, Sec. II.B.3); mu > 0; Nx, Ny >= 4; periodic sides paired.
 * opts may be NULL (defaults).  stream: a cudaStream_t or NULL.
 * Errors: EINVAL, ENOMEM, ECUDA; *out is NULL on failure. */
dvbm_status dvbm_create(dvbm_ctx** out, int lattice, int Nx, int Ny, double Pr, double gamma,
                        double mu, const dvbm_bc bcs[4], int storage, const dvbm_opts* opts,
                        void* stream);

/* Equilibrium initial conditions (Sec. III.A.3): populations = f^eq, g^eq of
 * the given rho, u_x, u_y, T at the cell centres; fills ghost layers; fixes
 * dt = cfl min(dx, dy) / max(|u| + sqrt(gamma R T)) over these fields unless
 * opts.dt > 0.  Resets the step counter.  Host fields (on_device = 0) pass
 * through a staging buffer of 4 Nx Ny doubles that the context allocates on
 * first use and keeps until dvbm_destroy.  The time step must respect the
 * explicit scheme's limits: max_i |v_i| dt / min(dx, dy) <= 1 (the fastest
 * population crosses at most one cell per step) and dt <= min(tau1, tau2) =
 * mu / p_max * min(1, 1/Pr) at the largest pressure p = rho R T of the given
 * fields (forward-Euler relaxation); otherwise EINVAL, and the context is left
 * as it was.  Errors: EINVAL (null pointer, rho <= 0 or T <= 0 or non-finite
 * input, dt beyond the limits), ENOMEM, ECUDA, ETIMEOUT. */
dvbm_status dvbm_init(dvbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                      const double* T, int on_device);

/* Advance n >= 0 explicit Euler steps (Eq. finalDiscretePDE), asynchronously
 * on the stream except for the instability checks (opts.check_every).
 * Errors: ESTATE (not initialised), EUNSTABLE, ETIMEOUT, ECUDA. */
dvbm_status dvbm_step(dvbm_ctx* ctx, int n);

/* rho, u_x, u_y, T of the current state (Sec. II.D.1 moments, T from
 * Eq. Total_energy_MB).  Any output pointer may be NULL to skip it.  Host
 * outputs (on_device = 0) go through the context's staging buffer (see
 * dvbm_init); the call returns once they are written.
 * Errors: EINVAL, ESTATE (no state yet), ENOMEM, ECUDA, ETIMEOUT. */
dvbm_status dvbm_moments(dvbm_ctx* ctx, double* rho, double* ux, double* uy, double* T,
                         int on_device);

/* Domain totals out[0..3] = mass, x-momentum, y-momentum, total energy
 * (sum over cells times dx dy).  Synchronous.  EUNSTABLE when a cell of the
 * current state has rho <= 0, T <= 0 or a non-finite value (out is filled
 * all the same).  Errors: EINVAL, ESTATE, EUNSTABLE, ECUDA, ETIMEOUT. */
dvbm_status dvbm_totals(dvbm_ctx* ctx, double out[4]);

/* Size in bytes of a state snapshot: the population planes [c][Ny][Nx] of the
 * storage type (double for FP64, float deviations for FP32DEV) plus one
 * 8-byte step counter at the end.  D2Q25: 50 planes, c = 5 p + q for f
 * (c < 25) and 25 + 5 p + q for g, x-node p and y-node q in the order
 * (0, +sqrt(5 - sqrt 10), -sqrt(5 - sqrt 10), +sqrt(5 + sqrt 10), -sqrt(5 + sqrt 10));
 * D2Q16: 32 planes, c = 4 p + q (f) and 16 + 4 p + q (g), node order
 * (+sqrt(3 - sqrt 6), -sqrt(3 - sqrt 6), +sqrt(3 + sqrt 6), -sqrt(3 + sqrt 6));
 * nodes times sqrt(R T_ref). */
size_t dvbm_state_bytes(const dvbm_ctx* ctx);

/* Copy the current state out / in (checkpoint / resume).  bytes must equal
 * dvbm_state_bytes.  set_state refills the ghost layers and clears the
 * instability flag (a run that returned EUNSTABLE resumes from a restored
 * state); the restored state is checked by the next step like any other.
 * Without a prior dvbm_init, set_state takes dt = opts.dt (> 0, else
 * ESTATE), subject to the one-cell-per-step limit of dvbm_init (else EINVAL).
 * Host buffers (on_device = 0) pass through a temporary device buffer.
 * Errors: EINVAL (null pointer, wrong size), ESTATE, ENOMEM, ECUDA, ETIMEOUT. */
dvbm_status dvbm_get_state(dvbm_ctx* ctx, void* buf, size_t bytes, int on_device);
dvbm_status dvbm_set_state(dvbm_ctx* ctx, const void* buf, size_t bytes, int on_device);

/* Record the forward run for dvbm_adjoint (or the stepwise adjoint below):
 * from the next dvbm_init on, keep the initial fields and a device copy of the
 * state every `every` steps (checkpoints; sqrt(n) is the usual choice).
 * every = 0 turns recording off.  Needs FP64 storage, the D2Q25 / split II
 * model and periodic boundaries; a band of a y-periodic grid (EXTERNAL y
 * sides) may record too, for the stepwise adjoint.  dvbm_set_state discards
 * the recording.  Errors: EINVAL. */
dvbm_status dvbm_record(dvbm_ctx* ctx, int every);

/* Discrete adjoint of the recorded run (a training pattern the paper does not
 * have; the forward map is Eq. finalDiscretePDE with equilibrium initial
 * conditions, dt held fixed).  Given device arrays [Ny][Nx] dL/drho and dL/dT
 * of the current state (either may be NULL = 0), writes the device arrays
 * dL/drho0, dL/dux0, dL/duy0, dL/dT0 of the initial fields and, to the host
 * array g_params, dL/dmu, dL/dPr, dL/dgamma.  Each checkpoint segment is
 * recomputed once, then stepped backwards with the hand-written adjoint step
 * kernel.  The state of the context is left unchanged.  Synchronous.  A band
 * (EXTERNAL sides) takes the stepwise adjoint below instead (EINVAL here).
 * Errors: ESTATE (no recording), EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
dvbm_status dvbm_adjoint(dvbm_ctx* ctx, const double* dL_drho, const double* dL_dT, double* g_rho0,
                         double* g_ux0, double* g_uy0, double* g_T0, double g_params[3]);

/* Stepwise adjoint, for a band of a slab-decomposed grid (EXTERNAL y sides),
 * whose adjoint steps need the neighbouring bands' rows at every step; it also
 * runs on a whole periodic grid.  With the rational limiter (beta = lp/lq,
 * the default) the arithmetic is that of dvbm_adjoint: the recompute records
 * each step's minmod branch codes and moments, and a band receives its
 * neighbours' code rows next to its edges.  Otherwise (or when the memory for
 * the codes is missing) the branches are derived from the recomputed states.
 *  - dvbm_adjoint_begin: lambda^N from the device arrays dL/drho, dL/dT of the
 *    band's current state (either may be NULL = 0), read by a kernel on the
 *    context's stream: they must stay valid until the stream has run it (at
 *    the latest, until dvbm_adjoint_finish returns).  Needs a recorded run.
 *  - dvbm_adjoint_advance: one action of the backward pass (restore a
 *    checkpoint, recompute one forward step of the segment, hand over that
 *    step's branch codes, or take one adjoint step back), in the same order on
 *    every band.  *halo says what needs the neighbouring bands' rows before
 *    the next call: 1 = the segment state just produced, 2 = the adjoint state
 *    just produced (also after dvbm_adjoint_begin), 3 = the branch-code rows
 *    of the step just recomputed; 0 = the pass is complete (call
 *    dvbm_adjoint_finish).
 *  - dvbm_adjoint_halo_pack / _unpack: as dvbm_halo_pack / _unpack, for what
 *    the last begin / advance named: two rows per side of a state in the
 *    [npop][2][Nx] double layout, or (*halo = 3) one row per side of branch
 *    codes, [npop][Nx] bytes at the start of the same buffers.  The same
 *    buffer rules.
 *  - dvbm_adjoint_finish: writes the device arrays dL/drho0, dL/dux0, dL/duy0,
 *    dL/dT0 of the band's initial fields and, to the host array g_params, the
 *    band's share of dL/dmu, dL/dPr, dL/dgamma (the grid's values are the sums
 *    over the bands).  Synchronous.
 * Everything but dvbm_adjoint_finish is stream-ordered without a host wait.
 * The state of the context is left unchanged.  Errors: ESTATE (no recording,
 * no pass begun, or finish before the pass is complete), EINVAL, ENOMEM,
 * ECUDA, ETIMEOUT. */
dvbm_status dvbm_adjoint_begin(dvbm_ctx* ctx, const double* dL_drho, const double* dL_dT);
dvbm_status dvbm_adjoint_advance(dvbm_ctx* ctx, int* halo);
dvbm_status dvbm_adjoint_halo_pack(dvbm_ctx* ctx, void* lo, void* hi);
dvbm_status dvbm_adjoint_halo_unpack(dvbm_ctx* ctx, const void* lo, const void* hi);
dvbm_status dvbm_adjoint_finish(dvbm_ctx* ctx, double* g_rho0, double* g_ux0, double* g_uy0, double* g_T0,
                                double g_params[3]);

/* Slab decomposition along y (multi-GPU, Sec. III.A.1; see DVBM_BC_EXTERNAL).
 * A halo buffer holds two rows of every population plane, layout
 * [npop][2][Nx] of the storage type (double for FP64, float deviations for
 * FP32DEV), rows in increasing y; dvbm_halo_bytes gives its size
 * (2 Nx npop element bytes).
 * dvbm_halo_pack writes the current state's two lowest interior rows
 * (y = 0, 1) to lo and its two highest (y = Ny - 2, Ny - 1) to hi: what the
 * lower and the upper neighbour need.  dvbm_halo_unpack writes lo into the
 * ghost rows below the band (y = -2, -1) and hi into those above it
 * (y = Ny, Ny + 1); every EXTERNAL side needs its buffer (else EINVAL), other
 * sides take NULL.  Pointers are device pointers on the context's device; the
 * copies are kernels on the context's stream (stream-ordered, no host wait).
 * Either pointer of dvbm_halo_pack may be NULL to skip that side.
 * Errors: EINVAL (null context, missing or unexpected buffer), ESTATE (no
 * state yet), ECUDA. */
size_t dvbm_halo_bytes(const dvbm_ctx* ctx);
dvbm_status dvbm_halo_pack(dvbm_ctx* ctx, void* lo, void* hi);
dvbm_status dvbm_halo_unpack(dvbm_ctx* ctx, const void* lo, const void* hi);

/* Replace the time step fixed at dvbm_init (or dvbm_set_state) by dt, e.g.
 * the smallest of the slabs' CFL steps so that every slab of a decomposed
 * grid steps with the same dt (Sec. III.A.3).  dt is checked against the
 * limits dvbm_init applies (one cell per step; the shortest relaxation time
 * of the field given to dvbm_init).  A run recorded for the adjoint keeps the
 * dt of its steps (the adjoint recomputes them): once it has stepped, a
 * different dt is refused.  Errors: EINVAL (dt <= 0, non-finite or beyond the
 * limits; the time step stays as it was), ESTATE (no state yet; a recorded
 * run that has stepped). */
dvbm_status dvbm_set_dt(dvbm_ctx* ctx, double dt);

/* Time step size fixed at dvbm_init (0 before). */
double dvbm_dt(const dvbm_ctx* ctx);

/* Number of steps taken since dvbm_init / dvbm_set_state. */
long long dvbm_steps_taken(const dvbm_ctx* ctx);

/* Last error message of ctx (or, if ctx is NULL, of the calling thread's last
 * failed dvbm_create).  Valid until the next call on that context (or the
 * thread's next dvbm_create). */
const char* dvbm_last_error(const dvbm_ctx* ctx);

/* Release the context and its device buffers (NULL is a no-op). */
void dvbm_destroy(dvbm_ctx* ctx);

/* Allocation-free CFL time step (the paper has no counterpart: this is a
 * service for callers that cannot allocate device memory, e.g. code inside a
 * framework whose caching allocator owns the whole device memory budget, or
 * loops where cudaMalloc/cudaFree would synchronise the device).
 * Computes dt = cfl * h / max over cells of (|u| + sqrt(gamma R T)) -- the rule
 * dvbm_init applies with h = min(dx, dy) -- from n device-resident doubles
 * per field, on `stream` (a cudaStream_t or NULL), and stores dt in the host
 * double *dt_out.  The call waits for the stream before it returns, for at
 * most 600 s (the library's default time limit; DVBM_ETIMEOUT beyond it, the
 * queued work staying queued).  No context, no device allocation: partial
 * maxima go to a fixed 64 KiB device array inside the library, held by every
 * GPU that loads it until the process exits.  Calls that overlap on the GPU
 * share that array and race: serialise them.  The first call on a device
 * looks up the array's device address.  Errors: EINVAL (null pointer,
 * n <= 0 or n > DVBM_NOALLOC_MAX_CELLS, bad gamma/R/cfl/h, or a field with
 * rho <= 0, T <= 0 or non-finite values), ETIMEOUT, ECUDA. */
#define DVBM_NOALLOC_MAX_CELLS 67108864LL
dvbm_status dvbm_cfl_dt_noalloc(const double* rho, const double* ux, const double* uy, const double* T,
                                long long n, double gamma, double R, double cfl, double h, void* stream,
                                double* dt_out);

#ifdef __cplusplus
}
#endif
#endif /* DVBM_H */
