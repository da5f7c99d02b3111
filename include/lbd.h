/*
 * lbd.h -- C ABI of the GB300 (sm_103a) solver for the coupled hybrid
 * lattice-Boltzmann / finite-difference time step of Fadda, Gonnella, Lamura &
 * Tiribocchi, "Lattice Boltzmann study of chemically-driven self-propelled
 * droplets" (arXiv 1711.10984), Section 2.
 *
 * Model (Section 2.1): order parameter phi, surfactant concentration psi (the
 * paper's c), total density rho (the paper's n), free energy Eq. (1) with
 * f_GL = a/2 phi^2 + b/4 phi^4 and B(psi) = B0 + B1 psi.  One time step
 * (Sections 2.2-2.3) is: force F = -phi grad mu_phi - psi grad mu_psi (Eq. (14),
 * mu_phi Eq. (3), mu_psi Eq. (5)); D2Q9 BGK collide-and-stream with Guo forcing
 * (Eqs. (10)-(13)); the two-step finite-difference update of phi and psi
 * (Eqs. (16)-(19)) with the surfactant source A Theta(R - |r - r_P|) and sink
 * -gamma (psi - c0) of Section 2.1.
 *
 * Readings where the paper is silent or garbled (the same as the test oracle):
 * Eq. (12) with the factor 1/2 on the quadratic term; a phi mobility M in front
 * of lap mu_phi (the paper's runs have M = 1); advection in conservative
 * donor-cell flux form; psi grad mu_psi = grad psi + psi grad m with
 * m = (B1/2)|grad phi|^2 (no logarithm is evaluated); isotropic D2Q9
 * gradient and Laplacian stencils; order force -> LB -> advection ->
 * diffusion, with u^n = (sum f e + F/2)/rho of the same step driving the
 * advection; activity off for t < t_on, then gamma on and
 * A(t) = min(A0 (t - t_on), A_max).
 *
 * Lattice: periodic nx x ny, site (x, y) at index y*nx + x in every host array.
 *
 * Conventions for every function:
 *   - return 0 (LBD_OK) or a negative LBD_E* code; lbd_strerror() names the code
 *     and lbd_last_error() returns the context's last message;
 *   - host pointers are read or written only during the call and never kept;
 *   - device memory is owned by the context and released by lbd_destroy();
 *   - work is queued on the CUDA stream given to lbd_create() (NULL = legacy
 *     default stream); functions that return host data synchronise that stream;
 *   - a CUDA error is sticky for the context: later calls return LBD_ECUDA.
 */
#ifndef LBD_H
#define LBD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBD_OK 0
#define LBD_EINVAL (-1)      /* bad argument (message in lbd_last_error)          */
#define LBD_ENOMEM (-2)      /* device or host allocation failed                  */
#define LBD_ECUDA (-3)       /* a CUDA call or kernel launch failed               */
#define LBD_ENONFINITE (-4)  /* a NaN or Inf in the fields                        */
#define LBD_EUNSTABLE (-5)   /* B(psi) <= 0 or psi <= 0 somewhere (Section 4 notes
                                that the droplet breaks up when B(c) <= 0)        */
#define LBD_ETIMEOUT (-6)    /* reserved: no kernel of the library waits on a
                                flag or a peer, so no call returns it           */

#define LBD_FP64 0           /* populations, phi, psi in double                   */
#define LBD_FP32 1           /* populations stored as float deviations f_i - w_i,
                                phi and psi in float; reductions in double        */

#define LBD_FROZEN_U 1u      /* advection uses the uniform velocity (ux0, uy0)    */
#define LBD_BODY_FORCE 2u    /* add the constant body force (fx, fy) to F         */
/* Two resting plates at y = -1/2 and y = ny - 1/2, x stays periodic (the
 * channel of Section 4; Section 2.2 takes its walls from another paper and
 * Section 2.3 asks for n.grad mu_phi = n.grad mu_c = 0 there).  LB: halfway
 * bounce-back, f_i(x, t+1) = f*_{-i}(x, t) for a population that would cross a
 * plate.  FD: every stencil sees phi, psi and the fields derived from them
 * mirrored across each plate (row -1-k is row k, row ny+k is row ny-1-k), so
 * their normal derivatives vanish; no advective flux crosses a plate; source
 * disks do not wrap through the plates.  Needs ny >= 8; steps run on the
 * stripe and tiled launch shapes (not the column-pair one) and in batches; not
 * available to lbd_adjoint (LBD_EINVAL). */
#define LBD_WALLS 16u

#define LBD_MAX_SOURCES 64

typedef struct { int32_t nx, ny; } lbd_grid;

/* Source disk Theta(R - |r - r_P|) of Section 2.1, inclusive, periodic minimum
 * image; several disks combine as a union.  Centre (x, y) in lattice units. */
typedef struct { double x, y, R; } lbd_source;

typedef struct {
    double a, b, B0, B1;   /* free energy Eq. (1): a < 0 for coexistence, b >= 0   */
    double M;              /* phi mobility multiplying lap mu_phi (Eq. (18))       */
    double D;              /* surfactant diffusion, L(psi) = D psi (Eq. (4))       */
    double tau;            /* BGK relaxation time (> 1/2), Eq. (10)                */
    double gamma, c0;      /* sink -gamma (psi - c0), on for t >= t_on             */
    double A0, A_max;      /* source strength A(t) = min(A0 (t - t_on), A_max)     */
    int64_t t_on;          /* activation step of source and sink                   */
    double fx, fy;         /* body force (LBD_BODY_FORCE)                          */
    double ux0, uy0;       /* frozen advection velocity (LBD_FROZEN_U)             */
    uint32_t flags;        /* LBD_FROZEN_U | LBD_BODY_FORCE | LBD_WALLS            */
    int32_t precision;     /* LBD_FP64 or LBD_FP32                                 */
    int32_t n_src;         /* number of entries of src used (0..LBD_MAX_SOURCES)   */
    int32_t reserved;      /* must be 0                                            */
    lbd_source src[LBD_MAX_SOURCES];
} lbd_params;

/* Global diagnostics, accumulated in double on the device. */
typedef struct {
    double sum_rho, sum_phi, sum_psi;  /* totals; conserved by the scheme (Eqs. (2), (4), (7)) */
    double cm_x, cm_y;                 /* centre of mass of the phi >= 0 region (Section 4),
                                          each site at its minimum image about the reference */
    double mass_pos;                   /* sum of phi over phi >= 0                           */
    double min_B, min_psi;             /* min of B0 + B1 psi and of psi                      */
    int64_t nonfinite;                 /* count of non-finite phi, psi and population values */
} lbd_diag;

typedef struct lbd_ctx lbd_ctx;

/* Name of an error code; never NULL. */
const char *lbd_strerror(int code);

/* Last error message of ctx (empty string if none); valid until the next call. */
const char *lbd_last_error(const lbd_ctx *ctx);

/* Create a solver on the current CUDA device.  grid: nx, ny in [4, 2^20].
 * params: copied; tau > 1/2, b >= 0, n_src in [0, LBD_MAX_SOURCES], R >= 0,
 * precision LBD_FP64 or LBD_FP32.  stream: a cudaStream_t (or NULL).
 * Initial state: rho = 1, u = 0, phi = psi = 0 until lbd_set_fields(); t = 0.
 * Allocates about (22 words + reduction scratch) per site on the device. */
int lbd_create(const lbd_grid *grid, const lbd_params *params, void *stream, lbd_ctx **out);

/* Replace the model parameters (same precision as at creation). */
int lbd_set_params(lbd_ctx *ctx, const lbd_params *params);

/* Set the state from host arrays of nx*ny doubles: populations become the
 * equilibrium f_i^eq(rho, u) of Eq. (12) (rho NULL = 1, ux/uy NULL = 0); phi and
 * psi are required.  Returns LBD_ENONFINITE for a NaN/Inf, LBD_EUNSTABLE if
 * B0 + B1 psi <= 0 or psi <= 0, LBD_EINVAL if rho <= 0, for the first such site in
 * index order (named by lbd_last_error); nothing is changed then.  The arrays
 * are uploaded and checked on the device.  Synchronises. */
int lbd_set_fields(lbd_ctx *ctx, const double *rho, const double *ux, const double *uy,
                   const double *phi, const double *psi);

/* lbd_set_fields with host arrays of nx*ny floats: the values are widened to
 * double on the device (exactly), then everything is as for lbd_set_fields
 * (same state, same verdicts, state unchanged on a rejected upload).  Half the
 * host-to-device bytes; meant for FP32 contexts, whose state holds no more than
 * float precision anyway.  For an FP32 context without rho and u the values go
 * straight into the context's second buffer set and are checked there (no
 * staging); otherwise a float staging area of 5*nx*ny floats is allocated on
 * first use.  LBD_ENOMEM if an allocation fails.  Synchronises. */
int lbd_set_fields_f32(lbd_ctx *ctx, const float *rho, const float *ux, const float *uy,
                       const float *phi, const float *psi);

/* Advance nsteps >= 0 coupled time steps (asynchronous on the stream).  With
 * run-time checks on (lbd_set_check), returns LBD_ENONFINITE or LBD_EUNSTABLE
 * once a check has found the state broken (message in lbd_last_error); the
 * verdict stays until the state is replaced (lbd_set_fields,
 * lbd_set_populations, lbd_init_droplets), and steps are refused meanwhile. */
int lbd_step(lbd_ctx *ctx, int64_t nsteps);

/* Run-time checks (Section 4: the droplet breaks up when B(c) <= 0).  With
 * every > 0, lbd_step queues the diagnostics reduction after each step whose
 * count t is a multiple of every, on the context's stream and without a host
 * synchronisation (up to 4 checks in flight; a fifth waits for the oldest).
 * A check fails when a site holds a non-finite value (LBD_ENONFINITE) or when
 * min B(psi) <= 0 or min psi <= 0 (LBD_EUNSTABLE).  Verdicts are read as the
 * checks complete: at the next lbd_step and, waiting for all of them, at
 * lbd_synchronize.  every = 0 (the default) turns the checks off. */
int lbd_set_check(lbd_ctx *ctx, int64_t every);

/* Copy the fields at the current time to host arrays of nx*ny doubles (any may
 * be NULL).  u is Eq. (11): (sum_i f_i e_i + F/2) / rho with the force of the
 * current phi, psi.  Synchronises the stream. */
int lbd_get_fields(lbd_ctx *ctx, double *rho, double *ux, double *uy, double *phi, double *psi);

/* lbd_get_fields into host arrays of nx*ny floats (the values of lbd_get_fields
 * rounded to float; for an FP32 context rho and u are computed in float and phi,
 * psi are stored in float, so nothing is lost).  Half the device-to-host bytes.
 * For an FP32 context phi and psi are copied from the state on a second stream
 * that the context creates on first use, while rho and u are evaluated; the
 * float staging area of lbd_set_fields_f32 is allocated on first use for rho
 * and u.  NULL skips a field.  All arrays are complete when the call returns.
 * Synchronises. */
int lbd_get_fields_f32(lbd_ctx *ctx, float *rho, float *ux, float *uy, float *phi, float *psi);

/* One droplet of a seeded initial state (lbd_init_droplets). */
typedef struct {
    double x, y, R;       /* centre and radius                                      */
    double psi_mean;      /* psi inside the droplet                                 */
    double psi_noise;     /* half-width of the uniform noise added inside           */
    double gx, gy;        /* linear psi ramp inside: + gx (x - x0)/R + gy (y - y0)/R */
} lbd_droplet_init;

/* Seeded initial state built on the device (the initial conditions of
 * Sections 3-4: tanh droplets in a surfactant bath), at rest (rho = 1, u = 0,
 * f = f^eq):  phi = phi_eq tanh(max_k (R_k - r_k) / xi), phi_eq = sqrt(-a/b),
 * r_k the minimum-image distance to droplet k (round half to even); xi <= 0
 * takes xi0 = sqrt(2 (B0 + B1 psi_bg) / -a).  psi = psi_bg, except at sites with
 * max_k (R_k - r_k) > 0, which take psi_mean + psi_noise (2 u - 1) + ramp of the
 * droplet k attaining the maximum, u = uniform in [0, 1) of SplitMix64 draw
 * y*nx + x of the stream `seed` ((draw >> 11) * 2^-53; draw k is the published
 * finaliser of seed + (k+1) * 0x9E3779B97F4A7C15).  1 <= n <= LBD_MAX_DROPLETS.
 * LBD_EUNSTABLE when the psi range this can produce reaches psi <= 0 or
 * B(psi) <= 0; t is unchanged.  Synchronises. */
int lbd_init_droplets(lbd_ctx *ctx, int32_t n, const lbd_droplet_init *d, double psi_bg,
                      double xi, uint64_t seed);

/* As lbd_get_fields, into caller-owned DEVICE arrays of nx*ny elements of the
 * context's precision (double for LBD_FP64, float for LBD_FP32), site (x,y) at
 * y*nx + x; any pointer may be NULL.  Asynchronous on the context's stream: the
 * arrays hold the fields once the stream reaches this point.  The pointers are
 * not checked (they must be device memory of the context's device). */
int lbd_get_fields_device(lbd_ctx *ctx, void *rho, void *ux, void *uy, void *phi, void *psi);

/* Copy the pre-collision populations f_i(r, t) to a host array of 9*nx*ny
 * doubles, plane i (velocity e_i) at offset i*nx*ny; velocities in the order
 * (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).  Synchronises. */
int lbd_get_populations(lbd_ctx *ctx, double *f);

/* Restore pre-collision populations f_i(r, t) from a host array laid out as
 * lbd_get_populations writes it (9 planes of nx*ny doubles), e.g. to resume
 * from a checkpoint: lbd_set_fields (phi, psi), then lbd_set_populations,
 * then lbd_set_time.  The values are stored in the context's precision (for
 * FP64 they round-trip to within the rounding of f - w).  LBD_ENONFINITE for
 * a NaN or Inf.  Synchronises. */
int lbd_set_populations(lbd_ctx *ctx, const double *f);

/* Global diagnostics at the current time.  (ref_x, ref_y) in [0,nx) x [0,ny)
 * is the reference point for the minimum-image centre of mass (pass the
 * previous centre to follow a moving droplet).  *out is filled in every case;
 * the return value is LBD_ENONFINITE if a site holds a non-finite value,
 * LBD_EUNSTABLE if min B(psi) <= 0 or min psi <= 0, LBD_OK otherwise (these two
 * verdicts are not sticky).  The FP64 form sums in double; the FP32 form
 * accumulates each thread's sites in float with compensated (Neumaier)
 * summation and combines the threads in double.  Synchronises. */
int lbd_diagnostics(lbd_ctx *ctx, double ref_x, double ref_y, lbd_diag *out);

/* One droplet of the current state (Section 4). */
typedef struct {
    double x, y;    /* centre of mass sum phi r / sum phi over its sites with phi >= 0,
                       wrapped into [0,nx) x [0,ny) (y not wrapped with LBD_WALLS) */
    double mass;    /* sum of phi over those sites                                  */
    double ux, uy;  /* phi-weighted mean fluid velocity (Eq. 11) over those sites   */
    int64_t sites;  /* number of those sites                                        */
} lbd_droplet;

#define LBD_MAX_DROPLETS 64

/* Track n droplets (1 <= n <= LBD_MAX_DROPLETS) at the current time: every site
 * with phi >= 0 belongs to the nearest of the n reference points ref_xy
 * (host array x0, y0, x1, y1, ..., each inside the lattice; minimum image in x,
 * and in y unless LBD_WALLS; ties to the lower index), and out[k] (host array
 * of n) receives the centre of mass of Section 4 of droplet k, taken as its
 * reference plus the phi-weighted mean minimum-image displacement, with its
 * mass, mean velocity and site count.  A droplet with no site gets NaN centre
 * and velocity.  Pass the previous centres to follow moving droplets.
 * LBD_EINVAL for a bad n or reference.  Synchronises. */
int lbd_droplets(lbd_ctx *ctx, int32_t n, const double *ref_xy, lbd_droplet *out);

/* Squirmer fit of Section 4 (Eq. 21) for the n droplets drops[] (as returned by
 * lbd_droplets for the current state): the phi = 0 contour is sampled where
 * phi changes sign along a lattice link (x to x+1, y to y+1, none through a
 * plate), point and velocity interpolated linearly along the link, each point
 * belonging to the nearest droplet centre.  In the droplet frame (velocity
 * minus (ux, uy)), with theta measured from the swimming direction e = u/|u|
 * (e = x if the droplet is at rest) towards z x e, the polar velocity
 * u_theta(theta) at the points is fitted by least squares to
 * b1 sin(theta) + (b2 / 2) sin(2 theta), all points weighted equally.  b1[k],
 * b2[k] (host arrays of n) receive the coefficients, NaN with fewer than two
 * points or a singular fit, points[k] (may be NULL) the number of points;
 * beta = b2 / b1 classifies the swimmer (beta < 0 pusher, > 0 puller).
 * LBD_EINVAL for a bad n or a non-finite centre.  Synchronises. */
int lbd_squirmer(lbd_ctx *ctx, int32_t n, const lbd_droplet *drops, double *b1, double *b2,
                 int64_t *points);

/* Select the launch shape of the step: bx output columns x by output rows per
 * CTA.  bx 32 or 64: tiled kernel; bx 118 or 246: stripe-marching kernel (one
 * column per thread); bx 116: FP32 stripe-marching kernel with 16-byte
 * population staging (periodic lattices with nx % 4 == 0; not valid with
 * LBD_WALLS).  The stripe kernels cut each stripe into row segments of at most
 * by rows, shorter (down to by / 2) where that fills the GPU's resident CTA
 * slots evenly.  Shapes not compiled in, or not valid for the
 * context's precision and lattice, return LBD_EINVAL.  All shapes of one kernel give bit-identical results; different
 * kernels agree to rounding. */
int lbd_set_tile(lbd_ctx *ctx, int32_t bx, int32_t by);

/* The context's current launch shape (either pointer may be NULL). */
int lbd_get_tile(const lbd_ctx *ctx, int32_t *bx, int32_t *by);

/* Tile shapes compiled into the library: writes up to cap pairs into bx[], by[]
 * and returns how many shapes exist. */
int lbd_tiles(int32_t *bx, int32_t *by, int32_t cap);

/* Time every compiled tile shape on this context's current state (reps launches
 * each, CUDA events on the context's stream) and keep the fastest; the trial
 * launches write only the scratch half of the double-buffered state, so the
 * state and t are unchanged.  The chosen shape is returned in *bx, *by (either
 * may be NULL).  Synchronises. */
int lbd_autotune(lbd_ctx *ctx, int32_t reps, int32_t *bx, int32_t *by);

/* Gradient of the droplet displacement, by a hand-written adjoint of the
 * coupled step.  From the current state at time t0 the solver runs nsteps
 * steps, keeping a checkpoint every ckpt_every steps, and evaluates
 *     L = X_cm(t0 + nsteps) - X_cm(t0),
 * X_cm the x centre of mass of the phi >= 0 region (Section 4), each site at
 * its minimum image about ref_x in [0, nx).  The reverse sweep restores each
 * checkpoint, recomputes its segment and applies the transposed step (in the
 * context's precision; dL/dB1 summed in double) to give dL/dpsi(t0) (host
 * array of nx*ny doubles, may be
 * NULL) and dL/dB1, B1 the surfactant coupling of B(psi) = B0 + B1 psi.
 * The upwind directions of the advection and the phi >= 0 mask are those of
 * the forward run.  On return the context holds the state at t0 + nsteps.
 * Device memory: (nsteps/ckpt_every + ckpt_every + 2) states plus 74 values
 * of the context's precision and one double per site, allocated for the call.  LBD_FROZEN_U and LBD_WALLS are not
 * supported.
 * Synchronises. */
int lbd_adjoint(lbd_ctx *ctx, int64_t nsteps, int32_t ckpt_every, double ref_x, double *loss,
                double *dL_dpsi0, double *dL_dB1);

/* Diagnostics of a state that the caller keeps in its own device memory, for
 * callers that cannot allocate device memory through cudaMalloc: code whose
 * device memory all comes from another allocator (a framework's caching pool,
 * a fixed arena reserved at start-up) and loops that must not pay the device
 * synchronisation a cudaMalloc or cudaFree can cause.  It computes the same
 * quantities as lbd_diagnostics (the paper has no counterpart of this entry
 * point) and allocates nothing: its reduction scratch is a fixed array of
 * 43,856 bytes (608 blocks x 9 partial sums, a completion counter, 9 results)
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits.
 *
 * Inputs (device pointers, caller-owned, read only): g = the 9 population
 * planes stored as deviations f_i - w_i from the rest weights, plane i at
 * offset i*pitch*ny elements, site (x, y) at y*pitch + x (the order of the
 * sites within a plane does not matter for the totals); phi, psi with the
 * same site layout; element type double (LBD_FP64) or float (LBD_FP32).
 * Output: *out, a host struct, filled in whenever the reduction ran; the
 * return value is then LBD_ENONFINITE, LBD_EUNSTABLE or LBD_OK as for
 * lbd_diagnostics.  B0, B1: B(psi) = B0 + B1 psi for min_B.
 * Limits: 1 <= nx, ny <= 2^20, nx <= pitch <= 2^40 with 9 pitch ny < 2^52,
 * ref in [0,nx) x [0,ny), and g, phi, psi device memory of the current device
 * (or managed memory); anything else (a host pointer, another GPU's buffer)
 * returns LBD_EINVAL before any work.  Works on the current CUDA device and
 * the given stream (NULL = legacy default); synchronises it.
 *
 * Every call looks up the device address of the scratch array
 * (cudaGetSymbolAddress with the caller's device current; the lookup
 * allocates nothing), so the address stays right after cudaDeviceReset and
 * under a non-primary context.  The first call on a device may load the
 * library's device code there: make that first call before any stream
 * capture.  All calls share the one array: calls that overlap on the GPU
 * (different streams or host threads) race on it and must be serialised by
 * the caller.  Every scratch slot a call reads is written earlier in the same
 * call, except the completion counter of the FP32 reduction, which starts at
 * zero when the device code loads and which every call leaves at zero. */
int lbd_diagnostics_static(int32_t nx, int32_t ny, int64_t pitch, int32_t precision,
                           const void *g, const void *phi, const void *psi, double B0, double B1,
                           double ref_x, double ref_y, void *stream, lbd_diag *out);

/* ---- batches of independent instances ------------------------------------
 * A batch holds n independent lattices (each with its own size and
 * parameters, all of one precision) whose steps run together: every step is
 * one persistent launch of the stripe-marching kernel over a work list of
 * (instance, stripe, row segment) items, and lbd_batch_step replays chunks of
 * 100 such launches from a captured CUDA graph (the activity schedule is
 * evaluated on the device from a device-side step count).  Instance k behaves
 * exactly like a context of its own: same state layout, same results; the
 * instances may mix periodic lattices and lattices with plates (LBD_WALLS). */
typedef struct lbd_batch lbd_batch;

/* grids[k], params[k]: as for lbd_create (params[k].precision must agree).
 * stream NULL: the batch creates and owns a non-blocking stream (graph capture
 * needs a stream other than the legacy default stream). */
int lbd_batch_create(int32_t n, const lbd_grid *grids, const lbd_params *params, void *stream,
                     lbd_batch **out);
const char *lbd_batch_last_error(const lbd_batch *b);
/* as lbd_set_fields / lbd_get_fields / lbd_diagnostics for instance k */
int lbd_batch_set_fields(lbd_batch *b, int32_t k, const double *rho, const double *ux,
                         const double *uy, const double *phi, const double *psi);
int lbd_batch_get_fields(lbd_batch *b, int32_t k, double *rho, double *ux, double *uy,
                         double *phi, double *psi);
int lbd_batch_diagnostics(lbd_batch *b, int32_t k, double ref_x, double ref_y, lbd_diag *out);
/* Advance every instance by nsteps (asynchronous on the batch stream). */
int lbd_batch_step(lbd_batch *b, int64_t nsteps);
/* Launch shape of the batched kernel: bx 116 (FP32 16-byte staged stripe kernel
 * for the periodic instances, which must then be 4k wide; instances with plates
 * take 118-column stripes of the stripe kernel), 118 or 246, by 32, 64 or 128.
 * FP32 batches start at 116 x 64 where it is valid, the others at 118 x 64. */
int lbd_batch_set_tile(lbd_batch *b, int32_t bx, int32_t by);
/* Time the batched launch for each shape (reps launches each, no state change)
 * and keep the fastest; returns it in *bx, *by (may be NULL). */
int lbd_batch_autotune(lbd_batch *b, int32_t reps, int32_t *bx, int32_t *by);
int lbd_batch_synchronize(lbd_batch *b);
/* The batch's current launch shape (either pointer may be NULL). */
int lbd_batch_get_tile(const lbd_batch *b, int32_t *bx, int32_t *by);
int lbd_batch_get_time(const lbd_batch *b, int64_t *t);
void lbd_batch_destroy(lbd_batch *b);

/* Current step count t. */
int lbd_get_time(const lbd_ctx *ctx, int64_t *t);

/* Set the step count t (used by the activity schedule). */
int lbd_set_time(lbd_ctx *ctx, int64_t t);

/* Block until the context's queued work is done; reports any CUDA error, then
 * the verdict of the run-time checks (LBD_ENONFINITE, LBD_EUNSTABLE). */
int lbd_synchronize(lbd_ctx *ctx);

/* Measurement support (the paper has no counterpart): the FP64 FMA rate of the
 * current device in flop/s, timed with CUDA events over one launch of
 * iters rounds of 8 independent FMA chains in each of 256 threads x 8 blocks
 * per SM (2 flops per FMA), after an untimed warm-up launch; the FP64 form of
 * the coupled step is bound by this rate.  Allocates and frees a small output
 * buffer; runs on a stream of its own and synchronises it.  LBD_EINVAL for
 * iters < 1 or a NULL output. */
int lbd_fp64_peak(int32_t iters, double *flops_per_s);

/* Test hook: the nth device or pinned-host allocation the library makes from
 * now on (counted over all contexts and threads) fails as if the memory were
 * exhausted; nth = 0 clears the hook.  The call that meets the failure returns
 * LBD_ENOMEM and leaves its context as it was (lbd_create returns no context).
 * LBD_EINVAL for nth < 0.  The paper has no counterpart: it exists so that the
 * out-of-memory paths can be tested without exhausting a GPU. */
int lbd_debug_fail_alloc(int32_t nth);

/* Release all device memory of ctx (NULL is allowed). */
void lbd_destroy(lbd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBD_H */
