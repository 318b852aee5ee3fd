/*
 * rlbm.h -- C ABI of the GB300 relativistic lattice Boltzmann (RLBM)
 * stream-collide library.
 *
 * The library advances a massless (ultra-relativistic) fluid on a periodic
 * 2D lattice with the method of Watson, "Two Dimensional Turbulence in a
 * Massless Fluid with a Relativistic Lattice Boltzmann Model"
 * (arXiv:2101.06187):
 *   - velocity space: the spherical "D3Q27" momentum node with one lattice
 *     node in z (Sec. 5), i.e. the 26 unit directions of the spherical
 *     degree-7 rule (faces 1/21, edges 4/105, corners 9/280); on a one-layer
 *     lattice the z-mirror pairs stream and collide alike, so the library
 *     stores 17 in-plane classes (their sums);
 *   - one step (Sec. 3.3, loop (b)-(e)): pull-streaming with linear
 *     interpolation from x - v_i (Sec. 3.2), moments T^{mu nu}
 *     (Eq. energyMomentumIntegral), the Landau-Lifshitz frame (eps, u^mu)
 *     (the eigenvalue problem closing Sec. 3.2), the truncated Juttner
 *     equilibrium (Eqs. rel_pdf_exp, rel_pdf_exp_coef, stressEnergyT with
 *     P = eps/3), Anderson-Witting relaxation (Eq. boltzmanneq_rel), and the
 *     projected driving term (Eq. forceTerm, App. B);
 *   - the stirring force of Sec. 5: random modes on a wavenumber shell,
 *     zero mean, redrawn every `redraw_period` steps.
 * Beyond the paper's one-layer lattice the same library runs the genuinely
 * two-dimensional massless gas on an 8-direction ring (RLBM_STENCIL_RING8_2D)
 * and the paper's node on a three-dimensional lattice (rlbm_create3d).
 * Lattice units: Delta x = Delta t = 1 (rlbm_opts.cfl sets Delta t / Delta x
 * otherwise); tau is the relaxation time in steps.
 * Signature (-,+,+,+).
 *
 * Conventions for every call:
 *   - Every call returns an rlbm_status.  After a CUDA error the handle's
 *     status is sticky: later calls return RLBM_ERR_CUDA until destroy.
 *     rlbm_last_error() gives a one-line message.
 *   - Host arrays are FP64, row-major (y, x), nx*ny elements, owned by the
 *     caller; device state is owned by the handle.
 *   - "Async" calls are ordered on the handle's CUDA stream and return
 *     before the GPU finishes; calls with host outputs synchronise it.
 *   - A handle is not thread-safe; use one handle per thread.
 */
#ifndef RLBM_H
#define RLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RLBM_API __attribute__((visibility("default")))
#else
#define RLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlbm rlbm_t;

typedef enum {
    RLBM_OK = 0,
    RLBM_ERR_ARG = 1,      /* invalid argument (size, tau, forcing band, NULL handle ...) */
    RLBM_ERR_ALLOC = 2,    /* device allocation failed */
    RLBM_ERR_CUDA = 3,     /* a CUDA call or kernel failed (sticky) */
    RLBM_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up */
    RLBM_ERR_NAN = 5,      /* a non-finite or non-physical (|v| >= 1, eps <= 0) state was found */
    RLBM_ERR_STATE = 6     /* call not valid in the handle's current state */
} rlbm_status;

/* Velocity stencil.
 * SPH26_SLAB: the paper's node (Sec. 3.1, Eq. 16, App. A): the 26-direction
 *   spherical rule on a one-layer (2D) lattice, stored as 17 in-plane
 *   classes; sound speed c_s^2 = 1/3 (P = eps/3).
 * RING8_2D: the genuinely two-dimensional massless gas the paper contrasts
 *   with its quasi-2D one (Sec. 3.1): 8 unit momenta in the plane at 45
 *   degree steps, weight 1/8, P = eps/2, c_s^2 = 1/2; the same step with the
 *   circle's angular polynomials (norms 1, 2, 4).  It runs the one node per
 *   thread kernel (GATHER), the packed-lane kernel (PACKED: FP32 compute
 *   with RLBM_LANDAU_FP32, nx even) or two steps per launch with the packed
 *   body (FUSED2, same conditions; its tiles run at a fixed 3 (256-thread)
 *   or 6 (128-thread) CTAs per SM whatever launch_budget says), at cfl 1 and
 *   fixed tau (eta_s 0), and is not available to ensembles.  rlbm_info_t.nclasses is 8 and the
 *   population arrays have 8 planes, in ring order k = 0..7 (angle k*45deg). */
typedef enum { RLBM_STENCIL_SPH26_SLAB = 0, RLBM_STENCIL_RING8_2D = 1 } rlbm_stencil;

/* Storage form of the populations.  All forms store the scaled deviation
 * q_c = (f_c - W_c eps0) / (W_c s) of each class from the rest equilibrium.
 * F64: FP64 storage and arithmetic.  F32: FP32 storage and arithmetic.
 * BF16 / F16: 16-bit storage, FP32 arithmetic. */
typedef enum { RLBM_F64 = 0, RLBM_F32 = 1, RLBM_BF16 = 2, RLBM_F16 = 3 } rlbm_dtype;

/* Precision of the per-node Landau-frame solve in the fused step of the
 * F32/16-bit forms (the F64 form always solves in FP64).  The solve is a
 * Newton iteration on the small deviation delta = E - eps, so FP32 keeps
 * full FP32 accuracy of eps and v.  RLBM_LANDAU_FP64 gives an FP64-accurate
 * frame: the FP64 Newton solve on the one-node-per-thread kernels, the FP32
 * frame refined by one double-float Newton step (residuals carried as pairs
 * of floats, within about 1e-12 of the FP64 solve) on the packed kernels.
 * rlbm_moments always returns an FP64-accurate frame (the refined one for
 * the F32/16-bit forms). */
typedef enum { RLBM_LANDAU_FP64 = 0, RLBM_LANDAU_FP32 = 1 } rlbm_landau;

/* Kernel variant of the fused step.  GATHER: one node per thread.
 * GATHER_VEC: a run of 4 nodes (2 for F64) along x per thread with 128-bit
 * (64-bit for 16-bit storage) loads and stores; needs nx divisible by that
 * run.  GATHER_VEC2: a run of 2 nodes (fewer registers); needs nx even.
 * PACKED: 2 nodes per thread whose arithmetic runs in packed FP32 lanes
 * (two nodes per instruction); FP32 compute with RLBM_LANDAU_FP32, nx even.
 * TMA: the packed body fed from shared memory: a persistent kernel whose
 * CTAs stage each 64 x 8 tile of all classes (with its halo) and the tile's
 * force through the tensor-memory accelerator, double-buffered, so the next
 * tile's copy overlaps the current tile's arithmetic; RLBM_F32 storage with
 * RLBM_LANDAU_FP32, nx even, SPH26_SLAB.  A wait on a tile copy that gives
 * up (bounded) makes the next synchronising call return RLBM_ERR_TIMEOUT.
 * TWOPASS: the packed body in two passes over the node pair's classes (the
 * first accumulates the moments pair by pair, the second gathers each pair
 * again and writes its update), so no thread keeps all 17 populations live
 * across the Landau solve: about half the registers, twice the resident
 * warps; same conditions as PACKED.
 * FUSED2: two time steps per launch (temporal blocking): each CTA updates
 * its tile plus a one-cell halo by one step into shared memory, then the
 * tile by a second step from there, so the state crosses HBM once per two
 * steps; the packed body, same conditions as PACKED.  Step counts are
 * split into launch pairs inside each forcing epoch (the force is constant
 * within one) and an odd remainder runs the packed single step; results
 * equal those of PACKED bit for bit.  block_x x block_y of the launch shape
 * is the output tile (64 x 16, 64 x 8, 32 x 16 or 128 x 8 nodes).
 * PACKED4: the packed body for 4 nodes per thread (two node pairs): each
 * class row around them is one aligned run of four values plus at most one
 * side value, half the loads per node of PACKED; results equal PACKED's bit
 * for bit.  Needs nx divisible by 4, CFL 1 and the one-layer lattice;
 * FP32 or 16-bit storage, either Landau precision (as PACKED).
 * The vector, TMA, two-pass and PACKED4 variants stream at CFL 1 only, the two-step
 * kernel at cfl <= 1 (halo 1), the packed kernel at any cfl (halo 2 above 1).
 * AUTO: the autotuned choice if one is cached for this lattice, else
 * GATHER. */
typedef enum {
    RLBM_KERNEL_AUTO = 0,
    RLBM_KERNEL_GATHER = 1,
    RLBM_KERNEL_GATHER_VEC = 2,
    RLBM_KERNEL_GATHER_VEC2 = 3,
    RLBM_KERNEL_PACKED = 4,
    RLBM_KERNEL_TMA = 5,
    RLBM_KERNEL_TWOPASS = 6,
    RLBM_KERNEL_FUSED2 = 7,
    RLBM_KERNEL_PACKED4 = 8
} rlbm_kernel;

/* Stirring force (Sec. 5).  Modes are the integer wavevectors k with
 * kmin <= |k| <= kmax (k = 0 excluded), one per Hermitian pair (ky > 0, or
 * ky = 0 and kx > 0), enumerated ky = 0..kmax, kx = -kmax..kmax.  In epoch e
 * = step / redraw_period, mode m draws Philox4x32-10 with counter
 * {e, m, 0, 0} (magnitude r*amp, phase) and {e, m, 1, 0} (direction), key
 * {seed & 0xffffffff, seed >> 32}; each word pair (a, b) becomes the double
 * (a * 2^21 + (b >> 11)) * 2^-53.  The force is
 *   F(x) = sum_m 2 r_m amp (cos th_m, sin th_m) cos(2 pi (kx x/nx + ky y/ny) + ph_m).
 * amp = 0 (or kmax = 0) disables forcing. */
typedef struct {
    int kmin;
    int kmax;
    double amp;
    uint64_t seed;
    int redraw_period; /* steps per epoch, >= 1 */
} rlbm_forcing;

/* Device allocator hooks.  alloc returns a device pointer of at least
 * `bytes` (aligned to 256 bytes) or NULL; free releases it.  NULL alloc
 * means cudaMalloc / cudaFree. */
typedef void *(*rlbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*rlbm_free_fn)(void *ptr, size_t bytes, void *ctx);

typedef struct {
    int dtype;            /* rlbm_dtype (default RLBM_F32) */
    int landau;           /* rlbm_landau (default RLBM_LANDAU_FP32) */
    int kernel;           /* rlbm_kernel (default RLBM_KERNEL_AUTO) */
    int use_graphs;       /* 1: replay chunks of two or more launches as CUDA graphs (default 1) */
    double eps0;          /* reference energy density of the deviation (default 1) */
    double scale;         /* s of the deviation; 0 = default: 1 (F64/F32, which accept only 1), 2^-6 (16-bit) */
    void *stream;         /* cudaStream_t the handle works on; NULL = legacy default stream */
    int device;           /* CUDA device ordinal; -1 = current device (default) */
    rlbm_alloc_fn alloc;  /* optional device allocator */
    rlbm_free_fn free;
    void *alloc_ctx;
    /* CFL number Delta t / Delta x (0 < cfl < 2, default 1): populations
     * stream cfl * v_i cells per step, interpolated bilinearly between the
     * cells around x - cfl v_i (Sec. 3.2, Sec. 5: Delta t = 0.05 on lattice
     * spacings 0.32, 0.16, 0.08, 0.04, i.e. cfl 0.156 ... 1.25).  cfl > 1
     * reaches two cells (halo 2) for the classes with cfl |v_i,a| > 1.
     * cfl != 1 runs the one-node-per-thread (GATHER) or the packed kernel
     * (PACKED), and cfl < 1 also the two-step kernel (FUSED2). */
    double cfl;
    /* eta/s > 0 switches the relaxation time to the paper's
     * tau_R = 5 (eta/s) / T with eps = 3 T^4 / pi^2 (Sec. 3.1-3.2), node by
     * node, in steps of dt (the physical time step); tau is then unused.
     * 0 (default): the constant tau of rlbm_create. */
    double eta_s;
    double dt;            /* time step for eta/s mode (default 1) */
    /* Failure-detection test hook (default 0).  1: the TMA kernel issues no
     * tile copies, so its bounded waits run out after one second, the
     * kernel leaves without touching memory it did not own, and the next
     * synchronising call returns RLBM_ERR_TIMEOUT (sticky); the state of
     * that step is undefined.  Nothing faults or hangs. */
    int test_unarmed_wait;
    /* Rounding of the 16-bit stores (rlbm_rounding).  RLBM_ROUND_NEAREST:
     * round to nearest even.  RLBM_ROUND_STOCHASTIC: round each stored value
     * up or down with probability given by its distance to the two
     * neighbours (the hardware's stochastic-rounding conversion), with random
     * bits hashed from the node, the class and the value itself, so runs
     * stay deterministic and checkpoints resume bitwise; nearest rounding's
     * error is a deterministic function of the smooth deviation field and
     * with BF16's 8-bit significand it shifts the time-averaged spectrum by
     * about 4%, stochastic rounding by a few tenths of a percent.  Needs
     * the packed kernels (PACKED, FUSED2) of the one-layer lattice.
     * RLBM_ROUND_DEFAULT (0): stochastic for BF16, nearest for FP16; for
     * ensembles nearest.  Ignored by the F32 and F64 forms. */
    int rounding;
} rlbm_opts;

typedef enum { RLBM_ROUND_DEFAULT = 0, RLBM_ROUND_NEAREST = 1, RLBM_ROUND_STOCHASTIC = 2 } rlbm_rounding;

typedef struct {
    int nx, ny, pitch;        /* lattice and row pitch (elements) of the device arrays */
    int nclasses;             /* stored classes: 17 (SPH26_SLAB) or 8 (RING8_2D) */
    int dtype;                /* rlbm_dtype */
    int kernel;               /* rlbm_kernel actually used */
    int block_x, block_y;     /* thread-block shape of the fused step */
    int nmodes;               /* forcing modes (0 = unforced) */
    int64_t step;             /* steps taken since init */
    double tau, eps0, scale;
    size_t bytes_per_node;    /* algorithmic HBM bytes per lattice update (a two-step launch moves the
                                 state once for two updates: half the single-step figure) */
    size_t device_bytes;      /* device memory held by the handle */
    const void *populations;  /* device pointer of the current state, [nclasses][nz][ny][pitch] of the storage type */
    int nz;                   /* layers: 1, or nz of a 3D lattice */
    int launch_budget;        /* register budget of the chosen launch: minimum resident blocks per SM
                                 asked of the compiler (256-thread blocks for the packed variants, except
                                 budget 5: 128; the launch's own blocks of at most 128 threads for PACKED4,
                                 3 or 4), CTAs per SM (TMA, FUSED2), else 1 */
    int steps_per_launch;     /* lattice steps one launch of the chosen kernel advances: 2 (FUSED2) or 1 */
} rlbm_info_t;

/* Fill *opts with the defaults listed above. */
RLBM_API void rlbm_opts_default(rlbm_opts *opts);

/* Create a lattice of nx x ny nodes (nx, ny >= 4, nx * ny <= 2^31,
 * ny <= 65535: the kernels put rows on the y dimension of the launch grid)
 * with relaxation time
 * tau > 1/2 (Eq. boltzmanneq_rel; eta = tau (eps + P)/5, Sec. 3.1) and
 * optional forcing (NULL = none; needs kmax < min(nx, ny)/2, amp >= 0,
 * 1 <= kmin <= kmax).  opts may be NULL (defaults).  The state starts as the
 * "flat" equilibrium eps = eps0, v = 0 (Sec. 5) at step 0.  Allocates all
 * device memory here; the step loop allocates nothing.
 * Errors: RLBM_ERR_ARG (bad size, tau, forcing, opts), RLBM_ERR_ALLOC,
 * RLBM_ERR_CUDA.  *out is NULL on error. */
RLBM_API rlbm_status rlbm_create(int nx, int ny, rlbm_stencil stencil, double tau, const rlbm_forcing *forcing,
                        const rlbm_opts *opts, rlbm_t **out);

/* Initialise with f = f_eq(eps, v) (step (a) of Sec. 3.3) from host FP64
 * fields eps (> 0) and 3-velocity vx, vy (|v| < 1), nx*ny each, row-major;
 * any NULL means eps = eps0 resp. v = 0.  Resets the step counter to 0.
 * The fields are copied from the caller's memory and checked on the device;
 * any entry with eps <= 0, |v| >= 1 or a non-finite value gives RLBM_ERR_ARG
 * and leaves the state unchanged.  Synchronous. */
RLBM_API rlbm_status rlbm_init_fields(rlbm_t *h, const double *eps, const double *vx, const double *vy);

/* Same, from device FP64 arrays (async on the handle's stream). */
RLBM_API rlbm_status rlbm_init_fields_device(rlbm_t *h, const double *d_eps, const double *d_vx, const double *d_vy);

/* Advance n >= 0 steps (async).  Each step: stream + collide + force, one
 * fused kernel; the force field is re-synthesised at each epoch start. */
RLBM_API rlbm_status rlbm_step(rlbm_t *h, int n);

/* Macroscopic fields seen by the next collision (post-stream moments and
 * Landau frame): eps and the 3-velocity v = u^i/u^0, nx*ny FP64 each on the
 * host (any may be NULL), and totals[3] = sum over nodes of (T^00, T^0x,
 * T^0y) in FP64 (may be NULL).  Synchronises.  Returns RLBM_ERR_NAN if any
 * node's solve failed (output entries of such nodes are NaN). */
RLBM_API rlbm_status rlbm_moments(rlbm_t *h, double *eps, double *vx, double *vy, double totals[3]);

/* Same into device FP64 buffers (nx*ny each; any may be NULL) and device
 * totals[3]; async, no NaN check. */
RLBM_API rlbm_status rlbm_moments_device(rlbm_t *h, double *d_eps, double *d_vx, double *d_vy, double *d_totals);

/* Energy spectrum E(n), n = 0..nshells-1 (Sec. 4): v_hat(k) = (1/(nx ny))
 * sum_x v(x) e^{-2 pi i (kx x/nx + ky y/ny)} of the 3-velocity field of
 * rlbm_moments, shell n = {k : |k| in [n - 1/2, n + 1/2)} with signed
 * integer wavenumbers, E(n) = 1/2 sum_shell |v_hat_x|^2 + |v_hat_y|^2.
 * Ek is a host array of nshells doubles.  Synchronises. */
RLBM_API rlbm_status rlbm_energy_spectrum(rlbm_t *h, int nshells, double *Ek);

/* Filtered RMS velocity (Sec. 5: the recorded velocities are filtered to
 * remove the driven band): sqrt of the lattice mean of |v_f|^2, where v_f
 * keeps only the Fourier modes of the 3-velocity with |k| < kf (signed
 * integer wavenumbers; kf = the lower edge of the driven band).  Computed on
 * the device from the same transform as rlbm_energy_spectrum (Parseval).
 * Synchronises. */
RLBM_API rlbm_status rlbm_filtered_velocity(rlbm_t *h, double kf, double *rms);

/* Time statistics of E(k) (App. C): rlbm_spectrum_sample adds the current
 * spectrum (nshells shells, as rlbm_energy_spectrum) to per-shell running
 * sums of E and E^2 kept on the device -- async, no host round trip, so a
 * long run can sample every N steps, N beyond the decorrelation time.
 * rlbm_spectrum_stats returns the time mean, the standard error of the mean
 * (sample standard deviation / sqrt(count); the reading of App. C's error
 * estimate for decorrelated samples) and the sample count (any output may
 * be NULL; synchronises).  rlbm_spectrum_reset clears the record.  All
 * samples of a record use the same nshells (else RLBM_ERR_STATE). */
RLBM_API rlbm_status rlbm_spectrum_sample(rlbm_t *h, int nshells);
RLBM_API rlbm_status rlbm_spectrum_stats(rlbm_t *h, int nshells, double *mean, double *sem, int *count);
RLBM_API rlbm_status rlbm_spectrum_reset(rlbm_t *h);

/* Decoded populations f_c = W_c (eps0 + s q_c) of the stored classes, host
 * FP64 [nclasses][ny][nx].  SPH26_SLAB class order: rest;
 * (1,0),(-1,0),(0,1),(0,-1); (a,0),(-a,0),(0,a),(0,-a);
 * (a,a),(-a,a),(a,-a),(-a,-a); (b,b),(-b,b),(b,-b),(-b,-b); a = 1/sqrt2,
 * b = 1/sqrt3.  RING8_2D: k = 0..7 at angle k*45 degrees.  Synchronises. */
RLBM_API rlbm_status rlbm_get_populations(rlbm_t *h, double *f);

/* Set the post-collision state from host FP64 populations in that layout
 * (encoded to the storage form; synchronous). */
RLBM_API rlbm_status rlbm_set_populations(rlbm_t *h, const double *f);

/* Force field of the current epoch (the one the next step uses), host FP64
 * nx*ny each.  Synchronises. */
RLBM_API rlbm_status rlbm_get_force(rlbm_t *h, double *Fx, double *Fy);

RLBM_API rlbm_status rlbm_get_info(rlbm_t *h, rlbm_info_t *info);

/* ---- Three-dimensional lattice ------------------------------------------
 * The paper's node (the 26-direction spherical rule, Landau frame,
 * equilibrium, Anderson-Witting relaxation and driving term of Sec. 3 and
 * App. A-B) on an nx x ny x nz periodic lattice: the three-dimensional model
 * the conclusion (Sec. 6) names as the next test.  All 26 directions are
 * stored (nclasses = 26), streamed by trilinear pull interpolation from
 * x - v_i (Sec. 3.2's linear interpolation in three dimensions, CFL 1);
 * the moments, frame and driving term keep every tensor component.  The
 * stirring force of Sec. 5 is carried to a 3D shell: integer k with
 * kmin <= |k| <= kmax, one mode per pair +-k (representative kz > 0, or
 * kz = 0 and ky > 0, or kz = ky = 0 and kx > 0, enumerated kz = 0..kmax,
 * ky = -kmax..kmax, kx = -kmax..kmax); mode m of epoch e draws
 * Philox(ctr = {e, m, 0, 0}, key = seed) -> magnitude r*amp, phase 2 pi u
 * and Philox(ctr = {e, m, 1, 0}, key) -> azimuth 2 pi u, mu = 2u - 1, the
 * direction (sqrt(1 - mu^2) cos az, sqrt(1 - mu^2) sin az, mu) uniform on
 * the sphere; F(x) = sum_m 2 r amp d cos(2 pi k.x/N + phi).  Populations
 * and fields are [.][z][y][x]; the device direction order is
 *   k = 0..2 faces (1,0,0), (0,1,0), (0,0,1); 3..8 edges (a,a,0), (a,-a,0),
 *   (a,0,a), (a,0,-a), (0,a,a), (0,a,-a); 9..12 corners (b,b,b), (b,b,-b),
 *   (b,-b,b), (b,-b,-b); k + 13 the opposite of k; a = 1/sqrt2, b = 1/sqrt3.
 * A 3D handle runs the one-node-per-thread kernel (GATHER, every storage
 * form) or the packed-lane kernel (PACKED: FP32 compute with
 * RLBM_LANDAU_FP32, nx even) at cfl 1 (eta_s allowed); rlbm_step,
 * rlbm_get/set_populations, rlbm_get_info, rlbm_autotune, rlbm_synchronize,
 * rlbm_last_error and rlbm_destroy apply to it, as do
 * rlbm_init_fields_device (v_z = 0) and the spectrum calls
 * (rlbm_energy_spectrum, rlbm_filtered_velocity, rlbm_spectrum_*), which
 * then bin |k| = (kx^2 + ky^2 + kz^2)^{1/2} over the three velocity
 * components; rlbm_init_fields, rlbm_moments[_device] and rlbm_get_force
 * return RLBM_ERR_STATE.  Errors as rlbm_create; nz >= 4, nx*ny*nz <= 2^31, nz <= 65535,
 * 2 kmax < min(nx, ny, nz). */
RLBM_API rlbm_status rlbm_create3d(int nx, int ny, int nz, double tau, const rlbm_forcing *forcing,
                                   const rlbm_opts *opts, rlbm_t **out);
/* f = f_eq of host FP64 fields, nx*ny*nz each ([z][y][x]; NULL: eps = 1,
 * v = 0), validated on the device first (RLBM_ERR_ARG, state untouched);
 * restarts the clock.  Synchronises. */
RLBM_API rlbm_status rlbm_init_fields3d(rlbm_t *h, const double *eps, const double *vx, const double *vy,
                                        const double *vz);
/* eps and v of the state the next collision sees (FP64 Landau frame), host
 * FP64 nx*ny*nz each (any may be NULL), and totals[4] = sum over nodes of
 * (T^00, T^0x, T^0y, T^0z) (may be NULL).  RLBM_ERR_NAN if a node has no
 * physical frame.  Synchronises. */
RLBM_API rlbm_status rlbm_moments3d(rlbm_t *h, double *eps, double *vx, double *vy, double *vz, double totals[4]);
/* Force of the current epoch, host FP64 nx*ny*nz each (any may be NULL). */
RLBM_API rlbm_status rlbm_get_force3d(rlbm_t *h, double *Fx, double *Fy, double *Fz);

/* Domain decomposition (no counterpart in the paper, which runs one
 * lattice per process; its step is local in space, so a lattice split into
 * slabs of rows with halo rows advances exactly like the whole lattice).
 * A slab is an ordinary lattice of ny_local + 2 H rows whose first and last
 * H rows are halo copies of the neighbouring slabs' edge rows, refreshed
 * before every H steps; the periodic pull inside the slab then gives the
 * interior rows exactly the whole lattice's values.
 * rlbm_set_force_frame: draw the stirring force (Sec. 5) in the frame of the
 *   whole nx_global x ny_global lattice, this lattice's node (x, y) being
 *   the global node (x + x0, y + y0) modulo the global sizes (y0 may be
 *   negative for halo rows).  The forcing shell must satisfy
 *   kmax < min(nx_global, ny_global)/2 (RLBM_ERR_ARG otherwise).  Not stored
 *   in checkpoints.  Synchronises.  RLBM_ERR_STATE for 3D lattices.
 * rlbm_halo_pack / rlbm_halo_unpack: copy rows [row, row + nrows) of the
 *   current state, every class with its pitch padding, to / from the
 *   caller's device buffer d_buf of nclasses * nrows * pitch elements of the
 *   storage type, laid out [class][row][pitch] (async on the handle's
 *   stream; RLBM_ERR_ARG for rows outside the lattice). */
RLBM_API rlbm_status rlbm_set_force_frame(rlbm_t *h, int nx_global, int ny_global, int x0, int y0);
RLBM_API rlbm_status rlbm_halo_pack(rlbm_t *h, int row, int nrows, void *d_buf);
RLBM_API rlbm_status rlbm_halo_unpack(rlbm_t *h, int row, int nrows, const void *d_buf);

/* Time every launch configuration of the fused step (kernel variant and
 * thread-block shape) for `reps` launches each (reps < 1: 20) on the
 * handle's lattice and keep the fastest per lattice step (a two-step launch
 * counts its time once for two steps).  The trial launches read the
 * current state and write only the spare buffer, so the simulation state is
 * unchanged.  The choice is cached per (nx, ny, dtype, landau, forced,
 * streaming mode) for handles created later in the process with
 * RLBM_KERNEL_AUTO (separately for each stencil).  Outputs may
 * be NULL.  Synchronises. */
RLBM_API rlbm_status rlbm_autotune(rlbm_t *h, int reps, int *kernel, int *block_x, int *block_y);

/* Pin the launch of the fused step to one of the configurations the
 * autotuner tries: kernel variant (rlbm_kernel, not AUTO), block_x x
 * block_y (the thread-block shape; the output tile for FUSED2) and
 * launch_budget (as reported in rlbm_info_t).  A handle created for a
 * fixed kernel accepts only that kernel.  One trial launch writes the spare
 * buffer (the state is unchanged).  RLBM_ERR_ARG if the configuration is
 * not on offer or does not fit the lattice (the handle stays usable).  Not
 * part of the paper: a service for reproducible timing and for tests that
 * cover every launch shape.  Synchronises. */
RLBM_API rlbm_status rlbm_set_launch(rlbm_t *h, int kernel, int block_x, int block_y, int launch_budget);

/* Allocation-free moments (no counterpart in the paper; a service for
 * callers that cannot allocate device memory, e.g. applications that run
 * on a memory budget fixed up front, loops that must not take the implicit
 * synchronisation of cudaMalloc, or hosts whose device memory belongs to
 * another framework's pool).  Computes what rlbm_moments_device computes
 * from a caller-owned population array of the paper's one-layer node:
 * stencil must be RLBM_STENCIL_SPH26_SLAB (anything else, e.g. the ring's
 * 8 planes or a 3D lattice's 26, is refused with RLBM_ERR_ARG: the call
 * cannot tell a layout from the pointer); d_q is the device state
 * [17][ny][pitch] of storage type `dtype` (for example
 * rlbm_info_t.populations and .pitch of a handle), eps0 and scale its
 * deviation parameters, and cfl the CFL number the lattice streams with
 * (rlbm_opts.cfl; 0 < cfl < 2; 1 for the default lattice), because the
 * moments are those of the streamed state and the pull depends on it.
 * d_eps, d_vx, d_vy (nx*ny FP64 each, any may be NULL) and d_totals (3
 * FP64, may be NULL) are caller-owned device outputs; d_bad (one int, may
 * be NULL) receives the number of nodes whose frame is not physical (their
 * outputs are NaN).  Async on `stream` (NULL = legacy default stream).
 * No device or host memory is allocated: the scratch (FP64 per-block
 * partial sums and the failed-node counter) lives in one static device
 * array of 1.5 MiB, held until the process exits by every GPU on which the
 * library's module is loaded.  With CUDA's default lazy module loading
 * that happens on the first use of the module on a device, which may
 * itself reserve device memory and synchronise: make the first call on a
 * device during set-up, before any stream capture (or load eagerly with
 * CUDA_MODULE_LOADING=EAGER).  That first call also looks the scratch
 * address up (cudaGetSymbolAddress) with that device current.  The lattice
 * must satisfy ceil(nx/32) * ceil(ny/8) <= RLBM_STATIC_MAX_BLOCKS (e.g.
 * 4096 x 4096); larger lattices get RLBM_ERR_ARG.  All calls on a device
 * share the scratch, which keeps the previous call's contents; each call
 * clears the counter and overwrites the partial sums it reads, so calls
 * that overlap on the GPU (different streams, no ordering) race: order
 * them on one stream.  Errors: RLBM_ERR_ARG, RLBM_ERR_CUDA (no handle, so
 * no message). */
#define RLBM_STATIC_MAX_BLOCKS 65536
RLBM_API rlbm_status rlbm_moments_static(int stencil, int dtype, const void *d_q, int nx, int ny, int pitch,
                                         double eps0, double scale, double cfl, double *d_eps, double *d_vx,
                                         double *d_vy, double *d_totals, int *d_bad, void *stream);

/* Checkpoint and resume (no counterpart in the paper).  A checkpoint holds
 * a header (lattice sizes, stencil, storage form, tau, eps0, scale, cfl,
 * eta/s, dt, the forcing parameters and the step counter) and the current
 * device state verbatim; because the stirring force is a counter-based
 * function of (seed, epoch), a handle created with the same arguments,
 * loaded from the checkpoint and stepped on reproduces the uninterrupted
 * run bitwise (same launch configuration).
 * rlbm_checkpoint_size: bytes a checkpoint of this handle takes.
 * rlbm_checkpoint_save: writes it into the caller's host buffer buf of len
 *   >= that size (synchronises; RLBM_ERR_ARG if len is short).
 * rlbm_checkpoint_load: restores state and step counter from buf; the
 *   header must match the handle's configuration exactly (RLBM_ERR_ARG
 *   otherwise, state untouched); the force of the restored epoch is
 *   re-synthesised by the next step.  Synchronises. */
RLBM_API rlbm_status rlbm_checkpoint_size(rlbm_t *h, size_t *bytes);
RLBM_API rlbm_status rlbm_checkpoint_save(rlbm_t *h, void *buf, size_t len);
RLBM_API rlbm_status rlbm_checkpoint_load(rlbm_t *h, const void *buf, size_t len);

/* Wait for all work queued on the handle's stream. */
RLBM_API rlbm_status rlbm_synchronize(rlbm_t *h);

/* ------------------------------------------------------------------------
 * Ensembles: many independent lattices (the paper's stirred runs, Sec. 5,
 * at several sizes, relaxation times and driven bands) advanced together.
 * Each member behaves exactly like an rlbm_t with the ensemble's options;
 * one step of the ensemble is a single launch over a flat list of tiles of
 * all members (a grid-stride loop, so the grid is sized to the GPU), and
 * chunks of two or more launches inside a forcing epoch replay as CUDA
 * graphs (a single launch goes directly).  All members
 * share one step counter, stream, storage form and the vector kernel (each
 * nx divisible by 4, or by 2 for F64). */
typedef struct rlbm_batch rlbm_batch_t;

typedef struct {
    int nx, ny;
    double tau;
    rlbm_forcing forcing; /* amp = 0: unforced member */
} rlbm_run_desc;

typedef struct {
    int nruns, dtype;
    int block_x, block_y, grid, ntiles; /* launch shape of the ensemble step */
    int64_t step;
    int64_t nodes;                      /* lattice nodes over all members */
    size_t bytes_per_step;              /* algorithmic HBM bytes per ensemble step (a two-step launch
                                           moves the state once for two steps: half the one-step figure) */
    size_t device_bytes;
    int kernel;                         /* body of the ensemble step: GATHER_VEC, PACKED or FUSED2 */
    int steps_per_launch;               /* 2 for the two-step body (FUSED2), else 1 */
} rlbm_batch_info_t;

/* Create nruns members (validation as rlbm_create, per member); all start at
 * rest at step 0.  opts->kernel picks the body of the ensemble step: AUTO
 * (the vector kernel until rlbm_batch_autotune chooses), GATHER_VEC, PACKED
 * or FUSED2 (FP32 compute with RLBM_LANDAU_FP32, nx even, fewer than 2^31
 * elements in a member's 17 planes); the autotuner then keeps that body.
 * Ensembles stream at CFL 1.  Errors: RLBM_ERR_ARG, RLBM_ERR_ALLOC,
 * RLBM_ERR_CUDA. */
RLBM_API rlbm_status rlbm_batch_create(int nruns, const rlbm_run_desc *runs, const rlbm_opts *opts,
                                       rlbm_batch_t **out);
/* The same call under the name rlbm_create_batch (identical arguments,
 * behaviour and errors), for callers that spell the constructors
 * rlbm_create*. */
RLBM_API rlbm_status rlbm_create_batch(int nruns, const rlbm_run_desc *runs, const rlbm_opts *opts,
                                       rlbm_batch_t **out);
/* Initialise member `run` as rlbm_init_fields does, at the ensemble's
 * current step (the step counter is shared and not reset). */
RLBM_API rlbm_status rlbm_batch_init_fields(rlbm_batch_t *b, int run, const double *eps, const double *vx,
                                            const double *vy);
/* Advance every member n steps (async). */
RLBM_API rlbm_status rlbm_batch_step(rlbm_batch_t *b, int n);
/* Per-member diagnostics, as the single-lattice calls (synchronise). */
RLBM_API rlbm_status rlbm_batch_moments(rlbm_batch_t *b, int run, double *eps, double *vx, double *vy,
                                        double totals[3]);
RLBM_API rlbm_status rlbm_batch_energy_spectrum(rlbm_batch_t *b, int run, int nshells, double *Ek);
RLBM_API rlbm_status rlbm_batch_get_populations(rlbm_batch_t *b, int run, double *f);
/* Time tile shapes and persistent grid sizes (multiples of the SM count,
 * or one block per tile) for the ensemble step and keep the fastest per
 * step; the bodies on offer are the vector kernel, the packed kernel and,
 * for FP32 compute with RLBM_LANDAU_FP32, two steps per launch through
 * shared memory (as RLBM_KERNEL_FUSED2, bit-identical to two packed steps;
 * block_x x block_y is then the tile in nodes).  The state is unchanged.
 * Outputs may be NULL.  Synchronises. */
RLBM_API rlbm_status rlbm_batch_autotune(rlbm_batch_t *b, int reps, int *block_x, int *block_y, int *grid);
RLBM_API rlbm_status rlbm_batch_get_info(rlbm_batch_t *b, rlbm_batch_info_t *info);
RLBM_API rlbm_status rlbm_batch_synchronize(rlbm_batch_t *b);
RLBM_API rlbm_status rlbm_batch_last_error(rlbm_batch_t *b, char *buf, size_t len);
/* Release the ensemble and all members (NULL-safe; synchronises). */
RLBM_API void rlbm_batch_destroy(rlbm_batch_t *b);

/* Copy the handle's last error message (NUL-terminated, truncated to len). */
RLBM_API rlbm_status rlbm_last_error(rlbm_t *h, char *buf, size_t len);

/* Release the handle and its device memory (NULL-safe; synchronises). */
RLBM_API void rlbm_destroy(rlbm_t *h);

RLBM_API const char *rlbm_status_string(rlbm_status s);

#ifdef __cplusplus
}
#endif
#endif /* RLBM_H */
