/*
 * biot.h -- C ABI of a single-GPU (sm_103a) solver for Biot's consolidation
 * model by the coupled lattice Boltzmann method of Lunowa & Wohlmuth,
 * "A lattice Boltzmann method for Biot's consolidation model of linear
 * poroelasticity" (arXiv 2409.11382).
 *
 * The problem (§2.1, eqs. elasticity, stress, flow, darcy) on the rectangle
 * (0, lx) x (0, ly):
 *     -div sigma + alpha grad p = f,   sigma = lambda div(eta) I + mu (grad eta + grad eta^T),
 *     d/dt (c0 p + alpha div eta) + div u = s,   u = -kappa grad p,
 * with p(0) = 0 and eta(0) = 0 (§3.6).  Each time step runs the pseudo-time
 * MRT LBM for elasticity inside its multigrid V-cycle (Alg. 4 with Alg. 2)
 * N_E times, then one SRT LBM step for the pressure (Alg. 3), coupled by the
 * centered update of eq. source:implicit -- together Alg. 5.
 *
 * Conventions for every entry point:
 *  - Return value: BIOT_OK (0) or a negative BIOT_ERR_* code; no exception or
 *    abort crosses the ABI.  biot_last_error() describes the last failure of
 *    the calling thread.
 *  - All pointers passed in are HOST pointers unless the name ends in
 *    "_device".  Inputs are copied before the call returns; the caller keeps
 *    ownership of every buffer it passes.
 *  - The handle owns all device memory it allocates; biot_destroy frees it.
 *  - A handle may be used by one host thread at a time.
 *  - Fields are stored y-major: value (x, y) of component c of an
 *    nx-by-ny field lives at [c * nx * ny + y * nx + x]; cell (x, y) has its
 *    centre at ((x + 1/2) h, (y + 1/2) h), h = lx / nx = ly / ny.
 */
#ifndef BIOT_GB300_H
#define BIOT_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BIOT_API __attribute__((visibility("default")))
#else
#define BIOT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------- */
#define BIOT_OK                 0
#define BIOT_ERR_INVALID_ARG   -1  /* a parameter violates a documented constraint */
#define BIOT_ERR_OOM           -2  /* device or host allocation failed */
#define BIOT_ERR_DIVERGED      -3  /* a non-finite residual was met (e.g. unstable coupling) */
#define BIOT_ERR_NOT_CONVERGED -4  /* a step reached ne_max V-cycles above tolerance (results kept) */
#define BIOT_ERR_CUDA          -5  /* a CUDA call failed; see biot_last_error() */
#define BIOT_ERR_TIMEOUT       -6  /* a bounded device-side wait gave up */
#define BIOT_ERR_NO_DEVICE     -7  /* no CUDA device is visible */

/* ---- storage precision of the populations --------------------------------- */
#define BIOT_FP64 0  /* all populations and arithmetic in FP64 (parity path) */
#define BIOT_FP32 1  /* FP32 elastic state and collisions on every multigrid level but
                        the coarsest, which is FP64 (Alg. 4 with l = 1); the
                        displacement moments of the finest level kept as double-float
                        (two FP32 planes); FP64 for residual norms and the divergence /
                        pressure accumulations of the coupling.  The solve at t = 0,
                        which starts from a zero iterate, runs on a temporary FP64 copy
                        of the problem for grids of at least 2048^2 cells (its state
                        then rounded into FP32 storage), and with double-float coarse
                        levels on smaller grids.  biot_params.options changes each of
                        these choices */
#define BIOT_FP32_COARSE64 2  /* BIOT_FP32 on the finest level (elastic state and flow
                                 populations), FP64 on every coarser multigrid level:
                                 the coarse-grid corrections are not rounded to FP32 */
#define BIOT_FP32_DEV16   3  /* BIOT_FP32, with the finest level's m_11, m_s, m_d -- the
                                 elastic state's deviation from its equilibrium (Tab. moments:
                                 their equilibria are zero) -- stored as IEEE FP16 values times a
                                 power of two fixed at creation from the boundary data, and
                                 collided in FP32.  Needs ne_fixed > 0 (the ghost moments 12, 21,
                                 22 are not stored) */
#define BIOT_FP32_DEVBF16 4  /* the same with bfloat16 storage */
/* In every precision the elastic state is stored as the MRT moments of the
 * populations (an exact change of basis, eqs. moments / moments:stress). */

/* ---- options of the FP32 paths (biot_params.options, bit flags) ------------
 * 0 selects the defaults described at BIOT_FP32.  They change rounding only:
 * the scheme, its iteration counts and its fixed point are the same.
 * BIOT_OPT_COLD_FP64 / _COLD_FP32 and BIOT_OPT_COARSE_LO_ALL / _OFF exclude
 * each other; BIOT_FP64 ignores all but BIOT_OPT_SEGMENTS. */
#define BIOT_OPT_COARSEST_STORAGE 1   /* the coarsest level in FP32 like the other coarse
                                         levels (faster on small instances) */
#define BIOT_OPT_COLD_FP64        2   /* the solve at t = 0 on an FP64 copy on every grid */
#define BIOT_OPT_COLD_FP32        4   /* ... on no grid (FP32 with double-float coarse levels) */
#define BIOT_OPT_COARSE_LO_ALL    8   /* double-float first moments on the FP32 coarse levels
                                         in every solve (default: in an FP32 solve at t = 0) */
#define BIOT_OPT_COARSE_LO_OFF   16   /* ... in no solve */
#define BIOT_OPT_SEGMENTS        32   /* a launch choice, honoured in every precision: the
                                         sweeps of the small coarse levels of a V-cycle (at most 16
                                         tiles each) as one thread-block-cluster launch per run of
                                         sweeps of one storage type (one cluster per instance in a
                                         batch) instead of one graph-launched kernel per sweep.
                                         Results are bitwise the same; on GB300 it is measured
                                         slower (graph launches cost about what the cluster
                                         barriers cost), so it is off by default */

/* ---- boundary condition types (§3.6) --------------------------------------- */
#define BIOT_PERIODIC  0  /* wrap-around streaming; must be set on both opposite sides
                             and for both fields */
#define BIOT_SYMMETRY  1  /* mirror (specular) reflection: a roller wall for the
                             displacement (normal displacement and shear stress vanish)
                             and a no-flux wall for the pressure */
#define BIOT_DIRICHLET 2  /* displacement: fullway bounce-back with a one-pseudo-step
                             delay, eq. BC:elasticity;  pressure: halfway
                             anti-bounce-back, eq. BC:pressure */
#define BIOT_NEUMANN   3  /* displacement: traction via halfway anti-bounce-back,
                             eq. BC:traction;  pressure: no-flow halfway bounce-back,
                             eq. BC:noFlow */
/* A population whose source lies beyond a corner follows the top/bottom rule,
 * except that a DIRICHLET or NEUMANN left/right wall wins over a SYMMETRY
 * top/bottom; two SYMMETRY walls reflect it twice. */

/* ---- sides ------------------------------------------------------------------ */
#define BIOT_BOTTOM 0  /* y = 0,  outward normal (0,-1) */
#define BIOT_RIGHT  1  /* x = lx, outward normal (1,0)  */
#define BIOT_TOP    2  /* y = ly, outward normal (0,1)  */
#define BIOT_LEFT   3  /* x = 0,  outward normal (-1,0) */

#define BIOT_MAX_LEVELS 16

/* Parameters of one instance (all dimensional, §2.1).  Lattice quantities
 * follow the scaling of §2.2 with L = h, T = dt, H = 1 (eps = h). */
typedef struct biot_params {
    int    nx, ny;     /* lattice cells of the finest grid (the paper's N_x, N_y);
                          both divisible by 2^(mg_levels-1) */
    double lx, ly;     /* domain size; lx/nx must equal ly/ny */
    double lambda, mu; /* Lame coefficients; mu > 0, lambda + mu > 0 */
    double alpha;      /* Biot-Willis coefficient, in [0, 1] */
    double c0;         /* specific storage coefficient, > 0 */
    double kappa;      /* permeability (viscosity-reduced), > 0 */
    double dt;         /* physical time step, > 0 */
    double r_coupling; /* ratio r of eq. source:implicit: 0 explicit, 0.5 centered, 1 implicit */
    int    mg_levels;  /* multigrid levels L >= 1 (Alg. 4) */
    int    K;          /* smoothing sweeps before and after the coarse correction, >= 1 */
    double gamma;      /* under-relaxation of eq. MG:smoother, in (0, 1] (paper: 0.75) */
    double tol;        /* stop the V-cycles of a step once the residual
                          max|g - ELASTIC_STEP(g)| <= tol * max(1, max|g|) (ne_fixed <= 0) */
    int    ne_max;     /* cap on V-cycles per step in tolerance mode */
    int    ne_fixed;   /* > 0: exactly this many V-cycles per step, MG(ne_fixed, K) */
    int    precision;  /* BIOT_FP64, BIOT_FP32, BIOT_FP32_COARSE64, BIOT_FP32_DEV16 or BIOT_FP32_DEVBF16 */
    int    options;    /* BIOT_OPT_* flags (0: defaults) */
    /* Multigrid cycles and pressure gradient (0 everywhere: the paper's V-cycle
     * of Alg. 4 and eq. pressure:gradient).  The paper leaves W- and F-cycles and
     * full multigrid to future work (§5); they are built here as the usual
     * definitions applied to Alg. 4's correction problem.  Batches take V-cycles
     * only. */
    int    cycle;      /* BIOT_CYCLE_V, BIOT_CYCLE_W (the coarse correction by two cycles
                          in succession) or BIOT_CYCLE_F (by an F-cycle, then a V-cycle) */
    int    fmg;        /* 1: the first cycle of every elastic solve is a full-multigrid
                          cycle: the finest defect restricted level by level, the coarsest
                          level solved, and each finer level started from the prolongated
                          solution below it and given one cycle */
    int    pgrad;      /* 0: eq. pressure:gradient (flux moment of f); 1: the central
                          difference of eq. pressure:gradient:alternative (§3.4) */
    int    K_level[BIOT_MAX_LEVELS];  /* smoothing sweeps before and after the coarse correction on
                          the level j steps below the finest (j = 0: the finest level); 0 takes
                          K.  biot_autotune_sweeps chooses them */
} biot_params;
#define BIOT_CYCLE_V 0
#define BIOT_CYCLE_W 1
#define BIOT_CYCLE_F 2

/* Boundary data of one side.  Profiles are sampled at the 2n+1 arc positions
 * k*h/2, k = 0..2n, along the side (n = nx for bottom/top, ny for left/right;
 * the arc runs in +x or +y), so that even k are cell faces and odd k cell
 * centres; a bounce-back rule evaluated at x + c/2 (eqs. BC:pressure,
 * BC:elasticity, BC:traction) reads the sample at its wall crossing. */
typedef struct biot_side {
    int eta_type;              /* BIOT_PERIODIC / SYMMETRY / DIRICHLET / NEUMANN */
    int p_type;                /* BIOT_PERIODIC / SYMMETRY / DIRICHLET / NEUMANN */
    const double *eta_profile; /* 2 x (2n+1), [component][k]: displacement eta_D (DIRICHLET)
                                  or traction t = sigma n (NEUMANN); NULL = zero */
    const double *p_profile;   /* 2n+1: pressure p_D (DIRICHLET); NULL = zero */
} biot_side;

typedef struct biot_stats {
    int     last_ne;        /* V-cycles of the last elastic solve */
    double  last_res;       /* residual max|g - ELASTIC_STEP(g)| over the populations of the finest
                               level, measured in its last smoothing sweep (FP64) */
    long    total_cycles;   /* V-cycles since creation */
    int     notconv_steps;  /* steps that hit ne_max */
    int     diverged;       /* 1 once a non-finite residual was met */
    long    nstep;          /* physical time steps taken */
    double  t;              /* current time nstep*dt */
    double  omega;          /* flow relaxation rate, eq. pressure:rate (lattice units) */
    double  omega_s, omega_d; /* elastic relaxation rates, Tab. moments */
    long    kernel_launches;  /* kernels launched since creation */
    size_t  device_bytes;     /* device memory held */
    double  last_res_l2;      /* (sum over cells and populations of (g - ELASTIC_STEP(g))^2)^(1/2) of the
                                 sweep that measured last_res, summed in FP64 (fixed V-cycle counts
                                 leave out the ghost moments 12, 21, 22, as in last_res) */
} biot_stats;

typedef struct biot_ctx *biot_handle;

/* Validate the parameters (constraints above; a PERIODIC side must face a
 * PERIODIC side for both fields) and create an instance at t = 0 with zero body force
 * and source.  Allocates all device memory of the multigrid hierarchy on the
 * current CUDA device.  On failure *out is NULL. */
BIOT_API int biot_create(const biot_params *p, const biot_side sides[4], biot_handle *out);

/* Free all device and host memory of the instance.  NULL is accepted. */
BIOT_API int biot_destroy(biot_handle h);

/* Launch all further work of the instance on this CUDA stream (a
 * cudaStream_t passed as void*); NULL selects the instance's own stream. */
BIOT_API int biot_set_stream(biot_handle h, void *cuda_stream);

/* Replace the solid body force f (2 x nx x ny, dimensional, NULL = zero) and
 * the fluid source s (nx x ny, NULL = zero) of eqs. elasticity / flow.  They
 * act from the next elastic solve on; before the first step they also enter
 * the initial populations of eqs. ICs / ICs:moments. */
BIOT_API int biot_set_sources(biot_handle h, const double *f_body, const double *s);

/* Replace the boundary data of one side (same layout as biot_side; the types
 * are fixed at creation).  NULL sets zero data.  The data act from the next
 * elastic solve on (the next step queued after this call); the current state
 * keeps the data it was solved with.  The arrays are copied into page-locked
 * staging before the call returns; the upload runs after the steps already
 * queued, without waiting for them. */
BIOT_API int biot_set_side_profile(biot_handle h, int side, const double *eta_profile, const double *p_profile);

/* Run n iterations of the time loop of Alg. 5 (elastic solve at t, flow step
 * to t + dt), followed by the elastic solve at the new time, so that
 * biot_read_u and biot_read_p refer to the same t.  Returns BIOT_OK,
 * BIOT_ERR_NOT_CONVERGED (a step hit ne_max; the state is kept) or
 * BIOT_ERR_DIVERGED (the state is no longer meaningful). */
BIOT_API int biot_step(biot_handle h, int n);

/* Pipelined stepping.  biot_step_async queues the same n steps as biot_step
 * on the instance's stream and returns without waiting for them (BIOT_OK, or
 * an error found while queueing them).  biot_sync waits for everything queued
 * on the instance -- steps and biot_read_async copies -- and reports the steps
 * queued since the last report: BIOT_OK, BIOT_ERR_NOT_CONVERGED or
 * BIOT_ERR_DIVERGED, as biot_step would have.  biot_set_side_profile and
 * biot_read_async do not wait for queued steps either, so a loop of
 * set_side_profile / step_async / read_async keeps the GPU busy while the host
 * prepares the next step.  In tolerance mode without CUDA graphs the V-cycle
 * loop needs the host after every V-cycle, and biot_step_async then runs as
 * biot_step. */
BIOT_API int biot_step_async(biot_handle h, int n);
BIOT_API int biot_sync(biot_handle h);

/* Step until t = round(T/dt)*dt (T not before the current time). */
BIOT_API int biot_solve_to(biot_handle h, double T);

/* Displacement eta (2 x nx x ny) of eq. displacement and its time. */
BIOT_API int biot_read_u(biot_handle h, double *eta, double *t_out);

/* Pressure p (nx x ny) of eq. pressure, p = p^ / c0, and its time. */
BIOT_API int biot_read_p(biot_handle h, double *p, double *t_out);

/* Stress (3 x nx x ny: sigma_11, sigma_12, sigma_22) of eqs. displacement /
 * moments:bared. */
BIOT_API int biot_read_stress(biot_handle h, double *sigma);

/* Read-out that overlaps later steps.  biot_read_async forms the same fields
 * as biot_read_u / biot_read_p / biot_read_stress at the current time (each
 * of eta, p, sigma may be NULL; same layouts) on the instance's stream, then
 * copies them to the host buffers on a copy stream of its own and returns
 * without waiting for the copy.  Steps issued afterwards run while it is in
 * flight: the fields are formed before them in stream order, so they are
 * those of the time returned in *t_out.
 * - The host buffers belong to the library until biot_read_wait returns: the
 *   caller neither reads nor frees them before.  Page-locked buffers (e.g.
 *   cudaHostAlloc) make the copy asynchronous; pageable ones are accepted, and
 *   then the copy may block the calling thread.
 * - At most two reads are in flight; a third waits on the device for the
 *   oldest one's copy before it overwrites that device staging buffer.  The
 *   two staging buffers (3 FP64 planes each, 6 with sigma) are allocated at
 *   the first call and held until biot_destroy.
 * - Errors: BIOT_ERR_INVALID_ARG (null handle, all three outputs NULL), the
 *   step errors of a pending solve, BIOT_ERR_OOM, BIOT_ERR_CUDA.
 * biot_read_wait blocks until every read issued so far has reached the host
 * (BIOT_OK also when none is in flight). */
BIOT_API int biot_read_async(biot_handle h, double *eta, double *p, double *sigma, double *t_out);
BIOT_API int biot_read_wait(biot_handle h);

BIOT_API int biot_stats_get(biot_handle h, biot_stats *out);

/* Static description of an error code, and the last error of this thread. */
BIOT_API const char *biot_error_string(int code);
BIOT_API const char *biot_last_error(void);

/* Kernel instrumentation: when enabled, every launch of the finest-level
 * smoothing sweep is bracketed by CUDA events on the instance's stream.
 * biot_sweep_timing_get synchronises the stream and returns the summed
 * device time (ms) and the number of such launches since the last enable. */
BIOT_API int biot_sweep_timing(biot_handle h, int enable);
BIOT_API int biot_sweep_timing_get(biot_handle h, double *ms_total, long *launches);

/* Checkpoint / resume.  biot_save writes the resumable state (flow populations,
 * finest elastic state, explicit force, divergence history, time and counters)
 * into a host buffer of biot_checkpoint_size bytes; biot_load restores it into an
 * instance created with the same grid, levels and precision (boundary data and
 * sources are not part of the checkpoint).  Stepping on from a loaded checkpoint
 * gives bitwise the result of the uninterrupted run. */
BIOT_API int biot_checkpoint_size(biot_handle h, size_t *bytes);
BIOT_API int biot_save(biot_handle h, void *buf, size_t size);
BIOT_API int biot_load(biot_handle h, const void *buf, size_t size);

/* Autotune the launch shape of the multigrid sweeps: for every level run as
 * strips (more than 256^2 cells) and both sweep modes (smoothing, residual +
 * restriction), time candidate strip heights (4 .. 96 rows) on a scratch
 * instance of the same shape (allocated for the call, then freed) and keep
 * the fastest for this instance.  Strip heights do not change the arithmetic:
 * results are bitwise the same as untuned.  rows_out / ms_out (may be NULL)
 * receive 2 values per level (smoothing, restriction; level 0 = coarsest) for
 * the first max_levels levels: the rows chosen (0 = not tuned) and the mean
 * time of one sweep (ms). */
BIOT_API int biot_autotune(biot_handle h, int *rows_out, double *ms_out, int max_levels);

/* Autotune the smoothing sweeps per multigrid level (biot_params.K_level).
 * On a scratch instance of the same problem (allocated for the call, then
 * freed), V-cycles run from the zero iterate of the solve at t = 0; for a
 * candidate set of per-level counts the tuner measures the time of a V-cycle
 * (CUDA events) and the residual contraction per V-cycle rho (the stopping-test
 * norm of consecutive V-cycles), and it minimises the time to reduce the
 * residual by a factor e, time / -ln(rho), by coordinate descent over the
 * levels with counts from 1 to 8.  The counts found are written to
 * K_out[0 .. L-1] (level j below the finest at K_out[j]) and, with apply != 0,
 * set for this instance (its captured graphs are dropped).  Changing the counts
 * changes the iteration, not its fixed point: with a fixed number of V-cycles
 * per step the results change within the solver's convergence; the FP64 oracle
 * takes the same counts.  Needs fixed V-cycles or tolerance mode alike;
 * batches take the counts through biot_params.K_level at creation. */
BIOT_API int biot_autotune_sweeps(biot_handle h, int apply, int *K_out, double *rho_out, double *ms_per_cycle_out);

/* ---- batched execution ----------------------------------------------------------
 * Many independent instances (different grids, materials, boundary data) advanced
 * together.  Each physical step of every instance is Alg. 5 exactly as in
 * biot_step -- same kernels, same arithmetic, bitwise the same result as the
 * instance stepped alone (FP64; FP32 within rounding, the kernel forms can
 * differ) -- but the launches of all instances are regrouped: the V-cycles are
 * aligned at the coarsest level and each phase is one work-list launch per
 * storage kind whose CTAs process strips or tiles of sweeps of different
 * instances; the flow steps are one work-list launch; the whole step is one
 * CUDA graph.
 * Instances need a fixed number of V-cycles (ne_fixed > 0) and equal K and
 * ne_fixed.  The batch owns its instances: read them with biot_read_u / _p /
 * _stress / biot_stats_get through biot_batch_instance, do not destroy them or
 * move them to another stream, and do not step them with biot_step. */
typedef struct biot_batch_s *biot_batch;

/* Create `count` instances (params[i], sides[4*i .. 4*i+3]); all device memory is
 * allocated here.  On failure *out is NULL and the message names the instance. */
BIOT_API int biot_batch_create(int count, const biot_params *params, const biot_side *sides, biot_batch *out);
BIOT_API int biot_batch_destroy(biot_batch b);
BIOT_API int biot_batch_size(biot_batch b, int *count);
/* Handle of instance i (owned by the batch). */
BIOT_API int biot_batch_instance(biot_batch b, int i, biot_handle *out);
/* n physical steps of every instance (plus the trailing elastic solve, as biot_step). */
BIOT_API int biot_batch_step(biot_batch b, int n);
/* As biot_step_async / biot_sync, for every instance of the batch. */
BIOT_API int biot_batch_step_async(biot_batch b, int n);
BIOT_API int biot_batch_sync(biot_batch b);
/* Kernel launches since creation, per captured step, and strip work items per step. */
BIOT_API int biot_batch_stats_get(biot_batch b, long *kernel_launches, long *launches_per_step,
                                  long *work_items_per_step);
/* biot_read_async for every instance of the batch in one call: eta[i], p[i],
 * sigma[i] are instance i's host buffers (an array may be NULL, and so may an
 * entry, which skips that field of that instance); t_out, if not NULL, receives
 * count times.  The same ownership rules as biot_read_async; the reads of
 * earlier instances stay issued when a later one fails.  biot_batch_read_wait
 * waits for every instance's reads. */
BIOT_API int biot_batch_read_async(biot_batch b, double *const *eta, double *const *p, double *const *sigma,
                                   double *t_out);
BIOT_API int biot_batch_read_wait(biot_batch b);

/* ---- serving: continuous batching of solve requests ---------------------------
 * A scheduler thread admits submitted solves in arrival order while the
 * device-memory budget (biot_estimate_bytes per request) and the resident-slot
 * limit allow, and keeps each admitted instance resident on its own CUDA stream.
 * It polls those streams without blocking: an instance whose queued work has
 * completed gets its next four time steps at once, so the residents' kernels
 * overlap on the GPU and none waits for another.  A finished instance
 * is read out (eta and p at the end time, as biot_read_u / biot_read_p) into host
 * memory and freed at once, which admits the next request.  Every request runs
 * the same kernels as biot_create + biot_solve_to, so its result does not depend
 * on what else is resident.  Times are seconds since biot_server_create. */
typedef struct biot_server_s *biot_server;

#define BIOT_REQ_QUEUED  0
#define BIOT_REQ_RUNNING 1
#define BIOT_REQ_DONE    2
#define BIOT_REQ_FAILED  3

typedef struct biot_request_info {
    int    state;         /* BIOT_REQ_* */
    int    status;        /* BIOT_OK or the error code of a failed request */
    double t_submit, t_start, t_done;
    int    nx, ny;
    long   steps;         /* physical steps to the end time */
    size_t device_bytes;  /* admission estimate */
} biot_request_info;

typedef struct biot_server_stats {
    int    queued, peak_resident;
    size_t used_bytes, peak_bytes;
    long   ticks, graph_launches;  /* ticks: scheduler passes that launched or finished work */
    long   graphs_reused;          /* step graphs taken over from a finished request of the same
                                      shape (cudaGraphExecUpdate) instead of instantiated */
} biot_server_stats;

/* Device bytes an instance with these parameters holds (allocation plus the
 * read-out buffer); validates the parameters. */
BIOT_API int biot_estimate_bytes(const biot_params *p, const biot_side sides[4], size_t *bytes);
/* Start a server on the current device with a device-memory budget and at most
 * max_resident instances resident at once. */
BIOT_API int biot_server_create(size_t mem_budget_bytes, int max_resident, biot_server *out);
/* Queue a solve to time T (copies all inputs); BIOT_ERR_OOM if it alone exceeds
 * the budget. */
BIOT_API int biot_server_submit(biot_server s, const biot_params *p, const biot_side sides[4], double T, uint64_t *id);
BIOT_API int biot_server_poll(biot_server s, uint64_t id, biot_request_info *info);
/* Block until the request is done (BIOT_OK), failed (its error code) or the
 * timeout expires (BIOT_ERR_TIMEOUT). */
BIOT_API int biot_server_wait(biot_server s, uint64_t id, double timeout_s);
/* Copy the result of a finished request: eta 2 x nx x ny, p nx x ny (either may
 * be NULL) and its time. */
BIOT_API int biot_server_fetch(biot_server s, uint64_t id, double *eta, double *p, double *t_out);
/* Forget a finished request (its result buffers are freed). */
BIOT_API int biot_server_release(biot_server s, uint64_t id);
BIOT_API int biot_server_stats_get(biot_server s, biot_server_stats *out);
/* Stop the scheduler; requests still queued or resident are dropped. */
BIOT_API int biot_server_destroy(biot_server s);

/* ---- read-out without device allocation ------------------------------------
 * The paper has no counterpart; this is a library convenience.
 *
 * biot_read_u stages the displacement in a device buffer that the instance
 * allocates with cudaMalloc on its first read.  Some callers cannot allocate at
 * that point: a process whose device memory is already handed out to another
 * allocator (a framework's caching pool, or other instances filling the GPU),
 * or a latency-critical loop that must not take the allocator's implicit
 * device-wide synchronisation.  biot_read_u_noalloc returns the same values as
 * biot_read_u but stages them in a fixed array that is part of the library
 * image (BIOT_NOALLOC_MAX_CELLS * 2 doubles = 4 MiB of device memory, held by
 * every GPU that loads the library until the process exits); it calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *  - Grids with more than BIOT_NOALLOC_MAX_CELLS cells (nx * ny) are rejected
 *    with BIOT_ERR_INVALID_ARG before any device work.
 *  - The first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture.
 *  - Every call shares the one array (per device).  The read-out kernel
 *    overwrites every value it copies back, so nothing needs clearing, but calls
 *    from different host threads whose GPU work overlaps (e.g. two instances on
 *    two streams) race on it: serialise them.
 *  - Like biot_read_u it may first run the pending elastic solve of the instance
 *    and returns after the values are in *eta (2 x nx x ny, host memory).  The
 *    one solve that would allocate -- the solve at t = 0 of an FP32 instance
 *    that runs it on an FP64 copy (grids of at least 2048^2 cells, or
 *    BIOT_OPT_COLD_FP64) -- is refused with BIOT_ERR_INVALID_ARG: step the
 *    instance or read it once with biot_read_u first.
 *  - The instance's device must be the current device (BIOT_ERR_INVALID_ARG
 *    otherwise); the array of that device is used. */
#define BIOT_NOALLOC_MAX_CELLS 262144
BIOT_API int biot_read_u_noalloc(biot_handle h, double *eta, double *t_out);

#ifdef __cplusplus
}
#endif
#endif /* BIOT_GB300_H */
