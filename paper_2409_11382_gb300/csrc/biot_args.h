// biot_args.h -- argument blocks passed by value from the host runtime to the
// sm_103a kernels, and the launcher declarations.  Plain structs of pointers
// and scalars; no torch types anywhere.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

namespace biot {

enum { SIDE_BOTTOM = 0, SIDE_RIGHT = 1, SIDE_TOP = 2, SIDE_LEFT = 3 };
enum { BC_PERIODIC = 0, BC_SYMMETRY = 1, BC_DIRICHLET = 2, BC_NEUMANN = 3 };
enum { SWEEP_SMOOTH = 0, SWEEP_RESTRICT = 1 };
// Residual words of a measured sweep: [0] max|g - g**| and [1] max|g| over the
// populations as ordered FP64 bits (atomicMax), [2] the FP64 sum of (g - g**)^2
// over every population of every cell (atomicAdd of a double).
constexpr int RES_WORDS = 3;

// One elastic sweep on one multigrid level: either the under-relaxed smoother
// of eq. MG:smoother, g <- (1-gamma) g + gamma ELASTIC_STEP(g - r, F~ + F_*(g)),
// or the residual + restriction of Alg. 4 (r_c = R(g - ELASTIC_STEP(...))).
// T is the storage type of this level, TC that of the next coarser level.
template <typename T, typename TC>
struct SweepArgs {
    int nx, ny;                  // cells of this level
    const T *g;                  // iterate: 8 moment planes of nx*ny (ignored when zero_init)
    T *gout;                     // smoothed iterate (SMOOTH) or nullptr (RESTRICT)
    const T *glo;                // low parts of m_10, m_01 (double-float, finest FP32 level) or nullptr
    T *glo_out;                  // their update (SMOOTH) or nullptr
    const T *r;                  // residual right-hand side (coarse levels) or nullptr
    const T *Ft;                 // explicit force F~, 2 planes (finest level) or nullptr
    const TC *gc;                // coarse correction added on load (prolongation) or nullptr
    TC *rc;                      // restricted residual (RESTRICT) or nullptr
    T *H[4];                     // fullway bounce-back history per Dirichlet side: 3 per wall cell
    const double *prof[4];       // boundary data per side, 2 x (2n+1) (finest level) or nullptr
    int bc[4];                   // displacement boundary type per side
    int hist_valid;              // 0: first ELASTIC_STEP after a reset (use current populations)
    int zero_init;               // 1: the iterate is identically zero (first sweep of a coarse solve)
    int mode;                    // SWEEP_SMOOTH or SWEEP_RESTRICT
    double gamma;                // under-relaxation
    double om_s, om_d;           // relaxation rates of Tab. moments
    double lm;                   // lambda^ + mu^
    double coef_fstar;           // alpha^2 r / 2 (self-dependence force)
    double c0h;                  // c0 * h (lattice traction per unit traction)
    unsigned long long *resmax;  // [RES_WORDS] max|g - g**|, max|g| (ordered bits), sum (g - g**)^2 (double), or nullptr
    int rows;                    // strip height of the launch (0: the default choice)
    int ghosts;                  // 1: load and store the ghost moments 12, 21, 22 (tolerance mode)
    // the same coefficients, evaluated once on the host in the storage type:
    T k_fs;   // coef_fstar * dD/dm_s = -(alpha^2 r / 2) * 3 / (2 (3 lm + 1))
    // halves of the even post-collision combinations S*_p of Tab. moments:inverse
    // as linear forms of the moments (eq. moments:collision:22 for m_22):
    //   S*_0/2 = k_hs m_s + k_hd m_d,   S*_1/2 = k_hs m_s - k_hd m_d,
    //   S*_2/2 = k_hd m_11 + k_h22 m_s, S*_3/2 = k_h22 m_s - k_hd m_11
    T k_hs;   // (1 - om_s) / 4 + 1 / (2 (12 lm + 4))
    T k_hd;   // (1 - om_d) / 4
    T k_h22;  // -1 / (4 (12 lm + 4))
    T k_gam;  // gamma
    // 16-bit deviation store of the finest FP32 level (BIOT_FP32_DEV16 / _DEVBF16):
    // the moments m_11, m_s, m_d -- the state's deviation from the equilibrium
    // values of Tab. moments, which are zero for them -- held as 16-bit values
    // times the power of two dsc; everything else as in FP32
    int dev;           // 0: none, 1: FP16, 2: BF16
    const void *gd;    // 3 planes (m_11, m_s, m_d) of the iterate, or nullptr
    void *gd_out;      // 3 planes of the smoothed iterate (SMOOTH), or nullptr
    float dsc, dinv;   // scale of the stored values and its inverse
    int dev_full;      // 1: also store m_11, m_s, m_d in FP32 (planes 2-4 of gout), for
                       // the flow step and the read-outs: the last sweep of a solve
};

// One CTA's work item of a batched sweep launch: strip (bx, by) of TY rows of
// the sweep jobs[job].
struct SweepItem {
    int job, bx, by, ty;
};

// Storage kind of a sweep launch (bit flags).
enum { SWEEP_V_COARSE = 1, SWEEP_V_LO = 2, SWEEP_V_RESTRICT = 4, SWEEP_V_NOGHOST = 8, SWEEP_V_TILE = 16,
       SWEEP_V_DEV16 = 32, SWEEP_V_DEVBF16 = 64, SWEEP_V_SEGMENT = 128 };
// Tile sweeps: levels of at most SWEEP_TILE_CELLS cells (single instance); tile
// shape per storage type.  The fused flow step works on FLOW_TILE_X x FLOW_TILE_Y tiles.
constexpr long SWEEP_TILE_CELLS = 256L * 256L;
inline void sweep_tile_shape(bool fp64, int *tx, int *ty) { *tx = fp64 ? 8 : 32; *ty = fp64 ? 2 : 8; }
constexpr int FLOW_TILE_X = 32, FLOW_TILE_Y = 8;

// Explicit part of the effective source (eq. source:implicit) per cell.
template <typename T>
struct SexpArgs {
    int nx, ny;
    const double *D1, *D2;  // lattice divergence at t - dt and t - 2 dt
    const double *src;      // fluid source s (dimensional) or nullptr
    double *SE;             // output: dt s - (alpha/h)[(1-r)(D1 - D2) - r D1]
    double dt, a_over_h, r;
};

// Explicit force F~ of a time step (finest level).
template <typename T>
struct ForceArgs {
    int nx, ny;
    const T *f;           // flow populations, 9 planes
    const double *SE;     // explicit source (SexpArgs output)
    const double *fbody;  // body force f (2 planes, dimensional) or nullptr
    T *Ft;                // output, 2 planes
    int perx, pery;       // periodic in x / y
    double omega, alpha_h, c0h2;
    T k_m3w, k_mah;       // -3 omega and -alpha h in the storage type (host-evaluated)
    int central;          // 1: grad of sum_i f_i by the central difference of
                          //    eq. pressure:gradient:alternative instead of -3 omega sum_i f_i c_i
};

// Fused flow step (Alg. 3) and explicit force of the next time step: D(t) of
// the final elastic iterate, s' of eq. source:implicit, p^ = sum f + s'/2,
// collision with source, streaming with the pressure walls, then
// F~(t + dt) = c0 h^2 f - alpha h [ -3 omega sum_i f_i(t+dt) c_i + 1/2 grad^c s'_exp(t+dt) ]
// with s'_exp(t+dt) = dt s - (alpha/h)[(1-r)(D(t) - D(t-dt)) - r D(t)].
template <typename T>
struct FlowFusedArgs {
    int nx, ny;
    const T *f;           // flow populations, 9 planes
    T *fout;              // streamed populations, 9 planes
    const T *ms;          // m_s plane of the finest elastic state
    const double *D1;     // D(t - dt)
    const T *dBprev;      // D(t - dt) - D(t - 2 dt) as the previous flow step rounded it
    double *Dnew;         // D(t), into the buffer of D(t - 2 dt) (which no CTA reads)
    T *dAout;             // D(t) - D(t - dt) rounded, for the next flow step
    const double *src;    // fluid source (dimensional) or nullptr
    const double *fbody;  // body force (2 planes) or nullptr
    T *Ft;                // explicit force of the next step, 2 planes
    const double *pprof[4];
    int bc[4];            // pressure boundary type per side
    int perx, pery;       // periodic in x / y (displacement sides; equal to the pressure sides)
    double dt, a_over_h, r, kD, c0, c0h2;
    T k_om, k_src, k_m3w, k_mah;  // omega, 1 - omega/2, -3 omega, -alpha h
    T k_a1r, k_ar;                // (alpha/h)(1 - r), (alpha/h) r
    T k_c2;                       // (alpha/h) r kD, evaluated in FP64 on the host and rounded
};

// Physical fields of the current state.
template <typename T>
struct ReadoutArgs {
    int nx, ny;
    const T *g, *f, *Ft;
    const T *glo;             // low parts of the first moments (double-float) or nullptr
    const double *D1, *D2, *src;
    double *eta, *p, *sigma;  // outputs (any may be nullptr)
    int perx, pery;
    double dt, a_over_h, r;
    double kD;  // dD/dm_s = -3 / (2 (3 lm + 1)) (host-evaluated)
    // host-evaluated coefficients: F_* = c_axis (m_s(E) - m_s(W)) + c_diag ((m_s(NE) + m_s(SE))
    // - (m_s(NW) + m_s(SW))) (and rotated), p = (...) inv_c0, and the stress
    // sigma_11,22 = c_s m_s +- c_d m_d, sigma_12 = c_11 m_11
    double c_axis, c_diag, inv_c0, c_s, c_d, c_11;
};

// Initial populations of eqs. ICs / ICs:moments.
template <typename T>
struct InitArgs {
    int nx, ny;
    T *f, *g;
    T *glo;  // low parts of the first moments (double-float) or nullptr
    const double *src, *fbody;
    double dt, c0h2;
};

// Device-side stopping test of the tolerance mode (the V-cycle loop of a time
// step runs inside a CUDA-graph WHILE node; no host read per V-cycle).
struct StopState {
    long long total;   // V-cycles run by the device loop since creation
    int ne;            // V-cycles of the current time step
    int last_ne;       // V-cycles of the last finished time step
    int notconv;       // time steps that stopped at ne_max
    int diverged;      // 1 once a non-finite residual was met
    double last_res, last_gn;
};
struct StopArgs {
    const unsigned long long *resmax;  // ordered bits of max|g - g**| and max|g|
    StopState *st;
    double tol;
    int ne_max;
    int first;                 // 1: the first V-cycle of the time step
    unsigned long long cond;   // cudaGraphConditionalHandle of the WHILE node
};
cudaError_t launch_stop_test(const StopArgs &a, cudaStream_t s);

template <typename T, typename TC> cudaError_t launch_sweep_mom(const SweepArgs<T, TC> &a, cudaStream_t s);
// n consecutive smoothing sweeps of one small FP64 level (at most
// SWEEP_CHAIN_MAX x SWEEP_CHAIN_MAX cells) in one launch: sweep k reads the
// output of sweep k-1 (ping-pong between a.g and a.gout), only the first
// sweep may start from zero (a.zero_init), the bounce-back history is valid
// after it.  The result lies in a.g for even n and in a.gout for odd n.
constexpr int SWEEP_CHAIN_MAX = 8;
template <typename T, typename TC> cudaError_t launch_sweep_chain(const SweepArgs<T, TC> &a, int n, cudaStream_t s);
// The jobs of one batched sweep launch, passed as a kernel parameter -- so that,
// as in a single-instance launch, the arguments sit in constant memory rather
// than in shared memory and registers.  Job j owns the work items
// start[j] .. start[j+1]-1, laid out row by row with sx[j] strips (or tiles) per
// row; ty[j] is its strip height (strip form).
constexpr int BATCH_MAX_JOBS = 96;
template <typename T, typename TC>
struct BatchParams {
    int njobs;
    int start[BATCH_MAX_JOBS + 1];
    int sx[BATCH_MAX_JOBS];
    int ty[BATCH_MAX_JOBS];
    SweepArgs<T, TC> job[BATCH_MAX_JOBS];
};
// Batched sweep: one launch of P.start[P.njobs] work items of storage kind
// `variant` (SWEEP_V_* flags).
template <typename T, typename TC>
cudaError_t launch_sweep_batch(int variant, const BatchParams<T, TC> &P, cudaStream_t s);
// Segment of a V-cycle: consecutive sweeps of small coarse levels of one
// storage family (T = float: levels of tkind float/float and float/double;
// T = double: double/double) run by one thread-block cluster in one launch, a
// cluster barrier between the sweeps.  A program is the sweeps of one
// instance's segment; one launch runs one program per cluster (one cluster per
// instance of a batch).  Each level of a program has one record: its sweep
// arguments with the parts that change from sweep to sweep (iterate buffers,
// prolongation source, restriction target, flags) taken from the sweep's job
// word.  Everything is a kernel parameter, so a launch captured in a graph
// needs no device table.
struct SegLevel {
    union {
        SweepArgs<double, double> dd;
        SweepArgs<float, double> fd;
        SweepArgs<float, float> ff;
    } a;                  // base arguments; g, gout, gc, rc, zero_init, hist_valid, mode set per sweep
    const void *buf[2];   // the level's two iterate buffers
    const void *cbuf[2];  // the next coarser level's two iterate buffers (prolongation source)
    void *crc;            // the next coarser level's residual right-hand side (restriction target)
    int tkind;            // 0: double/double, 1: float/double, 2: float/float
    int pad;
};
// Job word of one sweep: bits 0-3 the level record (relative to the program's
// first), bit 4 restriction, bit 5 the parity of the input buffer, bit 6 zero
// iterate, bit 7 prolongation (add the coarser level's buffer cbuf[bit 8]), bit 9
// history valid.
enum { SEGJ_LEVEL = 15, SEGJ_RESTRICT = 16, SEGJ_CUR = 32, SEGJ_ZERO = 64, SEGJ_PROL = 128, SEGJ_CCUR = 256,
       SEGJ_HIST = 512 };
// The arguments of job word w from its level record: the host builds the
// words with this function's inverse and checks that it reproduces every sweep.
template <typename T, typename TC>
__host__ __device__ inline void seg_patch(SweepArgs<T, TC> &a, const SegLevel &L, unsigned w)
{
    const int cur = (w & SEGJ_CUR) ? 1 : 0;
    const bool rs = (w & SEGJ_RESTRICT) != 0;
    a.g = static_cast<const T *>(L.buf[cur]);
    a.gout = rs ? nullptr : const_cast<T *>(static_cast<const T *>(L.buf[1 - cur]));
    a.gc = (w & SEGJ_PROL) ? static_cast<const TC *>(L.cbuf[(w & SEGJ_CCUR) ? 1 : 0]) : nullptr;
    a.rc = rs ? static_cast<TC *>(L.crc) : nullptr;
    a.zero_init = (w & SEGJ_ZERO) ? 1 : 0;
    a.hist_valid = (w & SEGJ_HIST) ? 1 : 0;
    a.mode = rs ? SWEEP_RESTRICT : SWEEP_SMOOTH;
}
constexpr int SEG_MAX_PROGS = 32, SEG_MAX_LEVELS = 60, SEG_MAX_JOBS = 1200;
constexpr int SEG_CLUSTER = 8;    // CTAs per cluster (the portable maximum)
constexpr int SEG_MAX_TILES = 2 * SEG_CLUSTER;  // tiles of a level in a segment: at most 2 per CTA
struct SegParams {
    int nprog;
    int ghosts;                   // 1: the ghost moments are loaded and stored (tolerance mode)
    int lev0[SEG_MAX_PROGS + 1];  // program p: level records lev0[p] .. lev0[p+1]-1
    int job0[SEG_MAX_PROGS + 1];  // program p: jobs job0[p] .. job0[p+1]-1
    SegLevel lev[SEG_MAX_LEVELS];
    unsigned job[SEG_MAX_JOBS];
};
// One launch of P.nprog clusters of cs CTAs (1 <= cs <= SEG_CLUSTER); T selects
// the storage family of every job.
template <typename T>
cudaError_t launch_sweep_segment(const SegParams &P, int cs, cudaStream_t s);
// Resident CTAs of a batched sweep launch (sweep_slots) and of a
// single-instance strip launch (sweep_strip_slots) of this kind on the current
// device, and the strip geometry of the two strip kernels (output columns per
// strip: 156 of a 160-thread CTA for single instances, 124 of a 128-thread CTA
// in batches, whose levels are at most 512 cells wide).
template <typename T, typename TC> int sweep_slots(int variant);
template <typename T, typename TC> int sweep_strip_slots(int variant);
constexpr int SWEEP_STRIP_COLS = 156;
constexpr int BATCH_STRIP_COLS = 124;

// Largest strip height of a sweep launch (rows) unless biot_autotune chose one.
inline int sweep_rows_cap() { return 32; }

// Rows per strip of a sweep over nx x ny cells given `slots` resident CTAs:
// the grid fills whole waves of slots, with the first wave count whose strips
// are at most sweep_rows_cap() rows tall.  Even (restriction pairs rows), >= 2.
inline int sweep_strip_rows(int nx, int ny, int slots)
{
    const int strips_x = (nx + SWEEP_STRIP_COLS - 1) / SWEEP_STRIP_COLS;
    const int cap = sweep_rows_cap();
    if (slots < 1) slots = 1;
    for (int waves = 1;; waves++) {
        long nsy = ((long)waves * slots) / strips_x;
        if (nsy < 1) nsy = 1;
        long ty = (ny + nsy - 1) / nsy;
        ty += ty & 1;
        if (ty < 2) ty = 2;
        if (ty <= cap || waves >= 64) return (int)ty;
    }
}
template <typename T> cudaError_t launch_sexp(const SexpArgs<T> &a, cudaStream_t s);
template <typename T> cudaError_t launch_force(const ForceArgs<T> &a, cudaStream_t s);
template <typename T> cudaError_t launch_readout(const ReadoutArgs<T> &a, cudaStream_t s);
template <typename T> cudaError_t launch_flow_fused(const FlowFusedArgs<T> &a, cudaStream_t s);
// Batched flow steps: one work item per FLOW_TILE_X x FLOW_TILE_Y tile of an instance (job).
template <typename T>
cudaError_t launch_flow_fused_batch(const FlowFusedArgs<T> *jobs, const SweepItem *items, int n, cudaStream_t s);

// The finest-level state of an FP64 instance narrowed into an FP32 instance:
// the 8 moment planes rounded to FP32, the first moments m_10, m_01 as
// double-float (high part + low part of the remainder), the 9 flow population
// planes and the 2 planes of F~ rounded to FP32.
struct NarrowArgs {
    size_t np;
    const double *g64, *f64, *ft64;
    float *g32, *glo32, *f32, *ft32;
};
cudaError_t launch_narrow_state(const NarrowArgs &a, cudaStream_t s);
template <typename T> cudaError_t launch_init(const InitArgs<T> &a, cudaStream_t s);

// The 16-bit deviation store written from the FP32 moment planes 2-4 (m_11,
// m_s, m_d): after the initial state, the FP64 cold start's hand-over and a
// checkpoint load.  dev: 1 FP16, 2 BF16.
struct DevEncodeArgs {
    size_t np;
    const float *g;  // planes 2-4 of an FP32 moment buffer (8 planes of np)
    void *gd;        // 3 planes of 16-bit values
    float dsc;
    int dev;
};
cudaError_t launch_dev_encode(const DevEncodeArgs &a, cudaStream_t s);

}  // namespace biot
