// biot_capi.cu -- host runtime and C ABI of the GB300 Biot solver.
//
// Owns the device memory of one instance (multigrid hierarchy, flow
// populations, coupling history) and drives Alg. 5: per time step the explicit
// force, N_E V-cycles of Alg. 4 built from fused elastic sweeps, then the
// flow step of Alg. 3.  Every arithmetic step runs in the sm_103a kernels of
// sweep_mom.cuh and field_kernels.cuh; this file only sequences launches and
// copies, and evaluates the per-instance coefficients once on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <new>
#include <string>
#include <vector>

#include "biot.h"
#include "biot_args.h"

using namespace biot;

namespace biot {
// A sweep prepared for a batched launch: its storage kind and arguments.
struct SweepJob {
    int tkind;    // 0: double/double, 1: float/double, 2: float/float
    int variant;  // SWEEP_V_* flags
    int level;
    SweepArgs<double, double> dd;
    SweepArgs<float, double> fd;
    SweepArgs<float, float> ff;
    int seg = -1;  // SWEEP_V_SEGMENT: index of its program among the instance's recorded ones
};
// The program of one segment of a V-cycle (sweep_segment.cuh): the records of
// its levels and one job word per sweep.
struct SegProg {
    int fam = 1;  // storage family: 0 double (tkind 0), 1 float (tkinds 1 and 2)
    int cs = 1;   // CTAs per cluster: the most tiles of any of its levels, at most SEG_CLUSTER
    std::vector<SegLevel> lev;
    std::vector<unsigned> job;
};
// A flow step prepared for a batched launch.
struct FlowRec {
    int fp64;
    FlowFusedArgs<float> f;
    FlowFusedArgs<double> d;
};
template <typename T> FlowFusedArgs<T> &flow_args(FlowRec &r);
template <> FlowFusedArgs<float> &flow_args<float>(FlowRec &r) { return r.f; }
template <> FlowFusedArgs<double> &flow_args<double>(FlowRec &r) { return r.d; }
template <typename T, typename TC> SweepArgs<T, TC> &job_args(SweepJob &j);
template <> SweepArgs<double, double> &job_args<double, double>(SweepJob &j) { return j.dd; }
template <> SweepArgs<float, double> &job_args<float, double>(SweepJob &j) { return j.fd; }
template <> SweepArgs<float, float> &job_args<float, float>(SweepJob &j) { return j.ff; }
}  // namespace biot

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                         \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return fail(BIOT_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));    \
    } while (0)

constexpr int MAX_LEVELS = 16;

// Double-float first moments on the FP32 coarse levels.  A V-cycle starts each
// coarse level from zero, so their low parts carry nothing from one V-cycle to
// the next and can be switched per solve.  They matter where the coarse
// corrections are displacement-sized: in the solve at t = 0, which starts from a
// zero iterate (a cold start); a warm-started step's corrections are of the
// size of the change over one time step.  Default: the cold-start solve only;
// BIOT_OPT_COARSE_LO_ALL takes them in every solve, BIOT_OPT_COARSE_LO_OFF never.
enum { COARSE_LO_OFF = 0, COARSE_LO_COLD = 1, COARSE_LO_ALL = 2 };
int coarse_lo_mode(const biot_params *p)
{
    if (p->options & BIOT_OPT_COARSE_LO_ALL) return COARSE_LO_ALL;
    if (p->options & BIOT_OPT_COARSE_LO_OFF) return COARSE_LO_OFF;
    return COARSE_LO_COLD;
}

// Precision of the coarsest level of the FP32 path: FP64 (default; Alg. 4 with
// l = 1 is the FP64 part of the mixed-precision multigrid), or FP32 like the
// other coarse levels with BIOT_OPT_COARSEST_STORAGE.
bool coarsest_fp64(const biot_params *p)
{
    return (p->options & BIOT_OPT_COARSEST_STORAGE) == 0;
}

// Smoothing sweeps of level index l (0 = coarsest) of an L-level hierarchy:
// the per-level count for the level L-1-l below the finest, or K.
int sweeps_of(const biot_params *p, int l)
{
    const int k = p->K_level[p->mg_levels - 1 - l];
    return k > 0 ? k : p->K;
}

struct Level {
    int nx = 0, ny = 0;
    size_t np = 0;
    bool fp64 = true;
    int rows[2] = {0, 0};  // strip height per sweep mode chosen by biot_autotune (0: default)
    void *g[2] = {nullptr, nullptr};
    void *glo[2] = {nullptr, nullptr};  // low parts of m_10, m_01 (finest FP32 level)
    void *gd[2] = {nullptr, nullptr};   // 16-bit deviation store: m_11, m_s, m_d (finest level, dev > 0)
    int cur = 0;
    void *r = nullptr;
    void *H[4] = {nullptr, nullptr, nullptr, nullptr};
    int hist_valid = 0;
};

// Executable step graphs of finished server requests, kept for the next
// request of the same shape: capturing a step is cheap, instantiating its graph
// is not, and cudaGraphExecUpdate moves a captured graph's arguments into an
// existing executable graph of the same topology.  Used by the server's
// scheduler thread only.
struct GraphKey {
    int nx, ny, L, K, ne_fixed, precision, options, cycle, fmg, pgrad;
    int bc[8];
    int K_level[BIOT_MAX_LEVELS];
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};
struct GraphCache {
    struct Entry {
        GraphKey key;
        int par;
        cudaGraphExec_t exec;
    };
    static constexpr size_t CAP = 64;
    std::deque<Entry> entries;
    std::atomic<long> reused{0}, rejected{0};  // read by biot_server_stats_get
    // an executable graph of this key and parity, updated to the captured graph g
    cudaGraphExec_t take(const GraphKey &key, int par, cudaGraph_t g)
    {
        for (auto it = entries.begin(); it != entries.end(); ++it) {
            if (it->par != par || !(it->key == key)) continue;
            cudaGraphExec_t e = it->exec;
            entries.erase(it);
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(e, g, &info) == cudaSuccess) {
                reused++;
                return e;
            }
            cudaGetLastError();
            cudaGraphExecDestroy(e);
            rejected++;
            return nullptr;
        }
        return nullptr;
    }
    void put(const GraphKey &key, int par, cudaGraphExec_t e)
    {
        entries.push_back({key, par, e});
        while (entries.size() > CAP) {
            cudaGraphExecDestroy(entries.front().exec);
            entries.pop_front();
        }
    }
    ~GraphCache()
    {
        for (Entry &e : entries) cudaGraphExecDestroy(e.exec);
    }
};

}  // namespace

struct biot_ctx {
    biot_params P{};
    int bc_eta[4]{}, bc_p[4]{};
    double *eta_prof[4]{}, *p_prof[4]{};  // device copies of the boundary data (finest level)
    // biot_set_side_profile stages the caller's data in page-locked memory and
    // uploads it in stream order: two slots per side, each reused once its
    // previous upload has run (an event), so the call never waits for the steps
    double *prof_stage[4][2] = {};
    cudaEvent_t prof_ev[4][2] = {};
    int prof_slot[4] = {};
    int notconv_reported = 0;  // notconv_steps when biot_step / biot_sync last reported
    double h = 0, lam = 0, mu = 0, kap = 0, omega = 0, om_s = 0, om_d = 0, lm = 0;
    int L = 0;
    bool fp32 = false;  // FP32 state (finest and middle levels)
    int dev = 0;        // finest level's deviation store: 0 none, 1 FP16, 2 BF16
    float dsc = 1.f, dinv = 1.f;  // its scale (a power of two) and inverse
    Level lv[MAX_LEVELS];
    void *f[2]{};
    int fcur = 0;
    double *D1 = nullptr, *D2 = nullptr, *SE = nullptr;
    void *dB[2] = {nullptr, nullptr};  // D(t - dt) - D(t - 2 dt) as rounded by the last flow step; by flow parity
    void *Ft = nullptr;
    double *src = nullptr, *fbody = nullptr;
    bool has_src = false, has_fbody = false;
    double *out = nullptr;  // readout scratch, 6 planes
    // biot_read_async: two device staging buffers (3 or 6 FP64 planes), a copy
    // stream, and per buffer the events "fields formed" and "copy done"
    double *aout[2] = {nullptr, nullptr};
    int aout_planes[2] = {0, 0};
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t aready[2] = {nullptr, nullptr}, acopied[2] = {nullptr, nullptr};
    bool ainflight[2] = {false, false};
    int aslot = 0;
    unsigned long long *resmax = nullptr;      // device [RES_WORDS]
    unsigned long long *resmax_host = nullptr; // pinned [RES_WORDS]
    // device-side stopping test (tolerance mode inside graphs)
    StopState *stop = nullptr;                 // device
    StopState *stop_host = nullptr;            // pinned mirror, copied at the end of each step
    bool pending_stop = false;                 // the mirror holds counters not yet applied
    long long stop_total_seen = 0;
    int stop_notconv_seen = 0;
    cudaStream_t aux_stream = nullptr;         // captures the WHILE node's body
    cudaStream_t stream = nullptr, own_stream = nullptr;
    long nstep = 0;
    bool solved = false, initialized = false, pending_res = false;
    bool cold_solve = false;  // the current elastic solve starts from a zero iterate (t = 0)
    bool cold64 = false;      // FP32 instance: run the solve at t = 0 on an FP64 shadow (cold_start_fp64)
    bool se_stale = true;   // SE must be recomputed from D1, D2 before k_force
    bool ft_fresh = false;  // the last flow step computed F~ of the next elastic solve
    // statistics
    int last_ne = 0;
    double last_res = 0;
    double last_res_l2 = 0;  // sqrt of the FP64 sum of squared residuals of that sweep
    long total_cycles = 0;
    int notconv_steps = 0;
    int diverged = 0;
    long launches = 0;
    size_t bytes = 0;
    // CUDA graphs of one time step (flow step + elastic solve) in fixed-cycle
    // mode, one per parity of the flow ping-pong buffer
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long graph_launches[2] = {0, 0};
    bool use_graphs = true;
    long epoch = 0;  // bumped whenever captured launch arguments become stale
    // instrumentation of the finest-level smoothing sweep
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::vector<void *> allocs;
    // measure the residual in the V-cycle being issued (set by elastic_solve)
    bool measure_cycle = true;
    // record mode (batched execution): sweeps are appended here instead of launched
    std::vector<biot::SweepJob> *rec = nullptr;
    std::vector<biot::FlowRec> *frec = nullptr;  // record mode: flow steps appended here
    std::vector<biot::SegProg> *segrec = nullptr;  // record mode: programs of the recorded segments
    bool in_seg = false;  // recording the sweeps of a segment (seg_vcycle)
    bool batched = false; // an instance of a batch (its steps are recorded and merged)
    // Allocation source of a server's instance: the server's stream-ordered
    // pool, so that freeing the instance synchronises only its own stream
    // (cudaFree would wait for every resident instance); its two pinned host
    // mirrors are lent from the server's arena for the same reason.
    cudaMemPool_t pool = nullptr;
    bool host_lent = false;
    int device = -1;  // the CUDA device current at biot_create (owns every buffer)
    GraphCache *gcache = nullptr;  // a server's cache of executable step graphs (see GraphCache)
};

namespace {

// What a server lends an instance it creates (see biot_ctx::pool).
struct Lend {
    cudaMemPool_t pool;
    unsigned long long *resmax_host;  // RES_WORDS values
    StopState *stop_host;
};

int dev_alloc(biot_ctx *h, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return BIOT_OK;
    cudaError_t e = h->pool ? cudaMallocFromPoolAsync(p, bytes, h->pool, h->stream) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BIOT_ERR_OOM : BIOT_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    h->bytes += bytes;
    e = cudaMemsetAsync(*p, 0, bytes, h->stream);
    if (e != cudaSuccess) return fail(BIOT_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    return BIOT_OK;
}

int side_cells(const biot_ctx *h, int side)
{
    return (side == BIOT_BOTTOM || side == BIOT_TOP) ? h->P.nx : h->P.ny;
}

int check_params(const biot_params *p, const biot_side *s)
{
    if (!p || !s) return fail(BIOT_ERR_INVALID_ARG, "null parameter block");
    if (p->mg_levels < 1 || p->mg_levels > MAX_LEVELS) return fail(BIOT_ERR_INVALID_ARG, "mg_levels out of range");
    if (p->nx < 1 || p->ny < 1) return fail(BIOT_ERR_INVALID_ARG, "grid must have at least one cell");
    const int div = 1 << (p->mg_levels - 1);
    if (p->nx % div || p->ny % div) return fail(BIOT_ERR_INVALID_ARG, "nx, ny must be divisible by 2^(mg_levels-1)");
    if ((long long)p->nx * p->ny > (1LL << 31)) return fail(BIOT_ERR_INVALID_ARG, "grid too large");
    if (!(p->lx > 0) || !(p->ly > 0)) return fail(BIOT_ERR_INVALID_ARG, "domain size must be positive");
    const double hx = p->lx / p->nx, hy = p->ly / p->ny;
    if (std::fabs(hx - hy) > 1e-12 * hx) return fail(BIOT_ERR_INVALID_ARG, "cells must be square (lx/nx == ly/ny)");
    if (!(p->mu > 0) || !(p->lambda + p->mu > 0)) return fail(BIOT_ERR_INVALID_ARG, "need mu > 0 and lambda + mu > 0");
    if (!(p->alpha >= 0 && p->alpha <= 1)) return fail(BIOT_ERR_INVALID_ARG, "alpha must lie in [0, 1]");
    if (!(p->c0 > 0) || !(p->kappa > 0) || !(p->dt > 0)) return fail(BIOT_ERR_INVALID_ARG, "c0, kappa, dt must be positive");
    if (!(p->r_coupling >= 0 && p->r_coupling <= 1)) return fail(BIOT_ERR_INVALID_ARG, "r_coupling must lie in [0, 1]");
    if (p->K < 1) return fail(BIOT_ERR_INVALID_ARG, "K must be >= 1");
    for (int j = 0; j < BIOT_MAX_LEVELS; j++)
        if (p->K_level[j] > 64) return fail(BIOT_ERR_INVALID_ARG, "K_level entries must not exceed 64");
    if (!(p->gamma > 0 && p->gamma <= 1)) return fail(BIOT_ERR_INVALID_ARG, "gamma must lie in (0, 1]");
    if (p->ne_fixed <= 0 && (p->ne_max < 1 || !(p->tol > 0))) return fail(BIOT_ERR_INVALID_ARG, "tolerance mode needs tol > 0 and ne_max >= 1");
    if (p->precision != BIOT_FP64 && p->precision != BIOT_FP32 && p->precision != BIOT_FP32_COARSE64 &&
        p->precision != BIOT_FP32_DEV16 && p->precision != BIOT_FP32_DEVBF16)
        return fail(BIOT_ERR_INVALID_ARG, "unknown precision");
    if ((p->precision == BIOT_FP32_DEV16 || p->precision == BIOT_FP32_DEVBF16) && p->ne_fixed <= 0)
        return fail(BIOT_ERR_INVALID_ARG, "the 16-bit deviation store needs a fixed number of V-cycles (ne_fixed > 0)");
    constexpr int known = BIOT_OPT_COARSEST_STORAGE | BIOT_OPT_COLD_FP64 | BIOT_OPT_COLD_FP32 |
                          BIOT_OPT_COARSE_LO_ALL | BIOT_OPT_COARSE_LO_OFF | BIOT_OPT_SEGMENTS;
    if (p->options & ~known) return fail(BIOT_ERR_INVALID_ARG, "unknown option flag");
    if (p->cycle < BIOT_CYCLE_V || p->cycle > BIOT_CYCLE_F) return fail(BIOT_ERR_INVALID_ARG, "unknown cycle");
    if (p->fmg != 0 && p->fmg != 1) return fail(BIOT_ERR_INVALID_ARG, "fmg must be 0 or 1");
    if (p->pgrad != 0 && p->pgrad != 1) return fail(BIOT_ERR_INVALID_ARG, "pgrad must be 0 or 1");
    if ((p->options & BIOT_OPT_COLD_FP64) && (p->options & BIOT_OPT_COLD_FP32))
        return fail(BIOT_ERR_INVALID_ARG, "BIOT_OPT_COLD_FP64 and BIOT_OPT_COLD_FP32 exclude each other");
    if ((p->options & BIOT_OPT_COARSE_LO_ALL) && (p->options & BIOT_OPT_COARSE_LO_OFF))
        return fail(BIOT_ERR_INVALID_ARG, "BIOT_OPT_COARSE_LO_ALL and BIOT_OPT_COARSE_LO_OFF exclude each other");
    for (int i = 0; i < 4; i++) {
        if (s[i].eta_type < BIOT_PERIODIC || s[i].eta_type > BIOT_NEUMANN || s[i].p_type < BIOT_PERIODIC || s[i].p_type > BIOT_NEUMANN)
            return fail(BIOT_ERR_INVALID_ARG, "unknown boundary type");
    }
    for (int a = 0; a < 2; a++) {
        const int b = a + 2;
        const bool pe = s[a].eta_type == BIOT_PERIODIC, pp = s[a].p_type == BIOT_PERIODIC;
        if (pe != (s[b].eta_type == BIOT_PERIODIC) || pp != (s[b].p_type == BIOT_PERIODIC) || pe != pp)
            return fail(BIOT_ERR_INVALID_ARG, "periodic sides must face periodic sides, for both fields");
    }
    return BIOT_OK;
}

int set_profiles(biot_ctx *h, int side, const double *eta, const double *p)
{
    const size_t m = 2 * (size_t)side_cells(h, side) + 1;
    if (eta) {
        if (!h->eta_prof[side]) {
            int rc = dev_alloc(h, (void **)&h->eta_prof[side], 2 * m * sizeof(double));
            if (rc) return rc;
        }
        CUDA_TRY(cudaMemcpyAsync(h->eta_prof[side], eta, 2 * m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    } else if (h->eta_prof[side]) {
        CUDA_TRY(cudaMemsetAsync(h->eta_prof[side], 0, 2 * m * sizeof(double), h->stream));
    }
    if (p) {
        if (!h->p_prof[side]) {
            int rc = dev_alloc(h, (void **)&h->p_prof[side], m * sizeof(double));
            if (rc) return rc;
        }
        CUDA_TRY(cudaMemcpyAsync(h->p_prof[side], p, m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    } else if (h->p_prof[side]) {
        CUDA_TRY(cudaMemsetAsync(h->p_prof[side], 0, m * sizeof(double), h->stream));
    }
    // Host sources may be pageable and reused by the caller after return.
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return BIOT_OK;
}

// As set_profiles, without waiting for the stream: the caller's data is copied
// into a page-locked staging slot on the host, and the upload from there runs
// in stream order after the steps already queued.
int set_profiles_staged(biot_ctx *h, int side, const double *eta, const double *p)
{
    const size_t m = 2 * (size_t)side_cells(h, side) + 1;
    const int k = h->prof_slot[side];
    double *&st = h->prof_stage[side][k];
    if (!st) {
        if (cudaMallocHost((void **)&st, 3 * m * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            st = nullptr;
            return fail(BIOT_ERR_OOM, "pinned host allocation failed (profile staging)");
        }
        CUDA_TRY(cudaEventCreateWithFlags(&h->prof_ev[side][k], cudaEventDisableTiming));
    } else {
        CUDA_TRY(cudaEventSynchronize(h->prof_ev[side][k]));  // the upload that last used this slot has run
    }
    if (eta) {
        if (!h->eta_prof[side]) {
            int rc = dev_alloc(h, (void **)&h->eta_prof[side], 2 * m * sizeof(double));
            if (rc) return rc;
        }
        std::memcpy(st, eta, 2 * m * sizeof(double));
        CUDA_TRY(cudaMemcpyAsync(h->eta_prof[side], st, 2 * m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    } else if (h->eta_prof[side]) {
        CUDA_TRY(cudaMemsetAsync(h->eta_prof[side], 0, 2 * m * sizeof(double), h->stream));
    }
    if (p) {
        if (!h->p_prof[side]) {
            int rc = dev_alloc(h, (void **)&h->p_prof[side], m * sizeof(double));
            if (rc) return rc;
        }
        std::memcpy(st + 2 * m, p, m * sizeof(double));
        CUDA_TRY(cudaMemcpyAsync(h->p_prof[side], st + 2 * m, m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    } else if (h->p_prof[side]) {
        CUDA_TRY(cudaMemsetAsync(h->p_prof[side], 0, m * sizeof(double), h->stream));
    }
    CUDA_TRY(cudaEventRecord(h->prof_ev[side][k], h->stream));
    h->prof_slot[side] = k ^ 1;
    return BIOT_OK;
}

// ---- kernel sequencing --------------------------------------------------------

// Large FP32 instances run their solve at t = 0 -- three V-cycles from a zero
// iterate, where every correction is displacement-sized -- on a temporary FP64
// copy of the problem and take over its state rounded to FP32 (the first moments
// as double-float).  The time steps themselves stay on the FP32 path.  The FP32
// rounding a cold start leaves behind grows with the grid: at 4096^2 it is the
// largest part of the pressure error after the first steps (1.1e-5 against 4e-6
// with the FP64 cold start), on grids up to 1024^2 it stays far below the 1e-5
// target.  So the FP64 cold start applies from 2048^2 cells (BIOT_OPT_COLD_FP64:
// every grid, BIOT_OPT_COLD_FP32: none).  Smaller grids, and large ones without
// room for the FP64 copy, solve with double-float coarse levels instead
// (coarse_lo_mode).
constexpr long long COLD_FP64_MIN_CELLS = 2048LL * 2048LL;
bool cold_fp64_for(const biot_params *p)
{
    if (p->options & BIOT_OPT_COLD_FP64) return true;
    if (p->options & BIOT_OPT_COLD_FP32) return false;
    return (long long)p->nx * p->ny >= COLD_FP64_MIN_CELLS;
}

// Whether the sweeps of level l use the double-float first moments: always on
// the finest FP32 level, on the coarse FP32 levels as coarse_lo_mode() says.
bool level_lo(const biot_ctx *h, int l, bool cold)
{
    if (!h->lv[l].glo[0]) return false;
    if (l == h->L - 1) return true;
    const int m = coarse_lo_mode(&h->P);
    return m == COARSE_LO_ALL || (m == COARSE_LO_COLD && cold);
}

template <typename T, typename TC>
int sweep_typed(biot_ctx *h, int l, int mode, bool zero_init, bool prolong, bool want_res, int chain)
{
    Level &Lv = h->lv[l];
    const bool fine = (l == h->L - 1);
    SweepArgs<T, TC> a{};
    a.nx = Lv.nx;
    a.ny = Lv.ny;
    a.g = static_cast<const T *>(Lv.g[Lv.cur]);
    a.gout = (mode == SWEEP_SMOOTH) ? static_cast<T *>(Lv.g[1 - Lv.cur]) : nullptr;
    const bool lo = level_lo(h, l, h->cold_solve);
    a.glo = lo ? static_cast<const T *>(Lv.glo[Lv.cur]) : nullptr;
    a.glo_out = (lo && mode == SWEEP_SMOOTH) ? static_cast<T *>(Lv.glo[1 - Lv.cur]) : nullptr;
    a.r = fine ? nullptr : static_cast<const T *>(Lv.r);
    a.Ft = fine ? static_cast<const T *>(h->Ft) : nullptr;
    a.gc = prolong ? static_cast<const TC *>(h->lv[l - 1].g[h->lv[l - 1].cur]) : nullptr;
    a.rc = (mode == SWEEP_RESTRICT) ? static_cast<TC *>(h->lv[l - 1].r) : nullptr;
    for (int s = 0; s < 4; s++) {
        a.H[s] = static_cast<T *>(Lv.H[s]);
        a.prof[s] = fine ? h->eta_prof[s] : nullptr;
        a.bc[s] = h->bc_eta[s];
    }
    a.hist_valid = Lv.hist_valid;
    a.zero_init = zero_init ? 1 : 0;
    a.mode = mode;
    a.gamma = h->P.gamma;
    a.om_s = h->om_s;
    a.om_d = h->om_d;
    a.lm = h->lm;
    a.coef_fstar = 0.5 * h->P.alpha * h->P.alpha * h->P.r_coupling;
    a.c0h = h->P.c0 * h->h;
    a.resmax = want_res ? h->resmax : nullptr;
    a.rows = Lv.rows[mode];
    a.ghosts = h->P.ne_fixed > 0 ? 0 : 1;
    a.k_fs = T(a.coef_fstar * (-1.5 / (3.0 * a.lm + 1.0)));
    {
        const double k22 = -1.0 / (12.0 * a.lm + 4.0);  // m_22 relaxation (eq. moments:collision:22)
        a.k_hs = T(0.25 * (1.0 - a.om_s) - 0.5 * k22);
        a.k_hd = T(0.25 * (1.0 - a.om_d));
        a.k_h22 = T(0.25 * k22);
    }
    a.k_gam = T(a.gamma);
    if (fine && h->dev) {
        a.dev = h->dev;
        a.gd = Lv.gd[Lv.cur];
        a.gd_out = mode == SWEEP_SMOOTH ? Lv.gd[1 - Lv.cur] : nullptr;
        a.dsc = h->dsc;
        a.dinv = h->dinv;
        a.dev_full = (mode == SWEEP_SMOOTH && want_res) ? 1 : 0;  // the last sweep of the solve
    }

    if (h->rec) {
        SweepJob j{};
        j.tkind = sizeof(T) == 8 ? 0 : (sizeof(TC) == 8 ? 1 : 2);
        j.variant = (fine ? 0 : SWEEP_V_COARSE) | (a.glo ? SWEEP_V_LO : 0) | (mode == SWEEP_RESTRICT ? SWEEP_V_RESTRICT : 0) |
                    (a.ghosts ? 0 : SWEEP_V_NOGHOST) | (a.dev == 1 ? SWEEP_V_DEV16 : a.dev == 2 ? SWEEP_V_DEVBF16 : 0);
        j.level = l;
        job_args<T, TC>(j) = a;
        h->rec->push_back(j);
        Lv.hist_valid = 1;
        if (mode == SWEEP_SMOOTH) Lv.cur ^= 1;
        return BIOT_OK;
    }
    const bool timed = h->timing && fine && mode == SWEEP_SMOOTH;
    if (timed) {
        while (h->ev.size() < h->ev_used + 2) {
            cudaEvent_t e;
            CUDA_TRY(cudaEventCreate(&e));
            h->ev.push_back(e);
        }
        CUDA_TRY(cudaEventRecord(h->ev[h->ev_used], h->stream));
    }
    if (chain > 1) CUDA_TRY((launch_sweep_chain<T, TC>(a, chain, h->stream)));
    else CUDA_TRY((launch_sweep_mom<T, TC>(a, h->stream)));
    if (timed) {
        CUDA_TRY(cudaEventRecord(h->ev[h->ev_used + 1], h->stream));
        h->ev_used += 2;
    }
    h->launches++;
    Lv.hist_valid = 1;
    if (mode == SWEEP_SMOOTH && (chain <= 1 || (chain & 1))) Lv.cur ^= 1;
    return BIOT_OK;
}

// chain > 1: that many smoothing sweeps of a small FP64 level in one launch.
int sweep(biot_ctx *h, int l, int mode, bool zero_init, bool prolong, bool want_res, int chain = 1)
{
    const bool t64 = h->lv[l].fp64;
    const bool c64 = (l > 0) ? h->lv[l - 1].fp64 : t64;
    if (t64) return sweep_typed<double, double>(h, l, mode, zero_init, prolong, want_res, chain);
    if (c64) return sweep_typed<float, double>(h, l, mode, zero_init, prolong, want_res, chain);
    return sweep_typed<float, float>(h, l, mode, zero_init, prolong, want_res, chain);
}

// ---------------------------------------------------------------------------
// Segments (BIOT_OPT_SEGMENTS).  The sweeps of the small coarse levels of a
// V-cycle -- every level from the segment's start level down to the coarsest,
// each of at most SEG_MAX_TILES tiles -- are recorded instead of launched, split
// into runs of one storage family, and each run becomes one cluster launch of
// k_sweep_segment (one cluster per instance).  Per-cell code and arguments are
// those of the separate tile launches, so results are bitwise the same.  A
// sweep inside a cluster costs what a graph-launched tile sweep costs (the
// cluster barrier takes the place of the launch gap), and a 64^2 level's 16
// tiles fall two to a CTA: measured slower than separate launches on GB300,
// hence not the default.
// ---------------------------------------------------------------------------
int seg_tiles_of(const biot_ctx *h, int l)
{
    int tx, ty;
    sweep_tile_shape(h->lv[l].fp64, &tx, &ty);
    return ((h->lv[l].nx + tx - 1) / tx) * ((h->lv[l].ny + ty - 1) / ty);
}

// The level where a V-cycle's segment starts (-1: none): the finest coarse
// level such that it and every coarser level have at most SEG_MAX_TILES tiles
// and no double-float first moments (which the tile form of a segment does not
// take).  cold: for the solve at t = 0.  With BIOT_OPT_SEGMENTS; without it,
// only an instance of a batch has one, and only its FP64 coarsest level: the
// 2K sweeps that a single instance runs as one chained launch.
int seg_start(const biot_ctx *h, bool cold)
{
    if (!(h->P.options & BIOT_OPT_SEGMENTS))
        return (h->batched && h->L > 1 && h->lv[0].fp64 && seg_tiles_of(h, 0) <= SEG_MAX_TILES) ? 0 : -1;
    int s = -1;
    for (int l = 0; l < h->L - 1; l++) {
        if (level_lo(h, l, cold) || seg_tiles_of(h, l) > SEG_MAX_TILES) break;
        s = l;
    }
    return s;
}

template <typename X>
bool seg_eq(const X &a, const X &b) { return std::memcmp(&a, &b, sizeof(X)) == 0; }

// Field by field (padding aside): are two sweeps' arguments the same?  The
// strip height `rows` is not compared: tile sweeps do not read it.
template <typename T, typename TC>
bool seg_same_args(const SweepArgs<T, TC> &a, const SweepArgs<T, TC> &b)
{
    bool ok = a.nx == b.nx && a.ny == b.ny && a.g == b.g && a.gout == b.gout && a.glo == b.glo &&
              a.glo_out == b.glo_out && a.r == b.r && a.Ft == b.Ft && a.gc == b.gc && a.rc == b.rc &&
              a.hist_valid == b.hist_valid && a.zero_init == b.zero_init && a.mode == b.mode &&
              seg_eq(a.gamma, b.gamma) && seg_eq(a.om_s, b.om_s) && seg_eq(a.om_d, b.om_d) && seg_eq(a.lm, b.lm) &&
              seg_eq(a.coef_fstar, b.coef_fstar) && seg_eq(a.c0h, b.c0h) && a.resmax == b.resmax &&
              a.ghosts == b.ghosts && seg_eq(a.k_fs, b.k_fs) && seg_eq(a.k_hs, b.k_hs) && seg_eq(a.k_hd, b.k_hd) &&
              seg_eq(a.k_h22, b.k_h22) && seg_eq(a.k_gam, b.k_gam) && a.dev == b.dev && a.gd == b.gd &&
              a.gd_out == b.gd_out && seg_eq(a.dsc, b.dsc) && seg_eq(a.dinv, b.dinv) && a.dev_full == b.dev_full;
    for (int i = 0; i < 4; i++) ok = ok && a.H[i] == b.H[i] && a.prof[i] == b.prof[i] && a.bc[i] == b.bc[i];
    return ok;
}

// Job word of one recorded sweep of level l (level record rel of the program),
// checked to reproduce the sweep's arguments through seg_patch.
template <typename T, typename TC>
int seg_word(const biot_ctx *h, const SweepArgs<T, TC> &a, int l, const SegLevel &L, int rel, unsigned *out)
{
    const Level &Lv = h->lv[l];
    unsigned w = (unsigned)rel;
    if (a.mode == SWEEP_RESTRICT) w |= SEGJ_RESTRICT;
    if (a.g == Lv.g[1]) w |= SEGJ_CUR;
    if (a.zero_init) w |= SEGJ_ZERO;
    if (a.gc) {
        w |= SEGJ_PROL;
        if (l > 0 && (const void *)a.gc == h->lv[l - 1].g[1]) w |= SEGJ_CCUR;
    }
    if (a.hist_valid) w |= SEGJ_HIST;
    SweepArgs<T, TC> b;
    std::memcpy(&b, &L.a, sizeof(b));
    seg_patch<T, TC>(b, L, w);
    if (a.resmax || a.glo || a.Ft || a.dev || !seg_same_args(a, b))
        return fail(BIOT_ERR_CUDA, "segment program: a sweep is not reproduced by its job word");
    *out = w;
    return BIOT_OK;
}

// The program of recorded sweeps rec[i0 .. i1) (one storage family).
int seg_build(const biot_ctx *h, const std::vector<SweepJob> &rec, size_t i0, size_t i1, SegProg &prog)
{
    prog.fam = rec[i0].tkind == 0 ? 0 : 1;
    prog.cs = 1;
    prog.lev.clear();
    prog.job.clear();
    std::vector<int> lvl;  // level of each record
    for (size_t k = i0; k < i1; k++) {
        const SweepJob &j = rec[k];
        const int l = j.level;
        int rel = (int)(std::find(lvl.begin(), lvl.end(), l) - lvl.begin());
        if (rel == (int)lvl.size()) {
            if (rel > SEGJ_LEVEL) return fail(BIOT_ERR_CUDA, "segment program: too many levels");
            SegLevel L;
            std::memset(&L, 0, sizeof(L));
            L.tkind = j.tkind;
            if (j.tkind == 0) L.a.dd = j.dd;
            else if (j.tkind == 1) L.a.fd = j.fd;
            else L.a.ff = j.ff;
            L.buf[0] = h->lv[l].g[0];
            L.buf[1] = h->lv[l].g[1];
            if (l > 0) {
                L.cbuf[0] = h->lv[l - 1].g[0];
                L.cbuf[1] = h->lv[l - 1].g[1];
                L.crc = h->lv[l - 1].r;
            }
            prog.lev.push_back(L);
            lvl.push_back(l);
        }
        const SegLevel &L = prog.lev[rel];
        if (L.tkind != j.tkind) return fail(BIOT_ERR_CUDA, "segment program: a level changed its storage kind");
        unsigned w = 0;
        int rc = j.tkind == 0 ? seg_word<double, double>(h, j.dd, l, L, rel, &w)
               : j.tkind == 1 ? seg_word<float, double>(h, j.fd, l, L, rel, &w)
                              : seg_word<float, float>(h, j.ff, l, L, rel, &w);
        if (rc) return rc;
        prog.job.push_back(w);
        prog.cs = std::max(prog.cs, std::min(SEG_CLUSTER, seg_tiles_of(h, l)));
    }
    if (prog.lev.size() > (size_t)SEG_MAX_LEVELS || prog.job.size() > (size_t)SEG_MAX_JOBS)
        return fail(BIOT_ERR_CUDA, "segment program: too many levels or sweeps for one launch");
    return BIOT_OK;
}

// Append program g to the launch parameters P (false: P is full).
bool seg_pack(SegParams &P, const SegProg &g)
{
    if (P.nprog >= SEG_MAX_PROGS || P.lev0[P.nprog] + (int)g.lev.size() > SEG_MAX_LEVELS ||
        P.job0[P.nprog] + (int)g.job.size() > SEG_MAX_JOBS)
        return false;
    const int p = P.nprog;
    std::copy(g.lev.begin(), g.lev.end(), P.lev + P.lev0[p]);
    std::copy(g.job.begin(), g.job.end(), P.job + P.job0[p]);
    P.lev0[p + 1] = P.lev0[p] + (int)g.lev.size();
    P.job0[p + 1] = P.job0[p] + (int)g.job.size();
    P.nprog = p + 1;
    return true;
}

cudaError_t seg_launch(int fam, const SegParams &P, int cs, cudaStream_t s)
{
    return fam == 0 ? launch_sweep_segment<double>(P, cs, s) : launch_sweep_segment<float>(P, cs, s);
}

int vcycle(biot_ctx *h, int l, bool zero_start, bool prolong_first, int kind);

// The V-cycle from level l down (a coarse-grid correction, zero start) as
// segments.  Single instance: one launch per run of one storage family, except
// that a run of the coarsest level's smoothing sweeps alone, FP64 and at most
// SWEEP_CHAIN_MAX^2 cells, keeps the chained launch.  Batch (record mode): one
// recorded job per run, whose program goes to segrec.
int seg_vcycle(biot_ctx *h, int l)
{
    std::vector<SweepJob> rec;
    std::vector<SweepJob> *outer = h->rec;
    h->rec = &rec;
    h->in_seg = true;
    int rc = vcycle(h, l, true, false, BIOT_CYCLE_V);
    h->rec = outer;
    h->in_seg = false;
    if (rc) return rc;
    std::unique_ptr<SegParams> P;
    for (size_t i = 0; i < rec.size();) {
        const int fam = rec[i].tkind == 0 ? 0 : 1;
        size_t j = i;
        while (j < rec.size() && (rec[j].tkind == 0 ? 0 : 1) == fam) j++;
        SegProg prog;
        if ((rc = seg_build(h, rec, i, j, prog))) return rc;
        if (outer) {
            if (!h->segrec) return fail(BIOT_ERR_CUDA, "segment recorded without a program list");
            SweepJob m{};
            m.tkind = fam == 0 ? 0 : 2;
            m.variant = SWEEP_V_SEGMENT | (h->P.ne_fixed > 0 ? SWEEP_V_NOGHOST : 0);
            m.level = rec[i].level;
            m.seg = (int)h->segrec->size();
            h->segrec->push_back(std::move(prog));
            outer->push_back(m);
        } else {
            bool chain = fam == 0 && h->lv[0].nx <= SWEEP_CHAIN_MAX && h->lv[0].ny <= SWEEP_CHAIN_MAX && j - i > 1;
            for (size_t k = i; k < j && chain; k++) chain = rec[k].level == 0 && rec[k].dd.mode == SWEEP_SMOOTH;
            if (chain) {
                CUDA_TRY((launch_sweep_chain<double, double>(rec[i].dd, (int)(j - i), h->stream)));
            } else {
                if (!P) P.reset(new (std::nothrow) SegParams());
                if (!P) return fail(BIOT_ERR_OOM, "segment launch parameters");
                P->nprog = 0;
                P->ghosts = h->P.ne_fixed > 0 ? 0 : 1;
                P->lev0[0] = P->job0[0] = 0;
                if (!seg_pack(*P, prog)) return fail(BIOT_ERR_CUDA, "segment program too large for one launch");
                CUDA_TRY(seg_launch(fam, *P, prog.cs, h->stream));
            }
            h->launches++;
        }
        i = j;
    }
    return BIOT_OK;
}

// ELASTIC_MULTIGRID (Alg. 4) on level l.  zero_start: the iterate is zero
// (coarse-grid correction of a finer level); prolong_first: the first sweep
// adds the prolongated iterate of level l - 1 to it (the finer levels of a
// full-multigrid cycle).  kind: how the coarse-grid correction problem is
// solved -- one cycle of Alg. 4 (V), two in succession (W), or an F-cycle
// followed by a V-cycle (F).
int vcycle(biot_ctx *h, int l, bool zero_start, bool prolong_first = false, int kind = BIOT_CYCLE_V)
{
    // a coarse-grid correction from the segment's start level down: as segments
    // (a single instance keeps the chained coarsest level when that is all)
    if (kind == BIOT_CYCLE_V && zero_start && !prolong_first && !h->in_seg && l == seg_start(h, h->cold_solve) &&
        (h->rec || l > 0))
        return seg_vcycle(h, l);
    const int K = sweeps_of(&h->P, l);
    const bool fine = (l == h->L - 1);
    int rc;
    // the coarsest level's 2K sweeps, when it is a small FP64 level below the
    // finest, in one launch (a batch records them one by one)
    const Level &Lv = h->lv[l];
    if (l == 0 && !fine && !h->rec && Lv.fp64 && Lv.nx <= SWEEP_CHAIN_MAX && Lv.ny <= SWEEP_CHAIN_MAX && !prolong_first)
        return sweep(h, 0, SWEEP_SMOOTH, zero_start, false, false, 2 * K);
    for (int k = 0; k < K; k++)
        if ((rc = sweep(h, l, SWEEP_SMOOTH, zero_start && k == 0, prolong_first && k == 0, false))) return rc;
    if (l > 0) {
        if ((rc = sweep(h, l, SWEEP_RESTRICT, false, false, false))) return rc;
        h->lv[l - 1].hist_valid = 0;
        if (kind == BIOT_CYCLE_V) {
            if ((rc = vcycle(h, l - 1, true))) return rc;
        } else if (kind == BIOT_CYCLE_W) {
            if ((rc = vcycle(h, l - 1, true, false, BIOT_CYCLE_W))) return rc;
            if ((rc = vcycle(h, l - 1, false, false, BIOT_CYCLE_W))) return rc;
        } else {
            if ((rc = vcycle(h, l - 1, true, false, BIOT_CYCLE_F))) return rc;
            if ((rc = vcycle(h, l - 1, false, false, BIOT_CYCLE_V))) return rc;
        }
    }
    for (int k = 0; k < K; k++)
        if ((rc = sweep(h, l, SWEEP_SMOOTH, false, l > 0 && k == 0, fine && k == K - 1 && h->measure_cycle))) return rc;
    return BIOT_OK;
}

// One full-multigrid cycle on the finest level's correction problem (nested
// iteration): the finest defect is restricted level by level (each coarse
// level passes on the defect of its zero iterate), the coarsest level is
// solved by its 2K sweeps from zero, every finer level starts from the
// prolongated solution of the level below and gets one cycle, and the finest
// level adds the prolongated correction and gets one cycle.
int fmg_cycle(biot_ctx *h, int kind)
{
    const int L = h->L;
    int rc;
    if (L < 2) return vcycle(h, 0, false, false, kind);
    if ((rc = sweep(h, L - 1, SWEEP_RESTRICT, false, false, false))) return rc;
    for (int l = L - 2; l >= 1; l--) {
        h->lv[l].hist_valid = 0;
        if ((rc = sweep(h, l, SWEEP_RESTRICT, true, false, false))) return rc;
    }
    h->lv[0].hist_valid = 0;
    if ((rc = vcycle(h, 0, true))) return rc;
    for (int l = 1; l <= L - 2; l++) {
        h->lv[l].hist_valid = 0;
        if ((rc = vcycle(h, l, true, true, kind))) return rc;
    }
    return vcycle(h, L - 1, false, true, kind);
}

// The cycle of the elastic solve: the first one of a solve is a full-multigrid
// cycle when fmg is set.
int solve_cycle(biot_ctx *h, bool first)
{
    return (first && h->P.fmg) ? fmg_cycle(h, h->P.cycle) : vcycle(h, h->L - 1, false, false, h->P.cycle);
}

template <typename T>
int force_typed(biot_ctx *h)
{
    if (h->ft_fresh) {  // computed by the fused flow step
        h->ft_fresh = false;
        return BIOT_OK;
    }
    SexpArgs<T> e{};
    e.nx = h->P.nx;
    e.ny = h->P.ny;
    e.D1 = h->D1;
    e.D2 = h->D2;
    e.src = h->has_src ? h->src : nullptr;
    e.SE = h->SE;
    e.dt = h->P.dt;
    e.a_over_h = h->P.alpha / h->h;
    e.r = h->P.r_coupling;
    if (h->se_stale) {
        CUDA_TRY(launch_sexp<T>(e, h->stream));
        h->launches++;
        h->se_stale = false;
    }
    ForceArgs<T> a{};
    a.nx = h->P.nx;
    a.ny = h->P.ny;
    a.f = static_cast<const T *>(h->f[h->fcur]);
    a.SE = h->SE;
    a.fbody = h->has_fbody ? h->fbody : nullptr;
    a.Ft = static_cast<T *>(h->Ft);
    a.perx = h->bc_eta[BIOT_LEFT] == BIOT_PERIODIC;
    a.pery = h->bc_eta[BIOT_BOTTOM] == BIOT_PERIODIC;
    a.omega = h->omega;
    a.alpha_h = h->P.alpha * h->h;
    a.c0h2 = h->P.c0 * h->h * h->h;
    a.k_m3w = T(-3.0 * a.omega);
    a.k_mah = T(-a.alpha_h);
    a.central = h->P.pgrad;
    CUDA_TRY(launch_force<T>(a, h->stream));
    h->launches++;
    return BIOT_OK;
}

int read_residual(biot_ctx *h)
{
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (h->pending_stop) {  // counters of device-driven tolerance-mode steps
        const StopState st = *h->stop_host;
        h->total_cycles += st.total - h->stop_total_seen;
        h->stop_total_seen = st.total;
        h->last_ne = st.last_ne;
        h->notconv_steps += st.notconv - h->stop_notconv_seen;
        h->stop_notconv_seen = st.notconv;
        h->pending_stop = false;
        if (st.diverged) {
            h->diverged = 1;
            h->pending_res = false;
            h->last_res = st.last_res;
            return fail(BIOT_ERR_DIVERGED, "non-finite pseudo-time residual: the coupled iteration diverged");
        }
    }
    double res, gn, sq;
    std::memcpy(&res, &h->resmax_host[0], sizeof(double));
    std::memcpy(&gn, &h->resmax_host[1], sizeof(double));
    std::memcpy(&sq, &h->resmax_host[2], sizeof(double));
    h->last_res = res;
    h->last_res_l2 = std::sqrt(sq);
    h->pending_res = false;
    if (!std::isfinite(res)) {
        h->diverged = 1;
        return fail(BIOT_ERR_DIVERGED, "non-finite pseudo-time residual: the coupled iteration diverged");
    }
    (void)gn;
    return BIOT_OK;
}

// Elasticity update of Alg. 5 at the current time.
int elastic_solve_device_loop(biot_ctx *h);
int elastic_solve(biot_ctx *h);
int ensure_initialized(biot_ctx *h);
int finish_pending(biot_ctx *h);
int dev_encode(biot_ctx *h);
void release(biot_ctx *h);
size_t estimate_bytes(const biot_params *p, const biot_side *sides);

constexpr int COLD_FALLBACK = 1;  // no room for the FP64 copy: solve on the FP32 path

// The solve at t = 0 of an FP32 instance on an FP64 copy of its problem (same
// parameters, boundary data and sources), then the copy's finest state narrowed
// into this instance.  Returns the solve's status, or COLD_FALLBACK when the copy
// cannot be allocated.
int cold_start_fp64(biot_ctx *h)
{
    biot_params p64 = h->P;
    p64.precision = BIOT_FP64;
    biot_side sides[4];
    for (int s = 0; s < 4; s++) sides[s] = biot_side{h->bc_eta[s], h->bc_p[s], nullptr, nullptr};
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return COLD_FALLBACK;
    }
    if (estimate_bytes(&p64, sides) + (64u << 20) > free_b) return COLD_FALLBACK;
    biot_handle s = nullptr;
    int rc = biot_create(&p64, sides, &s);
    if (rc) return rc == BIOT_ERR_OOM ? COLD_FALLBACK : rc;
    // the copy works on this instance's stream, after its own set-up
    if (cudaStreamSynchronize(s->own_stream) != cudaSuccess) rc = fail(BIOT_ERR_CUDA, "FP64 copy set-up failed");
    s->stream = h->stream;
    const size_t np = (size_t)h->P.nx * h->P.ny;
    for (int side = 0; side < 4 && !rc; side++) {
        const size_t m = 2 * (size_t)side_cells(h, side) + 1;
        if (h->eta_prof[side] && !(rc = dev_alloc(s, (void **)&s->eta_prof[side], 2 * m * sizeof(double))))
            if (cudaMemcpyAsync(s->eta_prof[side], h->eta_prof[side], 2 * m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
                rc = fail(BIOT_ERR_CUDA, "boundary data copy failed");
        if (!rc && h->p_prof[side] && !(rc = dev_alloc(s, (void **)&s->p_prof[side], m * sizeof(double))))
            if (cudaMemcpyAsync(s->p_prof[side], h->p_prof[side], m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
                rc = fail(BIOT_ERR_CUDA, "boundary data copy failed");
    }
    if (!rc && h->has_src && !(rc = dev_alloc(s, (void **)&s->src, np * sizeof(double)))) {
        if (cudaMemcpyAsync(s->src, h->src, np * sizeof(double), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            rc = fail(BIOT_ERR_CUDA, "source copy failed");
        s->has_src = true;
    }
    if (!rc && h->has_fbody && !(rc = dev_alloc(s, (void **)&s->fbody, 2 * np * sizeof(double)))) {
        if (cudaMemcpyAsync(s->fbody, h->fbody, 2 * np * sizeof(double), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            rc = fail(BIOT_ERR_CUDA, "body force copy failed");
        s->has_fbody = true;
    }
    int status = BIOT_OK;
    if (!rc) rc = ensure_initialized(s);
    if (!rc) {
        rc = elastic_solve(s);
        if (rc == BIOT_ERR_NOT_CONVERGED) {
            status = rc;
            rc = BIOT_OK;
        }
    }
    if (!rc) rc = finish_pending(s);
    if (!rc) {
        const Level &Ls = s->lv[s->L - 1];
        Level &Lh = h->lv[h->L - 1];
        NarrowArgs a{};
        a.np = np;
        a.g64 = static_cast<const double *>(Ls.g[Ls.cur]);
        a.f64 = static_cast<const double *>(s->f[s->fcur]);
        a.ft64 = static_cast<const double *>(s->Ft);
        a.g32 = static_cast<float *>(Lh.g[Lh.cur]);
        a.glo32 = static_cast<float *>(Lh.glo[Lh.cur]);
        a.f32 = static_cast<float *>(h->f[h->fcur]);
        a.ft32 = static_cast<float *>(h->Ft);
        if (!a.glo32) rc = fail(BIOT_ERR_CUDA, "FP32 instance without double-float first moments");
        else if (launch_narrow_state(a, h->stream) != cudaSuccess) rc = fail(BIOT_ERR_CUDA, "state hand-over launch failed");
        else if ((rc = dev_encode(h))) {
        } else if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = fail(BIOT_ERR_CUDA, "state hand-over failed");
    }
    if (!rc) {
        h->launches += s->launches + 1;
        h->total_cycles += s->total_cycles;
        h->notconv_steps += s->notconv_steps;
        h->last_ne = s->last_ne;
        h->last_res = s->last_res;
        h->last_res_l2 = s->last_res_l2;
        h->initialized = true;
        h->solved = true;
        h->pending_res = false;
        h->ft_fresh = false;
        h->se_stale = true;
        h->lv[h->L - 1].hist_valid = 0;
    }
    cudaStreamSynchronize(h->stream);
    s->stream = s->own_stream;
    release(s);
    return rc ? rc : status;
}

int elastic_solve(biot_ctx *h)
{
    int rc;
    if (h->cold64 && h->nstep == 0 && !h->solved && !h->rec) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CUDA_TRY(cudaStreamIsCapturing(h->stream, &cs));
        if (cs == cudaStreamCaptureStatusNone) {
            rc = cold_start_fp64(h);
            if (rc != COLD_FALLBACK) return rc;
        }
    }
    rc = h->fp32 ? force_typed<float>(h) : force_typed<double>(h);
    if (rc) return rc;
    h->lv[h->L - 1].hist_valid = 0;
    h->cold_solve = h->nstep == 0;
    const bool fixed = h->P.ne_fixed > 0;
    if (!fixed && !h->rec) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CUDA_TRY(cudaStreamIsCapturing(h->stream, &cs));
        if (cs == cudaStreamCaptureStatusActive) return elastic_solve_device_loop(h);
    }
    int ne = 0, status = BIOT_OK;
    for (;;) {
        const bool measure = !fixed || (ne + 1 == h->P.ne_fixed);
        h->measure_cycle = measure;
        if (measure) CUDA_TRY(cudaMemsetAsync(h->resmax, 0, RES_WORDS * sizeof(unsigned long long), h->stream));
        if ((rc = solve_cycle(h, ne == 0))) return rc;
        ne++;
        h->total_cycles++;
        if (fixed) {
            if (ne >= h->P.ne_fixed) {
                // (a batched step issues this copy after its merged sweeps)
                if (!h->rec)
                    CUDA_TRY(cudaMemcpyAsync(h->resmax_host, h->resmax, RES_WORDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
                h->pending_res = true;
                break;
            }
            continue;
        }
        CUDA_TRY(cudaMemcpyAsync(h->resmax_host, h->resmax, RES_WORDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
        if ((rc = read_residual(h))) return rc;
        double gn;
        std::memcpy(&gn, &h->resmax_host[1], sizeof(double));
        if (h->last_res <= h->P.tol * (gn > 1.0 ? gn : 1.0)) break;
        if (ne >= h->P.ne_max) {
            h->notconv_steps++;
            status = BIOT_ERR_NOT_CONVERGED;
            break;
        }
    }
    h->last_ne = ne;
    h->solved = true;
    return status;
}

// Tolerance mode inside a graph capture: the first V-cycle and its stopping
// test, then a WHILE node whose body is one more V-cycle and the test; the
// test kernel sets the node's condition.  Every V-cycle after the first of a
// step sees the same state transitions (each level's ping-pong parity returns
// after its 2K smoothing sweeps; the finest history is valid), so the body
// recorded once is exact for every iteration.
int stop_test(biot_ctx *h, int first, cudaGraphConditionalHandle cond)
{
    StopArgs a{};
    a.resmax = h->resmax;
    a.st = h->stop;
    a.tol = h->P.tol;
    a.ne_max = h->P.ne_max;
    a.first = first;
    a.cond = (unsigned long long)cond;
    CUDA_TRY(launch_stop_test(a, h->stream));
    h->launches++;
    return BIOT_OK;
}

int elastic_solve_device_loop(biot_ctx *h)
{
    int rc;
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &cg, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle cond;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, cg, 0, cudaGraphCondAssignDefault));
    // first V-cycle of the step
    h->measure_cycle = true;
    CUDA_TRY(cudaMemsetAsync(h->resmax, 0, RES_WORDS * sizeof(unsigned long long), h->stream));
    if ((rc = solve_cycle(h, true))) return rc;
    if ((rc = stop_test(h, 1, cond))) return rc;
    // WHILE node after it
    CUDA_TRY(cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &cg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CUDA_TRY(cudaStreamBeginCaptureToGraph(h->aux_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaStream_t main = h->stream;
    h->stream = h->aux_stream;
    rc = BIOT_OK;
    cudaError_t e = cudaMemsetAsync(h->resmax, 0, RES_WORDS * sizeof(unsigned long long), h->stream);
    if (e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    if (!rc) rc = solve_cycle(h, false);
    if (!rc) rc = stop_test(h, 0, cond);
    h->stream = main;
    cudaGraph_t body_out = body;
    e = cudaStreamEndCapture(h->aux_stream, &body_out);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(BIOT_ERR_CUDA, std::string("cudaStreamEndCapture (loop body): ") + cudaGetErrorString(e));
    CUDA_TRY(cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    // counters and the last residual back to the host once per step
    CUDA_TRY(cudaMemcpyAsync(h->resmax_host, h->resmax, RES_WORDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->stop_host, h->stop, sizeof(StopState), cudaMemcpyDeviceToHost, h->stream));
    h->pending_res = true;
    h->pending_stop = true;
    h->solved = true;
    return BIOT_OK;
}

template <typename T>
int flow_typed(biot_ctx *h)
{
    const Level &Lf = h->lv[h->L - 1];
    const size_t np = (size_t)h->P.nx * h->P.ny;
    FlowFusedArgs<T> a{};
    a.nx = h->P.nx;
    a.ny = h->P.ny;
    a.f = static_cast<const T *>(h->f[h->fcur]);
    a.fout = static_cast<T *>(h->f[1 - h->fcur]);
    a.ms = static_cast<const T *>(Lf.g[Lf.cur]) + 3 * np;
    a.D1 = h->D1;
    a.dBprev = static_cast<const T *>(h->dB[h->fcur]);
    a.Dnew = h->D2;  // D(t - 2 dt) is no longer read: D(t) takes its buffer
    a.dAout = static_cast<T *>(h->dB[1 - h->fcur]);
    a.src = h->has_src ? h->src : nullptr;
    a.fbody = h->has_fbody ? h->fbody : nullptr;
    a.Ft = static_cast<T *>(h->Ft);
    for (int i = 0; i < 4; i++) {
        a.pprof[i] = h->p_prof[i];
        a.bc[i] = h->bc_p[i];
    }
    a.perx = h->bc_eta[BIOT_LEFT] == BIOT_PERIODIC;
    a.pery = h->bc_eta[BIOT_BOTTOM] == BIOT_PERIODIC;
    a.dt = h->P.dt;
    a.a_over_h = h->P.alpha / h->h;
    a.r = h->P.r_coupling;
    a.kD = -1.5 / (3.0 * h->lm + 1.0);
    a.c0 = h->P.c0;
    a.c0h2 = h->P.c0 * h->h * h->h;
    a.k_om = T(h->omega);
    a.k_src = T(1.0 - 0.5 * h->omega);
    a.k_m3w = T(-3.0 * h->omega);
    a.k_mah = T(-(h->P.alpha * h->h));
    a.k_a1r = T(a.a_over_h * (1.0 - a.r));
    a.k_ar = T(a.a_over_h * a.r);
    a.k_c2 = T(a.a_over_h * a.r * a.kD);
    if (h->frec) {  // batched step: the batch launches it with the others
        FlowRec r{};
        r.fp64 = sizeof(T) == 8;
        flow_args<T>(r) = a;
        h->frec->push_back(r);
    } else {
        CUDA_TRY(launch_flow_fused<T>(a, h->stream));
        h->launches++;
    }
    std::swap(h->D1, h->D2);  // D1 <- D(t), D2 <- D(t - dt)
    h->ft_fresh = !h->P.pgrad;  // F~ of the next elastic solve is computed (eq. pressure:gradient)
    h->se_stale = true;   // the s'_exp buffer was used as scratch
    h->fcur ^= 1;
    h->nstep++;
    return BIOT_OK;
}

// The finest level's deviation store from its FP32 planes 2-4 (no-op without one).
int dev_encode(biot_ctx *h)
{
    if (!h->dev) return BIOT_OK;
    Level &Lf = h->lv[h->L - 1];
    DevEncodeArgs e{};
    e.np = (size_t)h->P.nx * h->P.ny;
    e.g = static_cast<const float *>(Lf.g[Lf.cur]);
    e.gd = Lf.gd[Lf.cur];
    e.dsc = h->dsc;
    e.dev = h->dev;
    CUDA_TRY(launch_dev_encode(e, h->stream));
    h->launches++;
    return BIOT_OK;
}

template <typename T>
int init_typed(biot_ctx *h)
{
    Level &Lf = h->lv[h->L - 1];
    InitArgs<T> a{};
    a.nx = h->P.nx;
    a.ny = h->P.ny;
    a.f = static_cast<T *>(h->f[h->fcur]);
    a.g = static_cast<T *>(Lf.g[Lf.cur]);
    a.glo = static_cast<T *>(Lf.glo[Lf.cur]);
    a.src = h->has_src ? h->src : nullptr;
    a.fbody = h->has_fbody ? h->fbody : nullptr;
    a.dt = h->P.dt;
    a.c0h2 = h->P.c0 * h->h * h->h;
    CUDA_TRY(launch_init<T>(a, h->stream));
    h->launches++;
    int rc = dev_encode(h);
    if (rc) return rc;
    h->initialized = true;
    return BIOT_OK;
}

int ensure_initialized(biot_ctx *h)
{
    if (h->initialized) return BIOT_OK;
    return h->fp32 ? init_typed<float>(h) : init_typed<double>(h);
}

int finish_pending(biot_ctx *h)
{
    if (!h->pending_res) return BIOT_OK;
    return read_residual(h);
}

template <typename T>
int readout_typed(biot_ctx *h, double *eta, double *p, double *sigma)
{
    const Level &Lf = h->lv[h->L - 1];
    ReadoutArgs<T> a{};
    a.nx = h->P.nx;
    a.ny = h->P.ny;
    a.g = static_cast<const T *>(Lf.g[Lf.cur]);
    a.glo = static_cast<const T *>(Lf.glo[Lf.cur]);
    a.f = static_cast<const T *>(h->f[h->fcur]);
    a.Ft = static_cast<const T *>(h->Ft);
    a.D1 = h->D1;
    a.D2 = h->D2;
    a.src = h->has_src ? h->src : nullptr;
    a.eta = eta;
    a.p = p;
    a.sigma = sigma;
    a.perx = h->bc_eta[BIOT_LEFT] == BIOT_PERIODIC;
    a.pery = h->bc_eta[BIOT_BOTTOM] == BIOT_PERIODIC;
    a.dt = h->P.dt;
    a.a_over_h = h->P.alpha / h->h;
    a.r = h->P.r_coupling;
    a.kD = -1.5 / (3.0 * h->lm + 1.0);
    const double coef_fstar = 0.5 * h->P.alpha * h->P.alpha * h->P.r_coupling;  // alpha^2 r / 2
    a.c_axis = coef_fstar * a.kD / 3.0;
    a.c_diag = coef_fstar * a.kD / 12.0;
    a.inv_c0 = 1.0 / h->P.c0;
    const double lm3 = 3.0 * h->lm, mu6 = 6.0 * h->mu, sc = -0.5 / (h->P.c0 * h->h);
    a.c_s = sc * lm3 / (lm3 + 1.0);   // mbar_s = 3 lm / (3 lm + 1) m_s
    a.c_d = sc * mu6 / (mu6 + 1.0);   // mbar_d = 6 mu / (6 mu + 1) m_d, same for m_11
    a.c_11 = 2.0 * a.c_d;
    CUDA_TRY(launch_readout<T>(a, h->stream));
    h->launches++;
    return BIOT_OK;
}

int readout(biot_ctx *h, double *eta_host, double *p_host, double *sigma_host)
{
    int rc;
    if ((rc = ensure_initialized(h))) return rc;
    if (!h->solved) {
        rc = elastic_solve(h);
        if (rc && rc != BIOT_ERR_NOT_CONVERGED) return rc;
    }
    if ((rc = finish_pending(h))) return rc;
    const size_t np = (size_t)h->P.nx * h->P.ny;
    if (!h->out) {
        if ((rc = dev_alloc(h, (void **)&h->out, 6 * np * sizeof(double)))) return rc;
    }
    double *deta = eta_host ? h->out : nullptr;
    double *dp = p_host ? h->out + 2 * np : nullptr;
    double *ds = sigma_host ? h->out + 3 * np : nullptr;
    rc = h->fp32 ? readout_typed<float>(h, deta, dp, ds) : readout_typed<double>(h, deta, dp, ds);
    if (rc) return rc;
    if (eta_host) CUDA_TRY(cudaMemcpyAsync(eta_host, deta, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (p_host) CUDA_TRY(cudaMemcpyAsync(p_host, dp, np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (sigma_host) CUDA_TRY(cudaMemcpyAsync(sigma_host, ds, 3 * np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return BIOT_OK;
}

// biot_read_async: fields formed on the instance's stream into staging buffer
// aslot, copied to the host on the copy stream; the buffer is reused only after
// its previous copy is done (a device-side wait).
int read_async(biot_ctx *h, double *eta_host, double *p_host, double *sigma_host)
{
    int rc;
    if ((rc = ensure_initialized(h))) return rc;
    if (!h->solved) {
        rc = elastic_solve(h);
        if (rc && rc != BIOT_ERR_NOT_CONVERGED) return rc;
    }
    // steps still queued keep their residual check pending: the read-out runs
    // after them in stream order, and the next synchronising call reports them
    if (!h->copy_stream) {
        CUDA_TRY(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; i++) {
            CUDA_TRY(cudaEventCreateWithFlags(&h->aready[i], cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&h->acopied[i], cudaEventDisableTiming));
        }
    }
    const int s = h->aslot;
    const size_t np = (size_t)h->P.nx * h->P.ny;
    const int planes = sigma_host ? 6 : 3;
    if (h->aout_planes[s] < planes) {
        if (h->aout[s]) {  // grow: the buffer's last copy must be done before it is freed
            CUDA_TRY(cudaEventSynchronize(h->acopied[s]));
            CUDA_TRY(cudaFree(h->aout[s]));
            h->bytes -= (size_t)h->aout_planes[s] * np * sizeof(double);
            h->aout[s] = nullptr;
            h->aout_planes[s] = 0;
            h->ainflight[s] = false;
        }
        cudaError_t e = cudaMalloc((void **)&h->aout[s], (size_t)planes * np * sizeof(double));
        if (e != cudaSuccess) {
            h->aout[s] = nullptr;
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? BIOT_ERR_OOM : BIOT_ERR_CUDA,
                        std::string("cudaMalloc (read-out staging): ") + cudaGetErrorString(e));
        }
        h->aout_planes[s] = planes;
        h->bytes += (size_t)planes * np * sizeof(double);
    }
    if (h->ainflight[s]) CUDA_TRY(cudaStreamWaitEvent(h->stream, h->acopied[s], 0));
    double *base = h->aout[s];
    double *deta = eta_host ? base : nullptr;
    double *dp = p_host ? base + 2 * np : nullptr;
    double *ds = sigma_host ? base + 3 * np : nullptr;
    rc = h->fp32 ? readout_typed<float>(h, deta, dp, ds) : readout_typed<double>(h, deta, dp, ds);
    if (rc) return rc;
    CUDA_TRY(cudaEventRecord(h->aready[s], h->stream));
    CUDA_TRY(cudaStreamWaitEvent(h->copy_stream, h->aready[s], 0));
    if (eta_host) CUDA_TRY(cudaMemcpyAsync(eta_host, deta, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, h->copy_stream));
    if (p_host) CUDA_TRY(cudaMemcpyAsync(p_host, dp, np * sizeof(double), cudaMemcpyDeviceToHost, h->copy_stream));
    if (sigma_host) CUDA_TRY(cudaMemcpyAsync(sigma_host, ds, 3 * np * sizeof(double), cudaMemcpyDeviceToHost, h->copy_stream));
    CUDA_TRY(cudaEventRecord(h->acopied[s], h->copy_stream));
    h->ainflight[s] = true;
    h->aslot = s ^ 1;
    return BIOT_OK;
}

void drop_graphs(biot_ctx *h)
{
    h->epoch++;
    for (int i = 0; i < 2; i++) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        h->graph[i] = nullptr;
    }
}

// One iteration of the time loop of Alg. 5 from a solved state: flow step to
// t + dt, then the elastic solve at t + dt.
int advance(biot_ctx *h)
{
    int rc = h->fp32 ? flow_typed<float>(h) : flow_typed<double>(h);
    if (rc) return rc;
    h->solved = false;
    rc = elastic_solve(h);
    return rc;
}

GraphKey graph_key(const biot_ctx *h)
{
    GraphKey k;
    std::memset(&k, 0, sizeof(k));
    k.nx = h->P.nx;
    k.ny = h->P.ny;
    k.L = h->L;
    k.K = h->P.K;
    k.ne_fixed = h->P.ne_fixed;
    k.precision = h->P.precision;
    k.options = h->P.options;
    k.cycle = h->P.cycle;
    k.fmg = h->P.fmg;
    k.pgrad = h->P.pgrad;
    for (int i = 0; i < 4; i++) {
        k.bc[i] = h->bc_eta[i];
        k.bc[4 + i] = h->bc_p[i];
    }
    for (int j = 0; j < BIOT_MAX_LEVELS; j++) k.K_level[j] = h->P.K_level[j];
    return k;
}

// advance() through a captured CUDA graph (fixed number of V-cycles: the
// launch sequence and every buffer parity repeat from step to step except the
// flow ping-pong, hence one graph per parity).
int advance_graph(biot_ctx *h)
{
    const int par = h->fcur;
    if (!h->graph[par]) {
        const long l0 = h->launches, c0 = h->total_cycles;
        CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int rc = advance(h);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(BIOT_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        h->graph[par] = h->gcache ? h->gcache->take(graph_key(h), par, g) : nullptr;
        e = h->graph[par] ? cudaSuccess : cudaGraphInstantiate(&h->graph[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->graph[par] = nullptr;
            return fail(BIOT_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
        h->graph_launches[par] = h->launches - l0;
        h->launches = l0;
        h->total_cycles = c0;
        // capture recorded the state transitions; replay them from the start state
        h->fcur ^= 1;
        std::swap(h->D1, h->D2);
        h->nstep -= 1;
    }
    CUDA_TRY(cudaGraphLaunch(h->graph[par], h->stream));
    h->launches += h->graph_launches[par];
    h->fcur ^= 1;
    std::swap(h->D1, h->D2);
    h->nstep += 1;
    if (h->P.ne_fixed > 0) {
        h->total_cycles += h->P.ne_fixed;
        h->last_ne = h->P.ne_fixed;
    } else {
        h->pending_stop = true;  // counters arrive with the step's read-back
    }
    h->solved = true;
    h->pending_res = true;
    return BIOT_OK;
}

void release(biot_ctx *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    drop_graphs(h);
    for (int i = 0; i < 2; i++) {
        if (h->aout[i]) cudaFree(h->aout[i]);
        if (h->aready[i]) cudaEventDestroy(h->aready[i]);
        if (h->acopied[i]) cudaEventDestroy(h->acopied[i]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->pool) {  // stream-ordered frees, complete before the server may destroy its pool
        for (void *p : h->allocs) cudaFreeAsync(p, h->stream);
        cudaStreamSynchronize(h->stream);
    } else {
        for (void *p : h->allocs) cudaFree(p);
    }
    h->allocs.clear();
    if (!h->host_lent) {
        if (h->resmax_host) cudaFreeHost(h->resmax_host);
        if (h->stop_host) cudaFreeHost(h->stop_host);
    }
    for (int side = 0; side < 4; side++)
        for (int k = 0; k < 2; k++) {
            if (h->prof_stage[side][k]) cudaFreeHost(h->prof_stage[side][k]);
            if (h->prof_ev[side][k]) cudaEventDestroy(h->prof_ev[side][k]);
        }
    if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char *biot_error_string(int code)
{
    switch (code) {
    case BIOT_OK: return "ok";
    case BIOT_ERR_INVALID_ARG: return "invalid argument";
    case BIOT_ERR_OOM: return "out of memory";
    case BIOT_ERR_DIVERGED: return "diverged";
    case BIOT_ERR_NOT_CONVERGED: return "not converged";
    case BIOT_ERR_CUDA: return "CUDA error";
    case BIOT_ERR_TIMEOUT: return "timeout";
    case BIOT_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown error";
    }
}

const char *biot_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace {

// biot_create, optionally with a server's pool and pinned mirrors (Lend).
int create_instance(const biot_params *p, const biot_side sides[4], biot_handle *out, const Lend *lend)
{
    if (!out) return fail(BIOT_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    int rc = check_params(p, sides);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(BIOT_ERR_NO_DEVICE, "no CUDA device visible");
    }
    biot_ctx *h = new (std::nothrow) biot_ctx();
    if (!h) return fail(BIOT_ERR_OOM, "host allocation failed");
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(BIOT_ERR_CUDA, "cudaGetDevice failed");
    }
    h->P = *p;
    h->L = p->mg_levels;
    h->fp32 = p->precision != BIOT_FP64;  // finest level and flow populations in FP32
    h->dev = p->precision == BIOT_FP32_DEV16 ? 1 : p->precision == BIOT_FP32_DEVBF16 ? 2 : 0;
    h->cold64 = h->fp32 && cold_fp64_for(p);
    h->h = p->lx / p->nx;
    h->lam = p->c0 * p->lambda;
    h->mu = p->c0 * p->mu;
    h->lm = h->lam + h->mu;
    h->kap = p->dt * p->kappa / (p->c0 * h->h * h->h);
    h->omega = 1.0 / (3.0 * h->kap + 0.5);
    h->om_s = 2.0 / (3.0 * h->lm + 1.0);
    h->om_d = 2.0 / (6.0 * h->mu + 1.0);
    for (int i = 0; i < 4; i++) {
        h->bc_eta[i] = sides[i].eta_type;
        h->bc_p[i] = sides[i].p_type;
    }
    if (h->dev) {
        // scale of the deviation store: the lattice stress c0 h sigma_ref of the
        // largest boundary traction (or of the stress lambda + 2 mu times the
        // largest boundary displacement over the domain size), taken to about 1,
        // so that FP16's normal range covers several decades on both sides
        double sref = 0.0;
        for (int i = 0; i < 4; i++) {
            if (!sides[i].eta_profile) continue;
            const size_t m = 2 * (size_t)((i == BIOT_BOTTOM || i == BIOT_TOP) ? p->nx : p->ny) + 1;
            double mx = 0.0;
            for (size_t k = 0; k < 2 * m; k++) mx = std::max(mx, std::fabs(sides[i].eta_profile[k]));
            if (sides[i].eta_type == BIOT_NEUMANN) sref = std::max(sref, mx);
            else if (sides[i].eta_type == BIOT_DIRICHLET) sref = std::max(sref, (p->lambda + 2.0 * p->mu) * mx / std::max(p->lx, p->ly));
        }
        if (!(sref > 0.0) || !std::isfinite(sref)) sref = 1.0;
        const int e = std::max(-60, std::min(60, (int)std::lround(-std::log2(p->c0 * h->h * sref))));
        h->dsc = std::ldexp(1.0f, e);
        h->dinv = std::ldexp(1.0f, -e);
    }
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(BIOT_ERR_CUDA, "cudaStreamCreate failed");
    }
    h->stream = h->own_stream;
    if (lend) {
        h->pool = lend->pool;
        h->resmax_host = lend->resmax_host;
        h->stop_host = lend->stop_host;
        h->host_lent = true;
    }

#define TRY_RC(x) do { int _r = (x); if (_r) { release(h); return _r; } } while (0)
    const size_t np = (size_t)p->nx * p->ny;
    const size_t tsz = h->fp32 ? sizeof(float) : sizeof(double);
    for (int l = 0; l < h->L; l++) {
        Level &Lv = h->lv[l];
        const int shift = h->L - 1 - l;
        Lv.nx = p->nx >> shift;
        Lv.ny = p->ny >> shift;
        Lv.np = (size_t)Lv.nx * Lv.ny;
        // FP64: the FP64 path; the coarsest level below a finer one unless
        // BIOT_OPT_COARSEST_STORAGE; with BIOT_FP32_COARSE64 every level below the finest
        Lv.fp64 = !h->fp32 || (l == 0 && h->L > 1 && coarsest_fp64(p)) || (p->precision == BIOT_FP32_COARSE64 && l < h->L - 1);
        const size_t esz = Lv.fp64 ? sizeof(double) : sizeof(float);
        TRY_RC(dev_alloc(h, &Lv.g[0], 8 * Lv.np * esz));
        TRY_RC(dev_alloc(h, &Lv.g[1], 8 * Lv.np * esz));
        if (!Lv.fp64 && (l == h->L - 1 || coarse_lo_mode(p) != COARSE_LO_OFF)) {  // double-float displacement moments
            TRY_RC(dev_alloc(h, &Lv.glo[0], 2 * Lv.np * esz));
            TRY_RC(dev_alloc(h, &Lv.glo[1], 2 * Lv.np * esz));
        }
        if (l < h->L - 1) TRY_RC(dev_alloc(h, &Lv.r, 8 * Lv.np * esz));
        if (l == h->L - 1 && h->dev) {  // 16-bit m_11, m_s, m_d
            TRY_RC(dev_alloc(h, &Lv.gd[0], 3 * Lv.np * 2));
            TRY_RC(dev_alloc(h, &Lv.gd[1], 3 * Lv.np * 2));
        }
        for (int s = 0; s < 4; s++) {
            if (h->bc_eta[s] != BIOT_DIRICHLET) continue;
            const int n = (s == BIOT_BOTTOM || s == BIOT_TOP) ? Lv.nx : Lv.ny;
            TRY_RC(dev_alloc(h, &Lv.H[s], 3 * (size_t)n * esz));
        }
    }
    TRY_RC(dev_alloc(h, &h->f[0], 9 * np * tsz));
    TRY_RC(dev_alloc(h, &h->f[1], 9 * np * tsz));
    TRY_RC(dev_alloc(h, &h->Ft, 2 * np * tsz));
    TRY_RC(dev_alloc(h, (void **)&h->D1, np * sizeof(double)));
    TRY_RC(dev_alloc(h, (void **)&h->D2, np * sizeof(double)));
    TRY_RC(dev_alloc(h, &h->dB[0], np * tsz));
    TRY_RC(dev_alloc(h, &h->dB[1], np * tsz));
    TRY_RC(dev_alloc(h, (void **)&h->SE, np * sizeof(double)));
    TRY_RC(dev_alloc(h, (void **)&h->resmax, RES_WORDS * sizeof(unsigned long long)));
    TRY_RC(dev_alloc(h, (void **)&h->stop, sizeof(StopState)));
    if (!h->host_lent && (cudaMallocHost((void **)&h->resmax_host, RES_WORDS * sizeof(unsigned long long)) != cudaSuccess ||
                          cudaMallocHost((void **)&h->stop_host, sizeof(StopState)) != cudaSuccess)) {
        cudaGetLastError();
        release(h);
        return fail(BIOT_ERR_OOM, "pinned host allocation failed");
    }
    std::memset(h->stop_host, 0, sizeof(StopState));
    if (cudaStreamCreateWithFlags(&h->aux_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->aux_stream = nullptr;
        release(h);
        return fail(BIOT_ERR_CUDA, "cudaStreamCreate failed");
    }
    for (int s = 0; s < 4; s++) TRY_RC(set_profiles(h, s, sides[s].eta_profile, sides[s].p_profile));
#undef TRY_RC
    *out = h;
    return BIOT_OK;
}

}  // namespace

extern "C" {

int biot_create(const biot_params *p, const biot_side sides[4], biot_handle *out)
{
    return create_instance(p, sides, out, nullptr);
}

int biot_destroy(biot_handle h)
{
    release(h);
    return BIOT_OK;
}

int biot_set_stream(biot_handle h, void *cuda_stream)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->own_stream;
    return BIOT_OK;
}

int biot_set_sources(biot_handle h, const double *f_body, const double *s)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    const size_t np = (size_t)h->P.nx * h->P.ny;
    const double *fb0 = h->fbody, *s0 = h->src;
    const bool hf0 = h->has_fbody, hs0 = h->has_src;
    int rc;
    if (f_body) {
        if (!h->fbody && (rc = dev_alloc(h, (void **)&h->fbody, 2 * np * sizeof(double)))) return rc;
        CUDA_TRY(cudaMemcpyAsync(h->fbody, f_body, 2 * np * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    h->has_fbody = f_body != nullptr;
    if (s) {
        if (!h->src && (rc = dev_alloc(h, (void **)&h->src, np * sizeof(double)))) return rc;
        CUDA_TRY(cudaMemcpyAsync(h->src, s, np * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    h->has_src = s != nullptr;
    h->se_stale = true;
    h->ft_fresh = false;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    // captured steps read the source buffers when they run; only a new buffer or
    // a source switched on or off makes them stale
    if (h->fbody != fb0 || h->src != s0 || h->has_fbody != hf0 || h->has_src != hs0) drop_graphs(h);
    h->solved = false;  // the elastic solve at the current time must see the new data
    return BIOT_OK;
}

int biot_set_side_profile(biot_handle h, int side, const double *eta_profile, const double *p_profile)
{
    if (!h || side < 0 || side > 3) return fail(BIOT_ERR_INVALID_ARG, "bad handle or side");
    const double *e0 = h->eta_prof[side], *p0 = h->p_prof[side];
    int rc = set_profiles_staged(h, side, eta_profile, p_profile);
    if (rc) return rc;
    // captured launches read the profile buffers when they run; only a newly
    // allocated buffer makes them stale
    if (h->eta_prof[side] != e0 || h->p_prof[side] != p0) drop_graphs(h);
    return BIOT_OK;
}

int biot_step(biot_handle h, int n)
{
    if (!h || n < 0) return fail(BIOT_ERR_INVALID_ARG, "bad handle or step count");
    if (h->diverged) return fail(BIOT_ERR_DIVERGED, "instance has diverged");
    int rc, status = BIOT_OK;
    if ((rc = ensure_initialized(h))) return rc;
    if (!h->solved) {
        rc = elastic_solve(h);
        if (rc == BIOT_ERR_NOT_CONVERGED) status = rc;
        else if (rc) return rc;
    }
    // Each step is one graph launch (fixed V-cycles, or the tolerance mode's
    // device-side loop); nothing is read back until the end: a diverged state
    // stays non-finite, so the last residual reveals it.
    const bool graphs = h->use_graphs && !h->timing;
    const int notconv0 = h->notconv_steps;
    for (int i = 0; i < n; i++) {
        if (!graphs && h->P.ne_fixed <= 0 && (rc = finish_pending(h))) return rc;
        rc = graphs ? advance_graph(h) : advance(h);
        if (rc == BIOT_ERR_NOT_CONVERGED) status = rc;
        else if (rc) return rc;
    }
    if ((rc = finish_pending(h))) return rc;
    if (h->notconv_steps > notconv0) status = BIOT_ERR_NOT_CONVERGED;
    h->notconv_reported = h->notconv_steps;
    return status;
}

int biot_step_async(biot_handle h, int n)
{
    if (!h || n < 0) return fail(BIOT_ERR_INVALID_ARG, "bad handle or step count");
    if (h->diverged) return fail(BIOT_ERR_DIVERGED, "instance has diverged");
    const bool graphs = h->use_graphs && !h->timing;
    if (!graphs && h->P.ne_fixed <= 0) {  // host-driven V-cycle loop: reads back after every step
        const int rc = biot_step(h, n);
        return rc == BIOT_ERR_NOT_CONVERGED ? BIOT_OK : rc;
    }
    int rc;
    if ((rc = ensure_initialized(h))) return rc;
    if (!h->solved) {
        rc = elastic_solve(h);
        if (rc && rc != BIOT_ERR_NOT_CONVERGED) return rc;
    }
    for (int i = 0; i < n; i++) {
        rc = graphs ? advance_graph(h) : advance(h);
        if (rc && rc != BIOT_ERR_NOT_CONVERGED) return rc;
    }
    return BIOT_OK;
}

int biot_sync(biot_handle h)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (h->copy_stream) {
        CUDA_TRY(cudaStreamSynchronize(h->copy_stream));
        h->ainflight[0] = h->ainflight[1] = false;
    }
    const int rc = finish_pending(h);
    if (rc) return rc;
    const bool nc = h->notconv_steps > h->notconv_reported;
    h->notconv_reported = h->notconv_steps;
    return nc ? BIOT_ERR_NOT_CONVERGED : BIOT_OK;
}

int biot_solve_to(biot_handle h, double T)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    const long target = (long)std::floor(T / h->P.dt + 0.5);
    if (target < h->nstep) return fail(BIOT_ERR_INVALID_ARG, "target time lies before the current time");
    return biot_step(h, (int)(target - h->nstep));
}

int biot_read_u(biot_handle h, double *eta, double *t_out)
{
    if (!h || !eta) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    int rc = readout(h, eta, nullptr, nullptr);
    if (t_out) *t_out = h->P.dt * (double)h->nstep;
    return rc;
}

int biot_read_p(biot_handle h, double *p, double *t_out)
{
    if (!h || !p) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    int rc = readout(h, nullptr, p, nullptr);
    if (t_out) *t_out = h->P.dt * (double)h->nstep;
    return rc;
}

int biot_read_stress(biot_handle h, double *sigma)
{
    if (!h || !sigma) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    return readout(h, nullptr, nullptr, sigma);
}

int biot_read_async(biot_handle h, double *eta, double *p, double *sigma, double *t_out)
{
    if (!h || (!eta && !p && !sigma)) return fail(BIOT_ERR_INVALID_ARG, "null handle or no output");
    int rc = read_async(h, eta, p, sigma);
    if (t_out) *t_out = h->P.dt * (double)h->nstep;
    return rc;
}

int biot_read_wait(biot_handle h)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    if (!h->copy_stream) return BIOT_OK;
    CUDA_TRY(cudaStreamSynchronize(h->copy_stream));
    h->ainflight[0] = h->ainflight[1] = false;
    return BIOT_OK;
}

int biot_stats_get(biot_handle h, biot_stats *o)
{
    if (!h || !o) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    int rc = finish_pending(h);
    o->last_ne = h->last_ne;
    o->last_res = h->last_res;
    o->last_res_l2 = h->last_res_l2;
    o->total_cycles = h->total_cycles;
    o->notconv_steps = h->notconv_steps;
    o->diverged = h->diverged;
    o->nstep = h->nstep;
    o->t = h->P.dt * (double)h->nstep;
    o->omega = h->omega;
    o->omega_s = h->om_s;
    o->omega_d = h->om_d;
    o->kernel_launches = h->launches;
    o->device_bytes = h->bytes;
    return rc == BIOT_ERR_DIVERGED ? BIOT_OK : rc;
}

int biot_sweep_timing(biot_handle h, int enable)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->timing = enable != 0;
    h->ev_used = 0;
    return BIOT_OK;
}

int biot_sweep_timing_get(biot_handle h, double *ms_total, long *launches)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    double total = 0.0;
    for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
        total += ms;
    }
    if (ms_total) *ms_total = total;
    if (launches) *launches = (long)(h->ev_used / 2);
    return BIOT_OK;
}

}  // extern "C"

// ============================================================================
// Read-out through a static device array (no allocation; see biot.h).
// ============================================================================
namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
// Staging array of biot_read_u_noalloc: the 2 displacement planes of at most
// BIOT_NOALLOC_MAX_CELLS cells.  In host code this name is only a stand-in for
// the device symbol; kernels get the address looked up by noalloc_scratch().
static __device__ __align__(256) double g_noalloc_eta[2 * (size_t)BIOT_NOALLOC_MAX_CELLS];

std::mutex g_noalloc_mu;
double *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the staging array on device dev, looked up once per device
// with that device current (the caller has checked that it is).
int noalloc_scratch(int dev, double **out)
{
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(BIOT_ERR_INVALID_ARG, "device ordinal out of range for the static read-out array");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_eta);
        if (e != cudaSuccess || !p)
            return fail(BIOT_ERR_CUDA, std::string("cudaGetSymbolAddress(static read-out array): ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_addr[dev];
    return BIOT_OK;
}

}  // namespace

extern "C" int biot_read_u_noalloc(biot_handle h, double *eta, double *t_out)
{
    if (!h || !eta) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    const size_t np = (size_t)h->P.nx * h->P.ny;
    if (np > (size_t)BIOT_NOALLOC_MAX_CELLS)
        return fail(BIOT_ERR_INVALID_ARG, "biot_read_u_noalloc: the grid has " + std::to_string(np) +
                                              " cells, more than the static read-out array holds (" +
                                              std::to_string(BIOT_NOALLOC_MAX_CELLS) + "); use biot_read_u");
    int cur = -1;
    CUDA_TRY(cudaGetDevice(&cur));
    if (cur != h->device)
        return fail(BIOT_ERR_INVALID_ARG, "biot_read_u_noalloc: the instance lives on device " + std::to_string(h->device) +
                                              " but device " + std::to_string(cur) + " is current; make it current first");
    // the solve at t = 0 of a large FP32 instance runs on an FP64 copy that
    // biot_create allocates: not on this path
    if (h->cold64 && h->nstep == 0 && !h->solved)
        return fail(BIOT_ERR_INVALID_ARG, "biot_read_u_noalloc: the pending solve at t = 0 of this instance allocates "
                                          "an FP64 copy; step it (biot_step) or read it with biot_read_u first");
    double *scratch = nullptr;
    int rc = noalloc_scratch(h->device, &scratch);
    if (rc) return rc;
    if ((rc = ensure_initialized(h))) return rc;
    if (!h->solved) {  // as biot_read_u: a step that hit ne_max still reads out
        rc = elastic_solve(h);
        if (rc && rc != BIOT_ERR_NOT_CONVERGED) return rc;
    }
    if ((rc = finish_pending(h))) return rc;
    rc = h->fp32 ? readout_typed<float>(h, scratch, nullptr, nullptr) : readout_typed<double>(h, scratch, nullptr, nullptr);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(eta, scratch, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (t_out) *t_out = h->P.dt * (double)h->nstep;
    return BIOT_OK;
}

// ============================================================================
// Batched execution of many instances (one CUDA graph per time step).
//
// Every instance keeps its own state and runs exactly the sweeps and flow steps
// of biot_step; only their launches are regrouped.  The V-cycles of all
// instances are aligned at the coarsest level: the down-legs end together and
// the up-legs start together, so a phase holds one level index of every
// instance deep enough to have it, and an instance with fewer levels waits in
// the outer phases.  Each phase is one work-list launch per storage kind, whose
// CTAs take strips (or, for levels of at most 128^2 cells and FP64 levels,
// tiles) of sweeps of different instances; the flow steps of all instances are
// one work-list launch.
// ============================================================================
namespace {

// In a batch, levels of at most this many cells run as tiles: a 128^2 level's
// rows would fill only 128 of the 248 columns of two strips.
constexpr long BATCH_TILE_MAX_CELLS = 128L * 128L;
// Whether the depth groups' branches of the step graph run at descending stream
// priorities, deepest first.
constexpr bool BATCH_BRANCH_PRIORITIES = true;
// Whether a batch runs the 2K sweeps of each instance's FP64 coarsest level as
// one segment launch (one cluster per instance) rather than 2K phase launches.
constexpr bool BATCH_COARSEST_SEGMENT = true;
long batch_tile_max_cells() { return BATCH_TILE_MAX_CELLS; }

// One sweep of the static schedule of an instance, or one segment (fam >= 0:
// a run of sweeps of one storage family, launched as one program).
struct PlanOp {
    int level, mode, key;
    int fam = -1;
};

// Mirror of vcycle(): the sweeps of one V-cycle from level l down, with their
// phase keys.  Instances are aligned at the coarsest level (level index 0): the
// down-legs end together and the up-legs start together, so every phase holds
// the same level index -- the same level size for hierarchies with equal
// coarsest grids -- of all instances deep enough to have it, and the FP64
// coarsest sweeps of all instances share their 2K phases.  Dmax: deepest
// coarsest-level index over the batch.
void plan_vcycle(const biot_ctx *h, int l, int K, int Dmax, std::vector<PlanOp> &out)
{
    // K: the largest per-level sweep count of the batch (the key spacing); this
    // level runs its own count Kl <= K of the sweeps of each leg
    const int Kl = sweeps_of(&h->P, l);
    const int bottom = Dmax * (K + 1);  // first key of the coarsest sweeps
    for (int k = 0; k < Kl; k++) out.push_back({l, SWEEP_SMOOTH, l == 0 ? bottom + k : (Dmax - l) * (K + 1) + k});
    if (l > 0) {
        out.push_back({l, SWEEP_RESTRICT, (Dmax - l) * (K + 1) + K});
        plan_vcycle(h, l - 1, K, Dmax, out);
    }
    for (int k = 0; k < Kl; k++)
        out.push_back({l, SWEEP_SMOOTH, l == 0 ? bottom + K + k : bottom + 2 * K + (l - 1) * K + k});
}

// The ops of the segments of one V-cycle's plan collapsed as seg_vcycle
// records them: the ops of the levels at or below the segment's start level are
// contiguous (the coarse-grid correction), and each run of one storage family
// among them becomes one op at the key of its first sweep.
void plan_segments(const biot_ctx *h, std::vector<PlanOp> &ops)
{
    const int s = seg_start(h, false);
    if (s < 0) return;
    std::vector<PlanOp> out;
    for (size_t i = 0; i < ops.size();) {
        if (ops[i].level > s) {
            out.push_back(ops[i++]);
            continue;
        }
        const int fam = h->lv[ops[i].level].fp64 ? 0 : 1;
        PlanOp m = ops[i];
        m.fam = fam;
        size_t j = i;
        while (j < ops.size() && ops[j].level <= s && (h->lv[ops[j].level].fp64 ? 0 : 1) == fam) j++;
        out.push_back(m);
        i = j;
    }
    ops.swap(out);
}

int op_tkind(const biot_ctx *h, const PlanOp &o);
int op_variant(const biot_ctx *h, const PlanOp &o);

int level_tkind(const biot_ctx *h, int l)
{
    const bool t64 = h->lv[l].fp64;
    const bool c64 = (l > 0) ? h->lv[l - 1].fp64 : t64;
    return t64 ? 0 : (c64 ? 1 : 2);
}

int level_variant(const biot_ctx *h, int l, int mode)
{
    const bool fine = l == h->L - 1;
    // in a batch the launches of a phase are large: strips except for the
    // smallest levels and FP64 levels
    const bool tile = (long)h->lv[l].nx * h->lv[l].ny <= batch_tile_max_cells() || h->lv[l].fp64;
    return (fine ? 0 : SWEEP_V_COARSE) | (level_lo(h, l, false) ? SWEEP_V_LO : 0) |
           (mode == SWEEP_RESTRICT ? SWEEP_V_RESTRICT : 0) | (h->P.ne_fixed > 0 ? SWEEP_V_NOGHOST : 0) |
           (tile ? SWEEP_V_TILE : 0) | (fine && h->dev == 1 ? SWEEP_V_DEV16 : 0) | (fine && h->dev == 2 ? SWEEP_V_DEVBF16 : 0);
}

int op_tkind(const biot_ctx *h, const PlanOp &o)
{
    return o.fam >= 0 ? (o.fam == 0 ? 0 : 2) : level_tkind(h, o.level);
}

int op_variant(const biot_ctx *h, const PlanOp &o)
{
    if (o.fam >= 0) return SWEEP_V_SEGMENT | (h->P.ne_fixed > 0 ? SWEEP_V_NOGHOST : 0);
    return level_variant(h, o.level, o.mode);
}

// Strip heights of one batched launch (levels of nx x ny cells): the fewest whole
// waves of `slots` resident CTAs whose share per level (in proportion to its
// cells) gives strips of at most sweep_rows_cap() rows.  Each level's strips
// stay within its share, so the launch's items never spill into a further,
// almost empty wave.  Heights are even and at least 2.
std::vector<int> batch_strip_rows(const std::vector<std::pair<int, int>> &dims, int slots)
{
    double cells = 0;
    for (const auto &d : dims) cells += (double)d.first * d.second;
    const int cap = sweep_rows_cap();
    std::vector<int> ty(dims.size(), 2);
    for (int waves = 1; waves <= 64; waves++) {
        bool ok = true;
        for (size_t g = 0; g < dims.size(); g++) {
            const int nx = dims[g].first, ny = dims[g].second;
            const long sx = (nx + BATCH_STRIP_COLS - 1) / BATCH_STRIP_COLS;
            const long share = (long)((double)waves * slots * ((double)nx * ny) / cells);
            long nsy = share / sx;
            if (nsy < 1) nsy = 1;
            long t = (ny + nsy - 1) / nsy;
            t += t & 1;
            if (t < 2) t = 2;
            ty[g] = (int)t;
            if (t > cap) ok = false;
        }
        if (ok) break;
    }
    return ty;
}

int tkind_slots(int tkind, int variant)
{
    return tkind == 0 ? sweep_slots<double, double>(variant)
         : tkind == 1 ? sweep_slots<float, double>(variant) : sweep_slots<float, float>(variant);
}

// The same for the single-instance strip kernel.
int tkind_strip_slots(int tkind, int variant)
{
    return tkind == 0 ? sweep_strip_slots<double, double>(variant)
         : tkind == 1 ? sweep_strip_slots<float, double>(variant) : sweep_strip_slots<float, float>(variant);
}

// One launch of the batched schedule.
struct BatchLaunch {
    int tkind, variant;
    size_t job_off, item_off;  // offsets into slots[tkind] and into the work items
    int njobs, nitems;
    int group;                 // the depth group whose branch of the step graph launches it
};

// A job of the schedule: which instance's which recorded sweep fills it.
struct BatchSlot {
    int inst, op;  // op: index into the instance's recorded sweeps of one step
};

}  // namespace

struct biot_batch_s {
    std::vector<biot_ctx *> inst;
    cudaStream_t stream = nullptr;
    int K = 0, ne = 0, Dmax = 0;
    std::vector<BatchLaunch> launches;            // in issue order
    std::vector<BatchSlot> slots[3];              // per tkind: the recorded sweep of each job
    std::vector<SweepItem> items;
    std::vector<size_t> nops;                     // recorded sweeps per instance and step
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::vector<long> epoch[2];                   // instance epochs the graphs were captured at
    // batched flow steps: per storage type (0 FP32, 1 FP64) the instances and their
    // tile work items
    std::vector<int> flow_inst[2];
    std::vector<SweepItem> flow_items[2];
    void *flow_dev[2][2] = {};                    // per graph parity, per type: FlowFusedArgs tables
    SweepItem *flow_items_dev[2] = {};
    long launches_per_step = 0, kernel_launches = 0, nstep = 0;
    std::vector<void *> allocs;
    // instances of equal depth (multigrid levels) form a group; the groups' phase
    // launches are independent chains, captured as parallel branches of the step
    // graph on streams of their own
    int ngroups = 1;
    std::vector<int> group_of;
    std::vector<cudaStream_t> branch;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
};

namespace {

int batch_alloc(biot_batch_s *b, void **p, size_t bytes)
{
    *p = nullptr;
    if (!bytes) return BIOT_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? BIOT_ERR_OOM : BIOT_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b->allocs.push_back(*p);
    return BIOT_OK;
}

// Static schedule of one time step: phases by key, launches per storage kind,
// strip work items sized so that each launch fills the GPU.
int batch_plan(biot_batch_s *b)
{
    const int n = (int)b->inst.size();
    std::vector<std::vector<PlanOp>> ops(n);
    // depth groups: instances with the same number of levels
    std::vector<int> depths;
    for (biot_ctx *h : b->inst)
        if (std::find(depths.begin(), depths.end(), h->L) == depths.end()) depths.push_back(h->L);
    std::sort(depths.begin(), depths.end(), std::greater<int>());  // deepest (usually largest) first
    b->ngroups = (int)depths.size();
    b->group_of.assign(n, 0);
    for (int i = 0; i < n; i++)
        b->group_of[i] = (int)(std::find(depths.begin(), depths.end(), b->inst[i]->L) - depths.begin());
    b->nops.assign(n, 0);
    std::vector<int> maxkey(b->ngroups, 0);
    for (int i = 0; i < n; i++) {
        const int Dg = b->inst[i]->L - 1;  // the group's depth: its own coarsest level aligns its V-cycles
        const int up = Dg * (b->K + 1) + 2 * b->K + Dg * b->K;
        std::vector<PlanOp> cyc;
        plan_vcycle(b->inst[i], b->inst[i]->L - 1, b->K, Dg, cyc);
        plan_segments(b->inst[i], cyc);
        for (int c = 0; c < b->ne; c++)
            for (const PlanOp &o : cyc) ops[i].push_back({o.level, o.mode, c * up + o.key, o.fam});
        b->nops[i] = ops[i].size();
        int &mk = maxkey[b->group_of[i]];
        for (const PlanOp &o : ops[i]) mk = o.key > mk ? o.key : mk;
    }
    b->launches.clear();
    b->items.clear();
    for (int t = 0; t < 3; t++) b->slots[t].clear();
    for (int g = 0; g < b->ngroups; g++) {
    // bucket the group's ops by key, then by (tkind, variant)
    std::vector<std::vector<BatchSlot>> bykey(maxkey[g] + 1);
    for (int i = 0; i < n; i++)
        if (b->group_of[i] == g)
            for (size_t j = 0; j < ops[i].size(); j++) bykey[ops[i][j].key].push_back({i, (int)j});
    for (int key = 0; key <= maxkey[g]; key++) {
        for (int tk = 0; tk < 3; tk++) {
            for (int v = 0; v < 256; v++) {  // every combination of the SWEEP_V_* flags
                std::vector<BatchSlot> grp;
                for (const BatchSlot &s : bykey[key]) {
                    const biot_ctx *h = b->inst[s.inst];
                    const PlanOp &o = ops[s.inst][s.op];
                    if (op_tkind(h, o) != tk || op_variant(h, o) != v) continue;
                    grp.push_back(s);
                }
                if (grp.empty()) continue;
                if (v & SWEEP_V_SEGMENT) {  // segments: one program per job, no work items
                    BatchLaunch L{tk, v, b->slots[tk].size(), b->items.size(), (int)grp.size(), 0, g};
                    for (const BatchSlot &sl : grp) b->slots[tk].push_back(sl);
                    b->launches.push_back(L);
                    continue;
                }
                const bool tile = (v & SWEEP_V_TILE) != 0;
                const int slots = tile ? 1 : tkind_slots(tk, v & ~SWEEP_V_TILE);
                if (!slots) return fail(BIOT_ERR_CUDA, "occupancy query of the batched sweep kernel failed");
                BatchLaunch L{tk, v, b->slots[tk].size(), b->items.size(), (int)grp.size(), 0, g};
                std::vector<int> tys;
                if (!tile) {
                    std::vector<std::pair<int, int>> dims;
                    for (const BatchSlot &s : grp) {
                        const Level &Lv = b->inst[s.inst]->lv[ops[s.inst][s.op].level];
                        dims.push_back({Lv.nx, Lv.ny});
                    }
                    tys = batch_strip_rows(dims, slots);
                }
                for (size_t g = 0; g < grp.size(); g++) {
                    const biot_ctx *h = b->inst[grp[g].inst];
                    const Level &Lv = h->lv[ops[grp[g].inst][grp[g].op].level];
                    if (tile) {  // tiles of the tile sweep
                        int tx, ty;
                        sweep_tile_shape(tk == 0, &tx, &ty);
                        for (int by = 0; by < (Lv.ny + ty - 1) / ty; by++)
                            for (int bx = 0; bx < (Lv.nx + tx - 1) / tx; bx++) b->items.push_back({(int)g, bx, by, 0});
                    } else {  // strips sized so that the launch fills whole waves of the GPU
                        const int ty = tys[g];
                        const int sx = (Lv.nx + BATCH_STRIP_COLS - 1) / BATCH_STRIP_COLS, sy = (Lv.ny + ty - 1) / ty;
                        for (int by = 0; by < sy; by++)
                            for (int bx = 0; bx < sx; bx++) b->items.push_back({(int)g, bx, by, ty});
                    }
                    b->slots[tk].push_back(grp[g]);
                }
                L.nitems = (int)(b->items.size() - L.item_off);
                b->launches.push_back(L);
            }
        }
    }
    }
    // the branch streams and the fork / join events of the step graph
    // the deepest group (usually the largest instances: the step's critical
    // path) gets the highest stream priority, the next ones lower ones; the
    // captured kernel nodes keep their stream's priority
    int prio_least = 0, prio_greatest = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    while ((int)b->branch.size() < b->ngroups) {
        cudaStream_t st;
        const int g = (int)b->branch.size();
        const int prio = BATCH_BRANCH_PRIORITIES ? std::min(prio_greatest + g, prio_least) : prio_least;
        CUDA_TRY(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio));
        b->branch.push_back(st);
        cudaEvent_t ev;
        CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        b->ev_join.push_back(ev);
    }
    if (!b->ev_fork) CUDA_TRY(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    // flow steps: one job per instance
    for (int t = 0; t < 2; t++) {
        b->flow_inst[t].clear();
        b->flow_items[t].clear();
    }
    for (int i = 0; i < n; i++) {
        const biot_ctx *h = b->inst[i];
        const int t = h->fp32 ? 0 : 1;
        const int job = (int)b->flow_inst[t].size();
        b->flow_inst[t].push_back(i);
        for (int by = 0; by < (h->P.ny + FLOW_TILE_Y - 1) / FLOW_TILE_Y; by++)
            for (int bx = 0; bx < (h->P.nx + FLOW_TILE_X - 1) / FLOW_TILE_X; bx++) b->flow_items[t].push_back({job, bx, by, 0});
    }
    int rc;
    for (int par = 0; par < 2; par++) {
        if ((rc = batch_alloc(b, &b->flow_dev[par][0], b->flow_inst[0].size() * sizeof(FlowFusedArgs<float>)))) return rc;
        if ((rc = batch_alloc(b, &b->flow_dev[par][1], b->flow_inst[1].size() * sizeof(FlowFusedArgs<double>)))) return rc;
    }
    for (int t = 0; t < 2; t++) {
        if ((rc = batch_alloc(b, (void **)&b->flow_items_dev[t], b->flow_items[t].size() * sizeof(SweepItem)))) return rc;
        if (!b->flow_items[t].empty())
            CUDA_TRY(cudaMemcpy(b->flow_items_dev[t], b->flow_items[t].data(), b->flow_items[t].size() * sizeof(SweepItem), cudaMemcpyHostToDevice));
    }
    return BIOT_OK;
}

// One planned launch of the batch as launches of at most BATCH_MAX_JOBS jobs,
// each with its parameter block: the recorded arguments of its sweeps and the
// geometry of their work items (job-major, row by row, as batch_plan lays them out).
template <typename T, typename TC>
cudaError_t batch_launch_typed(biot_batch_s *b, const BatchLaunch &L, std::vector<std::vector<SweepJob>> &rec,
                               cudaStream_t stream)
{
    std::unique_ptr<BatchParams<T, TC>> P(new (std::nothrow) BatchParams<T, TC>());
    if (!P) return cudaErrorMemoryAllocation;
    size_t it = L.item_off;
    const size_t it_end = L.item_off + L.nitems;
    for (int g0 = 0; g0 < L.njobs; g0 += BATCH_MAX_JOBS) {
        const int nj = std::min(BATCH_MAX_JOBS, L.njobs - g0);
        P->njobs = nj;
        int count = 0;
        for (int k = 0; k < nj; k++) {
            const BatchSlot &sl = b->slots[L.tkind][L.job_off + g0 + k];
            P->job[k] = job_args<T, TC>(rec[sl.inst][sl.op]);
            P->start[k] = count;
            P->sx[k] = 1;
            P->ty[k] = 0;
            for (; it < it_end && b->items[it].job == g0 + k; it++, count++) {
                const SweepItem &w = b->items[it];
                P->sx[k] = std::max(P->sx[k], w.bx + 1);
                P->ty[k] = w.ty;
            }
        }
        P->start[nj] = count;
        cudaError_t e = launch_sweep_batch<T, TC>(L.variant, *P, stream);
        if (e != cudaSuccess) return e;
    }
    return it == it_end ? cudaSuccess : cudaErrorInvalidValue;
}

// A planned launch of segments: the programs of its jobs packed into as few
// launches as the parameter block allows (*nl: how many).
cudaError_t batch_launch_segments(biot_batch_s *b, const BatchLaunch &L, std::vector<std::vector<SweepJob>> &rec,
                                  std::vector<std::vector<SegProg>> &segrec, cudaStream_t stream, long *nl)
{
    std::unique_ptr<SegParams> P(new (std::nothrow) SegParams());
    if (!P) return cudaErrorMemoryAllocation;
    const int fam = L.tkind == 0 ? 0 : 1;
    int cs = 1;
    auto reset = [&]() {
        P->nprog = 0;
        P->ghosts = (L.variant & SWEEP_V_NOGHOST) ? 0 : 1;
        P->lev0[0] = P->job0[0] = 0;
        cs = 1;
    };
    reset();
    for (int k = 0; k < L.njobs; k++) {
        const BatchSlot &sl = b->slots[L.tkind][L.job_off + k];
        const int gi = rec[sl.inst][sl.op].seg;
        if (gi < 0 || gi >= (int)segrec[sl.inst].size()) return cudaErrorInvalidValue;
        const SegProg &g = segrec[sl.inst][gi];
        if (g.fam != fam) return cudaErrorInvalidValue;
        if (!seg_pack(*P, g)) {
            if (P->nprog == 0) return cudaErrorInvalidValue;
            cudaError_t e = seg_launch(fam, *P, cs, stream);
            if (e != cudaSuccess) return e;
            (*nl)++;
            reset();
            if (!seg_pack(*P, g)) return cudaErrorInvalidValue;
        }
        cs = std::max(cs, g.cs);
    }
    if (P->nprog > 0) {
        cudaError_t e = seg_launch(fam, *P, cs, stream);
        if (e != cudaSuccess) return e;
        (*nl)++;
    }
    return cudaSuccess;
}

// Capture one time step of every instance (parity par of the flow buffers).
int batch_capture(biot_batch_s *b, int par)
{
    const int n = (int)b->inst.size();
    std::vector<std::vector<SweepJob>> rec(n);
    std::vector<std::vector<SegProg>> segrec(n);
    std::vector<FlowRec> frec;
    std::vector<long> l0(n), c0(n);
    CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = BIOT_OK;
    long nl = 0;
    for (int i = 0; i < n && !rc; i++) {
        biot_ctx *h = b->inst[i];
        l0[i] = h->launches;
        c0[i] = h->total_cycles;
        h->rec = &rec[i];
        h->frec = &frec;
        h->segrec = &segrec[i];
        rc = advance(h);  // flow steps and sweeps are recorded, launched below for all instances
        h->rec = nullptr;
        h->frec = nullptr;
        h->segrec = nullptr;
        if (!rc && frec.size() != (size_t)i + 1) rc = fail(BIOT_ERR_CUDA, "batched schedule: flow step not recorded");
        nl += h->launches - l0[i];
        if (!rc && rec[i].size() != b->nops[i]) rc = fail(BIOT_ERR_CUDA, "batched schedule does not match the recorded sweeps");
    }
    // every recorded sweep must be planned, and of the kind its planned launch instantiates
    {
        size_t planned = 0;
        for (const BatchLaunch &L : b->launches) planned += (size_t)L.njobs;
        size_t recorded = 0;
        for (int i = 0; i < n; i++) recorded += rec[i].size();
        if (!rc && planned != recorded) rc = fail(BIOT_ERR_CUDA, "batched schedule: a recorded sweep has no planned launch");
    }
    for (size_t k = 0; k < b->launches.size() && !rc; k++) {
        const BatchLaunch &L = b->launches[k];
        for (int j = 0; j < L.njobs && !rc; j++) {
            const BatchSlot &sl = b->slots[L.tkind][L.job_off + j];
            const SweepJob &r = rec[sl.inst][sl.op];
            if (r.tkind != L.tkind || r.variant != (L.variant & ~SWEEP_V_TILE))
                rc = fail(BIOT_ERR_CUDA, "batched schedule: a recorded sweep differs from its planned kind");
        }
    }
    // flow steps of all instances
    if (!rc && !b->flow_items[0].empty()) {
        cudaError_t e = launch_flow_fused_batch<float>(static_cast<const FlowFusedArgs<float> *>(b->flow_dev[par][0]),
                                                       b->flow_items_dev[0], (int)b->flow_items[0].size(), b->stream);
        if (e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("batched flow launch: ") + cudaGetErrorString(e));
        nl++;
    }
    if (!rc && !b->flow_items[1].empty()) {
        cudaError_t e = launch_flow_fused_batch<double>(static_cast<const FlowFusedArgs<double> *>(b->flow_dev[par][1]),
                                                        b->flow_items_dev[1], (int)b->flow_items[1].size(), b->stream);
        if (e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("batched flow launch: ") + cudaGetErrorString(e));
        nl++;
    }
    // the groups' phase launches as parallel branches (one group: on the main stream)
    const bool fork = b->ngroups > 1;
    if (!rc && fork) {
        cudaError_t e = cudaEventRecord(b->ev_fork, b->stream);
        for (int g = 0; g < b->ngroups && e == cudaSuccess; g++) e = cudaStreamWaitEvent(b->branch[g], b->ev_fork, 0);
        if (e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("batched graph fork: ") + cudaGetErrorString(e));
    }
    for (size_t k = 0; k < b->launches.size() && !rc; k++) {
        const BatchLaunch &L = b->launches[k];
        const cudaStream_t st = fork ? b->branch[L.group] : b->stream;
        if (L.variant & SWEEP_V_SEGMENT) {
            cudaError_t e = batch_launch_segments(b, L, rec, segrec, st, &nl);
            if (e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("batched segment launch: ") + cudaGetErrorString(e));
            continue;
        }
        cudaError_t e = L.tkind == 0 ? batch_launch_typed<double, double>(b, L, rec, st)
                      : L.tkind == 1 ? batch_launch_typed<float, double>(b, L, rec, st)
                                     : batch_launch_typed<float, float>(b, L, rec, st);
        if (e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("batched sweep launch: ") + cudaGetErrorString(e));
        nl++;
    }
    if (fork) {  // join every branch, also after an error, so that the capture can end
        for (int g = 0; g < b->ngroups; g++) {
            cudaError_t e = cudaEventRecord(b->ev_join[g], b->branch[g]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_join[g], 0);
            if (!rc && e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("batched graph join: ") + cudaGetErrorString(e));
        }
    }
    for (int i = 0; i < n && !rc; i++) {
        biot_ctx *h = b->inst[i];
        cudaError_t e = cudaMemcpyAsync(h->resmax_host, h->resmax, RES_WORDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream);
        if (e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (!rc && e != cudaSuccess) rc = fail(BIOT_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    if (!rc) {
        e = cudaGraphInstantiate(&b->graph[par], g, BATCH_BRANCH_PRIORITIES ? cudaGraphInstantiateFlagUseNodePriority : 0);
        if (e != cudaSuccess) {
            b->graph[par] = nullptr;
            rc = fail(BIOT_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
    }
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    {
        std::vector<FlowFusedArgs<float>> ff;
        std::vector<FlowFusedArgs<double>> fd;
        for (int i : b->flow_inst[0]) ff.push_back(frec[i].f);
        for (int i : b->flow_inst[1]) fd.push_back(frec[i].d);
        if (!ff.empty()) CUDA_TRY(cudaMemcpy(b->flow_dev[par][0], ff.data(), ff.size() * sizeof(ff[0]), cudaMemcpyHostToDevice));
        if (!fd.empty()) CUDA_TRY(cudaMemcpy(b->flow_dev[par][1], fd.data(), fd.size() * sizeof(fd[0]), cudaMemcpyHostToDevice));
    }
    b->launches_per_step = nl;
    b->epoch[par].clear();
    for (int i = 0; i < n; i++) b->epoch[par].push_back(b->inst[i]->epoch);
    // capture recorded the state transitions; replay them from the start state
    for (int i = 0; i < n; i++) {
        biot_ctx *h = b->inst[i];
        h->launches = l0[i];
        h->total_cycles = c0[i];
        h->fcur ^= 1;
        std::swap(h->D1, h->D2);
        h->nstep -= 1;
    }
    return BIOT_OK;
}

void batch_release(biot_batch_s *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (cudaStream_t st : b->branch) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : b->ev_join) cudaEventDestroy(ev);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (int i = 0; i < 2; i++)
        if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
    for (void *p : b->allocs) cudaFree(p);
    for (biot_ctx *h : b->inst) release(h);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // namespace

extern "C" {

int biot_batch_create(int count, const biot_params *params, const biot_side *sides, biot_batch *out)
{
    if (!out) return fail(BIOT_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (count < 1 || !params || !sides) return fail(BIOT_ERR_INVALID_ARG, "need count >= 1 and parameter / side arrays");
    for (int i = 0; i < count; i++) {
        if (params[i].ne_fixed <= 0) return fail(BIOT_ERR_INVALID_ARG, "batched instances need a fixed number of V-cycles (ne_fixed > 0)");
        if (params[i].ne_fixed != params[0].ne_fixed)
            return fail(BIOT_ERR_INVALID_ARG, "batched instances need equal ne_fixed");
        if (params[i].cycle != BIOT_CYCLE_V || params[i].fmg)
            return fail(BIOT_ERR_INVALID_ARG, "batched instances run V-cycles (cycle = BIOT_CYCLE_V, fmg = 0)");
    }
    biot_batch_s *b = new (std::nothrow) biot_batch_s();
    if (!b) return fail(BIOT_ERR_OOM, "host allocation failed");
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        b->stream = nullptr;
        delete b;
        return fail(BIOT_ERR_CUDA, "cudaStreamCreate failed");
    }
    b->K = 1;  // the largest sweep count of any level of any instance (phase-key spacing)
    for (int i = 0; i < count; i++)
        for (int l = 0; l < params[i].mg_levels && l < BIOT_MAX_LEVELS; l++)
            b->K = std::max(b->K, sweeps_of(&params[i], l));
    b->ne = params[0].ne_fixed;
    for (int i = 0; i < count; i++) {
        biot_handle h = nullptr;
        int rc = biot_create(&params[i], &sides[4 * i], &h);
        if (rc) {
            const std::string msg = "instance " + std::to_string(i) + ": " + g_last_error;
            batch_release(b);
            return fail(rc, msg);
        }
        b->inst.push_back(h);
        h->batched = BATCH_COARSEST_SEGMENT;
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            batch_release(b);
            return fail(BIOT_ERR_CUDA, "instance set-up failed");
        }
        h->stream = b->stream;
        b->Dmax = h->L - 1 > b->Dmax ? h->L - 1 : b->Dmax;
    }
    int rc = batch_plan(b);
    if (rc) {
        batch_release(b);
        return rc;
    }
    *out = b;
    return BIOT_OK;
}

int biot_batch_destroy(biot_batch b)
{
    batch_release(b);
    return BIOT_OK;
}

int biot_batch_size(biot_batch b, int *count)
{
    if (!b || !count) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    *count = (int)b->inst.size();
    return BIOT_OK;
}

int biot_batch_instance(biot_batch b, int i, biot_handle *out)
{
    if (!b || !out || i < 0 || i >= (int)b->inst.size()) return fail(BIOT_ERR_INVALID_ARG, "bad batch, index or output");
    *out = b->inst[i];
    return BIOT_OK;
}

int biot_batch_step(biot_batch b, int n)
{
    int rc = biot_batch_step_async(b, n);
    return rc ? rc : biot_batch_sync(b);
}

int biot_batch_sync(biot_batch b)
{
    if (!b) return fail(BIOT_ERR_INVALID_ARG, "null batch");
    int status = BIOT_OK, rc;
    for (biot_ctx *h : b->inst)
        if ((rc = biot_sync(h)) && status != BIOT_ERR_DIVERGED && status != BIOT_ERR_CUDA) status = rc;
    return status;
}

int biot_batch_step_async(biot_batch b, int n)
{
    if (!b || n < 0) return fail(BIOT_ERR_INVALID_ARG, "bad batch or step count");
    int rc;
    for (biot_ctx *h : b->inst) {
        if (h->diverged) return fail(BIOT_ERR_DIVERGED, "an instance of the batch has diverged");
        if (h->stream != b->stream) return fail(BIOT_ERR_INVALID_ARG, "an instance of the batch was moved to another stream");
        if ((rc = ensure_initialized(h))) return rc;
        if (!h->solved) {
            rc = elastic_solve(h);
            if (rc && rc != BIOT_ERR_NOT_CONVERGED) return rc;
        }
    }
    const int par = b->inst[0]->fcur;
    for (biot_ctx *h : b->inst)
        if (h->fcur != par) return fail(BIOT_ERR_INVALID_ARG, "instances of the batch were stepped separately");
    for (int par2 = 0; par2 < 2; par2++) {  // re-capture after an instance's arguments changed
        bool stale = false;
        for (size_t i = 0; i < b->inst.size() && b->graph[par2]; i++)
            stale = stale || b->epoch[par2][i] != b->inst[i]->epoch;
        if (stale) {
            cudaGraphExecDestroy(b->graph[par2]);
            b->graph[par2] = nullptr;
        }
    }
    for (int s = 0; s < n; s++) {
        const int p = b->inst[0]->fcur;
        if (!b->graph[p] && (rc = batch_capture(b, p))) return rc;
        CUDA_TRY(cudaGraphLaunch(b->graph[p], b->stream));
        b->kernel_launches += b->launches_per_step;
        b->nstep++;
        for (biot_ctx *h : b->inst) {
            h->fcur ^= 1;
            std::swap(h->D1, h->D2);
            h->nstep += 1;
            h->total_cycles += h->P.ne_fixed;
            h->last_ne = h->P.ne_fixed;
            h->solved = true;
            h->pending_res = true;
        }
    }
    return BIOT_OK;
}

int biot_batch_stats_get(biot_batch b, long *kernel_launches, long *launches_per_step, long *work_items_per_step)
{
    if (!b) return fail(BIOT_ERR_INVALID_ARG, "null batch");
    if (kernel_launches) *kernel_launches = b->kernel_launches;
    if (launches_per_step) *launches_per_step = b->launches_per_step;
    if (work_items_per_step) *work_items_per_step = (long)b->items.size();
    return BIOT_OK;
}

int biot_batch_read_async(biot_batch b, double *const *eta, double *const *p, double *const *sigma, double *t_out)
{
    if (!b || (!eta && !p && !sigma)) return fail(BIOT_ERR_INVALID_ARG, "null batch or no output");
    for (size_t i = 0; i < b->inst.size(); i++) {
        double *e = eta ? eta[i] : nullptr, *q = p ? p[i] : nullptr, *sg = sigma ? sigma[i] : nullptr;
        if (!e && !q && !sg) continue;
        const int rc = read_async(b->inst[i], e, q, sg);
        if (rc) return rc;
        if (t_out) t_out[i] = b->inst[i]->P.dt * (double)b->inst[i]->nstep;
    }
    return BIOT_OK;
}

int biot_batch_read_wait(biot_batch b)
{
    if (!b) return fail(BIOT_ERR_INVALID_ARG, "null batch");
    for (biot_ctx *h : b->inst) {
        const int rc = biot_read_wait(h);
        if (rc) return rc;
    }
    return BIOT_OK;
}

}  // extern "C"

// ============================================================================
// Serving: a request loop with continuous batching.
//
// A scheduler thread admits queued requests while the device-memory budget and
// the resident-slot limit allow, keeps every admitted instance (populations and
// multigrid hierarchy) resident on its own stream, and in each tick launches the
// next time steps of all resident instances before waiting for any of them, so
// that their kernels overlap on the GPU.  A finished instance is read out into
// host memory and freed at once, which admits the next request.
// ============================================================================
namespace {

size_t estimate_bytes(const biot_params *p, const biot_side *sides)
{
    const bool fp32 = p->precision != BIOT_FP64;
    const size_t tsz = fp32 ? 4 : 8, np = (size_t)p->nx * p->ny;
    size_t b = 0;
    for (int l = 0; l < p->mg_levels; l++) {
        const int shift = p->mg_levels - 1 - l;
        const size_t nx = (size_t)(p->nx >> shift), ny = (size_t)(p->ny >> shift), n = nx * ny;
        const bool fp64 = !fp32 || (l == 0 && p->mg_levels > 1 && coarsest_fp64(p)) ||
                          (p->precision == BIOT_FP32_COARSE64 && l < p->mg_levels - 1);
        const size_t esz = fp64 ? 8 : 4;
        b += 2 * 8 * n * esz;
        if (!fp64 && (l == p->mg_levels - 1 || coarse_lo_mode(p) != COARSE_LO_OFF)) b += 2 * 2 * n * esz;
        if (l < p->mg_levels - 1) b += 8 * n * esz;
        if (l == p->mg_levels - 1 && (p->precision == BIOT_FP32_DEV16 || p->precision == BIOT_FP32_DEVBF16))
            b += 2 * 3 * n * 2;
        for (int s = 0; s < 4; s++)
            if (sides && sides[s].eta_type == BIOT_DIRICHLET) b += 3 * ((s == BIOT_BOTTOM || s == BIOT_TOP) ? nx : ny) * esz;
    }
    b += (2 * 9 + 2 + 2) * np * tsz + 3 * np * 8 + RES_WORDS * sizeof(unsigned long long) + sizeof(StopState);
    for (int s = 0; s < 4; s++) {
        const size_t m = 2 * (size_t)((s == BIOT_BOTTOM || s == BIOT_TOP) ? p->nx : p->ny) + 1;
        if (sides && sides[s].eta_profile) b += 2 * m * 8;
        if (sides && sides[s].p_profile) b += m * 8;
    }
    b += 6 * np * 8;  // read-out buffer
    return b;
}

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

struct Request {
    uint64_t id = 0;
    biot_params P{};
    biot_side sides[4]{};
    std::vector<double> prof[4][2];  // owned copies of the boundary data
    long target = 0;                 // physical steps to take
    size_t bytes = 0;
    size_t shadow = 0;   // transient FP64 copy of the solve at t = 0 (cold_start_fp64)
    bool cold64 = false;
    int state = REQ_QUEUED, status = BIOT_OK;
    std::string error;
    double t_submit = 0, t_start = 0, t_done = 0;
    biot_ctx *h = nullptr;
    int host_slot = -1;     // the instance's pinned mirrors in the server's arena
    bool inflight = false;  // launched work not yet seen complete on the instance's stream
    std::vector<double> eta, p;
    double t_result = 0;
};

}  // namespace

struct biot_server_s {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    size_t budget = 0, used = 0, peak_used = 0;
    int max_resident = 0, peak_resident = 0;
    uint64_t next_id = 1;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request> req;
    std::vector<Request *> resident;  // worker thread only (map entries are stable)
    std::chrono::steady_clock::time_point t0;
    long ticks = 0, graph_launches = 0;
    int device = 0;
    // device memory of the instances (stream-ordered, kept up to the budget) and
    // their pinned host mirrors, one arena slot per resident instance
    cudaMemPool_t pool = nullptr;
    unsigned char *host_arena = nullptr;
    std::vector<int> free_slots;  // worker thread only
    GraphCache gcache;            // worker thread only
    static constexpr size_t SLOT_BYTES = 256;
    static_assert(RES_WORDS * sizeof(unsigned long long) + sizeof(StopState) <= SLOT_BYTES, "arena slot");
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

// Finish a resident request (worker thread, lock not held while reading out).
void server_finish(biot_server_s *S, Request &r, int status, const std::string &err)
{
    if (status == BIOT_OK) {
        const size_t np = (size_t)r.P.nx * r.P.ny;
        r.eta.resize(2 * np);
        r.p.resize(np);
        // eta and p of one read-out pass (the fields biot_read_u and biot_read_p return)
        int rc = readout(r.h, r.eta.data(), r.p.data(), nullptr);
        r.t_result = r.h->P.dt * (double)r.h->nstep;
        if (rc) {
            status = rc;
            r.error = g_last_error;
        }
    } else {
        r.error = err;
    }
    if (status == BIOT_OK && r.h->use_graphs) {  // the step graphs serve the next request of this shape
        for (int par = 0; par < 2; par++) {
            if (!r.h->graph[par]) continue;
            S->gcache.put(graph_key(r.h), par, r.h->graph[par]);
            r.h->graph[par] = nullptr;
        }
    }
    release(r.h);
    r.h = nullptr;
    if (r.host_slot >= 0) S->free_slots.push_back(r.host_slot);
    r.host_slot = -1;
    std::lock_guard<std::mutex> lock(S->mu);
    S->used -= r.bytes;
    r.status = status;
    r.state = status == BIOT_OK ? REQ_DONE : REQ_FAILED;
    r.t_done = S->now();
    S->cv_done.notify_all();
}

void server_loop(biot_server_s *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        // admission: memory budget and resident slots
        std::vector<Request *> admit;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            if (S->resident.empty())
                S->cv_work.wait(lock, [&] { return S->stop || !S->queue.empty(); });
            if (S->stop) break;
            while (!S->queue.empty() && (int)(S->resident.size() + admit.size()) < S->max_resident) {
                Request &r = S->req[S->queue.front()];
                if (S->used + r.bytes + r.shadow > S->budget) break;
                S->used += r.bytes + r.shadow;
                S->peak_used = S->used > S->peak_used ? S->used : S->peak_used;
                r.state = REQ_RUNNING;
                r.t_start = S->now();
                admit.push_back(&r);
                S->queue.pop_front();
            }
        }
        for (Request *r : admit) {
            biot_handle h = nullptr;
            int rc;
            if (S->host_arena && !S->free_slots.empty()) {
                r->host_slot = S->free_slots.back();
                S->free_slots.pop_back();
                unsigned char *slot = S->host_arena + (size_t)r->host_slot * biot_server_s::SLOT_BYTES;
                const Lend lend{S->pool, reinterpret_cast<unsigned long long *>(slot),
                                reinterpret_cast<StopState *>(slot + RES_WORDS * sizeof(unsigned long long))};
                rc = create_instance(&r->P, r->sides, &h, &lend);
            } else {
                rc = create_instance(&r->P, r->sides, &h, nullptr);
            }
            if (!rc) {
                h->cold64 = r->cold64;
                h->gcache = &S->gcache;
                rc = ensure_initialized(h);
            }
            if (!rc) {
                rc = elastic_solve(h);  // the solve at t = 0 (launch-only with fixed V-cycles)
                if (rc == BIOT_ERR_NOT_CONVERGED) rc = BIOT_OK;
            }
            {
                std::lock_guard<std::mutex> lock(S->mu);  // the FP64 copy is gone
                S->used -= r->shadow;
                r->shadow = 0;
            }
            r->h = h;
            r->inflight = h != nullptr;  // the solve at t = 0 is queued on its stream
            if (rc) {
                const std::string err = g_last_error;
                if (h) server_finish(S, *r, rc, err);
                else {
                    if (r->host_slot >= 0) S->free_slots.push_back(r->host_slot);
                    r->host_slot = -1;
                    std::lock_guard<std::mutex> lock(S->mu);
                    S->used -= r->bytes;
                    r->status = rc;
                    r->error = err;
                    r->state = REQ_FAILED;
                    r->t_done = S->now();
                    S->cv_done.notify_all();
                }
                continue;
            }
            S->resident.push_back(r);
        }
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->peak_resident = (int)S->resident.size() > S->peak_resident ? (int)S->resident.size() : S->peak_resident;
        }
        if (S->resident.empty()) continue;
        // one pass over the residents: an instance whose stream has drained is
        // checked (residual read-back, divergence), then finished at its end time
        // or given its next few steps; the others keep running meanwhile
        const int per_pass = 4;
        bool progressed = false;
        std::vector<Request *> keep;
        for (Request *rp : S->resident) {
            Request &r = *rp;
            const cudaError_t q = r.inflight ? cudaStreamQuery(r.h->stream) : cudaSuccess;
            if (q == cudaErrorNotReady) {
                keep.push_back(rp);
                continue;
            }
            progressed = true;
            int rc = BIOT_OK;
            if (q != cudaSuccess) {
                cudaGetLastError();
                rc = fail(BIOT_ERR_CUDA, std::string("instance stream: ") + cudaGetErrorString(q));
            }
            if (!rc) rc = finish_pending(r.h);  // the stream is idle: no wait
            r.inflight = false;
            if (!rc && r.h->nstep >= r.target) {
                server_finish(S, r, BIOT_OK, "");
                continue;
            }
            for (int j = 0; j < per_pass && !rc && r.h->nstep < r.target; j++) {
                rc = r.h->use_graphs ? advance_graph(r.h) : advance(r.h);
                if (rc == BIOT_ERR_NOT_CONVERGED) rc = BIOT_OK;
                S->graph_launches++;
            }
            if (rc) {
                server_finish(S, r, rc, g_last_error);
                continue;
            }
            r.inflight = true;
            keep.push_back(rp);
        }
        S->resident.swap(keep);
        if (progressed) S->ticks++;
        else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    // shutdown: drop whatever is resident
    for (Request *r : S->resident) {
        if (r->h) release(r->h);
        r->h = nullptr;
        if (r->host_slot >= 0) S->free_slots.push_back(r->host_slot);
        r->host_slot = -1;
    }
    S->resident.clear();
}

}  // namespace

extern "C" {

int biot_estimate_bytes(const biot_params *p, const biot_side sides[4], size_t *bytes)
{
    if (!p || !bytes) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    int rc = check_params(p, sides);
    if (rc) return rc;
    *bytes = estimate_bytes(p, sides);
    return BIOT_OK;
}

int biot_server_create(size_t mem_budget_bytes, int max_resident, biot_server *out)
{
    if (!out) return fail(BIOT_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (mem_budget_bytes == 0 || max_resident < 1) return fail(BIOT_ERR_INVALID_ARG, "need a memory budget and max_resident >= 1");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(BIOT_ERR_NO_DEVICE, "no CUDA device visible");
    }
    biot_server_s *S = new (std::nothrow) biot_server_s();
    if (!S) return fail(BIOT_ERR_OOM, "host allocation failed");
    S->budget = mem_budget_bytes;
    S->max_resident = max_resident;
    S->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&S->device);
    // the instances' allocation sources; without them instances allocate as biot_create does
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaMemPoolCreate(&S->pool, &props) == cudaSuccess) {
        uint64_t keep = mem_budget_bytes;  // memory returned by finished instances stays mapped up to the budget
        cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
        cudaGetLastError();
        S->pool = nullptr;
    }
    if (cudaMallocHost((void **)&S->host_arena, (size_t)max_resident * biot_server_s::SLOT_BYTES) == cudaSuccess) {
        for (int i = max_resident - 1; i >= 0; i--) S->free_slots.push_back(i);
    } else {
        cudaGetLastError();
        S->host_arena = nullptr;
    }
    try {
        S->worker = std::thread(server_loop, S);
    } catch (...) {
        if (S->pool) cudaMemPoolDestroy(S->pool);
        if (S->host_arena) cudaFreeHost(S->host_arena);
        delete S;
        return fail(BIOT_ERR_OOM, "cannot start the scheduler thread");
    }
    *out = S;
    return BIOT_OK;
}

int biot_server_submit(biot_server S, const biot_params *p, const biot_side sides[4], double T, uint64_t *id)
{
    if (!S || !p || !sides || !id) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    int rc = check_params(p, sides);
    if (rc) return rc;
    if (!(T >= 0)) return fail(BIOT_ERR_INVALID_ARG, "end time must be >= 0");
    Request r;
    r.P = *p;
    r.target = (long)std::floor(T / p->dt + 0.5);
    r.bytes = estimate_bytes(p, sides);
    if (p->precision != BIOT_FP64 && cold_fp64_for(p)) {
        biot_params p64 = *p;
        p64.precision = BIOT_FP64;
        r.shadow = estimate_bytes(&p64, sides);
        r.cold64 = true;
    }
    for (int s = 0; s < 4; s++) {
        r.sides[s] = sides[s];
        const size_t m = 2 * (size_t)((s == BIOT_BOTTOM || s == BIOT_TOP) ? p->nx : p->ny) + 1;
        if (sides[s].eta_profile) {
            r.prof[s][0].assign(sides[s].eta_profile, sides[s].eta_profile + 2 * m);
            r.sides[s].eta_profile = r.prof[s][0].data();
        }
        if (sides[s].p_profile) {
            r.prof[s][1].assign(sides[s].p_profile, sides[s].p_profile + m);
            r.sides[s].p_profile = r.prof[s][1].data();
        }
    }
    std::lock_guard<std::mutex> lock(S->mu);
    if (r.bytes > S->budget) return fail(BIOT_ERR_OOM, "the request alone needs more device memory than the server's budget");
    if (r.bytes + r.shadow > S->budget) {  // no room for the FP64 copy: FP32 cold start
        r.shadow = 0;
        r.cold64 = false;
    }
    r.id = S->next_id++;
    r.t_submit = S->now();
    *id = r.id;
    const uint64_t rid = r.id;
    Request &slot = S->req[rid];
    slot = std::move(r);
    for (int s = 0; s < 4; s++) {  // re-point the copies after the move
        if (!slot.prof[s][0].empty()) slot.sides[s].eta_profile = slot.prof[s][0].data();
        if (!slot.prof[s][1].empty()) slot.sides[s].p_profile = slot.prof[s][1].data();
    }
    S->queue.push_back(rid);
    S->cv_work.notify_one();
    return BIOT_OK;
}

int biot_server_poll(biot_server S, uint64_t id, biot_request_info *info)
{
    if (!S || !info) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->req.find(id);
    if (it == S->req.end()) return fail(BIOT_ERR_INVALID_ARG, "unknown request id");
    const Request &r = it->second;
    info->state = r.state;
    info->status = r.status;
    info->t_submit = r.t_submit;
    info->t_start = r.t_start;
    info->t_done = r.t_done;
    info->nx = r.P.nx;
    info->ny = r.P.ny;
    info->steps = r.target;
    info->device_bytes = r.bytes;
    return BIOT_OK;
}

int biot_server_wait(biot_server S, uint64_t id, double timeout_s)
{
    if (!S) return fail(BIOT_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->req.find(id);
    if (it == S->req.end()) return fail(BIOT_ERR_INVALID_ARG, "unknown request id");
    const bool ok = S->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0), [&] {
        return it->second.state == REQ_DONE || it->second.state == REQ_FAILED;
    });
    if (!ok) return fail(BIOT_ERR_TIMEOUT, "request not finished within the timeout");
    if (it->second.state == REQ_FAILED) return fail(it->second.status, it->second.error);
    return BIOT_OK;
}

int biot_server_fetch(biot_server S, uint64_t id, double *eta, double *p, double *t_out)
{
    if (!S) return fail(BIOT_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->req.find(id);
    if (it == S->req.end()) return fail(BIOT_ERR_INVALID_ARG, "unknown request id");
    Request &r = it->second;
    if (r.state == REQ_FAILED) return fail(r.status, r.error);
    if (r.state != REQ_DONE) return fail(BIOT_ERR_INVALID_ARG, "request not finished");
    if (eta) std::memcpy(eta, r.eta.data(), r.eta.size() * sizeof(double));
    if (p) std::memcpy(p, r.p.data(), r.p.size() * sizeof(double));
    if (t_out) *t_out = r.t_result;
    return BIOT_OK;
}

int biot_server_release(biot_server S, uint64_t id)
{
    if (!S) return fail(BIOT_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->req.find(id);
    if (it == S->req.end()) return fail(BIOT_ERR_INVALID_ARG, "unknown request id");
    if (it->second.state != REQ_DONE && it->second.state != REQ_FAILED) return fail(BIOT_ERR_INVALID_ARG, "request not finished");
    S->req.erase(it);
    return BIOT_OK;
}

int biot_server_stats_get(biot_server S, biot_server_stats *o)
{
    if (!S || !o) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lock(S->mu);
    o->queued = (int)S->queue.size();
    o->peak_resident = S->peak_resident;
    o->used_bytes = S->used;
    o->peak_bytes = S->peak_used;
    o->ticks = S->ticks;
    o->graph_launches = S->graph_launches;
    o->graphs_reused = S->gcache.reused.load();
    return BIOT_OK;
}

int biot_server_destroy(biot_server S)
{
    if (!S) return BIOT_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    // every instance is released (its frees completed on its stream)
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->host_arena) cudaFreeHost(S->host_arena);
    delete S;
    return BIOT_OK;
}

}  // extern "C"

// ============================================================================
// Autotuning of the sweep launch shape.
// ============================================================================
// Per-level smoothing counts (see biot.h).  One scratch instance with the
// caller's boundary data and sources; each candidate set of counts is run from
// the initial state for a few V-cycles, timed, and its residual contraction per
// V-cycle measured.
namespace {

struct SweepTrial {
    double rho = 1e30, ms = 0.0, cost = 1e300;
};

int sweep_trial(biot_ctx *c, cudaEvent_t e0, cudaEvent_t e1, SweepTrial &out)
{
    int rc;
    c->initialized = false;
    if ((rc = ensure_initialized(c))) return rc;
    c->ft_fresh = false;
    c->se_stale = true;
    if ((rc = c->fp32 ? force_typed<float>(c) : force_typed<double>(c))) return rc;
    c->lv[c->L - 1].hist_valid = 0;
    c->cold_solve = false;  // time the cycles as a time step runs them
    c->measure_cycle = true;
    constexpr int M = 5;
    double res[M];
    float ms_sum = 0.f;
    for (int m = 0; m < M; m++) {
        CUDA_TRY(cudaMemsetAsync(c->resmax, 0, RES_WORDS * sizeof(unsigned long long), c->stream));
        CUDA_TRY(cudaEventRecord(e0, c->stream));
        if ((rc = vcycle(c, c->L - 1, false, false, c->P.cycle))) return rc;
        CUDA_TRY(cudaEventRecord(e1, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->resmax_host, c->resmax, RES_WORDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (m > 0) ms_sum += ms;  // the first cycle includes one-off set-up
        std::memcpy(&res[m], &c->resmax_host[0], sizeof(double));
    }
    out.ms = ms_sum / (M - 1);
    // contraction from the second cycle on (the first leaves the start's transients)
    const double r1 = res[1], r4 = res[M - 1];
    if (!(r1 > 0.0) || !std::isfinite(r4)) {
        out.rho = 1e30;
        out.cost = 1e300;
        return BIOT_OK;
    }
    out.rho = std::pow(r4 / r1, 1.0 / (M - 2));
    out.cost = out.rho < 1.0 ? out.ms / -std::log(std::max(out.rho, 1e-30)) : 1e300;
    return BIOT_OK;
}

}  // namespace

extern "C" int biot_autotune_sweeps(biot_handle h, int apply, int *K_out, double *rho_out, double *ms_per_cycle_out)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    if (h->rec) return fail(BIOT_ERR_INVALID_ARG, "an instance of a batch: set K_level at creation");
    int rc;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    biot_side sides[4];
    for (int i = 0; i < 4; i++) sides[i] = biot_side{h->bc_eta[i], h->bc_p[i], nullptr, nullptr};
    biot_params p = h->P;
    p.options |= BIOT_OPT_COLD_FP32;  // the scratch copy never needs an FP64 copy of its own
    biot_handle c = nullptr;
    if ((rc = biot_create(&p, sides, &c))) return rc;
    // the caller's boundary data and sources: the residual of a zero iterate is theirs
    const size_t np = (size_t)h->P.nx * h->P.ny;
    for (int side = 0; side < 4 && !rc; side++) {
        const size_t m = 2 * (size_t)side_cells(h, side) + 1;
        if (h->eta_prof[side] && !(rc = dev_alloc(c, (void **)&c->eta_prof[side], 2 * m * sizeof(double))))
            if (cudaMemcpyAsync(c->eta_prof[side], h->eta_prof[side], 2 * m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                rc = fail(BIOT_ERR_CUDA, "boundary data copy failed");
        if (!rc && h->p_prof[side] && !(rc = dev_alloc(c, (void **)&c->p_prof[side], m * sizeof(double))))
            if (cudaMemcpyAsync(c->p_prof[side], h->p_prof[side], m * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                rc = fail(BIOT_ERR_CUDA, "boundary data copy failed");
    }
    if (!rc && h->has_src && !(rc = dev_alloc(c, (void **)&c->src, np * sizeof(double)))) {
        if (cudaMemcpyAsync(c->src, h->src, np * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            rc = fail(BIOT_ERR_CUDA, "source copy failed");
        c->has_src = true;
    }
    if (!rc && h->has_fbody && !(rc = dev_alloc(c, (void **)&c->fbody, 2 * np * sizeof(double)))) {
        if (cudaMemcpyAsync(c->fbody, h->fbody, 2 * np * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            rc = fail(BIOT_ERR_CUDA, "body force copy failed");
        c->has_fbody = true;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        cudaGetLastError();
        rc = fail(BIOT_ERR_CUDA, "cudaEventCreate failed");
    }
    const int L = h->L;
    std::vector<int> best(L);
    for (int j = 0; j < L; j++) best[j] = sweeps_of(&h->P, L - 1 - j);
    SweepTrial bt;
    auto run = [&](const std::vector<int> &K, SweepTrial &t) {
        for (int j = 0; j < BIOT_MAX_LEVELS; j++) c->P.K_level[j] = j < L ? K[j] : 0;
        return sweep_trial(c, e0, e1, t);
    };
    if (!rc) rc = run(best, bt);
    static const int cand[] = {1, 2, 3, 4, 6, 8};
    for (int pass = 0; pass < 2 && !rc; pass++) {
        bool changed = false;
        for (int j = 0; j < L && !rc; j++) {
            for (int k : cand) {
                if (k == best[j]) continue;
                std::vector<int> K = best;
                K[j] = k;
                SweepTrial t;
                if ((rc = run(K, t))) break;
                if (t.cost < 0.97 * bt.cost) {  // a clear gain, not timing noise
                    bt = t;
                    best = K;
                    changed = true;
                }
            }
        }
        if (!changed) break;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    release(c);
    if (rc) return rc;
    if (K_out)
        for (int j = 0; j < L; j++) K_out[j] = best[j];
    if (rho_out) *rho_out = bt.rho;
    if (ms_per_cycle_out) *ms_per_cycle_out = bt.ms;
    if (apply) {
        for (int j = 0; j < BIOT_MAX_LEVELS; j++) h->P.K_level[j] = j < L ? best[j] : 0;
        drop_graphs(h);
    }
    return BIOT_OK;
}

extern "C" int biot_autotune(biot_handle h, int *rows_out, double *ms_out, int max_levels)
{
    if (!h) return fail(BIOT_ERR_INVALID_ARG, "null handle");
    int rc;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    // a scratch instance of the same shape: timing does not touch the caller's state
    biot_side sides[4];
    for (int i = 0; i < 4; i++) sides[i] = biot_side{h->bc_eta[i], h->bc_p[i], nullptr, nullptr};
    biot_handle c = nullptr;
    if ((rc = biot_create(&h->P, sides, &c))) return rc;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        release(c);
        return fail(BIOT_ERR_CUDA, "cudaEventCreate failed");
    }
    static const int fixed_cand[] = {4, 8, 16, 24, 32, 48, 64, 96};
    int status = BIOT_OK;
    for (int l = 0; l < h->L && !status; l++) {
        Level &Lv = h->lv[l];
        for (int mode = 0; mode < 2 && !status; mode++) {
            if (mode == SWEEP_RESTRICT && l == 0) continue;
            int best = 0;
            double best_ms = 1e30;
            // tile-sized levels are not launched as strips: nothing to choose
            const bool strips = (long)Lv.nx * Lv.ny > (long)256 * 256;
            // candidates: fixed heights, and the heights whose strips fill exactly
            // 1, 2 or 3 waves of resident CTAs (tall strips repeat fewer halo rows)
            std::vector<int> cand(std::begin(fixed_cand), std::end(fixed_cand));
            const int slots = strips ? tkind_strip_slots(level_tkind(h, l), level_variant(h, l, mode) & ~SWEEP_V_TILE) : 0;
            const int sx = (Lv.nx + SWEEP_STRIP_COLS - 1) / SWEEP_STRIP_COLS;
            for (int w = 1; w <= 3 && slots > 0; w++) {
                const int nsy = w * slots / sx;
                if (nsy < 1) continue;
                int ty = (Lv.ny + nsy - 1) / nsy;
                ty += ty & 1;
                if ((Lv.ny + ty - 1) / ty * sx <= w * slots) cand.push_back(ty);
            }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            for (size_t k = 0; strips && k < cand.size() && !status; k++) {
                if (cand[k] > Lv.ny) break;
                c->lv[l].rows[mode] = cand[k];
                for (int w = 0; w < 2 && !status; w++) status = sweep(c, l, mode, false, false, false);
                if (status) break;
                if (cudaEventRecord(e0, c->stream) != cudaSuccess) status = fail(BIOT_ERR_CUDA, "cudaEventRecord");
                const int reps = 4;
                for (int r = 0; r < reps && !status; r++) status = sweep(c, l, mode, false, false, false);
                if (status) break;
                float ms = 0.f;
                if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                    status = fail(BIOT_ERR_CUDA, "timing the sweep failed");
                else if (ms / reps < best_ms) {
                    best_ms = ms / reps;
                    best = cand[k];
                }
                c->lv[l].rows[mode] = 0;
            }
            Lv.rows[mode] = best;
            if (rows_out && l < max_levels) rows_out[2 * l + mode] = best;
            if (ms_out && l < max_levels) ms_out[2 * l + mode] = best ? best_ms : 0.0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release(c);
    drop_graphs(h);  // graphs captured with the old shapes
    return status;
}

// ============================================================================
// Checkpoint / resume.
//
// The resumable state of an instance after a completed step is the current
// flow populations, the finest elastic state (moments and, in FP32, the low
// parts of the first moments), the explicit force F~ of the last solve and the
// divergence history D(t - dt), D(t - 2 dt); the coarse levels, residuals and
// bounce-back histories are rebuilt inside every time step.
// ============================================================================
namespace {

struct CkptHeader {
    uint64_t magic;  // "BIOTCKP1"
    int32_t nx, ny, levels, precision;
    int64_t nstep;
    int32_t solved, initialized, last_ne, notconv;
    int64_t total_cycles;
    double last_res;
    uint64_t payload;  // bytes after the header
};
constexpr uint64_t CKPT_MAGIC = 0x3150434B544F4942ull;

struct CkptPart {
    void *dev;
    size_t bytes;
};

std::vector<CkptPart> ckpt_parts(biot_ctx *h)
{
    const Level &Lf = h->lv[h->L - 1];
    const size_t np = (size_t)h->P.nx * h->P.ny;
    const size_t tsz = h->fp32 ? 4 : 8, esz = Lf.fp64 ? 8 : 4;
    std::vector<CkptPart> v;
    v.push_back({h->f[h->fcur], 9 * np * tsz});
    v.push_back({Lf.g[Lf.cur], 8 * np * esz});
    if (Lf.glo[Lf.cur]) v.push_back({Lf.glo[Lf.cur], 2 * np * esz});
    if (Lf.gd[Lf.cur]) v.push_back({Lf.gd[Lf.cur], 3 * np * 2});
    v.push_back({h->Ft, 2 * np * tsz});
    v.push_back({h->D1, np * sizeof(double)});
    v.push_back({h->D2, np * sizeof(double)});
    v.push_back({h->dB[h->fcur], np * tsz});  // the difference the next flow step reads
    return v;
}

}  // namespace

extern "C" {

int biot_checkpoint_size(biot_handle h, size_t *bytes)
{
    if (!h || !bytes) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    size_t n = sizeof(CkptHeader);
    for (const CkptPart &p : ckpt_parts(h)) n += p.bytes;
    *bytes = n;
    return BIOT_OK;
}

int biot_save(biot_handle h, void *buf, size_t size)
{
    if (!h || !buf) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    int rc;
    if ((rc = finish_pending(h))) return rc;
    size_t need = 0;
    biot_checkpoint_size(h, &need);
    if (size < need) return fail(BIOT_ERR_INVALID_ARG, "checkpoint buffer too small (see biot_checkpoint_size)");
    CkptHeader hd{};
    hd.magic = CKPT_MAGIC;
    hd.nx = h->P.nx;
    hd.ny = h->P.ny;
    hd.levels = h->L;
    hd.precision = h->P.precision;
    hd.nstep = h->nstep;
    hd.solved = h->solved;
    hd.initialized = h->initialized;
    hd.last_ne = h->last_ne;
    hd.notconv = h->notconv_steps;
    hd.total_cycles = h->total_cycles;
    hd.last_res = h->last_res;
    hd.payload = need - sizeof(CkptHeader);
    std::memcpy(buf, &hd, sizeof(hd));
    unsigned char *out = static_cast<unsigned char *>(buf) + sizeof(hd);
    for (const CkptPart &p : ckpt_parts(h)) {
        CUDA_TRY(cudaMemcpyAsync(out, p.dev, p.bytes, cudaMemcpyDeviceToHost, h->stream));
        out += p.bytes;
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return BIOT_OK;
}

int biot_load(biot_handle h, const void *buf, size_t size)
{
    if (!h || !buf || size < sizeof(CkptHeader)) return fail(BIOT_ERR_INVALID_ARG, "null argument or short buffer");
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    size_t need = 0;
    biot_checkpoint_size(h, &need);
    if (hd.magic != CKPT_MAGIC) return fail(BIOT_ERR_INVALID_ARG, "not a checkpoint of this library");
    if (hd.nx != h->P.nx || hd.ny != h->P.ny || hd.levels != h->L || hd.precision != h->P.precision ||
        hd.payload + sizeof(CkptHeader) != need || size < need)
        return fail(BIOT_ERR_INVALID_ARG, "checkpoint of a different grid, hierarchy or precision");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    const unsigned char *in = static_cast<const unsigned char *>(buf) + sizeof(hd);
    for (const CkptPart &p : ckpt_parts(h)) {
        CUDA_TRY(cudaMemcpyAsync(p.dev, in, p.bytes, cudaMemcpyHostToDevice, h->stream));
        in += p.bytes;
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->nstep = hd.nstep;
    h->solved = hd.solved != 0;
    h->initialized = hd.initialized != 0;
    h->last_ne = hd.last_ne;
    h->notconv_steps = hd.notconv;
    h->total_cycles = hd.total_cycles;
    h->last_res = hd.last_res;
    h->diverged = 0;
    h->pending_res = false;
    h->pending_stop = false;
    h->ft_fresh = false;  // F~ belongs to the solve at the saved time
    h->se_stale = true;
    drop_graphs(h);
    return BIOT_OK;
}

}  // extern "C"
