// biot_capi.cu -- host runtime and C ABI of the GB300 Biot solver.
//
// Owns the device memory of one instance (multigrid hierarchy, flow
// populations, coupling history) and drives Alg. 5: per time step the explicit
// force, N_E V-cycles of Alg. 4 built from fused elastic sweeps, then the
// flow step of Alg. 3.  Every arithmetic step runs in the sm_103a kernels of
// sweep_mom.cuh and field_kernels.cuh; this file only sequences launches and
// copies, and evaluates the per-instance coefficients once on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "biot.h"
#include "biot_args.h"

using namespace biot;

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

struct Level {
    int nx = 0, ny = 0;
    size_t np = 0;
    bool fp64 = true;
    void *g[2] = {nullptr, nullptr};
    void *glo[2] = {nullptr, nullptr};  // low parts of m_10, m_01 (finest FP32 level)
    int cur = 0;
    void *r = nullptr;
    void *H[4] = {nullptr, nullptr, nullptr, nullptr};
    int hist_valid = 0;
};

}  // namespace

struct biot_ctx {
    biot_params P{};
    int bc_eta[4]{}, bc_p[4]{};
    double *eta_prof[4]{}, *p_prof[4]{};  // device copies of the boundary data (finest level)
    double h = 0, lam = 0, mu = 0, kap = 0, omega = 0, om_s = 0, om_d = 0, lm = 0;
    int L = 0;
    bool fp32 = false;  // FP32 state (finest and middle levels)
    Level lv[MAX_LEVELS];
    void *f[2]{};
    int fcur = 0;
    double *D1 = nullptr, *D2 = nullptr, *SE = nullptr;
    void *Pp = nullptr, *Ss = nullptr;  // p^ and s' of the flow step (population type)
    void *Ft = nullptr;
    double *src = nullptr, *fbody = nullptr;
    bool has_src = false, has_fbody = false;
    double *out = nullptr;  // readout scratch, 6 planes
    unsigned long long *resmax = nullptr;      // device [2]
    unsigned long long *resmax_host = nullptr; // pinned [2]
    cudaStream_t stream = nullptr, own_stream = nullptr;
    long nstep = 0;
    bool solved = false, initialized = false, pending_res = false;
    bool se_stale = true;  // SE must be recomputed from D1, D2 (else the last flow step wrote it)
    // statistics
    int last_ne = 0;
    double last_res = 0;
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
    // instrumentation of the finest-level smoothing sweep
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::vector<void *> allocs;
};

namespace {

int dev_alloc(biot_ctx *h, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return BIOT_OK;
    cudaError_t e = cudaMalloc(p, bytes);
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
    if (!(p->gamma > 0 && p->gamma <= 1)) return fail(BIOT_ERR_INVALID_ARG, "gamma must lie in (0, 1]");
    if (p->ne_fixed <= 0 && (p->ne_max < 1 || !(p->tol > 0))) return fail(BIOT_ERR_INVALID_ARG, "tolerance mode needs tol > 0 and ne_max >= 1");
    if (p->precision != BIOT_FP64 && p->precision != BIOT_FP32) return fail(BIOT_ERR_INVALID_ARG, "unknown precision");
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

// ---- kernel sequencing --------------------------------------------------------

template <typename T, typename TC>
int sweep_typed(biot_ctx *h, int l, int mode, bool zero_init, bool prolong, bool want_res)
{
    Level &Lv = h->lv[l];
    const bool fine = (l == h->L - 1);
    SweepArgs<T, TC> a{};
    a.nx = Lv.nx;
    a.ny = Lv.ny;
    a.g = static_cast<const T *>(Lv.g[Lv.cur]);
    a.gout = (mode == SWEEP_SMOOTH) ? static_cast<T *>(Lv.g[1 - Lv.cur]) : nullptr;
    a.glo = static_cast<const T *>(Lv.glo[Lv.cur]);
    a.glo_out = (mode == SWEEP_SMOOTH) ? static_cast<T *>(Lv.glo[1 - Lv.cur]) : nullptr;
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
    a.k_fs = T(a.coef_fstar * (-1.5 / (3.0 * a.lm + 1.0)));
    a.k_ws = T(1.0 - a.om_s);
    a.k_wd = T(1.0 - a.om_d);
    a.k_22 = T(-1.0 / (12.0 * a.lm + 4.0));
    a.k_gam = T(a.gamma);

    const bool timed = h->timing && fine && mode == SWEEP_SMOOTH;
    if (timed) {
        while (h->ev.size() < h->ev_used + 2) {
            cudaEvent_t e;
            CUDA_TRY(cudaEventCreate(&e));
            h->ev.push_back(e);
        }
        CUDA_TRY(cudaEventRecord(h->ev[h->ev_used], h->stream));
    }
    CUDA_TRY((launch_sweep_mom<T, TC>(a, h->stream)));
    if (timed) {
        CUDA_TRY(cudaEventRecord(h->ev[h->ev_used + 1], h->stream));
        h->ev_used += 2;
    }
    h->launches++;
    Lv.hist_valid = 1;
    if (mode == SWEEP_SMOOTH) Lv.cur ^= 1;
    return BIOT_OK;
}

int sweep(biot_ctx *h, int l, int mode, bool zero_init, bool prolong, bool want_res)
{
    const bool t64 = h->lv[l].fp64;
    const bool c64 = (l > 0) ? h->lv[l - 1].fp64 : t64;
    if (t64) return sweep_typed<double, double>(h, l, mode, zero_init, prolong, want_res);
    if (c64) return sweep_typed<float, double>(h, l, mode, zero_init, prolong, want_res);
    return sweep_typed<float, float>(h, l, mode, zero_init, prolong, want_res);
}

// ELASTIC_MULTIGRID (Alg. 4) on level l; zero_start: the iterate is zero
// (coarse-grid correction of a finer level).
int vcycle(biot_ctx *h, int l, bool zero_start)
{
    const int K = h->P.K;
    const bool fine = (l == h->L - 1);
    int rc;
    for (int k = 0; k < K; k++)
        if ((rc = sweep(h, l, SWEEP_SMOOTH, zero_start && k == 0, false, false))) return rc;
    if (l > 0) {
        if ((rc = sweep(h, l, SWEEP_RESTRICT, false, false, false))) return rc;
        h->lv[l - 1].hist_valid = 0;
        if ((rc = vcycle(h, l - 1, true))) return rc;
    }
    for (int k = 0; k < K; k++)
        if ((rc = sweep(h, l, SWEEP_SMOOTH, false, l > 0 && k == 0, fine && k == K - 1))) return rc;
    return BIOT_OK;
}

template <typename T>
int force_typed(biot_ctx *h)
{
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
    CUDA_TRY(launch_force<T>(a, h->stream));
    h->launches++;
    return BIOT_OK;
}

int read_residual(biot_ctx *h)
{
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    double res, gn;
    std::memcpy(&res, &h->resmax_host[0], sizeof(double));
    std::memcpy(&gn, &h->resmax_host[1], sizeof(double));
    h->last_res = res;
    h->pending_res = false;
    if (!std::isfinite(res)) {
        h->diverged = 1;
        return fail(BIOT_ERR_DIVERGED, "non-finite pseudo-time residual: the coupled iteration diverged");
    }
    (void)gn;
    return BIOT_OK;
}

// Elasticity update of Alg. 5 at the current time.
int elastic_solve(biot_ctx *h)
{
    int rc;
    rc = h->fp32 ? force_typed<float>(h) : force_typed<double>(h);
    if (rc) return rc;
    h->lv[h->L - 1].hist_valid = 0;
    const bool fixed = h->P.ne_fixed > 0;
    int ne = 0, status = BIOT_OK;
    for (;;) {
        const bool measure = !fixed || (ne + 1 == h->P.ne_fixed);
        if (measure) CUDA_TRY(cudaMemsetAsync(h->resmax, 0, 2 * sizeof(unsigned long long), h->stream));
        if ((rc = vcycle(h, h->L - 1, false))) return rc;
        ne++;
        h->total_cycles++;
        if (fixed) {
            if (ne >= h->P.ne_fixed) {
                CUDA_TRY(cudaMemcpyAsync(h->resmax_host, h->resmax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
                h->pending_res = true;
                break;
            }
            continue;
        }
        CUDA_TRY(cudaMemcpyAsync(h->resmax_host, h->resmax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
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

template <typename T>
int flow_typed(biot_ctx *h)
{
    const Level &Lf = h->lv[h->L - 1];
    FlowMomentsArgs<T> m{};
    m.nx = h->P.nx;
    m.ny = h->P.ny;
    m.g = static_cast<const T *>(Lf.g[Lf.cur]);
    m.f = static_cast<const T *>(h->f[h->fcur]);
    m.D1 = h->D1;
    m.D2 = h->D2;
    m.src = h->has_src ? h->src : nullptr;
    m.P = static_cast<T *>(h->Pp);
    m.S = static_cast<T *>(h->Ss);
    m.Dnew = h->D2;  // D(t) overwrites D(t - 2 dt) cell by cell after it was read
    m.dt = h->P.dt;
    m.a_over_h = h->P.alpha / h->h;
    m.r = h->P.r_coupling;
    m.lm = h->lm;
    m.kD = -1.5 / (3.0 * h->lm + 1.0);
    m.SEnext = h->SE;  // the explicit source of the next elastic solve
    CUDA_TRY(launch_flow_moments<T>(m, h->stream));
    h->se_stale = false;
    h->launches++;
    std::swap(h->D1, h->D2);  // D1 <- D(t), D2 <- D(t - dt)

    FlowStreamArgs<T> s{};
    s.nx = h->P.nx;
    s.ny = h->P.ny;
    s.f = static_cast<const T *>(h->f[h->fcur]);
    s.fout = static_cast<T *>(h->f[1 - h->fcur]);
    s.P = static_cast<const T *>(h->Pp);
    s.S = static_cast<const T *>(h->Ss);
    for (int i = 0; i < 4; i++) {
        s.pprof[i] = h->p_prof[i];
        s.bc[i] = h->bc_p[i];
    }
    s.omega = h->omega;
    s.c0 = h->P.c0;
    s.k_om = T(h->omega);
    s.k_src = T(1.0 - 0.5 * h->omega);
    CUDA_TRY(launch_flow_stream<T>(s, h->stream));
    h->launches++;
    h->fcur ^= 1;
    h->nstep++;
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
    a.lm = h->lm;
    a.mu_hat = h->mu;
    a.coef_fstar = 0.5 * h->P.alpha * h->P.alpha * h->P.r_coupling;
    a.c0 = h->P.c0;
    a.c0h = h->P.c0 * h->h;
    a.kD = -1.5 / (3.0 * h->lm + 1.0);
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

void drop_graphs(biot_ctx *h)
{
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
        e = cudaGraphInstantiate(&h->graph[par], g, 0);
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
    h->total_cycles += h->P.ne_fixed;
    h->last_ne = h->P.ne_fixed;
    h->solved = true;
    h->pending_res = true;
    return BIOT_OK;
}

void release(biot_ctx *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    if (h->resmax_host) cudaFreeHost(h->resmax_host);
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

int biot_create(const biot_params *p, const biot_side sides[4], biot_handle *out)
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
    h->P = *p;
    h->L = p->mg_levels;
    h->fp32 = p->precision == BIOT_FP32;
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
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(BIOT_ERR_CUDA, "cudaStreamCreate failed");
    }
    h->stream = h->own_stream;

#define TRY_RC(x) do { int _r = (x); if (_r) { release(h); return _r; } } while (0)
    const size_t np = (size_t)p->nx * p->ny;
    const size_t tsz = h->fp32 ? sizeof(float) : sizeof(double);
    for (int l = 0; l < h->L; l++) {
        Level &Lv = h->lv[l];
        const int shift = h->L - 1 - l;
        Lv.nx = p->nx >> shift;
        Lv.ny = p->ny >> shift;
        Lv.np = (size_t)Lv.nx * Lv.ny;
        Lv.fp64 = !h->fp32 || (l == 0 && h->L > 1);  // coarsest level in FP64
        const size_t esz = Lv.fp64 ? sizeof(double) : sizeof(float);
        TRY_RC(dev_alloc(h, &Lv.g[0], 8 * Lv.np * esz));
        TRY_RC(dev_alloc(h, &Lv.g[1], 8 * Lv.np * esz));
        if (!Lv.fp64 && l == h->L - 1) {  // double-float displacement moments
            TRY_RC(dev_alloc(h, &Lv.glo[0], 2 * Lv.np * esz));
            TRY_RC(dev_alloc(h, &Lv.glo[1], 2 * Lv.np * esz));
        }
        if (l < h->L - 1) TRY_RC(dev_alloc(h, &Lv.r, 8 * Lv.np * esz));
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
    TRY_RC(dev_alloc(h, (void **)&h->SE, np * sizeof(double)));
    TRY_RC(dev_alloc(h, &h->Pp, np * tsz));
    TRY_RC(dev_alloc(h, &h->Ss, np * tsz));
    TRY_RC(dev_alloc(h, (void **)&h->resmax, 2 * sizeof(unsigned long long)));
    if (cudaMallocHost((void **)&h->resmax_host, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        h->resmax_host = nullptr;
        release(h);
        return fail(BIOT_ERR_OOM, "pinned host allocation failed");
    }
    for (int s = 0; s < 4; s++) TRY_RC(set_profiles(h, s, sides[s].eta_profile, sides[s].p_profile));
#undef TRY_RC
    *out = h;
    return BIOT_OK;
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
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    h->solved = false;
    return BIOT_OK;
}

int biot_set_side_profile(biot_handle h, int side, const double *eta_profile, const double *p_profile)
{
    if (!h || side < 0 || side > 3) return fail(BIOT_ERR_INVALID_ARG, "bad handle or side");
    int rc = set_profiles(h, side, eta_profile, p_profile);
    if (rc) return rc;
    drop_graphs(h);
    h->solved = false;
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
    // with a fixed number of V-cycles nothing is read back until the end: a
    // diverged state stays non-finite, so the last residual reveals it
    const bool graphs = h->P.ne_fixed > 0 && h->use_graphs && !h->timing;
    for (int i = 0; i < n; i++) {
        if (h->P.ne_fixed <= 0 && (rc = finish_pending(h))) return rc;
        rc = graphs ? advance_graph(h) : advance(h);
        if (rc == BIOT_ERR_NOT_CONVERGED) status = rc;
        else if (rc) return rc;
    }
    if ((rc = finish_pending(h))) return rc;
    return status;
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

int biot_stats_get(biot_handle h, biot_stats *o)
{
    if (!h || !o) return fail(BIOT_ERR_INVALID_ARG, "null argument");
    int rc = finish_pending(h);
    o->last_ne = h->last_ne;
    o->last_res = h->last_res;
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

// Device address of the staging array on the current device, looked up once
// per device with that device current.
int noalloc_scratch(double **out)
{
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
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
    double *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
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
