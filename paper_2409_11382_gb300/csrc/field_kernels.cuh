// field_kernels.cuh -- the per-cell kernels around the elastic sweeps:
// explicit force, flow step (Alg. 3), read-out of the physical fields and the
// initial state.  The elastic state is stored as MRT moments (sweep_mom.cuh).
#pragma once
#include "biot_common.cuh"

namespace biot {

// ---------------------------------------------------------------------------
// Explicit part of eq. source:implicit in lattice units (FP64):
//   s'_exp = dt s - (alpha/h)[(1-r)(D1 - D2) - r D1]
// (the iterate-dependent part -(alpha r/h) D(g) is added in the sweep).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_sexp(const SexpArgs<T> a)
{
    const size_t NP = (size_t)a.nx * a.ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= NP) return;
    const double d1 = a.D1[idx], d2 = a.D2[idx];
    const double s = a.src ? a.dt * a.src[idx] : 0.0;
    a.SE[idx] = s - a.a_over_h * ((1.0 - a.r) * (d1 - d2) - a.r * d1);
}

// Explicit force of a time step:
//   F~ = c0 h^2 f - alpha h [ -3 omega sum_i f_i c_i + 1/2 grad^c s'_exp ]
// (eqs. pressure:gradient and pressure:gradient:alternative).  The stencil
// differences of s'_exp are taken in FP64, the rest in the population type.
template <typename T>
__device__ __forceinline__ double se_at(const ForceArgs<T> &a, int x, int y)
{
    if (a.perx) x = wrapi(x, a.nx); else x = clampi(x, a.nx);
    if (a.pery) y = wrapi(y, a.ny); else y = clampi(y, a.ny);
    return a.SE[(size_t)y * a.nx + x];
}

template <typename T>
__global__ void __launch_bounds__(256) k_force(const ForceArgs<T> a)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.nx || y >= a.ny) return;
    const size_t NP = (size_t)a.nx * a.ny, idx = (size_t)y * a.nx + x;
    T f[9];
#pragma unroll
    for (int i = 1; i < 9; i++) f[i] = a.f[i * NP + idx];
    const T jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const T jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const double sE = se_at(a, x + 1, y), sW = se_at(a, x - 1, y);
    const double sN = se_at(a, x, y + 1), sS = se_at(a, x, y - 1);
    const double sNE = se_at(a, x + 1, y + 1), sNW = se_at(a, x - 1, y + 1);
    const double sSE = se_at(a, x + 1, y - 1), sSW = se_at(a, x - 1, y - 1);
    const T gx_ = T(sE - sW) * T(1.0 / 3.0) + (T(sNE - sNW) + T(sSE - sSW)) * T(1.0 / 12.0);
    const T gy_ = T(sN - sS) * T(1.0 / 3.0) + (T(sNE - sSE) + T(sNW - sSW)) * T(1.0 / 12.0);
    T gpx = a.k_m3w * jx + T(0.5) * gx_;
    T gpy = a.k_m3w * jy + T(0.5) * gy_;
    if (a.central) {
        // eq. pressure:gradient:alternative for sum_i f_i: 3 sum_i w_i c_i P(x + c_i)
        // (same stencil as grad^c s'_exp; ghosts of non-periodic walls are the
        // adjacent cell, as for s'_exp)
        auto P = [&](int xx, int yy) {
            if (a.perx) xx = wrapi(xx, a.nx); else xx = clampi(xx, a.nx);
            if (a.pery) yy = wrapi(yy, a.ny); else yy = clampi(yy, a.ny);
            const T *q = a.f + (size_t)yy * a.nx + xx;
            return ((q[0] + q[NP]) + (q[2 * NP] + q[3 * NP])) + ((q[4 * NP] + q[5 * NP]) + (q[6 * NP] + q[7 * NP])) + q[8 * NP];
        };
        const T pE = P(x + 1, y), pW = P(x - 1, y), pN = P(x, y + 1), pS = P(x, y - 1);
        const T pNE = P(x + 1, y + 1), pNW = P(x - 1, y + 1), pSE = P(x + 1, y - 1), pSW = P(x - 1, y - 1);
        gpx = (pE - pW) * T(1.0 / 3.0) + ((pNE + pSE) - (pNW + pSW)) * T(1.0 / 12.0) + T(0.5) * gx_;
        gpy = (pN - pS) * T(1.0 / 3.0) + ((pNE + pNW) - (pSE + pSW)) * T(1.0 / 12.0) + T(0.5) * gy_;
    }
    T fx = a.k_mah * gpx, fy = a.k_mah * gpy;
    if (a.fbody) {
        fx += T(a.c0h2 * a.fbody[idx]);
        fy += T(a.c0h2 * a.fbody[NP + idx]);
    }
    a.Ft[idx] = fx;
    a.Ft[NP + idx] = fy;
}

// ---------------------------------------------------------------------------
// Physical fields of the current state (FP64 outputs):
//   eta = mbar_10,01 with mbar = m + F/2, F = F~ + F_*(g)   (eq. displacement)
//   sigma = -(1/(2 c0 h)) [[mbar_s+mbar_d, 2 mbar_11], [2 mbar_11, mbar_s-mbar_d]]
//   p = (sum_i f_i + s'/2) / c0                              (eq. pressure)
// F_* = (alpha^2 r / 2) grad^c D with D = kD m_s (the D2Q9 central gradient)
// and s' of the flow step's source (centered coupling, eq. pressure:gradient).
// Arithmetic in the storage type T, except where the state carries more than T
// holds: the double-float displacement (high part + (low part + F/2)) and the
// FP64 divergence history, whose differences are formed in FP64.  On the FP64
// path everything is FP64.  GB300 runs FP64 at a small fraction of the FP32
// rate, so the FP32 path keeps FP64 to about a dozen operations per cell.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ms_at(const ReadoutArgs<T> &a, int x, int y)
{
    if (a.perx) x = wrapi(x, a.nx); else x = clampi(x, a.nx);
    if (a.pery) y = wrapi(y, a.ny); else y = clampi(y, a.ny);
    const size_t NP = (size_t)a.nx * a.ny;
    return a.g[3 * NP + (size_t)y * a.nx + x];
}

template <typename T>
__global__ void __launch_bounds__(256) k_readout(const ReadoutArgs<T> a)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.nx || y >= a.ny) return;
    const size_t NP = (size_t)a.nx * a.ny, idx = (size_t)y * a.nx + x;
    const T ms = a.g[3 * NP + idx];
    if (a.eta) {
        const T mE = ms_at(a, x + 1, y), mW = ms_at(a, x - 1, y);
        const T mN = ms_at(a, x, y + 1), mS = ms_at(a, x, y - 1);
        const T mNE = ms_at(a, x + 1, y + 1), mNW = ms_at(a, x - 1, y + 1);
        const T mSE = ms_at(a, x + 1, y - 1), mSW = ms_at(a, x - 1, y - 1);
        const T ca = T(a.c_axis), cd = T(a.c_diag);
        const T Fx = a.Ft[idx] + (ca * (mE - mW) + cd * ((mNE + mSE) - (mNW + mSW)));
        const T Fy = a.Ft[NP + idx] + (ca * (mN - mS) + cd * ((mNE + mNW) - (mSE + mSW)));
        const T lx = a.glo ? a.glo[idx] : T(0), ly = a.glo ? a.glo[NP + idx] : T(0);
        a.eta[idx] = (double)a.g[idx] + (double)(lx + T(0.5) * Fx);
        a.eta[NP + idx] = (double)a.g[NP + idx] + (double)(ly + T(0.5) * Fy);
    }
    if (a.sigma) {
        const double m11 = a.g[2 * NP + idx], md = a.g[4 * NP + idx];
        a.sigma[idx] = a.c_s * (double)ms + a.c_d * md;
        a.sigma[NP + idx] = a.c_11 * m11;
        a.sigma[2 * NP + idx] = a.c_s * (double)ms - a.c_d * md;
    }
    if (a.p) {
        const double dt_ = a.kD * (double)ms;
        const double d1 = a.D1[idx], d2 = a.D2[idx];
        const T q = T(1.0 - a.r) * T(d1 - d2) + T(a.r) * T(dt_ - d1);
        const T s0 = a.src ? T(a.dt * a.src[idx]) : T(0);
        const T sp = s0 - T(a.a_over_h) * q;
        const T* f = a.f + idx;
        const T sum = ((f[0] + f[NP]) + (f[2 * NP] + f[3 * NP])) + ((f[4 * NP] + f[5 * NP]) + (f[6 * NP] + f[7 * NP])) + f[8 * NP];
        a.p[idx] = (double)(sum + T(0.5) * sp) * a.inv_c0;
    }
}

// Initial state, eqs. ICs and ICs:moments with p(0) = 0, eta(0) = 0:
// f_i = -(1/2) w_i dt s(0);  moments m0_10,01 = -F/2, m0_12,21 = -F/6, others 0,
// with F = c0 h^2 f(0).
template <typename T>
__global__ void __launch_bounds__(256) k_init(const InitArgs<T> a)
{
    const size_t NP = (size_t)a.nx * a.ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= NP) return;
    const double s0 = a.src ? a.dt * a.src[idx] : 0.0;
#pragma unroll
    for (int i = 0; i < 9; i++) a.f[i * NP + idx] = T(-0.5 * w9(i) * s0);
    const double Fx = a.fbody ? a.c0h2 * a.fbody[idx] : 0.0;
    const double Fy = a.fbody ? a.c0h2 * a.fbody[NP + idx] : 0.0;
    const double m0[8] = {-0.5 * Fx, -0.5 * Fy, 0.0, 0.0, 0.0, -Fx / 6.0, -Fy / 6.0, 0.0};
#pragma unroll
    for (int k = 0; k < 8; k++) a.g[k * NP + idx] = T(m0[k]);
    if (a.glo) {
        a.glo[idx] = T(m0[0] - (double)T(m0[0]));
        a.glo[NP + idx] = T(m0[1] - (double)T(m0[1]));
    }
}

// ---------------------------------------------------------------------------
// Fused flow step + explicit force of the next step.  A CTA of 32 x 8 threads
// owns a 32 x 8 tile; it stages the tile and a 1-cell halo (34 x 10 cells):
// post-collision populations f* (eqs. pressure, pressure:equilibrium,
// pressure:collision, pressure:collision:source), and the three fields whose
// D2Q9 gradient gives grad^c s'_exp(t+dt): s0 = dt s, A = D(t) - D(t-dt) and
// m_s (D(t) = kD m_s).  Only the divergence history is FP64: D(t) is formed in
// FP64, differenced with D(t-dt) and D(t-2dt) in FP64, and the differences
// are rounded to the storage type; the gradient of D(t) itself is taken as
// kD times the difference of neighbouring m_s values of the state, which is
// exact for nearby values.  Ghost cells of non-periodic walls are the adjacent
// cell (even extension), as in the elastic sweep.
// ---------------------------------------------------------------------------
constexpr int FF_TX = 32, FF_TY = 8, FF_W = FF_TX + 2, FF_H = FF_TY + 2;
static_assert(FF_TX == FLOW_TILE_X && FF_TY == FLOW_TILE_Y, "flow tile shared with the batch planner");

template <typename T>
__device__ __forceinline__ int ff_src_index(const FlowFusedArgs<T> &a, int x, int y)
{
    if (a.perx) x = wrapi(x, a.nx); else x = clampi(x, a.nx);
    if (a.pery) y = wrapi(y, a.ny); else y = clampi(y, a.ny);
    return y * a.nx + x;
}

template <typename T>
struct FlowSmem {
    T fs[9][FF_H][FF_W];  // post-collision populations
    T qs0[FF_H][FF_W], qA[FF_H][FF_W], qms[FF_H][FF_W];
};

template <typename T>
__device__ __forceinline__ void flow_tile(const FlowFusedArgs<T> &a, int bx, int by, FlowSmem<T> &sm)
{
    auto &fs = sm.fs;
    auto &qs0 = sm.qs0;
    auto &qA = sm.qA;
    auto &qms = sm.qms;
    const int nx = a.nx, ny = a.ny;
    const size_t NP = (size_t)nx * ny;
    const int tid = threadIdx.x;
    const int x0 = bx * FF_TX, y0 = by * FF_TY;
    // stage: 340 cells over 256 threads
    for (int i = tid; i < FF_W * FF_H; i += FF_TX * FF_TY) {
        const int cx = i % FF_W, cy = i / FF_W;
        const int idx = ff_src_index(a, x0 - 1 + cx, y0 - 1 + cy);
        T fi[9];
        T sum = T(0);
#pragma unroll
        for (int k = 0; k < 9; k++) {
            fi[k] = a.f[k * NP + idx];
            sum += fi[k];
        }
        const T msv = a.ms[idx];
        const double dt_ = a.kD * (double)msv;  // D(t)
        const double d1 = a.D1[idx];
        const T dA = T(dt_ - d1);  // FP64 difference of the history
        const T dB = a.dBprev[idx];  // the same difference one step earlier
        const T s0 = a.src ? T(a.dt * a.src[idx]) : T(0);
        const T sp = s0 - (a.k_a1r * dB + a.k_ar * dA);  // s' of eq. source:implicit
        const T P = sum + T(0.5) * sp, S = sp;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const T wk = T(w9(k));
            fs[k][cy][cx] = fi[k] - a.k_om * (fi[k] - wk * P) + a.k_src * wk * S;
        }
        qs0[cy][cx] = s0;
        qA[cy][cx] = dA;
        qms[cy][cx] = msv;
        const int gx = x0 - 1 + cx, gy = y0 - 1 + cy;
        if (cx >= 1 && cx <= FF_TX && cy >= 1 && cy <= FF_TY && gx < nx && gy < ny) {
            a.Dnew[idx] = dt_;
            a.dAout[idx] = dA;
        }
    }
    __syncthreads();
    const int tx = tid % FF_TX, ty = tid / FF_TX;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= nx || y >= ny) return;
    const size_t idx = (size_t)y * nx + x;
    const int cx = tx + 1, cy = ty + 1;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;
    T fn[9];
    fn[0] = fs[0][cy][cx];
#pragma unroll
    for (int i = 1; i < 9; i++) {
        const int ex = ex9(i), ey = ey9(i);
        const int sx = x - ex, sy = y - ey;
        const bool outx = !perx && (sx < 0 || sx >= nx);
        const bool outy = !pery && (sy < 0 || sy >= ny);
        T v;
        if (!outx && !outy) {
            v = fs[i][cy - ey][cx - ex];
        } else {
            int side = outy ? (sy < 0 ? SIDE_BOTTOM : SIDE_TOP) : (sx < 0 ? SIDE_LEFT : SIDE_RIGHT);
            if (outy && outx) {
                const int vert = sx < 0 ? SIDE_LEFT : SIDE_RIGHT;
                if (a.bc[side] == BC_SYMMETRY && a.bc[vert] != BC_SYMMETRY) side = vert;
            }
            const int iout = opp9(i);
            const int type = a.bc[side];
            if (type == BC_SYMMETRY) {
                if (outy) {
                    if (outx) v = fs[dir9(-ex, -ey)][cy][cx];
                    else      v = fs[dir9(ex, -ey)][cy][cx - ex];
                } else {
                    v = fs[dir9(-ex, ey)][cy - ey][cx];
                }
            } else if (type == BC_NEUMANN) {
                v = fs[iout][cy][cx];
            } else {  // BC_DIRICHLET
                v = -fs[iout][cy][cx];
                if (a.pprof[side]) {
                    const bool horiz = (side == SIDE_BOTTOM || side == SIDE_TOP);
                    const int kk = horiz ? 2 * x + 1 - ex : 2 * y + 1 - ey;
                    v += T(2.0 * w9(i) * a.c0 * a.pprof[side][kk]);
                }
            }
        }
        fn[i] = v;
    }
#pragma unroll
    for (int i = 0; i < 9; i++) a.fout[i * NP + idx] = fn[i];
    // explicit force of the next step
    const T jx = (fn[1] - fn[3]) + (fn[5] - fn[6]) + (fn[8] - fn[7]);
    const T jy = (fn[2] - fn[4]) + (fn[5] + fn[6]) - (fn[7] + fn[8]);
    auto grad = [&](const T (&q)[FF_H][FF_W], T &gx, T &gy) {
        gx = (q[cy][cx + 1] - q[cy][cx - 1]) * T(1.0 / 3.0) +
             ((q[cy + 1][cx + 1] - q[cy + 1][cx - 1]) + (q[cy - 1][cx + 1] - q[cy - 1][cx - 1])) * T(1.0 / 12.0);
        gy = (q[cy + 1][cx] - q[cy - 1][cx]) * T(1.0 / 3.0) +
             ((q[cy + 1][cx + 1] - q[cy - 1][cx + 1]) + (q[cy + 1][cx - 1] - q[cy - 1][cx - 1])) * T(1.0 / 12.0);
    };
    T g0x, g0y, gAx, gAy, gmx, gmy;
    grad(qs0, g0x, g0y);
    grad(qA, gAx, gAy);
    grad(qms, gmx, gmy);
    // grad s'_exp = grad s0 - (alpha/h) [(1-r) grad A - r kD grad m_s]; the two
    // coefficients come from the host (FP64 products rounded to T), so the
    // kernel's FP64 work is the divergence history alone (GB300 issues FP64 at
    // 1/64 of the FP32 rate, and per-thread FP64 coefficients made this kernel
    // FP64-bound)
    const T c1 = a.k_a1r, c2 = a.k_c2;
    const T gx_ = (g0x - c1 * gAx) + c2 * gmx;
    const T gy_ = (g0y - c1 * gAy) + c2 * gmy;
    T fx = a.k_mah * (a.k_m3w * jx + T(0.5) * gx_);
    T fy = a.k_mah * (a.k_m3w * jy + T(0.5) * gy_);
    if (a.fbody) {
        fx += T(a.c0h2 * a.fbody[idx]);
        fy += T(a.c0h2 * a.fbody[NP + idx]);
    }
    a.Ft[idx] = fx;
    a.Ft[NP + idx] = fy;
}

template <typename T>
__global__ void __launch_bounds__(FF_TX * FF_TY) k_flow_fused(const FlowFusedArgs<T> a)
{
    __shared__ FlowSmem<T> sm;
    flow_tile<T>(a, blockIdx.x, blockIdx.y, sm);
}

// Batched form: CTA b processes tile (items[b].bx, items[b].by) of the flow step
// jobs[items[b].job] (one job per instance of a batch).
template <typename T>
__global__ void __launch_bounds__(FF_TX * FF_TY)
    k_flow_fused_batch(const FlowFusedArgs<T> *__restrict__ jobs, const SweepItem *__restrict__ items)
{
    __shared__ FlowSmem<T> sm;
    __shared__ FlowFusedArgs<T> sa;
    const SweepItem it = items[blockIdx.x];
    if (threadIdx.x == 0) sa = jobs[it.job];
    __syncthreads();
    flow_tile<T>(sa, it.bx, it.by, sm);
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_sexp_impl(const SexpArgs<T> &a, cudaStream_t s)
{
    const size_t n = (size_t)a.nx * a.ny;
    k_sexp<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_force_impl(const ForceArgs<T> &a, cudaStream_t s)
{
    dim3 grid((a.nx + 31) / 32, (a.ny + 7) / 8);
    k_force<T><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_readout_impl(const ReadoutArgs<T> &a, cudaStream_t s)
{
    dim3 grid((a.nx + 31) / 32, (a.ny + 7) / 8);
    k_readout<T><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flow_fused_impl(const FlowFusedArgs<T> &a, cudaStream_t s)
{
    dim3 grid((a.nx + FF_TX - 1) / FF_TX, (a.ny + FF_TY - 1) / FF_TY);
    k_flow_fused<T><<<grid, FF_TX * FF_TY, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flow_fused_batch_impl(const FlowFusedArgs<T> *jobs, const SweepItem *items, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_flow_fused_batch<T><<<n, FF_TX * FF_TY, 0, s>>>(jobs, items);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_impl(const InitArgs<T> &a, cudaStream_t s)
{
    const size_t n = (size_t)a.nx * a.ny;
    k_init<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace biot
