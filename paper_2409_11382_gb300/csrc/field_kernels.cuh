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
    const T gpx = a.k_m3w * jx + T(0.5) * gx_;
    const T gpy = a.k_m3w * jy + T(0.5) * gy_;
    T fx = a.k_mah * gpx, fy = a.k_mah * gpy;
    if (a.fbody) {
        fx += T(a.c0h2 * a.fbody[idx]);
        fy += T(a.c0h2 * a.fbody[NP + idx]);
    }
    a.Ft[idx] = fx;
    a.Ft[NP + idx] = fy;
}

// ---------------------------------------------------------------------------
// Flow step, part 1: D(t) of the final elastic iterate (eq. LBM:divergence), s' of
// eq. source:implicit and p^ = sum_i f_i + s'/2 (eq. pressure), all in FP64.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_flow_moments(const FlowMomentsArgs<T> a)
{
    const size_t NP = (size_t)a.nx * a.ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= NP) return;
    const double dt_ = a.kD * (double)a.g[3 * NP + idx];
    const double d1 = a.D1[idx], d2 = a.D2[idx];
    const double s0 = a.src ? a.dt * a.src[idx] : 0.0;
    const double sp = s0 - a.a_over_h * ((1.0 - a.r) * (d1 - d2) + a.r * (dt_ - d1));
    T sum = T(0);
#pragma unroll
    for (int i = 0; i < 9; i++) sum += a.f[i * NP + idx];
    a.P[idx] = T((double)sum + 0.5 * sp);
    a.S[idx] = T(sp);
    a.Dnew[idx] = dt_;
    // explicit source of the next time step, from D(t) and D(t - dt) (k_sexp's formula)
    if (a.SEnext) a.SEnext[idx] = s0 - a.a_over_h * ((1.0 - a.r) * (dt_ - d1) - a.r * dt_);
}

// Flow step, part 2: BGK collision with source (eqs. pressure:equilibrium,
// pressure:collision, pressure:collision:source), pull streaming and the
// pressure wall rules (eqs. BC:pressure, BC:noFlow; SYMMETRY = mirror).
template <typename T>
__device__ __forceinline__ T flow_post(const FlowStreamArgs<T> &a, size_t NP, size_t idx, int i)
{
    const T om = a.k_om;
    const T fi = a.f[(size_t)i * NP + idx];
    const T wi = T(w9(i));
    return fi - om * (fi - wi * a.P[idx]) + a.k_src * wi * a.S[idx];
}

template <typename T>
__global__ void __launch_bounds__(256) k_flow_stream(const FlowStreamArgs<T> a)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int nx = a.nx, ny = a.ny;
    if (x >= nx || y >= ny) return;
    const size_t NP = (size_t)nx * ny, idx = (size_t)y * nx + x;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;
    a.fout[idx] = flow_post(a, NP, idx, 0);
#pragma unroll
    for (int i = 1; i < 9; i++) {
        const int cx = ex9(i), cy = ey9(i);
        int sx = x - cx, sy = y - cy;
        const bool outx = !perx && (sx < 0 || sx >= nx);
        const bool outy = !pery && (sy < 0 || sy >= ny);
        if (perx) sx = wrapi(sx, nx);
        if (pery) sy = wrapi(sy, ny);
        T v;
        if (!outx && !outy) {
            v = flow_post(a, NP, (size_t)sy * nx + sx, i);
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
                    if (outx) v = flow_post(a, NP, idx, dir9(-cx, -cy));
                    else      v = flow_post(a, NP, (size_t)y * nx + sx, dir9(cx, -cy));
                } else {
                    v = flow_post(a, NP, (size_t)sy * nx + x, dir9(-cx, cy));
                }
            } else if (type == BC_NEUMANN) {
                v = flow_post(a, NP, idx, iout);
            } else {  // BC_DIRICHLET
                v = -flow_post(a, NP, idx, iout);
                if (a.pprof[side]) {
                    const bool horiz = (side == SIDE_BOTTOM || side == SIDE_TOP);
                    const int kk = horiz ? 2 * x + 1 - cx : 2 * y + 1 - cy;
                    v += T(2.0 * w9(i) * a.c0 * a.pprof[side][kk]);
                }
            }
        }
        a.fout[(size_t)i * NP + idx] = v;
    }
}

// ---------------------------------------------------------------------------
// Physical fields of the current state (FP64 outputs):
//   eta = mbar_10,01 with mbar = m + F/2, F = F~ + F_*(g)   (eq. displacement)
//   sigma = -(1/(2 c0 h)) [[mbar_s+mbar_d, 2 mbar_11], [2 mbar_11, mbar_s-mbar_d]]
//   p = (sum_i f_i + s'/2) / c0                              (eq. pressure)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double div_at(const ReadoutArgs<T> &a, int x, int y)
{
    if (a.perx) x = wrapi(x, a.nx); else x = clampi(x, a.nx);
    if (a.pery) y = wrapi(y, a.ny); else y = clampi(y, a.ny);
    const size_t NP = (size_t)a.nx * a.ny;
    return a.kD * (double)a.g[3 * NP + (size_t)y * a.nx + x];
}

template <typename T>
__global__ void __launch_bounds__(256) k_readout(const ReadoutArgs<T> a)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.nx || y >= a.ny) return;
    const size_t NP = (size_t)a.nx * a.ny, idx = (size_t)y * a.nx + x;
    double m10 = a.g[idx], m01 = a.g[NP + idx];
    if (a.glo) {  // low parts of the double-float first moments
        m10 += (double)a.glo[idx];
        m01 += (double)a.glo[NP + idx];
    }
    const double m11 = a.g[2 * NP + idx], ms = a.g[3 * NP + idx], md = a.g[4 * NP + idx];
    if (a.eta) {
        const double dE = div_at(a, x + 1, y), dW = div_at(a, x - 1, y);
        const double dN = div_at(a, x, y + 1), dS = div_at(a, x, y - 1);
        const double dNE = div_at(a, x + 1, y + 1), dNW = div_at(a, x - 1, y + 1);
        const double dSE = div_at(a, x + 1, y - 1), dSW = div_at(a, x - 1, y - 1);
        double Fx = a.coef_fstar * ((dE - dW) / 3.0 + ((dNE + dSE) - (dNW + dSW)) / 12.0);
        double Fy = a.coef_fstar * ((dN - dS) / 3.0 + ((dNE + dNW) - (dSE + dSW)) / 12.0);
        Fx += (double)a.Ft[idx];
        Fy += (double)a.Ft[NP + idx];
        a.eta[idx] = m10 + 0.5 * Fx;
        a.eta[NP + idx] = m01 + 0.5 * Fy;
    }
    if (a.sigma) {
        const double lm3 = 3.0 * a.lm, mu6 = 6.0 * a.mu_hat;
        const double mbs = lm3 / (lm3 + 1.0) * ms;
        const double mbd = mu6 / (mu6 + 1.0) * md;
        const double mb11 = mu6 / (mu6 + 1.0) * m11;
        const double sc = -0.5 / a.c0h;
        a.sigma[idx] = sc * (mbs + mbd);
        a.sigma[NP + idx] = sc * 2.0 * mb11;
        a.sigma[2 * NP + idx] = sc * (mbs - mbd);
    }
    if (a.p) {
        const double dt_ = a.kD * ms;
        const double d1 = a.D1[idx], d2 = a.D2[idx];
        const double s0 = a.src ? a.dt * a.src[idx] : 0.0;
        const double sp = s0 - a.a_over_h * ((1.0 - a.r) * (d1 - d2) + a.r * (dt_ - d1));
        double sum = 0.0;
#pragma unroll
        for (int i = 0; i < 9; i++) sum += (double)a.f[i * NP + idx];
        a.p[idx] = (sum + 0.5 * sp) / a.c0;
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
cudaError_t launch_flow_moments_impl(const FlowMomentsArgs<T> &a, cudaStream_t s)
{
    const size_t n = (size_t)a.nx * a.ny;
    k_flow_moments<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_flow_stream_impl(const FlowStreamArgs<T> &a, cudaStream_t s)
{
    dim3 grid((a.nx + 31) / 32, (a.ny + 7) / 8);
    k_flow_stream<T><<<grid, 256, 0, s>>>(a);
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
cudaError_t launch_init_impl(const InitArgs<T> &a, cudaStream_t s)
{
    const size_t n = (size_t)a.nx * a.ny;
    k_init<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace biot
