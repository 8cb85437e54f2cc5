// biot_kernels.cuh -- sm_103a kernels of the coupled LBM for Biot's
// consolidation model (Lunowa & Wohlmuth, arXiv 2409.11382).
//
// Data layout in HBM: structure-of-arrays planes, plane stride nx*ny, y-major.
//   elastic populations g: 8 planes, D2Q8 order 10, 01, -10, 0-1, 11, -11, -1-1, 1-1
//   flow populations f:    9 planes, D2Q9 order 00, 10, 01, -10, 0-1, 11, -11, -1-1, 1-1
// (Tab. velocities).  Everything is in lattice units of the level it lives
// on: dx = dt = dtau = 1, c_s^2 = 1/3; scaling of §2.2 with L = h, T = dt,
// H = 1, eps = h.
//
// Included by one translation unit per precision; the FP64 unit is compiled
// without FMA contraction.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "biot_args.h"

namespace biot {

// D2Q8 velocities and opposite directions.
__host__ __device__ constexpr int ex8(int k) { return (k == 0 || k == 4 || k == 7) ? 1 : (k == 2 || k == 5 || k == 6) ? -1 : 0; }
__host__ __device__ constexpr int ey8(int k) { return (k == 1 || k == 4 || k == 5) ? 1 : (k == 3 || k == 6 || k == 7) ? -1 : 0; }
__host__ __device__ constexpr int opp8(int k) { return k < 4 ? (k + 2) & 3 : 4 + ((k - 4 + 2) & 3); }
__host__ __device__ constexpr int dir8(int cx, int cy)
{
    return cy == 0 ? (cx > 0 ? 0 : 2)
         : cx == 0 ? (cy > 0 ? 1 : 3)
         : cy > 0 ? (cx > 0 ? 4 : 5) : (cx < 0 ? 6 : 7);
}
// D2Q9 velocities, weights, opposites.
__host__ __device__ constexpr int ex9(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
__host__ __device__ constexpr int ey9(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }
__host__ __device__ constexpr int opp9(int i) { return i == 0 ? 0 : i < 5 ? 1 + ((i - 1 + 2) & 3) : 5 + ((i - 5 + 2) & 3); }
__host__ __device__ constexpr int dir9(int cx, int cy)
{
    return (cx == 0 && cy == 0) ? 0
         : cy == 0 ? (cx > 0 ? 1 : 3)
         : cx == 0 ? (cy > 0 ? 2 : 4)
         : cy > 0 ? (cx > 0 ? 5 : 6) : (cx < 0 ? 7 : 8);
}
__host__ __device__ constexpr double w9(int i) { return i == 0 ? 4.0 / 9.0 : i < 5 ? 1.0 / 9.0 : 1.0 / 36.0; }

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// Slot of an outgoing direction in the 3-entry history record of a wall cell.
__device__ __forceinline__ int hslot(int side, int kout)
{
    switch (side) {
    case SIDE_BOTTOM: return kout == 3 ? 0 : kout == 6 ? 1 : 2;  // 0-1, -1-1, 1-1
    case SIDE_RIGHT:  return kout == 0 ? 0 : kout == 4 ? 1 : 2;  // 10, 11, 1-1
    case SIDE_TOP:    return kout == 1 ? 0 : kout == 4 ? 1 : 2;  // 01, 11, -11
    default:          return kout == 2 ? 0 : kout == 5 ? 1 : 2;  // -10, -11, -1-1
    }
}
__device__ __forceinline__ int hdir(int side, int j)
{
    switch (side) {
    case SIDE_BOTTOM: return j == 0 ? 3 : j == 1 ? 6 : 7;
    case SIDE_RIGHT:  return j == 0 ? 0 : j == 1 ? 4 : 7;
    case SIDE_TOP:    return j == 0 ? 1 : j == 1 ? 4 : 5;
    default:          return j == 0 ? 2 : j == 1 ? 5 : 6;
    }
}

// Collision of Alg. 2 in moment space (eqs. moments, moments:stress,
// moments:halfForce, moments:collision, Tab. moments, moments:collision:22)
// followed by the back-transformation of Tab. moments:inverse.  The moments
// m_12, m_21 and m_22 of the input are relaxed with rate 1 to values that do
// not depend on them, so only m_10, m_01, m_11, m_s, m_d are formed.
template <typename T>
__device__ __forceinline__ void elastic_collide(const T (&g)[8], T Fx, T Fy, T one_m_ws, T one_m_wd, T c22, T (&s)[8])
{
    const T dsum = (g[4] + g[5]) + (g[6] + g[7]);
    const T m10 = (g[0] - g[2]) + (g[4] - g[5]) + (g[7] - g[6]);
    const T m01 = (g[1] - g[3]) + (g[4] + g[5]) - (g[6] + g[7]);
    const T m11 = (g[4] - g[5]) + (g[6] - g[7]);
    const T ax = g[0] + g[2], ay = g[1] + g[3];
    const T ms = (ax + ay) + T(2) * dsum;
    const T md = ax - ay;
    const T a = m10 + Fx;                               // m*_10
    const T b = m01 + Fy;                               // m*_01
    const T q12 = (m10 + T(0.5) * Fx) * T(1.0 / 3.0);   // m*_12 = mbar_10 / 3
    const T q21 = (m01 + T(0.5) * Fy) * T(1.0 / 3.0);   // m*_21 = mbar_01 / 3
    const T ss = one_m_ws * ms;                         // m*_s
    const T sd = one_m_wd * md;                         // m*_d
    const T s11 = one_m_wd * m11;                       // m*_11
    const T s22 = c22 * ms;                             // m*_22 = -m_s / (12(lam+mu)+4)
    const T A = T(0.5) * (a - q12), B = T(0.5) * (b - q21);
    const T E0 = T(0.25) * (ss + sd) - T(0.5) * s22;
    const T E1 = T(0.25) * (ss - sd) - T(0.5) * s22;
    const T u = T(0.25) * (s22 + s11), v = T(0.25) * (s22 - s11);
    const T pp = T(0.25) * (q12 + q21), mm = T(0.25) * (q21 - q12);
    s[0] = E0 + A;
    s[2] = E0 - A;
    s[1] = E1 + B;
    s[3] = E1 - B;
    s[4] = u + pp;
    s[6] = u - pp;
    s[5] = v + mm;
    s[7] = v - mm;
}

template <typename T>
__device__ __forceinline__ T second_moment_sum(const T (&g)[8])
{
    return ((g[0] + g[2]) + (g[1] + g[3])) + T(2) * ((g[4] + g[5]) + (g[6] + g[7]));
}

// Lattice traction term eps * varsigma of eq. BC:traction for the incoming
// direction (cx, cy) at a wall, per unit of c0 h (the left-wall values are the
// paper's; the other walls follow by rotating the square).
__device__ __forceinline__ double traction_term(const double *prof, int side, int n, int x, int y, int cx, int cy)
{
    const bool horiz = (side == SIDE_BOTTOM || side == SIDE_TOP);
    const int kk = horiz ? 2 * x + 1 - cx : 2 * y + 1 - cy;
    const double t1 = prof[kk], t2 = prof[2 * n + 1 + kk];
    if (horiz) {
        const double nn = side == SIDE_TOP ? 1.0 : -1.0;
        return cx == 0 ? -nn * t2 : 0.5 * cx * t1;
    }
    const double nn = side == SIDE_RIGHT ? 1.0 : -1.0;
    return cy == 0 ? -nn * t1 : 0.5 * cy * t2;
}

// Displacement term -6 w c_out . eta_D of eq. BC:elasticity for the incoming
// direction (cx, cy) (outgoing -c), D2Q9 weights 1/9 and 1/36.
__device__ __forceinline__ double dirichlet_term(const double *prof, int side, int n, int x, int y, int cx, int cy)
{
    const bool horiz = (side == SIDE_BOTTOM || side == SIDE_TOP);
    const int kk = horiz ? 2 * x + 1 - cx : 2 * y + 1 - cy;
    const double e1 = prof[kk], e2 = prof[2 * n + 1 + kk];
    const double w = (cx != 0 && cy != 0) ? 6.0 / 36.0 : 6.0 / 9.0;
    return w * (cx * e1 + cy * e2);
}

__device__ __forceinline__ double nan_to_inf(double v) { return (v == v) ? v : (double)INFINITY; }

// ---------------------------------------------------------------------------
// Fused elastic sweep.  One CTA owns a TX x TY tile of cells.  It stages the
// iterate (plus a prolongated coarse correction) for the tile and a 2-cell
// halo in shared memory, forms the lattice divergence D(g) there, collides
// the tile and a 1-cell halo with F = F~ + (alpha^2 r/2) grad^c D(g), streams
// by pulling from shared memory, applies the wall rules of §3.6 and then
// either under-relaxes (eq. MG:smoother) or restricts the residual by the
// full sum of eq. MG:restriction.
// ---------------------------------------------------------------------------
template <int TX, int TY, typename T>
constexpr size_t sweep_smem_bytes()
{
    return sizeof(T) * (size_t)(17 * (TX + 4) * (TY + 4) + 8 * TX * TY);
}

template <typename T, typename TC>
__device__ __forceinline__ void load_cell(const SweepArgs<T, TC> &a, int x, int y, size_t NP, T (&v)[8])
{
    if (a.zero_init) {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = T(0);
    } else {
        const size_t idx = (size_t)y * a.nx + x;
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = a.g[k * NP + idx];
    }
    if (a.gc) {
        const int ncx = a.nx >> 1;
        const size_t NPc = NP >> 2;
        const size_t cidx = (size_t)(y >> 1) * ncx + (x >> 1);
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] += (T)a.gc[k * NPc + cidx];
    }
}

template <typename T, typename TC, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_elastic_sweep(const SweepArgs<T, TC> a)
{
    constexpr int NT = TX * TY;
    constexpr int BX = TX + 4, BY = TY + 4, BN = BX * BY;
    constexpr int QX = TX + 2, QN = (TX + 2) * (TY + 2);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sG = reinterpret_cast<T *>(smem_raw);  // [8][BN] iterate (+ correction)
    T *sGS = sG + 8 * BN;                      // [8][BN] post-collision
    T *sD = sGS + 8 * BN;                      // [BN] lattice divergence
    T *sR = sD + BN;                           // [8][NT] residual (restriction)
    __shared__ double red[2][NT / 32];

    const int nx = a.nx, ny = a.ny;
    const size_t NP = (size_t)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;
    const T cdiv = T(-1.5 / (3.0 * a.lm + 1.0));  // D = -3 m_s / (2(3(lam+mu)+1)), eq. LBM:divergence

    // Phase 1: iterate and divergence on the tile + 2 halo.  Outside a
    // non-periodic wall the divergence takes the value of the adjacent cell.
    for (int p = threadIdx.x; p < BN; p += NT) {
        const int bx = p % BX, by = p / BX;
        int gx = x0 + bx - 2, gy = y0 + by - 2;
        if (perx) gx = wrapi(gx, nx);
        if (pery) gy = wrapi(gy, ny);
        const bool in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny;
        T v[8];
        load_cell(a, clampi(gx, nx), clampi(gy, ny), NP, v);
        if (in) {
#pragma unroll
            for (int k = 0; k < 8; k++) sG[k * BN + p] = v[k];
        }
        sD[p] = cdiv * second_moment_sum(v);
    }
    __syncthreads();

    // Phase 2: collide the tile + 1 halo.
    const T one_m_ws = T(1.0 - a.om_s), one_m_wd = T(1.0 - a.om_d);
    const T c22 = T(-1.0 / (12.0 * a.lm + 4.0));
    const T cf = T(a.coef_fstar);
    for (int q = threadIdx.x; q < QN; q += NT) {
        const int bx = q % QX + 1, by = q / QX + 1;
        const int p = by * BX + bx;
        int gx = x0 + bx - 2, gy = y0 + by - 2;
        if (perx) gx = wrapi(gx, nx);
        if (pery) gy = wrapi(gy, ny);
        if ((unsigned)gx >= (unsigned)nx || (unsigned)gy >= (unsigned)ny) continue;
        const size_t idx = (size_t)gy * nx + gx;
        T v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = sG[k * BN + p];
        if (a.r) {
#pragma unroll
            for (int k = 0; k < 8; k++) v[k] -= a.r[k * NP + idx];
        }
        const T dE = sD[p + 1], dW = sD[p - 1], dN = sD[p + BX], dS = sD[p - BX];
        const T dNE = sD[p + BX + 1], dNW = sD[p + BX - 1], dSE = sD[p - BX + 1], dSW = sD[p - BX - 1];
        T Fx = cf * ((dE - dW) * T(1.0 / 3.0) + ((dNE + dSE) - (dNW + dSW)) * T(1.0 / 12.0));
        T Fy = cf * ((dN - dS) * T(1.0 / 3.0) + ((dNE + dNW) - (dSE + dSW)) * T(1.0 / 12.0));
        if (a.Ft) {
            Fx += a.Ft[idx];
            Fy += a.Ft[NP + idx];
        }
        T s[8];
        elastic_collide(v, Fx, Fy, one_m_ws, one_m_wd, c22, s);
#pragma unroll
        for (int k = 0; k < 8; k++) sGS[k * BN + p] = s[k];
    }
    __syncthreads();

    // Phase 3: stream (pull) with the wall rules, then relax or restrict.
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = x < nx && y < ny;
    double rmax = 0.0, gmax = 0.0;
    if (valid) {
        const int p = (ty + 2) * BX + (tx + 2);
        const size_t idx = (size_t)y * nx + x;
        T gcur[8], gss[8];
#pragma unroll
        for (int k = 0; k < 8; k++) gcur[k] = sG[k * BN + p];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int cx = ex8(k), cy = ey8(k);
            const int sx = x - cx, sy = y - cy;
            const bool outx = !perx && (sx < 0 || sx >= nx);
            const bool outy = !pery && (sy < 0 || sy >= ny);
            if (!outx && !outy) {
                gss[k] = sGS[k * BN + p - cx - cy * BX];
                continue;
            }
            int side = outy ? (sy < 0 ? SIDE_BOTTOM : SIDE_TOP) : (sx < 0 ? SIDE_LEFT : SIDE_RIGHT);
            if (outy && outx) {
                // corner: a bounce-back type side wall wins over a mirror top/bottom
                const int vert = sx < 0 ? SIDE_LEFT : SIDE_RIGHT;
                if (a.bc[side] == BC_SYMMETRY && a.bc[vert] != BC_SYMMETRY) side = vert;
            }
            const int kout = opp8(k);
            const int type = a.bc[side];
            if (type == BC_SYMMETRY) {
                // mirror image of the ghost source, normal velocity reversed
                if (outy) {
                    if (outx) gss[k] = sGS[dir8(-cx, -cy) * BN + p];
                    else      gss[k] = sGS[dir8(cx, -cy) * BN + p - cx];
                } else {
                    gss[k] = sGS[dir8(-cx, cy) * BN + p - cy * BX];
                }
            } else if (type == BC_NEUMANN) {
                T v = -sGS[kout * BN + p];
                if (a.prof[side]) {
                    const int n = (side == SIDE_BOTTOM || side == SIDE_TOP) ? nx : ny;
                    v += T(a.c0h * traction_term(a.prof[side], side, n, x, y, cx, cy));
                }
                gss[k] = v;
            } else {  // BC_DIRICHLET
                const int pos = (side == SIDE_BOTTOM || side == SIDE_TOP) ? x : y;
                T hv = a.hist_valid ? a.H[side][3 * pos + hslot(side, kout)] : sGS[kout * BN + p];
                if (a.prof[side]) {
                    const int n = (side == SIDE_BOTTOM || side == SIDE_TOP) ? nx : ny;
                    hv += T(dirichlet_term(a.prof[side], side, n, x, y, cx, cy));
                }
                gss[k] = hv;
            }
        }
        // history of the fullway bounce-back: this call's outgoing populations
        if (y == 0 && a.bc[SIDE_BOTTOM] == BC_DIRICHLET)
            for (int j = 0; j < 3; j++) a.H[SIDE_BOTTOM][3 * x + j] = sGS[hdir(SIDE_BOTTOM, j) * BN + p];
        if (y == ny - 1 && a.bc[SIDE_TOP] == BC_DIRICHLET)
            for (int j = 0; j < 3; j++) a.H[SIDE_TOP][3 * x + j] = sGS[hdir(SIDE_TOP, j) * BN + p];
        if (x == 0 && a.bc[SIDE_LEFT] == BC_DIRICHLET)
            for (int j = 0; j < 3; j++) a.H[SIDE_LEFT][3 * y + j] = sGS[hdir(SIDE_LEFT, j) * BN + p];
        if (x == nx - 1 && a.bc[SIDE_RIGHT] == BC_DIRICHLET)
            for (int j = 0; j < 3; j++) a.H[SIDE_RIGHT][3 * y + j] = sGS[hdir(SIDE_RIGHT, j) * BN + p];

        if (a.mode == SWEEP_SMOOTH) {
            const T gam = T(a.gamma), omg = T(1.0 - a.gamma);
#pragma unroll
            for (int k = 0; k < 8; k++) a.gout[k * NP + idx] = omg * gcur[k] + gam * gss[k];
            if (a.resmax) {
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    rmax = fmax(rmax, nan_to_inf(fabs((double)(gcur[k] - gss[k]))));
                    gmax = fmax(gmax, nan_to_inf(fabs((double)gcur[k])));
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) sR[k * NT + threadIdx.x] = gcur[k] - gss[k];
        }
    }
    if (a.mode == SWEEP_RESTRICT) {
        __syncthreads();
        constexpr int CXN = TX / 2, CN = (TX / 2) * (TY / 2);
        if (threadIdx.x < CN) {
            const int cxl = threadIdx.x % CXN, cyl = threadIdx.x / CXN;
            const int X = (x0 >> 1) + cxl, Y = (y0 >> 1) + cyl;
            const int ncx = nx >> 1, ncy = ny >> 1;
            if (X < ncx && Y < ncy) {
                const size_t NPc = NP >> 2;
                const int t00 = (2 * cyl) * TX + 2 * cxl;
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    TC v = (TC)sR[k * NT + t00];
                    v += (TC)sR[k * NT + t00 + 1];
                    v += (TC)sR[k * NT + t00 + TX];
                    v += (TC)sR[k * NT + t00 + TX + 1];
                    a.rc[k * NPc + (size_t)Y * ncx + X] = v;
                }
            }
        }
    }
    if (a.resmax) {
        // warp-shuffle then block reduction of the two maxima, one atomic per CTA
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) { red[0][warp] = rmax; red[1][warp] = gmax; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double r0 = 0.0, g0 = 0.0;
            for (int w = 0; w < NT / 32; w++) { r0 = fmax(r0, red[0][w]); g0 = fmax(g0, red[1][w]); }
            atomicMax(&a.resmax[0], (unsigned long long)__double_as_longlong(r0));
            atomicMax(&a.resmax[1], (unsigned long long)__double_as_longlong(g0));
        }
    }
}

// ---------------------------------------------------------------------------
// Explicit force of a time step:
//   F~ = c0 h^2 f - alpha h [ -3 omega sum_i f_i c_i + 1/2 grad^c s'_exp ]
// with s'_exp = dt s - (alpha/h)[(1-r)(D1 - D2) - r D1] (eqs. pressure:gradient,
// source:implicit; the iterate-dependent part is added in the sweep).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double sexp_at(const ForceArgs<T> &a, int x, int y)
{
    if (a.perx) x = wrapi(x, a.nx); else x = clampi(x, a.nx);
    if (a.pery) y = wrapi(y, a.ny); else y = clampi(y, a.ny);
    const size_t idx = (size_t)y * a.nx + x;
    const double d1 = a.D1[idx], d2 = a.D2[idx];
    const double s = a.src ? a.dt * a.src[idx] : 0.0;
    return s - a.a_over_h * ((1.0 - a.r) * (d1 - d2) - a.r * d1);
}

template <typename T>
__global__ void __launch_bounds__(256) k_force(const ForceArgs<T> a)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.nx || y >= a.ny) return;
    const size_t NP = (size_t)a.nx * a.ny, idx = (size_t)y * a.nx + x;
    double jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 1; i < 9; i++) {
        const double fi = (double)a.f[i * NP + idx];
        if (ex9(i)) jx += ex9(i) * fi;
        if (ey9(i)) jy += ey9(i) * fi;
    }
    const double sE = sexp_at(a, x + 1, y), sW = sexp_at(a, x - 1, y);
    const double sN = sexp_at(a, x, y + 1), sS = sexp_at(a, x, y - 1);
    const double sNE = sexp_at(a, x + 1, y + 1), sNW = sexp_at(a, x - 1, y + 1);
    const double sSE = sexp_at(a, x + 1, y - 1), sSW = sexp_at(a, x - 1, y - 1);
    const double gsx = (sE - sW) / 3.0 + ((sNE + sSE) - (sNW + sSW)) / 12.0;
    const double gsy = (sN - sS) / 3.0 + ((sNE + sNW) - (sSE + sSW)) / 12.0;
    const double gpx = -3.0 * a.omega * jx + 0.5 * gsx;
    const double gpy = -3.0 * a.omega * jy + 0.5 * gsy;
    double fx = -a.alpha_h * gpx, fy = -a.alpha_h * gpy;
    if (a.fbody) {
        fx += a.c0h2 * a.fbody[idx];
        fy += a.c0h2 * a.fbody[NP + idx];
    }
    a.Ft[idx] = (T)fx;
    a.Ft[NP + idx] = (T)fy;
}

// ---------------------------------------------------------------------------
// Flow step, part 1: D(t) of the final elastic iterate, s' of eq.
// source:implicit and p^ = sum_i f_i + s'/2 (eq. pressure), all in FP64.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_flow_moments(const FlowMomentsArgs<T> a)
{
    const size_t NP = (size_t)a.nx * a.ny;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= NP) return;
    T gv[8];
#pragma unroll
    for (int k = 0; k < 8; k++) gv[k] = a.g[k * NP + idx];
    const double dt_ = -1.5 / (3.0 * a.lm + 1.0) * (double)second_moment_sum(gv);
    const double d1 = a.D1[idx], d2 = a.D2[idx];
    const double s0 = a.src ? a.dt * a.src[idx] : 0.0;
    const double sp = s0 - a.a_over_h * ((1.0 - a.r) * (d1 - d2) + a.r * (dt_ - d1));
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < 9; i++) sum += (double)a.f[i * NP + idx];
    a.P[idx] = sum + 0.5 * sp;
    a.S[idx] = sp;
    a.Dnew[idx] = dt_;
}

// Flow step, part 2: BGK collision with source (eqs. pressure:equilibrium,
// pressure:collision, pressure:collision:source), pull streaming and the
// pressure wall rules (eqs. BC:pressure, BC:noFlow; SYMMETRY = mirror).
template <typename T>
__device__ __forceinline__ T flow_post(const FlowStreamArgs<T> &a, size_t NP, size_t idx, int i)
{
    const T om = T(a.omega);
    const T fi = a.f[(size_t)i * NP + idx];
    const T wi = T(w9(i));
    return fi - om * (fi - wi * T(a.P[idx])) + (T(1) - T(0.5) * om) * wi * T(a.S[idx]);
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
    const size_t NP = (size_t)a.nx * a.ny, idx = (size_t)y * a.nx + x;
    T gv[8];
#pragma unroll
    for (int k = 0; k < 8; k++) gv[k] = a.g[k * NP + idx];
    return -1.5 / (3.0 * a.lm + 1.0) * (double)second_moment_sum(gv);
}

template <typename T>
__global__ void __launch_bounds__(256) k_readout(const ReadoutArgs<T> a)
{
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (x >= a.nx || y >= a.ny) return;
    const size_t NP = (size_t)a.nx * a.ny, idx = (size_t)y * a.nx + x;
    double g[8];
#pragma unroll
    for (int k = 0; k < 8; k++) g[k] = (double)a.g[k * NP + idx];
    const double m10 = (g[0] - g[2]) + (g[4] - g[5]) + (g[7] - g[6]);
    const double m01 = (g[1] - g[3]) + (g[4] + g[5]) - (g[6] + g[7]);
    const double m11 = (g[4] - g[5]) + (g[6] - g[7]);
    const double ax = g[0] + g[2], ay = g[1] + g[3];
    const double ms = (ax + ay) + 2.0 * ((g[4] + g[5]) + (g[6] + g[7]));
    const double md = ax - ay;
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
        const double dt_ = -1.5 / (3.0 * a.lm + 1.0) * ms;
        const double d1 = a.D1[idx], d2 = a.D2[idx];
        const double s0 = a.src ? a.dt * a.src[idx] : 0.0;
        const double sp = s0 - a.a_over_h * ((1.0 - a.r) * (d1 - d2) + a.r * (dt_ - d1));
        double sum = 0.0;
#pragma unroll
        for (int i = 0; i < 9; i++) sum += (double)a.f[i * NP + idx];
        a.p[idx] = (sum + 0.5 * sp) / a.c0;
    }
}

// Initial populations, eqs. ICs and ICs:moments with p(0) = 0, eta(0) = 0:
// f_i = -(1/2) w_i dt s(0);  g = T m0 with m0_10,01 = -F/2, m0_12,21 = -F/6,
// F = c0 h^2 f(0) (the back-transformation written out).
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
    a.g[0 * NP + idx] = T(-Fx / 6.0);
    a.g[1 * NP + idx] = T(-Fy / 6.0);
    a.g[2 * NP + idx] = T(Fx / 6.0);
    a.g[3 * NP + idx] = T(Fy / 6.0);
    a.g[4 * NP + idx] = T(-(Fx + Fy) / 24.0);
    a.g[5 * NP + idx] = T((Fx - Fy) / 24.0);
    a.g[6 * NP + idx] = T((Fx + Fy) / 24.0);
    a.g[7 * NP + idx] = T((Fy - Fx) / 24.0);
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
constexpr int SWEEP_TX = 32, SWEEP_TY = 8;

template <typename T, typename TC>
cudaError_t launch_sweep_impl(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    constexpr size_t smem = sweep_smem_bytes<SWEEP_TX, SWEEP_TY, T>();
    auto kern = k_elastic_sweep<T, TC, SWEEP_TX, SWEEP_TY>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((a.nx + SWEEP_TX - 1) / SWEEP_TX, (a.ny + SWEEP_TY - 1) / SWEEP_TY);
    kern<<<grid, SWEEP_TX * SWEEP_TY, smem, s>>>(a);
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

#define BIOT_INSTANTIATE_LEVEL(T, TC)                                                              \
    template <> cudaError_t biot::launch_sweep<T, TC>(const biot::SweepArgs<T, TC> &a, cudaStream_t s) \
    {                                                                                              \
        return biot::launch_sweep_impl<T, TC>(a, s);                                               \
    }

#define BIOT_INSTANTIATE_FIELD(T)                                                                    \
    template <> cudaError_t biot::launch_force<T>(const biot::ForceArgs<T> &a, cudaStream_t s)         \
    { return biot::launch_force_impl<T>(a, s); }                                                     \
    template <> cudaError_t biot::launch_flow_moments<T>(const biot::FlowMomentsArgs<T> &a, cudaStream_t s) \
    { return biot::launch_flow_moments_impl<T>(a, s); }                                              \
    template <> cudaError_t biot::launch_flow_stream<T>(const biot::FlowStreamArgs<T> &a, cudaStream_t s) \
    { return biot::launch_flow_stream_impl<T>(a, s); }                                               \
    template <> cudaError_t biot::launch_readout<T>(const biot::ReadoutArgs<T> &a, cudaStream_t s)     \
    { return biot::launch_readout_impl<T>(a, s); }                                                   \
    template <> cudaError_t biot::launch_init<T>(const biot::InitArgs<T> &a, cudaStream_t s)           \
    { return biot::launch_init_impl<T>(a, s); }
