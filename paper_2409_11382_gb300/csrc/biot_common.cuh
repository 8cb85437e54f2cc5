// biot_common.cuh -- lattice tables and helpers shared by the sm_103a kernels
// of the coupled LBM for Biot's consolidation model (Lunowa & Wohlmuth,
// arXiv 2409.11382).
//
// Data layout in HBM: structure-of-arrays planes, plane stride nx*ny, y-major.
//   elastic state: 8 planes of MRT moments of the populations, in the column
//     order of Tab. moments:inverse (10, 01, 11, s, d, 12, 21, 22).  The moment
//     map of eqs. moments / moments:stress is an exact linear change of basis
//     of the D2Q8 populations, so storing moments is storing populations; it
//     keeps the small stress moments (s, d, 11, 22) at their own scale instead
//     of as differences of displacement-sized populations, which is what makes
//     FP32 storage accurate on large grids.
//   flow populations f: 9 planes, D2Q9 order 00, 10, 01, -10, 0-1, 11, -11, -1-1, 1-1
//     (Tab. velocities).
// Everything is in lattice units of the level it lives on: dx = dt = dtau = 1,
// c_s^2 = 1/3; scaling of §2.2 with L = h, T = dt, H = 1, eps = h.
//
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "biot_args.h"

namespace biot {

// ---------------------------------------------------------------------------
// Velocity sets.
// D2Q8 population index k: 10, 01, -10, 0-1, 11, -11, -1-1, 1-1.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex8(int k) { return (k == 0 || k == 4 || k == 7) ? 1 : (k == 2 || k == 5 || k == 6) ? -1 : 0; }
__host__ __device__ constexpr int ey8(int k) { return (k == 1 || k == 4 || k == 5) ? 1 : (k == 3 || k == 6 || k == 7) ? -1 : 0; }
__host__ __device__ constexpr int opp8(int k) { return k < 4 ? (k + 2) & 3 : 4 + ((k - 4 + 2) & 3); }
__host__ __device__ constexpr int dir8(int cx, int cy)
{
    return cy == 0 ? (cx > 0 ? 0 : 2)
         : cx == 0 ? (cy > 0 ? 1 : 3)
         : cy > 0 ? (cx > 0 ? 4 : 5) : (cx < 0 ? 6 : 7);
}
// Opposite pairs p: first member with velocity (1,0), (0,1), (1,1), (-1,1).
__host__ __device__ constexpr int pair_first(int p) { return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 4 : 5; }
__host__ __device__ constexpr int pair_second(int p) { return p == 0 ? 2 : p == 1 ? 3 : p == 2 ? 6 : 7; }
__host__ __device__ constexpr int pair_of(int k) { return (k == 0 || k == 2) ? 0 : (k == 1 || k == 3) ? 1 : (k == 4 || k == 6) ? 2 : 3; }
__host__ __device__ constexpr int sign_of(int k) { return (k == 0 || k == 1 || k == 4 || k == 5) ? 1 : -1; }
// Odd part of the post-collision populations of pair p,
//   A*_p = g*_first - g*_second = a_p . (m_10, m_01) + b_p . (F_x, F_y),
// from m*_10 = m_10 + F, m*_12 = (m_10 + F/2)/3 (and y alike) through
// Tab. moments:inverse.
__host__ __device__ constexpr double pa_x(int p) { return p == 0 ? 2.0 / 3.0 : p == 1 ? 0.0 : p == 2 ? 1.0 / 6.0 : -1.0 / 6.0; }
__host__ __device__ constexpr double pa_y(int p) { return p == 0 ? 0.0 : p == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double pb_x(int p) { return p == 0 ? 5.0 / 6.0 : p == 1 ? 0.0 : p == 2 ? 1.0 / 12.0 : -1.0 / 12.0; }
__host__ __device__ constexpr double pb_y(int p) { return p == 0 ? 0.0 : p == 1 ? 5.0 / 6.0 : 1.0 / 12.0; }

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

// Even / odd parts of the populations of a moment vector (Tab. moments:inverse
// written for opposite pairs): S_p = g_first + g_second, A_p = g_first - g_second.
template <typename T>
__device__ __forceinline__ void moments_to_pairs(const T (&m)[8], T (&S)[4], T (&A)[4])
{
    S[0] = T(0.5) * (m[3] + m[4]) - m[7];
    S[1] = T(0.5) * (m[3] - m[4]) - m[7];
    S[2] = T(0.5) * (m[2] + m[7]);
    S[3] = T(0.5) * (m[7] - m[2]);
    A[0] = m[0] - m[5];
    A[1] = m[1] - m[6];
    A[2] = T(0.5) * (m[5] + m[6]);
    A[3] = T(0.5) * (m[6] - m[5]);
}
// Moments of eqs. moments / moments:stress from the pair parts.
template <typename T>
__device__ __forceinline__ void pairs_to_moments(const T (&S)[4], const T (&A)[4], T (&m)[8])
{
    m[0] = (A[0] + A[2]) - A[3];
    m[1] = (A[1] + A[2]) + A[3];
    m[2] = S[2] - S[3];
    m[3] = (S[0] + S[1]) + T(2) * (S[2] + S[3]);
    m[4] = S[0] - S[1];
    m[5] = A[2] - A[3];
    m[6] = A[2] + A[3];
    m[7] = S[2] + S[3];
}
// max |g_k| over the populations of a moment vector (NaN -> +inf), in the
// storage type (a maximum is exact in any precision).
template <typename T>
__device__ __forceinline__ T pop_absmax(const T (&m)[8])
{
    T S[4], A[4];
    moments_to_pairs(m, S, A);
    T r = T(0);
#pragma unroll
    for (int p = 0; p < 4; p++) {
        const T u = fabs(T(0.5) * (S[p] + A[p]));
        const T v = fabs(T(0.5) * (S[p] - A[p]));
        r = fmax(r, (u == u) ? u : T(INFINITY));
        r = fmax(r, (v == v) ? v : T(INFINITY));
    }
    return r;
}

// Sum of the squared populations of a moment vector, sum_k g_k^2 =
// 1/2 sum_p (S_p^2 + A_p^2), in the storage type.
template <typename T>
__device__ __forceinline__ T pop_sumsq(const T (&m)[8])
{
    T S[4], A[4];
    moments_to_pairs(m, S, A);
    T r = T(0);
#pragma unroll
    for (int p = 0; p < 4; p++) r += S[p] * S[p] + A[p] * A[p];
    return T(0.5) * r;
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

// 16-bit values of the deviation store: DEV 1 = IEEE FP16, 2 = BF16, rounded
// to nearest on the way in.
template <int DEV>
__device__ __forceinline__ float dev_load(const void *p, size_t i)
{
    if constexpr (DEV == 1) return __half2float(static_cast<const __half *>(p)[i]);
    else return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
}
template <int DEV>
__device__ __forceinline__ void dev_store(void *p, size_t i, float v)
{
    if constexpr (DEV == 1) static_cast<__half *>(p)[i] = __float2half_rn(v);
    else static_cast<__nv_bfloat16 *>(p)[i] = __float2bfloat16_rn(v);
}

}  // namespace biot
