// sweep_mom.cuh -- fused elastic sweep on MOMENT storage (the FP32 path; also
// instantiated in FP64 for the coarsest level and for checking).
//
// The state of a cell is the vector of MRT moments of its D2Q8 populations in
// the column order of Tab. moments:inverse (10, 01, 11, s, d, 12, 21, 22).
// That is an exact change of basis (eqs. moments / moments:stress), so the
// scheme is unchanged; what changes is where rounding enters.  With FP32
// storage of populations, every sweep rounds each population at the scale of
// the displacement and the difference g - ELASTIC_STEP(g) -- which at the
// fixed point is the discrete momentum balance -- inherits that rounding as a
// spurious body force.  The elliptic solve amplifies such a force by ~N^2, so
// the FP32 result drifts from the FP64 one by ~N^2 * 6e-8 (4e-2 at 4096^2).
// Here the residual m - m** is formed from small quantities only:
//  * the even moments (s, d, 11, 22; the stress) are stored at their own scale;
//  * a population pulled from a neighbour y is split into a small part and
//    beta . (m_10, m_01)(x), the displacement-sized part written with the
//    target cell x's own first moments; the neighbour's displacement enters
//    only as m(y) - m(x), exact in floating point for nearby values;
//  * the beta parts of a pair cancel exactly away from walls, and m(x) - m**(x)
//    subtracts m(x) from itself symbolically rather than numerically;
//  * the first moments m_10, m_01 (the displacement) are carried as unevaluated
//    sums hi + lo of two values (double-float); on the finest FP32 level both
//    parts are stored, so the stored displacement is not rounded to FP32 either.
//    The other six moments do not need it: m_12, m_21, m_22 are overwritten by
//    the collision (rate 1) and s, d, 11 are stress-sized.
#pragma once
#include <stdlib.h>

#include "biot_common.cuh"

namespace biot {

// ---------------------------------------------------------------------------
// Row-streaming sweep.  A CTA of NT threads owns a strip of NT columns
// (x0-2 .. x0+NT-3) and TY rows; thread t owns column x0-2+t and walks down
// the strip.  Per output row y it (A) stores the moments of row y+2, prefetched
// into registers one iteration earlier, into a 3-row ring in shared memory and
// issues the loads of row y+3; (C) after a barrier collides row y+1 (it needs
// m_s of rows y..y+2 for F_*) into a 3-row ring of post-collision data; (E)
// after a barrier streams row y by pulling from rows y-1..y+1 of that ring,
// applies the wall rules, and relaxes or restricts.  The two outer columns on
// each side are halo: the outermost only supply m_s, the next ones are also
// collided; the NT-4 inner columns are written.  Strips overlap by 4 columns.
// The rings are planes (consecutive threads access consecutive elements, so
// the accesses are free of bank conflicts).  Values read by neighbouring
// threads have scalar planes: m_s in the raw ring, and in the post-collision
// ring the small part G_K of every outgoing population and the high parts of
// the first moments; values read only by the thread of the column are packed
// into 4-vectors (one 128-bit access each).  A pull thus reads one G_K and the
// one or two first moments its pair needs.
// FINE: finest level (explicit force F~, boundary data; double-float first
// moments when LO).  COARSE: residual right-hand side r, homogeneous walls.
// ---------------------------------------------------------------------------
// KIND bit 0: finest (0) or coarse (1) level; bit 1 (KIND_NOGHOST): the ghost
// moments m_12, m_21, m_22 are neither loaded nor stored.  Their relaxation rate
// is 1 (Tab. moments), so the collision overwrites them: the other moments, the
// restricted residual (coarse levels read r_0..r_4) and every output are
// independent of them, and only the residual norm contains them.  With fixed
// V-cycle counts they are elided (the norm then covers the other five moments'
// residuals); the tolerance mode keeps them for the paper's norm.
// KIND bits 2-3 (finest FP32 level without ghost moments only): m_11, m_s, m_d
// come from and go to the 16-bit deviation store, FP16 (KIND_DEV16) or BF16
// (KIND_DEVBF16).
enum { KIND_FINE = 0, KIND_COARSE = 1, KIND_NOGHOST = 2, KIND_DEV16 = 4, KIND_DEVBF16 = 8 };
__host__ __device__ constexpr bool kind_fine(int k) { return (k & 1) == 0; }
__host__ __device__ constexpr bool kind_ghosts(int k) { return (k & KIND_NOGHOST) == 0; }
__host__ __device__ constexpr int kind_dev(int k) { return (k & KIND_DEV16) ? 1 : (k & KIND_DEVBF16) ? 2 : 0; }

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;
};
template <typename T>
struct alignas(2 * sizeof(T)) V2 {
    T x, y;
};
template <int KIND, bool LO>
struct RingLayout {
    // values fetched per cell (fetch_cell): v0..v7 the 8 moments (the ghost
    // moments 0 when elided), then F~ (FINE, 2) or r_0..r_4 (COARSE, 5), then
    // the low parts of m_10, m_01 (LO)
    static constexpr int XV = 8;
    static constexpr int NXV = kind_fine(KIND) ? 2 : 5;
    static constexpr int LOV = XV + NXV;
    static constexpr int RV = LOV + (LO ? 2 : 0);
    // Raw ring: m_s on a scalar plane, q0 = (m_10, m_01, m_11, m_d) on a 4-vector
    // plane, and the cell's "extra" values e[0..NE) -- the ghost moments (when
    // kept), F~ or r, the low parts, in this order -- packed into 4-vector
    // planes, a remainder of two values into a 2-vector plane and of one value
    // into a scalar plane.
    static constexpr int EX = kind_ghosts(KIND) ? 3 : 0;  // first F~ / r value
    static constexpr int EL = EX + NXV;                    // first low part
    static constexpr int NE = EL + (LO ? 2 : 0);
    static constexpr int NE4 = (NE % 4 == 3) ? NE / 4 + 1 : NE / 4;
    static constexpr int NV4 = 1 + NE4;  // 4-vector planes per slot, q0 included
    static constexpr bool E2 = NE % 4 == 2;
    static constexpr bool E1 = NE % 4 == 1;
    // Post-collision ring: scalar planes G_0..G_7 (small parts of the outgoing
    // populations) and the high parts of the collision-input m_10, m_01.
    static constexpr int NPOST = 10;
    template <typename T>
    static constexpr size_t slot_bytes(int W)
    {
        return (size_t)W * (4 * NV4 + (E2 ? 2 : 0) + (E1 ? 1 : 0) + 1 + NPOST) * sizeof(T);
    }
};

template <typename T, int KIND, bool LO, int NT>
constexpr size_t rows_smem_bytes()
{
    return 3 * RingLayout<KIND, LO>::template slot_bytes<T>(NT);  // 3 slots
}

template <typename T>
struct PVal {
    // value = g + h + bx * m_10(x) + by * m_01(x): g stress-sized, h the small
    // target-relative part (kept apart so that a pair's sum and difference round
    // the stress-sized parts once)
    T g, h, bx, by;
};

// Shared-memory rings of W columns (slots: rows of the strip's window, or of
// the tile).
template <typename T, int W, int KIND, bool LO>
struct Rings {
    using L = RingLayout<KIND, LO>;
    V4<T> *q;   // [slot][NV4][W]  q0, packed extra values
    V2<T> *q2;  // [slot][W]       extra values, 2-vector remainder (E2)
    T *qs;      // [slot][W]       extra value, scalar remainder (E1)
    T *rms;     // [slot][W]       m_s
    T *post;    // [slot][NPOST][W] G_0..G_7, m_10, m_01 (high parts)
    __device__ __forceinline__ void carve(unsigned char *p, int slots)
    {
        q = reinterpret_cast<V4<T> *>(p);  // vectors first (alignment)
        q2 = reinterpret_cast<V2<T> *>(q + slots * L::NV4 * W);
        qs = reinterpret_cast<T *>(q2 + (L::E2 ? slots * W : 0));
        rms = qs + (L::E1 ? slots * W : 0);
        post = rms + slots * W;
    }
    __device__ __forceinline__ V4<T> &Q(int s, int j, int c) const { return q[(s * L::NV4 + j) * W + c]; }
    __device__ __forceinline__ T &ms(int s, int c) const { return rms[s * W + c]; }
    __device__ __forceinline__ T &G(int s, int k, int c) const { return post[(s * L::NPOST + k) * W + c]; }
    __device__ __forceinline__ T &MX(int s, int c) const { return post[(s * L::NPOST + 8) * W + c]; }
    __device__ __forceinline__ T &MY(int s, int c) const { return post[(s * L::NPOST + 9) * W + c]; }
    __device__ __forceinline__ void put_extras(int s, int c, const T (&e)[L::NE]) const
    {
#pragma unroll
        for (int j = 0; j < L::NE4; j++) {
            const int b = 4 * j;
            Q(s, 1 + j, c) = V4<T>{e[b], e[b + 1], e[b + 2 < L::NE ? b + 2 : b], b + 3 < L::NE ? e[b + 3] : T(0)};
        }
        if constexpr (L::E2) q2[s * W + c] = V2<T>{e[L::NE - 2], e[L::NE - 1]};
        if constexpr (L::E1) qs[s * W + c] = e[L::NE - 1];
    }
    __device__ __forceinline__ void get_extras(int s, int c, T (&e)[L::NE]) const
    {
#pragma unroll
        for (int j = 0; j < L::NE4; j++) {
            const V4<T> v = Q(s, 1 + j, c);
            const int b = 4 * j;
            e[b] = v.x;
            e[b + 1] = v.y;
            if (b + 2 < L::NE) e[b + 2 < L::NE ? b + 2 : b] = v.z;
            if (b + 3 < L::NE) e[b + 3 < L::NE ? b + 3 : b] = v.w;
        }
        if constexpr (L::E2) {
            const V2<T> v = q2[s * W + c];
            e[L::NE - 2] = v.x;
            e[L::NE - 1] = v.y;
        }
        if constexpr (L::E1) e[L::NE - 1] = qs[s * W + c];
    }
};

// Exact sum of two floating-point values: s + e == a + b.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e)
{
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// How a sweep's loads form the iterate: from the arguments at run time
// (a.zero_init, a.gc), or fixed at compile time -- the stored iterate, the
// stored iterate plus the prolongated coarse correction, or zero.
enum { FETCH_DYN = 0, FETCH_PLAIN = 1, FETCH_PROL = 2, FETCH_ZERO = 3, FETCH_ZPROL = 4 };

// Raw values of cell (gx, gy): moments of the iterate (+ prolongated coarse
// correction; with LO its first moments go to the low parts), F~ (FINE) or r
// (COARSE), low parts (LO).  Ghost cells of a non-periodic wall read the
// adjacent cell: only their m_s is used (even extension of the divergence).
// INB: the caller guarantees 0 <= gx < nx and 0 <= gy < ny.
template <typename T, typename TC, int KIND, bool LO, int RV, int FM = FETCH_DYN, bool INB = false>
__device__ __forceinline__ void fetch_cell(const SweepArgs<T, TC> &a, int gx, int gy, size_t NP, bool perx, bool pery,
                                           T (&v)[RV])
{
    using L = RingLayout<KIND, LO>;
    if constexpr (!INB) {
        if (perx) gx = wrapi(gx, a.nx);
        if (pery) gy = wrapi(gy, a.ny);
        gx = clampi(gx, a.nx);
        gy = clampi(gy, a.ny);
    }
    const size_t idx = (size_t)gy * a.nx + gx;
    constexpr int NM = kind_ghosts(KIND) ? 8 : 5;  // moment planes loaded
    const bool zero = FM == FETCH_ZERO || FM == FETCH_ZPROL || (FM == FETCH_DYN && a.zero_init);
    const bool prol = FM == FETCH_PROL || FM == FETCH_ZPROL || (FM == FETCH_DYN && a.gc != nullptr);
    constexpr int DEV = kind_dev(KIND);
    if (zero) {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = T(0);
    } else {
        const T *g = a.g + idx;
#pragma unroll
        for (int k = 0; k < NM; k++) {
            if (DEV && k >= 2 && k <= 4) v[k] = T(dev_load<DEV>(a.gd, (k - 2) * NP + idx)) * T(a.dinv);
            else v[k] = g[k * NP];
        }
#pragma unroll
        for (int k = NM; k < 8; k++) v[k] = T(0);
    }
    if (kind_fine(KIND)) {
        v[L::XV] = a.Ft[idx];
        v[L::XV + 1] = a.Ft[NP + idx];
    } else {
        const T *r = a.r + idx;
#pragma unroll
        for (int k = 0; k < 5; k++) v[L::XV + k] = r[k * NP];
    }
    if constexpr (LO) {
        v[L::LOV] = zero ? T(0) : a.glo[idx];
        v[L::LOV + 1] = zero ? T(0) : a.glo[NP + idx];
    }
    if (prol) {
        const size_t NPc = NP >> 2;
        const size_t cidx = (size_t)(gy >> 1) * (a.nx >> 1) + (gx >> 1);
        if constexpr (LO) {
            v[L::LOV] += (T)a.gc[cidx];
            v[L::LOV + 1] += (T)a.gc[NPc + cidx];
        } else {
            v[0] += (T)a.gc[cidx];
            v[1] += (T)a.gc[NPc + cidx];
        }
#pragma unroll
        for (int k = 2; k < NM; k++) v[k] += (T)a.gc[k * NPc + cidx];
    }
}

template <typename T, int W, int KIND, bool LO, int RV>
__device__ __forceinline__ void store_cell(const Rings<T, W, KIND, LO> &rg, int s, int c, const T (&v)[RV])
{
    using L = RingLayout<KIND, LO>;
    rg.ms(s, c) = v[3];
    rg.Q(s, 0, c) = V4<T>{v[0], v[1], v[2], v[4]};
    T e[L::NE];
#pragma unroll
    for (int i = 0; i < L::EX; i++) e[i] = v[5 + i];
#pragma unroll
    for (int i = 0; i < L::NXV; i++) e[L::EX + i] = v[L::XV + i];
#pragma unroll
    for (int i = 0; i < L::NE - L::EL; i++) e[L::EL + i] = v[L::LOV + i];
    rg.put_extras(s, c, e);
}

// Product rounded on its own, never fused into a neighbouring add: the pulls
// of wall cells and of interior cells are separate inlined copies of the same
// code, and an x-independent problem must give identical columns.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
// a * b + c with the rounding fixed by the source, not by the compiler's
// contraction choices: one fused multiply-add in either precision (the FP64
// kernels fuse nothing else).  The collision, pull, residual and relaxation
// arithmetic is shared by inlined copies in different kernels and loop forms;
// written with these, every copy rounds alike.  In FP64 the fused form also
// halves the FP64 instructions of these terms, and FP64 issue is what bounds
// the FP64 sweeps on this GPU.
__device__ __forceinline__ float mad_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mad_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// a_p . (x, y) / 2 for the odd coefficient vectors a_p of Tab. moments:inverse,
// zero terms omitted.
template <typename T, int P>
__device__ __forceinline__ T half_pa_dot(T x, T y)
{
    static_assert(pa_x(0) == 2.0 / 3.0 && pa_y(0) == 0.0 && pa_x(1) == 0.0 && pa_y(1) == 2.0 / 3.0 &&
                      pa_x(2) == 1.0 / 6.0 && pa_y(2) == 1.0 / 6.0 && pa_x(3) == -1.0 / 6.0 && pa_y(3) == 1.0 / 6.0,
                  "coefficients a_p");
    if constexpr (P == 0) return mul_rn(T(1.0 / 3.0), x);
    if constexpr (P == 1) return mul_rn(T(1.0 / 3.0), y);
    if constexpr (P == 2) return mul_rn(T(1.0 / 12.0), x + y);
    return mul_rn(T(1.0 / 12.0), y - x);
}

// Collision of the cell in raw slot s, column c (Alg. 2, first six lines, in
// moment space): even moments relaxed (Tab. moments, eq. moments:collision:22),
// odd part kept as first moments + force F = F~ + (alpha^2 r/2) grad^c D(g).
// Writes, per outgoing direction K of pair p and sign e, the part of
//   g*_K = 1/2 (S*_p + e A*_p),  A*_p = a_p . m + b_p . F  (Tab. moments:inverse)
// that does not contain the high parts of the first moments,
//   G_K = 1/2 (S*_p + e (a_p . m_lo + b_p . F)),
// and the high parts m_10, m_01 themselves: a pull adds e/2 a_p . (m_hi(source)
// - m_hi(target)), a difference of nearby values (exact), so that no
// displacement-sized value is ever rounded into a population.
template <typename T>
struct CollideOut {
    T G[8];   // G_0 .. G_7
    T mx, my; // high parts of the collision-input m_10, m_01
};

// The arithmetic of the collision from the cell's own values (moments m0..m4,
// extra values e in the raw-ring order of RingLayout) and m_s of its eight
// neighbours; shared by the ring and register forms of the strip sweep, so that
// both round identically.
template <typename T, typename TC, int KIND, bool LO, int NE>
__device__ __forceinline__ CollideOut<T> collide_math(const SweepArgs<T, TC> &a, T m0, T m1, T m2, T m3, T m4,
                                                     const T (&e)[NE], T dE, T dW, T dN, T dS, T dNE, T dNW, T dSE,
                                                     T dSW)
{
    using L = RingLayout<KIND, LO>;
    const T cf = a.k_fs;  // alpha^2 r/2 * dD/dm_s
    T Fx = mul_rn(cf, mad_rn(dE - dW, T(1.0 / 3.0), mul_rn((dNE + dSE) - (dNW + dSW), T(1.0 / 12.0))));
    T Fy = mul_rn(cf, mad_rn(dN - dS, T(1.0 / 3.0), mul_rn((dNE + dNW) - (dSE + dSW), T(1.0 / 12.0))));
    T lx = T(0), ly = T(0);  // low parts of the collision-input first moments (LO)
    if constexpr (kind_fine(KIND)) {
        Fx += e[L::EX];  // F~
        Fy += e[L::EX + 1];
        if constexpr (LO) {
            lx = e[L::EL];
            ly = e[L::EL + 1];
        }
    } else {  // minus the residual right-hand side r_0..r_4
        if constexpr (LO) {  // r_0, r_1 come off the low parts
            lx = e[L::EL] - e[L::EX];
            ly = e[L::EL + 1] - e[L::EX + 1];
        } else {
            m0 -= e[L::EX];
            m1 -= e[L::EX + 1];
        }
        m2 -= e[L::EX + 2];
        m3 -= e[L::EX + 3];
        m4 -= e[L::EX + 4];
    }
    // halves of the even combinations S*_p, one multiply and one fused multiply-add each
    const T hd = mul_rn(a.k_hd, m4), h22 = mul_rn(a.k_h22, m3);
    const T hS0 = mad_rn(a.k_hs, m3, hd), hS1 = mad_rn(a.k_hs, m3, -hd);
    const T hS2 = mad_rn(a.k_hd, m2, h22), hS3 = mad_rn(-a.k_hd, m2, h22);
    // G_K = S*_p/2 + e (a_p . m_lo + b_p . F)/2, b_p = (5/6, 0), (0, 5/6), (1/12, 1/12), (-1/12, 1/12)
    static_assert(pb_x(0) == 5.0 / 6.0 && pb_y(0) == 0.0 && pb_x(1) == 0.0 && pb_y(1) == 5.0 / 6.0 &&
                      pb_x(2) == 1.0 / 12.0 && pb_y(2) == 1.0 / 12.0 && pb_x(3) == -1.0 / 12.0 && pb_y(3) == 1.0 / 12.0,
                  "coefficients b_p");
    static_assert(pair_first(0) == 0 && pair_second(0) == 2 && pair_first(1) == 1 && pair_second(1) == 3 &&
                      pair_first(2) == 4 && pair_second(2) == 6 && pair_first(3) == 5 && pair_second(3) == 7,
                  "pairs");
    const T Fp = Fx + Fy, Fm = Fy - Fx;
    T G0, G1, G2, G3, G4, G5, G6, G7;
    if constexpr (LO) {  // odd parts without the high moments first (small), then one add each
        const T A0 = mad_rn(T(5.0 / 12.0), Fx, half_pa_dot<T, 0>(lx, ly));
        const T A1 = mad_rn(T(5.0 / 12.0), Fy, half_pa_dot<T, 1>(lx, ly));
        const T A2 = mad_rn(T(1.0 / 24.0), Fp, half_pa_dot<T, 2>(lx, ly));
        const T A3 = mad_rn(T(1.0 / 24.0), Fm, half_pa_dot<T, 3>(lx, ly));
        G0 = hS0 + A0;
        G2 = hS0 - A0;
        G1 = hS1 + A1;
        G3 = hS1 - A1;
        G4 = hS2 + A2;
        G6 = hS2 - A2;
        G5 = hS3 + A3;
        G7 = hS3 - A3;
    } else {  // one fused multiply-add each
        G0 = mad_rn(T(5.0 / 12.0), Fx, hS0);
        G2 = mad_rn(T(-5.0 / 12.0), Fx, hS0);
        G1 = mad_rn(T(5.0 / 12.0), Fy, hS1);
        G3 = mad_rn(T(-5.0 / 12.0), Fy, hS1);
        G4 = mad_rn(T(1.0 / 24.0), Fp, hS2);
        G6 = mad_rn(T(-1.0 / 24.0), Fp, hS2);
        G5 = mad_rn(T(1.0 / 24.0), Fm, hS3);
        G7 = mad_rn(T(-1.0 / 24.0), Fm, hS3);
    }
    CollideOut<T> o;
    o.G[0] = G0;
    o.G[1] = G1;
    o.G[2] = G2;
    o.G[3] = G3;
    o.G[4] = G4;
    o.G[5] = G5;
    o.G[6] = G6;
    o.G[7] = G7;
    o.mx = m0;
    o.my = m1;
    return o;
}

template <typename T, typename TC, int KIND, bool LO, int W>
__device__ __forceinline__ void collide_cell(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int sm, int s,
                                             int sp, int c)
{
    using L = RingLayout<KIND, LO>;
    const V4<T> q0 = rg.Q(s, 0, c);
    T e[L::NE];
    rg.get_extras(s, c, e);
    const T dE = rg.ms(s, c + 1), dW = rg.ms(s, c - 1), dN = rg.ms(sp, c), dS = rg.ms(sm, c);
    const T dNE = rg.ms(sp, c + 1), dNW = rg.ms(sp, c - 1), dSE = rg.ms(sm, c + 1), dSW = rg.ms(sm, c - 1);
    const CollideOut<T> o = collide_math<T, TC, KIND, LO, L::NE>(a, q0.x, q0.y, q0.z, rg.ms(s, c), q0.w, e, dE, dW, dN,
                                                                 dS, dNE, dNW, dSE, dSW);
#pragma unroll
    for (int k = 0; k < 8; k++) rg.G(s, k, c) = o.G[k];
    rg.MX(s, c) = o.mx;
    rg.MY(s, c) = o.my;
}

// Post-collision population K of the source cell in slot s, column c, split
// relative to the target's collision-input first moments (tx, ty high, tlx,
// tly low parts): sig = G_K + e/2 a_p . ((m_hi - t_hi) - t_lo).
template <typename T, bool LO, int K>
__device__ __forceinline__ PVal<T> pval_from(T g, T smx, T smy, T tx, T ty, T tlx, T tly)
{
    constexpr int p = pair_of(K);
    constexpr bool POS = sign_of(K) > 0;
    T dx = T(0), dy = T(0);
    if constexpr (pa_x(p) != 0.0) {
        dx = smx - tx;
        if constexpr (LO) dx -= tlx;
    }
    if constexpr (pa_y(p) != 0.0) {
        dy = smy - ty;
        if constexpr (LO) dy -= tly;
    }
    T h;
    if constexpr (p == 0) h = mul_rn(T(1.0 / 3.0), dx);
    else if constexpr (p == 1) h = mul_rn(T(1.0 / 3.0), dy);
    else if constexpr (p == 2) h = mul_rn(T(1.0 / 12.0), dx + dy);
    else h = mul_rn(T(1.0 / 12.0), dy - dx);
    static_assert(pa_x(0) == 2.0 / 3.0 && pa_y(1) == 2.0 / 3.0 && pa_x(2) == 1.0 / 6.0 && pa_y(2) == 1.0 / 6.0 &&
                      pa_x(3) == -1.0 / 6.0 && pa_y(3) == 1.0 / 6.0,
                  "h = a_p . (dx, dy) / 2");
    PVal<T> v;
    v.g = g;
    v.h = POS ? h : -h;
    v.bx = T(sign_of(K) * 0.5 * pa_x(p));
    v.by = T(sign_of(K) * 0.5 * pa_y(p));
    return v;
}

template <typename T, bool LO, int W, int KIND, int K>
__device__ __forceinline__ PVal<T> post_at(const Rings<T, W, KIND, LO> &rg, int s, int c, T tx, T ty, T tlx, T tly)
{
    constexpr int p = pair_of(K);
    const T smx = pa_x(p) != 0.0 ? rg.MX(s, c) : T(0);
    const T smy = pa_y(p) != 0.0 ? rg.MY(s, c) : T(0);
    return pval_from<T, LO, K>(rg.G(s, K, c), smx, smy, tx, ty, tlx, tly);
}

// Population of direction K arriving at cell (x, y) (ring column c0); sl[0..2]
// are the slots of rows y-1, y, y+1.
template <typename T, typename TC, int KIND, bool LO, int W, int K, bool WALL>
__device__ __forceinline__ PVal<T> pull(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int x, int y,
                                        const int (&sl)[3], int c0, T tx, T ty, T tlx, T tly, bool perx, bool pery)
{
    constexpr int cx = ex8(K), cy = ey8(K);
    const int s0 = sl[1];
    if (!WALL) return post_at<T, LO, W, KIND, K>(rg, sl[1 - cy], c0 - cx, tx, ty, tlx, tly);
    const int sx = x - cx, sy = y - cy;
    const bool outx = !perx && (sx < 0 || sx >= a.nx);
    const bool outy = !pery && (sy < 0 || sy >= a.ny);
    if (!outx && !outy) return post_at<T, LO, W, KIND, K>(rg, sl[1 - cy], c0 - cx, tx, ty, tlx, tly);
    int side = outy ? (sy < 0 ? SIDE_BOTTOM : SIDE_TOP) : (sx < 0 ? SIDE_LEFT : SIDE_RIGHT);
    if (outy && outx) {
        // corner: a bounce-back type side wall wins over a mirror top/bottom
        const int vert = sx < 0 ? SIDE_LEFT : SIDE_RIGHT;
        if (a.bc[side] == BC_SYMMETRY && a.bc[vert] != BC_SYMMETRY) side = vert;
    }
    const int type = a.bc[side];
    if (type == BC_SYMMETRY) {
        // mirror image of the ghost source, normal velocity reversed
        if (outy) {
            if (outx) return post_at<T, LO, W, KIND, dir8(-cx, -cy)>(rg, s0, c0, tx, ty, tlx, tly);
            return post_at<T, LO, W, KIND, dir8(cx, -cy)>(rg, s0, c0 - cx, tx, ty, tlx, tly);
        }
        return post_at<T, LO, W, KIND, dir8(-cx, cy)>(rg, sl[1 - cy], c0, tx, ty, tlx, tly);
    }
    constexpr int kout = opp8(K);
    const PVal<T> o = post_at<T, LO, W, KIND, kout>(rg, s0, c0, tx, ty, tlx, tly);
    const bool horiz = (side == SIDE_BOTTOM || side == SIDE_TOP);
    const int n = horiz ? a.nx : a.ny;
    PVal<T> v;
    if (type == BC_NEUMANN) {  // eq. BC:traction
        v.g = -o.g;
        v.h = -o.h;
        v.bx = -o.bx;
        v.by = -o.by;
        if (kind_fine(KIND) && a.prof[side]) v.g += T(a.c0h * traction_term(a.prof[side], side, n, x, y, cx, cy));
        return v;
    }
    // BC_DIRICHLET: eq. BC:elasticity, history = previous call's outgoing population
    if (a.hist_valid) {
        v.g = a.H[side][3 * (horiz ? x : y) + hslot(side, kout)];
        v.h = T(0);
        v.bx = T(0);
        v.by = T(0);
    } else {
        v = o;
    }
    if (kind_fine(KIND) && a.prof[side]) v.g += T(dirichlet_term(a.prof[side], side, n, x, y, cx, cy));
    return v;
}

// Pair p after streaming: S = g_first + g_second, A = g_first - g_second, each
// as a small part plus a beta part.  dB = (beta difference) - a_p vanishes
// exactly away from walls, as does the beta sum.
template <typename T>
struct PairOut {
    T Ss, As;      // small parts
    T bsx, bsy;    // beta sum (S)
    T dbx, dby;    // beta difference minus a_p (A)
};

template <typename T, int P>
__device__ __forceinline__ PairOut<T> pair_from(const PVal<T> &u, const PVal<T> &v);

template <typename T, typename TC, int KIND, bool LO, int W, int P, bool WALL>
__device__ __forceinline__ PairOut<T> pull_pair(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int x, int y,
                                                const int (&sl)[3], int c0, T tx, T ty, T tlx, T tly, bool perx, bool pery)
{
    const PVal<T> u = pull<T, TC, KIND, LO, W, pair_first(P), WALL>(a, rg, x, y, sl, c0, tx, ty, tlx, tly, perx, pery);
    const PVal<T> v = pull<T, TC, KIND, LO, W, pair_second(P), WALL>(a, rg, x, y, sl, c0, tx, ty, tlx, tly, perx, pery);
    return pair_from<T, P>(u, v);
}

template <typename T, int P>
__device__ __forceinline__ PairOut<T> pair_from(const PVal<T> &u, const PVal<T> &v)
{
    PairOut<T> o;
    o.Ss = (u.g + v.g) + (u.h + v.h);
    o.As = (u.g - v.g) + (u.h - v.h);
    o.bsx = u.bx + v.bx;
    o.bsy = u.by + v.by;
    o.dbx = (u.bx - v.bx) - T(pa_x(P));
    o.dby = (u.by - v.by) - T(pa_y(P));
    return o;
}

template <typename T, typename TC, bool LO, int W, int KIND, int K>
__device__ __forceinline__ void store_history(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int side, int pos,
                                              int s0, int c0, T tx, T ty, T tlx, T tly)
{
    const PVal<T> o = post_at<T, LO, W, KIND, K>(rg, s0, c0, tx, ty, tlx, tly);
    a.H[side][3 * pos + hslot(side, K)] = (o.g + o.h) + (mul_rn(o.bx, tx + tlx) + mul_rn(o.by, ty + tly));
}

// The streamed cell's own values, from its raw ring slot: the iterate's moments
// g, the low parts of m_10, m_01 (LO), and the collision-input first moments as
// the collision formed them (tx, ty high, tlx, tly low parts).
template <typename T>
struct OwnCell {
    T g[8];
    T lo[2];
    T tx, ty, tlx, tly;
};

template <typename T, int KIND, bool LO, int NE>
__device__ __forceinline__ OwnCell<T> own_from(T m0, T m1, T m2, T m3, T m4, const T (&e)[NE])
{
    using L = RingLayout<KIND, LO>;
    OwnCell<T> o;
    o.g[0] = m0;
    o.g[1] = m1;
    o.g[2] = m2;
    o.g[3] = m3;
    o.g[4] = m4;
#pragma unroll
    for (int i = 0; i < 3; i++) o.g[5 + i] = T(0);
    if constexpr (kind_ghosts(KIND)) {
        o.g[5] = e[0];
        o.g[6] = e[1];
        o.g[7] = e[2];
    }
    o.lo[0] = o.lo[1] = T(0);
    if constexpr (LO) {
        o.lo[0] = e[L::EL];
        o.lo[1] = e[L::EL + 1];
    }
    o.tx = o.g[0];
    o.ty = o.g[1];
    o.tlx = o.lo[0];
    o.tly = o.lo[1];
    if constexpr (!kind_fine(KIND)) {  // the same operations as collide_cell
        if constexpr (LO) {
            o.tlx = o.lo[0] - e[L::EX];
            o.tly = o.lo[1] - e[L::EX + 1];
        } else {
            o.tx = o.g[0] - e[L::EX];
            o.ty = o.g[1] - e[L::EX + 1];
        }
    }
    return o;
}

template <typename T, int W, int KIND, bool LO>
__device__ __forceinline__ OwnCell<T> own_cell(const Rings<T, W, KIND, LO> &rg, int s, int c)
{
    using L = RingLayout<KIND, LO>;
    const V4<T> q0 = rg.Q(s, 0, c);
    T e[L::NE];
    rg.get_extras(s, c, e);
    return own_from<T, KIND, LO, L::NE>(q0.x, q0.y, q0.z, rg.ms(s, c), q0.w, e);
}

// The wall-free part of the residual d = m - m** from the four streamed pairs
// (shared by the ring and register forms of the strip sweep).
template <typename T, int KIND, bool LO>
__device__ __forceinline__ void residual_core(const OwnCell<T> &own, const PairOut<T> &P0, const PairOut<T> &P1,
                                              const PairOut<T> &P2, const PairOut<T> &P3, T (&d)[8])
{
    const T(&gcur)[8] = own.g;
    const T tx = own.tx, ty = own.ty, tlx = own.tlx, tly = own.tly;
    const T mxf = tx + tlx, myf = ty + tly;  // full first moments: beta terms (walls) and the m_12, m_21 residuals
    // odd moments: m**_10 = (A0 + A2 - A3) = small + m_10(x) + dB-terms, etc.
    // (sum_p c_p a_p = (1,0), (0,1), (1/3,0), (0,1/3) for 10, 01, 12, 21)
    // residual rhs r_0, r_1 on coarse levels (0 on the finest): the iterate minus
    // the collision input, high and low parts differenced separately
    T r0 = gcur[0] - tx, r1 = gcur[1] - ty;
    if constexpr (LO && !kind_fine(KIND)) {
        r0 += own.lo[0] - tlx;
        r1 += own.lo[1] - tly;
    }
    d[0] = r0 - ((P0.As + P2.As) - P3.As);
    d[1] = r1 - ((P1.As + P2.As) + P3.As);
    d[5] = (gcur[5] - mul_rn(mxf, T(1.0 / 3.0))) - (P2.As - P3.As);
    d[6] = (gcur[6] - mul_rn(myf, T(1.0 / 3.0))) - (P2.As + P3.As);
    d[2] = gcur[2] - (P2.Ss - P3.Ss);
    d[3] = gcur[3] - ((P0.Ss + P1.Ss) + T(2) * (P2.Ss + P3.Ss));
    d[4] = gcur[4] - (P0.Ss - P1.Ss);
    d[7] = gcur[7] - (P2.Ss + P3.Ss);
}

// Residual d = m - m** of the cell (x, y) (small parts only, see the file
// comment); own: the cell's own values.
template <typename T, typename TC, int KIND, bool LO, int W, bool WALL>
__device__ __forceinline__ void residual_cell(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int x, int y,
                                              const int (&sl)[3], int c0, bool perx, bool pery, const OwnCell<T> &own,
                                              T (&d)[8])
{
    const int s0 = sl[1];
    const T(&gcur)[8] = own.g;
    const T tx = own.tx, ty = own.ty, tlx = own.tlx, tly = own.tly;
#define BIOT_PAIR(P) pull_pair<T, TC, KIND, LO, W, P, WALL>(a, rg, x, y, sl, c0, tx, ty, tlx, tly, perx, pery)
    const PairOut<T> P0 = BIOT_PAIR(0), P1 = BIOT_PAIR(1), P2 = BIOT_PAIR(2), P3 = BIOT_PAIR(3);
#undef BIOT_PAIR
    residual_core<T, KIND, LO>(own, P0, P1, P2, P3, d);
    const T mxf = tx + tlx, myf = ty + tly;
    constexpr bool GH = kind_ghosts(KIND);
    if (WALL) {
        // beta terms of the wall pulls; products rounded on their own (mul_rn), so
        // that no contraction choice of the compiler makes kernel forms differ
        d[0] -= mul_rn((P0.dbx + P2.dbx) - P3.dbx, mxf) + mul_rn((P0.dby + P2.dby) - P3.dby, myf);
        d[1] -= mul_rn((P1.dbx + P2.dbx) + P3.dbx, mxf) + mul_rn((P1.dby + P2.dby) + P3.dby, myf);
        d[5] -= mul_rn(P2.dbx - P3.dbx, mxf) + mul_rn(P2.dby - P3.dby, myf);
        d[6] -= mul_rn(P2.dbx + P3.dbx, mxf) + mul_rn(P2.dby + P3.dby, myf);
        d[2] -= mul_rn(P2.bsx - P3.bsx, mxf) + mul_rn(P2.bsy - P3.bsy, myf);
        d[3] -= mul_rn((P0.bsx + P1.bsx) + T(2) * (P2.bsx + P3.bsx), mxf) +
                mul_rn((P0.bsy + P1.bsy) + T(2) * (P2.bsy + P3.bsy), myf);
        d[4] -= mul_rn(P0.bsx - P1.bsx, mxf) + mul_rn(P0.bsy - P1.bsy, myf);
        d[7] -= mul_rn(P2.bsx + P3.bsx, mxf) + mul_rn(P2.bsy + P3.bsy, myf);
        // history of the fullway bounce-back: this call's outgoing populations
#define BIOT_HIST(SIDE, POS, K) store_history<T, TC, LO, W, KIND, K>(a, rg, SIDE, POS, s0, c0, tx, ty, tlx, tly)
        if (y == 0 && a.bc[SIDE_BOTTOM] == BC_DIRICHLET) { BIOT_HIST(SIDE_BOTTOM, x, 3); BIOT_HIST(SIDE_BOTTOM, x, 6); BIOT_HIST(SIDE_BOTTOM, x, 7); }
        if (y == a.ny - 1 && a.bc[SIDE_TOP] == BC_DIRICHLET) { BIOT_HIST(SIDE_TOP, x, 1); BIOT_HIST(SIDE_TOP, x, 4); BIOT_HIST(SIDE_TOP, x, 5); }
        if (x == 0 && a.bc[SIDE_LEFT] == BC_DIRICHLET) { BIOT_HIST(SIDE_LEFT, y, 2); BIOT_HIST(SIDE_LEFT, y, 5); BIOT_HIST(SIDE_LEFT, y, 6); }
        if (x == a.nx - 1 && a.bc[SIDE_RIGHT] == BC_DIRICHLET) { BIOT_HIST(SIDE_RIGHT, y, 0); BIOT_HIST(SIDE_RIGHT, y, 4); BIOT_HIST(SIDE_RIGHT, y, 7); }
#undef BIOT_HIST
    }
    if (!GH) d[5] = d[6] = d[7] = T(0);  // elided ghost moments (see KIND_NOGHOST)
}

// The smoothed iterate m - gamma d of the cell at idx (eq. MG:smoother in
// moment space): the first moments as (hi + lo) - gamma d renormalised into hi +
// lo with LO; m_11, m_s, m_d into the deviation store (and, in the last sweep of
// a solve, also in FP32) when the level has one.
template <typename T, typename TC, int KIND, bool LO>
__device__ __forceinline__ void store_smoothed(const SweepArgs<T, TC> &a, size_t idx, size_t NP, const OwnCell<T> &own,
                                               const T (&d)[8], T gam)
{
    constexpr int DEV = kind_dev(KIND);
    const T(&gcur)[8] = own.g;
    T *go = a.gout + idx;
#pragma unroll
    for (int k = 2; k < (kind_ghosts(KIND) ? 8 : 5); k++) {
        const T v = mad_rn(-gam, d[k], gcur[k]);
        if (DEV && k <= 4) {
            dev_store<DEV>(a.gd_out, (k - 2) * NP + idx, float(v * T(a.dsc)));
            if (a.dev_full) go[k * NP] = v;
        } else {
            go[k * NP] = v;
        }
    }
    if constexpr (LO) {
#pragma unroll
        for (int k = 0; k < 2; k++) {
            T hi, lw;
            two_sum(gcur[k], mad_rn(-gam, d[k], own.lo[k]), hi, lw);
            go[k * NP] = hi;
            a.glo_out[k * NP + idx] = lw;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 2; k++) go[k * NP] = mad_rn(-gam, d[k], gcur[k]);
    }
}

// One strip (column block bx, row block by of TY rows) of one sweep; the body
// of both the single-instance kernel and the batched work-list kernel.  The CTA
// has NT threads and a window of W = NT * CPT columns: thread t owns the ring
// columns t, t + NT, ..., so every plane access of a warp stays on consecutive
// words, and the per-row work that does not depend on the column -- ring slots,
// loop control, barriers, row predicates -- is shared by the thread's CPT cells.
// INT: the CTA's whole window -- columns x0-2 .. x0+W-3, rows y0-2 .. y1+2 --
// lies inside the grid (sweep_strip_interior), so no cell of it is a wall cell
// or reads a ghost or wrapped source: no clamping, no wall rules, no row tests.
template <typename T, typename TC, int NT, int CPT, int KIND, bool LO, bool RESTRICT, int FM, bool INT>
__device__ __forceinline__ void sweep_strip(const SweepArgs<T, TC> &a, int bx, int by, int TY, unsigned char *smem_raw,
                                            double (&red)[3][NT / 32])
{
    using L = RingLayout<KIND, LO>;
    constexpr int W = NT * CPT, RV = L::RV;
    static_assert(NT % 32 == 0 && NT % 2 == 0, "whole warps; even column offsets keep restriction pairs in one warp");
    Rings<T, W, KIND, LO> rg;
    rg.carve(smem_raw, 3);

    const int nx = a.nx, ny = a.ny;
    const size_t NP = (size_t)nx * ny;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;
    const int t = threadIdx.x;
    const int x0 = bx * (W - 4), y0 = by * TY;
    const int y1 = min(y0 + TY, ny);

    // this thread's columns x[j] = x0 - 2 + c[j], ring columns c[j] = t + j NT
    int xj[CPT], cj[CPT];
    bool loads[CPT], collides[CPT], writes[CPT], wall_col[CPT];
#pragma unroll
    for (int j = 0; j < CPT; j++) {
        cj[j] = t + j * NT;
        xj[j] = x0 - 2 + cj[j];
        if constexpr (INT) {
            loads[j] = true;
            collides[j] = cj[j] >= 1 && cj[j] < W - 1;
            writes[j] = cj[j] >= 2 && cj[j] < W - 2;
            wall_col[j] = false;
        } else {
            loads[j] = perx || xj[j] < nx + 2;  // a real, wrapped or ghost column
            collides[j] = cj[j] >= 1 && cj[j] < W - 1 && (perx || (xj[j] >= 0 && xj[j] < nx));
            writes[j] = cj[j] >= 2 && cj[j] < W - 2 && xj[j] < nx;
            wall_col[j] = !perx && (xj[j] == 0 || xj[j] == nx - 1);
        }
    }

    auto row_ok = [&](int y) { return INT || pery || (y >= 0 && y < ny); };

    T pv[CPT][RV];
    auto fetch_row = [&](int y) {
#pragma unroll
        for (int j = 0; j < CPT; j++)
            if (loads[j]) fetch_cell<T, TC, KIND, LO, RV, FM, INT>(a, xj[j], y, NP, perx, pery, pv[j]);
    };
    auto store_row = [&](int s) {
#pragma unroll
        for (int j = 0; j < CPT; j++)
            if (loads[j]) store_cell<T, W, KIND, LO, RV>(rg, s, cj[j], pv[j]);
    };
    auto collide_row = [&](int y, int sm, int s, int sp) {
        if (!row_ok(y)) return;
#pragma unroll
        for (int j = 0; j < CPT; j++)
            if (collides[j]) collide_cell<T, TC, KIND, LO, W>(a, rg, sm, s, sp, cj[j]);
    };

    // ring slots: rows y0-2, y0-1, y0 in slots 0, 1, 2; row r in slot (r - y0 + 2) % 3
    fetch_row(y0 - 2);
    store_row(0);
    fetch_row(y0 - 1);
    store_row(1);
    fetch_row(y0);
    store_row(2);
    __syncthreads();
    collide_row(y0 - 1, 0, 1, 2);
    fetch_row(y0 + 1);
    __syncthreads();
    store_row(0);
    fetch_row(y0 + 2);
    __syncthreads();
    collide_row(y0, 1, 2, 0);
    __syncthreads();

    T rmax = T(0), gmax = T(0);
    double rsum = 0.0;  // FP64 sum of the squared population residuals (measured sweeps)
    T acc[CPT][8];
#pragma unroll
    for (int j = 0; j < CPT; j++)
#pragma unroll
        for (int k = 0; k < 8; k++) acc[j][k] = T(0);
    const T gam = a.k_gam;
    // slots of rows y-1, y, y+1 (row y+2 reuses the slot of row y-1)
    int sa = 1, sb = 2, sc = 0;

    for (int y = y0; y < y1; y++) {
        store_row(sa);     // (A) prefetched row y+2 -> raw ring (slot of row y-1)
        fetch_row(y + 3);  //     prefetch row y+3
        __syncthreads();   // (C)
        collide_row(y + 1, sb, sc, sa);
        __syncthreads();   // (E)
        const int sl[3] = {sa, sb, sc};
        const bool wall_row = !INT && !pery && (y == 0 || y == ny - 1);
#pragma unroll
        for (int j = 0; j < CPT; j++) {
            const int x = xj[j], c = cj[j];
            T d[8];
#pragma unroll
            for (int k = 0; k < 8; k++) d[k] = T(0);
            if (writes[j]) {
                const OwnCell<T> own = own_cell<T, W, KIND, LO>(rg, sb, c);
                const T(&gcur)[8] = own.g;
                if (!INT && (wall_col[j] || wall_row)) residual_cell<T, TC, KIND, LO, W, true>(a, rg, x, y, sl, c, perx, pery, own, d);
                else residual_cell<T, TC, KIND, LO, W, false>(a, rg, x, y, sl, c, perx, pery, own, d);
                if (!RESTRICT) {
                    store_smoothed<T, TC, KIND, LO>(a, (size_t)y * nx + x, NP, own, d, gam);
                    if (a.resmax) {
                        rmax = fmax(rmax, pop_absmax(d));
                        gmax = fmax(gmax, pop_absmax(gcur));
                        rsum += (double)pop_sumsq(d);
                    }
                }
            }
            if (RESTRICT) {
                // full-sum restriction of eq. MG:restriction: pair rows, then columns
                // (columns x, x+1 with x even sit in lanes t, t+1 of one warp)
                const bool odd = ((y - y0) & 1) != 0;
#pragma unroll
                for (int k = 0; k < 8; k++) acc[j][k] = odd ? acc[j][k] + d[k] : d[k];
                if (odd) {
                    TC tot[8];
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        const TC mine = (TC)acc[j][k];
                        tot[k] = mine + __shfl_down_sync(0xffffffffu, mine, 1);
                    }
                    if (writes[j] && (x & 1) == 0) {
                        const size_t NPc = NP >> 2;
                        const size_t cidx = (size_t)(y >> 1) * (nx >> 1) + (x >> 1);
#pragma unroll
                        for (int k = 0; k < (kind_ghosts(KIND) ? 8 : 5); k++) a.rc[k * NPc + cidx] = tot[k];
                    }
                }
            }
        }
        const int s_old = sa;  // rotate: rows y, y+1, y+2 become y-1, y, y+1
        sa = sb;
        sb = sc;
        sc = s_old;
    }

    if (!RESTRICT && a.resmax) {
        // warp-shuffle then block reduction of the two maxima and the sum, one atomic each per CTA
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        }
        const int warp = t >> 5, lane = t & 31;
        if (lane == 0) {
            red[0][warp] = (double)rmax;
            red[1][warp] = (double)gmax;
            red[2][warp] = rsum;
        }
        __syncthreads();
        if (t == 0) {
            double r0 = 0.0, g0 = 0.0, q0 = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                r0 = fmax(r0, red[0][w]);
                g0 = fmax(g0, red[1][w]);
                q0 += red[2][w];
            }
            atomicMax(&a.resmax[0], (unsigned long long)__double_as_longlong(r0));
            atomicMax(&a.resmax[1], (unsigned long long)__double_as_longlong(g0));
            atomicAdd(reinterpret_cast<double *>(&a.resmax[2]), q0);
        }
    }
}

// ---------------------------------------------------------------------------
// Register form of the interior strip (fixed V-cycle counts: no ghost moments).
// The values only the column's own thread uses stay in registers instead of
// the shared rings: the raw values of rows y, y+1, y+2 (its moments, F~ or r,
// low parts), and of the post-collision data the populations 01 and 0-1 --
// which only the cell above and the cell below pull, both in this column --
// with m_01 of rows y-1 and y+1.  The rings keep what neighbouring columns
// read: m_s of three rows, and G_K of the other six directions with m_10,
// m_01 of three rows.  Shared-memory traffic per cell drops from 34 loads and
// 13 stores (six of them 128-bit) to 22 loads and 9 stores, all 32-bit.  The
// arithmetic is that of the ring form (collide_math, pval_from, pair_from,
// residual_core), so both forms round identically.  A row's global loads are
// issued two rows before its values are used, so that a whole row of work
// (two barriers, a collision and a residual) and more lies between a load and
// its first use.
// ---------------------------------------------------------------------------
constexpr int REG_POST_PLANES = 8;  // G_0, G_2, G_4, G_5, G_6, G_7, m_10, m_01
__host__ __device__ constexpr int reg_post_plane(int k) { return k == 0 ? 0 : k == 2 ? 1 : k - 2; }

template <typename T>
constexpr size_t reg_smem_bytes(int W)
{
    return (size_t)3 * W * (1 + REG_POST_PLANES) * sizeof(T);
}

template <typename T, typename TC, int NT, int KIND, bool LO, bool RESTRICT, int FM>
__device__ __forceinline__ void sweep_strip_reg(const SweepArgs<T, TC> &a, int bx, int by, int TY, unsigned char *smem_raw,
                                                double (&red)[3][NT / 32])
{
    static_assert(!kind_ghosts(KIND), "the register form serves fixed V-cycle counts");
    using L = RingLayout<KIND, LO>;
    constexpr int W = NT, RV = L::RV, XV = L::XV, NE = L::NE;
    static_assert(L::EX == 0 && NE == RV - XV, "extra values follow the moments in the fetched vector");
    T *rms = reinterpret_cast<T *>(smem_raw);  // [3][W]
    T *rpost = rms + 3 * W;                     // [3][REG_POST_PLANES][W]
    auto MSR = [&](int s, int c) -> T & { return rms[s * W + c]; };
    auto PST = [&](int s, int j, int c) -> T & { return rpost[(s * REG_POST_PLANES + j) * W + c]; };

    const int nx = a.nx;
    const size_t NP = (size_t)nx * a.ny;
    const int t = threadIdx.x;
    const int x0 = bx * (W - 4), y0 = by * TY;
    const int y1 = min(y0 + TY, a.ny);
    const int x = x0 - 2 + t;
    const bool collides = t >= 1 && t < W - 1;
    const bool writes = t >= 2 && t < W - 2;

    // fetched rows (pv the next, pv2 the one after: global loads are issued two
    // rows ahead of their use); raw values of rows y, y+1, y+2
    T pv[RV], pv2[RV], A[RV], B[RV], C[RV];
    auto fetch = [&](int yy) { fetch_cell<T, TC, KIND, LO, RV, FM, true>(a, x, yy, NP, false, false, pv); };
    auto fetch2 = [&](int yy) { fetch_cell<T, TC, KIND, LO, RV, FM, true>(a, x, yy, NP, false, false, pv2); };
    auto extras = [&](const T (&v)[RV], T (&e)[NE]) {
#pragma unroll
        for (int i = 0; i < NE; i++) e[i] = v[XV + i];
    };
    // collide the row whose raw values are R (ring slot s, neighbours' m_s in
    // slots sm / sp, own m_s below / above msS / msN): post data of the
    // neighbour-read directions to the ring, the rest returned
    auto collide = [&](const T (&R)[RV], T msS, T msN, int sm, int s, int sp, T &g1, T &g3, T &my) {
        T e[NE];
        extras(R, e);
        const CollideOut<T> o = collide_math<T, TC, KIND, LO, NE>(
            a, R[0], R[1], R[2], R[3], R[4], e, MSR(s, t + 1), MSR(s, t - 1), msN, msS, MSR(sp, t + 1),
            MSR(sp, t - 1), MSR(sm, t + 1), MSR(sm, t - 1));
        PST(s, 0, t) = o.G[0];
        PST(s, 1, t) = o.G[2];
#pragma unroll
        for (int k = 4; k < 8; k++) PST(s, k - 2, t) = o.G[k];
        PST(s, 6, t) = o.mx;
        PST(s, 7, t) = o.my;
        g1 = o.G[1];
        g3 = o.G[3];
        my = o.my;
    };

    // ring slots: row r in slot (r - y0 + 2) % 3; rows y0-2 .. y0+2 first
    T msm2;  // own m_s of row y0-2
    fetch(y0 - 2);
    msm2 = pv[3];
    MSR(0, t) = pv[3];
    fetch(y0 - 1);
#pragma unroll
    for (int i = 0; i < RV; i++) A[i] = pv[i];  // row y0-1
    MSR(1, t) = pv[3];
    fetch(y0);
#pragma unroll
    for (int i = 0; i < RV; i++) B[i] = pv[i];  // row y0
    MSR(2, t) = pv[3];
    __syncthreads();
    T g1m = T(0), mym = T(0), g1c = T(0), myc = T(0), g3n, myn, g1n;
    if (collides) collide(A, msm2, B[3], 0, 1, 2, g1m, g3n, mym);  // row y0-1
    fetch(y0 + 1);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RV; i++) C[i] = pv[i];  // row y0+1
    MSR(0, t) = pv[3];
    fetch(y0 + 2);
    fetch2(y0 + 3);  // y0 + 3 <= y1 + 1: inside the window
    __syncthreads();
    if (collides) collide(B, A[3], C[3], 1, 2, 0, g1c, g3n, myc);  // row y0
    __syncthreads();
    // from here: A = row y, B = row y+1, pv = row y+2 (C is rebuilt from it)
#pragma unroll
    for (int i = 0; i < RV; i++) {
        A[i] = B[i];
        B[i] = C[i];
    }

    T rmax = T(0), gmax = T(0);
    double rsum = 0.0;
    T acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = T(0);
    const T gam = a.k_gam;
    int sa = 1, sb = 2, sc = 0;  // slots of rows y-1, y, y+1

    for (int y = y0; y < y1; y++) {
#pragma unroll
        for (int i = 0; i < RV; i++) C[i] = pv[i];  // (A) row y+2
        MSR(sa, t) = C[3];
#pragma unroll
        for (int i = 0; i < RV; i++) pv[i] = pv2[i];  // row y+3
        if (y + 3 <= y1) fetch2(y + 4);  // row y+4 is the C of iteration y+2 (the last uses row y1+1)
        __syncthreads();  // (C)
        if (collides) collide(B, A[3], C[3], sb, sc, sa, g1n, g3n, myn);  // row y+1
        __syncthreads();  // (E)
        T d[8];
#pragma unroll
        for (int k = 0; k < 8; k++) d[k] = T(0);
        if (writes) {
            T e[NE];
            extras(A, e);
            const OwnCell<T> own = own_from<T, KIND, LO, NE>(A[0], A[1], A[2], A[3], A[4], e);
            const T tx = own.tx, ty = own.ty, tlx = own.tlx, tly = own.tly;
            // the eight pulls: (x - c) for direction c, rows y-1 (slot sa), y (sb), y+1 (sc)
            const PVal<T> p0 = pval_from<T, LO, 0>(PST(sb, 0, t - 1), PST(sb, 6, t - 1), T(0), tx, ty, tlx, tly);
            const PVal<T> p2 = pval_from<T, LO, 2>(PST(sb, 1, t + 1), PST(sb, 6, t + 1), T(0), tx, ty, tlx, tly);
            const PVal<T> p1 = pval_from<T, LO, 1>(g1m, T(0), mym, tx, ty, tlx, tly);
            const PVal<T> p3 = pval_from<T, LO, 3>(g3n, T(0), myn, tx, ty, tlx, tly);
            const PVal<T> p4 = pval_from<T, LO, 4>(PST(sa, 2, t - 1), PST(sa, 6, t - 1), PST(sa, 7, t - 1), tx, ty, tlx, tly);
            const PVal<T> p5 = pval_from<T, LO, 5>(PST(sa, 3, t + 1), PST(sa, 6, t + 1), PST(sa, 7, t + 1), tx, ty, tlx, tly);
            const PVal<T> p6 = pval_from<T, LO, 6>(PST(sc, 4, t + 1), PST(sc, 6, t + 1), PST(sc, 7, t + 1), tx, ty, tlx, tly);
            const PVal<T> p7 = pval_from<T, LO, 7>(PST(sc, 5, t - 1), PST(sc, 6, t - 1), PST(sc, 7, t - 1), tx, ty, tlx, tly);
            residual_core<T, KIND, LO>(own, pair_from<T, 0>(p0, p2), pair_from<T, 1>(p1, p3), pair_from<T, 2>(p4, p6),
                                       pair_from<T, 3>(p5, p7), d);
            d[5] = d[6] = d[7] = T(0);  // elided ghost moments
            if (!RESTRICT) {
                store_smoothed<T, TC, KIND, LO>(a, (size_t)y * nx + x, NP, own, d, gam);
                if (a.resmax) {
                    rmax = fmax(rmax, pop_absmax(d));
                    gmax = fmax(gmax, pop_absmax(own.g));
                    rsum += (double)pop_sumsq(d);
                }
            }
        }
        if (RESTRICT) {
            const bool odd = ((y - y0) & 1) != 0;
#pragma unroll
            for (int k = 0; k < 8; k++) acc[k] = odd ? acc[k] + d[k] : d[k];
            if (odd) {
                TC tot[8];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const TC mine = (TC)acc[k];
                    tot[k] = mine + __shfl_down_sync(0xffffffffu, mine, 1);
                }
                if (writes && (x & 1) == 0) {
                    const size_t NPc = NP >> 2;
                    const size_t cidx = (size_t)(y >> 1) * (nx >> 1) + (x >> 1);
#pragma unroll
                    for (int k = 0; k < 5; k++) a.rc[k * NPc + cidx] = tot[k];
                }
            }
        }
        // rotate: rows y, y+1, y+2 become y-1, y, y+1
#pragma unroll
        for (int i = 0; i < RV; i++) {
            A[i] = B[i];
            B[i] = C[i];
        }
        g1m = g1c;
        mym = myc;
        g1c = g1n;
        myc = myn;
        const int s_old = sa;
        sa = sb;
        sb = sc;
        sc = s_old;
    }

    if (!RESTRICT && a.resmax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        }
        const int warp = t >> 5, lane = t & 31;
        if (lane == 0) {
            red[0][warp] = (double)rmax;
            red[1][warp] = (double)gmax;
            red[2][warp] = rsum;
        }
        __syncthreads();
        if (t == 0) {
            double r0 = 0.0, g0 = 0.0, q0 = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                r0 = fmax(r0, red[0][w]);
                g0 = fmax(g0, red[1][w]);
                q0 += red[2][w];
            }
            atomicMax(&a.resmax[0], (unsigned long long)__double_as_longlong(r0));
            atomicMax(&a.resmax[1], (unsigned long long)__double_as_longlong(g0));
            atomicAdd(reinterpret_cast<double *>(&a.resmax[2]), q0);
        }
    }
}

// Whether strip (bx, by) of TY rows lies inside the grid with its whole window
// (the INT form of sweep_strip applies).
template <int W>
__device__ __forceinline__ bool sweep_strip_interior(int nx, int ny, int bx, int by, int TY)
{
    const int x0 = bx * (W - 4), y0 = by * TY, y1 = min(y0 + TY, ny);
    return x0 >= 2 && x0 + W - 3 <= nx - 1 && y0 >= 2 && y1 + 2 <= ny - 1;
}

template <typename T, typename TC, int NT, int CPT, int KIND, bool LO, bool RESTRICT, int FM>
__device__ __forceinline__ void sweep_strip_any(const SweepArgs<T, TC> &a, int bx, int by, int TY, unsigned char *smem_raw,
                                                double (&red)[3][NT / 32])
{
    static_assert(reg_smem_bytes<T>(NT) <= rows_smem_bytes<T, KIND, LO, NT * CPT>(),
                  "the register form's rings fit in the ring form's shared memory");
    if (sweep_strip_interior<NT * CPT>(a.nx, a.ny, bx, by, TY)) {
        if constexpr (CPT == 1 && !kind_ghosts(KIND))
            sweep_strip_reg<T, TC, NT, KIND, LO, RESTRICT, FM>(a, bx, by, TY, smem_raw, red);
        else
            sweep_strip<T, TC, NT, CPT, KIND, LO, RESTRICT, FM, true>(a, bx, by, TY, smem_raw, red);
    } else
        sweep_strip<T, TC, NT, CPT, KIND, LO, RESTRICT, FM, false>(a, bx, by, TY, smem_raw, red);
}

template <typename T, typename TC, int NT, int CPT, int KIND, bool LO, bool RESTRICT, int FM>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 896 / (NT * CPT) : 1) k_sweep_mom(const SweepArgs<T, TC> a, int TY)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][NT / 32];
    sweep_strip_any<T, TC, NT, CPT, KIND, LO, RESTRICT, FM>(a, blockIdx.x, blockIdx.y, TY, smem_raw, red);
}

// ---------------------------------------------------------------------------
// Tile sweep for small, latency-bound levels.  A CTA of (TX+4) x (TY+4) threads
// (rounded up to whole warps) stages its TX x TY tile and a 2-cell halo in one
// pass, collides the inner (TX+2) x (TY+2) cells and streams the tile: one
// global round trip and one pass of arithmetic per launch instead of a walk
// down a strip.  Rows of the tile are the ring slots of the strip kernel, so the
// same collision, pull and residual code runs.  Restriction sums 2 x 2 blocks
// of the tile (TX, TY even) through shared memory.
// ---------------------------------------------------------------------------
template <int TX, int TY>
struct TileShape {
    static constexpr int W = TX + 4, R = TY + 4, CELLS = W * R, NT = (CELLS + 31) / 32 * 32;
};

template <typename T, int TX, int TY, int KIND, bool LO>
constexpr size_t tile_smem_bytes()
{
    using S = TileShape<TX, TY>;
    return (size_t)S::R * RingLayout<KIND, LO>::template slot_bytes<T>(S::W) + (size_t)8 * TX * TY * sizeof(T);
}

template <typename T, typename TC, int TX, int TY, int KIND, bool LO, bool RESTRICT>
__device__ __forceinline__ void tile_body(const SweepArgs<T, TC> &a, int bx, int by, unsigned char *smem_raw,
                                          double (&red)[3][TileShape<TX, TY>::NT / 32])
{
    using L = RingLayout<KIND, LO>;
    using S = TileShape<TX, TY>;
    constexpr int W = S::W, R = S::R, RV = L::RV, NT = S::NT;
    Rings<T, W, KIND, LO> rg;  // slot = tile row
    rg.carve(smem_raw, R);
    T *dres = reinterpret_cast<T *>(smem_raw + R * L::template slot_bytes<T>(W));  // [8][TY][TX] residuals (restriction)

    const int nx = a.nx, ny = a.ny;
    const size_t NP = (size_t)nx * ny;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;
    const int tid = threadIdx.x;
    const bool live = tid < S::CELLS;
    const int c = tid % W, rrow = tid / W;  // ring column and slot
    const int x0 = bx * TX, y0 = by * TY;
    const int x = x0 - 2 + c, y = y0 - 2 + rrow;
    const bool xin = perx || (x >= 0 && x < nx);
    const bool yin = pery || (y >= 0 && y < ny);

    if (live && (perx || x < nx + 2) && (pery || y < ny + 2)) {
        T pv[RV];
        fetch_cell<T, TC, KIND, LO, RV>(a, x, y, NP, perx, pery, pv);
        store_cell<T, W, KIND, LO, RV>(rg, rrow, c, pv);
    }
    __syncthreads();
    if (live && c >= 1 && c < W - 1 && rrow >= 1 && rrow < R - 1 && xin && yin)
        collide_cell<T, TC, KIND, LO, W>(a, rg, rrow - 1, rrow, rrow + 1, c);
    __syncthreads();

    T rmax = T(0), gmax = T(0);
    double rsum = 0.0;
    const bool writes = live && c >= 2 && c < W - 2 && rrow >= 2 && rrow < R - 2 && x < nx && y < ny;
    // A warp with a wall cell among its written cells takes the wall form for
    // all of them: it then runs one form instead of both one after the other
    // (the slowest warp sets a tile's time at its barriers).  For a cell away
    // from the walls the wall form adds zero terms (exactly zero coefficients):
    // the values are the same, up to the sign of an exact zero.
    const bool wall_cell = writes && ((!perx && (x == 0 || x == nx - 1)) || (!pery && (y == 0 || y == ny - 1)));
    const bool wall = __any_sync(0xffffffffu, wall_cell);
    T d[8];
#pragma unroll
    for (int k = 0; k < 8; k++) d[k] = T(0);
    if (writes) {
        const int sl[3] = {rrow - 1, rrow, rrow + 1};
        const OwnCell<T> own = own_cell<T, W, KIND, LO>(rg, rrow, c);
        const T(&gcur)[8] = own.g;
        if (wall) residual_cell<T, TC, KIND, LO, W, true>(a, rg, x, y, sl, c, perx, pery, own, d);
        else residual_cell<T, TC, KIND, LO, W, false>(a, rg, x, y, sl, c, perx, pery, own, d);
        if (!RESTRICT) {
            store_smoothed<T, TC, KIND, LO>(a, (size_t)y * nx + x, NP, own, d, a.k_gam);
            if (a.resmax) {
                rmax = pop_absmax(d);
                gmax = pop_absmax(gcur);
                rsum = (double)pop_sumsq(d);
            }
        } else {
            const int i = (rrow - 2) * TX + (c - 2);
#pragma unroll
            for (int k = 0; k < 8; k++) dres[k * TX * TY + i] = d[k];
        }
    }
    if (RESTRICT) {
        // full-sum restriction of eq. MG:restriction over the 2 x 2 blocks of the tile
        __syncthreads();
        if (tid < (TX / 2) * (TY / 2)) {
            const int bx = tid % (TX / 2), by = tid / (TX / 2);
            const int xc = x0 / 2 + bx, yc = y0 / 2 + by;
            if (2 * xc < nx && 2 * yc < ny) {
                const size_t NPc = NP >> 2;
                const size_t cidx = (size_t)yc * (nx >> 1) + xc;
                const int i0 = (2 * by) * TX + 2 * bx;
#pragma unroll
                for (int k = 0; k < (kind_ghosts(KIND) ? 8 : 5); k++) {
                    const T *dk = dres + k * TX * TY + i0;
                    // rows first, then columns (the order of the strip kernel)
                    const TC r0 = (TC)(dk[0] + dk[TX]), r1 = (TC)(dk[1] + dk[TX + 1]);
                    a.rc[k * NPc + cidx] = r0 + r1;
                }
            }
        }
    }
    if (!RESTRICT && a.resmax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
            rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        }
        const int warp = tid >> 5, lane = tid & 31;
        if (lane == 0) {
            red[0][warp] = (double)rmax;
            red[1][warp] = (double)gmax;
            red[2][warp] = rsum;
        }
        __syncthreads();
        if (tid == 0) {
            double r0 = 0.0, g0 = 0.0, q0 = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                r0 = fmax(r0, red[0][w]);
                g0 = fmax(g0, red[1][w]);
                q0 += red[2][w];
            }
            atomicMax(&a.resmax[0], (unsigned long long)__double_as_longlong(r0));
            atomicMax(&a.resmax[1], (unsigned long long)__double_as_longlong(g0));
            atomicAdd(reinterpret_cast<double *>(&a.resmax[2]), q0);
        }
    }
}

template <typename T, typename TC, int TX, int TY, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(TileShape<TX, TY>::NT) k_sweep_tile(const SweepArgs<T, TC> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][TileShape<TX, TY>::NT / 32];
    tile_body<T, TC, TX, TY, KIND, LO, RESTRICT>(a, blockIdx.x, blockIdx.y, smem_raw, red);
}

// Tile shape per storage type: FP64 levels use small tiles, so that the few
// cells of a coarse FP64 level spread over many SMs (FP64 issue rate per SM is
// the limit there).
template <typename T> struct TileFor { static constexpr int X = 32, Y = 8; };
template <> struct TileFor<double> { static constexpr int X = 8, Y = 2; };
static_assert(TileFor<float>::X == 32 && TileFor<float>::Y == 8 && TileFor<double>::X == 8 && TileFor<double>::Y == 2,
              "tile shapes shared with the host planner (sweep_tile_shape)");

// Levels of at most this many cells use the tile sweep.
inline long sweep_tile_max_cells() { return SWEEP_TILE_CELLS; }

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
cudaError_t launch_tile(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    constexpr int TX = TileFor<T>::X, TY = TileFor<T>::Y;
    constexpr size_t smem = tile_smem_bytes<T, TX, TY, KIND, LO>();
    auto kern = k_sweep_tile<T, TC, TX, TY, KIND, LO, RESTRICT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
    kern<<<grid, TileShape<TX, TY>::NT, smem, s>>>(a);
    return cudaGetLastError();
}

// Strip sweep launch shape: SWEEP_NT threads, SWEEP_CPT cells of a row per
// thread.  Measured on the 4096^2 finest sweep (tuned strip heights; resident
// CTAs per SM from the register bound of __launch_bounds__): 128 threads
// 0.288 ms, 160: 0.257, 192: 0.265, 224: 0.302, 256: 0.271, 320: 0.315, 384:
// 0.289 ms.
constexpr int SWEEP_NT = 160, SWEEP_CPT = 1;
static_assert(SWEEP_NT * SWEEP_CPT - 4 == SWEEP_STRIP_COLS, "strip geometry shared with the host planner");

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
struct SweepKernel {
    static constexpr size_t smem = rows_smem_bytes<T, KIND, LO, SWEEP_NT * SWEEP_CPT>();
    template <int FM>
    static constexpr auto kernel() { return k_sweep_mom<T, TC, SWEEP_NT, SWEEP_CPT, KIND, LO, RESTRICT, FM>; }
    // kernel attributes and resident CTAs per device (set up on first use); the
    // fetch forms share one shape, and the plain form's occupancy stands for all
    static int slots()
    {
        static int n = 0;
        if (!n) {
            for (auto k : {kernel<FETCH_PLAIN>(), kernel<FETCH_PROL>(), kernel<FETCH_ZERO>(), kernel<FETCH_ZPROL>()})
                if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
            int dev = 0, sms = 0, per_sm = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) return 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel<FETCH_PLAIN>(), SWEEP_NT, smem) != cudaSuccess)
                return 0;
            n = sms * (per_sm > 0 ? per_sm : 1);
        }
        return n;
    }
};

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
cudaError_t launch_rows(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    if ((long)a.nx * a.ny <= sweep_tile_max_cells()) return launch_tile<T, TC, KIND, LO, RESTRICT>(a, s);
    using SK = SweepKernel<T, TC, KIND, LO, RESTRICT>;
    const int slots = SK::slots();
    if (!slots) return cudaGetLastError() != cudaSuccess ? cudaErrorUnknown : cudaErrorInvalidConfiguration;
    int ty = a.rows > 0 ? a.rows + (a.rows & 1) : sweep_strip_rows(a.nx, a.ny, slots);
    dim3 grid((a.nx + SWEEP_STRIP_COLS - 1) / SWEEP_STRIP_COLS, (a.ny + ty - 1) / ty);
    // the fetch form is fixed per launch
    auto k = a.zero_init && a.gc ? SK::template kernel<FETCH_ZPROL>()
           : a.zero_init         ? SK::template kernel<FETCH_ZERO>()
           : a.gc                ? SK::template kernel<FETCH_PROL>()
                                 : SK::template kernel<FETCH_PLAIN>();
    k<<<grid, SWEEP_NT, SK::smem, s>>>(a, ty);
    return cudaGetLastError();
}

// Storage kind of a launch from the SWEEP_V_* flags / the arguments.
template <typename T, typename TC, template <typename, typename, int, bool, bool> class F, typename... A>
auto dispatch_kind(bool coarse, bool lo, bool rs, bool ghosts, int dev, A &&...args)
{
    const int g = ghosts ? 0 : KIND_NOGHOST;
    if constexpr (sizeof(T) == 4) {  // the deviation store: finest FP32 level, low parts, no ghost moments
        if (dev && !coarse && lo && !ghosts) {
            if (dev == 1)
                return rs ? F<T, TC, KIND_FINE | KIND_NOGHOST | KIND_DEV16, true, true>::run(args...)
                          : F<T, TC, KIND_FINE | KIND_NOGHOST | KIND_DEV16, true, false>::run(args...);
            return rs ? F<T, TC, KIND_FINE | KIND_NOGHOST | KIND_DEVBF16, true, true>::run(args...)
                      : F<T, TC, KIND_FINE | KIND_NOGHOST | KIND_DEVBF16, true, false>::run(args...);
        }
    }
    if (coarse) {
        if constexpr (sizeof(T) == 4) {
            if (lo) {
                if (g) return rs ? F<T, TC, KIND_COARSE | KIND_NOGHOST, true, true>::run(args...) : F<T, TC, KIND_COARSE | KIND_NOGHOST, true, false>::run(args...);
                return rs ? F<T, TC, KIND_COARSE, true, true>::run(args...) : F<T, TC, KIND_COARSE, true, false>::run(args...);
            }
        }
        if (g) return rs ? F<T, TC, KIND_COARSE | KIND_NOGHOST, false, true>::run(args...) : F<T, TC, KIND_COARSE | KIND_NOGHOST, false, false>::run(args...);
        return rs ? F<T, TC, KIND_COARSE, false, true>::run(args...) : F<T, TC, KIND_COARSE, false, false>::run(args...);
    }
    if constexpr (sizeof(T) == 4) {  // double-float low parts exist only with FP32 storage
        if (lo) {
            if (g) return rs ? F<T, TC, KIND_FINE | KIND_NOGHOST, true, true>::run(args...) : F<T, TC, KIND_FINE | KIND_NOGHOST, true, false>::run(args...);
            return rs ? F<T, TC, KIND_FINE, true, true>::run(args...) : F<T, TC, KIND_FINE, true, false>::run(args...);
        }
    }
    if (g) return rs ? F<T, TC, KIND_FINE | KIND_NOGHOST, false, true>::run(args...) : F<T, TC, KIND_FINE | KIND_NOGHOST, false, false>::run(args...);
    return rs ? F<T, TC, KIND_FINE, false, true>::run(args...) : F<T, TC, KIND_FINE, false, false>::run(args...);
}

template <typename T, typename TC, int KIND, bool LO, bool RS>
struct RowsRun {
    static cudaError_t run(const SweepArgs<T, TC> &a, cudaStream_t s) { return launch_rows<T, TC, KIND, LO, RS>(a, s); }
};
template <typename T, typename TC, int KIND, bool LO, bool RS>
struct StripSlotsRun {
    static int run() { return SweepKernel<T, TC, KIND, LO, RS>::slots(); }
};

template <typename T, typename TC>
int sweep_strip_slots_impl(int v)
{
    return dispatch_kind<T, TC, StripSlotsRun>(v & SWEEP_V_COARSE, v & SWEEP_V_LO, v & SWEEP_V_RESTRICT,
                                               !(v & SWEEP_V_NOGHOST),
                                               (v & SWEEP_V_DEV16) ? 1 : (v & SWEEP_V_DEVBF16) ? 2 : 0);
}

// Level kind from the arguments: F~ present = finest level; low parts only
// with FP32 storage on the finest level.
template <typename T, typename TC>
cudaError_t launch_sweep_mom_impl(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    return dispatch_kind<T, TC, RowsRun>(a.Ft == nullptr, a.glo != nullptr, a.mode == SWEEP_RESTRICT, a.ghosts != 0,
                                         a.dev, a, s);
}

}  // namespace biot
