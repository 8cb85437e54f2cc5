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
// The rings are planes of 4-vectors (one 128-bit shared-memory access per
// group of four values of a cell; consecutive threads read consecutive
// vectors, so the accesses are free of bank conflicts).
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
enum { KIND_FINE = 0, KIND_COARSE = 1, KIND_NOGHOST = 2 };
__host__ __device__ constexpr bool kind_fine(int k) { return (k & 1) == 0; }
__host__ __device__ constexpr bool kind_ghosts(int k) { return (k & KIND_NOGHOST) == 0; }

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
    // raw values of a cell: v0..v7 the 8 moments; FINE: v8, v9 F~, v10, v11 the
    // low parts of m_10, m_01 (LO); COARSE: v8..v12 r_0..r_4, v13, v14 the low
    // parts (LO).
    static constexpr int XV = 8;
    static constexpr int LOV = kind_fine(KIND) ? 10 : 13;
    static constexpr int RV = kind_fine(KIND) ? 12 : (LO ? 15 : 13);  // values fetched per cell
    // In shared memory m_s (v3, read by the neighbours' F_* stencil) has a
    // plane of its own; the other values of a cell, used only by the thread of
    // its column, are packed into 4-vectors:
    //   q0 = (m_10, m_01, m_11, m_d), q1 = (m_12, m_21, m_22, v8),
    //   q2 = (v9, v10, v11, v12 or 0), q3 = (v13, v14, 0, 0) (COARSE with LO).
    static constexpr int NQ = (!kind_fine(KIND) && LO) ? 4 : 3;
};

template <typename T, int KIND, bool LO, int NT>
constexpr size_t rows_smem_bytes()
{
    // raw: m_s plane + NQ vector planes; post: 4 planes S*_p + 1 vector plane
    // (m_10, m_01, F_x, F_y) + (LO) a 2-vector plane of low parts; 3 slots each
    return (size_t)3 * NT *
           (sizeof(T) + RingLayout<KIND, LO>::NQ * sizeof(V4<T>) + 4 * sizeof(T) + sizeof(V4<T>) + (LO ? sizeof(V2<T>) : 0));
}

template <typename T>
struct PVal {
    T sig, bx, by;  // value = sig + bx * m_10(x) + by * m_01(x)
};

// Post-collision data a pull reads from its source cell.
template <typename T>
struct PostSrc {
    T S;           // even part S*_p of the pulled population's pair
    T mx, my;      // first moments (high parts with LO)
    T Fx, Fy;      // force of the collision
    T lx, ly;      // low parts of the first moments (LO), else 0
};

// Shared-memory rings of W columns and 3 slots.  Scalar planes are read by
// neighbouring threads (consecutive threads, consecutive words); vector planes
// by the thread of the column or as a whole 4-vector.
template <typename T, int W, int KIND, bool LO>
struct Rings {
    using L = RingLayout<KIND, LO>;
    T *rms;        // [3][W]     m_s
    V4<T> *raw4;   // [3][NQ][W]  q0, q1, q2 (, q3)
    T *postS;      // [3][4][W]  S*_0..3
    V4<T> *post4;  // [3][W]     (m_10, m_01, F_x, F_y)
    V2<T> *post2;  // [3][W]     low parts of m_10, m_01 (LO)
    __device__ __forceinline__ V4<T> &R4(int s, int q, int c) const { return raw4[(s * L::NQ + q) * W + c]; }
    // low parts of the first moments of the raw cell (LO)
    __device__ __forceinline__ V2<T> lo(int s, int c) const
    {
        if (kind_fine(KIND)) {
            const V4<T> q = R4(s, 2, c);
            return V2<T>{q.y, q.z};
        }
        const V4<T> q = R4(s, 3, c);
        return V2<T>{q.x, q.y};
    }
    __device__ __forceinline__ T &ms(int s, int c) const { return rms[s * W + c]; }
    __device__ __forceinline__ T &PS(int s, int p, int c) const { return postS[(s * 4 + p) * W + c]; }
    __device__ __forceinline__ V4<T> &P4(int s, int c) const { return post4[s * W + c]; }
    __device__ __forceinline__ V2<T> &P2(int s, int c) const { return post2[s * W + c]; }
    template <int PAIR>
    __device__ __forceinline__ PostSrc<T> src(int s, int c) const
    {
        PostSrc<T> o;
        o.S = PS(s, PAIR, c);
        const V4<T> q = P4(s, c);
        o.mx = q.x;
        o.my = q.y;
        o.Fx = q.z;
        o.Fy = q.w;
        if (LO) {
            const V2<T> l = P2(s, c);
            o.lx = l.x;
            o.ly = l.y;
        } else {
            o.lx = T(0);
            o.ly = T(0);
        }
        return o;
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

// Raw values of cell (gx, gy): moments of the iterate (+ prolongated coarse
// correction; with LO its first moments go to the low parts), F~ (FINE) or r
// (COARSE), low parts (LO).  Ghost cells of a non-periodic wall read the
// adjacent cell: only their m_s is used (even extension of the divergence).
template <typename T, typename TC, int KIND, bool LO, int RV>
__device__ __forceinline__ void fetch_cell(const SweepArgs<T, TC> &a, int gx, int gy, size_t NP, bool perx, bool pery,
                                           T (&v)[RV])
{
    using L = RingLayout<KIND, LO>;
    if (perx) gx = wrapi(gx, a.nx);
    if (pery) gy = wrapi(gy, a.ny);
    gx = clampi(gx, a.nx);
    gy = clampi(gy, a.ny);
    const size_t idx = (size_t)gy * a.nx + gx;
    constexpr int NM = kind_ghosts(KIND) ? 8 : 5;  // moment planes loaded
    if (a.zero_init) {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = T(0);
    } else {
        const T *g = a.g + idx;
#pragma unroll
        for (int k = 0; k < NM; k++) v[k] = g[k * NP];
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
    if (LO) {
        v[L::LOV] = a.zero_init ? T(0) : a.glo[idx];
        v[L::LOV + 1] = a.zero_init ? T(0) : a.glo[NP + idx];
    } else if (kind_fine(KIND)) {
        v[L::LOV] = T(0);
        v[L::LOV + 1] = T(0);
    }
    if (a.gc) {
        const size_t NPc = NP >> 2;
        const size_t cidx = (size_t)(gy >> 1) * (a.nx >> 1) + (gx >> 1);
        if (LO) {
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
    rg.ms(s, c) = v[3];
    rg.R4(s, 0, c) = V4<T>{v[0], v[1], v[2], v[4]};
    rg.R4(s, 1, c) = V4<T>{v[5], v[6], v[7], v[8]};
    rg.R4(s, 2, c) = V4<T>{v[9], v[10], v[11], RV > 12 ? v[12] : T(0)};
    if (RingLayout<KIND, LO>::NQ > 3) rg.R4(s, 3, c) = V4<T>{v[RV > 14 ? 13 : 0], v[RV > 14 ? 14 : 0], T(0), T(0)};
}

// Collision of the cell in raw slot s, column c (Alg. 2, first six lines, in
// moment space): even moments relaxed (Tab. moments, eq. moments:collision:22),
// odd part kept as first moments + force F = F~ + (alpha^2 r/2) grad^c D(g).
template <typename T, typename TC, int KIND, bool LO, int W>
__device__ __forceinline__ void collide_cell(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int sm, int s,
                                             int sp, int c)
{
    const V4<T> q0 = rg.R4(s, 0, c), q1 = rg.R4(s, 1, c), q2 = rg.R4(s, 2, c);
    T m0 = q0.x, m1 = q0.y, m2 = q0.z, m3 = rg.ms(s, c), m4 = q0.w;
    const T dE = rg.ms(s, c + 1), dW = rg.ms(s, c - 1), dN = rg.ms(sp, c), dS = rg.ms(sm, c);
    const T dNE = rg.ms(sp, c + 1), dNW = rg.ms(sp, c - 1), dSE = rg.ms(sm, c + 1), dSW = rg.ms(sm, c - 1);
    const T cf = a.k_fs;  // alpha^2 r/2 * dD/dm_s
    T Fx = cf * ((dE - dW) * T(1.0 / 3.0) + ((dNE + dSE) - (dNW + dSW)) * T(1.0 / 12.0));
    T Fy = cf * ((dN - dS) * T(1.0 / 3.0) + ((dNE + dNW) - (dSE + dSW)) * T(1.0 / 12.0));
    if (kind_fine(KIND)) {
        Fx += q1.w;  // F~
        Fy += q2.x;
    } else {           // minus the residual right-hand side r_0..r_4
        if (!LO) {
            m0 -= q1.w;
            m1 -= q2.x;
        }  // (with LO, r_0 and r_1 come off the low parts below)
        m2 -= q2.y;
        m3 -= q2.z;
        m4 -= q2.w;
    }
    const T ms = a.k_ws * m3, md = a.k_wd * m4, m11 = a.k_wd * m2, m22 = a.k_22 * m3;
    rg.PS(s, 0, c) = T(0.5) * (ms + md) - m22;
    rg.PS(s, 1, c) = T(0.5) * (ms - md) - m22;
    rg.PS(s, 2, c) = T(0.5) * (m11 + m22);
    rg.PS(s, 3, c) = T(0.5) * (m22 - m11);
    rg.P4(s, c) = V4<T>{m0, m1, Fx, Fy};
    if (LO) {
        if (kind_fine(KIND)) {
            rg.P2(s, c) = V2<T>{q2.y, q2.z};
        } else {
            const V4<T> q3 = rg.R4(s, 3, c);
            rg.P2(s, c) = V2<T>{q3.x - q1.w, q3.y - q2.x};
        }
    }
}

// Post-collision population K of a source cell, split relative to the target's
// collision-input first moments (tx, ty high, tlx, tly low parts):
//   g*_K = 1/2 (S*_p + e A*_p),  A*_p = a_p . m + b_p . F  (Tab. moments:inverse)
template <typename T, bool LO, int K>
__device__ __forceinline__ PVal<T> post_pop(const PostSrc<T> &q, T tx, T ty, T tlx, T tly)
{
    constexpr int p = pair_of(K);
    constexpr T e = T(sign_of(K));
    T dmx = q.mx - tx, dmy = q.my - ty;
    if (LO) {
        dmx += q.lx - tlx;
        dmy += q.ly - tly;
    }
    const T odd = (T(pa_x(p)) * dmx + T(pa_y(p)) * dmy) + (T(pb_x(p)) * q.Fx + T(pb_y(p)) * q.Fy);
    PVal<T> v;
    v.sig = T(0.5) * (q.S + e * odd);
    v.bx = e * T(0.5 * pa_x(p));
    v.by = e * T(0.5 * pa_y(p));
    return v;
}

template <typename T, bool LO, int W, int KIND, int K>
__device__ __forceinline__ PVal<T> post_at(const Rings<T, W, KIND, LO> &rg, int s, int c, T tx, T ty, T tlx, T tly)
{
    return post_pop<T, LO, K>(rg.template src<pair_of(K)>(s, c), tx, ty, tlx, tly);
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
        v.sig = -o.sig;
        v.bx = -o.bx;
        v.by = -o.by;
        if (kind_fine(KIND) && a.prof[side]) v.sig += T(a.c0h * traction_term(a.prof[side], side, n, x, y, cx, cy));
        return v;
    }
    // BC_DIRICHLET: eq. BC:elasticity, history = previous call's outgoing population
    if (a.hist_valid) {
        v.sig = a.H[side][3 * (horiz ? x : y) + hslot(side, kout)];
        v.bx = T(0);
        v.by = T(0);
    } else {
        v = o;
    }
    if (kind_fine(KIND) && a.prof[side]) v.sig += T(dirichlet_term(a.prof[side], side, n, x, y, cx, cy));
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

template <typename T, typename TC, int KIND, bool LO, int W, int P, bool WALL>
__device__ __forceinline__ PairOut<T> pull_pair(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int x, int y,
                                                const int (&sl)[3], int c0, T tx, T ty, T tlx, T tly, bool perx, bool pery)
{
    const PVal<T> u = pull<T, TC, KIND, LO, W, pair_first(P), WALL>(a, rg, x, y, sl, c0, tx, ty, tlx, tly, perx, pery);
    const PVal<T> v = pull<T, TC, KIND, LO, W, pair_second(P), WALL>(a, rg, x, y, sl, c0, tx, ty, tlx, tly, perx, pery);
    PairOut<T> o;
    o.Ss = u.sig + v.sig;
    o.As = u.sig - v.sig;
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
    a.H[side][3 * pos + hslot(side, K)] = o.sig + (o.bx * (tx + tlx) + o.by * (ty + tly));
}

// Residual d = m - m** of the cell (x, y) (small parts only, see the file
// comment); gcur: the iterate's moments.
template <typename T, typename TC, int KIND, bool LO, int W, bool WALL>
__device__ __forceinline__ void residual_cell(const SweepArgs<T, TC> &a, const Rings<T, W, KIND, LO> &rg, int x, int y,
                                              const int (&sl)[3], int c0, bool perx, bool pery, const T (&gcur)[8],
                                              T (&d)[8])
{
    const int s0 = sl[1];
    const V4<T> own = rg.P4(s0, c0);
    const T tx = own.x, ty = own.y;
    T tlx = T(0), tly = T(0);
    if (LO) {
        const V2<T> l = rg.P2(s0, c0);
        tlx = l.x;
        tly = l.y;
    }
#define BIOT_PAIR(P) pull_pair<T, TC, KIND, LO, W, P, WALL>(a, rg, x, y, sl, c0, tx, ty, tlx, tly, perx, pery)
    const PairOut<T> P0 = BIOT_PAIR(0), P1 = BIOT_PAIR(1), P2 = BIOT_PAIR(2), P3 = BIOT_PAIR(3);
#undef BIOT_PAIR
    const T mxf = tx + tlx, myf = ty + tly;  // full first moments: beta terms (walls) and the m_12, m_21 residuals
    // odd moments: m**_10 = (A0 + A2 - A3) = small + m_10(x) + dB-terms, etc.
    // (sum_p c_p a_p = (1,0), (0,1), (1/3,0), (0,1/3) for 10, 01, 12, 21)
    // residual rhs r_0, r_1 on coarse levels (0 on the finest): the iterate minus
    // the collision input, high and low parts differenced separately
    T r0 = gcur[0] - tx, r1 = gcur[1] - ty;
    if (LO && !kind_fine(KIND)) {
        const V2<T> gl = rg.lo(s0, c0);
        r0 += gl.x - tlx;
        r1 += gl.y - tly;
    }
    d[0] = r0 - ((P0.As + P2.As) - P3.As);
    d[1] = r1 - ((P1.As + P2.As) + P3.As);
    d[5] = (gcur[5] - mxf * T(1.0 / 3.0)) - (P2.As - P3.As);
    d[6] = (gcur[6] - myf * T(1.0 / 3.0)) - (P2.As + P3.As);
    d[2] = gcur[2] - (P2.Ss - P3.Ss);
    d[3] = gcur[3] - ((P0.Ss + P1.Ss) + T(2) * (P2.Ss + P3.Ss));
    d[4] = gcur[4] - (P0.Ss - P1.Ss);
    d[7] = gcur[7] - (P2.Ss + P3.Ss);
    constexpr bool GH = kind_ghosts(KIND);
    if (WALL) {
        d[0] -= ((P0.dbx + P2.dbx) - P3.dbx) * mxf + ((P0.dby + P2.dby) - P3.dby) * myf;
        d[1] -= ((P1.dbx + P2.dbx) + P3.dbx) * mxf + ((P1.dby + P2.dby) + P3.dby) * myf;
        d[5] -= (P2.dbx - P3.dbx) * mxf + (P2.dby - P3.dby) * myf;
        d[6] -= (P2.dbx + P3.dbx) * mxf + (P2.dby + P3.dby) * myf;
        d[2] -= (P2.bsx - P3.bsx) * mxf + (P2.bsy - P3.bsy) * myf;
        d[3] -= ((P0.bsx + P1.bsx) + T(2) * (P2.bsx + P3.bsx)) * mxf + ((P0.bsy + P1.bsy) + T(2) * (P2.bsy + P3.bsy)) * myf;
        d[4] -= (P0.bsx - P1.bsx) * mxf + (P0.bsy - P1.bsy) * myf;
        d[7] -= (P2.bsx + P3.bsx) * mxf + (P2.bsy + P3.bsy) * myf;
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

// One strip (column block bx, row block by of TY rows) of one sweep; the body
// of both the single-instance kernel and the batched work-list kernel.
template <typename T, typename TC, int NT, int KIND, bool LO, bool RESTRICT>
__device__ __forceinline__ void sweep_strip(const SweepArgs<T, TC> &a, int bx, int by, int TY, unsigned char *smem_raw,
                                            double (&red)[2][NT / 32])
{
    using L = RingLayout<KIND, LO>;
    constexpr int W = NT, RV = L::RV;
    Rings<T, W, KIND, LO> rg;
    rg.raw4 = reinterpret_cast<V4<T> *>(smem_raw);   // vectors first (alignment)
    rg.post4 = rg.raw4 + 3 * L::NQ * W;
    rg.post2 = reinterpret_cast<V2<T> *>(rg.post4 + 3 * W);
    rg.rms = reinterpret_cast<T *>(rg.post2 + (LO ? 3 * W : 0));
    rg.postS = rg.rms + 3 * W;

    const int nx = a.nx, ny = a.ny;
    const size_t NP = (size_t)nx * ny;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;
    const int t = threadIdx.x;
    const int x0 = bx * (NT - 4), y0 = by * TY;
    const int y1 = min(y0 + TY, ny);

    const int x = x0 - 2 + t;  // this thread's column (ring column t)
    const bool loads = perx || x < nx + 2;                           // a real, wrapped or ghost column
    const bool collides = t >= 1 && t < NT - 1 && (perx || (x >= 0 && x < nx));
    const bool writes = t >= 2 && t < NT - 2 && x < nx;
    const bool wall_col = !perx && (x == 0 || x == nx - 1);

    auto row_ok = [&](int y) { return pery || (y >= 0 && y < ny); };

    T pv[RV];
    auto fetch_row = [&](int y) {
        if (loads) fetch_cell<T, TC, KIND, LO, RV>(a, x, y, NP, perx, pery, pv);
    };
    auto store_row = [&](int s) {
        if (loads) store_cell<T, W, KIND, LO, RV>(rg, s, t, pv);
    };
    auto collide_row = [&](int y, int sm, int s, int sp) {
        if (collides && row_ok(y)) collide_cell<T, TC, KIND, LO, W>(a, rg, sm, s, sp, t);
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
    T acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = T(0);
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
        T d[8];
#pragma unroll
        for (int k = 0; k < 8; k++) d[k] = T(0);
        if (writes) {
            const V4<T> g0 = rg.R4(sb, 0, t), g1 = rg.R4(sb, 1, t);
            const T gcur[8] = {g0.x, g0.y, g0.z, rg.ms(sb, t), g0.w, g1.x, g1.y, g1.z};
            const bool wall = wall_col || (!pery && (y == 0 || y == ny - 1));
            if (wall) residual_cell<T, TC, KIND, LO, W, true>(a, rg, x, y, sl, t, perx, pery, gcur, d);
            else residual_cell<T, TC, KIND, LO, W, false>(a, rg, x, y, sl, t, perx, pery, gcur, d);
            if (!RESTRICT) {
                const size_t idx = (size_t)y * nx + x;
                T *go = a.gout + idx;
#pragma unroll
                for (int k = 2; k < (kind_ghosts(KIND) ? 8 : 5); k++) go[k * NP] = gcur[k] - gam * d[k];
                // first moments: (hi + lo) - gamma d, renormalised into hi + lo with LO
                if (LO) {
                    const V2<T> gl = rg.lo(sb, t);
                    const T lo[2] = {gl.x, gl.y};
#pragma unroll
                    for (int k = 0; k < 2; k++) {
                        T hi, lw;
                        two_sum(gcur[k], lo[k] - gam * d[k], hi, lw);
                        go[k * NP] = hi;
                        a.glo_out[k * NP + idx] = lw;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 2; k++) go[k * NP] = gcur[k] - gam * d[k];
                }
                if (a.resmax) {
                    rmax = fmax(rmax, pop_absmax(d));
                    gmax = fmax(gmax, pop_absmax(gcur));
                }
            }
        }
        if (RESTRICT) {
            // full-sum restriction of eq. MG:restriction: pair rows, then columns
            // (columns x, x+1 with x even sit in lanes t, t+1 of one warp)
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
                    for (int k = 0; k < (kind_ghosts(KIND) ? 8 : 5); k++) a.rc[k * NPc + cidx] = tot[k];
                }
            }
        }
        const int s_old = sa;  // rotate: rows y, y+1, y+2 become y-1, y, y+1
        sa = sb;
        sb = sc;
        sc = s_old;
    }

    if (!RESTRICT && a.resmax) {
        // warp-shuffle then block reduction of the two maxima, one atomic per CTA
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
        }
        const int warp = t >> 5, lane = t & 31;
        if (lane == 0) {
            red[0][warp] = (double)rmax;
            red[1][warp] = (double)gmax;
        }
        __syncthreads();
        if (t == 0) {
            double r0 = 0.0, g0 = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                r0 = fmax(r0, red[0][w]);
                g0 = fmax(g0, red[1][w]);
            }
            atomicMax(&a.resmax[0], (unsigned long long)__double_as_longlong(r0));
            atomicMax(&a.resmax[1], (unsigned long long)__double_as_longlong(g0));
        }
    }
}

template <typename T, typename TC, int NT, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 6 : 1) k_sweep_mom(const SweepArgs<T, TC> a, int TY)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2][NT / 32];
    sweep_strip<T, TC, NT, KIND, LO, RESTRICT>(a, blockIdx.x, blockIdx.y, TY, smem_raw, red);
}

// Batched form: CTA b processes work item items[b], a strip of the sweep
// described by jobs[items[b].job] (the jobs of one launch may belong to
// different instances and different multigrid levels of one storage kind).
template <typename T, typename TC, int NT, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 6 : 1)
    k_sweep_batch(const SweepArgs<T, TC> *__restrict__ jobs, const SweepItem *__restrict__ items)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2][NT / 32];
    __shared__ SweepArgs<T, TC> sa;
    const SweepItem it = items[blockIdx.x];
    if (threadIdx.x == 0) sa = jobs[it.job];
    __syncthreads();
    sweep_strip<T, TC, NT, KIND, LO, RESTRICT>(sa, it.bx, it.by, it.ty, smem_raw, red);
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
    return (size_t)S::R * S::W *
               (sizeof(T) + RingLayout<KIND, LO>::NQ * sizeof(V4<T>) + 4 * sizeof(T) + sizeof(V4<T>) + (LO ? sizeof(V2<T>) : 0)) +
           (size_t)8 * TX * TY * sizeof(T);
}

template <typename T, typename TC, int TX, int TY, int KIND, bool LO, bool RESTRICT>
__device__ __forceinline__ void tile_body(const SweepArgs<T, TC> &a, int bx, int by, unsigned char *smem_raw,
                                          double (&red)[2][TileShape<TX, TY>::NT / 32])
{
    using L = RingLayout<KIND, LO>;
    using S = TileShape<TX, TY>;
    constexpr int W = S::W, R = S::R, RV = L::RV, NT = S::NT;
    Rings<T, W, KIND, LO> rg;  // slot = tile row
    rg.raw4 = reinterpret_cast<V4<T> *>(smem_raw);
    rg.post4 = rg.raw4 + R * L::NQ * W;
    rg.post2 = reinterpret_cast<V2<T> *>(rg.post4 + R * W);
    rg.rms = reinterpret_cast<T *>(rg.post2 + (LO ? R * W : 0));
    rg.postS = rg.rms + R * W;
    T *dres = rg.postS + R * 4 * W;  // [8][TY][TX] residuals (restriction)

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
    const bool writes = live && c >= 2 && c < W - 2 && rrow >= 2 && rrow < R - 2 && x < nx && y < ny;
    T d[8];
#pragma unroll
    for (int k = 0; k < 8; k++) d[k] = T(0);
    if (writes) {
        const int sl[3] = {rrow - 1, rrow, rrow + 1};
        const V4<T> g0 = rg.R4(rrow, 0, c), g1 = rg.R4(rrow, 1, c);
        const T gcur[8] = {g0.x, g0.y, g0.z, rg.ms(rrow, c), g0.w, g1.x, g1.y, g1.z};
        const bool wall = (!perx && (x == 0 || x == nx - 1)) || (!pery && (y == 0 || y == ny - 1));
        if (wall) residual_cell<T, TC, KIND, LO, W, true>(a, rg, x, y, sl, c, perx, pery, gcur, d);
        else residual_cell<T, TC, KIND, LO, W, false>(a, rg, x, y, sl, c, perx, pery, gcur, d);
        if (!RESTRICT) {
            const size_t idx = (size_t)y * nx + x;
            T *go = a.gout + idx;
            const T gam = a.k_gam;
#pragma unroll
            for (int k = 2; k < (kind_ghosts(KIND) ? 8 : 5); k++) go[k * NP] = gcur[k] - gam * d[k];
            if (LO) {
                const V2<T> gl = rg.lo(rrow, c);
                const T lo[2] = {gl.x, gl.y};
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    T hi, lw;
                    two_sum(gcur[k], lo[k] - gam * d[k], hi, lw);
                    go[k * NP] = hi;
                    a.glo_out[k * NP + idx] = lw;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 2; k++) go[k * NP] = gcur[k] - gam * d[k];
            }
            if (a.resmax) {
                rmax = pop_absmax(d);
                gmax = pop_absmax(gcur);
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
        }
        const int warp = tid >> 5, lane = tid & 31;
        if (lane == 0) {
            red[0][warp] = (double)rmax;
            red[1][warp] = (double)gmax;
        }
        __syncthreads();
        if (tid == 0) {
            double r0 = 0.0, g0 = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                r0 = fmax(r0, red[0][w]);
                g0 = fmax(g0, red[1][w]);
            }
            atomicMax(&a.resmax[0], (unsigned long long)__double_as_longlong(r0));
            atomicMax(&a.resmax[1], (unsigned long long)__double_as_longlong(g0));
        }
    }
}

template <typename T, typename TC, int TX, int TY, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(TileShape<TX, TY>::NT) k_sweep_tile(const SweepArgs<T, TC> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2][TileShape<TX, TY>::NT / 32];
    tile_body<T, TC, TX, TY, KIND, LO, RESTRICT>(a, blockIdx.x, blockIdx.y, smem_raw, red);
}

// Batched form: CTA b processes tile (items[b].bx, items[b].by) of the sweep
// jobs[items[b].job] (items[b].ty is unused).
template <typename T, typename TC, int TX, int TY, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(TileShape<TX, TY>::NT)
    k_sweep_tile_batch(const SweepArgs<T, TC> *__restrict__ jobs, const SweepItem *__restrict__ items)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2][TileShape<TX, TY>::NT / 32];
    __shared__ SweepArgs<T, TC> sa;
    const SweepItem it = items[blockIdx.x];
    if (threadIdx.x == 0) sa = jobs[it.job];
    __syncthreads();
    tile_body<T, TC, TX, TY, KIND, LO, RESTRICT>(sa, it.bx, it.by, smem_raw, red);
}

// Tile shape per storage type: FP64 levels use small tiles, so that the few
// cells of a coarse FP64 level spread over many SMs (FP64 issue rate per SM is
// the limit there).
template <typename T> struct TileFor { static constexpr int X = 32, Y = 8; };
template <> struct TileFor<double> { static constexpr int X = 8, Y = 2; };
static_assert(TileFor<float>::X == 32 && TileFor<float>::Y == 8 && TileFor<double>::X == 8 && TileFor<double>::Y == 2,
              "tile shapes shared with the host planner (sweep_tile_shape)");

// Levels of at most this many cells use the tile sweep (default 256^2; the
// environment variable BIOT_SWEEP_TILE_MAX_CELLS overrides it, 0 disables).
inline long sweep_tile_max_cells()
{
    static long v = -1;
    if (v < 0) {
        const char *e = getenv("BIOT_SWEEP_TILE_MAX_CELLS");
        v = e ? atol(e) : SWEEP_TILE_CELLS;
        if (v < 0) v = 0;
    }
    return v;
}

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

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
cudaError_t launch_tile_batch(const SweepArgs<T, TC> *jobs, const SweepItem *items, int n, cudaStream_t s)
{
    constexpr int TX = TileFor<T>::X, TY = TileFor<T>::Y;
    constexpr size_t smem = tile_smem_bytes<T, TX, TY, KIND, LO>();
    auto kern = k_sweep_tile_batch<T, TC, TX, TY, KIND, LO, RESTRICT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (n <= 0) return cudaSuccess;
    kern<<<n, TileShape<TX, TY>::NT, smem, s>>>(jobs, items);
    return cudaGetLastError();
}

constexpr int SWEEP_NT = 128;
static_assert(SWEEP_NT - 4 == SWEEP_STRIP_COLS, "strip geometry shared with the host planner");

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
struct SweepKernel {
    static constexpr size_t smem = rows_smem_bytes<T, KIND, LO, SWEEP_NT>();
    // kernel attributes and resident CTAs per device (set up on first use)
    static int slots()
    {
        static int n = 0;
        if (!n) {
            auto k1 = k_sweep_mom<T, TC, SWEEP_NT, KIND, LO, RESTRICT>;
            auto k2 = k_sweep_batch<T, TC, SWEEP_NT, KIND, LO, RESTRICT>;
            if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
            if (cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
            int dev = 0, sms = 0, per_sm = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) return 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2, SWEEP_NT, smem) != cudaSuccess) return 0;
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
    dim3 grid((a.nx + SWEEP_NT - 5) / (SWEEP_NT - 4), (a.ny + ty - 1) / ty);
    k_sweep_mom<T, TC, SWEEP_NT, KIND, LO, RESTRICT><<<grid, SWEEP_NT, SK::smem, s>>>(a, ty);
    return cudaGetLastError();
}

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
cudaError_t launch_batch_v(const SweepArgs<T, TC> *jobs, const SweepItem *items, int n, cudaStream_t s)
{
    using SK = SweepKernel<T, TC, KIND, LO, RESTRICT>;
    if (n <= 0) return cudaSuccess;
    if (!SK::slots()) return cudaErrorInvalidConfiguration;
    k_sweep_batch<T, TC, SWEEP_NT, KIND, LO, RESTRICT><<<n, SWEEP_NT, SK::smem, s>>>(jobs, items);
    return cudaGetLastError();
}

// Storage kind of a launch from the SWEEP_V_* flags / the arguments.
template <typename T, typename TC, template <typename, typename, int, bool, bool> class F, typename... A>
auto dispatch_kind(bool coarse, bool lo, bool rs, bool ghosts, A &&...args)
{
    const int g = ghosts ? 0 : KIND_NOGHOST;
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
struct BatchRun {
    static cudaError_t run(bool tile, const SweepArgs<T, TC> *jobs, const SweepItem *items, int n, cudaStream_t s)
    {
        return tile ? launch_tile_batch<T, TC, KIND, LO, RS>(jobs, items, n, s)
                    : launch_batch_v<T, TC, KIND, LO, RS>(jobs, items, n, s);
    }
};
template <typename T, typename TC, int KIND, bool LO, bool RS>
struct SlotsRun {
    static int run() { return SweepKernel<T, TC, KIND, LO, RS>::slots(); }
};
template <typename T, typename TC, int KIND, bool LO, bool RS>
struct RowsRun {
    static cudaError_t run(const SweepArgs<T, TC> &a, cudaStream_t s) { return launch_rows<T, TC, KIND, LO, RS>(a, s); }
};

template <typename T, typename TC>
cudaError_t launch_sweep_batch_impl(int v, const SweepArgs<T, TC> *jobs, const SweepItem *items, int n, cudaStream_t s)
{
    return dispatch_kind<T, TC, BatchRun>(v & SWEEP_V_COARSE, v & SWEEP_V_LO, v & SWEEP_V_RESTRICT,
                                         !(v & SWEEP_V_NOGHOST), (v & SWEEP_V_TILE) != 0, jobs, items, n, s);
}

template <typename T, typename TC>
int sweep_slots_impl(int v)
{
    return dispatch_kind<T, TC, SlotsRun>(v & SWEEP_V_COARSE, v & SWEEP_V_LO, v & SWEEP_V_RESTRICT, !(v & SWEEP_V_NOGHOST));
}

// Level kind from the arguments: F~ present = finest level; low parts only
// with FP32 storage on the finest level.
template <typename T, typename TC>
cudaError_t launch_sweep_mom_impl(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    return dispatch_kind<T, TC, RowsRun>(a.Ft == nullptr, a.glo != nullptr, a.mode == SWEEP_RESTRICT, a.ghosts != 0, a, s);
}

}  // namespace biot
