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
// FINE: finest level (explicit force F~, boundary data; double-float first
// moments when LO).  COARSE: residual right-hand side r, homogeneous walls.
// ---------------------------------------------------------------------------
enum { KIND_FINE = 0, KIND_COARSE = 1 };

template <int KIND, bool LO>
struct RingLayout {
    // raw ring: 8 moments, then low parts (LO), then F~ (FINE) or r_0..r_4 (COARSE)
    static constexpr int LOV = 8;
    static constexpr int XV = LO ? 10 : 8;
    static constexpr int RV = XV + (KIND == KIND_FINE ? 2 : 5);
    // post ring: S*_0..3, m_10, m_01 (high), F_x, F_y, then low parts (LO)
    static constexpr int PV = LO ? 10 : 8;
};

template <typename T, int KIND, bool LO, int NT>
constexpr size_t rows_smem_bytes()
{
    return sizeof(T) * (size_t)(3 * (RingLayout<KIND, LO>::RV + RingLayout<KIND, LO>::PV) * NT);
}

template <typename T>
struct PVal {
    T sig, bx, by;  // value = sig + bx * m_10(x) + by * m_01(x)
};

// Shared-memory rings; element (slot, value, column).
template <typename T, int W, int RV, int PV>
struct Rings {
    T *raw;   // [3][RV][W]
    T *post;  // [3][PV][W]
    __device__ __forceinline__ T &R(int s, int v, int c) const { return raw[(s * RV + v) * W + c]; }
    __device__ __forceinline__ T &P(int s, int v, int c) const { return post[(s * PV + v) * W + c]; }
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
// correction; with LO its first moments go to the low parts), low parts, and
// F~ (FINE) or r (COARSE).  Ghost cells of a non-periodic wall read the
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
    if (a.zero_init) {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = T(0);
    } else {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = a.g[k * NP + idx];
    }
    if (LO) {
        v[L::LOV] = a.glo[idx];
        v[L::LOV + 1] = a.glo[NP + idx];
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
        for (int k = 2; k < 8; k++) v[k] += (T)a.gc[k * NPc + cidx];
    }
    if (KIND == KIND_FINE) {
        v[L::XV] = a.Ft[idx];
        v[L::XV + 1] = a.Ft[NP + idx];
    } else {
#pragma unroll
        for (int k = 0; k < 5; k++) v[L::XV + k] = a.r[k * NP + idx];
    }
}

// Collision of the cell in raw slot s, column c (Alg. 2, first six lines, in
// moment space): even moments relaxed (Tab. moments, eq. moments:collision:22),
// odd part kept as first moments + force F = F~ + (alpha^2 r/2) grad^c D(g).
template <typename T, typename TC, int KIND, bool LO, int W, int RV, int PV>
__device__ __forceinline__ void collide_cell(const SweepArgs<T, TC> &a, const Rings<T, W, RV, PV> &rg, int sm, int s,
                                             int sp, int c)
{
    using L = RingLayout<KIND, LO>;
    T m0 = rg.R(s, 0, c), m1 = rg.R(s, 1, c), m2 = rg.R(s, 2, c), m3 = rg.R(s, 3, c), m4 = rg.R(s, 4, c);
    const T dE = rg.R(s, 3, c + 1), dW = rg.R(s, 3, c - 1), dN = rg.R(sp, 3, c), dS = rg.R(sm, 3, c);
    const T dNE = rg.R(sp, 3, c + 1), dNW = rg.R(sp, 3, c - 1), dSE = rg.R(sm, 3, c + 1), dSW = rg.R(sm, 3, c - 1);
    const T cf = a.k_fs;  // alpha^2 r/2 * dD/dm_s
    T Fx = cf * ((dE - dW) * T(1.0 / 3.0) + ((dNE + dSE) - (dNW + dSW)) * T(1.0 / 12.0));
    T Fy = cf * ((dN - dS) * T(1.0 / 3.0) + ((dNE + dNW) - (dSE + dSW)) * T(1.0 / 12.0));
    if (KIND == KIND_FINE) {
        Fx += rg.R(s, L::XV, c);
        Fy += rg.R(s, L::XV + 1, c);
    } else {
        m0 -= rg.R(s, L::XV, c);
        m1 -= rg.R(s, L::XV + 1, c);
        m2 -= rg.R(s, L::XV + 2, c);
        m3 -= rg.R(s, L::XV + 3, c);
        m4 -= rg.R(s, L::XV + 4, c);
    }
    const T one_m_ws = a.k_ws, one_m_wd = a.k_wd;
    const T c22 = a.k_22;
    const T ms = one_m_ws * m3, md = one_m_wd * m4, m11 = one_m_wd * m2, m22 = c22 * m3;
    rg.P(s, 0, c) = T(0.5) * (ms + md) - m22;
    rg.P(s, 1, c) = T(0.5) * (ms - md) - m22;
    rg.P(s, 2, c) = T(0.5) * (m11 + m22);
    rg.P(s, 3, c) = T(0.5) * (m22 - m11);
    rg.P(s, 4, c) = m0;
    rg.P(s, 5, c) = m1;
    rg.P(s, 6, c) = Fx;
    rg.P(s, 7, c) = Fy;
    if (LO) {
        rg.P(s, 8, c) = rg.R(s, L::LOV, c);
        rg.P(s, 9, c) = rg.R(s, L::LOV + 1, c);
    }
}

// Post-collision population K of the cell in post slot s, column c, split
// relative to the target's collision-input first moments (high parts mx, my at
// slot s0, column c0; with LO the low parts are differenced alongside):
//   g*_K = 1/2 (S*_p + e A*_p),  A*_p = a_p . m + b_p . F  (Tab. moments:inverse)
template <typename T, bool LO, int W, int RV, int PV, int K>
__device__ __forceinline__ PVal<T> post_pop(const Rings<T, W, RV, PV> &rg, int s, int c, int s0, int c0, T mx, T my)
{
    constexpr int p = pair_of(K);
    constexpr T e = T(sign_of(K));
    T dmx = rg.P(s, 4, c) - mx, dmy = rg.P(s, 5, c) - my;
    if (LO) {
        dmx += rg.P(s, 8, c) - rg.P(s0, 8, c0);
        dmy += rg.P(s, 9, c) - rg.P(s0, 9, c0);
    }
    const T odd = (T(pa_x(p)) * dmx + T(pa_y(p)) * dmy) + (T(pb_x(p)) * rg.P(s, 6, c) + T(pb_y(p)) * rg.P(s, 7, c));
    PVal<T> v;
    v.sig = T(0.5) * (rg.P(s, p, c) + e * odd);
    v.bx = e * T(0.5 * pa_x(p));
    v.by = e * T(0.5 * pa_y(p));
    return v;
}

// Population of direction K arriving at cell (x, y) (ring column c0); sl[0..2]
// are the slots of rows y-1, y, y+1.
template <typename T, typename TC, int KIND, bool LO, int W, int RV, int PV, int K, bool WALL>
__device__ __forceinline__ PVal<T> pull(const SweepArgs<T, TC> &a, const Rings<T, W, RV, PV> &rg, int x, int y,
                                        const int (&sl)[3], int c0, T mx, T my, bool perx, bool pery)
{
    constexpr int cx = ex8(K), cy = ey8(K);
    const int s0 = sl[1];
    if (!WALL) return post_pop<T, LO, W, RV, PV, K>(rg, sl[1 - cy], c0 - cx, s0, c0, mx, my);
    const int sx = x - cx, sy = y - cy;
    const bool outx = !perx && (sx < 0 || sx >= a.nx);
    const bool outy = !pery && (sy < 0 || sy >= a.ny);
    if (!outx && !outy) return post_pop<T, LO, W, RV, PV, K>(rg, sl[1 - cy], c0 - cx, s0, c0, mx, my);
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
            if (outx) return post_pop<T, LO, W, RV, PV, dir8(-cx, -cy)>(rg, s0, c0, s0, c0, mx, my);
            return post_pop<T, LO, W, RV, PV, dir8(cx, -cy)>(rg, s0, c0 - cx, s0, c0, mx, my);
        }
        return post_pop<T, LO, W, RV, PV, dir8(-cx, cy)>(rg, sl[1 - cy], c0, s0, c0, mx, my);
    }
    constexpr int kout = opp8(K);
    const PVal<T> o = post_pop<T, LO, W, RV, PV, kout>(rg, s0, c0, s0, c0, mx, my);
    const bool horiz = (side == SIDE_BOTTOM || side == SIDE_TOP);
    const int n = horiz ? a.nx : a.ny;
    PVal<T> v;
    if (type == BC_NEUMANN) {  // eq. BC:traction
        v.sig = -o.sig;
        v.bx = -o.bx;
        v.by = -o.by;
        if (KIND == KIND_FINE && a.prof[side]) v.sig += T(a.c0h * traction_term(a.prof[side], side, n, x, y, cx, cy));
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
    if (KIND == KIND_FINE && a.prof[side]) v.sig += T(dirichlet_term(a.prof[side], side, n, x, y, cx, cy));
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

template <typename T, typename TC, int KIND, bool LO, int W, int RV, int PV, int P, bool WALL>
__device__ __forceinline__ PairOut<T> pull_pair(const SweepArgs<T, TC> &a, const Rings<T, W, RV, PV> &rg, int x, int y,
                                                const int (&sl)[3], int c0, T mx, T my, bool perx, bool pery)
{
    const PVal<T> u = pull<T, TC, KIND, LO, W, RV, PV, pair_first(P), WALL>(a, rg, x, y, sl, c0, mx, my, perx, pery);
    const PVal<T> v = pull<T, TC, KIND, LO, W, RV, PV, pair_second(P), WALL>(a, rg, x, y, sl, c0, mx, my, perx, pery);
    PairOut<T> o;
    o.Ss = u.sig + v.sig;
    o.As = u.sig - v.sig;
    o.bsx = u.bx + v.bx;
    o.bsy = u.by + v.by;
    o.dbx = (u.bx - v.bx) - T(pa_x(P));
    o.dby = (u.by - v.by) - T(pa_y(P));
    return o;
}

template <typename T, typename TC, bool LO, int W, int RV, int PV, int K>
__device__ __forceinline__ void store_history(const SweepArgs<T, TC> &a, const Rings<T, W, RV, PV> &rg, int side, int pos,
                                              int s0, int c0, T mx, T my)
{
    const PVal<T> o = post_pop<T, LO, W, RV, PV, K>(rg, s0, c0, s0, c0, mx, my);
    T mxf = mx, myf = my;
    if (LO) {
        mxf += rg.P(s0, 8, c0);
        myf += rg.P(s0, 9, c0);
    }
    a.H[side][3 * pos + hslot(side, K)] = o.sig + (o.bx * mxf + o.by * myf);
}

// Residual d = m - m** of the cell (x, y) (small parts only, see the file
// comment); gcur: the iterate's moments.
template <typename T, typename TC, int KIND, bool LO, int W, int RV, int PV, bool WALL>
__device__ __forceinline__ void residual_cell(const SweepArgs<T, TC> &a, const Rings<T, W, RV, PV> &rg, int x, int y,
                                              const int (&sl)[3], int c0, bool perx, bool pery, const T (&gcur)[8],
                                              T (&d)[8])
{
    const int s0 = sl[1];
    const T mx = rg.P(s0, 4, c0), my = rg.P(s0, 5, c0);
#define BIOT_PAIR(P) pull_pair<T, TC, KIND, LO, W, RV, PV, P, WALL>(a, rg, x, y, sl, c0, mx, my, perx, pery)
    const PairOut<T> P0 = BIOT_PAIR(0), P1 = BIOT_PAIR(1), P2 = BIOT_PAIR(2), P3 = BIOT_PAIR(3);
#undef BIOT_PAIR
    T mxf = mx, myf = my;  // full first moments: beta terms (walls) and the m_12, m_21 residuals
    if (LO) {
        mxf += rg.P(s0, 8, c0);
        myf += rg.P(s0, 9, c0);
    }
    // odd moments: m**_10 = (A0 + A2 - A3) = small + m_10(x) + dB-terms, etc.
    // (sum_p c_p a_p = (1,0), (0,1), (1/3,0), (0,1/3) for 10, 01, 12, 21)
    const T r0 = gcur[0] - mx, r1 = gcur[1] - my;  // = residual rhs r on coarse levels, 0 on the finest
    d[0] = r0 - ((P0.As + P2.As) - P3.As);
    d[1] = r1 - ((P1.As + P2.As) + P3.As);
    d[5] = (gcur[5] - mxf * T(1.0 / 3.0)) - (P2.As - P3.As);
    d[6] = (gcur[6] - myf * T(1.0 / 3.0)) - (P2.As + P3.As);
    d[2] = gcur[2] - (P2.Ss - P3.Ss);
    d[3] = gcur[3] - ((P0.Ss + P1.Ss) + T(2) * (P2.Ss + P3.Ss));
    d[4] = gcur[4] - (P0.Ss - P1.Ss);
    d[7] = gcur[7] - (P2.Ss + P3.Ss);
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
#define BIOT_HIST(SIDE, POS, K) store_history<T, TC, LO, W, RV, PV, K>(a, rg, SIDE, POS, s0, c0, mx, my)
        if (y == 0 && a.bc[SIDE_BOTTOM] == BC_DIRICHLET) { BIOT_HIST(SIDE_BOTTOM, x, 3); BIOT_HIST(SIDE_BOTTOM, x, 6); BIOT_HIST(SIDE_BOTTOM, x, 7); }
        if (y == a.ny - 1 && a.bc[SIDE_TOP] == BC_DIRICHLET) { BIOT_HIST(SIDE_TOP, x, 1); BIOT_HIST(SIDE_TOP, x, 4); BIOT_HIST(SIDE_TOP, x, 5); }
        if (x == 0 && a.bc[SIDE_LEFT] == BC_DIRICHLET) { BIOT_HIST(SIDE_LEFT, y, 2); BIOT_HIST(SIDE_LEFT, y, 5); BIOT_HIST(SIDE_LEFT, y, 6); }
        if (x == a.nx - 1 && a.bc[SIDE_RIGHT] == BC_DIRICHLET) { BIOT_HIST(SIDE_RIGHT, y, 0); BIOT_HIST(SIDE_RIGHT, y, 4); BIOT_HIST(SIDE_RIGHT, y, 7); }
#undef BIOT_HIST
    }
}

template <typename T, typename TC, int NT, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(NT) k_sweep_mom(const SweepArgs<T, TC> a, int TY)
{
    using L = RingLayout<KIND, LO>;
    constexpr int W = NT, RV = L::RV, PV = L::PV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Rings<T, W, RV, PV> rg;
    rg.raw = reinterpret_cast<T *>(smem_raw);
    rg.post = rg.raw + 3 * RV * W;
    __shared__ double red[2][NT / 32];

    const int nx = a.nx, ny = a.ny;
    const size_t NP = (size_t)nx * ny;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * (NT - 4), y0 = blockIdx.y * TY;
    const int y1 = min(y0 + TY, ny);
    const int base = y0 - 2;  // ring slot of row y: (y - base) % 3

    const int x = x0 - 2 + t;  // this thread's column (ring column t)
    const bool loads = perx || x < nx + 2;                           // a real, wrapped or ghost column
    const bool collides = t >= 1 && t < NT - 1 && (perx || (x >= 0 && x < nx));
    const bool writes = t >= 2 && t < NT - 2 && x < nx;
    const bool wall_col = !perx && (x == 0 || x == nx - 1);

    auto row_ok = [&](int y) { return pery || (y >= 0 && y < ny); };
    auto slot = [&](int y) { return (y - base) % 3; };

    T pv[RV];
    auto fetch_row = [&](int y) {
        if (loads) fetch_cell<T, TC, KIND, LO, RV>(a, x, y, NP, perx, pery, pv);
    };
    auto store_row = [&](int y) {
        if (loads) {
            const int s = slot(y);
#pragma unroll
            for (int k = 0; k < RV; k++) rg.R(s, k, t) = pv[k];
        }
    };
    auto collide_row = [&](int y) {
        if (collides && row_ok(y))
            collide_cell<T, TC, KIND, LO, W, RV, PV>(a, rg, slot(y - 1), slot(y), slot(y + 1), t);
    };

    // prologue: rows y0-2 .. y0+1 staged, rows y0-1 and y0 collided
    fetch_row(y0 - 2);
    store_row(y0 - 2);
    fetch_row(y0 - 1);
    store_row(y0 - 1);
    fetch_row(y0);
    store_row(y0);
    __syncthreads();
    collide_row(y0 - 1);
    fetch_row(y0 + 1);
    __syncthreads();
    store_row(y0 + 1);
    fetch_row(y0 + 2);
    __syncthreads();
    collide_row(y0);
    __syncthreads();

    T rmax = T(0), gmax = T(0);
    T acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = T(0);
    const T gam = a.k_gam;

    for (int y = y0; y < y1; y++) {
        store_row(y + 2);  // (A) prefetched row y+2 -> raw ring
        fetch_row(y + 3);  //     prefetch row y+3
        __syncthreads();   // (C)
        collide_row(y + 1);
        __syncthreads();   // (E)
        const int sr = slot(y);
        const int sl[3] = {slot(y - 1), sr, slot(y + 1)};
        T d[8];
#pragma unroll
        for (int k = 0; k < 8; k++) d[k] = T(0);
        if (writes) {
            T gcur[8];
#pragma unroll
            for (int k = 0; k < 8; k++) gcur[k] = rg.R(sr, k, t);
            const bool wall = wall_col || (!pery && (y == 0 || y == ny - 1));
            if (wall) residual_cell<T, TC, KIND, LO, W, RV, PV, true>(a, rg, x, y, sl, t, perx, pery, gcur, d);
            else residual_cell<T, TC, KIND, LO, W, RV, PV, false>(a, rg, x, y, sl, t, perx, pery, gcur, d);
            if (!RESTRICT) {
                const size_t idx = (size_t)y * nx + x;
#pragma unroll
                for (int k = 2; k < 8; k++) a.gout[k * NP + idx] = gcur[k] - gam * d[k];
                // first moments: (hi + lo) - gamma d, renormalised into hi + lo with LO
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    if (LO) {
                        T hi, lo;
                        two_sum(gcur[k], rg.R(sr, L::LOV + k, t) - gam * d[k], hi, lo);
                        a.gout[k * NP + idx] = hi;
                        a.glo_out[k * NP + idx] = lo;
                    } else {
                        a.gout[k * NP + idx] = gcur[k] - gam * d[k];
                    }
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
                    for (int k = 0; k < 8; k++) a.rc[k * NPc + cidx] = tot[k];
                }
            }
        }
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

constexpr int SWEEP_NT = 128;

// Rows per strip: enough strips to fill the GPU several times over, at most 64
// rows (the vertical halo costs 4 staged and 2 collided rows per strip), even
// (restriction pairs rows).
inline int strip_rows(int nx, int ny)
{
    const int strips_x = (nx + SWEEP_NT - 5) / (SWEEP_NT - 4);
    const long target = 640;  // about four resident strips per SM
    long ty = ((long)ny * strips_x + target - 1) / target;
    ty = ty < 2 ? 2 : (ty > 64 ? 64 : ty);
    ty += ty & 1;
    return (int)ty;
}

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
cudaError_t launch_rows(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    constexpr size_t smem = rows_smem_bytes<T, KIND, LO, SWEEP_NT>();
    auto kern = k_sweep_mom<T, TC, SWEEP_NT, KIND, LO, RESTRICT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int ty = strip_rows(a.nx, a.ny);
    dim3 grid((a.nx + SWEEP_NT - 5) / (SWEEP_NT - 4), (a.ny + ty - 1) / ty);
    kern<<<grid, SWEEP_NT, smem, s>>>(a, ty);
    return cudaGetLastError();
}

// Level kind from the arguments: F~ present = finest level; low parts only
// with FP32 storage on the finest level.
template <typename T, typename TC>
cudaError_t launch_sweep_mom_impl(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    const bool restrict_ = a.mode == SWEEP_RESTRICT;
    if (a.Ft) {
        if (a.glo) return restrict_ ? launch_rows<T, TC, KIND_FINE, true, true>(a, s) : launch_rows<T, TC, KIND_FINE, true, false>(a, s);
        return restrict_ ? launch_rows<T, TC, KIND_FINE, false, true>(a, s) : launch_rows<T, TC, KIND_FINE, false, false>(a, s);
    }
    return restrict_ ? launch_rows<T, TC, KIND_COARSE, false, true>(a, s) : launch_rows<T, TC, KIND_COARSE, false, false>(a, s);
}

}  // namespace biot
