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

template <int TX, int TY, typename T>
constexpr size_t mom_sweep_smem_bytes()
{
    return sizeof(T) * (size_t)(19 * (TX + 4) * (TY + 4) + 8 * TX * TY);
}

template <typename T>
struct PV {
    T sig, bx, by;  // value = sig + bx * m_10(x) + by * m_01(x)
};

// The iterate's moments at a cell (plus the prolongated coarse correction);
// lo receives the low parts of m_10, m_01 and the correction to them.
template <typename T, typename TC>
__device__ __forceinline__ void load_moments(const SweepArgs<T, TC> &a, int x, int y, size_t NP, T (&v)[8], T (&lo)[2])
{
    const size_t idx = (size_t)y * a.nx + x;
    if (a.zero_init) {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = T(0);
    } else {
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = a.g[k * NP + idx];
    }
    lo[0] = a.glo ? a.glo[idx] : T(0);
    lo[1] = a.glo ? a.glo[NP + idx] : T(0);
    if (a.gc) {
        const size_t NPc = NP >> 2;
        const size_t cidx = (size_t)(y >> 1) * (a.nx >> 1) + (x >> 1);
        lo[0] += (T)a.gc[cidx];
        lo[1] += (T)a.gc[NPc + cidx];
#pragma unroll
        for (int k = 2; k < 8; k++) v[k] += (T)a.gc[k * NPc + cidx];
    }
}

// Exact sum of two floating-point values: s + e == a + b.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e)
{
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename T, typename TC>
__device__ __forceinline__ T load_ms(const SweepArgs<T, TC> &a, int x, int y, size_t NP)
{
    T v = a.zero_init ? T(0) : a.g[3 * NP + (size_t)y * a.nx + x];
    if (a.gc) v += (T)a.gc[3 * (NP >> 2) + (size_t)(y >> 1) * (a.nx >> 1) + (x >> 1)];
    return v;
}

// Shared-memory planes of the sweep (all indexed by the tile + 2 box).
template <typename T, int BN>
struct MomSmem {
    T *M;    // [8][BN] iterate moments (tile + 1)
    T *MS;   // [BN]    m_s of the iterate (tile + 2)
    T *SS;   // [4][BN] even part S*_p = g*_first + g*_second after collision
    T *MI;   // [2][BN] first moments of the collision input g - r (high parts)
    T *ML;   // [2][BN] their low parts
    T *F;    // [2][BN] force of the collision
};

// Post-collision population K of the cell at box position q, split relative
// to the collision-input first moments (mx, my) of the target at box position
// q0 (high parts; the low parts are differenced alongside):
//   g*_K = 1/2 (S*_p + e A*_p),  A*_p = a_p . m + b_p . F  (Tab. moments:inverse)
template <typename T, int BN, int K>
__device__ __forceinline__ PV<T> post_pop(const MomSmem<T, BN> &s, int q, int q0, T mx, T my)
{
    constexpr int p = pair_of(K);
    constexpr T e = T(sign_of(K));
    const T dmx = (s.MI[q] - mx) + (s.ML[q] - s.ML[q0]);
    const T dmy = (s.MI[BN + q] - my) + (s.ML[BN + q] - s.ML[BN + q0]);
    const T odd = (T(pa_x(p)) * dmx + T(pa_y(p)) * dmy) + (T(pb_x(p)) * s.F[q] + T(pb_y(p)) * s.F[BN + q]);
    PV<T> v;
    v.sig = T(0.5) * (s.SS[p * BN + q] + e * odd);
    v.bx = e * T(0.5 * pa_x(p));
    v.by = e * T(0.5 * pa_y(p));
    return v;
}

// Population of direction K arriving at tile cell (x, y), box position q.
template <typename T, typename TC, int BN, int BX, int K>
__device__ __forceinline__ PV<T> pull(const SweepArgs<T, TC> &a, const MomSmem<T, BN> &s, int x, int y, int q,
                                      T mx, T my, bool perx, bool pery)
{
    constexpr int cx = ex8(K), cy = ey8(K);
    const int sx = x - cx, sy = y - cy;
    const bool outx = !perx && (sx < 0 || sx >= a.nx);
    const bool outy = !pery && (sy < 0 || sy >= a.ny);
    if (!outx && !outy) return post_pop<T, BN, K>(s, q - cx - cy * BX, q, mx, my);
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
            if (outx) return post_pop<T, BN, dir8(-cx, -cy)>(s, q, q, mx, my);
            return post_pop<T, BN, dir8(cx, -cy)>(s, q - cx, q, mx, my);
        }
        return post_pop<T, BN, dir8(-cx, cy)>(s, q - cy * BX, q, mx, my);
    }
    constexpr int kout = opp8(K);
    const PV<T> o = post_pop<T, BN, kout>(s, q, q, mx, my);
    const bool horiz = (side == SIDE_BOTTOM || side == SIDE_TOP);
    const int n = horiz ? a.nx : a.ny;
    PV<T> v;
    if (type == BC_NEUMANN) {  // eq. BC:traction
        v.sig = -o.sig;
        v.bx = -o.bx;
        v.by = -o.by;
        if (a.prof[side]) v.sig += T(a.c0h * traction_term(a.prof[side], side, n, x, y, cx, cy));
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
    if (a.prof[side]) v.sig += T(dirichlet_term(a.prof[side], side, n, x, y, cx, cy));
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

template <typename T, typename TC, int BN, int BX, int P>
__device__ __forceinline__ PairOut<T> pull_pair(const SweepArgs<T, TC> &a, const MomSmem<T, BN> &s, int x, int y,
                                                int q, T mx, T my, bool perx, bool pery)
{
    const PV<T> u = pull<T, TC, BN, BX, pair_first(P)>(a, s, x, y, q, mx, my, perx, pery);
    const PV<T> v = pull<T, TC, BN, BX, pair_second(P)>(a, s, x, y, q, mx, my, perx, pery);
    PairOut<T> o;
    o.Ss = u.sig + v.sig;
    o.As = u.sig - v.sig;
    o.bsx = u.bx + v.bx;
    o.bsy = u.by + v.by;
    o.dbx = (u.bx - v.bx) - T(pa_x(P));
    o.dby = (u.by - v.by) - T(pa_y(P));
    return o;
}

template <typename T, typename TC, int BN, int K>
__device__ __forceinline__ void store_history(const SweepArgs<T, TC> &a, const MomSmem<T, BN> &s, int side, int pos,
                                              int q, T mx, T my)
{
    const PV<T> o = post_pop<T, BN, K>(s, q, q, mx, my);
    const T mxf = mx + s.ML[q], myf = my + s.ML[BN + q];
    a.H[side][3 * pos + hslot(side, K)] = o.sig + (o.bx * mxf + o.by * myf);
}

template <typename T, typename TC, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_sweep_mom(const SweepArgs<T, TC> a)
{
    constexpr int NT = TX * TY;
    constexpr int BX = TX + 4, BY = TY + 4, BN = BX * BY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MomSmem<T, BN> s;
    s.M = reinterpret_cast<T *>(smem_raw);
    s.MS = s.M + 8 * BN;
    s.SS = s.MS + BN;
    s.MI = s.SS + 4 * BN;
    s.ML = s.MI + 2 * BN;
    s.F = s.ML + 2 * BN;
    T *sR = s.F + 2 * BN;  // [8][NT] residual of the tile (restriction)
    __shared__ double red[2][NT / 32];

    const int nx = a.nx, ny = a.ny;
    const size_t NP = (size_t)nx * ny;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const bool perx = a.bc[SIDE_LEFT] == BC_PERIODIC;
    const bool pery = a.bc[SIDE_BOTTOM] == BC_PERIODIC;

    // Phase 1: iterate moments on the tile + 1 box, m_s on the tile + 2 box.
    // Outside a non-periodic wall m_s (the divergence) takes the value of the
    // adjacent cell (even extension).
    for (int p = threadIdx.x; p < BN; p += NT) {
        const int bx = p % BX, by = p / BX;
        int gx = x0 + bx - 2, gy = y0 + by - 2;
        if (perx) gx = wrapi(gx, nx);
        if (pery) gy = wrapi(gy, ny);
        const bool in = (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny;
        const bool inner = bx >= 1 && bx <= TX + 2 && by >= 1 && by <= TY + 2;
        if (in && inner) {
            T v[8], lo[2];
            load_moments(a, gx, gy, NP, v, lo);
#pragma unroll
            for (int k = 0; k < 8; k++) s.M[k * BN + p] = v[k];
            s.ML[p] = lo[0];
            s.ML[BN + p] = lo[1];
            s.MS[p] = v[3];
        } else {
            s.MS[p] = load_ms(a, clampi(gx, nx), clampi(gy, ny), NP);
        }
    }
    __syncthreads();

    // Phase 2: collide the tile + 1 box (even moments relaxed, Tab. moments and
    // eq. moments:collision:22; the odd part is kept as first moments + force).
    const T one_m_ws = T(1.0 - a.om_s), one_m_wd = T(1.0 - a.om_d);
    const T c22 = T(-1.0 / (12.0 * a.lm + 4.0));
    const T cf = T(a.coef_fstar * (-1.5 / (3.0 * a.lm + 1.0)));  // alpha^2 r/2 * dD/dm_s
    constexpr int QX = TX + 2, QN = (TX + 2) * (TY + 2);
    for (int qq = threadIdx.x; qq < QN; qq += NT) {
        const int bx = qq % QX + 1, by = qq / QX + 1;
        const int p = by * BX + bx;
        int gx = x0 + bx - 2, gy = y0 + by - 2;
        if (perx) gx = wrapi(gx, nx);
        if (pery) gy = wrapi(gy, ny);
        if ((unsigned)gx >= (unsigned)nx || (unsigned)gy >= (unsigned)ny) continue;
        const size_t idx = (size_t)gy * nx + gx;
        T m0 = s.M[p], m1 = s.M[BN + p], m2 = s.M[2 * BN + p], m3 = s.M[3 * BN + p], m4 = s.M[4 * BN + p];
        if (a.r) {
            m0 -= a.r[idx];
            m1 -= a.r[NP + idx];
            m2 -= a.r[2 * NP + idx];
            m3 -= a.r[3 * NP + idx];
            m4 -= a.r[4 * NP + idx];
        }
        // F_* = (alpha^2 r/2) grad^c D(g), grad^c with the D2Q9 weights
        const T dE = s.MS[p + 1], dW = s.MS[p - 1], dN = s.MS[p + BX], dS = s.MS[p - BX];
        const T dNE = s.MS[p + BX + 1], dNW = s.MS[p + BX - 1], dSE = s.MS[p - BX + 1], dSW = s.MS[p - BX - 1];
        T Fx = cf * ((dE - dW) * T(1.0 / 3.0) + ((dNE + dSE) - (dNW + dSW)) * T(1.0 / 12.0));
        T Fy = cf * ((dN - dS) * T(1.0 / 3.0) + ((dNE + dNW) - (dSE + dSW)) * T(1.0 / 12.0));
        if (a.Ft) {
            Fx += a.Ft[idx];
            Fy += a.Ft[NP + idx];
        }
        const T ms = one_m_ws * m3, md = one_m_wd * m4, m11 = one_m_wd * m2, m22 = c22 * m3;
        s.SS[0 * BN + p] = T(0.5) * (ms + md) - m22;
        s.SS[1 * BN + p] = T(0.5) * (ms - md) - m22;
        s.SS[2 * BN + p] = T(0.5) * (m11 + m22);
        s.SS[3 * BN + p] = T(0.5) * (m22 - m11);
        s.MI[p] = m0;
        s.MI[BN + p] = m1;
        s.F[p] = Fx;
        s.F[BN + p] = Fy;
    }
    __syncthreads();

    // Phase 3: stream (pull) with the wall rules; residual d = m - m** from
    // small parts; then relax (m - gamma d) or restrict d.
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x = x0 + tx, y = y0 + ty;
    const bool valid = x < nx && y < ny;
    double rmax = 0.0, gmax = 0.0;
    if (valid) {
        const int q = (ty + 2) * BX + (tx + 2);
        const size_t idx = (size_t)y * nx + x;
        const T mx = s.MI[q], my = s.MI[BN + q];
        const PairOut<T> P0 = pull_pair<T, TC, BN, BX, 0>(a, s, x, y, q, mx, my, perx, pery);
        const PairOut<T> P1 = pull_pair<T, TC, BN, BX, 1>(a, s, x, y, q, mx, my, perx, pery);
        const PairOut<T> P2 = pull_pair<T, TC, BN, BX, 2>(a, s, x, y, q, mx, my, perx, pery);
        const PairOut<T> P3 = pull_pair<T, TC, BN, BX, 3>(a, s, x, y, q, mx, my, perx, pery);
        const T mxf = mx + s.ML[q], myf = my + s.ML[BN + q];  // beta terms only (walls)
        T gcur[8], d[8];
#pragma unroll
        for (int k = 0; k < 8; k++) gcur[k] = s.M[k * BN + q];
        // odd moments: m**_10 = (A0 + A2 - A3) = small + m_10(x) + dB-terms, etc.
        // (sum_p c_p a_p = (1,0), (0,1), (1/3,0), (0,1/3) for 10, 01, 12, 21)
        const T r0 = gcur[0] - mx, r1 = gcur[1] - my;  // = residual rhs r on coarse levels, 0 on the finest
        d[0] = r0 - ((P0.As + P2.As) - P3.As) - (((P0.dbx + P2.dbx) - P3.dbx) * mxf + ((P0.dby + P2.dby) - P3.dby) * myf);
        d[1] = r1 - ((P1.As + P2.As) + P3.As) - (((P1.dbx + P2.dbx) + P3.dbx) * mxf + ((P1.dby + P2.dby) + P3.dby) * myf);
        d[5] = (gcur[5] - mxf * T(1.0 / 3.0)) - (P2.As - P3.As) - ((P2.dbx - P3.dbx) * mxf + (P2.dby - P3.dby) * myf);
        d[6] = (gcur[6] - myf * T(1.0 / 3.0)) - (P2.As + P3.As) - ((P2.dbx + P3.dbx) * mxf + (P2.dby + P3.dby) * myf);
        // even moments from S = small + beta-sum terms
        d[2] = gcur[2] - (P2.Ss - P3.Ss) - ((P2.bsx - P3.bsx) * mxf + (P2.bsy - P3.bsy) * myf);
        d[3] = gcur[3] - ((P0.Ss + P1.Ss) + T(2) * (P2.Ss + P3.Ss))
               - (((P0.bsx + P1.bsx) + T(2) * (P2.bsx + P3.bsx)) * mxf + ((P0.bsy + P1.bsy) + T(2) * (P2.bsy + P3.bsy)) * myf);
        d[4] = gcur[4] - (P0.Ss - P1.Ss) - ((P0.bsx - P1.bsx) * mxf + (P0.bsy - P1.bsy) * myf);
        d[7] = gcur[7] - (P2.Ss + P3.Ss) - ((P2.bsx + P3.bsx) * mxf + (P2.bsy + P3.bsy) * myf);
        // history of the fullway bounce-back: this call's outgoing populations
        if (y == 0 && a.bc[SIDE_BOTTOM] == BC_DIRICHLET) {
            store_history<T, TC, BN, 3>(a, s, SIDE_BOTTOM, x, q, mx, my);
            store_history<T, TC, BN, 6>(a, s, SIDE_BOTTOM, x, q, mx, my);
            store_history<T, TC, BN, 7>(a, s, SIDE_BOTTOM, x, q, mx, my);
        }
        if (y == ny - 1 && a.bc[SIDE_TOP] == BC_DIRICHLET) {
            store_history<T, TC, BN, 1>(a, s, SIDE_TOP, x, q, mx, my);
            store_history<T, TC, BN, 4>(a, s, SIDE_TOP, x, q, mx, my);
            store_history<T, TC, BN, 5>(a, s, SIDE_TOP, x, q, mx, my);
        }
        if (x == 0 && a.bc[SIDE_LEFT] == BC_DIRICHLET) {
            store_history<T, TC, BN, 2>(a, s, SIDE_LEFT, y, q, mx, my);
            store_history<T, TC, BN, 5>(a, s, SIDE_LEFT, y, q, mx, my);
            store_history<T, TC, BN, 6>(a, s, SIDE_LEFT, y, q, mx, my);
        }
        if (x == nx - 1 && a.bc[SIDE_RIGHT] == BC_DIRICHLET) {
            store_history<T, TC, BN, 0>(a, s, SIDE_RIGHT, y, q, mx, my);
            store_history<T, TC, BN, 4>(a, s, SIDE_RIGHT, y, q, mx, my);
            store_history<T, TC, BN, 7>(a, s, SIDE_RIGHT, y, q, mx, my);
        }
        if (a.mode == SWEEP_SMOOTH) {
            const T gam = T(a.gamma);
#pragma unroll
            for (int k = 2; k < 8; k++) a.gout[k * NP + idx] = gcur[k] - gam * d[k];
            // first moments: (hi + lo) - gamma d, renormalised into hi + lo
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const T t = s.ML[k * BN + q] - gam * d[k];
                if (a.glo_out) {
                    T hi, lo;
                    two_sum(gcur[k], t, hi, lo);
                    a.gout[k * NP + idx] = hi;
                    a.glo_out[k * NP + idx] = lo;
                } else {
                    a.gout[k * NP + idx] = gcur[k] + t;
                }
            }
            if (a.resmax) {
                rmax = pop_absmax(d);
                gmax = pop_absmax(gcur);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) sR[k * NT + threadIdx.x] = d[k];
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
        if (lane == 0) {
            red[0][warp] = rmax;
            red[1][warp] = gmax;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
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

constexpr int MOM_TX = 32, MOM_TY = 8;

template <typename T, typename TC>
cudaError_t launch_sweep_mom_impl(const SweepArgs<T, TC> &a, cudaStream_t s)
{
    constexpr size_t smem = mom_sweep_smem_bytes<MOM_TX, MOM_TY, T>();
    auto kern = k_sweep_mom<T, TC, MOM_TX, MOM_TY>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((a.nx + MOM_TX - 1) / MOM_TX, (a.ny + MOM_TY - 1) / MOM_TY);
    kern<<<grid, MOM_TX * MOM_TY, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace biot
