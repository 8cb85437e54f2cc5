/*
 * biot_oracle.c -- FP64 CPU oracle for the coupled lattice Boltzmann method of
 * Lunowa & Wohlmuth, "A lattice Boltzmann method for Biot's consolidation model
 * of linear poroelasticity" (arXiv 2409.11382).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant with the CUDA library and includes
 * nothing from it.
 *
 * What it restates, in the paper's order and without any blocking or fusion:
 *   Alg. 5  semi-implicit LBM with multigrid (time loop),
 *   Alg. 4  ELASTIC_MULTIGRID (V-cycle, under-relaxed smoother eq. MG:smoother,
 *           restriction / prolongation eq. MG:restriction, self-dependence
 *           eq. MG:selfdependence),
 *   Alg. 2  ELASTIC_STEP (eqs. moments, moments:stress, moments:BC,
 *           moments:halfForce, moments:collision, Tab. moments,
 *           moments:collision:22, moments:inverse, Tab. moments:inverse),
 *   Alg. 3  FLOW_STEP (eqs. pressure, pressure:equilibrium, pressure:collision,
 *           pressure:collision:source, pressure:rate),
 *   §3.4    coupling (eqs. pressure:gradient, pressure:gradient:alternative,
 *           source:explicit, source:implicit, LBM:divergence),
 *   §3.6    initial conditions (eqs. ICs, ICs:moments) and the periodic,
 *           Dirichlet (BC:pressure, BC:elasticity) and Neumann (BC:noFlow,
 *           BC:traction) boundary schemes.
 *
 * Units.  Everything is computed in lattice units of the finest grid
 * (dx = dt = 1, c_s^2 = 1/3) using the dimensionless scaling of §2.2 with
 * L = dx (physical cell size h), T = dt (physical step), H = 1, so that
 * eps = h (§3.4, last paragraph).  With c0 the storage coefficient:
 *   lambda^ = c0 lambda, mu^ = c0 mu, kappa^ = dt kappa / (c0 h^2),
 *   p^ = c0 p,  lattice stress = c0 h sigma,  lattice force = c0 h^2 f_eff,
 *   lattice divergence D = h div(eta),  lattice source s' = dt s_eff.
 * Where a passage is ambiguous, garbled or silent, the reading taken is
 * stated as "Reading Rn" next to the code that uses it.
 *
 * Parity status: every routine here is pinned by the CPU tests under tests/
 * (moment-table identities, flow mass balance and diffusion decay, drained
 * elastic closed forms on each wall, a dense direct solve of the discrete
 * fixed point, Terzaghi's series solution, the manufactured periodic solution
 * and the coupling-stability behaviour of §4.1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LEVELS 16

/* Threads of the per-cell loops.  Only loops whose iterations write disjoint
 * cells run in parallel (collision, streaming, gradients, relaxation,
 * prolongation, flow step); every sum keeps its serial order, so the results
 * are bitwise those of one thread.  Default 1 (orc_set_threads). */
static int orc_threads = 1;
#define ORC_PAR_FOR _Pragma("omp parallel for schedule(static) if(orc_threads > 1) num_threads(orc_threads)")

enum { ORC_PERIODIC = 0, ORC_SYMMETRY = 1, ORC_DIRICHLET = 2, ORC_NEUMANN = 3 };
enum { SIDE_BOTTOM = 0, SIDE_RIGHT = 1, SIDE_TOP = 2, SIDE_LEFT = 3 };

typedef struct {
    int nx, ny;             /* lattice cells of the finest grid */
    double lx, ly;          /* domain size (lx/nx must equal ly/ny) */
    double lambda, mu;      /* Lame coefficients (dimensional) */
    double alpha, c0, kappa;/* Biot-Willis, storage, permeability */
    double dt;              /* physical time step */
    double r;               /* explicit / semi-implicit ratio of eq. source:implicit */
    int levels, K;          /* multigrid levels L and smoothing sweeps K */
    double gamma;           /* under-relaxation of eq. MG:smoother */
    double tol;             /* residual tolerance (used when ne_fixed <= 0) */
    int ne_max, ne_fixed;   /* cap on V-cycles; fixed V-cycle count when > 0 */
    int cycle;              /* 0: V-cycle (Alg. 4); 1: W-cycle; 2: F-cycle (reading R20) */
    int fmg;                /* 1: the first cycle of every elastic solve is a full-multigrid cycle (reading R21) */
    int pgrad;              /* 0: eq. pressure:gradient; 1: eq. pressure:gradient:alternative (reading R22) */
    int K_level[ORC_MAX_LEVELS]; /* smoothing sweeps of the level j below the finest (j = 0: finest);
                                    <= 0: K (reading R23) */
} orc_params;

typedef struct {
    int eta_type, p_type;
    const double *eta_profile; /* 2 x (2n+1): [component][k], position k*h/2 along the side */
    const double *p_profile;   /* (2n+1) */
} orc_side;

typedef struct {
    int nx, ny;
    double *g;      /* current iterate / correction, 8 per cell */
    double *r;      /* residual right-hand side, 8 per cell (NULL on the finest level) */
    double *gin;    /* g - r */
    double *gs;     /* post-collision populations of the last ELASTIC_STEP */
    double *gout;   /* result of the last ELASTIC_STEP (after streaming and BCs) */
    double *H;      /* post-collision populations of the previous ELASTIC_STEP (fullway BB) */
    double *F;      /* force used by the current ELASTIC_STEP, 2 per cell */
    double *D;      /* lattice divergence of the iterate, 1 per cell */
    int hist_valid;
} Level;

typedef struct {
    orc_params P;
    int side_eta[4], side_p[4];
    double *eta_prof[4], *p_prof[4];
    /* derived lattice parameters */
    double h, lam, mu, kap, omega, om_s, om_d;
    int L;
    Level lv[ORC_MAX_LEVELS];  /* lv[0] coarsest ... lv[L-1] finest */
    /* flow and coupling state on the finest grid */
    double *f, *fs, *fn;       /* 9 per cell: pre-collision, post-collision, streamed */
    double *D1, *D2, *Dt;      /* D(t - dt), D(t - 2 dt), D(t) */
    double *sexp;              /* explicit part of s_eff^im in lattice units */
    double *Pf;                /* sum_i f_i per cell (eq. pressure:gradient:alternative) */
    double *Ft;                /* explicit force F~ (2 per cell) */
    double *fbody, *src;       /* body force f (2 per cell) and source s (1 per cell), dimensional */
    double t;
    long nstep;
    int solved, initialized;
    /* statistics */
    int last_ne;
    double last_res, last_gnorm, last_res_l2;
    long total_cycles;
    int notconv_steps, diverged;
} Orc;

/* ---------------------------------------------------------------------------
 * Velocity sets, Tab. velocities (§3.1).
 * D2Q9, linear index i: 00, 10, 01, -10, 0-1, 11, -11, -1-1, 1-1.
 */
static const int CX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W9[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* D2Q8 (no rest velocity), Miller indices ij, in the row order of
 * Tab. moments:inverse: 10, 01, -10, 0-1, 11, -11, -1-1, 1-1. */
static const int CX8[8] = {1, 0, -1, 0, 1, -1, -1, 1};
static const int CY8[8] = {0, 1, 0, -1, 1, 1, -1, -1};

/* Tab. moments:inverse.  Reading R1: the printed column header "01, 10" is
 * swapped; the columns are (10, 01, 11, s, d, 12, 21, 22), the only order for
 * which the table inverts eqs. moments / moments:stress. */
static const double TINV[8][8] = {
    /*          10     01     11     s      d      12     21     22   */
    /* 10  */ { 0.5,   0.0,   0.0,   0.25,  0.25, -0.5,   0.0,  -0.5 },
    /* 01  */ { 0.0,   0.5,   0.0,   0.25, -0.25,  0.0,  -0.5,  -0.5 },
    /* -10 */ {-0.5,   0.0,   0.0,   0.25,  0.25,  0.5,   0.0,  -0.5 },
    /* 0-1 */ { 0.0,  -0.5,   0.0,   0.25, -0.25,  0.0,   0.5,  -0.5 },
    /* 11  */ { 0.0,   0.0,   0.25,  0.0,   0.0,   0.25,  0.25,  0.25},
    /* -11 */ { 0.0,   0.0,  -0.25,  0.0,   0.0,  -0.25,  0.25,  0.25},
    /* -1-1*/ { 0.0,   0.0,   0.25,  0.0,   0.0,  -0.25, -0.25,  0.25},
    /* 1-1 */ { 0.0,   0.0,  -0.25,  0.0,   0.0,   0.25, -0.25,  0.25},
};

static int ipow(int b, int e) { int v = 1; while (e-- > 0) v *= b; return v; }

static int q8_index(int cx, int cy)
{
    for (int k = 0; k < 8; k++) if (CX8[k] == cx && CY8[k] == cy) return k;
    return -1;
}
static int q9_index(int cx, int cy)
{
    for (int i = 0; i < 9; i++) if (CX9[i] == cx && CY9[i] == cy) return i;
    return -1;
}
/* D2Q9 weight of a D2Q8 direction (reading R2: eq. BC:elasticity uses the
 * D2Q9 weights 1/9 on the axes and 1/36 on the diagonals). */
static double w_of(int cx, int cy) { return W9[q9_index(cx, cy)]; }

/* ---------------------------------------------------------------------------
 * Raw moments m_ab = sum_ij i^a j^b g_ij, eq. moments.
 */
static double raw_moment(const double g[8], int a, int b)
{
    double m = 0.0;
    for (int k = 0; k < 8; k++) m += (double)(ipow(CX8[k], a) * ipow(CY8[k], b)) * g[k];
    return m;
}

/* Lattice divergence of eq. LBM:divergence with the half-collision moment of
 * eq. moments:bared: D = -mbar_s / (2 (lam+mu)),
 * mbar_s = 3(lam+mu)/(3(lam+mu)+1) m_s. */
static double divergence_of(const Orc *o, const double g[8])
{
    double ms = raw_moment(g, 2, 0) + raw_moment(g, 0, 2);
    double lm = o->lam + o->mu;
    double mbar_s = 3.0 * lm / (3.0 * lm + 1.0) * ms;
    return -mbar_s / (2.0 * lm);
}

/* Collision of Alg. 2 (first six lines): moments, half force, equilibrium,
 * second half force, relaxation, back-transformation. */
static void collide(const Orc *o, const double g[8], const double F[2], double gs[8])
{
    const double lm = o->lam + o->mu;
    /* eqs. moments, moments:stress, moments:BC */
    double m10 = raw_moment(g, 1, 0), m01 = raw_moment(g, 0, 1), m11 = raw_moment(g, 1, 1);
    double m20 = raw_moment(g, 2, 0), m02 = raw_moment(g, 0, 2);
    double m12 = raw_moment(g, 1, 2), m21 = raw_moment(g, 2, 1), m22 = raw_moment(g, 2, 2);
    double ms = m20 + m02, md = m20 - m02;
    double mf = m22 + ms / (12.0 * lm - 4.0);
    (void)mf; /* relaxed with omega_f = 1 to m_f^eq = 0; eq. moments:collision:22 below */
    /* eq. moments:halfForce, first half */
    double mb10 = m10 + 0.5 * F[0], mb01 = m01 + 0.5 * F[1];
    /* Tab. moments: equilibria */
    double eq_s = 0.0, eq_d = 0.0, eq_11 = 0.0, eq_12 = mb10 / 3.0, eq_21 = mb01 / 3.0;
    /* eq. moments:halfForce, second half (omega_10 = omega_01 = 0) */
    double ms10 = mb10 + 0.5 * F[0], ms01 = mb01 + 0.5 * F[1];
    /* eq. moments:collision with the rates of Tab. moments */
    double w_s = o->om_s, w_d = o->om_d, w_11 = o->om_d, w_12 = 1.0, w_21 = 1.0;
    double mss = ms - w_s * (ms - eq_s);
    double msd = md - w_d * (md - eq_d);
    double ms11 = m11 - w_11 * (m11 - eq_11);
    double ms12 = m12 - w_12 * (m12 - eq_12);
    double ms21 = m21 - w_21 * (m21 - eq_21);
    /* eq. moments:collision:22 */
    double ms22 = -ms / (12.0 * lm + 4.0);
    double mstar[8] = {ms10, ms01, ms11, mss, msd, ms12, ms21, ms22};
    /* eq. moments:inverse */
    for (int k = 0; k < 8; k++) {
        double v = 0.0;
        for (int nu = 0; nu < 8; nu++) v += TINV[k][nu] * mstar[nu];
        gs[k] = v;
    }
}

/* ---------------------------------------------------------------------------
 * Boundary data.  Profiles are sampled at the 2n+1 points k*h/2 along a side
 * (k even: cell faces, k odd: cell centres); a boundary scheme evaluated at
 * x + c/2 reads the sample at the wall crossing of the outgoing direction.
 */
static int side_len(const Orc *o, int side)
{
    return (side == SIDE_BOTTOM || side == SIDE_TOP) ? o->P.nx : o->P.ny;
}
static int crossing_index(int side, int x, int y, int cx_out, int cy_out)
{
    if (side == SIDE_BOTTOM || side == SIDE_TOP) return 2 * x + 1 + cx_out;
    return 2 * y + 1 + cy_out;
}
static double eta_data(const Orc *o, int side, int comp, int k)
{
    if (!o->eta_prof[side]) return 0.0;
    return o->eta_prof[side][comp * (2 * side_len(o, side) + 1) + k];
}
static double p_data(const Orc *o, int side, int k)
{
    if (!o->p_prof[side]) return 0.0;
    return o->p_prof[side][k];
}

/* Traction correction varsigma of eq. BC:traction for the incoming direction
 * (cx, cy) at a wall with outward normal n, from the traction t = sigma n.
 * The paper prints the left wall only; reading R11: axis directions get
 * -sigma_nn, diagonal ones -1/2 cx cy sigma_12 (this reproduces the printed
 * left-wall values and is covariant under the rotations of the square). */
static double varsigma(int side, int cx, int cy, double t1, double t2)
{
    int nxn = (side == SIDE_RIGHT) ? 1 : (side == SIDE_LEFT) ? -1 : 0;
    int nyn = (side == SIDE_TOP) ? 1 : (side == SIDE_BOTTOM) ? -1 : 0;
    double s12, snn;
    if (nyn != 0) { s12 = nyn * t1; snn = nyn * t2; }
    else          { s12 = nxn * t2; snn = nxn * t1; }
    if (cx == 0 || cy == 0) return -snn;
    return -0.5 * cx * cy * s12;
}

static int mirror(int s, int n) { return s < 0 ? -1 - s : 2 * n - 1 - s; }

/* Pull of one elastic population into cell (x,y) along direction k after
 * streaming (eq. streaming), resolving sources outside the domain by the
 * boundary schemes of §3.6.  Reading R13: periodic wraps first; a source
 * beyond one wall is handled by that wall's scheme; a source beyond a corner
 * by the top/bottom scheme, except that a bounce-back type side wall wins over
 * a SYMMETRY top/bottom (the mirror image of the side wall's bounce-back), and
 * two SYMMETRY walls reflect twice.  Reading R12: SYMMETRY (roller / no-flux
 * side) is specular reflection. */
static double pull_elastic(const Orc *o, const Level *Lv, int fine, int x, int y, int k,
                           const double *gs, const double *Hold)
{
    const int nx = Lv->nx, ny = Lv->ny;
    const int cx = CX8[k], cy = CY8[k];
    int sx = x - cx, sy = y - cy;
    if ((sx < 0 || sx >= nx) && o->side_eta[SIDE_LEFT] == ORC_PERIODIC) sx = (sx + nx) % nx;
    if ((sy < 0 || sy >= ny) && o->side_eta[SIDE_BOTTOM] == ORC_PERIODIC) sy = (sy + ny) % ny;
    int side = -1;
    if (sy < 0) side = SIDE_BOTTOM;
    else if (sy >= ny) side = SIDE_TOP;
    else if (sx < 0) side = SIDE_LEFT;
    else if (sx >= nx) side = SIDE_RIGHT;
    if (side < 0) return gs[8 * (sy * nx + sx) + k];
    if ((side == SIDE_BOTTOM || side == SIDE_TOP) && (sx < 0 || sx >= nx)) {
        int vert = sx < 0 ? SIDE_LEFT : SIDE_RIGHT;
        if (o->side_eta[side] == ORC_SYMMETRY && o->side_eta[vert] != ORC_SYMMETRY) side = vert;
    }

    const int type = o->side_eta[side];
    const int kout = q8_index(-cx, -cy);
    const double *here = gs + 8 * (y * nx + x);
    if (type == ORC_SYMMETRY) {
        int mx = sx, my = sy, rcx = cx, rcy = cy;
        if (side == SIDE_BOTTOM || side == SIDE_TOP) {
            my = mirror(sy, ny); rcy = -cy;
            if (mx < 0 || mx >= nx) { mx = mirror(mx, nx); rcx = -cx; } /* corner of two symmetry walls */
        } else {
            mx = mirror(sx, nx); rcx = -cx;
        }
        return gs[8 * (my * nx + mx) + q8_index(rcx, rcy)];
    }
    const int kk = crossing_index(side, x, y, -cx, -cy);
    if (type == ORC_NEUMANN) {
        /* eq. BC:traction (halfway anti-bounce-back), data term eps*varsigma =
         * c0 h varsigma(t) in lattice units; homogeneous on coarse levels */
        double v = -here[kout];
        if (fine) {
            double t1 = eta_data(o, side, 0, kk), t2 = eta_data(o, side, 1, kk);
            v += o->P.c0 * o->h * varsigma(side, cx, cy, t1, t2);
        }
        return v;
    }
    /* ORC_DIRICHLET: eq. BC:elasticity (fullway bounce-back with a delay of one
     * pseudo-time step).  Reading R10: g_ij(tau - dtau) is the post-collision
     * population of the previous ELASTIC_STEP call on this level; on the first
     * call after a reset the current one is used (g(-1,t) = g(0,t), §3.4). */
    double v = Hold[8 * (y * nx + x) + kout];
    if (fine) {
        double e1 = eta_data(o, side, 0, kk), e2 = eta_data(o, side, 1, kk);
        v -= 6.0 * w_of(-cx, -cy) * ((double)(-cx) * e1 + (double)(-cy) * e2);
    }
    return v;
}

/* ELASTIC_STEP (Alg. 2) on one level: gin are the pre-collision populations,
 * F the force per cell; the result (streamed, boundary conditions applied) is
 * written to gout.  Updates the history used by the fullway bounce-back. */
static void elastic_step(Orc *o, Level *Lv, int fine, const double *gin, const double *F, double *gout)
{
    const int n = Lv->nx * Lv->ny;
    ORC_PAR_FOR
    for (int c = 0; c < n; c++) collide(o, gin + 8 * c, F + 2 * c, Lv->gs + 8 * c);
    const double *Hold = Lv->hist_valid ? Lv->H : Lv->gs;
    ORC_PAR_FOR
    for (int y = 0; y < Lv->ny; y++)
        for (int x = 0; x < Lv->nx; x++)
            for (int k = 0; k < 8; k++)
                gout[8 * (y * Lv->nx + x) + k] = pull_elastic(o, Lv, fine, x, y, k, Lv->gs, Hold);
    memcpy(Lv->H, Lv->gs, sizeof(double) * 8 * (size_t)n);
    Lv->hist_valid = 1;
}

/* Neighbour value for the central-difference stencil of
 * eq. pressure:gradient:alternative.  Reading R14: outside a non-periodic
 * side the value of the adjacent interior cell is used (even extension). */
static double stencil_value(const Orc *o, const double *q, int nx, int ny, int x, int y)
{
    if (x < 0 || x >= nx) x = (o->side_eta[SIDE_LEFT] == ORC_PERIODIC) ? (x + nx) % nx : (x < 0 ? 0 : nx - 1);
    if (y < 0 || y >= ny) y = (o->side_eta[SIDE_BOTTOM] == ORC_PERIODIC) ? (y + ny) % ny : (y < 0 ? 0 : ny - 1);
    return q[y * nx + x];
}

/* eq. pressure:gradient:alternative in lattice units:
 * grad^c q(x) = sum_i w_i c_i q(x + c_i) / c_s^2 with c_s^2 = 1/3. */
static void central_gradient(const Orc *o, const double *q, int nx, int ny, int x, int y, double out[2])
{
    double gx = 0.0, gy = 0.0;
    for (int i = 0; i < 9; i++) {
        double v = stencil_value(o, q, nx, ny, x + CX9[i], y + CY9[i]);
        gx += W9[i] * CX9[i] * v;
        gy += W9[i] * CY9[i] * v;
    }
    out[0] = 3.0 * gx;
    out[1] = 3.0 * gy;
}

/* Self-dependence force of eq. MG:selfdependence.  Reading R8: in lattice
 * units the part of the force that depends on the current iterate through
 * grad p is F_*(g) = (alpha^2 r / 2) grad^c D(g); it follows from
 * eqs. source:implicit and pressure:gradient and is the same on every level. */
static void fstar(Orc *o, Level *Lv, const double *g, double *Fs)
{
    const int nx = Lv->nx, ny = Lv->ny;
    ORC_PAR_FOR
    for (int c = 0; c < nx * ny; c++) Lv->D[c] = divergence_of(o, g + 8 * c);
    const double coef = 0.5 * o->P.alpha * o->P.alpha * o->P.r;
    ORC_PAR_FOR
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double gr[2];
            central_gradient(o, Lv->D, nx, ny, x, y, gr);
            Fs[2 * (y * nx + x) + 0] = coef * gr[0];
            Fs[2 * (y * nx + x) + 1] = coef * gr[1];
        }
}

/* One smoothing or residual evaluation: gout = ELASTIC_STEP(g - r, F~ + F_*(g)). */
static void step_of_iterate(Orc *o, Level *Lv, int fine, const double *g, const double *Ft, double *gout)
{
    const int n = Lv->nx * Lv->ny;
    fstar(o, Lv, g, Lv->F);
    if (Ft) for (int c = 0; c < 2 * n; c++) Lv->F[c] += Ft[c];
    ORC_PAR_FOR
    for (int c = 0; c < 8 * n; c++) Lv->gin[c] = g[c] - (Lv->r ? Lv->r[c] : 0.0);
    elastic_step(o, Lv, fine, Lv->gin, Lv->F, gout);
}

static double absmax_nan_inf(double v) { return (v == v) ? fabs(v) : INFINITY; }

enum { CYC_V = 0, CYC_W = 1, CYC_F = 2 };

/* Pre- and post-smoothing sweeps of level index l (0 = coarsest): K of Alg. 4,
 * or the per-level count (reading R23). */
static int sweeps_of(const Orc *o, int l)
{
    int k = o->P.K_level[o->L - 1 - l];
    return k > 0 ? k : o->P.K;
}

/* ELASTIC_MULTIGRID (Alg. 4) on level index l (0 = coarsest); the iterate
 * Lv->g is updated in place; Ft is NULL on coarse levels (zero explicit force).
 * kind selects how the coarse-grid correction problem is solved (reading R20):
 * by one cycle of Alg. 4 (V), by two in succession (W), or by an F-cycle
 * followed by a V-cycle (F). */
static void multigrid(Orc *o, int l, const double *Ft, int kind)
{
    Level *Lv = &o->lv[l];
    const int fine = (l == o->L - 1);
    const int n = Lv->nx * Lv->ny;
    const double gam = o->P.gamma;
    const int K = sweeps_of(o, l);
    /* pre-smoothing, eq. MG:smoother */
    for (int k = 0; k < K; k++) {
        step_of_iterate(o, Lv, fine, Lv->g, Ft, Lv->gout);
        ORC_PAR_FOR
        for (int c = 0; c < 8 * n; c++) Lv->g[c] = (1.0 - gam) * Lv->g[c] + gam * Lv->gout[c];
    }
    if (l > 0) {
        Level *Lc = &o->lv[l - 1];
        /* residual eq. LBM:residual and restriction eq. MG:restriction (full sum) */
        step_of_iterate(o, Lv, fine, Lv->g, Ft, Lv->gout);
        memset(Lc->r, 0, sizeof(double) * 8 * (size_t)(Lc->nx * Lc->ny));
        for (int y = 0; y < Lv->ny; y++)
            for (int x = 0; x < Lv->nx; x++) {
                int pc = (y / 2) * Lc->nx + (x / 2);
                for (int k = 0; k < 8; k++)
                    Lc->r[8 * pc + k] += Lv->g[8 * (y * Lv->nx + x) + k] - Lv->gout[8 * (y * Lv->nx + x) + k];
            }
        /* coarse-grid correction: ELASTIC_MULTIGRID(0, r^c, 0, f_*, l-1), homogeneous BCs */
        memset(Lc->g, 0, sizeof(double) * 8 * (size_t)(Lc->nx * Lc->ny));
        Lc->hist_valid = 0;
        if (kind == CYC_V) {
            multigrid(o, l - 1, NULL, CYC_V);
        } else if (kind == CYC_W) {
            multigrid(o, l - 1, NULL, CYC_W);
            multigrid(o, l - 1, NULL, CYC_W);
        } else {
            multigrid(o, l - 1, NULL, CYC_F);
            multigrid(o, l - 1, NULL, CYC_V);
        }
        /* prolongation P = R^T (copy of the coarse value to its four cells) */
        ORC_PAR_FOR
        for (int y = 0; y < Lv->ny; y++)
            for (int x = 0; x < Lv->nx; x++) {
                int pc = (y / 2) * Lc->nx + (x / 2);
                for (int k = 0; k < 8; k++) Lv->g[8 * (y * Lv->nx + x) + k] += Lc->g[8 * pc + k];
            }
    }
    /* post-smoothing; on the finest level the last sweep also yields the
     * residual max|g - ELASTIC_STEP(g, F)| of the iterate it starts from
     * (reading R16: the stopping test of the adaptive variant, §3.4) */
    for (int k = 0; k < K; k++) {
        step_of_iterate(o, Lv, fine, Lv->g, Ft, Lv->gout);
        if (fine && k == K - 1) {
            double res = 0.0, gn = 0.0, sq = 0.0;
            for (int c = 0; c < 8 * n; c++) {
                double a = absmax_nan_inf(Lv->g[c] - Lv->gout[c]);
                double b = absmax_nan_inf(Lv->g[c]);
                if (a > res) res = a;
                if (b > gn) gn = b;
                sq += (Lv->g[c] - Lv->gout[c]) * (Lv->g[c] - Lv->gout[c]);
            }
            o->last_res = res;
            o->last_gnorm = gn;
            o->last_res_l2 = sqrt(sq); /* the 2-norm of the same residual */
        }
        ORC_PAR_FOR
        for (int c = 0; c < 8 * n; c++) Lv->g[c] = (1.0 - gam) * Lv->g[c] + gam * Lv->gout[c];
    }
}

/* Full-sum restriction (eq. MG:restriction) of the defect g - gout of level l
 * into the right-hand side r of level l - 1. */
static void restrict_defect(Orc *o, int l)
{
    Level *Lv = &o->lv[l], *Lc = &o->lv[l - 1];
    memset(Lc->r, 0, sizeof(double) * 8 * (size_t)(Lc->nx * Lc->ny));
    for (int y = 0; y < Lv->ny; y++)
        for (int x = 0; x < Lv->nx; x++) {
            int pc = (y / 2) * Lc->nx + (x / 2);
            for (int k = 0; k < 8; k++)
                Lc->r[8 * pc + k] += Lv->g[8 * (y * Lv->nx + x) + k] - Lv->gout[8 * (y * Lv->nx + x) + k];
        }
}

/* Prolongation P = R^T of level l - 1's iterate into level l: the copy of each
 * coarse value to its four cells, added to (add = 1) or replacing the iterate. */
static void prolong_into(Orc *o, int l, int add)
{
    Level *Lv = &o->lv[l], *Lc = &o->lv[l - 1];
    ORC_PAR_FOR
    for (int y = 0; y < Lv->ny; y++)
        for (int x = 0; x < Lv->nx; x++) {
            int pc = (y / 2) * Lc->nx + (x / 2);
            for (int k = 0; k < 8; k++) {
                double v = Lc->g[8 * pc + k];
                Lv->g[8 * (y * Lv->nx + x) + k] = add ? Lv->g[8 * (y * Lv->nx + x) + k] + v : v;
            }
        }
}

/* One full-multigrid cycle on the correction problem of the finest iterate
 * (reading R21; nested iteration): the finest defect is restricted level by
 * level -- each coarse level passing on the defect of its zero iterate, so every
 * level holds the right-hand side of the cycle of Alg. 4 that would reach it --
 * the coarsest level is solved by its 2K sweeps from zero, then each finer level
 * starts from the prolongated solution of the level below and runs one cycle of
 * the chosen kind, and the finest level takes the prolongated correction and
 * one cycle. */
static void fmg_cycle(Orc *o, const double *Ft, int kind)
{
    const int L = o->L;
    if (L < 2) { multigrid(o, 0, Ft, kind); return; }
    Level *Lf = &o->lv[L - 1];
    step_of_iterate(o, Lf, 1, Lf->g, Ft, Lf->gout);
    restrict_defect(o, L - 1);
    for (int l = L - 2; l >= 1; l--) {
        Level *Lv = &o->lv[l];
        memset(Lv->g, 0, sizeof(double) * 8 * (size_t)(Lv->nx * Lv->ny));
        Lv->hist_valid = 0;
        step_of_iterate(o, Lv, 0, Lv->g, NULL, Lv->gout);
        restrict_defect(o, l);
    }
    Level *L0 = &o->lv[0];
    memset(L0->g, 0, sizeof(double) * 8 * (size_t)(L0->nx * L0->ny));
    L0->hist_valid = 0;
    multigrid(o, 0, NULL, CYC_V);
    for (int l = 1; l <= L - 2; l++) {
        prolong_into(o, l, 0);
        o->lv[l].hist_valid = 0;
        multigrid(o, l, NULL, kind);
    }
    prolong_into(o, L - 1, 1);
    multigrid(o, L - 1, Ft, kind);
}

/* ---------------------------------------------------------------------------
 * Coupling, §3.4.
 */

/* Explicit part of eq. source:implicit in lattice units (s' = dt s_eff):
 * dt s - (alpha/eps)[(1-r)(D(t-dt) - D(t-2dt)) - r D(t-dt)]; the missing
 * term -(alpha r/eps) D(tau, t) depends on the current iterate.  The fluid
 * body force g of eq. darcy is zero in this implementation. */
static void explicit_source(Orc *o)
{
    const int n = o->P.nx * o->P.ny;
    const double a = o->P.alpha / o->h, r = o->P.r;
    ORC_PAR_FOR
    for (int c = 0; c < n; c++)
        o->sexp[c] = o->P.dt * o->src[c] - a * ((1.0 - r) * (o->D1[c] - o->D2[c]) - r * o->D1[c]);
}

/* Full eq. source:implicit with the final divergence D(t). */
static double full_source(const Orc *o, int c)
{
    const double a = o->P.alpha / o->h, r = o->P.r;
    return o->P.dt * o->src[c] - a * ((1.0 - r) * (o->D1[c] - o->D2[c]) + r * (o->Dt[c] - o->D1[c]));
}

/* Explicit force F~ = eps^2 (f - alpha grad* p) with the grad p part of
 * eq. pressure:gradient that does not depend on the iterate:
 * F~ = c0 h^2 f - alpha h [ -3 omega sum_i f_i c_i + 1/2 grad^c s'_exp ]. */
static void explicit_force(Orc *o)
{
    const int nx = o->P.nx, ny = o->P.ny;
    if (o->P.pgrad) {  /* the zeroth moments, for eq. pressure:gradient:alternative */
        ORC_PAR_FOR
        for (int c = 0; c < nx * ny; c++) {
            double sum = 0.0;
            for (int i = 0; i < 9; i++) sum += o->f[9 * c + i];
            o->Pf[c] = sum;
        }
    }
    ORC_PAR_FOR
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            int c = y * nx + x;
            double gs[2], gpx, gpy;
            central_gradient(o, o->sexp, nx, ny, x, y, gs);
            if (o->P.pgrad) {
                /* reading R22: grad^c of p^ = sum f + s'/2 by the central difference of
                 * eq. pressure:gradient:alternative, the iterate-dependent part of s'
                 * kept in F_*(g) as with eq. pressure:gradient */
                double gP[2];
                central_gradient(o, o->Pf, nx, ny, x, y, gP);
                gpx = gP[0] + 0.5 * gs[0];
                gpy = gP[1] + 0.5 * gs[1];
            } else {
                double jx = 0.0, jy = 0.0;
                for (int i = 0; i < 9; i++) { jx += o->f[9 * c + i] * CX9[i]; jy += o->f[9 * c + i] * CY9[i]; }
                gpx = -3.0 * o->omega * jx + 0.5 * gs[0];
                gpy = -3.0 * o->omega * jy + 0.5 * gs[1];
            }
            o->Ft[2 * c + 0] = o->P.c0 * o->h * o->h * o->fbody[2 * c + 0] - o->P.alpha * o->h * gpx;
            o->Ft[2 * c + 1] = o->P.c0 * o->h * o->h * o->fbody[2 * c + 1] - o->P.alpha * o->h * gpy;
        }
}

/* ---------------------------------------------------------------------------
 * FLOW_STEP (Alg. 3).
 */
static double pull_flow(const Orc *o, int x, int y, int i)
{
    const int nx = o->P.nx, ny = o->P.ny;
    const int cx = CX9[i], cy = CY9[i];
    int sx = x - cx, sy = y - cy;
    if ((sx < 0 || sx >= nx) && o->side_p[SIDE_LEFT] == ORC_PERIODIC) sx = (sx + nx) % nx;
    if ((sy < 0 || sy >= ny) && o->side_p[SIDE_BOTTOM] == ORC_PERIODIC) sy = (sy + ny) % ny;
    int side = -1;
    if (sy < 0) side = SIDE_BOTTOM;
    else if (sy >= ny) side = SIDE_TOP;
    else if (sx < 0) side = SIDE_LEFT;
    else if (sx >= nx) side = SIDE_RIGHT;
    if (side < 0) return o->fs[9 * (sy * nx + sx) + i];
    if ((side == SIDE_BOTTOM || side == SIDE_TOP) && (sx < 0 || sx >= nx)) {
        int vert = sx < 0 ? SIDE_LEFT : SIDE_RIGHT;
        if (o->side_p[side] == ORC_SYMMETRY && o->side_p[vert] != ORC_SYMMETRY) side = vert;
    }
    const int type = o->side_p[side];
    const int iout = q9_index(-cx, -cy);
    if (type == ORC_SYMMETRY) {
        int mx = sx, my = sy, rcx = cx, rcy = cy;
        if (side == SIDE_BOTTOM || side == SIDE_TOP) {
            my = mirror(sy, ny); rcy = -cy;
            if (mx < 0 || mx >= nx) { mx = mirror(mx, nx); rcx = -cx; }
        } else {
            mx = mirror(sx, nx); rcx = -cx;
        }
        return o->fs[9 * (my * nx + mx) + q9_index(rcx, rcy)];
    }
    const double fo = o->fs[9 * (y * nx + x) + iout];
    if (type == ORC_NEUMANN) return fo; /* eq. BC:noFlow (halfway bounce-back) */
    /* ORC_DIRICHLET: eq. BC:pressure (halfway anti-bounce-back), p^ = c0 p */
    int kk = crossing_index(side, x, y, -cx, -cy);
    return -fo + 2.0 * W9[iout] * o->P.c0 * p_data(o, side, kk);
}

static void flow_step(Orc *o)
{
    const int nx = o->P.nx, ny = o->P.ny, n = nx * ny;
    const double om = o->omega;
    ORC_PAR_FOR
    for (int c = 0; c < n; c++) {
        double sp = full_source(o, c);
        double sum = 0.0;
        for (int i = 0; i < 9; i++) sum += o->f[9 * c + i];
        double p = sum + 0.5 * sp;                        /* eq. pressure */
        for (int i = 0; i < 9; i++) {
            double feq = W9[i] * p;                        /* eq. pressure:equilibrium */
            double S = (1.0 - 0.5 * om) * W9[i] * sp;      /* eq. pressure:collision:source */
            o->fs[9 * c + i] = o->f[9 * c + i] - om * (o->f[9 * c + i] - feq) + S; /* eq. pressure:collision */
        }
    }
    ORC_PAR_FOR
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++)
            for (int i = 0; i < 9; i++) o->fn[9 * (y * nx + x) + i] = pull_flow(o, x, y, i);
    double *tmp = o->f; o->f = o->fn; o->fn = tmp;
    ORC_PAR_FOR
    for (int c = 0; c < n; c++) { o->D2[c] = o->D1[c]; o->D1[c] = o->Dt[c]; }
    o->nstep += 1;
    o->t = o->P.dt * (double)o->nstep;
}

/* ---------------------------------------------------------------------------
 * Initial conditions, eqs. ICs and ICs:moments (p(0) = 0, eta(0) = 0):
 * f_i = -(dt/2) w_i s(0) and g = T m0 with m0_10,01 = -F_eff(0)/2,
 * m0_12,21 = -F_eff(0)/6, other moments 0, F_eff(0) = c0 h^2 f(0).
 */
static void initial_conditions(Orc *o)
{
    const int n = o->P.nx * o->P.ny;
    Level *Lf = &o->lv[o->L - 1];
    for (int c = 0; c < n; c++) {
        double s0 = o->P.dt * o->src[c];
        for (int i = 0; i < 9; i++) o->f[9 * c + i] = -0.5 * W9[i] * s0;
        double Fx = o->P.c0 * o->h * o->h * o->fbody[2 * c], Fy = o->P.c0 * o->h * o->h * o->fbody[2 * c + 1];
        double m0[8] = {-0.5 * Fx, -0.5 * Fy, 0.0, 0.0, 0.0, -Fx / 6.0, -Fy / 6.0, 0.0};
        for (int k = 0; k < 8; k++) {
            double v = 0.0;
            for (int nu = 0; nu < 8; nu++) v += TINV[k][nu] * m0[nu];
            Lf->g[8 * c + k] = v;
        }
    }
    o->initialized = 1;
}

/* Elasticity update of Alg. 5 at the current time t. */
static int elastic_solve(Orc *o)
{
    Level *Lf = &o->lv[o->L - 1];
    const int n = o->P.nx * o->P.ny;
    explicit_source(o);
    explicit_force(o);
    Lf->hist_valid = 0;
    int ne = 0, status = 0;
    for (;;) {
        if (ne == 0 && o->P.fmg) fmg_cycle(o, o->Ft, o->P.cycle);
        else multigrid(o, o->L - 1, o->Ft, o->P.cycle);
        ne++;
        o->total_cycles++;
        if (!isfinite(o->last_res)) { o->diverged = 1; status = -3; break; }
        if (o->P.ne_fixed > 0) { if (ne >= o->P.ne_fixed) break; continue; }
        double thr = o->P.tol * (o->last_gnorm > 1.0 ? o->last_gnorm : 1.0);
        if (o->last_res <= thr) break;
        if (ne >= o->P.ne_max) { o->notconv_steps++; status = -4; break; }
    }
    o->last_ne = ne;
    ORC_PAR_FOR
    for (int c = 0; c < n; c++) o->Dt[c] = divergence_of(o, Lf->g + 8 * c);
    o->solved = 1;
    return status;
}

/* ---------------------------------------------------------------------------
 * Public entry points (loaded through ctypes by the tests).
 */
static int validate(const orc_params *p, const orc_side s[4])
{
    if (!p || !s) return -1;
    if (p->nx <= 0 || p->ny <= 0 || p->levels < 1 || p->levels > ORC_MAX_LEVELS || p->K < 1) return -1;
    int div = 1 << (p->levels - 1);
    if (p->nx % div || p->ny % div) return -1;
    if (!(p->lx > 0 && p->ly > 0) || fabs(p->lx / p->nx - p->ly / p->ny) > 1e-12 * (p->lx / p->nx)) return -1;
    if (!(p->c0 > 0 && p->kappa > 0 && p->dt > 0 && p->lambda + p->mu > 0 && p->mu > 0)) return -1;
    if (!(p->gamma > 0 && p->gamma <= 1) || p->r < 0 || p->r > 1) return -1;
    if (p->cycle < 0 || p->cycle > 2 || (p->fmg != 0 && p->fmg != 1) || (p->pgrad != 0 && p->pgrad != 1)) return -1;
    for (int j = 0; j < ORC_MAX_LEVELS; j++) if (p->K_level[j] > 64) return -1;
    for (int pair = 0; pair < 2; pair++) {
        int a = pair, b = pair + 2;
        if ((s[a].eta_type == ORC_PERIODIC) != (s[b].eta_type == ORC_PERIODIC)) return -1;
        if ((s[a].p_type == ORC_PERIODIC) != (s[b].p_type == ORC_PERIODIC)) return -1;
        if ((s[a].eta_type == ORC_PERIODIC) != (s[a].p_type == ORC_PERIODIC)) return -1;
    }
    return 0;
}

void orc_destroy(void *h);

/* Threads of the per-cell loops (1 = serial, the default); results do not
 * depend on it. */
void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return orc_threads; }
int orc_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

void *orc_create(const orc_params *p, const orc_side sides[4])
{
    if (validate(p, sides)) return NULL;
    Orc *o = (Orc *)calloc(1, sizeof(Orc));
    o->P = *p;
    o->L = p->levels;
    o->h = p->lx / p->nx;
    o->lam = p->c0 * p->lambda;
    o->mu = p->c0 * p->mu;
    o->kap = p->dt * p->kappa / (p->c0 * o->h * o->h);
    o->omega = 1.0 / (3.0 * o->kap + 0.5); /* eq. pressure:rate, c_s^2 = 1/3, dt = 1 */
    o->om_s = 2.0 / (3.0 * (o->lam + o->mu) + 1.0);
    o->om_d = 2.0 / (6.0 * o->mu + 1.0);
    for (int s = 0; s < 4; s++) {
        o->side_eta[s] = sides[s].eta_type;
        o->side_p[s] = sides[s].p_type;
        int m = 2 * side_len(o, s) + 1;
        if (sides[s].eta_profile) {
            o->eta_prof[s] = (double *)malloc(sizeof(double) * 2 * m);
            memcpy(o->eta_prof[s], sides[s].eta_profile, sizeof(double) * 2 * m);
        }
        if (sides[s].p_profile) {
            o->p_prof[s] = (double *)malloc(sizeof(double) * m);
            memcpy(o->p_prof[s], sides[s].p_profile, sizeof(double) * m);
        }
    }
    for (int l = 0; l < o->L; l++) {
        Level *Lv = &o->lv[l];
        int shift = o->L - 1 - l;
        Lv->nx = p->nx >> shift;
        Lv->ny = p->ny >> shift;
        size_t n = (size_t)Lv->nx * Lv->ny;
        Lv->g = (double *)calloc(8 * n, sizeof(double));
        Lv->r = (l == o->L - 1) ? NULL : (double *)calloc(8 * n, sizeof(double));
        Lv->gin = (double *)calloc(8 * n, sizeof(double));
        Lv->gs = (double *)calloc(8 * n, sizeof(double));
        Lv->gout = (double *)calloc(8 * n, sizeof(double));
        Lv->H = (double *)calloc(8 * n, sizeof(double));
        Lv->F = (double *)calloc(2 * n, sizeof(double));
        Lv->D = (double *)calloc(n, sizeof(double));
    }
    size_t n = (size_t)p->nx * p->ny;
    o->f = (double *)calloc(9 * n, sizeof(double));
    o->fs = (double *)calloc(9 * n, sizeof(double));
    o->fn = (double *)calloc(9 * n, sizeof(double));
    o->D1 = (double *)calloc(n, sizeof(double));
    o->D2 = (double *)calloc(n, sizeof(double));
    o->Dt = (double *)calloc(n, sizeof(double));
    o->sexp = (double *)calloc(n, sizeof(double));
    o->Pf = (double *)calloc(n, sizeof(double));
    o->Ft = (double *)calloc(2 * n, sizeof(double));
    o->fbody = (double *)calloc(2 * n, sizeof(double));
    o->src = (double *)calloc(n, sizeof(double));
    if (!o->f || !o->fn || !o->src || !o->lv[o->L - 1].H) { orc_destroy(o); return NULL; }
    return o;
}

void orc_destroy(void *h)
{
    Orc *o = (Orc *)h;
    if (!o) return;
    for (int l = 0; l < ORC_MAX_LEVELS; l++) {
        Level *Lv = &o->lv[l];
        free(Lv->g); free(Lv->r); free(Lv->gin); free(Lv->gs); free(Lv->gout);
        free(Lv->H); free(Lv->F); free(Lv->D);
    }
    for (int s = 0; s < 4; s++) { free(o->eta_prof[s]); free(o->p_prof[s]); }
    free(o->f); free(o->fs); free(o->fn); free(o->D1); free(o->D2); free(o->Dt);
    free(o->sexp); free(o->Pf); free(o->Ft); free(o->fbody); free(o->src);
    free(o);
}

/* Body force f (2 per cell, dimensional) and fluid source s (1 per cell);
 * either may be NULL (zero).  They apply from the next elastic solve on. */
int orc_set_sources(void *h, const double *fbody, const double *src)
{
    Orc *o = (Orc *)h;
    size_t n = (size_t)o->P.nx * o->P.ny;
    if (fbody) memcpy(o->fbody, fbody, sizeof(double) * 2 * n); else memset(o->fbody, 0, sizeof(double) * 2 * n);
    if (src) memcpy(o->src, src, sizeof(double) * n); else memset(o->src, 0, sizeof(double) * n);
    o->solved = 0; /* the elastic solve at the current time must see the new data */
    return 0;
}

/* n iterations of the time loop of Alg. 5, followed by the elasticity update
 * at the final time so that displacement and pressure refer to the same t
 * (reading R15).  Returns 0, -3 (diverged) or -4 (a step hit ne_max). */
int orc_step(void *h, int nsteps)
{
    Orc *o = (Orc *)h;
    int status = 0, st;
    if (!o->initialized) initial_conditions(o);
    for (int i = 0; i < nsteps; i++) {
        if (!o->solved) { st = elastic_solve(o); if (st == -3) return st; if (st) status = st; }
        flow_step(o);
        o->solved = 0;
    }
    if (!o->solved) { st = elastic_solve(o); if (st == -3) return st; if (st) status = st; }
    return status;
}

int orc_solve_to(void *h, double T)
{
    Orc *o = (Orc *)h;
    long target = (long)floor(T / o->P.dt + 0.5);
    long n = target - o->nstep;
    if (n < 0) return -1;
    return orc_step(h, (int)n);
}

/* Displacement eta = (mbar_10, mbar_01), eq. displacement, with
 * mbar = m + F/2 and F = F~ + F_*(g) of the final iterate. eta: [2][ny][nx]. */
int orc_read_u(void *h, double *eta, double *t_out)
{
    Orc *o = (Orc *)h;
    Level *Lf = &o->lv[o->L - 1];
    const int n = o->P.nx * o->P.ny;
    if (!o->initialized) initial_conditions(o);
    if (!o->solved) elastic_solve(o);
    fstar(o, Lf, Lf->g, Lf->F);
    for (int c = 0; c < n; c++) {
        eta[c] = raw_moment(Lf->g + 8 * c, 1, 0) + 0.5 * (o->Ft[2 * c] + Lf->F[2 * c]);
        eta[n + c] = raw_moment(Lf->g + 8 * c, 0, 1) + 0.5 * (o->Ft[2 * c + 1] + Lf->F[2 * c + 1]);
    }
    if (t_out) *t_out = o->t;
    return 0;
}

/* Pressure p = (sum_i f_i + s'/2) / c0, eq. pressure, with s' of eq.
 * source:implicit at the final divergence. p: [ny][nx]. */
int orc_read_p(void *h, double *p, double *t_out)
{
    Orc *o = (Orc *)h;
    const int n = o->P.nx * o->P.ny;
    if (!o->initialized) initial_conditions(o);
    if (!o->solved) elastic_solve(o);
    for (int c = 0; c < n; c++) {
        double sum = 0.0;
        for (int i = 0; i < 9; i++) sum += o->f[9 * c + i];
        p[c] = (sum + 0.5 * full_source(o, c)) / o->P.c0;
    }
    if (t_out) *t_out = o->t;
    return 0;
}

/* Stress, eq. displacement with eq. moments:bared, converted from lattice
 * stress (c0 h sigma) to sigma. sigma: [3][ny][nx] = (11, 12, 22). */
int orc_read_stress(void *h, double *sigma)
{
    Orc *o = (Orc *)h;
    Level *Lf = &o->lv[o->L - 1];
    const int n = o->P.nx * o->P.ny;
    if (!o->initialized) initial_conditions(o);
    if (!o->solved) elastic_solve(o);
    const double lm = o->lam + o->mu;
    const double scale = 1.0 / (o->P.c0 * o->h);
    for (int c = 0; c < n; c++) {
        const double *g = Lf->g + 8 * c;
        double m20 = raw_moment(g, 2, 0), m02 = raw_moment(g, 0, 2), m11 = raw_moment(g, 1, 1);
        double mbs = 3.0 * lm / (3.0 * lm + 1.0) * (m20 + m02);
        double mbd = 6.0 * o->mu / (6.0 * o->mu + 1.0) * (m20 - m02);
        double mb11 = 6.0 * o->mu / (6.0 * o->mu + 1.0) * m11;
        sigma[c] = -0.5 * (mbs + mbd) * scale;
        sigma[n + c] = -0.5 * 2.0 * mb11 * scale;
        sigma[2 * n + c] = -0.5 * (mbs - mbd) * scale;
    }
    return 0;
}

typedef struct {
    int last_ne;
    double last_res;
    long total_cycles;
    int notconv_steps;
    int diverged;
    long nstep;
    double t;
    double omega, om_s, om_d, kap_lattice;
    double last_res_l2;
} orc_stats;

int orc_stats_get(void *h, orc_stats *s)
{
    Orc *o = (Orc *)h;
    s->last_ne = o->last_ne;
    s->last_res = o->last_res;
    s->total_cycles = o->total_cycles;
    s->notconv_steps = o->notconv_steps;
    s->diverged = o->diverged;
    s->nstep = o->nstep;
    s->t = o->t;
    s->omega = o->omega;
    s->om_s = o->om_s;
    s->om_d = o->om_d;
    s->kap_lattice = o->kap;
    s->last_res_l2 = o->last_res_l2;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Component access for the pins (tests only).
 */

/* Post-collision populations of one cell for given material (lattice units). */
void orc_collide_cell(double lam_hat, double mu_hat, const double g[8], const double F[2], double gs[8])
{
    Orc o;
    memset(&o, 0, sizeof(o));
    o.lam = lam_hat;
    o.mu = mu_hat;
    o.om_s = 2.0 / (3.0 * (lam_hat + mu_hat) + 1.0);
    o.om_d = 2.0 / (6.0 * mu_hat + 1.0);
    collide(&o, g, F, gs);
}

void orc_inverse_table(double out[64]) { memcpy(out, TINV, sizeof(TINV)); }

void orc_velocities(int cx8[8], int cy8[8], int cx9[9], int cy9[9], double w9[9])
{
    memcpy(cx8, CX8, sizeof(CX8)); memcpy(cy8, CY8, sizeof(CY8));
    memcpy(cx9, CX9, sizeof(CX9)); memcpy(cy9, CY9, sizeof(CY9)); memcpy(w9, W9, sizeof(W9));
}

/* Prepare the explicit force of the current time (as the elastic solve does). */
int orc_prepare_elastic(void *h)
{
    Orc *o = (Orc *)h;
    if (!o->initialized) initial_conditions(o);
    explicit_source(o);
    explicit_force(o);
    return 0;
}

/* Fixed-point map of the finest level with halfway (undelayed) Dirichlet
 * bounce-back: out = ELASTIC_STEP(g, F~ + F_*(g)). */
int orc_fixed_point_map(void *h, const double *g, double *out)
{
    Orc *o = (Orc *)h;
    Level *Lf = &o->lv[o->L - 1];
    Lf->hist_valid = 0;
    step_of_iterate(o, Lf, 1, g, o->Ft, out);
    Lf->hist_valid = 0;
    return 0;
}

/* One V-cycle on the finest level with the prepared F~; returns the residual
 * measured in its last smoothing sweep. */
double orc_vcycle(void *h, int reset_history)
{
    Orc *o = (Orc *)h;
    if (reset_history) o->lv[o->L - 1].hist_valid = 0;
    multigrid(o, o->L - 1, o->Ft, o->P.cycle);
    return o->last_res;
}

/* One plain (non-multigrid) pseudo-time step of Alg. 1 on the finest level. */
int orc_plain_pseudo_step(void *h)
{
    Orc *o = (Orc *)h;
    Level *Lf = &o->lv[o->L - 1];
    step_of_iterate(o, Lf, 1, Lf->g, o->Ft, Lf->gout);
    memcpy(Lf->g, Lf->gout, sizeof(double) * 8 * (size_t)(Lf->nx * Lf->ny));
    return 0;
}

int orc_get_g(void *h, double *g)
{
    Orc *o = (Orc *)h;
    Level *Lf = &o->lv[o->L - 1];
    memcpy(g, Lf->g, sizeof(double) * 8 * (size_t)(Lf->nx * Lf->ny));
    return 0;
}
int orc_set_g(void *h, const double *g)
{
    Orc *o = (Orc *)h;
    Level *Lf = &o->lv[o->L - 1];
    memcpy(Lf->g, g, sizeof(double) * 8 * (size_t)(Lf->nx * Lf->ny));
    o->solved = 0;
    return 0;
}
int orc_get_f(void *h, double *f)
{
    Orc *o = (Orc *)h;
    memcpy(f, o->f, sizeof(double) * 9 * (size_t)(o->P.nx * o->P.ny));
    return 0;
}
int orc_set_f(void *h, const double *f)
{
    Orc *o = (Orc *)h;
    memcpy(o->f, f, sizeof(double) * 9 * (size_t)(o->P.nx * o->P.ny));
    o->initialized = 1;
    o->solved = 0;
    return 0;
}
