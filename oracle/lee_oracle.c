/*
 * lee_oracle.c -- plain, slow FP64 CPU oracle of the ghost-point immersed
 * boundary / ADE impedance / 2D linearized Euler method of
 * "A high-order ghost-point immersed boundary method coupled with auxiliary
 * differential equations for time-domain impedance walls".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; it is written from the paper.
 *
 * Every routine follows the paper's steps in its order and notation:
 *   Sec. 2.1  Eq. 1            linearized Euler equations (rho0 = c0 = 1)
 *   Sec. 2.2  Eq. DRP_s        7-point DRP first derivative (antisymmetric)
 *   Sec. 2.3-2.5               MSD impedance, poles, residues, ADE states
 *   Sec. 3.1  Eqs. ns-rotation, ns-ellipse, ns-poly2d .. ns-readout, ns-ghost
 *   Sec. 3.2                   six coupling steps per RK stage per ghost point
 * Readings where the paper is silent:
 *   RK coefficients: 2N-storage Jameson alpha = (1/4, 1/3, 1/2, 1); a classical
 *   Butcher RK4 mode is kept for cross-checks.  The source time factor enters
 *   each stage as the moment of sin(w t) over the step that keeps the scheme
 *   4th order (stage_forcing).  One-sided stencils in the three outer layers:
 *   the 7-point one-sided DRP stencils of Tam and Webb (J. Comput. Phys. 107,
 *   1993), the scheme the paper cites for its boundary rows (Sec. 2.2), on
 *   nodes 0..6 from the edge.  Radiation condition of Tam and Webb in the three
 *   outer layers (Secs. 4.1-4.2): dq/dt = -(cos th dq/dx + sin th dq/dy +
 *   q/(2 rho)), polar about the domain centre, no source there; where a wall
 *   meets the band, a derivative whose 7-node window holds a non-fluid node is
 *   left out of the condition (its one-sided row would otherwise feed ghost
 *   values from clouds clipped by the box back into the node).  The paper adds
 *   no damping (Sec. 4.3); an absorbing ramp over the W outer layers (rate
 *   (kappa/h) ((W - d)/W)^2 at distance d from the edge) is available as an
 *   opt-in departure (orc_set_sponge), off by default, for runs longer than
 *   this closure stays stable: its semi-discrete operator has eigenvalues with
 *   a small positive real part (grid-scale modes at the band).  Normal n points from the wall into the fluid;
 *   u_n (positive into the wall) = -u.n, so the Dirichlet datum for w = u.n is
 *   -u_n and the Neumann datum for dp/dn is +du_n/dt.  Critical damping uses
 *   the double-pole (Jordan) form of the same admittance.  A cloud clipped by
 *   the domain edge lowers the fit degree k = m from 4 step by step; one that
 *   cannot carry a plane (nodes on a single line) takes the constant fit (the
 *   cloud mean) with a linear normal extrapolation (m = 1).
 * Parity unpinned: none of the functions below (each has a pin in the tests).
 * The one-sided stencil rows are pinned by their Taylor moments and by
 * polynomial exactness; the band as a whole (one-sided rows + radiation
 * condition) by the free-field Gaussian pulse against its exact solution.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#define ORC_MAXCL 160
#define ORC_MAXPOLE 8

/* ---------------------------------------------------------------- types */
typedef struct {
    int target;                 /* storage index of the ghost node            */
    double bpx, bpy;            /* boundary point BP (Sec. 3.1)               */
    double nx, ny;              /* wall normal, wall -> fluid                 */
    double r;                   /* r = d / h, d = |GP - BP|                   */
    int m;                      /* extrapolation degree m (= k, or 1 if k = 0) */
    int k;                      /* degree of the cloud fit actually used       */
    int ncl;                    /* cloud size N                               */
    int cl[ORC_MAXCL];          /* cloud storage indices                      */
    double *L;                  /* (m+1) x ncl read-out rows at P_0..P_m      */
    double c[5];                /* Dirichlet factors c_i(r), Eq. ns-ghost     */
    double ct[5];               /* Neumann factors  c~_i(r), Eq. ns-ghost     */
    double ell[5];              /* free extrapolation: Q(-r) = sum ell_i f_i  */
} orc_ghost;

typedef struct {
    int nx, ny;
    double h, cfl, dt, x0, y0;
    int per_x, per_y;
    int wall;                   /* 0 none, 1 line, 2 cylinder */
    double wa, wb, wc;          /* line: point, angle / cylinder: centre, radius */
    int rigid;
    double R, M, K;
    int regime;                 /* 0 rigid, 1 complex pair, 2 real poles, 3 double pole, 4 rational */
    double A[2][2], bv[2], cv[2];
    /* general rational admittance (Eq. Yrational): N real poles lam_k with
     * residues A_k, M complex pairs s_k = al_k + i be_k with q_k = B_k + i C_k */
    int nreal, npair;
    double lam[ORC_MAXPOLE], Ares[ORC_MAXPOLE];
    double al[ORC_MAXPOLE], be[ORC_MAXPOLE], Bres[ORC_MAXPOLE], Cres[ORC_MAXPOLE];
    int ns;                     /* ADE states per ghost: 2 (MSD, rigid) or N + 2M */
    double s_amp, s_x, s_y, s_b, s_omega;
    unsigned char *kind;        /* 0 solid, 1 fluid, 2 ghost */
    double *q[3];               /* Q^n: p, u, v */
    int ng;
    orc_ghost *g;
    double *X;                  /* ADE state X^n, ng x 2 */
    long step;
    int nprobe;
    int *pidx;                  /* nprobe x 16 */
    double *pw;                 /* nprobe x 16 */
    double *phist;              /* pcap x nprobe */
    long pcap, prec;
    int n_reduced;              /* ghosts whose degree was lowered */
    const double *bc_override;  /* test hook: (w_BP, dp/dn_BP) per ghost */
    int f32_storage;            /* emulate FP32 storage of the field (tolerance studies) */
    int sponge_w;               /* opt-in absorbing ramp: width in cells (0 = off) */
    double sponge_k;            /* and strength kappa (rate kappa / h at the edge) */
    double *work;               /* stage work arrays of orc_run (allocated once) */
    size_t work_n;
    char err[256];
} orc_t;

/* DRP coefficients, Sec. 2.2 (a_{-k} = -a_k) */
static const double ORC_A1 = 0.770882380518;
static const double ORC_A2 = -0.166705904415;
static const double ORC_A3 = 0.020843142770;

/* ------------------------------------------------------------ creation */
orc_t *orc_create(int nx, int ny, double h, double cfl, double x0, double y0,
                  int per_x, int per_y)
{
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    o->nx = nx; o->ny = ny; o->h = h; o->cfl = cfl; o->dt = cfl * h;
    o->x0 = x0; o->y0 = y0; o->per_x = per_x; o->per_y = per_y;
    o->rigid = 1;
    size_t n = (size_t)nx * ny;
    o->kind = (unsigned char *)calloc(n, 1);
    for (int f = 0; f < 3; f++) o->q[f] = (double *)calloc(n, sizeof(double));
    return o;
}

static void orc_free_ghosts(orc_t *o)
{
    if (o->g) {
        for (int i = 0; i < o->ng; i++) free(o->g[i].L);
        free(o->g);
    }
    o->g = NULL;
    free(o->X); o->X = NULL;
    o->ng = 0;
}

void orc_destroy(orc_t *o)
{
    if (!o) return;
    orc_free_ghosts(o);
    free(o->kind);
    for (int f = 0; f < 3; f++) free(o->q[f]);
    free(o->pidx); free(o->pw); free(o->phist);
    free(o->work);
    free(o);
}

const char *orc_error(orc_t *o) { return o->err; }

/* Reduced-storage emulation: round the stored field (stage results, ghost
 * values, initial field) as any implementation that keeps the bulk field in a
 * narrower format must.  mode 1: single precision (the FP32 error floor);
 * mode 2: bfloat16, 8 significant bits rounded to nearest even, single
 * precision's exponent range (subnormals on the 2^-133 grid; no value here
 * comes near the overflow limit), for the storage-precision study. */
void orc_set_f32_storage(orc_t *o, int on) { o->f32_storage = on; }
static double round_bf16(double v)
{
    if (v == 0.0 || !isfinite(v)) return v;
    if (fabs(v) < 0x1p-126) return nearbyint(v * 0x1p133) * 0x1p-133;   /* subnormal grid, 2^-133 */
    int e;
    double m = frexp(v, &e);            /* v = m 2^e, 0.5 <= |m| < 1 */
    m = nearbyint(m * 256.0) / 256.0;   /* 8 significant bits, ties to even */
    return ldexp(m, e);
}
static double stored(const orc_t *o, double v)
{
    if (o->f32_storage == 1) return (double)(float)v;
    if (o->f32_storage == 2) return round_bf16(v);
    return v;
}

/* Opt-in absorbing ramp over the `width` outer layers of every non-periodic
 * edge, damping rate (kappa / h) ((width - d) / width)^2 at distance d < width
 * cells; width = 0 turns it off (the default, as in the paper). */
void orc_set_sponge(orc_t *o, int width, double kappa) { o->sponge_w = width > 0 ? width : 0; o->sponge_k = kappa; }

void orc_set_none(orc_t *o) { o->wall = 0; }
void orc_set_line(orc_t *o, double xw, double yw, double angle)
{ o->wall = 1; o->wa = xw; o->wb = yw; o->wc = angle; }
void orc_set_cylinder(orc_t *o, double xc, double yc, double rad)
{ o->wall = 2; o->wa = xc; o->wb = yc; o->wc = rad; }
void orc_set_rigid(orc_t *o) { o->rigid = 1; o->nreal = o->npair = 0; }
void orc_set_msd(orc_t *o, double R, double M, double K)
{ o->rigid = 0; o->R = R; o->M = M; o->K = K; o->nreal = o->npair = 0; }

/* General rational admittance of Eq. Yrational with Y_inf = 0: nreal real
 * poles lam[k] < 0 with real residues A[k], npair complex-conjugate pairs
 * s_k = al[k] + i be[k] (al < 0, be > 0) with residues q_k = B[k] + i C[k];
 * nreal + 2 npair <= ORC_MAXPOLE states per ghost (Eq. ADEgeneral).
 * Returns 0, or -1 for counts out of range. */
int orc_set_rational(orc_t *o, int nreal, const double *lam, const double *A,
                     int npair, const double *al, const double *be, const double *B, const double *C)
{
    if (nreal < 0 || npair < 0 || nreal + 2 * npair < 1 || nreal + 2 * npair > ORC_MAXPOLE) return -1;
    o->rigid = 0; o->nreal = nreal; o->npair = npair;
    for (int k = 0; k < nreal; k++) { o->lam[k] = lam[k]; o->Ares[k] = A[k]; }
    for (int k = 0; k < npair; k++) { o->al[k] = al[k]; o->be[k] = be[k]; o->Bres[k] = B[k]; o->Cres[k] = C[k]; }
    return 0;
}
void orc_set_monopole(orc_t *o, double xs, double ys, double amp, double w, double omega)
{
    o->s_amp = amp; o->s_x = xs; o->s_y = ys; o->s_omega = omega;
    o->s_b = log(2.0) / (w * w);           /* b = ln 2 / w^2, Sec. 4.3 */
}

static double node_x(const orc_t *o, int i) { return o->x0 + i * o->h; }
static double node_y(const orc_t *o, int j) { return o->y0 + j * o->h; }

/* Fluid test of the wall geometry, evaluated exactly as written. */
static int is_fluid_xy(const orc_t *o, double x, double y)
{
    if (o->wall == 1) {
        double nx = -sin(o->wc), ny = cos(o->wc);
        double phi = (x - o->wa) * nx + (y - o->wb) * ny;
        return phi > 0.0;
    }
    if (o->wall == 2) {
        double dx = x - o->wa, dy = y - o->wb;
        return dx * dx + dy * dy > o->wc * o->wc;
    }
    return 1;
}

/* ------------------------------------------------- MSD impedance, Sec. 2.5 */
static void orc_ade_coeffs(int rigid, double R, double M, double K,
                           int *regime, double A[2][2], double bv[2], double cv[2])
{
    memset(A, 0, 4 * sizeof(double)); bv[0] = bv[1] = 0; cv[0] = cv[1] = 0;
    if (rigid) { *regime = 0; return; }          /* Y -> 0: u_n == 0, Sec. 2.4 */
    double a = R / (2.0 * M);
    double disc = a * a - K / M;                 /* (R/2M)^2 - K/M */
    if (fabs(disc) <= 1e-10 * a * a) {
        /* double pole lambda = -R/2M: Y = (1/M)[1/(s-l) + l/(s-l)^2];
         * Phi1' = l Phi1 + p, Phi2' = l Phi2 + Phi1, u_n = (Phi1 + l Phi2)/M */
        double l = -a;
        *regime = 3;
        A[0][0] = l; A[0][1] = 0; A[1][0] = 1; A[1][1] = l;
        bv[0] = 1; bv[1] = 0;
        cv[0] = 1.0 / M; cv[1] = l / M;
    } else if (disc < 0) {
        /* s1 = -a + i beta; q1 = s1 / [M (s1 - s2)] = B1 + i C1 */
        double beta = sqrt(-disc);
        double s1r = -a, s1i = beta;
        double dr = 0.0, di = 2.0 * beta;        /* s1 - s2 */
        double den = M * (dr * dr + di * di);
        double B1 = (s1r * dr + s1i * di) / den;
        double C1 = (s1i * dr - s1r * di) / den;
        *regime = 1;
        A[0][0] = -a; A[0][1] = -beta; A[1][0] = beta; A[1][1] = -a;
        bv[0] = 1; bv[1] = 0;
        cv[0] = 2.0 * B1; cv[1] = -2.0 * C1;     /* u_n = 2B1 Psi1 - 2C1 Psi2 */
    } else {
        /* two real poles, residues A_k = l_k / [M (l_k - l_other)] */
        double sq = sqrt(disc);
        double l1 = -a + sq, l2 = -a - sq;
        *regime = 2;
        A[0][0] = l1; A[1][1] = l2;
        bv[0] = 1; bv[1] = 1;
        cv[0] = l1 / (M * (l1 - l2));
        cv[1] = l2 / (M * (l2 - l1));
    }
}

int orc_ade_regime(double R, double M, double K, double *out_A, double *out_b, double *out_c)
{
    int reg; double A[2][2], b[2], c[2];
    orc_ade_coeffs(0, R, M, K, &reg, A, b, c);
    out_A[0] = A[0][0]; out_A[1] = A[0][1]; out_A[2] = A[1][0]; out_A[3] = A[1][1];
    out_b[0] = b[0]; out_b[1] = b[1]; out_c[0] = c[0]; out_c[1] = c[1];
    return reg;
}

/* RK4 stability polynomial modulus at z = pole * dt (complex). */
static double rk4_mod(double zr, double zi)
{
    /* P(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, Horner in complex arithmetic */
    double pr = 1.0 / 24.0, pi = 0.0;
    double cs[4] = {1.0 / 6.0, 0.5, 1.0, 1.0};
    for (int k = 0; k < 4; k++) {
        double tr = pr * zr - pi * zi, ti = pr * zi + pi * zr;
        pr = tr + cs[k]; pi = ti;
    }
    return sqrt(pr * pr + pi * pi);
}

/* Returns max |P(pole dt)| over the admittance poles (0 for a rigid wall). */
double orc_ade_stability(double R, double M, double K, double dt)
{
    double a = R / (2.0 * M);
    double disc = a * a - K / M;
    if (disc < 0) return rk4_mod(-a * dt, sqrt(-disc) * dt);
    double sq = sqrt(disc);
    double m1 = rk4_mod((-a + sq) * dt, 0.0), m2 = rk4_mod((-a - sq) * dt, 0.0);
    return m1 > m2 ? m1 : m2;
}

static double ipow_d(double x, int e) { double r = 1.0; while (e-- > 0) r *= x; return r; }

/* ------------------------------------------------- stage forcing */
/*
 * Forcing value used by stage k (k = 1..4) of the 2N-storage scheme for a
 * prescribed time factor phi(t) = sin(omega t).  Expanding the four stages,
 * the forcing enters Q(n+1) as dt f4 + dt^2/2 L f3 + dt^3/6 L^2 f2 + dt^4/24 L^3 f1,
 * while the exact solution has sum_j L^j int_0^dt (dt-s)^j / j! phi(tn+s) ds.
 * Matching term by term gives f_k = (j+1)!/dt^(j+1) int_0^dt (dt-s)^j/j! phi
 * with j = 4 - k, which keeps the scheme 4th order with a time-dependent
 * source.  The integral is evaluated by 8-point Gauss-Legendre quadrature.
 */
static const double GL8_X[4] = {0.1834346424956498, 0.5255324099163290,
                                0.7966664774136267, 0.9602898564975363};
static const double GL8_W[4] = {0.3626837833783620, 0.3137066458778873,
                                0.2223810344533745, 0.1012285362903763};

static double stage_forcing(double omega, double tn, double dt, int k)
{
    int j = 4 - k;
    double fact = 1.0, jf = 1.0;
    for (int i = 2; i <= j + 1; i++) fact *= i;      /* (j+1)! */
    for (int i = 2; i <= j; i++) jf *= i;            /* j!     */
    double acc = 0.0;
    for (int q = 0; q < 8; q++) {
        double xq = q < 4 ? -GL8_X[3 - q] : GL8_X[q - 4];
        double wq = q < 4 ? GL8_W[3 - q] : GL8_W[q - 4];
        double sq = 0.5 * dt * (1.0 + xq);
        acc += wq * ipow_d(dt - sq, j) / jf * sin(omega * (tn + sq));
    }
    acc *= 0.5 * dt;
    return fact / ipow_d(dt, j + 1) * acc;
}

double orc_stage_forcing(double omega, double tn, double dt, int k)
{ return stage_forcing(omega, tn, dt, k); }

/* ------------------------------------------------------------ setup */
/* Lagrange basis on nodes sg[0..m]: value and derivative of basis i at s
 * (extended precision, rounded to FP64 by the caller). */
static long double lag_val(const long double *sg, int m, int i, long double s)
{
    long double v = 1.0L;
    for (int j = 0; j <= m; j++) if (j != i) v *= (s - sg[j]) / (sg[i] - sg[j]);
    return v;
}
static long double lag_der(const long double *sg, int m, int i, long double s)
{
    long double d = 0.0L;
    for (int k = 0; k <= m; k++) {
        if (k == i) continue;
        long double t = 1.0L / (sg[i] - sg[k]);
        for (int j = 0; j <= m; j++) if (j != i && j != k) t *= (s - sg[j]) / (sg[i] - sg[j]);
        d += t;
    }
    return d;
}

/* Monomials of total degree <= k: ordered by degree, then alpha descending. */
static int monomials(int k, int *al, int *be)
{
    int n = 0;
    for (int d = 0; d <= k; d++)
        for (int a = d; a >= 0; a--) { al[n] = a; be[n] = d - a; n++; }
    return n;
}


/*
 * Least-squares read-out rows (Eqs. ns-poly2d .. ns-readout).  The fit
 * a = (V^T V)^{-1} V^T f is evaluated through a thin QR of the column-scaled
 * Vandermonde matrix computed by modified Gram-Schmidt with one
 * re-orthogonalisation pass, in extended precision (long double) and rounded
 * to FP64 at the end; L_i = v(P_i)^T a-map, i.e. L_i = Q R^{-T} D v(P_i)
 * with D the column scaling.
 * Returns 0 on success, 1 if the cloud is rank deficient at this degree.
 */
typedef long double xreal;

static xreal xpow(xreal x, int e) { xreal r = 1.0L; while (e-- > 0) r *= x; return r; }

static int lsq_rows(int N, const double *xp, const double *yp, int k, double *L)
{
    int al[15], be[15];
    int nm = monomials(k, al, be);
    if (N < nm) return 1;
    xreal *Q = (xreal *)malloc(sizeof(xreal) * N * nm);
    xreal R[15][15];
    xreal D[15];
    memset(R, 0, sizeof(R));
    for (int j = 0; j < nm; j++) {
        xreal s = 0.0L;
        for (int e = 0; e < N; e++) {
            xreal v = xpow(xp[e], al[j]) * xpow(yp[e], be[j]);
            Q[e * nm + j] = v;
            s += v * v;
        }
        D[j] = s > 0 ? 1.0L / sqrtl(s) : 1.0L;
        for (int e = 0; e < N; e++) Q[e * nm + j] *= D[j];
    }
    for (int j = 0; j < nm; j++) {
        for (int pass = 0; pass < 2; pass++) {
            for (int i = 0; i < j; i++) {
                xreal dot = 0.0L;
                for (int e = 0; e < N; e++) dot += Q[e * nm + i] * Q[e * nm + j];
                R[i][j] += dot;
                for (int e = 0; e < N; e++) Q[e * nm + j] -= dot * Q[e * nm + i];
            }
        }
        xreal nrm = 0.0L;
        for (int e = 0; e < N; e++) nrm += Q[e * nm + j] * Q[e * nm + j];
        nrm = sqrtl(nrm);
        R[j][j] = nrm;
        if (nrm > 0) for (int e = 0; e < N; e++) Q[e * nm + j] /= nrm;
    }
    xreal rmax = 0.0L, rmin = 1e300L;
    for (int j = 0; j < nm; j++) {
        xreal a = fabsl(R[j][j]);
        if (a > rmax) rmax = a;
        if (a < rmin) rmin = a;
    }
    if (!(rmin > 1e-10L * rmax)) { free(Q); return 1; }
    for (int i = 0; i <= k; i++) {
        /* v(P_i): x' = i, y' = 0 */
        xreal z[15];
        for (int j = 0; j < nm; j++) {
            xreal v = (be[j] == 0 ? xpow((xreal)i, al[j]) : 0.0L) * D[j];
            for (int l = 0; l < j; l++) v -= R[l][j] * z[l];
            z[j] = v / R[j][j];              /* R^T z = D v  (forward) */
        }
        for (int e = 0; e < N; e++) {
            xreal s = 0.0L;
            for (int j = 0; j < nm; j++) s += Q[e * nm + j] * z[j];
            L[i * N + e] = (double)s;
        }
    }
    free(Q);
    return 0;
}

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* Stencil footprint of a fluid node along one axis: [lo, hi] (unwrapped). */
static void footprint(int i, int n, int per, int *lo, int *hi)
{
    if (per) { *lo = i - 3; *hi = i + 3; return; }
    if (i < 3) { *lo = 0; *hi = 6; return; }           /* one-sided rows read nodes 0..6 */
    if (i > n - 4) { *lo = n - 7; *hi = n - 1; return; }
    *lo = i - 3; *hi = i + 3;
}

static int build_ghost(orc_t *o, orc_ghost *G, int gi, int gj)
{
    const double h = o->h;
    double x = node_x(o, gi), y = node_y(o, gj);
    G->target = gj * o->nx + gi;
    double d;
    if (o->wall == 2) {
        double gx = x - o->wa, gy = y - o->wb;
        double rho = sqrt(gx * gx + gy * gy);
        if (!(rho > 0)) return 2;
        G->nx = gx / rho; G->ny = gy / rho;
        G->bpx = o->wa + o->wc * G->nx;
        G->bpy = o->wb + o->wc * G->ny;
        d = o->wc - rho;
    } else {
        G->nx = -sin(o->wc); G->ny = cos(o->wc);
        double phi = (x - o->wa) * G->nx + (y - o->wb) * G->ny;
        d = -phi;
        G->bpx = x + d * G->nx;
        G->bpy = y + d * G->ny;
    }
    G->r = d / h;
    /* elliptical cloud, Eq. ns-ellipse, R_n = 2k = 8, R_t = k/2 + 1 = 3 */
    double fx = (G->bpx - o->x0) / h, fy = (G->bpy - o->y0) / h;
    int ilo = (int)floor(fx) - 9, ihi = (int)ceil(fx) + 9;
    int jlo = (int)floor(fy) - 9, jhi = (int)ceil(fy) + 9;
    double xp[ORC_MAXCL], yp[ORC_MAXCL];
    int N = 0;
    for (int j = jlo; j <= jhi; j++) {
        if (!o->per_y && (j < 0 || j >= o->ny)) continue;
        for (int i = ilo; i <= ihi; i++) {
            if (!o->per_x && (i < 0 || i >= o->nx)) continue;
            int s = wrap(j, o->ny) * o->nx + wrap(i, o->nx);
            if (o->kind[s] != 1) continue;
            double ddx = node_x(o, i) - G->bpx, ddy = node_y(o, j) - G->bpy;
            double xr = (G->nx * ddx + G->ny * ddy) / h;
            double yr = (-G->ny * ddx + G->nx * ddy) / h;
            double qv = (xr * xr) / 64.0 + (yr * yr) / 9.0;
            if (qv <= 1.0) {
                if (N >= ORC_MAXCL) return 3;
                G->cl[N] = s; xp[N] = xr; yp[N] = yr; N++;
            }
        }
    }
    G->ncl = N;
    /* degree k = m = 4; lowered step by step down to 1 when the cloud (clipped
     * by the domain edge) cannot carry it.  A cloud that cannot carry even a
     * plane (all its nodes on one line: a steep wall leaving the box) gets the
     * constant fit, whose prediction is the cloud mean everywhere, and the
     * normal extrapolation keeps m = 1 (L_0 = L_1 = 1/N). */
    int k;
    G->L = (double *)malloc(sizeof(double) * 5 * (N > 0 ? N : 1));
    for (k = 4; k >= 1; k--)
        if (lsq_rows(N, xp, yp, k, G->L) == 0) break;
    G->k = k >= 1 ? k : 0;
    if (k < 1) {
        if (N < 1) return 4;
        for (int e = 0; e < N; e++) G->L[e] = G->L[N + e] = 1.0 / N;
        k = 1;
    }
    G->m = k;
    /* Step 2 of Sec. 3.1: Lagrange factors along the normal.
     * Dirichlet / Neumann: nodes {-r, 1..m}, evaluated (value / slope) at s = 0.
     * Free: nodes {0..m}, evaluated at s = -r. */
    long double sg[5], s0[5];
    sg[0] = -(long double)G->r;
    for (int i = 1; i <= k; i++) sg[i] = i;
    for (int i = 0; i <= k; i++) s0[i] = i;
    for (int i = 0; i <= k; i++) {
        G->c[i] = (double)lag_val(sg, k, i, 0.0L);
        G->ct[i] = (double)lag_der(sg, k, i, 0.0L);
        G->ell[i] = (double)lag_val(s0, k, i, -(long double)G->r);
    }
    return 0;
}

int orc_setup(orc_t *o)
{
    const int nx = o->nx, ny = o->ny;
    orc_free_ghosts(o);
    o->err[0] = 0;
    orc_ade_coeffs(o->rigid, o->R, o->M, o->K, &o->regime, o->A, o->bv, o->cv);
    o->ns = 2;
    if (!o->rigid && o->nreal + o->npair > 0) { o->regime = 4; o->ns = o->nreal + 2 * o->npair; }
    /* mask: fluid / solid (Sec. 3.1) */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++)
            o->kind[j * nx + i] = is_fluid_xy(o, node_x(o, i), node_y(o, j)) ? 1 : 0;
    /* ghost points: solid nodes inside the stencil of some fluid node */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            if (o->kind[j * nx + i] != 1) continue;
            int lo, hi;
            footprint(i, nx, o->per_x, &lo, &hi);
            for (int a = lo; a <= hi; a++) {
                int s = j * nx + wrap(a, nx);
                if (o->kind[s] == 0) o->kind[s] = 2;
            }
            footprint(j, ny, o->per_y, &lo, &hi);
            for (int b = lo; b <= hi; b++) {
                int s = wrap(b, ny) * nx + i;
                if (o->kind[s] == 0) o->kind[s] = 2;
            }
        }
    int ng = 0;
    for (int s = 0; s < nx * ny; s++) ng += o->kind[s] == 2;
    o->ng = ng;
    o->g = (orc_ghost *)calloc(ng > 0 ? ng : 1, sizeof(orc_ghost));
    o->X = (double *)calloc((size_t)o->ns * (ng > 0 ? ng : 1), sizeof(double));
    int *gs = (int *)malloc(sizeof(int) * (ng > 0 ? ng : 1));
    int c = 0;
    for (int s = 0; s < nx * ny; s++) if (o->kind[s] == 2) gs[c++] = s;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(|:bad)
    for (int g = 0; g < ng; g++) {
        int rc = build_ghost(o, &o->g[g], gs[g] % nx, gs[g] / nx);
        if (rc) bad |= 1 << rc;
    }
    free(gs);
    o->n_reduced = 0;
    for (int g = 0; g < ng; g++) o->n_reduced += o->g[g].k < 4;
    o->step = 0;
    if (bad) { snprintf(o->err, sizeof(o->err), "ghost setup failed (mask %d)", bad); return bad; }
    return 0;
}

int orc_n_ghost(orc_t *o) { return o->ng; }
int orc_n_reduced(orc_t *o) { return o->n_reduced; }
int orc_regime(orc_t *o) { return o->regime; }
double orc_dt(orc_t *o) { return o->dt; }

/* degree k of a ghost's cloud fit (0: constant fit, see build_ghost) */
int orc_ghost_fit_degree(orc_t *o, int g) { return o->g[g].k; }

void orc_ghost_meta(orc_t *o, int g, int *target, double *meta, int *m, int *ncl)
{
    orc_ghost *G = &o->g[g];
    *target = G->target;
    meta[0] = G->bpx; meta[1] = G->bpy; meta[2] = G->nx; meta[3] = G->ny; meta[4] = G->r;
    *m = G->m; *ncl = G->ncl;
}

/* Export of one ghost's cloud and its read-out rows L_0..L_m ((m+1) x ncl). */
void orc_ghost_rows(orc_t *o, int g, int *cl, double *L, double *c, double *ct, double *ell)
{
    orc_ghost *G = &o->g[g];
    for (int e = 0; e < G->ncl; e++) cl[e] = G->cl[e];
    memcpy(L, G->L, sizeof(double) * (G->m + 1) * G->ncl);
    for (int i = 0; i <= G->m; i++) { c[i] = G->c[i]; ct[i] = G->ct[i]; ell[i] = G->ell[i]; }
}

void orc_get_kind(orc_t *o, unsigned char *out) { memcpy(out, o->kind, (size_t)o->nx * o->ny); }

/* ------------------------------------------------- initial conditions */
void orc_init_pulse(orc_t *o, double xs, double ys, double amp, double w)
{
    double b = log(2.0) / (w * w);
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            int s = j * o->nx + i;
            double dx = node_x(o, i) - xs, dy = node_y(o, j) - ys;
            o->q[0][s] = o->kind[s] == 1 ? stored(o, amp * exp(-b * (dx * dx + dy * dy))) : 0.0;
            o->q[1][s] = 0.0; o->q[2][s] = 0.0;
        }
    memset(o->X, 0, sizeof(double) * o->ns * (o->ng > 0 ? o->ng : 1));
    o->step = 0; o->prec = 0;
}

/* Wave packet of Sec. 4.1, propagating along direction ang:
 * p0 = (a/2) exp(-alpha^2 s^2) cos(2 pi k s), (u0, v0) = p0 (cos ang, sin ang). */
void orc_init_packet(orc_t *o, double xs, double ys, double ang, double amp, double k, double alpha)
{
    double ca = cos(ang), sa = sin(ang);
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            int sidx = j * o->nx + i;
            double s = (node_x(o, i) - xs) * ca + (node_y(o, j) - ys) * sa;
            double p = o->kind[sidx] == 1
                     ? 0.5 * amp * exp(-alpha * alpha * s * s) * cos(2.0 * M_PI * k * s) : 0.0;
            o->q[0][sidx] = stored(o, p); o->q[1][sidx] = stored(o, p * ca); o->q[2][sidx] = stored(o, p * sa);
        }
    memset(o->X, 0, sizeof(double) * o->ns * (o->ng > 0 ? o->ng : 1));
    o->step = 0; o->prec = 0;
}

void orc_get_field(orc_t *o, int which, double *out)
{ memcpy(out, o->q[which], sizeof(double) * o->nx * o->ny); }
void orc_set_field(orc_t *o, int which, const double *in)
{ memcpy(o->q[which], in, sizeof(double) * o->nx * o->ny); }
void orc_get_ade(orc_t *o, double *out) { memcpy(out, o->X, sizeof(double) * o->ns * o->ng); }
void orc_set_ade(orc_t *o, const double *in) { memcpy(o->X, in, sizeof(double) * o->ns * o->ng); }
int orc_n_states(orc_t *o) { return o->ns; }
long orc_get_step(orc_t *o) { return o->step; }

/* ------------------------------------------------------------ probes */
int orc_set_probes(orc_t *o, int n, const double *xy, long cap)
{
    free(o->pidx); free(o->pw); free(o->phist);
    o->nprobe = n; o->pcap = cap; o->prec = 0;
    o->pidx = (int *)calloc((size_t)16 * (n > 0 ? n : 1), sizeof(int));
    o->pw = (double *)calloc((size_t)16 * (n > 0 ? n : 1), sizeof(double));
    o->phist = (double *)calloc((size_t)(cap > 0 ? cap : 1) * (n > 0 ? n : 1), sizeof(double));
    int invalid = 0;
    for (int p = 0; p < n; p++) {
        double fx = (xy[2 * p] - o->x0) / o->h, fy = (xy[2 * p + 1] - o->y0) / o->h;
        int i0 = (int)floor(fx) - 1, j0 = (int)floor(fy) - 1;
        double xi = fx - i0, eta = fy - j0;
        int ok = i0 >= 0 && j0 >= 0 && i0 + 3 < o->nx && j0 + 3 < o->ny;
        for (int b = 0; ok && b < 4; b++)
            for (int a = 0; a < 4; a++)
                if (o->kind[(j0 + b) * o->nx + i0 + a] != 1) ok = 0;
        if (ok) {
            /* 4 x 4 tensor Lagrange interpolation of degree 3 */
            long double sn[4] = {0, 1, 2, 3};
            for (int b = 0; b < 4; b++)
                for (int a = 0; a < 4; a++) {
                    o->pidx[16 * p + 4 * b + a] = (j0 + b) * o->nx + i0 + a;
                    o->pw[16 * p + 4 * b + a] = (double)(lag_val(sn, 3, a, xi) * lag_val(sn, 3, b, eta));
                }
        } else {
            int i = (int)floor(fx + 0.5), j = (int)floor(fy + 0.5);
            if (i < 0 || j < 0 || i >= o->nx || j >= o->ny || o->kind[j * o->nx + i] != 1) {
                invalid++;
                continue;           /* records 0 */
            }
            o->pidx[16 * p] = j * o->nx + i;
            o->pw[16 * p] = 1.0;
        }
    }
    return invalid;
}

static void record_probes(orc_t *o)
{
    if (o->nprobe == 0 || o->prec >= o->pcap) return;
    for (int p = 0; p < o->nprobe; p++) {
        double s = 0.0;
        for (int e = 0; e < 16; e++) s += o->pw[16 * p + e] * o->q[0][o->pidx[16 * p + e]];
        o->phist[o->prec * o->nprobe + p] = s;
    }
    o->prec++;
}

long orc_get_probes(orc_t *o, double *out)
{
    memcpy(out, o->phist, sizeof(double) * o->prec * o->nprobe);
    return o->prec;
}

/* ------------------------------------------------------------ operator */
/* One-sided 7-point DRP stencils of Tam and Webb (1993) for the three nodes
 * nearest an edge: row r (node r from the edge) holds the coefficients of
 * nodes 0..6, so that df/dx at node r = (1/h) sum_k TW[r][k] f_k.  Each row is
 * exact for polynomials of degree <= 4 (to the 9 printed digits). */
static const double ORC_TW[3][7] = {
    {-2.192280339, 4.748611401, -5.108851915, 4.461567104, -2.833498741, 1.128328861, -0.203876371},
    {-0.209337622, -1.084875676, 2.147776050, -1.388928322, 0.768949766, -0.281814650, 0.048230454},
    {0.049041958, -0.468840357, -0.474760914, 1.273274737, -0.518484526, 0.166138533, -0.026369431}};

/* First derivative along an axis of n nodes at index i, reading f[k * stride]
 * (k wrapped when the axis is periodic).  Sec. 2.2: the DRP stencil in the
 * interior; the one-sided DRP stencils in the three outer layers of a
 * non-periodic axis (at the far edge the mirror image: nodes n-1, n-2, ...
 * with the signs reversed). */
static double deriv1(const double *f, int stride, int n, int i, int per, double h)
{
#define F(k) f[(size_t)wrap((k), n) * stride]
    if (per || (i >= 3 && i <= n - 4))
        return (ORC_A1 * (F(i + 1) - F(i - 1)) + ORC_A2 * (F(i + 2) - F(i - 2)) +
                ORC_A3 * (F(i + 3) - F(i - 3))) / h;
    double s = 0.0;
    if (i < 3) {
        for (int k = 0; k < 7; k++) s += ORC_TW[i][k] * F(k);
    } else {
        const int r = n - 1 - i;                 /* row counted from the far edge */
        for (int k = 0; k < 7; k++) s -= ORC_TW[r][k] * F(n - 1 - k);
    }
    return s / h;
#undef F
}

static double dx_at(const orc_t *o, const double *f, int i, int j)
{ return deriv1(f + (size_t)j * o->nx, 1, o->nx, i, o->per_x, o->h); }

static double dy_at(const orc_t *o, const double *f, int i, int j)
{ return deriv1(f + i, o->nx, o->ny, j, o->per_y, o->h); }

/* 1D derivative operator on a bare array (pin: polynomial exactness). */
void orc_deriv_1d(int n, const double *f, double h, int per, double *out)
{
    for (int i = 0; i < n; i++) out[i] = deriv1(f, 1, n, i, per, h);
}

/* Opt-in absorbing ramp near the non-periodic edges (off unless
 * orc_set_sponge gave it a width W): damping rate at node (i, j),
 * (kappa / h) ((W - d) / W)^2 for a distance d < W (in cells) to the nearest
 * edge, 0 elsewhere. */
static double sponge_rate(const orc_t *o, int i, int j)
{
    const int W = o->sponge_w;
    if (W <= 0) return 0.0;
    int d = 1 << 30;
    if (!o->per_x) { if (i < d) d = i; if (o->nx - 1 - i < d) d = o->nx - 1 - i; }
    if (!o->per_y) { if (j < d) d = j; if (o->ny - 1 - j < d) d = o->ny - 1 - j; }
    if (d >= W) return 0.0;
    double r = (double)(W - d) / W;
    return o->sponge_k / o->h * r * r;
}

static int in_band(const orc_t *o, int i, int j)
{
    return (!o->per_x && (i < 3 || i > o->nx - 4)) || (!o->per_y && (j < 3 || j > o->ny - 4));
}

/*
 * Steps 2-3 of Sec. 3.2 for one ghost: the ADE derivative xd of the states x
 * forced by p_BP, the wall normal velocity u_n and its time derivative.
 * MSD wall (Sec. 2.5): the 2 x 2 form of its regime.  Rational admittance:
 * Eq. ADEgeneral state by state (real poles first, then the pairs) and
 * Eq. unGeneral with Y_inf = 0.
 */
static void ade_eval(const orc_t *o, const double *x, double pbp, double *xd, double *un, double *dun)
{
    if (o->regime != 4) {
        xd[0] = o->A[0][0] * x[0] + o->A[0][1] * x[1] + o->bv[0] * pbp;
        xd[1] = o->A[1][0] * x[0] + o->A[1][1] * x[1] + o->bv[1] * pbp;
        *un = o->cv[0] * x[0] + o->cv[1] * x[1];
        *dun = o->cv[0] * xd[0] + o->cv[1] * xd[1];
        return;
    }
    double u = 0.0, du = 0.0;
    for (int k = 0; k < o->nreal; k++) {
        const double phi = x[k];
        const double dphi = o->lam[k] * phi + pbp;                          /* Eq. ADEgeneral a */
        xd[k] = dphi;
        u += o->Ares[k] * phi;                                              /* Eq. unGeneral */
        du += o->Ares[k] * dphi;
    }
    for (int k = 0; k < o->npair; k++) {
        const double *psi = x + o->nreal + 2 * k;
        double *dpsi = xd + o->nreal + 2 * k;
        dpsi[0] = o->al[k] * psi[0] - o->be[k] * psi[1] + pbp;             /* Eq. ADEgeneral b */
        dpsi[1] = o->al[k] * psi[1] + o->be[k] * psi[0];                   /* Eq. ADEgeneral c */
        u += 2.0 * (o->Bres[k] * psi[0] - o->Cres[k] * psi[1]);
        du += 2.0 * (o->Bres[k] * dpsi[0] - o->Cres[k] * dpsi[1]);
    }
    *un = u;
    *dun = du;
}

/*
 * One evaluation of the semi-discrete right-hand side of Q = [p; u; v; X]
 * (Sec. 3.2).  Steps 1-5 fill the ghost nodes of q (in place) and give the
 * ADE derivative Xd; step 6 evaluates the DRP / radiation right-hand side at
 * every fluid node (0 elsewhere).  sigma is the source time factor of this
 * evaluation, s = a exp(-b r^2) sigma (Sec. 4.3).
 */
static void orc_rhs(orc_t *o, double *q[3], const double *X, double sigma, double *rq[3], double *Xd)
{
    const int nx = o->nx, ny = o->ny;
    const double h = o->h;
#pragma omp parallel for schedule(static)
    for (int g = 0; g < o->ng; g++) {
        orc_ghost *G = &o->g[g];
        const int m = G->m, N = G->ncl;
        double Pp[5], Pw[5], Pt[5];
        for (int i = 0; i <= m; i++) {
            double sp = 0, sw = 0, st = 0;
            const double *Li = G->L + (size_t)i * N;
            for (int e = 0; e < N; e++) {
                int s = G->cl[e];
                double uu = q[1][s], vv = q[2][s];
                sp += Li[e] * q[0][s];
                sw += Li[e] * (G->nx * uu + G->ny * vv);      /* w = u . n   */
                st += Li[e] * (-G->ny * uu + G->nx * vv);     /* t = u . tau */
            }
            Pp[i] = sp; Pw[i] = sw; Pt[i] = st;
        }
        /* 1: pressure at the boundary point */
        double pbp = Pp[0];
        /* 2-3: ADE derivative at this stage, wall normal velocity and its
         * time derivative */
        const double *x = X + (size_t)o->ns * g;
        double *xd = Xd + (size_t)o->ns * g;
        double un, dun;
        ade_eval(o, x, pbp, xd, &un, &dun);
        /* 4: boundary data: w_BP = -u_n (Dirichlet), dp/dn_BP = +du_n/dt (Neumann) */
        double gD = -un, gN = dun;
        if (o->bc_override) { gD = o->bc_override[2 * g]; gN = o->bc_override[2 * g + 1]; }
        /* 5: Lagrange extrapolation along the normal, Eq. ns-ghost */
        double np = h * gN, nw = gD, tg = 0.0;
        for (int i = 1; i <= m; i++) { np -= G->ct[i] * Pp[i]; nw -= G->c[i] * Pw[i]; }
        for (int i = 0; i <= m; i++) tg += G->ell[i] * Pt[i];
        double pg = np / G->ct[0];
        double wg = nw / G->c[0];
        q[0][G->target] = stored(o, pg);
        q[1][G->target] = stored(o, wg * G->nx - tg * G->ny);
        q[2][G->target] = stored(o, wg * G->ny + tg * G->nx);
    }
    /* 6: right-hand side at fluid nodes */
    const double xc = o->x0 + 0.5 * (nx - 1) * h, yc = o->y0 + 0.5 * (ny - 1) * h;
    const double samp = o->s_amp != 0.0 ? o->s_amp * sigma : 0.0;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int s = j * nx + i;
            if (o->kind[s] != 1) { rq[0][s] = rq[1][s] = rq[2][s] = 0.0; continue; }
            if (in_band(o, i, j)) {
                double rx = node_x(o, i) - xc, ry = node_y(o, j) - yc;
                double rho = sqrt(rx * rx + ry * ry);
                double ct = rx / rho, st = ry / rho;
                /* where a wall meets the band, a derivative whose stencil
                 * window holds a non-fluid node is left out of the radiation
                 * condition (reading for walls that reach the outer boundary) */
                int wx = 1, wy = 1, lo, hi;
                footprint(i, nx, o->per_x, &lo, &hi);
                for (int a = lo; a <= hi; a++) if (o->kind[j * nx + wrap(a, nx)] != 1) wx = 0;
                footprint(j, ny, o->per_y, &lo, &hi);
                for (int b = lo; b <= hi; b++) if (o->kind[wrap(b, ny) * nx + i] != 1) wy = 0;
                for (int f = 0; f < 3; f++) {
                    double dr = 0.0;
                    if (wx) dr += ct * dx_at(o, q[f], i, j);
                    if (wy) dr += st * dy_at(o, q[f], i, j);
                    rq[f][s] = -(dr + q[f][s] / (2.0 * rho));
                }
            } else {
                double src = 0.0;
                if (samp != 0.0) {
                    double dx = node_x(o, i) - o->s_x, dy = node_y(o, j) - o->s_y;
                    src = samp * exp(-o->s_b * (dx * dx + dy * dy));
                }
                rq[0][s] = -(dx_at(o, q[1], i, j) + dy_at(o, q[2], i, j)) + src;
                rq[1][s] = -dx_at(o, q[0], i, j);
                rq[2][s] = -dy_at(o, q[0], i, j);
            }
            double sr = sponge_rate(o, i, j);
            if (sr != 0.0)
                for (int f = 0; f < 3; f++) rq[f][s] -= sr * q[f][s];
        }
}

/*
 * Advance nsteps time steps.  classical = 0: the four-stage 2N-storage scheme
 * Q(k) = Q(n) + alpha_k dt RHS(Q(k-1)), alpha = (1/4, 1/3, 1/2, 1), the ADE
 * states advanced by the same stages; classical = 1: Butcher RK4.
 */
void orc_run(orc_t *o, long nsteps, int classical)
{
    const size_t n = (size_t)o->nx * o->ny;
    const int ng = o->ng;
    const double dt = o->dt;
    /* work arrays: allocated on the first call and kept, so that repeated
     * short runs time the method and not the allocator */
    const size_t nsx = (size_t)o->ns * ng;       /* ADE states of all ghosts */
    size_t gx = (size_t)o->ns * (ng > 0 ? ng : 1);
    size_t need = 9 * n + 3 * gx;
    if (o->work_n < need) {
        free(o->work);
        o->work = (double *)malloc(sizeof(double) * need);
        o->work_n = need;
    }
    double *qs[3], *rq[3], *acc[3];
    for (int f = 0; f < 3; f++) {
        qs[f] = o->work + (size_t)f * n;
        rq[f] = o->work + (size_t)(3 + f) * n;
        acc[f] = o->work + (size_t)(6 + f) * n;
    }
    double *Xs = o->work + 9 * n;
    double *Xd = Xs + gx;
    double *Xacc = Xd + gx;
    static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
    for (long st = 0; st < nsteps; st++) {
        const double tn = (double)o->step * dt;
        if (!classical) {
            for (int f = 0; f < 3; f++) memcpy(qs[f], o->q[f], sizeof(double) * n);
            memcpy(Xs, o->X, sizeof(double) * nsx);
            for (int k = 0; k < 4; k++) {
                orc_rhs(o, qs, Xs, stage_forcing(o->s_omega, tn, dt, k + 1), rq, Xd);
                const double ad = alpha[k] * dt;
#pragma omp parallel for schedule(static)
                for (size_t s = 0; s < n; s++)
                    for (int f = 0; f < 3; f++)
                        qs[f][s] = o->kind[s] == 1 ? stored(o, o->q[f][s] + ad * rq[f][s]) : 0.0;
                for (size_t g = 0; g < nsx; g++) Xs[g] = o->X[g] + ad * Xd[g];
            }
            for (int f = 0; f < 3; f++) memcpy(o->q[f], qs[f], sizeof(double) * n);
            memcpy(o->X, Xs, sizeof(double) * nsx);
        } else {
            static const double cw[4] = {1.0, 2.0, 2.0, 1.0};
            static const double cf[4] = {0.5, 0.5, 1.0, 0.0};
            static const double tc[4] = {0.0, 0.5, 0.5, 1.0};
            for (int f = 0; f < 3; f++) { memcpy(qs[f], o->q[f], sizeof(double) * n); memset(acc[f], 0, sizeof(double) * n); }
            memcpy(Xs, o->X, sizeof(double) * nsx);
            memset(Xacc, 0, sizeof(double) * gx);
            for (int k = 0; k < 4; k++) {
                orc_rhs(o, qs, Xs, sin(o->s_omega * (tn + tc[k] * dt)), rq, Xd);
                for (size_t s = 0; s < n; s++)
                    for (int f = 0; f < 3; f++) {
                        acc[f][s] += cw[k] * rq[f][s];
                        qs[f][s] = o->kind[s] == 1 ? o->q[f][s] + cf[k] * dt * rq[f][s] : 0.0;
                    }
                for (size_t g = 0; g < nsx; g++) {
                    Xacc[g] += cw[k] * Xd[g];
                    Xs[g] = o->X[g] + cf[k] * dt * Xd[g];
                }
            }
            for (size_t s = 0; s < n; s++)
                for (int f = 0; f < 3; f++)
                    o->q[f][s] = o->kind[s] == 1 ? o->q[f][s] + dt / 6.0 * acc[f][s] : 0.0;
            for (size_t g = 0; g < nsx; g++) o->X[g] += dt / 6.0 * Xacc[g];
        }
        o->step++;
        record_probes(o);
    }
}

/* Fill the ghost nodes of the current Q^n from the current X^n (steps 1-5)
 * and return them in the field; used by tests of the ghost fill alone. */
void orc_fill_ghosts(orc_t *o, double *Xd_out)
{
    const size_t n = (size_t)o->nx * o->ny;
    double *rq[3];
    for (int f = 0; f < 3; f++) rq[f] = (double *)malloc(sizeof(double) * n);
    double *Xd = (double *)malloc(sizeof(double) * o->ns * (o->ng > 0 ? o->ng : 1));
    orc_rhs(o, o->q, o->X, sin(o->s_omega * (double)o->step * o->dt), rq, Xd);
    if (Xd_out) memcpy(Xd_out, Xd, sizeof(double) * o->ns * o->ng);
    for (int f = 0; f < 3; f++) free(rq[f]);
    free(Xd);
}

/* Test hook: fill the ghost nodes from given boundary data per ghost,
 * bc[2g] = w = u.n at BP (Dirichlet) and bc[2g+1] = dp/dn at BP (Neumann),
 * instead of the data supplied by the ADE (steps 4-5 of Sec. 3.2 alone). */
void orc_fill_ghosts_bc(orc_t *o, const double *bc)
{
    o->bc_override = bc;
    orc_fill_ghosts(o, NULL);
    o->bc_override = NULL;
}

/* Evaluate the right-hand side at the current state (after a ghost fill). */
void orc_eval_rhs(orc_t *o, double t, double *rp, double *ru, double *rv, double *Xd)
{
    double *rq[3] = {rp, ru, rv};
    orc_rhs(o, o->q, o->X, sin(o->s_omega * t), rq, Xd);
}

/* Acoustic energy of the fluid nodes: E = 1/2 h^2 sum (p^2 + u^2 + v^2). */
double orc_energy(orc_t *o)
{
    double e = 0.0;
    for (size_t s = 0; s < (size_t)o->nx * o->ny; s++)
        if (o->kind[s] == 1) e += o->q[0][s] * o->q[0][s] + o->q[1][s] * o->q[1][s] + o->q[2][s] * o->q[2][s];
    return 0.5 * o->h * o->h * e;
}

/*
 * The rational-admittance ADE alone (Eqs. ADEgeneral, unGeneral), forced by
 * p_BP(t) = sin(omega t) and advanced by the four stages with the same stage
 * forcing moments as the source; returns u_n after each step.
 * Pin: u_n equals the convolution of the kernel y(t) of Eq. Yrational's
 * inverse Laplace transform with the forcing, up to O(dt^4).
 */
void orc_rational_drive(int nreal, const double *lam, const double *A, int npair, const double *al,
                        const double *be, const double *B, const double *C, double dt, long nsteps,
                        double omega, double *un_out)
{
    orc_t o;
    memset(&o, 0, sizeof o);
    orc_set_rational(&o, nreal, lam, A, npair, al, be, B, C);
    o.regime = 4;
    o.ns = nreal + 2 * npair;
    static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
    double X[ORC_MAXPOLE] = {0}, Xs[ORC_MAXPOLE], Xd[ORC_MAXPOLE], un, dun;
    for (long n = 0; n < nsteps; n++) {
        memcpy(Xs, X, sizeof X);
        for (int k = 0; k < 4; k++) {
            ade_eval(&o, Xs, stage_forcing(omega, (double)n * dt, dt, k + 1), Xd, &un, &dun);
            for (int i = 0; i < o.ns; i++) Xs[i] = X[i] + alpha[k] * dt * Xd[i];
        }
        memcpy(X, Xs, sizeof X);
        ade_eval(&o, X, 0.0, Xd, &un, &dun);
        un_out[n] = un;
    }
}

/*
 * The wall ODE alone (Sec. 2.5), forced by p_BP(t) = sin(omega t) and advanced
 * by the same four stages (with the same stage forcing moments as the
 * source); returns u_n after each step and the final state.
 * Pin: the steady response equals Y(i omega) sin, up to O(dt^4).
 */
void orc_ade_drive(double R, double M, double K, double dt, long nsteps, double omega,
                   double *un_out, double *X_out)
{
    int reg; double A[2][2], b[2], c[2];
    orc_ade_coeffs(0, R, M, K, &reg, A, b, c);
    static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};
    double X[2] = {0, 0}, Xs[2];
    for (long n = 0; n < nsteps; n++) {
        Xs[0] = X[0]; Xs[1] = X[1];
        for (int k = 0; k < 4; k++) {
            double p = stage_forcing(omega, (double)n * dt, dt, k + 1);
            double d0 = A[0][0] * Xs[0] + A[0][1] * Xs[1] + b[0] * p;
            double d1 = A[1][0] * Xs[0] + A[1][1] * Xs[1] + b[1] * p;
            Xs[0] = X[0] + alpha[k] * dt * d0;
            Xs[1] = X[1] + alpha[k] * dt * d1;
        }
        X[0] = Xs[0]; X[1] = Xs[1];
        un_out[n] = c[0] * X[0] + c[1] * X[1];
    }
    X_out[0] = X[0]; X_out[1] = X[1];
}
