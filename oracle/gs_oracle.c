/*
 * gs_oracle.c -- plain FP64 CPU oracle for the TMSmesh 2.0 meshing path
 * (Liu, Chen & Lu, "Efficient and qualified mesh generation for Gaussian
 * molecular surface using piecewise trilinear polynomial approximation").
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg call this code.  It shares nothing with the
 * CUDA library: both implement the same readings of the paper independently.
 *
 * Everything is brute force and in the paper's order: every atom is visited
 * for every cube and every point (no cell lists), sums run in ascending atom
 * index, the SVD is a textbook one-sided Jacobi iteration.  Build with
 * -O2 -ffp-contract=off and no fast-math.
 *
 * Parity status: every function is pinned by a test against a closed form,
 * a library routine or brute force, except the per-cube triangulation of
 * general (non-sphere) inputs, whose pins are invariants (closed manifold,
 * |g - c| = 0 at points, single-valued pieces) rather than exact values.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads: the loops over cubes and points run in parallel when built with
 * OpenMP.  Every cube's and point's result depends on that cube or point
 * alone, and results are collected in input order, so the output does not
 * depend on the thread count. */
static int g_threads = 0; /* 0: OpenMP's default */
int or_set_threads(int n)
{
    g_threads = n < 0 ? 0 : n;
#ifdef _OPENMP
    return g_threads ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}
#ifdef _OPENMP
#define OR_NT (g_threads ? g_threads : omp_get_max_threads())
#endif

/* ------------------------------------------------------------------ */
/* Key format (shared *format*, not code, with the CUDA library):      */
/*   bits  0..17 x, 18..35 y, 36..53 z  (lattice coordinates)          */
/*   bits 54..58 type, 59..63 level                                    */
/* type 0..2   : surface point on a cube edge along axis 0/1/2; xyz =  */
/*               finest-lattice coords of the edge's lower endpoint    */
/* type 8..19  : extreme point, 8 + 4*axis + 2*side + rank; xyz =      */
/*               finest-lattice coords of the face's lower corner;     */
/*               side 1 = the fold belongs to the cube on the + side   */
/* type 20..31 : critical point, 20 + 4*(a+b-1) + 2*i + j for roots i  */
/*               of the a-fold and j of the b-fold (a < b); xyz = the  */
/*               cube's lower corner (finest lattice)                  */
/* cube keys (own namespace): type 30, xyz at the cube's own level     */
/* lattice-vertex keys (own namespace): type 31, finest coords, lvl 0  */
/* ------------------------------------------------------------------ */
#define OK_BITS 18
#define OK_MASK ((1ull << OK_BITS) - 1)
#define T_CUBE 30u
#define T_VERT 31u

static uint64_t okey(uint64_t x, uint64_t y, uint64_t z, unsigned type, unsigned level)
{
    return x | (y << 18) | (z << 36) | ((uint64_t)type << 54) | ((uint64_t)level << 59);
}
static void okey_xyz(uint64_t k, int64_t *x, int64_t *y, int64_t *z)
{
    *x = (int64_t)(k & OK_MASK);
    *y = (int64_t)((k >> 18) & OK_MASK);
    *z = (int64_t)((k >> 36) & OK_MASK);
}
static unsigned okey_level(uint64_t k) { return (unsigned)(k >> 59); }

/* status codes (same meaning as the library's) */
#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_OOM -2
#define OR_ERR_CAP -3

/* decisions */
#define DEC_DISCARD 0
#define DEC_ACCEPT 1
#define DEC_SPLIT 2
#define DEC_FORCED 3 /* accepted because the level is max_depth */

/* ================================================================== */
/* Problem setup: eq (Gaussian1) and the neighbourhood truncation.     */
/* ================================================================== */

typedef struct {
    int64_t n;
    const double *xyz; /* [n,3] */
    const double *r;   /* [n] */
    double D, c, cutoff_rel, precision, min_edge;
    int max_depth;
    double *R2;     /* per-atom squared cutoff radius */
    double pad;     /* max cutoff radius */
    double origin[3];
    int64_t nroot[3];
    double h0;
    int child_mode;   /* 0: children re-projected from the atoms; 1: re-expansion of the parent's P~ */
    int order;        /* 0: bound test, then precision test; 1: literal order of steps 2 and 3 */
    int norm;         /* size of the high-order coefficients: 0 sum of |.|, 1 max |.|, 2 sqrt of sum of squares */
    int conform;      /* mixed-size neighbours: 0 constrained vertex values with at most one level between
                         cubes that share a face or an edge; 1 equal sizes across every shared face and edge */
    int resolve;      /* 1: decisions and vertex signs whose margin is in band are re-decided in quad precision */
} oprob;

/* Terms exp(-D(|x-xi|^2 - ri^2)) below cutoff_rel*c are dropped:
 *   term >= cutoff_rel*c  <=>  |x-xi|^2 <= ri^2 + K/D,  K = -ln(cutoff_rel*c). */
static double cut_K(double cutoff_rel, double c) { return -log(cutoff_rel * c); }
static void gl_init(void);

static int oprob_init(oprob *P, int64_t n, const double *xyz, const double *r, double D, double c,
                      double cutoff_rel, double precision, double min_edge, int max_depth)
{
    if (n <= 0 || !(D > 0) || !(c > 0) || !(precision > 0) || !(min_edge > 0) || max_depth < 0 ||
        max_depth > 20 || !(cutoff_rel > 0) || !(cutoff_rel < 1))
        return OR_ERR_ARG;
    memset(P, 0, sizeof(*P));
    gl_init(); /* before any parallel loop reads the nodes */
    P->n = n; P->xyz = xyz; P->r = r; P->D = D; P->c = c; P->cutoff_rel = cutoff_rel;
    P->precision = precision; P->min_edge = min_edge; P->max_depth = max_depth;
    P->R2 = (double *)malloc(sizeof(double) * (size_t)n);
    if (!P->R2) return OR_ERR_OOM;
    double K = cut_K(cutoff_rel, c);
    double KD = K / D;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double r2max = 0;
    for (int64_t i = 0; i < n; i++) {
        double ri = r[i];
        P->R2[i] = ri * ri + KD;
        if (P->R2[i] > r2max) r2max = P->R2[i];
        for (int a = 0; a < 3; a++) {
            double v = xyz[3 * i + a];
            if (!isfinite(v) || !isfinite(ri) || ri < 0) { free(P->R2); P->R2 = NULL; return OR_ERR_ARG; }
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    }
    /* Root grid (section 2.2, "very coarse" initial grid): edge h0 =
     * min_edge * 2^max_depth, origin aligned to h0, covering the atoms'
     * bounding box grown by the largest cutoff radius. */
    P->pad = sqrt(r2max);
    P->h0 = ldexp(min_edge, max_depth);
    for (int a = 0; a < 3; a++) {
        P->origin[a] = P->h0 * floor((lo[a] - P->pad) / P->h0);
        int64_t m = (int64_t)ceil((hi[a] + P->pad - P->origin[a]) / P->h0);
        P->nroot[a] = m < 1 ? 1 : m;
        if ((P->nroot[a] << max_depth) + 1 > (int64_t)OK_MASK) { free(P->R2); P->R2 = NULL; return OR_ERR_ARG; }
    }
    return OR_OK;
}

static void oprob_free(oprob *P) { free(P->R2); P->R2 = NULL; }

/* cube edge at level l */
static double lvl_h(const oprob *P, int l) { return ldexp(P->min_edge, P->max_depth - l); }
/* world coordinate of lattice index i at level l along axis a */
static double lat_x(const oprob *P, int a, int64_t i, int l) { return P->origin[a] + (double)i * lvl_h(P, l); }
/* world coordinate at fraction f of the level-l edge that starts at lattice
 * index i (the index's own lattice coordinate when f is 0 or 1) */
static double wfrac(const oprob *P, int a, int64_t i, int l, double f)
{
    if (f == 0) return lat_x(P, a, i, l);
    if (f == 1) return lat_x(P, a, i + 1, l);
    return lat_x(P, a, i, l) + f * lvl_h(P, l);
}

/* ================================================================== */
/* Gauss-Legendre rule (nodes by Newton iteration on P_n).              */
/* ================================================================== */

static void gauss_legendre(int q, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < q; i++) {
        double t = cos(pi * (i + 0.75) / (q + 0.5));
        double dp = 1;
        for (int it = 0; it < 100; it++) {
            double p0 = 1, p1 = t;
            for (int k = 2; k <= q; k++) {
                double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1; p1 = p2;
            }
            /* p1 = P_q(t), p0 = P_{q-1}(t) */
            dp = q * (t * p1 - p0) / (t * t - 1);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = t;
        w[i] = 2.0 / ((1 - t * t) * dp * dp);
    }
}

#define OR_Q 24
static double gl_x[OR_Q], gl_w[OR_Q];
static int gl_ready = 0;
static void gl_init(void)
{
    if (!gl_ready) { gauss_legendre(OR_Q, gl_x, gl_w); gl_ready = 1; }
}

static double leg(int j, double t)
{
    switch (j) {
    case 0: return 1.0;
    case 1: return t;
    case 2: return (3.0 * t * t - 1.0) / 2.0;
    default: return (5.0 * t * t * t - 3.0 * t) / 2.0;
    }
}

/* ================================================================== */
/* Per-axis Legendre projection with the C0 endpoint correction        */
/* (eqs poly2_1..poly2_3, the alpha/beta/gamma integrals, eqs poly3,    */
/* condition1, pn and alpha; n = 3).                                   */
/* f(x) = exp(-D (x - xi)^2) on [a,b]; t = (2x-(a+b))/(b-a).            */
/* alpha_j = (2j+1)/(b-a) * int_a^b f(x) L_j(t(x)) dx                   */
/*         = (2j+1)/2 * int_{-1}^{1} f(x(t)) L_j(t) dt                  */
/* (the orthogonal L2 projection; the printed prefactor 2/(b-a) and     */
/* the integrand phi(t) are read as this projection).                  */
/* ================================================================== */

void or_axis_projection(double xi, double a, double b, double D, int q, double *out4)
{
    double xs[64], ws[64];
    if (q < 1) q = 1;
    if (q > 64) q = 64;
    gauss_legendre(q, xs, ws);
    double m = 0.5 * (a + b), hh = 0.5 * (b - a);
    for (int j = 0; j < 4; j++) {
        double s = 0;
        for (int k = 0; k < q; k++) {
            double x = m + hh * xs[k];
            double d = x - xi;
            s += ws[k] * exp(-D * d * d) * leg(j, xs[k]);
        }
        out4[j] = 0.5 * (2 * j + 1) * s;
    }
}

/* C0 correction: add eps0 L_2 + eps1 L_3 so that the cubic equals f at
 * both ends (L_j(1) = 1, L_j(-1) = (-1)^j). */
void or_axis_coeffs(double xi, double a, double b, double D, double *out4)
{
    gl_init();
    double m = 0.5 * (a + b), hh = 0.5 * (b - a);
    double al[4];
    for (int j = 0; j < 4; j++) {
        double s = 0;
        for (int k = 0; k < OR_Q; k++) {
            double d = (m + hh * gl_x[k]) - xi;
            s += gl_w[k] * exp(-D * d * d) * leg(j, gl_x[k]);
        }
        al[j] = 0.5 * (2 * j + 1) * s;
    }
    double fa = exp(-D * (a - xi) * (a - xi));
    double fb = exp(-D * (b - xi) * (b - xi));
    double eR = fb - (al[0] + al[1] + al[2] + al[3]);
    double eL = fa - (al[0] - al[1] + al[2] - al[3]);
    double e0 = 0.5 * (eR + eL), e1 = 0.5 * (eR - eL);
    out4[0] = al[0];
    out4[1] = al[1];
    out4[2] = al[2] + e0;
    out4[3] = al[3] + e1;
}

/* squared distance from point x to the box [lo, lo+h]^3, axes in order */
static double box_dist2(const double *lo, const double *hi, const double *x)
{
    double s = 0;
    for (int a = 0; a < 3; a++) {
        double d = 0;
        if (lo[a] - x[a] > 0) d = lo[a] - x[a];
        else if (x[a] - hi[a] > 0) d = x[a] - hi[a];
        s += d * d;
    }
    return s;
}

/* Coefficient tensor A (eqs polynew, tensor1, tensor2): A[j][k][l] =
 * sum_i e^{D r_i^2} atilde_j(x) btilde_k(y) gtilde_l(z), j<->x, k<->y,
 * l<->z, over atoms whose cutoff sphere meets the box; returns the count. */
static int64_t cube_tensor(const oprob *P, const double *lo, const double *hi, double *A)
{
    memset(A, 0, 64 * sizeof(double));
    int64_t cnt = 0;
    for (int64_t i = 0; i < P->n; i++) {
        const double *x = P->xyz + 3 * i;
        if (box_dist2(lo, hi, x) > P->R2[i]) continue;
        cnt++;
        double w = exp(P->D * P->r[i] * P->r[i]);
        double ax[4], ay[4], az[4];
        or_axis_coeffs(x[0], lo[0], hi[0], P->D, ax);
        or_axis_coeffs(x[1], lo[1], hi[1], P->D, ay);
        or_axis_coeffs(x[2], lo[2], hi[2], P->D, az);
        for (int j = 0; j < 4; j++)
            for (int k = 0; k < 4; k++)
                for (int l = 0; l < 4; l++) A[16 * j + 4 * k + l] += w * ax[j] * ay[k] * az[l];
    }
    return cnt;
}

/* ================================================================== */
/* One-sided (Hestenes) Jacobi SVD of an m x n matrix by rows.          */
/* On return rows of M are mutually orthogonal and Q (m x m) holds the   */
/* accumulated rotations: M_in = Q^T M_out.                             */
/* ================================================================== */

static void jacobi_rows(double *M, int m, int n, double *Q)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) Q[i * m + j] = (i == j);
    for (int sweep = 0; sweep < 80; sweep++) {
        int rotated = 0;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) {
                double al = 0, be = 0, ga = 0;
                for (int k = 0; k < n; k++) {
                    al += M[p * n + k] * M[p * n + k];
                    be += M[q * n + k] * M[q * n + k];
                    ga += M[p * n + k] * M[q * n + k];
                }
                if (ga == 0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                rotated = 1;
                double zeta = (be - al) / (2 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1 + zeta * zeta));
                double cs = 1 / sqrt(1 + t * t), sn = cs * t;
                for (int k = 0; k < n; k++) {
                    double mp = M[p * n + k], mq = M[q * n + k];
                    M[p * n + k] = cs * mp - sn * mq;
                    M[q * n + k] = sn * mp + cs * mq;
                }
                for (int k = 0; k < m; k++) {
                    double qp = Q[p * m + k], qq = Q[q * m + k];
                    Q[p * m + k] = cs * qp - sn * qq;
                    Q[q * m + k] = sn * qp + cs * qq;
                }
            }
        if (!rotated) break;
    }
}

/* SVD of an m x n (m <= n, m <= 4) row-major matrix: X = sum_p s_p u_p v_p^T
 * with s sorted descending; u: [m][m] (u_p in row p), v: [m][n]. */
void or_svd_rows(const double *X, int m, int n, double *s, double *u, double *v)
{
    double M[64], Q[16];
    memcpy(M, X, sizeof(double) * (size_t)(m * n));
    jacobi_rows(M, m, n, Q);
    double sv[4];
    int order[4];
    for (int p = 0; p < m; p++) {
        double s2 = 0;
        for (int k = 0; k < n; k++) s2 += M[p * n + k] * M[p * n + k];
        sv[p] = sqrt(s2);
        order[p] = p;
    }
    /* stable insertion sort by descending singular value */
    for (int i = 1; i < m; i++) {
        int o = order[i], j = i - 1;
        while (j >= 0 && sv[order[j]] < sv[o]) { order[j + 1] = order[j]; j--; }
        order[j + 1] = o;
    }
    for (int i = 0; i < m; i++) {
        int p = order[i];
        s[i] = sv[p];
        for (int k = 0; k < m; k++) u[i * m + k] = Q[p * m + k];
        for (int k = 0; k < n; k++) v[i * n + k] = sv[p] > 0 ? M[p * n + k] / sv[p] : 0.0;
    }
}

/* exact range of the cubic sum_j c_j L_j(t) on [-1,1]: endpoints and the
 * real zeros of the derivative inside the interval */
void or_cubic_bounds(const double *cf, double *lo, double *hi)
{
    double c0 = cf[0], c1 = cf[1], c2 = cf[2], c3 = cf[3];
    double m0 = c0 - 0.5 * c2, m1 = c1 - 1.5 * c3, m2 = 1.5 * c2, m3 = 2.5 * c3;
    double vals[4];
    int nv = 0;
    vals[nv++] = c0 + c1 + c2 + c3;
    vals[nv++] = c0 - c1 + c2 - c3;
    /* p'(t) = m1 + 2 m2 t + 3 m3 t^2 */
    double A2 = 3 * m3, B2 = 2 * m2, C2 = m1;
    double roots[2];
    int nr = 0;
    if (A2 == 0) {
        if (B2 != 0) roots[nr++] = -C2 / B2;
    } else {
        double disc = B2 * B2 - 4 * A2 * C2;
        if (disc >= 0) {
            double sq = sqrt(disc);
            double qq = -0.5 * (B2 + (B2 >= 0 ? sq : -sq));
            if (qq != 0) { roots[nr++] = qq / A2; roots[nr++] = C2 / qq; }
            else roots[nr++] = 0.0; /* B2 == 0 and disc == 0 -> C2 == 0 */
        }
    }
    for (int i = 0; i < nr; i++) {
        double t = roots[i];
        if (t > -1 && t < 1) vals[nv++] = m0 + t * (m1 + t * (m2 + t * m3));
    }
    double a = vals[0], b = vals[0];
    for (int i = 1; i < nv; i++) { if (vals[i] < a) a = vals[i]; if (vals[i] > b) b = vals[i]; }
    *lo = a; *hi = b;
}

/* smallest j with sum_{i<=j} s_i >= 0.99 * sum s (eq SVD3); returns count.
 * rel (nullable) is lowered to the smallest |sum_{i<=j} s_i - 0.99 sum s| /
 * sum s over the rules evaluated (those up to the deciding one). */
static int rank99_m(const double *s, int m, double *rel)
{
    double tot = 0;
    for (int i = 0; i < m; i++) tot += s[i];
    double acc = 0;
    for (int j = 0; j < m; j++) {
        acc += s[j];
        if (rel && tot > 0) {
            double d = fabs(acc - 0.99 * tot) / tot;
            if (d < *rel) *rel = d;
        }
        if (acc >= 0.99 * tot) return j + 1;
    }
    return m;
}

/* ================================================================== */
/* Bounds of Ptilde on the cube (section 2.2.2): two-level truncated    */
/* SVD (eqs matrix1, SVD1-SVD7), 1-D cubic bounds, interval products,    */
/* residual bound (eq bound1), U and L (eqs bound2, bound3).             */
/* Unfolding read as A1[j][4k+l] (rows follow x, as U^i(x) requires).    */
/* out[0]=L out[1]=U out[2]=sum|R| out[3]=sum of |high-order| entries    */
/* out[4]=rank j  out[5]=sum of inner ranks                              */
/* ================================================================== */

static void or_bounds_r(const double *A, double *out, double *rank_rel);
void or_bounds(const double *A, double *out) { or_bounds_r(A, out, NULL); }

/* rank_rel (nullable): the smallest relative distance of a rank rule from
 * its threshold, as rank99_m */
static void or_bounds_r(const double *A, double *out, double *rank_rel)
{
    double s[4], u[16], v[64];
    or_svd_rows(A, 4, 16, s, u, v);
    double high = 0;
    for (int j = 0; j < 4; j++)
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++)
                if (j >= 2 || k >= 2 || l >= 2) high += fabs(A[16 * j + 4 * k + l]);
    double stot = s[0] + s[1] + s[2] + s[3];
    if (stot == 0) {
        out[0] = out[1] = out[2] = 0; out[3] = high; out[4] = 0; out[5] = 0;
        return;
    }
    int jr = rank99_m(s, 4, rank_rel);
    double At[64];
    memset(At, 0, sizeof(At));
    double M = 0, m = 0;
    int inner = 0;
    for (int i = 0; i < jr; i++) {
        double Vi[16], d[4], w[16], z[16];
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++) Vi[4 * k + l] = v[16 * i + 4 * k + l];
        or_svd_rows(Vi, 4, 4, d, w, z);
        int ji = rank99_m(d, 4, rank_rel);
        inner += ji;
        double Myz = 0, myz = 0;
        for (int k = 0; k < ji; k++) {
            double ly, hy, lz, hz;
            or_cubic_bounds(w + 4 * k, &ly, &hy);
            or_cubic_bounds(z + 4 * k, &lz, &hz);
            double p[4] = {hy * hz, hy * lz, ly * hz, ly * lz};
            double pmx = p[0], pmn = p[0];
            for (int t = 1; t < 4; t++) { if (p[t] > pmx) pmx = p[t]; if (p[t] < pmn) pmn = p[t]; }
            Myz += d[k] * pmx;
            myz += d[k] * pmn;
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++)
                    for (int cc = 0; cc < 4; cc++)
                        At[16 * a + 4 * b + cc] += s[i] * u[4 * i + a] * d[k] * w[4 * k + b] * z[4 * k + cc];
        }
        double lx, hx;
        or_cubic_bounds(u + 4 * i, &lx, &hx);
        double p[4] = {hx * Myz, hx * myz, lx * Myz, lx * myz};
        double pmx = p[0], pmn = p[0];
        for (int t = 1; t < 4; t++) { if (p[t] > pmx) pmx = p[t]; if (p[t] < pmn) pmn = p[t]; }
        M += s[i] * pmx;
        m += s[i] * pmn;
    }
    double sr = 0;
    for (int t = 0; t < 64; t++) sr += fabs(A[t] - At[t]);
    out[0] = m - sr;
    out[1] = M + sr;
    out[2] = sr;
    out[3] = high;
    out[4] = jr;
    out[5] = inner;
}

/* Decision (steps 1-3 of section 2.2, reading: bound test first, then the
 * trilinear-fit test, forced acceptance at max_depth). */
static int or_decide_r(const double *A, double c, double precision, int level, int max_depth, double *out6,
                       double *rank_rel)
{
    or_bounds_r(A, out6, rank_rel);
    double L = out6[0], U = out6[1];
    if (out6[4] == 0) return DEC_DISCARD; /* A == 0 */
    if (!(L <= c && c <= U)) return DEC_DISCARD;
    if (out6[3] <= precision) return DEC_ACCEPT;
    if (level >= max_depth) return DEC_FORCED;
    return DEC_SPLIT;
}
int or_decide(const double *A, double c, double precision, int level, int max_depth, double *out6)
{
    return or_decide_r(A, c, precision, level, max_depth, out6, NULL);
}

/* The alternative readings of section 2.2.3 and of steps 2-3 of section 2.2.
 * norm: the size of the coefficients A_jkl with max(j,k,l) >= 2 measured as
 * the sum of magnitudes (0), the largest magnitude (1) or the Euclidean norm
 * (2).  order 1 takes steps 2 and 3 as printed: a root cube goes through the
 * bound test (step 2) and, when kept, is divided (step 3); each child's
 * polynomial is then computed and, if its higher-order coefficients are under
 * the bound, the child is accepted as trilinear; otherwise it returns to
 * step 2 (bound test, then division).  A child without atoms (A = 0) has no
 * surface and is discarded under both orders. */
double or_high_norm(const double *A, int norm)
{
    double sum = 0, mx = 0, sq = 0;
    for (int j = 0; j < 4; j++)
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++) {
                if (j < 2 && k < 2 && l < 2) continue;
                double v = A[16 * j + 4 * k + l];
                sum += fabs(v);
                if (fabs(v) > mx) mx = fabs(v);
                sq += v * v;
            }
    if (norm == 1) return mx;
    if (norm == 2) return sqrt(sq);
    return sum;
}

static int or_decide_ex_r(const double *A, double c, double precision, int level, int max_depth, int order,
                          int norm, double *out6, double *rank_rel)
{
    if (order == 0 && norm == 0) return or_decide_r(A, c, precision, level, max_depth, out6, rank_rel);
    or_bounds_r(A, out6, rank_rel);
    out6[3] = or_high_norm(A, norm);
    double L = out6[0], U = out6[1];
    int has_atoms = out6[4] != 0;
    int trilinear = out6[3] <= precision;
    int straddles = L <= c && c <= U;
    if (!has_atoms) return DEC_DISCARD;
    if (order == 1) {
        if (level > 0 && trilinear) return DEC_ACCEPT;   /* step 3 on a child */
        if (!straddles) return DEC_DISCARD;               /* step 2 */
        if (level >= max_depth) return DEC_FORCED;
        return DEC_SPLIT;                                 /* step 3: divide */
    }
    if (!straddles) return DEC_DISCARD;
    if (trilinear) return DEC_ACCEPT;
    if (level >= max_depth) return DEC_FORCED;
    return DEC_SPLIT;
}
int or_decide_ex(const double *A, double c, double precision, int level, int max_depth, int order, int norm,
                 double *out6)
{
    return or_decide_ex_r(A, c, precision, level, max_depth, order, norm, out6, NULL);
}

/* ================================================================== */
/* Field at points (eq Gaussian1, same truncation, point distance).      */
/* ================================================================== */

static double phi_at(const oprob *P, const double *x, double *grad)
{
    double s = 0, g0 = 0, g1 = 0, g2 = 0;
    for (int64_t i = 0; i < P->n; i++) {
        const double *xi = P->xyz + 3 * i;
        double dx = x[0] - xi[0], dy = x[1] - xi[1], dz = x[2] - xi[2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > P->R2[i]) continue;
        double t = exp(-P->D * (d2 - P->r[i] * P->r[i]));
        s += t;
        g0 += -2 * P->D * dx * t;
        g1 += -2 * P->D * dy * t;
        g2 += -2 * P->D * dz * t;
    }
    if (grad) { grad[0] = g0; grad[1] = g1; grad[2] = g2; }
    return s;
}

/* ================================================================== */
/* Quad-precision resolution (the decision-margin policy).  A decision   */
/* or a vertex sign whose margin lies within 1e-10 of its threshold is   */
/* taken again with every step in IEEE binary128 (113-bit significand):  */
/* the Gauss-Legendre nodes, the 1-D coefficients with their C0          */
/* correction, the tensor, the Jacobi SVDs, the cubic ranges, the 99%    */
/* rank rules and the bounds of section 2.2.2; or the field sum of eq    */
/* (Gaussian1) at the vertex.  The atoms taken are those of the FP64      */
/* cutoff test (the truncation is part of the definition, not a          */
/* rounding).  x86-64: __float128 (libquadmath); AArch64: long double.   */
/* ================================================================== */
#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 oq;
#define QL(x) x##Q
#define QEXP expq
#define QSQRT sqrtq
#define QFABS fabsq
#define QCOS cosq
#define OR_HAVE_QUAD 1
#elif defined(__aarch64__) && (__LDBL_MANT_DIG__ == 113)
typedef long double oq;
#define QL(x) x##L
#define QEXP expl
#define QSQRT sqrtl
#define QFABS fabsl
#define QCOS cosl
#define OR_HAVE_QUAD 1
#else
#define OR_HAVE_QUAD 0
#endif

#if OR_HAVE_QUAD
static oq q_leg(int j, oq t)
{
    switch (j) {
    case 0: return 1;
    case 1: return t;
    case 2: return (3 * t * t - 1) / 2;
    default: return (5 * t * t * t - 3 * t) / 2;
    }
}

/* nodes and weights of the q-point rule, Newton on P_q from the usual guesses */
static void q_gauss_legendre(int q, oq *x, oq *w)
{
    const oq pi = (oq)QL(3.14159265358979323846264338327950288);
    for (int i = 0; i < q; i++) {
        oq t = QCOS(pi * ((oq)i + (oq)QL(0.75)) / ((oq)q + (oq)QL(0.5))), dp = 1;
        for (int it = 0; it < 200; it++) {
            oq p0 = 1, p1 = t;
            for (int k = 2; k <= q; k++) {
                oq p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = q * (t * p1 - p0) / (t * t - 1);
            oq dt = p1 / dp;
            t -= dt;
            if (QFABS(dt) < (oq)QL(1e-33)) break;
        }
        x[i] = t;
        w[i] = 2 / ((1 - t * t) * dp * dp);
    }
}

/* or_axis_coeffs in quad: the projection of exp(-D (x - xi)^2) on [a, b]
 * onto L_0..L_3 by the 24-point rule, then the C0 endpoint correction */
static void q_axis_coeffs(const oq *gx, const oq *gw, oq xi, oq a, oq b, oq D, oq *out4)
{
    oq m = (a + b) / 2, hh = (b - a) / 2, al[4];
    for (int j = 0; j < 4; j++) {
        oq s = 0;
        for (int k = 0; k < OR_Q; k++) {
            oq d = (m + hh * gx[k]) - xi;
            s += gw[k] * QEXP(-D * d * d) * q_leg(j, gx[k]);
        }
        al[j] = (oq)(2 * j + 1) / 2 * s;
    }
    oq fa = QEXP(-D * (a - xi) * (a - xi)), fb = QEXP(-D * (b - xi) * (b - xi));
    oq eR = fb - (al[0] + al[1] + al[2] + al[3]), eL = fa - (al[0] - al[1] + al[2] - al[3]);
    out4[0] = al[0];
    out4[1] = al[1];
    out4[2] = al[2] + (eR + eL) / 2;
    out4[3] = al[3] + (eR - eL) / 2;
}

static void q_jacobi_rows(oq *M, int m, int n, oq *Q)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) Q[i * m + j] = (i == j);
    for (int sweep = 0; sweep < 120; sweep++) {
        int rotated = 0;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) {
                oq al = 0, be = 0, ga = 0;
                for (int k = 0; k < n; k++) {
                    al += M[p * n + k] * M[p * n + k];
                    be += M[q * n + k] * M[q * n + k];
                    ga += M[p * n + k] * M[q * n + k];
                }
                if (ga == 0 || QFABS(ga) <= (oq)QL(1e-32) * QSQRT(al * be)) continue;
                rotated = 1;
                oq zeta = (be - al) / (2 * ga);
                oq t = (zeta >= 0 ? (oq)1 : (oq)-1) / (QFABS(zeta) + QSQRT(1 + zeta * zeta));
                oq cs = 1 / QSQRT(1 + t * t), sn = cs * t;
                for (int k = 0; k < n; k++) {
                    oq mp = M[p * n + k], mq = M[q * n + k];
                    M[p * n + k] = cs * mp - sn * mq;
                    M[q * n + k] = sn * mp + cs * mq;
                }
                for (int k = 0; k < m; k++) {
                    oq qp = Q[p * m + k], qq = Q[q * m + k];
                    Q[p * m + k] = cs * qp - sn * qq;
                    Q[q * m + k] = sn * qp + cs * qq;
                }
            }
        if (!rotated) break;
    }
}

static void q_svd_rows(const oq *X, int m, int n, oq *s, oq *u, oq *v)
{
    oq M[64], Q[16], sv[4];
    int order[4];
    memcpy(M, X, sizeof(oq) * (size_t)(m * n));
    q_jacobi_rows(M, m, n, Q);
    for (int p = 0; p < m; p++) {
        oq s2 = 0;
        for (int k = 0; k < n; k++) s2 += M[p * n + k] * M[p * n + k];
        sv[p] = QSQRT(s2);
        order[p] = p;
    }
    for (int i = 1; i < m; i++) {
        int o = order[i], j = i - 1;
        while (j >= 0 && sv[order[j]] < sv[o]) { order[j + 1] = order[j]; j--; }
        order[j + 1] = o;
    }
    for (int i = 0; i < m; i++) {
        int p = order[i];
        s[i] = sv[p];
        for (int k = 0; k < m; k++) u[i * m + k] = Q[p * m + k];
        for (int k = 0; k < n; k++) v[i * n + k] = sv[p] > 0 ? M[p * n + k] / sv[p] : 0;
    }
}

static void q_cubic_bounds(const oq *cf, oq *lo, oq *hi)
{
    oq c0 = cf[0], c1 = cf[1], c2 = cf[2], c3 = cf[3];
    oq m0 = c0 - c2 / 2, m1 = c1 - 3 * c3 / 2, m2 = 3 * c2 / 2, m3 = 5 * c3 / 2;
    oq vals[4], roots[2];
    int nv = 0, nr = 0;
    vals[nv++] = c0 + c1 + c2 + c3;
    vals[nv++] = c0 - c1 + c2 - c3;
    oq A2 = 3 * m3, B2 = 2 * m2, C2 = m1;
    if (A2 == 0) {
        if (B2 != 0) roots[nr++] = -C2 / B2;
    } else {
        oq disc = B2 * B2 - 4 * A2 * C2;
        if (disc >= 0) {
            oq sq = QSQRT(disc);
            oq qq = -(B2 + (B2 >= 0 ? sq : -sq)) / 2;
            if (qq != 0) { roots[nr++] = qq / A2; roots[nr++] = C2 / qq; }
            else roots[nr++] = 0;
        }
    }
    for (int i = 0; i < nr; i++) {
        oq t = roots[i];
        if (t > -1 && t < 1) vals[nv++] = m0 + t * (m1 + t * (m2 + t * m3));
    }
    oq a = vals[0], b = vals[0];
    for (int i = 1; i < nv; i++) { if (vals[i] < a) a = vals[i]; if (vals[i] > b) b = vals[i]; }
    *lo = a; *hi = b;
}

static int q_rank99(const oq *s, int m)
{
    oq tot = 0, acc = 0, thr;
    for (int i = 0; i < m; i++) tot += s[i];
    thr = (oq)QL(0.99) * tot;
    for (int j = 0; j < m; j++) {
        acc += s[j];
        if (acc >= thr) return j + 1;
    }
    return m;
}

/* or_bounds in quad: out = L, U, sum|R|, rank */
static void q_bounds(const oq *A, oq *out)
{
    oq s[4], u[16], v[64], At[64], Mx = 0, mn = 0;
    q_svd_rows(A, 4, 16, s, u, v);
    oq stot = s[0] + s[1] + s[2] + s[3];
    if (stot == 0) { out[0] = out[1] = out[2] = out[3] = 0; return; }
    int jr = q_rank99(s, 4);
    for (int t = 0; t < 64; t++) At[t] = 0;
    for (int i = 0; i < jr; i++) {
        oq Vi[16], d[4], w[16], z[16], Myz = 0, myz = 0;
        for (int t = 0; t < 16; t++) Vi[t] = v[16 * i + t];
        q_svd_rows(Vi, 4, 4, d, w, z);
        int ji = q_rank99(d, 4);
        for (int k = 0; k < ji; k++) {
            oq ly, hy, lz, hz;
            q_cubic_bounds(w + 4 * k, &ly, &hy);
            q_cubic_bounds(z + 4 * k, &lz, &hz);
            oq p[4] = {hy * hz, hy * lz, ly * hz, ly * lz}, pmx = p[0], pmn = p[0];
            for (int t = 1; t < 4; t++) { if (p[t] > pmx) pmx = p[t]; if (p[t] < pmn) pmn = p[t]; }
            Myz += d[k] * pmx;
            myz += d[k] * pmn;
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++)
                    for (int cc = 0; cc < 4; cc++)
                        At[16 * a + 4 * b + cc] += s[i] * u[4 * i + a] * d[k] * w[4 * k + b] * z[4 * k + cc];
        }
        oq lx, hx;
        q_cubic_bounds(u + 4 * i, &lx, &hx);
        oq p[4] = {hx * Myz, hx * myz, lx * Myz, lx * myz}, pmx = p[0], pmn = p[0];
        for (int t = 1; t < 4; t++) { if (p[t] > pmx) pmx = p[t]; if (p[t] < pmn) pmn = p[t]; }
        Mx += s[i] * pmx;
        mn += s[i] * pmn;
    }
    oq sr = 0;
    for (int t = 0; t < 64; t++) sr += QFABS(A[t] - At[t]);
    out[0] = mn - sr;
    out[1] = Mx + sr;
    out[2] = sr;
    out[3] = jr;
}

/* the tensor of cube [lo, hi] in quad (the atoms of the FP64 cutoff test) */
static int64_t q_cube_tensor(const oprob *P, const double *lo, const double *hi, oq *A)
{
    oq gx[OR_Q], gw[OR_Q];
    q_gauss_legendre(OR_Q, gx, gw);
    for (int t = 0; t < 64; t++) A[t] = 0;
    int64_t cnt = 0;
    const oq D = P->D;
    for (int64_t i = 0; i < P->n; i++) {
        const double *x = P->xyz + 3 * i;
        if (box_dist2(lo, hi, x) > P->R2[i]) continue;
        cnt++;
        oq ri = P->r[i], w = QEXP(D * ri * ri), ax[4], ay[4], az[4];
        q_axis_coeffs(gx, gw, x[0], lo[0], hi[0], D, ax);
        q_axis_coeffs(gx, gw, x[1], lo[1], hi[1], D, ay);
        q_axis_coeffs(gx, gw, x[2], lo[2], hi[2], D, az);
        for (int j = 0; j < 4; j++)
            for (int k = 0; k < 4; k++)
                for (int l = 0; l < 4; l++) A[16 * j + 4 * k + l] += w * ax[j] * ay[k] * az[l];
    }
    return cnt;
}

static int quad_decide(const oprob *P, const double *lo, const double *hi, int level, int *dec)
{
    oq A[64], b[4];
    q_cube_tensor(P, lo, hi, A);
    q_bounds(A, b);
    oq high = 0, mx = 0, sq = 0;
    for (int j = 0; j < 4; j++)
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++) {
                if (j < 2 && k < 2 && l < 2) continue;
                oq v = QFABS(A[16 * j + 4 * k + l]);
                high += v;
                if (v > mx) mx = v;
                sq += v * v;
            }
    if (P->norm == 1) high = mx;
    else if (P->norm == 2) high = QSQRT(sq);
    const oq c = P->c, prec = P->precision;
    const int straddles = b[0] <= c && c <= b[1], trilinear = high <= prec;
    if (b[3] == 0) *dec = DEC_DISCARD;
    else if (P->order == 1 && level > 0 && trilinear) *dec = DEC_ACCEPT;
    else if (!straddles) *dec = DEC_DISCARD;
    else if (P->order == 0 && trilinear) *dec = DEC_ACCEPT;
    else if (level >= P->max_depth) *dec = DEC_FORCED;
    else *dec = DEC_SPLIT;
    return 0;
}

/* eq (Gaussian1) at x in quad, the atoms of the FP64 cutoff test */
static int quad_phi(const oprob *P, const double *x, double *phi)
{
    oq s = 0;
    const oq D = P->D;
    for (int64_t i = 0; i < P->n; i++) {
        const double *xi = P->xyz + 3 * i;
        double dx = x[0] - xi[0], dy = x[1] - xi[1], dz = x[2] - xi[2];
        if (dx * dx + dy * dy + dz * dz > P->R2[i]) continue;
        oq qx = (oq)x[0] - (oq)xi[0], qy = (oq)x[1] - (oq)xi[1], qz = (oq)x[2] - (oq)xi[2], ri = P->r[i];
        s += QEXP(-D * (qx * qx + qy * qy + qz * qz - ri * ri));
    }
    *phi = (double)s;
    return 0;
}

/* pins of the quad path: the 1-D coefficients and the field as hi + lo
 * pairs of doubles (value = hi + lo to ~1e-32 relative) */
int or_axis_coeffs_quad(double xi, double a, double b, double D, double *hi4, double *lo4)
{
    oq gx[OR_Q], gw[OR_Q], o[4];
    q_gauss_legendre(OR_Q, gx, gw);
    q_axis_coeffs(gx, gw, xi, a, b, D, o);
    for (int j = 0; j < 4; j++) {
        hi4[j] = (double)o[j];
        lo4[j] = (double)(o[j] - (oq)hi4[j]);
    }
    return OR_OK;
}

int or_field_quad(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
                  int64_t np, const double *pts, double *hi, double *lo)
{
    oprob P;
    int e = oprob_init(&P, n, xyz, r, D, c, cutoff_rel, 1.0, 0.25, 0);
    if (e) return e;
    const oq Dq = D;
    for (int64_t k = 0; k < np; k++) {
        const double *x = pts + 3 * k;
        oq s = 0;
        for (int64_t i = 0; i < n; i++) {
            const double *xi = xyz + 3 * i;
            double dx = x[0] - xi[0], dy = x[1] - xi[1], dz = x[2] - xi[2];
            if (dx * dx + dy * dy + dz * dz > P.R2[i]) continue;
            oq qx = (oq)x[0] - (oq)xi[0], qy = (oq)x[1] - (oq)xi[1], qz = (oq)x[2] - (oq)xi[2], ri = r[i];
            s += QEXP(-Dq * (qx * qx + qy * qy + qz * qz - ri * ri));
        }
        hi[k] = (double)s;
        lo[k] = (double)(s - (oq)hi[k]);
    }
    oprob_free(&P);
    return OR_OK;
}

/* the bounds of section 2.2.2 in quad for a tensor given as hi + lo pairs:
 * out = L, U, sum|R|, rank (rounded to double) */
int or_bounds_quad(const double *Ahi, const double *Alo, double *out4)
{
    oq A[64], b[4];
    for (int t = 0; t < 64; t++) A[t] = (oq)Ahi[t] + (oq)Alo[t];
    q_bounds(A, b);
    for (int t = 0; t < 4; t++) out4[t] = (double)b[t];
    return OR_OK;
}
int or_have_quad(void) { return 1; }
#else
static int quad_decide(const oprob *P, const double *lo, const double *hi, int level, int *dec)
{
    (void)P; (void)lo; (void)hi; (void)level; (void)dec;
    return -1;
}
static int quad_phi(const oprob *P, const double *x, double *phi)
{
    (void)P; (void)x; (void)phi;
    return -1;
}
int or_have_quad(void) { return 0; }
#endif

/* ================================================================== */
/* Sorted uint64 sets                                                   */
/* ================================================================== */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}
static int64_t find_u64(const uint64_t *arr, int64_t n, uint64_t k)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (arr[mid] == k) return mid;
        if (arr[mid] < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}
static int64_t sort_unique(uint64_t *a, int64_t n)
{
    if (n <= 0) return 0;
    qsort(a, (size_t)n, sizeof(uint64_t), cmp_u64);
    int64_t m = 1;
    for (int64_t i = 1; i < n; i++)
        if (a[i] != a[m - 1]) a[m++] = a[i];
    return m;
}

typedef struct { uint64_t *a; int64_t n, cap; } vec64;
static int v_push(vec64 *v, uint64_t x)
{
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 1024;
        uint64_t *p = (uint64_t *)realloc(v->a, sizeof(uint64_t) * (size_t)nc);
        if (!p) return OR_ERR_OOM;
        v->a = p; v->cap = nc;
    }
    v->a[v->n++] = x;
    return OR_OK;
}

/* ================================================================== */
/* Adaptive partition (steps 1-3 of section 2.2), level by level.        */
/* ================================================================== */

typedef struct {
    int64_t examined[21], discarded[21], accepted[21], forced[21], split[21];
    int64_t pair_terms;       /* (cube, atom) terms inside the cutoff */
    int64_t conformity_splits;
    int64_t vertex_terms;
    int64_t n_vertices_lattice;
    int64_t n_cubes_final, n_cubes_surface;
    int64_t open_faces, degenerate_ears, loop_errors;
    double min_margin;        /* smallest |c-L|,|U-c|,|precision-high| seen (relative) */
    int64_t constrained_vertices; /* lattice vertices whose value is a coarser cube's interpolant */
    int64_t agreement_splits;     /* cubes split because a constrained value fell on the other side of c */
    /* decisions whose margin is below 1e-10 relative: [0] bound test, min(c-L, U-c) against |c|+|L|+|U|;
     * [1] precision test, |precision - sum|high|| against their sum; [2] a 99% rank rule, |sum_{i<=j} s_i -
     * 0.99 sum s| against sum s (outer and inner rules); [3] vertex sign, |value - c| against c, over the
     * final lattice values */
    int64_t near[4];
    int64_t resolved_cubes, resolved_vertices; /* re-decided in quad precision (resolve mode) */
    int64_t resolved_changed;                  /* cubes whose decision the quad evaluation changed */
    int64_t vertex_sign_changed;               /* vertices whose side of c the quad value changed */
} ostats;

static void cube_box(const oprob *P, uint64_t key, double *lo, double *hi)
{
    int64_t x, y, z;
    okey_xyz(key, &x, &y, &z);
    int l = (int)okey_level(key);
    int64_t ix[3] = {x, y, z};
    for (int a = 0; a < 3; a++) {
        lo[a] = lat_x(P, a, ix[a], l);
        hi[a] = lat_x(P, a, ix[a] + 1, l);
    }
}

/* Child tensor by re-expansion (the other reading of the child tensor, eq
 * childtensor): the Legendre coefficients, on child box c8, of the parent's
 * polynomial P~ = sum A_jkl L_j(s_x) L_k(s_y) L_l(s_z).  On the child's
 * local coordinates t in [-1,1]^3 the parent coordinate is s = (t + sigma)/2,
 * sigma = -1 for the lower half and +1 for the upper.  Coefficient
 * B_pqr = prod (2p+1)/2 times the integral of P~(s(t)) L_p L_q L_r over the
 * child cube, by 4-point Gauss-Legendre per axis (exact: degree <= 6). */
void or_child_reexpand(const double *A, int c8, double *B)
{
    double t4[4], w4[4];
    gauss_legendre(4, t4, w4);
    double sg[3] = {(c8 & 1) ? 1.0 : -1.0, ((c8 >> 1) & 1) ? 1.0 : -1.0, ((c8 >> 2) & 1) ? 1.0 : -1.0};
    for (int q = 0; q < 64; q++) B[q] = 0.0;
    for (int ix = 0; ix < 4; ix++)
        for (int iy = 0; iy < 4; iy++)
            for (int iz = 0; iz < 4; iz++) {
                double tx = t4[ix], ty = t4[iy], tz = t4[iz];
                double sx = (tx + sg[0]) / 2.0, sy = (ty + sg[1]) / 2.0, sz = (tz + sg[2]) / 2.0;
                double f = 0.0;
                for (int j = 0; j < 4; j++)
                    for (int k = 0; k < 4; k++)
                        for (int l = 0; l < 4; l++) f += A[16 * j + 4 * k + l] * leg(j, sx) * leg(k, sy) * leg(l, sz);
                double w = w4[ix] * w4[iy] * w4[iz];
                for (int p = 0; p < 4; p++)
                    for (int q = 0; q < 4; q++)
                        for (int r = 0; r < 4; r++)
                            B[16 * p + 4 * q + r] += (2 * p + 1) / 2.0 * (2 * q + 1) / 2.0 * (2 * r + 1) / 2.0 * w * f *
                                                     leg(p, tx) * leg(q, ty) * leg(r, tz);
            }
}

#define OR_NEAR 1e-10
static int quad_decide(const oprob *P, const double *lo, const double *hi, int level, int *dec);
static int quad_phi(const oprob *P, const double *x, double *phi);

static int partition(const oprob *P, vec64 *accepted, ostats *st, uint8_t *dec_log_unused)
{
    (void)dec_log_unused;
    vec64 cur = {0}, nxt = {0};
    for (int64_t z = 0; z < P->nroot[2]; z++)
        for (int64_t y = 0; y < P->nroot[1]; y++)
            for (int64_t x = 0; x < P->nroot[0]; x++)
                if (v_push(&cur, okey((uint64_t)x, (uint64_t)y, (uint64_t)z, T_CUBE, 0))) return OR_ERR_OOM;
    st->min_margin = INFINITY;
    /* child_mode 1: the tensors of the current cubes (children of the split
     * cubes of the previous level, in the order of cur) */
    double *curA = NULL, *nxtA = NULL;
    int64_t nxt_cap = 0;
    int e = OR_OK;
    for (int l = 0; l <= P->max_depth && cur.n > 0; l++) {
        st->examined[l] = cur.n;
        nxt.n = 0;
        /* each cube's tensor and decision depend on that cube alone: computed
         * in parallel, then taken in order */
        uint8_t *dec = (uint8_t *)malloc((size_t)cur.n);
        uint8_t *near = (uint8_t *)malloc((size_t)cur.n);   /* bits: bound, precision, rank; 8 resolved, 16 changed */
        double *marg = (double *)malloc(sizeof(double) * (size_t)cur.n);
        int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * (size_t)cur.n);
        double *keepA = P->child_mode == 1 ? (double *)malloc(sizeof(double) * 64 * (size_t)cur.n) : NULL;
        if (!dec || !near || !marg || !pairs || (P->child_mode == 1 && !keepA)) {
            free(dec); free(near); free(marg); free(pairs); free(keepA);
            e = OR_ERR_OOM;
            break;
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(OR_NT)
#endif
        for (int64_t q = 0; q < cur.n; q++) {
            double lo[3], hi[3], A[64], o6[6];
            cube_box(P, cur.a[q], lo, hi);
            pairs[q] = 0;
            if (P->child_mode == 1 && l > 0) memcpy(A, curA + 64 * q, sizeof(A));
            else pairs[q] = cube_tensor(P, lo, hi, A);
            double rrel = INFINITY;
            int d = or_decide_ex_r(A, P->c, P->precision, l, P->max_depth, P->order, P->norm, o6, &rrel);
            double mg = INFINITY;
            unsigned nb = 0;
            if (o6[4] > 0) {
                double scale = fabs(P->c) + fabs(o6[0]) + fabs(o6[1]);
                double mb = fmin(fabs(P->c - o6[0]), fabs(o6[1] - P->c)) / scale;
                mg = mb;
                if (mb < OR_NEAR) nb |= 1;
                if (rrel < OR_NEAR) nb |= 4;
                if (d != DEC_DISCARD) {
                    double mp = fabs(P->precision - o6[3]) / (P->precision + o6[3]);
                    mg = fmin(mg, mp);
                    if (mp < OR_NEAR) nb |= 2;
                }
            }
            if (nb && P->resolve && !(P->child_mode == 1 && l > 0)) {
                /* in band: the decision again, every step in quad precision */
                int dq = d;
                if (quad_decide(P, lo, hi, l, &dq) == 0) {
                    nb |= 8;
                    if (dq != d) { nb |= 16; d = dq; }
                }
            }
            dec[q] = (uint8_t)d;
            near[q] = (uint8_t)nb;
            marg[q] = mg;
            if (keepA) memcpy(keepA + 64 * q, A, sizeof(A));
        }
        for (int64_t q = 0; q < cur.n && !e; q++) {
            int d = dec[q];
            st->pair_terms += pairs[q];
            if (marg[q] < st->min_margin) st->min_margin = marg[q];
            for (int k = 0; k < 3; k++) st->near[k] += (near[q] >> k) & 1;
            st->resolved_cubes += (near[q] >> 3) & 1;
            st->resolved_changed += (near[q] >> 4) & 1;
            if (d == DEC_DISCARD) { st->discarded[l]++; continue; }
            if (d == DEC_ACCEPT || d == DEC_FORCED) {
                if (d == DEC_ACCEPT) st->accepted[l]++; else st->forced[l]++;
                if (v_push(accepted, cur.a[q])) e = OR_ERR_OOM;
                continue;
            }
            st->split[l]++;
            int64_t x, y, zz;
            okey_xyz(cur.a[q], &x, &y, &zz);
            for (int c8 = 0; c8 < 8 && !e; c8++) {
                if (v_push(&nxt, okey((uint64_t)(2 * x + (c8 & 1)), (uint64_t)(2 * y + ((c8 >> 1) & 1)),
                                      (uint64_t)(2 * zz + ((c8 >> 2) & 1)), T_CUBE, (unsigned)(l + 1)))) {
                    e = OR_ERR_OOM;
                    break;
                }
                if (P->child_mode == 1) {
                    if (nxt.n > nxt_cap) {
                        nxt_cap = 2 * nxt.n + 64;
                        double *g = (double *)realloc(nxtA, sizeof(double) * 64 * (size_t)nxt_cap);
                        if (!g) { e = OR_ERR_OOM; break; }
                        nxtA = g;
                    }
                    or_child_reexpand(keepA + 64 * q, c8, nxtA + 64 * (nxt.n - 1));
                }
            }
        }
        free(dec); free(near); free(marg); free(pairs); free(keepA);
        if (e) break;
        vec64 t = cur; cur = nxt; nxt = t;
        free(curA);
        curA = nxtA;
        nxtA = NULL;
        nxt_cap = 0;
    }
    free(cur.a); free(nxt.a);
    free(curA); free(nxtA);
    return e;
}

/* ================================================================== */
/* Mixed-size neighbours (section 2.3: the points of the neighbouring   */
/* cubes that lie in the current cube are taken into its loops, so that  */
/* cubes of different sizes join without cracks).                       */
/*                                                                       */
/* Reading (conform = 0): the accepted cubes keep their sizes, except    */
/* that a cube touching a cube two or more levels finer along a face or  */
/* an edge is split (to a fixpoint), so cubes that share a face or an    */
/* edge differ by at most one level.  A lattice vertex on a face or an   */
/* edge of a coarser final cube takes that cube's interpolant there      */
/* (constrain_values below), which makes the piecewise trilinear g       */
/* continuous; the triangulation then takes the finer neighbours' points */
/* on a shared face into the coarser cube's face curve, and the coarser  */
/* cube's extreme points into the finer cubes' curves.                   */
/* Reading conform = 1: every accepted cube touching any finer one is    */
/* split, until all cubes sharing a face or an edge have one size.       */
/* ================================================================== */

/* does the cube touch, along a face or an edge, a cube at least min_gap
 * levels finer? */
static int touches_finer(const uint64_t *S, int64_t n, uint64_t key, int max_depth, int min_gap)
{
    int64_t x, y, z;
    okey_xyz(key, &x, &y, &z);
    int l = (int)okey_level(key);
    for (int lf = l + min_gap; lf <= max_depth; lf++) {
        int64_t s = (int64_t)1 << (lf - l);
        int64_t I0[3] = {x * s, y * s, z * s};
        for (int64_t a = -1; a <= s; a++)
            for (int64_t b = -1; b <= s; b++)
                for (int64_t cc = -1; cc <= s; cc++) {
                    int out = (a < 0 || a >= s) + (b < 0 || b >= s) + (cc < 0 || cc >= s);
                    if (out == 0 || out == 3) continue;
                    int64_t X = I0[0] + a, Y = I0[1] + b, Z = I0[2] + cc;
                    if (X < 0 || Y < 0 || Z < 0) continue;
                    if (find_u64(S, n, okey((uint64_t)X, (uint64_t)Y, (uint64_t)Z, T_CUBE, (unsigned)lf)) >= 0)
                        return 1;
                }
    }
    return 0;
}

static int conformity(const oprob *P, vec64 *S, ostats *st)
{
    for (int pass = 0; pass < 64; pass++) {
        S->n = sort_unique(S->a, S->n);
        vec64 out = {0};
        int64_t splits = 0;
        for (int64_t i = 0; i < S->n; i++) {
            uint64_t k = S->a[i];
            int l = (int)okey_level(k);
            if (l < P->max_depth && touches_finer(S->a, S->n, k, P->max_depth, P->conform ? 1 : 2)) {
                int64_t x, y, z;
                okey_xyz(k, &x, &y, &z);
                for (int c8 = 0; c8 < 8; c8++)
                    if (v_push(&out, okey((uint64_t)(2 * x + (c8 & 1)), (uint64_t)(2 * y + ((c8 >> 1) & 1)),
                                          (uint64_t)(2 * z + ((c8 >> 2) & 1)), T_CUBE, (unsigned)(l + 1))))
                        return OR_ERR_OOM;
                splits++;
            } else if (v_push(&out, k)) return OR_ERR_OOM;
        }
        free(S->a);
        *S = out;
        st->conformity_splits += splits;
        if (splits == 0) { S->n = sort_unique(S->a, S->n); return OR_OK; }
    }
    return OR_ERR_CAP;
}

/* replace the cubes listed in R (sorted, unique, all members of S) by their
 * eight children */
static int split_listed(vec64 *S, const uint64_t *R, int64_t nr, int64_t *nsplit)
{
    vec64 out = {0};
    *nsplit = 0;
    for (int64_t i = 0; i < S->n; i++) {
        uint64_t k = S->a[i];
        if (find_u64(R, nr, k) < 0) {
            if (v_push(&out, k)) { free(out.a); return OR_ERR_OOM; }
            continue;
        }
        int64_t x, y, z;
        okey_xyz(k, &x, &y, &z);
        unsigned l = okey_level(k);
        for (int c8 = 0; c8 < 8; c8++)
            if (v_push(&out, okey((uint64_t)(2 * x + (c8 & 1)), (uint64_t)(2 * y + ((c8 >> 1) & 1)),
                                  (uint64_t)(2 * z + ((c8 >> 2) & 1)), T_CUBE, l + 1))) {
                free(out.a);
                return OR_ERR_OOM;
            }
        (*nsplit)++;
    }
    free(S->a);
    *S = out;
    S->n = sort_unique(S->a, S->n);
    return OR_OK;
}

/* Constrained vertex values.  A lattice vertex that lies on a face or an
 * edge of a coarser final cube without being one of its corners takes the
 * bilinear (face) or linear (edge) interpolant of that cube's corner values;
 * the coarsest cube touching the vertex decides, and the values are set
 * coarse to fine, so the corners it reads are final.  With these values the
 * trilinear functions of two cubes sharing a face agree on the whole face
 * (conforming hanging-node constraints of octree finite elements), so their
 * level curves there coincide.  Every other vertex keeps its field value.
 * The interpolant depends only on the face or edge (its corners in global
 * axis order and the vertex's fractions along it), not on which cube holds
 * it. */
typedef struct {
    int lev;          /* level of the constraining face or edge; -1: free (psi = phi) */
    int nsrc;         /* 2 (edge) or 4 (face) */
    int64_t src[4];   /* vertex indices: edge lower, upper; face (u0,w0) (u1,w0) (u0,w1) (u1,w1) */
    double t[2];      /* fractions along the edge, or along u and w on the face */
} ocons;

static int64_t vert_index(const uint64_t *vk, int64_t nv, int64_t X, int64_t Y, int64_t Z)
{
    if (X < 0 || Y < 0 || Z < 0) return -1;
    return find_u64(vk, nv, okey((uint64_t)X, (uint64_t)Y, (uint64_t)Z, T_VERT, 0));
}

static int constrain_values(const oprob *P, const uint64_t *cubes, int64_t nc, const uint64_t *vk, int64_t nv,
                            const double *phi, double *psi, ocons *cons)
{
    const int md = P->max_depth;
    for (int64_t i = 0; i < nv; i++) {
        ocons *K = &cons[i];
        K->lev = -1;
        K->nsrc = 0;
        psi[i] = phi[i];
        if (P->conform) continue;
        int64_t X[3];
        okey_xyz(vk[i], &X[0], &X[1], &X[2]);
        for (int l = 0; l < md; l++) {
            int64_t s = (int64_t)1 << (md - l);
            int al[3], na = 0;
            for (int a = 0; a < 3; a++) { al[a] = X[a] % s == 0; na += al[a]; }
            if (na == 0) continue;
            /* level-l cubes whose closed box holds the vertex */
            int found = 0;
            for (int c8 = 0; c8 < 8 && !found; c8++) {
                int64_t Q[3];
                int ok = 1;
                for (int a = 0; a < 3; a++) {
                    int bit = (c8 >> a) & 1;
                    if (!al[a] && bit) { ok = 0; break; }
                    Q[a] = X[a] / s - (al[a] && bit ? 1 : 0);
                    if (Q[a] < 0) { ok = 0; break; }
                }
                if (ok && find_u64(cubes, nc, okey((uint64_t)Q[0], (uint64_t)Q[1], (uint64_t)Q[2], T_CUBE,
                                                   (unsigned)l)) >= 0)
                    found = 1;
            }
            if (!found) continue;
            if (na == 3) break; /* a corner of the coarsest cube touching it: free */
            /* the face (one aligned axis) or edge (two) of level l holding it */
            int un[2], nu = 0;
            for (int a = 0; a < 3; a++)
                if (!al[a]) un[nu++] = a;
            int64_t base[3];
            for (int a = 0; a < 3; a++) base[a] = al[a] ? X[a] : (X[a] / s) * s;
            K->lev = l;
            K->nsrc = nu == 1 ? 2 : 4;
            for (int k = 0; k < nu; k++) K->t[k] = (double)(X[un[k]] - base[un[k]]) / (double)s;
            for (int q = 0; q < K->nsrc; q++) {
                int64_t Y[3] = {base[0], base[1], base[2]};
                for (int k = 0; k < nu; k++) Y[un[k]] += ((q >> k) & 1) ? s : 0;
                K->src[q] = vert_index(vk, nv, Y[0], Y[1], Y[2]);
                if (K->src[q] < 0) return OR_ERR_CAP;
            }
            break;
        }
    }
    /* coarse to fine: a source's own constraint is of a coarser level */
    for (int l = 0; l < md; l++)
        for (int64_t i = 0; i < nv; i++) {
            const ocons *K = &cons[i];
            if (K->lev != l) continue;
            if (K->nsrc == 2) {
                double a = psi[K->src[0]], b = psi[K->src[1]];
                psi[i] = a + K->t[0] * (b - a);
            } else {
                double q00 = psi[K->src[0]], q10 = psi[K->src[1]], q01 = psi[K->src[2]], q11 = psi[K->src[3]];
                double e0 = q00 + K->t[0] * (q10 - q00);
                double e1 = q01 + K->t[0] * (q11 - q01);
                psi[i] = e0 + K->t[1] * (e1 - e0);
            }
        }
    return OR_OK;
}

/* Disagreement (the split rule for cubes of different sizes): a vertex
 * whose constrained value and field value lie on different sides of c
 * would put the surface where the finer cubes, or the cubes discarded next
 * to them, have none.  Every final cube of the constraining level that
 * holds such a vertex on its boundary is listed for splitting. */
static int disagreeing_cubes(const oprob *P, const uint64_t *cubes, int64_t nc, const uint64_t *vk, int64_t nv,
                             const double *phi, const double *psi, const ocons *cons, vec64 *R)
{
    const int md = P->max_depth;
    const double c = P->c;
    for (int64_t i = 0; i < nv; i++) {
        if (cons[i].lev < 0 || (psi[i] >= c) == (phi[i] >= c)) continue;
        int l = cons[i].lev;
        int64_t s = (int64_t)1 << (md - l);
        int64_t X[3];
        okey_xyz(vk[i], &X[0], &X[1], &X[2]);
        for (int c8 = 0; c8 < 8; c8++) {
            int64_t Q[3];
            int ok = 1;
            for (int a = 0; a < 3; a++) {
                int al = X[a] % s == 0, bit = (c8 >> a) & 1;
                if (!al && bit) { ok = 0; break; }
                Q[a] = X[a] / s - (al && bit ? 1 : 0);
                if (Q[a] < 0) { ok = 0; break; }
            }
            if (!ok) continue;
            uint64_t k = okey((uint64_t)Q[0], (uint64_t)Q[1], (uint64_t)Q[2], T_CUBE, (unsigned)l);
            if (find_u64(cubes, nc, k) >= 0 && v_push(R, k)) return OR_ERR_OOM;
        }
    }
    R->n = sort_unique(R->a, R->n);
    return OR_OK;
}

/* ================================================================== */
/* Per-cube trilinear surface (eq linear1) and its triangulation         */
/* (section 2.3, eqs intersection, curve, fold1, critical).              */
/* Local coordinates in [0,1]^3; corner v = bx + 2 by + 4 bz.            */
/* ================================================================== */

typedef struct {
    double p[3];   /* local coords */
    double w[3];   /* world coords, computed in the frame of the cube (or edge) the point belongs to */
    uint64_t key;
    int kind;      /* 0 edge point, 1 own extreme point, 2 neighbour's extreme point, 3 critical point */
    int nb[4];     /* fold neighbours: extreme point -> nb[0]; critical point -> +a, -a, +b, -b */
    int fa, fb;    /* critical point: the two fold axes (fa < fb) */
    int rh;        /* critical point: (+a, +b, outward normal) is right-handed */
} opoint;

#define MAXP 64
#define FPMAX 20 /* points inserted into one face curve */
#ifdef OR_DEBUG
#include <stdio.h>
#define LOOPERR(site) do { st->loop_errors++; fprintf(stderr, "looperr site %d cube %llx\n", site, (unsigned long long)ckey); } while (0)
#else
#define LOOPERR(site) (st->loop_errors++)
#endif

/* other two axes of a in increasing order */
static void other_axes(int a, int *u, int *v)
{
    *u = a == 0 ? 1 : 0;
    *v = a == 2 ? 1 : 2;
}

/* corner value with per-axis bits */
static double gv(const double *g, int bx, int by, int bz) { return g[bx | (by << 1) | (bz << 2)]; }

/* Fold lines along axis a (eq fold1): g = A(u,v) + s B(u,v) with s the
 * coordinate along a; the fold set {dg/ds = 0, g = c} = {B = 0, A = c} is a
 * set of segments parallel to a at the (u,v) roots.  Returns the roots that
 * lie strictly inside the unit square, ordered by u then v. */
static int fold_roots(const double *g, int a, double c, double ru[2], double rv[2])
{
    int ua, va;
    other_axes(a, &ua, &va);
    double A00, A10, A01, A11, B00, B10, B01, B11;
    int b[3];
    double F0[4], F1[4];
    for (int iv = 0; iv < 2; iv++)
        for (int iu = 0; iu < 2; iu++) {
            b[a] = 0; b[ua] = iu; b[va] = iv;
            F0[iu + 2 * iv] = gv(g, b[0], b[1], b[2]);
            b[a] = 1;
            F1[iu + 2 * iv] = gv(g, b[0], b[1], b[2]);
        }
    A00 = F0[0]; A10 = F0[1]; A01 = F0[2]; A11 = F0[3];
    B00 = F1[0] - F0[0]; B10 = F1[1] - F0[1]; B01 = F1[2] - F0[2]; B11 = F1[3] - F0[3];
    /* bilinear monomials: A = a0 + a1 u + a2 v + a3 uv (minus c), B likewise */
    double a0 = A00 - c, a1 = A10 - A00, a2 = A01 - A00, a3 = A11 - A10 - A01 + A00;
    double b0 = B00, b1 = B10 - B00, b2 = B01 - B00, b3 = B11 - B10 - B01 + B00;
    if (b0 == 0 && b1 == 0 && b2 == 0 && b3 == 0) return 0; /* g independent of s: no fold */
    /* eliminate v: from B = 0, v (b2 + b3 u) = -(b0 + b1 u);  A = 0 gives
     * (a0 + a1 u)(b2 + b3 u) - (a2 + a3 u)(b0 + b1 u) = 0 */
    double q2 = a1 * b3 - a3 * b1;
    double q1 = a0 * b3 + a1 * b2 - a2 * b1 - a3 * b0;
    double q0 = a0 * b2 - a2 * b0;
    double us[2];
    int nu = 0;
    if (q2 == 0) {
        if (q1 != 0) us[nu++] = -q0 / q1;
    } else {
        double disc = q1 * q1 - 4 * q2 * q0;
        if (disc >= 0) {
            double sq = sqrt(disc);
            double qq = -0.5 * (q1 + (q1 >= 0 ? sq : -sq));
            if (qq != 0) { us[nu++] = qq / q2; us[nu++] = q0 / qq; }
            else us[nu++] = 0.0;
            if (nu == 2 && us[0] == us[1]) nu = 1;
        }
    }
    /* both end faces must carry a face curve for the segment to end on it */
    int f0in = 0, f1in = 0;
    for (int k = 0; k < 4; k++) { f0in += F0[k] >= c; f1in += F1[k] >= c; }
    if (f0in == 0 || f0in == 4 || f1in == 0 || f1in == 4) return 0;
    double sa = fabs(a0) + fabs(a1) + fabs(a2) + fabs(a3);
    double sb = fabs(b0) + fabs(b1) + fabs(b2) + fabs(b3);
    int nr = 0;
    for (int i = 0; i < nu; i++) {
        double u = us[i];
        if (!(u > 0 && u < 1)) continue;
        /* v from B = 0 or from A = c, whichever is better conditioned at u
         * (B = 0 degenerates when B has a factor (b2 + b3 u) vanishing at the
         * root; A = c likewise); keep a candidate only if it solves both */
        double dB = b2 + b3 * u, dA = a2 + a3 * u;
        double cand[2];
        int nc = 0;
        if (fabs(dB) >= fabs(dA)) {
            if (dB != 0) cand[nc++] = -(b0 + b1 * u) / dB;
            if (dA != 0) cand[nc++] = -(a0 + a1 * u) / dA;
        } else {
            if (dA != 0) cand[nc++] = -(a0 + a1 * u) / dA;
            if (dB != 0) cand[nc++] = -(b0 + b1 * u) / dB;
        }
        for (int k = 0; k < nc; k++) {
            double v = cand[k];
            if (!(v > 0 && v < 1)) continue;
            if (fabs(a0 + a1 * u + a2 * v + a3 * u * v) > 1e-9 * sa) continue;
            if (fabs(b0 + b1 * u + b2 * v + b3 * u * v) > 1e-9 * sb) continue;
            ru[nr] = u; rv[nr] = v; nr++;
            break;
        }
    }
    if (nr == 2 && (ru[1] < ru[0] || (ru[1] == ru[0] && rv[1] < rv[0]))) {
        double t = ru[0]; ru[0] = ru[1]; ru[1] = t;
        t = rv[0]; rv[0] = rv[1]; rv[1] = t;
    }
    return nr;
}

typedef struct {
    const oprob *P;
    const uint64_t *cubes; int64_t ncubes;
    const uint64_t *vkeys; const double *vphi; int64_t nv;
} omesh_ctx;

static int lookup_phi(const omesh_ctx *M, int64_t X, int64_t Y, int64_t Z, double *out)
{
    if (X < 0 || Y < 0 || Z < 0) return 0;
    int64_t i = find_u64(M->vkeys, M->nv, okey((uint64_t)X, (uint64_t)Y, (uint64_t)Z, T_VERT, 0));
    if (i < 0) return 0;
    *out = M->vphi[i];
    return 1;
}

/* 8 corner values of the level-l cube at lattice (x,y,z); 0 if missing */
static int cube_values(const omesh_ctx *M, int l, int64_t x, int64_t y, int64_t z, double *g)
{
    int64_t s = (int64_t)1 << (M->P->max_depth - l);
    for (int v = 0; v < 8; v++)
        if (!lookup_phi(M, (x + (v & 1)) * s, (y + ((v >> 1) & 1)) * s, (z + ((v >> 2) & 1)) * s, &g[v]))
            return 0;
    return 1;
}

typedef struct { uint64_t k[3]; int64_t piece; } otri;
typedef struct { otri *t; int64_t n, cap; int64_t piece; } vtri;
static int t_push(vtri *v, uint64_t a, uint64_t b, uint64_t c)
{
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 1024;
        otri *p = (otri *)realloc(v->t, sizeof(otri) * (size_t)nc);
        if (!p) return OR_ERR_OOM;
        v->t = p; v->cap = nc;
    }
    v->t[v->n].k[0] = a; v->t[v->n].k[1] = b; v->t[v->n].k[2] = c;
    v->t[v->n].piece = v->piece;
    v->n++;
    return OR_OK;
}

typedef struct { uint64_t key; double x[3]; } overt;
typedef struct { overt *p; int64_t n, cap; } vvert;
static int p_push(vvert *v, uint64_t key, const double *x)
{
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 1024;
        overt *p = (overt *)realloc(v->p, sizeof(overt) * (size_t)nc);
        if (!p) return OR_ERR_OOM;
        v->p = p; v->cap = nc;
    }
    v->p[v->n].key = key;
    memcpy(v->p[v->n].x, x, sizeof(double) * 3);
    v->n++;
    return OR_OK;
}

/* 2-D orientation of (a,b,c) in the plane of axes (i,j) */
static double orient2(const double *a, const double *b, const double *c, int i, int j)
{
    return (b[i] - a[i]) * (c[j] - a[j]) - (b[j] - a[j]) * (c[i] - a[i]);
}

/* Ear clipping (two-ears theorem; Meisters) of one single-valued piece,
 * projected along the axis of largest |Newell normal|.  The clipped ear is
 * always the valid (convex, empty) ear whose tip has the smallest key. */
static int ear_clip(const opoint *pts, const int *poly, int n, vtri *tris, ostats *st)
{
    double N[3] = {0, 0, 0};
    for (int i = 0; i < n; i++) {
        const double *p = pts[poly[i]].p, *q = pts[poly[(i + 1) % n]].p;
        N[0] += (p[1] - q[1]) * (p[2] + q[2]);
        N[1] += (p[2] - q[2]) * (p[0] + q[0]);
        N[2] += (p[0] - q[0]) * (p[1] + q[1]);
    }
    int k = 0;
    if (fabs(N[1]) > fabs(N[k])) k = 1;
    if (fabs(N[2]) > fabs(N[k])) k = 2;
    int ia = (k + 1) % 3, ib = (k + 2) % 3;
    double sg = N[k] >= 0 ? 1.0 : -1.0;
    int idx[MAXP];
    int m = n;
    for (int i = 0; i < n; i++) idx[i] = poly[i];
    while (m > 3) {
        int best = -1, fb = -1;
        for (int i = 0; i < m; i++) {
            int a = idx[(i + m - 1) % m], b = idx[i], c = idx[(i + 1) % m];
            double cr = sg * orient2(pts[a].p, pts[b].p, pts[c].p, ia, ib);
            if (fb < 0 || pts[b].key < pts[idx[fb]].key) fb = i;
            if (!(cr > 0)) continue;
            int empty = 1;
            for (int j = 0; j < m && empty; j++) {
                int d = idx[j];
                if (d == a || d == b || d == c) continue;
                const double *pd = pts[d].p;
                double s1 = sg * orient2(pts[a].p, pts[b].p, pd, ia, ib);
                double s2 = sg * orient2(pts[b].p, pts[c].p, pd, ia, ib);
                double s3 = sg * orient2(pts[c].p, pts[a].p, pd, ia, ib);
                if (s1 >= 0 && s2 >= 0 && s3 >= 0) empty = 0;
            }
            if (!empty) continue;
            if (best < 0 || pts[b].key < pts[idx[best]].key) best = i;
        }
        if (best < 0) { best = fb; st->degenerate_ears++; }
        int a = idx[(best + m - 1) % m], b = idx[best], c = idx[(best + 1) % m];
        if (a != b && b != c && a != c)
            if (t_push(tris, pts[a].key, pts[b].key, pts[c].key)) return OR_ERR_OOM;
        for (int j = best; j < m - 1; j++) idx[j] = idx[j + 1];
        m--;
    }
    if (m == 3 && idx[0] != idx[1] && idx[1] != idx[2] && idx[0] != idx[2])
        if (t_push(tris, pts[idx[0]].key, pts[idx[1]].key, pts[idx[2]].key)) return OR_ERR_OOM;
    return OR_OK;
}

static int new_point(opoint *pts, int *np, int kind)
{
    if (*np >= MAXP) return -1;
    opoint *p = &pts[*np];
    memset(p, 0, sizeof(*p));
    p->kind = kind;
    p->nb[0] = p->nb[1] = p->nb[2] = p->nb[3] = -1;
    return (*np)++;
}

static int triangulate_cube(const omesh_ctx *M, uint64_t ckey, vtri *tris, vvert *verts, ostats *st)
{
    const oprob *P = M->P;
    int l = (int)okey_level(ckey);
    int64_t cx, cy, cz;
    okey_xyz(ckey, &cx, &cy, &cz);
    int64_t s = (int64_t)1 << (P->max_depth - l);
    int64_t C[3] = {cx, cy, cz};
    double g[8];
    if (!cube_values(M, l, cx, cy, cz, g)) return OR_ERR_CAP;
    double c = P->c;
    int nin = 0;
    for (int v = 0; v < 8; v++) nin += g[v] >= c;
    if (nin == 0 || nin == 8) return OR_OK;
    st->n_cubes_surface++;

    opoint pts[MAXP];
    int np = 0;
    const int fine_ok = P->conform == 0 && l < P->max_depth;
    const int64_t s2 = s / 2; /* the finer level's step (with fine_ok) */
    /* edge points (eq intersection): eid[a][o1][o2], o1/o2 = bits of the
     * other two axes in increasing axis order.  An edge that a finer cube
     * touches is halved (its midpoint is a lattice vertex): the point is the
     * crossing on the half where the sign changes, keyed by that half. */
    int eid[3][2][2];
    for (int a = 0; a < 3; a++) {
        int ua, va;
        other_axes(a, &ua, &va);
        for (int o1 = 0; o1 < 2; o1++)
            for (int o2 = 0; o2 < 2; o2++) {
                int b0[3], b1[3];
                b0[a] = 0; b1[a] = 1; b0[ua] = b1[ua] = o1; b0[va] = b1[va] = o2;
                double g0 = gv(g, b0[0], b0[1], b0[2]), g1 = gv(g, b1[0], b1[1], b1[2]);
                eid[a][o1][o2] = -1;
                if ((g0 >= c) == (g1 >= c)) continue;
                int id = new_point(pts, &np, 0);
                if (id < 0) { LOOPERR(9); return OR_OK; }
                opoint *p = &pts[id];
                int64_t L[3];
                L[a] = C[a] * s; L[ua] = (C[ua] + o1) * s; L[va] = (C[va] + o2) * s;
                double gm;
                int64_t Lm[3] = {L[0], L[1], L[2]};
                Lm[a] += s2;
                if (fine_ok && lookup_phi(M, Lm[0], Lm[1], Lm[2], &gm)) {
                    int half = (g0 >= c) == (gm >= c); /* 0: first half, 1: second */
                    double ga = half ? gm : g0, gb = half ? g1 : gm;
                    double t = (c - ga) / (gb - ga);
                    p->p[a] = (half + t) * 0.5;
                    L[a] += half * s2;
                    p->key = okey((uint64_t)L[0], (uint64_t)L[1], (uint64_t)L[2], (unsigned)a, (unsigned)(l + 1));
                    p->w[a] = wfrac(P, a, 2 * C[a] + half, l + 1, t);
                } else {
                    double t = (c - g0) / (g1 - g0);
                    p->p[a] = t;
                    p->key = okey((uint64_t)L[0], (uint64_t)L[1], (uint64_t)L[2], (unsigned)a, (unsigned)l);
                    p->w[a] = wfrac(P, a, C[a], l, t);
                }
                p->p[ua] = o1; p->p[va] = o2;
                p->w[ua] = lat_x(P, ua, L[ua], P->max_depth);
                p->w[va] = lat_x(P, va, L[va], P->max_depth);
                eid[a][o1][o2] = id;
            }
    }
    /* Own fold lines (eq fold1) along each axis: a segment across the cube
     * whose ends on the two faces normal to the axis are extreme points
     * (eq curve).  A neighbour's folds end on the face it shares with this
     * cube; they become further points of that face curve. */
    int fp[3][2][FPMAX];
    int nfp[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    double fr[3][2][2];   /* own roots: fr[a][r] = (u, v) */
    int fend[3][2][2];    /* own fold ends: fend[a][r][side] */
    int nfr[3];
    for (int a = 0; a < 3; a++) {
        double ru[2], rv[2];
        nfr[a] = fold_roots(g, a, c, ru, rv);
        for (int r = 0; r < nfr[a]; r++) { fr[a][r][0] = ru[r]; fr[a][r][1] = rv[r]; }
    }
    /* Critical points (eq critical): in the slice through an a-fold line
     * normal to a third axis, the level set of the bilinear slice function
     * is a pair of crossing lines, so fold lines of two axes meet whenever
     * their roots share the coordinate of the remaining axis.  That shared
     * coordinate is one number; the later fold takes the earlier fold's
     * value, so every segment along a fold line is exactly axis-parallel. */
    int xing[12][4], nx = 0;
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++) {
            int cc = 3 - a - b;
            int ua, va, ub, vb;
            other_axes(a, &ua, &va);
            other_axes(b, &ub, &vb);
            for (int i = 0; i < nfr[a]; i++)
                for (int j = 0; j < nfr[b]; j++) {
                    double ca = fr[a][i][cc == ua ? 0 : 1];
                    double cb = fr[b][j][cc == ub ? 0 : 1];
                    if (fabs(ca - cb) > 1e-9) continue;
                    fr[b][j][cc == ub ? 0 : 1] = ca;
                    xing[nx][0] = a; xing[nx][1] = i; xing[nx][2] = b; xing[nx][3] = j;
                    nx++;
                }
        }
    for (int a = 0; a < 3; a++) {
        int ua, va;
        other_axes(a, &ua, &va);
        for (int r = 0; r < nfr[a]; r++) {
            for (int sd = 0; sd < 2; sd++) {
                int id = new_point(pts, &np, 1);
                if (id < 0) { LOOPERR(9); return OR_OK; }
                opoint *p = &pts[id];
                p->p[a] = sd; p->p[ua] = fr[a][r][0]; p->p[va] = fr[a][r][1];
                int64_t L[3] = {C[0] * s, C[1] * s, C[2] * s};
                L[a] = (C[a] + sd) * s;
                /* face at sd=0: this cube lies on its + side; sd=1: - side */
                unsigned type = 8u + 4u * (unsigned)a + 2u * (unsigned)(sd == 0) + (unsigned)r;
                p->key = okey((uint64_t)L[0], (uint64_t)L[1], (uint64_t)L[2], type, (unsigned)l);
                for (int q = 0; q < 3; q++) p->w[q] = wfrac(P, q, C[q], l, p->p[q]);
                fend[a][r][sd] = id;
                fp[a][sd][nfp[a][sd]++] = id;
            }
        }
        /* Across each face normal to a: the points of the neighbouring cubes
         * that lie on it (section 2.3).  A neighbour of the same size adds its
         * a-fold ends; finer neighbours (four tiles of the face) add their
         * a-fold ends and the points on the face's inner half-lines, which
         * are their edges; a coarser neighbour adds those of its a-fold ends
         * that fall in this face (the quarter of its face that this cube
         * covers, halves taken as [0, 1/2) and [1/2, 1]).  All of them lie
         * on this face's level curve: the tiles' and this face's values are
         * one bilinear function (constrained vertex values). */
        for (int sd = 0; sd < 2; sd++) {
            int64_t N[3] = {C[0], C[1], C[2]};
            N[a] += sd ? 1 : -1;
            if (N[a] < 0) continue;
            uint64_t nk = okey((uint64_t)N[0], (uint64_t)N[1], (uint64_t)N[2], T_CUBE, (unsigned)l);
            if (find_u64(M->cubes, M->ncubes, nk) >= 0) {
                double gn[8];
                if (!cube_values(M, l, N[0], N[1], N[2], gn)) return OR_ERR_CAP;
                double nu_[2], nv_[2];
                int nn = fold_roots(gn, a, c, nu_, nv_);
                for (int r = 0; r < nn; r++) {
                    int id = new_point(pts, &np, 2);
                    if (id < 0 || nfp[a][sd] >= FPMAX) { LOOPERR(9); return OR_OK; }
                    opoint *p = &pts[id];
                    p->p[a] = sd; p->p[ua] = nu_[r]; p->p[va] = nv_[r];
                    int64_t L[3] = {C[0] * s, C[1] * s, C[2] * s};
                    L[a] = (C[a] + sd) * s;
                    /* the neighbour lies on the + side of the shared face iff sd = 1 */
                    unsigned type = 8u + 4u * (unsigned)a + 2u * (unsigned)(sd == 1) + (unsigned)r;
                    p->key = okey((uint64_t)L[0], (uint64_t)L[1], (uint64_t)L[2], type, (unsigned)l);
                    for (int q = 0; q < 3; q++) p->w[q] = wfrac(P, q, C[q], l, p->p[q]);
                    fp[a][sd][nfp[a][sd]++] = id;
                }
                continue;
            }
            if (P->conform) continue;
            /* the neighbouring cube's side of the shared plane */
            const int side_n = sd ? 0 : 1;
            const int64_t plane = (C[a] + sd) * s; /* finest-lattice coordinate of the face */
            if (fine_ok) {
                int tex[2][2];
                int64_t T[2][2][3];
                int ntile = 0;
                for (int iv = 0; iv < 2; iv++)
                    for (int iu = 0; iu < 2; iu++) {
                        int64_t *t3 = T[iu][iv];
                        t3[a] = 2 * N[a] + side_n; t3[ua] = 2 * C[ua] + iu; t3[va] = 2 * C[va] + iv;
                        tex[iu][iv] = find_u64(M->cubes, M->ncubes,
                                               okey((uint64_t)t3[0], (uint64_t)t3[1], (uint64_t)t3[2], T_CUBE,
                                                    (unsigned)(l + 1))) >= 0;
                        ntile += tex[iu][iv];
                    }
                if (ntile > 0) {
                    /* the tiles' fold ends on this face */
                    for (int iv = 0; iv < 2; iv++)
                        for (int iu = 0; iu < 2; iu++) {
                            if (!tex[iu][iv]) continue;
                            const int64_t *t3 = T[iu][iv];
                            double gt[8];
                            if (!cube_values(M, l + 1, t3[0], t3[1], t3[2], gt)) return OR_ERR_CAP;
                            double tu[2], tv[2];
                            int nn = fold_roots(gt, a, c, tu, tv);
                            for (int r = 0; r < nn; r++) {
                                int id = new_point(pts, &np, 2);
                                if (id < 0 || nfp[a][sd] >= FPMAX) { LOOPERR(9); return OR_OK; }
                                opoint *p = &pts[id];
                                p->p[a] = sd; p->p[ua] = (iu + tu[r]) * 0.5; p->p[va] = (iv + tv[r]) * 0.5;
                                int64_t L[3] = {t3[0] * s2, t3[1] * s2, t3[2] * s2};
                                L[a] = plane;
                                unsigned type = 8u + 4u * (unsigned)a + 2u * (unsigned)(side_n == 0) + (unsigned)r;
                                p->key = okey((uint64_t)L[0], (uint64_t)L[1], (uint64_t)L[2], type, (unsigned)(l + 1));
                                p->w[a] = lat_x(P, a, plane, P->max_depth);
                                p->w[ua] = wfrac(P, ua, t3[ua], l + 1, tu[r]);
                                p->w[va] = wfrac(P, va, t3[va], l + 1, tv[r]);
                                fp[a][sd][nfp[a][sd]++] = id;
                            }
                        }
                    /* the inner half-lines: along u at v = 1/2 (halves k),
                     * then along v at u = 1/2; a half-line is an edge of the
                     * tiles on either side of it */
                    for (int dir = 0; dir < 2; dir++)
                        for (int k = 0; k < 2; k++) {
                            int along = dir ? va : ua, across = dir ? ua : va;
                            int has = dir ? (tex[0][k] || tex[1][k]) : (tex[k][0] || tex[k][1]);
                            if (!has) continue;
                            int64_t L0[3];
                            L0[a] = plane;
                            L0[along] = C[along] * s + k * s2;
                            L0[across] = C[across] * s + s2;
                            int64_t L1[3] = {L0[0], L0[1], L0[2]};
                            L1[along] += s2;
                            double ga, gb;
                            if (!lookup_phi(M, L0[0], L0[1], L0[2], &ga) || !lookup_phi(M, L1[0], L1[1], L1[2], &gb)) {
                                LOOPERR(10);
                                return OR_OK;
                            }
                            if ((ga >= c) == (gb >= c)) continue;
                            int id = new_point(pts, &np, 2);
                            if (id < 0 || nfp[a][sd] >= FPMAX) { LOOPERR(9); return OR_OK; }
                            opoint *p = &pts[id];
                            double t = (c - ga) / (gb - ga);
                            p->p[a] = sd; p->p[along] = (k + t) * 0.5; p->p[across] = 0.5;
                            p->key = okey((uint64_t)L0[0], (uint64_t)L0[1], (uint64_t)L0[2], (unsigned)along,
                                          (unsigned)(l + 1));
                            p->w[a] = lat_x(P, a, plane, P->max_depth);
                            p->w[along] = wfrac(P, along, 2 * C[along] + k, l + 1, t);
                            p->w[across] = lat_x(P, across, L0[across], P->max_depth);
                            fp[a][sd][nfp[a][sd]++] = id;
                        }
                    continue;
                }
            }
            if (l > 0) {
                int64_t Q[3] = {N[0] >> 1, N[1] >> 1, N[2] >> 1};
                if (find_u64(M->cubes, M->ncubes,
                             okey((uint64_t)Q[0], (uint64_t)Q[1], (uint64_t)Q[2], T_CUBE, (unsigned)(l - 1))) < 0)
                    continue;
                double gq[8];
                if (!cube_values(M, l - 1, Q[0], Q[1], Q[2], gq)) return OR_ERR_CAP;
                double qu_[2], qv_[2];
                int nn = fold_roots(gq, a, c, qu_, qv_);
                const int64_t su = C[ua] - 2 * Q[ua], sv = C[va] - 2 * Q[va]; /* this face's quarter */
                for (int r = 0; r < nn; r++) {
                    if ((qu_[r] >= 0.5) != (su == 1) || (qv_[r] >= 0.5) != (sv == 1)) continue;
                    int id = new_point(pts, &np, 2);
                    if (id < 0 || nfp[a][sd] >= FPMAX) { LOOPERR(9); return OR_OK; }
                    opoint *p = &pts[id];
                    p->p[a] = sd; p->p[ua] = 2.0 * qu_[r] - (double)su; p->p[va] = 2.0 * qv_[r] - (double)sv;
                    int64_t L[3] = {Q[0] * 2 * s, Q[1] * 2 * s, Q[2] * 2 * s};
                    L[a] = plane;
                    unsigned type = 8u + 4u * (unsigned)a + 2u * (unsigned)(side_n == 0) + (unsigned)r;
                    p->key = okey((uint64_t)L[0], (uint64_t)L[1], (uint64_t)L[2], type, (unsigned)(l - 1));
                    p->w[a] = lat_x(P, a, plane, P->max_depth);
                    p->w[ua] = wfrac(P, ua, Q[ua], l - 1, qu_[r]);
                    p->w[va] = wfrac(P, va, Q[va], l - 1, qv_[r]);
                    fp[a][sd][nfp[a][sd]++] = id;
                }
            }
        }
    }
    int chain[3][2][4];   /* points along each own fold line, ordered by the fold coordinate */
    int nch[3][2];
    for (int a = 0; a < 3; a++)
        for (int r = 0; r < nfr[a]; r++) { chain[a][r][0] = fend[a][r][0]; nch[a][r] = 1; }
    for (int t = 0; t < nx; t++) {
        int a = xing[t][0], i = xing[t][1], b = xing[t][2], j = xing[t][3];
        int cc = 3 - a - b;
        int ua, va, ub, vb;
        other_axes(a, &ua, &va);
        other_axes(b, &ub, &vb);
        int id = new_point(pts, &np, 3);
        if (id < 0) { LOOPERR(9); return OR_OK; }
        opoint *p = &pts[id];
        p->p[a] = fr[b][j][a == ub ? 0 : 1];
        p->p[b] = fr[a][i][b == ua ? 0 : 1];
        p->p[cc] = fr[a][i][cc == ua ? 0 : 1];
        for (int q = 0; q < 3; q++) p->w[q] = wfrac(P, q, C[q], l, p->p[q]);
        p->fa = a; p->fb = b;
        /* outward normal = -grad g = -(dg/dx_cc) e_cc at the point */
        double w[3] = {p->p[0], p->p[1], p->p[2]};
        double dgc = 0;
        for (int v = 0; v < 8; v++) {
            double f = 1;
            for (int q = 0; q < 3; q++) {
                int bit = (v >> q) & 1;
                if (q == cc) f *= bit ? 1.0 : -1.0;
                else f *= bit ? w[q] : 1.0 - w[q];
            }
            dgc += f * g[v];
        }
        int even = (a == 0 && b == 1) || (a == 1 && b == 2) ? 1 : 0; /* (a,b,cc) cyclic */
        p->rh = (even == (dgc < 0));
        if (dgc == 0) LOOPERR(1);
        p->key = okey((uint64_t)(C[0] * s), (uint64_t)(C[1] * s), (uint64_t)(C[2] * s),
                      20u + 4u * (unsigned)(a + b - 1) + 2u * (unsigned)i + (unsigned)j, (unsigned)l);
        if (nch[a][i] < 3) chain[a][i][nch[a][i]++] = id;
        if (nch[b][j] < 3) chain[b][j][nch[b][j]++] = id;
    }
    /* close the chains, sort interior points along the fold axis, link */
    for (int a = 0; a < 3; a++)
        for (int r = 0; r < nfr[a]; r++) {
            int *ch = chain[a][r];
            int n = nch[a][r];
            if (n == 3 && pts[ch[2]].p[a] < pts[ch[1]].p[a]) { int t = ch[1]; ch[1] = ch[2]; ch[2] = t; }
            ch[n++] = fend[a][r][1];
            nch[a][r] = n;
            for (int k = 0; k + 1 < n; k++) {
                int p0 = ch[k], p1 = ch[k + 1];
                /* p0 -> p1 is the + direction along a */
                if (pts[p0].kind == 3) pts[p0].nb[pts[p0].fa == a ? 0 : 2] = p1;
                else pts[p0].nb[0] = p1;
                if (pts[p1].kind == 3) pts[p1].nb[pts[p1].fa == a ? 1 : 3] = p0;
                else pts[p1].nb[0] = p0;
            }
        }

    /* Face curves: arcs of the bilinear face function between edge points,
     * extreme points inserted in order along their branch, oriented so that
     * the inside (g >= c) is on the right seen from outside the cube.  All
     * face decisions use the face's own (u,v) frame (global axis order), so
     * both cubes sharing the face take the same ones. */
    int next[MAXP];
    for (int i = 0; i < np; i++) next[i] = -1;
    for (int a = 0; a < 3; a++) {
        int ua, va;
        other_axes(a, &ua, &va);
        for (int sd = 0; sd < 2; sd++) {
            double h[2][2];
            int b[3];
            for (int iu = 0; iu < 2; iu++)
                for (int iv = 0; iv < 2; iv++) {
                    b[a] = sd; b[ua] = iu; b[va] = iv;
                    h[iu][iv] = gv(g, b[0], b[1], b[2]);
                }
            /* face edges: E0 v=0, E1 u=1, E2 v=1, E3 u=0 */
            int ep[4];
            for (int e = 0; e < 4; e++) {
                int along = (e == 0 || e == 2) ? ua : va;
                int fixed_other = (e == 0 || e == 2) ? va : ua;
                int fixed_val = (e == 1 || e == 2) ? 1 : 0;
                int bits[3];
                bits[along] = 0; bits[a] = sd; bits[fixed_other] = fixed_val;
                int o1, o2;
                other_axes(along, &o1, &o2);
                ep[e] = eid[along][bits[o1]][bits[o2]];
            }
            int ncross = (ep[0] >= 0) + (ep[1] >= 0) + (ep[2] >= 0) + (ep[3] >= 0);
            if (ncross == 0) {
                if (nfp[a][sd] > 0) LOOPERR(2);
                continue;
            }
            int hs = (sd ? 1 : -1) * (a == 1 ? -1 : 1);
            double stq[4];
            stq[0] = hs * (h[1][0] - h[0][0]);
            stq[1] = hs * (h[1][1] - h[1][0]);
            stq[2] = -hs * (h[1][1] - h[0][1]);
            stq[3] = -hs * (h[0][1] - h[0][0]);
            int arcs[2][2];
            int narc = 0, around00 = 0;
            double us = 0;
            if (ncross == 2) {
                int e1 = -1, e2 = -1;
                for (int e = 0; e < 4; e++)
                    if (ep[e] >= 0) { if (e1 < 0) e1 = e; else e2 = e; }
                arcs[0][0] = e1; arcs[0][1] = e2;
                narc = 1;
            } else if (ncross == 4) {
                double d = h[0][0] - h[1][0] - h[0][1] + h[1][1];
                double hsad = (h[0][0] * h[1][1] - h[1][0] * h[0][1]) / d;
                us = (h[0][0] - h[0][1]) / d;
                int in00 = h[0][0] >= c;
                int separated = hsad < c;
                around00 = (in00 && separated) || (!in00 && !separated);
                if (around00) { arcs[0][0] = 0; arcs[0][1] = 3; arcs[1][0] = 2; arcs[1][1] = 1; }
                else { arcs[0][0] = 0; arcs[0][1] = 1; arcs[1][0] = 2; arcs[1][1] = 3; }
                narc = 2;
            } else {
                LOOPERR(3);
                continue;
            }
            for (int ai = 0; ai < narc; ai++) {
                int e1 = arcs[ai][0], e2 = arcs[ai][1];
                int P1 = ep[e1], P2 = ep[e2];
                int st1 = stq[e1] > 0, st2 = stq[e2] > 0;
                if (st1 == st2) { LOOPERR(4); continue; }
                int S = st1 ? P1 : P2, T = st1 ? P2 : P1;
                int mid[FPMAX], nm = 0;
                for (int t = 0; t < nfp[a][sd]; t++) {
                    int id = fp[a][sd][t];
                    if (narc == 2) {
                        int branch_lowu = pts[id].p[ua] < us;
                        int arc_lowu = (ai == 0) ? around00 : !around00;
                        if (branch_lowu != arc_lowu) continue;
                    }
                    mid[nm++] = id;
                }
                double du = pts[T].p[ua] - pts[S].p[ua], dv = pts[T].p[va] - pts[S].p[va];
                int ax = fabs(du) >= fabs(dv) ? ua : va;
                double sgn = (ax == ua ? du : dv) >= 0 ? 1.0 : -1.0;
                for (int i1 = 1; i1 < nm; i1++) {
                    int x = mid[i1], j = i1 - 1;
                    while (j >= 0) {
                        double kx = sgn * pts[x].p[ax], kj = sgn * pts[mid[j]].p[ax];
                        if (kj > kx || (kj == kx && pts[mid[j]].key > pts[x].key)) { mid[j + 1] = mid[j]; j--; }
                        else break;
                    }
                    mid[j + 1] = x;
                }
                int seq[FPMAX + 2], ns = 0;
                seq[ns++] = S;
                for (int i1 = 0; i1 < nm; i1++) seq[ns++] = mid[i1];
                seq[ns++] = T;
                for (int i1 = 0; i1 + 1 < ns; i1++) {
                    if (next[seq[i1]] >= 0) LOOPERR(5);
                    next[seq[i1]] = seq[i1 + 1];
                }
            }
        }
    }
    for (int i = 0; i < np; i++)
        if (pts[i].kind != 3 && next[i] < 0) { LOOPERR(6); return OR_OK; }

    /* Pieces: trace every face of the graph formed by the loops and the fold
     * segments, keeping the face on the left (seen from outside).  After a
     * loop edge into an own extreme point the walk turns onto its fold; after
     * a fold segment into an extreme point it continues along the loop; at a
     * critical point it takes the segment next clockwise from the one it
     * arrived on. */
    int used_loop[MAXP], used_fold[MAXP][4];
    for (int i = 0; i < np; i++) { used_loop[i] = 0; used_fold[i][0] = used_fold[i][1] = used_fold[i][2] = used_fold[i][3] = 0; }
    for (int i0 = 0; i0 < np; i0++) {
        if (pts[i0].kind == 3 || used_loop[i0]) continue;
        int poly[2 * MAXP], n = 0;
        int cur = i0, slot = -1; /* slot < 0: loop edge from cur; else fold slot */
        int ok = 1;
        for (int steps = 0;; steps++) {
            if (steps > 4 * MAXP || n >= 2 * MAXP) { ok = 0; break; }
            poly[n++] = cur;
            int nx;
            if (slot < 0) { used_loop[cur] = 1; nx = next[cur]; }
            else { used_fold[cur][slot] = 1; nx = pts[cur].nb[slot]; }
            if (nx < 0) { ok = 0; break; }
            int nslot;
            if (slot < 0) {
                nslot = pts[nx].kind == 1 ? 0 : -1;
            } else if (pts[nx].kind != 3) {
                nslot = -1;
            } else {
                /* arrived at a critical point from cur: direction back to cur */
                opoint *X = &pts[nx];
                int back = -1;
                for (int k = 0; k < 4; k++) if (X->nb[k] == cur) back = k;
                /* slots: 0 +a, 1 -a, 2 +b, 3 -b; clockwise successor */
                static const int cw_rh[4] = {3, 2, 0, 1};  /* +a->-b, -a->+b, +b->+a, -b->-a */
                static const int cw_lh[4] = {2, 3, 1, 0};  /* +a->+b, -a->-b, +b->-a, -b->+a */
                if (back < 0) { ok = 0; break; }
                nslot = X->rh ? cw_rh[back] : cw_lh[back];
                if (X->nb[nslot] < 0) { ok = 0; break; }
            }
            cur = nx;
            slot = nslot;
            if (slot < 0 && cur == i0) break;
            if (slot < 0 && used_loop[cur]) { ok = 0; break; }
            if (slot >= 0 && used_fold[cur][slot]) { ok = 0; break; }
        }
        if (!ok) { LOOPERR(7); continue; }
        if (n >= 3 && n <= MAXP) {
            tris->piece++;
            int r = ear_clip(pts, poly, n, tris, st);
            if (r) return r;
        } else if (n > MAXP) LOOPERR(8);
    }
    /* world positions, each computed in its owner's frame */
    for (int i = 0; i < np; i++)
        if (p_push(verts, pts[i].key, pts[i].w)) return OR_ERR_OOM;
    return OR_OK;
}

/* Triangulate every listed cube.  Cubes are independent (each reads only the
 * shared, read-only field and cube set), so blocks of cubes run in parallel
 * into their own buffers, which are then appended in cube order with the
 * piece numbers offset: the result is that of the sequential loop. */
static int triangulate_all(const omesh_ctx *M, const uint64_t *cubes, int64_t n, vtri *tris, vvert *verts,
                           ostats *st)
{
    const int64_t BS = 2048;
    int64_t nb = (n + BS - 1) / BS;
    if (nb == 0) return OR_OK;
    vtri *bt = (vtri *)calloc((size_t)nb, sizeof(vtri));
    vvert *bv = (vvert *)calloc((size_t)nb, sizeof(vvert));
    ostats *bs = (ostats *)calloc((size_t)nb, sizeof(ostats));
    int *be = (int *)calloc((size_t)nb, sizeof(int));
    if (!bt || !bv || !bs || !be) { free(bt); free(bv); free(bs); free(be); return OR_ERR_OOM; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(OR_NT)
#endif
    for (int64_t b = 0; b < nb; b++) {
        int64_t i1 = (b + 1) * BS < n ? (b + 1) * BS : n;
        for (int64_t i = b * BS; i < i1 && !be[b]; i++) be[b] = triangulate_cube(M, cubes[i], &bt[b], &bv[b], &bs[b]);
    }
    int e = OR_OK;
    for (int64_t b = 0; b < nb; b++) {
        if (be[b] && !e) e = be[b];
        st->n_cubes_surface += bs[b].n_cubes_surface;
        st->degenerate_ears += bs[b].degenerate_ears;
        st->loop_errors += bs[b].loop_errors;
        for (int64_t i = 0; i < bt[b].n && !e; i++) {
            otri *t = &bt[b].t[i];
            if (t_push(tris, t->k[0], t->k[1], t->k[2])) { e = OR_ERR_OOM; break; }
            tris->t[tris->n - 1].piece = t->piece + tris->piece;
        }
        tris->piece += bt[b].piece;
        for (int64_t i = 0; i < bv[b].n && !e; i++)
            if (p_push(verts, bv[b].p[i].key, bv[b].p[i].x)) e = OR_ERR_OOM;
        free(bt[b].t);
        free(bv[b].p);
    }
    free(bt); free(bv); free(bs); free(be);
    return e;
}

/* phi at lattice-vertex keys (finest lattice), one point at a time */
/* resolve mode: a value within 1e-10 c of c is summed again in quad
 * precision (and rounded once); *resolved and *changed count those values
 * and those whose side of c changed */
static void lattice_field(const oprob *P, const uint64_t *vk, int64_t n, double *vphi, int64_t *resolved,
                          int64_t *changed)
{
    int64_t nr = 0, nc = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(OR_NT) reduction(+ : nr, nc)
#endif
    for (int64_t i = 0; i < n; i++) {
        int64_t x, y, z;
        okey_xyz(vk[i], &x, &y, &z);
        double p[3] = {lat_x(P, 0, x, P->max_depth), lat_x(P, 1, y, P->max_depth), lat_x(P, 2, z, P->max_depth)};
        vphi[i] = phi_at(P, p, NULL);
        double q;
        if (P->resolve && fabs(vphi[i] - P->c) < OR_NEAR * P->c && quad_phi(P, p, &q) == 0) {
            nr++;
            if ((q < P->c) != (vphi[i] < P->c)) nc++;
            vphi[i] = q;
        }
    }
    if (resolved) *resolved = nr;
    if (changed) *changed = nc;
}

static int cmp_vert(const void *a, const void *b)
{
    uint64_t x = ((const overt *)a)->key, y = ((const overt *)b)->key;
    return x < y ? -1 : x > y;
}

/* ================================================================== */
/* Public entry points (ctypes)                                         */
/* ================================================================== */

typedef struct {
    int64_t n_vertices, n_triangles, n_cubes, n_accepted_pre;
    double *vertices;     /* [nv,3] */
    uint64_t *vkeys;      /* [nv] sorted */
    int32_t *triangles;   /* [nt,3] */
    int64_t *tri_piece;   /* [nt] piece each triangle came from */
    uint64_t *cube_keys;  /* [n_cubes] final accepted cubes, sorted */
    uint64_t *pre_keys;   /* accepted cubes before conformity, sorted */
    int64_t n_lattice;
    uint64_t *lattice_keys; double *lattice_phi; /* vertex field at cube corners */
    double *lattice_psi;  /* the values the trilinear functions take: phi, or the constrained interpolant */
    ostats st;
} or_mesh_out;

void or_mesh_free(or_mesh_out *o)
{
    free(o->vertices); free(o->vkeys); free(o->triangles); free(o->tri_piece); free(o->cube_keys); free(o->pre_keys);
    free(o->lattice_keys); free(o->lattice_phi); free(o->lattice_psi);
    memset(o, 0, sizeof(*o));
}

int or_root_grid(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
                 double min_edge, int max_depth, double *origin, int64_t *nroot, double *pad)
{
    oprob P;
    int e = oprob_init(&P, n, xyz, r, D, c, cutoff_rel, 1.0, min_edge, max_depth);
    if (e) return e;
    for (int a = 0; a < 3; a++) { origin[a] = P.origin[a]; nroot[a] = P.nroot[a]; }
    *pad = P.pad;
    oprob_free(&P);
    return OR_OK;
}

int or_field(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
             int64_t npts, const double *pts, double *phi, double *grad)
{
    oprob P;
    int e = oprob_init(&P, n, xyz, r, D, c, cutoff_rel, 1.0, 1.0, 0);
    if (e) return e;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(OR_NT)
#endif
    for (int64_t i = 0; i < npts; i++) phi[i] = phi_at(&P, pts + 3 * i, grad ? grad + 3 * i : NULL);
    oprob_free(&P);
    return OR_OK;
}

/* tensor A of the cube [lo, lo+h]^3 (brute force over atoms) */
int64_t or_cube_tensor(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
                       const double *lo, double h, double *A)
{
    oprob P;
    if (oprob_init(&P, n, xyz, r, D, c, cutoff_rel, 1.0, 1.0, 0)) return -1;
    double hi[3] = {lo[0] + h, lo[1] + h, lo[2] + h};
    int64_t cnt = cube_tensor(&P, lo, hi, A);
    oprob_free(&P);
    return cnt;
}

/* tensors and decisions for listed cube keys (type 30) of the problem's grid */
int or_cube_batch(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
                  double precision, double min_edge, int max_depth, int64_t ncubes, const uint64_t *keys,
                  double *A_out, double *bounds_out, int32_t *dec_out)
{
    oprob P;
    int e = oprob_init(&P, n, xyz, r, D, c, cutoff_rel, precision, min_edge, max_depth);
    if (e) return e;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(OR_NT)
#endif
    for (int64_t q = 0; q < ncubes; q++) {
        double lo[3], hi[3], A[64], o6[6];
        cube_box(&P, keys[q], lo, hi);
        cube_tensor(&P, lo, hi, A);
        dec_out[q] = or_decide(A, c, precision, (int)okey_level(keys[q]), max_depth, o6);
        if (A_out) memcpy(A_out + 64 * q, A, sizeof(A));
        if (bounds_out) memcpy(bounds_out + 6 * q, o6, sizeof(o6));
    }
    oprob_free(&P);
    return OR_OK;
}

/* the whole path: partition, conformity, vertex field, triangulation, weld */
/* resolve: 1 takes every in-band decision and vertex sign again in quad
 * precision (OR_ERR_ARG where the compiler has no binary128 type) */
int or_mesh_ex2(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
                double precision, double min_edge, int max_depth, int child_mode, int order, int norm, int conform,
                int resolve, or_mesh_out *out)
{
    memset(out, 0, sizeof(*out));
    if (resolve != 0 && (resolve != 1 || !or_have_quad())) return OR_ERR_ARG;
    oprob P;
    int e = oprob_init(&P, n, xyz, r, D, c, cutoff_rel, precision, min_edge, max_depth);
    if (e) return e;
    P.resolve = resolve;
    if (child_mode != 0 && child_mode != 1) { oprob_free(&P); return OR_ERR_ARG; }
    if (order != 0 && order != 1) { oprob_free(&P); return OR_ERR_ARG; }
    if (norm < 0 || norm > 2) { oprob_free(&P); return OR_ERR_ARG; }
    if (conform != 0 && conform != 1) { oprob_free(&P); return OR_ERR_ARG; }
    P.conform = conform;
    P.child_mode = child_mode;
    P.order = order;
    P.norm = norm;
    ostats *st = &out->st;
    vec64 acc = {0};
    e = partition(&P, &acc, st, NULL);
    if (e) goto done;
    acc.n = sort_unique(acc.a, acc.n);
    out->n_accepted_pre = acc.n;
    out->pre_keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(acc.n ? acc.n : 1));
    if (acc.n) memcpy(out->pre_keys, acc.a, sizeof(uint64_t) * (size_t)acc.n);
    e = conformity(&P, &acc, st);
    if (e) goto done;
    /* lattice vertices of the final cubes, their field values, and the
     * constrained values; cubes of different sizes that disagree are split
     * and the whole repeated (to a fixpoint) */
    {
        vec64 vk = {0};
        double *vphi = NULL, *vpsi = NULL;
        for (int iter = 0;; iter++) {
            free(vk.a); free(vphi); free(vpsi);
            vk.a = NULL; vk.n = vk.cap = 0; vphi = vpsi = NULL;
            if (iter > 64) { e = OR_ERR_CAP; goto done; }
            for (int64_t i = 0; i < acc.n; i++) {
                int64_t x, y, z;
                okey_xyz(acc.a[i], &x, &y, &z);
                int l = (int)okey_level(acc.a[i]);
                int64_t s = (int64_t)1 << (max_depth - l);
                for (int v = 0; v < 8; v++)
                    if (v_push(&vk, okey((uint64_t)((x + (v & 1)) * s), (uint64_t)((y + ((v >> 1) & 1)) * s),
                                         (uint64_t)((z + ((v >> 2) & 1)) * s), T_VERT, 0))) { e = OR_ERR_OOM; goto done; }
            }
            vk.n = sort_unique(vk.a, vk.n);
            vphi = (double *)malloc(sizeof(double) * (size_t)(vk.n ? vk.n : 1));
            vpsi = (double *)malloc(sizeof(double) * (size_t)(vk.n ? vk.n : 1));
            ocons *cons = (ocons *)malloc(sizeof(ocons) * (size_t)(vk.n ? vk.n : 1));
            if (!vphi || !vpsi || !cons) { free(cons); free(vk.a); free(vphi); free(vpsi); e = OR_ERR_OOM; goto done; }
            int64_t vres = 0, vchg = 0;
            lattice_field(&P, vk.a, vk.n, vphi, &vres, &vchg);
            st->resolved_vertices = vres;
            st->vertex_sign_changed = vchg;
            e = constrain_values(&P, acc.a, acc.n, vk.a, vk.n, vphi, vpsi, cons);
            vec64 R = {0};
            if (!e) e = disagreeing_cubes(&P, acc.a, acc.n, vk.a, vk.n, vphi, vpsi, cons, &R);
            int64_t ncons = 0;
            for (int64_t i = 0; i < vk.n; i++) ncons += cons[i].lev >= 0;
            free(cons);
            if (!e && R.n > 0) {
                int64_t ns = 0;
                e = split_listed(&acc, R.a, R.n, &ns);
                st->agreement_splits += ns;
                if (!e) e = conformity(&P, &acc, st);
            }
            int64_t nr = R.n;
            free(R.a);
            if (e) { free(vk.a); free(vphi); free(vpsi); goto done; }
            if (nr == 0) {
                st->constrained_vertices = ncons;
                for (int64_t i = 0; i < vk.n; i++) st->near[3] += fabs(vpsi[i] - c) < OR_NEAR * c;
                break;
            }
        }
        st->n_cubes_final = acc.n;
        st->n_vertices_lattice = vk.n;
        out->n_lattice = vk.n;
        out->lattice_keys = vk.a;
        out->lattice_phi = vphi;
        out->lattice_psi = vpsi;
        omesh_ctx M = {&P, acc.a, acc.n, vk.a, vpsi, vk.n};
        vtri tris = {0};
        vvert verts = {0};
        e = triangulate_all(&M, acc.a, acc.n, &tris, &verts, st);
        if (e) { free(tris.t); free(verts.p); goto done; }
        /* weld: unique keys (sorted), triangles remapped to indices */
        if (verts.n) qsort(verts.p, (size_t)verts.n, sizeof(overt), cmp_vert);
        int64_t m = 0;
        for (int64_t i = 0; i < verts.n; i++)
            if (m == 0 || verts.p[i].key != verts.p[m - 1].key) verts.p[m++] = verts.p[i];
        out->n_vertices = m;
        out->vertices = (double *)malloc(sizeof(double) * 3 * (size_t)(m ? m : 1));
        out->vkeys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
        for (int64_t i = 0; i < m; i++) {
            out->vkeys[i] = verts.p[i].key;
            memcpy(out->vertices + 3 * i, verts.p[i].x, sizeof(double) * 3);
        }
        out->n_triangles = tris.n;
        out->triangles = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(tris.n ? tris.n : 1));
        out->tri_piece = (int64_t *)malloc(sizeof(int64_t) * (size_t)(tris.n ? tris.n : 1));
        for (int64_t i = 0; i < tris.n; i++) out->tri_piece[i] = tris.t[i].piece;
        for (int64_t i = 0; i < tris.n; i++)
            for (int j = 0; j < 3; j++) {
                int64_t id = find_u64(out->vkeys, m, tris.t[i].k[j]);
                out->triangles[3 * i + j] = (int32_t)id;
                if (id < 0) st->loop_errors++;
            }
        free(tris.t);
        free(verts.p);
    }
    out->n_cubes = acc.n;
    out->cube_keys = acc.a;
    acc.a = NULL;
done:
    free(acc.a);
    oprob_free(&P);
    if (e) or_mesh_free(out);
    return e;
}

int or_mesh_ex(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
               double precision, double min_edge, int max_depth, int child_mode, int order, int norm, int conform,
               or_mesh_out *out)
{
    return or_mesh_ex2(n, xyz, r, D, c, cutoff_rel, precision, min_edge, max_depth, child_mode, order, norm, conform,
                       0, out);
}

/* partition only (level loop), returns the accepted cubes (sorted) */
int or_mesh(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
            double precision, double min_edge, int max_depth, or_mesh_out *out)
{
    return or_mesh_ex(n, xyz, r, D, c, cutoff_rel, precision, min_edge, max_depth, 0, 0, 0, 0, out);
}

int or_partition(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
                 double precision, double min_edge, int max_depth, or_mesh_out *out)
{
    memset(out, 0, sizeof(*out));
    oprob P;
    int e = oprob_init(&P, n, xyz, r, D, c, cutoff_rel, precision, min_edge, max_depth);
    if (e) return e;
    vec64 acc = {0};
    e = partition(&P, &acc, &out->st, NULL);
    if (!e) {
        acc.n = sort_unique(acc.a, acc.n);
        out->n_accepted_pre = acc.n;
        out->pre_keys = acc.a;
        acc.a = NULL;
    }
    free(acc.a);
    oprob_free(&P);
    return e;
}


/* Triangulate a uniform grid of given corner values (all cubes accepted at
 * one level, unit spacing, origin 0): the per-cube path on exact trilinear
 * data.  values: [(nz+1)][(ny+1)][(nx+1)], x fastest. */
int or_mesh_grid(int64_t nx, int64_t ny, int64_t nz, const double *values, double c, or_mesh_out *out)
{
    memset(out, 0, sizeof(*out));
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx > 4096 || ny > 4096 || nz > 4096) return OR_ERR_ARG;
    oprob P;
    memset(&P, 0, sizeof(P));
    P.c = c; P.min_edge = 1.0; P.max_depth = 0; P.h0 = 1.0;
    P.nroot[0] = nx; P.nroot[1] = ny; P.nroot[2] = nz;
    int64_t nc = nx * ny * nz, nv = (nx + 1) * (ny + 1) * (nz + 1);
    uint64_t *cubes = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nc);
    uint64_t *vk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nv);
    double *vp = (double *)malloc(sizeof(double) * (size_t)nv);
    if (!cubes || !vk || !vp) { free(cubes); free(vk); free(vp); return OR_ERR_OOM; }
    int64_t q = 0;
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) cubes[q++] = okey((uint64_t)x, (uint64_t)y, (uint64_t)z, T_CUBE, 0);
    qsort(cubes, (size_t)nc, sizeof(uint64_t), cmp_u64);
    /* keys sort by (z, y, x) because z occupies the high bits */
    q = 0;
    for (int64_t z = 0; z <= nz; z++)
        for (int64_t y = 0; y <= ny; y++)
            for (int64_t x = 0; x <= nx; x++) {
                vk[q] = okey((uint64_t)x, (uint64_t)y, (uint64_t)z, T_VERT, 0);
                vp[q] = values[q];
                q++;
            }
    omesh_ctx M = {&P, cubes, nc, vk, vp, nv};
    vtri tris = {0};
    vvert verts = {0};
    int e = triangulate_all(&M, cubes, nc, &tris, &verts, &out->st);
    if (!e) {
        if (verts.n) qsort(verts.p, (size_t)verts.n, sizeof(overt), cmp_vert);
        int64_t m = 0;
        for (int64_t i = 0; i < verts.n; i++)
            if (m == 0 || verts.p[i].key != verts.p[m - 1].key) verts.p[m++] = verts.p[i];
        out->n_vertices = m;
        out->vertices = (double *)malloc(sizeof(double) * 3 * (size_t)(m ? m : 1));
        out->vkeys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
        for (int64_t i = 0; i < m; i++) {
            out->vkeys[i] = verts.p[i].key;
            memcpy(out->vertices + 3 * i, verts.p[i].x, sizeof(double) * 3);
        }
        out->n_triangles = tris.n;
        out->triangles = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(tris.n ? tris.n : 1));
        out->tri_piece = (int64_t *)malloc(sizeof(int64_t) * (size_t)(tris.n ? tris.n : 1));
        for (int64_t i = 0; i < tris.n; i++) out->tri_piece[i] = tris.t[i].piece;
        for (int64_t i = 0; i < tris.n; i++)
            for (int j = 0; j < 3; j++) {
                int64_t id = find_u64(out->vkeys, m, tris.t[i].k[j]);
                out->triangles[3 * i + j] = (int32_t)id;
                if (id < 0) out->st.loop_errors++;
            }
    }
    free(tris.t); free(verts.p);
    out->n_cubes = nc;
    out->cube_keys = cubes;
    free(vk); free(vp);
    if (e) or_mesh_free(out);
    return e;
}

int or_sizeof_mesh_out(void) { return (int)sizeof(or_mesh_out); }
int or_sizeof_stats(void) { return (int)sizeof(ostats); }

/* ================================================================== */
/* Derivatives of the mesh.  The paper defines none; these are the chain */
/* rule applied to its construction, with the cube set and the topology  */
/* held fixed.  A vertex is a function of the lattice values it is        */
/* computed from (eqs intersection, fold1, critical); the lattice values  */
/* are functions of the atoms (eq Gaussian1).                             */
/* ================================================================== */

/* Fold equations of axis a at (u,v): A = bilinear(lower face) - c,
 * B = bilinear(upper face) - bilinear(lower face), their partials in (u,v)
 * and in each corner value. */
static void fold_eqs(const double *g, int a, double c, double u, double v, double *A, double *B, double dA[2],
                     double dB[2], double dAg[8], double dBg[8])
{
    int ua, va;
    other_axes(a, &ua, &va);
    *A = -c; *B = 0.0;
    dA[0] = dA[1] = dB[0] = dB[1] = 0.0;
    for (int k = 0; k < 8; k++) dAg[k] = dBg[k] = 0.0;
    for (int k = 0; k < 4; k++) {
        int ku = k & 1, kv = k >> 1;
        double wu = ku ? u : 1.0 - u, wv = kv ? v : 1.0 - v, w = wu * wv;
        double dwdu = (ku ? 1.0 : -1.0) * wv, dwdv = wu * (kv ? 1.0 : -1.0);
        int b[3];
        b[a] = 0; b[ua] = ku; b[va] = kv;
        int il = b[0] | (b[1] << 1) | (b[2] << 2);
        b[a] = 1;
        int iu = b[0] | (b[1] << 1) | (b[2] << 2);
        double dlt = g[iu] - g[il];
        *A += w * g[il];
        *B += w * dlt;
        dA[0] += dwdu * g[il]; dA[1] += dwdv * g[il];
        dB[0] += dwdu * dlt;   dB[1] += dwdv * dlt;
        dAg[il] += w;
        dBg[iu] += w;
        dBg[il] -= w;
    }
}

/* d(u,v)/dg_k of a fold root of axis a: the 2x2 system
 * [dA/du dA/dv; dB/du dB/dv] (du, dv) = -(dA/dg_k, dB/dg_k), by Cramer's rule */
static void fold_root_derivs(const double *g, int a, double c, double u, double v, double du[8], double dv[8])
{
    double A, B, dA[2], dB[2], dAg[8], dBg[8];
    fold_eqs(g, a, c, u, v, &A, &B, dA, dB, dAg, dBg);
    double det = dA[0] * dB[1] - dA[1] * dB[0];
    for (int k = 0; k < 8; k++) {
        double r1 = -dAg[k], r2 = -dBg[k];
        du[k] = det != 0.0 ? (r1 * dB[1] - dA[1] * r2) / det : 0.0;
        dv[k] = det != 0.0 ? (dA[0] * r2 - r1 * dB[0]) / det : 0.0;
    }
}

static int64_t lattice_index(const or_mesh_out *m, int64_t X, int64_t Y, int64_t Z)
{
    return find_u64(m->lattice_keys, m->n_lattice, okey((uint64_t)X, (uint64_t)Y, (uint64_t)Z, T_VERT, 0));
}

/* dL/d(atom centres [n,3]), dL/d(radii [n]), dL/dD from dL/dp [nv,3] given in
 * the order of or_mesh's vertices (sorted keys).  Outputs overwritten. */
int or_mesh_grad(int64_t n, const double *xyz, const double *r, double D, double c, double cutoff_rel,
                 double precision, double min_edge, int max_depth, int64_t nv, const double *dLdp, double *g_xyz,
                 double *g_r, double *g_D)
{
    or_mesh_out m;
    int e = or_mesh(n, xyz, r, D, c, cutoff_rel, precision, min_edge, max_depth, &m);
    if (e) return e;
    if (nv != m.n_vertices) { or_mesh_free(&m); return OR_ERR_ARG; }
    oprob P;
    e = oprob_init(&P, n, xyz, r, D, c, cutoff_rel, precision, min_edge, max_depth);
    if (e) { or_mesh_free(&m); return e; }
    double *lam = (double *)calloc((size_t)(m.n_lattice ? m.n_lattice : 1), sizeof(double));
    ocons *cons = (ocons *)malloc(sizeof(ocons) * (size_t)(m.n_lattice ? m.n_lattice : 1));
    double *psi = (double *)malloc(sizeof(double) * (size_t)(m.n_lattice ? m.n_lattice : 1));
    if (!lam || !cons || !psi) e = OR_ERR_OOM;
    if (!e) e = constrain_values(&P, m.cube_keys, m.n_cubes, m.lattice_keys, m.n_lattice, m.lattice_phi, psi, cons);
    /* the vertices are functions of the values the trilinear functions take (psi) */
    omesh_ctx M = {&P, m.cube_keys, m.n_cubes, m.lattice_keys, psi, m.n_lattice};
    for (int64_t i = 0; i < nv && !e; i++) {
        const double *G = dLdp + 3 * i;
        uint64_t K = m.vkeys[i];
        unsigned type = (unsigned)((K >> 54) & 31u);
        int l = (int)okey_level(K);
        int64_t L[3];
        okey_xyz(K, &L[0], &L[1], &L[2]);
        int64_t s = (int64_t)1 << (max_depth - l);
        double h = lvl_h(&P, l);
        if (type <= 2) {
            /* edge point (eq intersection): t = (c - g0)/(g1 - g0) along axis a */
            int a = (int)type;
            int64_t L1[3] = {L[0], L[1], L[2]};
            L1[a] += s;
            int64_t i0 = lattice_index(&m, L[0], L[1], L[2]), i1 = lattice_index(&m, L1[0], L1[1], L1[2]);
            if (i0 < 0 || i1 < 0) { e = OR_ERR_CAP; break; }
            double g0 = psi[i0], g1 = psi[i1];
            double t = (c - g0) / (g1 - g0);
            lam[i0] += G[a] * h * (-(1.0 - t) / (g1 - g0));
            lam[i1] += G[a] * h * (-t / (g1 - g0));
            continue;
        }
        /* extreme point (fold end on a face) or critical point: the cube */
        int64_t C[3] = {L[0] / s, L[1] / s, L[2] / s};
        int fa, fr, fb = -1, fj = 0;
        if (type >= 8 && type < 20) {
            int code = (int)type - 8;
            fa = code >> 2;
            fr = code & 1;
            if (!((code >> 1) & 1)) C[fa] -= 1;   /* the end on the owner's upper face */
        } else if (type >= 20 && type < 32) {
            int code = (int)type - 20, pr = code >> 2;
            fa = pr == 2 ? 1 : 0;
            fb = pr == 0 ? 1 : 2;
            fr = (code >> 1) & 1;
            fj = code & 1;
        } else {
            continue;
        }
        double g[8];
        if (!cube_values(&M, l, C[0], C[1], C[2], g)) { e = OR_ERR_CAP; break; }
        int64_t li[8];
        for (int v = 0; v < 8; v++) {
            li[v] = lattice_index(&m, (C[0] + (v & 1)) * s, (C[1] + ((v >> 1) & 1)) * s, (C[2] + ((v >> 2) & 1)) * s);
            if (li[v] < 0) { e = OR_ERR_CAP; break; }
        }
        if (e) break;
        double ru[2], rv[2], du[8], dv[8], dp[3][8];
        memset(dp, 0, sizeof(dp));
        int ua, va;
        other_axes(fa, &ua, &va);
        if (fold_roots(g, fa, c, ru, rv) <= fr) { e = OR_ERR_CAP; break; }
        fold_root_derivs(g, fa, c, ru[fr], rv[fr], du, dv);
        if (fb < 0) {
            for (int v = 0; v < 8; v++) { dp[ua][v] = du[v]; dp[va][v] = dv[v]; }
        } else {
            /* eq critical: coordinate fa from the b-root, the others from the a-root */
            int cc = 3 - fa - fb, ub, vb;
            for (int v = 0; v < 8; v++) {
                dp[fb][v] = fb == ua ? du[v] : dv[v];
                dp[cc][v] = cc == ua ? du[v] : dv[v];
            }
            other_axes(fb, &ub, &vb);
            if (fold_roots(g, fb, c, ru, rv) <= fj) { e = OR_ERR_CAP; break; }
            fold_root_derivs(g, fb, c, ru[fj], rv[fj], du, dv);
            for (int v = 0; v < 8; v++) dp[fa][v] = fa == ub ? du[v] : dv[v];
        }
        for (int v = 0; v < 8; v++) lam[li[v]] += h * (G[0] * dp[0][v] + G[1] * dp[1][v] + G[2] * dp[2][v]);
    }
    /* constrained values are interpolants of their sources: fine to coarse,
     * each passes its adjoint on with the interpolation weights */
    for (int l = max_depth - 1; l >= 0 && !e; l--)
        for (int64_t k = 0; k < m.n_lattice; k++) {
            const ocons *K = &cons[k];
            if (K->lev != l || lam[k] == 0.0) continue;
            if (K->nsrc == 2) {
                lam[K->src[0]] += lam[k] * (1.0 - K->t[0]);
                lam[K->src[1]] += lam[k] * K->t[0];
            } else {
                double tu = K->t[0], tw = K->t[1];
                lam[K->src[0]] += lam[k] * (1.0 - tu) * (1.0 - tw);
                lam[K->src[1]] += lam[k] * tu * (1.0 - tw);
                lam[K->src[2]] += lam[k] * (1.0 - tu) * tw;
                lam[K->src[3]] += lam[k] * tu * tw;
            }
            lam[k] = 0.0;
        }
    /* the field (eq Gaussian1, truncated): dt/dx_i = 2D t (p - x_i),
     * dt/dr_i = 2D t r_i, dt/dD = -t (|p - x_i|^2 - r_i^2), all atoms */
    for (int64_t i = 0; i < n; i++) { g_xyz[3 * i] = g_xyz[3 * i + 1] = g_xyz[3 * i + 2] = 0.0; g_r[i] = 0.0; }
    *g_D = 0.0;
    for (int64_t k = 0; k < m.n_lattice && !e; k++) {
        if (lam[k] == 0.0) continue;
        int64_t x, y, z;
        okey_xyz(m.lattice_keys[k], &x, &y, &z);
        double p[3] = {lat_x(&P, 0, x, max_depth), lat_x(&P, 1, y, max_depth), lat_x(&P, 2, z, max_depth)};
        for (int64_t i = 0; i < n; i++) {
            double d[3] = {p[0] - xyz[3 * i], p[1] - xyz[3 * i + 1], p[2] - xyz[3 * i + 2]};
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (d2 > P.R2[i]) continue;
            double t = exp(-D * (d2 - r[i] * r[i]));
            for (int q = 0; q < 3; q++) g_xyz[3 * i + q] += lam[k] * 2.0 * D * t * d[q];
            g_r[i] += lam[k] * 2.0 * D * t * r[i];
            *g_D -= lam[k] * t * (d2 - r[i] * r[i]);
        }
    }
    free(lam);
    free(cons);
    free(psi);
    oprob_free(&P);
    or_mesh_free(&m);
    return e;
}

/* enclosed volume and area of a closed outward mesh (plain sums) */
void or_volume_area(int64_t nv, const double *v, int64_t nt, const int32_t *t, double *out2)
{
    (void)nv;
    double vol = 0.0, area = 0.0;
    for (int64_t i = 0; i < nt; i++) {
        const double *p0 = v + 3 * t[3 * i], *p1 = v + 3 * t[3 * i + 1], *p2 = v + 3 * t[3 * i + 2];
        double c12[3] = {p1[1] * p2[2] - p1[2] * p2[1], p1[2] * p2[0] - p1[0] * p2[2], p1[0] * p2[1] - p1[1] * p2[0]};
        vol += (p0[0] * c12[0] + p0[1] * c12[1] + p0[2] * c12[2]) / 6.0;
        double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]}, e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        area += 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    }
    out2[0] = vol;
    out2[1] = area;
}
