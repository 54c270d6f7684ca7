/*
 * nl_oracle.c -- plain, slow FP64 CPU reference for the nonlocal operator
 * library.  TEST INFRASTRUCTURE ONLY: nothing on the product path may link,
 * load or call this file.  It shares no code, header, table or constant with
 * the CUDA library; it is written directly from the paper's definitions:
 *
 *   Tian & Engquist, "Fast algorithm for computing nonlocal operators with
 *   finite interaction distance" (arXiv 1905.08375).
 *
 *   Eq. (2.1)  nonlocal diffusion  L u(x) = int_{H_x} w(x,y) (u(y)-u(x)) dy
 *   Eq. (2.2)  kernel  w = C(x,y) / delta^{d+2} * gamma(|y-x| / delta)
 *   Eq. (1.2)  linear bond force  f = w(x,y) [e.(u(y)-u(x))] e
 *   Sec. 3     splitting gamma = kappa + p^{2K} chi, Hermite-matched p^{2K}; the direct
 *              sum serves all three profiles (gamma, kappa and p^{2K})
 *   Eq. (3.1)  volume constraint u = 0 outside Omega = [0,1]^d
 *   Eq. (3.3)  L^P u = C/delta^{d+2} ( int_{H_x cap Omega} u - |H_x| u(x) )
 *   Algorithm 1 (recur), Algorithm 2 (cube/ball test), Steps 1-3, Eq. (3.5)
 *   Sec. 4     outlook: a fast algorithm for peridynamics (here: degree 0 over the
 *              leaf set, or_fast_pd_leafset)
 *
 * Conventions (readings of the paper, stated once here):
 *   - grid: n nodes per dimension, h = 1/n, node i at x_i = (i + 1/2) h
 *     (cell-centred; one node per leaf cell), flat index x fastest.
 *   - horizon test: lattice offset o (integer, units of h) is inside the
 *     open ball of node i iff  (double)|o|^2 < R2_i,  R2_i = (delta_i n)^2
 *     evaluated in FP64.  Cell tests use half-units of h (integers), with
 *     threshold 4 R2_i.
 *   - exterior rule: for a node y outside Omega, u(y) = 0 (volume
 *     constraint) and every coefficient field (a, c, delta) takes the value
 *     of the row's own node x.
 *   - quadrature: nodal Riemann sum with weight h^d (the paper's AC weights
 *     are not given in the paper); j = i is excluded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

enum { OR_POWER = 0, OR_POLY = 1, OR_KAPPA = 2 };
enum { OR_COEF_NONE = 0, OR_COEF_X = 1, OR_COEF_XY = 2 };
enum { OR_SELF_DISCRETE = 0, OR_SELF_PAPER = 1 };

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* number of OpenMP threads of the following calls (timing only; results do not depend on it) */
void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------ */
/* Small helpers                                                       */
/* ------------------------------------------------------------------ */

static int64_t num_nodes(int d, int n)
{
    int64_t N = 1;
    for (int k = 0; k < d; ++k) N *= n;
    return N;
}

/* flat index -> per-dimension index (unused dimensions are 0) */
static void unflatten(int64_t f, int d, int n, int64_t c[3])
{
    c[0] = c[1] = c[2] = 0;
    for (int k = 0; k < d; ++k) { c[k] = f % n; f /= n; }
}

static int64_t flatten(const int64_t c[3], int d, int n)
{
    int64_t f = 0;
    for (int k = d - 1; k >= 0; --k) f = f * n + c[k];
    return f;
}

/* Surface measure of the unit sphere S^{d-1}: 2, 2 pi, 4 pi. */
double or_sphere_area(int d)
{
    if (d == 1) return 2.0;
    if (d == 2) return 2.0 * OR_PI;
    return 4.0 * OR_PI;
}

/*
 * Normalisation of Eq. (2.2) used here: (1/(2d)) int_{B_delta} |xi|^2 w = 1
 * for w = sigma delta^{-(d+2)} (|xi|/delta)^{-alpha}, so that L -> Laplacian
 * (the 1-D condition printed after Eq. (2.2) gives L -> u''/2 instead).
 * int_{B_1} |s|^{2-alpha} ds = |S^{d-1}| / (d+2-alpha), hence
 * sigma = 2d (d+2-alpha) / |S^{d-1}|.
 */
double or_sigma(int d, double alpha, double scale, int normalize)
{
    if (!normalize) return scale;
    return scale * 2.0 * d * (d + 2.0 - alpha) / or_sphere_area(d);
}

/*
 * Sec. 3: p^{2K}(s) = sum_{m=0}^{K} p_m s^{2m} matches gamma(s) = s^{-alpha}
 * and its first K derivatives at s = 1.  Row j of the linear system:
 *   sum_m p_m (2m)(2m-1)...(2m-j+1) = (-alpha)(-alpha-1)...(-alpha-j+1).
 * Solved by Gaussian elimination with partial pivoting.
 */
int or_poly_coeffs(int K, double alpha, double *p)
{
    if (K < 0 || K > 8) return 1;
    int m = K + 1;
    double A[9][10];
    for (int j = 0; j < m; ++j) {
        for (int c = 0; c < m; ++c) {
            double f = 1.0;
            for (int t = 0; t < j; ++t) f *= (double)(2 * c - t);
            A[j][c] = f;
        }
        double g = 1.0;
        for (int t = 0; t < j; ++t) g *= (-alpha - t);
        A[j][m] = g;
    }
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return 2;
        if (piv != col)
            for (int c = 0; c <= m; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
        for (int r = 0; r < m; ++r) {
            if (r == col) continue;
            double f = A[r][col] / A[col][col];
            for (int c = col; c <= m; ++c) A[r][c] -= f * A[col][c];
        }
    }
    for (int j = 0; j < m; ++j) p[j] = A[j][m] / A[j][j];
    return 0;
}

/* Radial profile gamma(s) of Eq. (2.2) for 0 < s < 1: s^{-alpha} (POWER), p^{2K}(s) (POLY), or
 * the other part of the splitting of Sec. 3, gamma = kappa + p^{2K} chi:
 * kappa(s) = s^{-alpha} - p^{2K}(s) (KAPPA). */
static double profile(int family, double alpha, int K, const double *p, double s)
{
    if (family == OR_POWER) return pow(s, -alpha);
    double r = 0.0, s2 = s * s, sp = 1.0;
    for (int m = 0; m <= K; ++m) { r += p[m] * sp; sp *= s2; }
    if (family == OR_KAPPA) return pow(s, -alpha) - r;
    return r;
}

/* ------------------------------------------------------------------ */
/* Direct scalar operator, Eq. (2.1)-(2.2)                             */
/* ------------------------------------------------------------------ */

typedef struct {
    int d, n, family, K, coef, symmetric;
    double alpha, sigma, h;
    const double *delta, *a, *p;
} scalar_op;

/*
 * Weight w_ij * c_ij of the bond from node i (coords ci) to lattice
 * offset o.  Returns 0 when the bond is outside the horizon(s).
 *   one-sided (non-divergence type, Sec. 2 case (a)):  w_ij uses delta_i.
 *   symmetric (divergence type, Sec. 2 case (b)):
 *       w^s_ij = (w_ij + w_ji)/2, each half with its own node's ball.
 */
static double bond_weight(const scalar_op *op, const int64_t ci[3], int64_t fi,
                          const int64_t o[3], int *inside_out, int64_t *fj_out)
{
    const int d = op->d, n = op->n;
    int64_t o2 = 0, cj[3];
    int inside = 1;
    for (int k = 0; k < 3; ++k) {
        cj[k] = ci[k] + o[k];
        o2 += o[k] * o[k];
        if (k < d && (cj[k] < 0 || cj[k] >= n)) inside = 0;
    }
    *inside_out = inside;
    *fj_out = inside ? flatten(cj, d, n) : -1;
    if (o2 == 0) return 0.0;
    const double r = sqrt((double)o2) * op->h;             /* |x_j - x_i| */
    const double di = op->delta[fi];
    const double R2i = (di * n) * (di * n);
    double wi = 0.0;
    if ((double)o2 < R2i)
        wi = op->sigma * pow(di, -(d + 2.0)) * profile(op->family, op->alpha, op->K, op->p, r / di);
    double w = wi;
    if (op->symmetric && inside) {
        const double dj = op->delta[*fj_out];
        const double R2j = (dj * n) * (dj * n);
        double wj = 0.0;
        if ((double)o2 < R2j)
            wj = op->sigma * pow(dj, -(d + 2.0)) * profile(op->family, op->alpha, op->K, op->p, r / dj);
        w = 0.5 * (wi + wj);
    }
    if (w == 0.0) return 0.0;
    double c = 1.0;
    if (op->coef == OR_COEF_X) c = op->a[fi];
    else if (op->coef == OR_COEF_XY) c = op->a[fi] * (inside ? op->a[*fj_out] : op->a[fi]);
    return w * c;
}

static int64_t box_halfwidth(const scalar_op *op, int64_t N)
{
    double rmax = 0.0;
    for (int64_t f = 0; f < N; ++f) if (op->delta[f] * op->n > rmax) rmax = op->delta[f] * op->n;
    return (int64_t)ceil(rmax);
}

/*
 * (L u)_i = h^d sum_{j != i} w_ij c_ij (u_j - u_i), u_j = 0 outside Omega.
 * u, out: [nrhs][N].  idx (optional): compute only the listed nodes; out is
 * then [nrhs][nidx].
 */
int or_direct_scalar(int d, int n, const double *delta, int family, double alpha, int K,
                     const double *p, double sigma, int coef, const double *a, int symmetric,
                     int nrhs, const double *u, double *out, const int64_t *idx, int64_t nidx)
{
    if (d < 1 || d > 3 || n < 1) return 1;
    if (symmetric && coef == OR_COEF_X) return 2;
    scalar_op op = { d, n, family, K, coef, symmetric, alpha, sigma, 1.0 / n, delta, a, p };
    const int64_t N = num_nodes(d, n);
    const int64_t M = idx ? nidx : N;
    const int64_t B = box_halfwidth(&op, N);
    const double hd = pow(op.h, d);
    const int64_t bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < M; ++q) {
        const int64_t fi = idx ? idx[q] : q;
        int64_t ci[3];
        unflatten(fi, d, n, ci);
        for (int r = 0; r < nrhs; ++r) {
            const double *ur = u + (int64_t)r * N;
            const double ui = ur[fi];
            double acc = 0.0;
            for (int64_t oz = -bz; oz <= bz; ++oz)
                for (int64_t oy = -by; oy <= by; ++oy)
                    for (int64_t ox = -B; ox <= B; ++ox) {
                        int64_t o[3] = { ox, oy, oz }, fj;
                        int inside;
                        double wc = bond_weight(&op, ci, fi, o, &inside, &fj);
                        if (wc == 0.0) continue;
                        double uj = inside ? ur[fj] : 0.0;
                        acc += wc * (uj - ui);
                    }
            out[(int64_t)r * M + q] = hd * acc;
        }
    }
    return 0;
}

/* Diagonal of -L (the Jacobi preconditioner): h^d sum_{j != i} w_ij c_ij. */
int or_direct_diag(int d, int n, const double *delta, int family, double alpha, int K,
                   const double *p, double sigma, int coef, const double *a, int symmetric,
                   double *diag)
{
    if (symmetric && coef == OR_COEF_X) return 2;
    scalar_op op = { d, n, family, K, coef, symmetric, alpha, sigma, 1.0 / n, delta, a, p };
    const int64_t N = num_nodes(d, n);
    const int64_t B = box_halfwidth(&op, N);
    const double hd = pow(op.h, d);
    const int64_t bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t fi = 0; fi < N; ++fi) {
        int64_t ci[3];
        unflatten(fi, d, n, ci);
        double acc = 0.0;
        for (int64_t oz = -bz; oz <= bz; ++oz)
            for (int64_t oy = -by; oy <= by; ++oy)
                for (int64_t ox = -B; ox <= B; ++ox) {
                    int64_t o[3] = { ox, oy, oz }, fj;
                    int inside;
                    acc += bond_weight(&op, ci, fi, o, &inside, &fj);
                }
        diag[fi] = hd * acc;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Linear bond-based peridynamics, Eq. (1.1)-(1.2)                      */
/* ------------------------------------------------------------------ */

/*
 * (L_PD u)_i = h^d sum_{0<|xi|<delta_i} sigma c_ij (xi xi^T / |xi|^3) (u_j - u_i)
 * with xi = x_j - x_i, c_ij = (c_i + c_j)/2 (c_j = c_i outside Omega),
 * u_j = 0 outside Omega.  The micromodulus of Eq. (1.2) is sigma c_ij / |xi|,
 * applied along the unit bond vector e = xi/|xi|.
 * u, out: [nrhs][d][N] (component planes).  idx as above.
 */
int or_pd_direct(int d, int n, const double *delta, const double *c, double sigma,
                 int nrhs, const double *u, double *out, const int64_t *idx, int64_t nidx)
{
    if (d < 1 || d > 3 || n < 1) return 1;
    const int64_t N = num_nodes(d, n);
    const int64_t M = idx ? nidx : N;
    const double h = 1.0 / n, hd = pow(h, d);
    double rmax = 0.0;
    for (int64_t f = 0; f < N; ++f) if (delta[f] * n > rmax) rmax = delta[f] * n;
    const int64_t B = (int64_t)ceil(rmax);
    const int64_t bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < M; ++q) {
        const int64_t fi = idx ? idx[q] : q;
        int64_t ci[3];
        unflatten(fi, d, n, ci);
        const double R2i = (delta[fi] * n) * (delta[fi] * n);
        for (int r = 0; r < nrhs; ++r) {
            const double *ur = u + (int64_t)r * d * N;
            double acc[3] = { 0, 0, 0 };
            for (int64_t oz = -bz; oz <= bz; ++oz)
                for (int64_t oy = -by; oy <= by; ++oy)
                    for (int64_t ox = -B; ox <= B; ++ox) {
                        int64_t o[3] = { ox, oy, oz }, cj[3];
                        int64_t o2 = ox * ox + oy * oy + oz * oz;
                        if (o2 == 0 || !((double)o2 < R2i)) continue;
                        int inside = 1;
                        for (int k = 0; k < 3; ++k) {
                            cj[k] = ci[k] + o[k];
                            if (k < d && (cj[k] < 0 || cj[k] >= n)) inside = 0;
                        }
                        const int64_t fj = inside ? flatten(cj, d, n) : -1;
                        double xi[3], du[3], xdu = 0.0, len2 = 0.0;
                        for (int k = 0; k < d; ++k) {
                            xi[k] = (double)o[k] * h;
                            len2 += xi[k] * xi[k];
                            double uj = inside ? ur[(int64_t)k * N + fj] : 0.0;
                            du[k] = uj - ur[(int64_t)k * N + fi];
                            xdu += xi[k] * du[k];
                        }
                        const double len = sqrt(len2);
                        const double cij = 0.5 * (c[fi] + (inside ? c[fj] : c[fi]));
                        const double f = sigma * cij * xdu / (len2 * len);
                        for (int k = 0; k < d; ++k) acc[k] += f * xi[k];
                    }
            for (int k = 0; k < d; ++k) out[((int64_t)r * d + k) * M + q] = hd * acc[k];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Fast algorithm of Sec. 3                                             */
/* ------------------------------------------------------------------ */

/* Multi-indices alpha with |alpha| <= 2K in d dimensions. */
static int moment_list(int d, int K, int al[][3])
{
    int M = 0, D = 2 * K;
    for (int a2 = 0; a2 <= (d > 2 ? D : 0); ++a2)
        for (int a1 = 0; a1 <= (d > 1 ? D : 0); ++a1)
            for (int a0 = 0; a0 <= D; ++a0)
                if (a0 + a1 + a2 <= D) { al[M][0] = a0; al[M][1] = a1; al[M][2] = a2; ++M; }
    return M;
}

static double binom(int a, int b)
{
    double r = 1.0;
    for (int t = 1; t <= b; ++t) r = r * (a - b + t) / t;
    return r;
}

/*
 * Step 2 (bottom-up partial sums).  For K > 0 the paper asks for the sums
 * sum_{x_k in Q} x_k^m u(x_k); here they are taken about each panel's centre
 * in units of its half-width, t = (x - c_Q)/(w_Q/2), which is the same
 * information re-expanded exactly (binomial shift) and avoids the
 * cancellation of raw monomials.  At a leaf the node sits at the centre, so
 * mu_0 = v and every higher moment is 0.  Parent from child (s in {0,1}^d):
 *   t_parent = (t_child + 2s - 1)/2.
 * pyr[l] holds (2^l)^d panels x M moments, panel-major.
 */
static double **build_pyramid(int d, int L, int K, const double *v)
{
    int al[512][3];
    const int M = moment_list(d, K, al);
    double **pyr = (double **)calloc(L + 1, sizeof(double *));
    for (int l = 0; l <= L; ++l) {
        int64_t P = num_nodes(d, 1 << l);
        pyr[l] = (double *)calloc((size_t)(P * M), sizeof(double));
    }
    const int64_t N = num_nodes(d, 1 << L);
    for (int64_t f = 0; f < N; ++f) pyr[L][f * M + 0] = v[f];
    for (int l = L - 1; l >= 0; --l) {
        const int np = 1 << l;
        const int64_t P = num_nodes(d, np);
        for (int64_t f = 0; f < P; ++f) {
            int64_t kp[3];
            unflatten(f, d, np, kp);
            for (int sz = 0; sz <= (d > 2); ++sz)
                for (int sy = 0; sy <= (d > 1); ++sy)
                    for (int sx = 0; sx <= 1; ++sx) {
                        int s[3] = { sx, sy, sz };
                        int64_t kc[3] = { 2 * kp[0] + sx, 2 * kp[1] + sy, 2 * kp[2] + sz };
                        int64_t fc = flatten(kc, d, 2 * np);
                        for (int ia = 0; ia < M; ++ia)
                            for (int ib = 0; ib < M; ++ib) {
                                double coef = 1.0;
                                int ok = 1;
                                for (int k = 0; k < d; ++k) {
                                    int A = al[ia][k], Bq = al[ib][k];
                                    if (Bq > A) { ok = 0; break; }
                                    double sg = (s[k] ? 1.0 : -1.0);
                                    coef *= binom(A, Bq) * pow(sg, A - Bq) * pow(0.5, A);
                                }
                                if (ok) pyr[l][f * M + ia] += coef * pyr[l + 1][fc * M + ib];
                            }
                    }
        }
    }
    return pyr;
}

static void free_pyramid(double **pyr, int L)
{
    for (int l = 0; l <= L; ++l) free(pyr[l]);
    free(pyr);
}

/* Geometry of Step 1, in half-units of h (integers): node X = 2 i + 1,
 * panel k of level l spans [k S, (k+1) S], S = 2^{L-l+1}. */
typedef struct {
    int d, L;
    int64_t X[3];
    double R2x4;          /* 4 R2_i: squared radius in half-units */
    int64_t *lev, *pk;    /* output list: level and flat panel index */
    int64_t cnt, cap;
    int64_t calls;        /* number of recur calls (N_d(x) of Step 1) */
} recur_ctx;

/* All 2^d corners strictly inside the open ball (full containment test). */
static int all_corners_inside(const recur_ctx *c, const int64_t lo[3], const int64_t hi[3])
{
    for (int m = 0; m < (1 << c->d); ++m) {
        int64_t dist2 = 0;
        for (int k = 0; k < c->d; ++k) {
            int64_t x = ((m >> k) & 1) ? hi[k] : lo[k];
            dist2 += (x - c->X[k]) * (x - c->X[k]);
        }
        if (!((double)dist2 < c->R2x4)) return 0;
    }
    return 1;
}

/* Algorithm 2: squared distance from the ball centre to the box, dmin < r^2. */
static int box_meets_ball(const recur_ctx *c, const int64_t lo[3], const int64_t hi[3])
{
    int64_t dmin = 0;
    for (int k = 0; k < c->d; ++k) {
        if (lo[k] > c->X[k]) dmin += (lo[k] - c->X[k]) * (lo[k] - c->X[k]);
        else if (hi[k] < c->X[k]) dmin += (hi[k] - c->X[k]) * (hi[k] - c->X[k]);
    }
    return (double)dmin < c->R2x4;
}

static void include_panel(recur_ctx *c, int l, int64_t f)
{
    if (c->cnt == c->cap) {
        c->cap = c->cap ? 2 * c->cap : 256;
        c->lev = (int64_t *)realloc(c->lev, c->cap * sizeof(int64_t));
        c->pk = (int64_t *)realloc(c->pk, c->cap * sizeof(int64_t));
    }
    c->lev[c->cnt] = l;
    c->pk[c->cnt] = f;
    c->cnt++;
}

/* Algorithm 1. */
static void recur(recur_ctx *c, int l, const int64_t k[3])
{
    c->calls++;
    const int64_t S = (int64_t)2 << (c->L - l);
    int64_t lo[3] = { 0, 0, 0 }, hi[3] = { 0, 0, 0 };
    for (int q = 0; q < c->d; ++q) { lo[q] = k[q] * S; hi[q] = (k[q] + 1) * S; }
    if (all_corners_inside(c, lo, hi)) {
        include_panel(c, l, flatten(k, c->d, 1 << l));
        return;
    }
    if (box_meets_ball(c, lo, hi)) {
        if (l < c->L) {
            for (int m = 0; m < (1 << c->d); ++m) {
                int64_t kc[3] = { 0, 0, 0 };
                for (int q = 0; q < c->d; ++q) kc[q] = 2 * k[q] + ((m >> q) & 1);
                recur(c, l + 1, kc);
            }
        } else {
            include_panel(c, l, flatten(k, c->d, 1 << l));
        }
    }
}

/* Step 1 for one node: the list of (level, panel) of the decomposition of
 * H_x cap Omega.  Returns the count; writes at most cap entries. */
int64_t or_tree_decompose(int d, int L, double delta_i, int64_t node, int64_t *lev,
                          int64_t *pk, int64_t cap, int64_t *calls)
{
    recur_ctx c;
    memset(&c, 0, sizeof(c));
    c.d = d; c.L = L;
    const int n = 1 << L;
    int64_t ci[3];
    unflatten(node, d, n, ci);
    for (int k = 0; k < 3; ++k) c.X[k] = 2 * ci[k] + 1;
    c.R2x4 = 4.0 * ((delta_i * n) * (delta_i * n));
    int64_t root[3] = { 0, 0, 0 };
    recur(&c, 0, root);
    for (int64_t t = 0; t < c.cnt && t < cap; ++t) { lev[t] = c.lev[t]; pk[t] = c.pk[t]; }
    if (calls) *calls = c.calls;
    int64_t cnt = c.cnt;
    free(c.lev); free(c.pk);
    return cnt;
}

/* Self term of Eq. (3.3).  PAPER: the continuous |H_x|-type integral
 * int_{B_delta} p(|xi|/delta) dxi = |S^{d-1}| delta^d sum_m p_m/(2m+d).
 * DISCRETE: h^d sum over every lattice cell (inside or outside Omega) that
 * meets the open ball, of p(|x_k - x_i|/delta) b_k, where b = a (XY
 * coefficient; exterior cells take a_i) or 1. */
static double self_term(int d, int n, int K, const double *p, int self_mode, int coef,
                        const double *a, int64_t fi, const int64_t ci[3], double di)
{
    if (self_mode == OR_SELF_PAPER) {
        double s = 0.0;
        for (int m = 0; m <= K; ++m) s += p[m] / (2.0 * m + d);
        return or_sphere_area(d) * pow(di, d) * s;
    }
    const double h = 1.0 / n;
    const double R2x4 = 4.0 * ((di * n) * (di * n));
    const int64_t B = (int64_t)ceil(di * n) + 1;
    const int64_t bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
    double acc = 0.0;
    for (int64_t oz = -bz; oz <= bz; ++oz)
        for (int64_t oy = -by; oy <= by; ++oy)
            for (int64_t ox = -B; ox <= B; ++ox) {
                int64_t o[3] = { ox, oy, oz }, cj[3];
                int64_t dmin = 0, o2 = 0;
                int inside = 1;
                for (int k = 0; k < d; ++k) {
                    /* node at 2i+1, cell i+o spans [2(i+o), 2(i+o)+2] */
                    int64_t lo = 2 * (ci[k] + o[k]), hi = lo + 2, X = 2 * ci[k] + 1;
                    if (lo > X) dmin += (lo - X) * (lo - X);
                    else if (hi < X) dmin += (hi - X) * (hi - X);
                    o2 += o[k] * o[k];
                    cj[k] = ci[k] + o[k];
                    if (cj[k] < 0 || cj[k] >= n) inside = 0;
                }
                if (!((double)dmin < R2x4)) continue;
                double b = 1.0;
                if (coef == OR_COEF_XY) b = inside ? a[flatten(cj, d, n)] : a[fi];
                acc += profile(OR_POLY, 0.0, K, p, sqrt((double)o2) * h / di) * b;
            }
    return pow(h, d) * acc;
}

/*
 * O1: the fast algorithm as the paper states it.  Step 1: recur() per
 * node; Step 2: the moment pyramid; Step 3: Eq. (3.5) summed over the
 * decomposition, each panel's integral of P(x,.) v obtained from its
 * moments; then Eq. (3.3).  Kernel: P = sigma A_x delta_x^{-(d+2)} p^{2K}.
 * v = a u for the XY coefficient (a(y) folded into the summed field), else u.
 * u, out: [nrhs][N]; panels (optional, per computed node): panel count.
 */
int or_fast_tree(int d, int L, const double *delta, int K, const double *p, double sigma,
                 int coef, const double *a, int self_mode, int nrhs, const double *u,
                 double *out, const int64_t *idx, int64_t nidx, int64_t *panels)
{
    if (d < 1 || d > 3 || L < 0 || L > 20 || K < 0 || K > 3) return 1;
    if (self_mode == OR_SELF_PAPER && coef == OR_COEF_XY) return 2;
    const int n = 1 << L;
    const int64_t N = num_nodes(d, n);
    const int64_t M = idx ? nidx : N;
    const double h = 1.0 / n, hd = pow(h, d);
    int al[512][3];
    const int nm = moment_list(d, K, al);
    double *v = (double *)malloc(sizeof(double) * N);
    for (int r = 0; r < nrhs; ++r) {
        const double *ur = u + (int64_t)r * N;
        for (int64_t f = 0; f < N; ++f) v[f] = (coef == OR_COEF_XY) ? a[f] * ur[f] : ur[f];
        double **pyr = build_pyramid(d, L, K, v);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t q = 0; q < M; ++q) {
            const int64_t fi = idx ? idx[q] : q;
            int64_t ci[3];
            unflatten(fi, d, n, ci);
            const double di = delta[fi];
            const double R2x4 = 4.0 * ((di * n) * (di * n));
            int64_t cap = 1 << 12;
            int64_t *lev = (int64_t *)malloc(cap * sizeof(int64_t));
            int64_t *pk = (int64_t *)malloc(cap * sizeof(int64_t));
            int64_t cnt = or_tree_decompose(d, L, di, fi, lev, pk, cap, NULL);
            if (cnt > cap) {
                cap = cnt;
                lev = (int64_t *)realloc(lev, cap * sizeof(int64_t));
                pk = (int64_t *)realloc(pk, cap * sizeof(int64_t));
                or_tree_decompose(d, L, di, fi, lev, pk, cap, NULL);
            }
            if (panels && r == 0) panels[q] = cnt;
            double G = 0.0;
            for (int64_t t = 0; t < cnt; ++t) {
                const int l = (int)lev[t];
                int64_t kp[3];
                unflatten(pk[t], d, 1 << l, kp);
                const int64_t S = (int64_t)2 << (L - l);
                /* q(t) = p(|B + H t| / (2 rho)) as a polynomial in t, with
                 * B = panel centre - node and H = half-width (half-units). */
                double Bv[3] = { 0, 0, 0 };
                for (int k = 0; k < d; ++k) Bv[k] = (double)(kp[k] * S + S / 2 - (2 * ci[k] + 1));
                const double H = (double)(S / 2);
                /* dense coefficient arrays over exponents 0..2K per dimension */
                const int E = 2 * K + 1;
                double qc[7 * 7 * 7], rc[7 * 7 * 7], tmp[7 * 7 * 7];
                memset(qc, 0, sizeof(qc));
                memset(rc, 0, sizeof(rc));
                /* rc = |B + H t|^2 / (4 R2) */
                for (int k = 0; k < d; ++k) {
                    int e1[3] = { 0, 0, 0 }, e2[3] = { 0, 0, 0 };
                    e1[k] = 1; e2[k] = 2;
                    rc[0] += Bv[k] * Bv[k] / R2x4;
                    rc[e1[0] + E * (e1[1] + E * e1[2])] += 2.0 * Bv[k] * H / R2x4;
                    rc[e2[0] + E * (e2[1] + E * e2[2])] += H * H / R2x4;
                }
                /* qc = sum_m p_m rc^m, accumulated with a running power */
                double pw[7 * 7 * 7];
                memset(pw, 0, sizeof(pw));
                pw[0] = 1.0;
                for (int m = 0; m <= K; ++m) {
                    for (int e = 0; e < E * E * E; ++e) qc[e] += p[m] * pw[e];
                    if (m == K) break;
                    memset(tmp, 0, sizeof(tmp));
                    for (int e0 = 0; e0 < E; ++e0)
                        for (int e1 = 0; e1 < E; ++e1)
                            for (int e2 = 0; e2 < E; ++e2) {
                                double pv = pw[e0 + E * (e1 + E * e2)];
                                if (pv == 0.0) continue;
                                for (int f0 = 0; f0 <= 2; ++f0)
                                    for (int f1 = 0; f1 <= 2; ++f1)
                                        for (int f2 = 0; f2 <= 2; ++f2) {
                                            double rv = rc[f0 + E * (f1 + E * f2)];
                                            if (rv == 0.0) continue;
                                            int g0 = e0 + f0, g1 = e1 + f1, g2 = e2 + f2;
                                            if (g0 >= E || g1 >= E || g2 >= E) continue;
                                            tmp[g0 + E * (g1 + E * g2)] += pv * rv;
                                        }
                            }
                    memcpy(pw, tmp, sizeof(tmp));
                }
                const double *mu = pyr[l] + pk[t] * nm;
                for (int ia = 0; ia < nm; ++ia)
                    G += qc[al[ia][0] + E * (al[ia][1] + E * al[ia][2])] * mu[ia];
            }
            G *= hd;
            const double Sx = self_term(d, n, K, p, self_mode, coef, a, fi, ci, di);
            double Ax = (coef == OR_COEF_NONE) ? 1.0 : a[fi];
            out[(int64_t)r * M + q] = sigma * Ax * pow(di, -(d + 2.0)) * (G - ur[fi] * Sx);
            free(lev);
            free(pk);
        }
        free_pyramid(pyr, L);
    }
    free(v);
    return 0;
}

/*
 * O2: the same quantity as a plain sum over the leaf set
 *   LS(i) = { leaf cells k in Omega : dmin(cell_k, x_i) < delta_i },
 * which is exactly the union of the panels Algorithm 1 includes:
 *   G_i = h^d sum_{k in LS(i)} p(|x_k - x_i|/delta_i) v_k.
 */
int or_fast_leafset(int d, int L, const double *delta, int K, const double *p, double sigma,
                    int coef, const double *a, int self_mode, int nrhs, const double *u,
                    double *out, const int64_t *idx, int64_t nidx, int64_t *cells)
{
    if (d < 1 || d > 3 || L < 0 || L > 20 || K < 0) return 1;
    if (self_mode == OR_SELF_PAPER && coef == OR_COEF_XY) return 2;
    const int n = 1 << L;
    const int64_t N = num_nodes(d, n);
    const int64_t M = idx ? nidx : N;
    const double h = 1.0 / n, hd = pow(h, d);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < M; ++q) {
        const int64_t fi = idx ? idx[q] : q;
        int64_t ci[3];
        unflatten(fi, d, n, ci);
        const double di = delta[fi];
        const double R2x4 = 4.0 * ((di * n) * (di * n));
        const int64_t B = (int64_t)ceil(di * n) + 1;
        const int64_t bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
        const double Sx = self_term(d, n, K, p, self_mode, coef, a, fi, ci, di);
        const double Ax = (coef == OR_COEF_NONE) ? 1.0 : a[fi];
        for (int r = 0; r < nrhs; ++r) {
            const double *ur = u + (int64_t)r * N;
            double G = 0.0;
            int64_t count = 0;
            for (int64_t oz = -bz; oz <= bz; ++oz)
                for (int64_t oy = -by; oy <= by; ++oy)
                    for (int64_t ox = -B; ox <= B; ++ox) {
                        int64_t o[3] = { ox, oy, oz }, cj[3];
                        int64_t dmin = 0, o2 = 0;
                        int inside = 1;
                        for (int k = 0; k < d; ++k) {
                            int64_t lo = 2 * (ci[k] + o[k]), hi = lo + 2, X = 2 * ci[k] + 1;
                            if (lo > X) dmin += (lo - X) * (lo - X);
                            else if (hi < X) dmin += (hi - X) * (hi - X);
                            o2 += o[k] * o[k];
                            cj[k] = ci[k] + o[k];
                            if (cj[k] < 0 || cj[k] >= n) inside = 0;
                        }
                        if (!inside || !((double)dmin < R2x4)) continue;
                        const int64_t fj = flatten(cj, d, n);
                        const double vj = (coef == OR_COEF_XY) ? a[fj] * ur[fj] : ur[fj];
                        G += profile(OR_POLY, 0.0, K, p, sqrt((double)o2) * h / di) * vj;
                        ++count;
                    }
            if (cells && r == 0) cells[q] = count;
            out[(int64_t)r * M + q] = sigma * Ax * pow(di, -(d + 2.0)) * (hd * G - ur[fi] * Sx);
        }
    }
    return 0;
}

/*
 * Symmetrised leaf-set operator of the polynomial kernel (a project extension: the paper's
 * fast algorithm, Sec. 3, is stated for C(x), delta(x) only; its case (b) of Sec. 2, the
 * divergence type with symmetric C and delta, is not covered).  With the leaf-set relation
 *   k ~ i  iff  cell_k meets the open ball B(x_i, delta_i)
 * (the quadrature set of Algorithm 1) and the one-sided weight
 *   w_i(k) = C_ik delta_i^{-(d+2)} p(|x_k - x_i| / delta_i) [k ~ i],
 * the symmetrised weight of a node pair in Omega is (w_i(k) + w_k(i)) / 2, each half with its
 * own node's horizon; a cell outside Omega takes a_k = a_i and delta_k = delta_i (so both
 * halves agree there: the cell-to-node distance is the same both ways) and u_k = 0:
 *   (L u)_i = sigma h^d sum_{k != i} w^s_ik (u_k - u_i).
 * C = 1 (coef NONE) or a_i a_k (coef XY).  u, out: [nrhs][N]; idx as above.
 */
int or_fast_sym_leafset(int d, int L, const double *delta, int K, const double *p, double sigma,
                        int coef, const double *a, int nrhs, const double *u, double *out,
                        const int64_t *idx, int64_t nidx)
{
    if (d < 1 || d > 3 || L < 0 || L > 20 || K < 0) return 1;
    if (coef != OR_COEF_NONE && coef != OR_COEF_XY) return 2;
    const int n = 1 << L;
    const int64_t N = num_nodes(d, n);
    const int64_t M = idx ? nidx : N;
    const double h = 1.0 / n, hd = pow(h, d);
    double dmax = 0.0;
    for (int64_t f = 0; f < N; ++f) if (delta[f] > dmax) dmax = delta[f];
    const int64_t B = (int64_t)ceil(dmax * n) + 1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < M; ++q) {
        const int64_t fi = idx ? idx[q] : q;
        int64_t ci[3];
        unflatten(fi, d, n, ci);
        const double di = delta[fi];
        const double ai = (coef == OR_COEF_XY) ? a[fi] : 1.0;
        const double R2i4 = 4.0 * ((di * n) * (di * n));
        const int64_t bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
        for (int r = 0; r < nrhs; ++r) {
            const double *ur = u + (int64_t)r * N;
            double acc = 0.0;
            for (int64_t oz = -bz; oz <= bz; ++oz)
                for (int64_t oy = -by; oy <= by; ++oy)
                    for (int64_t ox = -B; ox <= B; ++ox) {
                        int64_t o[3] = { ox, oy, oz }, ck[3];
                        int64_t dmin = 0, o2 = 0;
                        int inside = 1;
                        for (int k = 0; k < d; ++k) {
                            /* half units: cell_k spans [2 c_k, 2 c_k + 2], node i at 2 c_i + 1 */
                            int64_t lo = 2 * (ci[k] + o[k]), hi = lo + 2, X = 2 * ci[k] + 1;
                            if (lo > X) dmin += (lo - X) * (lo - X);
                            else if (hi < X) dmin += (hi - X) * (hi - X);
                            o2 += o[k] * o[k];
                            ck[k] = ci[k] + o[k];
                            if (ck[k] < 0 || ck[k] >= n) inside = 0;
                        }
                        if (o2 == 0) continue;
                        const double rr = sqrt((double)o2) * h;
                        const int64_t fk = inside ? flatten(ck, d, n) : -1;
                        const double ak = (coef == OR_COEF_XY && inside) ? a[fk] : ai;
                        const double dk = inside ? delta[fk] : di;
                        const double R2k4 = 4.0 * ((dk * n) * (dk * n));
                        const double wi = ((double)dmin < R2i4)
                            ? pow(di, -(d + 2.0)) * profile(OR_POLY, 0.0, K, p, rr / di) : 0.0;
                        const double wk = ((double)dmin < R2k4)
                            ? pow(dk, -(d + 2.0)) * profile(OR_POLY, 0.0, K, p, rr / dk) : 0.0;
                        const double w = 0.5 * (wi + wk) * ai * ak;
                        if (w == 0.0) continue;
                        const double uk = inside ? ur[fk] : 0.0;
                        acc += w * (uk - ur[fi]);
                    }
            out[(int64_t)r * M + q] = sigma * hd * acc;
        }
    }
    return 0;
}

/*
 * Fast-path peridynamics (the polynomial micromodulus of the paper's outlook): the bond tensor
 * xi xi^T / |xi|^3 of Eq. (1.2), i.e. xi xi^T gamma(|xi|/delta_i) / delta_i^3 with the profile
 * gamma(s) = s^{-3}, is replaced by xi xi^T p^{2K}(|xi|/delta_i) / delta_i^3, p^{2K} the even
 * polynomial of degree 2K matching s^{-3} and its first K derivatives at s = 1 (the splitting
 * of Sec. 3 applied to this profile; K = 0 gives p = 1), and the sum runs over the leaf set of
 * Algorithm 1 (every leaf cell, inside Omega or not, that meets the open ball of x_i):
 *   (L u)_i = h^d sum_{k in LS(i), k != i} sigma c_ik p(|xi|/delta_i) (xi xi^T / delta_i^3)
 *             (u_k - u_i),
 * c_ik = (c_i + c_k)/2, with u_k = 0 and c_k = c_i for cells outside Omega.  p holds p_0..p_K
 * (p(s) = sum_m p_m s^{2m}).  u, out: [nrhs][d][N].  idx as above.
 */
int or_fast_pd_leafset(int d, int L, const double *delta, const double *c, double sigma, int K,
                       const double *p, int nrhs, const double *u, double *out,
                       const int64_t *idx, int64_t nidx)
{
    if (d < 1 || d > 3 || L < 0 || L > 20 || K < 0 || K > 7 || !p) return 1;
    const int n = 1 << L;
    const int64_t N = num_nodes(d, n);
    const int64_t M = idx ? nidx : N;
    const double h = 1.0 / n, hd = pow(h, d);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < M; ++q) {
        const int64_t fi = idx ? idx[q] : q;
        int64_t ci[3];
        unflatten(fi, d, n, ci);
        const double di = delta[fi];
        const double R2x4 = 4.0 * ((di * n) * (di * n));
        const int64_t B = (int64_t)ceil(di * n) + 1;
        const int64_t bz = d > 2 ? B : 0, by = d > 1 ? B : 0;
        const double pre = sigma * hd / (di * di * di);
        for (int r = 0; r < nrhs; ++r) {
            const double *ur = u + (int64_t)r * d * N;
            double acc[3] = { 0, 0, 0 };
            for (int64_t oz = -bz; oz <= bz; ++oz)
                for (int64_t oy = -by; oy <= by; ++oy)
                    for (int64_t ox = -B; ox <= B; ++ox) {
                        int64_t o[3] = { ox, oy, oz }, cj[3];
                        int64_t dmin = 0;
                        int inside = 1;
                        for (int k = 0; k < d; ++k) {
                            int64_t lo = 2 * (ci[k] + o[k]), hi = lo + 2, X = 2 * ci[k] + 1;
                            if (lo > X) dmin += (lo - X) * (lo - X);
                            else if (hi < X) dmin += (hi - X) * (hi - X);
                            cj[k] = ci[k] + o[k];
                            if (cj[k] < 0 || cj[k] >= n) inside = 0;
                        }
                        if (!((double)dmin < R2x4)) continue;
                        if (ox == 0 && oy == 0 && oz == 0) continue;
                        const int64_t fj = inside ? flatten(cj, d, n) : -1;
                        double xi[3], xdu = 0.0;
                        for (int k = 0; k < d; ++k) {
                            xi[k] = (double)o[k] * h;
                            const double uj = inside ? ur[(int64_t)k * N + fj] : 0.0;
                            xdu += xi[k] * (uj - ur[(int64_t)k * N + fi]);
                        }
                        double r2 = 0.0;                  /* |xi|^2 / delta_i^2 */
                        for (int k = 0; k < d; ++k) r2 += xi[k] * xi[k];
                        r2 /= di * di;
                        double w = 0.0, pw = 1.0;          /* p(s) = sum_m p_m s^{2m} */
                        for (int m = 0; m <= K; ++m) { w += p[m] * pw; pw *= r2; }
                        const double cik = 0.5 * (c[fi] + (inside ? c[fj] : c[fi]));
                        for (int k = 0; k < d; ++k) acc[k] += cik * w * xdu * xi[k];
                    }
            for (int k = 0; k < d; ++k) out[((int64_t)r * d + k) * M + q] = pre * acc[k];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Conjugate gradients on -L x = f (the Krylov use of Sec. 4)           */
/* ------------------------------------------------------------------ */

typedef struct {
    int kind;             /* 0 scalar (symmetric variant), 1 peridynamics */
    int d, n, family, K, coef;
    double alpha, sigma;
    const double *delta, *a, *p, *c;
} cg_op;

static void cg_apply_neg(const cg_op *op, const double *x, double *y)
{
    const int64_t N = num_nodes(op->d, op->n);
    int64_t len = op->kind == 0 ? N : N * op->d;
    if (op->kind == 0)
        or_direct_scalar(op->d, op->n, op->delta, op->family, op->alpha, op->K, op->p, op->sigma,
                         op->coef, op->a, 1, 1, x, y, NULL, 0);
    else
        or_pd_direct(op->d, op->n, op->delta, op->c, op->sigma, 1, x, y, NULL, 0);
    for (int64_t t = 0; t < len; ++t) y[t] = -y[t];
}

static double dot(const double *x, const double *y, int64_t len)
{
    double s = 0.0;
    for (int64_t t = 0; t < len; ++t) s += x[t] * y[t];
    return s;
}

/*
 * Preconditioned CG for -L x = f, x0 = 0.  precond: 0 none, 1 Jacobi
 * (inverse diagonal in dinv, length of x).  Stops when ||f + L x|| <=
 * rtol ||f|| with the residual recomputed from the operator.
 */
int or_cg(int kind, int d, int n, const double *delta, int family, double alpha, int K,
          const double *p, double sigma, int coef, const double *a, const double *c,
          const double *dinv, const double *f, double *x, double rtol, int maxit,
          int *iters, double *relres)
{
    cg_op op = { kind, d, n, family, K, coef, alpha, sigma, delta, a, p, c };
    const int64_t N = num_nodes(d, n);
    const int64_t len = kind == 0 ? N : N * d;
    double *r = (double *)malloc(len * sizeof(double));
    double *z = (double *)malloc(len * sizeof(double));
    double *pp = (double *)malloc(len * sizeof(double));
    double *q = (double *)malloc(len * sizeof(double));
    for (int64_t t = 0; t < len; ++t) { x[t] = 0.0; r[t] = f[t]; }
    const double fn = sqrt(dot(f, f, len));
    for (int64_t t = 0; t < len; ++t) z[t] = dinv ? dinv[t] * r[t] : r[t];
    memcpy(pp, z, len * sizeof(double));
    double rz = dot(r, z, len);
    int it = 0;
    double rel = fn > 0 ? sqrt(dot(r, r, len)) / fn : 0.0;
    while (it < maxit && rel > rtol) {
        cg_apply_neg(&op, pp, q);
        const double alpha_k = rz / dot(pp, q, len);
        for (int64_t t = 0; t < len; ++t) { x[t] += alpha_k * pp[t]; r[t] -= alpha_k * q[t]; }
        for (int64_t t = 0; t < len; ++t) z[t] = dinv ? dinv[t] * r[t] : r[t];
        const double rz_new = dot(r, z, len);
        const double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t t = 0; t < len; ++t) pp[t] = z[t] + beta * pp[t];
        ++it;
        rel = sqrt(dot(r, r, len)) / fn;
    }
    /* true residual */
    cg_apply_neg(&op, x, q);
    for (int64_t t = 0; t < len; ++t) q[t] = f[t] - q[t];
    *relres = fn > 0 ? sqrt(dot(q, q, len)) / fn : 0.0;
    *iters = it;
    free(r); free(z); free(pp); free(q);
    return *relres <= rtol ? 0 : 5;
}
