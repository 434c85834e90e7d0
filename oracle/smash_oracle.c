/*
 * smash_oracle.c -- plain, slow, serial CPU oracle for the SMASH H^2 path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this code.  It shares nothing with the CUDA library:
 * every step is written out here from the paper (Cai, Chow, Saad, Xi,
 * "SMASH: Structured Matrix Approximation by Separation and Hierarchy").
 *
 * What it computes, in the paper's order:
 *   - dense brute force  z_i = sum_j kappa(x_i, y_j) q_j  (Neumaier-compensated),
 *     the plain definition of A q (Sections 1.2 and 2.2);
 *   - adaptive partitioning of the bounding cube (Section 3.1);
 *   - admissible leaves L (3.3) and inadmissible leaves L^- (3.4) with the
 *     well-separation test of Definition 2.1 applied to node cells (4.6);
 *   - interpolation bases U^_i from Lagrange polynomials at Chebyshev anchors
 *     of the node cell (2.2) and the basis choice discussed around (3.1);
 *   - compr = strong rank-revealing QR of U^_i^T (Theorem 2.4, s = f = 2)
 *     giving the interpolative decomposition (2.11)/(2.14);
 *   - the bottom-up H^2 construction (3.16)-(3.20);
 *   - the node-wise H^2 matvec of Section 3.4 (upward, coupling, downward,
 *     near field).
 *
 * Readings of the paper that are not fixed by its text are applied exactly
 * as the design notes list them: cube normalisation, Morton digit order,
 * split iff count > leaf_size, cell-based admissibility, Chebyshev anchors
 * of the first kind, ascending skeleton order, QR with column pivoting
 * stopped at |R_jj| <= tol |R_00|, followed by Gu-Eisenstat swaps until
 * max_ij (A_ij^2 + gamma_j^2 / omega_i^2) <= f^2.
 *
 * Compile with -ffp-contract=off: a*b+c below is two rounded operations unless
 * it is written as fma(a, b, c), the IEEE fused multiply-add (one rounding);
 * the dot products, norms and triangular solves use fma.
 *
 * The loops over the nodes of one level, over the nodes of the matvec passes
 * and over the rows of the dense product carry OpenMP pragmas.  Each
 * iteration writes only its own node's (or row's) results, so a build with
 * -fopenmp computes the same bits on several host threads; the default build
 * ignores the pragmas and runs serially.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_MAXP 64
#define ORC_MAX_SWAPS 1000

enum { ORC_K_LOG = 0, ORC_K_INVR = 1, ORC_K_YUKAWA = 2, ORC_K_CAUCHY = 3, ORC_K_DLP1 = 4, ORC_K_DLP2 = 5 };

/* ------------------------------------------------------------------------ */
/* kernels (2.1) with the diagonal value 0                                   */
/* ------------------------------------------------------------------------ */

double orc_kernel(int kid, int d, const double *x, const double *y)
{
    if (kid == ORC_K_CAUCHY) {
        double t = x[0] - y[0];
        return t == 0.0 ? 0.0 : 1.0 / t;
    }
    double r2 = 0.0;
    for (int a = 0; a < d; ++a) {
        double t = x[a] - y[a];
        r2 += t * t;
    }
    if (r2 == 0.0)
        return 0.0;
    /* Section 6.4: the gradient in y of Phi(x, y) = -(1/2 pi) log|x - y| is
     * -(1/2 pi) (y - x) / |x - y|^2; kernels 4 and 5 are its two components (d = 2) */
    if (kid == ORC_K_DLP1) return -(y[0] - x[0]) / (2.0 * ORC_PI * r2);
    if (kid == ORC_K_DLP2) return -(y[1] - x[1]) / (2.0 * ORC_PI * r2);
    double r = sqrt(r2);
    switch (kid) {
    case ORC_K_LOG: return log(r);
    case ORC_K_INVR: return 1.0 / r;
    case ORC_K_YUKAWA: return exp(-r) / r;
    default: return 0.0;
    }
}

/* Neumaier-compensated dense product for selected rows:
 * out[t*nrhs+c] = sum_j kappa(x[rows[t]], y[j]) q[j*nrhs+c]. */
void orc_dense_rows(const double *x, int64_t nx, const double *y, int64_t ny, int d, int kid,
                    const double *q, int nrhs, const int64_t *rows, int64_t nrows, double *out)
{
    (void)nx;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nrows; ++t) {
        double *sum = malloc(sizeof(double) * (size_t)nrhs);
        double *comp = malloc(sizeof(double) * (size_t)nrhs);
        const double *xi = x + rows[t] * d;
        for (int c = 0; c < nrhs; ++c) { sum[c] = 0.0; comp[c] = 0.0; }
        for (int64_t j = 0; j < ny; ++j) {
            double k = orc_kernel(kid, d, xi, y + j * d);
            for (int c = 0; c < nrhs; ++c) {
                double v = k * q[j * nrhs + c];
                double s = sum[c] + v;
                if (fabs(sum[c]) >= fabs(v))
                    comp[c] += (sum[c] - s) + v;
                else
                    comp[c] += (v - s) + sum[c];
                sum[c] = s;
            }
        }
        for (int c = 0; c < nrhs; ++c)
            out[t * nrhs + c] = sum[c] + comp[c];
        free(sum);
        free(comp);
    }
}

/* ------------------------------------------------------------------------ */
/* Section 6.1 parameter heuristic                                           */
/* ------------------------------------------------------------------------ */

int orc_suggest_rank(double eps, double tau)
{
    double v = log(eps) / log(tau);
    if (eps < 1e-8)
        return (int)floor(v - 20.0);
    if (eps < 1e-6)
        return (int)floor(v - 15.0);
    int r = (int)floor(v - 10.0);
    return r > 5 ? r : 5;
}

/* ------------------------------------------------------------------------ */
/* Section 3.1: bounding cube and Morton keys                                */
/* ------------------------------------------------------------------------ */

int orc_bits_per_dim(int d) { return d == 1 ? 62 : (d == 2 ? 31 : 21); }

/* Smallest axis-aligned cube [lo, lo+s]^d holding X and Y (y may be NULL).
 * s = largest extent times (1 + 2^-40), or 1 when all points coincide. */
void orc_bounding_cube(const double *x, int64_t nx, const double *y, int64_t ny, int d,
                       double *lo, double *s)
{
    double hi[3];
    for (int a = 0; a < d; ++a) { lo[a] = x[a]; hi[a] = x[a]; }
    for (int64_t i = 0; i < nx; ++i)
        for (int a = 0; a < d; ++a) {
            double v = x[i * d + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    if (y)
        for (int64_t i = 0; i < ny; ++i)
            for (int a = 0; a < d; ++a) {
                double v = y[i * d + a];
                if (v < lo[a]) lo[a] = v;
                if (v > hi[a]) hi[a] = v;
            }
    double ext = 0.0;
    for (int a = 0; a < d; ++a)
        if (hi[a] - lo[a] > ext) ext = hi[a] - lo[a];
    *s = ext > 0.0 ? ext * (1.0 + 0x1p-40) : 1.0;
}

/* Integer cell coordinate of one coordinate value at the finest level:
 * floor((v - lo)/s * 2^b), clamped to [0, 2^b - 1]. */
static uint64_t orc_quantize(double v, double lo, double s, int b)
{
    double t = (v - lo) / s;
    double f = floor(t * ldexp(1.0, b));
    uint64_t top = (((uint64_t)1) << b) - 1;
    if (!(f > 0.0))
        return 0;
    if (f >= ldexp(1.0, b))
        return top;
    uint64_t q = (uint64_t)f;
    return q > top ? top : q;
}

/* Morton key: b digits of d bits, most significant digit first; within a
 * digit, dimension 0 is the most significant bit. */
uint64_t orc_morton_key(const double *pt, int d, const double *lo, double s)
{
    int b = orc_bits_per_dim(d);
    uint64_t q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a)
        q[a] = orc_quantize(pt[a], lo[a], s, b);
    uint64_t key = 0;
    for (int l = 0; l < b; ++l)
        for (int a = 0; a < d; ++a)
            key = (key << 1) | ((q[a] >> (b - 1 - l)) & 1u);
    return key;
}

void orc_morton_keys(const double *pts, int64_t n, int d, const double *lo, double s, uint64_t *keys)
{
    for (int64_t i = 0; i < n; ++i)
        keys[i] = orc_morton_key(pts + i * d, d, lo, s);
}

typedef struct { uint64_t key; int64_t idx; } orc_kv;

static int orc_kv_cmp(const void *pa, const void *pb)
{
    const orc_kv *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/* Stable sort of the points by key: perm[p] = original index at sorted position p. */
static void orc_sort_points(const double *pts, int64_t n, int d, const double *lo, double s,
                            int64_t *perm, uint64_t *keys_sorted, double *pts_sorted)
{
    orc_kv *kv = malloc(sizeof(orc_kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        kv[i].key = orc_morton_key(pts + i * d, d, lo, s);
        kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(orc_kv), orc_kv_cmp);
    for (int64_t p = 0; p < n; ++p) {
        perm[p] = kv[p].idx;
        keys_sorted[p] = kv[p].key;
        for (int a = 0; a < d; ++a)
            pts_sorted[p * d + a] = pts[kv[p].idx * d + a];
    }
    free(kv);
}

/* ------------------------------------------------------------------------ */
/* Definition 2.1 on cells                                                    */
/* ------------------------------------------------------------------------ */

/* Cells are dyadic cubes: a node at level l (root = 1) with integer cell
 * coordinates c has side h_l = s 2^(1-l), centre lo + (c + 1/2) h_l and
 * radius sqrt(d) h_l / 2 (the smallest ball around the cube).  In units of
 * half the finer cell, u = s 2^-m with m = max(li, lj), the centres are the
 * integers (2c+1) 2^(m-l) and the radii sqrt(d) 2^(m-l).  (2.3) squared:
 *     d (2^(m-li) + 2^(m-lj))^2  <=  tau^2 sum_a D_a^2,
 * D the integer centre difference.  Returns 1 when well-separated. */
int orc_admissible(int d, int li, const uint64_t *ci, int lj, const uint64_t *cj, double tau)
{
    int m = li > lj ? li : lj;
    double e = ldexp(1.0, m - li) + ldexp(1.0, m - lj);
    double lhs = (double)d * (e * e);
    double sum = 0.0;
    for (int a = 0; a < d; ++a) {
        uint64_t Ci = (2 * ci[a] + 1) << (m - li);
        uint64_t Cj = (2 * cj[a] + 1) << (m - lj);
        uint64_t D = Ci >= Cj ? Ci - Cj : Cj - Ci;
        double Dd = (double)D;
        sum = sum + Dd * Dd;
    }
    double tau2 = tau * tau;
    return lhs <= tau2 * sum;
}

/* ------------------------------------------------------------------------ */
/* (2.2): Lagrange polynomials at Chebyshev points, tensor basis             */
/* ------------------------------------------------------------------------ */

/* Chebyshev points of the first kind on [-1, 1]. */
void orc_chebyshev(int p, double *t)
{
    for (int m = 0; m < p; ++m)
        t[m] = cos((double)(2 * m + 1) * ORC_PI / (double)(2 * p));
}

/* Weights of the Lagrange polynomials of the anchors:
 * w_m = 1 / prod_{n != m} (t_m - t_n). */
void orc_lagrange_weights(int p, const double *anchors, double *w)
{
    for (int m = 0; m < p; ++m) {
        double den = 1.0;
        for (int n = 0; n < p; ++n)
            if (n != m) den = den * (anchors[m] - anchors[n]);
        w[m] = 1.0 / den;
    }
}

/* ell_m(t) = prod_{n != m} (t - t_n) / (t_m - t_n) = w_m prod_{n != m} (t - t_n). */
double orc_lagrange(int p, const double *anchors, const double *w, int m, double t)
{
    double v = w[m];
    for (int n = 0; n < p; ++n)
        if (n != m) v = v * (t - anchors[n]);
    return v;
}

/* Transpose of the interpolation basis of one cell, evaluated at npts points:
 * Mt[kk * npts + c] = prod_a ell_{k_a}(t_a(x_c)), kk = (k_0 p + k_1) p + k_2
 * (last dimension fastest), t_a = (x_a - centre_a) / (h/2) in [-1, 1].
 * The cell: level l (root 1) with integer coordinates cell[] in the cube
 * [lo, lo+s]^d. */
void orc_basis_t(int d, int p, const double *anchors, const double *lo, double s, int level,
                 const uint64_t *cell, const double *pts, int npts, double *Mt)
{
    double h = ldexp(s, 1 - level);
    double half = 0.5 * h;
    int r = 1;
    for (int a = 0; a < d; ++a) r *= p;
    double L[3][ORC_MAXP], wts[ORC_MAXP];
    orc_lagrange_weights(p, anchors, wts);
    for (int c = 0; c < npts; ++c) {
        for (int a = 0; a < d; ++a) {
            double centre = lo[a] + ((double)cell[a] + 0.5) * h;
            double t = (pts[c * d + a] - centre) / half;
            for (int m = 0; m < p; ++m)
                L[a][m] = orc_lagrange(p, anchors, wts, m, t);
        }
        for (int kk = 0; kk < r; ++kk) {
            int rem = kk, idx[3] = {0, 0, 0};
            for (int a = d - 1; a >= 0; --a) { idx[a] = rem % p; rem /= p; }
            double v = L[0][idx[0]];
            for (int a = 1; a < d; ++a) v = v * L[a][idx[a]];
            Mt[(size_t)kk * npts + c] = v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Theorem 2.4: strong rank-revealing QR and the ID (2.11)                   */
/* ------------------------------------------------------------------------ */

/* One Householder step on column j of W (r x m row-major), rows j..r-1,
 * applied to the columns j+1..m-1.  Afterwards W[j][j] = R_jj and the
 * entries below it are zero. */
static void orc_householder(double *W, int r, int m, int j, double *v)
{
    double alpha = W[(size_t)j * m + j];
    double sigma = 0.0;
    for (int i = j + 1; i < r; ++i) {
        double x = W[(size_t)i * m + j];
        sigma = fma(x, x, sigma);
    }
    if (sigma == 0.0)
        return; /* already triangular in this column: H = I */
    double nrm = sqrt(fma(alpha, alpha, sigma));
    double beta = alpha <= 0.0 ? nrm : -nrm;
    double tau = (beta - alpha) / beta;
    double den = alpha - beta;
    v[j] = 1.0;
    for (int i = j + 1; i < r; ++i)
        v[i] = W[(size_t)i * m + j] / den;
    for (int c = j + 1; c < m; ++c) {
        double w = W[(size_t)j * m + c];
        for (int i = j + 1; i < r; ++i)
            w = fma(v[i], W[(size_t)i * m + c], w);
        double tw = tau * w;
        W[(size_t)j * m + c] = W[(size_t)j * m + c] - tw;
        for (int i = j + 1; i < r; ++i)
            W[(size_t)i * m + c] = fma(-tw, v[i], W[(size_t)i * m + c]);
    }
    W[(size_t)j * m + j] = beta;
    for (int i = j + 1; i < r; ++i)
        W[(size_t)i * m + j] = 0.0;
}

/* Householder QR of W (r x m).  pivot = 1: column pivoting on the largest
 * remaining column norm (ties: lowest position), stopping before step j
 * when |R_jj| <= tol |R_00|; returns the number of steps k.  pivot = 0:
 * exactly ksteps steps in the given column order. */
static int orc_qr(double *W, int r, int m, int *perm, int pivot, int ksteps, double tol,
                  double *nrm2, double *v)
{
    int kmax = pivot ? (r < m ? r : m) : ksteps;
    double r00 = 0.0;
    for (int j = 0; j < kmax; ++j) {
        if (pivot) {
            for (int c = j; c < m; ++c) {
                double s2 = 0.0;
                for (int i = j; i < r; ++i) {
                    double x = W[(size_t)i * m + c];
                    s2 = fma(x, x, s2);
                }
                nrm2[c] = s2;
            }
            int piv = j;
            for (int c = j + 1; c < m; ++c)
                if (nrm2[c] > nrm2[piv]) piv = c;
            double nrm = sqrt(nrm2[piv]);
            if (j == 0) {
                r00 = nrm;
                if (nrm == 0.0) return 0;
            } else if (nrm <= tol * r00) {
                return j;
            }
            if (piv != j) {
                for (int i = 0; i < r; ++i) {
                    double t = W[(size_t)i * m + j];
                    W[(size_t)i * m + j] = W[(size_t)i * m + piv];
                    W[(size_t)i * m + piv] = t;
                }
                int tp = perm[j]; perm[j] = perm[piv]; perm[piv] = tp;
            }
        }
        orc_householder(W, r, m, j, v);
    }
    return kmax;
}

/* compr (2.14) on Mt = U^_i^T (r x m, row-major; not modified).
 * Output: perm (m entries; perm[0..k) are the selected columns = skeleton
 * positions, perm[k..m) the rest), *k_out, A = R11^{-1} R12 (k x (m-k),
 * row-major) and the number of Gu-Eisenstat swaps (-1 if the cap was hit).
 * A must hold k*(m-k) doubles with k <= min(r, m). */
int orc_compr(const double *Mt, int r, int m, double tol, double f, int *perm, int *k_out,
              double *A, int *nswaps_out)
{
    double *W = malloc(sizeof(double) * (size_t)r * (size_t)(m > 0 ? m : 1));
    double *nrm2 = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *v = malloc(sizeof(double) * (size_t)(r > 0 ? r : 1));
    for (int c = 0; c < m; ++c) perm[c] = c;
    memcpy(W, Mt, sizeof(double) * (size_t)r * (size_t)m);
    int k = orc_qr(W, r, m, perm, 1, 0, tol, nrm2, v);
    int nsw = 0;
    int mk = m - k;
    double *X = malloc(sizeof(double) * (size_t)(k > 0 ? k * k : 1));
    double *rho = malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double *g2 = malloc(sizeof(double) * (size_t)(mk > 0 ? mk : 1));
    for (;;) {
        if (k == 0 || mk == 0) break;
        /* A = R11^{-1} R12 by back substitution, one column at a time */
        for (int u = 0; u < mk; ++u)
            for (int t = k - 1; t >= 0; --t) {
                double s = W[(size_t)t * m + k + u];
                for (int q = t + 1; q < k; ++q)
                    s = fma(-W[(size_t)t * m + q], A[(size_t)q * mk + u], s);
                A[(size_t)t * mk + u] = s / W[(size_t)t * m + t];
            }
        /* X = R11^{-1}; 1/omega_t^2 = squared norm of row t of X */
        for (int c = 0; c < k; ++c)
            for (int t = k - 1; t >= 0; --t) {
                double s = (t == c) ? 1.0 : 0.0;
                for (int q = t + 1; q < k; ++q)
                    s = fma(-W[(size_t)t * m + q], X[(size_t)q * k + c], s);
                X[(size_t)t * k + c] = s / W[(size_t)t * m + t];
            }
        for (int t = 0; t < k; ++t) {
            double s = 0.0;
            for (int c = 0; c < k; ++c) {
                double x = X[(size_t)t * k + c];
                s = fma(x, x, s);
            }
            rho[t] = s;
        }
        /* gamma_u^2 = squared norm of column u of R22 */
        for (int u = 0; u < mk; ++u) {
            double s = 0.0;
            for (int i = k; i < r; ++i) {
                double x = W[(size_t)i * m + k + u];
                s = fma(x, x, s);
            }
            g2[u] = s;
        }
        double best = -1.0;
        int bt = 0, bu = 0;
        for (int t = 0; t < k; ++t)
            for (int u = 0; u < mk; ++u) {
                double a = A[(size_t)t * mk + u];
                double val = fma(a, a, g2[u] * rho[t]);
                if (val > best) { best = val; bt = t; bu = u; }
            }
        if (best <= f * f) break;
        if (nsw >= ORC_MAX_SWAPS) { nsw = -1; break; }
        int tp = perm[bt]; perm[bt] = perm[k + bu]; perm[k + bu] = tp;
        ++nsw;
        /* rebuild the permuted matrix and re-triangularise its first k columns */
        for (int i = 0; i < r; ++i)
            for (int c = 0; c < m; ++c)
                W[(size_t)i * m + c] = Mt[(size_t)i * m + perm[c]];
        orc_qr(W, r, m, perm, 0, k, tol, nrm2, v);
    }
    *k_out = k;
    *nswaps_out = nsw;
    free(W); free(nrm2); free(v); free(X); free(rho); free(g2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The H^2 representation                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int m, k, nswaps;
    int64_t *ibar;    /* m working-set point indices (sorted positions) */
    int64_t *skel;    /* k skeleton indices, ascending */
    int64_t *rest;    /* m-k others, ascending */
    int32_t *skel_loc, *rest_loc; /* their positions in ibar */
    double *G;        /* (m-k) x k, row-major: rows = rest, columns = skel */
} orc_comp;

typedef struct {
    int level, leaf, parent, child0, nchild;
    int64_t rs, rc, cs, cc;
    uint64_t cell[3];
} orc_node;

typedef struct orc_h2 {
    int d, kid, leaf, p, r, same, b;
    double tau, tol, f;
    int64_t nx, ny;
    double lo[3], s;
    double anchors[ORC_MAXP];
    int64_t *permx, *permy;
    uint64_t *keyx, *keyy;
    double *xs, *ys;
    int L;
    int64_t *lvl_off; /* nodes of level l (1-based) are gids [lvl_off[l-1], lvl_off[l]) */
    int nnodes, cap;
    orc_node *nodes;
    int64_t *adm_ptr, *near_ptr;
    int32_t *adm_col, *near_col;
    int64_t nadm, nnear;
    orc_comp *rowc, *colc;
    /* the Taylor-expansion representation of 1/(x - y) on C (Section 2.1):
     * rt terms, coefficients cl[l] = (l/e)(2 pi rt)^(1/(2 rt)) of (2.5), the
     * diagonal value d_x of (2.1); G of every node is complex, (m-k) x k
     * interleaved (re, im) */
    int cplx, rt;
    double cl[ORC_MAXP];
    double dx_re, dx_im;
    /* HSS (Section 3.3.1): the nearfield sets N_i of (A.1) in CSR by node,
     * and the number of truncated-SVD vectors s_i appended to each basis */
    int hss;
    double eps_svd;
    int64_t *nf_ptr;
    int32_t *nf_col;
    int32_t *svd_rows, *svd_cols;
} orc_h2;

/* growable pair list */
typedef struct { uint64_t *v; int64_t n, cap; } orc_pairs;

static void orc_pairs_push(orc_pairs *p, int i, int j)
{
    if (p->n == p->cap) {
        p->cap = p->cap ? 2 * p->cap : 1024;
        p->v = realloc(p->v, sizeof(uint64_t) * (size_t)p->cap);
    }
    p->v[p->n++] = ((uint64_t)(uint32_t)i << 32) | (uint32_t)j;
}

static int orc_u64_cmp(const void *pa, const void *pb)
{
    uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
    return a < b ? -1 : (a > b);
}

static int orc_new_node(orc_h2 *h)
{
    if (h->nnodes == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 256;
        h->nodes = realloc(h->nodes, sizeof(orc_node) * (size_t)h->cap);
    }
    memset(&h->nodes[h->nnodes], 0, sizeof(orc_node));
    return h->nnodes++;
}

/* digit of a key that selects the child of a level-l node */
static int orc_digit(uint64_t key, int d, int b, int l)
{
    return (int)((key >> (d * (b - l))) & ((1u << d) - 1));
}

/* Section 3.1: level-by-level bisection of every box with more than leaf
 * points (rows or columns) along all d axes; empty boxes are dropped. */
static void orc_build_tree(orc_h2 *h)
{
    int d = h->d, b = h->b;
    h->lvl_off = malloc(sizeof(int64_t) * (size_t)(b + 3));
    int root = orc_new_node(h);
    orc_node *rt = &h->nodes[root];
    rt->level = 1; rt->parent = -1; rt->child0 = -1;
    rt->rs = 0; rt->rc = h->nx; rt->cs = 0; rt->cc = h->ny;
    int64_t big = rt->rc > rt->cc ? rt->rc : rt->cc;
    rt->leaf = !(big > h->leaf && 1 <= b);
    h->lvl_off[0] = 0;
    h->lvl_off[1] = 1;
    int l = 1;
    for (;;) {
        int64_t first = h->lvl_off[l - 1], last = h->lvl_off[l];
        for (int64_t g = first; g < last; ++g) {
            if (h->nodes[g].leaf) continue;
            int64_t rcur = h->nodes[g].rs, rend = h->nodes[g].rs + h->nodes[g].rc;
            int64_t ccur = h->nodes[g].cs, cend = h->nodes[g].cs + h->nodes[g].cc;
            h->nodes[g].child0 = -1;
            h->nodes[g].nchild = 0;
            for (int dig = 0; dig < (1 << d); ++dig) {
                int64_t r0 = rcur, c0 = ccur;
                while (rcur < rend && orc_digit(h->keyx[rcur], d, b, l) == dig) ++rcur;
                while (ccur < cend && orc_digit(h->keyy[ccur], d, b, l) == dig) ++ccur;
                if (rcur - r0 + ccur - c0 == 0) continue;
                int c = orc_new_node(h);
                orc_node *nd = &h->nodes[c];
                orc_node *par = &h->nodes[g];
                nd->level = l + 1;
                nd->parent = (int)g;
                nd->child0 = -1;
                nd->rs = r0; nd->rc = rcur - r0;
                nd->cs = c0; nd->cc = ccur - c0;
                for (int a = 0; a < d; ++a)
                    nd->cell[a] = 2 * par->cell[a] + (uint64_t)((dig >> (d - 1 - a)) & 1);
                int64_t cnt = nd->rc > nd->cc ? nd->rc : nd->cc;
                nd->leaf = !(cnt > h->leaf && (l + 1) <= b);
                if (par->child0 < 0) par->child0 = c;
                par->nchild++;
            }
        }
        if (h->nnodes == last) break;
        ++l;
        h->lvl_off[l] = h->nnodes;
    }
    h->L = l;
}

/* (3.3)/(3.4) by dual traversal from (root, root). */
static void orc_visit(const orc_h2 *h, int i, int j, orc_pairs *adm, orc_pairs *near)
{
    const orc_node *a = &h->nodes[i], *b = &h->nodes[j];
    if (a->rc == 0 || b->cc == 0) return; /* empty block */
    if (orc_admissible(h->d, a->level, a->cell, b->level, b->cell, h->tau)) {
        orc_pairs_push(adm, i, j);
    } else if (a->leaf && b->leaf) {
        orc_pairs_push(near, i, j);
    } else if (!a->leaf && !b->leaf) {
        for (int ci = 0; ci < a->nchild; ++ci)
            for (int cj = 0; cj < b->nchild; ++cj)
                orc_visit(h, a->child0 + ci, b->child0 + cj, adm, near);
    } else if (a->leaf) {
        for (int cj = 0; cj < b->nchild; ++cj)
            orc_visit(h, i, b->child0 + cj, adm, near);
    } else {
        for (int ci = 0; ci < a->nchild; ++ci)
            orc_visit(h, a->child0 + ci, j, adm, near);
    }
}

static void orc_to_csr(int nnodes, orc_pairs *p, int64_t **ptr, int32_t **col)
{
    qsort(p->v, (size_t)p->n, sizeof(uint64_t), orc_u64_cmp);
    *ptr = calloc((size_t)nnodes + 1, sizeof(int64_t));
    *col = malloc(sizeof(int32_t) * (size_t)(p->n > 0 ? p->n : 1));
    for (int64_t e = 0; e < p->n; ++e) {
        (*ptr)[(p->v[e] >> 32) + 1]++;
        (*col)[e] = (int32_t)(p->v[e] & 0xffffffffu);
    }
    for (int g = 0; g < nnodes; ++g) (*ptr)[g + 1] += (*ptr)[g];
}

/* compr (3.16) on one node and one side; writes the canonical form. */
static void orc_compress_node(orc_h2 *h, int g, int side)
{
    orc_node *nd = &h->nodes[g];
    orc_comp *cp = side == 0 ? &h->rowc[g] : &h->colc[g];
    const double *pts = side == 0 ? h->xs : h->ys;
    int d = h->d, r = h->r;
    /* working set (3.6)/(3.18) */
    int m;
    if (nd->leaf) {
        m = (int)(side == 0 ? nd->rc : nd->cc);
        int64_t st = side == 0 ? nd->rs : nd->cs;
        cp->ibar = malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        for (int c = 0; c < m; ++c) cp->ibar[c] = st + c;
    } else {
        m = 0;
        for (int c = 0; c < nd->nchild; ++c)
            m += (side == 0 ? h->rowc : h->colc)[nd->child0 + c].k;
        cp->ibar = malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        int pos = 0;
        for (int c = 0; c < nd->nchild; ++c) {
            orc_comp *ch = &(side == 0 ? h->rowc : h->colc)[nd->child0 + c];
            for (int t = 0; t < ch->k; ++t) cp->ibar[pos++] = ch->skel[t];
        }
    }
    cp->m = m;
    if (m == 0) {
        cp->k = 0;
        return;
    }
    double *P = malloc(sizeof(double) * (size_t)m * (size_t)d);
    for (int c = 0; c < m; ++c)
        for (int a = 0; a < d; ++a) P[c * d + a] = pts[cp->ibar[c] * d + a];
    double *Mt = malloc(sizeof(double) * (size_t)r * (size_t)m);
    orc_basis_t(d, h->p, h->anchors, h->lo, h->s, nd->level, nd->cell, P, m, Mt);
    int *perm = malloc(sizeof(int) * (size_t)m);
    int kmax = r < m ? r : m;
    double *A = malloc(sizeof(double) * (size_t)(kmax * (m - 1) + 1));
    int k, nsw;
    orc_compr(Mt, r, m, h->tol, h->f, perm, &k, A, &nsw);
    cp->k = k;
    cp->nswaps = nsw;
    /* canonical form: skeleton and rest each in ascending position order */
    int *sel = calloc((size_t)m, sizeof(int));
    for (int t = 0; t < k; ++t) sel[perm[t]] = 1;
    int *rank = malloc(sizeof(int) * (size_t)m); /* position -> sorted index */
    int ns = 0, nr = 0;
    for (int pos = 0; pos < m; ++pos) rank[pos] = sel[pos] ? ns++ : nr++;
    cp->skel = malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    cp->rest = malloc(sizeof(int64_t) * (size_t)(m - k > 0 ? m - k : 1));
    cp->skel_loc = malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    cp->rest_loc = malloc(sizeof(int32_t) * (size_t)(m - k > 0 ? m - k : 1));
    cp->G = malloc(sizeof(double) * (size_t)((m - k) * k > 0 ? (m - k) * k : 1));
    for (int pos = 0; pos < m; ++pos) {
        if (sel[pos]) { cp->skel[rank[pos]] = cp->ibar[pos]; cp->skel_loc[rank[pos]] = pos; }
        else { cp->rest[rank[pos]] = cp->ibar[pos]; cp->rest_loc[rank[pos]] = pos; }
    }
    int mk = m - k;
    for (int t = 0; t < k; ++t)
        for (int u = 0; u < mk; ++u)
            cp->G[(size_t)rank[perm[k + u]] * k + rank[perm[t]]] = A[(size_t)t * mk + u];
    free(P); free(Mt); free(perm); free(A); free(sel); free(rank);
}

void orc_free(orc_h2 *h);
static void orc_structure(orc_h2 *h, const double *x, int64_t nx, const double *y, int64_t ny);

/* Build: returns NULL on invalid input.  y == NULL means Y = X. */
orc_h2 *orc_build(const double *x, int64_t nx, const double *y, int64_t ny, int d, int kid,
                  int leaf, int p, double tau, double tol, double f)
{
    if (d < 1 || d > 3 || nx < 1 || leaf < 1 || p < 1 || p > ORC_MAXP || !(tol > 0.0) ||
        !(tau > 0.0 && tau < 1.0) || !(f > 1.0))
        return NULL;
    if (kid < 0 || kid > 5 || (kid == ORC_K_CAUCHY && d != 1) || ((kid == ORC_K_DLP1 || kid == ORC_K_DLP2) && d != 2))
        return NULL;
    if (y && ny < 1) return NULL;
    for (int64_t i = 0; i < nx * d; ++i) if (!isfinite(x[i])) return NULL;
    if (y) for (int64_t i = 0; i < ny * d; ++i) if (!isfinite(y[i])) return NULL;
    orc_h2 *h = calloc(1, sizeof(orc_h2));
    h->d = d; h->kid = kid; h->leaf = leaf; h->p = p; h->tau = tau; h->tol = tol; h->f = f;
    h->r = 1;
    for (int a = 0; a < d; ++a) h->r *= p;
    orc_chebyshev(p, h->anchors);
    orc_structure(h, x, nx, y, ny);
    h->rowc = calloc((size_t)h->nnodes, sizeof(orc_comp));
    h->colc = h->same ? h->rowc : calloc((size_t)h->nnodes, sizeof(orc_comp));
    /* (3.16)-(3.18): levels L..2, bottom-up */
    for (int l = h->L; l >= 2; --l) {
        #pragma omp parallel for schedule(dynamic)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) {
            orc_compress_node(h, (int)g, 0);
            if (!h->same) orc_compress_node(h, (int)g, 1);
        }
    }
    return h;
}

/* Sections 3.1 and 3.2: bounding cube, sorted points, the adaptive tree and
 * the lists L (3.3) and L^- (3.4), for h->d, h->leaf and h->tau. */
static void orc_structure(orc_h2 *h, const double *x, int64_t nx, const double *y, int64_t ny)
{
    int d = h->d;
    h->same = (y == NULL);
    h->nx = nx; h->ny = y ? ny : nx;
    h->b = orc_bits_per_dim(d);
    orc_bounding_cube(x, nx, y, ny, d, h->lo, &h->s);
    h->permx = malloc(sizeof(int64_t) * (size_t)nx);
    h->keyx = malloc(sizeof(uint64_t) * (size_t)nx);
    h->xs = malloc(sizeof(double) * (size_t)nx * d);
    orc_sort_points(x, nx, d, h->lo, h->s, h->permx, h->keyx, h->xs);
    if (h->same) {
        h->permy = h->permx; h->keyy = h->keyx; h->ys = h->xs;
    } else {
        h->permy = malloc(sizeof(int64_t) * (size_t)ny);
        h->keyy = malloc(sizeof(uint64_t) * (size_t)ny);
        h->ys = malloc(sizeof(double) * (size_t)ny * d);
        orc_sort_points(y, ny, d, h->lo, h->s, h->permy, h->keyy, h->ys);
    }
    orc_build_tree(h);
    orc_pairs adm = {0}, near = {0};
    orc_visit(h, 0, 0, &adm, &near);
    h->nadm = adm.n; h->nnear = near.n;
    orc_to_csr(h->nnodes, &adm, &h->adm_ptr, &h->adm_col);
    orc_to_csr(h->nnodes, &near, &h->near_ptr, &h->near_col);
    free(adm.v); free(near.v);
}

static void orc_free_comp(orc_comp *c, int n)
{
    if (!c) return;
    for (int g = 0; g < n; ++g) {
        free(c[g].ibar); free(c[g].skel); free(c[g].rest);
        free(c[g].skel_loc); free(c[g].rest_loc); free(c[g].G);
    }
    free(c);
}

void orc_free(orc_h2 *h)
{
    if (!h) return;
    free(h->nf_ptr); free(h->nf_col);
    if (h->svd_cols != h->svd_rows) free(h->svd_cols);
    free(h->svd_rows);
    if (!h->same) { free(h->permy); free(h->keyy); free(h->ys); orc_free_comp(h->colc, h->nnodes); }
    free(h->permx); free(h->keyx); free(h->xs);
    orc_free_comp(h->rowc, h->nnodes);
    free(h->lvl_off); free(h->nodes);
    free(h->adm_ptr); free(h->adm_col); free(h->near_ptr); free(h->near_col);
    free(h);
}

/* ------------------------------------------------------------------------ */
/* Section 3.4: node-wise H^2 matvec, z = A^ q (q: ny x nrhs, z: nx x nrhs)   */
/* ------------------------------------------------------------------------ */

/* need == NULL: every node.  Otherwise only the nodes flagged in need get
 * their coupling, downward and near-field work, and only the rows of the
 * flagged leaves of z are written (the upward pass is always complete).
 * absval != 0: the same passes with every factor replaced by its magnitude
 * (|q|, |G|, |kappa|), so that each output is the sum of the magnitudes of
 * the terms the plain matvec adds up for it, step by step.  A sum of terms
 * t_1..t_n computed in floating point differs from the exact sum by at most
 * a small multiple of the unit roundoff times sum |t_i|; this is that scale
 * for every row of A^ q. */
#define ORC_ABS(v) (absval ? fabs(v) : (v))
static int orc_matvec_masked(const orc_h2 *h, const double *q, double *z, int nrhs, const unsigned char *need,
                             int absval)
{
    int d = h->d;
    int64_t nx = h->nx, ny = h->ny;
    double *qs = malloc(sizeof(double) * (size_t)ny * nrhs);
    double *zs = calloc((size_t)nx * nrhs, sizeof(double));
    for (int64_t pnt = 0; pnt < ny; ++pnt)
        for (int c = 0; c < nrhs; ++c) qs[pnt * nrhs + c] = ORC_ABS(q[h->permy[pnt] * nrhs + c]);
    double **qhat = calloc((size_t)h->nnodes, sizeof(double *));
    double **zhat = calloc((size_t)h->nnodes, sizeof(double *));
    /* step 1: upward pass, q^_i = V_i^T q|_i at leaves, sum_c W_c^T q^_c above */
    for (int l = h->L; l >= 2; --l) {
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) {
            const orc_node *nd = &h->nodes[g];
            const orc_comp *cp = &h->colc[g];
            int m = cp->m, k = cp->k;
            double *in = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1) * nrhs);
            if (nd->leaf) {
                memcpy(in, qs + nd->cs * nrhs, sizeof(double) * (size_t)m * nrhs);
            } else {
                int pos = 0;
                for (int c = 0; c < nd->nchild; ++c) {
                    int kc = h->colc[nd->child0 + c].k;
                    memcpy(in + (size_t)pos * nrhs, qhat[nd->child0 + c], sizeof(double) * (size_t)kc * nrhs);
                    pos += kc;
                }
            }
            qhat[g] = calloc((size_t)(k > 0 ? k : 1) * nrhs, sizeof(double));
            for (int t = 0; t < k; ++t)
                for (int c = 0; c < nrhs; ++c) {
                    double s = in[(size_t)cp->skel_loc[t] * nrhs + c];
                    for (int u = 0; u < m - k; ++u)
                        s = s + ORC_ABS(cp->G[(size_t)u * k + t]) * in[(size_t)cp->rest_loc[u] * nrhs + c];
                    qhat[g][(size_t)t * nrhs + c] = s;
                }
            free(in);
        }
    }
    /* step 2: coupling, z^_i = sum_{(i,j) in L} A|_{i^ x j^} q^_j  (3.19) */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int g = 0; g < h->nnodes; ++g) {
        const orc_comp *ci = &h->rowc[g];
        zhat[g] = calloc((size_t)(ci->k > 0 ? ci->k : 1) * nrhs, sizeof(double));
        if (need && !need[g]) continue;
        for (int64_t e = h->adm_ptr[g]; e < h->adm_ptr[g + 1]; ++e) {
            int j = h->adm_col[e];
            const orc_comp *cj = &h->colc[j];
            for (int a = 0; a < ci->k; ++a) {
                const double *xa = h->xs + ci->skel[a] * d;
                for (int bb = 0; bb < cj->k; ++bb) {
                    double kv = ORC_ABS(orc_kernel(h->kid, d, xa, h->ys + cj->skel[bb] * d));
                    for (int c = 0; c < nrhs; ++c)
                        zhat[g][(size_t)a * nrhs + c] += kv * qhat[j][(size_t)bb * nrhs + c];
                }
            }
        }
    }
    /* step 3: downward pass, z^_c += R_c z^_i, and z|_i = U_i z^_i at leaves */
    for (int l = 2; l <= h->L; ++l) {
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) {
            if (need && !need[g]) continue;
            const orc_node *nd = &h->nodes[g];
            const orc_comp *cp = &h->rowc[g];
            int m = cp->m, k = cp->k;
            double *out = calloc((size_t)(m > 0 ? m : 1) * nrhs, sizeof(double));
            for (int t = 0; t < k; ++t)
                for (int c = 0; c < nrhs; ++c)
                    out[(size_t)cp->skel_loc[t] * nrhs + c] = zhat[g][(size_t)t * nrhs + c];
            for (int u = 0; u < m - k; ++u)
                for (int c = 0; c < nrhs; ++c) {
                    double s = 0.0;
                    for (int t = 0; t < k; ++t)
                        s = s + ORC_ABS(cp->G[(size_t)u * k + t]) * zhat[g][(size_t)t * nrhs + c];
                    out[(size_t)cp->rest_loc[u] * nrhs + c] = s;
                }
            if (nd->leaf) {
                for (int64_t a = 0; a < (int64_t)m * nrhs; ++a) zs[nd->rs * nrhs + a] += out[a];
            } else {
                int pos = 0;
                for (int c = 0; c < nd->nchild; ++c) {
                    int kc = h->rowc[nd->child0 + c].k;
                    for (int64_t a = 0; a < (int64_t)kc * nrhs; ++a)
                        zhat[nd->child0 + c][a] += out[(size_t)pos * nrhs + a];
                    pos += kc;
                }
            }
            free(out);
        }
    }
    /* near field (3.20): z|_i += A|_{i x j} q|_j for (i,j) in L^- */
    #pragma omp parallel for schedule(dynamic, 16)
    for (int g = 0; g < h->nnodes; ++g) {
        if (need && !need[g]) continue;
        const orc_node *ni = &h->nodes[g];
        for (int64_t e = h->near_ptr[g]; e < h->near_ptr[g + 1]; ++e) {
            const orc_node *nj = &h->nodes[h->near_col[e]];
            for (int64_t a = ni->rs; a < ni->rs + ni->rc; ++a)
                for (int64_t bb = nj->cs; bb < nj->cs + nj->cc; ++bb) {
                    double kv = ORC_ABS(orc_kernel(h->kid, d, h->xs + a * d, h->ys + bb * d));
                    for (int c = 0; c < nrhs; ++c) zs[a * nrhs + c] += kv * qs[bb * nrhs + c];
                }
        }
    }
    if (!need) {
        for (int64_t pnt = 0; pnt < nx; ++pnt)
            for (int c = 0; c < nrhs; ++c) z[h->permx[pnt] * nrhs + c] = zs[pnt * nrhs + c];
    } else {
        for (int g = 0; g < h->nnodes; ++g) {
            if (!need[g] || !h->nodes[g].leaf) continue;
            for (int64_t pnt = h->nodes[g].rs; pnt < h->nodes[g].rs + h->nodes[g].rc; ++pnt)
                for (int c = 0; c < nrhs; ++c) z[h->permx[pnt] * nrhs + c] = zs[pnt * nrhs + c];
        }
    }
    for (int g = 0; g < h->nnodes; ++g) { free(qhat[g]); free(zhat[g]); }
    free(qhat); free(zhat); free(qs); free(zs);
    return 0;
}

#undef ORC_ABS

int orc_matvec(const orc_h2 *h, const double *q, double *z, int nrhs)
{
    return orc_matvec_masked(h, q, z, nrhs, NULL, 0);
}

/* Rows of A^ q for the points of the given leaves only (gids), computed
 * exactly as orc_matvec computes them: the full upward pass, then coupling,
 * downward and near-field work on the leaves and their ancestors.  Rows of
 * other points in z are left untouched. */
int orc_matvec_leaves(const orc_h2 *h, const double *q, double *z, int nrhs, const int32_t *leaves,
                      int64_t nleaves)
{
    unsigned char *need = calloc((size_t)h->nnodes, 1);
    for (int64_t t = 0; t < nleaves; ++t) {
        int g = leaves[t];
        if (g < 0 || g >= h->nnodes || !h->nodes[g].leaf) { free(need); return -1; }
        while (g >= 0) { need[g] = 1; g = h->nodes[g].parent; }
    }
    int st = orc_matvec_masked(h, q, z, nrhs, need, 0);
    free(need);
    return st;
}

/* Row scales of A^ q: the matvec above with every factor replaced by its
 * magnitude (see orc_matvec_masked).  leaves == NULL: every row; otherwise
 * only the rows of the given leaves are written. */
int orc_matvec_abs(const orc_h2 *h, const double *q, double *z, int nrhs, const int32_t *leaves,
                   int64_t nleaves)
{
    if (!leaves) return orc_matvec_masked(h, q, z, nrhs, NULL, 1);
    unsigned char *need = calloc((size_t)h->nnodes, 1);
    for (int64_t t = 0; t < nleaves; ++t) {
        int g = leaves[t];
        if (g < 0 || g >= h->nnodes || !h->nodes[g].leaf) { free(need); return -1; }
        while (g >= 0) { need[g] = 1; g = h->nodes[g].parent; }
    }
    int st = orc_matvec_masked(h, q, z, nrhs, need, 1);
    free(need);
    return st;
}

/* ------------------------------------------------------------------------ */
/* introspection                                                             */
/* ------------------------------------------------------------------------ */

enum {
    ORC_Q_NX = 0, ORC_Q_NY, ORC_Q_L, ORC_Q_NNODES, ORC_Q_NADM, ORC_Q_NNEAR, ORC_Q_SAME,
    ORC_Q_SKEL_ROW, ORC_Q_REST_ROW, ORC_Q_G_ROW, ORC_Q_SKEL_COL, ORC_Q_REST_COL, ORC_Q_G_COL,
    ORC_Q_R, ORC_Q_SWAPS_ROW, ORC_Q_SWAPS_COL, ORC_Q_BADSWAP, ORC_Q_NNF
};

static void orc_comp_totals(const orc_comp *c, int n, int64_t *ts, int64_t *tr, int64_t *tg,
                            int64_t *sw, int64_t *bad)
{
    *ts = *tr = *tg = *sw = *bad = 0;
    for (int g = 0; g < n; ++g) {
        *ts += c[g].k;
        *tr += c[g].m - c[g].k;
        *tg += (int64_t)(c[g].m - c[g].k) * c[g].k;
        if (c[g].nswaps > 0) *sw += c[g].nswaps;
        if (c[g].nswaps < 0) *bad += 1;
    }
}

int64_t orc_query(const orc_h2 *h, int what)
{
    int64_t ts, tr, tg, sw, bad;
    switch (what) {
    case ORC_Q_NX: return h->nx;
    case ORC_Q_NY: return h->ny;
    case ORC_Q_L: return h->L;
    case ORC_Q_NNODES: return h->nnodes;
    case ORC_Q_NADM: return h->nadm;
    case ORC_Q_NNEAR: return h->nnear;
    case ORC_Q_SAME: return h->same;
    case ORC_Q_R: return h->r;
    default: break;
    }
    int col = (what == ORC_Q_SKEL_COL || what == ORC_Q_REST_COL || what == ORC_Q_G_COL ||
               what == ORC_Q_SWAPS_COL);
    orc_comp_totals(col ? h->colc : h->rowc, h->nnodes, &ts, &tr, &tg, &sw, &bad);
    switch (what) {
    case ORC_Q_SKEL_ROW: case ORC_Q_SKEL_COL: return ts;
    case ORC_Q_REST_ROW: case ORC_Q_REST_COL: return tr;
    case ORC_Q_G_ROW: case ORC_Q_G_COL: return tg;
    case ORC_Q_SWAPS_ROW: case ORC_Q_SWAPS_COL: return sw;
    case ORC_Q_BADSWAP: return bad;
    case ORC_Q_NNF: return h->nf_ptr ? h->nf_ptr[h->nnodes] : 0;
    default: return -1;
    }
}

void orc_export_geometry(const orc_h2 *h, double *lo, double *s, int64_t *permx, int64_t *permy,
                         uint64_t *keyx, uint64_t *keyy)
{
    for (int a = 0; a < h->d; ++a) lo[a] = h->lo[a];
    *s = h->s;
    memcpy(permx, h->permx, sizeof(int64_t) * (size_t)h->nx);
    memcpy(permy, h->permy, sizeof(int64_t) * (size_t)h->ny);
    memcpy(keyx, h->keyx, sizeof(uint64_t) * (size_t)h->nx);
    memcpy(keyy, h->keyy, sizeof(uint64_t) * (size_t)h->ny);
}

void orc_export_nodes(const orc_h2 *h, int64_t *lvl_off, int32_t *level, int32_t *leaf,
                      int32_t *parent, int32_t *child0, int32_t *nchild, int64_t *rs, int64_t *rc,
                      int64_t *cs, int64_t *cc, uint64_t *cell)
{
    for (int l = 0; l <= h->L; ++l) lvl_off[l] = h->lvl_off[l];
    for (int g = 0; g < h->nnodes; ++g) {
        const orc_node *n = &h->nodes[g];
        level[g] = n->level; leaf[g] = n->leaf; parent[g] = n->parent;
        child0[g] = n->leaf ? -1 : n->child0; nchild[g] = n->leaf ? 0 : n->nchild;
        rs[g] = n->rs; rc[g] = n->rc; cs[g] = n->cs; cc[g] = n->cc;
        for (int a = 0; a < 3; ++a) cell[g * 3 + a] = a < h->d ? n->cell[a] : 0;
    }
}

void orc_export_lists(const orc_h2 *h, int64_t *adm_ptr, int32_t *adm_col, int64_t *near_ptr,
                      int32_t *near_col)
{
    memcpy(adm_ptr, h->adm_ptr, sizeof(int64_t) * (size_t)(h->nnodes + 1));
    memcpy(near_ptr, h->near_ptr, sizeof(int64_t) * (size_t)(h->nnodes + 1));
    memcpy(adm_col, h->adm_col, sizeof(int32_t) * (size_t)h->nadm);
    memcpy(near_col, h->near_col, sizeof(int32_t) * (size_t)h->nnear);
}

/* Per node in gid order: m, k, and concatenated skeleton, rest, G. */
void orc_export_comp(const orc_h2 *h, int side, int32_t *m, int32_t *k, int64_t *skel,
                     int64_t *rest, double *G)
{
    const orc_comp *c = side == 0 ? h->rowc : h->colc;
    int64_t ps = 0, pr = 0, pg = 0;
    for (int g = 0; g < h->nnodes; ++g) {
        m[g] = c[g].m; k[g] = c[g].k;
        int mk = c[g].m - c[g].k;
        for (int t = 0; t < c[g].k; ++t) skel[ps++] = c[g].skel[t];
        for (int u = 0; u < mk; ++u) rest[pr++] = c[g].rest[u];
        for (int64_t e = 0; e < (int64_t)mk * c[g].k; ++e) G[pg++] = c[g].G[e];
    }
}

/* ------------------------------------------------------------------------ */
/* Section 2.1: the Taylor expansion (2.4)-(2.5) of 1/(x - y) on C, and the  */
/* H^2 construction (3.16)-(3.20) and matvec (Section 3.4) built on it       */
/* ------------------------------------------------------------------------ */
/* Points are complex numbers x = x_0 + i x_1 (d = 2).  Complex values are
 * pairs of doubles and every operation is written out in real arithmetic, so
 * the order of the roundings is the one written here. */

typedef struct { double re, im; } orc_cx;

static orc_cx cx_mul(orc_cx a, orc_cx b)
{
    orc_cx c = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return c;
}

/* a * conj(b) */
static orc_cx cx_mulc(orc_cx a, orc_cx b)
{
    orc_cx c = {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
    return c;
}

static orc_cx cx_div(orc_cx a, orc_cx b)
{
    double den = b.re * b.re + b.im * b.im;
    orc_cx c = {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
    return c;
}

static double cx_abs2(orc_cx a) { return fma(a.re, a.re, a.im * a.im); }

/* kappa of (2.1): 1/(x - y) for x != y, d_x where the points coincide */
static orc_cx orc_cauchy_c(const double *x, const double *y, double dx_re, double dx_im)
{
    orc_cx t = {x[0] - y[0], x[1] - y[1]};
    if (t.re == 0.0 && t.im == 0.0) {
        orc_cx dv = {dx_re, dx_im};
        return dv;
    }
    double den = t.re * t.re + t.im * t.im;
    orc_cx v = {t.re / den, -t.im / den};
    return v;
}

double orc_cauchy_c_entry(const double *x, const double *y, double dx_re, double dx_im, double *out_im)
{
    orc_cx v = orc_cauchy_c(x, y, dx_re, dx_im);
    *out_im = v.im;
    return v.re;
}

/* The factors of (2.5) that do not depend on the node:
 * cl[l] = (l/e) (2 pi r)^(1/(2r)), so that eta_{v,l} = (cl[l] / delta_v)^l. */
void orc_taylor_coefficients(int r, double *cl)
{
    double rho = pow(2.0 * ORC_PI * (double)r, 1.0 / (2.0 * (double)r));
    for (int l = 0; l < r; ++l) cl[l] = ((double)l / exp(1.0)) * rho;
}

/* phi_{a,l}(x - a) = eta_{a,l} (x - a)^l / l!  of (2.5), l = 0..r-1, at npts
 * points (pts: npts x 2), as the rows of Mt (r x npts complex, interleaved):
 * with u = (x - a)/delta and w = cl[l] u, phi_l = w^l / l!, formed as l
 * steps v <- (v w) / j. */
void orc_taylor_basis_t(int r, const double *cl, double a_re, double a_im, double delta, const double *pts,
                        int npts, double *Mt)
{
    for (int c = 0; c < npts; ++c) {
        orc_cx u = {(pts[2 * c] - a_re) / delta, (pts[2 * c + 1] - a_im) / delta};
        for (int l = 0; l < r; ++l) {
            orc_cx w = {cl[l] * u.re, cl[l] * u.im};
            orc_cx v = {1.0, 0.0};
            for (int j = 1; j <= l; ++j) {
                v = cx_mul(v, w);
                v.re = v.re / (double)j;
                v.im = v.im / (double)j;
            }
            Mt[2 * ((size_t)l * npts + c)] = v.re;
            Mt[2 * ((size_t)l * npts + c) + 1] = v.im;
        }
    }
}

/* Complex Householder step on column j of W (r x m complex, row-major),
 * in the convention of LAPACK's elementary reflectors: H = I - tau v v^H
 * with v_j = 1 and real beta, H^H [alpha; x] = [beta; 0],
 * beta = -sign(Re alpha) sqrt(|alpha|^2 + |x|^2), tau = (beta - alpha)/beta,
 * v = x / (alpha - beta); H^H is applied to the columns j+1..m-1. */
static void orc_householder_c(orc_cx *W, int r, int m, int j, orc_cx *v)
{
    orc_cx alpha = W[(size_t)j * m + j];
    double sigma = 0.0;
    for (int i = j + 1; i < r; ++i) {
        orc_cx x = W[(size_t)i * m + j];
        sigma = fma(x.re, x.re, sigma);
        sigma = fma(x.im, x.im, sigma);
    }
    if (sigma == 0.0 && alpha.im == 0.0)
        return; /* already triangular with a real diagonal entry: H = I */
    double nrm = sqrt(fma(alpha.re, alpha.re, fma(alpha.im, alpha.im, sigma)));
    double beta = alpha.re <= 0.0 ? nrm : -nrm;
    orc_cx tau = {(beta - alpha.re) / beta, -alpha.im / beta};
    orc_cx den = {alpha.re - beta, alpha.im};
    v[j].re = 1.0; v[j].im = 0.0;
    for (int i = j + 1; i < r; ++i) v[i] = cx_div(W[(size_t)i * m + j], den);
    for (int c = j + 1; c < m; ++c) {
        /* w = v^H W[:, c] */
        orc_cx w = W[(size_t)j * m + c];
        for (int i = j + 1; i < r; ++i) {
            orc_cx x = W[(size_t)i * m + c];
            w.re = fma(v[i].re, x.re, fma(v[i].im, x.im, w.re));
            w.im = fma(v[i].re, x.im, fma(-v[i].im, x.re, w.im));
        }
        /* W[:, c] -= conj(tau) w v */
        orc_cx tw = cx_mulc(w, tau);
        W[(size_t)j * m + c].re = W[(size_t)j * m + c].re - tw.re;
        W[(size_t)j * m + c].im = W[(size_t)j * m + c].im - tw.im;
        for (int i = j + 1; i < r; ++i) {
            orc_cx y = cx_mul(tw, v[i]);
            W[(size_t)i * m + c].re = W[(size_t)i * m + c].re - y.re;
            W[(size_t)i * m + c].im = W[(size_t)i * m + c].im - y.im;
        }
    }
    W[(size_t)j * m + j].re = beta;
    W[(size_t)j * m + j].im = 0.0;
    for (int i = j + 1; i < r; ++i) { W[(size_t)i * m + j].re = 0.0; W[(size_t)i * m + j].im = 0.0; }
}

/* Complex counterpart of orc_qr: pivot on the largest remaining column norm
 * (ties: lowest position), rank cut |R_jj| <= tol |R_00|. */
static int orc_qr_c(orc_cx *W, int r, int m, int *perm, int pivot, int ksteps, double tol, double *nrm2,
                    orc_cx *v)
{
    int kmax = pivot ? (r < m ? r : m) : ksteps;
    double r00 = 0.0;
    for (int j = 0; j < kmax; ++j) {
        if (pivot) {
            for (int c = j; c < m; ++c) {
                double s2 = 0.0;
                for (int i = j; i < r; ++i) {
                    orc_cx x = W[(size_t)i * m + c];
                    s2 = fma(x.re, x.re, s2);
                    s2 = fma(x.im, x.im, s2);
                }
                nrm2[c] = s2;
            }
            int piv = j;
            for (int c = j + 1; c < m; ++c)
                if (nrm2[c] > nrm2[piv]) piv = c;
            double nrm = sqrt(nrm2[piv]);
            if (j == 0) {
                r00 = nrm;
                if (nrm == 0.0) return 0;
            } else if (nrm <= tol * r00) {
                return j;
            }
            if (piv != j) {
                for (int i = 0; i < r; ++i) {
                    orc_cx t = W[(size_t)i * m + j];
                    W[(size_t)i * m + j] = W[(size_t)i * m + piv];
                    W[(size_t)i * m + piv] = t;
                }
                int tp = perm[j]; perm[j] = perm[piv]; perm[piv] = tp;
            }
        }
        orc_householder_c(W, r, m, j, v);
    }
    return kmax;
}

/* compr (2.14) on a complex Mt (r x m, interleaved): Theorem 2.4 with the
 * same steps as orc_compr; A = R11^{-1} R12 (k x (m-k), interleaved). */
int orc_compr_c(const double *Mt_in, int r, int m, double tol, double f, int *perm, int *k_out, double *A_out,
                int *nswaps_out)
{
    const orc_cx *Mt = (const orc_cx *)Mt_in;
    orc_cx *A = (orc_cx *)A_out;
    orc_cx *W = malloc(sizeof(orc_cx) * (size_t)r * (size_t)(m > 0 ? m : 1));
    double *nrm2 = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    orc_cx *v = malloc(sizeof(orc_cx) * (size_t)(r > 0 ? r : 1));
    for (int c = 0; c < m; ++c) perm[c] = c;
    memcpy(W, Mt, sizeof(orc_cx) * (size_t)r * (size_t)m);
    int k = orc_qr_c(W, r, m, perm, 1, 0, tol, nrm2, v);
    int nsw = 0;
    int mk = m - k;
    orc_cx *X = malloc(sizeof(orc_cx) * (size_t)(k > 0 ? k * k : 1));
    double *rho = malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    double *g2 = malloc(sizeof(double) * (size_t)(mk > 0 ? mk : 1));
    for (;;) {
        if (k == 0 || mk == 0) break;
        /* A = R11^{-1} R12 by back substitution, one column at a time */
        for (int u = 0; u < mk; ++u)
            for (int t = k - 1; t >= 0; --t) {
                orc_cx s = W[(size_t)t * m + k + u];
                for (int q = t + 1; q < k; ++q) {
                    orc_cx y = cx_mul(W[(size_t)t * m + q], A[(size_t)q * mk + u]);
                    s.re = s.re - y.re;
                    s.im = s.im - y.im;
                }
                A[(size_t)t * mk + u] = cx_div(s, W[(size_t)t * m + t]);
            }
        /* X = R11^{-1}; 1/omega_t^2 = squared norm of row t of X */
        for (int c = 0; c < k; ++c)
            for (int t = k - 1; t >= 0; --t) {
                orc_cx s = {(t == c) ? 1.0 : 0.0, 0.0};
                for (int q = t + 1; q < k; ++q) {
                    orc_cx y = cx_mul(W[(size_t)t * m + q], X[(size_t)q * k + c]);
                    s.re = s.re - y.re;
                    s.im = s.im - y.im;
                }
                X[(size_t)t * k + c] = cx_div(s, W[(size_t)t * m + t]);
            }
        for (int t = 0; t < k; ++t) {
            double s = 0.0;
            for (int c = 0; c < k; ++c) {
                s = fma(X[(size_t)t * k + c].re, X[(size_t)t * k + c].re, s);
                s = fma(X[(size_t)t * k + c].im, X[(size_t)t * k + c].im, s);
            }
            rho[t] = s;
        }
        /* gamma_u^2 = squared norm of column u of R22 */
        for (int u = 0; u < mk; ++u) {
            double s = 0.0;
            for (int i = k; i < r; ++i) {
                s = fma(W[(size_t)i * m + k + u].re, W[(size_t)i * m + k + u].re, s);
                s = fma(W[(size_t)i * m + k + u].im, W[(size_t)i * m + k + u].im, s);
            }
            g2[u] = s;
        }
        double best = -1.0;
        int bt = 0, bu = 0;
        for (int t = 0; t < k; ++t)
            for (int u = 0; u < mk; ++u) {
                orc_cx a = A[(size_t)t * mk + u];
                double val = fma(a.re, a.re, fma(a.im, a.im, g2[u] * rho[t]));
                if (val > best) { best = val; bt = t; bu = u; }
            }
        if (best <= f * f) break;
        if (nsw >= ORC_MAX_SWAPS) { nsw = -1; break; }
        int tp = perm[bt]; perm[bt] = perm[k + bu]; perm[k + bu] = tp;
        ++nsw;
        for (int i = 0; i < r; ++i)
            for (int c = 0; c < m; ++c)
                W[(size_t)i * m + c] = Mt[(size_t)i * m + perm[c]];
        orc_qr_c(W, r, m, perm, 0, k, tol, nrm2, v);
    }
    *k_out = k;
    *nswaps_out = nsw;
    free(W); free(nrm2); free(v); free(X); free(rho); free(g2);
    return 0;
}

/* (3.16)-(3.18) for one node with the Taylor basis of its cell: centre a =
 * the cell centre, radius delta = half the cell diagonal (Definition 2.1 on
 * the cell, as (4.6) does). */
static void orc_compress_node_c(orc_h2 *h, int g)
{
    orc_node *nd = &h->nodes[g];
    orc_comp *cp = &h->rowc[g];
    int r = h->rt;
    int m;
    if (nd->leaf) {
        m = (int)nd->rc;
        cp->ibar = malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        for (int c = 0; c < m; ++c) cp->ibar[c] = nd->rs + c;
    } else {
        m = 0;
        for (int c = 0; c < nd->nchild; ++c) m += h->rowc[nd->child0 + c].k;
        cp->ibar = malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        int pos = 0;
        for (int c = 0; c < nd->nchild; ++c) {
            orc_comp *ch = &h->rowc[nd->child0 + c];
            for (int t = 0; t < ch->k; ++t) cp->ibar[pos++] = ch->skel[t];
        }
    }
    cp->m = m;
    if (m == 0) { cp->k = 0; return; }
    double hc = ldexp(h->s, 1 - nd->level);
    double a_re = h->lo[0] + ((double)nd->cell[0] + 0.5) * hc;
    double a_im = h->lo[1] + ((double)nd->cell[1] + 0.5) * hc;
    double delta = 0.5 * hc * sqrt(2.0);
    double *P = malloc(sizeof(double) * (size_t)m * 2);
    for (int c = 0; c < m; ++c) { P[2 * c] = h->xs[cp->ibar[c] * 2]; P[2 * c + 1] = h->xs[cp->ibar[c] * 2 + 1]; }
    double *Mt = malloc(sizeof(double) * 2 * (size_t)r * (size_t)m);
    orc_taylor_basis_t(r, h->cl, a_re, a_im, delta, P, m, Mt);
    int *perm = malloc(sizeof(int) * (size_t)m);
    int kmax = r < m ? r : m;
    double *A = malloc(sizeof(double) * 2 * (size_t)(kmax * (m - 1) + 1));
    int k, nsw;
    orc_compr_c(Mt, r, m, h->tol, h->f, perm, &k, A, &nsw);
    cp->k = k;
    cp->nswaps = nsw;
    int *sel = calloc((size_t)m, sizeof(int));
    for (int t = 0; t < k; ++t) sel[perm[t]] = 1;
    int *rank = malloc(sizeof(int) * (size_t)m);
    int ns = 0, nr = 0;
    for (int pos = 0; pos < m; ++pos) rank[pos] = sel[pos] ? ns++ : nr++;
    cp->skel = malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    cp->rest = malloc(sizeof(int64_t) * (size_t)(m - k > 0 ? m - k : 1));
    cp->skel_loc = malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    cp->rest_loc = malloc(sizeof(int32_t) * (size_t)(m - k > 0 ? m - k : 1));
    cp->G = malloc(sizeof(double) * 2 * (size_t)((m - k) * k > 0 ? (m - k) * k : 1));
    for (int pos = 0; pos < m; ++pos) {
        if (sel[pos]) { cp->skel[rank[pos]] = cp->ibar[pos]; cp->skel_loc[rank[pos]] = pos; }
        else { cp->rest[rank[pos]] = cp->ibar[pos]; cp->rest_loc[rank[pos]] = pos; }
    }
    int mk = m - k;
    for (int t = 0; t < k; ++t)
        for (int u = 0; u < mk; ++u) {
            size_t dst = (size_t)rank[perm[k + u]] * k + rank[perm[t]];
            cp->G[2 * dst] = A[2 * ((size_t)t * mk + u)];
            cp->G[2 * dst + 1] = A[2 * ((size_t)t * mk + u) + 1];
        }
    free(P); free(Mt); free(perm); free(A); free(sel); free(rank);
}

/* H^2 approximation of A = [kappa(x_i, x_j)] with kappa of (2.1) on C (X = Y,
 * points n x 2 read as x_0 + i x_1), bases from the Taylor expansion (2.4)
 * with r terms, separation ratio tau, rank cut tol, SRRQR bound f.  Returns
 * NULL on invalid input. */
orc_h2 *orc_build_taylor(const double *x, int64_t n, int leaf, int r, double tau, double tol, double f,
                         double dx_re, double dx_im)
{
    if (n < 1 || leaf < 1 || r < 1 || r > ORC_MAXP || !(tol > 0.0) || !(tau > 0.0 && tau < 1.0) || !(f > 1.0))
        return NULL;
    for (int64_t i = 0; i < n * 2; ++i) if (!isfinite(x[i])) return NULL;
    orc_h2 *h = calloc(1, sizeof(orc_h2));
    h->d = 2; h->kid = -1; h->leaf = leaf; h->p = 0; h->r = r; h->tau = tau; h->tol = tol; h->f = f;
    h->cplx = 1; h->rt = r; h->dx_re = dx_re; h->dx_im = dx_im;
    orc_taylor_coefficients(r, h->cl);
    orc_structure(h, x, n, NULL, 0);
    h->rowc = calloc((size_t)h->nnodes, sizeof(orc_comp));
    h->colc = h->rowc;
    for (int l = h->L; l >= 2; --l) {
        #pragma omp parallel for schedule(dynamic)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) orc_compress_node_c(h, (int)g);
    }
    return h;
}

/* Section 3.4 on the complex representation: z = A^ q with q, z n x nrhs
 * complex (interleaved), in the caller's order.  Steps as in
 * orc_matvec_masked (upward with [I G^T] P^T, coupling (3.19), downward,
 * near field (3.20) with kappa(x, x) = d_x); absval != 0 replaces every factor
 * by its magnitude and writes real row scales to z (n x nrhs doubles). */
int orc_matvec_taylor(const orc_h2 *h, const double *q_in, double *z_out, int nrhs, int absval)
{
    if (!h->cplx) return -1;
    int64_t n = h->nx;
    const orc_cx *q = (const orc_cx *)q_in;
    orc_cx *qs = malloc(sizeof(orc_cx) * (size_t)n * nrhs);
    orc_cx *zs = calloc((size_t)n * nrhs, sizeof(orc_cx));
    for (int64_t pnt = 0; pnt < n; ++pnt)
        for (int c = 0; c < nrhs; ++c) {
            orc_cx v = q[h->permx[pnt] * nrhs + c];
            if (absval) { v.re = sqrt(cx_abs2(v)); v.im = 0.0; }
            qs[pnt * nrhs + c] = v;
        }
    orc_cx **qhat = calloc((size_t)h->nnodes, sizeof(orc_cx *));
    orc_cx **zhat = calloc((size_t)h->nnodes, sizeof(orc_cx *));
#define ORC_GC(cp, idx) (absval ? (orc_cx){sqrt(cx_abs2(((const orc_cx *)(cp)->G)[idx])), 0.0} \
                                : ((const orc_cx *)(cp)->G)[idx])
    for (int l = h->L; l >= 2; --l) {
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) {
            const orc_node *nd = &h->nodes[g];
            const orc_comp *cp = &h->rowc[g];
            int m = cp->m, k = cp->k;
            orc_cx *in = malloc(sizeof(orc_cx) * (size_t)(m > 0 ? m : 1) * nrhs);
            if (nd->leaf) {
                memcpy(in, qs + nd->rs * nrhs, sizeof(orc_cx) * (size_t)m * nrhs);
            } else {
                int pos = 0;
                for (int c = 0; c < nd->nchild; ++c) {
                    int kc = h->rowc[nd->child0 + c].k;
                    memcpy(in + (size_t)pos * nrhs, qhat[nd->child0 + c], sizeof(orc_cx) * (size_t)kc * nrhs);
                    pos += kc;
                }
            }
            qhat[g] = calloc((size_t)(k > 0 ? k : 1) * nrhs, sizeof(orc_cx));
            for (int t = 0; t < k; ++t)
                for (int c = 0; c < nrhs; ++c) {
                    orc_cx s = in[(size_t)cp->skel_loc[t] * nrhs + c];
                    for (int u = 0; u < m - k; ++u) {
                        orc_cx y = cx_mul(ORC_GC(cp, (size_t)u * k + t), in[(size_t)cp->rest_loc[u] * nrhs + c]);
                        s.re = s.re + y.re;
                        s.im = s.im + y.im;
                    }
                    qhat[g][(size_t)t * nrhs + c] = s;
                }
            free(in);
        }
    }
    #pragma omp parallel for schedule(dynamic, 16)
    for (int g = 0; g < h->nnodes; ++g) {
        const orc_comp *ci = &h->rowc[g];
        zhat[g] = calloc((size_t)(ci->k > 0 ? ci->k : 1) * nrhs, sizeof(orc_cx));
        for (int64_t e = h->adm_ptr[g]; e < h->adm_ptr[g + 1]; ++e) {
            int j = h->adm_col[e];
            const orc_comp *cj = &h->rowc[j];
            for (int a = 0; a < ci->k; ++a)
                for (int bb = 0; bb < cj->k; ++bb) {
                    orc_cx kv = orc_cauchy_c(h->xs + ci->skel[a] * 2, h->xs + cj->skel[bb] * 2, h->dx_re, h->dx_im);
                    if (absval) { kv.re = sqrt(cx_abs2(kv)); kv.im = 0.0; }
                    for (int c = 0; c < nrhs; ++c) {
                        orc_cx y = cx_mul(kv, qhat[j][(size_t)bb * nrhs + c]);
                        zhat[g][(size_t)a * nrhs + c].re += y.re;
                        zhat[g][(size_t)a * nrhs + c].im += y.im;
                    }
                }
        }
    }
    for (int l = 2; l <= h->L; ++l) {
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) {
            const orc_node *nd = &h->nodes[g];
            const orc_comp *cp = &h->rowc[g];
            int m = cp->m, k = cp->k;
            orc_cx *out = calloc((size_t)(m > 0 ? m : 1) * nrhs, sizeof(orc_cx));
            for (int t = 0; t < k; ++t)
                for (int c = 0; c < nrhs; ++c)
                    out[(size_t)cp->skel_loc[t] * nrhs + c] = zhat[g][(size_t)t * nrhs + c];
            for (int u = 0; u < m - k; ++u)
                for (int c = 0; c < nrhs; ++c) {
                    orc_cx s = {0.0, 0.0};
                    for (int t = 0; t < k; ++t) {
                        orc_cx y = cx_mul(ORC_GC(cp, (size_t)u * k + t), zhat[g][(size_t)t * nrhs + c]);
                        s.re = s.re + y.re;
                        s.im = s.im + y.im;
                    }
                    out[(size_t)cp->rest_loc[u] * nrhs + c] = s;
                }
            if (nd->leaf) {
                for (int64_t a = 0; a < (int64_t)m * nrhs; ++a) {
                    zs[nd->rs * nrhs + a].re += out[a].re;
                    zs[nd->rs * nrhs + a].im += out[a].im;
                }
            } else {
                int pos = 0;
                for (int c = 0; c < nd->nchild; ++c) {
                    int kc = h->rowc[nd->child0 + c].k;
                    for (int64_t a = 0; a < (int64_t)kc * nrhs; ++a) {
                        zhat[nd->child0 + c][a].re += out[(size_t)pos * nrhs + a].re;
                        zhat[nd->child0 + c][a].im += out[(size_t)pos * nrhs + a].im;
                    }
                    pos += kc;
                }
            }
            free(out);
        }
    }
#undef ORC_GC
    #pragma omp parallel for schedule(dynamic, 16)
    for (int g = 0; g < h->nnodes; ++g) {
        const orc_node *ni = &h->nodes[g];
        for (int64_t e = h->near_ptr[g]; e < h->near_ptr[g + 1]; ++e) {
            const orc_node *nj = &h->nodes[h->near_col[e]];
            for (int64_t a = ni->rs; a < ni->rs + ni->rc; ++a)
                for (int64_t bb = nj->cs; bb < nj->cs + nj->cc; ++bb) {
                    orc_cx kv = orc_cauchy_c(h->xs + a * 2, h->xs + bb * 2, h->dx_re, h->dx_im);
                    if (absval) { kv.re = sqrt(cx_abs2(kv)); kv.im = 0.0; }
                    for (int c = 0; c < nrhs; ++c) {
                        orc_cx y = cx_mul(kv, qs[bb * nrhs + c]);
                        zs[a * nrhs + c].re += y.re;
                        zs[a * nrhs + c].im += y.im;
                    }
                }
        }
    }
    for (int64_t pnt = 0; pnt < n; ++pnt)
        for (int c = 0; c < nrhs; ++c) {
            orc_cx v = zs[pnt * nrhs + c];
            if (absval) {
                z_out[h->permx[pnt] * nrhs + c] = v.re;
            } else {
                z_out[2 * (h->permx[pnt] * nrhs + c)] = v.re;
                z_out[2 * (h->permx[pnt] * nrhs + c) + 1] = v.im;
            }
        }
    for (int g = 0; g < h->nnodes; ++g) { free(qhat[g]); free(zhat[g]); }
    free(qhat); free(zhat); free(qs); free(zs);
    return 0;
}

/* Dense rows of A q for kappa of (2.1) on C (Neumaier-compensated sums of
 * the real and imaginary parts): out[t] = sum_j kappa(x_rows[t], x_j) q_j. */
void orc_dense_rows_taylor(const double *x, int64_t n, const double *q_in, int nrhs, const int64_t *rows,
                           int64_t nrows, double dx_re, double dx_im, double *out)
{
    const orc_cx *q = (const orc_cx *)q_in;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nrows; ++t) {
        double *sum = calloc((size_t)2 * nrhs, sizeof(double));
        double *comp = calloc((size_t)2 * nrhs, sizeof(double));
        for (int64_t j = 0; j < n; ++j) {
            orc_cx kv = orc_cauchy_c(x + rows[t] * 2, x + j * 2, dx_re, dx_im);
            for (int c = 0; c < nrhs; ++c) {
                orc_cx y = cx_mul(kv, q[j * nrhs + c]);
                double parts[2] = {y.re, y.im};
                for (int p = 0; p < 2; ++p) {
                    double *sm = &sum[2 * c + p], *cm = &comp[2 * c + p];
                    double v = parts[p];
                    double s2 = *sm + v;
                    if (fabs(*sm) >= fabs(v)) *cm += (*sm - s2) + v;
                    else *cm += (v - s2) + *sm;
                    *sm = s2;
                }
            }
        }
        for (int c = 0; c < nrhs; ++c) {
            out[2 * (t * nrhs + c)] = sum[2 * c] + comp[2 * c];
            out[2 * (t * nrhs + c) + 1] = sum[2 * c + 1] + comp[2 * c + 1];
        }
        free(sum);
        free(comp);
    }
}

/* Per node (gid order): m, k, skeleton and rest indices (sorted positions)
 * and the complex G ((m-k) x k interleaved) of the Taylor representation. */
void orc_export_taylor(const orc_h2 *h, int32_t *m, int32_t *k, int64_t *skel, int64_t *rest, double *G)
{
    int64_t ps = 0, pr = 0, pg = 0;
    for (int g = 0; g < h->nnodes; ++g) {
        const orc_comp *c = &h->rowc[g];
        m[g] = c->m; k[g] = c->k;
        for (int t = 0; t < c->k; ++t) skel[ps++] = c->skel[t];
        for (int u = 0; u < c->m - c->k; ++u) rest[pr++] = c->rest[u];
        int64_t ng = (int64_t)(c->m - c->k) * c->k;
        if (ng > 0) memcpy(G + 2 * pg, c->G, sizeof(double) * 2 * (size_t)ng);
        pg += ng;
    }
}

/* ------------------------------------------------------------------------ */
/* Section 3.3.1 and Appendix A: HSS construction                           */
/* ------------------------------------------------------------------------ */
/* The HSS tree is binary: the partition of Section 3.1 in one dimension.  The
 * lists become (3.5): L = sibling pairs at every level, L^- = the diagonal
 * blocks of the leaves.  Each node's basis is the interpolation basis (2.2)
 * joined with a basis of its nearfield block row (3.7), compressed together
 * by (3.9); the matvec of Section 3.4 then applies the HSS generators with
 * these lists unchanged. */

#define ORC_JACOBI_EPS 1e-15
#define ORC_JACOBI_SWEEPS 60
#define ORC_JACOBI_FLOOR 1e-30

/* One-sided Jacobi SVD of the rows of B (m x n, row-major, overwritten):
 * plane rotations of row pairs (p, q), p < q, in the round-robin order of
 * Brent and Luk (rounds of disjoint pairs), sweep after sweep until a sweep
 * rotates no pair (|b_p . b_q| <= eps |b_p| |b_q|) or the sweep cap.  A pair
 * whose norm product |b_p| |b_q| is below 1e-30 of the squared Frobenius
 * norm of the input is not rotated: with more rows than columns the surplus
 * rows tend to zero and would otherwise keep exchanging roundoff.  JT (m x
 * m) starts as the identity and takes the same rotations, so that the input
 * equals JT^T B with mutually orthogonal rows of B: row p of JT is the left
 * singular vector of the singular value sig[p] = |b_p|.  Returns the sweeps. */
int orc_jacobi_rows(double *B, int m, int n, double *JT, double *sig)
{
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) JT[(size_t)i * m + j] = i == j ? 1.0 : 0.0;
    int M = m + (m & 1);
    int sweeps = 0;
    double frob2 = 0.0;
    for (size_t e = 0; e < (size_t)m * n; ++e) frob2 = fma(B[e], B[e], frob2);
    const double floor_ab = ORC_JACOBI_FLOOR * frob2;
    for (; sweeps < ORC_JACOBI_SWEEPS && m > 1; ++sweeps) {
        int rotated = 0;
        for (int rr = 0; rr < M - 1; ++rr)
            for (int i = 0; i < M / 2; ++i) {
                int a, b;
                if (i == 0) { a = M - 1; b = rr; }
                else { a = (rr + i) % (M - 1); b = (rr - i + (M - 1)) % (M - 1); }
                int p = a < b ? a : b, q = a < b ? b : a;
                if (q >= m) continue;
                double *bp = B + (size_t)p * n, *bq = B + (size_t)q * n;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int e = 0; e < n; ++e) {
                    al = fma(bp[e], bp[e], al);
                    be = fma(bq[e], bq[e], be);
                    ga = fma(bp[e], bq[e], ga);
                }
                const double nab = sqrt(al) * sqrt(be);
                if (ga == 0.0 || !(fabs(ga) > ORC_JACOBI_EPS * nab) || !(nab > floor_ab)) continue;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double sn = c * t;
                for (int e = 0; e < n; ++e) {
                    double u = bp[e], v = bq[e];
                    bp[e] = c * u - sn * v;
                    bq[e] = sn * u + c * v;
                }
                double *jp = JT + (size_t)p * m, *jq = JT + (size_t)q * m;
                for (int e = 0; e < m; ++e) {
                    double u = jp[e], v = jq[e];
                    jp[e] = c * u - sn * v;
                    jq[e] = sn * u + c * v;
                }
                rotated = 1;
            }
        if (!rotated) break;
    }
    for (int p = 0; p < m; ++p) {
        double s2 = 0.0;
        for (int e = 0; e < n; ++e) s2 = fma(B[(size_t)p * n + e], B[(size_t)p * n + e], s2);
        sig[p] = sqrt(s2);
    }
    return sweeps;
}

/* (3.7)/(3.11): the left singular vectors of A (m x n, destroyed) whose
 * singular values exceed eps_svd times the largest, in descending order of
 * the value (ties: lower index first), as the rows of ST (s x m); returns s. */
int orc_truncated_svd_rows(double *A, int m, int n, double eps_svd, double *ST)
{
    if (m == 0 || n == 0) return 0;
    double *JT = malloc(sizeof(double) * (size_t)m * m);
    double *sig = malloc(sizeof(double) * (size_t)m);
    int *used = calloc((size_t)m, sizeof(int));
    orc_jacobi_rows(A, m, n, JT, sig);
    double smax = 0.0;
    for (int p = 0; p < m; ++p) if (sig[p] > smax) smax = sig[p];
    int s = 0;
    for (;;) {
        int best = -1;
        for (int p = 0; p < m; ++p)
            if (!used[p] && (best < 0 || sig[p] > sig[best])) best = p;
        if (best < 0 || !(sig[best] > eps_svd * smax) || !(sig[best] > 0.0)) break;
        used[best] = 1;
        memcpy(ST + (size_t)s * m, JT + (size_t)best * m, sizeof(double) * (size_t)m);
        ++s;
    }
    free(JT); free(sig); free(used);
    return s;
}

/* working set of node g on a side: leaves own their points, parents the
 * concatenated skeletons of their children ((3.6), (3.14)) */
static int64_t *orc_working_set(const orc_h2 *h, int g, int side, int *m_out)
{
    const orc_node *nd = &h->nodes[g];
    const orc_comp *cs = side == 0 ? h->rowc : h->colc;
    int m;
    int64_t *ib;
    if (nd->leaf) {
        m = (int)(side == 0 ? nd->rc : nd->cc);
        int64_t st = side == 0 ? nd->rs : nd->cs;
        ib = malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        for (int c = 0; c < m; ++c) ib[c] = st + c;
    } else {
        m = 0;
        for (int c = 0; c < nd->nchild; ++c) m += cs[nd->child0 + c].k;
        ib = malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        int pos = 0;
        for (int c = 0; c < nd->nchild; ++c) {
            const orc_comp *ch = &cs[nd->child0 + c];
            for (int t = 0; t < ch->k; ++t) ib[pos++] = ch->skel[t];
        }
    }
    *m_out = m;
    return ib;
}

/* (3.9)/(3.13) for node g on one side: the nearfield block row (side 0:
 * rows i_bar^row, columns j_bar^col of j in N_i) or block column (side 1,
 * transposed), its truncated SVD, and compr of [U^_i, S_i]. */
static void orc_compress_node_hss(orc_h2 *h, int g, int side)
{
    orc_node *nd = &h->nodes[g];
    orc_comp *cp = side == 0 ? &h->rowc[g] : &h->colc[g];
    const double *pts = side == 0 ? h->xs : h->ys;
    const double *opts = side == 0 ? h->ys : h->xs;
    int r = h->r, m;
    cp->ibar = orc_working_set(h, g, side, &m);
    cp->m = m;
    if (m == 0) { cp->k = 0; return; }
    /* the columns of the nearfield block: the other side's working sets of N_i */
    int n = 0;
    int64_t **js = malloc(sizeof(int64_t *) * (size_t)(h->nf_ptr[g + 1] - h->nf_ptr[g] + 1));
    int *jm = malloc(sizeof(int) * (size_t)(h->nf_ptr[g + 1] - h->nf_ptr[g] + 1));
    for (int64_t e = h->nf_ptr[g]; e < h->nf_ptr[g + 1]; ++e) {
        js[e - h->nf_ptr[g]] = orc_working_set(h, h->nf_col[e], 1 - side, &jm[e - h->nf_ptr[g]]);
        n += jm[e - h->nf_ptr[g]];
    }
    double *A = malloc(sizeof(double) * (size_t)m * (size_t)(n > 0 ? n : 1));
    int col = 0;
    for (int64_t e = h->nf_ptr[g]; e < h->nf_ptr[g + 1]; ++e) {
        int64_t t = e - h->nf_ptr[g];
        for (int b = 0; b < jm[t]; ++b, ++col)
            for (int a = 0; a < m; ++a) {
                const double *pa = pts + cp->ibar[a], *pb = opts + js[t][b];
                A[(size_t)a * n + col] = side == 0 ? orc_kernel(h->kid, 1, pa, pb) : orc_kernel(h->kid, 1, pb, pa);
            }
        free(js[t]);
    }
    free(js); free(jm);
    int smax = m < n ? m : n;
    double *ST = malloc(sizeof(double) * (size_t)(smax > 0 ? smax : 1) * (size_t)m);
    int s = orc_truncated_svd_rows(A, m, n, h->eps_svd, ST);
    free(A);
    (side == 0 ? h->svd_rows : h->svd_cols)[g] = s;
    /* [U^_i, S_i]^T: the interpolation basis rows, then the singular vectors */
    int rr = r + s;
    double *Mt = malloc(sizeof(double) * (size_t)rr * (size_t)m);
    double *P = malloc(sizeof(double) * (size_t)m);
    for (int c = 0; c < m; ++c) P[c] = pts[cp->ibar[c]];
    orc_basis_t(1, h->p, h->anchors, h->lo, h->s, nd->level, nd->cell, P, m, Mt);
    memcpy(Mt + (size_t)r * m, ST, sizeof(double) * (size_t)s * m);
    free(ST); free(P);
    int *perm = malloc(sizeof(int) * (size_t)m);
    int kmax = rr < m ? rr : m;
    double *Aid = malloc(sizeof(double) * (size_t)(kmax * (m - 1) + 1));
    int k, nsw;
    orc_compr(Mt, rr, m, h->tol, h->f, perm, &k, Aid, &nsw);
    cp->k = k;
    cp->nswaps = nsw;
    int *sel = calloc((size_t)m, sizeof(int));
    for (int t = 0; t < k; ++t) sel[perm[t]] = 1;
    int *rank = malloc(sizeof(int) * (size_t)m);
    int ns = 0, nr = 0;
    for (int pos = 0; pos < m; ++pos) rank[pos] = sel[pos] ? ns++ : nr++;
    cp->skel = malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    cp->rest = malloc(sizeof(int64_t) * (size_t)(m - k > 0 ? m - k : 1));
    cp->skel_loc = malloc(sizeof(int32_t) * (size_t)(k > 0 ? k : 1));
    cp->rest_loc = malloc(sizeof(int32_t) * (size_t)(m - k > 0 ? m - k : 1));
    cp->G = malloc(sizeof(double) * (size_t)((m - k) * k > 0 ? (m - k) * k : 1));
    for (int pos = 0; pos < m; ++pos) {
        if (sel[pos]) { cp->skel[rank[pos]] = cp->ibar[pos]; cp->skel_loc[rank[pos]] = pos; }
        else { cp->rest[rank[pos]] = cp->ibar[pos]; cp->rest_loc[rank[pos]] = pos; }
    }
    int mk = m - k;
    for (int t = 0; t < k; ++t)
        for (int u = 0; u < mk; ++u)
            cp->G[(size_t)rank[perm[k + u]] * k + rank[perm[t]]] = Aid[(size_t)t * mk + u];
    free(Mt); free(perm); free(Aid); free(sel); free(rank);
}

static int orc_i32_cmp(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

/* HSS approximation (Section 3.3.1) of A = [kappa(x_i, y_j)] for points on a
 * line (d = 1; y == NULL: Y = X), interpolation order p, separation ratio tau
 * for the nearfield sets, SRRQR rank cut tol and bound f, truncated-SVD
 * tolerance eps_svd of (3.8).  NULL on invalid input. */
orc_h2 *orc_build_hss(const double *x, int64_t nx, const double *y, int64_t ny, int kid, int leaf, int p,
                      double tau, double tol, double eps_svd, double f)
{
    if (nx < 1 || leaf < 1 || p < 1 || p > ORC_MAXP || !(tol > 0.0) || !(eps_svd > 0.0) ||
        !(tau > 0.0 && tau < 1.0) || !(f > 1.0) || kid < 0 || kid > ORC_K_CAUCHY)
        return NULL;
    if (y && ny < 1) return NULL;
    for (int64_t i = 0; i < nx; ++i) if (!isfinite(x[i])) return NULL;
    if (y) for (int64_t i = 0; i < ny; ++i) if (!isfinite(y[i])) return NULL;
    orc_h2 *h = calloc(1, sizeof(orc_h2));
    h->d = 1; h->kid = kid; h->leaf = leaf; h->p = p; h->r = p; h->tau = tau; h->tol = tol; h->f = f;
    h->hss = 1; h->eps_svd = eps_svd;
    orc_chebyshev(p, h->anchors);
    orc_structure(h, x, nx, y, ny);
    /* (3.5): L = siblings, L^- = leaves with themselves */
    free(h->adm_ptr); free(h->adm_col); free(h->near_ptr); free(h->near_col);
    orc_pairs adm = {0}, near = {0};
    for (int g = 0; g < h->nnodes; ++g) {
        if (h->nodes[g].parent >= 0) {
            const orc_node *pn = &h->nodes[h->nodes[g].parent];
            for (int c = 0; c < pn->nchild; ++c)
                if (pn->child0 + c != g) orc_pairs_push(&adm, g, pn->child0 + c);
        }
        if (h->nodes[g].leaf) orc_pairs_push(&near, g, g);
    }
    h->nadm = adm.n; h->nnear = near.n;
    orc_to_csr(h->nnodes, &adm, &h->adm_ptr, &h->adm_col);
    orc_to_csr(h->nnodes, &near, &h->near_ptr, &h->near_col);
    free(adm.v); free(near.v);
    /* (A.1), top-down: N_root empty; N_i = siblings of i, the children k of
     * nodes of N_{p_i} with (i, k) not well separated, and the leaves of
     * N_{p_i} not well separated from i; ascending node id */
    h->nf_ptr = calloc((size_t)h->nnodes + 1, sizeof(int64_t));
    int32_t **lists = calloc((size_t)h->nnodes, sizeof(int32_t *));
    int *lcount = calloc((size_t)h->nnodes, sizeof(int));
    for (int l = 2; l <= h->L; ++l)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) {
            const orc_node *ni = &h->nodes[g];
            const orc_node *pn = &h->nodes[ni->parent];
            int cap = pn->nchild, cnt = 0;
            for (int t = 0; t < lcount[ni->parent]; ++t) {
                const orc_node *kq = &h->nodes[lists[ni->parent][t]];
                cap += kq->leaf ? 1 : kq->nchild;
            }
            int32_t *v = malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
            for (int c = 0; c < pn->nchild; ++c)
                if (pn->child0 + c != g) v[cnt++] = pn->child0 + c;
            for (int t = 0; t < lcount[ni->parent]; ++t) {
                int kq = lists[ni->parent][t];
                const orc_node *nk = &h->nodes[kq];
                if (nk->leaf) {
                    if (!orc_admissible(1, ni->level, ni->cell, nk->level, nk->cell, tau)) v[cnt++] = kq;
                } else {
                    for (int c = 0; c < nk->nchild; ++c) {
                        const orc_node *ch = &h->nodes[nk->child0 + c];
                        if (!orc_admissible(1, ni->level, ni->cell, ch->level, ch->cell, tau)) v[cnt++] = nk->child0 + c;
                    }
                }
            }
            qsort(v, (size_t)cnt, sizeof(int32_t), orc_i32_cmp);
            lists[g] = v;
            lcount[g] = cnt;
        }
    for (int g = 0; g < h->nnodes; ++g) h->nf_ptr[g + 1] = h->nf_ptr[g] + lcount[g];
    h->nf_col = malloc(sizeof(int32_t) * (size_t)(h->nf_ptr[h->nnodes] > 0 ? h->nf_ptr[h->nnodes] : 1));
    for (int g = 0; g < h->nnodes; ++g) {
        if (lcount[g]) memcpy(h->nf_col + h->nf_ptr[g], lists[g], sizeof(int32_t) * (size_t)lcount[g]);
        free(lists[g]);
    }
    free(lists); free(lcount);
    h->rowc = calloc((size_t)h->nnodes, sizeof(orc_comp));
    h->colc = h->same ? h->rowc : calloc((size_t)h->nnodes, sizeof(orc_comp));
    h->svd_rows = calloc((size_t)h->nnodes, sizeof(int32_t));
    h->svd_cols = h->same ? h->svd_rows : calloc((size_t)h->nnodes, sizeof(int32_t));
    /* (3.9)-(3.14): levels L..2, bottom-up; each node needs the working sets
     * of its nearfield nodes, which are complete once the level below is */
    for (int l = h->L; l >= 2; --l) {
        #pragma omp parallel for schedule(dynamic)
        for (int64_t g = h->lvl_off[l - 1]; g < h->lvl_off[l]; ++g) {
            orc_compress_node_hss(h, (int)g, 0);
            if (!h->same) orc_compress_node_hss(h, (int)g, 1);
        }
    }
    return h;
}

/* N_i in CSR (nf_ptr: nnodes + 1, nf_col: nf_ptr[nnodes]) and the numbers
 * of singular vectors s_i per node and side */
void orc_export_hss(const orc_h2 *h, int64_t *nf_ptr, int32_t *nf_col, int32_t *svd_rows, int32_t *svd_cols)
{
    memcpy(nf_ptr, h->nf_ptr, sizeof(int64_t) * ((size_t)h->nnodes + 1));
    if (h->nf_ptr[h->nnodes]) memcpy(nf_col, h->nf_col, sizeof(int32_t) * (size_t)h->nf_ptr[h->nnodes]);
    memcpy(svd_rows, h->svd_rows, sizeof(int32_t) * (size_t)h->nnodes);
    memcpy(svd_cols, h->svd_cols, sizeof(int32_t) * (size_t)h->nnodes);
}

