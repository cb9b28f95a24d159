/*
 * sph_oracle.c -- plain, slow, obviously correct FP64 CPU oracle of one SPH
 * time step (paper Section 3, Algorithm 1: build tree, find neighbours and
 * smoothing length, SPH kernels, new time step, update).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header
 * or constant with the CUDA path, and the CUDA path never calls it.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction:
 * every +, -, * and / below is rounded on its own, in the order written).
 *
 * The paper prints none of the SPH equations; each function states the
 * textbook definition it follows (Monaghan 1992 forms, M4 cubic spline of
 * Table 1) and the reading taken where the paper is silent.
 *
 * Parallel loops are in gather form (each i writes only its own outputs), so
 * results do not depend on the number of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t eos;         /* 0 = Tait, 1 = ideal gas */
    int32_t n_target;    /* target neighbour count (100) */
    int32_t n_tol;       /* accepted |n - n_target| (5) */
    int32_t max_h_iter;  /* h iterations before giving up */
    int32_t periodic_z;  /* 1: minimum image along z with period lz */
    int32_t kernel;      /* 0 = M4 cubic spline, 1 = Wendland C2, 2 = sinc (Table 1) */
    int32_t gradients;   /* 0 = kernel derivatives, 1 = IAD (Table 1) */
    int32_t sinc_n;      /* exponent n of the sinc kernel (kernel 2) */
    double rho0, c0, gamma, alpha, beta, eta2, cfl, lz;
} orc_params;

static const double ORC_PI = 3.14159265358979323846;

void orc_set_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * M4 cubic spline in 3D (Table 1, "M4 spline"), support 2h, q = r/h,
 * sigma = 1/(pi h^3):
 *   W = sigma (1 - 1.5 q^2 + 0.75 q^3)   0 <= q < 1
 *   W = sigma 0.25 (2 - q)^3             1 <= q < 2
 *   W = 0                                otherwise
 * and its radial derivative dW/dr = (1/(pi h^4)) f(q) with
 *   f = -3 q + 2.25 q^2 (q < 1),  f = -0.75 (2 - q)^2 (1 <= q < 2).
 * ------------------------------------------------------------------------- */
double orc_W(double r, double h)
{
    double q = r / h;
    double sigma = 1.0 / (ORC_PI * h * h * h);
    if (q < 1.0) return sigma * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) {
        double t = 2.0 - q;
        return sigma * (0.25 * t * t * t);
    }
    return 0.0;
}

double orc_dWdr(double r, double h)
{
    double q = r / h;
    double k = 1.0 / (ORC_PI * h * h * h * h);
    if (q < 1.0) return k * (-3.0 * q + 2.25 * q * q);
    if (q < 2.0) {
        double t = 2.0 - q;
        return k * (-0.75 * t * t);
    }
    return 0.0;
}

/* ---------------------------------------------------------------------------
 * Kernel variants (Tables 1 and 2 name the M4 spline, the Wendland and the
 * sinc kernels; the paper prints none of them, so each is the textbook form
 * in 3D with support 2h, written for q = r/h):
 *
 *  Wendland C2 (Wendland 1995, compact support H = 2h):
 *    W     = 21/(16 pi h^3) (1 - q/2)^4 (1 + 2 q)         q < 2
 *    dW/dr = -105/(16 pi h^4) q (1 - q/2)^3              q < 2
 *  since d/dq [(1 - q/2)^4 (1 + 2q)] = 2 (1 - q/2)^3 ((1 - q/2) - (1 + 2q))
 *  = -5 q (1 - q/2)^3.
 *
 *  Sinc (Cabezon, Garcia-Senz and Relano 2008), x = pi q / 2, S(x) = sin x / x:
 *    W     = B_n / h^3 S(x)^n                            q < 2
 *    dW/dr = B_n / h^4 (pi / 2) n S(x)^(n-1) S'(x),  S'(x) = (x cos x - sin x) / x^2
 *  with S(0) = 1, S'(0) = 0 and the normalisation
 *    B_n = 1 / (4 pi int_0^2 q^2 S(pi q / 2)^n dq)
 *  taken by composite Simpson quadrature (orc_sinc_norm).
 * ------------------------------------------------------------------------- */
static double orc_ipow(double v, int k)
{
    double r = 1.0;
    for (int e = 0; e < k; ++e) r = r * v;
    return r;
}

static double orc_sinc(double x)
{
    return x == 0.0 ? 1.0 : sin(x) / x;
}

static double orc_dsinc(double x)
{
    return x == 0.0 ? 0.0 : (x * cos(x) - sin(x)) / (x * x);
}

/* B_n by composite Simpson on [0, 2] with 2^16 panels, Kahan-summed. */
double orc_sinc_norm(int n)
{
    const int64_t panels = INT64_C(1) << 16;
    const double hq = 2.0 / (double)panels;
    double sum = 0.0, comp = 0.0;
    for (int64_t k = 0; k <= panels; ++k) {
        double q = hq * (double)k;
        double f = q * q * orc_ipow(orc_sinc(0.5 * ORC_PI * q), n);
        double wgt = (k == 0 || k == panels) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
        double y = wgt * f - comp;
        double t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    double integral = sum * hq / 3.0;
    return 1.0 / (4.0 * ORC_PI * integral);
}

/* The selected kernel with its normalisation evaluated once per call. */
typedef struct {
    int kind, n;
    double Bn; /* sinc normalisation (kind 2) */
} orc_kern;

static orc_kern orc_kern_of(const orc_params *P)
{
    orc_kern k = {P->kernel, P->sinc_n, 0.0};
    if (k.kind == 2) k.Bn = orc_sinc_norm(k.n);
    return k;
}

static double orc_kW(const orc_kern *K, double r, double h)
{
    if (K->kind == 0) return orc_W(r, h);
    double q = r / h;
    if (!(q < 2.0)) return 0.0;
    if (K->kind == 1) {
        double t = 1.0 - 0.5 * q;
        return 21.0 / (16.0 * ORC_PI * h * h * h) * (t * t * t * t * (1.0 + 2.0 * q));
    }
    return K->Bn / (h * h * h) * orc_ipow(orc_sinc(0.5 * ORC_PI * q), K->n);
}

static double orc_kdWdr(const orc_kern *K, double r, double h)
{
    if (K->kind == 0) return orc_dWdr(r, h);
    double q = r / h;
    if (!(q < 2.0)) return 0.0;
    if (K->kind == 1) {
        double t = 1.0 - 0.5 * q;
        return -105.0 / (16.0 * ORC_PI * h * h * h * h) * (q * t * t * t);
    }
    double x = 0.5 * ORC_PI * q;
    return K->Bn / (h * h * h * h) * (0.5 * ORC_PI) *
           ((double)K->n * orc_ipow(orc_sinc(x), K->n - 1) * orc_dsinc(x));
}

double orc_kernel_W(const orc_params *P, double r, double h)
{
    orc_kern K = orc_kern_of(P);
    return orc_kW(&K, r, h);
}

double orc_kernel_dWdr(const orc_params *P, double r, double h)
{
    orc_kern K = orc_kern_of(P);
    return orc_kdWdr(&K, r, h);
}

/* Pair vector r_ij = r_i - r_j; along z the minimum image with period lz when
 * periodic_z is set (Section 5.1.1: the patch is periodic in Z). */
static inline void orc_pair(const orc_params *P, const double *x, const double *y,
                            const double *z, int64_t i, int64_t j, double *d)
{
    d[0] = x[i] - x[j];
    d[1] = y[i] - y[j];
    double dz = z[i] - z[j];
    if (P->periodic_z) {
        double half = 0.5 * P->lz;
        if (dz > half) dz = dz - P->lz;
        else if (dz < -half) dz = dz + P->lz;
    }
    d[2] = dz;
}

/* r^2 = (dx dx + dy dy) + dz dz, left to right, each operation rounded. */
static inline double orc_r2(const double *d)
{
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* Gather radius test r_ij^2 < (2 h)^2 with a strict "<". */
static inline double orc_support2(double h)
{
    double s = 2.0 * h;
    return s * s;
}

/* ---------------------------------------------------------------------------
 * Uniform cell grid (Algorithm 1 step 1 replaced by a cell list): particles
 * binned by floor((x - lo) / w); a query of radius R visits every cell whose
 * index range overlaps [x - R, x + R] (one extra cell each side, so the
 * candidate set is a superset), then applies the exact pair test.
 * ------------------------------------------------------------------------- */
typedef struct {
    double lo[3], w[3];
    int n[3];
    int periodic_z;
    double lz;
    int64_t *start; /* ncells + 1 */
    int64_t *order; /* particle ids grouped by cell, ascending id within a cell */
} orc_grid;

static int orc_cell1(double v, double lo, double w, int n)
{
    double f = floor((v - lo) / w);
    if (f < 0.0) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (int)f;
}

static int orc_grid_build(orc_grid *g, const orc_params *P, int64_t n, const double *x,
                          const double *y, const double *z, double cell_w)
{
    const double *c[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            if (c[d][i] < mn) mn = c[d][i];
            if (c[d][i] > mx) mx = c[d][i];
        }
        if (n == 0) { mn = 0.0; mx = 0.0; }
        double ext = mx - mn;
        double w = cell_w > 0.0 ? cell_w : 1.0;
        int cnt = (int)fmin(256.0, floor(ext / w) + 1.0);
        if (cnt < 1) cnt = 1;
        if ((double)cnt * w <= ext) w = ext / ((double)cnt - 0.5);
        g->lo[d] = mn;
        g->w[d] = w;
        g->n[d] = cnt;
    }
    g->periodic_z = P->periodic_z;
    g->lz = P->lz;
    if (P->periodic_z) {
        double w = cell_w > 0.0 ? cell_w : P->lz;
        int cnt = (int)floor(P->lz / w);
        if (cnt < 1) cnt = 1;
        if (cnt > 256) cnt = 256;
        g->lo[2] = -0.5 * P->lz;
        g->w[2] = P->lz / (double)cnt;
        g->n[2] = cnt;
    }
    int64_t ncell = (int64_t)g->n[0] * g->n[1] * g->n[2];
    g->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *cell = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!g->start || !g->order || !cell) {
        free(g->start); free(g->order); free(cell);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        int kx = orc_cell1(x[i], g->lo[0], g->w[0], g->n[0]);
        int ky = orc_cell1(y[i], g->lo[1], g->w[1], g->n[1]);
        int kz = orc_cell1(z[i], g->lo[2], g->w[2], g->n[2]);
        cell[i] = ((int64_t)kz * g->n[1] + ky) * g->n[0] + kx;
        g->start[cell[i] + 1] += 1;
    }
    for (int64_t k = 0; k < ncell; ++k) g->start[k + 1] += g->start[k];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t) + 8);
    if (!fill) { free(g->start); free(g->order); free(cell); return -1; }
    memcpy(fill, g->start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) g->order[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
    return 0;
}

static void orc_grid_free(orc_grid *g)
{
    free(g->start);
    free(g->order);
}

/* Index range of cells to visit along axis d for a query interval [v-R, v+R]. */
static void orc_range(const orc_grid *g, int d, double v, double R, int *k0, int *k1)
{
    double a = floor((v - R - g->lo[d]) / g->w[d]) - 1.0;
    double b = floor((v + R - g->lo[d]) / g->w[d]) + 1.0;
    if (d == 2 && g->periodic_z) {
        if (b - a + 1.0 >= (double)g->n[2]) { *k0 = 0; *k1 = g->n[2] - 1; return; }
        *k0 = (int)a;  /* may be negative or >= n: wrapped by the caller */
        *k1 = (int)b;
        return;
    }
    if (a < 0.0) a = 0.0;
    if (b > (double)(g->n[d] - 1)) b = (double)(g->n[d] - 1);
    *k0 = (int)a;
    *k1 = (int)b;
}

static inline int orc_wrap(int k, int n)
{
    int r = k % n;
    return r < 0 ? r + n : r;
}

/* Visit every candidate j of the query (cells overlapping radius R) and call
 * visit(ctx, j). Each particle is visited at most once. */
typedef void (*orc_visit_fn)(void *ctx, int64_t j);

static void orc_grid_query(const orc_grid *g, double px, double py, double pz, double R,
                           orc_visit_fn visit, void *ctx)
{
    int x0, x1, y0, y1, z0, z1;
    orc_range(g, 0, px, R, &x0, &x1);
    orc_range(g, 1, py, R, &y0, &y1);
    orc_range(g, 2, pz, R, &z0, &z1);
    for (int kz = z0; kz <= z1; ++kz) {
        int cz = g->periodic_z ? orc_wrap(kz, g->n[2]) : kz;
        for (int ky = y0; ky <= y1; ++ky)
            for (int kx = x0; kx <= x1; ++kx) {
                int64_t c = ((int64_t)cz * g->n[1] + ky) * g->n[0] + kx;
                for (int64_t e = g->start[c]; e < g->start[c + 1]; ++e) visit(ctx, g->order[e]);
            }
    }
}

/* ---------------------------------------------------------------------------
 * Neighbour counting (Algorithm 1 step 2; footnote of Section 3: the run aims
 * at a target neighbour count which sets h). Gather set of i at radius 2h:
 *   N_i(h) = { j != i : r_ij^2 < (2h)^2 },  n_i = |N_i|.
 * ------------------------------------------------------------------------- */
typedef struct {
    const orc_params *P;
    const double *x, *y, *z;
    int64_t i;
    double s2;
    int64_t count;
} orc_count_ctx;

static void orc_count_visit(void *vctx, int64_t j)
{
    orc_count_ctx *c = (orc_count_ctx *)vctx;
    if (j == c->i) return;
    double d[3];
    orc_pair(c->P, c->x, c->y, c->z, c->i, j, d);
    if (orc_r2(d) < c->s2) c->count += 1;
}

int64_t orc_count_brute(const orc_params *P, int64_t n, const double *x, const double *y,
                        const double *z, int64_t i, double h)
{
    orc_count_ctx c = {P, x, y, z, i, orc_support2(h), 0};
    for (int64_t j = 0; j < n; ++j) orc_count_visit(&c, j);
    return c.count;
}

static int64_t orc_count_grid(const orc_grid *g, const orc_params *P, const double *x,
                              const double *y, const double *z, int64_t i, double h)
{
    orc_count_ctx c = {P, x, y, z, i, orc_support2(h), 0};
    orc_grid_query(g, x[i], y[i], z[i], 2.0 * h, orc_count_visit, &c);
    return c.count;
}

/* ---------------------------------------------------------------------------
 * Smoothing-length iteration (reading of the Section 3 footnote; the paper
 * gives no update rule). Bracketing search that uses only correctly rounded
 * + - * and compares, so every conforming implementation reaches the same
 * bits:
 *   lo = 0, hi = +inf, h = h_in
 *   repeat up to max_h_iter counts:
 *     n = |N_i(h)|;  if |n - n_target| <= n_tol: converged
 *     if n < n_target - n_tol: lo = h, h = (hi == inf) ? 1.25 h : (lo + hi) / 2
 *     else:                    hi = h, h = (lo == 0)   ? 0.8 h  : (lo + hi) / 2
 * The returned h is the last one counted; nnb is its count. A particle that
 * never lands in the band keeps that h and conv = 0.
 * ------------------------------------------------------------------------- */
static double orc_h_search(const orc_params *P, int64_t i, double h0,
                           int64_t (*count)(const void *, int64_t, double), const void *cctx,
                           int32_t *nnb, uint8_t *conv)
{
    double h = h0, lo = 0.0, hi = INFINITY;
    int64_t lowb = (int64_t)P->n_target - P->n_tol;
    int64_t highb = (int64_t)P->n_target + P->n_tol;
    *conv = 0;
    for (int it = 0; it < P->max_h_iter; ++it) {
        int64_t k = count(cctx, i, h);
        *nnb = (int32_t)k;
        if (k >= lowb && k <= highb) { *conv = 1; return h; }
        if (it == P->max_h_iter - 1) break;
        if (k < lowb) {
            lo = h;
            h = isinf(hi) ? h * 1.25 : 0.5 * (lo + hi);
        } else {
            hi = h;
            h = (lo == 0.0) ? h * 0.8 : 0.5 * (lo + hi);
        }
    }
    return h;
}

typedef struct {
    const orc_grid *g;
    const orc_params *P;
    const double *x, *y, *z;
    int64_t n;
} orc_hctx;

static int64_t orc_hcount_grid(const void *v, int64_t i, double h)
{
    const orc_hctx *c = (const orc_hctx *)v;
    return orc_count_grid(c->g, c->P, c->x, c->y, c->z, i, h);
}

static int64_t orc_hcount_brute(const void *v, int64_t i, double h)
{
    const orc_hctx *c = (const orc_hctx *)v;
    return orc_count_brute(c->P, c->n, c->x, c->y, c->z, i, h);
}

static double orc_max(int64_t n, const double *a)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (a[i] > m) m = a[i];
    return m;
}

/* Returns the number of particles that did not converge, or -1 on allocation
 * failure. brute != 0 counts over all pairs instead of the cell grid. */
int64_t orc_h_iterate(const orc_params *P, int64_t n, const double *x, const double *y,
                      const double *z, const double *h_in, double *h_out, int32_t *nnb,
                      uint8_t *conv, int brute)
{
    orc_grid g;
    memset(&g, 0, sizeof g);
    if (!brute && orc_grid_build(&g, P, n, x, y, z, 2.0 * orc_max(n, h_in)) != 0) return -1;
    orc_hctx c = {&g, P, x, y, z, n};
    int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : bad)
    for (int64_t i = 0; i < n; ++i) {
        h_out[i] = orc_h_search(P, i, h_in[i], brute ? orc_hcount_brute : orc_hcount_grid, &c,
                                &nnb[i], &conv[i]);
        if (!conv[i]) bad += 1;
    }
    if (!brute) orc_grid_free(&g);
    return bad;
}

/* ---------------------------------------------------------------------------
 * Symmetric interaction set (reading; the paper is silent): the forces sum
 * over S_i = { j != i : r_ij^2 < (2h_i)^2  or  r_ij^2 < (2h_j)^2 }, which is
 * symmetric in (i, j) as antisymmetric pair forces need. The density sums
 * over the gather subset N_i (first condition).
 *
 * CSR layout: row i holds first the entries of N_i in ascending j, then those
 * of S_i \ N_i in ascending j; ngather[i] = |N_i|.
 * ------------------------------------------------------------------------- */
typedef struct {
    const orc_params *P;
    const double *x, *y, *z, *h;
    int64_t i;
    double si2;
    int64_t *buf;   /* candidate list: j, tagged by (j << 1) | outer */
    int64_t len, cap;
    int oom;
} orc_sym_ctx;

static void orc_sym_visit(void *vctx, int64_t j)
{
    orc_sym_ctx *c = (orc_sym_ctx *)vctx;
    if (j == c->i) return;
    double d[3];
    orc_pair(c->P, c->x, c->y, c->z, c->i, j, d);
    double r2 = orc_r2(d);
    int in_i = r2 < c->si2;
    int in_j = r2 < orc_support2(c->h[j]);
    if (!(in_i || in_j)) return;
    if (c->len == c->cap) {
        int64_t nc = c->cap ? 2 * c->cap : 256;
        int64_t *nb = (int64_t *)realloc(c->buf, (size_t)nc * sizeof(int64_t));
        if (!nb) { c->oom = 1; return; }
        c->buf = nb;
        c->cap = nc;
    }
    c->buf[c->len++] = (j << 1) | (in_i ? 0 : 1);
}

static int orc_cmp_i64(const void *a, const void *b)
{
    int64_t u = *(const int64_t *)a, v = *(const int64_t *)b;
    return (u > v) - (u < v);
}

/* Gather row i of S_i into c->buf, sorted so that N_i comes first. */
static void orc_sym_row(const orc_grid *g, orc_sym_ctx *c, int brute, int64_t n, double hmax)
{
    c->len = 0;
    if (brute) {
        for (int64_t j = 0; j < n; ++j) orc_sym_visit(c, j);
    } else {
        double hi = c->h[c->i];
        double R = 2.0 * (hi > hmax ? hi : hmax);
        orc_grid_query(g, c->x[c->i], c->y[c->i], c->z[c->i], R, orc_sym_visit, c);
    }
    /* key: outer flag first, then j: sort (outer, j) lexicographically */
    for (int64_t k = 0; k < c->len; ++k) {
        int64_t v = c->buf[k];
        c->buf[k] = ((v & 1) << 62) | (v >> 1);
    }
    qsort(c->buf, (size_t)c->len, sizeof(int64_t), orc_cmp_i64);
}

/* Pass 1: counts[i] = |S_i|. Returns 0, or -1 on allocation failure. */
int orc_csr_count(const orc_params *P, int64_t n, const double *x, const double *y,
                  const double *z, const double *h, int64_t *counts, int brute)
{
    orc_grid g;
    memset(&g, 0, sizeof g);
    double hmax = orc_max(n, h);
    if (!brute && orc_grid_build(&g, P, n, x, y, z, 2.0 * hmax) != 0) return -1;
    int fail = 0;
#pragma omp parallel reduction(| : fail)
    {
        orc_sym_ctx c = {P, x, y, z, h, 0, 0.0, NULL, 0, 0, 0};
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            c.i = i;
            c.si2 = orc_support2(h[i]);
            orc_sym_row(&g, &c, brute, n, hmax);
            counts[i] = c.len;
        }
        fail |= c.oom;
        free(c.buf);
    }
    if (!brute) orc_grid_free(&g);
    return fail ? -1 : 0;
}

/* Pass 2: offsets[n+1] (given, exclusive prefix of counts), idx[nnz],
 * ngather[n]. */
int orc_csr_fill(const orc_params *P, int64_t n, const double *x, const double *y,
                 const double *z, const double *h, const int64_t *offsets, int32_t *idx,
                 int32_t *ngather, int brute)
{
    orc_grid g;
    memset(&g, 0, sizeof g);
    double hmax = orc_max(n, h);
    if (!brute && orc_grid_build(&g, P, n, x, y, z, 2.0 * hmax) != 0) return -1;
    int fail = 0;
#pragma omp parallel reduction(| : fail)
    {
        orc_sym_ctx c = {P, x, y, z, h, 0, 0.0, NULL, 0, 0, 0};
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            c.i = i;
            c.si2 = orc_support2(h[i]);
            orc_sym_row(&g, &c, brute, n, hmax);
            if (c.len != offsets[i + 1] - offsets[i]) { fail = 1; continue; }
            int32_t ng = 0;
            for (int64_t k = 0; k < c.len; ++k) {
                int64_t v = c.buf[k];
                if (!(v >> 62)) ng += 1;
                idx[offsets[i] + k] = (int32_t)(v & ((INT64_C(1) << 62) - 1));
            }
            ngather[i] = ng;
        }
        fail |= c.oom;
        free(c.buf);
    }
    if (!brute) orc_grid_free(&g);
    return fail ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Density summation (Section 3, Algorithm 1 step 3, the density): standard volume elements,
 *   rho_i = m_i W(0, h_i) + sum_{j in N_i} m_j W(r_ij, h_i),
 * with W the selected kernel.
 * ------------------------------------------------------------------------- */
void orc_density(const orc_params *P, int64_t n, const double *x, const double *y,
                 const double *z, const double *m, const double *h, const int64_t *offsets,
                 const int32_t *idx, const int32_t *ngather, double *rho)
{
    orc_kern K = orc_kern_of(P);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = m[i] * orc_kW(&K, 0.0, h[i]);
        for (int64_t e = offsets[i]; e < offsets[i] + ngather[i]; ++e) {
            int64_t j = idx[e];
            double d[3];
            orc_pair(P, x, y, z, i, j, d);
            s = s + m[j] * orc_kW(&K, sqrt(orc_r2(d)), h[i]);
        }
        rho[i] = s;
    }
}

/* ---------------------------------------------------------------------------
 * Integral approach to derivatives, IAD (the gradients column of Table 1;
 * Garcia-Senz, Cabezon and Escartin 2012). With volume elements V_j = m_j /
 * rho_j and the gather set N_i, the symmetric 3x3 matrix
 *   tau_i = sum_{j in N_i} V_j W(r_ij, h_i) (r_j - r_i) (r_j - r_i)^T
 * is inverted, C_i = tau_i^(-1) (adjugate over determinant; a singular tau
 * gives C_i = 0). Stored per particle as (xx, xy, xz, yy, yz, zz).
 * The IAD gradient of a field f,
 *   grad f_i = C_i sum_{j in N_i} V_j (f_j - f_i) W(r_ij, h_i) (r_j - r_i),
 * is exact for every linear f, because the sum is then tau_i grad f.
 * ------------------------------------------------------------------------- */
static void orc_inv3(const double *t, double *cm)
{
    double a = t[0], b = t[1], c = t[2], d = t[3], e = t[4], f = t[5];
    /* cofactors of the symmetric matrix [[a b c] [b d e] [c e f]] */
    double c00 = d * f - e * e, c01 = c * e - b * f, c02 = b * e - c * d;
    double c11 = a * f - c * c, c12 = b * c - a * e, c22 = a * d - b * b;
    double det = a * c00 + b * c01 + c * c02;
    if (det == 0.0) {
        for (int k = 0; k < 6; ++k) cm[k] = 0.0;
        return;
    }
    cm[0] = c00 / det; cm[1] = c01 / det; cm[2] = c02 / det;
    cm[3] = c11 / det; cm[4] = c12 / det; cm[5] = c22 / det;
}

void orc_iad(const orc_params *P, int64_t n, const double *x, const double *y, const double *z,
             const double *m, const double *h, const double *rho, const int64_t *offsets,
             const int32_t *idx, const int32_t *ngather, double *cmat)
{
    orc_kern K = orc_kern_of(P);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int64_t e = offsets[i]; e < offsets[i] + ngather[i]; ++e) {
            int64_t j = idx[e];
            double d[3];
            orc_pair(P, x, y, z, i, j, d);
            double r = sqrt(orc_r2(d));
            double w = m[j] / rho[j] * orc_kW(&K, r, h[i]);
            /* (r_j - r_i) = -d; the outer product is the same for +-d */
            t[0] = t[0] + w * d[0] * d[0];
            t[1] = t[1] + w * d[0] * d[1];
            t[2] = t[2] + w * d[0] * d[2];
            t[3] = t[3] + w * d[1] * d[1];
            t[4] = t[4] + w * d[1] * d[2];
            t[5] = t[5] + w * d[2] * d[2];
        }
        orc_inv3(t, cmat + 6 * i);
    }
}

/* C v for the symmetric matrix c = (xx, xy, xz, yy, yz, zz). */
static void orc_symv(const double *c, const double *v, double *o)
{
    o[0] = c[0] * v[0] + c[1] * v[1] + c[2] * v[2];
    o[1] = c[1] * v[0] + c[3] * v[1] + c[4] * v[2];
    o[2] = c[2] * v[0] + c[4] * v[1] + c[5] * v[2];
}

void orc_iad_gradient(const orc_params *P, int64_t n, const double *x, const double *y,
                      const double *z, const double *m, const double *h, const double *rho,
                      const int64_t *offsets, const int32_t *idx, const int32_t *ngather,
                      const double *cmat, const double *f, double *gx, double *gy, double *gz)
{
    orc_kern K = orc_kern_of(P);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int64_t e = offsets[i]; e < offsets[i] + ngather[i]; ++e) {
            int64_t j = idx[e];
            double d[3];
            orc_pair(P, x, y, z, i, j, d);
            double r = sqrt(orc_r2(d));
            double w = m[j] / rho[j] * (f[j] - f[i]) * orc_kW(&K, r, h[i]);
            for (int k = 0; k < 3; ++k) s[k] = s[k] - w * d[k]; /* r_j - r_i = -d */
        }
        double g[3];
        orc_symv(cmat + 6 * i, s, g);
        gx[i] = g[0];
        gy[i] = g[1];
        gz[i] = g[2];
    }
}

/* ---------------------------------------------------------------------------
 * Equation of state.
 *  Tait (square patch): p = (c0^2 rho0 / 7) (x^7 - 1), x = rho/rho0, with
 *    x^7 = ((x^2)^2 x^2) x; sound speed c = sqrt(dp/drho) = c0 x^3.
 *  Ideal gas (Evrard, Section 5.1.2, gamma = 5/3): p = (gamma - 1) rho u,
 *    c = sqrt(gamma (gamma - 1) u).
 * ------------------------------------------------------------------------- */
void orc_eos(const orc_params *P, int64_t n, const double *rho, const double *u, double *p,
             double *c)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (P->eos == 0) {
            double xr = rho[i] / P->rho0;
            double x2 = xr * xr;
            double x4 = x2 * x2;
            double x7 = (x4 * x2) * xr;
            p[i] = (P->c0 * P->c0 * P->rho0 / 7.0) * (x7 - 1.0);
            c[i] = P->c0 * (x2 * xr);
        } else {
            p[i] = (P->gamma - 1.0) * rho[i] * u[i];
            c[i] = sqrt(P->gamma * (P->gamma - 1.0) * u[i]);
        }
    }
}

/* ---------------------------------------------------------------------------
 * Momentum and energy with Monaghan artificial viscosity (Section 3,
 * Algorithm 1 step 3: the accelerations and the rates of change of the
 * internal energy; Table 1: standard volume elements, gradients from kernel
 * derivatives). For j in S_i:
 *   r_ij = r_i - r_j, v_ij = v_i - v_j, r = |r_ij|
 *   Fbar_ij = (dW/dr(r, h_i) + dW/dr(r, h_j)) / 2 / r  (each zero outside its
 *             own support), so grad_i Wbar_ij = Fbar_ij r_ij
 *   A_i = p_i / rho_i^2
 *   if v_ij . r_ij < 0:
 *      hb = (h_i + h_j)/2, cb = (c_i + c_j)/2, rhob = (rho_i + rho_j)/2
 *      mu_ij = hb (v_ij . r_ij) / (r^2 + eta2 hb^2)
 *      Pi_ij = (-alpha cb mu_ij + beta mu_ij^2) / rhob
 *   else mu_ij = Pi_ij = 0
 *   a_i   = - sum_j m_j (A_i + A_j + Pi_ij) Fbar_ij r_ij
 *   du_i  = A_i sum_j m_j Fbar_ij (v_ij . r_ij)
 *           + 1/2 sum_j m_j Pi_ij Fbar_ij (v_ij . r_ij)
 *   mumax_i = max_j |mu_ij|
 * A pair at zero separation contributes nothing. dW/dr is the selected
 * kernel's.
 *
 * IAD gradients (gradients = 1) replace the symmetrised kernel gradient
 * Fbar_ij r_ij by the symmetrised IAD one,
 *   G_ij = 1/2 (W(r, h_i) C_i (r_j - r_i) + W(r, h_j) C_j (r_j - r_i))
 * (the IAD estimate of grad_i W(r_ij, h) at each particle's own h and C;
 * each W zero outside its own support), in every place it appears:
 *   a_i  = - sum_j m_j (A_i + A_j + Pi_ij) G_ij
 *   du_i = A_i sum_j m_j G_ij . v_ij + 1/2 sum_j m_j Pi_ij G_ij . v_ij
 * G_ji = -G_ij, so total momentum and total energy are conserved as with
 * kernel derivatives (angular momentum is not: G_ij need not be parallel to
 * r_ij).
 * ------------------------------------------------------------------------- */
static void orc_iad_pair(const orc_kern *K, const double *cmat, int64_t i, int64_t j,
                         const double *h, double r, const double *d, double *G)
{
    double rji[3] = {-d[0], -d[1], -d[2]};
    double ui[3], uj[3];
    orc_symv(cmat + 6 * i, rji, ui);
    orc_symv(cmat + 6 * j, rji, uj);
    double wi = orc_kW(K, r, h[i]), wj = orc_kW(K, r, h[j]);
    for (int k = 0; k < 3; ++k) G[k] = 0.5 * (wi * ui[k] + wj * uj[k]);
}

void orc_forces(const orc_params *P, int64_t n, const double *x, const double *y,
                const double *z, const double *vx, const double *vy, const double *vz,
                const double *m, const double *h, const double *rho, const double *p,
                const double *c, const int64_t *offsets, const int32_t *idx, const double *cmat,
                double *ax, double *ay, double *az, double *du, double *mumax)
{
    orc_kern K = orc_kern_of(P);
    int iad = P->gradients == 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double Ai = p[i] / (rho[i] * rho[i]);
        double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0, sv = 0.0, mum = 0.0;
        for (int64_t e = offsets[i]; e < offsets[i + 1]; ++e) {
            int64_t j = idx[e];
            double d[3];
            orc_pair(P, x, y, z, i, j, d);
            double r2 = orc_r2(d);
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double wx = vx[i] - vx[j], wy = vy[i] - vy[j], wz = vz[i] - vz[j];
            double vr = (wx * d[0] + wy * d[1]) + wz * d[2];
            double Pi = 0.0, mu = 0.0;
            if (vr < 0.0) {
                double hb = 0.5 * (h[i] + h[j]);
                double cb = 0.5 * (c[i] + c[j]);
                double rb = 0.5 * (rho[i] + rho[j]);
                mu = hb * vr / (r2 + P->eta2 * hb * hb);
                Pi = (-P->alpha * cb * mu + P->beta * mu * mu) / rb;
            }
            double Aj = p[j] / (rho[j] * rho[j]);
            if (iad) {
                double G[3];
                orc_iad_pair(&K, cmat, i, j, h, r, d, G);
                double Gv = (G[0] * wx + G[1] * wy) + G[2] * wz;
                double g = m[j] * (Ai + Aj + Pi);
                sx = sx + g * G[0];
                sy = sy + g * G[1];
                sz = sz + g * G[2];
                sp = sp + m[j] * Gv;
                sv = sv + m[j] * Pi * Gv;
            } else {
                double Fb = 0.5 * (orc_kdWdr(&K, r, h[i]) + orc_kdWdr(&K, r, h[j])) / r;
                double g = m[j] * (Ai + Aj + Pi) * Fb;
                sx = sx + g * d[0];
                sy = sy + g * d[1];
                sz = sz + g * d[2];
                sp = sp + m[j] * Fb * vr;
                sv = sv + m[j] * Pi * Fb * vr;
            }
            double amu = fabs(mu);
            if (amu > mum) mum = amu;
        }
        ax[i] = -sx;
        ay[i] = -sy;
        az[i] = -sz;
        du[i] = Ai * sp + 0.5 * sv;
        mumax[i] = mum;
    }
}

/* Conditioning scales of the force sums, for comparing two implementations
 * whose sums round differently: per particle the sums of the magnitudes of
 * the terms that the definitions above add up,
 *   sa_i  = sum_j m_j |A_i + A_j + Pi_ij| |g_ij|
 *   sdu_i = |A_i| sum_j m_j |g_ij| |v_ij| + 1/2 sum_j m_j |Pi_ij| |g_ij| |v_ij|
 * with g_ij = Fbar_ij r_ij, or G_ij with IAD gradients,
 *   smu_i = max_j hb |v_ij| |r_ij| / (r^2 + eta2 hb^2)
 * Rounding in v_ij . r_ij alone is bounded by a few ulps of |v_ij| |r_ij|, so
 * a field whose exact value is zero (du and mu under rigid rotation) carries
 * noise of order 1e-16 of these scales in any implementation. */
void orc_forces_scale(const orc_params *P, int64_t n, const double *x, const double *y,
                      const double *z, const double *vx, const double *vy, const double *vz,
                      const double *m, const double *h, const double *rho, const double *p,
                      const double *c, const int64_t *offsets, const int32_t *idx,
                      const double *cmat, double *sa, double *sdu, double *smu)
{
    orc_kern K = orc_kern_of(P);
    int iad = P->gradients == 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double Ai = p[i] / (rho[i] * rho[i]);
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
        for (int64_t e = offsets[i]; e < offsets[i + 1]; ++e) {
            int64_t j = idx[e];
            double d[3];
            orc_pair(P, x, y, z, i, j, d);
            double r2 = orc_r2(d);
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            /* |grad|: |Fbar_ij| r, or |G_ij| with IAD */
            double gabs;
            if (iad) {
                double G[3];
                orc_iad_pair(&K, cmat, i, j, h, r, d, G);
                gabs = sqrt((G[0] * G[0] + G[1] * G[1]) + G[2] * G[2]);
            } else {
                gabs = fabs(0.5 * (orc_kdWdr(&K, r, h[i]) + orc_kdWdr(&K, r, h[j])) / r) * r;
            }
            double wx = vx[i] - vx[j], wy = vy[i] - vy[j], wz = vz[i] - vz[j];
            double vr = (wx * d[0] + wy * d[1]) + wz * d[2];
            double vabs = sqrt((wx * wx + wy * wy) + wz * wz);
            double hb = 0.5 * (h[i] + h[j]);
            double Pi = 0.0;
            if (vr < 0.0) {
                double cb = 0.5 * (c[i] + c[j]);
                double rb = 0.5 * (rho[i] + rho[j]);
                double mu = hb * vr / (r2 + P->eta2 * hb * hb);
                Pi = (-P->alpha * cb * mu + P->beta * mu * mu) / rb;
            }
            double Aj = p[j] / (rho[j] * rho[j]);
            s1 = s1 + m[j] * fabs(Ai + Aj + Pi) * gabs;
            s2 = s2 + m[j] * gabs * vabs;
            s3 = s3 + m[j] * fabs(Pi) * gabs * vabs;
            double mus = hb * vabs * r / (r2 + P->eta2 * hb * hb);
            if (mus > s4) s4 = mus;
        }
        sa[i] = s1;
        sdu[i] = fabs(Ai) * s2 + 0.5 * s3;
        smu[i] = s4;
    }
}

/* ---------------------------------------------------------------------------
 * New time step (Algorithm 1 step 5; reading: Monaghan's Courant form with
 * the viscous signal term, CFL factor from the workload):
 *   dt = cfl * min_i h_i / (c_i + 1.2 (alpha c_i + beta mumax_i)).
 * Returns +inf for n == 0.
 * ------------------------------------------------------------------------- */
double orc_dt(const orc_params *P, int64_t n, const double *h, const double *c,
              const double *mumax)
{
    double best = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double v = h[i] / (c[i] + 1.2 * (P->alpha * c[i] + P->beta * mumax[i]));
        if (v < best) best = v;
    }
    return P->cfl * best;
}

/* ---------------------------------------------------------------------------
 * Update velocity and position (Algorithm 1 step 6; leapfrog read as
 * kick-drift): v += dt a; u += dt du; x += dt v (new v); then z is wrapped
 * back into [-lz/2, lz/2) when periodic.
 * ------------------------------------------------------------------------- */
void orc_leapfrog(const orc_params *P, int64_t n, double dt, double *x, double *y, double *z,
                  double *vx, double *vy, double *vz, double *u, const double *ax,
                  const double *ay, const double *az, const double *du)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        vx[i] = vx[i] + dt * ax[i];
        vy[i] = vy[i] + dt * ay[i];
        vz[i] = vz[i] + dt * az[i];
        u[i] = u[i] + dt * du[i];
        x[i] = x[i] + dt * vx[i];
        y[i] = y[i] + dt * vy[i];
        z[i] = z[i] + dt * vz[i];
        if (P->periodic_z) {
            double half = 0.5 * P->lz;
            if (z[i] >= half) z[i] = z[i] - P->lz;
            else if (z[i] < -half) z[i] = z[i] + P->lz;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Whole time step, Algorithm 1 order: neighbours and h, density, EOS, (the
 * IAD matrices when selected), forces, dt, update. State arrays are updated in place; rho, p, c, a, du,
 * mumax receive the values of the last step's force evaluation. stats (may be
 * NULL) receives { nnz of the last step, non-converged particles summed over
 * the steps }. Returns 0, or -1 on allocation failure.
 * ------------------------------------------------------------------------- */
int orc_step(const orc_params *P, int64_t n, int nsteps, double *x, double *y, double *z,
             double *vx, double *vy, double *vz, const double *m, double *h, double *u,
             double *rho, double *p, double *c, double *ax, double *ay, double *az, double *du,
             double *mumax, double *time, double *dt_out, int64_t *stats)
{
    int32_t *nnb = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *ng = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    uint8_t *conv = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    int64_t *off = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    double *hn = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *cm = P->gradients == 1 ? (double *)malloc((size_t)(n > 0 ? n : 1) * 6 * sizeof(double))
                                   : NULL;
    int rc = 0;
    int64_t bad_total = 0, nnz = 0;
    if (!nnb || !ng || !conv || !off || !hn || (P->gradients == 1 && !cm)) { rc = -1; goto done; }
    for (int s = 0; s < nsteps; ++s) {
        int64_t bad = orc_h_iterate(P, n, x, y, z, h, hn, nnb, conv, 0);
        if (bad < 0) { rc = -1; goto done; }
        bad_total += bad;
        memcpy(h, hn, (size_t)n * sizeof(double));
        if (orc_csr_count(P, n, x, y, z, h, off + 1, 0) != 0) { rc = -1; goto done; }
        off[0] = 0;
        for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i];
        nnz = off[n];
        int32_t *idx = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
        if (!idx) { rc = -1; goto done; }
        if (orc_csr_fill(P, n, x, y, z, h, off, idx, ng, 0) != 0) { free(idx); rc = -1; goto done; }
        orc_density(P, n, x, y, z, m, h, off, idx, ng, rho);
        orc_eos(P, n, rho, u, p, c);
        if (P->gradients == 1) orc_iad(P, n, x, y, z, m, h, rho, off, idx, ng, cm);
        orc_forces(P, n, x, y, z, vx, vy, vz, m, h, rho, p, c, off, idx, cm, ax, ay, az, du,
                   mumax);
        free(idx);
        double dt = orc_dt(P, n, h, c, mumax);
        orc_leapfrog(P, n, dt, x, y, z, vx, vy, vz, u, ax, ay, az, du);
        *time = *time + dt;
        *dt_out = dt;
    }
done:
    if (stats) { stats[0] = nnz; stats[1] = bad_total; }
    free(nnb); free(ng); free(conv); free(off); free(hn); free(cm);
    return rc;
}
