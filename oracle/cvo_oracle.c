/*
 * FP64 CPU oracle for the Continuous Visual Odometry (CVO) pair sums.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent reference the CUDA
 * path is checked against. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product library never does.
 * It shares no code, header or constant with the CUDA sources.
 *
 * What it computes, for a fixed cloud X = {x_i, f_i} (the target), a moving
 * cloud Z = {z_j, g_j} (the source) and a pose P = (R, T) that maps Z into
 * X's frame (P is the paper's h^{-1}, Sec. 3 "Calculating the Gradient",
 * where z~_j = h^{-1} z_j):
 *
 *   z~_j  = R z_j + T
 *   e_ij  = x_i - z~_j
 *   k_ij  = sigma^2 exp(-|e_ij|^2 / (2 ell^2))          squared-exponential
 *                                                        kernel, Sec. 3
 *   c_ij  = label inner product (Sec. 2 remark defining c_ij):
 *             COLOR_NONE   : 1
 *             COLOR_KERNEL : exp(-|f_i - g_j|^2 / (2 ell_c^2))
 *             COLOR_DOT    : s <f_i, g_j>   (Sec. 5 remark, s = 1e-5)
 *   F     = sum_ij c_ij k_ij                             Eq. (scalar)
 *
 * Kernel sparsification (Sec. 5, Table 1): a pair whose spatial kernel value
 * exp(-|e|^2/2ell^2) is below kcut is dropped, i.e. a pair is kept iff
 * |e|^2 <= r_c^2 = 2 ell^2 ln(1/kcut). kcut <= 0 keeps every pair.
 *
 * Gradient (Eq. 3_gradient, with the sign convention fixed by differentiating
 * F along the left perturbation P <- exp(t xi) P, xi = (omega, v)):
 *   dF/domega = (1/ell^2) sum_ij w_ij (z~_j x e_ij)
 *   dF/dv     = (1/ell^2) sum_ij w_ij e_ij,          w_ij = c_ij k_ij
 * These are returned unscaled; dividing by a^2 and b^2 (Eq. metric, n = 3)
 * is the caller's job.
 *
 * Step-size sums (Eq. fourth): along a direction xi, the exponent of each
 * pair's kernel at exp(t xi) P is alpha + beta t + gamma t^2 + delta t^3 +
 * eps t^4 + O(t^5) with, for u1 = omega x z~ + v and u_k = omega x u_{k-1},
 *   alpha = -|e|^2 / (2 ell^2)
 *   beta  =  <e,u1> / ell^2
 *   gamma = (<e,u2> - |u1|^2) / (2 ell^2)
 *   delta = (<e,u3>/6 - <u1,u2>/2) / ell^2
 *   eps   = (<e,u4>/24 - <u1,u3>/6 - |u2|^2/8) / ell^2
 * (the exact expansion of -|x - exp(t xi) z~|^2 / 2ell^2; the coefficients
 * printed with Eq. fourth are not this expansion), and exp(beta t + ...)
 * = 1 + g1 t + g2 t^2 + g3 t^3 + g4 t^4 + O(t^5) with g1..g4 composed exactly
 * as printed with Eq. fourth. The returned sums are S0 = sum w and
 * S_m = sum w g_m, so G(t) = F(exp(t xi) P) ~ S0 + S1 t + S2 t^2 + S3 t^3 +
 * S4 t^4.
 *
 * Two searches give the same sums bit for bit: the exhaustive loop over
 * every target point (orc_pair_sums*) and a grid search over the 27 cells
 * of edge r_c around each source point (orc_pair_sums_grid*), which visits
 * its candidates in the exhaustive loop's order. The grid search is what
 * makes whole solves of large clouds affordable on the CPU.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_COLOR_NONE 0
#define ORC_COLOR_KERNEL 1
#define ORC_COLOR_DOT 2

/* Number of doubles returned per source point by orc_pair_sums_per_j. */
#define ORC_NOUT 13 /* F, dFdw[3], dFdv[3], nnz, S0..S4 */

typedef struct {
    double ell;         /* spatial lengthscale */
    double sigma;       /* kernel signal standard deviation */
    double kcut;        /* sparsification threshold on exp(-d^2/2ell^2); <= 0: off */
    int color_mode;     /* ORC_COLOR_* */
    double ell_color;   /* appearance lengthscale (COLOR_KERNEL) */
    double color_scale; /* label inner-product scale (COLOR_DOT) */
} orc_params;

static void cross3(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Label inner product c_ij (Sec. 2 remark; Sec. 5 remark for COLOR_DOT). */
static double label_product(const double* fi, const double* gj, int D, const orc_params* p) {
    if (p->color_mode == ORC_COLOR_NONE || D <= 0) return 1.0;
    if (p->color_mode == ORC_COLOR_DOT) {
        double s = 0.0;
        for (int d = 0; d < D; ++d) s += fi[d] * gj[d];
        return p->color_scale * s;
    }
    double q = 0.0;
    for (int d = 0; d < D; ++d) {
        double df = fi[d] - gj[d];
        q += df * df;
    }
    return exp(-q / (2.0 * p->ell_color * p->ell_color));
}

/* Contribution of the pair (i, j) to out[], if it survives the cutoff:
 * zt = z~_j, gj its features, u = {u1, u2, u3, u4} for the step sums (NULL:
 * no step sums). Both search modes call exactly this, so they keep the same
 * pairs and, adding them in the same order, give the same bits. */
static void add_pair(const double* X, const double* FX, int64_t i, const double zt[3],
                     const double* gj, int D, const orc_params* prm, const double (*u)[3],
                     double out[ORC_NOUT]) {
    const double ell2 = prm->ell * prm->ell;
    const double sig2 = prm->sigma * prm->sigma;
    const int use_cut = prm->kcut > 0.0;
    const double rc2 = use_cut ? 2.0 * ell2 * log(1.0 / prm->kcut) : 0.0;
    const double* xv = X + 3 * i;
    double e[3] = {xv[0] - zt[0], xv[1] - zt[1], xv[2] - zt[2]};
    double d2 = dot3(e, e);
    if (use_cut && d2 > rc2) return;
    double alpha = -d2 / (2.0 * ell2);
    double k = sig2 * exp(alpha);
    double c = label_product(FX ? FX + (int64_t)D * i : NULL, gj, D, prm);
    double w = c * k;
    out[0] += w;
    double zxe[3];
    cross3(zt, e, zxe);
    for (int r = 0; r < 3; ++r) {
        out[1 + r] += w * zxe[r] / ell2;
        out[4 + r] += w * e[r] / ell2;
    }
    out[7] += 1.0;
    if (u) {
        const double* u1 = u[0];
        const double* u2 = u[1];
        const double* u3 = u[2];
        const double* u4 = u[3];
        double beta = dot3(e, u1) / ell2;
        double gamma = (dot3(e, u2) - dot3(u1, u1)) / (2.0 * ell2);
        double delta = (dot3(e, u3) / 6.0 - dot3(u1, u2) / 2.0) / ell2;
        double eps = (dot3(e, u4) / 24.0 - dot3(u1, u3) / 6.0 - dot3(u2, u2) / 8.0) / ell2;
        double g1 = beta;
        double g2 = gamma + 0.5 * beta * beta;
        double g3 = delta + beta * gamma + beta * beta * beta / 6.0;
        double g4 = eps + beta * delta + 0.5 * beta * beta * gamma + 0.5 * gamma * gamma +
                    beta * beta * beta * beta / 24.0;
        out[8] += w;
        out[9] += w * g1;
        out[10] += w * g2;
        out[11] += w * g3;
        out[12] += w * g4;
    }
}

/* z~_j = R z_j + T (P row-major 4x4) and, when xi is given, the vectors of
 * the step sums: u1 = omega x z~ + v, u_k = omega x u_{k-1}. */
static void source_terms(const double* zj, const double* P, const double* xi, double zt[3],
                         double u[4][3]) {
    for (int r = 0; r < 3; ++r)
        zt[r] = P[4 * r + 0] * zj[0] + P[4 * r + 1] * zj[1] + P[4 * r + 2] * zj[2] + P[4 * r + 3];
    if (xi) {
        const double* om = xi;
        const double* v = xi + 3;
        cross3(om, zt, u[0]);
        for (int r = 0; r < 3; ++r) u[0][r] += v[r];
        cross3(om, u[0], u[1]);
        cross3(om, u[1], u[2]);
        cross3(om, u[2], u[3]);
    }
}

/* All contributions of source point j, summed over every target point i. */
static void sums_for_j(const double* X, const double* FX, int64_t N,
                       const double* zj, const double* gj, int D,
                       const double* P, const orc_params* prm,
                       const double* xi, double out[ORC_NOUT]) {
    memset(out, 0, sizeof(double) * ORC_NOUT);
    double zt[3], u[4][3];
    source_terms(zj, P, xi, zt, u);
    for (int64_t i = 0; i < N; ++i)
        add_pair(X, FX, i, zt, gj, D, prm, xi ? (const double(*)[3])u : NULL, out);
}

/*
 * Per-source-point sums. For each listed source index js[q] (or every j when
 * js == NULL, in which case nq must equal M), writes ORC_NOUT doubles to
 * out_j[q*ORC_NOUT ...]: F_j, dF/domega_j[3], dF/dv_j[3], nnz_j, S0_j..S4_j
 * (the S terms are zero when xi == NULL).
 * X: N x 3, FX: N x D (may be NULL when D == 0), Z: M x 3, FZ: M x D.
 * Returns 0, or -1 on a bad argument.
 */
int orc_pair_sums_per_j(const double* X, const double* FX, int64_t N,
                        const double* Z, const double* FZ, int64_t M, int D,
                        const double* P, const orc_params* prm, const double* xi,
                        const int64_t* js, int64_t nq, double* out_j) {
    if (!X || !Z || !P || !prm || !out_j || N < 0 || M < 0 || D < 0 || nq < 0) return -1;
    if (D > 0 && (!FX || !FZ)) return -1;
    if (!js && nq != M) return -1;
    if (!(prm->ell > 0.0)) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < nq; ++q) {
        int64_t j = js ? js[q] : q;
        double o[ORC_NOUT];
        if (j < 0 || j >= M) {
            for (int r = 0; r < ORC_NOUT; ++r) o[r] = NAN;
        } else {
            sums_for_j(X, FX, N, Z + 3 * j, D > 0 ? FZ + (int64_t)D * j : NULL, D, P, prm, xi, o);
        }
        memcpy(out_j + q * ORC_NOUT, o, sizeof(o));
    }
    return 0;
}

/*
 * Whole-cloud sums: out[ORC_NOUT] = sum over j of the per-j sums, added in
 * increasing j (a fixed order, so the result does not depend on threading).
 */
int orc_pair_sums(const double* X, const double* FX, int64_t N,
                  const double* Z, const double* FZ, int64_t M, int D,
                  const double* P, const orc_params* prm, const double* xi, double* out) {
    if (!out) return -1;
    double* per = (double*)malloc(sizeof(double) * ORC_NOUT * (size_t)(M > 0 ? M : 1));
    if (!per) return -2;
    int rc = orc_pair_sums_per_j(X, FX, N, Z, FZ, M, D, P, prm, xi, NULL, M, per);
    if (rc == 0) {
        for (int r = 0; r < ORC_NOUT; ++r) out[r] = 0.0;
        for (int64_t j = 0; j < M; ++j)
            for (int r = 0; r < ORC_NOUT; ++r) out[r] += per[j * ORC_NOUT + r];
    }
    free(per);
    return rc;
}

/*
 * Grid search (Sec. 5 sparsification, in the oracle's own form): the same sums,
 * visiting for each source point only the target points of the 27 cells of
 * edge h >= r_c around it, which hold every point within the cutoff. The
 * cells are a dense grid over the bounding box of X, its edge enlarged when
 * the box would need more than ORC_GRID_MAX_CELLS cells (a wider cell still
 * holds every neighbour). Each source point's candidates are put in
 * increasing target index and passed through add_pair, so that the kept
 * pairs, the terms and the order in which they are added are those of the
 * exhaustive loop: the results are the same bits. Needs kcut in (0, 1).
 */
#define ORC_GRID_MAX_CELLS (1LL << 24)

typedef struct {
    double lo[3], h;
    int64_t n[3];
    int64_t* start;   /* n0 n1 n2 + 1 offsets into idx */
    int64_t* idx;     /* target indices sorted by cell, increasing within a cell */
} orc_grid;

static int cmp_i64(const void* a, const void* b) {
    const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

static int grid_build(const double* X, int64_t N, double rc, orc_grid* g) {
    memset(g, 0, sizeof(*g));
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            if (X[3 * i + a] < lo[a]) lo[a] = X[3 * i + a];
            if (X[3 * i + a] > hi[a]) hi[a] = X[3 * i + a];
        }
    if (N == 0)
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = 0.0;
    double h = rc;
    for (;;) {
        double cells = 1.0;
        for (int a = 0; a < 3; ++a) cells *= floor((hi[a] - lo[a]) / h) + 1.0;
        if (cells <= (double)ORC_GRID_MAX_CELLS) break;
        h *= 1.5;
    }
    g->h = h;
    int64_t total = 1;
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = lo[a];
        g->n[a] = (int64_t)floor((hi[a] - lo[a]) / h) + 1;
        total *= g->n[a];
    }
    g->start = (int64_t*)calloc((size_t)total + 1, sizeof(int64_t));
    g->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!g->start || !g->idx || !cell) {
        free(cell);
        return -2;
    }
    /* counting sort by cell, stable in i */
    for (int64_t i = 0; i < N; ++i) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int64_t)floor((X[3 * i + a] - lo[a]) / h);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= g->n[a]) c[a] = g->n[a] - 1;
        }
        cell[i] = c[0] + g->n[0] * (c[1] + g->n[1] * c[2]);
        g->start[cell[i] + 1] += 1;
    }
    for (int64_t c = 0; c < total; ++c) g->start[c + 1] += g->start[c];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)total);
    if (!fill) {
        free(cell);
        return -2;
    }
    memcpy(fill, g->start, sizeof(int64_t) * (size_t)total);
    for (int64_t i = 0; i < N; ++i) g->idx[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
    return 0;
}

static void grid_free(orc_grid* g) {
    free(g->start);
    free(g->idx);
}

/* Source point j's sums over the target points of the 27 cells around z~_j;
 * buf holds at least N entries. */
static void grid_sums_for_j(const orc_grid* g, const double* X, const double* FX, int64_t N,
                            const double* zj, const double* gj, int D, const double* P,
                            const orc_params* prm, const double* xi, int64_t* buf,
                            double out[ORC_NOUT]) {
    memset(out, 0, sizeof(double) * ORC_NOUT);
    double zt[3], u[4][3];
    source_terms(zj, P, xi, zt, u);
    int64_t c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
        const double q = floor((zt[a] - g->lo[a]) / g->h);
        /* cells c with |c - q| <= 1, clipped to the grid (q may lie outside it) */
        double lo = q - 1.0, hi = q + 1.0;
        if (lo < 0.0) lo = 0.0;
        if (hi > (double)(g->n[a] - 1)) hi = (double)(g->n[a] - 1);
        if (!(lo <= hi)) return; /* no cell within reach (or a non-finite point) */
        c0[a] = (int64_t)lo;
        c1[a] = (int64_t)hi;
    }
    int64_t k = 0;
    for (int64_t cz = c0[2]; cz <= c1[2]; ++cz)
        for (int64_t cy = c0[1]; cy <= c1[1]; ++cy)
            for (int64_t cx = c0[0]; cx <= c1[0]; ++cx) {
                const int64_t c = cx + g->n[0] * (cy + g->n[1] * cz);
                for (int64_t p = g->start[c]; p < g->start[c + 1]; ++p) buf[k++] = g->idx[p];
            }
    qsort(buf, (size_t)k, sizeof(int64_t), cmp_i64);
    (void)N;
    for (int64_t q = 0; q < k; ++q)
        add_pair(X, FX, buf[q], zt, gj, D, prm, xi ? (const double(*)[3])u : NULL, out);
}

/* orc_pair_sums_per_j with the grid search. Returns 0, -1 on a bad argument
 * (including kcut outside (0, 1)), -2 when memory runs out. */
int orc_pair_sums_grid_per_j(const double* X, const double* FX, int64_t N,
                             const double* Z, const double* FZ, int64_t M, int D,
                             const double* P, const orc_params* prm, const double* xi,
                             const int64_t* js, int64_t nq, double* out_j) {
    if (!X || !Z || !P || !prm || !out_j || N < 0 || M < 0 || D < 0 || nq < 0) return -1;
    if (D > 0 && (!FX || !FZ)) return -1;
    if (!js && nq != M) return -1;
    if (!(prm->ell > 0.0) || !(prm->kcut > 0.0 && prm->kcut < 1.0)) return -1;
    /* a cell edge a little above r_c: two points within r_c of each other
     * then lie in neighbouring cells even after the rounding of the cell
     * coordinates */
    const double rc = prm->ell * sqrt(2.0 * log(1.0 / prm->kcut)) * (1.0 + 1e-9);
    orc_grid g;
    int rc_build = grid_build(X, N, rc, &g);
    if (rc_build != 0) {
        grid_free(&g);
        return rc_build;
    }
    int fail = 0;
#pragma omp parallel
    {
        int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < nq; ++q) {
            int64_t j = js ? js[q] : q;
            double o[ORC_NOUT];
            if (!buf || j < 0 || j >= M) {
                for (int r = 0; r < ORC_NOUT; ++r) o[r] = NAN;
            } else {
                grid_sums_for_j(&g, X, FX, N, Z + 3 * j, D > 0 ? FZ + (int64_t)D * j : NULL, D,
                                P, prm, xi, buf, o);
            }
            memcpy(out_j + q * ORC_NOUT, o, sizeof(o));
        }
        free(buf);
    }
    grid_free(&g);
    return fail ? -2 : 0;
}

/* orc_pair_sums with the grid search (same fixed order over j). */
int orc_pair_sums_grid(const double* X, const double* FX, int64_t N,
                       const double* Z, const double* FZ, int64_t M, int D,
                       const double* P, const orc_params* prm, const double* xi, double* out) {
    if (!out) return -1;
    double* per = (double*)malloc(sizeof(double) * ORC_NOUT * (size_t)(M > 0 ? M : 1));
    if (!per) return -2;
    int rc = orc_pair_sums_grid_per_j(X, FX, N, Z, FZ, M, D, P, prm, xi, NULL, M, per);
    if (rc == 0) {
        for (int r = 0; r < ORC_NOUT; ++r) out[r] = 0.0;
        for (int64_t j = 0; j < M; ++j)
            for (int r = 0; r < ORC_NOUT; ++r) out[r] += per[j * ORC_NOUT + r];
    }
    free(per);
    return rc;
}

/* Threads the oracle uses (for reporting the CPU baseline). */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
