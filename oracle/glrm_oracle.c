/*
 * FP64 CPU oracle for the generalized low rank model (GLRM) fitting method of
 * Udell, Horn, Zadeh and Boyd, "Generalized Low Rank Models" (arXiv 1410.0342).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  It shares no code, header, table or helper
 * with the CUDA library, and the product path never calls it: only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Problem (eq. gpca, Section 4; eq. apca, Section 5):
 *     minimize  sum_{(i,j) in Omega} L_j(x_i . y_j, A_ij) + sum_i r(x_i) + sum_j rt(y_j)
 * with X (m x k, rows x_i) and Y (k x n, columns y_j).  Y is held here as its
 * transpose Yt (n x k, row j = y_j), both row-major.
 *
 * Everything is double precision, loops are plain and run in index order.
 * OpenMP only spreads independent rows (X-step) or columns (Y-step) over
 * threads, which the paper names as the natural parallelism of the method
 * (Section 7.2, "Choosing a step size", last paragraph); every result is
 * written to its own slot and every sum runs in a fixed order, so the output
 * does not depend on the thread count.
 *
 * Readings of the paper taken where it is silent or inconsistent:
 *  - quadratic loss is (u-a)^2 and the quadratic regulariser gamma*||x||^2
 *    (eq. qpca, Section 2);
 *  - Huber with threshold delta: 0.5 x^2 if |x| <= delta, else
 *    delta*(|x| - delta/2); delta = 1 is the paper's function (Section 4.3);
 *  - at a kink of the hinge / ordinal hinge a term's derivative is 0;
 *  - Boolean data is coded -1/+1 and decodes to +1 when u >= 0;
 *  - an ordinal decode tie goes to the smaller level;
 *  - the step-size safeguard (Section 7.2) rejects a step that increases the
 *    row (column) objective: the factor is kept and alpha shrinks by 0.7; a
 *    step that does not increase it is kept and alpha grows by 1.05;
 *  - alpha starts at 1/max(n_i, 1) (scale 1 divided by the observation count);
 *  - the row objective uses the general regulariser r(x), which is +inf for
 *    the nonnegativity indicator at an infeasible point.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { LOSS_QUAD = 0, LOSS_HUBER = 1, LOSS_HINGE = 2, LOSS_LOGISTIC = 3, LOSS_ORDINAL = 4,
       LOSS_L1 = 5, LOSS_QUANTILE = 6 };
enum { REG_ZERO = 0, REG_QUAD = 1, REG_L1 = 2, REG_NONNEG = 3 };

static double pos(double v) { return v > 0.0 ? v : 0.0; }

/* ---------------------------------------------------------------- losses */

/* L(u, a).  Quadratic (eq. qpca), Huber (Section 4.3, "Huber PCA"), hinge
 * (Section 5.2, "Boolean PCA"), logistic (Section 5.2, "Logistic PCA"),
 * ordinal hinge (eq. ord-pca), l1 |a - u| (Section 4.2, robust PCA) and the
 * quantile loss alpha (a - u)_+ + (1 - alpha) (u - a)_+ with alpha = param
 * (Section 4.2, "Quantile PCA"). */
double oracle_loss(int kind, double param, int levels, double u, double a)
{
    switch (kind) {
    case LOSS_QUAD:
        return (u - a) * (u - a);
    case LOSS_HUBER: {
        double x = fabs(u - a), d = param;
        return x <= d ? 0.5 * x * x : d * (x - 0.5 * d);
    }
    case LOSS_HINGE:
        return pos(1.0 - a * u);
    case LOSS_LOGISTIC: {
        /* log(1 + exp(-a u)), evaluated without overflow */
        double z = -a * u;
        return z > 0.0 ? z + log1p(exp(-z)) : log1p(exp(z));
    }
    case LOSS_ORDINAL: {
        double s = 0.0;
        int lev = (int)a;
        for (int ap = 1; ap <= lev - 1; ++ap) s += pos(1.0 - u + ap);
        for (int ap = lev + 1; ap <= levels; ++ap) s += pos(1.0 + u - ap);
        return s;
    }
    case LOSS_L1:
        return fabs(a - u);
    case LOSS_QUANTILE:
        return param * pos(a - u) + (1.0 - param) * pos(u - a);
    }
    return NAN;
}

/* dL/du (a subgradient at kinks, taken as 0 there). */
double oracle_dloss(int kind, double param, int levels, double u, double a)
{
    switch (kind) {
    case LOSS_QUAD:
        return 2.0 * (u - a);
    case LOSS_HUBER: {
        double x = u - a, d = param;
        if (x > d) return d;
        if (x < -d) return -d;
        return x;
    }
    case LOSS_HINGE:
        return (1.0 - a * u) > 0.0 ? -a : 0.0;
    case LOSS_LOGISTIC:
        /* d/du log(1+exp(-a u)) = -a / (1 + exp(a u)) */
        return -a / (1.0 + exp(a * u));
    case LOSS_ORDINAL: {
        double s = 0.0;
        int lev = (int)a;
        for (int ap = 1; ap <= lev - 1; ++ap)
            if (1.0 - u + ap > 0.0) s -= 1.0;
        for (int ap = lev + 1; ap <= levels; ++ap)
            if (1.0 + u - ap > 0.0) s += 1.0;
        return s;
    }
    case LOSS_L1:
        return u > a ? 1.0 : (u < a ? -1.0 : 0.0);
    case LOSS_QUANTILE:
        return u > a ? 1.0 - param : (u < a ? -param : 0.0);
    }
    return NAN;
}

/* Imputation (Section 5.3): argmin over the loss's domain of L(u, a).
 * Real-valued losses (quadratic, Huber, l1, quantile) return u; Boolean losses return sign(u) with sign(0)=+1;
 * the ordinal hinge is minimised by trying every level 1..d (ties to the
 * smaller level). */
double oracle_decode(int kind, int levels, double u)
{
    switch (kind) {
    case LOSS_QUAD:
    case LOSS_HUBER:
    case LOSS_L1:
    case LOSS_QUANTILE:
        return u;
    case LOSS_HINGE:
    case LOSS_LOGISTIC:
        return u >= 0.0 ? 1.0 : -1.0;
    case LOSS_ORDINAL: {
        int best = 1;
        double bestv = oracle_loss(LOSS_ORDINAL, 0.0, levels, u, 1.0);
        for (int a = 2; a <= levels; ++a) {
            double v = oracle_loss(LOSS_ORDINAL, 0.0, levels, u, (double)a);
            if (v < bestv) { bestv = v; best = a; }
        }
        return (double)best;
    }
    }
    return NAN;
}

/* ----------------------------------------------------------- regularisers */

/* r(x) for the quadratic (gamma ||x||^2, eq. qpca), l1 (lambda ||x||_1,
 * Section 3.2 "Sparse PCA"), nonnegativity indicator (Section 3.2, "NNMF") and
 * zero regularisers. */
double oracle_reg(int kind, double w, int k, const double *x)
{
    double s = 0.0;
    switch (kind) {
    case REG_ZERO:
        return 0.0;
    case REG_QUAD:
        for (int c = 0; c < k; ++c) s += x[c] * x[c];
        return w * s;
    case REG_L1:
        for (int c = 0; c < k; ++c) s += fabs(x[c]);
        return w * s;
    case REG_NONNEG:
        for (int c = 0; c < k; ++c)
            if (x[c] < 0.0) return INFINITY;
        return 0.0;
    }
    return NAN;
}

/* prox_{alpha r}(z) = argmin_x alpha r(x) + 0.5 ||x - z||^2 (Section 7.2,
 * "Proximal gradient method").  All four regularisers are separable, so the
 * minimiser is taken coordinate by coordinate:
 *   quadratic:  alpha w x^2 + 0.5 (x-z)^2  ->  x = z / (1 + 2 alpha w)
 *   l1:         alpha w |x| + 0.5 (x-z)^2  ->  soft threshold at alpha w
 *   nonneg:     projection onto x >= 0     ->  max(z, 0)
 *   zero:       x = z                                                    */
void oracle_prox(int kind, double w, double alpha, int k, const double *z, double *out)
{
    for (int c = 0; c < k; ++c) {
        double v = z[c];
        switch (kind) {
        case REG_ZERO:
            out[c] = v;
            break;
        case REG_QUAD:
            out[c] = v / (1.0 + 2.0 * alpha * w);
            break;
        case REG_L1: {
            double t = alpha * w;
            out[c] = v > t ? v - t : (v < -t ? v + t : 0.0);
            break;
        }
        case REG_NONNEG:
            out[c] = v > 0.0 ? v : 0.0;
            break;
        default:
            out[c] = NAN;
        }
    }
}

/* Offsets (Section 3.4, "Offsets and scaling"): the model's factors carry one
 * extra coordinate, here the last one (index k-1).  The regulariser of a row
 * of X becomes r'(x) = r(x_1 .. x_{k-1}) if x_k = 1, +inf otherwise, and that
 * of a column of Y becomes r~'(y) = r~(y_1 .. y_{k-1}): the offset column of X
 * is the constant 1 and the offset row of Y (the column offsets mu_j) is not
 * penalised.  role: 0 none, 1 a row of X, 2 a column of Y. */
static double reg_vec(int kind, double w, int k, const double *x, int role)
{
    if (role == 0) return oracle_reg(kind, w, k, x);
    double r = oracle_reg(kind, w, k - 1, x);
    if (role == 1 && x[k - 1] != 1.0) return INFINITY;
    return r;
}

/* prox of the regulariser above: r's prox on the first k-1 coordinates; the
 * last one is projected onto {1} (a row of X) or left as it is (a column of Y). */
static void prox_vec(int kind, double w, double alpha, int k, const double *z, double *out, int role)
{
    if (role == 0) {
        oracle_prox(kind, w, alpha, k, z, out);
        return;
    }
    oracle_prox(kind, w, alpha, k - 1, z, out);
    out[k - 1] = role == 1 ? 1.0 : z[k - 1];
}

/* ------------------------------------------------------------- Omega lists */

/* The observed set is given as coordinate triples (row, col, value) sorted by
 * row then column.  From it the oracle builds, by counting, its own list of
 * the entries of every row (columns ascending) and of every column (rows
 * ascending). */
typedef struct {
    int64_t m, n, nnz;
    int64_t *rstart;  /* m+1 */
    int32_t *rcol;    /* nnz, column of each entry of the row lists */
    double *rval;
    int64_t *cstart;  /* n+1 */
    int32_t *crow;    /* nnz, row of each entry of the column lists */
    double *cval;
} omega_lists;

static void lists_free(omega_lists *L)
{
    free(L->rstart); free(L->rcol); free(L->rval);
    free(L->cstart); free(L->crow); free(L->cval);
}

static int lists_build(omega_lists *L, int64_t m, int64_t n, int64_t nnz,
                       const int32_t *row, const int32_t *col, const double *val)
{
    L->m = m; L->n = n; L->nnz = nnz;
    L->rstart = calloc((size_t)m + 1, sizeof(int64_t));
    L->cstart = calloc((size_t)n + 1, sizeof(int64_t));
    L->rcol = malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    L->rval = malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    L->crow = malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    L->cval = malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    if (!L->rstart || !L->cstart || !L->rcol || !L->rval || !L->crow || !L->cval) return -1;
    for (int64_t e = 0; e < nnz; ++e) {
        if (row[e] < 0 || row[e] >= m || col[e] < 0 || col[e] >= n) return -2;
        L->rstart[row[e] + 1]++;
        L->cstart[col[e] + 1]++;
    }
    for (int64_t i = 0; i < m; ++i) L->rstart[i + 1] += L->rstart[i];
    for (int64_t j = 0; j < n; ++j) L->cstart[j + 1] += L->cstart[j];
    int64_t *rfill = malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
    int64_t *cfill = malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (!rfill || !cfill) { free(rfill); free(cfill); return -1; }
    memcpy(rfill, L->rstart, sizeof(int64_t) * (size_t)m);
    memcpy(cfill, L->cstart, sizeof(int64_t) * (size_t)n);
    /* entries arrive sorted by (row, col): the fills below keep each row's
     * columns ascending and each column's rows ascending */
    for (int64_t e = 0; e < nnz; ++e) {
        int64_t p = rfill[row[e]]++;
        L->rcol[p] = col[e];
        L->rval[p] = val[e];
        int64_t q = cfill[col[e]]++;
        L->crow[q] = row[e];
        L->cval[q] = val[e];
    }
    free(rfill); free(cfill);
    return 0;
}

static double dot(int k, const double *a, const double *b)
{
    double s = 0.0;
    for (int c = 0; c < k; ++c) s += a[c] * b[c];
    return s;
}

/* Loss part of the objective of one factor vector v against the list of its
 * observed entries: sum_e L(v . W[idx[e]], a[e]).  In the X-step v = x_i and
 * W = Yt, and an entry's loss is that of its column idx[e]; in the Y-step
 * v = y_j, W = X, and every entry uses column j's loss (fixed_col = j). */
typedef struct {
    const int32_t *kind;
    const double *param;
    const int32_t *levels;
    const double *w; /* per-column loss weights (Section 4.3 scaling); NULL: all 1 */
} loss_table;

static double col_weight(const loss_table *lt, int64_t j) { return lt->w ? lt->w[j] : 1.0; }

static double list_loss(int k, const double *v, const double *W, const int32_t *idx,
                        const double *a, int64_t cnt, const loss_table *lt, int64_t fixed_col)
{
    double s = 0.0;
    for (int64_t e = 0; e < cnt; ++e) {
        int64_t j = fixed_col >= 0 ? fixed_col : idx[e];
        double u = dot(k, v, W + (int64_t)idx[e] * k);
        s += col_weight(lt, j) * oracle_loss(lt->kind[j], lt->param[j], lt->levels[j], u, a[e]);
    }
    return s;
}

/* One proximal-gradient update of v with the step-size safeguard
 * (Section 7.2, "Proximal gradient method" and "Choosing a step size"):
 *   g     = sum_e L'(v . w_e, a_e) w_e
 *   v+    = prox_{alpha r}(v - alpha g)
 *   keep v+ and alpha *= 1.05 if f(v+) <= f(v), else keep v and alpha *= 0.7,
 * with f(v) = sum_e L(v . w_e, a_e) + r(v).
 * Returns 1 when the step was accepted.  *fkept receives f of the kept vector. */
static int update_vector(int k, double *v, double *alpha, const double *W, const int32_t *idx,
                         const double *a, int64_t cnt, const loss_table *lt, int64_t fixed_col,
                         int rkind, double rw, int role, double *fkept, double *rkept)
{
    double g[k], z[k], vp[k];
    for (int c = 0; c < k; ++c) g[c] = 0.0;
    for (int64_t e = 0; e < cnt; ++e) {
        int64_t j = fixed_col >= 0 ? fixed_col : idx[e];
        const double *w = W + (int64_t)idx[e] * k;
        double u = dot(k, v, w);
        double r = col_weight(lt, j) * oracle_dloss(lt->kind[j], lt->param[j], lt->levels[j], u, a[e]);
        for (int c = 0; c < k; ++c) g[c] += r * w[c];
    }
    for (int c = 0; c < k; ++c) z[c] = v[c] - (*alpha) * g[c];
    prox_vec(rkind, rw, *alpha, k, z, vp, role);
    double r_old = reg_vec(rkind, rw, k, v, role);
    double r_new = reg_vec(rkind, rw, k, vp, role);
    double f_old = list_loss(k, v, W, idx, a, cnt, lt, fixed_col) + r_old;
    double f_new = list_loss(k, vp, W, idx, a, cnt, lt, fixed_col) + r_new;
    if (f_new <= f_old) {
        for (int c = 0; c < k; ++c) v[c] = vp[c];
        *alpha *= 1.05;
        *fkept = f_new;
        *rkept = r_new;
        return 1;
    }
    *alpha *= 0.7;
    *fkept = f_old;
    *rkept = r_old;
    return 0;
}

static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Full objective (eq. gpca):  sum over Omega of L (rows ascending, then each
 * row's columns ascending) + sum_i r(x_i) + sum_j rt(y_j). */
static double objective_lists(const omega_lists *L, int k, const double *X, const double *Yt,
                              const loss_table *lt, int rxk, double rxw, int ryk, double ryw, int offset)
{
    double *rowsum = malloc(sizeof(double) * (size_t)(L->m ? L->m : 1));
    int64_t i;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < L->m; ++i)
        rowsum[i] = list_loss(k, X + i * k, Yt, L->rcol + L->rstart[i], L->rval + L->rstart[i],
                              L->rstart[i + 1] - L->rstart[i], lt, -1);
    double F = 0.0;
    for (i = 0; i < L->m; ++i) F += rowsum[i];
    for (i = 0; i < L->m; ++i) F += reg_vec(rxk, rxw, k, X + i * k, offset ? 1 : 0);
    for (int64_t j = 0; j < L->n; ++j) F += reg_vec(ryk, ryw, k, Yt + j * k, offset ? 2 : 0);
    free(rowsum);
    return F;
}

double oracle_objective(int64_t m, int64_t n, int k, int64_t nnz, const int32_t *row,
                        const int32_t *col, const double *val, const int32_t *lkind,
                        const double *lparam, const int32_t *llevels, int rxk, double rxw,
                        int ryk, double ryw, int offset, const double *wcol, const double *X,
                        const double *Yt, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    if (lists_build(&L, m, n, nnz, row, col, val)) { lists_free(&L); return NAN; }
    set_threads(nthreads);
    loss_table lt = { lkind, lparam, llevels, wcol };
    double F = objective_lists(&L, k, X, Yt, &lt, rxk, rxw, ryk, ryw, offset);
    lists_free(&L);
    return F;
}

/* Loss part of the gradient (Section 7.2, "Gradient method"):
 *   GX[i] = sum_{j in Omega_i} L'_j(x_i . y_j, A_ij) y_j
 *   GYt[j] = sum_{i in Omega_j} L'_j(x_i . y_j, A_ij) x_i               */
int oracle_gradient(int64_t m, int64_t n, int k, int64_t nnz, const int32_t *row,
                    const int32_t *col, const double *val, const int32_t *lkind,
                    const double *lparam, const int32_t *llevels, const double *wcol,
                    const double *X, const double *Yt, double *GX, double *GYt, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    int rc = lists_build(&L, m, n, nnz, row, col, val);
    if (rc) { lists_free(&L); return rc; }
    set_threads(nthreads);
    int64_t i, j;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < m; ++i) {
        double *g = GX + i * k;
        for (int c = 0; c < k; ++c) g[c] = 0.0;
        for (int64_t e = L.rstart[i]; e < L.rstart[i + 1]; ++e) {
            int32_t jj = L.rcol[e];
            double u = dot(k, X + i * k, Yt + (int64_t)jj * k);
            double r = (wcol ? wcol[jj] : 1.0) * oracle_dloss(lkind[jj], lparam[jj], llevels[jj], u, L.rval[e]);
            for (int c = 0; c < k; ++c) g[c] += r * Yt[(int64_t)jj * k + c];
        }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (j = 0; j < n; ++j) {
        double *h = GYt + j * k;
        for (int c = 0; c < k; ++c) h[c] = 0.0;
        for (int64_t e = L.cstart[j]; e < L.cstart[j + 1]; ++e) {
            int32_t ii = L.crow[e];
            double u = dot(k, X + (int64_t)ii * k, Yt + j * k);
            double r = (wcol ? wcol[j] : 1.0) * oracle_dloss(lkind[j], lparam[j], llevels[j], u, L.cval[e]);
            for (int c = 0; c < k; ++c) h[c] += r * X[(int64_t)ii * k + c];
        }
    }
    lists_free(&L);
    return 0;
}

/* Magnitude of the terms of each gradient coordinate (the scale of the
 * rounding error of any summation of them):
 *   SX[i] = sum_{j in Omega_i} |L'_j(x_i . y_j, A_ij)| |y_j|   (elementwise)
 *   SYt[j] = sum_{i in Omega_j} |L'_j(x_i . y_j, A_ij)| |x_i|
 * Same loops as oracle_gradient with absolute values. */
int oracle_gradient_abs(int64_t m, int64_t n, int k, int64_t nnz, const int32_t *row,
                        const int32_t *col, const double *val, const int32_t *lkind,
                        const double *lparam, const int32_t *llevels, const double *X,
                        const double *Yt, double *SX, double *SYt, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    int rc = lists_build(&L, m, n, nnz, row, col, val);
    if (rc) { lists_free(&L); return rc; }
    set_threads(nthreads);
    int64_t i, j;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < m; ++i) {
        double *g = SX + i * k;
        for (int c = 0; c < k; ++c) g[c] = 0.0;
        for (int64_t e = L.rstart[i]; e < L.rstart[i + 1]; ++e) {
            int32_t jj = L.rcol[e];
            double u = dot(k, X + i * k, Yt + (int64_t)jj * k);
            double r = fabs(oracle_dloss(lkind[jj], lparam[jj], llevels[jj], u, L.rval[e]));
            for (int c = 0; c < k; ++c) g[c] += r * fabs(Yt[(int64_t)jj * k + c]);
        }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (j = 0; j < n; ++j) {
        double *h = SYt + j * k;
        for (int c = 0; c < k; ++c) h[c] = 0.0;
        for (int64_t e = L.cstart[j]; e < L.cstart[j + 1]; ++e) {
            int32_t ii = L.crow[e];
            double u = dot(k, X + (int64_t)ii * k, Yt + j * k);
            double r = fabs(oracle_dloss(lkind[j], lparam[j], llevels[j], u, L.cval[e]));
            for (int c = 0; c < k; ++c) h[c] += r * fabs(X[(int64_t)ii * k + c]);
        }
    }
    lists_free(&L);
    return 0;
}

/* How far each gradient coordinate can move when every product u = x_i . y_j
 * is perturbed by at most delta = u_rel * sum_c |x_ic y_jc| (the rounding
 * bound of a low-precision dot product):
 *   VX[i] = sum_{j in Omega_i} (L'_j(u + delta) - L'_j(u - delta)) |y_j|
 *   VYt[j] = sum_{i in Omega_j} (L'_j(u + delta) - L'_j(u - delta)) |x_i|
 * Every loss here is convex, so L' is nondecreasing and the difference is
 * the variation of L' over [u - delta, u + delta]: the jump of the
 * subgradient when a kink lies in that interval (hinge, ordinal hinge), about
 * 2 delta L'' for smooth losses. */
int oracle_gradient_variation(int64_t m, int64_t n, int k, int64_t nnz, const int32_t *row,
                              const int32_t *col, const double *val, const int32_t *lkind,
                              const double *lparam, const int32_t *llevels, const double *X,
                              const double *Yt, double u_rel, double *VX, double *VYt,
                              int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    int rc = lists_build(&L, m, n, nnz, row, col, val);
    if (rc) { lists_free(&L); return rc; }
    set_threads(nthreads);
    int64_t i, j;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < m; ++i) {
        double *g = VX + i * k;
        for (int c = 0; c < k; ++c) g[c] = 0.0;
        for (int64_t e = L.rstart[i]; e < L.rstart[i + 1]; ++e) {
            int32_t jj = L.rcol[e];
            const double *x = X + i * k, *y = Yt + (int64_t)jj * k;
            double u = dot(k, x, y), a = 0.0;
            for (int c = 0; c < k; ++c) a += fabs(x[c] * y[c]);
            double d = u_rel * a;
            double v = oracle_dloss(lkind[jj], lparam[jj], llevels[jj], u + d, L.rval[e]) -
                       oracle_dloss(lkind[jj], lparam[jj], llevels[jj], u - d, L.rval[e]);
            for (int c = 0; c < k; ++c) g[c] += v * fabs(y[c]);
        }
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (j = 0; j < n; ++j) {
        double *h = VYt + j * k;
        for (int c = 0; c < k; ++c) h[c] = 0.0;
        for (int64_t e = L.cstart[j]; e < L.cstart[j + 1]; ++e) {
            int32_t ii = L.crow[e];
            const double *x = X + (int64_t)ii * k, *y = Yt + j * k;
            double u = dot(k, x, y), a = 0.0;
            for (int c = 0; c < k; ++c) a += fabs(x[c] * y[c]);
            double d = u_rel * a;
            double v = oracle_dloss(lkind[j], lparam[j], llevels[j], u + d, L.cval[e]) -
                       oracle_dloss(lkind[j], lparam[j], llevels[j], u - d, L.cval[e]);
            for (int c = 0; c < k; ++c) h[c] += v * fabs(x[c]);
        }
    }
    lists_free(&L);
    return 0;
}

/* Alternating proximal-gradient sweeps (Algorithm 2 with the proximal
 * gradient update and the per-row/per-column step-size rule of Section 7.2).
 * Sweep t updates every row x_i against Y^{t-1}, then every column y_j against
 * the new X^t.  alpha_x (m) and alpha_y (n) carry the step sizes between
 * calls; a caller starting a fit sets them to 1/max(n_i,1) and 1/max(m_j,1).
 * history[t] receives the objective after sweep t; accepts[2t], accepts[2t+1]
 * receive the number of accepted row and column steps of sweep t. */
int oracle_proxgrad(int64_t m, int64_t n, int k, int64_t nnz, const int32_t *row,
                    const int32_t *col, const double *val, const int32_t *lkind,
                    const double *lparam, const int32_t *llevels, int rxk, double rxw, int ryk,
                    double ryw, int offset, const double *wcol, double *X, double *Yt, double *alpha_x,
                    double *alpha_y, int nsweeps, double *history, int64_t *accepts, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    int rc = lists_build(&L, m, n, nnz, row, col, val);
    if (rc) { lists_free(&L); return rc; }
    set_threads(nthreads);
    loss_table lt = { lkind, lparam, llevels, wcol };
    double *fx = malloc(sizeof(double) * (size_t)(m ? m : 1));
    double *rx = malloc(sizeof(double) * (size_t)(m ? m : 1));
    double *fy = malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *ry = malloc(sizeof(double) * (size_t)(n ? n : 1));
    int *ax = malloc(sizeof(int) * (size_t)(m ? m : 1));
    int *ay = malloc(sizeof(int) * (size_t)(n ? n : 1));
    for (int t = 0; t < nsweeps; ++t) {
        int64_t i, j;
#pragma omp parallel for schedule(dynamic, 64)
        for (i = 0; i < m; ++i) {
            int64_t b = L.rstart[i];
            ax[i] = update_vector(k, X + i * k, alpha_x + i, Yt, L.rcol + b, L.rval + b,
                                  L.rstart[i + 1] - b, &lt, -1, rxk, rxw, offset ? 1 : 0, fx + i, rx + i);
        }
#pragma omp parallel for schedule(dynamic, 4)
        for (j = 0; j < n; ++j) {
            int64_t b = L.cstart[j];
            ay[j] = update_vector(k, Yt + j * k, alpha_y + j, X, L.crow + b, L.cval + b,
                                  L.cstart[j + 1] - b, &lt, j, ryk, ryw, offset ? 2 : 0, fy + j, ry + j);
        }
        int64_t na = 0, nb = 0;
        for (i = 0; i < m; ++i) na += ax[i];
        for (j = 0; j < n; ++j) nb += ay[j];
        if (accepts) { accepts[2 * t] = na; accepts[2 * t + 1] = nb; }
        if (history)
            history[t] = objective_lists(&L, k, X, Yt, &lt, rxk, rxw, ryk, ryw, offset);
    }
    free(fx); free(rx); free(fy); free(ry); free(ax); free(ay);
    lists_free(&L);
    return 0;
}

/* Cholesky factorisation G = C C^T of a symmetric positive definite k x k
 * matrix (lower triangle of C written over G), then the two triangular solves
 * C w = b and C^T x = w.  Textbook column-by-column algorithm. */
static int chol_solve(int k, double *G, double *b)
{
    for (int c = 0; c < k; ++c) {
        double d = G[c * k + c];
        for (int p = 0; p < c; ++p) d -= G[c * k + p] * G[c * k + p];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        G[c * k + c] = d;
        for (int r = c + 1; r < k; ++r) {
            double s = G[r * k + c];
            for (int p = 0; p < c; ++p) s -= G[r * k + p] * G[c * k + p];
            G[r * k + c] = s / d;
        }
    }
    for (int r = 0; r < k; ++r) {
        double s = b[r];
        for (int p = 0; p < r; ++p) s -= G[r * k + p] * b[p];
        b[r] = s / G[r * k + r];
    }
    for (int r = k - 1; r >= 0; --r) {
        double s = b[r];
        for (int p = r + 1; p < k; ++p) s -= G[p * k + r] * b[p];
        b[r] = s / G[r * k + r];
    }
    return 0;
}

/* Exact minimisation of sum_e (v . w_e - a_e)^2 + gamma ||v||^2 over v:
 * (sum_e w_e w_e^T + gamma I) v = sum_e a_e w_e  (Section 2.4, "Parallelizing
 * alternating minimization" and "Caching factorizations", with the Gram matrix
 * restricted to the observed entries as in Section 2.5). */
static int solve_vector(int k, double *v, const double *W, const int32_t *idx, const double *a,
                        int64_t cnt, double gamma)
{
    double G[k * k], b[k];
    for (int p = 0; p < k * k; ++p) G[p] = 0.0;
    for (int c = 0; c < k; ++c) b[c] = 0.0;
    for (int64_t e = 0; e < cnt; ++e) {
        const double *w = W + (int64_t)idx[e] * k;
        for (int r = 0; r < k; ++r) {
            b[r] += a[e] * w[r];
            for (int c = 0; c < k; ++c) G[r * k + c] += w[r] * w[c];
        }
    }
    for (int c = 0; c < k; ++c) G[c * k + c] += gamma;
    if (chol_solve(k, G, b)) return -1;
    for (int c = 0; c < k; ++c) v[c] = b[c];
    return 0;
}

/* Alternating minimisation for quadratic loss and quadratic regularisation
 * (Algorithm 1 with the closed-form row and column problems): every x_i is
 * the exact minimiser against Y^{t-1}, then every y_j against X^t.
 * history[t] receives the objective (quadratic loss, gamma ||.||^2 on both
 * factors) after sweep t. */
int oracle_als(int64_t m, int64_t n, int k, int64_t nnz, const int32_t *row, const int32_t *col,
               const double *val, double gamma, double *X, double *Yt, int nsweeps,
               double *history, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    int rc = lists_build(&L, m, n, nnz, row, col, val);
    if (rc) { lists_free(&L); return rc; }
    set_threads(nthreads);
    int32_t *kind = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    double *param = malloc(sizeof(double) * (size_t)(n ? n : 1));
    int32_t *lev = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    for (int64_t j = 0; j < n; ++j) { kind[j] = LOSS_QUAD; param[j] = 0.0; lev[j] = 0; }
    loss_table lt = { kind, param, lev, NULL };
    int bad = 0;
    for (int t = 0; t < nsweeps && !bad; ++t) {
        int64_t i, j;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
        for (i = 0; i < m; ++i) {
            int64_t b = L.rstart[i];
            bad |= solve_vector(k, X + i * k, Yt, L.rcol + b, L.rval + b, L.rstart[i + 1] - b, gamma) != 0;
        }
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
        for (j = 0; j < n; ++j) {
            int64_t b = L.cstart[j];
            bad |= solve_vector(k, Yt + j * k, X, L.crow + b, L.cval + b, L.cstart[j + 1] - b, gamma) != 0;
        }
        if (history)
            history[t] = objective_lists(&L, k, X, Yt, &lt, REG_QUAD, gamma, REG_QUAD, gamma, 0);
    }
    free(kind); free(param); free(lev);
    lists_free(&L);
    return bad ? -3 : 0;
}

/* Prox-prox update of one factor vector for quadratic loss (Section 7.2,
 * "Prox-prox method", with the cached factorisation of Section 7.3): with
 * f(v) = sum_e (v . w_e - a_e)^2, G = sum_e w_e w_e^T and b = sum_e a_e w_e,
 *   prox_{alpha f}(v) = argmin_v' alpha f(v') + 1/2 ||v' - v||^2
 *                     = (2 alpha G + I)^{-1} (2 alpha b + v),
 * then v <- prox_{alpha r}(prox_{alpha f}(v)), `inner` times with the same
 * factorisation of 2 alpha G + I. */
static int proxprox_vector(int k, double *v, const double *W, const int32_t *idx, const double *a,
                           int64_t cnt, double alpha, int inner, int rkind, double rw)
{
    double G[k * k], Gc[k * k], b[k], rhs[k];
    for (int p = 0; p < k * k; ++p) G[p] = 0.0;
    for (int c = 0; c < k; ++c) b[c] = 0.0;
    for (int64_t e = 0; e < cnt; ++e) {
        const double *w = W + (int64_t)idx[e] * k;
        for (int r = 0; r < k; ++r) {
            b[r] += a[e] * w[r];
            for (int c = 0; c < k; ++c) G[r * k + c] += w[r] * w[c];
        }
    }
    for (int t = 0; t < inner; ++t) {
        /* the factorisation is recomputed here for plainness; it does not
         * change between the inner iterations */
        for (int p = 0; p < k * k; ++p) Gc[p] = 2.0 * alpha * G[p];
        for (int c = 0; c < k; ++c) Gc[c * k + c] += 1.0;
        for (int c = 0; c < k; ++c) rhs[c] = 2.0 * alpha * b[c] + v[c];
        if (chol_solve(k, Gc, rhs)) return -1;
        oracle_prox(rkind, rw, alpha, k, rhs, v);
    }
    return 0;
}

/* Alternating prox-prox sweeps for quadratic loss and any regulariser: every
 * row x_i takes `inner` prox-prox updates against Y^{t-1}, then every column
 * y_j against X^t.  history[t] receives the objective after sweep t. */
int oracle_proxprox(int64_t m, int64_t n, int k, int64_t nnz, const int32_t *row, const int32_t *col,
                    const double *val, int rxk, double rxw, int ryk, double ryw, double alpha, int inner,
                    double *X, double *Yt, int nsweeps, double *history, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    int rc = lists_build(&L, m, n, nnz, row, col, val);
    if (rc) { lists_free(&L); return rc; }
    set_threads(nthreads);
    int32_t *kind = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    double *param = malloc(sizeof(double) * (size_t)(n ? n : 1));
    int32_t *lev = malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    for (int64_t j = 0; j < n; ++j) { kind[j] = LOSS_QUAD; param[j] = 0.0; lev[j] = 0; }
    loss_table lt = { kind, param, lev, NULL };
    int bad = 0;
    for (int t = 0; t < nsweeps && !bad; ++t) {
        int64_t i, j;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
        for (i = 0; i < m; ++i) {
            int64_t b = L.rstart[i];
            bad |= proxprox_vector(k, X + i * k, Yt, L.rcol + b, L.rval + b, L.rstart[i + 1] - b, alpha,
                                   inner, rxk, rxw) != 0;
        }
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
        for (j = 0; j < n; ++j) {
            int64_t b = L.cstart[j];
            bad |= proxprox_vector(k, Yt + j * k, X, L.crow + b, L.cval + b, L.cstart[j + 1] - b, alpha,
                                   inner, ryk, ryw) != 0;
        }
        if (history)
            history[t] = objective_lists(&L, k, X, Yt, &lt, rxk, rxw, ryk, ryw, 0);
    }
    free(kind); free(param); free(lev);
    lists_free(&L);
    return bad ? -3 : 0;
}

/* Column statistics for the automatic scaling of Section 4.3 ("Offsets and
 * scaling"): for each column j with observed entries a_i,
 *   mu_j      = argmin_mu sum_i L_j(mu, a_i),
 *   sigma2_j  = sum_i L_j(mu_j, a_i) / (n_j - 1)     (NaN when n_j < 2).
 * The sum is convex in mu; it is minimised directly by golden-section search
 * on [min a - 32, max a + 32] down to an interval of 1e-13 of its width.
 * The search compares sums, so their rounding error limits where it can place
 * the minimiser: the sums are compensated (Neumaier), which keeps them
 * accurate to a few units of rounding whatever the column's length.  Where
 * the minimisers form an interval (a median of an even count, a quantile,
 * the flat bottom of a hinge sum) mu_j is its smallest point: a bisection
 * for the least x whose sum is within rounding of the minimum. */
static double col_sum(int kind, double param, int levels, const double *a, int64_t cnt, double mu)
{
    double s = 0.0, c = 0.0;
    for (int64_t e = 0; e < cnt; ++e) {
        double v = oracle_loss(kind, param, levels, mu, a[e]);
        double t = s + v;
        c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
        s = t;
    }
    return s + c;
}

int oracle_column_stats(int64_t m, int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                        const double *val, const int32_t *lkind, const double *lparam,
                        const int32_t *llevels, double *mu, double *sigma2, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    int rc = lists_build(&L, m, n, nnz, row, col, val);
    if (rc) { lists_free(&L); return rc; }
    set_threads(nthreads);
    int64_t j;
#pragma omp parallel for schedule(dynamic, 4)
    for (j = 0; j < n; ++j) {
        const double *a = L.cval + L.cstart[j];
        const int64_t cnt = L.cstart[j + 1] - L.cstart[j];
        if (cnt == 0) { mu[j] = NAN; sigma2[j] = NAN; continue; }
        double lo = a[0], hi = a[0];
        for (int64_t e = 1; e < cnt; ++e) { lo = a[e] < lo ? a[e] : lo; hi = a[e] > hi ? a[e] : hi; }
        lo -= 32.0;
        hi += 32.0;
        const double gr = 0.5 * (sqrt(5.0) - 1.0), width = hi - lo, lo0 = lo;
        double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
        double f1 = col_sum(lkind[j], lparam[j], llevels[j], a, cnt, x1);
        double f2 = col_sum(lkind[j], lparam[j], llevels[j], a, cnt, x2);
        while (hi - lo > 1e-13 * width) {
            if (f1 <= f2) {
                hi = x2; x2 = x1; f2 = f1;
                x1 = hi - gr * (hi - lo);
                f1 = col_sum(lkind[j], lparam[j], llevels[j], a, cnt, x1);
            } else {
                lo = x1; x1 = x2; f1 = f2;
                x2 = lo + gr * (hi - lo);
                f2 = col_sum(lkind[j], lparam[j], llevels[j], a, cnt, x2);
            }
        }
        /* the minimisers of S_j form an interval (a flat bottom for the
         * piecewise-linear losses); take its smallest point: the least x in
         * the bracket with S(x) within rounding of the minimum found */
        double best = 0.5 * (lo + hi);
        const double smin = col_sum(lkind[j], lparam[j], llevels[j], a, cnt, best);
        const double slack = 4e-15 * (fabs(smin) > 1.0 ? fabs(smin) : 1.0);
        double l0 = lo0, h0 = best;
        for (int it = 0; it < 200 && h0 - l0 > 1e-15 * width; ++it) {
            const double mid = 0.5 * (l0 + h0);
            if (col_sum(lkind[j], lparam[j], llevels[j], a, cnt, mid) <= smin + slack) h0 = mid;
            else l0 = mid;
        }
        mu[j] = h0;
        sigma2[j] = cnt > 1 ? col_sum(lkind[j], lparam[j], llevels[j], a, cnt, mu[j]) / (double)(cnt - 1) : NAN;
    }
    lists_free(&L);
    return 0;
}

/* Per observed entry, in the order given: w_j L_j'(x_i . y_j, A_ij) (w_j = 1
 * when wcol is NULL) -- the entries of the loss gradient G in dL(Z) at
 * Z = X Y (Section 7.6, eq. convex-certificate), 0 at a kink. */
int oracle_entry_derivs(int64_t nnz, int k, const int32_t *row, const int32_t *col, const double *val,
                        const int32_t *lkind, const double *lparam, const int32_t *llevels, const double *wcol,
                        const double *X, const double *Yt, double *out)
{
    for (int64_t e = 0; e < nnz; ++e) {
        const int32_t i = row[e], j = col[e];
        const double u = dot(k, X + (int64_t)i * k, Yt + (int64_t)j * k);
        out[e] = (wcol ? wcol[j] : 1.0) * oracle_dloss(lkind[j], lparam[j], llevels[j], u, val[e]);
    }
    return 0;
}

/* ------------------------------------------- multi-dimensional losses */

/* Section 6 ("Multi-dimensional loss functions", eq. mpca): feature j of the
 * table is represented by a block Y_j of d_j columns of Y, and entry (i, j)
 * costs L_j(x_i Y_j, A_ij) with u = x_i Y_j in R^{d_j}.  Feature kinds:
 *  - FEAT_SCALAR: d_j = 1 and one of the scalar losses above;
 *  - FEAT_CATEGORICAL with d labels 1..d ("Categorical PCA", one-vs-all):
 *        L(u, a) = (1 - u_a)_+ + sum_{a' != a} (1 + u_a')_+,   d_j = d;
 *  - FEAT_ORDINAL_MD with d levels 1..d (eq. ord-mpca):
 *        L(u, a) = sum_{a'=1}^{d-1} (1 - s(a, a') u_a')_+,       d_j = d - 1,
 *    reading the printed indicator I_{a > a'} as the sign s = +1 if a > a'
 *    and -1 otherwise (with a 0/1 indicator every term with a <= a' would be
 *    the constant 1 and the loss could not prefer low levels).
 * Kinks take derivative 0.  u is indexed from 0: u[l] is column l + 1. */
enum { FEAT_SCALAR = 0, FEAT_CATEGORICAL = 1, FEAT_ORDINAL_MD = 2 };

int oracle_feature_dim(int fkind, int levels)
{
    switch (fkind) {
    case FEAT_SCALAR: return 1;
    case FEAT_CATEGORICAL: return levels;
    case FEAT_ORDINAL_MD: return levels - 1;
    }
    return -1;
}

double oracle_mloss(int fkind, int levels, const double *u, double a)
{
    const int lab = (int)a;
    double s = 0.0;
    if (fkind == FEAT_CATEGORICAL) {
        for (int l = 1; l <= levels; ++l)
            s += l == lab ? pos(1.0 - u[l - 1]) : pos(1.0 + u[l - 1]);
        return s;
    }
    if (fkind == FEAT_ORDINAL_MD) {
        for (int ap = 1; ap <= levels - 1; ++ap) {
            const double sg = lab > ap ? 1.0 : -1.0;
            s += pos(1.0 - sg * u[ap - 1]);
        }
        return s;
    }
    return NAN;
}

/* Gradient of oracle_mloss with respect to u (d_j entries into g). */
void oracle_mgrad(int fkind, int levels, const double *u, double a, double *g)
{
    const int lab = (int)a;
    if (fkind == FEAT_CATEGORICAL) {
        for (int l = 1; l <= levels; ++l)
            g[l - 1] = l == lab ? (1.0 - u[l - 1] > 0.0 ? -1.0 : 0.0) : (1.0 + u[l - 1] > 0.0 ? 1.0 : 0.0);
        return;
    }
    if (fkind == FEAT_ORDINAL_MD) {
        for (int ap = 1; ap <= levels - 1; ++ap) {
            const double sg = lab > ap ? 1.0 : -1.0;
            g[ap - 1] = 1.0 - sg * u[ap - 1] > 0.0 ? -sg : 0.0;
        }
    }
}

/* Imputation of a multi-dimensional feature: the categorical label is
 * argmax_l u_l (Section 6, "Categorical PCA"; the first of equal maxima); the
 * ordinal level is argmin_a L(u, a) over a = 1..d by trying every level (the
 * general rule of Section 5.3; ties to the smaller level). */
double oracle_mdecode(int fkind, int levels, const double *u)
{
    if (fkind == FEAT_CATEGORICAL) {
        int best = 1;
        for (int l = 2; l <= levels; ++l)
            if (u[l - 1] > u[best - 1]) best = l;
        return (double)best;
    }
    if (fkind == FEAT_ORDINAL_MD) {
        int best = 1;
        double bestv = oracle_mloss(fkind, levels, u, 1.0);
        for (int a = 2; a <= levels; ++a) {
            double v = oracle_mloss(fkind, levels, u, (double)a);
            if (v < bestv) { bestv = v; best = a; }
        }
        return (double)best;
    }
    return NAN;
}

/* The feature model of one problem: per feature its kind, label / level
 * count, scalar loss (FEAT_SCALAR), and first column of its block in Y
 * (first[j] .. first[j] + d_j - 1; first[nf] = d, the embedded width). */
typedef struct {
    int64_t nf;
    const int32_t *fkind, *flev, *lkind, *llev;
    const double *lparam;
    int64_t *first;
} feat_model;

/* u = x Y_j (d_j entries; Yt holds Y's columns as rows of k). */
static void block_u(const feat_model *F, int k, int64_t j, const double *x, const double *Yt, double *u)
{
    const int64_t c0 = F->first[j], d = F->first[j + 1] - c0;
    for (int64_t l = 0; l < d; ++l) u[l] = dot(k, x, Yt + (c0 + l) * k);
}

static double entry_loss(const feat_model *F, int64_t j, const double *u, double a)
{
    if (F->fkind[j] == FEAT_SCALAR) return oracle_loss(F->lkind[j], F->lparam[j], F->llev[j], u[0], a);
    return oracle_mloss(F->fkind[j], F->flev[j], u, a);
}

static void entry_grad(const feat_model *F, int64_t j, const double *u, double a, double *g)
{
    if (F->fkind[j] == FEAT_SCALAR) g[0] = oracle_dloss(F->lkind[j], F->lparam[j], F->llev[j], u[0], a);
    else oracle_mgrad(F->fkind[j], F->flev[j], u, a, g);
}

static int model_build(feat_model *F, int64_t nf, const int32_t *fkind, const int32_t *flev,
                       const int32_t *lkind, const double *lparam, const int32_t *llev)
{
    F->nf = nf; F->fkind = fkind; F->flev = flev; F->lkind = lkind; F->lparam = lparam; F->llev = llev;
    F->first = malloc(sizeof(int64_t) * (size_t)(nf + 1));
    if (!F->first) return -1;
    F->first[0] = 0;
    for (int64_t j = 0; j < nf; ++j) {
        int d = oracle_feature_dim(fkind[j], flev[j]);
        if (d < 1) return -2;
        F->first[j + 1] = F->first[j] + d;
    }
    return 0;
}

static int64_t model_dmax(const feat_model *F)
{
    int64_t dm = 1;
    for (int64_t j = 0; j < F->nf; ++j) dm = F->first[j + 1] - F->first[j] > dm ? F->first[j + 1] - F->first[j] : dm;
    return dm;
}

/* Loss of row i's entries at factor row x. */
static double mrow_loss(const feat_model *F, int k, const double *x, const double *Yt, const omega_lists *L,
                        int64_t i, double *u)
{
    double s = 0.0;
    for (int64_t e = L->rstart[i]; e < L->rstart[i + 1]; ++e) {
        const int64_t j = L->rcol[e];
        block_u(F, k, j, x, Yt, u);
        s += entry_loss(F, j, u, L->rval[e]);
    }
    return s;
}

static double mobjective_lists(const feat_model *F, const omega_lists *L, int k, const double *X, const double *Yt,
                               int rxk, double rxw, int ryk, double ryw)
{
    const int64_t dmax = model_dmax(F);
    double *rowsum = malloc(sizeof(double) * (size_t)(L->m ? L->m : 1));
    int64_t i;
#pragma omp parallel
    {
        double *u = malloc(sizeof(double) * (size_t)dmax);
#pragma omp for schedule(dynamic, 64)
        for (i = 0; i < L->m; ++i) rowsum[i] = mrow_loss(F, k, X + i * k, Yt, L, i, u);
        free(u);
    }
    double tot = 0.0;
    for (i = 0; i < L->m; ++i) tot += rowsum[i];
    for (i = 0; i < L->m; ++i) tot += oracle_reg(rxk, rxw, k, X + i * k);
    for (int64_t c = 0; c < F->first[F->nf]; ++c) tot += oracle_reg(ryk, ryw, k, Yt + c * k);
    free(rowsum);
    return tot;
}

/* Objective of eq. mpca: sum over Omega of L_j(x_i Y_j, A_ij) (rows
 * ascending, then features ascending) + sum_i r(x_i) + sum over the d
 * columns of Y of rt(y).  Omega: triples (row, feature, value) sorted by row
 * then feature; Yt is d x k. */
double oracle_mobjective(int64_t m, int64_t nf, int k, int64_t nnz, const int32_t *row, const int32_t *feat,
                         const double *val, const int32_t *fkind, const int32_t *flev, const int32_t *lkind,
                         const double *lparam, const int32_t *llev, int rxk, double rxw, int ryk, double ryw,
                         const double *X, const double *Yt, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    feat_model F;
    memset(&F, 0, sizeof F);
    double out = NAN;
    if (!lists_build(&L, m, nf, nnz, row, feat, val) && !model_build(&F, nf, fkind, flev, lkind, lparam, llev)) {
        set_threads(nthreads);
        out = mobjective_lists(&F, &L, k, X, Yt, rxk, rxw, ryk, ryw);
    }
    free(F.first);
    lists_free(&L);
    return out;
}

/* Alternating proximal-gradient sweeps on eq. mpca (Algorithm 2 with the
 * update and step-size rule of Section 7.2).  X-step: row x_i against the
 * blocks of its observed features, g = sum_j sum_l dL/du_l y_{j,l}, the rule
 * on f(x) = sum_j L_j(x Y_j, A_ij) + r(x).  Y-step: the block Y_j is
 * updated one column y_{j,l} at a time, each with its own step size and
 * accept test on f(y) = sum_i L_j(x_i Y_j[l <- y], A_ij) + rt(y), the other
 * columns held at their values from the start of the Y-step.  The losses of
 * this section are sums of one term per column of the block and rt is a sum
 * over columns, so minimising over Y_j separates exactly into these column
 * problems (the paper notes the one-vs-all loss's separability); each column
 * taking its own step size is the reading taken here.  Step sizes start at
 * 1 / max(count, 1) with count the number of scalar loss terms: sum of d_j
 * over a row's observed features, the observation count of feature j for each
 * column of its block.  alpha_y has d entries; accepts[2t], accepts[2t+1]
 * count accepted rows and columns of Y in sweep t. */
int oracle_mproxgrad(int64_t m, int64_t nf, int k, int64_t nnz, const int32_t *row, const int32_t *feat,
                     const double *val, const int32_t *fkind, const int32_t *flev, const int32_t *lkind,
                     const double *lparam, const int32_t *llev, int rxk, double rxw, int ryk, double ryw,
                     double *X, double *Yt, double *alpha_x, double *alpha_y, int nsweeps, double *history,
                     int64_t *accepts, int nthreads)
{
    omega_lists L;
    memset(&L, 0, sizeof L);
    feat_model F;
    memset(&F, 0, sizeof F);
    int rc = lists_build(&L, m, nf, nnz, row, feat, val);
    if (!rc) rc = model_build(&F, nf, fkind, flev, lkind, lparam, llev);
    if (rc) { free(F.first); lists_free(&L); return rc; }
    set_threads(nthreads);
    const int64_t D = F.first[nf], dmax = model_dmax(&F);
    int64_t *cfeat = malloc(sizeof(int64_t) * (size_t)(D ? D : 1));
    double *Yold = malloc(sizeof(double) * (size_t)(D ? D : 1) * (size_t)k);
    int *ax = malloc(sizeof(int) * (size_t)(m ? m : 1));
    int *ay = malloc(sizeof(int) * (size_t)(D ? D : 1));
    for (int64_t j = 0; j < nf; ++j)
        for (int64_t c = F.first[j]; c < F.first[j + 1]; ++c) cfeat[c] = j;
    for (int t = 0; t < nsweeps; ++t) {
        int64_t i, c;
#pragma omp parallel
        {
            double *u = malloc(sizeof(double) * (size_t)dmax);
            double *gu = malloc(sizeof(double) * (size_t)dmax);
            double g[k], z[k], xp[k];
#pragma omp for schedule(dynamic, 64)
            for (i = 0; i < m; ++i) {
                double *x = X + i * k;
                for (int q = 0; q < k; ++q) g[q] = 0.0;
                for (int64_t e = L.rstart[i]; e < L.rstart[i + 1]; ++e) {
                    const int64_t j = L.rcol[e];
                    block_u(&F, k, j, x, Yt, u);
                    entry_grad(&F, j, u, L.rval[e], gu);
                    for (int64_t l = 0; l < F.first[j + 1] - F.first[j]; ++l)
                        for (int q = 0; q < k; ++q) g[q] += gu[l] * Yt[(F.first[j] + l) * k + q];
                }
                for (int q = 0; q < k; ++q) z[q] = x[q] - alpha_x[i] * g[q];
                oracle_prox(rxk, rxw, alpha_x[i], k, z, xp);
                const double f_old = mrow_loss(&F, k, x, Yt, &L, i, u) + oracle_reg(rxk, rxw, k, x);
                const double f_new = mrow_loss(&F, k, xp, Yt, &L, i, u) + oracle_reg(rxk, rxw, k, xp);
                if (f_new <= f_old) {
                    for (int q = 0; q < k; ++q) x[q] = xp[q];
                    alpha_x[i] *= 1.05;
                    ax[i] = 1;
                } else {
                    alpha_x[i] *= 0.7;
                    ax[i] = 0;
                }
            }
            free(u);
            free(gu);
        }
        memcpy(Yold, Yt, sizeof(double) * (size_t)D * (size_t)k);
#pragma omp parallel
        {
            double *u = malloc(sizeof(double) * (size_t)dmax);
            double *gu = malloc(sizeof(double) * (size_t)dmax);
            double g[k], z[k], yp[k];
#pragma omp for schedule(dynamic, 4)
            for (c = 0; c < D; ++c) {
                const int64_t j = cfeat[c], l = c - F.first[j];
                const double *y = Yold + c * k;
                for (int q = 0; q < k; ++q) g[q] = 0.0;
                for (int64_t e = L.cstart[j]; e < L.cstart[j + 1]; ++e) {
                    const double *x = X + (int64_t)L.crow[e] * k;
                    block_u(&F, k, j, x, Yold, u);
                    entry_grad(&F, j, u, L.cval[e], gu);
                    for (int q = 0; q < k; ++q) g[q] += gu[l] * x[q];
                }
                for (int q = 0; q < k; ++q) z[q] = y[q] - alpha_y[c] * g[q];
                oracle_prox(ryk, ryw, alpha_y[c], k, z, yp);
                double f_old = oracle_reg(ryk, ryw, k, y), f_new = oracle_reg(ryk, ryw, k, yp);
                for (int64_t e = L.cstart[j]; e < L.cstart[j + 1]; ++e) {
                    const double *x = X + (int64_t)L.crow[e] * k;
                    block_u(&F, k, j, x, Yold, u);
                    f_old += entry_loss(&F, j, u, L.cval[e]);
                    u[l] = dot(k, x, yp);
                    f_new += entry_loss(&F, j, u, L.cval[e]);
                }
                if (f_new <= f_old) {
                    for (int q = 0; q < k; ++q) Yt[c * k + q] = yp[q];
                    alpha_y[c] *= 1.05;
                    ay[c] = 1;
                } else {
                    alpha_y[c] *= 0.7;
                    ay[c] = 0;
                }
            }
            free(u);
            free(gu);
        }
        int64_t na = 0, nb = 0;
        for (i = 0; i < m; ++i) na += ax[i];
        for (c = 0; c < D; ++c) nb += ay[c];
        if (accepts) { accepts[2 * t] = na; accepts[2 * t + 1] = nb; }
        if (history) history[t] = mobjective_lists(&F, &L, k, X, Yt, rxk, rxw, ryk, ryw);
    }
    free(cfeat); free(Yold); free(ax); free(ay);
    free(F.first);
    lists_free(&L);
    return 0;
}

int oracle_num_threads(int nthreads) { return set_threads(nthreads); }
