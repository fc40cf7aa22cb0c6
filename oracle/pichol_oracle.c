/*
 * Plain FP64 CPU oracle for piCholesky cross-validation (Kuang, Gittens, Hamid,
 * "Cholesky Factor Interpolation for Efficient Approximate Cross-Validation").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA path is checked against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA library and must never be linked into
 * it.
 *
 * Every routine is a definition written out with plain loops in double
 * precision: no fusion and no reordering of any sum beyond what the definition
 * states.  The one restructuring is a loop interchange in the Gram routine,
 * which keeps the order of every sum.  OpenMP is used only to run independent
 * units (groups of Gram rows, the entries of one Cholesky column, independent
 * right-hand sides, the rows of a hold-out error) side by side; it never
 * changes the order of a sum, so every result is the same from run to run.
 *
 * Matrices are row-major: element (i, j) of an r x s matrix M is M[i*s + j].
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

/*
 * Normal-equation blocks of a set of rows (Sec. 3.1, Eq. 2: H = X^T X and
 * g = X^T y).  Rows [skip0, skip1) are left out, so with the fold's own rows
 * skipped this gives the training-set Hessian H_f and right-hand side B_f of
 * fold f directly, without any cross-fold shortcut.
 *   X : n x d,  Y : n x c
 *   H : d x d (both triangles written), B : d x c
 */
void orc_normal_blocks(int64_t n, int64_t d, int64_t c,
                       const double* X, const double* Y,
                       int64_t skip0, int64_t skip1,
                       double* H, double* B)
{
    /* H[i][j] = sum over kept rows r (ascending) of X[r][i] * X[r][j].  The
     * rows of H are handled in groups of 32 so that each row of X is read
     * once per group; the order of every sum is still r = 0, 1, ..., n-1. */
    const int64_t grp = 32;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i0 = 0; i0 < d; i0 += grp) {
        int64_t i1 = (i0 + grp < d) ? i0 + grp : d;
        for (int64_t i = i0; i < i1; ++i) {
            for (int64_t j = 0; j < d; ++j) H[i * d + j] = 0.0;
            for (int64_t o = 0; o < c; ++o) B[i * c + o] = 0.0;
        }
        for (int64_t r = 0; r < n; ++r) {
            if (r >= skip0 && r < skip1) continue;
            const double* x = X + r * d;
            for (int64_t i = i0; i < i1; ++i) {
                double xi = x[i];
                double* Hi = H + i * d;
                for (int64_t j = 0; j <= i; ++j) Hi[j] += xi * x[j];
                for (int64_t o = 0; o < c; ++o) B[i * c + o] += xi * Y[r * c + o];
            }
        }
    }
    /* mirror the lower triangle into the upper one */
    for (int64_t i = 0; i < d; ++i)
        for (int64_t j = i + 1; j < d; ++j)
            H[i * d + j] = H[j * d + i];
}

/*
 * Cholesky factor A = L L^T of a symmetric positive-definite d x d matrix
 * (Sec. 3.2), column by column (Cholesky-Crout order):
 *   L[j][j] = sqrt(A[j][j] - sum_{p<j} L[j][p]^2),
 *   L[i][j] = (A[i][j] - sum_{p<j} L[i][p] L[j][p]) / L[j][j]   for i > j.
 * Each sum runs over p = 0, 1, ..., j-1 in order.  The entries of one column
 * below the diagonal are independent of each other and are computed side by
 * side.  Only the lower triangle of A is read; L is written in full (upper
 * triangle zero).
 * Returns -1 on success, else the index of the first pivot that is not
 * positive (L is then only partly defined).
 */
int64_t orc_cholesky(int64_t d, const double* A, double* L)
{
    memset(L, 0, (size_t)(d * d) * sizeof(double));
    for (int64_t j = 0; j < d; ++j) {
        double s = A[j * d + j];
        for (int64_t p = 0; p < j; ++p) s -= L[j * d + p] * L[j * d + p];
        if (!(s > 0.0)) return j;
        double ljj = sqrt(s);
        L[j * d + j] = ljj;
        #pragma omp parallel for schedule(static) if (d - j > 256)
        for (int64_t i = j + 1; i < d; ++i) {
            double t = A[i * d + j];
            for (int64_t p = 0; p < j; ++p) t -= L[i * d + p] * L[j * d + p];
            L[i * d + j] = t / ljj;
        }
    }
    return -1;
}

/*
 * Forward substitution L Z = B (Sec. 3.2, first triangular solve), c columns.
 * L: d x d lower, B, Z: d x c.
 */
void orc_forward(int64_t d, int64_t c, const double* L, const double* B, double* Z)
{
    #pragma omp parallel for if (c > 1)
    for (int64_t o = 0; o < c; ++o) {
        for (int64_t i = 0; i < d; ++i) {
            double s = B[i * c + o];
            for (int64_t p = 0; p < i; ++p)
                s -= L[i * d + p] * Z[p * c + o];
            Z[i * c + o] = s / L[i * d + i];
        }
    }
}

/*
 * Back substitution L^T W = Z (Sec. 3.2, second triangular solve), c columns.
 */
void orc_backward(int64_t d, int64_t c, const double* L, const double* Z, double* W)
{
    #pragma omp parallel for if (c > 1)
    for (int64_t o = 0; o < c; ++o) {
        for (int64_t i = d - 1; i >= 0; --i) {
            double s = Z[i * c + o];
            for (int64_t p = i + 1; p < d; ++p)
                s -= L[p * d + i] * W[p * c + o];
            W[i * c + o] = s / L[i * d + i];
        }
    }
}

/*
 * Hold-out sum of squared residuals ||Y_v - X_v W||_F^2 over the n_v held-out
 * rows, evaluated directly row by row (Sec. 3.1: the lambda with the smallest
 * hold-out error is picked).  X_v: n_v x d, Y_v: n_v x c, W: d x c.
 */
double orc_holdout_sse(int64_t nv, int64_t d, int64_t c,
                       const double* Xv, const double* Yv, const double* W)
{
    /* the rows' sums are independent units; their total is then taken in row
     * order r = 0, 1, ..., n_v - 1 (NaN if the scratch row cannot be had) */
    double* rows = (double*)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    if (!rows) return NAN;
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nv; ++r) {
        double row = 0.0;
        for (int64_t o = 0; o < c; ++o) {
            double pred = 0.0;
            for (int64_t p = 0; p < d; ++p)
                pred += Xv[r * d + p] * W[p * c + o];
            double e = Yv[r * c + o] - pred;
            row += e * e;
        }
        rows[r] = row;
    }
    double total = 0.0;
    for (int64_t r = 0; r < nv; ++r) total += rows[r];
    free(rows);
    return total;
}

/*
 * Least-squares polynomial fit of Algorithm 1: Theta minimising
 * ||T - V Theta||_F, V: g x p (p = r + 1, g >= p, full column rank),
 * T: g x D, Theta: p x D.
 *
 * Algorithm 1 writes the minimiser through the normal equations
 * (V^T V)^{-1} V^T T.  The same minimiser is computed here by Householder QR
 * of V, which does not square the condition number of V:
 *   V = Q R,  Theta = R^{-1} (Q^T T)[0:p].
 * Returns 0, 1 if R has a zero diagonal (V rank deficient), or 2 if the
 * scratch matrices cannot be had.
 */
int orc_lstsq_householder(int64_t g, int64_t p, const double* V,
                          int64_t D, const double* T, double* Theta)
{
    double* R = (double*)malloc((size_t)(g * p) * sizeof(double));
    double* QT = (double*)malloc((size_t)(g * D) * sizeof(double));
    double* v = (double*)malloc((size_t)g * sizeof(double));
    if (!R || !QT || !v) { free(R); free(QT); free(v); return 2; }
    memcpy(R, V, (size_t)(g * p) * sizeof(double));
    memcpy(QT, T, (size_t)(g * D) * sizeof(double));
    int rc = 0;
    for (int64_t k = 0; k < p; ++k) {
        /* Householder vector for column k, rows k..g-1 */
        double norm = 0.0;
        for (int64_t i = k; i < g; ++i) norm += R[i * p + k] * R[i * p + k];
        norm = sqrt(norm);
        if (norm == 0.0) { rc = 1; break; }
        double alpha = (R[k * p + k] > 0.0) ? -norm : norm;
        for (int64_t i = 0; i < g; ++i) v[i] = 0.0;
        v[k] = R[k * p + k] - alpha;
        for (int64_t i = k + 1; i < g; ++i) v[i] = R[i * p + k];
        double vv = 0.0;
        for (int64_t i = k; i < g; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        /* apply H = I - 2 v v^T / (v^T v) to R (columns k..p-1) */
        for (int64_t j = k; j < p; ++j) {
            double s = 0.0;
            for (int64_t i = k; i < g; ++i) s += v[i] * R[i * p + j];
            s = 2.0 * s / vv;
            for (int64_t i = k; i < g; ++i) R[i * p + j] -= s * v[i];
        }
        /* ... and to every column of T */
        #pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < D; ++j) {
            double s = 0.0;
            for (int64_t i = k; i < g; ++i) s += v[i] * QT[i * D + j];
            s = 2.0 * s / vv;
            for (int64_t i = k; i < g; ++i) QT[i * D + j] -= s * v[i];
        }
    }
    if (rc == 0) {
        for (int64_t k = 0; k < p; ++k)
            if (R[k * p + k] == 0.0) rc = 1;
    }
    if (rc == 0) {
        /* back substitution R Theta = (Q^T T)[0:p] */
        #pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < D; ++j) {
            for (int64_t i = p - 1; i >= 0; --i) {
                double s = QT[i * D + j];
                for (int64_t l = i + 1; l < p; ++l) s -= R[i * p + l] * Theta[l * D + j];
                Theta[i * D + j] = s / R[i * p + i];
            }
        }
    }
    free(R); free(QT); free(v);
    return rc;
}

/*
 * Row-wise vectorisation of the lower triangle of a d x d matrix (Sec. 5,
 * "row-wise" order): entries (0,0), (1,0), (1,1), (2,0), ... ; D = d(d+1)/2.
 * The ordering does not change the fitted coefficients entrywise, so the
 * oracle uses the plainest one.
 */
void orc_vec_lower(int64_t d, const double* L, double* v)
{
    int64_t idx = 0;
    for (int64_t i = 0; i < d; ++i)
        for (int64_t j = 0; j <= i; ++j)
            v[idx++] = L[i * d + j];
}

/* Inverse of orc_vec_lower; the upper triangle is zeroed. */
void orc_unvec_lower(int64_t d, const double* v, double* L)
{
    int64_t idx = 0;
    memset(L, 0, (size_t)(d * d) * sizeof(double));
    for (int64_t i = 0; i < d; ++i)
        for (int64_t j = 0; j <= i; ++j)
            L[i * d + j] = v[idx++];
}

/*
 * Interpolated factor entries (Sec. 3.3, evaluation of the D polynomials at a
 * new lambda_t): vec(L_t) = sum_m phi_m(lambda_t) Theta[m, :].
 * phi: p basis values at lambda_t, Theta: p x D, out: D.
 */
void orc_eval_poly(int64_t p, int64_t D, const double* phi, const double* Theta, double* out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < D; ++j) {
        double s = 0.0;
        for (int64_t m = 0; m < p; ++m) s += phi[m] * Theta[m * D + j];
        out[j] = s;
    }
}
