/*
 * Plain, slow, double-precision CPU oracle for Gaussian belief propagation
 * (GaBP) on nonsymmetric sparse systems A x = b.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline / reference leg load this library.  It shares no code, header,
 * table or helper with the CUDA library; it is written from the paper's
 * equations in the paper's notation, not for speed.
 *
 * Matrix: CSR with n rows, int64 row pointers, int32 column indices sorted
 * within each row, double values.
 *
 * Graph (Sec. 2.3): the directed edge j -> i exists iff A_ij != 0 and i != j.
 *
 * Message storage: the message sent from node j to node i lives in the CSR
 * slot p of the matrix entry (i, j):
 *     lt[p] = tilde-Lambda_{ji},   mm[p] = m_{ji}
 * with the reparametrisation m_ji = mu_ji Lambda_ji and
 * tilde-Lambda_ji = Lambda_ji / A_ji (eq. nonsymmetric_GaBP_messages).
 * Slots on the diagonal or holding an explicit zero carry no message and are
 * kept at zero.
 *
 * Every loop over rows is independent of every other row, so the optional
 * OpenMP pragmas change nothing in the results (the residual uses max, which
 * is exact in any order).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_BREAKDOWN 4

/* A_ij by binary search in row i; 0 where the entry is not stored. */
static double aval(const int64_t *indptr, const int32_t *indices, const double *data,
                   int64_t i, int64_t j)
{
    int64_t lo = indptr[i], hi = indptr[i + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int64_t c = indices[mid];
        if (c == j) return data[mid];
        if (c < j) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Beliefs (eq. nonsymmetric_GaBP_rules, second line):
 *   beta_i = A_ii + sum_{j in N(i)} tilde-Lambda_ji A_ji
 *   mu_i   = (b_i + sum_{j in N(i)} m_ji) / beta_i
 * where N(i) are the nodes j with an edge j -> i (A_ij != 0).
 */
void oracle_beliefs(int64_t n, const int64_t *indptr, const int32_t *indices,
                    const double *data, const double *b, const double *lt,
                    const double *mm, double *mu, double *beta)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double prec = aval(indptr, indices, data, i, i);
        double mean = b[i];
        for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
            int64_t j = indices[p];
            if (j == i || data[p] == 0.0) continue;
            prec += lt[p] * aval(indptr, indices, data, j, i); /* tilde-Lambda_ji A_ji */
            mean += mm[p];                                      /* m_ji */
        }
        beta[i] = prec;
        mu[i] = mean / prec;
    }
}

/*
 * One synchronous (flood, Sec. 2.2) update of every message from the
 * previous ones (eq. nonsymmetric_GaBP_rules, first line).  For the edge
 * j -> i:
 *   tilde-Lambda_ji <- -A_ij / (A_jj + sum_{k in N(j) \ i} tilde-Lambda_kj A_kj)
 *   m_ji            <- tilde-Lambda_ji (b_j + sum_{k in N(j) \ i} m_kj)
 * The sums run literally over the neighbours k of j other than i.
 * Returns ORACLE_BREAKDOWN if a denominator is zero or not finite.
 */
int oracle_update(int64_t n, const int64_t *indptr, const int32_t *indices,
                  const double *data, const double *b, const double *lt_old,
                  const double *mm_old, double *lt_new, double *mm_new)
{
    int breakdown = 0;
    int64_t i;
#pragma omp parallel for schedule(static) reduction(| : breakdown)
    for (i = 0; i < n; ++i) {
        for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
            int64_t j = indices[p];
            if (j == i || data[p] == 0.0) {
                lt_new[p] = 0.0;
                mm_new[p] = 0.0;
                continue;
            }
            /* message j -> i: aggregate at node j excluding what came from i */
            double den = aval(indptr, indices, data, j, j);
            double num = b[j];
            for (int64_t q = indptr[j]; q < indptr[j + 1]; ++q) {
                int64_t k = indices[q];
                if (k == j || k == i || data[q] == 0.0) continue;
                den += lt_old[q] * aval(indptr, indices, data, k, j); /* tilde-Lambda_kj A_kj */
                num += mm_old[q];                                     /* m_kj */
            }
            if (den == 0.0 || !isfinite(den)) breakdown |= 1;
            double lt_ji = -data[p] / den; /* -A_ij / (...) */
            lt_new[p] = lt_ji;
            mm_new[p] = lt_ji * num;
        }
    }
    return breakdown ? ORACLE_BREAKDOWN : ORACLE_OK;
}

/* max_i |b_i - (A x)_i|  (the stopping quantity of Algorithm 1). */
double oracle_residual_inf(int64_t n, const int64_t *indptr, const int32_t *indices,
                           const double *data, const double *b, const double *x)
{
    double worst = 0.0;
    int nan_seen = 0;
    int64_t i;
#pragma omp parallel for schedule(static) reduction(max : worst) reduction(| : nan_seen)
    for (i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) s -= data[p] * x[indices[p]];
        double a = fabs(s);
        if (a != a) nan_seen = 1;
        else if (a > worst) worst = a;
    }
    return nan_seen ? NAN : worst;
}

/* r = b - A x (full vector), used by the error-correction smoother (Algorithm 3). */
void oracle_residual(int64_t n, const int64_t *indptr, const int32_t *indices,
                     const double *data, const double *b, const double *x, double *r)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) s -= data[p] * x[indices[p]];
        r[i] = s;
    }
}

/*
 * `nsweeps` flood sweeps in the order of Algorithm 1: every sweep first
 * forms the beliefs x from the current messages and then replaces all
 * messages at once from the current ones.  The state (lt, mm) is updated in
 * place through the scratch pair (lt2, mm2) of the same length.  On return x
 * holds the beliefs of the last sweep and beta their precisions.
 */
int oracle_sweeps(int64_t n, const int64_t *indptr, const int32_t *indices,
                  const double *data, const double *b, int nsweeps, double *lt, double *mm,
                  double *lt2, double *mm2, double *x, double *beta)
{
    int64_t nnz = indptr[n];
    int status = ORACLE_OK;
    for (int s = 0; s < nsweeps; ++s) {
        oracle_beliefs(n, indptr, indices, data, b, lt, mm, x, beta);
        status |= oracle_update(n, indptr, indices, data, b, lt, mm, lt2, mm2);
        memcpy(lt, lt2, (size_t)nnz * sizeof(double));
        memcpy(mm, mm2, (size_t)nnz * sizeof(double));
    }
    return status;
}

/*
 * `nsweeps` sweeps of Algorithm 1 with a coloured schedule (Sec. 5.1: red-black
 * and 4-colour GaBP process one colour class at a time).  color[j] in
 * [0, ncolors) must give adjacent nodes different colours.  One sweep visits
 * the colours in order; for every node j of the current colour it forms the
 * belief x_j from the current messages and then replaces every message j -> i
 * it sends (eq. nonsymmetric_GaBP_rules), in place.  The messages into a node
 * of the current colour come from nodes of other colours, so the order of the
 * nodes inside one colour does not matter.
 */
int oracle_sweeps_colored(int64_t n, const int64_t *indptr, const int32_t *indices,
                          const double *data, const double *b, const int32_t *color,
                          int ncolors, int nsweeps, double *lt, double *mm, double *x,
                          double *beta)
{
    int breakdown = 0;
    for (int s = 0; s < nsweeps; ++s) {
        for (int c = 0; c < ncolors; ++c) {
            int64_t j;
            /* beliefs of the colour class from the current messages */
#pragma omp parallel for schedule(static)
            for (j = 0; j < n; ++j) {
                if (color[j] != c) continue;
                double prec = aval(indptr, indices, data, j, j);
                double mean = b[j];
                for (int64_t p = indptr[j]; p < indptr[j + 1]; ++p) {
                    int64_t k = indices[p];
                    if (k == j || data[p] == 0.0) continue;
                    prec += lt[p] * aval(indptr, indices, data, k, j);
                    mean += mm[p];
                }
                beta[j] = prec;
                x[j] = mean / prec;
            }
            /* messages sent by the colour class: j -> i lives in row i at column j */
            int64_t i;
#pragma omp parallel for schedule(static) reduction(| : breakdown)
            for (i = 0; i < n; ++i) {
                for (int64_t p = indptr[i]; p < indptr[i + 1]; ++p) {
                    int64_t jj = indices[p];
                    if (jj == i || color[jj] != c) continue;
                    if (data[p] == 0.0) {
                        lt[p] = 0.0;
                        mm[p] = 0.0;
                        continue;
                    }
                    double den = aval(indptr, indices, data, jj, jj);
                    double num = b[jj];
                    for (int64_t q = indptr[jj]; q < indptr[jj + 1]; ++q) {
                        int64_t k = indices[q];
                        if (k == jj || k == i || data[q] == 0.0) continue;
                        den += lt[q] * aval(indptr, indices, data, k, jj);
                        num += mm[q];
                    }
                    if (den == 0.0 || !isfinite(den)) breakdown |= 1;
                    double lt_ji = -data[p] / den;
                    lt[p] = lt_ji;
                    mm[p] = lt_ji * num;
                }
            }
        }
    }
    return breakdown ? ORACLE_BREAKDOWN : ORACLE_OK;
}
