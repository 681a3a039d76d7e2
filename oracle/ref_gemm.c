/*
 * FP64 reference GEMM -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library.  The CUDA product path never links it.
 *
 * What it computes is the plain definition of the operation the Stream-K
 * method accelerates (paper, Introduction and Background: general
 * matrix-matrix multiplication; the method only re-partitions the k-sum):
 *
 *     C[i][j] = alpha * sum_k A[i][k] * B[k][j] + beta * C0[i][j]
 *     S[i][j] =         sum_k |A[i][k]| * |B[k][j]|
 *
 * in IEEE double, as a triple loop over (i, j, k) with rows split across
 * host threads.  S is the scale of the normwise error bound.  Operands are
 * addressed through explicit element strides, so any storage order works:
 * element (i, k) of A is A[i * a_rs + k * a_cs], and so on.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static double dot_entry(int64_t i, int64_t j, int64_t K,
                        const double *A, int64_t a_rs, int64_t a_cs,
                        const double *B, int64_t b_rs, int64_t b_cs,
                        double *abs_out)
{
    double acc = 0.0, s = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        double a = A[i * a_rs + k * a_cs];
        double b = B[k * b_rs + j * b_cs];
        acc += a * b;
        s += fabs(a) * fabs(b);
    }
    if (abs_out) *abs_out = s;
    return acc;
}

/* Full product.  C0 may be NULL when beta == 0; S may be NULL. */
void oracle_gemm_f64(int64_t M, int64_t N, int64_t K,
                     const double *A, int64_t a_rs, int64_t a_cs,
                     const double *B, int64_t b_rs, int64_t b_cs,
                     double alpha, double beta,
                     const double *C0, int64_t c0_rs, int64_t c0_cs,
                     double *C, int64_t c_rs, int64_t c_cs,
                     double *S, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            double s;
            double acc = dot_entry(i, j, K, A, a_rs, a_cs, B, b_rs, b_cs, &s);
            double c = alpha * acc;
            if (beta != 0.0 && C0) c += beta * C0[i * c0_rs + j * c0_cs];
            C[i * c_rs + j * c_cs] = c;
            if (S) S[i * c_rs + j * c_cs] = s;
        }
    }
}

/* Selected entries only: for p < count, (rows[p], cols[p]).  Used to check
 * products too large to form in full on the host. */
void oracle_gemm_entries_f64(int64_t count, const int64_t *rows, const int64_t *cols,
                             int64_t K,
                             const double *A, int64_t a_rs, int64_t a_cs,
                             const double *B, int64_t b_rs, int64_t b_cs,
                             double alpha, double beta,
                             const double *C0, int64_t c0_rs, int64_t c0_cs,
                             double *C_out, double *S_out, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t p = 0; p < count; ++p) {
        int64_t i = rows[p], j = cols[p];
        double s;
        double acc = dot_entry(i, j, K, A, a_rs, a_cs, B, b_rs, b_cs, &s);
        double c = alpha * acc;
        if (beta != 0.0 && C0) c += beta * C0[i * c0_rs + j * c0_cs];
        C_out[p] = c;
        if (S_out) S_out[p] = s;
    }
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
