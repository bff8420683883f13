/*
 * mp_oracle.h -- CPU oracle for multi-component (DD/TD/QD) arithmetic and GEMM.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, scalar reference that the
 * GPU path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the library's product path never
 * does.  It shares no source with the CUDA kernels.
 *
 * Conventions
 *   - A multi-component number with P components (P = 2 DD, 3 TD, 4 QD) is P
 *     binary64 values, component 0 the most significant (Sec. 2).
 *   - Vectors and matrices are structure-of-arrays: one binary64 plane per
 *     component (Sec. 2.5, Fig. 1).  Matrices are row-major (Sec. 3).
 *   - Every + - * is a separately rounded binary64 operation (round to nearest
 *     even); the only fused operations are the explicit fma() calls that the
 *     algorithms name.  The file must be compiled with -ffp-contract=off.
 */
#ifndef MP_ORACLE_H
#define MP_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* error-free transformations, Sec. 2.1 */
void or_quick_two_sum(double a, double b, double *s, double *e);
void or_two_sum(double a, double b, double *s, double *e);
void or_two_prod(double a, double b, double *p, double *e);

/* helpers used by Alg. 3-6 */
void or_three_sum(double *a, double *b, double *c);
void or_three_sum2(double *a, double *b, double *c);
void or_renorm5(const double c[5], double r[4]);
void or_vec_sum(int n, const double *x, double *e);
void or_vseb(int n, const double *e, int k, double *r);

/* scalar multi-component operations; x, y, r are arrays of P components */
void or_dd_add(const double x[2], const double y[2], double r[2]);   /* Alg. 1 */
void or_dd_mul(const double x[2], const double y[2], double r[2]);   /* Alg. 2 */
void or_td_add(const double x[3], const double y[3], double r[3]);   /* Alg. 3 */
void or_td_addq(const double x[3], const double y[3], double r[3]);  /* Sec. 2.3, TDaddq */
void or_td_mul(const double x[3], const double y[3], double r[3]);   /* Alg. 4 */
void or_qd_add(const double x[4], const double y[4], double r[4]);   /* Alg. 5 */
void or_qd_mul(const double x[4], const double y[4], double r[4]);   /* Alg. 6 */
void or_td_mulq(const double x[3], const double y[3], double r[3]);  /* Sec. 2.3, TDmulq */
void or_td_mul_acc(const double x[3], const double y[3], double r[3]); /* Sec. 2.3, accurate TD product */
void or_qd_add_acc(const double x[4], const double y[4], double r[4]); /* accurate QD addition */

/* elementwise over SoA planes, Sec. 2.5: r_i = x_i (op) y_i, op 0 = add, 1 = mul.
 * P in {2,3,4}; the TD add is TDaddq (the paper's default TD addition). */
int or_vec_op(int P, int op, int64_t n, const double *const *x,
              const double *const *y, double *const *r);
/* elementwise EFTs: which 0 = QuickTwoSum, 1 = TwoSum, 2 = TwoProd */
int or_vec_eft(int which, int64_t n, const double *a, const double *b,
               double *s, double *e);

/* C := A B (Eq. 1), k-sequential: acc starts at zero and, for p = 0..k-1 in
 * order, acc = add(acc, mul(A[i,p], B[p,j])).  Row-major planes, leading
 * dimensions in elements.  nthreads > 1 splits the rows of C across OpenMP
 * threads; each entry is still computed by the same sequence. */
int or_gemm(int P, int64_t m, int64_t n, int64_t k,
            const double *const *A, int64_t lda,
            const double *const *B, int64_t ldb,
            double *const *C, int64_t ldc, int nthreads);

/* The binary64-only product: C := A B (Eq. 1) with acc = fma(a_ip, b_pj, acc)
 * for p = 0..k-1 in order from acc = +0; single row-major planes. */
int or_dgemm(int64_t m, int64_t n, int64_t k,
             const double *A, int64_t lda,
             const double *B, int64_t ldb,
             double *C, int64_t ldc, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
