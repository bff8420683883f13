/*
 * mp_oracle.c -- CPU oracle for DD/TD/QD arithmetic and GEMM (Kouya,
 * "Acceleration of multiple precision matrix multiplication based on
 * multi-component floating-point arithmetic using AVX2", arXiv 2101.06584).
 *
 * TEST INFRASTRUCTURE ONLY: a plain scalar restatement of the paper's
 * algorithms used to check the GPU library.  It is not part of the library's
 * product path and shares no code with it.
 *
 * Build with -O2 -ffp-contract=off (no contraction of a*b+c into an fma; the
 * only fused operations are the explicit fma() calls the algorithms name).
 *
 * Helpers the paper uses without defining (ThreeSum, ThreeSum2, Renorm,
 * VecSum, VSEB, Merge) follow the works it cites for them: the QD library of
 * Hida, Li and Bailey for ThreeSum/ThreeSum2/Renorm, and Fabiano, Muller and
 * Picot's triple-word arithmetic for VecSum/VSEB/Merge.  Renorm is written as
 * the branch-driven loop that Sec. 2 describes.
 */
#include "mp_oracle.h"
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Sec. 2.1 */

/* QuickTwoSum: s = fl(a+b), e = b - (s - a); a+b = s+e exactly when |a| >= |b|. */
void or_quick_two_sum(double a, double b, double *s, double *e)
{
    double sum = a + b;
    double bv = sum - a;
    *e = b - bv;
    *s = sum;
}

/* TwoSum: s = fl(a+b) and the exact error e = (a+b) - s, no ordering needed. */
void or_two_sum(double a, double b, double *s, double *e)
{
    double sum = a + b;
    double bv = sum - a;
    double av = sum - bv;
    double ea = a - av;
    double eb = b - bv;
    *e = ea + eb;
    *s = sum;
}

/* TwoProd with FMA: p = fl(a*b), e = fma(a, b, -p) = a*b - p exactly. */
void or_two_prod(double a, double b, double *p, double *e)
{
    double prod = a * b;
    *e = fma(a, b, -prod);
    *p = prod;
}

/* ------------------------------------------------ helpers of Alg. 3 - 6 */

/* ThreeSum (QD library): (a,b,c) -> (a',b',c') with a'+b'+c' = a+b+c exactly. */
void or_three_sum(double *a, double *b, double *c)
{
    double t1, t2, t3, na, nb, nc;
    or_two_sum(*a, *b, &t1, &t2);
    or_two_sum(*c, t1, &na, &t3);
    or_two_sum(t2, t3, &nb, &nc);
    *a = na;
    *b = nb;
    *c = nc;
}

/* ThreeSum2 (QD library): like ThreeSum, but the two low terms are added
 * with one rounding and c is left untouched. */
void or_three_sum2(double *a, double *b, double *c)
{
    double t1, t2, t3, na;
    or_two_sum(*a, *b, &t1, &t2);
    or_two_sum(*c, t1, &na, &t3);
    *a = na;
    *b = t2 + t3;
}

/* Renorm of five terms into four (QD renormalisation), as the loop of Sec. 2:
 * a bottom-up QuickTwoSum pass, then a top-down pass that emits a component
 * each time the running sum leaves a nonzero error; once three components are
 * emitted the remaining terms are folded into the last one with plain adds. */
void or_renorm5(const double c[5], double r[4])
{
    double t[5];
    double s = c[4];
    for (int i = 3; i >= 0; --i) {
        double hi, lo;
        or_quick_two_sum(c[i], s, &hi, &lo);
        t[i + 1] = lo;
        s = hi;
    }
    t[0] = s;

    r[0] = r[1] = r[2] = r[3] = 0.0;
    int k = 0;
    s = t[0];
    for (int i = 1; i <= 4; ++i) {
        if (k == 3) {
            s = s + t[i];
        } else {
            double hi, lo;
            or_quick_two_sum(s, t[i], &hi, &lo);
            if (lo != 0.0) {
                r[k] = hi;
                k = k + 1;
                s = lo;
            } else {
                s = hi;
            }
        }
    }
    r[k] = s;
}

/* VecSum (Fabiano, Muller, Picot): a TwoSum chain from the last term to the
 * first; e[0] is the rounded total, and sum(e) = sum(x) exactly. */
void or_vec_sum(int n, const double *x, double *e)
{
    double s = x[n - 1];
    for (int i = n - 2; i >= 0; --i) {
        double hi, lo;
        or_two_sum(x[i], s, &hi, &lo);
        e[i + 1] = lo;
        s = hi;
    }
    e[0] = s;
}

/* VSEB(k), VecSum with branch (Fabiano, Muller, Picot): compacts n terms into
 * k components with a QuickTwoSum chain that starts a new component whenever
 * the error is nonzero and returns as soon as k components are complete.
 * Components never written stay +0. */
void or_vseb(int n, const double *e, int k, double *r)
{
    for (int i = 0; i < k; ++i)
        r[i] = 0.0;
    int j = 0;
    double eps = e[0];
    for (int i = 0; i <= n - 2; ++i) {
        double hi, lo;
        or_quick_two_sum(eps, e[i + 1], &hi, &lo);
        r[j] = hi;
        if (lo != 0.0) {
            if (j >= k - 1)
                return;
            j = j + 1;
            eps = lo;
        } else {
            eps = hi;
        }
    }
    if (eps != 0.0 && j <= k - 1)
        r[j] = eps;
}

/* ------------------------------------------------------------- Sec. 2.2 */

/* Alg. 1, DDadd: TwoSum of the leading parts, the trailing parts added with
 * one rounding, then QuickTwoSum. */
void or_dd_add(const double x[2], const double y[2], double r[2])
{
    double s, e, w;
    or_two_sum(x[0], y[0], &s, &e);
    w = x[1] + y[1];
    e = e + w;
    or_quick_two_sum(s, e, &r[0], &r[1]);
}

/* Alg. 2, DDmul: TwoProd of the leading parts plus the two cross products. */
void or_dd_mul(const double x[2], const double y[2], double r[2])
{
    double p1, p2, w1, w2, w3;
    or_two_prod(x[0], y[0], &p1, &p2);
    w1 = x[0] * y[1];
    w2 = x[1] * y[0];
    w3 = w1 + w2;
    p2 = p2 + w3;
    or_quick_two_sum(p1, p2, &r[0], &r[1]);
}

/* ------------------------------------------------------------- Sec. 2.3 */

/* Merge step of Alg. 3: the six components of x and y sorted by decreasing
 * magnitude.  x and y are each already in decreasing order, so a two-way
 * merge suffices; on equal magnitude the component of x comes first. */
static void merge6(const double x[3], const double y[3], double z[6])
{
    int i = 0, j = 0;
    for (int o = 0; o < 6; ++o) {
        if (j >= 3 || (i < 3 && fabs(x[i]) >= fabs(y[j])))
            z[o] = x[i++];
        else
            z[o] = y[j++];
    }
}

/* Alg. 3, TDadd: Merge, VecSum, VSEB(3). */
void or_td_add(const double x[3], const double y[3], double r[3])
{
    double z[6], e[6];
    merge6(x, y, z);
    or_vec_sum(6, z, e);
    or_vseb(6, e, 3, r);
}

/* Alg. 5, QDadd (sloppy): componentwise sums and their exact errors, the
 * errors folded in with TwoSum/ThreeSum/ThreeSum2, then Renorm. */
void or_qd_add(const double x[4], const double y[4], double r[4])
{
    double s0, s1, s2, s3, v0, v1, v2, v3, u0, u1, u2, u3, w0, w1, w2, w3;
    double t0, t1, t2, t3;

    s0 = x[0] + y[0];
    s1 = x[1] + y[1];
    s2 = x[2] + y[2];
    s3 = x[3] + y[3];

    v0 = s0 - x[0];
    v1 = s1 - x[1];
    v2 = s2 - x[2];
    v3 = s3 - x[3];

    u0 = s0 - v0;
    u1 = s1 - v1;
    u2 = s2 - v2;
    u3 = s3 - v3;

    w0 = x[0] - u0;
    w1 = x[1] - u1;
    w2 = x[2] - u2;
    w3 = x[3] - u3;

    u0 = y[0] - v0;
    u1 = y[1] - v1;
    u2 = y[2] - v2;
    u3 = y[3] - v3;

    t0 = w0 + u0;
    t1 = w1 + u1;
    t2 = w2 + u2;
    t3 = w3 + u3; /* used below although the listing forms only t0..t2 */

    or_two_sum(s1, t0, &s1, &t0);
    or_three_sum(&s2, &t0, &t1);
    or_three_sum2(&s3, &t0, &t2);
    t0 = (t0 + t1) + t3;

    double c[5] = {s0, s1, s2, s3, t0};
    or_renorm5(c, r);
}

/* TDaddq (Sec. 2.3): QDadd applied to TD operands padded with a zero fourth
 * component; the fourth component of the result is dropped. */
void or_td_addq(const double x[3], const double y[3], double r[3])
{
    double x4[4] = {x[0], x[1], x[2], 0.0};
    double y4[4] = {y[0], y[1], y[2], 0.0};
    double r4[4];
    or_qd_add(x4, y4, r4);
    r[0] = r4[0];
    r[1] = r4[1];
    r[2] = r4[2];
}

/* Alg. 4, TDmul ("fast" triple-word product of Fabiano, Muller, Picot). */
void or_td_mul(const double x[3], const double y[3], double r[3])
{
    double z00up, z00lo, z01up, z01lo, z10up, z10lo;
    or_two_prod(x[0], y[0], &z00up, &z00lo);
    or_two_prod(x[0], y[1], &z01up, &z01lo);
    or_two_prod(x[1], y[0], &z10up, &z10lo);

    double bin[3] = {z00lo, z01up, z10up};
    double b[3];
    or_vec_sum(3, bin, b);

    double c = fma(x[1], y[1], b[2]);
    double z31 = fma(x[0], y[2], z10lo);
    double z32 = fma(x[2], y[0], z01lo);
    double z3 = z31 + z32;
    double s3 = c + z3;

    double ein[4] = {z00up, b[0], b[1], s3};
    double e[4];
    or_vec_sum(4, ein, e);

    r[0] = e[0];
    or_vseb(3, &e[1], 2, &r[1]);
}

/* ------------------------------------------------------------- Sec. 2.4 */

/* Alg. 6, QDmul (sloppy).  The listing's first line, s0 = x0 + y0, is
 * overwritten before any use and is therefore not computed. */
void or_qd_mul(const double x[4], const double y[4], double r[4])
{
    double p0, p1, p2, p3, p4, p5, q0, q1, q2, q3, q4, q5;
    double s0, s1, s2, t0, t1;

    or_two_prod(x[0], y[0], &p0, &q0);
    or_two_prod(x[0], y[1], &p1, &q1);
    or_two_prod(x[1], y[0], &p2, &q2);
    or_two_prod(x[0], y[2], &p3, &q3);
    or_two_prod(x[1], y[1], &p4, &q4);
    or_two_prod(x[2], y[0], &p5, &q5);

    or_three_sum(&p1, &p2, &q0);
    or_three_sum(&p2, &q1, &q2);
    or_three_sum(&p3, &p4, &p5);

    or_two_sum(p2, p3, &s0, &t0);
    or_two_sum(q1, p4, &s1, &t1);
    s2 = q2 + p5;
    or_two_sum(s1, t0, &s1, &t0);
    s2 = s2 + (t0 + t1);

    s1 = s1 + x[0] * y[3];
    s1 = s1 + x[1] * y[2];
    s1 = s1 + x[2] * y[1];
    s1 = s1 + x[3] * y[0];
    s1 = s1 + q0;
    s1 = s1 + q3;
    s1 = s1 + q4;
    s1 = s1 + q5;

    double c[5] = {p0, p1, s0, s1, s2};
    or_renorm5(c, r);
}

/* ------------------------------------------ variants of Sec. 2.3 - 2.4 */

/* Stable sort by decreasing magnitude (insertion sort): equal magnitudes keep
 * their order, so for operands that are each already in decreasing order the
 * result is the two-way merge of Alg. 3 with the first operand first on ties. */
static void sort_by_magnitude(int n, double *z)
{
    for (int i = 1; i < n; ++i) {
        double v = z[i];
        int j = i;
        while (j > 0 && fabs(v) > fabs(z[j - 1])) {
            z[j] = z[j - 1];
            j = j - 1;
        }
        z[j] = v;
    }
}

/* TDmulq (Sec. 2.3, the trial TD product): QDmul (Alg. 6) applied to TD
 * operands padded with a zero fourth component; the fourth component of the
 * result is dropped. */
void or_td_mulq(const double x[3], const double y[3], double r[3])
{
    double x4[4] = {x[0], x[1], x[2], 0.0};
    double y4[4] = {y[0], y[1], y[2], 0.0};
    double r4[4];
    or_qd_mul(x4, y4, r4);
    r[0] = r4[0];
    r[1] = r4[1];
    r[2] = r4[2];
}

/* The normalisation of the accurate variants, after the IEEE-style QD
 * addition of Hida, Li and Bailey: n >= 2 terms, sorted by decreasing
 * magnitude, are added one by one into a two-term accumulator (u, v).  A term
 * t gives (s1, e1) = TwoSum(v, t) and (s, e2) = TwoSum(u, s1), so that
 * u + v + t = s + e2 + e1 exactly; when both errors are nonzero, s is final
 * and is emitted as the next component and the accumulator becomes (e2, e1);
 * otherwise the accumulator becomes s and the nonzero error.  Renorm turns
 * the components and the rest into four.  Readings: once four components are
 * out, the accumulator and the terms not yet added are summed into a fifth
 * term with plain additions, in order; if the terms run out first, the
 * accumulator's two terms follow the emitted components. */
static void accumulate_sorted(int n, const double *z, double r[4])
{
    double u, v;
    or_quick_two_sum(z[0], z[1], &u, &v);
    double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int k = 0, i = 2;
    while (i < n && k < 4) {
        double s1, e1, s, e2;
        or_two_sum(v, z[i], &s1, &e1);
        or_two_sum(u, s1, &s, &e2);
        i = i + 1;
        if (e2 != 0.0 && e1 != 0.0) {
            c[k] = s;
            k = k + 1;
            u = e2;
            v = e1;
        } else if (e1 == 0.0) {
            u = s;
            v = e2;
        } else {
            u = s;
            v = e1;
        }
    }
    if (k < 4) {
        c[k] = u;
        c[k + 1] = v;
    } else {
        double t = u + v;
        for (; i < n; ++i)
            t = t + z[i];
        c[4] = t;
    }
    or_renorm5(c, r);
}

/* Accurate TD product (Sec. 2.3 names the "accurate" triple-word product of
 * Fabiano, Muller and Picot without giving its steps).  Reading: every
 * partial product x_i y_j with i + j <= 2 is split exactly by TwoProd; the
 * terms of order three (the errors of the order-two products, then x2 y1 and
 * x1 y2 by fma) are summed with one rounding each; x2 y2 is dropped.  The ten
 * terms, sorted by decreasing magnitude, go through the accurate
 * normalisation above; as in TDaddq and TDmulq, the fourth component is
 * dropped. */
void or_td_mul_acc(const double x[3], const double y[3], double r[3])
{
    double p00, q00, p01, q01, p10, q10, p02, q02, p11, q11, p20, q20;
    or_two_prod(x[0], y[0], &p00, &q00);
    or_two_prod(x[0], y[1], &p01, &q01);
    or_two_prod(x[1], y[0], &p10, &q10);
    or_two_prod(x[0], y[2], &p02, &q02);
    or_two_prod(x[1], y[1], &p11, &q11);
    or_two_prod(x[2], y[0], &p20, &q20);
    double t3 = (q02 + q11) + q20;
    t3 = fma(x[2], y[1], t3);
    t3 = fma(x[1], y[2], t3);

    double z[10] = {p00, q00, p01, p10, q01, q10, p02, p11, p20, t3};
    double r4[4];
    sort_by_magnitude(10, z);
    accumulate_sorted(10, z, r4);
    r[0] = r4[0];
    r[1] = r4[1];
    r[2] = r4[2];
}

/* Accurate QD addition (the IEEE-style addition of Hida, Li and Bailey): the
 * eight components sorted by decreasing magnitude (x first on ties), then
 * the accurate normalisation above. */
void or_qd_add_acc(const double x[4], const double y[4], double r[4])
{
    double z[8];
    for (int c = 0; c < 4; ++c) {
        z[c] = x[c];
        z[4 + c] = y[c];
    }
    sort_by_magnitude(8, z);
    accumulate_sorted(8, z, r);
}

/* --------------------------------------------------------- dispatch */

static void mp_add(int P, const double *x, const double *y, double *r)
{
    if (P == 2)
        or_dd_add(x, y, r);
    else if (P == 3)
        or_td_addq(x, y, r);
    else
        or_qd_add(x, y, r);
}

static void mp_mul(int P, const double *x, const double *y, double *r)
{
    if (P == 2)
        or_dd_mul(x, y, r);
    else if (P == 3)
        or_td_mul(x, y, r);
    else
        or_qd_mul(x, y, r);
}

/* Elementwise ops of SoA vectors (Sec. 2.5).  op: 0 add, 1 mul (the GEMM's
 * pair for P); 2 TDadd (Alg. 3), 3 TDmulq, 4 accurate TD product (P = 3);
 * 5 accurate QD addition (P = 4). */
int or_vec_op(int P, int op, int64_t n, const double *const *x,
              const double *const *y, double *const *r)
{
    if (P < 2 || P > 4 || op < 0 || op > 5 || n < 0)
        return -1;
    if ((op >= 2 && op <= 4 && P != 3) || (op == 5 && P != 4))
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        double xv[4], yv[4], rv[4];
        for (int c = 0; c < P; ++c) {
            xv[c] = x[c][i];
            yv[c] = y[c][i];
        }
        if (op == 0)
            mp_add(P, xv, yv, rv);
        else if (op == 1)
            mp_mul(P, xv, yv, rv);
        else if (op == 2)
            or_td_add(xv, yv, rv);
        else if (op == 3)
            or_td_mulq(xv, yv, rv);
        else if (op == 4)
            or_td_mul_acc(xv, yv, rv);
        else
            or_qd_add_acc(xv, yv, rv);
        for (int c = 0; c < P; ++c)
            r[c][i] = rv[c];
    }
    return 0;
}

int or_vec_eft(int which, int64_t n, const double *a, const double *b,
               double *s, double *e)
{
    if (which < 0 || which > 2 || n < 0)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (which == 0)
            or_quick_two_sum(a[i], b[i], &s[i], &e[i]);
        else if (which == 1)
            or_two_sum(a[i], b[i], &s[i], &e[i]);
        else
            or_two_prod(a[i], b[i], &s[i], &e[i]);
    }
    return 0;
}

/* ------------------------------------------------------------- Sec. 3 */

/* Eq. 1, c_ij = sum_k a_ik b_kj, with the sum taken in increasing k from a
 * zero accumulator, one multi-component mul and add per term. */
int or_gemm(int P, int64_t m, int64_t n, int64_t k,
            const double *const *A, int64_t lda,
            const double *const *B, int64_t ldb,
            double *const *C, int64_t ldc, int nthreads)
{
    if (P < 2 || P > 4 || m < 0 || n < 0 || k < 0)
        return -1;
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t p = 0; p < k; ++p) {
                double a[4], b[4], prod[4], sum[4];
                for (int c = 0; c < P; ++c) {
                    a[c] = A[c][i * lda + p];
                    b[c] = B[c][p * ldb + j];
                }
                mp_mul(P, a, b, prod);
                mp_add(P, acc, prod, sum);
                for (int c = 0; c < P; ++c)
                    acc[c] = sum[c];
            }
            for (int c = 0; c < P; ++c)
                C[c][i * ldc + j] = acc[c];
        }
    }
    return 0;
}

/* Eq. 1 in plain binary64 (Sec. 1: the 53-bit format the multi-component
 * numbers extend; Sec. 3 counts the digits a product loses): c_ij = sum_k
 * a_ik b_kj with one fused multiply-add per term, acc = fma(a_ik, b_kj, acc),
 * k increasing from acc = +0.  The FP64-only GEMM the DD/TD/QD products are
 * compared with. */
int or_dgemm(int64_t m, int64_t n, int64_t k,
             const double *A, int64_t lda,
             const double *B, int64_t ldb,
             double *C, int64_t ldc, int nthreads)
{
    if (m < 0 || n < 0 || k < 0)
        return -1;
    if (nthreads < 1)
        nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int64_t p = 0; p < k; ++p)
                acc = fma(A[i * lda + p], B[p * ldb + j], acc);
            C[i * ldc + j] = acc;
        }
    }
    return 0;
}
