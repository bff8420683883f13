// mp_arith.cuh -- device-side multi-component (DD/TD/QD) arithmetic.
//
// The operations of Kouya, arXiv 2101.06584, Sec. 2: error-free
// transformations (Sec. 2.1), DDadd/DDmul (Alg. 1-2), TDadd (Alg. 3),
// TDaddq (Sec. 2.3), TDmul (Alg. 4), QDadd/QDmul (Alg. 5-6) with the
// renormalisation of the QD library and VecSum/VSEB of Fabiano, Muller and
// Picot, which the paper uses without restating.
//
// Every function takes a policy f that performs the rounded binary64
// operations (add, sub, mul, fma) and the three transformations of Sec. 2.1
// (two_sum, quick_two_sum, two_prod).  Rn issues each as an explicit
// __fma_rn intrinsic, so the compiler cannot contract or reorder them: each
// function performs the same sequence of IEEE binary64 operations as the
// paper's algorithm and therefore returns the same bits as any other faithful
// implementation.  RnInt computes chosen transformations on the integer
// pipes instead, with the same bits for every input.  Data-dependent branches (the nonzero tests of VSEB and
// Renorm) are written as selects that pick exactly the value the branch
// would; the tests themselves look at the bit pattern with integer
// instructions so they do not occupy the FP64 pipe.
#pragma once
#include <cstdint>

#include "soft_fp64.cuh"

namespace mp {

// Rounded binary64 operations.  On GB300 a DFMA whose operands are ordinary
// registers issues at about 1.19x the rate of DADD or DMUL (or of a DFMA with
// a compile-time-constant operand), so every operation is issued as a fused
// multiply-add that rounds to exactly the same value:
//   a + b = fma(a, 1, b),   a - b = fma(b, -1, a),   a * b = fma(a, b, -0)
// (the product with +-1 is exact; adding -0 changes no value and keeps the
// sign of a zero product).  `one`, `neg_zero` and `zero` (+0, used wherever
// an algorithm adds a constant zero) are loaded at run time from a table
// indexed by the lane (make_rn), so they live in per-thread registers and no
// compiler stage can fold them or treat them as uniform constants.
struct Rn {
    double one;       // +1.0
    double neg_zero;  // -0.0
    double zero;      // +0.0
    __device__ __forceinline__ double add(double a, double b) const { return __fma_rn(a, one, b); }
    __device__ __forceinline__ double sub(double a, double b) const { return __fma_rn(b, -one, a); }
    __device__ __forceinline__ double mul(double a, double b) const { return __fma_rn(a, b, neg_zero); }
    __device__ __forceinline__ double fma(double a, double b, double c) const { return __fma_rn(a, b, c); }

    // Sec. 2.1 as operation sequences on the FP64 pipe.
    // FastTwoSum (QuickTwoSum): s = fl(a + b), e = b - (s - a).
    __device__ __forceinline__ void quick_two_sum(double a, double b, double& s, double& e) const
    {
        const double sum = add(a, b);
        e = sub(b, sub(sum, a));
        s = sum;
    }
    // TwoSum: s = fl(a + b) and e = (a + b) - s exactly.
    __device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) const
    {
        const double sum = add(a, b);
        const double bv = sub(sum, a);
        const double av = sub(sum, bv);
        e = add(sub(a, av), sub(b, bv));
        s = sum;
    }
    // TwoProd with FMA: p = fl(a b), e = a b - p exactly.
    __device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) const
    {
        const double prod = mul(a, b);
        e = fma(a, b, -prod);
        p = prod;
    }
};

// Rn with the transformations that MASK names computed on the integer pipes
// from one exact sum or product (soft_fp64.cuh): bit 0 TwoSum, bit 1
// FastTwoSum, bit 2 TwoProd.  Each returns the same bits as Rn's sequence for
// every input, so a kernel may take any mask; the FP64 pipe then runs only
// the remaining operations while the integer pipes of the same warps run the
// rest.  RnInt<0> is Rn.
template <unsigned MASK>
struct RnInt : Rn {
    __device__ __forceinline__ explicit RnInt(const Rn& r) : Rn(r) {}
    __device__ __forceinline__ void quick_two_sum(double a, double b, double& s, double& e) const
    {
        if constexpr ((MASK & 2u) != 0u) {
            const soft::Pair r = soft::two_sum<true>(a, b);
            s = r.hi;
            e = r.lo;
        } else {
            Rn::quick_two_sum(a, b, s, e);
        }
    }
    __device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) const
    {
        if constexpr ((MASK & 1u) != 0u) {
            const soft::Pair r = soft::two_sum<false>(a, b);
            s = r.hi;
            e = r.lo;
        } else {
            Rn::two_sum(a, b, s, e);
        }
    }
    __device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) const
    {
        if constexpr ((MASK & 4u) != 0u) {
            const soft::Pair r = soft::two_prod(a, b);
            p = r.hi;
            e = r.lo;
        } else {
            Rn::two_prod(a, b, p, e);
        }
    }
};

static __device__ double rn_constants[96] = {
    1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0,
    1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0,
    -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0,
    -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0, -0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
    0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};

// The Rn constants, read through a volatile pointer at a lane-dependent
// address into per-thread registers.
__device__ __forceinline__ Rn make_rn()
{
    const volatile double* p = rn_constants;
    const int lane = static_cast<int>(threadIdx.x & 31u);
    return Rn{p[lane], p[32 + lane], p[64 + lane]};
}

// The bit tests below work on the two 32-bit words of a double.  Written on
// the whole 64-bit pattern they cost FP64-pipe instructions, which every
// kernel built on these helpers keeps saturated (measured on GB300: QDadd 93
// FP64-pipe instructions per element that way, 87 -- its arithmetic alone --
// with these); 64-bit integer shifts and compares by themselves stay off that
// pipe, so the one-word tests evidently become floating-point comparisons.

// x != 0 (true for every value but +0 and -0), tested on the bit pattern.
__device__ __forceinline__ bool nonzero(double x)
{
    return ((static_cast<unsigned>(__double2hiint(x)) << 1) | static_cast<unsigned>(__double2loint(x))) != 0u;
}

// |a| >= |b| for finite a, b: the bit patterns without the sign compared as
// unsigned integers, high words first.
__device__ __forceinline__ bool abs_ge(double a, double b)
{
    const unsigned ha = static_cast<unsigned>(__double2hiint(a)) & 0x7fffffffu;
    const unsigned hb = static_cast<unsigned>(__double2hiint(b)) & 0x7fffffffu;
    const unsigned la = static_cast<unsigned>(__double2loint(a));
    const unsigned lb = static_cast<unsigned>(__double2loint(b));
    return ha > hb || (ha == hb && la >= lb);
}

// ------------------------------------------------------------- Sec. 2.1

// The transformations of Sec. 2.1, as the policy f computes them.
template <class F>
__device__ __forceinline__ void quick_two_sum(const F& f, double a, double b, double& s, double& e)
{
    f.quick_two_sum(a, b, s, e);
}

template <class F>
__device__ __forceinline__ void two_sum(const F& f, double a, double b, double& s, double& e)
{
    f.two_sum(a, b, s, e);
}

template <class F>
__device__ __forceinline__ void two_prod(const F& f, double a, double b, double& p, double& e)
{
    f.two_prod(a, b, p, e);
}

// ------------------------------------------------- helpers of Alg. 3 - 6

// ThreeSum: (a, b, c) -> (a', b', c'), same exact sum.
template <class F>
__device__ __forceinline__ void three_sum(const F& f, double& a, double& b, double& c)
{
    double t1, t2, t3;
    two_sum(f, a, b, t1, t2);
    two_sum(f, c, t1, a, t3);
    two_sum(f, t2, t3, b, c);
}

// ThreeSum2: as ThreeSum with the two low terms added in one rounding.
template <class F>
__device__ __forceinline__ void three_sum2(const F& f, double& a, double& b, double c)
{
    double t1, t2, t3;
    two_sum(f, a, b, t1, t2);
    two_sum(f, c, t1, a, t3);
    b = f.add(t2, t3);
}

// Renorm of five terms into four: a bottom-up QuickTwoSum pass, then a
// top-down pass that emits a component whenever the QuickTwoSum error is
// nonzero, folding everything after the third emitted component into the
// fourth.  k counts emitted components; r_k selects stand in for indexing.
template <class F>
__device__ __forceinline__ void renorm5(const F& f, double c0, double c1, double c2, double c3, double c4,
                                        double& r0, double& r1, double& r2, double& r3)
{
    double s, t0, t1, t2, t3, t4;
    quick_two_sum(f, c3, c4, s, t4);
    quick_two_sum(f, c2, s, s, t3);
    quick_two_sum(f, c1, s, s, t2);
    quick_two_sum(f, c0, s, t0, t1);

    r0 = 0.0; r1 = 0.0; r2 = 0.0; r3 = 0.0;
    int k = 0;
    double hi, lo;
    bool emit;

    // term 1 (k == 0 here)
    quick_two_sum(f, t0, t1, hi, lo);
    emit = nonzero(lo);
    r0 = emit ? hi : r0;
    k = emit ? 1 : 0;
    s = emit ? lo : hi;

    // term 2 (k <= 1)
    quick_two_sum(f, s, t2, hi, lo);
    emit = nonzero(lo);
    r0 = (emit && k == 0) ? hi : r0;
    r1 = (emit && k == 1) ? hi : r1;
    k += emit ? 1 : 0;
    s = emit ? lo : hi;

    // term 3 (k <= 2)
    quick_two_sum(f, s, t3, hi, lo);
    emit = nonzero(lo);
    r0 = (emit && k == 0) ? hi : r0;
    r1 = (emit && k == 1) ? hi : r1;
    r2 = (emit && k == 2) ? hi : r2;
    k += emit ? 1 : 0;
    s = emit ? lo : hi;

    // term 4: with three components out, the sum is a plain add, which is
    // exactly the QuickTwoSum's rounded sum
    quick_two_sum(f, s, t4, hi, lo);
    emit = nonzero(lo) && k < 3;
    r0 = (emit && k == 0) ? hi : r0;
    r1 = (emit && k == 1) ? hi : r1;
    r2 = (emit && k == 2) ? hi : r2;
    k += emit ? 1 : 0;
    s = emit ? lo : hi;

    r0 = (k == 0) ? s : r0;
    r1 = (k == 1) ? s : r1;
    r2 = (k == 2) ? s : r2;
    r3 = (k == 3) ? s : r3;
}

// VecSum of three / four terms: TwoSum chain from the last term up.
template <class F>
__device__ __forceinline__ void vec_sum3(const F& f, double x0, double x1, double x2,
                                         double& e0, double& e1, double& e2)
{
    double s;
    two_sum(f, x1, x2, s, e2);
    two_sum(f, x0, s, e0, e1);
}

template <class F>
__device__ __forceinline__ void vec_sum4(const F& f, double x0, double x1, double x2, double x3,
                                         double& e0, double& e1, double& e2, double& e3)
{
    double s;
    two_sum(f, x2, x3, s, e3);
    two_sum(f, x1, s, s, e2);
    two_sum(f, x0, s, e0, e1);
}

// VSEB(2) on three terms.  Following the loop: the first QuickTwoSum writes
// r0 and either moves to r1 (nonzero error) or carries its sum on; the second
// writes the current slot; after it the loop returns if both slots are done,
// otherwise a nonzero remainder lands in the current slot.
template <class F>
__device__ __forceinline__ void vseb2_of3(const F& f, double e0, double e1, double e2, double& r0, double& r1)
{
    double h1, l1, h2, l2;
    quick_two_sum(f, e0, e1, h1, l1);
    const bool nz1 = nonzero(l1);
    quick_two_sum(f, nz1 ? l1 : h1, e2, h2, l2);
    const bool nz2 = nonzero(l2);
    r0 = nz1 ? h1 : h2;
    r1 = nz1 ? h2 : (nz2 ? l2 : 0.0);
}

// VSEB(3) on six terms (used by the merge-based TDadd).
template <class F>
__device__ __forceinline__ void vseb3_of6(const F& f, const double e[6], double& r0, double& r1, double& r2)
{
    r0 = 0.0; r1 = 0.0; r2 = 0.0;
    int j = 0;
    bool done = false;
    double eps = e[0];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double hi, lo;
        quick_two_sum(f, eps, e[i + 1], hi, lo);
        const bool w = !done;
        r0 = (w && j == 0) ? hi : r0;
        r1 = (w && j == 1) ? hi : r1;
        r2 = (w && j == 2) ? hi : r2;
        const bool nz = nonzero(lo);
        const bool finish = w && nz && j >= 2;
        const bool adv = w && nz && j < 2;
        eps = w ? (nz ? lo : hi) : eps;
        j += adv ? 1 : 0;
        done = done || finish;
    }
    const bool tail = !done && nonzero(eps);
    r0 = (tail && j == 0) ? eps : r0;
    r1 = (tail && j == 1) ? eps : r1;
    r2 = (tail && j == 2) ? eps : r2;
}

// ------------------------------------------------------------- Sec. 2.2

// Alg. 1, DDadd.
template <class F>
__device__ __forceinline__ void dd_add(const F& f, const double x[2], const double y[2], double r[2])
{
    double s, e;
    two_sum(f, x[0], y[0], s, e);
    const double w = f.add(x[1], y[1]);
    e = f.add(e, w);
    quick_two_sum(f, s, e, r[0], r[1]);
}

// Alg. 2, DDmul.
template <class F>
__device__ __forceinline__ void dd_mul(const F& f, const double x[2], const double y[2], double r[2])
{
    double p1, p2;
    two_prod(f, x[0], y[0], p1, p2);
    const double w1 = f.mul(x[0], y[1]);
    const double w2 = f.mul(x[1], y[0]);
    const double w3 = f.add(w1, w2);
    p2 = f.add(p2, w3);
    quick_two_sum(f, p1, p2, r[0], r[1]);
}

// ------------------------------------------------------------- Sec. 2.3

// Alg. 4, TDmul (the "fast" triple-word product).
template <class F>
__device__ __forceinline__ void td_mul(const F& f, const double x[3], const double y[3], double r[3])
{
    double z00up, z00lo, z01up, z01lo, z10up, z10lo;
    two_prod(f, x[0], y[0], z00up, z00lo);
    two_prod(f, x[0], y[1], z01up, z01lo);
    two_prod(f, x[1], y[0], z10up, z10lo);
    double b0, b1, b2;
    vec_sum3(f, z00lo, z01up, z10up, b0, b1, b2);
    const double c = f.fma(x[1], y[1], b2);
    const double z31 = f.fma(x[0], y[2], z10lo);
    const double z32 = f.fma(x[2], y[0], z01lo);
    const double z3 = f.add(z31, z32);
    const double s3 = f.add(c, z3);
    double e0, e1, e2, e3;
    vec_sum4(f, z00up, b0, b1, s3, e0, e1, e2, e3);
    r[0] = e0;
    vseb2_of3(f, e1, e2, e3, r[1], r[2]);
}

// ------------------------------------------------------------- Sec. 2.4

// Alg. 5, QDadd (sloppy); t3 is the error of the fourth componentwise sum.
// With ZERO4 the fourth components of both operands are +0 (TDaddq): then
// s3, v3, u3, w3 and t3 are all exactly +0 in round-to-nearest, and those six
// operations are replaced by the constant.
template <bool ZERO4, class F>
__device__ __forceinline__ void qd_add_impl(const F& f, const double x[4], const double y[4], double r[4])
{
    double s0, s1, s2, s3, t0, t1, t2, t3;
    two_sum(f, x[0], y[0], s0, t0);
    two_sum(f, x[1], y[1], s1, t1);
    two_sum(f, x[2], y[2], s2, t2);
    if (ZERO4) {
        s3 = f.zero;
        t3 = f.zero;
    } else {
        two_sum(f, x[3], y[3], s3, t3);
    }
    two_sum(f, s1, t0, s1, t0);
    three_sum(f, s2, t0, t1);
    three_sum2(f, s3, t0, t2);
    t0 = f.add(f.add(t0, t1), t3);
    renorm5(f, s0, s1, s2, s3, t0, r[0], r[1], r[2], r[3]);
}

template <class F>
__device__ __forceinline__ void qd_add(const F& f, const double x[4], const double y[4], double r[4])
{
    qd_add_impl<false>(f, x, y, r);
}

// TDaddq (Sec. 2.3): QDadd on operands padded with a zero fourth component,
// the fourth result component dropped.
template <class F>
__device__ __forceinline__ void td_addq(const F& f, const double x[3], const double y[3], double r[3])
{
    const double x4[4] = {x[0], x[1], x[2], f.zero};
    const double y4[4] = {y[0], y[1], y[2], f.zero};
    double r4[4];
    qd_add_impl<true>(f, x4, y4, r4);
    r[0] = r4[0];
    r[1] = r4[1];
    r[2] = r4[2];
}

// Alg. 3, TDadd: Merge (by decreasing magnitude, x first on ties), VecSum,
// VSEB(3).
template <class F>
__device__ __forceinline__ void td_add_merge(const F& f, const double x[3], const double y[3], double r[3])
{
    double z[6];
    int i = 0, j = 0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
        const double xi = (i == 0) ? x[0] : (i == 1) ? x[1] : x[2];
        const double yj = (j == 0) ? y[0] : (j == 1) ? y[1] : y[2];
        const bool takex = (j >= 3) || (i < 3 && abs_ge(xi, yj));
        z[o] = takex ? xi : yj;
        i += takex ? 1 : 0;
        j += takex ? 0 : 1;
    }
    double e[6];
    double s = z[5];
#pragma unroll
    for (int t = 4; t >= 0; --t)
        two_sum(f, z[t], s, s, e[t + 1]);
    e[0] = s;
    vseb3_of6(f, e, r[0], r[1], r[2]);
}

// Alg. 6, QDmul (sloppy).  The listing's first line is dead and omitted.
template <class F>
__device__ __forceinline__ void qd_mul(const F& f, const double x[4], const double y[4], double r[4])
{
    double p0, p1, p2, p3, p4, p5, q0, q1, q2, q3, q4, q5;
    two_prod(f, x[0], y[0], p0, q0);
    two_prod(f, x[0], y[1], p1, q1);
    two_prod(f, x[1], y[0], p2, q2);
    two_prod(f, x[0], y[2], p3, q3);
    two_prod(f, x[1], y[1], p4, q4);
    two_prod(f, x[2], y[0], p5, q5);
    three_sum(f, p1, p2, q0);
    three_sum(f, p2, q1, q2);
    three_sum(f, p3, p4, p5);
    double s0, s1, s2, t0, t1;
    two_sum(f, p2, p3, s0, t0);
    two_sum(f, q1, p4, s1, t1);
    s2 = f.add(q2, p5);
    two_sum(f, s1, t0, s1, t0);
    s2 = f.add(s2, f.add(t0, t1));
    s1 = f.add(s1, f.mul(x[0], y[3]));
    s1 = f.add(s1, f.mul(x[1], y[2]));
    s1 = f.add(s1, f.mul(x[2], y[1]));
    s1 = f.add(s1, f.mul(x[3], y[0]));
    s1 = f.add(s1, q0);
    s1 = f.add(s1, q3);
    s1 = f.add(s1, q4);
    s1 = f.add(s1, q5);
    renorm5(f, p0, p1, s0, s1, s2, r[0], r[1], r[2], r[3]);
}

// ------------------------------------------ variants of Sec. 2.3 - 2.4

// TDmulq (Sec. 2.3, the trial TD product): QDmul on operands padded with a
// zero fourth component, the fourth result component dropped.  The padding is
// the register zero, so every operation on it runs as written and the signs
// of zero results agree with the same steps on the host.
template <class F>
__device__ __forceinline__ void td_mulq(const F& f, const double x[3], const double y[3], double r[3])
{
    const double x4[4] = {x[0], x[1], x[2], f.zero};
    const double y4[4] = {y[0], y[1], y[2], f.zero};
    double r4[4];
    qd_mul(f, x4, y4, r4);
    r[0] = r4[0];
    r[1] = r4[1];
    r[2] = r4[2];
}

// Stable sort of N values by decreasing magnitude: the insertion sort
// unrolled into adjacent compare-exchanges that swap only when the later
// entry is strictly larger in magnitude.  Once an inserted value stops, the
// exchanges below it meet a sorted prefix and do nothing, so the network
// gives exactly the insertion sort's order, equal magnitudes unmoved.
template <int N>
__device__ __forceinline__ void sort_by_magnitude(double z[N])
{
#pragma unroll
    for (int i = 1; i < N; ++i) {
#pragma unroll
        for (int j = i; j > 0; --j) {
            const bool sw = !abs_ge(z[j - 1], z[j]);
            const double a = z[j - 1], b = z[j];
            z[j - 1] = sw ? b : a;
            z[j] = sw ? a : b;
        }
    }
}

// The normalisation of the accurate variants (after the IEEE-style QD
// addition of Hida, Li and Bailey): N sorted terms are added one by one into
// a two-term accumulator (u, v).  A term t gives (s1, e1) = TwoSum(v, t) and
// (s, e2) = TwoSum(u, s1); with both errors nonzero s is emitted as the next
// component and the accumulator becomes (e2, e1), otherwise s and the nonzero
// error.  After four components the accumulator and the remaining terms are
// summed into a fifth term with plain additions; if the terms run out first
// the accumulator's two terms follow the components.  Renorm ends it.  The
// emission count k selects the slot, so nothing is indexed dynamically.
template <int N, class F>
__device__ __forceinline__ void accumulate_sorted(const F& f, const double z[N], double r[4])
{
    double u, v;
    quick_two_sum(f, z[0], z[1], u, v);
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0, tail = 0.0;
    int k = 0;
#pragma unroll
    for (int i = 2; i < N; ++i) {
        const bool live = k < 4;
        double s1, e1, s, e2;
        two_sum(f, v, z[i], s1, e1);
        two_sum(f, u, s1, s, e2);
        const bool nz1 = nonzero(e1);
        const bool emit = live && nz1 && nonzero(e2);
        c0 = (emit && k == 0) ? s : c0;
        c1 = (emit && k == 1) ? s : c1;
        c2 = (emit && k == 2) ? s : c2;
        c3 = (emit && k == 3) ? s : c3;
        const double nu = emit ? e2 : s;
        const double nv = (emit || nz1) ? e1 : e2;
        // the term joins the tail once four components are out
        tail = live ? tail : f.add(tail, z[i]);
        u = live ? nu : u;
        v = live ? nv : v;
        k += emit ? 1 : 0;
        // the fourth emission starts the tail with the accumulator
        tail = (emit && k == 4) ? f.add(u, v) : tail;
    }
    const bool left = k < 4;
    const double c4 = left ? ((k == 3) ? v : 0.0) : tail;
    c3 = (left && k == 3) ? u : (left && k == 2) ? v : c3;
    c2 = (left && k == 2) ? u : (left && k == 1) ? v : c2;
    c1 = (left && k == 1) ? u : (left && k == 0) ? v : c1;
    c0 = (left && k == 0) ? u : c0;
    renorm5(f, c0, c1, c2, c3, c4, r[0], r[1], r[2], r[3]);
}

// Accurate TD product: every x_i y_j with i + j <= 2 split exactly by
// TwoProd; the order-three terms (the order-two products' errors, then x2 y1
// and x1 y2 by fma) summed with one rounding each; x2 y2 dropped.  The ten
// terms, stably sorted by decreasing magnitude, go through the accurate
// normalisation; the fourth component is dropped.
template <class F>
__device__ __forceinline__ void td_mul_acc(const F& f, const double x[3], const double y[3], double r[3])
{
    double z[10];
    double q02, q11, q20;
    two_prod(f, x[0], y[0], z[0], z[1]);
    two_prod(f, x[0], y[1], z[2], z[4]);
    two_prod(f, x[1], y[0], z[3], z[5]);
    two_prod(f, x[0], y[2], z[6], q02);
    two_prod(f, x[1], y[1], z[7], q11);
    two_prod(f, x[2], y[0], z[8], q20);
    double t3 = f.add(f.add(q02, q11), q20);
    t3 = f.fma(x[2], y[1], t3);
    z[9] = f.fma(x[1], y[2], t3);
    sort_by_magnitude<10>(z);
    double r4[4];
    accumulate_sorted<10>(f, z, r4);
    r[0] = r4[0];
    r[1] = r4[1];
    r[2] = r4[2];
}

// Accurate QD addition (the IEEE-style addition of Hida, Li and Bailey): the
// eight components stably sorted by decreasing magnitude, x first on ties,
// then the accurate normalisation.
template <class F>
__device__ __forceinline__ void qd_add_acc(const F& f, const double x[4], const double y[4], double r[4])
{
    double z[8] = {x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3]};
    sort_by_magnitude<8>(z);
    accumulate_sorted<8>(f, z, r);
}

// ------------------------------------------------ generic by component count

template <int P> struct Ops;
template <> struct Ops<2> {
    template <class F> static __device__ __forceinline__ void mul(const F& f, const double* x, const double* y, double* r) { dd_mul(f, x, y, r); }
    template <class F> static __device__ __forceinline__ void add(const F& f, const double* x, const double* y, double* r) { dd_add(f, x, y, r); }
};
template <> struct Ops<3> {
    template <class F> static __device__ __forceinline__ void mul(const F& f, const double* x, const double* y, double* r) { td_mul(f, x, y, r); }
    template <class F> static __device__ __forceinline__ void add(const F& f, const double* x, const double* y, double* r) { td_addq(f, x, y, r); }
};
template <> struct Ops<4> {
    template <class F> static __device__ __forceinline__ void mul(const F& f, const double* x, const double* y, double* r) { qd_mul(f, x, y, r); }
    template <class F> static __device__ __forceinline__ void add(const F& f, const double* x, const double* y, double* r) { qd_add(f, x, y, r); }
};

// acc = add(acc, mul(a, b)): one multiply-add of the GEMM, a from A, b from B.
// For P = 1 (the binary64-only product) it is acc = fma(a, b, acc), one
// rounding per term -- the plain FP64 GEMM the multi-component forms are
// compared with.
template <int P, class F>
__device__ __forceinline__ void mad(const F& f, double* acc, const double* a, const double* b)
{
    if constexpr (P == 1) {
        acc[0] = f.fma(a[0], b[0], acc[0]);
    } else {
        double prod[P], sum[P];
        Ops<P>::mul(f, a, b, prod);
        Ops<P>::add(f, acc, prod, sum);
#pragma unroll
        for (int c = 0; c < P; ++c) acc[c] = sum[c];
    }
}

}  // namespace mp
