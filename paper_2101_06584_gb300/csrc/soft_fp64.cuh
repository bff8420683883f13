// soft_fp64.cuh -- the error-free transformations of Sec. 2.1 computed on the
// integer pipes, with the bits of the binary64 operation sequences.
//
// GB300 issues about two FP64 lanes per clock per SM, a small fraction of its
// integer throughput.  The transformations are the bulk of every DD/TD/QD
// multiply-add, and each has a plain definition: TwoSum(a, b) =
// (fl(a + b), a + b - fl(a + b)) and TwoProd(a, b) = (fl(a b),
// fl(a b - fl(a b))), round to nearest even.  Computed from ONE exact integer
// sum (or product) of the significands, both outputs come out of a single
// alignment and rounding, where the floating-point sequences need six
// (TwoSum), three (FastTwoSum) or two (TwoProd) rounded operations.  The
// results are the bits those sequences give, signed zeros included, for every
// finite input whose sum does not overflow; the other inputs (non-finite
// operands, an overflowing sum or product, a product error below the
// subnormal range, FastTwoSum with |b| > |a|) run the sequence itself on the
// FP64 pipe, out of line -- inline, the compiler may if-convert it into
// predicated FP64 instructions that issue on every call.
//
// Representation used throughout: a finite nonzero x is m 2^(e - 1075) with
// an integer significand m < 2^53 and an effective biased exponent e >= 1
// (m has bit 52 set for normal numbers, e = 1 for subnormal ones).
//
// Rounding of a sum: the larger operand's significand is placed at bit 56,
// leaving four bits below its last place, and the smaller one is aligned
// below it with one extra bit.  That is the aligned value shifted left by
// one, with its lowest bit set when anything was shifted out.  The set bit
// stands for a remainder strictly inside (0, 2) units of that bit, and the
// computed sum or difference is then odd, so the exact result lies strictly
// between the two even integers next to it: the computed bits from bit 1 up
// are those of the exact result, and the set lowest bit marks its nonzero
// remainder.  Rounding at bit 4 (guard bit 3, sticky bits 0-2, after at most
// a one-place normalisation when a bit was shifted out) therefore rounds the
// exact result, for subtraction as well as addition.
#pragma once
#include <cstdint>

namespace mp {
namespace soft {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kFrac = 0x000fffffffffffffull;
constexpr uint64_t kHidden = 0x0010000000000000ull;

// Classification reads the two 32-bit words of a double.  A test written on
// the whole 64-bit pattern (zero, infinite or NaN, a nonzero exponent, the
// sign) can be turned back into a floating-point comparison by the compiler,
// which then occupies the FP64 pipe these routines exist to spare; tests on
// one word cannot.
struct Words {
    unsigned hi, lo;
};
__device__ __forceinline__ Words words(double x)
{
    return Words{static_cast<unsigned>(__double2hiint(x)), static_cast<unsigned>(__double2loint(x))};
}
__device__ __forceinline__ double from_bits(uint64_t b) { return __longlong_as_double(static_cast<long long>(b)); }
// Infinity or NaN.
__device__ __forceinline__ bool special(Words w) { return (w.hi & 0x7ff00000u) == 0x7ff00000u; }
// +0 or -0.
__device__ __forceinline__ bool is_zero(Words w) { return ((w.hi << 1) | w.lo) == 0u; }
// |a| > |b| for finite a, b.
__device__ __forceinline__ bool mag_gt(Words a, Words b)
{
    const unsigned ha = a.hi & 0x7fffffffu, hb = b.hi & 0x7fffffffu;
    return ha > hb || (ha == hb && a.lo > b.lo);
}
// The biased exponent field, the sign bit (as kSign or 0) and the fraction.
__device__ __forceinline__ int expo(Words w) { return static_cast<int>((w.hi >> 20) & 0x7ffu); }
__device__ __forceinline__ uint64_t sign_of(Words w) { return static_cast<uint64_t>(w.hi & 0x80000000u) << 32; }
__device__ __forceinline__ uint64_t frac(Words w)
{
    return (static_cast<uint64_t>(w.hi & 0x000fffffu) << 32) | w.lo;
}

// The significand of a finite nonzero x normalised to bit 52 and its
// exponent (below 1 for subnormal x).
__device__ __forceinline__ void unpack_normalised(Words w, uint64_t& m, int& e)
{
    const int ef = expo(w);
    const uint64_t f = frac(w);
    if (ef) {
        m = f | kHidden;
        e = ef;
    } else {
        const int sh = __clzll(static_cast<long long>(f)) - 11;
        m = f << sh;
        e = 1 - sh;
    }
}

// sign | q 2^(e - 1075) for q < 2^53 (a q below 2^52 is subnormal, then e
// is 1); e >= 2047 gives infinity.
__device__ __forceinline__ double pack(uint64_t sign, uint64_t q, int e)
{
    if (e >= 2047) return from_bits(sign | 0x7ff0000000000000ull);
    const uint64_t field = (q >> 52) ? static_cast<uint64_t>(e) : 0ull;
    return from_bits(sign | (field << 52) | (q & kFrac));
}

// sign | mag 2^(eu - 1075), eu >= 1, for a value known to be representable
// (no bit is lost: the error terms of the transformations).
__device__ __forceinline__ double exact_scaled(uint64_t sign, uint64_t mag, int eu)
{
    const int L = 63 - __clzll(static_cast<long long>(mag));
    const int e = eu + L - 52;
    if (e >= 1) {
        const uint64_t q = L >= 52 ? (mag >> (L - 52)) : (mag << (52 - L));
        return from_bits(sign | (static_cast<uint64_t>(e) << 52) | (q & kFrac));
    }
    return from_bits(sign | (mag << (eu - 1)));
}

// The rounded sum of |X| >= |Y| (finite, Y nonzero): significand q < 2^53
// and exponent e of fl(X + Y), or q = 0 for an exact zero.  mx, my, ex, ey
// as in the header.
__device__ __forceinline__ void round_sum(uint64_t mx, int ex, uint64_t my, int ey, bool subtract, uint64_t& q,
                                          int& e)
{
    const int d = ex - ey;
    const uint64_t xa = mx << 4;
    const uint64_t xb = my << 3;
    uint64_t yb;
    if (d < 64) {
        const uint64_t al = xb >> d;
        const uint64_t lost = (d != 0 && (xb << (64 - d)) != 0ull) ? 1ull : 0ull;
        yb = (al << 1) | lost;
    } else {
        yb = 1ull;
    }
    uint64_t r = subtract ? xa - yb : xa + yb;
    e = ex;
    if (r == 0ull) {
        q = 0ull;
        return;
    }
    if (r >> 57) {
        r = (r >> 1) | (r & 1ull);
        ++e;
    } else {
        const int lz = __clzll(static_cast<long long>(r)) - 7;
        const int sh = lz < e - 1 ? lz : e - 1;
        r <<= sh;
        e -= sh;
    }
    q = r >> 4;
    const bool g = (r >> 3) & 1ull;
    const bool below = (r & 7ull) != 0ull;
    q += (g && (below || (q & 1ull))) ? 1ull : 0ull;
    if (q >> 53) {
        q >>= 1;
        ++e;
    }
}

// The significand and effective exponent of a finite nonzero operand.
__device__ __forceinline__ void operand(Words w, uint64_t& m, int& e)
{
    const int ef = expo(w);
    m = frac(w) | (ef ? kHidden : 0ull);
    e = ef ? ef : 1;
}

// The two outputs of a transformation.
struct Pair {
    double hi, lo;
};

// The operation sequences on the FP64 pipe, for the rare inputs.
static __device__ __noinline__ Pair two_sum_seq(double a, double b)
{
    const double s = __dadd_rn(a, b);
    const double bv = __dsub_rn(s, a);
    const double av = __dsub_rn(s, bv);
    return Pair{s, __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv))};
}

static __device__ __noinline__ Pair fast_two_sum_seq(double a, double b)
{
    const double s = __dadd_rn(a, b);
    return Pair{s, __dsub_rn(b, __dsub_rn(s, a))};
}

static __device__ __noinline__ Pair two_prod_seq(double x, double y)
{
    const double p = __dmul_rn(x, y);
    return Pair{p, __fma_rn(x, y, -p)};
}

// TwoSum (QUICK false) or FastTwoSum (QUICK true) of (a, b): s = fl(a + b)
// and the error e, returned with exactly the bits of the operation sequences
//   TwoSum:      s = a + b, bv = s - a, av = s - bv, e = (a - av) + (b - bv)
//   FastTwoSum:  s = a + b, e = b - (s - a).
// Both sequences give e = a + b - s exactly whenever FastTwoSum's |a| >= |b|
// holds (and always for TwoSum); an exact zero error is +0 except that
// FastTwoSum returns b itself when b is a zero.
//
// The error comes from the exact sum in units of the smaller operand's last
// place u:  a + b = (mx 2^d +- my) u  and  s = q 2^(es - ey) u, so
// e / u = (mx 2^d +- my) - q 2^(es - ey).  |e| <= ulp(s) / 2 keeps that
// difference below 2^55, so it is computed modulo 2^64 although the two
// terms may not fit.  A gap d > 54 leaves s = the larger operand and e = the
// smaller one (|smaller| < a quarter of the larger one's last place).
template <bool QUICK>
__device__ __forceinline__ Pair two_sum(double a, double b)
{
    Words X = words(a), Y = words(b);
    if (special(X) || special(Y)) return QUICK ? fast_two_sum_seq(a, b) : two_sum_seq(a, b);
    if (mag_gt(Y, X)) {
        if (QUICK) return fast_two_sum_seq(a, b);
        const Words t = X;
        X = Y;
        Y = t;
    }
    if (is_zero(Y)) {
        const double s = is_zero(X) ? from_bits(sign_of(X) & sign_of(Y)) : __hiloint2double(X.hi, X.lo);
        return Pair{s, QUICK ? b : from_bits(0ull)};
    }
    const uint64_t sa = sign_of(X);
    const bool subtract = ((X.hi ^ Y.hi) >> 31) != 0u;
    uint64_t mx, my;
    int ex, ey;
    operand(X, mx, ex);
    operand(Y, my, ey);
    const int d = ex - ey;
    if (d > 54) return Pair{__hiloint2double(X.hi, X.lo), __hiloint2double(Y.hi, Y.lo)};
    uint64_t q;
    int es;
    round_sum(mx, ex, my, ey, subtract, q, es);
    if (q == 0ull) return Pair{from_bits(0ull), from_bits(0ull)};
    if (es >= 2047) return QUICK ? fast_two_sum_seq(a, b) : two_sum_seq(a, b);   // overflow
    const double s = pack(sa, q, es);
    const int sh = es - ey;
    if (sh <= 0) return Pair{s, from_bits(0ull)};                                  // s is exact
    const uint64_t R = subtract ? (mx << d) - my : (mx << d) + my;
    const int64_t ei = static_cast<int64_t>(R - (q << sh));
    if (ei == 0) return Pair{s, from_bits(0ull)};
    const uint64_t mag = ei < 0 ? static_cast<uint64_t>(-ei) : static_cast<uint64_t>(ei);
    return Pair{s, exact_scaled(sa ^ (ei < 0 ? kSign : 0ull), mag, ey)};
}

// TwoProd: p = fl(x y) and e = fl(x y - p), the bits of the sequence
// p = x * y, e = fma(x, y, -p).  From the exact 106-bit product P of the
// significands, p is P rounded at bit s (52 or 53) and e / 2^(ea + eb - 2150)
// = P - q 2^s, at most 2^(s-1) in magnitude, so it is computed from the low
// 64 bits of P.  That e is representable needs its last place 2^(ea + eb -
// 2150) at or above 2^-1074, i.e. ea + eb >= 1076.  A zero operand gives
// p = the signed zero and e = +0.
__device__ __forceinline__ Pair two_prod(double x, double y)
{
    const Words a = words(x), b = words(y);
    if (special(a) || special(b)) return two_prod_seq(x, y);
    const uint64_t sign = sign_of(a) ^ sign_of(b);
    if (is_zero(a) || is_zero(b)) return Pair{from_bits(sign), from_bits(0ull)};
    uint64_t ma, mb;
    int ea, eb;
    unpack_normalised(a, ma, ea);
    unpack_normalised(b, mb, eb);
    const uint64_t lo = ma * mb;
    const uint64_t hi = __umul64hi(ma, mb);
    const int top = (hi >> 41) ? 105 : 104;
    int E = ea + eb - 1023 + (top - 104);
    if (ea + eb < 1076 || E >= 2046) return two_prod_seq(x, y);
    const int s = top - 52;
    uint64_t q = (hi << (64 - s)) | (lo >> s);
    const bool g = (lo >> (s - 1)) & 1ull;
    const bool below = (lo & ((1ull << (s - 1)) - 1ull)) != 0ull;
    q += (g && (below || (q & 1ull))) ? 1ull : 0ull;
    const int64_t rem = static_cast<int64_t>(lo - (q << s));
    if (q >> 53) {
        q >>= 1;
        ++E;
    }
    const double p = from_bits(sign | (static_cast<uint64_t>(E) << 52) | (q & kFrac));
    if (rem == 0) return Pair{p, from_bits(0ull)};
    const uint64_t mag = rem < 0 ? static_cast<uint64_t>(-rem) : static_cast<uint64_t>(rem);
    return Pair{p, exact_scaled(sign ^ (rem < 0 ? kSign : 0ull), mag, ea + eb - 1075)};
}

}  // namespace soft
}  // namespace mp
