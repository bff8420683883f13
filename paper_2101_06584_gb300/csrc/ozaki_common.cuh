// ozaki_common.cuh -- what the slicing form (ozaki.cu) and the CRT form (crt.cu)
// share: the scaled-integer machinery (digit and residue cursors), the
// scale and slice kernels, the tcgen05/TMA/mbarrier helpers, and the host
// side of slicing both operands and of the TMA tensor maps of the slices.
// Included by those two translation units only; everything here has
// internal linkage or is inline.
#pragma once
#include "mp_arith.cuh"
#include "ozaki.h"

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdlib>
#include <mutex>

namespace mpg {


namespace {

constexpr int TILE = 64;         // padding granularity of the rows of op(A) and op(B)
constexpr int KPAD = 128;        // padding granularity of k (the largest k-step)

__device__ __forceinline__ uint64_t abs_bits(double x)
{
    return static_cast<uint64_t>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// ilogb of a positive finite binary64 given by its magnitude bits.
__device__ __forceinline__ int ilogb_bits(uint64_t b)
{
    const int E = static_cast<int>(b >> 52);
    if (E) return E - 1023;
    const uint64_t frac = b & ((1ull << 52) - 1);
    return (63 - __clzll(static_cast<long long>(frac))) - 1074;
}

// Signed integer mantissa and exponent: x = M * 2^e (M = 0 for +-0).
__device__ __forceinline__ void decompose(double x, int64_t& M, int& e)
{
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(x));
    const int E = static_cast<int>((b >> 52) & 0x7ff);
    const uint64_t frac = b & ((1ull << 52) - 1);
    int64_t m;
    if (E == 0) { m = static_cast<int64_t>(frac); e = -1074; }
    else        { m = static_cast<int64_t>(frac | (1ull << 52)); e = E - 1075; }
    M = (b >> 63) ? -m : m;
}

// floor(W * 2^sh) and whether bits were dropped, for sh < 0.
__device__ __forceinline__ __int128 floor_shift(__int128 W, int sh, bool& frac)
{
    if (sh >= 0) { frac = false; return W << sh; }
    if (sh <= -127) { frac = (W != 0); return W < 0 ? -1 : 0; }
    const int r = -sh;
    const __int128 mask = (static_cast<__int128>(1) << r) - 1;
    frac = (W & mask) != 0;
    return W >> r;   // arithmetic shift: floor
}

// X = floor((hi + lo) 2^(F - sigma)) exactly, sticky = whether X is inexact.
__device__ __forceinline__ __int128 fixed_point(double hi, double lo, int sigma, int F, bool& sticky)
{
    int64_t Mh, Ml;
    int eh, el;
    decompose(hi, Mh, eh);
    decompose(lo, Ml, el);
    if (Mh == 0 && Ml != 0) { Mh = Ml; eh = el; Ml = 0; }
    int sh = eh - sigma + F, sl = el - sigma + F;
    if (Ml != 0 && sl > sh) {        // unnormalised input: larger exponent first
        const int64_t tm = Mh; Mh = Ml; Ml = tm;
        const int ts = sh; sh = sl; sl = ts;
    }
    if (Mh == 0) { sticky = false; return 0; }
    if (Ml == 0) return floor_shift(Mh, sh, sticky);
    if (sh >= 0) {
        bool f;
        const __int128 lowp = floor_shift(Ml, sl, f);
        sticky = f;
        return (static_cast<__int128>(Mh) << sh) + lowp;
    }
    const int d = sh - sl;            // > 0 here: lo below hi
    if (d <= 74) {
        const __int128 W = (static_cast<__int128>(Mh) << d) + Ml;
        return floor_shift(W, sl, sticky);
    }
    // lo lies more than 74 bits below hi's last bit: it only decides the
    // floor when hi is itself an integer in these units
    bool fh;
    __int128 X = floor_shift(Mh, sh, fh);
    if (!fh && Ml < 0) X -= 1;
    sticky = true;
    return X;
}

}  // namespace

// Digits of a fixed-point value held with the current digit's unit at bit
// 120 of a 128-bit two's-complement integer (hi, lo): |value| < 2^126.  Each
// step takes the nearest integer of value / 2^120 (ties to even unless
// `sticky` says the true value lies above the held one), subtracts it, and
// moves the next digit's unit up by the 7 bits of the base.
struct DigitCursor {
    uint64_t hi, lo;
    bool sticky;
    __device__ __forceinline__ int next()
    {
        const int64_t t = static_cast<int64_t>(hi + (1ull << 55)) >> 56;          // nearest, ties up
        const bool tie = lo == 0 && (hi & ((1ull << 56) - 1)) == (1ull << 55);
        const int64_t d = (tie && !sticky && (t & 1)) ? t - 1 : t;                // ties to even
        hi -= static_cast<uint64_t>(d) << 56;                                      // |value| <= 2^119
        hi = (hi << 7) | (lo >> 57);
        lo <<= 7;
        return static_cast<int>(d);
    }
};

// The digit cursor of (hi + lo) 2^-sigma with S digits: R = floor((hi + lo)
// 2^(F - sigma)), F = 7S + 12, |R| < 2^(F-1), shifted left by 115 - 7S so that
// the first digit's unit 2^(F-7) sits at bit 120.
__device__ __forceinline__ DigitCursor ozaki_cursor(double hi, double lo, int sigma, int S)
{
    const int F = 7 * S + 12;
    bool sticky;
    const unsigned __int128 R = static_cast<unsigned __int128>(fixed_point(hi, lo, sigma, F, sticky)) << (115 - 7 * S);
    return DigitCursor{static_cast<uint64_t>(R >> 64), static_cast<uint64_t>(R), sticky};
}

// ------------------------------------------------- wide digits (TD, QD)
//
// For P >= 3 components the S digits need up to 7S + 12 bits below the scale
// plus guard bits, beyond 128.  Each component is floored to a multiple of
// 2^(sigma - F - 64) (F = 7S + 12) and the floored parts are summed exactly
// in a 384-bit two's-complement integer (six 64-bit words, word 0 least
// significant); the digits are those of that sum, ties to even decided
// exactly.  Nothing of the method's arithmetic is approximated: the floor is
// part of the definition, 64 bits below the last digit.

constexpr int kWideWords = 6;
constexpr int kGuardBits = 64;

struct Wide {
    uint64_t w[kWideWords];
};

// W += M * 2^sh for a signed |M| < 2^53 and 0 <= sh (fits by construction).
__device__ __forceinline__ void wide_add_shifted(Wide& W, int64_t M, int sh)
{
    const int wi = sh >> 6, bo = sh & 63;
    const uint64_t ext = M < 0 ? ~0ull : 0ull;
    uint64_t part[kWideWords];
#pragma unroll
    for (int i = 0; i < kWideWords; ++i) part[i] = i < wi ? 0ull : ext;
    const uint64_t lo = static_cast<uint64_t>(M) << bo;
    const uint64_t hi = bo == 0 ? ext : static_cast<uint64_t>(M >> (64 - bo));
#pragma unroll
    for (int i = 0; i < kWideWords; ++i) {
        if (i == wi) part[i] = lo;
        if (i == wi + 1) part[i] = hi;
    }
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < kWideWords; ++i) {
        const uint64_t a = W.w[i], b = part[i];
        const uint64_t s1 = a + b;
        const uint64_t c1 = s1 < a;
        const uint64_t s2 = s1 + carry;
        const uint64_t c2 = s2 < s1;
        W.w[i] = s2;
        carry = c1 | c2;
    }
}

// W += v for a small signed v at bit 0.
__device__ __forceinline__ void wide_add_small(Wide& W, int64_t v)
{
    wide_add_shifted(W, v, 0);
}

// Digits of a 384-bit fixed-point value with the current digit's unit at bit
// 376 (|value| < 2^382); as DigitCursor, with every tie exact.
struct WideCursor {
    uint64_t w[kWideWords];
    __device__ __forceinline__ int next()
    {
        const int64_t t = static_cast<int64_t>(w[5] + (1ull << 55)) >> 56;        // nearest, ties up
        bool tie = (w[5] & ((1ull << 56) - 1)) == (1ull << 55);
#pragma unroll
        for (int i = 0; i < 5; ++i) tie = tie && w[i] == 0;
        const int64_t d = (tie && (t & 1)) ? t - 1 : t;                           // ties to even
        w[5] -= static_cast<uint64_t>(d) << 56;
#pragma unroll
        for (int i = 5; i > 0; --i) w[i] = (w[i] << 7) | (w[i - 1] >> 57);
        w[0] <<= 7;
        return static_cast<int>(d);
    }
};

// The digit cursor of the sum of the P components, each floored at
// 2^(sigma - F - 64), F = 7S + 12: the floored sum W (|W| < 2^(F+63)) shifted
// left by 307 - 7S so that the first digit's unit 2^(F+57) sits at bit 376.
template <int P>
__device__ __forceinline__ WideCursor ozaki_cursor_wide(const double (&c)[P], int sigma, int S)
{
    const int F = 7 * S + 12;
    Wide W;
#pragma unroll
    for (int i = 0; i < kWideWords; ++i) W.w[i] = 0ull;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        int64_t M;
        int e;
        decompose(c[i], M, e);
        if (M == 0) continue;
        const int sh = e - sigma + F + kGuardBits;
        if (sh >= 0) wide_add_shifted(W, M, sh);
        else if (sh > -64) wide_add_small(W, M >> (-sh));      // arithmetic shift: floor
        else wide_add_small(W, M < 0 ? -1 : 0);
    }
    // shift left by L = 307 - 7S (27 <= L <= 300): whole words first, with
    // unrolled selects so that W stays in registers, then the bits
    const int L = 307 - 7 * S, ws = L >> 6, bs = L & 63;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k < ws) {
#pragma unroll
            for (int i = kWideWords - 1; i > 0; --i) W.w[i] = W.w[i - 1];
            W.w[0] = 0ull;
        }
    }
    WideCursor cur;
#pragma unroll
    for (int i = kWideWords - 1; i > 0; --i) cur.w[i] = bs ? (W.w[i] << bs) | (W.w[i - 1] >> (64 - bs)) : W.w[i];
    cur.w[0] = W.w[0] << bs;
    return cur;
}

// ------------------------------------------------------- CRT residues
//
// The CRT form (Ozaki scheme II; not in the paper): each scaled entry of
// op(A) and op(B) becomes an integer A' (the nearest integer, ties to even,
// of the sum of its components each floored to a multiple of
// 2^(sigma - beta - 64), in units of 2^(sigma - beta)), whose residues modulo
// N pairwise coprime moduli m_i <= 256 -- symmetric representatives, so
// |r| <= 128, exact in int8 and in bf16 -- replace the digits of the slicing
// form.  The product of each residue pair is exact on the tensor cores; the
// integer product A'B' is recovered from its residues (Garner's mixed radix)
// and rounded to P binary64 components.

namespace crt {
constexpr int kMaxModuli = 49;
constexpr int kLimbs = 12;                        // |A'| < 2^192 in 16-bit limbs

struct Tables {
    int count;
    int m[kMaxModuli];                            // 256, 255, 253, 251, 247, ...
    uint32_t magic[kMaxModuli];                   // floor(2^32 / m) + 1
    uint32_t pw8[kMaxModuli][kLimbs / 2];         // byte t of word w: 2^(8 (4w + t)) mod m_i
    uint32_t big[kMaxModuli];                     // m_i ceil(2^28 / m_i): a multiple of m_i above every limb sum
    uint32_t half[kMaxModuli];                    // floor(m_i / 2)
};

constexpr int gcd_c(int a, int b)
{
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// The moduli: pairwise coprime integers taken greedily from 256 downward.
constexpr Tables make_tables()
{
    Tables t{};
    int n = 0;
    for (int m = 256; m > 1 && n < kMaxModuli; --m) {
        bool ok = true;
        for (int i = 0; i < n; ++i) ok = ok && gcd_c(m, t.m[i]) == 1;
        if (ok) t.m[n++] = m;
    }
    t.count = n;
    for (int i = 0; i < n; ++i) {
        const uint32_t m = static_cast<uint32_t>(t.m[i]);
        t.magic[i] = static_cast<uint32_t>((1ull << 32) / m + 1);
        for (int w = 0; w < kLimbs / 2; ++w) {
            uint32_t word = 0;
            for (int b = 0; b < 4; ++b) {
                uint32_t v = 1 % m;
                for (int e = 0; e < 4 * w + b; ++e) v = static_cast<uint32_t>((static_cast<uint64_t>(v) << 8) % m);
                word |= v << (8 * b);
            }
            t.pw8[i][w] = word;
        }
        t.big[i] = m * (((1u << 28) + m - 1) / m);
        t.half[i] = m / 2;
    }
    return t;
}

constexpr Tables kHost = make_tables();
static_assert(kHost.count == kMaxModuli, "49 pairwise coprime moduli up to 256");
static __constant__ Tables kDev = kHost;

// x mod m_i for x < 2^32 (one Barrett step: the estimate is the quotient or
// one more).
__device__ __forceinline__ uint32_t mod_small(uint32_t x, int i)
{
    const uint32_t m = static_cast<uint32_t>(kDev.m[i]);
    const uint32_t q = __umulhi(x, kDev.magic[i]);
    const int r = static_cast<int>(x - q * m);
    return static_cast<uint32_t>(r < 0 ? r + static_cast<int>(m) : r);
}
}  // namespace crt

// A' of the P components: each floored at 2^(sigma - beta - 64), summed
// exactly in WW 64-bit words (64 fraction bits below the unit 2^(sigma - beta)),
// rounded to the nearest integer (ties to even); in two's complement, WW - 1
// words, least significant first.  WW is the fewest words that hold the
// beta-bit integer with its sign and the fraction word (3 for beta <= 96 up to
// 6 for beta <= 316).
template <int WW>
__device__ __forceinline__ void wide_add_shifted_n(uint64_t (&W)[WW], int64_t M, int sh)
{
    const int wi = sh >> 6, bo = sh & 63;
    const uint64_t ext = M < 0 ? ~0ull : 0ull;
    const uint64_t lo = static_cast<uint64_t>(M) << bo;
    const uint64_t hi = bo == 0 ? ext : static_cast<uint64_t>(M >> (64 - bo));
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < WW; ++i) {
        const uint64_t b = i < wi ? 0ull : (i == wi ? lo : (i == wi + 1 ? hi : ext));
        const uint64_t s1 = W[i] + b;
        const uint64_t c1 = s1 < b;
        const uint64_t s2 = s1 + carry;
        const uint64_t c2 = s2 < s1;
        W[i] = s2;
        carry = c1 | c2;
    }
}

template <int P, int WW>
__device__ __forceinline__ void scaled_integer(const double (&c)[P], int sigma, int beta, uint64_t (&I)[WW - 1])
{
    uint64_t W[WW];
#pragma unroll
    for (int i = 0; i < WW; ++i) W[i] = 0ull;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        int64_t M;
        int e;
        decompose(c[i], M, e);
        if (M == 0) continue;
        const int sh = e - sigma + beta + kGuardBits;
        if (sh >= 0) wide_add_shifted_n<WW>(W, M, sh);
        else if (sh > -64) wide_add_shifted_n<WW>(W, M >> (-sh), 0);      // arithmetic shift: floor
        else wide_add_shifted_n<WW>(W, M < 0 ? -1 : 0, 0);
    }
    // integer part (words 1.., floor) and the fraction in word 0
    const uint64_t f = W[0];
    const bool up = f > (1ull << 63) || (f == (1ull << 63) && (W[1] & 1ull));
    uint64_t carry = up ? 1ull : 0ull;
#pragma unroll
    for (int i = 0; i < WW - 1; ++i) {
        const uint64_t v = W[i + 1] + carry;
        carry = (carry && v == 0) ? 1ull : 0ull;
        I[i] = v;
    }
}

// The magnitude of a scaled integer as NL / 2 32-bit words (NL 16-bit limbs),
// least significant first, and its sign.
template <int NL>
struct ResLimbs {
    uint32_t l[NL / 2];
    bool neg;
};

template <int NL, int WI>
__device__ __forceinline__ ResLimbs<NL> limbs_of(uint64_t (&I)[WI])
{
    static_assert(NL % 2 == 0 && NL <= 4 * WI, "limbs beyond the integer");
    ResLimbs<NL> x;
    x.neg = (I[WI - 1] >> 63) != 0;
    if (x.neg) {                                     // magnitude: two's complement negation
        uint64_t cc = 1;
#pragma unroll
        for (int i = 0; i < WI; ++i) {
            const uint64_t v = ~I[i] + cc;
            cc = (cc && v == 0) ? 1ull : 0ull;
            I[i] = v;
        }
    }
#pragma unroll
    for (int j = 0; j < NL / 2; ++j) x.l[j] = static_cast<uint32_t>(I[j / 2] >> (32 * (j % 2)));
    return x;
}

// The constants of modulus i, read once per plane and shared by the
// thread's elements.
template <int NL>
struct ModConst {
    uint32_t pw[NL / 2];                             // bytes 2^(8 j) mod m, four to a word
    uint32_t m, magic, big, half;
};

template <int NL>
__device__ __forceinline__ ModConst<NL> mod_const(int i)
{
    ModConst<NL> k;
#pragma unroll
    for (int j = 0; j < NL / 2; ++j) k.pw[j] = crt::kDev.pw8[i][j];
    k.m = static_cast<uint32_t>(crt::kDev.m[i]);
    k.magic = crt::kDev.magic[i];
    k.big = crt::kDev.big[i];
    k.half = crt::kDev.half[i];
    return k;
}

// The symmetric residue of (-1)^neg sum_j b_j 2^(8 j) modulo m (b_j the bytes
// of the magnitude), in [-floor(m/2), ceil(m/2) - 1]: s = sum_j b_j (2^(8 j)
// mod m), four bytes at a time (dp4a; s < 24 * 255 * 255 < 2^21), made
// nonnegative as big - s for a negative integer, shifted by floor(m/2) and
// reduced by one Barrett step (the estimate is the quotient or one more, and
// the unsigned minimum of r and r + m keeps the one in [0, m)).
template <int NL>
__device__ __forceinline__ int sym_residue(const ResLimbs<NL>& x, const ModConst<NL>& k)
{
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < NL / 2; ++j) s = __dp4a(x.l[j], k.pw[j], s);
    s = x.neg ? k.big - s : s;
    const uint32_t t = s + k.half;
    const uint32_t r0 = t - __umulhi(t, k.magic) * k.m;
    const uint32_t r1 = r0 + k.m;
    return static_cast<int>(r0 < r1 ? r0 : r1) - static_cast<int>(k.half);
}

template <int NL, int P, int WW>
__device__ __forceinline__ void residue_limbs(const double (&c)[P], int sigma, int beta, ResLimbs<NL>& hi)
{
    uint64_t I[WW - 1];
    scaled_integer<P, WW>(c, sigma, beta, I);
    hi = limbs_of<NL, WW - 1>(I);
}

// Word q of a WI-word two's-complement integer, its sign beyond the top.
template <int WI>
__device__ __forceinline__ uint64_t word_at(const uint64_t (&x)[WI], int q)
{
    uint64_t r = (x[WI - 1] >> 63) ? ~0ull : 0ull;
#pragma unroll
    for (int k = 0; k < WI; ++k) r = (k == q) ? x[k] : r;
    return r;
}

// Split integers: A' = A1 2^w + A0 with A0 in [-2^(w-1), 2^(w-1)); hi gets
// A1, lo gets A0 (w = beta / 2).
template <int NL, int P, int WWS>
__device__ __forceinline__ void split_limbs(const double (&c)[P], int sigma, int beta, ResLimbs<NL>& hi,
                                            ResLimbs<NL>& lo)
{
    constexpr int WW = WWS - 1;
    uint64_t I[WW];
    scaled_integer<P, WWS>(c, sigma, beta, I);
    const int w = beta / 2;
    // A0: the low w bits, sign-extended from bit w - 1
    const int wi = w >> 6, wb = w & 63;
    const bool low_neg = (word_at<WW>(I, (w - 1) >> 6) >> ((w - 1) & 63)) & 1ull;
    uint64_t A0[WW], D[WW];
#pragma unroll
    for (int k = 0; k < WW; ++k) {
        const uint64_t keep = k < wi ? ~0ull : (k == wi ? (wb ? ((1ull << wb) - 1) : 0ull) : 0ull);
        A0[k] = (I[k] & keep) | (low_neg ? ~keep : 0ull);
    }
    // A1 = (A' - A0) >> w, exact
    uint64_t borrow = 0;
#pragma unroll
    for (int k = 0; k < WW; ++k) {
        const uint64_t d = I[k] - A0[k] - borrow;
        borrow = (I[k] < A0[k] || (I[k] == A0[k] && borrow)) ? 1ull : 0ull;
        D[k] = d;
    }
    uint64_t A1[WW];
#pragma unroll
    for (int k = 0; k < WW; ++k) {
        const uint64_t a = word_at<WW>(D, k + wi), b = word_at<WW>(D, k + wi + 1);
        A1[k] = wb ? (a >> wb) | (b << (64 - wb)) : a;
    }
    hi = limbs_of<NL, WW>(A1);
    lo = limbs_of<NL, WW>(A0);
}

// ------------------------------------------------------------------ scale

// One warp per vector whose elements are contiguous (stride 1, vectors ld apart).
static __global__ void ozaki_scale_contig(const double* __restrict__ hi, int64_t count, int64_t len,
                                   int64_t ld, int* __restrict__ out)
{
    const int64_t v = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= count) return;
    uint64_t mx = 0;
    for (int64_t p = lane; p < len; p += 32) {
        const uint64_t b = abs_bits(hi[v * ld + p]);
        mx = b > mx ? b : mx;
    }
    for (int off = 16; off; off >>= 1) {
        const uint64_t o = __shfl_xor_sync(0xffffffffu, mx, off);
        mx = o > mx ? o : mx;
    }
    if (lane == 0) out[v] = mx ? ilogb_bits(mx) + 2 : 0;
}

// Vectors whose elements are ld apart (vectors adjacent): blocks of 32
// vectors x 32 warps, each over one chunk of `rows` elements, so that the
// grid covers the SMs even when the vectors are few (1024 columns are only
// 32 blocks of all the rows).  A block's maximum per vector goes into
// out[v] with an integer atomicMax as ilogb + 2 + kScaleBias (out zeroed
// beforehand; 0 stays for an all-zero vector); ozaki_scale_decode removes
// the bias.
constexpr int kScaleBias = 4096;                   // above -(ilogb + 2) of any binary64
static __global__ void __launch_bounds__(1024) ozaki_scale_strided(const double* __restrict__ hi, int64_t count,
                                                                    int64_t len, int64_t ld, int64_t rows,
                                                                    int* __restrict__ out)
{
    __shared__ unsigned long long smax[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t v = static_cast<int64_t>(blockIdx.x) * 32 + tx;
    const int64_t p0 = static_cast<int64_t>(blockIdx.y) * rows;
    const int64_t p1 = p0 + rows < len ? p0 + rows : len;
    if (ty == 0) smax[tx] = 0;
    __syncthreads();
    uint64_t mx = 0;
    if (v < count) {
#pragma unroll 4
        for (int64_t p = p0 + ty; p < p1; p += 32) {
            const uint64_t b = abs_bits(hi[p * ld + v]);
            mx = b > mx ? b : mx;
        }
    }
    atomicMax(&smax[tx], static_cast<unsigned long long>(mx));
    __syncthreads();
    if (ty == 0 && v < count) {
        const uint64_t m = smax[tx];
        if (m) atomicMax(out + v, ilogb_bits(m) + 2 + kScaleBias);
    }
}

// out[v] for v < count without the bias of ozaki_scale_strided; 0 for the
// padding up to `padded`.
static __global__ void ozaki_scale_decode(int* out, int64_t count, int64_t padded)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < count) out[i] = out[i] ? out[i] - kScaleBias : 0;
    else if (i < padded) out[i] = 0;
}

static __global__ void ozaki_fill_int(int* out, int64_t from, int64_t to)
{
    const int64_t i = from + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < to) out[i] = 0;
}

// ------------------------------------------------------------------ slice

// Slice storage: int8 digits for the int8 tensor path, or the same digits as
// bf16 (exact: |d| <= 64 needs 7 bits of significand) for the bf16 path.
template <typename T> struct DigitStore;
template <> struct DigitStore<int8_t> {
    static __device__ __forceinline__ uint32_t bits(int8_t d) { return static_cast<uint8_t>(d); }
    static constexpr int kBits = 8;
};
template <> struct DigitStore<uint16_t> {
    // |d| <= 128 is exact in binary32 (1.5 2^23 + d, less 1.5 2^23) and in
    // bf16, whose bits are then the upper half of the binary32's
    static __device__ __forceinline__ uint32_t bits(int8_t d)
    {
        const float f = __int_as_float(0x4B400000 + static_cast<int>(d)) - 12582912.0f;
        return __float_as_uint(f) >> 16;
    }
    static constexpr int kBits = 16;
};

// Four consecutive digits packed little-endian and stored at out (4 * sizeof(T) bytes).
template <typename T>
__device__ __forceinline__ void store4(T* out, int8_t d0, int8_t d1, int8_t d2, int8_t d3)
{
    if constexpr (sizeof(T) == 1) {
        *reinterpret_cast<uint32_t*>(out) = DigitStore<T>::bits(d0) | (DigitStore<T>::bits(d1) << 8) |
                                            (DigitStore<T>::bits(d2) << 16) | (DigitStore<T>::bits(d3) << 24);
    } else {
        uint2 v;
        v.x = DigitStore<T>::bits(d0) | (DigitStore<T>::bits(d1) << 16);
        v.y = DigitStore<T>::bits(d2) | (DigitStore<T>::bits(d3) << 16);
        *reinterpret_cast<uint2*>(out) = v;
    }
}

// Rows of the sliced operand are contiguous in memory (element (r, p) at
// base[r*ld + p]).  One thread per 4 consecutive p; rows up to `rows_pad`,
// columns up to kp, zero outside [rows) x [len).
template <int P>
struct Planes {
    const double* c[P];
};

// The digit cursor of element `off` of the component planes.
template <int P> struct CursorOf { using T = WideCursor; };
template <> struct CursorOf<2> { using T = DigitCursor; };

template <int P>
__device__ __forceinline__ typename CursorOf<P>::T element_cursor(const Planes<P>& pl, int64_t off, int sigma, int S)
{
    if constexpr (P == 2) {
        return ozaki_cursor(pl.c[0][off], pl.c[1][off], sigma, S);
    } else {
        double c[P];
#pragma unroll
        for (int i = 0; i < P; ++i) c[i] = pl.c[i][off];
        return ozaki_cursor_wide<P>(c, sigma, S);
    }
}
// A cursor whose digits are all zero (padding).
template <int P>
__device__ __forceinline__ typename CursorOf<P>::T zero_cursor()
{
    typename CursorOf<P>::T c;
    if constexpr (P == 2) {
        c.hi = 0;
        c.lo = 0;
        c.sticky = false;
    } else {
#pragma unroll
        for (int i = 0; i < kWideWords; ++i) c.w[i] = 0;
    }
    return c;
}

// KIND 0: the slicing form's digits (S of them).  KIND >= 1: the CRT
// form's residues, one plane per modulus, from the magnitude of each scaled
// integer in NL 16-bit limbs: KIND 1-4 one integer (S = N planes) with
// NL = 6, 8, 10, 12 (beta up to 96, 128, 160, 192 bits); KIND 5-7 split
// integers (S = 2N planes: A1's residues, then A0's) with NL = 6, 8, 12 per
// half (w = beta / 2 up to 96, 128, 192 bits).
constexpr int kind_limbs(int kind)
{
    return kind == 1 || kind == 5 ? 6 : kind == 2 || kind == 6 ? 8 : kind == 3 ? 10 : 12;
}
constexpr bool kind_split(int kind) { return kind >= 5; }
// 64-bit words of the exact sum of the components (fraction word included)
constexpr int kind_words(int kind)
{
    return kind == 1 ? 3 : kind <= 3 ? 4 : kind <= 5 ? 5 : 6;
}
constexpr int residue_kind(int beta, int halves = 1)
{
    if (halves == 2) return beta / 2 <= 96 ? 5 : beta / 2 <= 128 ? 6 : 7;
    return beta <= 96 ? 1 : beta <= 128 ? 2 : beta <= 160 ? 3 : 4;
}

template <int P, int KIND>
__device__ __forceinline__ typename CursorOf<P>::T make_cursor(const Planes<P>& pl, int64_t off, bool valid,
                                                               int sigma, int S)
{
    return valid ? element_cursor<P>(pl, off, sigma, S) : zero_cursor<P>();
}

// The limbs of element `off` (zero when not valid): hi, and lo with split
// integers.
template <int P, int KIND>
__device__ __forceinline__ void make_limbs(const Planes<P>& pl, int64_t off, bool valid, int sigma, int beta,
                                           ResLimbs<kind_limbs(KIND)>& hi, ResLimbs<kind_limbs(KIND)>& lo)
{
    constexpr int NL = kind_limbs(KIND);
    double c[P];
#pragma unroll
    for (int i = 0; i < P; ++i) c[i] = valid ? pl.c[i][off] : 0.0;
    if constexpr (kind_split(KIND)) split_limbs<NL, P, kind_words(KIND)>(c, sigma, beta, hi, lo);
    else residue_limbs<NL, P, kind_words(KIND)>(c, sigma, beta, hi);
}

// Plane s of the residues: modulus i of A1 (or of the one integer) for
// s < N, of A0 for s >= N with split integers.
template <int KIND>
__device__ __forceinline__ void residue_plane(int s, int S, int& i, bool& second)
{
    const int n = kind_split(KIND) ? S / 2 : S;
    second = kind_split(KIND) && s >= n;
    i = second ? s - n : s;
}

template <int P, typename T, int KIND = 0>
__global__ void ozaki_slice_rows(const Planes<P> pl, int64_t rows, int64_t len, int64_t ld,
                                 const int* __restrict__ sig, int S, int64_t rows_pad, int64_t kp,
                                 T* __restrict__ out, int beta = 0)
{
    const int64_t quads = kp / 4;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= rows_pad * quads) return;
    const int64_t r = t / quads;
    const int64_t p0 = (t % quads) * 4;
    const int sg = r < rows ? sig[r] : 0;
    T* o = out + r * kp + p0;
    const int64_t plane = rows_pad * kp;
    if constexpr (KIND == 0) {
        typename CursorOf<P>::T cur[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t p = p0 + u;
            cur[u] = make_cursor<P, KIND>(pl, r * ld + p, r < rows && p < len, sg, S);
        }
        for (int s = 0; s < S; ++s, o += plane) {
            const int d0 = cur[0].next(), d1 = cur[1].next(), d2 = cur[2].next(), d3 = cur[3].next();
            store4(o, static_cast<int8_t>(d0), static_cast<int8_t>(d1), static_cast<int8_t>(d2),
                   static_cast<int8_t>(d3));
        }
    } else {
        constexpr int NL = kind_limbs(KIND);
        ResLimbs<NL> hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t p = p0 + u;
            make_limbs<P, KIND>(pl, r * ld + p, r < rows && p < len, sg, beta, hi[u], lo[u]);
        }
        for (int s = 0; s < S; ++s, o += plane) {
            int i;
            bool second;
            residue_plane<KIND>(s, S, i, second);
            const ModConst<NL> k = mod_const<NL>(i);
            int d[4];
            if (second) {
#pragma unroll
                for (int u = 0; u < 4; ++u) d[u] = sym_residue<NL>(lo[u], k);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) d[u] = sym_residue<NL>(hi[u], k);
            }
            store4(o, static_cast<int8_t>(d[0]), static_cast<int8_t>(d[1]), static_cast<int8_t>(d[2]),
                   static_cast<int8_t>(d[3]));
        }
    }
}

// Rows of the sliced operand are strided (element (r, p) at base[p*ld + r]):
// a 32 x 32 tile is read with r fastest, sliced, transposed through shared
// memory and written with p fastest.
template <int P, typename T, int KIND = 0>
__global__ void __launch_bounds__(256)
ozaki_slice_cols(const Planes<P> pl, int64_t rows, int64_t len, int64_t ld,
                 const int* __restrict__ sig, int S, int64_t rows_pad, int64_t kp,
                 T* __restrict__ out, int beta = 0)
{
    constexpr int CHUNK = 16;               // digits (residues) staged per pass
    __shared__ int8_t tile[CHUNK][32][36];
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int64_t p0 = static_cast<int64_t>(blockIdx.y) * 32;
    const int tr = threadIdx.x & 31;        // r within the tile
    const int tp = threadIdx.x >> 5;        // 0..7: p = tp, tp + 8, tp + 16, tp + 24
    const int64_t r = r0 + tr;
    const int sg = r < rows ? sig[r] : 0;
    // write: each thread writes 4 consecutive p of one row r
    const int wr = threadIdx.x >> 3;        // 0..31 row within tile
    const int wq = (threadIdx.x & 7) * 4;   // p offset
    const int64_t row = r0 + wr;
    auto flush = [&](int s0, int cnt) {
        __syncthreads();
        if (row < rows_pad && p0 + wq < kp) {
            for (int s = 0; s < cnt; ++s)
                store4(out + (static_cast<int64_t>(s0 + s) * rows_pad + row) * kp + p0 + wq, tile[s][wr][wq],
                       tile[s][wr][wq + 1], tile[s][wr][wq + 2], tile[s][wr][wq + 3]);
        }
        __syncthreads();
    };
    if constexpr (KIND == 0) {
        typename CursorOf<P>::T cur[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t p = p0 + tp + 8 * u;
            cur[u] = make_cursor<P, KIND>(pl, p * ld + r, r < rows && p < len, sg, S);
        }
        for (int s0 = 0; s0 < S; s0 += CHUNK) {
            const int cnt = S - s0 < CHUNK ? S - s0 : CHUNK;
            for (int s = 0; s < cnt; ++s) {
#pragma unroll
                for (int u = 0; u < 4; ++u) tile[s][tr][tp + 8 * u] = static_cast<int8_t>(cur[u].next());
            }
            flush(s0, cnt);
        }
    } else {
        constexpr int NL = kind_limbs(KIND);
        ResLimbs<NL> hi[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t p = p0 + tp + 8 * u;
            make_limbs<P, KIND>(pl, p * ld + r, r < rows && p < len, sg, beta, hi[u], lo[u]);
        }
        for (int s0 = 0; s0 < S; s0 += CHUNK) {
            const int cnt = S - s0 < CHUNK ? S - s0 : CHUNK;
            for (int s = 0; s < cnt; ++s) {
                int i;
                bool second;
                residue_plane<KIND>(s0 + s, S, i, second);
                const ModConst<NL> k = mod_const<NL>(i);
                if (second) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) tile[s][tr][tp + 8 * u] = static_cast<int8_t>(sym_residue<NL>(lo[u], k));
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) tile[s][tr][tp + 8 * u] = static_cast<int8_t>(sym_residue<NL>(hi[u], k));
                }
            }
            flush(s0, cnt);
        }
    }
}

// ------------------------------------------------- cp.async and mma.sync

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------- tcgen05 helpers

namespace tc {
constexpr int BM = 128;
constexpr int KE = 64;                                   // box width in bf16 elements (128 bytes)
constexpr int KB = 2;                                    // boxes per stage: 128 values of k
constexpr int STAGES = 3;
constexpr int A_BYTES = BM * KE * 2;                     // one A box, 16 KB
constexpr int SEG_STAGES = 2048 / (KE * KB);             // stages per fp32 segment
static_assert(KPAD % (KE * KB) == 0, "stage k");
constexpr int TMEM_COLS = 512;
constexpr unsigned long long TIMEOUT_NS = 1000000000ull;

// Tile of TD and QD: TMEM holds two sets of two BN-column fp32 accumulators
// (one per weight of a block) and BN group sums of GW 32-bit words each
// (4 BN + GW BN <= 512).  A stage holds one A slice tile and the B slice tiles
// of the block's (at most) two weights.
template <int P> struct Cfg {
    static_assert(P == 3 || P == 4, "DD runs on CTA pairs");
    static constexpr int BN = 64;
    static constexpr int GW = 4;
    static constexpr int B_BYTES = BN * KE * 2;                   // one B box, 8 KB
    static constexpr int A_STAGE = KB * A_BYTES;                  // 32 KB
    static constexpr int B_STAGE = KB * B_BYTES;                  // 16 KB per weight
    static constexpr int STAGE_BYTES = A_STAGE + 2 * B_STAGE;     // 64 KB
    static constexpr int SET_COLS = 2 * BN;                  // accumulator sets at columns 0 and 2 BN
    static constexpr int GRP_COL = 4 * BN;
    static_assert(GRP_COL + GW * BN <= TMEM_COLS, "TMEM columns");
    // instruction descriptor: kind::f16, bf16 A and B (K-major), fp32 D, M = 128, N = BN
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                      ((static_cast<uint32_t>(BN) >> 3) << 17) | ((128u >> 4) << 24);
};
}  // namespace tc

struct TcArgs {
    const int* sig;
    const int* tau;
    double* C[4];
    int64_t ldc, m, n, kp;
    int S, tiles_m, tiles_n;
    int* err;
    long long* scratch;     // CTA-pair engine: per CTA, two [BN][BM] buffers of finished group sums
    int test_abort;         // test of the abort path: the producer gives up before its first load
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait with a suspend-time hint in ns.  Measured on GB300 in the MMA
// thread: any hint, against none, frees about 100 cycles per stage.
template <unsigned HINT>
__device__ __forceinline__ bool mbar_try_hint(uint64_t* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(HINT)
        : "memory");
    return ok != 0;
}
constexpr unsigned kHintIssue = 20;        // waits of the MMA-issuing thread
constexpr unsigned kHintIdle = 10000;      // waits of the producer and the epilogue
// Bounded wait: false after about a second, or once another role aborted.
template <unsigned HINT>
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag)
{
    if (mbar_try_hint<HINT>(b, parity)) return true;      // the common case reads no clock
    const unsigned long long t0 = gtimer();
    while (!mbar_try_hint<HINT>(b, parity)) {
        if (*abort_flag) return false;
        if (gtimer() - t0 > tc::TIMEOUT_NS) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    return static_cast<uint64_t>((saddr & 0x3FFFF) >> 4) | (1ull << 16) |
           (static_cast<uint64_t>(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void umma(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}
#define MPG_R32(r) "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), \
    "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), \
    "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), \
    "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
#define MPG_W32(r) "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), \
    "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), \
    "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), \
    "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : MPG_R32(r)
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        ::"r"(taddr), MPG_W32(r)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// A group sum as GW little-endian 32-bit TMEM words.
template <typename T, int GW>
__device__ __forceinline__ T group_load(const uint32_t* w)
{
    unsigned __int128 u = 0;
#pragma unroll
    for (int i = GW - 1; i >= 0; --i) u = (u << 32) | w[i];
    return static_cast<T>(u);
}
template <typename T, int GW>
__device__ __forceinline__ void group_store(uint32_t* w, T v)
{
#pragma unroll
    for (int i = 0; i < GW; ++i) w[i] = static_cast<uint32_t>(v >> (32 * i));
}

// ------------------------------------------------- CTA pairs (clusters of two)

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_index()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// The shared::cluster address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_cl(uint64_t* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
template <unsigned HINT>
__device__ __forceinline__ bool mbar_try_cl_hint(uint64_t* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity), "r"(HINT)
        : "memory");
    return ok != 0;
}
template <unsigned HINT>
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* b, unsigned parity, volatile int* abort_flag)
{
    if (mbar_try_cl_hint<HINT>(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_cl_hint<HINT>(b, parity)) {
        if (*abort_flag) return false;
        if (gtimer() - t0 > tc::TIMEOUT_NS) return false;
    }
    return true;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t caddr, int v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(caddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, int x, int y, int z,
                                                 uint32_t bar_caddr)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar_caddr)
        : "memory");
}
__device__ __forceinline__ void umma_pair(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
// Arrive on the barrier at this address in both CTAs once the MMAs issued so far complete.
__device__ __forceinline__ void umma_commit_both(uint64_t* bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
        ::"r"(smem_u32(bar)), "h"(static_cast<uint16_t>(3)) : "memory");
}
__device__ __forceinline__ void umma_commit_pair_local(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

// ------------------------------------------------------------------ host

static int64_t round_up(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

static unsigned blocks_for(int64_t threads, int per) { return static_cast<unsigned>((threads + per - 1) / per); }

// Slice one operand: vectors (rows of op(A) or columns of op(B)) of length
// len; `contig` says whether a vector's elements are adjacent in memory.
template <int P, typename T, int KIND = 0>
static cudaError_t slice_operand(const Planes<P>& pl, int64_t count, int64_t len, int64_t ld,
                                 bool contig, int S, int64_t count_pad, int64_t kp, T* out,
                                 int* sig, cudaStream_t s, int beta = 0)
{
    const double* lead = pl.c[0];
    if (contig) {
        ozaki_scale_contig<<<blocks_for(count * 32, 256), 256, 0, s>>>(lead, count, len, ld, sig);
        if (count_pad > count)
            ozaki_fill_int<<<blocks_for(count_pad - count, 256), 256, 0, s>>>(sig, count, count_pad);
    } else {
        // row chunks so that about two blocks per SM run
        const int64_t col_blocks = (count + 31) / 32;
        const int64_t want = col_blocks > 0 ? (2 * static_cast<int64_t>(num_sms()) + col_blocks - 1) / col_blocks : 1;
        int64_t rows = (len + want - 1) / want;
        rows = rows < 256 ? 256 : (rows + 31) / 32 * 32;
        const int64_t chunks = len > 0 ? (len + rows - 1) / rows : 1;
        if (chunks > 65535) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(sig, 0, static_cast<size_t>(count) * sizeof(int), s);
        if (e != cudaSuccess) return e;
        if (count > 0)
            ozaki_scale_strided<<<dim3(static_cast<unsigned>(col_blocks), static_cast<unsigned>(chunks)), 1024, 0, s>>>(
            lead, count, len, ld, rows, sig);
        if (count_pad > 0) ozaki_scale_decode<<<blocks_for(count_pad, 256), 256, 0, s>>>(sig, count, count_pad);
    }
    if (contig) {
        ozaki_slice_rows<P, T, KIND><<<blocks_for(count_pad * (kp / 4), 128), 128, 0, s>>>(
            pl, count, len, ld, sig, S, count_pad, kp, out, beta);
    } else {
        const dim3 grid(static_cast<unsigned>(count_pad / 32), static_cast<unsigned>(kp / 32));
        ozaki_slice_cols<P, T, KIND><<<grid, 256, 0, s>>>(pl, count, len, ld, sig, S, count_pad, kp, out, beta);
    }
    return cudaGetLastError();
}

// A second stream for slicing op(B) while op(A) is sliced on the caller's
// stream (the two are independent and neither fills the GPU alone), with the
// events that fork it from and join it back to the caller's stream, so the
// call stays ordered on that stream and can be captured into a CUDA graph.
// One set per host thread and device: concurrent callers never share events.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    unsigned long long ctx = 0;     // the context they were created in
    ~SideStream()
    {
        // at thread exit; errors (e.g. a runtime already unloaded) are moot
        if (join) cudaEventDestroy(join);
        if (fork) cudaEventDestroy(fork);
        if (s) cudaStreamDestroy(s);
    }
};

// The calling thread's side stream and events on the current device
// (created on first use; one set per host thread and device).
cudaError_t side_stream(SideStream** out);

// Slices op(A) on stream s and op(B) on the side stream, joined back to s.
template <int P, typename T, int KIND = 0>
static cudaError_t slice_both(const GemmArgs<P>& g, int S, const OzakiLayout& L, T* sa, T* sb, int* sig,
                              int* tau, cudaStream_t s, int beta = 0)
{
    Planes<P> pa, pb;
    for (int c = 0; c < P; ++c) {
        pa.c[c] = g.A[c];
        pb.c[c] = g.B[c];
    }
    SideStream* ss = nullptr;
    cudaError_t e = side_stream(&ss);
    if (e == cudaSuccess) e = cudaEventRecord(ss->fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->s, ss->fork, 0);
    // op(A) row i: contiguous unless A is stored transposed; op(B) column j:
    // contiguous only if B is stored transposed
    if (e == cudaSuccess)
        e = slice_operand<P, T, KIND>(pb, g.n, g.k, g.ldb, g.trans_b != 0, S, L.np, L.kp, sb, tau, ss->s, beta);
    if (e == cudaSuccess) e = cudaEventRecord(ss->join, ss->s);
    if (e == cudaSuccess)
        e = slice_operand<P, T, KIND>(pa, g.m, g.k, g.lda, !g.trans_a, S, L.mp, L.kp, sa, sig, s, beta);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ss->join, 0);
    return e;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// A [S][rows][kp] bf16 slice array as a 3-D TMA tensor; boxes of 64 (k) x
// box_rows x 1, 128-byte swizzle (the UMMA K-major layout).
static bool slice_map(CUtensorMap* map, void* base, int S, int64_t rows, int64_t kp, int box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {static_cast<cuuint64_t>(kp), static_cast<cuuint64_t>(rows),
                                static_cast<cuuint64_t>(S)};
    const cuuint64_t strides[2] = {static_cast<cuuint64_t>(kp) * 2, static_cast<cuuint64_t>(rows * kp) * 2};
    const cuuint32_t box[3] = {tc::KE, static_cast<cuuint32_t>(box_rows), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Test of the tcgen05 engines' abort path: with MPGEMM_TEST_TC_ABORT=1 in the
// environment the producer gives up before issuing any load, as if its first
// bounded wait had run out; every other role then finds the abort flag with
// nothing in flight, the kernel releases TMEM and returns, and the workspace
// header holds code 1 (C is not computed).
static int tc_test_abort()
{
    const char* v = getenv("MPGEMM_TEST_TC_ABORT");
    return v && v[0] == '1' && v[1] == '\0';
}

}  // namespace mpg
