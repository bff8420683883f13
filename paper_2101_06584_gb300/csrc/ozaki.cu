// ozaki.cu -- the INT8 error-free slicing form of the DD GEMM, C := op(A) op(B).
//
// Not in the paper: the product of Sec. 3 (Eq. 1) in DD computed with an
// Ozaki-style error-free splitting so that the multiplications run on the
// tensor cores, with binary64 kept to the slicing and to the error-free
// accumulation of the slice products into DD.
//
//   scale   sigma_i = ilogb(max_p |hi(a_ip)|) + 2 for row i of op(A), tau_j for
//           column j of op(B) (0 for an all-zero vector): |a| 2^-sigma < 1/2.
//   slice   x_0 = a 2^-sigma; for s = 1..S: y = 2^7 x_{s-1}, d_s = nearest
//           integer to y (ties to even), x_s = y - d_s.  |d_s| <= 64, so the
//           digits are int8.  Computed exactly in 128-bit fixed point.
//   product for w = S+1 down to 2: P_w = sum over s + t = w of A^(s) B^(t),
//           int8 x int8 -> int32 on the tensor cores (mma.sync m16n8k32 s8;
//           GB300's tcgen05 has no int8 kind).  Exact while
//           S * k * 64 * 64 < 2^31.
//   accumulate  acc = DDadd(acc, (P_w 2^(sigma_i + tau_j - 7w), 0)) (Alg. 1),
//           the int32 turned into that exact binary64 with integer operations.
//
// Workspace (caller-provided, 256-byte aligned), with mp, np, kp the sizes
// rounded up to 64 and the padding zero:
//   [S][mp][kp] int8 slices of op(A), row-major;
//   [S][np][kp] int8 slices of op(B)^T (column j of op(B) as a row);
//   [mp] int32 sigma; [np] int32 tau.
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
    uint32_t pw16[kMaxModuli][kLimbs];            // 2^(16 j) mod m_i
    uint32_t pm[kMaxModuli][kMaxModuli];          // (m_0 ... m_(j-1)) mod m_i, j < i
    uint32_t inv[kMaxModuli];                     // (m_0 ... m_(i-1))^-1 mod m_i
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
        uint32_t p = 1;
        for (int j = 0; j < kLimbs; ++j) {
            t.pw16[i][j] = p;
            p = static_cast<uint32_t>((static_cast<uint64_t>(p) << 16) % m);
        }
        uint32_t q = 1 % m;
        for (int j = 0; j < i; ++j) {
            t.pm[i][j] = q;
            q = static_cast<uint32_t>((static_cast<uint64_t>(q) * static_cast<uint32_t>(t.m[j])) % m);
        }
        uint32_t inv = 0;
        for (uint32_t x = 1; x < m; ++x)
            if ((static_cast<uint64_t>(q) * x) % m == 1) { inv = x; break; }
        t.inv[i] = i == 0 ? 1 % m : inv;
    }
    return t;
}

constexpr Tables kHost = make_tables();
static_assert(kHost.count == kMaxModuli, "49 pairwise coprime moduli up to 256");
__constant__ Tables kDev = kHost;

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

// Residues of one scaled entry, one modulus per next(): the symmetric
// representative of A' mod m_i, i = 0, 1, ...  NL 16-bit limbs hold |A'|
// (|A'| <= 2^(beta - 1): NL = 4, 8 or 12 for beta up to 64, 128, 192).
template <int NL>
struct ResidueCursor {
    uint32_t limb[NL];                // |A'| in 16-bit limbs, least significant first
    bool neg;
    int idx;
    __device__ __forceinline__ int next()
    {
        const int i = idx++;
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < NL; ++j) s += limb[j] * crt::kDev.pw16[i][j];
        const int m = crt::kDev.m[i];
        int r = static_cast<int>(crt::mod_small(s, i));
        if (neg && r) r = m - r;
        return r >= (m + 1) / 2 ? r - m : r;
    }
};

// A' of the P components: each floored at 2^(sigma - beta - 64), summed
// exactly in 384 bits, rounded to the nearest integer (ties to even) in units
// of 2^(sigma - beta); in two's complement, five 64-bit words, least
// significant first (beta <= 316).
template <int P>
__device__ __forceinline__ void scaled_integer(const double (&c)[P], int sigma, int beta, uint64_t (&I)[kWideWords - 1])
{
    Wide W;
#pragma unroll
    for (int i = 0; i < kWideWords; ++i) W.w[i] = 0ull;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        int64_t M;
        int e;
        decompose(c[i], M, e);
        if (M == 0) continue;
        const int sh = e - sigma + beta + kGuardBits;
        if (sh >= 0) wide_add_shifted(W, M, sh);
        else if (sh > -64) wide_add_small(W, M >> (-sh));      // arithmetic shift: floor
        else wide_add_small(W, M < 0 ? -1 : 0);
    }
    // integer part (words 1..5, floor) and the fraction in word 0
    const uint64_t f = W.w[0];
    const bool up = f > (1ull << 63) || (f == (1ull << 63) && (W.w[1] & 1ull));
#pragma unroll
    for (int i = 0; i < kWideWords - 1; ++i) I[i] = W.w[i + 1];
    uint64_t carry = up ? 1ull : 0ull;
#pragma unroll
    for (int i = 0; i < kWideWords - 1; ++i) {
        const uint64_t s = I[i] + carry;
        carry = (carry && s == 0) ? 1ull : 0ull;
        I[i] = s;
    }
}

// The residue cursor of a two's-complement integer: its sign and magnitude
// in NL 16-bit limbs.
template <int NL>
__device__ __forceinline__ ResidueCursor<NL> cursor_of(uint64_t (&I)[kWideWords - 1])
{
    ResidueCursor<NL> cur;
    cur.neg = (I[kWideWords - 2] >> 63) != 0;
    if (cur.neg) {                                   // magnitude: two's complement negation
        uint64_t cc = 1;
#pragma unroll
        for (int i = 0; i < kWideWords - 1; ++i) {
            const uint64_t s = ~I[i] + cc;
            cc = (cc && s == 0) ? 1ull : 0ull;
            I[i] = s;
        }
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) cur.limb[j] = static_cast<uint32_t>(I[j / 4] >> (16 * (j % 4))) & 0xffffu;
    cur.idx = 0;
    return cur;
}

template <int NL, int P>
__device__ __forceinline__ ResidueCursor<NL> residue_cursor(const double (&c)[P], int sigma, int beta)
{
    uint64_t I[kWideWords - 1];
    scaled_integer<P>(c, sigma, beta, I);
    return cursor_of<NL>(I);
}

// Word q of a five-word two's-complement integer, its sign beyond the top.
__device__ __forceinline__ uint64_t word_at(const uint64_t (&x)[kWideWords - 1], int q)
{
    uint64_t r = (x[kWideWords - 2] >> 63) ? ~0ull : 0ull;
#pragma unroll
    for (int k = 0; k < kWideWords - 1; ++k) r = (k == q) ? x[k] : r;
    return r;
}

// Split integers: residues of A1 for moduli 0..N-1, then of A0, where
// A' = A1 2^w + A0 with A0 in [-2^(w-1), 2^(w-1)).
template <int NL>
struct SplitResidueCursor {
    ResidueCursor<NL> hi, lo;
    int n, idx;
    __device__ __forceinline__ int next() { return idx++ < n ? hi.next() : lo.next(); }
};

template <int NL, int P>
__device__ __forceinline__ SplitResidueCursor<NL> split_residue_cursor(const double (&c)[P], int sigma, int beta,
                                                                       int n)
{
    constexpr int WW = kWideWords - 1;
    uint64_t I[WW];
    scaled_integer<P>(c, sigma, beta, I);
    const int w = beta / 2;
    // A0: the low w bits, sign-extended from bit w - 1
    const int wi = w >> 6, wb = w & 63;
    const bool low_neg = (word_at(I, (w - 1) >> 6) >> ((w - 1) & 63)) & 1ull;
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
        const uint64_t a = word_at(D, k + wi), b = word_at(D, k + wi + 1);
        A1[k] = wb ? (a >> wb) | (b << (64 - wb)) : a;
    }
    SplitResidueCursor<NL> cur;
    cur.hi = cursor_of<NL>(A1);
    cur.lo = cursor_of<NL>(A0);
    cur.n = n;
    cur.idx = 0;
    return cur;
}

// ------------------------------------------------------------------ scale

// One warp per vector whose elements are contiguous (stride 1, vectors ld apart).
__global__ void ozaki_scale_contig(const double* __restrict__ hi, int64_t count, int64_t len,
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

// Vectors whose elements are ld apart (vectors adjacent): a block of 32 x 32
// threads covers 32 vectors, each column of threads a 32-way split of the
// elements (coalesced rows of 32 vectors), reduced in shared memory.
__global__ void __launch_bounds__(1024) ozaki_scale_strided(const double* __restrict__ hi, int64_t count,
                                                           int64_t len, int64_t ld, int* __restrict__ out)
{
    __shared__ unsigned long long smax[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t v = static_cast<int64_t>(blockIdx.x) * 32 + tx;
    if (ty == 0) smax[tx] = 0;
    __syncthreads();
    uint64_t mx = 0;
    if (v < count) {
#pragma unroll 4
        for (int64_t p = ty; p < len; p += 32) {
            const uint64_t b = abs_bits(hi[p * ld + v]);
            mx = b > mx ? b : mx;
        }
    }
    atomicMax(&smax[tx], static_cast<unsigned long long>(mx));
    __syncthreads();
    if (ty == 0 && v < count) {
        const uint64_t m = smax[tx];
        out[v] = m ? ilogb_bits(m) + 2 : 0;
    }
}

// Zero the exponent padding [count, padded).
__global__ void ozaki_fill_int(int* out, int64_t from, int64_t to)
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
    static __device__ __forceinline__ uint32_t bits(int8_t d)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(static_cast<float>(d)));
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

// KIND 0: the slicing form's digits (S of them); KIND 1: the CRT form's
// residues (S moduli, beta bits per scaled entry).
// KIND 1, 2, 3: residues with 12, 8 or 4 limbs (beta up to 192, 128, 64 bits);
// KIND 4, 5: split integers (2N planes: A1's residues, then A0's) with 8 or
// 12 limbs per half (w = beta / 2 up to 128 or 192 bits).
template <int P, int KIND> struct KindCursor { using T = typename CursorOf<P>::T; };
template <int P> struct KindCursor<P, 1> { using T = ResidueCursor<12>; };
template <int P> struct KindCursor<P, 2> { using T = ResidueCursor<8>; };
template <int P> struct KindCursor<P, 3> { using T = ResidueCursor<4>; };
template <int P> struct KindCursor<P, 4> { using T = SplitResidueCursor<8>; };
template <int P> struct KindCursor<P, 5> { using T = SplitResidueCursor<12>; };
constexpr int residue_kind(int beta, int halves = 1)
{
    return halves == 2 ? (beta / 2 <= 128 ? 4 : 5) : (beta <= 64 ? 3 : beta <= 128 ? 2 : 1);
}

template <int P, int KIND>
__device__ __forceinline__ typename KindCursor<P, KIND>::T make_cursor(const Planes<P>& pl, int64_t off, bool valid,
                                                                      int sigma, int S, int beta)
{
    if constexpr (KIND == 0) {
        return valid ? element_cursor<P>(pl, off, sigma, S) : zero_cursor<P>();
    } else if constexpr (KIND <= 3) {
        double c[P];
#pragma unroll
        for (int i = 0; i < P; ++i) c[i] = valid ? pl.c[i][off] : 0.0;
        return residue_cursor<KIND == 1 ? 12 : KIND == 2 ? 8 : 4, P>(c, sigma, beta);
    } else {
        double c[P];
#pragma unroll
        for (int i = 0; i < P; ++i) c[i] = valid ? pl.c[i][off] : 0.0;
        return split_residue_cursor<KIND == 4 ? 8 : 12, P>(c, sigma, beta, S / 2);
    }
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
    typename KindCursor<P, KIND>::T cur[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t p = p0 + u;
        cur[u] = make_cursor<P, KIND>(pl, r * ld + p, r < rows && p < len, sg, S, beta);
    }
    T* o = out + r * kp + p0;
    const int64_t plane = rows_pad * kp;
    for (int s = 0; s < S; ++s, o += plane) {
        const int d0 = cur[0].next(), d1 = cur[1].next(), d2 = cur[2].next(), d3 = cur[3].next();
        store4(o, static_cast<int8_t>(d0), static_cast<int8_t>(d1), static_cast<int8_t>(d2), static_cast<int8_t>(d3));
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
    typename KindCursor<P, KIND>::T cur[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t p = p0 + tp + 8 * u;
        cur[u] = make_cursor<P, KIND>(pl, p * ld + r, r < rows && p < len, sg, S, beta);
    }
    // write: each thread writes 4 consecutive p of one row r
    const int wr = threadIdx.x >> 3;        // 0..31 row within tile
    const int wq = (threadIdx.x & 7) * 4;   // p offset
    const int64_t row = r0 + wr;
    for (int s0 = 0; s0 < S; s0 += CHUNK) {
        const int cnt = S - s0 < CHUNK ? S - s0 : CHUNK;
        for (int s = 0; s < cnt; ++s) {
#pragma unroll
            for (int u = 0; u < 4; ++u) tile[s][tr][tp + 8 * u] = static_cast<int8_t>(cur[u].next());
        }
        __syncthreads();
        if (row < rows_pad && p0 + wq < kp) {
            for (int s = 0; s < cnt; ++s)
                store4(out + (static_cast<int64_t>(s0 + s) * rows_pad + row) * kp + p0 + wq, tile[s][wr][wq],
                       tile[s][wr][wq + 1], tile[s][wr][wq + 2], tile[s][wr][wq + 3]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ product

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

// u 2^E as binary64 (0 < u <= 2^53), assembled from its bits with integer
// operations only: the group-end splits run next to the FP64 additions, and
// integer <-> binary64 conversions would share the FP64 pipe with them.  As
// ldexp of the binary64 u by E: exact in the normal range; below it rounded
// to the nearest multiple of 2^-1074, ties to even (gradual underflow; a part
// that rounds to zero keeps its sign); above it +-inf.  `exact` is cleared
// when the result is not u 2^E exactly.
__device__ __forceinline__ double pow2_scaled(bool neg, uint64_t u, int E, bool& exact)
{
    const int msb = 63 - __clzll(static_cast<long long>(u));
    const int ef = msb + E + 1023;                    // biased exponent of the leading bit
    const uint64_t sign = static_cast<uint64_t>(neg) << 63;
    if (ef >= 2047) {
        exact = false;
        return __longlong_as_double(static_cast<long long>(sign | 0x7ff0000000000000ull));
    }
    if (ef >= 1) {
        const uint64_t mant = msb <= 52 ? (u << (52 - msb)) & ((1ull << 52) - 1) : 0ull;   // u = 2^53: 0
        return __longlong_as_double(static_cast<long long>(sign | (static_cast<uint64_t>(ef) << 52) | mant));
    }
    // below the normal range: in units of 2^-1074 the value is u 2^t, and
    // msb + t <= 51, so a left shift stays below 2^52
    const int t = E + 1074;
    uint64_t m;
    if (t >= 0) {
        m = u << t;
    } else if (t <= -64) {
        m = 0;                                        // u <= 2^53: below half a unit
        exact = false;
    } else {
        const int sr = -t;
        const uint64_t q = u >> sr, rem = u & ((1ull << sr) - 1), half = 1ull << (sr - 1);
        m = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
        if (rem) exact = false;
    }
    return __longlong_as_double(static_cast<long long>(sign | m));   // m = 2^52 is the least normal
}

// The split of the magnitude u (< 2^128) of a group sum: q 2^sh = RN(u) with
// q <= 2^53 (ties to even), rest = u - q 2^sh (|rest| <= 2^(sh-1)).
__device__ __forceinline__ void round53(unsigned __int128 u, uint64_t& q, int& sh, int64_t& rest)
{
    const uint64_t uh = static_cast<uint64_t>(u >> 64), ul = static_cast<uint64_t>(u);
    const int nb = uh ? 128 - __clzll(static_cast<long long>(uh)) : 64 - __clzll(static_cast<long long>(ul));
    sh = 0;
    rest = 0;
    if (nb <= 53) {
        q = ul;
        return;
    }
    sh = nb - 53;
    q = static_cast<uint64_t>(u >> sh);
    const uint64_t rem = static_cast<uint64_t>(u - (static_cast<unsigned __int128>(q) << sh));
    const uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) {
        q += 1;
        rest = static_cast<int64_t>(rem) - static_cast<int64_t>(1ull << sh);
    } else {
        rest = static_cast<int64_t>(rem);
    }
}

// The split of a group sum v times 2^e: hi = RN(v) 2^e (ties to even), lo =
// (v - RN(v)) 2^e, each scaled as pow2_scaled does; a zero remainder is +0.
// Returns whether both parts are exact (always, unless a part leaves the
// normal binary64 range).
__device__ __forceinline__ bool split_parts(bool neg, uint64_t q, int sh, int64_t rest, int e, double& hi, double& lo)
{
    bool exact = true;
    hi = pow2_scaled(neg, q, sh + e, exact);
    lo = rest == 0 ? 0.0
                   : pow2_scaled(neg != (rest < 0), static_cast<uint64_t>(rest < 0 ? -rest : rest), e, exact);
    return exact;
}
__device__ __forceinline__ bool split_exact(long long v, int e, double& hi, double& lo)
{
    if (v == 0) {
        hi = 0.0;
        lo = 0.0;
        return true;
    }
    const bool neg = v < 0;
    const uint64_t u = neg ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
    const int nb = 64 - __clzll(static_cast<long long>(u));
    const int sh = nb > 53 ? nb - 53 : 0;
    uint64_t q = u >> sh;
    int64_t rest = 0;
    if (sh) {
        const uint64_t rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) {
            q += 1;
            rest = static_cast<int64_t>(rem) - static_cast<int64_t>(1ull << sh);
        } else {
            rest = static_cast<int64_t>(rem);
        }
    }
    return split_parts(neg, q, sh, rest, e, hi, lo);
}
__device__ __forceinline__ bool split_exact(__int128 v, int e, double& hi, double& lo)
{
    if (v == 0) {
        hi = 0.0;
        lo = 0.0;
        return true;
    }
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
    uint64_t q;
    int sh;
    int64_t rest;
    round53(u, q, sh, rest);
    return split_parts(neg, q, sh, rest, e, hi, lo);
}

// The exact group sums of precision P: 64-bit integers for DD, 128-bit for TD and QD.
template <int P> struct GroupSum { using T = __int128; };
template <> struct GroupSum<2> { using T = long long; };

struct OzakiGemmArgs {
    const void* sa;     // [S][mp][kp] digits (int8 or bf16)
    const void* sb;     // [S][np][kp]
    const int* sig;     // [mp]
    const int* tau;     // [np]
    double* C[4];       // the P output planes
    int64_t ldc, m, n, mp, np, kp;
    int S;
};

// Iteration cursor over (weight w, pair s, k tile), weights from S+1 down to 2.
struct Cursor {
    int w, s, kt;
    __device__ __forceinline__ void advance(int S, int KT)
    {
        if (++kt < KT) return;
        kt = 0;
        const int smax = w - 1 < S ? w - 1 : S;
        if (++s <= smax) return;
        --w;
        s = w - S > 1 ? w - S : 1;
    }
};

// Iteration of the CTA-pair engine: the groups of G weights from the least
// significant (S+1, ..., S+2-G, then the next G, ...), and inside a group
// the slice s of op(A) outermost: for s = 1, 2, ..., every weight w of the
// group with w > s, largest first, then the k tiles of the pair (s, w - s).
// Consecutive pairs share their A slice, which then stays in L2, while each
// pair still fills its own accumulator segments; the integer group sums do
// not depend on the order in which their weights' products arrive.
struct GroupCursor {
    int wtop, wbot;     // the current group's weights
    int s, w, kt;
    __device__ __forceinline__ void begin(int S, int G, int top)
    {
        wtop = top;
        wbot = top - G + 1 > 2 ? top - G + 1 : 2;
        s = 1;
        w = top;
        kt = 0;
        (void)S;
    }
    // the next stage; pair_end / group_end describe the stage just passed
    __device__ __forceinline__ void advance(int S, int G, int KT, bool& pair_end, bool& group_end)
    {
        pair_end = false;
        group_end = false;
        if (++kt < KT) return;
        kt = 0;
        pair_end = true;
        const int wlow = wbot > s + 1 ? wbot : s + 1;
        if (w - 1 >= wlow) {
            --w;
            return;
        }
        const int smax = wtop - 1 < S ? wtop - 1 : S;
        if (s + 1 <= smax) {
            ++s;
            w = wtop;
            return;
        }
        group_end = true;
        if (wbot > 2) begin(S, G, wbot - 1);
    }
};

// CTA of WM x WN warps; each warp owns MT x NT fragments of 16 x 8 outputs,
// so the CTA tile is (WM*MT*16) x (WN*NT*8).  Slice tiles of KS bytes of k
// are staged through a STG-deep cp.async pipeline.  P output components;
// ozaki_group(P) weights are combined exactly in integers and each group is
// added, split exactly into two binary64, with the precision's add.
template <int P, int MT, int NT, int WM, int WN, int STG, int MINB, int KS>
__global__ void __launch_bounds__(WM * WN * 32, MINB) ozaki_gemm_kernel(const OzakiGemmArgs g)
{
    constexpr int NTHR = WM * WN * 32;
    constexpr int BM = WM * MT * 16;
    constexpr int BN = WN * NT * 8;
    constexpr int SROW = KS + 16;     // smem row stride in bytes: conflict-free fragment loads
    constexpr int CPR = KS / 16;      // 16-byte chunks per row
    __shared__ __align__(16) int8_t As[STG][BM * SROW];
    __shared__ __align__(16) int8_t Bs[STG][BN * SROW];

    const mp::Rn f = mp::make_rn();
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int wm = warp / WN, wn = warp % WN;
    const int64_t m0 = static_cast<int64_t>(blockIdx.y) * BM;
    const int64_t n0 = static_cast<int64_t>(blockIdx.x) * BN;
    const int S = g.S;
    const int KT = static_cast<int>(g.kp / KS);
    const int total = (S * (S + 1) / 2) * KT;

    // exponents of this thread's rows and columns
    int sg[MT][2], tu[NT][2];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) sg[mt][h] = g.sig[m0 + wm * MT * 16 + mt * 16 + gq + h * 8];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) tu[nt][h] = g.tau[n0 + wn * NT * 8 + nt * 8 + 2 * tq + h];

    double acc[MT][NT][4][P];
    int ci[MT][NT][4];
    using G = typename GroupSum<P>::T;
    constexpr int kGroup = ozaki_group(P);
    G grp[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int c = 0; c < P; ++c) acc[mt][nt][r][c] = 0.0;
                ci[mt][nt][r] = 0;
                grp[mt][nt][r] = 0;
            }

    auto load = [&](int stage, const Cursor& c) {
        const int8_t* a = static_cast<const int8_t*>(g.sa) +
                          ((static_cast<int64_t>(c.s - 1) * g.mp + m0) * g.kp) + static_cast<int64_t>(c.kt) * KS;
        const int8_t* b = static_cast<const int8_t*>(g.sb) +
                          ((static_cast<int64_t>(c.w - c.s - 1) * g.np + n0) * g.kp) + static_cast<int64_t>(c.kt) * KS;
        // (BM + BN) rows of KS bytes in 16-byte chunks
        for (int chunk = tid; chunk < (BM + BN) * CPR; chunk += NTHR) {
            const int row = chunk / CPR, col = (chunk % CPR) * 16;
            if (row < BM)
                cp_async16(&As[stage][row * SROW + col], a + static_cast<int64_t>(row) * g.kp + col);
            else
                cp_async16(&Bs[stage][(row - BM) * SROW + col],
                           b + static_cast<int64_t>(row - BM) * g.kp + col);
        }
    };

    Cursor ld{S + 1, 1, 0}, cm{S + 1, 1, 0};
#pragma unroll
    for (int st = 0; st < STG - 1; ++st) {
        if (st < total) load(st, ld);
        ld.advance(S, KT);
        cp_async_commit();
    }

    for (int it = 0; it < total; ++it) {
        cp_async_wait<STG - 2>();
        __syncthreads();
        {
            const int nxt = it + STG - 1;
            if (nxt < total) load(nxt % STG, ld);
            ld.advance(S, KT);
            cp_async_commit();
        }
        const int8_t* as = As[it % STG];
        const int8_t* bs = Bs[it % STG];
#pragma unroll
        for (int kk = 0; kk < KS; kk += 32) {
            uint32_t af[MT][4], bf[NT][2];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int r = wm * MT * 16 + mt * 16 + gq;
                af[mt][0] = *reinterpret_cast<const uint32_t*>(as + r * SROW + kk + 4 * tq);
                af[mt][1] = *reinterpret_cast<const uint32_t*>(as + (r + 8) * SROW + kk + 4 * tq);
                af[mt][2] = *reinterpret_cast<const uint32_t*>(as + r * SROW + kk + 16 + 4 * tq);
                af[mt][3] = *reinterpret_cast<const uint32_t*>(as + (r + 8) * SROW + kk + 16 + 4 * tq);
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int c = wn * NT * 8 + nt * 8 + gq;
                bf[nt][0] = *reinterpret_cast<const uint32_t*>(bs + c * SROW + kk + 4 * tq);
                bf[nt][1] = *reinterpret_cast<const uint32_t*>(bs + c * SROW + kk + 16 + 4 * tq);
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) mma_s8(ci[mt][nt], af[mt], bf[nt]);
        }
        // end of a weight: fold its exact integer sums into the accumulators
        const int w = cm.w;
        cm.advance(S, KT);
        if (cm.w != w || it == total - 1) {
            // position of w in its group, counted from the least significant
            // weight S+1; the group ends at its last weight or at w = 2
            const int j = (S + 1 - w) % kGroup;
            const bool group_end = j == kGroup - 1 || w == 2;
            const int wmax = w + j;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        grp[mt][nt][r] += static_cast<G>(ci[mt][nt][r]) << (7 * j);
                        ci[mt][nt][r] = 0;
                        if (group_end) {
                            double y[P];
                            split_exact(grp[mt][nt][r], sg[mt][r >> 1] + tu[nt][r & 1] - 7 * wmax, y[0], y[1]);
#pragma unroll
                            for (int c = 2; c < P; ++c) y[c] = f.zero;
                            double z[P];
                            mp::Ops<P>::add(f, acc[mt][nt][r], y, z);
#pragma unroll
                            for (int c = 0; c < P; ++c) acc[mt][nt][r][c] = z[c];
                            grp[mt][nt][r] = 0;
                        }
                    }
        }
    }
    cp_async_wait<0>();

#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int64_t row = m0 + wm * MT * 16 + mt * 16 + gq + (r >> 1) * 8;
                const int64_t col = n0 + wn * NT * 8 + nt * 8 + 2 * tq + (r & 1);
                if (row < g.m && col < g.n) {
#pragma unroll
                    for (int c = 0; c < P; ++c) g.C[c][row * g.ldc + col] = acc[mt][nt][r][c];
                }
            }
}

// ------------------------------------------------------- CRT products
//
// One modulus per grid z: Q_i = R_A,i R_B,i^T on mma.sync m16n8k32 s8 (exact
// int32: |Q_i| <= k 2^14 < 2^31), reduced to its symmetric residue mod m_i
// and stored as int8 [N][mp][np].  With split integers three products per
// modulus (grid z = 3N): hh = R(A1) R(B1)^T, mid = R(A1) R(B0)^T +
// R(A0) R(B1)^T (two k loops into one accumulator, |mid| <= 2k 2^14 < 2^31),
// ll = R(A0) R(B0)^T.  CTA of WM x WN warps, MT x NT fragments
// of 16 x 8 per warp, KS bytes of k per cp.async stage (STG stages).

struct CrtGemmArgs {
    const int8_t* ra;       // [N][mp][kp] residues of op(A) ([2N]: A1's, then A0's, with split integers)
    const int8_t* rb;       // [N][np][kp] residues of op(B)^T (likewise)
    int8_t* out;            // [N][mp][np] residues of the products ([3N]: hh, mid, ll)
    int64_t mp, np, kp;
    int N, split;
};

// Split integers: the operand planes of sub-product s of modulus i (s = 0:
// A1 B1, 1: A1 B0, 2: A0 B1, 3: A0 B0) and the product each one adds to
// (0: hh, 1: mid, 2: ll).
__host__ __device__ constexpr int split_plane_a(int s, int i, int N) { return s < 2 ? i : N + i; }
__host__ __device__ constexpr int split_plane_b(int s, int i, int N) { return (s & 1) ? N + i : i; }
__host__ __device__ constexpr int split_output(int s) { return s == 0 ? 0 : (s == 3 ? 2 : 1); }

template <int MT, int NT, int WM, int WN, int STG, int KS>
__global__ void __launch_bounds__(WM * WN * 32) crt_gemm_kernel(const CrtGemmArgs g)
{
    constexpr int NTHR = WM * WN * 32;
    constexpr int BM = WM * MT * 16;
    constexpr int BN = WN * NT * 8;
    constexpr int SROW = KS + 16;     // smem row stride in bytes: conflict-free fragment loads
    constexpr int CPR = KS / 16;      // 16-byte chunks per row
    extern __shared__ __align__(16) int8_t csm[];
    int8_t* As = csm;                              // [STG][BM * SROW]
    int8_t* Bs = csm + STG * BM * SROW;            // [STG][BN * SROW]

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int wm = warp / WN, wn = warp % WN;
    const int64_t m0 = static_cast<int64_t>(blockIdx.y) * BM;
    const int64_t n0 = static_cast<int64_t>(blockIdx.x) * BN;
    // plane z of the output: modulus z (or, with split integers, product
    // z / N of modulus z % N, the middle one summing two sub-products)
    const int z = blockIdx.z;
    const int mi = g.split ? z % g.N : z;
    const int o = g.split ? z / g.N : 0;
    const int s0 = o == 0 ? 0 : (o == 1 ? 1 : 3);
    const int nsub = o == 1 ? 2 : 1;
    const int KT1 = static_cast<int>(g.kp / KS);
    const int KT = nsub * KT1;
    auto plane_a = [&](int sub) { return g.split ? split_plane_a(s0 + sub, mi, g.N) : mi; };
    auto plane_b = [&](int sub) { return g.split ? split_plane_b(s0 + sub, mi, g.N) : mi; };

    int ci[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) ci[mt][nt][r] = 0;

    auto load = [&](int stage, int kt) {
        const int sub = kt >= KT1 ? 1 : 0;
        const int kk = kt - sub * KT1;
        const int8_t* a = g.ra + (static_cast<int64_t>(plane_a(sub)) * g.mp + m0) * g.kp;
        const int8_t* b = g.rb + (static_cast<int64_t>(plane_b(sub)) * g.np + n0) * g.kp;
        for (int chunk = tid; chunk < (BM + BN) * CPR; chunk += NTHR) {
            const int row = chunk / CPR, col = (chunk % CPR) * 16;
            if (row < BM)
                cp_async16(As + stage * BM * SROW + row * SROW + col,
                           a + static_cast<int64_t>(row) * g.kp + static_cast<int64_t>(kk) * KS + col);
            else
                cp_async16(Bs + stage * BN * SROW + (row - BM) * SROW + col,
                           b + static_cast<int64_t>(row - BM) * g.kp + static_cast<int64_t>(kk) * KS + col);
        }
    };
#pragma unroll
    for (int st = 0; st < STG - 1; ++st) {
        if (st < KT) load(st, st);
        cp_async_commit();
    }
    for (int it = 0; it < KT; ++it) {
        cp_async_wait<STG - 2>();
        __syncthreads();
        if (it + STG - 1 < KT) load((it + STG - 1) % STG, it + STG - 1);
        cp_async_commit();
        const int8_t* as = As + (it % STG) * BM * SROW;
        const int8_t* bs = Bs + (it % STG) * BN * SROW;
#pragma unroll
        for (int kk = 0; kk < KS; kk += 32) {
            uint32_t af[MT][4], bf[NT][2];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int r = wm * MT * 16 + mt * 16 + gq;
                af[mt][0] = *reinterpret_cast<const uint32_t*>(as + r * SROW + kk + 4 * tq);
                af[mt][1] = *reinterpret_cast<const uint32_t*>(as + (r + 8) * SROW + kk + 4 * tq);
                af[mt][2] = *reinterpret_cast<const uint32_t*>(as + r * SROW + kk + 16 + 4 * tq);
                af[mt][3] = *reinterpret_cast<const uint32_t*>(as + (r + 8) * SROW + kk + 16 + 4 * tq);
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int c = wn * NT * 8 + nt * 8 + gq;
                bf[nt][0] = *reinterpret_cast<const uint32_t*>(bs + c * SROW + kk + 4 * tq);
                bf[nt][1] = *reinterpret_cast<const uint32_t*>(bs + c * SROW + kk + 16 + 4 * tq);
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) mma_s8(ci[mt][nt], af[mt], bf[nt]);
        }
    }
    cp_async_wait<0>();

    const int m = crt::kDev.m[mi];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t row = m0 + wm * MT * 16 + mt * 16 + gq + h * 8;
                const int64_t col = n0 + wn * NT * 8 + nt * 8 + 2 * tq;
                int8_t rr[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int v = ci[mt][nt][2 * h + u];
                    const uint32_t mag = static_cast<uint32_t>(v < 0 ? -v : v);
                    int r = static_cast<int>(crt::mod_small(mag, mi));
                    if (v < 0 && r) r = m - r;
                    rr[u] = static_cast<int8_t>(r >= (m + 1) / 2 ? r - m : r);
                }
                char2 pk;
                pk.x = rr[0];
                pk.y = rr[1];
                *reinterpret_cast<char2*>(g.out + (static_cast<int64_t>(z) * g.mp + row) * g.np + col) = pk;
            }
}

// ------------------------------------------------------- CRT recovery
//
// Per output: the residues of Q_i give the mixed-radix digits of A'B' (Garner:
// v_i = (r_i - (v_0 + v_1 m_0 + ... ) mod m_i) (m_0 ... m_(i-1))^-1 mod m_i,
// all in small integers), Horner's rule turns them into the integer X in
// [0, M) (11 32-bit limbs), X >= ceil(M/2) is taken as X - M, and the P
// components of X 2^(sigma_i + tau_j - 2 beta) are rounded to nearest (ties
// to even) one after another, each from the exact remainder of the previous
// ones, with integer operations only.

namespace crt {
constexpr int kRecLimbs = 11;                     // M < 2^352
}

struct CrtRecArgs {
    const int8_t* res;      // [N][mp][np] residues of the products ([3N]: hh, mid, ll with split integers)
    const int* sig;
    const int* tau;
    double* C[4];
    int64_t ldc, m, n, mp, np;
    int N, beta;
    int w;                  // split integers: C' = P_hh 2^(2w) + P_mid 2^w + P_ll
    uint32_t M[crt::kRecLimbs];          // the product of the moduli
    uint32_t H[crt::kRecLimbs];          // ceil(M / 2)
    // the CRT weights W_i = (M / m_i) c_i, c_i = (M / m_i)^-1 mod m_i, so that
    // X = sum_i r_i W_i - M floor(sum_i r_i c_i / m_i) for residues r_i in [0, m_i)
    uint32_t W[crt::kMaxModuli][crt::kRecLimbs];
    float f[crt::kMaxModuli];             // c_i / m_i
};

// Big unsigned integers of L 32-bit limbs, least significant first, kept in
// registers: every index below is a compile-time constant after unrolling.
template <int L>
__device__ __forceinline__ uint32_t limb_at(const uint32_t (&u)[L], int w)
{
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) r = (k == w) ? u[k] : r;
    return r;
}

template <int L>
__device__ __forceinline__ int bit_length(const uint32_t (&u)[L])
{
    int bl = 0;
#pragma unroll
    for (int k = 0; k < L; ++k)
        if (u[k]) bl = 32 * k + (32 - __clz(static_cast<int>(u[k])));
    return bl;
}

// Bits [pos, pos + 53) of u, pos >= 0.
template <int L>
__device__ __forceinline__ uint64_t bits53(const uint32_t (&u)[L], int pos)
{
    const int w = pos >> 5, off = pos & 31;
    const unsigned __int128 x = static_cast<unsigned __int128>(limb_at<L>(u, w)) |
                                (static_cast<unsigned __int128>(limb_at<L>(u, w + 1)) << 32) |
                                (static_cast<unsigned __int128>(limb_at<L>(u, w + 2)) << 64);
    return static_cast<uint64_t>(x >> off) & ((1ull << 53) - 1);
}

__device__ __forceinline__ uint32_t low_mask(int s, int lo)
{
    return s >= lo + 32 ? 0xffffffffu : (s <= lo ? 0u : ((1u << (s - lo)) - 1u));
}

// Whether any bit of u below position pos is set.
template <int L>
__device__ __forceinline__ bool any_below(const uint32_t (&u)[L], int pos)
{
    bool any = false;
#pragma unroll
    for (int k = 0; k < L; ++k) any = any || (u[k] & low_mask(pos, 32 * k)) != 0u;
    return any;
}

// u = u mod 2^s (s >= 1), then, when `complement`, u = 2^s - u (u != 0).
template <int L>
__device__ __forceinline__ void low_bits(uint32_t (&u)[L], int s, bool complement)
{
#pragma unroll
    for (int k = 0; k < L; ++k) u[k] &= low_mask(s, 32 * k);
    if (!complement) return;
    uint32_t carry = 1;
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const uint64_t t = static_cast<uint64_t>(~u[k]) + carry;
        u[k] = static_cast<uint32_t>(t) & low_mask(s, 32 * k);
        carry = static_cast<uint32_t>(t >> 32);
    }
}

// RN((-1)^neg u 2^e) as binary64 (ties to even; gradual underflow; +-inf
// above the range); u and neg become the exact remainder (magnitude, sign).
template <int L>
__device__ __forceinline__ double rn_component(uint32_t (&u)[L], bool& neg, int e)
{
    const int bl = bit_length<L>(u);
    if (bl == 0) return 0.0;
    const uint64_t sign = neg ? (1ull << 63) : 0ull;
    const int E = bl - 1 + e;
    int qx = E >= -1022 ? E - 52 : -1074;
    const int s = qx - e;
    uint64_t q;
    if (s <= 0) {                                     // exactly representable
        q = bits53<L>(u, 0) << (-s);
#pragma unroll
        for (int k = 0; k < L; ++k) u[k] = 0u;
    } else {
        q = bits53<L>(u, s);
        const bool half = (limb_at<L>(u, (s - 1) >> 5) >> ((s - 1) & 31)) & 1u;
        const bool up = half && ((q & 1ull) || any_below<L>(u, s - 1));
        low_bits<L>(u, s, up);
        if (up) {
            ++q;
            neg = !neg;
        }
        if (q == (1ull << 53)) {
            q = 1ull << 52;
            ++qx;
        }
    }
    if (q == 0) return __longlong_as_double(static_cast<long long>(sign));     // a signed zero
    if (q >= (1ull << 52) && qx + 52 > 1023) {                                  // beyond the range
#pragma unroll
        for (int k = 0; k < L; ++k) u[k] = 0u;
        return __longlong_as_double(static_cast<long long>(sign | 0x7ff0000000000000ull));
    }
    const uint64_t bits = q >= (1ull << 52)
                              ? (static_cast<uint64_t>(qx + 52 + 1023) << 52) | (q - (1ull << 52))
                              : q;                    // subnormal: qx = -1074
    return __longlong_as_double(static_cast<long long>(sign | bits));
}

// The integer X in [0, M) from the column sums S (limbs of 64 bits, S < 2^14 M)
// and the quotient estimate qf (see the recovery kernel below), centred to
// [-M/2, M/2) as magnitude Y and sign; crt_finish rounds it to the P
// components of output (row, col).
template <int L>
__device__ __forceinline__ void crt_centre(const CrtRecArgs& g, const uint64_t (&S)[L + 1], float qf,
                                           uint32_t (&Y)[L], bool& neg)
{
    // carries: S as L + 1 32-bit limbs
    uint32_t X[L + 1];
    uint64_t carry = 0;
#pragma unroll
    for (int k = 0; k <= L; ++k) {
        const uint64_t v = S[k] + carry;
        X[k] = static_cast<uint32_t>(v);
        carry = v >> 32;
    }
    // X -= q M, then one correction by M either way
    const uint32_t q = static_cast<uint32_t>(floorf(qf));
    uint64_t mc = 0;
    int64_t borrow = 0;
#pragma unroll
    for (int k = 0; k <= L; ++k) {
        const uint64_t pm = static_cast<uint64_t>(k < L ? g.M[k] : 0u) * q + mc;
        mc = pm >> 32;
        const int64_t d = static_cast<int64_t>(X[k]) - static_cast<int64_t>(static_cast<uint32_t>(pm)) + borrow;
        X[k] = static_cast<uint32_t>(d);
        borrow = d >> 32;                              // 0 or -1
    }
    if (static_cast<int32_t>(X[L]) < 0) {             // q was one too large: add M back
        uint64_t c = 0;
#pragma unroll
        for (int k = 0; k <= L; ++k) {
            const uint64_t v = static_cast<uint64_t>(X[k]) + (k < L ? g.M[k] : 0u) + c;
            X[k] = static_cast<uint32_t>(v);
            c = v >> 32;
        }
    } else {                                          // q one too small: X >= M
        bool ge = X[L] != 0u, decided = X[L] != 0u;
#pragma unroll
        for (int k = L - 1; k >= 0; --k) {
            if (!decided && X[k] != g.M[k]) {
                ge = X[k] > g.M[k];
                decided = true;
            }
        }
        if (!decided) ge = true;
        if (ge) {
            int64_t b2 = 0;
#pragma unroll
            for (int k = 0; k <= L; ++k) {
                const int64_t d = static_cast<int64_t>(X[k]) - static_cast<int64_t>(k < L ? g.M[k] : 0u) + b2;
                X[k] = static_cast<uint32_t>(d);
                b2 = d >> 32;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < L; ++k) Y[k] = X[k];
    // Y >= ceil(M/2): the value is Y - M < 0, magnitude M - Y
    bool ge = true, decided = false;
#pragma unroll
    for (int k = L - 1; k >= 0; --k) {
        if (!decided && Y[k] != g.H[k]) {
            ge = Y[k] > g.H[k];
            decided = true;
        }
    }
    neg = false;
    if (ge) {
        uint64_t bw = 0;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const uint64_t d = static_cast<uint64_t>(g.M[k]) - Y[k] - bw;
            Y[k] = static_cast<uint32_t>(d);
            bw = (d >> 63) & 1ull;
        }
        neg = true;
    }
}

template <int P, int L>
__device__ __forceinline__ void crt_finish(const CrtRecArgs& g, const uint64_t (&S)[L + 1], float qf, int64_t row,
                                           int64_t col)
{
    uint32_t Y[L];
    bool neg;
    crt_centre<L>(g, S, qf, Y, neg);
    const int e = g.sig[row] + g.tau[col] - 2 * g.beta;
#pragma unroll
    for (int c = 0; c < P; ++c) g.C[c][row * g.ldc + col] = rn_component<L>(Y, neg, e);
}

// NB: the moduli count rounded up to a multiple of 8 (the loops below are
// unrolled NB times and skip moduli i >= N); L = NB / 4 limbs (at most 11)
// hold the product of NB moduli <= 256.  The integer in [0, M) congruent to
// the residues is sum_i r_i W_i - q M with q = floor(sum_i r_i c_i / m_i):
// the sum is accumulated exactly in 64-bit columns (each term below 2^40), q
// is estimated in binary32 (off by at most one: the sum is below 2^14 and its
// rounding error far below one) and corrected by one addition or subtraction
// of M.  Each thread takes four consecutive outputs of a row (one 4-byte load
// per modulus; the residue rows are padded to a multiple of 128).
template <int P, int NB>
__global__ void __launch_bounds__(256) crt_recover_kernel(const __grid_constant__ CrtRecArgs g)
{
    constexpr int L = NB / 4 < crt::kRecLimbs ? NB / 4 : crt::kRecLimbs;
    const int64_t quads = (g.n + 3) / 4;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= g.m * quads) return;
    const int64_t row = t / quads, col0 = (t % quads) * 4;
    const int N = g.N;
    uint64_t S[4][L + 1];
    float qf[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        qf[u] = 0.0f;
#pragma unroll
        for (int k = 0; k <= L; ++k) S[u][k] = 0ull;
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        if (i < N) {
            const int mi = crt::kDev.m[i];
            const char4 r4 = *reinterpret_cast<const char4*>(g.res + (static_cast<int64_t>(i) * g.mp + row) * g.np + col0);
            const int rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = rr[u] < 0 ? rr[u] + mi : rr[u];
                const uint32_t ru = static_cast<uint32_t>(r);
#pragma unroll
                for (int k = 0; k < L; ++k) S[u][k] += static_cast<uint64_t>(g.W[i][k]) * ru;
                qf[u] = __fmaf_rn(static_cast<float>(r), g.f[i], qf[u]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (col0 + u < g.n) crt_finish<P, L>(g, S[u], qf[u], row, col0 + u);
}

// Z += (-1)^neg Y 2^shift in two's complement (LC limbs; the sum stays in range).
template <int L, int LC>
__device__ __forceinline__ void add_shifted(uint32_t (&Z)[LC], const uint32_t (&Y)[L], bool neg, int shift)
{
    const int sw = shift >> 5, sb = shift & 31;
    uint64_t carry = neg ? 1ull : 0ull;                 // -T = ~T + 1
#pragma unroll
    for (int k = 0; k < LC; ++k) {
        const uint32_t hi = limb_at<L>(Y, k - sw);
        const uint32_t lo = sb ? limb_at<L>(Y, k - sw - 1) >> (32 - sb) : 0u;
        uint32_t t = (hi << sb) | lo;
        if (neg) t = ~t;
        const uint64_t v = static_cast<uint64_t>(Z[k]) + t + carry;
        Z[k] = static_cast<uint32_t>(v);
        carry = v >> 32;
    }
}

// Split integers: the three products hh, mid, ll of each output recovered as
// above (each in [-M/2, M/2)), combined exactly as C' = P_hh 2^(2w) +
// P_mid 2^w + P_ll in LC = 2L + 1 32-bit limbs (|C'| < M 2^(2w) <= 2^(64L)),
// and rounded to P components.  Two outputs per thread.
template <int P, int NB>
__global__ void __launch_bounds__(256) crt_recover2_kernel(const __grid_constant__ CrtRecArgs g)
{
    constexpr int L = NB / 4 < crt::kRecLimbs ? NB / 4 : crt::kRecLimbs;
    constexpr int LC = 2 * L + 1;
    const int64_t pairs = (g.n + 1) / 2;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= g.m * pairs) return;
    const int64_t row = t / pairs, col0 = (t % pairs) * 2;
    const int N = g.N;
    uint32_t Z[2][LC];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int k = 0; k < LC; ++k) Z[u][k] = 0u;
#pragma unroll 1
    for (int part = 0; part < 3; ++part) {
        uint64_t S[2][L + 1];
        float qf[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            qf[u] = 0.0f;
#pragma unroll
            for (int k = 0; k <= L; ++k) S[u][k] = 0ull;
        }
        const int8_t* res = g.res + static_cast<int64_t>(part) * N * g.mp * g.np;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            if (i < N) {
                const int mi = crt::kDev.m[i];
                const char2 r2 = *reinterpret_cast<const char2*>(res + (static_cast<int64_t>(i) * g.mp + row) * g.np + col0);
                const int rr[2] = {r2.x, r2.y};
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int r = rr[u] < 0 ? rr[u] + mi : rr[u];
                    const uint32_t ru = static_cast<uint32_t>(r);
#pragma unroll
                    for (int k = 0; k < L; ++k) S[u][k] += static_cast<uint64_t>(g.W[i][k]) * ru;
                    qf[u] = __fmaf_rn(static_cast<float>(r), g.f[i], qf[u]);
                }
            }
        }
        const int shift = (2 - part) * g.w;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            uint32_t Y[L];
            bool neg;
            crt_centre<L>(g, S[u], qf[u], Y, neg);
            add_shifted<L, LC>(Z[u], Y, neg, shift);
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t col = col0 + u;
        if (col >= g.n) continue;
        bool neg = (Z[u][LC - 1] >> 31) != 0;
        if (neg) {                                      // magnitude
            uint64_t c = 1;
#pragma unroll
            for (int k = 0; k < LC; ++k) {
                const uint64_t v = static_cast<uint64_t>(~Z[u][k]) + c;
                Z[u][k] = static_cast<uint32_t>(v);
                c = v >> 32;
            }
        }
        const int e = g.sig[row] + g.tau[col] - 2 * g.beta;
#pragma unroll
        for (int c = 0; c < P; ++c) g.C[c][row * g.ldc + col] = rn_component<LC>(Z[u], neg, e);
    }
}


// ------------------------------------------------------- tcgen05 engine
//
// The bf16 digits on the 5th-generation tensor cores, TD and QD (DD runs on
// CTA pairs, below).  A persistent CTA per SM owns 128 x 64 tiles of C.  Warp 0
// streams 128 x 128 (A) and 64 x 128 (B) bf16 slice tiles of op(A) and
// op(B)^T, two 64-wide boxes each, into shared memory with TMA (128-byte
// swizzle, 4-stage mbarrier ring: eight MMAs per barrier wait).
// Warp 1 owns 512 TMEM columns and issues tcgen05.mma.cta_group::1.kind::f16
// (M = 128, N = 64, K = 16, fp32 accumulation), filling one of two TMEM
// accumulators per segment: the k tiles of one weight, at most 2048 values of
// k, so every fp32 partial sum of integer products of at most 2^12 stays an
// exact integer below 2^23.  Warps 2-5 (one TMEM lane quadrant each, one row
// of the tile per thread) drain each segment: fp32 -> int, shifted into that
// thread's exact 128-bit group sums held in TMEM after the accumulators (4
// columns per output); at the end of a group
// they split the group value exactly into two binary64 and add it to C with
// the precision's add.  The integer weight sums equal those of the int8 path,
// so the result is bit-identical to it.  Every wait is bounded (about 1 s): on
// a timeout the kernel records an error code in the workspace header, drains
// what it issued, frees TMEM and returns.

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

// Iteration over the stages of one TD/QD tile on the tcgen05 engine.  The
// weights S+1, S, ..., 2 are cut into the accumulation groups of G weights
// (from the least significant end), and each group into blocks of two
// consecutive weights (w, w - 1), a lone last weight forming a block of its
// own, so no block spans two groups.  A block's stages run over the pair
// index s = 1 .. w - 1 and, for each s, the k tiles: the stage multiplies the
// A slice s by the B slices w - s and (while s <= w - 2) w - 1 - s, so one A
// tile feeds both weights' accumulators.  The integer group sums do not depend
// on the order in which their weights' products arrive, so the result is that
// of the weight-by-weight order.
struct BlockCursor {
    int wh;     // the block's larger weight
    int two;    // 1 when the block also holds wh - 1
    int s, kt;
    __device__ __forceinline__ void begin(int S, int G, int w)
    {
        wh = w;
        const int j = (S + 1 - w) % G;
        two = (j + 1 < G && w - 1 >= 2) ? 1 : 0;
        s = 1;
        kt = 0;
    }
    // whether the current stage carries the pair of weight wh - 1
    __device__ __forceinline__ bool lo() const { return two && s <= wh - 2; }
    // the next stage; returns true when that starts a new block
    __device__ __forceinline__ bool advance(int S, int G, int KT)
    {
        if (++kt < KT) return false;
        kt = 0;
        if (++s <= wh - 1) return false;
        begin(S, G, wh - 1 - two);
        return true;
    }
    // index of weight w within its group, and whether it closes the group
    static __device__ __forceinline__ int index(int S, int G, int w) { return (S + 1 - w) % G; }
    static __device__ __forceinline__ bool closes(int S, int G, int w) { return index(S, G, w) == G - 1 || w == 2; }
};

// Stages of one tile: sum over the blocks of (wh - 1) KT.
__device__ __forceinline__ int tile_stages(int S, int G, int KT)
{
    int n = 0;
    for (int w = S + 1; w >= 2;) {
        const int j = (S + 1 - w) % G;
        const int two = (j + 1 < G && w - 1 >= 2) ? 1 : 0;
        n += (w - 1) * KT;
        w -= 1 + two;
    }
    return n;
}

template <int P>
__global__ void __launch_bounds__(192, 1)
ozaki_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const TcArgs g)
{
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[tc::STAGES], empty[tc::STAGES], accf[2], acce[2], fin;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    using Cf = tc::Cfg<P>;
    using G = typename GroupSum<P>::T;
    constexpr int BN = Cf::BN, GW = Cf::GW, OPW = 32 / GW;   // outputs per 32 group columns
    constexpr int kGroup = ozaki_group(P);
    __shared__ int s_tau[BN];

    const uint32_t raw = smem_u32(dsm);
    uint8_t* stage0 = dsm + (((raw + 1023u) & ~1023u) - raw);   // 1024-aligned for the swizzle
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abortp = &abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < tc::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 128);
        }
        mbar_init(&fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(tc::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    const int S = g.S;
    const int KT = static_cast<int>(g.kp / (tc::KE * tc::KB));
    const int per_tile = tile_stages(S, kGroup, KT);
    const int ntiles = g.tiles_m * g.tiles_n;
    auto fail = [&](int code) {
        *abortp = 1;
        atomicCAS(g.err, 0, code);
    };

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            if (g.test_abort) {
                // as if the first wait had run out: nothing has been loaded,
                // so no role has anything in flight when it sees the abort
                fail(1);
                ok = false;
            }
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int m0 = (tile % g.tiles_m) * tc::BM, n0 = (tile / g.tiles_m) * BN;
                BlockCursor c;
                c.begin(S, kGroup, S + 1);
                for (int i = 0; i < per_tile; ++i, ++it) {
                    const uint32_t st = it % tc::STAGES, ph = (it / tc::STAGES) & 1u;
                    if (!mbar_wait<kHintIdle>(&empty[st], ph ^ 1u, abortp)) { fail(1); ok = false; break; }
                    uint8_t* sa = stage0 + st * Cf::STAGE_BYTES;
                    const bool lo = c.lo();
                    mbar_expect_tx(&full[st], Cf::A_STAGE + (lo ? 2 : 1) * Cf::B_STAGE);
#pragma unroll
                    for (int q = 0; q < tc::KB; ++q) {
                        const int x = (c.kt * tc::KB + q) * tc::KE;
                        tma_load_3d(sa + q * tc::A_BYTES, &tmA, x, m0, c.s - 1, &full[st]);
                        tma_load_3d(sa + Cf::A_STAGE + q * Cf::B_BYTES, &tmB, x, n0, c.wh - c.s - 1, &full[st]);
                        if (lo)
                            tma_load_3d(sa + Cf::A_STAGE + Cf::B_STAGE + q * Cf::B_BYTES, &tmB, x, n0,
                                        c.wh - 1 - c.s - 1, &full[st]);
                    }
                    c.advance(S, kGroup, KT);
                }
            }
            // the last loads issued must have landed before the CTA exits
            for (uint32_t j = 0; j < tc::STAGES && j < it; ++j) {
                const uint32_t k = it - 1 - j;
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&full[k % tc::STAGES], (k / tc::STAGES) & 1u) && gtimer() - t0 < tc::TIMEOUT_NS) {
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            uint32_t it = 0, seg = 0;
            int pend = -1;          // accumulator set whose commit waits for the next stage
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                BlockCursor c;
                c.begin(S, kGroup, S + 1);
                int seg_stages = 0;
                bool lo_started = false;
                uint32_t b = 0;
                for (int i = 0; i < per_tile; ++i, ++it) {
                    if (seg_stages == 0) {
                        b = seg & 1u;
                        lo_started = false;
                        if (!mbar_wait<kHintIssue>(&acce[b], ((seg >> 1) & 1u) ^ 1u, abortp)) { fail(2); ok = false; break; }
                    }
                    const uint32_t st = it % tc::STAGES, ph = (it / tc::STAGES) & 1u;
                    if (!mbar_wait<kHintIssue>(&full[st], ph, abortp)) { fail(3); ok = false; break; }
                    tc_fence_after();
                    if (pend >= 0) {
                        umma_commit(&accf[pend]);
                        pend = -1;
                    }
                    const bool lo = c.lo();
                    const uint32_t sa = smem_u32(stage0 + st * Cf::STAGE_BYTES);
                    const uint32_t d_hi = tmem + b * Cf::SET_COLS, d_lo = d_hi + BN;
#pragma unroll
                    for (int q = 0; q < tc::KB; ++q) {
                        const uint64_t da = umma_desc(sa + q * tc::A_BYTES);
                        const uint64_t dh = umma_desc(sa + Cf::A_STAGE + q * Cf::B_BYTES);
                        const uint64_t dl = umma_desc(sa + Cf::A_STAGE + Cf::B_STAGE + q * Cf::B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < tc::KE / 16; ++kk) {
                            const uint32_t more = (q > 0 || kk > 0) ? 1u : 0u;
                            umma(d_hi, da + 2ull * kk, dh + 2ull * kk, Cf::IDESC, (seg_stages > 0 || more) ? 1u : 0u);
                            if (lo) umma(d_lo, da + 2ull * kk, dl + 2ull * kk, Cf::IDESC, (lo_started || more) ? 1u : 0u);
                        }
                    }
                    umma_commit(&empty[st]);
                    lo_started = lo_started || lo;
                    ++seg_stages;
                    const bool block_end = c.advance(S, kGroup, KT);
                    if (block_end || seg_stages == tc::SEG_STAGES) {
                        pend = static_cast<int>(b);
                        ++seg;
                        seg_stages = 0;
                    }
                }
            }
            if (pend >= 0) umma_commit(&accf[pend]);
            // every MMA issued has completed before TMEM is released
            umma_commit(&fin);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(&fin, 0u) && gtimer() - t0 < tc::TIMEOUT_NS) {
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const mp::Rn f = mp::make_rn();
        const int q = warp & 3;                          // TMEM lane quadrant of this warp
        const int r = 32 * q + lane;                     // row of the tile
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        const uint32_t grp = tmem + lane_off + Cf::GRP_COL;
        uint32_t zero32[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) zero32[t] = 0u;
        uint32_t seg = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int m0 = (tile % g.tiles_m) * tc::BM, n0 = (tile / g.tiles_m) * BN;
            const int64_t row = m0 + r;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (r < BN) s_tau[r] = g.tau[n0 + r];
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const int sg = g.sig[row];
#pragma unroll
            for (int c0 = 0; c0 < GW * BN; c0 += 32) tmem_st32(grp + c0, zero32);
            tmem_wait_st();
            BlockCursor c;
            c.begin(S, kGroup, S + 1);
            int seg_stages = 0;
            bool lo_used = false;
            bool first_group = true;
            for (int i = 0; i < per_tile; ++i) {
                ++seg_stages;
                lo_used = lo_used || c.lo();
                const int wh = c.wh, two = c.two;
                const bool block_end = c.advance(S, kGroup, KT);
                if (!block_end && seg_stages != tc::SEG_STAGES) continue;
                seg_stages = 0;
                const bool use_lo = lo_used;
                lo_used = false;
                const uint32_t b = seg & 1u;
                // the decision must be warp-uniform: the TMEM loads below are .sync.aligned
                if (!__all_sync(0xffffffffu, mbar_wait<kHintIdle>(&accf[b], (seg >> 1) & 1u, abortp))) {
                    fail(4);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int jh = BlockCursor::index(S, kGroup, wh);     // the lower weight is jh + 1
                const uint32_t acc = tmem + lane_off + b * Cf::SET_COLS;
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    uint32_t fh[32], fl[32];
                    tmem_ld32(acc + c0, fh);
                    if (use_lo) tmem_ld32(acc + BN + c0, fl);
                    tmem_wait_ld();
#pragma unroll
                    for (int h = 0; h < GW; ++h) {
                        uint32_t gw[32];
                        tmem_ld32(grp + GW * c0 + 32 * h, gw);
                        tmem_wait_ld();
#pragma unroll
                        for (int t = 0; t < OPW; ++t) {
                            G add = static_cast<G>(__float2int_rn(__uint_as_float(fh[OPW * h + t]))) << (7 * jh);
                            if (use_lo)
                                add += static_cast<G>(__float2int_rn(__uint_as_float(fl[OPW * h + t]))) << (7 * (jh + 1));
                            group_store<G, GW>(gw + GW * t, group_load<G, GW>(gw + GW * t) + add);
                        }
                        tmem_st32(grp + GW * c0 + 32 * h, gw);
                    }
                    tmem_wait_st();
                }
                tc_fence_before();
                mbar_arrive(&acce[b]);
                ++seg;
                const int wl = wh - two;
                if (!(block_end && BlockCursor::closes(S, kGroup, wl))) continue;
                // end of a group: add its exact value to C
                const int wmax = wl + BlockCursor::index(S, kGroup, wl);
                for (int c0 = 0; c0 < GW * BN; c0 += 32) {
                    uint32_t gw[32];
                    tmem_ld32(grp + c0, gw);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < OPW; ++t) {
                        const int64_t col = n0 + c0 / GW + t;
                        if (row >= g.m || col >= g.n) continue;
                        double y[P], accv[P], zz[P];
                        const bool exact = split_exact(group_load<G, GW>(gw + GW * t),
                                                       sg + s_tau[c0 / GW + t] - 7 * wmax, y[0], y[1]);
#pragma unroll
                        for (int cc = 2; cc < P; ++cc) y[cc] = f.zero;
                        if (first_group && exact) {
                            // TDaddq / QDadd of zero and an exact split (no
                            // negative zero) is the split itself
#pragma unroll
                            for (int cc = 0; cc < P; ++cc) g.C[cc][row * g.ldc + col] = y[cc];
                            continue;
                        }
                        // a first group whose split left the normal range is
                        // added to zero as written
#pragma unroll
                        for (int cc = 0; cc < P; ++cc) accv[cc] = first_group ? f.zero : g.C[cc][row * g.ldc + col];
                        mp::Ops<P>::add(f, accv, y, zz);
#pragma unroll
                        for (int cc = 0; cc < P; ++cc) g.C[cc][row * g.ldc + col] = zz[cc];
                    }
                    tmem_st32(grp + c0, zero32);
                }
                tmem_wait_st();
                first_group = false;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::TMEM_COLS));
    }
}

// ----------------------------------------------- CRT form on tcgen05
//
// The residue products on the 5th-generation tensor cores: residues as bf16
// (exact: |r| <= 128), TMA-loaded 128 x 128 tiles of op(A) and op(B)^T,
// tcgen05.mma kind::f16 with M = N = 128 and fp32 accumulation in tensor
// memory.  A product of two residues is at most 2^14, so an accumulator is
// drained after at most 1024 values of k (8 stages) while every partial sum
// is an integer below 2^24, exact in fp32; the drains add it to an exact
// int32 sum per output kept in tensor memory, and at the end of a modulus the
// sum's symmetric residue is stored as int8.  With split integers each
// modulus runs four sub-products (A1 B1, A1 B0, A0 B1, A0 B0); the two middle
// ones add into one sum.  Warp roles, barriers, bounded waits and the abort
// protocol are those of the slicing engine.

namespace tcc {
constexpr int BM = 128;
constexpr int BN = 128;
constexpr int KE = 64;
constexpr int KB = 2;                                     // 128 values of k per stage
constexpr int STAGES = 3;
constexpr int BOX = BM * KE * 2;                          // one 128 x 64 bf16 box, 16 KB
constexpr int STAGE_BYTES = 2 * KB * BOX;                 // A and B, 64 KB
constexpr int SEG_STAGES = 1024 / (KE * KB);              // fp32 exact: 1024 k per drain
constexpr int SUM_COL = 2 * BN;                           // int32 sums after two accumulators
constexpr int TMEM_COLS = 512;
static_assert(SUM_COL + BN <= TMEM_COLS, "TMEM columns");
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((static_cast<uint32_t>(BN) >> 3) << 17) |
                           ((128u >> 4) << 24);
}  // namespace tcc

struct CrtTcArgs {
    int8_t* out;            // [N][mp][np] residues of the products ([3N] with split integers)
    int64_t mp, np, kp;
    int N, tiles_m, tiles_n;
    int* err;
    int test_abort;
    int split;              // 1: split integers, four sub-products per modulus
};

__global__ void __launch_bounds__(192, 1)
crt_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const CrtTcArgs g)
{
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[tcc::STAGES], empty[tcc::STAGES], accf[2], acce[2], fin;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const uint32_t raw = smem_u32(dsm);
    uint8_t* stage0 = dsm + (((raw + 1023u) & ~1023u) - raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int* abortp = &abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < tcc::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 128);
        }
        mbar_init(&fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(tcc::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int KT = static_cast<int>(g.kp / (tcc::KE * tcc::KB));
    const int NSUB = g.split ? 4 : 1;                    // sub-products per modulus
    const int per_tile = g.N * NSUB * KT;
    const int ntiles = g.tiles_m * g.tiles_n;
    auto fail = [&](int code) {
        *abortp = 1;
        atomicCAS(g.err, 0, code);
    };
    // a segment ends after SEG_STAGES stages or at the end of a modulus
    auto seg_end = [&](int kt, int seg_stages) { return kt == KT - 1 || seg_stages == tcc::SEG_STAGES; };

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            if (g.test_abort) {
                fail(1);
                ok = false;
            }
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                const int m0 = (tile % g.tiles_m) * tcc::BM, n0 = (tile / g.tiles_m) * tcc::BN;
                for (int i = 0; i < per_tile; ++i, ++it) {
                    const int mi = i / (NSUB * KT), sub = (i / KT) % NSUB, kt = i % KT;
                    const int pa = g.split ? split_plane_a(sub, mi, g.N) : mi;
                    const int pb = g.split ? split_plane_b(sub, mi, g.N) : mi;
                    const uint32_t st = it % tcc::STAGES, ph = (it / tcc::STAGES) & 1u;
                    if (!mbar_wait<kHintIdle>(&empty[st], ph ^ 1u, abortp)) { fail(1); ok = false; break; }
                    uint8_t* sa = stage0 + st * tcc::STAGE_BYTES;
                    mbar_expect_tx(&full[st], tcc::STAGE_BYTES);
#pragma unroll
                    for (int q = 0; q < tcc::KB; ++q) {
                        const int x = (kt * tcc::KB + q) * tcc::KE;
                        tma_load_3d(sa + q * tcc::BOX, &tmA, x, m0, pa, &full[st]);
                        tma_load_3d(sa + (tcc::KB + q) * tcc::BOX, &tmB, x, n0, pb, &full[st]);
                    }
                }
            }
            for (uint32_t j = 0; j < tcc::STAGES && j < it; ++j) {
                const uint32_t k = it - 1 - j;
                const unsigned long long t0 = gtimer();
                while (!mbar_try(&full[k % tcc::STAGES], (k / tcc::STAGES) & 1u) && gtimer() - t0 < tc::TIMEOUT_NS) {
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, seg = 0;
            int pend = -1;
            bool ok = true;
            for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                int seg_stages = 0;
                uint32_t b = 0;
                for (int i = 0; i < per_tile; ++i, ++it) {
                    const int kt = i % KT;
                    if (seg_stages == 0) {
                        b = seg & 1u;
                        if (!mbar_wait<kHintIssue>(&acce[b], ((seg >> 1) & 1u) ^ 1u, abortp)) { fail(2); ok = false; break; }
                    }
                    const uint32_t st = it % tcc::STAGES, ph = (it / tcc::STAGES) & 1u;
                    if (!mbar_wait<kHintIssue>(&full[st], ph, abortp)) { fail(3); ok = false; break; }
                    tc_fence_after();
                    if (pend >= 0) {
                        umma_commit(&accf[pend]);
                        pend = -1;
                    }
                    const uint32_t sa = smem_u32(stage0 + st * tcc::STAGE_BYTES);
#pragma unroll
                    for (int q = 0; q < tcc::KB; ++q) {
                        const uint64_t da = umma_desc(sa + q * tcc::BOX);
                        const uint64_t db = umma_desc(sa + (tcc::KB + q) * tcc::BOX);
#pragma unroll
                        for (int kk = 0; kk < tcc::KE / 16; ++kk)
                            umma(tmem + b * tcc::BN, da + 2ull * kk, db + 2ull * kk, tcc::IDESC,
                                 (seg_stages > 0 || q > 0 || kk > 0) ? 1u : 0u);
                    }
                    umma_commit(&empty[st]);
                    ++seg_stages;
                    if (seg_end(kt, seg_stages)) {
                        pend = static_cast<int>(b);
                        ++seg;
                        seg_stages = 0;
                    }
                }
            }
            if (pend >= 0) umma_commit(&accf[pend]);
            umma_commit(&fin);
            const unsigned long long t0 = gtimer();
            while (!mbar_try(&fin, 0u) && gtimer() - t0 < tc::TIMEOUT_NS) {
            }
        }
    } else {
        const int q = warp & 3;
        const int r = 32 * q + lane;
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        const uint32_t sums = tmem + lane_off + tcc::SUM_COL;
        uint32_t seg = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int m0 = (tile % g.tiles_m) * tcc::BM, n0 = (tile / g.tiles_m) * tcc::BN;
            int seg_stages = 0;
            bool first = true;                            // first segment of an output product
            for (int i = 0; i < per_tile; ++i) {
                const int mi = i / (NSUB * KT), sub = (i / KT) % NSUB, kt = i % KT;
                ++seg_stages;
                if (!seg_end(kt, seg_stages)) continue;
                seg_stages = 0;
                const uint32_t b = seg & 1u;
                if (!__all_sync(0xffffffffu, mbar_wait<kHintIdle>(&accf[b], (seg >> 1) & 1u, abortp))) {
                    fail(4);
                    ok = false;
                    break;
                }
                tc_fence_after();
                // the middle product of split integers continues over two sub-products
                const bool last = kt == KT - 1 && !(g.split && sub == 1);
                const int plane = g.split ? split_output(sub) * g.N + mi : mi;
                const int m = crt::kDev.m[mi];
                for (int c0 = 0; c0 < tcc::BN; c0 += 32) {
                    uint32_t fv[32], sv[32];
                    tmem_ld32(tmem + lane_off + b * tcc::BN + c0, fv);
                    if (!first) tmem_ld32(sums + c0, sv);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        const int add = __float2int_rn(__uint_as_float(fv[t]));
                        sv[t] = first ? static_cast<uint32_t>(add) : sv[t] + static_cast<uint32_t>(add);
                    }
                    if (!last) {
                        tmem_st32(sums + c0, sv);
                    } else {
                        // symmetric residue of each exact sum, 32 consecutive bytes of this row
                        uint32_t pk[8];
#pragma unroll
                        for (int w = 0; w < 8; ++w) pk[w] = 0u;
#pragma unroll
                        for (int t = 0; t < 32; ++t) {
                            const int v = static_cast<int>(sv[t]);
                            const uint32_t mag = static_cast<uint32_t>(v < 0 ? -v : v);
                            int rr = static_cast<int>(crt::mod_small(mag, mi));
                            if (v < 0 && rr) rr = m - rr;
                            rr = rr >= (m + 1) / 2 ? rr - m : rr;
                            pk[t >> 2] |= (static_cast<uint32_t>(rr) & 0xffu) << (8 * (t & 3));
                        }
                        uint4* dst = reinterpret_cast<uint4*>(g.out + (static_cast<int64_t>(plane) * g.mp + m0 + r) * g.np +
                                                              n0 + c0);
                        dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    }
                }
                tmem_wait_st();
                tc_fence_before();
                mbar_arrive(&acce[b]);
                ++seg;
                first = last;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcc::TMEM_COLS));
    }
}

// ------------------------------------------------- tcgen05 engine, CTA pairs
//
// DD on pairs of SMs (a cluster of two CTAs, tcgen05 .cta_group::2).  The pair
// owns a 256 x 128 tile of C; each CTA holds 128 rows of it in its own TMEM
// (two 128-column fp32 accumulators and the 64-bit group sums, exactly as in
// the single-CTA engine, so the epilogue and the result are the same).  Each
// CTA's TMA loads its 128 rows of the op(A) slice tile and its half (64 rows)
// of the op(B)^T slice tile, 128 values of k per stage (two 64-wide boxes
// each), and signals the leader CTA's barrier; the leader's MMA thread issues
// tcgen05.mma.cta_group::2 with M = 256, N = 128, which reads A from both CTAs
// and B halves from both, and releases a stage in both CTAs with one
// multicast commit.  A finished accumulator is committed after the next
// stage's barrier wait, not right behind the stage's own commit: two commits
// in a row stall the issuing thread.  The FP64 work of a finished group is
// done by four adder warps (warps 6-9): a drain warp copies its rows' 64-bit
// group sums to a per-CTA buffer in global memory and goes on draining, and
// the adder of its lane quadrant splits them and adds them to C in order.  Compared with a 128 x 128 tile per SM this loads a
// quarter fewer bytes per product and waits once per eight MMAs instead of
// four.  Epilogue warps of both CTAs signal the leader when an accumulator
// has been drained.  Every wait is bounded; a role that gives up sets the
// abort flag of both CTAs.

namespace tc2 {
constexpr int BM = 128;                                  // rows per CTA (the pair covers 256)
constexpr int BN = 128;                                  // columns of the pair's tile
constexpr int KE = 64;                                   // box width in bf16 (128 bytes)
constexpr int KB = 2;                                    // boxes per stage: 128 values of k
constexpr int STAGES = 4;
constexpr int A_BOX = BM * KE * 2;                       // 16 KB
constexpr int B_BOX = (BN / 2) * KE * 2;                 // 8 KB
constexpr int STAGE_BYTES = KB * (A_BOX + B_BOX);        // 48 KB per CTA
constexpr int SEG_STAGES = 2048 / (KE * KB);             // stages per fp32 segment
constexpr int GW = 2;                                    // 64-bit group sums
constexpr int ACC_COLS = BN;
constexpr int GRP_COL = 2 * BN;
constexpr int TMEM_COLS = 512;
constexpr int EPI_ARRIVALS = 8;                          // 4 drain warps in each CTA
constexpr int THREADS = 320;                             // producer, MMA, 4 drain, 4 adder warps
constexpr int SCRATCH_BYTES = 2 * BN * BM * 8;           // per CTA: two buffers of 64-bit group sums
static_assert(GRP_COL + GW * BN <= TMEM_COLS, "TMEM columns");
static_assert(2048 % (KE * KB) == 0 && KPAD % (KE * KB) == 0, "stage k");
// kind::f16, bf16 A and B (K-major), fp32 D, M = 256, N = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((static_cast<uint32_t>(BN) >> 3) << 17) |
                           ((256u >> 4) << 24);
}  // namespace tc2

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
__device__ __forceinline__ void umma_pair(uint32_t d, uint64_t da, uint64_t db, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(da), "l"(db), "r"(tc2::IDESC), "r"(acc));
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

// Bounded wait until the shared counter reaches `target` (false after about a
// second or once another role aborted).
__device__ __forceinline__ bool wait_count(const volatile int* f, int target, volatile int* abort_flag)
{
    if (*f >= target) return true;
    const unsigned long long t0 = gtimer();
    while (*f < target) {
        if (*abort_flag) return false;
        if (gtimer() - t0 > tc::TIMEOUT_NS) return false;
        __nanosleep(128);
    }
    return true;
}

template <int P>
__global__ void __launch_bounds__(tc2::THREADS, 1)
ozaki_tc_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const TcArgs g)
{
    static_assert(P == 2, "the CTA-pair engine keeps 64-bit group sums (DD)");
    using G = typename GroupSum<P>::T;
    constexpr int BN = tc2::BN, GW = tc2::GW, OPW = 32 / GW;
    constexpr int kGroup = ozaki_group(P);
    extern __shared__ uint8_t dsm[];
    __shared__ __align__(8) uint64_t full[tc2::STAGES], empty[tc2::STAGES], accf[2], acce[2], fin;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int s_tau[BN];
    // drain -> adder hand-over, per TMEM lane quadrant: buffers filled and
    // released so far, a finish flag, and each buffer's tile and weight
    __shared__ int ready_gen[4], done_gen[4], fin_flag[4];
    __shared__ int meta[4][2][3];

    const uint32_t raw = smem_u32(dsm);
    uint8_t* stage0 = dsm + (((raw + 1023u) & ~1023u) - raw);   // 1024-aligned for the swizzle
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    volatile int* abortp = &abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < tc2::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], tc2::EPI_ARRIVALS);
        }
        mbar_init(&fin, 1);
        abort_flag = 0;
        for (int i = 0; i < 4; ++i) ready_gen[i] = done_gen[i] = fin_flag[i] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        // both CTAs of the pair allocate together
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(tc2::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    __syncwarp();
    cluster_sync_all();        // barriers of both CTAs initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    const int S = g.S;
    const int KT = static_cast<int>(g.kp / (tc2::KE * tc2::KB));
    const int per_tile = (S * (S + 1) / 2) * KT;
    const int ntiles = g.tiles_m * g.tiles_n;
    const int cid = static_cast<int>(cluster_index()), ncl = static_cast<int>(cluster_count());
    const uint32_t peer_abort = cluster_addr(&abort_flag, rank ^ 1u);
    auto fail = [&](int code) {
        *abortp = 1;
        st_cluster(peer_abort, 1);
        atomicCAS(g.err, 0, code);
    };

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            if (g.test_abort) {
                // as if the first wait had run out, in both CTAs of the pair:
                // nothing has been loaded, so nothing is in flight
                fail(1);
                ok = false;
            }
            for (int tile = cid; tile < ntiles && ok; tile += ncl) {
                const int ma = (tile % g.tiles_m) * 2 * tc2::BM + static_cast<int>(rank) * tc2::BM;
                const int nb = (tile / g.tiles_m) * BN + static_cast<int>(rank) * (BN / 2);
                GroupCursor c;
                c.begin(S, kGroup, S + 1);
                for (int i = 0; i < per_tile; ++i, ++it) {
                    const uint32_t st = it % tc2::STAGES, ph = (it / tc2::STAGES) & 1u;
                    if (!mbar_wait_cl<kHintIdle>(&empty[st], ph ^ 1u, abortp)) { fail(1); ok = false; break; }
                    uint8_t* sa = stage0 + st * tc2::STAGE_BYTES;
                    const uint32_t bar = cluster_addr(&full[st], 0);
                    if (rank == 0) mbar_expect_tx(&full[st], 2 * tc2::STAGE_BYTES);
#pragma unroll
                    for (int q = 0; q < tc2::KB; ++q) {
                        const int x = (c.kt * tc2::KB + q) * tc2::KE;
                        tma_load_3d_pair(sa + q * tc2::A_BOX, &tmA, x, ma, c.s - 1, bar);
                        tma_load_3d_pair(sa + tc2::KB * tc2::A_BOX + q * tc2::B_BOX, &tmB, x, nb, c.w - c.s - 1, bar);
                    }
                    bool pe, ge;
                    c.advance(S, kGroup, KT, pe, ge);
                }
            }
            // every stage's last release has arrived (the leader's MMAs have
            // read this CTA's loads) before the CTA may exit
            for (uint32_t j = 0; j < tc2::STAGES && j < it; ++j) {
                const uint32_t k = it - 1 - j;
                const unsigned long long t0 = gtimer();
                while (!mbar_try_cl(&empty[k % tc2::STAGES], (k / tc2::STAGES) & 1u) &&
                       gtimer() - t0 < tc::TIMEOUT_NS) {
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA (leader only)
        if (lane == 0 && rank == 0) {
            uint32_t it = 0, seg = 0;
            int pend = -1;          // accumulator whose commit waits for the next stage
            bool ok = true;
            for (int tile = cid; tile < ntiles && ok; tile += ncl) {
                GroupCursor c;
                c.begin(S, kGroup, S + 1);
                int seg_stages = 0;
                uint32_t b = 0;
                for (int i = 0; i < per_tile; ++i, ++it) {
                    if (seg_stages == 0) {
                        b = seg & 1u;
                        if (!mbar_wait_cl<kHintIssue>(&acce[b], ((seg >> 1) & 1u) ^ 1u, abortp)) { fail(2); ok = false; break; }
                    }
                    const uint32_t st = it % tc2::STAGES, ph = (it / tc2::STAGES) & 1u;
                    if (!mbar_wait_cl<kHintIssue>(&full[st], ph, abortp)) { fail(3); ok = false; break; }
                    tc_fence_after();
                    if (pend >= 0) {
                        umma_commit_both(&accf[pend]);
                        pend = -1;
                    }
                    const uint32_t sa = smem_u32(stage0 + st * tc2::STAGE_BYTES);
#pragma unroll
                    for (int q = 0; q < tc2::KB; ++q) {
                        const uint64_t da = umma_desc(sa + q * tc2::A_BOX);
                        const uint64_t db = umma_desc(sa + tc2::KB * tc2::A_BOX + q * tc2::B_BOX);
#pragma unroll
                        for (int kk = 0; kk < tc2::KE / 16; ++kk)
                            umma_pair(tmem + b * tc2::ACC_COLS, da + 2ull * kk, db + 2ull * kk,
                                      (seg_stages > 0 || q > 0 || kk > 0) ? 1u : 0u);
                    }
                    umma_commit_both(&empty[st]);
                    ++seg_stages;
                    bool pair_end, group_end;
                    c.advance(S, kGroup, KT, pair_end, group_end);
                    if (pair_end || seg_stages == tc2::SEG_STAGES) {
                        pend = static_cast<int>(b);
                        ++seg;
                        seg_stages = 0;
                    }
                }
            }
            if (pend >= 0) umma_commit_both(&accf[pend]);
            // every MMA issued has completed before TMEM is released
            umma_commit_pair_local(&fin);
            const unsigned long long t0 = gtimer();
            while (!mbar_try_cl(&fin, 0u) && gtimer() - t0 < tc::TIMEOUT_NS) {
            }
        }
    } else if (warp < 6) {
        // ---------------------------------------------------------- epilogue
        const mp::Rn f = mp::make_rn();
        const int q = warp & 3;                          // TMEM lane quadrant of this warp
        const int r = 32 * q + lane;                     // row of this CTA's half of the tile
        const uint32_t lane_off = static_cast<uint32_t>(32 * q) << 16;
        const uint32_t grp = tmem + lane_off + tc2::GRP_COL;
        const uint32_t lead_acce0 = cluster_addr(&acce[0], 0), lead_acce1 = cluster_addr(&acce[1], 0);
        uint32_t zero32[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) zero32[t] = 0u;
        long long* const scr = g.scratch + static_cast<int64_t>(blockIdx.x) * 2 * BN * tc2::BM;
        int issued = 0;                                  // groups handed to the adder warp
        uint32_t seg = 0;
        bool ok = true;
        for (int tile = cid; tile < ntiles && ok; tile += ncl) {
            const int m0 = (tile % g.tiles_m) * 2 * tc2::BM + static_cast<int>(rank) * tc2::BM;
            const int n0 = (tile / g.tiles_m) * BN;
            const int64_t row = m0 + r;
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (r < BN) s_tau[r] = g.tau[n0 + r];
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const int sg = g.sig[row];
#pragma unroll
            for (int c0 = 0; c0 < GW * BN; c0 += 32) tmem_st32(grp + c0, zero32);
            tmem_wait_st();
            GroupCursor c;
            c.begin(S, kGroup, S + 1);
            int seg_stages = 0;
            bool first_group = true;
            for (int i = 0; i < per_tile; ++i) {
                ++seg_stages;
                const int w = c.w;
                bool pair_end, group_end;
                c.advance(S, kGroup, KT, pair_end, group_end);
                if (!pair_end && seg_stages != tc2::SEG_STAGES) continue;
                seg_stages = 0;
                const uint32_t b = seg & 1u;
                // the decision must be warp-uniform: the TMEM loads below are .sync.aligned
                if (!__all_sync(0xffffffffu, mbar_wait_cl<kHintIdle>(&accf[b], (seg >> 1) & 1u, abortp))) {
                    fail(4);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int j = (S + 1 - w) % kGroup;
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    uint32_t fv[32];
                    tmem_ld32(tmem + lane_off + b * tc2::ACC_COLS + c0, fv);
                    tmem_wait_ld();
#pragma unroll
                    for (int h = 0; h < GW; ++h) {
                        uint32_t gw[32];
                        tmem_ld32(grp + GW * c0 + 32 * h, gw);
                        tmem_wait_ld();
#pragma unroll
                        for (int t = 0; t < OPW; ++t) {
                            const int add = __float2int_rn(__uint_as_float(fv[OPW * h + t]));
                            const G V = group_load<G, GW>(gw + GW * t) + (static_cast<G>(add) << (7 * j));
                            group_store<G, GW>(gw + GW * t, V);
                        }
                        tmem_st32(grp + GW * c0 + 32 * h, gw);
                    }
                    tmem_wait_st();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(b ? lead_acce1 : lead_acce0);
                ++seg;
                if (!group_end) continue;
                // end of a group: the first of a tile goes to C as it is
                // (DDadd((0, 0), y) is y exactly: an exact split with no
                // negative zero); a later one is handed to this quadrant's
                // adder warp, which adds it to C while the drains go on
                const int wmax = w + j;
                const int bi = issued & 1;
                long long* const buf = scr + static_cast<int64_t>(bi) * BN * tc2::BM;
                if (!first_group && issued >= 2 &&
                    !__all_sync(0xffffffffu, wait_count(&done_gen[q], issued - 1, abortp))) {
                    fail(6);
                    ok = false;
                    break;
                }
                for (int c0 = 0; c0 < GW * BN; c0 += 32) {
                    uint32_t gw[32];
                    tmem_ld32(grp + c0, gw);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < OPW; ++t) {
                        const int cc = c0 / GW + t;
                        const G V = group_load<G, GW>(gw + GW * t);
                        if (first_group) {
                            const int64_t col = n0 + cc;
                            if (row < g.m && col < g.n) {
                                double y[2];
                                if (!split_exact(V, sg + s_tau[cc] - 7 * wmax, y[0], y[1])) {
                                    // a part left the normal range: DDadd to zero as written
                                    const double z[2] = {f.zero, f.zero};
                                    double r2[2];
                                    mp::Ops<2>::add(f, z, y, r2);
                                    y[0] = r2[0];
                                    y[1] = r2[1];
                                }
                                g.C[0][row * g.ldc + col] = y[0];
                                g.C[1][row * g.ldc + col] = y[1];
                            }
                        } else {
                            buf[static_cast<int64_t>(cc) * tc2::BM + r] = V;      // coalesced over the warp
                        }
                    }
                    tmem_st32(grp + c0, zero32);
                }
                tmem_wait_st();
                if (!first_group) {
                    if (lane == 0) {
                        meta[q][bi][0] = m0;
                        meta[q][bi][1] = n0;
                        meta[q][bi][2] = wmax;
                    }
                    __threadfence_block();
                    __syncwarp();
                    if (lane == 0) *static_cast<volatile int*>(&ready_gen[q]) = issued + 1;
                    ++issued;
                }
                first_group = false;
            }
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) *static_cast<volatile int*>(&fin_flag[q]) = 1;
    } else {
        // ------------------------------------------------------------ adder
        // Finished groups of this quadrant's 32 rows: split each group sum
        // exactly and add it to C with DDadd, in the order the groups ended.
        const mp::Rn f = mp::make_rn();
        const int q = warp & 3;
        const int r = 32 * q + lane;
        const long long* const scr = g.scratch + static_cast<int64_t>(blockIdx.x) * 2 * BN * tc2::BM;
        const volatile int* const rdy = &ready_gen[q];
        const volatile int* const fin_q = &fin_flag[q];
        int processed = 0;
        for (;;) {
            // next group, or the end of the drains
            const unsigned long long t0 = gtimer();
            bool have = *rdy > processed;
            while (!have) {
                if (*fin_q) {
                    __threadfence_block();           // the drain warp raised fin after its last hand-over
                    have = *rdy > processed;
                    break;
                }
                if (*abortp || gtimer() - t0 > tc::TIMEOUT_NS) break;
                __nanosleep(256);
                have = *rdy > processed;
            }
            if (!__all_sync(0xffffffffu, have)) {
                if (!*fin_q && !*abortp) fail(5);
                break;
            }
            __threadfence_block();
            const int bi = processed & 1;
            const int m0 = meta[q][bi][0], n0 = meta[q][bi][1], wmax = meta[q][bi][2];
            const long long* const buf = scr + static_cast<int64_t>(bi) * BN * tc2::BM;
            const int64_t row = m0 + r;
            if (row < g.m) {
                const int sg = g.sig[row];
#pragma unroll 4
                for (int cc = 0; cc < BN; ++cc) {
                    const int64_t col = n0 + cc;
                    if (col >= g.n) break;
                    double y[P], acc[P], zz[P];
                    split_exact(static_cast<long long>(buf[static_cast<int64_t>(cc) * tc2::BM + r]),
                                sg + g.tau[col] - 7 * wmax, y[0], y[1]);
#pragma unroll
                    for (int h = 0; h < P; ++h) acc[h] = g.C[h][row * g.ldc + col];
                    mp::Ops<P>::add(f, acc, y, zz);
#pragma unroll
                    for (int h = 0; h < P; ++h) g.C[h][row * g.ldc + col] = zz[h];
                }
            }
            __threadfence_block();
            __syncwarp();
            ++processed;
            if (lane == 0) *static_cast<volatile int*>(&done_gen[q]) = processed;
        }
    }

    tc_fence_before();
    __syncthreads();
    __syncwarp();
    cluster_sync_all();        // no remote arrival or TMA into this CTA is outstanding
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc2::TMEM_COLS));
    }
}

// ------------------------------------------------------- fixed scratch

// Scratch for callers that cannot allocate device memory (see
// mpgemm_dd_int8_static in include/mpgemm.h).  Every device that loads the
// library holds this array until the process exits.  Each call rewrites every
// byte of it that it later reads (slices and padding, exponents and padding),
// so nothing has to be cleared between calls.
static __device__ __align__(256) unsigned char g_static_scratch[kOzakiStaticScratchBytes];

namespace {
std::mutex g_static_mu;
void* g_static_ptr[64] = {nullptr};
unsigned long long g_static_ctx[64] = {0};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
}  // namespace

// Unique id of the calling thread's current CUDA context, 0 if there is none
// or the driver cannot say.  A device reset ends the primary context; the
// next one gets a new id, which is how the caches below notice that the
// handles and addresses they hold belong to a context that is gone.
static unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    unsigned long long id = 0;
    return get_id(ctx, &id) == CUDA_SUCCESS ? id : 0;
}

cudaError_t ozaki_static_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_static_ptr[dev] || ctx == 0 || ctx != g_static_ctx[dev]) {
        // In host code the array's name is only a stand-in: the kernels need
        // the device address, looked up with the device current -- once per
        // context (again after a device reset replaced the context, and on
        // every call if the context's id cannot be read).
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
        g_static_ctx[dev] = current_context_id();
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

// ------------------------------------------------------------------ host

static int64_t round_up(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

OzakiLayout ozaki_layout(int S, int64_t m, int64_t n, int64_t k, int elem_bytes)
{
    OzakiLayout L;
    L.S = S;
    L.mp = round_up(m > 0 ? m : 1, TILE);
    L.np = round_up(n > 0 ? n : 1, TILE);
    L.kp = round_up(k > 0 ? k : 1, KPAD);
    L.offA = 0;
    L.offB = round_up(static_cast<int64_t>(S) * L.mp * L.kp * elem_bytes, 256);
    L.offSig = L.offB + round_up(static_cast<int64_t>(S) * L.np * L.kp * elem_bytes, 256);
    L.offTau = L.offSig + round_up(L.mp * 4, 256);
    L.total = L.offTau + round_up(L.np * 4, 256);
    L.offScr = L.total;
    return L;
}

static unsigned blocks_for(int64_t threads, int per) { return static_cast<unsigned>((threads + per - 1) / per); }

// Slice one operand: vectors (rows of op(A) or columns of op(B)) of length
// len; `contig` says whether a vector's elements are adjacent in memory.
template <int P, typename T, int KIND = 0>
static cudaError_t slice_operand(const Planes<P>& pl, int64_t count, int64_t len, int64_t ld,
                                 bool contig, int S, int64_t count_pad, int64_t kp, T* out,
                                 int* sig, cudaStream_t s, int beta = 0)
{
    const double* lead = pl.c[0];
    if (contig) ozaki_scale_contig<<<blocks_for(count * 32, 256), 256, 0, s>>>(lead, count, len, ld, sig);
    else ozaki_scale_strided<<<blocks_for(count, 32), 1024, 0, s>>>(lead, count, len, ld, sig);
    if (count_pad > count)
        ozaki_fill_int<<<blocks_for(count_pad - count, 256), 256, 0, s>>>(sig, count, count_pad);
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

static cudaError_t side_stream(SideStream** out)
{
    thread_local SideStream per_dev[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    SideStream& ss = per_dev[dev];
    const unsigned long long ctx = current_context_id();
    if (ss.s && ctx != 0 && ctx != ss.ctx) {
        // created in a context that a device reset has ended: the handles
        // went with it, so they are dropped, not destroyed
        ss.s = nullptr;
        ss.fork = ss.join = nullptr;
    }
    if (!ss.s) {
        e = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        ss.ctx = current_context_id();
    }
    *out = &ss;
    return cudaSuccess;
}

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

// ----------------------------------------------------- tcgen05 host side

OzakiLayout ozaki_tc_layout(int P, int S, int64_t m, int64_t n, int64_t k)
{
    OzakiLayout L;
    L.S = S;
    // DD runs on CTA pairs (256 x 128 tiles), TD/QD on single CTAs (128 x 64)
    L.mp = round_up(m > 0 ? m : 1, P == 2 ? 2 * tc2::BM : tc::BM);
    L.np = round_up(n > 0 ? n : 1, P == 2 ? tc2::BN : tc::Cfg<4>::BN);
    L.kp = round_up(k > 0 ? k : 1, KPAD);
    L.offA = 256;                                     // bytes 0..255: header (error code)
    L.offB = L.offA + round_up(static_cast<int64_t>(S) * L.mp * L.kp * 2, 256);
    L.offSig = L.offB + round_up(static_cast<int64_t>(S) * L.np * L.kp * 2, 256);
    L.offTau = L.offSig + round_up(L.mp * 4, 256);
    L.offScr = L.offTau + round_up(L.np * 4, 256);
    // DD: the pair kernel's hand-over buffers, one area per CTA (at most one
    // CTA per SM)
    L.total = L.offScr + (P == 2 ? static_cast<int64_t>(num_sms()) * tc2::SCRATCH_BYTES : 0);
    return L;
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

// Clusters of two CTAs of the pair kernel that fit on the device at once.
static cudaError_t pair_clusters(int* out)
{
    static std::mutex mu;
    static int cached[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!cached[dev]) {
        const int smem = tc2::STAGES * tc2::STAGE_BYTES + 1024;
        e = cudaFuncSetAttribute(ozaki_tc_pair_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(tc2::THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, ozaki_tc_pair_kernel<2>, &cfg);
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        cached[dev] = n;
    }
    *out = cached[dev];
    return cudaSuccess;
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

template <int P>
static cudaError_t launch_ozaki_tc(const GemmArgs<P>& g, int S, void* ws, cudaStream_t s)
{
    using Cf = tc::Cfg<P>;
    const OzakiLayout L = ozaki_tc_layout(P, S, g.m, g.n, g.k);
    int8_t* base = static_cast<int8_t*>(ws);
    int* err = reinterpret_cast<int*>(base);
    uint16_t* sa = reinterpret_cast<uint16_t*>(base + L.offA);
    uint16_t* sb = reinterpret_cast<uint16_t*>(base + L.offB);
    int* sig = reinterpret_cast<int*>(base + L.offSig);
    int* tau = reinterpret_cast<int*>(base + L.offTau);
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = slice_both<P>(g, S, L, sa, sb, sig, tau, s);
    if (e != cudaSuccess) return e;
    CUtensorMap ma, mb;
    if constexpr (P == 2) {
        if (!slice_map(&ma, sa, S, L.mp, L.kp, tc2::BM) || !slice_map(&mb, sb, S, L.np, L.kp, tc2::BN / 2))
            return cudaErrorInvalidValue;
        TcArgs a{sig, tau, {g.C[0], g.C[1], nullptr, nullptr}, g.ldc, g.m, g.n, L.kp, S,
                 static_cast<int>(L.mp / (2 * tc2::BM)), static_cast<int>(L.np / tc2::BN), err,
                 reinterpret_cast<long long*>(base + L.offScr), tc_test_abort()};
        int clusters = 0;
        e = pair_clusters(&clusters);
        if (e != cudaSuccess) return e;
        const int tiles = a.tiles_m * a.tiles_n;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * static_cast<unsigned>(tiles < clusters ? tiles : clusters));
        cfg.blockDim = dim3(tc2::THREADS);
        cfg.dynamicSmemBytes = tc2::STAGES * tc2::STAGE_BYTES + 1024;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, ozaki_tc_pair_kernel<2>, ma, mb, a);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    } else {
        if (!slice_map(&ma, sa, S, L.mp, L.kp, tc::BM) || !slice_map(&mb, sb, S, L.np, L.kp, Cf::BN))
            return cudaErrorInvalidValue;
        TcArgs a{sig, tau, {nullptr, nullptr, nullptr, nullptr}, g.ldc, g.m, g.n, L.kp, S,
                 static_cast<int>(L.mp / tc::BM), static_cast<int>(L.np / Cf::BN), err, nullptr,
                 tc_test_abort()};
        for (int c = 0; c < P; ++c) a.C[c] = g.C[c];
        const int smem = tc::STAGES * Cf::STAGE_BYTES + 1024;
        e = cudaFuncSetAttribute(ozaki_tc_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        const int tiles = a.tiles_m * a.tiles_n;
        const int grid = tiles < num_sms() ? tiles : num_sms();
        ozaki_tc_kernel<P><<<grid, 192, smem, s>>>(ma, mb, a);
        return cudaGetLastError();
    }
}

template <int P>
cudaError_t launch_ozaki(const GemmArgs<P>& g, int S, void* ws, cudaStream_t s, int variant, int engine)
{
    if (engine == 1) return launch_ozaki_tc<P>(g, S, ws, s);
    const OzakiLayout L = ozaki_layout(S, g.m, g.n, g.k, 1);
    int8_t* base = static_cast<int8_t*>(ws);
    int* sig = reinterpret_cast<int*>(base + L.offSig);
    int* tau = reinterpret_cast<int*>(base + L.offTau);
    int8_t* sa = base + L.offA;
    int8_t* sb = base + L.offB;
    cudaError_t e = slice_both<P>(g, S, L, sa, sb, sig, tau, s);
    if (e != cudaSuccess) return e;
    OzakiGemmArgs a{base + L.offA, base + L.offB, sig, tau, {nullptr, nullptr, nullptr, nullptr},
                    g.ldc, g.m, g.n, L.mp, L.np, L.kp, S};
    for (int c = 0; c < P; ++c) a.C[c] = g.C[c];
    if constexpr (P == 2) {
        // int8 tilings (DD 4096^3, S = 13 on GB300, 3-weight groups: 0 -> 88 ms,
        // 1 -> 91.5, 2 -> 90; the 64 x 64 tilings cannot hold 32 outputs'
        // 128-bit group sums in registers)
        switch (variant) {
        case 1: {   // 64 x 32 CTA tile, 4 warps of 32 x 16, 4 stages of 64 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 32), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 2, 2, 2, 2, 4, 3, 64><<<grid, 128, 0, s>>>(a);
            break;
        }
        case 2: {   // 64 x 32 CTA tile, 4 warps of 16 x 32, 4 stages of 64 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 32), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 1, 4, 4, 1, 4, 3, 64><<<grid, 128, 0, s>>>(a);
            break;
        }
        default: {  // 64 x 32 CTA tile, 4 warps of 32 x 16, 3 stages of 128 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 32), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 2, 2, 2, 2, 3, 3, 128><<<grid, 128, 0, s>>>(a);
            break;
        }
        }
    } else {
        // TD/QD: 64 x 16 CTA tile, 4 warps of 16 x 16 (8 outputs each), 3 stages of 128 bytes
        (void)variant;
        const dim3 grid(static_cast<unsigned>(L.np / 16), static_cast<unsigned>(L.mp / 64));
        ozaki_gemm_kernel<P, 1, 2, 4, 1, 3, 3, 128><<<grid, 128, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template cudaError_t launch_ozaki<2>(const GemmArgs<2>&, int, void*, cudaStream_t, int, int);
template cudaError_t launch_ozaki<3>(const GemmArgs<3>&, int, void*, cudaStream_t, int, int);
template cudaError_t launch_ozaki<4>(const GemmArgs<4>&, int, void*, cudaStream_t, int, int);


// ----------------------------------------------------- CRT form, host side

OzakiLayout crt_layout(int N, int64_t m, int64_t n, int64_t k, int engine, int halves)
{
    OzakiLayout L;
    const int elem_bytes = engine == 1 ? 2 : 1;
    const int64_t planes = static_cast<int64_t>(N) * halves;        // residue planes per operand
    const int64_t products = halves == 2 ? 3 * static_cast<int64_t>(N) : N;
    L.S = N;
    L.mp = round_up(m > 0 ? m : 1, 128);
    L.np = round_up(n > 0 ? n : 1, 128);
    L.kp = round_up(k > 0 ? k : 1, KPAD);
    L.offA = engine == 1 ? 256 : 0;                    // tcgen05: a 256-byte header (error code)
    L.offB = L.offA + round_up(planes * L.mp * L.kp * elem_bytes, 256);
    L.offSig = L.offB + round_up(planes * L.np * L.kp * elem_bytes, 256);
    L.offTau = L.offSig + round_up(L.mp * 4, 256);
    L.offScr = L.offTau + round_up(L.np * 4, 256);      // [N or 3N][mp][np] int8 residues of the products
    L.total = L.offScr + round_up(products * L.mp * L.np, 256);
    return L;
}

// M = m_0 ... m_(N-1) in 32-bit limbs.
static void crt_modulus(int N, uint32_t (&M)[crt::kRecLimbs])
{
    for (int k = 0; k < crt::kRecLimbs; ++k) M[k] = 0;
    M[0] = 1;
    for (int i = 0; i < N; ++i) {
        uint64_t carry = 0;
        for (int k = 0; k < crt::kRecLimbs; ++k) {
            const uint64_t p = static_cast<uint64_t>(M[k]) * static_cast<uint32_t>(crt::kHost.m[i]) + carry;
            M[k] = static_cast<uint32_t>(p);
            carry = p >> 32;
        }
    }
}

int crt_beta(int N, int64_t k, int halves)
{
    if (N < 1 || N > crt::kMaxModuli || k < 0 || (halves != 1 && halves != 2)) return -1;
    uint32_t T[crt::kRecLimbs];
    crt_modulus(N, T);
    // T = floor((M - 1) / k): the largest beta with k 2^(2 beta - 1) < M is
    // floor(bitlength(T) / 2)
    for (int w = 0; w < crt::kRecLimbs; ++w) {
        if (T[w]--) break;                 // M - 1 (M >= 2)
    }
    const uint64_t d = static_cast<uint64_t>(k > 0 ? k : 1);
    uint64_t rem = 0;
    for (int w = crt::kRecLimbs - 1; w >= 0; --w) {
        const uint64_t cur = (rem << 32) | T[w];
        T[w] = static_cast<uint32_t>(cur / d);
        rem = cur % d;
    }
    int bl = 0;
    for (int w = 0; w < crt::kRecLimbs; ++w)
        if (T[w]) bl = 32 * w + (32 - __builtin_clz(T[w]));
    // split integers: the largest w with k 2^(2w) < M, i.e. 2^(2w) <= T
    if (halves == 2) return bl >= 1 ? 2 * ((bl - 1) / 2) : 0;
    return bl / 2;
}

template <int P>
static cudaError_t crt_recover(const GemmArgs<P>& g, int N, int beta, int halves, const OzakiLayout& L,
                               const int* sig, const int* tau, const int8_t* rq, cudaStream_t s);

// Residues of both operands, with as few 16-bit limbs as beta needs (split
// integers: 2N planes, A1's residues then A0's).
template <int P, typename T>
static cudaError_t crt_residues(const GemmArgs<P>& g, int N, int halves, const OzakiLayout& L, T* ra, T* rb,
                                int* sig, int* tau, cudaStream_t s, int beta)
{
    switch (residue_kind(beta, halves)) {
    case 5: return slice_both<P, T, 5>(g, 2 * N, L, ra, rb, sig, tau, s, beta);
    case 4: return slice_both<P, T, 4>(g, 2 * N, L, ra, rb, sig, tau, s, beta);
    case 3: return slice_both<P, T, 3>(g, N, L, ra, rb, sig, tau, s, beta);
    case 2: return slice_both<P, T, 2>(g, N, L, ra, rb, sig, tau, s, beta);
    default: return slice_both<P, T, 1>(g, N, L, ra, rb, sig, tau, s, beta);
    }
}

template <int P>
cudaError_t launch_crt(const GemmArgs<P>& g, int N, void* ws, cudaStream_t s, int engine, int halves)
{
    const int beta = crt_beta(N, g.k, halves);
    if (beta < 1 || beta > crt_max_beta(halves)) return cudaErrorInvalidValue;
    const int planes = N * halves;
    const OzakiLayout L = crt_layout(N, g.m, g.n, g.k, engine, halves);
    int8_t* base = static_cast<int8_t*>(ws);
    int* sig = reinterpret_cast<int*>(base + L.offSig);
    int* tau = reinterpret_cast<int*>(base + L.offTau);
    int8_t* rq = base + L.offScr;
    cudaError_t e;
    if (engine == 1) {
        int* err = reinterpret_cast<int*>(base);
        uint16_t* sa = reinterpret_cast<uint16_t*>(base + L.offA);
        uint16_t* sb = reinterpret_cast<uint16_t*>(base + L.offB);
        e = cudaMemsetAsync(err, 0, sizeof(int), s);
        if (e == cudaSuccess) e = crt_residues<P, uint16_t>(g, N, halves, L, sa, sb, sig, tau, s, beta);
        if (e != cudaSuccess) return e;
        CUtensorMap ma, mb;
        if (!slice_map(&ma, sa, planes, L.mp, L.kp, tcc::BM) || !slice_map(&mb, sb, planes, L.np, L.kp, tcc::BN))
            return cudaErrorInvalidValue;
        const CrtTcArgs a{rq, L.mp, L.np, L.kp, N, static_cast<int>(L.mp / tcc::BM),
                          static_cast<int>(L.np / tcc::BN), err, tc_test_abort(), halves == 2 ? 1 : 0};
        const int smem = tcc::STAGES * tcc::STAGE_BYTES + 1024;
        e = cudaFuncSetAttribute(crt_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        const int tiles = a.tiles_m * a.tiles_n;
        const int grid = tiles < num_sms() ? tiles : num_sms();
        crt_tc_kernel<<<grid, 192, smem, s>>>(ma, mb, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return crt_recover<P>(g, N, beta, halves, L, sig, tau, rq, s);
    }
    int8_t* ra = base + L.offA;
    int8_t* rb = base + L.offB;
    e = crt_residues<P, int8_t>(g, N, halves, L, ra, rb, sig, tau, s, beta);
    if (e != cudaSuccess) return e;
    // 128 x 128 CTA tile, 8 warps of 64 x 32, 4 stages of 64 bytes of k
    constexpr int MT = 4, NT = 4, WM = 2, WN = 4, STG = 4, KS = 64;
    constexpr int smem = STG * (WM * MT * 16 + WN * NT * 8) * (KS + 16);
    e = cudaFuncSetAttribute(crt_gemm_kernel<MT, NT, WM, WN, STG, KS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const CrtGemmArgs ga{ra, rb, rq, L.mp, L.np, L.kp, N, halves == 2 ? 1 : 0};
    const dim3 grid(static_cast<unsigned>(L.np / 128), static_cast<unsigned>(L.mp / 128),
                    static_cast<unsigned>(halves == 2 ? 3 * N : N));
    crt_gemm_kernel<MT, NT, WM, WN, STG, KS><<<grid, WM * WN * 32, smem, s>>>(ga);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return crt_recover<P>(g, N, beta, halves, L, sig, tau, rq, s);
}

// The recovery kernel over the products' residues rq.
template <int P>
static cudaError_t crt_recover(const GemmArgs<P>& g, int N, int beta, int halves, const OzakiLayout& L,
                               const int* sig, const int* tau, const int8_t* rq, cudaStream_t s)
{
    CrtRecArgs ra_{rq, sig, tau, {nullptr, nullptr, nullptr, nullptr}, g.ldc, g.m, g.n, L.mp, L.np, N, beta, 0,
                   {}, {}};
    if (halves == 2) ra_.w = beta / 2;
    for (int c = 0; c < P; ++c) ra_.C[c] = g.C[c];
    crt_modulus(N, ra_.M);
    // H = ceil(M / 2) = (M + 1) >> 1
    uint32_t M1[crt::kRecLimbs];
    for (int k = 0; k < crt::kRecLimbs; ++k) M1[k] = ra_.M[k];
    for (int k = 0; k < crt::kRecLimbs; ++k)
        if (++M1[k]) break;
    for (int k = 0; k < crt::kRecLimbs; ++k)
        ra_.H[k] = (M1[k] >> 1) | (k + 1 < crt::kRecLimbs ? (M1[k + 1] << 31) : 0u);
    // W_i = (M / m_i) c_i with c_i the inverse of (M / m_i) mod m_i
    for (int i = 0; i < N; ++i) {
        const uint64_t mi = static_cast<uint64_t>(crt::kHost.m[i]);
        uint32_t Q[crt::kRecLimbs];
        uint64_t rem = 0;
        for (int k = crt::kRecLimbs - 1; k >= 0; --k) {      // Q = M / m_i (exact)
            const uint64_t cur = (rem << 32) | ra_.M[k];
            Q[k] = static_cast<uint32_t>(cur / mi);
            rem = cur % mi;
        }
        uint64_t qm = 0;                                      // Q mod m_i
        for (int k = crt::kRecLimbs - 1; k >= 0; --k) qm = ((qm << 32) | Q[k]) % mi;
        uint64_t c = 0;
        for (uint64_t x = 1; x < mi; ++x)
            if ((qm * x) % mi == 1) { c = x; break; }
        if (mi == 1) c = 0;
        uint64_t carry = 0;
        for (int k = 0; k < crt::kRecLimbs; ++k) {
            const uint64_t v = static_cast<uint64_t>(Q[k]) * c + carry;
            ra_.W[i][k] = static_cast<uint32_t>(v);
            carry = v >> 32;
        }
        ra_.f[i] = static_cast<float>(static_cast<double>(c) / static_cast<double>(mi));
    }
    if (halves == 2) {
        const unsigned grid2 = blocks_for(g.m * ((g.n + 1) / 2), 256);     // two outputs per thread
        switch ((N + 7) / 8) {
        case 1: crt_recover2_kernel<P, 8><<<grid2, 256, 0, s>>>(ra_); break;
        case 2: crt_recover2_kernel<P, 16><<<grid2, 256, 0, s>>>(ra_); break;
        case 3: crt_recover2_kernel<P, 24><<<grid2, 256, 0, s>>>(ra_); break;
        case 4: crt_recover2_kernel<P, 32><<<grid2, 256, 0, s>>>(ra_); break;
        case 5: crt_recover2_kernel<P, 40><<<grid2, 256, 0, s>>>(ra_); break;
        default: crt_recover2_kernel<P, 48><<<grid2, 256, 0, s>>>(ra_); break;
        }
        return cudaGetLastError();
    }
    const int64_t outs = g.m * ((g.n + 3) / 4);        // four outputs per thread
    const unsigned grid = blocks_for(outs, 256);
    switch ((N + 7) / 8) {
    case 1: crt_recover_kernel<P, 8><<<grid, 256, 0, s>>>(ra_); break;
    case 2: crt_recover_kernel<P, 16><<<grid, 256, 0, s>>>(ra_); break;
    case 3: crt_recover_kernel<P, 24><<<grid, 256, 0, s>>>(ra_); break;
    case 4: crt_recover_kernel<P, 32><<<grid, 256, 0, s>>>(ra_); break;
    case 5: crt_recover_kernel<P, 40><<<grid, 256, 0, s>>>(ra_); break;
    case 6: crt_recover_kernel<P, 48><<<grid, 256, 0, s>>>(ra_); break;
    default: crt_recover_kernel<P, 56><<<grid, 256, 0, s>>>(ra_); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_crt<2>(const GemmArgs<2>&, int, void*, cudaStream_t, int, int);
template cudaError_t launch_crt<3>(const GemmArgs<3>&, int, void*, cudaStream_t, int, int);
template cudaError_t launch_crt<4>(const GemmArgs<4>&, int, void*, cudaStream_t, int, int);

}  // namespace mpg
