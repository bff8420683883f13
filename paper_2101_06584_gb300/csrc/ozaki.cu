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

#include <cuda_bf16.h>

#include <cstdint>
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

// The S digits of (hi + lo) 2^-sigma (nearest, ties to even).
__device__ __forceinline__ void ozaki_digits(double hi, double lo, int sigma, int S, int8_t* out)
{
    const int F = 7 * S + 12;
    bool sticky;
    __int128 R = fixed_point(hi, lo, sigma, F, sticky);
    for (int s = 1; s <= S; ++s) {
        const int q = F - 7 * s;
        const __int128 U = static_cast<__int128>(1) << q;
        const __int128 half = U >> 1;
        __int128 dd = (R + half) >> q;                       // nearest, ties up
        if (!sticky && (R & (U - 1)) == half && (dd & 1)) dd -= 1;   // ties to even
        R -= dd << q;
        out[s - 1] = static_cast<int8_t>(static_cast<int>(dd));
    }
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

// The S digits of the sum of the P components, each floored at
// 2^(sigma - F - 64) (nearest, ties to even).
template <int P>
__device__ __forceinline__ void ozaki_digits_wide(const double (&c)[P], int sigma, int S, int8_t* out)
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
    for (int s = 1; s <= S; ++s) {
        const int q = F + kGuardBits - 7 * s;     // bit position of the digit's unit (>= 76)
        const int wq = q >> 6, bq = q & 63;
        // t = floor((W + 2^(q-1)) / 2^q) from a copy with the half added
        Wide H = W;
        wide_add_shifted(H, 1, q - 1);
        // bits q .. q+63 as a signed 64-bit value; |t| <= 65, so the bits
        // above q + 7 are copies of the sign
        int64_t t;
        if (wq + 1 < kWideWords) {
            const uint64_t hi = bq == 0 ? 0ull : (H.w[wq + 1] << (64 - bq));
            t = static_cast<int64_t>((H.w[wq] >> bq) | hi);
        } else {
            t = static_cast<int64_t>(H.w[wq]) >> bq;            // arithmetic: top word
        }
        // a tie leaves no bits below q after adding the half
        bool below_zero = (H.w[wq] & ((bq == 0) ? 0ull : ((1ull << bq) - 1))) == 0;
#pragma unroll
        for (int i = 0; i < kWideWords; ++i)
            if (i < wq) below_zero = below_zero && H.w[i] == 0ull;
        if (below_zero && (t & 1)) t -= 1;
        wide_add_shifted(W, -t, q);
        out[s - 1] = static_cast<int8_t>(t);
    }
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

// One thread per vector whose elements are ld apart (vectors adjacent).
__global__ void ozaki_scale_strided(const double* __restrict__ hi, int64_t count, int64_t len,
                                    int64_t ld, int* __restrict__ out)
{
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= count) return;
    uint64_t mx = 0;
    for (int64_t p = 0; p < len; ++p) {
        const uint64_t b = abs_bits(hi[p * ld + v]);
        mx = b > mx ? b : mx;
    }
    out[v] = mx ? ilogb_bits(mx) + 2 : 0;
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

// The S digits of element `off` of the component planes.
template <int P>
__device__ __forceinline__ void element_digits(const Planes<P>& pl, int64_t off, int sigma, int S,
                                               int8_t* out)
{
    if constexpr (P == 2) {
        ozaki_digits(pl.c[0][off], pl.c[1][off], sigma, S, out);
    } else {
        double c[P];
#pragma unroll
        for (int i = 0; i < P; ++i) c[i] = pl.c[i][off];
        ozaki_digits_wide<P>(c, sigma, S, out);
    }
}

template <int P, typename T>
__global__ void ozaki_slice_rows(const Planes<P> pl, int64_t rows, int64_t len, int64_t ld,
                                 const int* __restrict__ sig, int S, int64_t rows_pad, int64_t kp,
                                 T* __restrict__ out)
{
    const int64_t quads = kp / 4;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= rows_pad * quads) return;
    const int64_t r = t / quads;
    const int64_t p0 = (t % quads) * 4;
    int8_t dg[4][kOzakiMaxSlicesWide];
    const int sg = r < rows ? sig[r] : 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t p = p0 + u;
        if (r < rows && p < len) {
            element_digits<P>(pl, r * ld + p, sg, S, dg[u]);
        } else {
            for (int s = 0; s < S; ++s) dg[u][s] = 0;
        }
    }
    for (int s = 0; s < S; ++s)
        store4(out + (static_cast<int64_t>(s) * rows_pad + r) * kp + p0, dg[0][s], dg[1][s], dg[2][s],
               dg[3][s]);
}

// Rows of the sliced operand are strided (element (r, p) at base[p*ld + r]):
// a 32 x 32 tile is read with r fastest, sliced, transposed through shared
// memory and written with p fastest.
template <int P, typename T>
__global__ void __launch_bounds__(256)
ozaki_slice_cols(const Planes<P> pl, int64_t rows, int64_t len, int64_t ld,
                 const int* __restrict__ sig, int S, int64_t rows_pad, int64_t kp,
                 T* __restrict__ out)
{
    constexpr int SMAX = P == 2 ? kOzakiMaxSlices : kOzakiMaxSlicesWide;
    __shared__ int8_t tile[SMAX][32][36];
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 32;
    const int64_t p0 = static_cast<int64_t>(blockIdx.y) * 32;
    const int tr = threadIdx.x & 31;        // r within the tile
    const int tp = threadIdx.x >> 5;        // 0..7
    const int64_t r = r0 + tr;
    const int sg = r < rows ? sig[r] : 0;
    for (int pp = tp; pp < 32; pp += 8) {
        const int64_t p = p0 + pp;
        int8_t dg[SMAX];
        if (r < rows && p < len) {
            element_digits<P>(pl, p * ld + r, sg, S, dg);
        } else {
            for (int s = 0; s < S; ++s) dg[s] = 0;
        }
        for (int s = 0; s < S; ++s) tile[s][tr][pp] = dg[s];
    }
    __syncthreads();
    // write: each thread writes 4 consecutive p of one row r
    const int wr = threadIdx.x >> 3;        // 0..31 row within tile
    const int wq = (threadIdx.x & 7) * 4;   // p offset
    const int64_t row = r0 + wr;
    if (row < rows_pad && p0 + wq < kp) {
        for (int s = 0; s < S; ++s)
            store4(out + (static_cast<int64_t>(s) * rows_pad + row) * kp + p0 + wq, tile[s][wr][wq],
                   tile[s][wr][wq + 1], tile[s][wr][wq + 2], tile[s][wr][wq + 3]);
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

// v * 2^e as a binary64, exactly (v an int32, result in the normal range),
// built with integer operations.
__device__ __forceinline__ double scaled_int(int v, int e)
{
    if (v == 0) return 0.0;
    const unsigned u = v < 0 ? 0u - static_cast<unsigned>(v) : static_cast<unsigned>(v);
    const int lz = __clz(static_cast<int>(u));
    const int ex = 31 - lz + e;
    const uint64_t mant = (static_cast<uint64_t>(u) << (21 + lz)) & ((1ull << 52) - 1);
    const uint64_t bits = (static_cast<uint64_t>(v < 0) << 63) |
                          (static_cast<uint64_t>(ex + 1023) << 52) | mant;
    return __longlong_as_double(static_cast<long long>(bits));
}

// v * 2^e as a binary64, exactly (|v| < 2^53, result in the normal range).
__device__ __forceinline__ double scaled_int64(int64_t v, int e)
{
    if (v == 0) return 0.0;
    const uint64_t u = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
    const int lz = __clzll(static_cast<long long>(u));
    const int ex = 63 - lz + e;
    const uint64_t mant = (u << (lz - 11)) & ((1ull << 52) - 1);
    const uint64_t bits = (static_cast<uint64_t>(v < 0) << 63) |
                          (static_cast<uint64_t>(ex + 1023) << 52) | mant;
    return __longlong_as_double(static_cast<long long>(bits));
}

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

// CTA of WM x WN warps; each warp owns MT x NT fragments of 16 x 8 outputs,
// so the CTA tile is (WM*MT*16) x (WN*NT*8).  Slice tiles of KS bytes of k
// are staged through a STG-deep cp.async pipeline.  P output components:
// DD adds every weight's sum; TD/QD combine three weights exactly in int64
// first and add the group.
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
    int64_t grp[MT][NT][4];
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
            // TD/QD: position of w in its group of three, counted from the
            // least significant weight S+1; the group ends at its third
            // weight or at w = 2
            const int j = (S + 1 - w) % 3;
            const bool group_end = (P == 2) || j == 2 || w == 2;
            const int wmax = P == 2 ? w : w + j;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        double y[P];
                        if constexpr (P == 2) {
                            y[0] = scaled_int(ci[mt][nt][r], sg[mt][r >> 1] + tu[nt][r & 1] - 7 * w);
                        } else {
                            grp[mt][nt][r] += static_cast<int64_t>(ci[mt][nt][r]) << (7 * j);
                            y[0] = scaled_int64(grp[mt][nt][r], sg[mt][r >> 1] + tu[nt][r & 1] - 7 * wmax);
                        }
                        ci[mt][nt][r] = 0;
                        if (group_end) {
#pragma unroll
                            for (int c = 1; c < P; ++c) y[c] = f.zero;
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

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The same weight sums with the digits as bf16 on the bf16 tensor path
// (mma.sync m16n8k16, fp32 accumulation).  On GB300 this runs no faster than
// the int8 kernel (DD 4096^3, S = 13: 89.7 vs 87.8 ms): at the bf16 rate its
// fragment loads would need ~185 B/clk/SM of shared memory, more than the SM
// delivers, and larger warp tiles do not fit beside the DD accumulators.  Every product is an integer of at
// most 2^12 and every partial sum an integer; the fp32 fragments are drained
// into the int32 weight sums every 2048 values of k, so no partial sum exceeds
// 2^23 and each is exactly representable: the int32 sums, and so the result,
// equal those of the int8 path bit for bit.
template <int MT, int NT, int WM, int WN, int STG, int MINB, int KSE>
__global__ void __launch_bounds__(WM * WN * 32, MINB) ozaki_gemm_bf16_kernel(const OzakiGemmArgs g)
{
    constexpr int NTHR = WM * WN * 32;
    constexpr int BM = WM * MT * 16;
    constexpr int BN = WN * NT * 8;
    constexpr int SROWE = KSE + 8;        // row stride in elements: conflict-free fragment loads
    constexpr int CPR = KSE * 2 / 16;     // 16-byte chunks per row
    constexpr int FLUSH = 2048 / KSE;     // k-tiles between drains of the fp32 fragments
    __shared__ __align__(16) uint16_t As[STG][BM * SROWE];
    __shared__ __align__(16) uint16_t Bs[STG][BN * SROWE];

    const mp::Rn f = mp::make_rn();
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const int wm = warp / WN, wn = warp % WN;
    const int64_t m0 = static_cast<int64_t>(blockIdx.y) * BM;
    const int64_t n0 = static_cast<int64_t>(blockIdx.x) * BN;
    const int S = g.S;
    const int KT = static_cast<int>(g.kp / KSE);
    const int total = (S * (S + 1) / 2) * KT;

    int sg[MT][2], tu[NT][2];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) sg[mt][h] = g.sig[m0 + wm * MT * 16 + mt * 16 + gq + h * 8];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) tu[nt][h] = g.tau[n0 + wn * NT * 8 + nt * 8 + 2 * tq + h];

    double acc0[MT][NT][4], acc1[MT][NT][4];
    float cf[MT][NT][4];
    int ci[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                acc0[mt][nt][r] = 0.0; acc1[mt][nt][r] = 0.0; cf[mt][nt][r] = 0.f; ci[mt][nt][r] = 0;
            }

    auto load = [&](int stage, const Cursor& c) {
        const uint16_t* a = static_cast<const uint16_t*>(g.sa) +
                            ((static_cast<int64_t>(c.s - 1) * g.mp + m0) * g.kp) + static_cast<int64_t>(c.kt) * KSE;
        const uint16_t* b = static_cast<const uint16_t*>(g.sb) +
                            ((static_cast<int64_t>(c.w - c.s - 1) * g.np + n0) * g.kp) + static_cast<int64_t>(c.kt) * KSE;
        for (int chunk = tid; chunk < (BM + BN) * CPR; chunk += NTHR) {
            const int row = chunk / CPR, col = (chunk % CPR) * 8;
            if (row < BM)
                cp_async16(&As[stage][row * SROWE + col], a + static_cast<int64_t>(row) * g.kp + col);
            else
                cp_async16(&Bs[stage][(row - BM) * SROWE + col],
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

    int since = 0;
    for (int it = 0; it < total; ++it) {
        cp_async_wait<STG - 2>();
        __syncthreads();
        {
            const int nxt = it + STG - 1;
            if (nxt < total) load(nxt % STG, ld);
            ld.advance(S, KT);
            cp_async_commit();
        }
        const uint16_t* as = As[it % STG];
        const uint16_t* bs = Bs[it % STG];
#pragma unroll
        for (int kk = 0; kk < KSE; kk += 16) {
            uint32_t af[MT][4], bf[NT][2];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const int r = wm * MT * 16 + mt * 16 + gq;
                af[mt][0] = *reinterpret_cast<const uint32_t*>(as + r * SROWE + kk + 2 * tq);
                af[mt][1] = *reinterpret_cast<const uint32_t*>(as + (r + 8) * SROWE + kk + 2 * tq);
                af[mt][2] = *reinterpret_cast<const uint32_t*>(as + r * SROWE + kk + 8 + 2 * tq);
                af[mt][3] = *reinterpret_cast<const uint32_t*>(as + (r + 8) * SROWE + kk + 8 + 2 * tq);
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int c = wn * NT * 8 + nt * 8 + gq;
                bf[nt][0] = *reinterpret_cast<const uint32_t*>(bs + c * SROWE + kk + 2 * tq);
                bf[nt][1] = *reinterpret_cast<const uint32_t*>(bs + c * SROWE + kk + 8 + 2 * tq);
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) mma_bf16(cf[mt][nt], af[mt], bf[nt]);
        }
        const int w = cm.w;
        cm.advance(S, KT);
        const bool weight_end = (cm.w != w || it == total - 1);
        if (++since == FLUSH || weight_end) {
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        ci[mt][nt][r] += __float2int_rn(cf[mt][nt][r]);
                        cf[mt][nt][r] = 0.f;
                    }
            since = 0;
        }
        if (weight_end) {
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int e = sg[mt][r >> 1] + tu[nt][r & 1] - 7 * w;
                        const double x[2] = {acc0[mt][nt][r], acc1[mt][nt][r]};
                        const double y[2] = {scaled_int(ci[mt][nt][r], e), f.zero};
                        double z[2];
                        mp::dd_add(f, x, y, z);
                        acc0[mt][nt][r] = z[0];
                        acc1[mt][nt][r] = z[1];
                        ci[mt][nt][r] = 0;
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
                    g.C[0][row * g.ldc + col] = acc0[mt][nt][r];
                    g.C[1][row * g.ldc + col] = acc1[mt][nt][r];
                }
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
}  // namespace

cudaError_t ozaki_static_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        // In host code the array's name is only a stand-in: the kernels need
        // the device address, looked up once per device with it current.
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
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
    return L;
}

static unsigned blocks_for(int64_t threads, int per) { return static_cast<unsigned>((threads + per - 1) / per); }

// Slice one operand: vectors (rows of op(A) or columns of op(B)) of length
// len; `contig` says whether a vector's elements are adjacent in memory.
template <int P, typename T>
static cudaError_t slice_operand(const Planes<P>& pl, int64_t count, int64_t len, int64_t ld,
                                 bool contig, int S, int64_t count_pad, int64_t kp, T* out,
                                 int* sig, cudaStream_t s)
{
    const double* lead = pl.c[0];
    if (contig) ozaki_scale_contig<<<blocks_for(count * 32, 256), 256, 0, s>>>(lead, count, len, ld, sig);
    else ozaki_scale_strided<<<blocks_for(count, 256), 256, 0, s>>>(lead, count, len, ld, sig);
    if (count_pad > count)
        ozaki_fill_int<<<blocks_for(count_pad - count, 256), 256, 0, s>>>(sig, count, count_pad);
    if (contig) {
        ozaki_slice_rows<P, T><<<blocks_for(count_pad * (kp / 4), 128), 128, 0, s>>>(
            pl, count, len, ld, sig, S, count_pad, kp, out);
    } else {
        const dim3 grid(static_cast<unsigned>(count_pad / 32), static_cast<unsigned>(kp / 32));
        ozaki_slice_cols<P, T><<<grid, 256, 0, s>>>(pl, count, len, ld, sig, S, count_pad, kp, out);
    }
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_ozaki(const GemmArgs<P>& g, int S, void* ws, cudaStream_t s, int variant, int engine)
{
    const int eb = engine == 1 ? 2 : 1;
    const OzakiLayout L = ozaki_layout(S, g.m, g.n, g.k, eb);
    int8_t* base = static_cast<int8_t*>(ws);
    int* sig = reinterpret_cast<int*>(base + L.offSig);
    int* tau = reinterpret_cast<int*>(base + L.offTau);
    Planes<P> pa, pb;
    for (int c = 0; c < P; ++c) {
        pa.c[c] = g.A[c];
        pb.c[c] = g.B[c];
    }
    cudaError_t e;
    // op(A) row i: contiguous unless A is stored transposed; op(B) column j:
    // contiguous only if B is stored transposed
    if (engine == 1) {
        uint16_t* sa = reinterpret_cast<uint16_t*>(base + L.offA);
        uint16_t* sb = reinterpret_cast<uint16_t*>(base + L.offB);
        e = slice_operand(pa, g.m, g.k, g.lda, !g.trans_a, S, L.mp, L.kp, sa, sig, s);
        if (e == cudaSuccess) e = slice_operand(pb, g.n, g.k, g.ldb, g.trans_b != 0, S, L.np, L.kp, sb, tau, s);
    } else {
        int8_t* sa = base + L.offA;
        int8_t* sb = base + L.offB;
        e = slice_operand(pa, g.m, g.k, g.lda, !g.trans_a, S, L.mp, L.kp, sa, sig, s);
        if (e == cudaSuccess) e = slice_operand(pb, g.n, g.k, g.ldb, g.trans_b != 0, S, L.np, L.kp, sb, tau, s);
    }
    if (e != cudaSuccess) return e;
    OzakiGemmArgs a{base + L.offA, base + L.offB, sig, tau, {nullptr, nullptr, nullptr, nullptr},
                    g.ldc, g.m, g.n, L.mp, L.np, L.kp, S};
    for (int c = 0; c < P; ++c) a.C[c] = g.C[c];
    if constexpr (P == 2) {
        if (engine == 1) {
            // 64 x 32 CTA tile, 4 warps of 32 x 16, 3 stages of 64 bf16
            const dim3 grid(static_cast<unsigned>(L.np / 32), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_bf16_kernel<2, 2, 2, 2, 3, 3, 64><<<grid, 128, 0, s>>>(a);
            return cudaGetLastError();
        }
        // int8 tilings, measured at DD 4096^3, S = 13 on GB300: 0 -> 88 ms, 1 -> 102,
        // 2 -> 91.5, 3 -> 90, 4 -> 96
        switch (variant) {
        case 1: {   // 64 x 64 CTA tile, 4 warps of 32 x 32, 3 stages of 64 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 64), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 2, 4, 2, 2, 3, 1, 64><<<grid, 128, 0, s>>>(a);
            break;
        }
        case 2: {   // 64 x 32 CTA tile, 4 warps of 32 x 16, 4 stages of 64 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 32), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 2, 2, 2, 2, 4, 4, 64><<<grid, 128, 0, s>>>(a);
            break;
        }
        case 3: {   // 64 x 32 CTA tile, 4 warps of 16 x 32, 4 stages of 64 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 32), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 1, 4, 4, 1, 4, 4, 64><<<grid, 128, 0, s>>>(a);
            break;
        }
        case 4: {   // 64 x 64 CTA tile, 8 warps of 32 x 16, 4 stages of 64 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 64), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 2, 2, 2, 4, 4, 2, 64><<<grid, 256, 0, s>>>(a);
            break;
        }
        default: {  // 64 x 32 CTA tile, 4 warps of 32 x 16, 3 stages of 128 bytes
            const dim3 grid(static_cast<unsigned>(L.np / 32), static_cast<unsigned>(L.mp / 64));
            ozaki_gemm_kernel<2, 2, 2, 2, 2, 3, 4, 128><<<grid, 128, 0, s>>>(a);
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

}  // namespace mpg
