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
#include "ozaki_common.cuh"

namespace mpg {

// ------------------------------------------------------------------ product

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
                            umma_pair(tmem + b * tc2::ACC_COLS, da + 2ull * kk, db + 2ull * kk, tc2::IDESC,
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

cudaError_t side_stream(SideStream** out)
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

}  // namespace mpg
