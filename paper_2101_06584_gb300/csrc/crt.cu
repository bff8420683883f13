// crt.cu -- the CRT form (Ozaki scheme II) of C := op(A) op(B), not in the
// paper: residue products on mma.sync s8 or on tcgen05, exact recovery of
// the integer product and its rounding to P binary64 components.  The
// residues themselves come from the shared slice kernels (ozaki_common.cuh).
#include "ozaki_common.cuh"

namespace mpg {

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
// Per output: the integer in [-floor(M/2), ceil(M/2)) congruent to the
// residues of the product (A'B' itself, since |A'B'| < M/2), and the P
// components of that integer times 2^(sigma_i + tau_j - 2 beta), each the
// nearest binary64 (ties to even) of what the previous ones leave, with
// integer operations only.
//
// The integer comes from the CRT weights W_i = (M / m_i) c_i, with c_i the
// inverse of M / m_i modulo m_i: for residues r_i in [0, m_i),
// S = sum_i r_i W_i is congruent to A'B' and S / M = sum_i r_i c_i / m_i.
// S is accumulated exactly in 64-bit columns of 32-bit limbs; the quotient
// q = floor(S / M + 1/2) is estimated in binary32 (off by at most one: the
// sum is below 2^14 and its rounding error far below one half), and
// Z = S - q M, corrected once by M either way, is the centred integer in
// two's complement.
//
// Rounding a two's-complement Z: with b the bit length of Z (of ~Z when Z is
// negative) and s = max(b - 53, -1074 - e) the exponent of the last place
// kept, the component is 2^s times Q + up, where Q = floor(Z / 2^s) and up
// rounds by the bit below s and the bits under it (ties to even).  What it
// leaves, Z - (Q + up) 2^s, has the same bits as Z below s and only sign
// bits from s upward (ones when up, the remainder being negative then).  So
// every component is read from the original bit pattern of Z: a position p
// below which the bits are Z's own, the sign pattern above it, and three
// bit masks over the limbs (nonzero, not all ones, any nonzero below) that
// give bit lengths and sticky bits without scanning.  The limbs live in a
// per-thread column of shared memory, where a limb at a computed index is
// one load.

namespace crt {
constexpr int kRecLimbs = 11;                     // M < 2^352
constexpr int kRecGroups = (kMaxModuli + 3) / 4;  // moduli in groups of four
}

struct CrtRecArgs {
    const int8_t* res;      // [N][mp][np] residues of the products ([3N] with split integers: hh, mid, ll)
    const int* sig;
    const int* tau;
    double* C[4];
    int64_t ldc, m, n, mp, np;
    int N, beta;
    int w;                  // split integers: C' = P_hh 2^(2w) + P_mid 2^w + P_ll
    uint32_t M[crt::kRecLimbs];          // the product of the moduli
    uint32_t H[crt::kRecLimbs];          // ceil(M / 2)
    uint32_t F[crt::kRecLimbs];          // floor(M / 2)
    uint32_t M16[2 * crt::kRecLimbs];     // M in 16-bit limbs (one per word)
    uint32_t K16[2 * crt::kRecLimbs + 1]; // 128 sum_i W_i in 16-bit limbs (the bias of the residues)
    int64_t KF;                          // 128 sum_i floor(2^24 c_i / m_i)
    // the CRT weights W_i = (M / m_i) c_i, c_i = (M / m_i)^-1 mod m_i, as bytes:
    // byte t of Wd[g][j] is byte j of W_(4g+t) (zero for 4g + t >= N)
    uint32_t Wd[crt::kRecGroups][4 * crt::kRecLimbs];
    // likewise the three bytes of floor(2^24 c_i / m_i)
    uint32_t Fd[crt::kRecGroups][3];
};

constexpr int kRecThreads = 256;

// A per-thread column of LC 32-bit limbs in shared memory (limb k of this
// thread at col[k * kRecThreads]), least significant first.
struct LimbCol {
    uint32_t* col;
    __device__ __forceinline__ uint32_t get(int k) const { return col[k * kRecThreads]; }
    __device__ __forceinline__ void set(int k, uint32_t v) const { col[k * kRecThreads] = v; }
};

// Bit masks over the LC limbs of Z: limb k nonzero, limb k not all ones, and
// any limb below k nonzero.
struct LimbMasks {
    uint32_t nz0, nz1, below;
};

template <int LC>
__device__ __forceinline__ LimbMasks limb_masks(const uint32_t (&z)[LC])
{
    LimbMasks mk{0u, 0u, 0u};
    bool any = false;
#pragma unroll
    for (int k = 0; k < LC; ++k) {
        if (any) mk.below |= 1u << k;
        if (z[k] != 0u) mk.nz0 |= 1u << k;
        if (z[k] != ~0u) mk.nz1 |= 1u << k;
        any = any || z[k] != 0u;
    }
    return mk;
}

template <int LC>
__device__ __forceinline__ LimbMasks limb_masks(const LimbCol& z)
{
    LimbMasks mk{0u, 0u, 0u};
    bool any = false;
#pragma unroll
    for (int k = 0; k < LC; ++k) {
        const uint32_t v = z.get(k);
        if (any) mk.below |= 1u << k;
        if (v != 0u) mk.nz0 |= 1u << k;
        if (v != ~0u) mk.nz1 |= 1u << k;
        any = any || v != 0u;
    }
    return mk;
}

// Bits [pos, pos + 64) of the remainder: Z's own bits below p, sx above.
template <int LC>
__device__ __forceinline__ uint64_t window64(const LimbCol& z, int pos, int p, uint32_t sx)
{
    const int w = pos >> 5, r = pos & 31;
    const uint32_t x0 = z.get(w < LC ? w : LC - 1);
    const uint32_t x1 = z.get(w + 1 < LC ? w + 1 : LC - 1);
    const uint32_t x2 = z.get(w + 2 < LC ? w + 2 : LC - 1);
    uint64_t v = static_cast<uint64_t>(__funnelshift_r(x0, x1, r)) |
                 (static_cast<uint64_t>(__funnelshift_r(x1, x2, r)) << 32);
    const int cut = p - pos;                           // bits of Z kept in the window (>= 1)
    if (cut < 64) {
        const uint64_t keep = (1ull << cut) - 1ull;
        v = (v & keep) | (sx ? ~keep : 0ull);
    }
    return v;
}

// The P components of Z 2^e, Z a two's-complement integer of LC limbs.
template <int LC, int P>
__device__ __forceinline__ void round_components(const LimbCol& z, const LimbMasks& mk, int e, double* const* C,
                                                 int64_t off)
{
    int p = 32 * LC;                                   // Z's own bits lie below p
    uint32_t sx = (z.get(LC - 1) >> 31) ? ~0u : 0u;    // the remainder's sign pattern above p
    bool done = false;
#pragma unroll
    for (int c = 0; c < P; ++c) {
        double out = 0.0;
        if (!done) {
            // b: bit length of the remainder (of its complement when negative)
            int b = 0;
            {
                const int w = p >> 5, r = p & 31;
                uint32_t v = 0u;
                if (r) v = (z.get(w) ^ sx) & ((1u << r) - 1u);
                if (v) {
                    b = 32 * w + 32 - __clz(static_cast<int>(v));
                } else {
                    const uint32_t lower = w >= 32 ? ~0u : ((1u << w) - 1u);
                    const uint32_t m = (sx ? mk.nz1 : mk.nz0) & lower;
                    if (m) {
                        const int t = 31 - __clz(static_cast<int>(m));
                        b = 32 * t + 32 - __clz(static_cast<int>(z.get(t) ^ sx));
                    }
                }
            }
            if (b == 0 && !sx) {
                done = true;                           // exactly zero: this and the rest are +0
            } else {
                int s = b - 53;
                if (s < -1074 - e) s = -1074 - e;
                if (s >= p) {
                    // below the subnormal range: |remainder| <= 2^(p-1) <= 2^(s-1)
                    // rounds to a zero of its sign, and stays the remainder
                    C[c][off] = sx ? -0.0 : 0.0;
                    continue;
                }
                int64_t q;                             // the component is q 2^(s + e)
                bool up = false;
                if (s <= 0) {                          // the remainder itself: exact
                    q = static_cast<int64_t>(window64<LC>(z, 0, p, sx) << (-s));
                    done = true;
                } else {
                    const int64_t Q = static_cast<int64_t>(window64<LC>(z, s, p, sx) << 9) >> 9;
                    const int h = s - 1;               // the half bit (h < p)
                    const uint32_t lh = z.get(h >> 5);
                    const bool half = (lh >> (h & 31)) & 1u;
                    const bool sticky = ((mk.below >> (h >> 5)) & 1u) || (lh & ((1u << (h & 31)) - 1u));
                    up = half && (sticky || (Q & 1));
                    q = Q + (up ? 1 : 0);
                    if (!half && !sticky) done = true; // nothing left below
                }
                const bool neg = q < 0 || (q == 0 && sx);
                uint64_t mag = static_cast<uint64_t>(q < 0 ? -q : q);
                int ex = s + e;
                const uint64_t sign = neg ? (1ull << 63) : 0ull;
                if (mag == 0) {
                    out = __longlong_as_double(static_cast<long long>(sign));
                } else {
                    if (mag == (1ull << 53)) {
                        mag = 1ull << 52;
                        ++ex;
                    }
                    if (mag >= (1ull << 52)) {
                        const int biased = ex + 52 + 1023;
                        if (biased > 2046) {
                            out = __longlong_as_double(static_cast<long long>(sign | 0x7ff0000000000000ull));
                            done = true;       // after an infinity the rest are +0
                        } else {
                            out = __longlong_as_double(static_cast<long long>(
                                sign | (static_cast<uint64_t>(biased) << 52) | (mag - (1ull << 52))));
                        }
                    } else {                   // subnormal: ex = -1074
                        out = __longlong_as_double(static_cast<long long>(sign | mag));
                    }
                }
                p = s;
                sx = up ? ~0u : 0u;
            }
        }
        C[c][off] = out;
    }
}

// The centred integer of one product (its residues r_i at res[i * plane],
// i < N) as L limbs of two's complement.  NB: N rounded up to a multiple of
// 8 (the unrolled bound of the loops); L = NB / 4 limbs, at most 11, hold M.
// The residues, biased to r_i + 128 in [0, 256) (the top bit of each byte
// flipped) and four to a register, meet the bytes of the CRT weights in
// dot products of four (dp4a): column j sums (r_i + 128) byte_j(W_i) over the
// moduli (below 13 * 4 * 255 * 255 < 2^22), so sum_j col_j 2^(8j) - K, with
// K = 128 sum_i W_i, is S = sum_i r_i W_i, congruent to A'B' modulo M.  Three
// more columns against the bytes of floor(2^24 c_i / m_i) give 2^24 S / M to
// within 49 * 128 units, whence q = floor(S / M + 1/2) up to one either way.
// The columns, paired into 16-bit columns less K and q M, are carried into
// limbs, and one addition or subtraction of M centres the result.  Residues
// of moduli i >= N (up to NB) are read from plane N - 1 and meet zero
// weights.
template <int NB, int L>
__device__ __forceinline__ void crt_centred(const CrtRecArgs& g, const int8_t* res, int64_t plane, int N,
                                            uint32_t (&Z)[L])
{
    constexpr int G = NB / 4;
    constexpr int D = 4 * L;
    uint32_t r4[G];
    const uint8_t* rp = reinterpret_cast<const uint8_t*>(res);
#pragma unroll
    for (int q4 = 0; q4 < G; ++q4) {
        uint32_t v = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v |= static_cast<uint32_t>(*rp) << (8 * t);
            if (4 * q4 + t + 1 < N) rp += plane;
        }
        r4[q4] = v ^ 0x80808080u;
    }
    unsigned S[D], Q[3] = {0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < D; ++j) S[j] = 0u;
#pragma unroll
    for (int q4 = 0; q4 < G; ++q4) {
        if (4 * q4 < N) {
#pragma unroll
            for (int j = 0; j < D; ++j) S[j] = __dp4a(r4[q4], g.Wd[q4][j], S[j]);
#pragma unroll
            for (int j = 0; j < 3; ++j) Q[j] = __dp4a(r4[q4], g.Fd[q4][j], Q[j]);
        }
    }
    const int64_t qfix = static_cast<int64_t>(Q[0]) + (static_cast<int64_t>(Q[1]) << 8) +
                         (static_cast<int64_t>(Q[2]) << 16) - g.KF + (1ll << 23);
    const int q = static_cast<int>(qfix >> 24);
    // 16-bit columns of S - q M (|.| < 2^31), carried into L + 1 limbs
    uint32_t X[L + 1];
    int carry = 0;
#pragma unroll
    for (int k = 0; k <= 2 * L; ++k) {
        const int c = (k < 2 * L ? static_cast<int>(S[2 * k] + S[2 * k + 1] * 256u) -
                                       q * static_cast<int>(g.M16[k])
                                 : 0) -
                      static_cast<int>(g.K16[k]);
        const int v = c + carry;
        carry = v >> 16;                               // arithmetic: floor
        const uint32_t u = static_cast<uint32_t>(v) & 0xffffu;
        if (k & 1) X[k >> 1] |= u << 16;
        else X[k >> 1] = u;
    }
    X[L] |= static_cast<uint32_t>(carry) << 16;        // the sign above
    // X in [-3M/2, 3M/2): X >= ceil(M/2) -> X - M; X < -floor(M/2) -> X + M
    int64_t b1 = 0, b2 = 0;
#pragma unroll
    for (int k = 0; k <= L; ++k) {
        const uint32_t hk = k < L ? g.H[k] : 0u, fk = k < L ? g.F[k] : 0u;
        const int64_t xs = k < L ? static_cast<int64_t>(X[k]) : static_cast<int64_t>(static_cast<int32_t>(X[k]));
        const int64_t d1 = xs - static_cast<int64_t>(hk) + b1;
        b1 = d1 >> 32;
        const int64_t d2 = xs + static_cast<int64_t>(fk) + b2;
        b2 = d2 >> 32;
    }
    const bool ge = b1 >= 0, lt = b2 < 0;              // the signs of X - H and X + F
    uint64_t c2 = ge ? 1u : 0u;                        // X - M = X + ~M + 1
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const uint32_t mk = g.M[k];
        const uint32_t a = ge ? ~mk : (lt ? mk : 0u);
        const uint64_t v = static_cast<uint64_t>(X[k]) + a + c2;
        Z[k] = static_cast<uint32_t>(v);
        c2 = v >> 32;
    }
}

template <int P, int NB>
__global__ void __launch_bounds__(kRecThreads) crt_recover_kernel(const __grid_constant__ CrtRecArgs g)
{
    constexpr int L = NB / 4 < crt::kRecLimbs ? NB / 4 : crt::kRecLimbs;
    __shared__ uint32_t cols[L * kRecThreads];
    const int64_t t = static_cast<int64_t>(blockIdx.x) * kRecThreads + threadIdx.x;
    if (t >= g.m * g.n) return;
    const int64_t row = t / g.n, col = t % g.n;
    uint32_t Z[L];
    crt_centred<NB, L>(g, g.res + row * g.np + col, g.mp * g.np, g.N, Z);
    const LimbCol zc{cols + threadIdx.x};
#pragma unroll
    for (int k = 0; k < L; ++k) zc.set(k, Z[k]);
    const LimbMasks mk = limb_masks<L>(Z);
    round_components<L, P>(zc, mk, g.sig[row] + g.tau[col] - 2 * g.beta, g.C, row * g.ldc + col);
}

// Split integers: the three products hh, mid, ll of each output, each
// centred as above, combined exactly into C' = P_hh 2^(2w) + P_mid 2^w +
// P_ll in LC = 2L + 1 limbs (|C'| < M 2^(2w) <= 2^(64L)) in the thread's
// shared-memory column, and rounded to P components.
template <int P, int NB>
__global__ void __launch_bounds__(kRecThreads) crt_recover2_kernel(const __grid_constant__ CrtRecArgs g)
{
    constexpr int L = NB / 4 < crt::kRecLimbs ? NB / 4 : crt::kRecLimbs;
    constexpr int LC = 2 * L + 1;
    __shared__ uint32_t cols[LC * kRecThreads];
    const int64_t t = static_cast<int64_t>(blockIdx.x) * kRecThreads + threadIdx.x;
    if (t >= g.m * g.n) return;
    const int64_t row = t / g.n, col = t % g.n;
    const int64_t plane = g.mp * g.np;
    const int8_t* res = g.res + row * g.np + col;
    const LimbCol zc{cols + threadIdx.x};
    {   // ll, sign-extended
        uint32_t Z[L];
        crt_centred<NB, L>(g, res + 2 * static_cast<int64_t>(g.N) * plane, plane, g.N, Z);
        const uint32_t ext = (Z[L - 1] >> 31) ? ~0u : 0u;
#pragma unroll
        for (int k = 0; k < LC; ++k) zc.set(k, k < L ? Z[k] : ext);
    }
#pragma unroll
    for (int part = 1; part >= 0; --part) {            // mid (shift w), then hh (shift 2w)
        uint32_t Z[L];
        crt_centred<NB, L>(g, res + static_cast<int64_t>(part) * g.N * plane, plane, g.N, Z);
        const int shift = (2 - part) * g.w;
        const int sw = shift >> 5, sb = shift & 31;
        const uint32_t ext = (Z[L - 1] >> 31) ? ~0u : 0u;
        // column limb k + sw gains limb k of Z 2^sb (L + 1 limbs, then the sign)
        uint64_t carry = 0;
#pragma unroll
        for (int k = 0; k < LC; ++k) {
            if (k + sw < LC) {
                const uint32_t lo = k == 0 ? 0u : (k - 1 < L ? Z[k - 1] : ext);
                const uint32_t hi = k < L ? Z[k] : ext;
                const uint32_t a = __funnelshift_l(lo, hi, sb);
                const uint64_t v = static_cast<uint64_t>(zc.get(k + sw)) + a + carry;
                zc.set(k + sw, static_cast<uint32_t>(v));
                carry = v >> 32;
            }
        }
    }
    const LimbMasks mk = limb_masks<LC>(zc);
    round_components<LC, P>(zc, mk, g.sig[row] + g.tau[col] - 2 * g.beta, g.C, row * g.ldc + col);
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
// ones add into one sum.  The work is cut into (modulus, tile) items, taken
// modulus-major by the persistent CTAs in turn: the products of different
// moduli share nothing, so all SMs are busy even when the tiles are fewer
// than the SMs (64 tiles at 1024^3), and the CTAs running at the same time
// read the residue planes of the same modulus, which stay in L2.  Warp roles,
// barriers, bounded waits and the abort protocol are those of the slicing
// engine.

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
    const int per_item = NSUB * KT;                      // stages of one (modulus, tile) item
    const int ntiles = g.tiles_m * g.tiles_n;
    const int nitems = g.N * ntiles;
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
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int mi = item / ntiles, tile = item % ntiles;
                const int m0 = (tile % g.tiles_m) * tcc::BM, n0 = (tile / g.tiles_m) * tcc::BN;
                for (int i = 0; i < per_item; ++i, ++it) {
                    const int sub = i / KT, kt = i % KT;
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
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                int seg_stages = 0;
                uint32_t b = 0;
                for (int i = 0; i < per_item; ++i, ++it) {
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
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int mi = item / ntiles, tile = item % ntiles;
            const int m0 = (tile % g.tiles_m) * tcc::BM, n0 = (tile / g.tiles_m) * tcc::BN;
            int seg_stages = 0;
            bool first = true;                            // first segment of an output product
            for (int i = 0; i < per_item; ++i) {
                const int sub = i / KT, kt = i % KT;
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
    case 7: return slice_both<P, T, 7>(g, 2 * N, L, ra, rb, sig, tau, s, beta);
    case 6: return slice_both<P, T, 6>(g, 2 * N, L, ra, rb, sig, tau, s, beta);
    case 5: return slice_both<P, T, 5>(g, 2 * N, L, ra, rb, sig, tau, s, beta);
    case 4: return slice_both<P, T, 4>(g, N, L, ra, rb, sig, tau, s, beta);
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
        const int64_t items = static_cast<int64_t>(N) * a.tiles_m * a.tiles_n;
        if (items > 0x7fffffff) return cudaErrorInvalidValue;
        const int grid = items < num_sms() ? static_cast<int>(items) : num_sms();
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
    // F = floor(M / 2) = M - H
    int64_t bw = 0;
    for (int k = 0; k < crt::kRecLimbs; ++k) {
        const int64_t d = static_cast<int64_t>(ra_.M[k]) - static_cast<int64_t>(ra_.H[k]) + bw;
        ra_.F[k] = static_cast<uint32_t>(d);
        bw = d >> 32;
    }
    for (int k = 0; k < 2 * crt::kRecLimbs; ++k) ra_.M16[k] = (ra_.M[k / 2] >> (16 * (k % 2))) & 0xffffu;
    // W_i = (M / m_i) c_i with c_i the inverse of (M / m_i) mod m_i, as bytes
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
        const int grp = i / 4, sh = 8 * (i % 4);
        uint32_t Wfull[crt::kRecLimbs];
        for (int k = 0; k < crt::kRecLimbs; ++k) {
            const uint64_t v = static_cast<uint64_t>(Q[k]) * c + carry;
            const uint32_t w = static_cast<uint32_t>(v);
            Wfull[k] = w;
            carry = v >> 32;
            for (int t = 0; t < 4; ++t) ra_.Wd[grp][4 * k + t] |= ((w >> (8 * t)) & 0xffu) << sh;
        }
        const uint32_t fr = static_cast<uint32_t>((c << 24) / mi);     // floor(2^24 c / m_i) < 2^24
        for (int t = 0; t < 3; ++t) ra_.Fd[grp][t] |= ((fr >> (8 * t)) & 0xffu) << sh;
        ra_.KF += 128 * static_cast<int64_t>(fr);
        // K += 128 W_i in 16-bit limbs
        uint64_t kc = 0;
        for (int k = 0; k < 2 * crt::kRecLimbs + 1; ++k) {
            const uint32_t w16 = k / 2 < crt::kRecLimbs ? (Wfull[k / 2] >> (16 * (k % 2))) & 0xffffu : 0u;
            const uint64_t v = static_cast<uint64_t>(ra_.K16[k]) + 128ull * w16 + kc;
            ra_.K16[k] = static_cast<uint32_t>(v & 0xffffu);
            kc = v >> 16;
        }
    }
    const unsigned grid = blocks_for(g.m * g.n, kRecThreads);         // one output per thread
    if (grid == 0) return cudaSuccess;
    if (halves == 2) {
        switch ((N + 7) / 8) {
        case 1: crt_recover2_kernel<P, 8><<<grid, kRecThreads, 0, s>>>(ra_); break;
        case 2: crt_recover2_kernel<P, 16><<<grid, kRecThreads, 0, s>>>(ra_); break;
        case 3: crt_recover2_kernel<P, 24><<<grid, kRecThreads, 0, s>>>(ra_); break;
        case 4: crt_recover2_kernel<P, 32><<<grid, kRecThreads, 0, s>>>(ra_); break;
        case 5: crt_recover2_kernel<P, 40><<<grid, kRecThreads, 0, s>>>(ra_); break;
        default: crt_recover2_kernel<P, 48><<<grid, kRecThreads, 0, s>>>(ra_); break;
        }
        return cudaGetLastError();
    }
    switch ((N + 7) / 8) {
    case 1: crt_recover_kernel<P, 8><<<grid, kRecThreads, 0, s>>>(ra_); break;
    case 2: crt_recover_kernel<P, 16><<<grid, kRecThreads, 0, s>>>(ra_); break;
    case 3: crt_recover_kernel<P, 24><<<grid, kRecThreads, 0, s>>>(ra_); break;
    case 4: crt_recover_kernel<P, 32><<<grid, kRecThreads, 0, s>>>(ra_); break;
    case 5: crt_recover_kernel<P, 40><<<grid, kRecThreads, 0, s>>>(ra_); break;
    case 6: crt_recover_kernel<P, 48><<<grid, kRecThreads, 0, s>>>(ra_); break;
    default: crt_recover_kernel<P, 56><<<grid, kRecThreads, 0, s>>>(ra_); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_crt<2>(const GemmArgs<2>&, int, void*, cudaStream_t, int, int);
template cudaError_t launch_crt<3>(const GemmArgs<3>&, int, void*, cudaStream_t, int, int);
template cudaError_t launch_crt<4>(const GemmArgs<4>&, int, void*, cudaStream_t, int, int);

}  // namespace mpg
