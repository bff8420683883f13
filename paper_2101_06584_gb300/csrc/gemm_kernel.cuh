// gemm_kernel.cuh -- FP64-EFT GEMM kernels, C := op(A) op(B) (Sec. 3, Eq. 1).
//
// Both kernels are bound by arithmetic, not operand traffic: a DD
// multiply-add is 20 binary64 operations, TD 128, QD 210, against roughly two
// FP64 lanes per clock per SM on GB300.  With the operation sequences (policy
// Rn) the goal is to keep the FP64 pipe fed with independent work while
// issuing no FP64 instruction the algorithms do not need; with the policy
// RnInt<mask> the transformations in the mask run on the integer pipes beside
// it (QD: 78 of the 210 operations stay on the FP64 pipe with TwoSum moved),
// and the bound becomes the latency of those integer chains.
//
// gemm_kseq_kernel: a CTA owns a BM x BN tile of C; each thread owns TM x TN
//   entries (strided so that smem reads are broadcasts / consecutive) and
//   accumulates each one over p = 0..k-1 in order.  A and B tiles of BK
//   columns/rows are staged through shared memory for all P planes.  The
//   result is bit-identical to the k-sequential definition.
// gemm_splitk_warp_kernel: for small m*n, `S` lanes of a warp share one
//   output, each summing a contiguous k chunk in order; the partial sums are
//   combined by a butterfly of __shfl_xor_sync with the lower chunk always the
//   left operand, so every lane ends with the same, deterministic value.
#pragma once
#include "internal.h"
#include "mp_arith.cuh"

namespace mpg {

// Shared-memory staging of one k-sequential tile: all P planes of a BK-wide
// slab of A (k-major, padded) and of B.
template <int P, int BM, int BN, int BK>
struct KseqSmem {
    double As[P][BK][BM + 1];
    double Bs[P][BK][BN];
};

// One BM x BN tile of C = op(A) op(B) at (m0, n0), computed by a CTA of
// (BM/TM)*(BN/TN) threads.  Every entry is accumulated by one thread over
// p = 0..k-1 in order.  Threads none of whose entries lie inside C skip the
// arithmetic (they still take part in staging and barriers).
template <int P, int BM, int BN, int BK, int TM, int TN, class F>
__device__ __forceinline__ void kseq_tile(const GemmArgs<P>& g, int64_t m0, int64_t n0,
                                          KseqSmem<P, BM, BN, BK>& sm, const F& f)
{
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int TX = BN / TN;
    constexpr int TY = BM / TM;
    const int tid = threadIdx.x;
    const int tx = tid % TX;
    const int ty = tid / TX;
    const bool active = (m0 + ty < g.m) && (n0 + tx < g.n);

    double acc[TM][TN][P];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j)
#pragma unroll
            for (int c = 0; c < P; ++c) acc[i][j][c] = 0.0;

    for (int64_t k0 = 0; k0 < g.k; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NT) {
            int i, kk;
            if (!g.trans_a) { kk = e % BK; i = e / BK; }
            else            { i = e % BM; kk = e / BM; }
            const int64_t gi = m0 + i, gk = k0 + kk;
            const bool ok = gi < g.m && gk < g.k;
            const int64_t off = g.trans_a ? gk * g.lda + gi : gi * g.lda + gk;
#pragma unroll
            for (int c = 0; c < P; ++c) sm.As[c][kk][i] = ok ? g.A[c][off] : 0.0;
        }
        for (int e = tid; e < BK * BN; e += NT) {
            int kk, j;
            if (!g.trans_b) { j = e % BN; kk = e / BN; }
            else            { kk = e % BK; j = e / BK; }
            const int64_t gj = n0 + j, gk = k0 + kk;
            const bool ok = gj < g.n && gk < g.k;
            const int64_t off = g.trans_b ? gj * g.ldb + gk : gk * g.ldb + gj;
#pragma unroll
            for (int c = 0; c < P; ++c) sm.Bs[c][kk][j] = ok ? g.B[c][off] : 0.0;
        }
        __syncthreads();

        if (active) {
            const int kmax = static_cast<int>(g.k - k0 < BK ? g.k - k0 : BK);
#pragma unroll 1
            for (int kk = 0; kk < kmax; ++kk) {
                double a[TM][P], b[TN][P];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int c = 0; c < P; ++c) a[i][c] = sm.As[c][kk][ty + i * TY];
#pragma unroll
                for (int j = 0; j < TN; ++j)
#pragma unroll
                    for (int c = 0; c < P; ++c) b[j][c] = sm.Bs[c][kk][tx + j * TX];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) mp::mad<P>(f, acc[i][j], a[i], b[j]);
            }
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gi = m0 + ty + i * TY;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gj = n0 + tx + j * TX;
            if (gi < g.m && gj < g.n) {
#pragma unroll
                for (int c = 0; c < P; ++c) g.C[c][gi * g.ldc + gj] = acc[i][j][c];
            }
        }
    }
}

// INTS: the transformations run on the integer pipes (mp::RnInt's mask).
template <int P, int BM, int BN, int BK, int TM, int TN, unsigned INTS>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kseq_kernel(const GemmArgs<P> g)
{
    __shared__ KseqSmem<P, BM, BN, BK> sm;
    const mp::RnInt<INTS> f(mp::make_rn());
    kseq_tile<P, BM, BN, BK, TM, TN>(g, static_cast<int64_t>(blockIdx.y) * BM,
                                     static_cast<int64_t>(blockIdx.x) * BN, sm, f);
}

template <int P, int S>
__global__ void __launch_bounds__(256)
gemm_splitk_warp_kernel(const GemmArgs<P> g)
{
    constexpr int OUT_PER_WARP = 32 / S;
    const mp::Rn f = mp::make_rn();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t out = warp * OUT_PER_WARP + lane / S;
    const int part = lane % S;
    const int64_t total = g.m * g.n;
    const bool valid = out < total;
    const int64_t i = valid ? out / g.n : 0;
    const int64_t j = valid ? out % g.n : 0;

    // contiguous chunk [p0, p1) of k for this lane
    const int64_t chunk = (g.k + S - 1) / S;
    const int64_t p0 = valid ? (part * chunk < g.k ? part * chunk : g.k) : 0;
    const int64_t p1 = valid ? (p0 + chunk < g.k ? p0 + chunk : g.k) : 0;

    double acc[P];
#pragma unroll
    for (int c = 0; c < P; ++c) acc[c] = 0.0;
    for (int64_t p = p0; p < p1; ++p) {
        double a[P], b[P];
        const int64_t offa = g.trans_a ? p * g.lda + i : i * g.lda + p;
        const int64_t offb = g.trans_b ? j * g.ldb + p : p * g.ldb + j;
#pragma unroll
        for (int c = 0; c < P; ++c) {
            a[c] = g.A[c][offa];
            b[c] = g.B[c][offb];
        }
        mp::mad<P>(f, acc, a, b);
    }

    // butterfly over the S lanes of this output: at each level the lane whose
    // chunk comes first supplies the left operand, so both partners compute
    // the same sum.
#pragma unroll
    for (int off = 1; off < S; off <<= 1) {
        double other[P], lo[P], hi[P], sum[P];
#pragma unroll
        for (int c = 0; c < P; ++c) other[c] = __shfl_xor_sync(0xffffffffu, acc[c], off);
        const bool lower = (part & off) == 0;
#pragma unroll
        for (int c = 0; c < P; ++c) {
            lo[c] = lower ? acc[c] : other[c];
            hi[c] = lower ? other[c] : acc[c];
        }
        mp::Ops<P>::add(f, lo, hi, sum);
#pragma unroll
        for (int c = 0; c < P; ++c) acc[c] = sum[c];
    }
    if (valid && part == 0) {
#pragma unroll
        for (int c = 0; c < P; ++c) g.C[c][i * g.ldc + j] = acc[c];
    }
}

template <int P>
__global__ void zero_kernel(const GemmArgs<P> g)
{
    const int64_t total = g.m * g.n;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = t / g.n, j = t % g.n;
#pragma unroll
        for (int c = 0; c < P; ++c) g.C[c][i * g.ldc + j] = 0.0;
    }
}

template <int P, int BM, int BN, int BK, int TM, int TN, unsigned INTS = 0>
cudaError_t launch_kseq_cfg(const GemmArgs<P>& g, cudaStream_t s)
{
    const dim3 grid(static_cast<unsigned>((g.n + BN - 1) / BN),
                    static_cast<unsigned>((g.m + BM - 1) / BM));
    gemm_kseq_kernel<P, BM, BN, BK, TM, TN, INTS><<<grid, (BM / TM) * (BN / TN), 0, s>>>(g);
    return cudaGetLastError();
}

template <int P, int S>
cudaError_t launch_splitk_cfg(const GemmArgs<P>& g, cudaStream_t s)
{
    const int64_t outs = g.m * g.n;
    const int64_t threads = outs * S;
    const int64_t blocks = (threads + 255) / 256;
    gemm_splitk_warp_kernel<P, S><<<static_cast<unsigned>(blocks), 256, 0, s>>>(g);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_splitk_impl(const GemmArgs<P>& g, int split, cudaStream_t s)
{
    switch (split) {
    case 2: return launch_splitk_cfg<P, 2>(g, s);
    case 4: return launch_splitk_cfg<P, 4>(g, s);
    case 8: return launch_splitk_cfg<P, 8>(g, s);
    case 16: return launch_splitk_cfg<P, 16>(g, s);
    case 32: return launch_splitk_cfg<P, 32>(g, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int P>
cudaError_t launch_zero_impl(const GemmArgs<P>& g, cudaStream_t s)
{
    const int64_t total = g.m * g.n;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    zero_kernel<P><<<static_cast<unsigned>(blocks), 256, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace mpg
