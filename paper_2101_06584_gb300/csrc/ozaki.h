// ozaki.h -- host-side interface of the INT8 error-free slicing DD GEMM.
#pragma once
#include "internal.h"

namespace mpg {

constexpr int kOzakiMaxSlices = 16;       // DD: 128-bit exact fixed point
constexpr int kOzakiMaxSlicesWide = 40;   // TD, QD: 384-bit floored fixed point
constexpr int kOzakiDefaultSlices = 14;
// Weights combined exactly per add: DD 5 (sums below 2^60, 64-bit integers),
// TD 11 (below 2^102) and QD 10 (below 2^95) in 128-bit integers.  Eleven TD
// weights make the default 22 slices two groups.
constexpr int ozaki_group(int P) { return P == 2 ? 5 : P == 3 ? 11 : 10; }

// Workspace layout for S slices of an m x n x k product (byte offsets).
struct OzakiLayout {
    int S;
    int64_t mp, np, kp;
    int64_t offA, offB, offSig, offTau, offScr, total;
};
// elem_bytes: 1 for int8 digits, 2 for bf16 digits
OzakiLayout ozaki_layout(int S, int64_t m, int64_t n, int64_t k, int elem_bytes = 1);
// Workspace of the tcgen05 engine: a 256-byte header (int32 error code of the
// last call: 0, or the role whose bounded wait expired), bf16 slices with rows
// of op(A) padded to 256 (DD) or 128 and columns of op(B) to 128 (DD) or 64,
// exponents, and for DD two 128 x 128 buffers of 64-bit group sums per SM.
OzakiLayout ozaki_tc_layout(int P, int S, int64_t m, int64_t n, int64_t k);

// Largest k for which the int32 weight sums are exact: S * k * 64 * 64 < 2^31.
inline int64_t ozaki_k_limit(int S) { return (2147483647LL) / (static_cast<int64_t>(S) * 64 * 64); }

// engine 0: int8 digits on mma.sync s8 (for DD, variant 0..2 selects the CTA
// tiling, 0 the default); engine 1: bf16 digits on tcgen05 (TMEM accumulators).
template <int P>
cudaError_t launch_ozaki(const GemmArgs<P>& g, int S, void* ws, cudaStream_t s, int variant = 0,
                         int engine = 0);

// The CRT form (Ozaki scheme II): N moduli (pairwise coprime, <= 256, at most
// kCrtMaxModuli), beta bits per scaled entry.  Workspace: residues of op(A)
// [N][mp][kp] and of op(B)^T [N][np][kp] (int8; mp, np rounded up to 128, kp
// to 128), int32 exponents, and the products' residues [N][mp][np] (int8).
// halves = 2 (split integers, A' = A1 2^w + A0): [2N] residue planes per
// operand (A1's, then A0's) and [3N] product planes (hh, mid, ll).
constexpr int kCrtMaxModuli = 49;
inline int64_t crt_k_limit(int halves = 1) { return (2147483647LL) / (halves * 128 * 128); }
// The most bits a scaled entry may keep: 192 for one integer (three 64-bit
// residue cursors' worth), 316 with split integers (the 384-bit sum of the
// floored components with its 64 guard bits).
inline int crt_max_beta(int halves) { return halves == 2 ? 316 : 192; }
// engine 0: int8 residues (mma.sync); engine 1: bf16 residues after a 256-byte
// header (tcgen05).
OzakiLayout crt_layout(int N, int64_t m, int64_t n, int64_t k, int engine = 0, int halves = 1);
// The largest beta with k 2^(2 beta - 1) < m_0 ... m_(N-1) (halves = 2:
// beta = 2w for the largest w with k 2^(2w) < m_0 ... m_(N-1)); -1 for a bad
// N or halves.
int crt_beta(int N, int64_t k, int halves = 1);
template <int P>
cudaError_t launch_crt(const GemmArgs<P>& g, int N, void* ws, cudaStream_t s, int engine = 0, int halves = 1);

// Size of the library's fixed scratch array and its device address on the
// current device (looked up on first use per device).
constexpr int64_t kOzakiStaticScratchBytes = 32LL << 20;
cudaError_t ozaki_static_scratch(void** out);

}  // namespace mpg
