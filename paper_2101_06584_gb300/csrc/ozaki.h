// ozaki.h -- host-side interface of the INT8 error-free slicing DD GEMM.
#pragma once
#include "internal.h"

namespace mpg {

constexpr int kOzakiMaxSlices = 16;
constexpr int kOzakiDefaultSlices = 14;

// Workspace layout for S slices of an m x n x k product (byte offsets).
struct OzakiLayout {
    int S;
    int64_t mp, np, kp;
    int64_t offA, offB, offSig, offTau, total;
};
OzakiLayout ozaki_layout(int S, int64_t m, int64_t n, int64_t k);

// Largest k for which the int32 weight sums are exact: S * k * 64 * 64 < 2^31.
inline int64_t ozaki_k_limit(int S) { return (2147483647LL) / (static_cast<int64_t>(S) * 64 * 64); }

// variant 0..4: CTA tilings of the slice-product kernel (0 is the default)
cudaError_t launch_ozaki_dd(const GemmArgs<2>& g, int S, void* ws, cudaStream_t s, int variant = 0);

// Size of the library's fixed scratch array and its device address on the
// current device (looked up on first use per device).
constexpr int64_t kOzakiStaticScratchBytes = 32LL << 20;
cudaError_t ozaki_static_scratch(void** out);

}  // namespace mpg
