// gemm_d.cu -- the binary64-only GEMM (P = 1): C := A B with every c_ij
// accumulated in order p = 0..k-1 as acc = fma(a_ip, b_pj, acc) from acc = +0.
// It is the plain FP64 product against which the DD/TD/QD forms' accuracy is
// reported (the paper's problem, Sec. 3, Eq. 1, in binary64 alone; Sec. 3
// remarks on the decimal digits its own test products lose).  Same k-sequential
// kernel as the multi-component precisions, one DFMA per multiply-add.
#include "gemm_kernel.cuh"

namespace mpg {
namespace {
constexpr int P = 1;
const TileInfo kTiles[] = {
    {64, 64, 16, 4, 4, 256},
    {32, 32, 16, 2, 2, 256},
    {16, 16, 16, 1, 1, 256},
    {8, 8, 16, 1, 1, 64},
};
constexpr int kNumTiles = static_cast<int>(sizeof(kTiles) / sizeof(kTiles[0]));
}  // namespace

template <>
int num_tiles<P>() { return kNumTiles; }

template <>
TileInfo tile_info<P>(int t) { return kTiles[t]; }

// The largest tile whose last wave keeps the SMs busy: a 4 x 4 register block
// feeds 16 DFMAs from 8 shared-memory loads, 1 x 1 one from two.
template <>
int default_tile<P>(int64_t m, int64_t n, int64_t)
{
    return pick_tile<P>(m, n, {0, 1, 2, 3});
}

template <>
cudaError_t launch_gemm_kseq<P>(const GemmArgs<P>& g, int tile, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_kseq_cfg<P, 64, 64, 16, 4, 4>(g, s);
    case 1: return launch_kseq_cfg<P, 32, 32, 16, 2, 2>(g, s);
    case 2: return launch_kseq_cfg<P, 16, 16, 16, 1, 1>(g, s);
    case 3: return launch_kseq_cfg<P, 8, 8, 16, 1, 1>(g, s);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_gemm_splitk<P>(const GemmArgs<P>&, int, cudaStream_t)
{
    return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_zero<P>(const GemmArgs<P>& g, cudaStream_t s)
{
    return launch_zero_impl<P>(g, s);
}

}  // namespace mpg
