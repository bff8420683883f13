// gemm_td.cu -- instantiations of the FP64-EFT GEMM kernels for P = 3.
#include "gemm_kernel.cuh"

namespace mpg {
namespace {
constexpr int P = 3;
const TileInfo kTiles[] = {
    {16, 16, 16, 1, 1, 256},
    {32, 16, 16, 2, 1, 256},
    {32, 32, 16, 2, 2, 256},
    {8, 8, 16, 1, 1, 64},
    {16, 16, 16, 1, 1, 256, 1},
    {8, 8, 16, 1, 1, 64, 1},
    {16, 8, 16, 1, 1, 128, 1},
    {16, 16, 32, 1, 1, 256, 1},
    {16, 16, 16, 1, 1, 256, 5},
};
constexpr int kNumTiles = static_cast<int>(sizeof(kTiles) / sizeof(kTiles[0]));
}  // namespace

template <>
int num_tiles<P>() { return kNumTiles; }

template <>
TileInfo tile_info<P>(int t) { return kTiles[t]; }

// 16 x 16, or 8 x 8 where 16 x 16 leaves much of the last wave's SMs idle
// (one entry per thread either way); with TwoSum on the integer pipes when
// the product has enough outputs for them (int_tiles_pay).
template <>
int default_tile<P>(int64_t m, int64_t n, int64_t)
{
    return int_tiles_pay(m, n) ? pick_tile<P>(m, n, {4, 5}) : pick_tile<P>(m, n, {0, 3});
}

template <>
cudaError_t launch_gemm_kseq<P>(const GemmArgs<P>& g, int tile, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_kseq_cfg<P, 16, 16, 16, 1, 1>(g, s);
    case 1: return launch_kseq_cfg<P, 32, 16, 16, 2, 1>(g, s);
    case 2: return launch_kseq_cfg<P, 32, 32, 16, 2, 2>(g, s);
    case 3: return launch_kseq_cfg<P, 8, 8, 16, 1, 1>(g, s);
    case 4: return launch_kseq_cfg<P, 16, 16, 16, 1, 1, 1>(g, s);
    case 5: return launch_kseq_cfg<P, 8, 8, 16, 1, 1, 1>(g, s);
    case 6: return launch_kseq_cfg<P, 16, 8, 16, 1, 1, 1>(g, s);
    case 7: return launch_kseq_cfg<P, 16, 16, 32, 1, 1, 1>(g, s);
    case 8: return launch_kseq_cfg<P, 16, 16, 16, 1, 1, 5>(g, s);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_gemm_splitk<P>(const GemmArgs<P>& g, int split, cudaStream_t s)
{
    return launch_splitk_impl<P>(g, split, s);
}

template <>
cudaError_t launch_zero<P>(const GemmArgs<P>& g, cudaStream_t s)
{
    return launch_zero_impl<P>(g, s);
}

}  // namespace mpg
