// gemm_dd.cu -- instantiations of the FP64-EFT GEMM kernels for P = 2.
#include "gemm_kernel.cuh"

namespace mpg {
namespace {
constexpr int P = 2;
const TileInfo kTiles[] = {
    {32, 32, 16, 2, 2, 256},
    {16, 16, 16, 1, 1, 256},
    {32, 16, 16, 2, 1, 256},
    {64, 32, 16, 2, 2, 512},
    {64, 64, 16, 4, 4, 256},
    {8, 8, 16, 1, 1, 64},
    {8, 8, 128, 1, 1, 64},
    {32, 32, 16, 2, 2, 256, 3},
    {16, 16, 16, 1, 1, 256, 7},
    {8, 8, 16, 1, 1, 64, 3},
    {16, 16, 16, 1, 1, 256, 3},
    {32, 32, 16, 2, 2, 256, 7},
    {8, 8, 128, 1, 1, 64, 3},
};
constexpr int kNumTiles = static_cast<int>(sizeof(kTiles) / sizeof(kTiles[0]));
}  // namespace

template <>
int num_tiles<P>() { return kNumTiles; }

template <>
TileInfo tile_info<P>(int t) { return kTiles[t]; }

// 32 x 32, 16 x 16 or 8 x 8 (one entry per thread), by the last wave's
// occupancy.  One warp per SM sub-partition already keeps its FP64 pipe busy,
// so small tiles trade nothing but staging for the idle SMs they fill.  The
// 8 x 8 tile stages 128 values of k at a time (34 KB of shared memory): a
// 128^3 product is then one load and one barrier per CTA instead of eight,
// 94 -> 90 us back to back and 108 -> 95 us after an L2 flush on GB300.
//
// With enough outputs (int_tiles_pay) the 16 x 16 or 8 x 8 tiles that run
// TwoSum and FastTwoSum on the integer pipes: 19.7 ms at 1024^3 against
// 34.4 ms for the best FP64-pipe tile.
template <>
int default_tile<P>(int64_t m, int64_t n, int64_t)
{
    return int_tiles_pay(m, n) ? pick_tile<P>(m, n, {10, 9}) : pick_tile<P>(m, n, {0, 1, 6});
}

template <>
cudaError_t launch_gemm_kseq<P>(const GemmArgs<P>& g, int tile, cudaStream_t s)
{
    switch (tile) {
    case 0: return launch_kseq_cfg<P, 32, 32, 16, 2, 2>(g, s);
    case 1: return launch_kseq_cfg<P, 16, 16, 16, 1, 1>(g, s);
    case 2: return launch_kseq_cfg<P, 32, 16, 16, 2, 1>(g, s);
    case 3: return launch_kseq_cfg<P, 64, 32, 16, 2, 2>(g, s);
    case 4: return launch_kseq_cfg<P, 64, 64, 16, 4, 4>(g, s);
    case 5: return launch_kseq_cfg<P, 8, 8, 16, 1, 1>(g, s);
    case 6: return launch_kseq_cfg<P, 8, 8, 128, 1, 1>(g, s);
    case 7: return launch_kseq_cfg<P, 32, 32, 16, 2, 2, 3>(g, s);
    case 8: return launch_kseq_cfg<P, 16, 16, 16, 1, 1, 7>(g, s);
    case 9: return launch_kseq_cfg<P, 8, 8, 16, 1, 1, 3>(g, s);
    case 10: return launch_kseq_cfg<P, 16, 16, 16, 1, 1, 3>(g, s);
    case 11: return launch_kseq_cfg<P, 32, 32, 16, 2, 2, 7>(g, s);
    case 12: return launch_kseq_cfg<P, 8, 8, 128, 1, 1, 3>(g, s);
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
