// probe.cu -- pipe throughput probes used as roofline denominators.
//
// GB300 executes binary64 add/mul/fma at roughly two lanes per clock per SM;
// this kernel measures that ceiling at the clocks of the calling run.  Each
// thread runs 8 independent chains of the chosen instruction so latency is
// hidden; the caller times the launch with events and divides the lane
// operations (blocks * 256 * iters * 8) by the elapsed time.  The operands are
// registers (read through a volatile pointer), the form the GEMM kernels use;
// DADD and DMUL issue at about 0.84x the DFMA rate on GB300.
#include "mpgemm.h"
#include "internal.h"
#include "soft_fp64.cuh"

namespace mpg {

static __device__ double probe_constants[2] = {0.9999999, 1e-7};

template <int KIND>
__global__ void __launch_bounds__(256) fp64_probe_kernel(int iters, double* out)
{
    const volatile double* pc = probe_constants;
    const double a = pc[0], b = pc[1];
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if constexpr (KIND == 0) x[j] = __dadd_rn(x[j], b);
            else if constexpr (KIND == 1) x[j] = __dmul_rn(x[j], a);
            else x[j] = __fma_rn(x[j], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s = __dadd_rn(s, x[j]);
    out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

// The int8 tensor-pipe rate of the warp-level MMA the INT8 slicing form
// uses: each warp issues `iters` rounds of 4 independent
// mma.sync.m16n8k32.s8 (8192 int8 operations each).
__global__ void __launch_bounds__(256) mma_s8_probe_kernel(int iters, double* out)
{
    const volatile double* pc = probe_constants;
    unsigned a0 = threadIdx.x + static_cast<unsigned>(pc[0] > 2.0), a1 = a0 * 3u, a2 = a0 * 5u,
             a3 = a0 * 7u, b0 = a0 * 11u, b1 = a0 * 13u;
    int d[4][4] = {};
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                "{%8,%9}, {%0,%1,%2,%3};\n"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
    int s = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) s += d[c][j];
    out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = static_cast<double>(s);
}

// The integer-pipe rates of the transformations as RnInt computes them
// (soft_fp64.cuh): each thread runs 4 independent chains of TwoSum (KIND 4),
// FastTwoSum (5) or TwoProd (6); every error term is folded into a running
// XOR so none is dead.  Transformations = blocks*256*iters*4.
template <int KIND>
__global__ void __launch_bounds__(256) int_eft_probe_kernel(int iters, double* out)
{
    const volatile double* pc = probe_constants;
    const double a = pc[0], b = pc[1];
    double x[4];
    long long acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = 1.0 + threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            mp::soft::Pair r;
            if constexpr (KIND == 4) r = mp::soft::two_sum<false>(x[j], b);
            else if constexpr (KIND == 5) r = mp::soft::two_sum<true>(x[j], b);
            else r = mp::soft::two_prod(x[j], a);
            x[j] = r.hi;
            acc ^= __double_as_longlong(r.lo);
        }
    }
    double s = __longlong_as_double(acc & 0x3fffffffffffffffll);
#pragma unroll
    for (int j = 0; j < 4; ++j) s = __dadd_rn(s, x[j]);
    out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

}  // namespace mpg

extern "C" int mpgemm_peak_probe(int kind, int blocks, int iters, double* out)
{
    using namespace mpg;
    if (kind < 0 || kind > 6 || blocks < 1 || iters < 1 || !out)
        return set_error(MPG_EINVAL, "mpgemm_peak_probe: kind 0..6, blocks >= 1, iters >= 1, out non-NULL");
    clear_error();
    cudaStream_t s = current_stream();
    switch (kind) {
    case 0: fp64_probe_kernel<0><<<blocks, 256, 0, s>>>(iters, out); break;
    case 1: fp64_probe_kernel<1><<<blocks, 256, 0, s>>>(iters, out); break;
    case 2: fp64_probe_kernel<2><<<blocks, 256, 0, s>>>(iters, out); break;
    case 3: mma_s8_probe_kernel<<<blocks, 256, 0, s>>>(iters, out); break;
    case 4: int_eft_probe_kernel<4><<<blocks, 256, 0, s>>>(iters, out); break;
    case 5: int_eft_probe_kernel<5><<<blocks, 256, 0, s>>>(iters, out); break;
    default: int_eft_probe_kernel<6><<<blocks, 256, 0, s>>>(iters, out); break;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPG_OK : set_error(MPG_ECUDA, cudaGetErrorString(e));
}
