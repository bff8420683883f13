// elementwise.cu -- elementwise EFTs and DD/TD/QD add/mul over SoA vectors
// (Sec. 2.1-2.5), with the TD/QD variants of Sec. 2.3-2.4.  Each element is independent; a grid-stride loop with one
// element per thread per iteration keeps loads coalesced per plane.  Every
// kernel here is FP64-bound on GB300 (e.g. a DD add is 11 FP64 operations for
// 48 bytes of traffic), so there is no staging.
#include "internal.h"
#include "mp_arith.cuh"

namespace mpg {

template <int P>
struct VecArgs {
    const double* x[P];
    const double* y[P];
    double* r[P];
    int64_t n;
};

template <int P, int OP>
__global__ void __launch_bounds__(256) vec_kernel(const VecArgs<P> a)
{
    const mp::Rn f = mp::make_rn();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n;
         i += stride) {
        double x[P], y[P], r[P];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            x[c] = a.x[c][i];
            y[c] = a.y[c][i];
        }
        if constexpr (OP == 0) {
            mp::Ops<P>::add(f, x, y, r);
        } else if constexpr (OP == 1) {
            mp::Ops<P>::mul(f, x, y, r);
        } else if constexpr (OP == 2) {
            static_assert(P == 3, "merge-based add is the TD addition of Alg. 3");
            mp::td_add_merge(f, x, y, r);
        } else if constexpr (OP == 3) {
            static_assert(P == 3, "TDmulq is a TD product");
            mp::td_mulq(f, x, y, r);
        } else if constexpr (OP == 4) {
            static_assert(P == 3, "the accurate product is a TD product");
            mp::td_mul_acc(f, x, y, r);
        } else {
            static_assert(P == 4, "the accurate addition is a QD addition");
            mp::qd_add_acc(f, x, y, r);
        }
#pragma unroll
        for (int c = 0; c < P; ++c) a.r[c][i] = r[c];
    }
}

// DD add / mul with four adjacent elements per thread and iteration: each of
// the four operand planes is read as two double2 (16-byte loads, 32 bytes per
// thread, 1 KB contiguous per warp and plane) and all four elements' loads
// are issued before any result is stored, so each thread keeps four times the
// bytes in flight.  A DD operation is only 9-11 FP64 operations per 48 bytes,
// the least work per byte of all the elementwise operations, and one element
// per thread leaves the FP64 pipe waiting on memory.  Requires 16-byte aligned
// planes (checked by the host); the last n mod 4 elements are done by one
// thread with scalar loads.
template <int OP>
__global__ void __launch_bounds__(256) vec_dd_x4_kernel(const VecArgs<2> a)
{
    const mp::Rn f = mp::make_rn();
    const int64_t quads = a.n >> 2;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const double2* x0 = reinterpret_cast<const double2*>(a.x[0]);
    const double2* x1 = reinterpret_cast<const double2*>(a.x[1]);
    const double2* y0 = reinterpret_cast<const double2*>(a.y[0]);
    const double2* y1 = reinterpret_cast<const double2*>(a.y[1]);
    double2* r0 = reinterpret_cast<double2*>(a.r[0]);
    double2* r1 = reinterpret_cast<double2*>(a.r[1]);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < quads; i += stride) {
        double2 u0[2], u1[2], v0[2], v1[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            u0[h] = x0[2 * i + h];
            u1[h] = x1[2 * i + h];
            v0[h] = y0[2 * i + h];
            v1[h] = y1[2 * i + h];
        }
        double o0[4], o1[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int h = e >> 1;
            const bool hi = e & 1;
            double x[2] = {hi ? u0[h].y : u0[h].x, hi ? u1[h].y : u1[h].x};
            double y[2] = {hi ? v0[h].y : v0[h].x, hi ? v1[h].y : v1[h].x};
            double r[2];
            if constexpr (OP == 0) mp::dd_add(f, x, y, r);
            else mp::dd_mul(f, x, y, r);
            o0[e] = r[0];
            o1[e] = r[1];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            r0[2 * i + h] = make_double2(o0[2 * h], o0[2 * h + 1]);
            r1[2 * i + h] = make_double2(o1[2 * h], o1[2 * h + 1]);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int64_t t = quads * 4; t < a.n; ++t) {
            double x[2] = {a.x[0][t], a.x[1][t]}, y[2] = {a.y[0][t], a.y[1][t]}, r[2];
            if constexpr (OP == 0) mp::dd_add(f, x, y, r);
            else mp::dd_mul(f, x, y, r);
            a.r[0][t] = r[0];
            a.r[1][t] = r[1];
        }
    }
}

// INTS: 0 for the operation sequences on the FP64 pipe, 7 for the integer-pipe
// form of all three transformations (mp::RnInt).
template <int W, unsigned INTS>
__global__ void __launch_bounds__(256)
eft_kernel(int64_t n, const double* a, const double* b, double* s,
           double* e)
{
    const mp::RnInt<INTS> f(mp::make_rn());
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        double hi, lo;
        if constexpr (W == 0) mp::quick_two_sum(f, a[i], b[i], hi, lo);
        else if constexpr (W == 1) mp::two_sum(f, a[i], b[i], hi, lo);
        else mp::two_prod(f, a[i], b[i], hi, lo);
        s[i] = hi;
        e[i] = lo;
    }
}

// Grid of a grid-stride kernel: enough blocks for n items of 256 threads,
// at most the blocks that are resident on all SMs at once (from the
// kernel's occupancy, looked up once per kernel), so every block stays
// resident to the end and no second, partial wave leaves SM sub-partitions
// without warps.  Each elementwise op is FP64-bound, and the FP64 pipe of a
// sub-partition idles when it has no warp ready.
template <typename K>
static unsigned grid_for(K kernel, int64_t n)
{
    static int per_sm = 0;                 // one cache per kernel instantiation
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b < 1) b = 1;
        per_sm = b;
    }
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = static_cast<int64_t>(num_sms()) * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return static_cast<unsigned>(blocks);
}

template <int P>
cudaError_t launch_vec(int op, int64_t n, const double* const* x, const double* const* y,
                       double* const* r, cudaStream_t s)
{
    VecArgs<P> a;
    for (int c = 0; c < P; ++c) {
        a.x[c] = x[c];
        a.y[c] = y[c];
        a.r[c] = r[c];
    }
    a.n = n;
    if constexpr (P == 2) {
        bool aligned = true;
        for (int c = 0; c < P; ++c)
            aligned = aligned && (reinterpret_cast<uintptr_t>(x[c]) | reinterpret_cast<uintptr_t>(y[c]) |
                                  reinterpret_cast<uintptr_t>(r[c])) % 16 == 0;
        if (aligned && (op == 0 || op == 1)) {
            const int64_t q = n / 4 > 0 ? n / 4 : 1;
            if (op == 0) vec_dd_x4_kernel<0><<<grid_for(vec_dd_x4_kernel<0>, q), 256, 0, s>>>(a);
            else vec_dd_x4_kernel<1><<<grid_for(vec_dd_x4_kernel<1>, q), 256, 0, s>>>(a);
            return cudaGetLastError();
        }
    }
    // op codes: 0 add, 1 mul (the GEMM's pair for P); 2 TDadd (Alg. 3),
    // 3 TDmulq, 4 accurate TD product; 5 accurate QD addition
    if (op == 0) vec_kernel<P, 0><<<grid_for(vec_kernel<P, 0>, n), 256, 0, s>>>(a);
    else if (op == 1) vec_kernel<P, 1><<<grid_for(vec_kernel<P, 1>, n), 256, 0, s>>>(a);
    else if constexpr (P == 3) {
        if (op == 2) vec_kernel<P, 2><<<grid_for(vec_kernel<P, 2>, n), 256, 0, s>>>(a);
        else if (op == 3) vec_kernel<P, 3><<<grid_for(vec_kernel<P, 3>, n), 256, 0, s>>>(a);
        else if (op == 4) vec_kernel<P, 4><<<grid_for(vec_kernel<P, 4>, n), 256, 0, s>>>(a);
        else return cudaErrorInvalidValue;
    } else if constexpr (P == 4) {
        if (op == 5) vec_kernel<P, 5><<<grid_for(vec_kernel<P, 5>, n), 256, 0, s>>>(a);
        else return cudaErrorInvalidValue;
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_vec<2>(int, int64_t, const double* const*, const double* const*,
                                   double* const*, cudaStream_t);
template cudaError_t launch_vec<3>(int, int64_t, const double* const*, const double* const*,
                                   double* const*, cudaStream_t);
template cudaError_t launch_vec<4>(int, int64_t, const double* const*, const double* const*,
                                   double* const*, cudaStream_t);

template <unsigned INTS>
static cudaError_t launch_eft_form(int which, int64_t n, const double* a, const double* b, double* s, double* e,
                                   cudaStream_t st)
{
    switch (which) {
    case 0: eft_kernel<0, INTS><<<grid_for(eft_kernel<0, INTS>, n), 256, 0, st>>>(n, a, b, s, e); break;
    case 1: eft_kernel<1, INTS><<<grid_for(eft_kernel<1, INTS>, n), 256, 0, st>>>(n, a, b, s, e); break;
    case 2: eft_kernel<2, INTS><<<grid_for(eft_kernel<2, INTS>, n), 256, 0, st>>>(n, a, b, s, e); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_eft(int which, bool int_pipes, int64_t n, const double* a, const double* b, double* s,
                       double* e, cudaStream_t st)
{
    return int_pipes ? launch_eft_form<7>(which, n, a, b, s, e, st) : launch_eft_form<0>(which, n, a, b, s, e, st);
}

}  // namespace mpg
