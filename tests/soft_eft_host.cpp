// Host build of the device arithmetic, for the CPU tests: soft_fp64.cuh
// (the integer-pipe error-free transformations) and mp_arith.cuh (the
// DD/TD/QD operations under each arithmetic policy) compiled as plain C++,
// with the CUDA bit-cast, count and high-multiply intrinsics they use written
// out for the host and their binary64 operations on the host's IEEE
// arithmetic.  Built with -ffp-contract=off so every operation rounds once.
#include <cmath>
#include <cstdint>
#include <cstring>

#define __device__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))

static inline int __double2hiint(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return static_cast<int>(static_cast<uint32_t>(b >> 32));
}
static inline int __double2loint(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return static_cast<int>(static_cast<uint32_t>(b));
}
static inline double __hiloint2double(int hi, int lo)
{
    const uint64_t b = (static_cast<uint64_t>(static_cast<uint32_t>(hi)) << 32) | static_cast<uint32_t>(lo);
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}
static inline long long __double_as_longlong(double x)
{
    long long b;
    std::memcpy(&b, &x, 8);
    return b;
}
static inline double __longlong_as_double(long long b)
{
    double d;
    std::memcpy(&d, &b, 8);
    return d;
}
static inline int __clzll(long long x)
{
    return x == 0 ? 64 : __builtin_clzll(static_cast<unsigned long long>(x));
}
static inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b)
{
    return static_cast<unsigned long long>((static_cast<unsigned __int128>(a) * b) >> 64);
}
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }

struct HostThreadIdx {
    unsigned x;
};
static const HostThreadIdx threadIdx = {0u};

#include "mp_arith.cuh"

// which: 0 QuickTwoSum, 1 TwoSum, 2 TwoProd, elementwise over n pairs.
extern "C" void soft_eft_host(int which, long n, const double* a, const double* b, double* s, double* e)
{
    for (long i = 0; i < n; ++i) {
        const mp::soft::Pair r = which == 0   ? mp::soft::two_sum<true>(a[i], b[i])
                                 : which == 1 ? mp::soft::two_sum<false>(a[i], b[i])
                                              : mp::soft::two_prod(a[i], b[i]);
        s[i] = r.hi;
        e[i] = r.lo;
    }
}

// acc := add(acc, mul(a, b)), the GEMM's multiply-add of precision P, on
// n AoS values (P doubles each), with the transformations in `mask` computed
// on the integer pipes (mp::RnInt<mask>; 0 = the operation sequences).
template <int P, unsigned MASK>
static void mad_n(long n, double* acc, const double* a, const double* b)
{
    const mp::RnInt<MASK> f(mp::make_rn());
    for (long i = 0; i < n; ++i) mp::mad<P>(f, acc + P * i, a + P * i, b + P * i);
}

template <int P>
static void mad_mask(unsigned mask, long n, double* acc, const double* a, const double* b)
{
    switch (mask) {
    case 0: mad_n<P, 0>(n, acc, a, b); break;
    case 1: mad_n<P, 1>(n, acc, a, b); break;
    case 2: mad_n<P, 2>(n, acc, a, b); break;
    case 3: mad_n<P, 3>(n, acc, a, b); break;
    case 4: mad_n<P, 4>(n, acc, a, b); break;
    case 5: mad_n<P, 5>(n, acc, a, b); break;
    case 6: mad_n<P, 6>(n, acc, a, b); break;
    default: mad_n<P, 7>(n, acc, a, b); break;
    }
}

extern "C" void mad_host(int P, unsigned mask, long n, double* acc, const double* a, const double* b)
{
    if (P == 2) mad_mask<2>(mask, n, acc, a, b);
    else if (P == 3) mad_mask<3>(mask, n, acc, a, b);
    else mad_mask<4>(mask, n, acc, a, b);
}
