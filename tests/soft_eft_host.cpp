// Host build of the integer-pipe error-free transformations, for the CPU
// tests: the device header compiled as plain C++, with the CUDA bit-cast,
// count and high-multiply intrinsics it uses written out for the host and
// its rare-input sequences on the host's IEEE binary64 operations.  Built
// with -ffp-contract=off so every operation rounds once.
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

#include "soft_fp64.cuh"

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
