// abi.cu -- the extern "C" entry points of include/mpgemm.h: argument
// validation on the host (no launch on a bad argument), dispatch to the
// kernels on the calling thread's stream, and error reporting.
#include "mpgemm.h"
#include "internal.h"
#include "ozaki.h"

#include <cstdarg>
#include <cstdio>
#include <cstring>

namespace mpg {

namespace {
thread_local char g_err[512] = "";
thread_local cudaStream_t g_stream = nullptr;

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    return fail(MPG_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Byte range [lo, hi) touched by a rows x cols plane with leading dimension ld.
struct Range {
    uintptr_t lo, hi;
};
Range plane_range(const void* p, int64_t rows, int64_t cols, int64_t ld)
{
    if (!p || rows <= 0 || cols <= 0) return {0, 0};
    const uintptr_t lo = reinterpret_cast<uintptr_t>(p);
    const uint64_t elems = static_cast<uint64_t>(rows - 1) * static_cast<uint64_t>(ld) +
                           static_cast<uint64_t>(cols);
    return {lo, lo + elems * sizeof(double)};
}
bool overlap(Range a, Range b)
{
    return a.lo < a.hi && b.lo < b.hi && a.lo < b.hi && b.lo < a.hi;
}
}  // namespace

int num_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        cache[dev] = v;
    }
    return cache[dev];
}

cudaStream_t current_stream() { return g_stream; }
void clear_error() { g_err[0] = '\0'; }
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

// ------------------------------------------------------------ validation

static int check_vec(int P, int64_t n, const double* const* x, const double* const* y,
                     double* const* r)
{
    if (n < 0) return fail(MPG_EINVAL, "n must be >= 0 (got %lld)", (long long)n);
    if (n == 0) return MPG_OK;
    if (!x || !y || !r) return fail(MPG_EINVAL, "plane pointer arrays must not be NULL");
    for (int c = 0; c < P; ++c)
        if (!x[c] || !y[c] || !r[c])
            return fail(MPG_EINVAL, "component plane %d is NULL", c);
    for (int c = 0; c < P; ++c) {
        const Range rc = plane_range(r[c], 1, n, n);
        for (int d = 0; d < P; ++d) {
            if (d != c && overlap(rc, plane_range(r[d], 1, n, n)))
                return fail(MPG_EINVAL, "output planes %d and %d overlap", c, d);
            for (const double* in : {x[d], y[d]}) {
                const Range ri = plane_range(in, 1, n, n);
                const bool same = (d == c && in == r[c]);
                if (!same && overlap(rc, ri))
                    return fail(MPG_EINVAL, "output plane %d partially overlaps an input plane", c);
            }
        }
    }
    return MPG_OK;
}

template <int P>
static int vec_call(int op, int64_t n, const double* const* x, const double* const* y,
                    double* const* r)
{
    clear_error();
    int rc = check_vec(P, n, x, y, r);
    if (rc != MPG_OK || n == 0) return rc;
    cudaError_t e = launch_vec<P>(op, n, x, y, r, g_stream);
    return e == cudaSuccess ? MPG_OK : cuda_fail(e, "elementwise launch");
}

static int eft_call(int which, bool int_pipes, int64_t n, const double* a, const double* b, double* s, double* e)
{
    clear_error();
    if (which < 0 || which > 2) return fail(MPG_EINVAL, "which must be 0, 1 or 2 (got %d)", which);
    if (n < 0) return fail(MPG_EINVAL, "n must be >= 0 (got %lld)", (long long)n);
    if (n == 0) return MPG_OK;
    if (!a || !b || !s || !e) return fail(MPG_EINVAL, "NULL pointer with n > 0");
    const Range rs = plane_range(s, 1, n, n), re = plane_range(e, 1, n, n);
    if (overlap(rs, re)) return fail(MPG_EINVAL, "s and e overlap");
    for (const double* in : {a, b}) {
        const Range ri = plane_range(in, 1, n, n);
        if ((overlap(rs, ri) && in != s) || (overlap(re, ri) && in != e))
            return fail(MPG_EINVAL, "an output partially overlaps an input");
    }
    cudaError_t err = launch_eft(which, int_pipes, n, a, b, s, e, g_stream);
    return err == cudaSuccess ? MPG_OK : cuda_fail(err, "eft launch");
}

template <int P>
int check_gemm(const GemmArgs<P>& g)
{
    if (g.m < 0 || g.n < 0 || g.k < 0)
        return fail(MPG_EINVAL, "m, n, k must be >= 0 (got %lld, %lld, %lld)", (long long)g.m,
                    (long long)g.n, (long long)g.k);
    // stored shapes of A and B
    const int64_t ar = g.trans_a ? g.k : g.m, ac = g.trans_a ? g.m : g.k;
    const int64_t br = g.trans_b ? g.n : g.k, bc = g.trans_b ? g.k : g.n;
    const int64_t one = 1;
    if (g.lda < (ac > one ? ac : one))
        return fail(MPG_EINVAL, "lda (%lld) must be >= max(1, %lld)", (long long)g.lda, (long long)ac);
    if (g.ldb < (bc > one ? bc : one))
        return fail(MPG_EINVAL, "ldb (%lld) must be >= max(1, %lld)", (long long)g.ldb, (long long)bc);
    if (g.ldc < (g.n > one ? g.n : one))
        return fail(MPG_EINVAL, "ldc (%lld) must be >= max(1, %lld)", (long long)g.ldc, (long long)g.n);
    const bool needA = g.m > 0 && g.k > 0 && g.n > 0;
    const bool needB = needA;
    const bool needC = g.m > 0 && g.n > 0;
    for (int c = 0; c < P; ++c) {
        if (needA && !g.A[c]) return fail(MPG_EINVAL, "A plane %d is NULL", c);
        if (needB && !g.B[c]) return fail(MPG_EINVAL, "B plane %d is NULL", c);
        if (needC && !g.C[c]) return fail(MPG_EINVAL, "C plane %d is NULL", c);
    }
    if (!needC) return MPG_OK;
    for (int c = 0; c < P; ++c) {
        const Range rc = plane_range(g.C[c], g.m, g.n, g.ldc);
        for (int d = 0; d < P; ++d) {
            if (d != c && overlap(rc, plane_range(g.C[d], g.m, g.n, g.ldc)))
                return fail(MPG_EINVAL, "C planes %d and %d overlap", c, d);
            if (needA && overlap(rc, plane_range(g.A[d], ar, ac, g.lda)))
                return fail(MPG_EINVAL, "C plane %d overlaps A plane %d", c, d);
            if (needB && overlap(rc, plane_range(g.B[d], br, bc, g.ldb)))
                return fail(MPG_EINVAL, "C plane %d overlaps B plane %d", c, d);
        }
    }
    return MPG_OK;
}

template int check_gemm<1>(const GemmArgs<1>&);
template int check_gemm<2>(const GemmArgs<2>&);
template int check_gemm<3>(const GemmArgs<3>&);
template int check_gemm<4>(const GemmArgs<4>&);

constexpr int kMaxStrassenLevels = 8;

// Slice-count limits and defaults per precision.
static int ozaki_max_slices(int P) { return P == 2 ? kOzakiMaxSlices : kOzakiMaxSlicesWide; }
static int ozaki_default_slices(int P) { return P == 2 ? kOzakiDefaultSlices : P == 3 ? 22 : 29; }

template <int P>
static int ozaki_call(const GemmArgs<P>& g, const mpgemm_opts* o)
{
    const int engine = o->algo == MPG_ALGO_BF16_SLICES ? 1 : 0;
    const int S = o->slices ? o->slices : ozaki_default_slices(P);
    if (S < 1 || S > ozaki_max_slices(P))
        return fail(MPG_EINVAL, "slices must be in 1..%d for P = %d (got %d)", ozaki_max_slices(P), P, S);
    if (g.k > ozaki_k_limit(S))
        return fail(MPG_EUNSUPPORTED, "k = %lld exceeds %lld, the largest k whose %d-slice int32 "
                    "sums are exact", (long long)g.k, (long long)ozaki_k_limit(S), S);
    const OzakiLayout L = engine == 1 ? ozaki_tc_layout(P, S, g.m, g.n, g.k) : ozaki_layout(S, g.m, g.n, g.k, 1);
    if (L.mp / 64 > 65535) return fail(MPG_EINVAL, "m too large for the slicing form's grid");
    if (!o->workspace) return fail(MPG_EWORKSPACE, "the slicing form needs a workspace of %lld bytes",
                                   (long long)L.total);
    if (reinterpret_cast<uintptr_t>(o->workspace) % 256)
        return fail(MPG_EWORKSPACE, "workspace must be 256-byte aligned");
    if (o->workspace_bytes < static_cast<size_t>(L.total))
        return fail(MPG_EWORKSPACE, "workspace of %zu bytes is smaller than the %lld needed",
                    o->workspace_bytes, (long long)L.total);
    const Range rw{reinterpret_cast<uintptr_t>(o->workspace),
                   reinterpret_cast<uintptr_t>(o->workspace) + static_cast<uintptr_t>(L.total)};
    const int64_t ar = g.trans_a ? g.k : g.m, ac = g.trans_a ? g.m : g.k;
    const int64_t br = g.trans_b ? g.n : g.k, bc = g.trans_b ? g.k : g.n;
    for (int c = 0; c < P; ++c) {
        if (overlap(rw, plane_range(g.A[c], ar, ac, g.lda)) || overlap(rw, plane_range(g.B[c], br, bc, g.ldb)) ||
            overlap(rw, plane_range(g.C[c], g.m, g.n, g.ldc)))
            return fail(MPG_EWORKSPACE, "workspace overlaps an operand");
    }
    const int variant = o->tile > 0 ? o->tile - 1 : 0;
    if (variant > 2) return fail(MPG_EINVAL, "INT8 tile id %d out of range 1..3", o->tile);
    cudaError_t e = launch_ozaki<P>(g, S, o->workspace, g_stream, variant, engine);
    return e == cudaSuccess ? MPG_OK : cuda_fail(e, "slicing gemm launch");
}

static bool is_crt(int algo)
{
    return algo == MPG_ALGO_INT8_CRT || algo == MPG_ALGO_BF16_CRT || algo == MPG_ALGO_INT8_CRT_SPLIT ||
           algo == MPG_ALGO_BF16_CRT_SPLIT;
}
static int crt_engine(int algo) { return algo == MPG_ALGO_BF16_CRT || algo == MPG_ALGO_BF16_CRT_SPLIT ? 1 : 0; }
static int crt_halves(int algo) { return algo == MPG_ALGO_INT8_CRT_SPLIT || algo == MPG_ALGO_BF16_CRT_SPLIT ? 2 : 1; }
static int crt_default_moduli(int P, int halves)
{
    if (halves == 2) return P == 2 ? 16 : P == 3 ? 22 : 30;
    return P == 2 ? 28 : P == 3 ? 44 : kCrtMaxModuli;
}

template <int P>
static int crt_call(const GemmArgs<P>& g, const mpgemm_opts* o)
{
    const int halves = crt_halves(o->algo);
    const int N = o->slices ? o->slices : crt_default_moduli(P, halves);
    if (N < 1 || N > kCrtMaxModuli)
        return fail(MPG_EINVAL, "the CRT form takes 1..%d moduli (got %d)", kCrtMaxModuli, N);
    if (g.k > crt_k_limit(halves))
        return fail(MPG_EUNSUPPORTED, "k = %lld exceeds %lld, the largest k whose residue products sum "
                    "exactly in int32", (long long)g.k, (long long)crt_k_limit(halves));
    const int beta = crt_beta(N, g.k, halves);
    if (beta < 1)
        return fail(MPG_EUNSUPPORTED, "%d moduli leave no bits for k = %lld (their product must exceed %s)", N,
                    (long long)g.k, halves == 2 ? "4k" : "2k");
    if (beta > crt_max_beta(halves))
        return fail(MPG_EUNSUPPORTED, "%d moduli give %d bits at k = %lld, more than the %d the form keeps", N,
                    beta, (long long)g.k, crt_max_beta(halves));
    const int engine = crt_engine(o->algo);
    const OzakiLayout L = crt_layout(N, g.m, g.n, g.k, engine, halves);
    if (L.mp / 128 > 65535) return fail(MPG_EINVAL, "m too large for the CRT form's grid");
    if (!o->workspace) return fail(MPG_EWORKSPACE, "the CRT form needs a workspace of %lld bytes",
                                   (long long)L.total);
    if (reinterpret_cast<uintptr_t>(o->workspace) % 256)
        return fail(MPG_EWORKSPACE, "workspace must be 256-byte aligned");
    if (o->workspace_bytes < static_cast<size_t>(L.total))
        return fail(MPG_EWORKSPACE, "workspace of %zu bytes is smaller than the %lld needed",
                    o->workspace_bytes, (long long)L.total);
    const Range rw{reinterpret_cast<uintptr_t>(o->workspace),
                   reinterpret_cast<uintptr_t>(o->workspace) + static_cast<uintptr_t>(L.total)};
    const int64_t ar = g.trans_a ? g.k : g.m, ac = g.trans_a ? g.m : g.k;
    const int64_t br = g.trans_b ? g.n : g.k, bc = g.trans_b ? g.k : g.n;
    for (int c = 0; c < P; ++c) {
        if (overlap(rw, plane_range(g.A[c], ar, ac, g.lda)) || overlap(rw, plane_range(g.B[c], br, bc, g.ldb)) ||
            overlap(rw, plane_range(g.C[c], g.m, g.n, g.ldc)))
            return fail(MPG_EWORKSPACE, "workspace overlaps an operand");
    }
    cudaError_t e = launch_crt<P>(g, N, o->workspace, g_stream, engine, halves);
    return e == cudaSuccess ? MPG_OK : cuda_fail(e, "CRT gemm launch");
}

template <int P>
static int gemm_call(const mpgemm_opts* o, int64_t m, int64_t n, int64_t k,
                     const double* const* A, int64_t lda, const double* const* B, int64_t ldb,
                     double* const* C, int64_t ldc)
{
    clear_error();
    if (!A || !B || !C) return fail(MPG_EINVAL, "plane pointer arrays must not be NULL");
    GemmArgs<P> g;
    for (int c = 0; c < P; ++c) {
        g.A[c] = A[c];
        g.B[c] = B[c];
        g.C[c] = C[c];
    }
    g.m = m; g.n = n; g.k = k; g.lda = lda; g.ldb = ldb; g.ldc = ldc;
    g.trans_a = o ? (o->trans_a != 0) : 0;
    g.trans_b = o ? (o->trans_b != 0) : 0;
    int rc = check_gemm<P>(g);
    if (rc != MPG_OK) return rc;
    if (m == 0 || n == 0) return MPG_OK;
    const int algo = o ? o->algo : MPG_ALGO_AUTO;
    if (algo != MPG_ALGO_AUTO && algo != MPG_ALGO_FP64_EFT && algo != MPG_ALGO_INT8_OZAKI &&
        algo != MPG_ALGO_BF16_SLICES && !is_crt(algo))
        return fail(MPG_EINVAL, "unknown algorithm %d", algo);
    const bool crt = is_crt(algo);
    const bool sliced = algo == MPG_ALGO_INT8_OZAKI || algo == MPG_ALGO_BF16_SLICES || crt;
    const int split = o ? o->split_k : 0;
    const int levels = o ? o->strassen : 0;
    if (P == 1 && (sliced || split > 1 || levels != 0))
        return fail(MPG_EINVAL, "the binary64-only product (P = 1) takes no slicing, split_k or strassen option");
    cudaError_t e;
    if (k == 0) {
        e = launch_zero<P>(g, g_stream);
        return e == cudaSuccess ? MPG_OK : cuda_fail(e, "zero launch");
    }
    if constexpr (P >= 2) {
        if (sliced) {
            if (o->strassen) return fail(MPG_EINVAL, "strassen applies to the FP64-EFT algorithm only");
            return crt ? crt_call(g, o) : ozaki_call(g, o);
        }
        if (levels < 0 || levels > kMaxStrassenLevels)
            return fail(MPG_EINVAL, "strassen must be in 0..%d (got %d)", kMaxStrassenLevels, levels);
        if (levels > 0) {
            if (g.trans_a || g.trans_b) return fail(MPG_EUNSUPPORTED, "the Strassen form takes untransposed operands");
            if (split > 1) return fail(MPG_EINVAL, "split_k and strassen cannot be combined");
            const int64_t bytes = strassen_workspace_elems(P, m, n, k, levels) * 8;
            if (bytes > 0) {
                if (!o->workspace) return fail(MPG_EWORKSPACE, "the Strassen form needs a workspace of %lld bytes",
                                               (long long)bytes);
                if (reinterpret_cast<uintptr_t>(o->workspace) % 256)
                    return fail(MPG_EWORKSPACE, "workspace must be 256-byte aligned");
                if (o->workspace_bytes < static_cast<size_t>(bytes))
                    return fail(MPG_EWORKSPACE, "workspace of %zu bytes is smaller than the %lld needed",
                                o->workspace_bytes, (long long)bytes);
                const Range rw{reinterpret_cast<uintptr_t>(o->workspace),
                               reinterpret_cast<uintptr_t>(o->workspace) + static_cast<uintptr_t>(bytes)};
                for (int c = 0; c < P; ++c) {
                    if (overlap(rw, plane_range(g.A[c], m, k, g.lda)) || overlap(rw, plane_range(g.B[c], k, n, g.ldb)) ||
                        overlap(rw, plane_range(g.C[c], m, n, g.ldc)))
                        return fail(MPG_EWORKSPACE, "workspace overlaps an operand");
                }
            }
            e = launch_strassen<P>(g, levels, static_cast<double*>(o->workspace), g_stream);
            return e == cudaSuccess ? MPG_OK : cuda_fail(e, "strassen launch");
        }
        if (split > 1) {
            if (split != 2 && split != 4 && split != 8 && split != 16 && split != 32)
                return fail(MPG_EINVAL, "split_k must be 0, 1, 2, 4, 8, 16 or 32 (got %d)", split);
            e = launch_gemm_splitk<P>(g, split, g_stream);
            return e == cudaSuccess ? MPG_OK : cuda_fail(e, "split-k gemm launch");
        }
    }
    if (split < 0) return fail(MPG_EINVAL, "split_k must be >= 0 (got %d)", split);
    int tile = o ? o->tile : 0;
    if (tile <= 0) {
        // a remembered choice of this shape's bucket, if its grid fits, else the occupancy rule
        const int tuned = tuned_tile_index(P, m, n, k, num_tiles<P>());
        tile = default_tile<P>(m, n, k);
        if (tuned >= 0) {
            const TileInfo tt = tile_info<P>(tuned);
            if ((n + tt.bn - 1) / tt.bn <= 2147483647LL && (m + tt.bm - 1) / tt.bm <= 65535LL) tile = tuned;
        }
    } else {
        tile -= 1;
    }
    if (tile >= num_tiles<P>()) return fail(MPG_EINVAL, "tile id %d out of range", tile + 1);
    const TileInfo ti = tile_info<P>(tile);
    if ((n + ti.bn - 1) / ti.bn > 2147483647LL || (m + ti.bm - 1) / ti.bm > 65535LL)
        return fail(MPG_EINVAL, "matrix too large for the grid of tile %d", tile + 1);
    e = launch_gemm_kseq<P>(g, tile, g_stream);
    return e == cudaSuccess ? MPG_OK : cuda_fail(e, "gemm launch");
}

}  // namespace mpg

using namespace mpg;

extern "C" {

const char* mpgemm_last_error(void) { return g_err; }

int mpgemm_set_stream(void* stream)
{
    g_stream = static_cast<cudaStream_t>(stream);
    return MPG_OK;
}

void* mpgemm_get_stream(void) { return static_cast<void*>(g_stream); }

int mpgemm_version(void) { return 106; }

int mp_quick_two_sum(int64_t n, const double* a, const double* b, double* s, double* e)
{ return eft_call(0, false, n, a, b, s, e); }
int mp_two_sum(int64_t n, const double* a, const double* b, double* s, double* e)
{ return eft_call(1, false, n, a, b, s, e); }
int mp_two_prod(int64_t n, const double* a, const double* b, double* s, double* e)
{ return eft_call(2, false, n, a, b, s, e); }
int mp_eft_int(int which, int64_t n, const double* a, const double* b, double* s, double* e)
{ return eft_call(which, true, n, a, b, s, e); }

int mp_dd_add(int64_t n, const double* const x[2], const double* const y[2], double* const r[2])
{ return vec_call<2>(0, n, x, y, r); }
int mp_dd_mul(int64_t n, const double* const x[2], const double* const y[2], double* const r[2])
{ return vec_call<2>(1, n, x, y, r); }
int mp_td_add(int64_t n, const double* const x[3], const double* const y[3], double* const r[3])
{ return vec_call<3>(0, n, x, y, r); }
int mp_td_add_merge(int64_t n, const double* const x[3], const double* const y[3], double* const r[3])
{ return vec_call<3>(2, n, x, y, r); }
int mp_td_mul(int64_t n, const double* const x[3], const double* const y[3], double* const r[3])
{ return vec_call<3>(1, n, x, y, r); }
int mp_qd_add(int64_t n, const double* const x[4], const double* const y[4], double* const r[4])
{ return vec_call<4>(0, n, x, y, r); }
int mp_qd_mul(int64_t n, const double* const x[4], const double* const y[4], double* const r[4])
{ return vec_call<4>(1, n, x, y, r); }
int mp_td_mul_q(int64_t n, const double* const x[3], const double* const y[3], double* const r[3])
{ return vec_call<3>(3, n, x, y, r); }
int mp_td_mul_accurate(int64_t n, const double* const x[3], const double* const y[3], double* const r[3])
{ return vec_call<3>(4, n, x, y, r); }
int mp_qd_add_accurate(int64_t n, const double* const x[4], const double* const y[4], double* const r[4])
{ return vec_call<4>(5, n, x, y, r); }

int mpgemm_dd(int64_t m, int64_t n, int64_t k, const double* const A[2], int64_t lda,
              const double* const B[2], int64_t ldb, double* const C[2], int64_t ldc)
{ return gemm_call<2>(nullptr, m, n, k, A, lda, B, ldb, C, ldc); }
int mpgemm_td(int64_t m, int64_t n, int64_t k, const double* const A[3], int64_t lda,
              const double* const B[3], int64_t ldb, double* const C[3], int64_t ldc)
{ return gemm_call<3>(nullptr, m, n, k, A, lda, B, ldb, C, ldc); }
int mpgemm_qd(int64_t m, int64_t n, int64_t k, const double* const A[4], int64_t lda,
              const double* const B[4], int64_t ldb, double* const C[4], int64_t ldc)
{ return gemm_call<4>(nullptr, m, n, k, A, lda, B, ldb, C, ldc); }

int mpgemm_d(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B, int64_t ldb,
             double* C, int64_t ldc)
{
    const double* const a[1] = {A};
    const double* const b[1] = {B};
    double* const c[1] = {C};
    return gemm_call<1>(nullptr, m, n, k, a, lda, b, ldb, c, ldc);
}

int mpgemm_ex(int P, const mpgemm_opts* opts, int64_t m, int64_t n, int64_t k,
              const double* const* A, int64_t lda, const double* const* B, int64_t ldb,
              double* const* C, int64_t ldc)
{
    switch (P) {
    case 1: return gemm_call<1>(opts, m, n, k, A, lda, B, ldb, C, ldc);
    case 2: return gemm_call<2>(opts, m, n, k, A, lda, B, ldb, C, ldc);
    case 3: return gemm_call<3>(opts, m, n, k, A, lda, B, ldb, C, ldc);
    case 4: return gemm_call<4>(opts, m, n, k, A, lda, B, ldb, C, ldc);
    default: clear_error(); return fail(MPG_EINVAL, "P must be 1, 2, 3 or 4 (got %d)", P);
    }
}

size_t mpgemm_workspace_size(int P, const mpgemm_opts* opts, int64_t m, int64_t n, int64_t k)
{
    if (!opts || P < 2 || P > 4 || m < 0 || n < 0 || k < 0) return 0;
    if ((opts->algo == MPG_ALGO_AUTO || opts->algo == MPG_ALGO_FP64_EFT) && opts->strassen > 0 &&
        opts->strassen <= kMaxStrassenLevels)
        return static_cast<size_t>(strassen_workspace_elems(P, m, n, k, opts->strassen) * 8);
    if (is_crt(opts->algo)) {
        const int halves = crt_halves(opts->algo);
        const int N = opts->slices ? opts->slices : crt_default_moduli(P, halves);
        if (N < 1 || N > kCrtMaxModuli) return 0;
        return static_cast<size_t>(crt_layout(N, m, n, k, crt_engine(opts->algo), halves).total);
    }
    if (opts->algo != MPG_ALGO_INT8_OZAKI && opts->algo != MPG_ALGO_BF16_SLICES) return 0;
    const int S = opts->slices ? opts->slices : ozaki_default_slices(P);
    if (S < 1 || S > ozaki_max_slices(P)) return 0;
    if (opts->algo == MPG_ALGO_BF16_SLICES) return static_cast<size_t>(ozaki_tc_layout(P, S, m, n, k).total);
    return static_cast<size_t>(ozaki_layout(S, m, n, k, 1).total);
}

int mpgemm_dd_int8_static(int64_t m, int64_t n, int64_t k, const double* const A[2], int64_t lda,
                          const double* const B[2], int64_t ldb, double* const C[2], int64_t ldc,
                          int slices)
{
    clear_error();
    if (!A || !B || !C) return fail(MPG_EINVAL, "plane pointer arrays must not be NULL");
    GemmArgs<2> g;
    for (int c = 0; c < 2; ++c) {
        g.A[c] = A[c];
        g.B[c] = B[c];
        g.C[c] = C[c];
    }
    g.m = m; g.n = n; g.k = k; g.lda = lda; g.ldb = ldb; g.ldc = ldc;
    g.trans_a = 0;
    g.trans_b = 0;
    int rc = check_gemm<2>(g);
    if (rc != MPG_OK) return rc;
    if (m == 0 || n == 0) return MPG_OK;
    const int S = slices ? slices : kOzakiDefaultSlices;
    if (S < 1 || S > kOzakiMaxSlices)
        return fail(MPG_EINVAL, "slices must be in 1..%d (got %d)", kOzakiMaxSlices, S);
    if (k > ozaki_k_limit(S))
        return fail(MPG_EUNSUPPORTED, "k = %lld exceeds %lld, the largest k whose %d-slice int32 "
                    "sums are exact", (long long)k, (long long)ozaki_k_limit(S), S);
    cudaError_t e;
    if (k == 0) {
        e = launch_zero<2>(g, g_stream);
        return e == cudaSuccess ? MPG_OK : cuda_fail(e, "zero launch");
    }
    const OzakiLayout L = ozaki_layout(S, m, n, k);
    if (L.total > kOzakiStaticScratchBytes)
        return fail(MPG_EWORKSPACE, "this product needs %lld bytes of scratch with %d slices; the "
                    "library's fixed array holds %lld (use mpgemm_ex with a workspace instead)",
                    (long long)L.total, S, (long long)kOzakiStaticScratchBytes);
    void* ws = nullptr;
    e = ozaki_static_scratch(&ws);
    if (e != cudaSuccess) return cuda_fail(e, "looking up the fixed scratch array");
    e = launch_ozaki<2>(g, S, ws, g_stream);
    return e == cudaSuccess ? MPG_OK : cuda_fail(e, "INT8 slicing gemm launch");
}

int mpgemm_crt_beta(int moduli, int64_t k)
{
    clear_error();
    if (moduli < 1 || moduli > kCrtMaxModuli || k < 0)
        return fail(MPG_EINVAL, "moduli must be in 1..%d and k >= 0 (got %d, %lld)", kCrtMaxModuli, moduli,
                    (long long)k);
    return crt_beta(moduli, k);
}

int mpgemm_crt_split_beta(int moduli, int64_t k)
{
    clear_error();
    if (moduli < 1 || moduli > kCrtMaxModuli || k < 0)
        return fail(MPG_EINVAL, "moduli must be in 1..%d and k >= 0 (got %d, %lld)", kCrtMaxModuli, moduli,
                    (long long)k);
    return crt_beta(moduli, k, 2);
}

int mpgemm_num_tiles(int P)
{
    switch (P) {
    case 1: return num_tiles<1>();
    case 2: return num_tiles<2>();
    case 3: return num_tiles<3>();
    case 4: return num_tiles<4>();
    default: return 0;
    }
}

int mpgemm_default_tile(int P, int64_t m, int64_t n, int64_t k)
{
    clear_error();
    if (m < 0 || n < 0 || k < 0)
        return fail(MPG_EINVAL, "m, n, k must be >= 0 (got %lld, %lld, %lld)", (long long)m, (long long)n,
                    (long long)k);
    switch (P) {
    case 1: return default_tile<1>(m, n, k) + 1;
    case 2: return default_tile<2>(m, n, k) + 1;
    case 3: return default_tile<3>(m, n, k) + 1;
    case 4: return default_tile<4>(m, n, k) + 1;
    default: return fail(MPG_EINVAL, "P must be 1, 2, 3 or 4 (got %d)", P);
    }
}

int mpgemm_tc_status(const void* workspace)
{
    clear_error();
    if (!workspace) return fail(MPG_EINVAL, "workspace is NULL");
    cudaError_t e = cudaStreamSynchronize(g_stream);
    int code = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&code, workspace, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the workspace header");
    if (code != 0) {
        static const char* const kRole[] = {"", "the producer (a stage to refill)", "the MMA issuer (a free accumulator)",
                                            "the MMA issuer (a loaded stage)", "a drain warp (a finished accumulator)",
                                            "an adder warp (a finished group)", "a drain warp (a free hand-over buffer)"};
        fail(MPG_OK, "a bounded wait gave up: %s; C is incomplete",
             code > 0 && code < 7 ? kRole[code] : "unknown role");
    }
    return code;
}

int mpgemm_tile_info(int P, int id, int info[6])
{
    clear_error();
    const int nt = mpgemm_num_tiles(P);
    if (nt == 0 || id < 1 || id > nt || !info) return fail(MPG_EINVAL, "unknown tile %d for P = %d", id, P);
    TileInfo t = P == 1 ? tile_info<1>(id - 1) : P == 2 ? tile_info<2>(id - 1)
                 : P == 3 ? tile_info<3>(id - 1) : tile_info<4>(id - 1);
    info[0] = t.bm; info[1] = t.bn; info[2] = t.bk; info[3] = t.tm; info[4] = t.tn; info[5] = t.threads;
    return MPG_OK;
}

int mpgemm_tile_int_ops(int P, int id)
{
    clear_error();
    const int nt = mpgemm_num_tiles(P);
    if (nt == 0 || id < 1 || id > nt) return fail(MPG_EINVAL, "unknown tile %d for P = %d", id, P);
    const TileInfo t = P == 1 ? tile_info<1>(id - 1) : P == 2 ? tile_info<2>(id - 1)
                       : P == 3 ? tile_info<3>(id - 1) : tile_info<4>(id - 1);
    return t.ints;
}

}  // extern "C"
