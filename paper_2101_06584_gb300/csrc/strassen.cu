// strassen.cu -- the Strassen form of the DD/TD/QD GEMM (Sec. 3): for even
// dimensions C := A B from seven products of half-size blocks,
//
//   M1 = (A11 + A22)(B11 + B22)     M5 = (A11 + A12) B22
//   M2 = (A21 + A22) B11            M6 = (A21 - A11)(B11 + B12)
//   M3 = A11 (B12 - B22)            M7 = (A12 - A22)(B21 + B22)
//   M4 = A22 (B21 - B11)
//   C11 = ((M1 + M4) - M5) + M7     C12 = M3 + M5
//   C21 = M2 + M4                   C22 = ((M1 - M2) + M3) + M6
//
// recursively `levels` times while m, n and k are even; the leaf products are
// the k-sequential kernel.  "+" is the precision's GEMM addition (DDadd,
// TDaddq, QDadd) and x - y is x + (-y), so every result is bit-identical to
// the same steps on the host.  Blocks are strided views of the operands; the
// sums and the seven products live in the caller's workspace.  On GB300 the
// leaves are FP64-bound, so each level removes an eighth of the work for
// O(n^2) block additions.
#include "internal.h"
#include "mp_arith.cuh"

namespace mpg {

template <int P>
struct MatArgs {
    const double* x[P];
    const double* y[P];
    double* r[P];
    int64_t rows, cols, ldx, ldy, ldr;
};

// r = x + y, or x + (-y) for SUB, elementwise over a rows x cols block; r may
// be x itself.
template <int P, bool SUB>
__global__ void __launch_bounds__(256) mat_addsub_kernel(const MatArgs<P> a)
{
    const mp::Rn f = mp::make_rn();
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= a.cols) return;
    for (int64_t i = blockIdx.y; i < a.rows; i += gridDim.y) {
        double x[P], y[P], r[P];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            x[c] = a.x[c][i * a.ldx + j];
            const double v = a.y[c][i * a.ldy + j];
            y[c] = SUB ? -v : v;
        }
        mp::Ops<P>::add(f, x, y, r);
#pragma unroll
        for (int c = 0; c < P; ++c) a.r[c][i * a.ldr + j] = r[c];
    }
}

namespace {

// A rows x cols block of P planes with leading dimension ld.
template <int P, typename T>
struct Block {
    T* c[P];
    int64_t ld;
    Block sub(int64_t i, int64_t j) const
    {
        Block b = *this;
        for (int q = 0; q < P; ++q) b.c[q] = c[q] + i * ld + j;
        return b;
    }
};
template <int P> using CBlock = Block<P, const double>;
template <int P> using MBlock = Block<P, double>;

// A contiguous rows x cols block carved from the workspace.
template <int P>
MBlock<P> carve(double*& ws, int64_t rows, int64_t cols)
{
    MBlock<P> b;
    for (int q = 0; q < P; ++q) {
        b.c[q] = ws;
        ws += rows * cols;
    }
    b.ld = cols;
    return b;
}

template <int P>
CBlock<P> as_const(const MBlock<P>& m)
{
    CBlock<P> b;
    for (int q = 0; q < P; ++q) b.c[q] = m.c[q];
    b.ld = m.ld;
    return b;
}

template <int P, bool SUB>
cudaError_t addsub(const CBlock<P>& x, const CBlock<P>& y, const MBlock<P>& r, int64_t rows, int64_t cols,
                   cudaStream_t s)
{
    MatArgs<P> a;
    for (int q = 0; q < P; ++q) {
        a.x[q] = x.c[q];
        a.y[q] = y.c[q];
        a.r[q] = r.c[q];
    }
    a.rows = rows;
    a.cols = cols;
    a.ldx = x.ld;
    a.ldy = y.ld;
    a.ldr = r.ld;
    const dim3 grid(static_cast<unsigned>((cols + 255) / 256),
                    static_cast<unsigned>(rows < 1024 ? rows : 1024));
    mat_addsub_kernel<P, SUB><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t leaf(const CBlock<P>& A, const CBlock<P>& B, const MBlock<P>& C, int64_t m, int64_t n, int64_t k,
                 cudaStream_t s)
{
    GemmArgs<P> g;
    for (int q = 0; q < P; ++q) {
        g.A[q] = A.c[q];
        g.B[q] = B.c[q];
        g.C[q] = C.c[q];
    }
    g.m = m;
    g.n = n;
    g.k = k;
    g.lda = A.ld;
    g.ldb = B.ld;
    g.ldc = C.ld;
    g.trans_a = 0;
    g.trans_b = 0;
    return launch_gemm_kseq<P>(g, default_tile<P>(m, n, k), s);
}

bool splits(int64_t m, int64_t n, int64_t k) { return m % 2 == 0 && n % 2 == 0 && k % 2 == 0 && m && n && k; }

template <int P>
cudaError_t strassen_rec(const CBlock<P>& A, const CBlock<P>& B, const MBlock<P>& C, int64_t m, int64_t n,
                         int64_t k, int levels, double* ws, cudaStream_t s)
{
    if (levels <= 0 || !splits(m, n, k)) return leaf<P>(A, B, C, m, n, k, s);
    const int64_t m2 = m / 2, n2 = n / 2, k2 = k / 2;
    const CBlock<P> A11 = A.sub(0, 0), A12 = A.sub(0, k2), A21 = A.sub(m2, 0), A22 = A.sub(m2, k2);
    const CBlock<P> B11 = B.sub(0, 0), B12 = B.sub(0, n2), B21 = B.sub(k2, 0), B22 = B.sub(k2, n2);
    double* w = ws;
    const MBlock<P> TA = carve<P>(w, m2, k2), TB = carve<P>(w, k2, n2);
    MBlock<P> M[7];
    for (int i = 0; i < 7; ++i) M[i] = carve<P>(w, m2, n2);
    double* inner = w;
    const CBlock<P> ta = as_const(TA), tb = as_const(TB);
    cudaError_t e = cudaSuccess;
    auto add = [&](const CBlock<P>& x, const CBlock<P>& y, const MBlock<P>& r, int64_t rr, int64_t cc) {
        if (e == cudaSuccess) e = addsub<P, false>(x, y, r, rr, cc, s);
    };
    auto sub = [&](const CBlock<P>& x, const CBlock<P>& y, const MBlock<P>& r, int64_t rr, int64_t cc) {
        if (e == cudaSuccess) e = addsub<P, true>(x, y, r, rr, cc, s);
    };
    auto rec = [&](const CBlock<P>& x, const CBlock<P>& y, const MBlock<P>& r) {
        if (e == cudaSuccess) e = strassen_rec<P>(x, y, r, m2, n2, k2, levels - 1, inner, s);
    };
    add(A11, A22, TA, m2, k2);
    add(B11, B22, TB, k2, n2);
    rec(ta, tb, M[0]);
    add(A21, A22, TA, m2, k2);
    rec(ta, B11, M[1]);
    sub(B12, B22, TB, k2, n2);
    rec(A11, tb, M[2]);
    sub(B21, B11, TB, k2, n2);
    rec(A22, tb, M[3]);
    add(A11, A12, TA, m2, k2);
    rec(ta, B22, M[4]);
    sub(A21, A11, TA, m2, k2);
    add(B11, B12, TB, k2, n2);
    rec(ta, tb, M[5]);
    sub(A12, A22, TA, m2, k2);
    add(B21, B22, TB, k2, n2);
    rec(ta, tb, M[6]);
    CBlock<P> m_[7];
    for (int i = 0; i < 7; ++i) m_[i] = as_const(M[i]);
    const MBlock<P> C11 = C.sub(0, 0), C12 = C.sub(0, n2), C21 = C.sub(m2, 0), C22 = C.sub(m2, n2);
    add(m_[0], m_[3], C11, m2, n2);
    sub(as_const(C11), m_[4], C11, m2, n2);
    add(as_const(C11), m_[6], C11, m2, n2);
    add(m_[2], m_[4], C12, m2, n2);
    add(m_[1], m_[3], C21, m2, n2);
    sub(m_[0], m_[1], C22, m2, n2);
    add(as_const(C22), m_[2], C22, m2, n2);
    add(as_const(C22), m_[5], C22, m2, n2);
    return e;
}

}  // namespace

int64_t strassen_workspace_elems(int P, int64_t m, int64_t n, int64_t k, int levels)
{
    if (levels <= 0 || !splits(m, n, k)) return 0;
    const int64_t m2 = m / 2, n2 = n / 2, k2 = k / 2;
    return static_cast<int64_t>(P) * (m2 * k2 + k2 * n2 + 7 * m2 * n2) +
           strassen_workspace_elems(P, m2, n2, k2, levels - 1);
}

template <int P>
cudaError_t launch_strassen(const GemmArgs<P>& g, int levels, double* ws, cudaStream_t s)
{
    CBlock<P> A, B;
    MBlock<P> C;
    for (int q = 0; q < P; ++q) {
        A.c[q] = g.A[q];
        B.c[q] = g.B[q];
        C.c[q] = g.C[q];
    }
    A.ld = g.lda;
    B.ld = g.ldb;
    C.ld = g.ldc;
    return strassen_rec<P>(A, B, C, g.m, g.n, g.k, levels, ws, s);
}

template cudaError_t launch_strassen<2>(const GemmArgs<2>&, int, double*, cudaStream_t);
template cudaError_t launch_strassen<3>(const GemmArgs<3>&, int, double*, cudaStream_t);
template cudaError_t launch_strassen<4>(const GemmArgs<4>&, int, double*, cudaStream_t);

}  // namespace mpg
