// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mpg {

// Plane pointers and shape of one GEMM, C := op(A) op(B).
template <int P>
struct GemmArgs {
    const double* A[P];
    const double* B[P];
    double* C[P];
    int64_t m, n, k, lda, ldb, ldc;
    int trans_a, trans_b;
};

struct TileInfo {
    int bm, bn, bk, tm, tn, threads;
};

// k-sequential FP64-EFT GEMM with tile configuration `tile` (0-based).
template <int P>
cudaError_t launch_gemm_kseq(const GemmArgs<P>& g, int tile, cudaStream_t s);
template <int P>
int num_tiles();
template <int P>
TileInfo tile_info(int tile);
// default tile for a shape
template <int P>
int default_tile(int64_t m, int64_t n, int64_t k);

// Warp split-K FP64-EFT GEMM: `split` lanes share one output, each summing a
// contiguous chunk of k, combined by shuffles.  split in {2,4,8,16,32}.
template <int P>
cudaError_t launch_gemm_splitk(const GemmArgs<P>& g, int split, cudaStream_t s);

// Host-side validation of a GEMM's arguments (MPG_OK or an error code with
// the thread's message set).
template <int P>
int check_gemm(const GemmArgs<P>& g);

// Strassen form: `levels` levels of Strassen's seven products over the
// k-sequential kernel (untransposed operands); workspace in doubles.
int64_t strassen_workspace_elems(int P, int64_t m, int64_t n, int64_t k, int levels);
template <int P>
cudaError_t launch_strassen(const GemmArgs<P>& g, int levels, double* ws, cudaStream_t s);

// C := 0 (all planes), for k == 0.
template <int P>
cudaError_t launch_zero(const GemmArgs<P>& g, cudaStream_t s);

// Elementwise kernels.  op: 0 add, 1 mul, 2 merge-based add (P == 3 only).
template <int P>
cudaError_t launch_vec(int op, int64_t n, const double* const* x, const double* const* y,
                       double* const* r, cudaStream_t s);
// which: 0 QuickTwoSum, 1 TwoSum, 2 TwoProd
cudaError_t launch_eft(int which, int64_t n, const double* a, const double* b, double* s,
                       double* e, cudaStream_t st);

int num_sms();
cudaStream_t current_stream();
void clear_error();
int set_error(int code, const char* msg);

}  // namespace mpg
