// internal.h -- declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <initializer_list>
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

// A k-sequential tile: CTA tile bm x bn, k slab bk, tm x tn outputs per
// thread; ints names the transformations run on the integer pipes (the mask
// of mp::RnInt: 1 TwoSum, 2 FastTwoSum, 4 TwoProd; 0 for none).
struct TileInfo {
    int bm, bn, bk, tm, tn, threads;
    int ints;
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

// Elementwise kernels.  op: 0 add, 1 mul (the GEMM's pair for P); 2 TDadd
// (Alg. 3), 3 TDmulq, 4 accurate TD product (P == 3); 5 accurate QD addition
// (P == 4).
template <int P>
cudaError_t launch_vec(int op, int64_t n, const double* const* x, const double* const* y,
                       double* const* r, cudaStream_t s);
// which: 0 QuickTwoSum, 1 TwoSum, 2 TwoProd; int_pipes: the integer-pipe form
// (mp::RnInt) instead of the operation sequence.
cudaError_t launch_eft(int which, bool int_pipes, int64_t n, const double* a, const double* b, double* s,
                       double* e, cudaStream_t st);

int num_sms();

// The default tile among `cands` (tile ids, largest tile first): the first
// whose CTAs, dealt round-robin to the SMs, keep at least 90% of the SMs'
// time busy -- ctas / (sms * ceil(ctas / sms)) -- else the one that comes
// closest.  Every tile gives the same, k-sequential result, so this only
// trades staging per output against idle SMs in the last wave.
template <int P>
int pick_tile(int64_t m, int64_t n, std::initializer_list<int> cands)
{
    const int64_t sms = num_sms();
    int best = *cands.begin();
    double best_eff = -1.0;
    for (const int t : cands) {
        const TileInfo ti = tile_info<P>(t);
        const int64_t ctas = ((m + ti.bm - 1) / ti.bm) * ((n + ti.bn - 1) / ti.bn);
        const int64_t per_sm = (ctas + sms - 1) / sms;
        const double eff = per_sm > 0 ? static_cast<double>(ctas) / static_cast<double>(sms * per_sm) : 0.0;
        if (eff >= 0.9) return t;
        if (eff > best_eff) {
            best_eff = eff;
            best = t;
        }
    }
    return best;
}

// Whether an m x n product has enough outputs for the tiles that compute
// transformations on the integer pipes: a transformation there is a chain of
// some fifty dependent integer instructions, whose latency takes many warps
// per SM to hide.  On GB300, against the best FP64-pipe tile, they run
// 1.7-2.0x faster at 1024^2 outputs (about 6900 per SM), 1.2-1.6x faster at
// 256^2 (about 430 per SM) and 1.6x slower at 128^2 (about 110 per SM); the
// rule takes them from 256 outputs per SM.
inline bool int_tiles_pay(int64_t m, int64_t n)
{
    return m * n >= static_cast<int64_t>(256) * num_sms();
}

cudaStream_t current_stream();
void clear_error();
int set_error(int code, const char* msg);

// Autotuner cache (tune.cu): keys "device|gemm:P:bm:bn:bk" (the bits of m,
// n, k rounded up to powers of two) and "device|batch:P:count:hash".
int tune_bucket(int64_t x);
void gemm_tune_key(int P, int64_t m, int64_t n, int64_t k, char* out, size_t cap);
void batch_tune_key(int P, int count, uint64_t shapes_hash, char* out, size_t cap);
bool tune_lookup(const char* key, int* choice, float* ms);
void tune_store(const char* key, int choice, float ms);
int tuned_tile_index(int P, int64_t m, int64_t n, int64_t k, int ntiles);

}  // namespace mpg
