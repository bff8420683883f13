/*
 * mpgemm.h -- C ABI of the GB300 multi-component (DD/TD/QD) GEMM library.
 *
 * Implements the hot path of T. Kouya, "Acceleration of multiple precision
 * matrix multiplication based on multi-component floating-point arithmetic
 * using AVX2" (arXiv 2101.06584): the matrix product C := A B of Sec. 3,
 * Eq. 1, in double-double (DD, 2 components), triple-double (TD, 3) and
 * quad-double (QD, 4) arithmetic, built from the error-free transformations
 * of Sec. 2.1 and the additions/multiplications of Sec. 2.2-2.4 (Alg. 1-6).
 *
 * Data layout (Sec. 2.5, Fig. 1; Sec. 3 row-major): a P-component vector or
 * matrix is P separate planes of binary64, plane 0 the most significant
 * component.  A matrix plane is row-major: element (i, j) of plane c of X is
 * X[c][i * ldx + j].  Arguments of the form `const double *const X[P]` are
 * host arrays of P DEVICE pointers.
 *
 * Ownership: every pointer is owned by the caller.  The library allocates no
 * device memory; calls that need scratch take a caller-provided workspace.
 * Kernels run asynchronously on the calling thread's current stream (see
 * mpgemm_set_stream); a call returns once the work is enqueued.
 *
 * Errors: every entry point returns an mpg_status.  Invalid arguments are
 * detected on the host and return MPG_EINVAL without launching anything; a
 * failed launch returns MPG_ECUDA.  mpgemm_last_error() gives a message for
 * the calling thread's most recent failure.  Faults during asynchronous
 * execution surface at the caller's next synchronisation.
 *
 * Numerics: inputs are finite binary64 components; the results of the
 * elementwise operations and of the k-sequential GEMM are the exact bits of
 * the paper's algorithms (round to nearest even, no contraction other than
 * the algorithms' own FMAs).  Non-finite inputs give unspecified output.
 */
#ifndef MPGEMM_H
#define MPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mpg_status {
    MPG_OK = 0,
    MPG_EINVAL = -1,       /* invalid argument; nothing was launched */
    MPG_ECUDA = -2,        /* a CUDA call or launch failed */
    MPG_EWORKSPACE = -3,   /* workspace missing, too small or misaligned */
    MPG_EUNSUPPORTED = -4  /* valid request the library does not support */
} mpg_status;

/* Message describing the calling thread's most recent failure ("" if none). */
const char *mpgemm_last_error(void);

/* Set / get the CUDA stream (a cudaStream_t, NULL = legacy default stream)
 * on which the calling thread's subsequent calls enqueue their kernels. */
int mpgemm_set_stream(void *stream);
void *mpgemm_get_stream(void);

/* Library ABI version (major * 100 + minor): 101 adds the TD/QD variants,
 * mpgemm_default_tile and mpgemm_tc_status to 100; 102 adds mpgemm_d and
 * P = 1 in mpgemm_ex, mpgemm_num_tiles, mpgemm_tile_info and
 * mpgemm_default_tile; 103 adds MPG_ALGO_INT8_CRT, MPG_ALGO_BF16_CRT and
 * mpgemm_crt_beta; 104 adds MPG_ALGO_INT8_CRT_SPLIT, MPG_ALGO_BF16_CRT_SPLIT
 * and mpgemm_crt_split_beta; 105 adds mpgemm_autotune, mpgemm_tuned_tile and
 * mpgemm_tune_cache_reset; 106 adds mpgemm_tile_int_ops, mp_eft_int and the
 * tiles that compute error-free transformations on the integer pipes. */
int mpgemm_version(void);

/* ---------------------------------------------------------------------
 * Elementwise error-free transformations, Sec. 2.1, over n-vectors:
 *   QuickTwoSum: s_i = fl(a_i + b_i), e_i = b_i - (s_i - a_i)
 *   TwoSum:      s_i = fl(a_i + b_i), e_i = (a_i + b_i) - s_i exactly
 *   TwoProd:     s_i = fl(a_i b_i),   e_i = fma(a_i, b_i, -s_i)
 * a, b, s, e: device arrays of n binary64; s and e must not overlap a or b
 * unless identical to them.  n = 0 is a no-op; n < 0 or a NULL pointer with
 * n > 0 is MPG_EINVAL.
 * ------------------------------------------------------------------- */
int mp_quick_two_sum(int64_t n, const double *a, const double *b, double *s, double *e);
int mp_two_sum(int64_t n, const double *a, const double *b, double *s, double *e);
int mp_two_prod(int64_t n, const double *a, const double *b, double *s, double *e);
/* The same three transformations (which: 0 QuickTwoSum, 1 TwoSum, 2 TwoProd)
 * computed on the integer pipes, the form the tiles of mpgemm_tile_int_ops
 * use: both outputs from one exact integer sum or product of the
 * significands, with the bits of the operation sequences above for every
 * input (non-finite operands, overflow, a product error below the subnormal
 * range and QuickTwoSum with |b| > |a| run the sequence).  Arguments and
 * errors as above; a `which` outside 0..2 is MPG_EINVAL. */
int mp_eft_int(int which, int64_t n, const double *a, const double *b, double *s, double *e);

/* ---------------------------------------------------------------------
 * Elementwise multi-component add/mul of SoA vectors (Sec. 2.5):
 * r_i = x_i (+|*) y_i for i < n.
 *   mp_dd_add  Alg. 1        mp_dd_mul  Alg. 2
 *   mp_td_add  TDaddq, Sec. 2.3 (QDadd with zero fourth components; the
 *              paper's default TD addition)
 *   mp_td_add_merge  Alg. 3 (Merge, VecSum, VSEB(3))
 *   mp_td_mul  Alg. 4        mp_qd_add  Alg. 5        mp_qd_mul  Alg. 6
 * x, y, r: host arrays of P device pointers to n binary64 each.  r may
 * alias x or y exactly (in place); partial overlap is not allowed.
 * ------------------------------------------------------------------- */
int mp_dd_add(int64_t n, const double *const x[2], const double *const y[2], double *const r[2]);
int mp_dd_mul(int64_t n, const double *const x[2], const double *const y[2], double *const r[2]);
int mp_td_add(int64_t n, const double *const x[3], const double *const y[3], double *const r[3]);
int mp_td_add_merge(int64_t n, const double *const x[3], const double *const y[3], double *const r[3]);
int mp_td_mul(int64_t n, const double *const x[3], const double *const y[3], double *const r[3]);
int mp_qd_add(int64_t n, const double *const x[4], const double *const y[4], double *const r[4]);
int mp_qd_mul(int64_t n, const double *const x[4], const double *const y[4], double *const r[4]);

/* ---------------------------------------------------------------------
 * Variants of the TD/QD operations (Sec. 2.3-2.4), same arguments and rules
 * as the calls above:
 *   mp_td_mul_q  TDmulq, the trial TD product of Sec. 2.3: QDmul (Alg. 6) on
 *                operands padded with a zero fourth component, the fourth
 *                result component dropped.
 *   mp_td_mul_accurate  the accurate TD product (Sec. 2.3 names it; its steps
 *                are this library's): each x_i y_j with i + j <= 2 split
 *                exactly by TwoProd, the order-three terms summed with one
 *                rounding each -- (q02 + q11) + q20, then fma(x2, y1, .), then
 *                fma(x1, y2, .) -- and x2 y2 dropped.  The ten terms
 *                (p00, q00, p01, p10, q01, q10, p02, p11, p20, t3), stably
 *                sorted by decreasing magnitude, go through the accurate
 *                normalisation below; the fourth component is dropped.
 *                Within 2^-158 of the exact product, relative to it.
 *   mp_qd_add_accurate  the accurate (IEEE-style) QD addition of Hida, Li and
 *                Bailey: the eight components (x0..x3, y0..y3) stably sorted
 *                by decreasing magnitude, then the accurate normalisation.
 *                Within 2^-211 of the exact sum relative to |x + y|, also
 *                under cancellation (the sloppy mp_qd_add is bounded only
 *                relative to |x| + |y|).
 * The accurate normalisation: the sorted terms are added one by one into a
 * two-term accumulator (u, v); a term t gives (s1, e1) = TwoSum(v, t) and
 * (s, e2) = TwoSum(u, s1); if both errors are nonzero s is emitted as the
 * next component and (u, v) = (e2, e1), else u = s and v is the nonzero
 * error (e2 when both are zero).  After four components the accumulator and
 * the remaining terms are summed, in order, into a fifth term; if the terms
 * run out first, u and v follow the components.  Renorm (Sec. 2.4) of the
 * five terms gives the result.  Every result is bit-identical to these steps
 * in binary64 with round-to-nearest-even.
 * ------------------------------------------------------------------- */
int mp_td_mul_q(int64_t n, const double *const x[3], const double *const y[3], double *const r[3]);
int mp_td_mul_accurate(int64_t n, const double *const x[3], const double *const y[3], double *const r[3]);
int mp_qd_add_accurate(int64_t n, const double *const x[4], const double *const y[4], double *const r[4]);

/* ---------------------------------------------------------------------
 * GEMM, Sec. 3, Eq. 1: C := A B with A m x k, B k x n, C m x n, each a set
 * of P row-major device planes.  C is overwritten (there is no alpha/beta,
 * as in the paper).  Requirements: m, n, k >= 0; lda >= max(1, k),
 * ldb >= max(1, n), ldc >= max(1, n); no NULL plane where the matrix is
 * non-empty; C must not overlap A or B.  k = 0 sets C to zero; m = 0 or
 * n = 0 is a no-op.
 *
 * These calls run the k-sequential FP64-EFT kernel: every c_ij is
 * accumulated by one thread as acc = add(acc, mul(a_ip, b_pj)) for
 * p = 0, 1, ..., k-1 from acc = 0, with mul/add the paper's DD (Alg. 1-2),
 * TD (Alg. 4, TDaddq) or QD (Alg. 5-6) operations, a_ip the left operand.
 * The result is bit-identical to that sequence evaluated anywhere else.
 * ------------------------------------------------------------------- */
int mpgemm_dd(int64_t m, int64_t n, int64_t k,
              const double *const A[2], int64_t lda,
              const double *const B[2], int64_t ldb,
              double *const C[2], int64_t ldc);
int mpgemm_td(int64_t m, int64_t n, int64_t k,
              const double *const A[3], int64_t lda,
              const double *const B[3], int64_t ldb,
              double *const C[3], int64_t ldc);
int mpgemm_qd(int64_t m, int64_t n, int64_t k,
              const double *const A[4], int64_t lda,
              const double *const B[4], int64_t ldb,
              double *const C[4], int64_t ldc);

/* The binary64-only product: C := A B of Sec. 3, Eq. 1 evaluated in plain
 * binary64, the arithmetic the multi-component formats extend (Sec. 1) and
 * against which Sec. 3 counts the decimal digits a product loses.  A, B, C
 * are single row-major device planes (m x k, k x n, m x n) with the
 * requirements of mpgemm_dd.  Every c_ij is accumulated by one thread as
 * acc = fma(a_ip, b_pj, acc) for p = 0, 1, ..., k-1 from acc = +0, so the
 * result is bit-identical to that sequence evaluated anywhere else and within
 * k * 2^-53 (|A| |B|)_ij of the exact product.  Given the leading planes of
 * DD/TD/QD operands it is the FP64-only GEMM that the multi-component
 * results are compared with.  mpgemm_ex with P = 1 takes the same product
 * with transposes and a tile choice (no slicing, split_k or strassen). */
int mpgemm_d(int64_t m, int64_t n, int64_t k,
             const double *A, int64_t lda,
             const double *B, int64_t ldb,
             double *C, int64_t ldc);

/* Algorithms selectable through mpgemm_ex. */
typedef enum mpg_algo {
    MPG_ALGO_AUTO = 0,       /* the FP64-EFT kernel (k-sequential unless split_k > 1) */
    MPG_ALGO_FP64_EFT = 1,   /* FP64 error-free transformations on the CUDA cores */
    MPG_ALGO_INT8_OZAKI = 2, /* DD/TD/QD: error-free INT8 slicing on the tensor cores */
    MPG_ALGO_BF16_SLICES = 3, /* DD/TD/QD: the same digits as bf16 on tcgen05 (TMEM accumulators) */
    MPG_ALGO_INT8_CRT = 4,    /* DD/TD/QD: residues modulo small coprime moduli on the tensor cores */
    MPG_ALGO_BF16_CRT = 5,    /* DD/TD/QD: the same residues as bf16 on tcgen05 (TMEM accumulators) */
    MPG_ALGO_INT8_CRT_SPLIT = 6, /* the CRT form with split integers (about twice the bits), mma.sync */
    MPG_ALGO_BF16_CRT_SPLIT = 7  /* the same on tcgen05 */
} mpg_algo;

/* Options of mpgemm_ex.  Zero-initialised options give the plain call. */
typedef struct mpgemm_opts {
    int trans_a;    /* 1: A is given as its k x m transpose (element (i,p) at A[c][p*lda+i]) */
    int trans_b;    /* 1: B is given as its n x k transpose (element (p,j) at B[c][j*ldb+p]) */
    int algo;       /* an mpg_algo */
    int split_k;    /* 0/1: k-sequential.  s > 1: the k range is cut into s contiguous
                       chunks, summed separately and combined with the precision's
                       add in a fixed tree order (not bit-identical to k-sequential;
                       within the same error bound) */
    int slices;     /* INT8_OZAKI: slices per operand, 0 = default */
    int tile;       /* FP64_EFT: tile configuration id 1..mpgemm_num_tiles(P);
                       INT8_OZAKI: slice-product tiling 1..3; 0 or -1 = library choice
                       (FP64_EFT: the largest of a few tiles whose CTAs keep at least
                       90% of the SMs busy in the last wave; every tile gives the
                       same result) */
    void *workspace;          /* device scratch for algorithms that need it */
    size_t workspace_bytes;
    int strassen;   /* FP64_EFT / AUTO: levels of Strassen's algorithm (0..8, 0 = none;
                       untransposed operands, split_k 0 or 1): see below */
} mpgemm_opts;

/* C := op(A) op(B) with the options above; P in {2, 3, 4} (or 1, the
 * binary64-only product of mpgemm_d); lda/ldb must cover the stored
 * (possibly transposed) shapes. */
int mpgemm_ex(int P, const mpgemm_opts *opts, int64_t m, int64_t n, int64_t k,
              const double *const *A, int64_t lda,
              const double *const *B, int64_t ldb,
              double *const *C, int64_t ldc);

/* MPG_ALGO_INT8_OZAKI (not in the paper).  C := op(A) op(B) via an
 * error-free splitting whose products run on the tensor cores.  For DD:
 *   sigma_i = ilogb(max_p |a_ip[0]|) + 2 per row of op(A) (0 for a zero row),
 *   tau_j likewise per column of op(B); S = opts->slices (default 14, 1..16)
 *   balanced base-2^7 digits of a 2^-sigma, each the nearest integer (ties to
 *   even) of the exact scaled remainder; for w = S+1 down to 2 the int32 sum
 *   P_w of the slice products with s + t = w (exact: requires
 *   S * k * 4096 < 2^31, else MPG_EUNSUPPORTED); the weight sums combined
 *   exactly G = 5 at a time from the least significant weight (w = S+1,
 *   ..., S-3, then S-4, ...; the last group may be shorter),
 *   V = P_w + 2^7 P_(w-1) + ... + 2^28 P_(w-4) (|V| < 2^60), V split exactly
 *   into hi = RN(V) (ties to even) and lo = V - hi, and from acc = 0,
 *   acc = DDadd(acc, (hi 2^e, lo 2^e)), e = sigma_i + tau_j - 7w (Alg. 1),
 *   w the group's largest weight.  hi 2^e and lo 2^e are scaled as C's
 *   ldexp: exact in the normal binary64 range (every product but the
 *   tiniest and the largest); below it rounded to the nearest multiple of
 *   2^-1074, ties to even, a zero keeping its sign; above it +-inf.
 * The result is deterministic and bit-identical to those steps evaluated
 * anywhere; its error against the exact product shrinks by ~2^-7 per slice.
 * Needs opts->workspace: 256-byte aligned, mpgemm_workspace_size() bytes, not
 * overlapping A, B or C.  Layout (mp, np = m, n rounded up to 64, kp = k
 * rounded up to 128, padding zero; each region starts on a 256-byte boundary):
 *   int8  [S][mp][kp]  slices of op(A);   int8 [S][np][kp] slices of op(B)^T;
 *   int32 [mp] sigma;                     int32 [np] tau.
 * The workspace holds these values after the call.
 * For TD and QD (P = 3, 4; S default 22 / 29, 1..40): each component is
 * first floored to a multiple of 2^(sigma - 7S - 12 - 64) and the digits are
 * those of the sum of the floored components (computed exactly in 384-bit
 * integers); the groups hold G = 11 (TD, |V| < 2^102) or 10 (QD, |V| < 2^95)
 * weights and are added with
 * TDaddq / QDadd (Sec. 2.3, Alg. 5) of (hi 2^e, lo 2^e, 0, ...).
 *
 * MPG_ALGO_BF16_SLICES (DD/TD/QD; not in the paper): the same digits, scales,
 * weight sums and accumulation, with the slice products on the 5th-generation
 * tensor cores: the digits are stored as bf16 (exact: |d| <= 64), loaded by
 * TMA, multiplied by tcgen05.mma (kind::f16, M = 128, N = 128 for DD and 64
 * for TD/QD, fp32 accumulation in
 * tensor memory), and each accumulator is drained into exact integer sums
 * after at most 2048 values of k of one weight, so every fp32 partial sum is
 * an integer below 2^23 and exact.  The result is bit-identical to
 * MPG_ALGO_INT8_OZAKI.  Workspace: a 256-byte header whose first int32 is 0
 * after a normal run (a device-side wait that exceeded about a second leaves
 * the code of the waiting role there), then the digits as bf16 with rows
 * padded to 128 ([S][mp][kp] for op(A); 256 for DD) and to N ([S][np][kp] for
 * op(B)^T), then the int32 exponents, then for DD 256 KB per SM in which
 * finished groups wait for their additions to C; mpgemm_workspace_size gives
 * the total. */

/* MPG_ALGO_INT8_CRT (not in the paper; the Chinese-remainder form, also
 * called Ozaki scheme II).  C := op(A) op(B) for P = 2, 3, 4 with N =
 * opts->slices moduli (default 28 for DD, 44 for TD, 49 for QD; 1..49):
 *   moduli  m_0 = 256, m_1 = 255, 253, 251, 247, ...: the pairwise coprime
 *           integers <= 256 taken greedily from 256 downward (49 of them);
 *           M = m_0 ... m_(N-1).
 *   bits    beta = mpgemm_crt_beta(N, k), the largest beta with
 *           k 2^(2 beta - 1) < M (MPG_EUNSUPPORTED if there is none).
 *   scale   sigma_i, tau_j as for MPG_ALGO_INT8_OZAKI.
 *   integers A'_ip = the nearest integer (ties to even) of the sum of the
 *           components of a_ip, each first floored to a multiple of
 *           2^(sigma_i - beta - 64), in units of 2^(sigma_i - beta);
 *           |A'| <= 2^(beta - 1); B' likewise with tau_j.
 *   residues r(x, m) in [-floor(m/2), ceil(m/2) - 1] (|r| <= 128, int8).
 *   products Q_i = r(A', m_i) r(B', m_i)^T on mma.sync m16n8k32 s8, exact in
 *           int32 (k <= 131071, else MPG_EUNSUPPORTED).
 *   recover C' = the integer in [-M/2, M/2) congruent to Q_i mod m_i for
 *           every i, which is A'B' exactly.
 *   output  the P components of C' 2^(sigma_i + tau_j - 2 beta), each the
 *           nearest binary64 (ties to even; gradual underflow, +-inf above
 *           the range) of the exact remainder of the previous ones.
 * The result is deterministic and bit-identical to these steps evaluated
 * anywhere; its error against the exact product is about 2^-beta relative to
 * the row and column scales (beta is about 170 at most, so QD results carry
 * fewer bits than the QD format).  Workspace (mpgemm_workspace_size, 256-byte
 * aligned, not overlapping A, B or C), with mp, np, kp = m, n, k rounded up
 * to 128 and each region on a 256-byte boundary: int8 [N][mp][kp] residues
 * of op(A), int8 [N][np][kp] of op(B)^T, int32 [mp] sigma, int32 [np] tau,
 * int8 [N][mp][np] residues of the products.
 *
 * MPG_ALGO_BF16_CRT: the same residues, products and result (bit-identical
 * to MPG_ALGO_INT8_CRT), with the residues stored as bf16 (exact: |r| <= 128),
 * loaded by TMA and multiplied by tcgen05.mma (kind::f16, M = N = 128, fp32
 * accumulation in tensor memory); each accumulator is drained into an exact
 * int32 sum after at most 1024 values of k, so every fp32 partial sum is an
 * integer below 2^24.  Workspace: a 256-byte header whose first int32 is 0
 * after a normal run (else the code of the role whose bounded wait gave up,
 * read by mpgemm_tc_status), then the regions above with the residues of
 * op(A) and op(B)^T as bf16 (2 bytes each). */

/* beta of the CRT form for N moduli and inner dimension k (>= 1 when the
 * form applies, 0 when the moduli's product is too small); MPG_EINVAL for N
 * outside 1..49 or k < 0. */
int mpgemm_crt_beta(int moduli, int64_t k);

/* MPG_ALGO_INT8_CRT_SPLIT (not in the paper): the CRT form with each scaled
 * integer split in two, for about twice the bits that one integer product
 * of the same moduli can carry.  With N = opts->slices moduli (default 16 for
 * DD, 22 for TD, 30 for QD; 1..49):
 *   bits    beta = mpgemm_crt_split_beta(N, k) = 2w for the largest w with
 *           k 2^(2w) < M; MPG_EUNSUPPORTED when there is none or beta > 316.
 *   integers A', B' as for MPG_ALGO_INT8_CRT with this beta.
 *   split   A' = A1 2^w + A0 with A0 the representative of A' mod 2^w in
 *           [-2^(w-1), 2^(w-1)) and A1 = (A' - A0) / 2^w; B' likewise.
 *   products per modulus m_i, exact in int32 (k <= 65535, else
 *           MPG_EUNSUPPORTED): hh = r(A1) r(B1)^T, mid = r(A1) r(B0)^T +
 *           r(A0) r(B1)^T, ll = r(A0) r(B0)^T.
 *   recover P_hh, P_mid, P_ll = the integers in [-M/2, M/2) congruent to
 *           them (each is below k 2^(2w-1) < M/2 in magnitude), and
 *           C' = P_hh 2^(2w) + P_mid 2^w + P_ll = A'B' exactly.
 *   output  as for MPG_ALGO_INT8_CRT, with 2 beta = 4w.
 * 3N products of the residues instead of N, for twice the bits: with 30
 * moduli beta is about 210, enough for QD.  Workspace as for
 * MPG_ALGO_INT8_CRT with [2N] residue planes per operand (A1's residues for
 * m_0..m_(N-1), then A0's) and [3N] product planes (hh, mid, ll).
 * MPG_ALGO_BF16_CRT_SPLIT: the same on tcgen05 as MPG_ALGO_BF16_CRT (the
 * two middle sub-products add into one exact int32 sum), bit-identical. */
int mpgemm_crt_split_beta(int moduli, int64_t k);

/* After an MPG_ALGO_BF16_SLICES call with this workspace: synchronises the
 * calling thread's stream and returns the code in the workspace header.  0
 * after a normal run.  A positive code names the role whose bounded wait
 * (about a second) gave up, the kernel having then stopped every role and
 * released its resources: 1 the producer (a stage to refill), 2 the MMA
 * issuer (a free accumulator), 3 the MMA issuer (a loaded stage), 4 a drain
 * warp (a finished accumulator), 5 an adder warp (a finished group), 6 a
 * drain warp (a free hand-over buffer); C is then incomplete, and
 * mpgemm_last_error() says which.  MPG_EINVAL for a NULL workspace,
 * MPG_ECUDA if the header cannot be read. */
int mpgemm_tc_status(const void *workspace);

/* The Strassen form (Sec. 3: the paper's divide-and-conquer alternative to
 * the block algorithm).  With opts->strassen = L > 0, C := A B is computed
 * from Strassen's seven products of half-size blocks,
 *   M1 = (A11 + A22)(B11 + B22)   M2 = (A21 + A22) B11   M3 = A11 (B12 - B22)
 *   M4 = A22 (B21 - B11)          M5 = (A11 + A12) B22   M6 = (A21 - A11)(B11 + B12)
 *   M7 = (A12 - A22)(B21 + B22)
 *   C11 = ((M1 + M4) - M5) + M7   C12 = M3 + M5   C21 = M2 + M4
 *   C22 = ((M1 - M2) + M3) + M6,
 * applied L times while m, n and k are even (an odd or zero dimension ends the
 * recursion); the leaf products are the k-sequential GEMM of mpgemm_dd/td/qd.
 * "+" is the precision's addition (DDadd Alg. 1, TDaddq Sec. 2.3, QDadd
 * Alg. 5) elementwise, x - y is x + (-y) with every component of y negated,
 * and each sum is evaluated left to right.  The result is deterministic and
 * bit-identical to those steps evaluated anywhere; it is not bit-identical to
 * the block algorithm, and its error bound grows with L.  Workspace:
 * mpgemm_workspace_size bytes (256-byte aligned, not overlapping A, B or C):
 * per level P (m/2 k/2 + k/2 n/2 + 7 m/2 n/2) binary64 values. */

/* Bytes of workspace mpgemm_ex needs for these options and sizes (0 if none). */
size_t mpgemm_workspace_size(int P, const mpgemm_opts *opts, int64_t m, int64_t n, int64_t k);

/* ---------------------------------------------------------------------
 * Batched GEMM (not in the paper): many independent k-sequential products
 * C_i := op(A_i) op(B_i) of Sec. 3, Eq. 1, all in precision P, executed by
 * one persistent kernel launch that the plan captures in a CUDA graph.
 * Each C_i is bit-identical to mpgemm_ex on that problem alone.
 * ------------------------------------------------------------------- */
typedef struct mpgemm_problem {
    int64_t m, n, k;
    const double *A[4];   /* first P entries used; stored shapes as in mpgemm_ex */
    int64_t lda;
    const double *B[4];
    int64_t ldb;
    double *C[4];
    int64_t ldc;
    int trans_a, trans_b;
} mpgemm_problem;

typedef struct mpgemm_batch_plan mpgemm_batch_plan;

/* Workspace bytes a plan over these problems may need (any policy). */
size_t mpgemm_batch_workspace_size(int P, int count, const mpgemm_problem *problems);

/* Validate every problem (as mpgemm_ex; a bad one fails the whole call with
 * its message), split them into output tiles -- 16 x 16 for problems with
 * m*n below the policy's threshold, 32 x 32 otherwise; policy 0..4 =
 * threshold 0, 2048, 8192, 32768, never; policy 5 = 16 x 16 tiles throughout
 * with the error-free transformations on the integer pipes (TwoSum, and for
 * P = 2 FastTwoSum, as in mpgemm_tile_int_ops; same results) -- sort the
 * tiles by decreasing work,
 * copy the descriptors into `workspace` (device, 256-byte aligned, caller-
 * owned, kept alive and unmodified while the plan is used) on the current
 * stream and wait for that copy, and capture one persistent launch in a CUDA
 * graph.  The problems' matrices are not read until mpgemm_batch_run.
 * *out receives a host-side handle (free with mpgemm_batch_plan_destroy). */
int mpgemm_batch_plan_create(int P, int count, const mpgemm_problem *problems, int policy,
                             void *workspace, size_t workspace_bytes, mpgemm_batch_plan **out);

/* Replay the plan's graph on the calling thread's current stream.  Runs of
 * one plan must not overlap on the GPU (they share the tile counter). */
int mpgemm_batch_run(const mpgemm_batch_plan *plan);

/* info = {tiles, CTAs in the persistent grid, policy, problem count}. */
int mpgemm_batch_plan_info(const mpgemm_batch_plan *plan, int64_t info[4]);

int mpgemm_batch_plan_destroy(mpgemm_batch_plan *plan);

/* Autotuner: build a plan for every policy, time `reps` graph replays of
 * each on the current stream (writing the problems' C), and return the
 * fastest policy and its time per run in milliseconds.  The choice is
 * remembered for this exact list of shapes (see mpgemm_autotune): a later
 * call for the same list returns it without measuring (and writes no C). */
int mpgemm_batch_autotune(int P, int count, const mpgemm_problem *problems, void *workspace,
                          size_t workspace_bytes, int reps, int *best_policy, float *best_ms);

/* DD C := A B through the INT8 slicing form (as mpgemm_ex with
 * MPG_ALGO_INT8_OZAKI and no transposes) without a caller workspace.  The
 * paper has no counterpart: this call exists for callers that cannot
 * allocate device memory -- code running inside a host framework that owns
 * all device memory through its own pool and forbids raw allocations, or a
 * latency-critical loop that cannot afford cudaMalloc's implicit
 * synchronisation -- so it allocates no device memory and calls no cudaMalloc,
 * cudaFree or allocating library routine.
 * Its scratch is a fixed 32 MiB array inside the library, present on every
 * device that loads it until the process exits.  Products whose scratch
 * (mpgemm_workspace_size with algo MPG_ALGO_INT8_OZAKI) exceeds 32 MiB are
 * rejected with MPG_EWORKSPACE before anything is launched; e.g. DD
 * 1024 x 1024 x 1024 with 14 slices fits.  slices = 0 means 14.
 * First-call work: the first call in a device's context looks up the array's
 * device address (cudaGetSymbolAddress, with that device current), and the
 * first call of each host thread on a device creates the stream on which op(B)
 * is sliced and its two fork/join events (driver resources, not device
 * memory).  Make those first calls before any stream capture and outside
 * latency-critical loops.  A device reset (cudaDeviceReset) ends the context
 * the address and the stream belong to; the library notices the new context
 * (by its id) and repeats that first-call work on the next call, which should
 * then also come before any capture.  Every call uses the same array and each call
 * writes every scratch byte it reads, so a call never depends on what an
 * earlier one left there; but calls whose execution overlaps on the GPU
 * (different streams, or different host threads without ordering) race on
 * the array and must be serialised by the caller. */
int mpgemm_dd_int8_static(int64_t m, int64_t n, int64_t k,
                          const double *const A[2], int64_t lda,
                          const double *const B[2], int64_t ldb,
                          double *const C[2], int64_t ldc, int slices);

/* ---------------------------------------------------------------------
 * Autotuner (no counterpart in the paper).  Every FP64-EFT tile gives the
 * same k-sequential result, so the tile is a matter of speed and can be
 * chosen by measurement.  mpgemm_autotune times every tile id on the caller's
 * operands (`reps` calls each after one warm-up, CUDA events on the calling
 * thread's stream, synchronising; C is written with the same result every
 * time; not for use inside a stream capture), returns the fastest id and
 * its time in milliseconds, and remembers it for the device (name and SM
 * count), P and the shape's bucket: m, n and k each rounded up to a power of
 * two.  mpgemm_ex with algo AUTO or FP64_EFT and tile 0 then takes the
 * remembered tile of its bucket, before the rule of mpgemm_default_tile.
 * Choices live in memory and, when the environment variable
 * MPGEMM_TUNE_CACHE names a file, in that JSON file: read at the first
 * lookup, rewritten (through a temporary file and a rename) after every new
 * choice; lines that do not parse are ignored and a file that cannot be
 * written leaves the choices in memory.  The same cache holds the policies
 * of mpgemm_batch_autotune.  MPG_EINVAL when no tile can run the call (the
 * message of the last tile's refusal is kept).
 * ------------------------------------------------------------------- */
int mpgemm_autotune(int P, int64_t m, int64_t n, int64_t k,
                    const double *const *A, int64_t lda, const double *const *B, int64_t ldb,
                    double *const *C, int64_t ldc, int reps, int *best_tile, float *best_ms);
/* The remembered tile id (1-based) of the bucket of (P, m, n, k) on the
 * current device, or 0 if there is none. */
int mpgemm_tuned_tile(int P, int64_t m, int64_t n, int64_t k);
/* Forget the choices in memory; the next lookup reads MPGEMM_TUNE_CACHE
 * (as the environment then has it) again. */
void mpgemm_tune_cache_reset(void);

/* Number of FP64-EFT tile configurations for precision P (1..4), and a description
 * of configuration id (BM, BN, BK, TM, TN, threads); returns MPG_EINVAL for
 * an unknown id. */
int mpgemm_num_tiles(int P);
int mpgemm_tile_info(int P, int id, int info[6]);
/* Which error-free transformations (Sec. 2.1) tile `id` of precision P
 * computes on the integer pipes instead of as binary64 operation sequences
 * on the FP64 pipe: a mask of 1 TwoSum, 2 FastTwoSum (QuickTwoSum), 4
 * TwoProd; 0 for none.  Such a tile forms each transformation's two outputs
 * from one exact integer sum or product of the significands, with the bits
 * the operation sequence gives for every input (rare inputs -- non-finite,
 * overflowing, or a product error below the subnormal range -- run the
 * sequence itself), so every tile still returns the same C.  MPG_EINVAL for
 * an unknown id. */
int mpgemm_tile_int_ops(int P, int id);

/* The FP64-EFT tile id (1-based) that mpgemm_ex uses for an m x n x k product
 * when opts->tile is 0 and the autotuner remembers none: of the candidates (binary64-only: 64x64, 32x32,
 * 16x16, 8x8; DD: 32x32, 16x16, 8x8 staging 128 values of k; TD/QD: 16x16, 8x8), the first whose CTAs,
 * dealt round-robin to the device's SMs,
 * keep at least 90% of them busy -- ctas / (sms * ceil(ctas / sms)) -- else
 * the closest.  For P = 2, 3, 4 with m * n >= 256 * sms the candidates are
 * the 16x16 and 8x8 tiles that compute TwoSum (and for DD FastTwoSum) on the
 * integer pipes (mpgemm_tile_int_ops), which need that many outputs to hide
 * the integer pipes' latency.  Uses the current device's SM count (152 when
 * there is no device).  MPG_EINVAL for an unknown P or a negative
 * dimension. */
int mpgemm_default_tile(int P, int64_t m, int64_t n, int64_t k);

/* ---------------------------------------------------------------------
 * Measurement aid (no counterpart in the paper): pipe throughput probes used
 * as roofline denominators.  Launches `blocks` CTAs of 256 threads and writes
 * one double per thread to out[blocks * 256] (device, caller-owned); the
 * caller times the launch.
 *   kind 0/1/2: `iters` rounds of 8 independent binary64 add / mul / fma per
 *     thread with register operands; lane-operations = blocks*256*iters*8.
 *   kind 3: `iters` rounds of 4 independent mma.sync.m16n8k32 s8 per warp;
 *     int8 operations = blocks*8*iters*4*8192.
 *   kind 4/5/6: `iters` rounds of 4 independent TwoSum / FastTwoSum /
 *     TwoProd per thread computed on the integer pipes (the form of the tiles
 *     mpgemm_tile_int_ops reports); transformations = blocks*256*iters*4.
 * ------------------------------------------------------------------- */
int mpgemm_peak_probe(int kind, int blocks, int iters, double *out);

#ifdef __cplusplus
}
#endif
#endif /* MPGEMM_H */
