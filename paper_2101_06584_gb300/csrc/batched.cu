// batched.cu -- many uneven FP64-EFT GEMMs in one persistent launch.
//
// Not in the paper.  A plan turns `count` problems C_i := op(A_i) op(B_i)
// (each a k-sequential DD/TD/QD product of Sec. 3, Eq. 1) into one list of
// output tiles, sorted by decreasing work, and stores it with the problem
// descriptors in a caller-provided device workspace.  A persistent kernel
// with one or more CTAs per SM claims tiles in that order through an atomic
// counter (no spin-waits; the last CTA to finish resets the counter for the
// next launch), so large tiles start first and small ones fill the tail.
// Each tile is computed exactly as by mpgemm_ex, so every C_i is
// bit-identical to its separate k-sequential product.  The plan captures the
// single launch in a CUDA graph; running the plan replays the graph.
//
// Tile kinds: 0 = 16 x 16 outputs, 1 thread each; 1 = 32 x 32 outputs, 2 x 2
// per thread; both 256 threads.  A policy decides the kind per problem:
// kind 1 when m * n >= threshold(policy), else kind 0.  Policies 0-4 run the
// arithmetic on the FP64 pipe; policy 5 puts every problem in 16 x 16 tiles
// whose transformations run on the integer pipes as in the GEMM tiles of
// mpgemm_tile_int_ops (TwoSum, and for DD FastTwoSum), same bits.
#include "mpgemm.h"
#include "gemm_kernel.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace mpg {

namespace {

struct BatchItem {
    int problem;
    int kind;
    int tile_m;
    int tile_n;
};

template <int P>
struct BatchDev {
    unsigned* counters;          // [0] next item, [1] CTAs finished
    const GemmArgs<P>* probs;
    const BatchItem* items;
    int n_items;
};

constexpr int kNumPolicies = 6;
constexpr int kIntPolicy = 5;
const int64_t kPolicyThreshold[kNumPolicies] = {0, 2048, 8192, 32768, INT64_MAX, INT64_MAX};

// The transformations policy kIntPolicy computes on the integer pipes.
template <int P>
constexpr unsigned int_mask() { return P == 2 ? 3u : 1u; }

template <int P>
__host__ __device__ constexpr size_t batch_smem_bytes()
{
    return sizeof(KseqSmem<P, 32, 32, 16>) > sizeof(KseqSmem<P, 16, 16, 16>)
               ? sizeof(KseqSmem<P, 32, 32, 16>)
               : sizeof(KseqSmem<P, 16, 16, 16>);
}

// The persistent loop.  INTS: the transformations on the integer pipes
// (mp::RnInt's mask); with a nonzero mask every item is a 16 x 16 tile.
template <int P, unsigned INTS>
__device__ __forceinline__ void batched_body(const BatchDev<P>& b)
{
    __shared__ __align__(16) unsigned char smem[batch_smem_bytes<P>()];
    __shared__ int s_item;
    const mp::RnInt<INTS> f(mp::make_rn());
    for (;;) {
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(&b.counters[0], 1u));
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= b.n_items) break;
        const BatchItem w = b.items[it];
        const GemmArgs<P> g = b.probs[w.problem];
        if (INTS != 0u || w.kind == 0) {
            kseq_tile<P, 16, 16, 16, 1, 1>(g, static_cast<int64_t>(w.tile_m) * 16,
                                           static_cast<int64_t>(w.tile_n) * 16,
                                           *reinterpret_cast<KseqSmem<P, 16, 16, 16>*>(smem), f);
        } else if constexpr (INTS == 0u) {
            kseq_tile<P, 32, 32, 16, 2, 2>(g, static_cast<int64_t>(w.tile_m) * 32,
                                           static_cast<int64_t>(w.tile_n) * 32,
                                           *reinterpret_cast<KseqSmem<P, 32, 32, 16>*>(smem), f);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&b.counters[1], 1u);
        if (done == gridDim.x - 1) {
            atomicExch(&b.counters[0], 0u);
            atomicExch(&b.counters[1], 0u);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(256) batched_kernel(const BatchDev<P> b)
{
    batched_body<P, 0u>(b);
}

// Policy kIntPolicy.  Three CTAs per SM (at most 85 registers, as the GEMM's
// own 16 x 16 integer-pipe tile uses) give the integer pipes the warps that
// hide their latency.
template <int P>
__global__ void __launch_bounds__(256, 3) batched_int_kernel(const BatchDev<P> b)
{
    batched_body<P, int_mask<P>()>(b);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <int P>
size_t problems_bytes(int count) { return align256(sizeof(GemmArgs<P>) * static_cast<size_t>(count)); }

int64_t tiles_of(int64_t m, int64_t n, int kind)
{
    const int64_t t = kind == 0 ? 16 : 32;
    return ((m + t - 1) / t) * ((n + t - 1) / t);
}

}  // namespace

struct BatchPlanImpl {
    int P = 0, count = 0, policy = 0, n_items = 0, grid = 0, device = -1;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

template <int P>
static int build_plan(int count, const mpgemm_problem* probs, int policy, void* ws, size_t bytes,
                      BatchPlanImpl* plan)
{
    std::vector<GemmArgs<P>> args(static_cast<size_t>(count));
    std::vector<BatchItem> items;
    std::vector<double> work;
    for (int i = 0; i < count; ++i) {
        const mpgemm_problem& q = probs[i];
        GemmArgs<P>& g = args[static_cast<size_t>(i)];
        for (int c = 0; c < P; ++c) {
            g.A[c] = q.A[c];
            g.B[c] = q.B[c];
            g.C[c] = q.C[c];
        }
        g.m = q.m; g.n = q.n; g.k = q.k; g.lda = q.lda; g.ldb = q.ldb; g.ldc = q.ldc;
        g.trans_a = q.trans_a != 0;
        g.trans_b = q.trans_b != 0;
        const int rc = check_gemm<P>(g);
        if (rc != MPG_OK) return rc;
        if (g.m == 0 || g.n == 0) continue;
        const int kind = (g.m * g.n >= kPolicyThreshold[policy]) ? 1 : 0;
        const int t = kind == 0 ? 16 : 32;
        for (int64_t tm = 0; tm * t < g.m; ++tm)
            for (int64_t tn = 0; tn * t < g.n; ++tn) {
                items.push_back({i, kind, static_cast<int>(tm), static_cast<int>(tn)});
                const int64_t rows = std::min<int64_t>(t, g.m - tm * t);
                const int64_t cols = std::min<int64_t>(t, g.n - tn * t);
                // k = 0 tiles still write zeros: give them a token cost
                work.push_back(static_cast<double>(rows * cols) * static_cast<double>(g.k > 0 ? g.k : 1));
            }
    }
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b2) { return work[a] > work[b2]; });
    std::vector<BatchItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];

    const size_t need = 256 + problems_bytes<P>(count) + align256(sizeof(BatchItem) * sorted.size());
    if (need > bytes) {
        char msg[160];
        snprintf(msg, sizeof(msg), "batch workspace of %zu bytes is smaller than the %zu needed", bytes, need);
        return set_error(MPG_EWORKSPACE, msg);
    }
    unsigned char* base = static_cast<unsigned char*>(ws);
    BatchDev<P> d;
    d.counters = reinterpret_cast<unsigned*>(base);
    d.probs = reinterpret_cast<const GemmArgs<P>*>(base + 256);
    d.items = reinterpret_cast<const BatchItem*>(base + 256 + problems_bytes<P>(count));
    d.n_items = static_cast<int>(sorted.size());

    // upload (synchronously: the host vectors go out of scope)
    cudaStream_t s = current_stream();
    const unsigned zero[2] = {0u, 0u};
    cudaError_t e = cudaMemcpyAsync(base, zero, sizeof(zero), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && count)
        e = cudaMemcpyAsync(base + 256, args.data(), sizeof(GemmArgs<P>) * args.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !sorted.empty())
        e = cudaMemcpyAsync(base + 256 + problems_bytes<P>(count), sorted.data(),
                            sizeof(BatchItem) * sorted.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(MPG_ECUDA, cudaGetErrorString(e));

    const bool ints = policy == kIntPolicy;
    int per_sm = 0;
    e = ints ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_int_kernel<P>, 256, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<P>, 256, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int grid = num_sms() * per_sm;
    if (grid > d.n_items) grid = d.n_items > 0 ? d.n_items : 1;

    // one launch, captured in a graph
    e = cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (ints) batched_int_kernel<P><<<grid, 256, 0, plan->cap_stream>>>(d);
        else batched_kernel<P><<<grid, 256, 0, plan->cap_stream>>>(d);
        const cudaError_t le = cudaGetLastError();
        e = cudaStreamEndCapture(plan->cap_stream, &plan->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
    if (e != cudaSuccess) return set_error(MPG_ECUDA, cudaGetErrorString(e));

    plan->P = P;
    plan->count = count;
    plan->policy = policy;
    plan->n_items = d.n_items;
    plan->grid = grid;
    plan->ws = ws;
    plan->ws_bytes = bytes;
    cudaGetDevice(&plan->device);
    return MPG_OK;
}

template <int P>
static size_t batch_ws_size(int count, const mpgemm_problem* probs)
{
    // the largest tile list of any policy: every problem in 16 x 16 tiles
    size_t items = 0;
    for (int i = 0; i < count; ++i)
        if (probs[i].m > 0 && probs[i].n > 0) items += static_cast<size_t>(tiles_of(probs[i].m, probs[i].n, 0));
    return 256 + problems_bytes<P>(count) + align256(sizeof(BatchItem) * items);
}

static void release(BatchPlanImpl* p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    delete p;
}

}  // namespace mpg

using namespace mpg;

struct mpgemm_batch_plan : BatchPlanImpl {};

extern "C" {

size_t mpgemm_batch_workspace_size(int P, int count, const mpgemm_problem* problems)
{
    if (count < 0 || (count > 0 && !problems)) return 0;
    switch (P) {
    case 2: return batch_ws_size<2>(count, problems);
    case 3: return batch_ws_size<3>(count, problems);
    case 4: return batch_ws_size<4>(count, problems);
    default: return 0;
    }
}

int mpgemm_batch_plan_create(int P, int count, const mpgemm_problem* problems, int policy,
                             void* workspace, size_t workspace_bytes, mpgemm_batch_plan** out)
{
    clear_error();
    if (!out) return set_error(MPG_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (P < 2 || P > 4) return set_error(MPG_EINVAL, "P must be 2, 3 or 4");
    if (count < 0 || (count > 0 && !problems)) return set_error(MPG_EINVAL, "bad problem list");
    if (policy < 0 || policy >= kNumPolicies) return set_error(MPG_EINVAL, "policy must be in 0..5");
    if (!workspace) return set_error(MPG_EWORKSPACE, "a batch needs a workspace");
    if (reinterpret_cast<uintptr_t>(workspace) % 256)
        return set_error(MPG_EWORKSPACE, "workspace must be 256-byte aligned");
    mpgemm_batch_plan* plan = new (std::nothrow) mpgemm_batch_plan();
    if (!plan) return set_error(MPG_EINVAL, "out of host memory");
    int rc;
    switch (P) {
    case 2: rc = build_plan<2>(count, problems, policy, workspace, workspace_bytes, plan); break;
    case 3: rc = build_plan<3>(count, problems, policy, workspace, workspace_bytes, plan); break;
    default: rc = build_plan<4>(count, problems, policy, workspace, workspace_bytes, plan); break;
    }
    if (rc != MPG_OK) {
        release(plan);
        return rc;
    }
    *out = plan;
    return MPG_OK;
}

int mpgemm_batch_run(const mpgemm_batch_plan* plan)
{
    clear_error();
    if (!plan || !plan->exec) return set_error(MPG_EINVAL, "not a prepared plan");
    const cudaError_t e = cudaGraphLaunch(plan->exec, current_stream());
    return e == cudaSuccess ? MPG_OK : set_error(MPG_ECUDA, cudaGetErrorString(e));
}

int mpgemm_batch_plan_info(const mpgemm_batch_plan* plan, int64_t info[4])
{
    clear_error();
    if (!plan || !info) return set_error(MPG_EINVAL, "NULL argument");
    info[0] = plan->n_items;
    info[1] = plan->grid;
    info[2] = plan->policy;
    info[3] = plan->count;
    return MPG_OK;
}

int mpgemm_batch_plan_destroy(mpgemm_batch_plan* plan)
{
    release(plan);
    return MPG_OK;
}

int mpgemm_batch_autotune(int P, int count, const mpgemm_problem* problems, void* workspace,
                          size_t workspace_bytes, int reps, int* best_policy, float* best_ms)
{
    clear_error();
    if (!best_policy) return set_error(MPG_EINVAL, "best_policy must not be NULL");
    if (reps < 1) reps = 1;
    // a remembered choice for this exact list of shapes (FNV-1a over m, n, k
    // and the transposes of every problem) is returned without measuring
    char key[512] = "";
    if (problems && count > 0) {
        uint64_t h = 1469598103934665603ull;
        auto mix = [&](int64_t v) {
            for (int b = 0; b < 8; ++b) {
                h ^= static_cast<uint64_t>(v >> (8 * b)) & 0xffu;
                h *= 1099511628211ull;
            }
        };
        for (int i = 0; i < count; ++i) {
            mix(problems[i].m);
            mix(problems[i].n);
            mix(problems[i].k);
            mix(problems[i].trans_a * 2 + problems[i].trans_b);
        }
        batch_tune_key(P, count, h, key, sizeof(key));
        int pol = -1;
        float ms = 0.f;
        if (tune_lookup(key, &pol, &ms) && pol >= 0 && pol < kNumPolicies) {
            *best_policy = pol;
            if (best_ms) *best_ms = ms;
            return MPG_OK;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(MPG_ECUDA, "event creation failed");
    float best = 0.f;
    int arg = -1;
    int rc = MPG_OK;
    for (int pol = 0; pol < kNumPolicies && rc == MPG_OK; ++pol) {
        mpgemm_batch_plan* plan = nullptr;
        rc = mpgemm_batch_plan_create(P, count, problems, pol, workspace, workspace_bytes, &plan);
        if (rc != MPG_OK) break;
        cudaStream_t s = current_stream();
        rc = mpgemm_batch_run(plan);                       // warm-up
        if (rc == MPG_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && rc == MPG_OK; ++r) rc = mpgemm_batch_run(plan);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(MPG_ECUDA, "timing failed");
        }
        if (rc == MPG_OK) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= static_cast<float>(reps);
            if (arg < 0 || ms < best) { best = ms; arg = pol; }
        }
        mpgemm_batch_plan_destroy(plan);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MPG_OK) return rc;
    if (key[0]) tune_store(key, arg, best);
    *best_policy = arg;
    if (best_ms) *best_ms = best;
    return MPG_OK;
}

}  // extern "C"
