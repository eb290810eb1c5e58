// Bellman-Ford single-source shortest paths (Section 4.2): repeated tropical
// matrix-vector products P <- P (+) A (x) P, with A_ii = 0 keeping P's own
// entries, until no distance changes; a change in round |V| means a reachable
// negative cycle.
//
// The product is applied to the frontier only: in each round the out-edges of
// the vertices whose distance decreased in the previous round are relaxed with
// an atomic minimum on the distance vector, and a vertex whose distance
// decreased joins the next frontier once (a per-vertex round stamp).  Vertices
// at the additive identity never relax, so the fixed point is the one of full
// relaxation; for fp32 it is the minimum over paths of the rounded left-to-right
// path sums, because a rounded add is monotone in each operand.
//
// Two drivers: a host loop with one launch per round that reads the frontier
// size back each round, and one cooperative launch that runs every round with a
// grid barrier (bounded spin) and tests convergence on the device.
#include <cooperative_groups.h>

#include <mutex>

#include "stc_internal.cuh"

namespace {

constexpr int BF_NT = 512;
constexpr int BF_U = 8;  // out-edges per lane whose atomic minima are in flight together
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 22;  // iterations of ~0.5 us each (~2 s)

template <int ALG> struct BfT;
template <> struct BfT<ALG_MP_I32> {
    using W = int; using D = int;  // stored distance representation
    static __device__ __forceinline__ D init() { return STC_MIN_PLUS_I32_IDENTITY; }
    static __device__ __forceinline__ D zero() { return 0; }
    static __device__ __forceinline__ D relax(D du, W w) { return du + w; }
    static __device__ __forceinline__ D amin(D* p, D v) { return atomicMin(p, v); }
    static __device__ __forceinline__ bool less(D a, D b) { return a < b; }
};
template <> struct BfT<ALG_MP_F32> {
    using W = float; using D = unsigned;  // order-preserving key of the fp32 distance
    static __device__ __forceinline__ D init() { return f32_to_ordered(__int_as_float(0x7f800000)); }
    static __device__ __forceinline__ D zero() { return f32_to_ordered(0.0f); }
    static __device__ __forceinline__ D relax(D du, W w) {
        return f32_to_ordered(__fadd_rn(ordered_to_f32(du), w));
    }
    static __device__ __forceinline__ D amin(D* p, D v) { return atomicMin(p, v); }
    static __device__ __forceinline__ bool less(D a, D b) { return a < b; }
};

struct BfArgs {
    int64_t n, nnz;
    const int64_t* __restrict__ ptr;
    const int32_t* __restrict__ col;
    const void* __restrict__ w;
    int32_t* frontier[2];
    int* stamp;
    int* cnt;  // three rotating frontier counters
    unsigned long long* relax;  // edge relaxations performed
};

template <int ALG>
__global__ void k_bf_init(BfArgs a, typename BfT<ALG>::D* dist, int32_t source) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < a.n;
         v += int64_t(gridDim.x) * blockDim.x) {
        dist[v] = v == source ? BfT<ALG>::zero() : BfT<ALG>::init();
        a.stamp[v] = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.frontier[0][0] = source;
        a.cnt[0] = 1;
        a.cnt[1] = 0;
        a.cnt[2] = 0;
    }
}

// Relax the out-edges of frontier entries [0, cnt_cur); one warp per frontier
// vertex, lanes over its edges.  Warps are numbered across the grid.
template <int ALG>
__device__ __forceinline__ void relax_round(const BfArgs& a, typename BfT<ALG>::D* dist, int r,
                                            const int32_t* __restrict__ cur, int ncur,
                                            int32_t* __restrict__ next, int* cnt_next) {
    using T = BfT<ALG>;
    const int lane = threadIdx.x & 31;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const auto* W = static_cast<const typename T::W*>(a.w);
    unsigned long long nrelax = 0;
    for (int64_t e = warp; e < ncur; e += nwarps) {
        int32_t u = cur[e];
        int64_t lo, hi;
        row_range(a.ptr, u, a.nnz, lo, hi);
        nrelax += (unsigned long long)(hi - lo);
        typename T::D du = *(volatile typename T::D*)&dist[u];
        // BF_U edges a lane at a time, their atomics issued together (a hub's row
        // is long and sets the round's length)
        for (int64_t p0 = lo + lane; p0 < hi; p0 += 32 * BF_U) {
            int32_t v[BF_U];
            typename T::D cand[BF_U], old[BF_U];
#pragma unroll
            for (int k = 0; k < BF_U; ++k) {
                const int64_t p = p0 + 32 * k;
                v[k] = -1;
                if (p < hi) {
                    const int32_t x = a.col[p];
                    if ((uint64_t)x < (uint64_t)a.n) {
                        v[k] = x;
                        cand[k] = T::relax(du, W[p]);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < BF_U; ++k)
                if (v[k] >= 0) old[k] = T::amin(&dist[v[k]], cand[k]);
#pragma unroll
            for (int k = 0; k < BF_U; ++k)
                if (v[k] >= 0 && T::less(cand[k], old[k]) && atomicExch(&a.stamp[v[k]], r) != r)
                    next[atomicAdd(cnt_next, 1)] = v[k];
        }
    }
    if (lane == 0 && nrelax) atomicAdd(a.relax, nrelax);
}

template <int ALG>
__global__ void __launch_bounds__(BF_NT) k_bf_round(BfArgs a, typename BfT<ALG>::D* dist, int r) {
    const int ncur = a.cnt[r % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[(r + 2) % 3] = 0;  // counter of round r+2's frontier
    relax_round<ALG>(a, dist, r, a.frontier[r & 1], ncur, a.frontier[(r + 1) & 1], &a.cnt[(r + 1) % 3]);
}

// Grid-wide barrier of `expected` blocks (gridDim.x in the solvers) with a
// bounded spin: after spin_limit polls of ~0.5 us it gives up, raises
// STC_FLAG_TIMEOUT and returns false, so a block that never arrives ends the
// kernel with a status instead of a hang.
__device__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned expected, long long spin_limit, int* flags,
                             int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g0 = *(volatile unsigned*)gen;
        __threadfence();
        unsigned arrived = atomicAdd(count, 1u);
        if (arrived == expected - 1) {
            *(volatile unsigned*)count = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*(volatile unsigned*)gen == g0) {
                if (++spins > spin_limit) {
                    ok = 0;
                    atomicOr(flags, STC_FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Failure-detection self test: every block of a cooperative launch enters a grid
// barrier that expects `expected` blocks; passed counts the blocks that got
// through.
__global__ void k_barrier_selftest(unsigned* bar, unsigned expected, long long spin_limit, int* flags,
                                   int* passed) {
    __shared__ int s_ok;
    if (grid_barrier(&bar[0], &bar[1], expected, spin_limit, flags, &s_ok) && threadIdx.x == 0)
        atomicAdd(passed, 1);
}

template <int ALG>
__global__ void __launch_bounds__(BF_NT) k_bf_persistent(BfArgs a, typename BfT<ALG>::D* dist,
                                                         unsigned* bar, int* flags, int* rounds_out) {
    __shared__ int s_ok;
    int r = 0;
    int changed_rounds = 0;
    for (;;) {
        const int ncur = *(volatile int*)&a.cnt[r % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[(r + 2) % 3] = 0;
        relax_round<ALG>(a, dist, r, a.frontier[r & 1], ncur, a.frontier[(r + 1) & 1],
                         &a.cnt[(r + 1) % 3]);
        if (!grid_barrier(&bar[0], &bar[1], gridDim.x, BARRIER_SPIN_LIMIT, flags, &s_ok)) return;
        const int nnext = *(volatile int*)&a.cnt[(r + 1) % 3];
        if (nnext == 0) break;
        ++changed_rounds;
        ++r;
        if (int64_t(changed_rounds) >= a.n) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flags, STC_FLAG_NEG_CYCLE);
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *rounds_out = changed_rounds;
}

// Arguments of the cached graph's kernels, read from the handle's device
// parameter block (rewritten by every call before the graph is launched).
struct BfGraphParams {
    BfArgs a;
    void* dist;
    int* d_round;
    int* d_changed;
};

template <int ALG>
__global__ void __launch_bounds__(BF_NT) k_bf_round_g(const BfGraphParams* __restrict__ p) {
    using D = typename BfT<ALG>::D;
    const BfArgs a = p->a;
    D* dist = static_cast<D*>(p->dist);
    const int r = *p->d_round;
    const int ncur = a.cnt[r % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[(r + 2) % 3] = 0;
    relax_round<ALG>(a, dist, r, a.frontier[r & 1], ncur, a.frontier[(r + 1) & 1], &a.cnt[(r + 1) % 3]);
}

// Termination test of the graph form (one thread): stop when the round produced
// an empty frontier, or flag a negative cycle when |V| rounds all changed
// something; otherwise advance the round and run the body again.
__global__ void k_bf_check_g(const BfGraphParams* __restrict__ p, int* flags, cudaGraphConditionalHandle loop) {
    const BfArgs a = p->a;
    const int r = *p->d_round;
    const int nnext = a.cnt[(r + 1) % 3];
    unsigned go = 0;
    if (nnext > 0) {
        const int changed = *p->d_changed + 1;
        *p->d_changed = changed;
        if (int64_t(changed) >= a.n) {
            atomicOr(flags, STC_FLAG_NEG_CYCLE);
        } else {
            *p->d_round = r + 1;
            go = 1;
        }
    }
    cudaGraphSetConditional(loop, go);
}

// The cached graph of algebra ALG: WHILE{k_bf_round_g -> k_bf_check_g}, built and
// instantiated once per handle; its kernel arguments are the parameter block.
template <int ALG>
cudaError_t bf_graph_exec(stc_handle* h, cudaGraphExec_t* out) {
    const int idx = ALG == ALG_MP_I32 ? 0 : 1;
    if (h->bf_exec[idx]) {
        *out = h->bf_exec[idx];
        return cudaSuccess;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    do {
        if (e != cudaSuccess) break;
        cudaGraphConditionalHandle loop;
        if ((e = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode, n1, n2;
        if ((e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp)) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        const BfGraphParams* params = static_cast<const BfGraphParams*>(h->d_params);
        int* flags = h->d_flags;
        void* round_args[] = {&params};
        cudaKernelNodeParams kp = {};
        kp.func = (void*)k_bf_round_g<ALG>;
        kp.gridDim = dim3(h->num_sms * 4);
        kp.blockDim = dim3(BF_NT);
        kp.kernelParams = round_args;
        if ((e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &kp)) != cudaSuccess) break;
        void* check_args[] = {&params, &flags, &loop};
        cudaKernelNodeParams kc = {};
        kc.func = (void*)k_bf_check_g;
        kc.gridDim = dim3(1);
        kc.blockDim = dim3(1);
        kc.kernelParams = check_args;
        if ((e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &kc)) != cudaSuccess) break;
        e = cudaGraphInstantiate(&exec, graph, 0);
    } while (0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        return e;
    }
    h->bf_graph[idx] = graph;
    h->bf_exec[idx] = exec;
    *out = exec;
    return cudaSuccess;
}

template <int ALG>
__global__ void k_bf_finish(int64_t n, const typename BfT<ALG>::D* key, void* out) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += int64_t(gridDim.x) * blockDim.x) {
        if (ALG == ALG_MP_F32)
            static_cast<float*>(out)[v] = ordered_to_f32(static_cast<unsigned>(key[v]));
    }
}

template <int ALG>
stc_status run_bf(stc_handle* h, const stc_csr* G, int32_t source, void* dist_out, int32_t* rounds_out,
                  int64_t* relax_out, int persistent, stc_stream s) {
    using D = typename BfT<ALG>::D;
    StcScratch sc(h, s);
    const int64_t n = G->nrows;
    BfArgs a;
    a.n = n;
    a.nnz = G->nnz;
    a.ptr = G->rowptr;
    a.col = G->col;
    a.w = G->val;
    a.frontier[0] = sc.get<int32_t>(size_t(n));
    a.frontier[1] = sc.get<int32_t>(size_t(n));
    a.stamp = sc.get<int>(size_t(n));
    int* ints = sc.get<int>(16);  // [0..2] counters, [4..5] barrier, [6] rounds, [8..9] relaxations,
                                  // [10] round and [11] changed rounds of the graph form
    D* dist = ALG == ALG_MP_I32 ? reinterpret_cast<D*>(dist_out) : sc.get<D>(size_t(n));
    if (sc.failed) return STC_ERR_OOM;
    a.cnt = ints;
    a.relax = reinterpret_cast<unsigned long long*>(ints + 8);
    stc_mark(h, s, 0);
    STC_CUDA_TRY(cudaMemsetAsync(ints, 0, 16 * sizeof(int), s));
    stc_status st = stc_validate_csr_async(h, G, s);
    if (st != STC_OK) return st;
    int64_t blocks = (n + 255) / 256;
    if (blocks > int64_t(h->num_sms) * 8) blocks = int64_t(h->num_sms) * 8;
    k_bf_init<ALG><<<unsigned(blocks), 256, 0, s>>>(a, dist, source);
    STC_LAUNCH_CHECK();
    stc_count(h);
    stc_mark(h, s, 1);

    int rounds = 0;
    if (persistent == 1) {
        int per_sm = 0;
        STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bf_persistent<ALG>, BF_NT, 0));
        if (per_sm < 1) return STC_ERR_CUDA;
        int grid = per_sm * h->num_sms;
        unsigned* bar = reinterpret_cast<unsigned*>(ints + 4);
        int* flags = h->d_flags;
        int* d_rounds = ints + 6;
        void* args[] = {&a, &dist, &bar, &flags, &d_rounds};
        STC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_bf_persistent<ALG>, dim3(grid), dim3(BF_NT),
                                                 args, 0, s));
        stc_count(h);
        stc_mark(h, s, 2);
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[0], d_rounds, sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[2], a.relax, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[1], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        rounds = reinterpret_cast<int*>(&h->h_stage[0])[0];
    } else if (persistent == 2) {
        // graph form: the handle's cached graph (conditional WHILE node repeating
        // {round, check}); this call's arguments go to its parameter block first
        static_assert(sizeof(BfGraphParams) <= STC_PARAM_BYTES, "parameter block");
        int* d_round = ints + 10;
        int* d_changed = ints + 11;
        cudaGraphExec_t exec = nullptr;
        STC_CUDA_TRY(bf_graph_exec<ALG>(h, &exec));
        BfGraphParams* hp = static_cast<BfGraphParams*>(h->h_params);
        hp->a = a;
        hp->dist = dist;
        hp->d_round = d_round;
        hp->d_changed = d_changed;
        STC_CUDA_TRY(cudaMemcpyAsync(h->d_params, hp, sizeof(BfGraphParams), cudaMemcpyHostToDevice, s));
        STC_CUDA_TRY(cudaGraphLaunch(exec, s));
        stc_count(h, 2);  // the body's two kernels (repeated on the device)
        stc_mark(h, s, 2);
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[0], d_changed, sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[1], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[2], a.relax, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        rounds = reinterpret_cast<int*>(&h->h_stage[0])[0];
    } else {
        // plain form: one launch per round, frontier size read back each round
        int grid = h->num_sms * 4;
        int* h_cnt = reinterpret_cast<int*>(&h->h_stage[0]);
        for (int r = 0;; ++r) {
            k_bf_round<ALG><<<grid, BF_NT, 0, s>>>(a, dist, r);
            STC_LAUNCH_CHECK();
            stc_count(h);
            STC_CUDA_TRY(cudaMemcpyAsync(h_cnt, &a.cnt[(r + 1) % 3], sizeof(int), cudaMemcpyDeviceToHost, s));
            STC_CUDA_TRY(cudaStreamSynchronize(s));
            if (*h_cnt == 0) break;
            ++rounds;
            if (int64_t(rounds) >= n) {
                int f = STC_FLAG_NEG_CYCLE;
                STC_CUDA_TRY(cudaMemcpyAsync(h->d_flags, &f, sizeof(int), cudaMemcpyHostToDevice, s));
                break;
            }
        }
        stc_mark(h, s, 2);
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[1], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[2], a.relax, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (ALG == ALG_MP_F32) {
        k_bf_finish<ALG><<<unsigned(blocks), 256, 0, s>>>(n, dist, dist_out);
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    if (rounds_out) *rounds_out = rounds;
    if (relax_out) *relax_out = h->h_stage[2];
    int flags = reinterpret_cast<int*>(&h->h_stage[1])[0];
    if (flags) {
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(flags);
    }
    return STC_OK;
}

}  // namespace

stc_status stc_bellman_ford_impl(stc_handle* h, int alg, const stc_csr* G, int32_t source, void* dist,
                                 int32_t* rounds, int64_t* relax, int32_t persistent, stc_stream s) {
    if (alg == ALG_MP_I32) return run_bf<ALG_MP_I32>(h, G, source, dist, rounds, relax, persistent, s);
    return run_bf<ALG_MP_F32>(h, G, source, dist, rounds, relax, persistent, s);
}

extern "C" stc_status stc_selftest_barrier(stc_handle* h, int32_t missing, int32_t spin_limit,
                                           stc_stream s) {
    if (!h || missing < 0 || missing > 1 || spin_limit < 1 || spin_limit > (1 << 24)) return STC_ERR_INVALID_ARG;
    StcScratch sc(h, s);
    int* ints = sc.get<int>(4);  // [0..1] barrier, [2] passed
    if (!ints) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(ints, 0, 4 * sizeof(int), s));
    unsigned* bar = reinterpret_cast<unsigned*>(ints);
    unsigned expected = 2u + unsigned(missing);
    long long limit = spin_limit;
    int* flags = h->d_flags;
    int* passed = ints + 2;
    void* args[] = {&bar, &expected, &limit, &flags, &passed};
    STC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_barrier_selftest, dim3(2), dim3(32), args, 0, s));
    stc_count(h);
    int* st = reinterpret_cast<int*>(&h->h_stage[0]);
    st[0] = st[1] = 0;
    STC_CUDA_TRY(cudaMemcpyAsync(&st[0], passed, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaMemcpyAsync(&st[1], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    if (st[1]) {
        const int f = st[1];
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(f);
    }
    return st[0] == 2 ? STC_OK : STC_ERR_CUDA;
}

// ----------------------------------------------------------------- allocation-free variant
//
// stc_bellman_ford_noalloc serves callers that cannot allocate device memory
// while they run (host callbacks, real-time loops, processes that hand out
// memory only from fixed pools).  It runs the same kernels as the persistent
// driver above, with every piece of working memory carved from one file-scope
// device array instead of the handle's allocator.

namespace {

// Header of the scratch array (bytes):
//   [0, 12)   int[0..2]   frontier and work counters
//   [16, 24)  int[4..5]   grid-barrier state
//   [24, 28)  int[6]      round count
//   [28, 32)  int[7]      device flags
//   [32, 48)  u64[2]      CSR validation counters
//   [64, 72)  u64         relaxation counter (written by every round, not read back)
// then, per vertex, the two frontier slots, the round stamp and the fp32 distance key.
constexpr size_t NOALLOC_HEADER = 256;
constexpr size_t NOALLOC_RELAX_OFFSET = 64;
static_assert(NOALLOC_RELAX_OFFSET + sizeof(unsigned long long) <= NOALLOC_HEADER,
              "the relaxation counter must sit inside the cleared header");
constexpr size_t NOALLOC_VAL_OFFSET = 32;
static_assert(8 * sizeof(int) <= NOALLOC_VAL_OFFSET, "the validation counters follow the flags");
static_assert(NOALLOC_VAL_OFFSET + 2 * sizeof(unsigned long long) <= NOALLOC_RELAX_OFFSET,
              "the counters and flags must end before the relaxation counter");
// per vertex: two frontier slots, a round stamp and an fp32 distance key
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + size_t(STC_NOALLOC_BF_MAX_VERTICES) * 16;

// Held by every GPU that loads the library, until the process exits.  Host code
// must not pass this name to a kernel: on the host it is only a stand-in symbol.
// Its device address is looked up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_bf_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set-up on first use).
stc_status noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return STC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bf_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return STC_ERR_CUDA;
        }
        g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_addr[dev];
    return STC_OK;
}

template <int ALG>
stc_status run_bf_noalloc(const stc_csr* G, int32_t source, void* dist_out, int32_t* rounds_out,
                          stc_stream s) {
    using D = typename BfT<ALG>::D;
    const int64_t n = G->nrows;
    int dev = 0, num_sms = 0;
    STC_CUDA_TRY(cudaGetDevice(&dev));
    STC_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned char* base = nullptr;
    stc_status st = noalloc_scratch(dev, &base);
    if (st != STC_OK) return st;
    int* ints = reinterpret_cast<int*>(base);  // [0..2] counters, [4..5] barrier, [6] rounds, [7] flags
    BfArgs a;
    a.n = n;
    a.nnz = G->nnz;
    a.ptr = G->rowptr;
    a.col = G->col;
    a.w = G->val;
    a.cnt = ints;
    a.relax = reinterpret_cast<unsigned long long*>(base + NOALLOC_RELAX_OFFSET);
    a.frontier[0] = reinterpret_cast<int32_t*>(base + NOALLOC_HEADER);
    a.frontier[1] = a.frontier[0] + n;
    a.stamp = a.frontier[1] + n;
    D* dist = ALG == ALG_MP_I32 ? reinterpret_cast<D*>(dist_out) : reinterpret_cast<D*>(a.stamp + n);
    unsigned* bar = reinterpret_cast<unsigned*>(ints + 4);
    int* d_rounds = ints + 6;
    int* flags = ints + 7;

    // the previous call's counters, barrier state and flags are left behind: clear them
    STC_CUDA_TRY(cudaMemsetAsync(base, 0, NOALLOC_HEADER, s));
    if ((st = stc_validate_csr_flags_async(G, flags,
                                           reinterpret_cast<unsigned long long*>(base + NOALLOC_VAL_OFFSET), num_sms,
                                           s)) != STC_OK)
        return st;
    int64_t blocks = (n + 255) / 256;
    if (blocks > int64_t(num_sms) * 8) blocks = int64_t(num_sms) * 8;
    k_bf_init<ALG><<<unsigned(blocks), 256, 0, s>>>(a, dist, source);
    STC_LAUNCH_CHECK();
    int per_sm = 0;
    STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bf_persistent<ALG>, BF_NT, 0));
    if (per_sm < 1) return STC_ERR_CUDA;
    void* args[] = {&a, &dist, &bar, &flags, &d_rounds};
    STC_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_bf_persistent<ALG>, dim3(per_sm * num_sms),
                                             dim3(BF_NT), args, 0, s));
    if (ALG == ALG_MP_F32) {
        k_bf_finish<ALG><<<unsigned(blocks), 256, 0, s>>>(n, dist, dist_out);
        STC_LAUNCH_CHECK();
    }
    int host[2] = {0, 0};  // rounds, flags
    STC_CUDA_TRY(cudaMemcpyAsync(host, d_rounds, sizeof(host), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    if (rounds_out) *rounds_out = host[0];
    return host[1] ? stc_flags_to_status(host[1]) : STC_OK;
}

}  // namespace

extern "C" stc_status stc_bellman_ford_noalloc(stc_algebra alg, const stc_csr* G, int32_t source,
                                               void* dist_out, int32_t* rounds_out, stc_stream stream) {
    if (!dist_out) return STC_ERR_INVALID_ARG;
    if (alg != STC_MIN_PLUS_I32 && alg != STC_MIN_PLUS_F32) return STC_ERR_ALGEBRA;
    stc_status st = stc_check_csr_host(G);
    if (st != STC_OK) return st;
    if (G->nrows != G->ncols) return STC_ERR_SHAPE;
    if (G->nrows > STC_NOALLOC_BF_MAX_VERTICES) return STC_ERR_CAPACITY;
    if (source < 0 || source >= G->nrows) return STC_ERR_INVALID_ARG;
    if (alg == STC_MIN_PLUS_I32) return run_bf_noalloc<ALG_MP_I32>(G, source, dist_out, rounds_out, stream);
    return run_bf_noalloc<ALG_MP_F32>(G, source, dist_out, rounds_out, stream);
}
