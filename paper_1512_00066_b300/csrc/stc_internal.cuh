// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <vector>

#include "stc.h"

// ----------------------------------------------------------------- handle

struct stc_handle {
    int device = 0;
    int num_sms = 0;
    int smem_optin = 0;  // max dynamic shared memory per block (opt-in)
    stc_alloc_fn alloc = nullptr;
    stc_free_fn free_fn = nullptr;
    void* ctx = nullptr;
    int* d_flags = nullptr;        // 64 device bytes: error flags (STC_FLAG_* bits) at 0,
                                   // the validation counters at STC_VAL_COUNTER_OFFSET
    int64_t* h_stage = nullptr;    // pinned host staging, 64 int64
    bool timing = false;           // record phase events
    cudaEvent_t ev[9] = {};        // phase boundary events (created on first use)
    int nphases = 0;               // phases recorded by the last timed call
    int64_t launches = 0;          // kernels launched by this handle
    int round_driver = 1;          // multi-round loops: 0 host-driven, 1 CUDA graph
    cudaStream_t aux = nullptr;    // second stream for concurrent launches (created on first use)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // Bellman-Ford CUDA graph per algebra (0: int32, 1: fp32), instantiated on the
    // first graph-driven call and reused by later ones: its kernels read their
    // arguments from the device parameter block, which each call rewrites
    cudaGraph_t bf_graph[2] = {};
    cudaGraphExec_t bf_exec[2] = {};
    void* d_params = nullptr;  // device parameter block, STC_PARAM_BYTES
    void* h_params = nullptr;  // pinned host staging of that block
    // tuned light-row threshold per (algebra, ceil(log2 output columns)): -128 unknown,
    // -1 no light launch, L > 0 rows with ub < 2^L
    signed char tune_light[6][40];
    stc_handle() {
        for (auto& row : tune_light)
            for (auto& x : row) x = -128;
    }
};

constexpr size_t STC_PARAM_BYTES = 4096;
constexpr size_t STC_VAL_COUNTER_OFFSET = 16;  // two u64 after the flag word

// The auxiliary stream; run work on it between stc_fork and stc_join (stream order
// of `s` is kept: the auxiliary work starts after what is queued on `s` and `s`
// resumes after it).
stc_status stc_fork(stc_handle* h, stc_stream s, cudaStream_t* aux);
stc_status stc_join(stc_handle* h, stc_stream s);
int stc_log2_ceil(int64_t x);

// Record phase boundary `idx` (0 = start of the call) when timing is enabled.
void stc_mark(stc_handle* h, stc_stream s, int idx);
// Count `n` kernel launches.
inline void stc_count(stc_handle* h, int n = 1) { h->launches += n; }

// Device-side error flag bits (accumulated with atomicOr).
enum : int {
    STC_FLAG_SHAPE = 1,
    STC_FLAG_UNSORTED = 2,
    STC_FLAG_TIMEOUT = 4,
    STC_FLAG_NEG_CYCLE = 8,
    STC_FLAG_INTERNAL = 16,
    STC_FLAG_INVALID = 32,
};

stc_status stc_flags_to_status(int flags);

void* stc_alloc_bytes(stc_handle* h, size_t bytes, stc_stream s);
void stc_free_bytes(stc_handle* h, void* p, stc_stream s);

// Scratch allocations released (stream-ordered) when the object goes out of scope.
struct StcScratch {
    stc_handle* h;
    stc_stream s;
    std::vector<void*> ptrs;
    bool failed = false;
    StcScratch(stc_handle* h_, stc_stream s_) : h(h_), s(s_) {}
    template <class T>
    T* get(size_t count) {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        void* p = stc_alloc_bytes(h, bytes, s);
        if (!p) { failed = true; return nullptr; }
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~StcScratch() {
        for (void* p : ptrs) stc_free_bytes(h, p, s);
    }
};

#define STC_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) { (void)cudaGetLastError(); return STC_ERR_CUDA; } \
    } while (0)

#define STC_LAUNCH_CHECK() STC_CUDA_TRY(cudaGetLastError())

// ----------------------------------------------------------------- CSR checks

stc_status stc_check_csr_host(const stc_csr* m);
// Enqueue the device-side validation of a CSR matrix; raises STC_FLAG_SHAPE /
// STC_FLAG_UNSORTED in h->d_flags.
stc_status stc_validate_csr_async(stc_handle* h, const stc_csr* m, stc_stream s);
// Validation of `count` matrices (host descriptors) in one launch.
stc_status stc_validate_many_async(stc_handle* h, StcScratch& sc, const stc_csr* mats, int count, stc_stream s);
// The same check raising its flags in `flags` (a device int); needs no handle.
// `counters` are two device u64, zero before the launch (the kernel leaves them zero).
stc_status stc_validate_csr_flags_async(const stc_csr* m, int* flags, unsigned long long* counters, int num_sms,
                                        stc_stream s);
// The handle's pair of validation counters.
unsigned long long* stc_val_counters(stc_handle* h);

// ----------------------------------------------------------------- algebra ids

constexpr int ALG_PT_F32 = STC_PLUS_TIMES_F32;
constexpr int ALG_PT_F64 = STC_PLUS_TIMES_F64;
constexpr int ALG_MP_I32 = STC_MIN_PLUS_I32;
constexpr int ALG_MP_F32 = STC_MIN_PLUS_F32;
constexpr int ALG_BOOL = STC_OR_AND_BOOL;
constexpr int ALG_MULTPATH = STC_MULTPATH_I32_F64;
// Internal algebra (not in stc_algebra): paths (w, h) of Tiskin's path doubling,
// (+) = lexicographic minimum of (w, h), (x) = (w1 + w2, h1 + h2).
constexpr int ALG_PATH = 6;
struct PathVal {
    int32_t w, h;
};

size_t stc_val_bytes(int alg, char operand);  // 'A', 'B' or 'C'

// ----------------------------------------------------------------- device helpers

#ifdef __CUDACC__

// (distance, multiplicity) element as loaded by the device: one 16-byte access.
struct __align__(16) DSig {
    int d;
    int pad;
    double s;
};

__device__ __forceinline__ void row_range(const int64_t* __restrict__ ptr, int64_t i, int64_t nnz,
                                          int64_t& lo, int64_t& hi) {
    int64_t a = ptr[i], b = ptr[i + 1];
    a = a < 0 ? 0 : (a > nnz ? nnz : a);
    b = b < a ? a : (b > nnz ? nnz : b);
    lo = a;
    hi = b;
}

// Monotone map of fp32 bit patterns to uint32: unsigned order equals float order
// (for non-NaN values).
__device__ __forceinline__ unsigned f32_to_ordered(float x) {
    unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_f32(unsigned k) {
    unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// Block-wide exclusive scan of one int per thread.  Returns the exclusive prefix;
// `total` receives the block sum.  s_warp must hold NT/32 + 1 ints.  Contains
// __syncthreads; every thread of the block must call it.
template <int NT, class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T w = lane < NT / 32 ? s_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) s_warp[lane] = w;  // inclusive warp prefix
        if (lane == NT / 32 - 1) s_warp[NT / 32] = w;
    }
    __syncthreads();
    T excl = x - v + (wid > 0 ? s_warp[wid - 1] : T(0));
    total = s_warp[NT / 32];
    __syncthreads();
    return excl;
}

#endif  // __CUDACC__

// ----------------------------------------------------------------- internal entry points

stc_status stc_spgemm_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                           const stc_opts* opts, stc_stream s);
stc_status stc_spgemm_batched_impl(stc_handle* h, int alg, int nb, const stc_csr* A, const stc_csr* B,
                                   stc_csr* C, const stc_opts* opts, stc_stream s);
stc_status stc_spmm_impl(stc_handle* h, int alg, const stc_csr* A, const void* X, int64_t ldx,
                         int32_t ncol, void* Y, int64_t ldy, int32_t accumulate, stc_stream s);
stc_status stc_apsp_tiskin_impl(stc_handle* h, const stc_csr* G, stc_csr* P_out, int32_t* rounds_out,
                                int64_t* products_out, stc_stream s);
stc_status stc_apsp_impl(stc_handle* h, const stc_csr* G, stc_csr* P_out, int32_t* squarings_out, stc_stream s);
stc_status stc_bellman_ford_impl(stc_handle* h, int alg, const stc_csr* G, int32_t source,
                                 void* dist, int32_t* rounds, int64_t* relaxations,
                                 int32_t persistent, stc_stream s);

stc_status stc_mfbc_sssp_impl(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsrc,
                              int32_t* d_out, double* sigma_out, int32_t* rounds_out, stc_stream s);
stc_status stc_mfbc_impl(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsrc, int32_t batch,
                         double* bc, stc_stream s);

stc_status stc_features_impl(stc_handle* h, StcScratch& sc, const stc_csr* A, const stc_csr* B, float* feat,
                             stc_stream s);
stc_status stc_mlp_forward_tc_impl(stc_handle* h, const float* w, const float* feat, int64_t n, float* y,
                                   stc_stream s);
stc_status stc_mlp_forward_impl(stc_handle* h, const float* w, const float* feat, int64_t n, float* y,
                                stc_stream s);
stc_status stc_mlp_grad_impl(stc_handle* h, const float* w, const float* feat, const float* target,
                             const int32_t* idx, int64_t n, float scale, float* grad, float* loss, stc_stream s);
stc_status stc_mlp_adam_impl(stc_handle* h, float* w, float* m, float* v, float* grad, int64_t step, float lr,
                             stc_stream s);
stc_status stc_spgemm_masked_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, const stc_csr* M,
                                  void* c_val, const stc_opts* opts, stc_stream s);
stc_status stc_autotune_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, int32_t* best_out,
                             int32_t* cand_out, float* ms_out, int32_t* ncand_out, stc_stream s);
stc_status stc_calibrate_accumulate_impl(stc_handle* h, int alg, double* rate, stc_stream s);
stc_status stc_row_counts_impl(stc_handle* h, const stc_csr* A, const stc_csr* B, int64_t* counts,
                               const stc_opts* opts, stc_stream s);
stc_status stc_spgemm_learned_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                                   const float* weights, float margin, stc_learned_stats* stats,
                                   const stc_opts* opts, stc_stream s);

// Inclusive scan in place of n int64 values (device), using scratch from sc.
stc_status stc_inclusive_scan_i64(stc_handle* h, StcScratch& sc, int64_t* data, int64_t n,
                                  stc_stream s);
