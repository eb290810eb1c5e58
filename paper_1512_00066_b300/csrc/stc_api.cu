// C-ABI entry points, handle, allocator plumbing, CSR validation and the
// device-wide scan used to turn per-row counts into row pointers.
#include <cstdio>
#include <cstring>
#include <vector>

#include "stc_internal.cuh"

// ----------------------------------------------------------------- statuses

static const char* k_status_text[] = {
    "ok",
    "invalid argument",
    "shape mismatch or malformed row pointers",
    "columns not strictly ascending or out of range",
    "algebra not supported by this entry point",
    "allocation failed",
    "CUDA runtime error",
    "negative cycle reachable from the source",
    "bounded device-side wait timed out",
    "graph larger than the fixed scratch of the allocation-free entry point",
};

extern "C" const char* stc_status_str(stc_status s) {
    int i = static_cast<int>(s);
    if (i < 0 || i >= static_cast<int>(sizeof(k_status_text) / sizeof(k_status_text[0])))
        return "unknown status";
    return k_status_text[i];
}

extern "C" int32_t stc_version(void) { return 100; }

stc_status stc_flags_to_status(int f) {
    if (f & STC_FLAG_SHAPE) return STC_ERR_SHAPE;
    if (f & STC_FLAG_UNSORTED) return STC_ERR_UNSORTED;
    if (f & STC_FLAG_TIMEOUT) return STC_ERR_TIMEOUT;
    if (f & STC_FLAG_NEG_CYCLE) return STC_ERR_NEG_CYCLE;
    if (f & STC_FLAG_INTERNAL) return STC_ERR_CUDA;
    if (f & STC_FLAG_INVALID) return STC_ERR_INVALID_ARG;
    return STC_OK;
}

size_t stc_val_bytes(int alg, char operand) {
    switch (alg) {
    case ALG_PT_F32: return 4;
    case ALG_PT_F64: return 8;
    case ALG_MP_I32: return 4;
    case ALG_MP_F32: return 4;
    case ALG_BOOL: return 1;
    case ALG_MULTPATH: return operand == 'A' ? 4 : 16;
    case ALG_PATH: return 8;
    default: return 0;
    }
}

// ----------------------------------------------------------------- handle

extern "C" stc_status stc_create(stc_handle** out, stc_alloc_fn alloc, stc_free_fn free_fn,
                                 void* ctx) {
    if (!out) return STC_ERR_INVALID_ARG;
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return STC_ERR_INVALID_ARG;
    stc_handle* h = new stc_handle();
    h->alloc = alloc;
    h->free_fn = free_fn;
    h->ctx = ctx;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) !=
            cudaSuccess ||
        cudaMalloc(&h->d_flags, 64) != cudaSuccess ||
        cudaMemset(h->d_flags, 0, 64) != cudaSuccess ||
        cudaMallocHost(&h->h_stage, 64 * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&h->d_params, STC_PARAM_BYTES) != cudaSuccess ||
        cudaMallocHost(&h->h_params, STC_PARAM_BYTES) != cudaSuccess) {
        (void)cudaGetLastError();
        if (h->d_flags) cudaFree(h->d_flags);
        if (h->h_stage) cudaFreeHost(h->h_stage);
        if (h->d_params) cudaFree(h->d_params);
        delete h;
        return STC_ERR_CUDA;
    }
    *out = h;
    return STC_OK;
}

stc_status stc_fork(stc_handle* h, stc_stream s, cudaStream_t* aux) {
    if (!h->aux) {
        STC_CUDA_TRY(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        STC_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        STC_CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    STC_CUDA_TRY(cudaEventRecord(h->ev_fork, s));
    STC_CUDA_TRY(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    *aux = h->aux;
    return STC_OK;
}

stc_status stc_join(stc_handle* h, stc_stream s) {
    STC_CUDA_TRY(cudaEventRecord(h->ev_join, h->aux));
    STC_CUDA_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
    return STC_OK;
}

int stc_log2_ceil(int64_t x) {
    int l = 0;
    while (l < 62 && (int64_t(1) << l) < x) ++l;
    return l;
}

extern "C" void stc_destroy(stc_handle* h) {
    if (!h) return;
    if (h->aux) {
        cudaStreamSynchronize(h->aux);
        cudaStreamDestroy(h->aux);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    for (int a = 0; a < 2; ++a) {
        if (h->bf_exec[a]) cudaGraphExecDestroy(h->bf_exec[a]);
        if (h->bf_graph[a]) cudaGraphDestroy(h->bf_graph[a]);
    }
    if (h->d_flags) cudaFree(h->d_flags);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    if (h->d_params) cudaFree(h->d_params);
    if (h->h_params) cudaFreeHost(h->h_params);
    delete h;
}

void* stc_alloc_bytes(stc_handle* h, size_t bytes, stc_stream s) {
    if (bytes == 0) bytes = 16;
    if (h->alloc) return h->alloc(bytes, h->ctx, s);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

void stc_free_bytes(stc_handle* h, void* p, stc_stream s) {
    if (!p) return;
    if (h->free_fn) h->free_fn(p, h->ctx, s);
    else (void)cudaFreeAsync(p, s);
}

extern "C" void stc_free(stc_handle* h, void* ptr, stc_stream stream) {
    if (h) stc_free_bytes(h, ptr, stream);
}

extern "C" stc_status stc_check_device_status(stc_handle* h, stc_stream s) {
    if (!h) return STC_ERR_INVALID_ARG;
    int f = 0;
    STC_CUDA_TRY(cudaMemcpyAsync(&f, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
    return stc_flags_to_status(f);
}

// ----------------------------------------------------------------- instrumentation

void stc_mark(stc_handle* h, stc_stream s, int idx) {
    if (!h->timing || idx < 0 || idx >= 9) return;
    if (!h->ev[idx] && cudaEventCreate(&h->ev[idx]) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    if (cudaEventRecord(h->ev[idx], s) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    h->nphases = idx;
}

extern "C" stc_status stc_set_timing(stc_handle* h, int32_t enable) {
    if (!h) return STC_ERR_INVALID_ARG;
    h->timing = enable != 0;
    h->nphases = 0;
    return STC_OK;
}

extern "C" int32_t stc_phase_times(stc_handle* h, float* ms_out, int32_t max_phases) {
    if (!h || !h->timing || h->nphases <= 0) return 0;
    int n = h->nphases;
    if (cudaEventSynchronize(h->ev[n]) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    for (int i = 0; i < n && i < max_phases; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) != cudaSuccess) {
            (void)cudaGetLastError();
            ms = -1.f;
        }
        if (ms_out) ms_out[i] = ms;
    }
    return n;
}

extern "C" int64_t stc_kernel_launches(const stc_handle* h) { return h ? h->launches : 0; }

// ----------------------------------------------------------------- CSR validation

stc_status stc_check_csr_host(const stc_csr* m) {
    if (!m) return STC_ERR_INVALID_ARG;
    if (m->nrows < 0 || m->ncols < 0 || m->nnz < 0) return STC_ERR_INVALID_ARG;
    if (m->nrows >= INT32_MAX || m->ncols > INT32_MAX) return STC_ERR_INVALID_ARG;
    if (!m->rowptr) return STC_ERR_INVALID_ARG;
    if (m->nnz > 0 && (!m->col || !m->val)) return STC_ERR_INVALID_ARG;
    return STC_OK;
}

// Validation works on a flat index over each matrix's row pointers and columns:
// element e < nrows checks row e's pointer pair (0 <= ptr[e] <= ptr[e+1] <= nnz),
// element nrows + p checks column p (0 <= col[p] < ncols).  Order: a position p > 0
// with col[p-1] >= col[p] (a descent) is legal only where a row opens.  Every
// non-empty row opens at a distinct position, so the columns are strictly ascending
// within rows exactly when the number of descents equals the number of descents
// at row openings; elements add +1 per descent and -1 per descent at an opening
// into a counter, and the last block to finish checks it for zero and clears it.
// A block takes VAL_TILE consecutive elements of one matrix; `tile0` numbers each
// matrix's first tile, and in a batch tile_mat[tile] names the tile's matrix.
struct CsrView {
    int64_t nrows, ncols, nnz;
    const int64_t* ptr;
    const int32_t* col;
    int64_t tile0;
};

constexpr int VAL_NT = 256;
constexpr int VAL_PER = 8;
constexpr int64_t VAL_TILE = int64_t(VAL_NT) * VAL_PER;

static int64_t val_tiles(int64_t nrows, int64_t nnz) {
    const int64_t t = (nrows + nnz + VAL_TILE - 1) / VAL_TILE;
    return t > 0 ? t : 1;
}

// Eight blocks per SM at most, striding over the tiles.
static unsigned val_grid(int64_t tiles, int num_sms) {
    const int64_t cap = int64_t(num_sms > 0 ? num_sms : 1) * 8;
    return unsigned(tiles < cap ? tiles : cap);
}

// Tile t of matrix m: raises flag bits in `bad`, adds descents minus descents at row
// openings to `net`.
__device__ __forceinline__ void val_tile(const CsrView& m, int64_t t, int& bad, long long& net) {
    if (t == 0 && threadIdx.x == 0 && (m.ptr[0] != 0 || m.ptr[m.nrows] != m.nnz)) bad |= STC_FLAG_SHAPE;
    const int64_t e0 = t * VAL_TILE + threadIdx.x;  // this thread's elements: e0 + j * VAL_NT
    const int64_t nel = m.nrows + m.nnz;
    if (t * VAL_TILE >= m.nrows && m.nnz > 0) {
        // a tile of entries only: every load is issued before any is used (indexes
        // clamped into the array; out-of-range elements are masked afterwards)
        const int64_t p0 = e0 - m.nrows;
        int32_t c[VAL_PER], cp[VAL_PER];
#pragma unroll
        for (int j = 0; j < VAL_PER; ++j) {
            int64_t p = p0 + int64_t(j) * VAL_NT;
            p = p < m.nnz ? p : m.nnz - 1;
            c[j] = m.col[p];
            cp[j] = m.col[p > 0 ? p - 1 : 0];
        }
#pragma unroll
        for (int j = 0; j < VAL_PER; ++j) {
            const int64_t p = p0 + int64_t(j) * VAL_NT;
            if (p < m.nnz) {
                if (c[j] < 0 || c[j] >= m.ncols) bad |= STC_FLAG_UNSORTED;
                if (p > 0 && cp[j] >= c[j]) ++net;
            }
        }
    } else if ((t + 1) * VAL_TILE <= m.nrows) {
        // a tile of row pointers only
        int64_t lo[VAL_PER], hi[VAL_PER];
#pragma unroll
        for (int j = 0; j < VAL_PER; ++j) {
            const int64_t r = e0 + int64_t(j) * VAL_NT;
            lo[j] = m.ptr[r];
            hi[j] = m.ptr[r + 1];
        }
        int32_t a[VAL_PER], c[VAL_PER];
#pragma unroll
        for (int j = 0; j < VAL_PER; ++j) {
            const bool ok = lo[j] >= 0 && hi[j] >= lo[j] && hi[j] <= m.nnz;
            if (!ok) bad |= STC_FLAG_SHAPE;
            const bool opens = ok && lo[j] > 0 && lo[j] < hi[j];
            a[j] = opens ? m.col[lo[j] - 1] : 0;
            c[j] = opens ? m.col[lo[j]] : 1;
        }
#pragma unroll
        for (int j = 0; j < VAL_PER; ++j)
            if (a[j] >= c[j]) --net;
    } else {
        // the tile where the row pointers end and the entries begin
        for (int j = 0; j < VAL_PER; ++j) {
            const int64_t e = e0 + int64_t(j) * VAL_NT;
            if (e < m.nrows) {
                const int64_t lo = m.ptr[e], hi = m.ptr[e + 1];
                if (lo < 0 || hi < lo || hi > m.nnz) bad |= STC_FLAG_SHAPE;
                else if (lo > 0 && lo < hi && m.col[lo - 1] >= m.col[lo]) --net;
            } else if (e < nel) {
                const int64_t p = e - m.nrows;
                const int32_t c = m.col[p];
                if (c < 0 || c >= m.ncols) bad |= STC_FLAG_UNSORTED;
                if (p > 0 && m.col[p - 1] >= c) ++net;
            }
        }
    }
}

// views == null: the single matrix `one` (tile0 = 0).  Blocks stride over the
// `tiles` tiles (one counter update per block).  cnt: [0] the descent balance (two's
// complement), [1] finished blocks; zero before the launch, zero after it.
__global__ void __launch_bounds__(VAL_NT) k_validate_tiles(CsrView one, const CsrView* __restrict__ views,
                                                           const int* __restrict__ tile_mat, int64_t tiles,
                                                           int* flags, unsigned long long* cnt) {
    __shared__ long long s_net[VAL_NT / 32];
    int bad = 0;
    long long net = 0;
    for (int64_t tg = blockIdx.x; tg < tiles; tg += gridDim.x) {
        const CsrView m = views ? views[tile_mat[tg]] : one;
        val_tile(m, tg - m.tile0, bad, net);
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) net += __shfl_xor_sync(0xffffffffu, net, o);
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(flags, bad);
        s_net[threadIdx.x >> 5] = net;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long tot = 0;
        for (int w = 0; w < VAL_NT / 32; ++w) tot += s_net[w];
        if (tot) atomicAdd(&cnt[0], static_cast<unsigned long long>(tot));
        __threadfence();
        if (atomicAdd(&cnt[1], 1ull) == gridDim.x - 1ull) {
            __threadfence();
            if (atomicAdd(&cnt[0], 0ull) != 0ull) atomicOr(flags, STC_FLAG_UNSORTED);
            cnt[0] = 0ull;
            cnt[1] = 0ull;
        }
    }
}

static CsrView view_of(const stc_csr* m) {
    return CsrView{m->nrows, m->ncols, m->nnz, m->rowptr, m->col, 0};
}

unsigned long long* stc_val_counters(stc_handle* h) {
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(h->d_flags) +
                                                 STC_VAL_COUNTER_OFFSET);
}

stc_status stc_validate_csr_async(stc_handle* h, const stc_csr* m, stc_stream s) {
    const stc_status st = stc_validate_csr_flags_async(m, h->d_flags, stc_val_counters(h), h->num_sms, s);
    if (st == STC_OK) stc_count(h);
    return st;
}

// Validation of many matrices in one launch.
stc_status stc_validate_many_async(stc_handle* h, StcScratch& sc, const stc_csr* mats, int count, stc_stream s) {
    if (count == 1) return stc_validate_csr_async(h, mats, s);
    std::vector<CsrView> v(count);
    int64_t tiles = 0;
    for (int i = 0; i < count; ++i) {
        v[i] = view_of(mats + i);
        v[i].tile0 = tiles;
        tiles += val_tiles(mats[i].nrows, mats[i].nnz);
    }
    if (tiles > INT32_MAX) return STC_ERR_INVALID_ARG;
    std::vector<int> tm(static_cast<size_t>(tiles));
    for (int i = 0; i < count; ++i) {
        const int64_t end = i + 1 < count ? v[i + 1].tile0 : tiles;
        for (int64_t t = v[i].tile0; t < end; ++t) tm[size_t(t)] = i;
    }
    CsrView* d = sc.get<CsrView>(size_t(count));
    int* d_tm = sc.get<int>(size_t(tiles));
    if (sc.failed) return STC_ERR_OOM;
    // copies from pageable memory return once the source has been staged, so the
    // host vectors may go out of scope right after them
    STC_CUDA_TRY(cudaMemcpyAsync(d, v.data(), sizeof(CsrView) * count, cudaMemcpyHostToDevice, s));
    STC_CUDA_TRY(cudaMemcpyAsync(d_tm, tm.data(), sizeof(int) * size_t(tiles), cudaMemcpyHostToDevice, s));
    k_validate_tiles<<<val_grid(tiles, h->num_sms), VAL_NT, 0, s>>>(CsrView{}, d, d_tm, tiles, h->d_flags,
                                                                     stc_val_counters(h));
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

// Same validation with the flag word and the two counters supplied by the caller
// (no handle).
stc_status stc_validate_csr_flags_async(const stc_csr* m, int* flags, unsigned long long* counters, int num_sms,
                                        stc_stream s) {
    const int64_t tiles = val_tiles(m->nrows, m->nnz);
    if (tiles > INT32_MAX) return STC_ERR_INVALID_ARG;
    k_validate_tiles<<<val_grid(tiles, num_sms), VAL_NT, 0, s>>>(view_of(m), nullptr, nullptr, tiles, flags,
                                                                  counters);
    STC_LAUNCH_CHECK();
    return STC_OK;
}

// ----------------------------------------------------------------- scan

constexpr int SCAN_NT = 512;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_TILE = SCAN_NT * SCAN_PER_THREAD;

// Phase 1: inclusive scan of each tile in place; tile totals to `part`.
__global__ void __launch_bounds__(SCAN_NT) k_scan_tiles(int64_t* data, int64_t n, int64_t* part) {
    __shared__ int64_t s_warp[SCAN_NT / 32 + 1];
    int64_t base = int64_t(blockIdx.x) * SCAN_TILE + int64_t(threadIdx.x) * SCAN_PER_THREAD;
    int64_t v[SCAN_PER_THREAD];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER_THREAD; ++j) {
        int64_t idx = base + j;
        v[j] = idx < n ? data[idx] : 0;
        sum += v[j];
        v[j] = sum;
    }
    int64_t total;
    int64_t excl = block_exclusive_scan<SCAN_NT, int64_t>(sum, s_warp, total);
#pragma unroll
    for (int j = 0; j < SCAN_PER_THREAD; ++j) {
        int64_t idx = base + j;
        if (idx < n) data[idx] = v[j] + excl;
    }
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Phase 2: one block turns the tile totals into exclusive tile offsets.
__global__ void __launch_bounds__(SCAN_NT) k_scan_parts(int64_t* part, int64_t nparts) {
    __shared__ int64_t s_warp[SCAN_NT / 32 + 1];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < nparts; b += SCAN_NT) {
        int64_t idx = b + threadIdx.x;
        int64_t v = idx < nparts ? part[idx] : 0;
        int64_t total;
        int64_t excl = block_exclusive_scan<SCAN_NT, int64_t>(v, s_warp, total);
        int64_t carry = s_carry;
        if (idx < nparts) part[idx] = carry + excl;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + total;
        __syncthreads();
    }
}

// Phase 3: add each tile's offset.
__global__ void __launch_bounds__(SCAN_NT) k_scan_add(int64_t* data, int64_t n, const int64_t* part) {
    if (blockIdx.x == 0) return;
    int64_t off = part[blockIdx.x];
    int64_t base = int64_t(blockIdx.x) * SCAN_TILE;
    for (int j = threadIdx.x; j < SCAN_TILE; j += SCAN_NT) {
        int64_t idx = base + j;
        if (idx < n) data[idx] += off;
    }
}

stc_status stc_inclusive_scan_i64(stc_handle* h, StcScratch& sc, int64_t* data, int64_t n,
                                  stc_stream s) {
    if (n <= 0) return STC_OK;
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t* part = sc.get<int64_t>(size_t(tiles));
    if (!part) return STC_ERR_OOM;
    k_scan_tiles<<<(unsigned)tiles, SCAN_NT, 0, s>>>(data, n, part);
    STC_LAUNCH_CHECK();
    stc_count(h);
    if (tiles > 1) {
        k_scan_parts<<<1, SCAN_NT, 0, s>>>(part, tiles);
        STC_LAUNCH_CHECK();
        k_scan_add<<<(unsigned)tiles, SCAN_NT, 0, s>>>(data, n, part);
        STC_LAUNCH_CHECK();
        stc_count(h, 2);
    }
    return STC_OK;
}

// ----------------------------------------------------------------- public entry points

static bool alg_valid(int alg) { return alg >= 0 && alg <= ALG_MULTPATH; }

extern "C" stc_status stc_contract_spgemm(stc_handle* h, stc_algebra alg, const stc_csr* A,
                                          const stc_csr* B, stc_csr* C, const stc_opts* opts,
                                          stc_stream stream) {
    if (!h || !C) return STC_ERR_INVALID_ARG;
    if (!alg_valid(alg)) return STC_ERR_ALGEBRA;
    stc_status st = stc_check_csr_host(A);
    if (st != STC_OK) return st;
    if ((st = stc_check_csr_host(B)) != STC_OK) return st;
    if (A->ncols != B->nrows) return STC_ERR_SHAPE;
    if (opts) {
        for (int r : opts->reserved)
            if (r != 0) return STC_ERR_INVALID_ARG;
        if (opts->light_rows < -1 || opts->light_rows > 30) return STC_ERR_INVALID_ARG;
        int w = opts->window_cols;
        if (w != 0 && (w < 1024 || (w & (w - 1)) != 0)) return STC_ERR_INVALID_ARG;
    }
    return stc_spgemm_impl(h, alg, A, B, C, opts, stream);
}

extern "C" stc_status stc_contract_spgemm_batched(stc_handle* h, stc_algebra alg, int32_t nbatch,
                                                  const stc_csr* A, const stc_csr* B, stc_csr* C,
                                                  const stc_opts* opts, stc_stream stream) {
    if (!h || !A || !B || !C || nbatch < 1 || nbatch > 65535) return STC_ERR_INVALID_ARG;
    if (!alg_valid(alg)) return STC_ERR_ALGEBRA;
    int64_t rows = 0;
    for (int32_t b = 0; b < nbatch; ++b) {
        stc_status st = stc_check_csr_host(&A[b]);
        if (st != STC_OK) return st;
        if ((st = stc_check_csr_host(&B[b])) != STC_OK) return st;
        if (A[b].ncols != B[b].nrows) return STC_ERR_SHAPE;
        if (B[b].ncols > (1 << 18)) return STC_ERR_INVALID_ARG;
        rows += A[b].nrows;
    }
    if (rows >= INT32_MAX) return STC_ERR_INVALID_ARG;
    if (opts)
        for (int r : opts->reserved)
            if (r != 0) return STC_ERR_INVALID_ARG;
        if (opts->light_rows < -1 || opts->light_rows > 30) return STC_ERR_INVALID_ARG;
    return stc_spgemm_batched_impl(h, alg, nbatch, A, B, C, opts, stream);
}

extern "C" stc_status stc_contract_spmm(stc_handle* h, stc_algebra alg, const stc_csr* A,
                                        const void* X, int64_t ldx, int32_t ncol, void* Y,
                                        int64_t ldy, int32_t accumulate, stc_stream stream) {
    if (!h) return STC_ERR_INVALID_ARG;
    if (!alg_valid(alg)) return STC_ERR_ALGEBRA;
    stc_status st = stc_check_csr_host(A);
    if (st != STC_OK) return st;
    if (ncol < 0 || ldx < ncol || ldy < ncol) return STC_ERR_INVALID_ARG;
    if (ncol > 0 && A->nrows > 0 && !Y) return STC_ERR_INVALID_ARG;
    if (ncol > 0 && A->ncols > 0 && !X) return STC_ERR_INVALID_ARG;
    return stc_spmm_impl(h, alg, A, X, ldx, ncol, Y, ldy, accumulate, stream);
}

extern "C" stc_status stc_contract_spmv(stc_handle* h, stc_algebra alg, const stc_csr* A,
                                        const void* x, void* y, int32_t accumulate,
                                        stc_stream stream) {
    return stc_contract_spmm(h, alg, A, x, 1, 1, y, 1, accumulate, stream);
}

extern "C" stc_status stc_bellman_ford(stc_handle* h, stc_algebra alg, const stc_csr* G,
                                       int32_t source, void* dist_out, int32_t* rounds_out,
                                       int64_t* relaxations_out, int32_t persistent,
                                       stc_stream stream) {
    if (!h || !dist_out) return STC_ERR_INVALID_ARG;
    if (alg != STC_MIN_PLUS_I32 && alg != STC_MIN_PLUS_F32) return STC_ERR_ALGEBRA;
    stc_status st = stc_check_csr_host(G);
    if (st != STC_OK) return st;
    if (G->nrows != G->ncols) return STC_ERR_SHAPE;
    if (source < 0 || source >= G->nrows) return STC_ERR_INVALID_ARG;
    if (persistent < 0 || persistent > 2) return STC_ERR_INVALID_ARG;
    return stc_bellman_ford_impl(h, alg, G, source, dist_out, rounds_out, relaxations_out, persistent,
                                 stream);
}

static stc_status mfbc_args(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsources) {
    if (!h || !sources || nsources <= 0 || !G) return STC_ERR_INVALID_ARG;
    // val may be NULL here: unit lengths
    stc_csr structure = *G;
    if (!structure.val) structure.val = structure.col;
    stc_status st = stc_check_csr_host(&structure);
    if (st != STC_OK) return st;
    if (G->nrows != G->ncols) return STC_ERR_SHAPE;
    for (int32_t i = 0; i < nsources; ++i)
        if (sources[i] < 0 || sources[i] >= G->nrows) return STC_ERR_INVALID_ARG;
    return STC_OK;
}

extern "C" stc_status stc_mfbc_sssp(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsources,
                                    int32_t* d_out, double* sigma_out, int32_t* rounds_out, stc_stream stream) {
    stc_status st = mfbc_args(h, G, sources, nsources);
    if (st != STC_OK) return st;
    if (nsources > 256 || !d_out || !sigma_out) return STC_ERR_INVALID_ARG;
    return stc_mfbc_sssp_impl(h, G, sources, nsources, d_out, sigma_out, rounds_out, stream);
}

extern "C" stc_status stc_contract_spgemm_masked(stc_handle* h, stc_algebra alg, const stc_csr* A,
                                                 const stc_csr* B, const stc_csr* M, void* c_val,
                                                 const stc_opts* opts, stc_stream stream) {
    if (!h || !M) return STC_ERR_INVALID_ARG;
    if (!alg_valid(alg)) return STC_ERR_ALGEBRA;
    stc_status st = stc_check_csr_host(A);
    if (st != STC_OK) return st;
    if ((st = stc_check_csr_host(B)) != STC_OK) return st;
    stc_csr mstruct = *M;  // the mask's values are not read
    if (!mstruct.val) mstruct.val = mstruct.col;
    if ((st = stc_check_csr_host(&mstruct)) != STC_OK) return st;
    if (A->ncols != B->nrows || M->nrows != A->nrows || M->ncols != B->ncols) return STC_ERR_SHAPE;
    if (M->nnz > 0 && !c_val) return STC_ERR_INVALID_ARG;
    if (opts) {
        for (int r : opts->reserved)
            if (r != 0) return STC_ERR_INVALID_ARG;
        if (opts->window_cols != 0 || opts->light_rows < -1 || opts->light_rows > 30) return STC_ERR_INVALID_ARG;
    }
    return stc_spgemm_masked_impl(h, alg, A, B, M, c_val, opts, stream);
}

extern "C" stc_status stc_apsp_path_doubling(stc_handle* h, const stc_csr* G, stc_csr* P_out,
                                             int32_t* squarings_out, stc_stream stream) {
    if (!h || !P_out) return STC_ERR_INVALID_ARG;
    stc_status st = stc_check_csr_host(G);
    if (st != STC_OK) return st;
    if (G->nrows != G->ncols) return STC_ERR_SHAPE;
    return stc_apsp_impl(h, G, P_out, squarings_out, stream);
}

extern "C" stc_status stc_apsp_tiskin(stc_handle* h, const stc_csr* G, stc_csr* P_out, int32_t* rounds_out,
                                      int64_t* products_out, stc_stream stream) {
    if (!h || !P_out) return STC_ERR_INVALID_ARG;
    stc_status st = stc_check_csr_host(G);
    if (st != STC_OK) return st;
    if (G->nrows != G->ncols) return STC_ERR_SHAPE;
    return stc_apsp_tiskin_impl(h, G, P_out, rounds_out, products_out, stream);
}

extern "C" stc_status stc_autotune_spgemm(stc_handle* h, stc_algebra alg, const stc_csr* A, const stc_csr* B,
                                          int32_t* best_out, int32_t* cand_out, float* ms_out, int32_t* ncand_out,
                                          stc_stream stream) {
    if (!h) return STC_ERR_INVALID_ARG;
    if (!alg_valid(alg)) return STC_ERR_ALGEBRA;
    stc_status st = stc_check_csr_host(A);
    if (st != STC_OK) return st;
    if ((st = stc_check_csr_host(B)) != STC_OK) return st;
    if (A->ncols != B->nrows) return STC_ERR_SHAPE;
    return stc_autotune_impl(h, alg, A, B, best_out, cand_out, ms_out, ncand_out, stream);
}

// Tuning files: "stc-tune 1 <SM count> <device name, blanks as '_'>" then lines
// "<algebra> <ceil(log2 columns)> <light-row threshold>".
static void device_tag(int device, char* name, size_t n) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(name, n, "unknown");
        return;
    }
    snprintf(name, n, "%s", prop.name);
    for (char* c = name; *c; ++c)
        if (*c == ' ' || *c == '\t') *c = '_';
}

extern "C" stc_status stc_tune_save(const stc_handle* h, const char* path) {
    if (!h || !path) return STC_ERR_INVALID_ARG;
    char name[256];
    device_tag(h->device, name, sizeof(name));
    FILE* f = fopen(path, "w");
    if (!f) return STC_ERR_INVALID_ARG;
    fprintf(f, "stc-tune 1 %d %s\n", h->num_sms, name);
    for (int a = 0; a < 6; ++a)
        for (int c = 0; c < 40; ++c)
            if (h->tune_light[a][c] != -128) fprintf(f, "%d %d %d\n", a, c, int(h->tune_light[a][c]));
    const bool ok = fclose(f) == 0;
    return ok ? STC_OK : STC_ERR_INVALID_ARG;
}

extern "C" stc_status stc_tune_load(stc_handle* h, const char* path) {
    if (!h || !path) return STC_ERR_INVALID_ARG;
    FILE* f = fopen(path, "r");
    if (!f) return STC_ERR_INVALID_ARG;
    char magic[32], dev[256], name[256];
    int version = 0, sms = 0;
    if (fscanf(f, "%31s %d %d %255s", magic, &version, &sms, dev) != 4 || strcmp(magic, "stc-tune") != 0 ||
        version != 1) {
        fclose(f);
        return STC_ERR_INVALID_ARG;
    }
    device_tag(h->device, name, sizeof(name));
    if (sms != h->num_sms || strcmp(dev, name) != 0) {
        fclose(f);
        return STC_ERR_INVALID_ARG;
    }
    signed char t[6][40];
    memcpy(t, h->tune_light, sizeof(t));
    int a, c, v;
    int n;
    while ((n = fscanf(f, "%d %d %d", &a, &c, &v)) == 3) {
        if (a < 0 || a >= 6 || c < 0 || c >= 40 || v < -1 || v == 0 || v > 30) {
            fclose(f);
            return STC_ERR_INVALID_ARG;
        }
        t[a][c] = static_cast<signed char>(v);
    }
    const bool clean = n == EOF;
    fclose(f);
    if (!clean) return STC_ERR_INVALID_ARG;
    memcpy(h->tune_light, t, sizeof(t));
    return STC_OK;
}

extern "C" stc_status stc_set_round_driver(stc_handle* h, int32_t driver) {
    if (!h || driver < 0 || driver > 1) return STC_ERR_INVALID_ARG;
    h->round_driver = driver;
    return STC_OK;
}

extern "C" stc_status stc_mfbc(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsources,
                               int32_t batch, double* bc_out, stc_stream stream) {
    stc_status st = mfbc_args(h, G, sources, nsources);
    if (st != STC_OK) return st;
    if (batch < 1 || batch > 256 || !bc_out) return STC_ERR_INVALID_ARG;
    return stc_mfbc_impl(h, G, sources, nsources, batch, bc_out, stream);
}

extern "C" stc_status stc_contract_spgemm_learned(stc_handle* h, stc_algebra alg, const stc_csr* A,
                                                  const stc_csr* B, stc_csr* C, const float* weights, float margin,
                                                  stc_learned_stats* stats, const stc_opts* opts,
                                                  stc_stream stream) {
    if (!h || !C) return STC_ERR_INVALID_ARG;
    if (!alg_valid(alg)) return STC_ERR_ALGEBRA;
    stc_status st = stc_check_csr_host(A);
    if (st != STC_OK) return st;
    if ((st = stc_check_csr_host(B)) != STC_OK) return st;
    if (A->ncols != B->nrows) return STC_ERR_SHAPE;
    if (!(margin >= 0.0f) || margin > 64.0f) return STC_ERR_INVALID_ARG;
    if (opts)
        for (int r : opts->reserved)
            if (r != 0) return STC_ERR_INVALID_ARG;
        if (opts->light_rows < -1 || opts->light_rows > 30) return STC_ERR_INVALID_ARG;
    return stc_spgemm_learned_impl(h, alg, A, B, C, weights, margin, stats, opts, stream);
}

extern "C" stc_status stc_calibrate_accumulate(stc_handle* h, stc_algebra alg, double* updates_per_s,
                                               stc_stream stream) {
    if (!h || !updates_per_s) return STC_ERR_INVALID_ARG;
    return stc_calibrate_accumulate_impl(h, int(alg), updates_per_s, stream);
}
