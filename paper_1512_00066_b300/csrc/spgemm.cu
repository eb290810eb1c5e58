// SpGEMM C = A (x) B over the library's algebras: the plain two-pass method.
//
//   row analysis   ub_i = sum over stored k of row i of A of nnz(B_k)   (products of row i)
//   binning        rows with ub_i > 0 listed heaviest first (log2 bins of ub_i)
//   window table   for every row k of B and column window w, the offset of the
//                  first entry of B_k with column >= w * W (only when the columns
//                  do not fit one window)
//   symbolic       exact nnz of each output row: bitmap of the union of the
//                  column sets in shared memory, popcount
//   scan           row pointers of C
//   numeric        per output row and column window: a dense shared-memory
//                  accumulator of W entries combined with the algebra's additive
//                  operator through shared-memory atomics, a presence bitmap, then
//                  a compaction of the window in column order straight into C
//
// The contraction is the one of Section 3.3.1 (C["ij"] = A["ik"]*B["kj"]) over the
// structures of Section 3.1 and the pairwise functions of Section 3.3.2.  One CTA
// owns one output row at a time (persistent CTAs pull rows from a device counter);
// inside the CTA the products of a chunk of up to NT stored entries of A_i are
// spread evenly over the threads (a block scan of the segment lengths, then a
// binary search of each product's segment), so hub rows of B do not serialise on
// one thread.
#include "stc_internal.cuh"

namespace {

constexpr int SP_NT = 512;   // threads per CTA of the symbolic and numeric kernels
constexpr int NBINS = 48;    // bin 0: ub == 0; bin b >= 1: 2^(b-1) <= ub < 2^b
constexpr int SYM_MAX_COLS = 1 << 19;  // symbolic bitmap width (64 KB)

struct SpgArgs {
    int64_t nA, K, ncols, nnzA, nnzB;
    const int64_t* __restrict__ a_ptr;
    const int32_t* __restrict__ a_col;
    const void* __restrict__ a_val;
    const int64_t* __restrict__ b_ptr;
    const int32_t* __restrict__ b_col;
    const void* __restrict__ b_val;
    const int32_t* __restrict__ woff;  // [K][nwin+1] or null when nwin == 1
    int W;                             // numeric window width, power of two
    int nwin;                          // number of numeric windows
};

// ----------------------------------------------------------------- algebra traits

template <int ALG> struct Tr;

template <> struct Tr<ALG_PT_F32> {
    using A = float; using B = float; using C = float; using Acc = double;
    static __device__ __forceinline__ Acc empty() { return 0.0; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        atomicAdd(&acc[c], double(a) * double(b));
    }
    static __device__ __forceinline__ C out(Acc v) { return float(v); }
};
template <> struct Tr<ALG_PT_F64> {
    using A = double; using B = double; using C = double; using Acc = double;
    static __device__ __forceinline__ Acc empty() { return 0.0; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        atomicAdd(&acc[c], a * b);
    }
    static __device__ __forceinline__ C out(Acc v) { return v; }
};
template <> struct Tr<ALG_MP_I32> {
    using A = int; using B = int; using C = int; using Acc = int;
    // INT_MAX, not the additive identity: every flushed entry has at least one
    // product, and min(INT_MAX, x) == x for every representable sum.
    static __device__ __forceinline__ Acc empty() { return INT_MAX; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        atomicMin(&acc[c], a + b);
    }
    static __device__ __forceinline__ C out(Acc v) { return v; }
};
template <> struct Tr<ALG_MP_F32> {
    using A = float; using B = float; using C = float; using Acc = unsigned;
    static __device__ __forceinline__ Acc empty() { return 0xffffffffu; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        atomicMin(&acc[c], f32_to_ordered(__fadd_rn(a, b)));
    }
    static __device__ __forceinline__ C out(Acc v) { return ordered_to_f32(v); }
};
template <> struct Tr<ALG_BOOL> {
    using A = uint8_t; using B = uint8_t; using C = uint8_t; using Acc = unsigned;
    static __device__ __forceinline__ Acc empty() { return 0u; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        if (a != 0 && b != 0 && acc[c] == 0u) atomicOr(&acc[c], 1u);
    }
    static __device__ __forceinline__ C out(Acc v) { return uint8_t(v != 0u); }
};
template <> struct Tr<ALG_MULTPATH> {
    using A = int; using B = DSig; using C = DSig; using Acc = int;  // distance part
    static __device__ __forceinline__ Acc empty() { return INT_MAX; }
};

// ----------------------------------------------------------------- row analysis + binning

__device__ __forceinline__ int bin_of(int64_t ub) { return ub == 0 ? 0 : 64 - __clzll(ub); }

__global__ void k_row_ub(SpgArgs g, int64_t* __restrict__ ub, int* __restrict__ bin_count) {
    __shared__ int s_bins[NBINS];
    for (int t = threadIdx.x; t < NBINS; t += blockDim.x) s_bins[t] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = warp; i < g.nA; i += nwarps) {
        int64_t lo, hi;
        row_range(g.a_ptr, i, g.nnzA, lo, hi);
        int64_t s = 0;
        for (int64_t p = lo + lane; p < hi; p += 32) {
            int32_t k = g.a_col[p];
            if ((uint64_t)k < (uint64_t)g.K) {
                int64_t bl, bh;
                row_range(g.b_ptr, k, g.nnzB, bl, bh);
                s += bh - bl;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            ub[i] = s;
            atomicAdd(&s_bins[bin_of(s)], 1);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NBINS; t += blockDim.x)
        if (s_bins[t]) atomicAdd(&bin_count[t], s_bins[t]);
}

// Exclusive offsets of the bins, heaviest bin first; empty rows (bin 0) are not listed.
__global__ void k_bin_offsets(const int* __restrict__ bin_count, int* __restrict__ cursor,
                              int* __restrict__ nlist) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int off = 0;
        for (int b = NBINS - 1; b >= 1; --b) {
            cursor[b] = off;
            off += bin_count[b];
        }
        cursor[0] = off;
        *nlist = off;
    }
}

// Scatter of row ids into their bins (order inside a bin is arbitrary: rows are
// independent).  Block-aggregated: one global atomic per bin per block.
__global__ void __launch_bounds__(512) k_bin_scatter(int64_t nA, const int64_t* __restrict__ ub,
                                                     int* __restrict__ cursor,
                                                     int32_t* __restrict__ rowlist) {
    __shared__ int s_cnt[NBINS];
    __shared__ int s_base[NBINS];
    for (int t = threadIdx.x; t < NBINS; t += blockDim.x) s_cnt[t] = 0;
    __syncthreads();
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int bin = 0, local = 0;
    if (i < nA) {
        bin = bin_of(ub[i]);
        if (bin > 0) local = atomicAdd(&s_cnt[bin], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NBINS; t += blockDim.x)
        s_base[t] = (t > 0 && s_cnt[t]) ? atomicAdd(&cursor[t], s_cnt[t]) : 0;
    __syncthreads();
    if (i < nA && bin > 0) rowlist[s_base[bin] + local] = int32_t(i);
}

// woff[k*(nwin+1) + w] = position inside B_k of the first column >= w*W.
__global__ void k_window_offsets(SpgArgs g, int32_t* __restrict__ woff) {
    int64_t stride = int64_t(g.nwin) + 1;
    int64_t total = g.K * stride;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        int64_t k = idx / stride;
        int64_t w = idx - k * stride;
        int64_t lo, hi;
        row_range(g.b_ptr, k, g.nnzB, lo, hi);
        int64_t target = w * int64_t(g.W);
        int64_t a = lo, b = hi;  // first p in [lo, hi) with col >= target
        while (a < b) {
            int64_t m = (a + b) >> 1;
            if (int64_t(g.b_col[m]) < target) a = m + 1; else b = m;
        }
        woff[idx] = int32_t(a - lo);
    }
}

// ----------------------------------------------------------------- chunked product walk

template <int NT>
struct ChunkSmem {
    int pre[NT];        // exclusive prefix of the segment lengths of the chunk
    int64_t lo[NT];     // first B position of each segment
    int warp[NT / 32 + 1];
};

// Load the chunk [p0, p0+NT) of A_i (p < ahi), restricted to numeric windows
// [wl, wh) of each B row; returns the number of products.  Every thread calls it.
template <int NT, class AT, bool WITH_VAL>
__device__ __forceinline__ int load_chunk(const SpgArgs& g, int64_t p0, int64_t ahi, int wl, int wh,
                                          ChunkSmem<NT>& cs, AT* s_aval) {
    int64_t p = p0 + threadIdx.x;
    int len = 0;
    int64_t lo = 0;
    AT av = AT();
    if (p < ahi) {
        int32_t k = g.a_col[p];
        if ((uint64_t)k < (uint64_t)g.K) {
            int64_t bl, bh;
            row_range(g.b_ptr, k, g.nnzB, bl, bh);
            if (g.woff) {
                const int32_t* wo = g.woff + int64_t(k) * (g.nwin + 1);
                int64_t s = bl + wo[wl], e = bl + wo[wh];
                if (e > bh) e = bh;
                if (s > e) s = e;
                lo = s;
                len = int(e - s);
            } else {
                lo = bl;
                len = int(bh - bl);
            }
            if (WITH_VAL) av = static_cast<const AT*>(g.a_val)[p];
        }
    }
    int total;
    int ex = block_exclusive_scan<NT, int>(len, cs.warp, total);
    cs.pre[threadIdx.x] = ex;
    cs.lo[threadIdx.x] = lo;
    if (WITH_VAL) s_aval[threadIdx.x] = av;
    __syncthreads();
    return total;
}

// Largest j with pre[j] <= f (pre non-decreasing, pre[0] == 0 <= f).
template <int NT>
__device__ __forceinline__ int find_seg(const int* pre, int f) {
    int j = 0;
#pragma unroll
    for (int step = NT / 2; step > 0; step >>= 1)
        if (pre[j + step] <= f) j += step;
    return j;
}

// Persistent-CTA row loop: returns the next listed row or -1.
__device__ __forceinline__ int next_row(int* counter, int nlist, const int32_t* rowlist, int* s_row) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int r = atomicAdd(counter, 1);
        *s_row = r < nlist ? rowlist[r] : -1;
    }
    __syncthreads();
    return *s_row;
}

// ----------------------------------------------------------------- symbolic

template <int NT>
__global__ void __launch_bounds__(NT, 2)
k_symbolic(SpgArgs g, int R, const int32_t* __restrict__ rowlist, const int* __restrict__ nlist_ptr,
           int* __restrict__ counter, int64_t* __restrict__ row_nnz) {
    extern __shared__ uint4 smem_raw[];
    uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw);
    __shared__ ChunkSmem<NT> cs;
    __shared__ int s_row;
    __shared__ int64_t s_red[NT / 32 + 1];
    const int Ws = g.W * R;
    const int NWs = Ws >> 5;
    for (int w = threadIdx.x; w < NWs; w += NT) bits[w] = 0u;
    const int nlist = *nlist_ptr;
    const int nws = (g.nwin + R - 1) / R;
    for (;;) {
        int i = next_row(counter, nlist, rowlist, &s_row);
        if (i < 0) break;
        int64_t alo, ahi;
        row_range(g.a_ptr, i, g.nnzA, alo, ahi);
        int64_t count = 0;
        for (int ws = 0; ws < nws; ++ws) {
            const int wl = ws * R;
            const int wh = min(wl + R, g.nwin);
            const int64_t c0 = int64_t(wl) * g.W;
            for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
                int total = load_chunk<NT, int, false>(g, p0, ahi, wl, wh, cs, nullptr);
                for (int f = threadIdx.x; f < total; f += NT) {
                    int j = find_seg<NT>(cs.pre, f);
                    int64_t p = cs.lo[j] + (f - cs.pre[j]);
                    int64_t c = int64_t(g.b_col[p]) - c0;
                    if ((uint64_t)c < (uint64_t)Ws) atomicOr(&bits[c >> 5], 1u << (c & 31));
                }
                __syncthreads();
            }
            int64_t local = 0;
            for (int w = threadIdx.x; w < NWs; w += NT) {
                uint32_t b = bits[w];
                if (b) {
                    local += __popc(b);
                    bits[w] = 0u;
                }
            }
            int64_t tot;
            (void)block_exclusive_scan<NT, int64_t>(local, s_red, tot);
            count += tot;
        }
        if (threadIdx.x == 0) row_nnz[i] = count;
    }
}

// ----------------------------------------------------------------- numeric

template <int ALG>
__device__ __forceinline__ void store_out(void* c_val, int64_t pos, typename Tr<ALG>::Acc v) {
    static_cast<typename Tr<ALG>::C*>(c_val)[pos] = Tr<ALG>::out(v);
}

// Compact the window's present columns in ascending order to C, reset the
// accumulator entries and the bitmap.  Returns the number of entries written.
template <int ALG, int NT, class FlushOne>
__device__ __forceinline__ int flush_window(uint32_t* bits, int NW, int64_t out0, int64_t out_end,
                                            int* s_warp, FlushOne flush_one) {
    const int WPT = (NW + NT - 1) / NT;
    const int w0 = threadIdx.x * WPT;
    const int w1 = min(w0 + WPT, NW);
    int cnt = 0;
    for (int w = w0; w < w1; ++w) cnt += __popc(bits[w]);
    int total;
    int ex = block_exclusive_scan<NT, int>(cnt, s_warp, total);
    int64_t pos = out0 + ex;
    for (int w = w0; w < w1; ++w) {
        uint32_t b = bits[w];
        if (!b) continue;
        bits[w] = 0u;
        while (b) {
            int bit = __ffs(b) - 1;
            b &= b - 1;
            int cl = (w << 5) + bit;
            flush_one(cl, pos, pos < out_end);
            ++pos;
        }
    }
    __syncthreads();
    return total;
}

template <int ALG, int NT>
__global__ void __launch_bounds__(NT, 2)
k_numeric(SpgArgs g, const int32_t* __restrict__ rowlist, const int* __restrict__ nlist_ptr,
          int* __restrict__ counter, const int64_t* __restrict__ c_ptr, int32_t* __restrict__ c_col,
          void* __restrict__ c_val, int* __restrict__ flags) {
    using T = Tr<ALG>;
    using AT = typename T::A;
    using BT = typename T::B;
    using Acc = typename T::Acc;
    extern __shared__ uint4 smem_raw[];
    const int W = g.W;
    const int NW = W >> 5;
    Acc* acc = reinterpret_cast<Acc*>(smem_raw);
    double* sig = reinterpret_cast<double*>(acc + W);  // multiplicities (multpath only)
    uint32_t* bits = ALG == ALG_MULTPATH ? reinterpret_cast<uint32_t*>(sig + W)
                                         : reinterpret_cast<uint32_t*>(acc + W);
    __shared__ ChunkSmem<NT> cs;
    __shared__ AT s_aval[NT];
    __shared__ int s_row;
    __shared__ int s_warp[NT / 32 + 1];

    for (int c = threadIdx.x; c < W; c += NT) {
        acc[c] = T::empty();
        if (ALG == ALG_MULTPATH) sig[c] = 0.0;
    }
    for (int w = threadIdx.x; w < NW; w += NT) bits[w] = 0u;
    const int nlist = *nlist_ptr;
    const BT* __restrict__ bval = static_cast<const BT*>(g.b_val);
    auto* cval = static_cast<typename T::C*>(c_val);

    for (;;) {
        int i = next_row(counter, nlist, rowlist, &s_row);
        if (i < 0) break;
        int64_t alo, ahi;
        row_range(g.a_ptr, i, g.nnzA, alo, ahi);
        const int64_t o0 = c_ptr[i], o1 = c_ptr[i + 1];
        int64_t base = 0;
        for (int w = 0; w < g.nwin; ++w) {
            const int64_t c0 = int64_t(w) * W;
            for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
                int total = load_chunk<NT, AT, true>(g, p0, ahi, w, w + 1, cs, s_aval);
                for (int f = threadIdx.x; f < total; f += NT) {
                    int j = find_seg<NT>(cs.pre, f);
                    int64_t p = cs.lo[j] + (f - cs.pre[j]);
                    int64_t c = int64_t(g.b_col[p]) - c0;
                    if ((uint64_t)c >= (uint64_t)W) continue;
                    const AT a = s_aval[j];
                    const BT b = bval[p];
                    if constexpr (ALG == ALG_MULTPATH) {
                        atomicMin(&acc[c], a + b.d);
                    } else {
                        T::combine(acc, int(c), a, b);
                    }
                    atomicOr(&bits[c >> 5], 1u << (c & 31));
                }
                __syncthreads();
            }
            if constexpr (ALG == ALG_MULTPATH) {
                // second walk: add the multiplicities of the products at the minimum
                for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
                    int total = load_chunk<NT, AT, true>(g, p0, ahi, w, w + 1, cs, s_aval);
                    for (int f = threadIdx.x; f < total; f += NT) {
                        int j = find_seg<NT>(cs.pre, f);
                        int64_t p = cs.lo[j] + (f - cs.pre[j]);
                        int64_t c = int64_t(g.b_col[p]) - c0;
                        if ((uint64_t)c >= (uint64_t)W) continue;
                        const BT b = bval[p];
                        if (s_aval[j] + b.d == acc[c]) atomicAdd(&sig[c], b.s);
                    }
                    __syncthreads();
                }
            }
            int wrote;
            if constexpr (ALG == ALG_MULTPATH) {
                wrote = flush_window<ALG, NT>(bits, NW, o0 + base, o1, s_warp,
                    [&](int cl, int64_t pos, bool ok) {
                        if (ok) {
                            c_col[pos] = int32_t(c0 + cl);
                            DSig r;
                            r.d = acc[cl];
                            r.pad = 0;
                            r.s = sig[cl];
                            cval[pos] = r;
                        }
                        acc[cl] = T::empty();
                        sig[cl] = 0.0;
                    });
            } else {
                wrote = flush_window<ALG, NT>(bits, NW, o0 + base, o1, s_warp,
                    [&](int cl, int64_t pos, bool ok) {
                        if (ok) {
                            c_col[pos] = int32_t(c0 + cl);
                            cval[pos] = T::out(acc[cl]);
                        }
                        acc[cl] = T::empty();
                    });
            }
            base += wrote;
        }
        if (threadIdx.x == 0 && base != o1 - o0) atomicOr(flags, STC_FLAG_INTERNAL);
    }
}

// ----------------------------------------------------------------- host side

int64_t pow2_ceil(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

int numeric_window_max(int alg) {
    switch (alg) {
    case ALG_PT_F32:
    case ALG_PT_F64: return 8192;    // 64 KB of fp64 accumulators
    case ALG_MULTPATH: return 4096;  // 48 KB of (int, fp64)
    default: return 16384;           // 64 KB of 32-bit accumulators
    }
}

size_t numeric_smem_bytes(int alg, int W) {
    size_t acc = (alg == ALG_PT_F32 || alg == ALG_PT_F64) ? 8 : 4;
    size_t per = acc + (alg == ALG_MULTPATH ? 8 : 0);
    return per * size_t(W) + size_t(W / 32) * 4;
}

template <class K>
stc_status launch_persistent(stc_handle* h, K kernel, size_t smem, int& grid) {
    STC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int per_sm = 0;
    STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, SP_NT, smem));
    if (per_sm < 1) return STC_ERR_CUDA;
    grid = per_sm * h->num_sms;
    return STC_OK;
}

template <int ALG>
stc_status run_numeric(stc_handle* h, const SpgArgs& g, const int32_t* rowlist, const int* nlist,
                       int* counter, const int64_t* c_ptr, int32_t* c_col, void* c_val, int64_t nA,
                       stc_stream s) {
    size_t smem = numeric_smem_bytes(ALG, g.W);
    int grid = 0;
    auto kern = k_numeric<ALG, SP_NT>;
    stc_status st = launch_persistent(h, kern, smem, grid);
    if (st != STC_OK) return st;
    if (int64_t(grid) > nA) grid = int(nA > 0 ? nA : 1);
    kern<<<grid, SP_NT, smem, s>>>(g, rowlist, nlist, counter, c_ptr, c_col, c_val, h->d_flags);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

}  // namespace

stc_status stc_spgemm_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                           const stc_opts* opts, stc_stream s) {
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->nnz = 0;
    C->rowptr = nullptr;
    C->col = nullptr;
    C->val = nullptr;
    const int64_t nA = A->nrows;
    const size_t vbytes = stc_val_bytes(alg, 'C');

    int64_t* c_ptr = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(nA + 1) * 8, s));
    if (!c_ptr) return STC_ERR_OOM;
    int32_t* c_col = nullptr;
    void* c_val = nullptr;
    auto fail = [&](stc_status st) {
        stc_free_bytes(h, c_ptr, s);
        if (c_col) stc_free_bytes(h, c_col, s);
        if (c_val) stc_free_bytes(h, c_val, s);
        return st;
    };
    stc_mark(h, s, 0);
    if (cudaMemsetAsync(c_ptr, 0, size_t(nA + 1) * 8, s) != cudaSuccess) return fail(STC_ERR_CUDA);

    const bool validate = !(opts && opts->skip_validation);
    stc_status st;
    if (validate) {
        if ((st = stc_validate_csr_async(h, A, s)) != STC_OK) return fail(st);
        if ((st = stc_validate_csr_async(h, B, s)) != STC_OK) return fail(st);
    }
    stc_mark(h, s, 1);

    SpgArgs g;
    g.nA = nA;
    g.K = A->ncols;
    g.ncols = B->ncols;
    g.nnzA = A->nnz;
    g.nnzB = B->nnz;
    g.a_ptr = A->rowptr;
    g.a_col = A->col;
    g.a_val = A->val;
    g.b_ptr = B->rowptr;
    g.b_col = B->col;
    g.b_val = B->val;
    g.woff = nullptr;
    const int64_t ncp = pow2_ceil(B->ncols > 0 ? B->ncols : 1);
    int64_t W = numeric_window_max(alg);
    if (opts && opts->window_cols) W = opts->window_cols;
    if (ncp < W) W = ncp < 32 ? 32 : ncp;
    g.W = int(W);
    g.nwin = int((B->ncols + W - 1) / W);
    if (g.nwin < 1) g.nwin = 1;
    const bool trivial = nA == 0 || A->nnz == 0 || B->nnz == 0 || B->ncols == 0;
    if (numeric_smem_bytes(alg, g.W) > size_t(h->smem_optin) - 24 * 1024) return fail(STC_ERR_INVALID_ARG);

    {
        StcScratch sc(h, s);
        int32_t* rowlist = nullptr;
        int* ints = nullptr;
        if (!trivial) {
            int64_t Ws = ncp < SYM_MAX_COLS ? ncp : SYM_MAX_COLS;
            if (Ws < W) Ws = W;
            const int R = int(Ws / W);
            int64_t* ub = sc.get<int64_t>(size_t(nA));
            rowlist = sc.get<int32_t>(size_t(nA));
            ints = sc.get<int>(2 * NBINS + 8);
            if (sc.failed) return fail(STC_ERR_OOM);
            if (cudaMemsetAsync(ints, 0, sizeof(int) * (2 * NBINS + 8), s) != cudaSuccess)
                return fail(STC_ERR_CUDA);
            int* bin_count = ints;
            int* cursor = ints + NBINS;
            int* nlist = ints + 2 * NBINS;
            int* counters = ints + 2 * NBINS + 1;  // [0] symbolic, [1] numeric
            if (g.nwin > 1) {
                int32_t* woff = sc.get<int32_t>(size_t(g.K) * size_t(g.nwin + 1));
                if (!woff) return fail(STC_ERR_OOM);
                g.woff = woff;
                int64_t tot = g.K * (g.nwin + 1);
                int64_t blocks = (tot + 255) / 256;
                if (blocks > int64_t(h->num_sms) * 32) blocks = int64_t(h->num_sms) * 32;
                k_window_offsets<<<unsigned(blocks > 0 ? blocks : 1), 256, 0, s>>>(g, woff);
                if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
                stc_count(h);
            }
            {
                int64_t blocks = (nA * 32 + 255) / 256;
                if (blocks > int64_t(h->num_sms) * 16) blocks = int64_t(h->num_sms) * 16;
                k_row_ub<<<unsigned(blocks), 256, 0, s>>>(g, ub, bin_count);
                k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
                k_bin_scatter<<<unsigned((nA + 511) / 512), 512, 0, s>>>(nA, ub, cursor, rowlist);
                if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
                stc_count(h, 3);
            }
            stc_mark(h, s, 2);
            {
                size_t smem = size_t(Ws / 32) * 4;
                int grid = 0;
                auto kern = k_symbolic<SP_NT>;
                if ((st = launch_persistent(h, kern, smem, grid)) != STC_OK) return fail(st);
                if (int64_t(grid) > nA) grid = int(nA);
                kern<<<grid, SP_NT, smem, s>>>(g, R, rowlist, nlist, counters, c_ptr + 1);
                if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
                stc_count(h);
            }
            stc_mark(h, s, 3);
            if ((st = stc_inclusive_scan_i64(h, sc, c_ptr + 1, nA, s)) != STC_OK) return fail(st);
        } else {
            stc_mark(h, s, 2);
            stc_mark(h, s, 3);
        }
        // the single synchronisation: nnz(C) and the validation flags
        if (cudaMemcpyAsync(&h->h_stage[0], c_ptr + nA, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(&h->h_stage[1], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(STC_ERR_CUDA);
        }
        const int64_t nnz = h->h_stage[0];
        const int flags = int(reinterpret_cast<int*>(&h->h_stage[1])[0]);
        if (flags) {
            (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
            return fail(stc_flags_to_status(flags));
        }
        if (nnz < 0) return fail(STC_ERR_CUDA);
        c_col = static_cast<int32_t*>(stc_alloc_bytes(h, size_t(nnz) * 4, s));
        c_val = stc_alloc_bytes(h, size_t(nnz) * vbytes, s);
        if (!c_col || !c_val) return fail(STC_ERR_OOM);
        stc_mark(h, s, 4);
        if (!trivial && nnz > 0) {
            int* nlist = ints + 2 * NBINS;
            int* counters = ints + 2 * NBINS + 1;
            switch (alg) {
            case ALG_PT_F32: st = run_numeric<ALG_PT_F32>(h, g, rowlist, nlist, counters + 1, c_ptr, c_col, c_val, nA, s); break;
            case ALG_PT_F64: st = run_numeric<ALG_PT_F64>(h, g, rowlist, nlist, counters + 1, c_ptr, c_col, c_val, nA, s); break;
            case ALG_MP_I32: st = run_numeric<ALG_MP_I32>(h, g, rowlist, nlist, counters + 1, c_ptr, c_col, c_val, nA, s); break;
            case ALG_MP_F32: st = run_numeric<ALG_MP_F32>(h, g, rowlist, nlist, counters + 1, c_ptr, c_col, c_val, nA, s); break;
            case ALG_BOOL: st = run_numeric<ALG_BOOL>(h, g, rowlist, nlist, counters + 1, c_ptr, c_col, c_val, nA, s); break;
            case ALG_MULTPATH: st = run_numeric<ALG_MULTPATH>(h, g, rowlist, nlist, counters + 1, c_ptr, c_col, c_val, nA, s); break;
            default: st = STC_ERR_ALGEBRA;
            }
            if (st != STC_OK) return fail(st);
        }
        stc_mark(h, s, 5);
        C->nnz = nnz;
    }
    C->rowptr = c_ptr;
    C->col = c_col;
    C->val = c_val;
    return STC_OK;
}
