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
constexpr int BIN_COPY = NBINS;       // rows with a single stored A entry (rank path)
constexpr int NBINS_ALL = NBINS + 1;
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
    const int32_t* __restrict__ ctab;  // rank path: [K][ncell+1] per-cell offsets in B rows, or null
    int ncell;                         // rank path: 1024-column cells of the output
    int col_base;                      // added to every written column (column slabs of a wide B)
    int64_t bm_off;                    // warp-per-row passes: first bitmap word of this matrix's rows
};

// Rows of one matrix (table == null: `one`) or of a batch of independent
// matrices whose rows are numbered consecutively (row_off[b] = first global row
// of matrix b, row_off[nb] = total).
struct SpgRows {
    SpgArgs one;
    const SpgArgs* __restrict__ table;
    const int64_t* __restrict__ row_off;
    int nb;
};

// Where the numeric rank kernel writes a row.  Plain form: ptr = C's row
// pointers (cap == null), and a row must fill exactly its slot.  Learned form:
// ptr = scratch offsets, cap = predicted capacity; the exact count goes to nnz[],
// a row larger than its capacity is listed in ovf[] and not written.
struct RankOut {
    const int64_t* __restrict__ ptr;
    const int64_t* __restrict__ cap;
    int64_t* __restrict__ nnz;
    int32_t* __restrict__ ovf;
    int* __restrict__ novf;
    const float* __restrict__ pred;  // predicted log2(1 + nnz), or null
    double* __restrict__ err;        // sum of |pred - log2(1 + nnz)|
    // Learned form: a row larger than its capacity is written to the overflow pool
    // [pool_base, pool_base + pool_cap) of the scratch instead (bump allocation in
    // *pool_used) and listed in ovf only when the pool is full.  where[gi] (may be
    // null) receives the scratch offset the row was written at, or -1.
    unsigned long long* __restrict__ pool_used;
    int64_t pool_base, pool_cap;
    int64_t* __restrict__ where;
    int* __restrict__ n_over;  // rows larger than their capacity, pooled or not (may be null)
};

__device__ __forceinline__ int batch_of(const SpgRows& R, int64_t gi) {
    int lo = 0, hi = R.nb - 1;  // last b with row_off[b] <= gi
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (R.row_off[mid] <= gi) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ----------------------------------------------------------------- algebra traits

template <int ALG> struct Tr;

template <> struct Tr<ALG_PT_F32> {
    // fp32 products summed with fp32 shared-memory atomics (B300's fp64 rate is a
    // small fraction of its fp32 rate)
    using A = float; using B = float; using C = float; using Acc = float;
    static __device__ __forceinline__ Acc empty() { return 0.0f; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        atomicAdd(&acc[c], __fmul_rn(a, b));
    }
    static __device__ __forceinline__ C out(Acc v) { return v; }
    // the output of an entry with exactly one product (added to an empty accumulator)
    static __device__ __forceinline__ C one(A a, B b) { return __fadd_rn(0.0f, __fmul_rn(a, b)); }
    static __device__ __forceinline__ C identity() { return 0.0f; }  // of (+)
};
template <> struct Tr<ALG_PT_F64> {
    using A = double; using B = double; using C = double; using Acc = double;
    static __device__ __forceinline__ Acc empty() { return 0.0; }
    // acc[c] = fma(a, b, acc[c]) by compare-and-swap: one FP64 instruction per
    // product.  The shared-memory fp64 add of a rounded product (atomicAdd, or
    // red.shared.add.f64 with no return) runs faster in isolation on B300 (0.82
    // against 0.44 updates per clock per SM; random targets, 1024 threads per SM),
    // but was slower inside this kernel both ways (R-MAT 18 numeric phase 27.5 and
    // 27.7 ms against 25.1-25.5 ms); the bits are compared, so a NaN ends the loop
    // like any other value
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        unsigned long long* p = reinterpret_cast<unsigned long long*>(&acc[c]);
        unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(p);
        for (;;) {
            const unsigned long long want = __double_as_longlong(__fma_rn(a, b, __longlong_as_double(old)));
            const unsigned long long seen = atomicCAS(p, old, want);
            if (seen == old) break;
            old = seen;
        }
    }
    static __device__ __forceinline__ C out(Acc v) { return v; }
    static __device__ __forceinline__ C one(A a, B b) { return __dadd_rn(0.0, __dmul_rn(a, b)); }
    static __device__ __forceinline__ C identity() { return 0.0; }
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
    static __device__ __forceinline__ C one(A a, B b) { return a + b; }
    static __device__ __forceinline__ C identity() { return STC_MIN_PLUS_I32_IDENTITY; }
};
template <> struct Tr<ALG_MP_F32> {
    using A = float; using B = float; using C = float; using Acc = unsigned;
    static __device__ __forceinline__ Acc empty() { return 0xffffffffu; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        atomicMin(&acc[c], f32_to_ordered(__fadd_rn(a, b)));
    }
    static __device__ __forceinline__ C out(Acc v) { return ordered_to_f32(v); }
    static __device__ __forceinline__ C one(A a, B b) { return ordered_to_f32(f32_to_ordered(__fadd_rn(a, b))); }
    static __device__ __forceinline__ C identity() { return __int_as_float(0x7f800000); }  // +inf
};
template <> struct Tr<ALG_BOOL> {
    using A = uint8_t; using B = uint8_t; using C = uint8_t; using Acc = unsigned;
    static __device__ __forceinline__ Acc empty() { return 0u; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        if (a != 0 && b != 0 && acc[c] == 0u) atomicOr(&acc[c], 1u);
    }
    static __device__ __forceinline__ C out(Acc v) { return uint8_t(v != 0u); }
    static __device__ __forceinline__ C one(A a, B b) { return uint8_t(a != 0 && b != 0); }
    static __device__ __forceinline__ C identity() { return 0; }
};
template <> struct Tr<ALG_PATH> {
    // lexicographic (w, h) as one 64-bit key: w with its sign bit flipped, then h
    using A = PathVal; using B = PathVal; using C = PathVal; using Acc = unsigned long long;
    static __device__ __forceinline__ Acc key(int32_t w, int32_t h) {
        return (Acc(uint32_t(w) ^ 0x80000000u) << 32) | uint32_t(h);
    }
    static __device__ __forceinline__ Acc empty() { return ~0ull; }
    static __device__ __forceinline__ void combine(Acc* acc, int c, A a, B b) {
        const Acc k = key(a.w + b.w, a.h + b.h);
        if (k < acc[c]) atomicMin(&acc[c], k);
    }
    static __device__ __forceinline__ C out(Acc v) {
        C o;
        o.w = int32_t(uint32_t(v >> 32) ^ 0x80000000u);
        o.h = int32_t(uint32_t(v));
        return o;
    }
    static __device__ __forceinline__ C one(A a, B b) {
        C o;
        o.w = a.w + b.w;
        o.h = a.h + b.h;
        return o;
    }
};
template <> struct Tr<ALG_MULTPATH> {
    using A = int; using B = DSig; using C = DSig; using Acc = int;  // distance part
    static __device__ __forceinline__ Acc empty() { return INT_MAX; }
    static __device__ __forceinline__ C one(A a, B b) {
        DSig o;
        o.d = a + b.d;
        o.pad = 0;
        o.s = 0.0 + b.s;
        return o;
    }
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

// Exclusive offsets of the bins, heaviest bin first; empty rows (bin 0) are not
// listed.  *nlist counts the rows of bins 1..NBINS-1; the rows of BIN_COPY (when
// used) follow them.
__global__ void k_bin_offsets(const int* __restrict__ bin_count, int* __restrict__ cursor,
                              int* __restrict__ nlist) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int off = 0;
        for (int b = NBINS - 1; b >= 1; --b) {
            cursor[b] = off;
            off += bin_count[b];
        }
        *nlist = off;
        cursor[BIN_COPY] = off;
        cursor[0] = off + bin_count[BIN_COPY];
    }
}

// Scatter of row ids into their bins (order inside a bin is arbitrary: rows are
// independent).  Block-aggregated: one global atomic per bin per block.
// Sizes of the heavy prefix (bins above L) and the light suffix (bins 1..L) of
// the row list.
__global__ void k_split_counts(const int* __restrict__ bin_count, int L, int* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int heavy = 0, light = 0;
        for (int b = 1; b < NBINS; ++b) (b > L ? heavy : light) += bin_count[b];
        out[0] = heavy;
        out[1] = light;
    }
}

// single (may be null): non-zero for the rows of BIN_COPY.
__global__ void __launch_bounds__(512) k_bin_scatter(int64_t nA, const int64_t* __restrict__ ub,
                                                     const int64_t* __restrict__ single,
                                                     int* __restrict__ cursor,
                                                     int32_t* __restrict__ rowlist) {
    __shared__ int s_cnt[NBINS_ALL];
    __shared__ int s_base[NBINS_ALL];
    for (int t = threadIdx.x; t < NBINS_ALL; t += blockDim.x) s_cnt[t] = 0;
    __syncthreads();
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int bin = 0, local = 0;
    if (i < nA) {
        bin = (single && single[i] > 0) ? BIN_COPY : bin_of(ub[i]);
        if (bin > 0) local = atomicAdd(&s_cnt[bin], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NBINS_ALL; t += blockDim.x)
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

// find_seg for a warp-uniform f, by two ballot rounds: over coarse[g] = pre[32 g]
// to pick the group of 32 entries, then over that group (every lane of the warp
// calls it with the same f; NT a multiple of 32, <= 1024).
template <int NT>
__device__ __forceinline__ int find_seg_warp(const int* pre, const int* coarse, int f, int lane) {
    constexpr int G = NT / 32;
    const unsigned m1 = __ballot_sync(0xffffffffu, lane < G && coarse[lane] <= f);
    const int grp = 31 - __clz(m1);  // m1 != 0: pre[0] == 0 <= f
    const unsigned m2 = __ballot_sync(0xffffffffu, pre[grp * 32 + lane] <= f);
    return grp * 32 + 31 - __clz(m2);
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

// ----------------------------------------------------------------- rank-indexed accumulator
//
// For outputs of at most RK_MAX_COLS columns: one CTA owns an output row and
// keeps its whole column bitmap in shared memory (1 bit per column, plus one
// summary bit per 32-bit word).  The products of the row are walked as warp
// tasks: each task is up to RK_SUB consecutive entries of one B row, read by the
// 32 lanes of a warp with coalesced loads (the few stored entries of A_i index
// long B rows, so segment-per-warp beats product-per-thread here).
//
//  symbolic  bitmap of the union of the column sets, popcount of touched words
//  numeric   1) bitmap again; 2) per 1024-column cell the popcount prefix of its
//            words and the cells' exclusive prefix give every present column its
//            rank, i.e. its position in the output row; the columns are written
//            to C in order; 3) the values are accumulated in shared memory
//            indexed by rank, with the algebra's additive operator as a
//            shared-memory atomic, then written to C coalesced.  Rows with more
//            entries than the value buffer are cut into rank windows made of
//            whole cells; a table of per-cell offsets inside every B row restricts
//            each window's walk to that window's columns.

constexpr int RK_SUB = 256;                 // B entries per warp task
// B entries per warp task of the numeric pass's value walk.  A row's products are a
// few dozen tasks for the CTA's 32 warps, so shorter tasks balance the warps better
// where products are expensive: fp64 (+,x) (a compare-and-swap of a DFMA each) takes
// 64, fp32 (+,x) 128, the other algebras RK_SUB (each the fastest measured at R-MAT 18)
constexpr int value_task_entries(int alg) {
    return alg == ALG_PT_F64 ? 64 : alg == ALG_PT_F32 ? 128 : RK_SUB;
}
constexpr int RK_CELL_SHIFT = 10;           // 1024-column cells (32 bitmap words)
constexpr int RK_CELL = 1 << RK_CELL_SHIFT;
constexpr int RK_MAX_COLS = 1 << 18;        // 32 KB bitmap
constexpr int RK_NT = 1024;     // numeric kernel: one CTA per SM, large value buffer
constexpr int RK_SYM_NT = 256;  // symbolic kernel: more rows in flight per SM
constexpr int RK_SYM_MINB = 5;  // its CTAs per SM (34 KB of shared memory each at 2^18 columns)
constexpr size_t RK_SMEM_TARGET = 224 * 1024;  // one CTA per SM
constexpr double RK_RECORD_BUDGET = 24e9;        // bytes of stored rank records
constexpr int RK_SPARSE_MAX_WORDS = 4096;         // sparse record: at most this many non-zero words
// (+,x) fp32: a row of A with more than F32_WIDE_ROW stored entries can give an
// output entry more terms than plain fp32 summation serves well, so such rows are
// summed with compensation: beside each fp32 accumulator an fp32 correction
// collects the exact rounding errors of the products (fma) and of the accumulating
// adds (two-sum on the value the atomic add returns), and the entry is the rounded
// sum of the two.  In the CTA numeric kernel the corrections take the
// column-per-rank buffer, and the row's output columns are expanded from its
// bitmap at write-out; the warp-per-row kernels leave such rows to it.
constexpr int64_t F32_WIDE_ROW = 1024;
constexpr int64_t NO_WIDE_ROWS = INT64_MAX;
__host__ __device__ constexpr int64_t wide_len_of(int alg) { return alg == ALG_PT_F32 ? F32_WIDE_ROW : NO_WIDE_ROWS; }

template <int NT>
struct TaskSmem {
    int pre[NT];         // exclusive prefix of the warp-task counts of the chunk's segments
    int coarse[NT / 32]; // pre[32 g], contiguous (read by 32 lanes without bank conflicts)
    int len[NT];         // segment length
    int64_t lo[NT];      // first B position of the segment
    int warp[NT / 32 + 1];
    int next;            // next unclaimed warp task (warps claim tasks dynamically)
};

// Segments of the chunk [p0, p0+NT) of A_i: whole B rows, or (ctab != null) the
// part of each B row inside cells [cl, ch).  Returns the number of warp tasks.
template <int NT, class AT, bool WITH_VAL, int SUB = RK_SUB>
__device__ __forceinline__ int load_tasks(const SpgArgs& g, const int32_t* __restrict__ ctab, int ncell,
                                          int64_t p0, int64_t ahi, int cl, int ch, TaskSmem<NT>& ts,
                                          AT* s_aval) {
    int64_t p = p0 + threadIdx.x;
    int len = 0;
    int64_t lo = 0;
    AT av = AT();
    if (p < ahi) {
        int32_t k = g.a_col[p];
        if ((uint64_t)k < (uint64_t)g.K) {
            int64_t bl, bh;
            row_range(g.b_ptr, k, g.nnzB, bl, bh);
            if (ctab) {
                const int32_t* t = ctab + int64_t(k) * (ncell + 1);
                int64_t s = bl + t[cl], e = bl + t[ch];
                if (e > bh) e = bh;
                if (s > e) s = e;
                bl = s;
                bh = e;
            }
            lo = bl;
            len = int(bh - bl);
            if (WITH_VAL) av = static_cast<const AT*>(g.a_val)[p];
        }
    }
    int total;
    int ex = block_exclusive_scan<NT, int>((len + SUB - 1) / SUB, ts.warp, total);
    ts.pre[threadIdx.x] = ex;
    if ((threadIdx.x & 31) == 0) ts.coarse[threadIdx.x >> 5] = ex;
    ts.len[threadIdx.x] = len;
    ts.lo[threadIdx.x] = lo;
    if (WITH_VAL) s_aval[threadIdx.x] = av;
    if (threadIdx.x == 0) ts.next = NT / 32;  // tasks 0..NT/32-1 go to warps 0..NT/32-1
    __syncthreads();
    return total;
}

// Run op(p, col, j) for every product of the loaded chunk (p: B position,
// j: index of the A entry in the chunk).  Columns are loaded SUB/32 at a time.
template <int NT, int SUB = RK_SUB, class Op>
__device__ __forceinline__ void walk_tasks(const SpgArgs& g, TaskSmem<NT>& ts, int ntasks, Op op) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int U = SUB / 32;
    for (int t = wid; t < ntasks;) {
        const int j = find_seg_warp<NT>(ts.pre, ts.coarse, t, lane);
        const int64_t start = ts.lo[j] + int64_t(t - ts.pre[j]) * SUB;
        const int64_t end = ts.lo[j] + ts.len[j];
        // warp-uniform number of 32-entry steps of this task (short B rows stop early)
        const int64_t span = end - start;
        const int nu = span >= SUB ? U : int((span + 31) >> 5);
        int col[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u < nu) {
                const int64_t p = start + lane + 32 * u;
                col[u] = p < end ? g.b_col[p] : -1;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u < nu) {
                const int64_t p = start + lane + 32 * u;
                if (p < end) op(p, col[u], j);
            }
        }
        int nt = 0;
        if (lane == 0) nt = atomicAdd(&ts.next, 1);
        t = __shfl_sync(0xffffffffu, nt, 0);
    }
}

// Symbolic walk: set the bitmap bit of every product's column.  All the task's
// bitmap reads are issued before its atomics (a read after an atomic would wait
// for it), and the summary bits are derived from the bitmap afterwards.
template <int NT, int SUB = RK_SUB, int STRIDE = 1>
__device__ __forceinline__ void walk_tasks_bits(const SpgArgs& g, TaskSmem<NT>& ts, int ntasks,
                                                uint32_t* bits) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int U = SUB / 32;
    for (int t = wid; t < ntasks;) {
        const int j = find_seg_warp<NT>(ts.pre, ts.coarse, t, lane);
        const int64_t start = ts.lo[j] + int64_t(t - ts.pre[j]) * SUB;
        const int64_t end = ts.lo[j] + ts.len[j];
        const int64_t span = end - start;
        const int nu = span >= SUB ? U : int((span + 31) >> 5);
        int col[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            col[u] = -1;
            if (u < nu) {
                const int64_t p = start + lane + 32 * u;
                if (p < end) col[u] = g.b_col[p];
            }
        }
        int nt = 0;
        if (lane == 0) nt = atomicAdd(&ts.next, 1);
        uint32_t cur[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            cur[u] = (u < nu && (uint64_t)col[u] < (uint64_t)g.ncols) ? bits[(col[u] >> 5) * STRIDE] : ~0u;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u < nu && (uint64_t)col[u] < (uint64_t)g.ncols) {
                const uint32_t m = 1u << (col[u] & 31);
                if (!(cur[u] & m)) atomicOr(&bits[(col[u] >> 5) * STRIDE], m);
            }
        }
        t = __shfl_sync(0xffffffffu, nt, 0);
    }
}

// Numeric walk: load the task's columns and B values up front, map every valid
// column to its rank in the current window with rank_of, calling on_rank(r, col)
// for the ranks in [0, rcount), then apply upd(r, col, b, a) to those.  All the
// rank lookups of a task are issued before its first accumulator update: the
// compiler cannot move a bitmap read past an atomic on the same shared memory.
template <int NT, class AT, class BT, int SUB = RK_SUB, class RankF, class OnRankF, class UpdF>
__device__ __forceinline__ void walk_tasks_rank(const SpgArgs& g, TaskSmem<NT>& ts, int ntasks,
                                                const AT* s_aval, const BT* __restrict__ bval, int rcount,
                                                RankF rank_of, OnRankF on_rank, UpdF upd) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int U = SUB / 32;
    for (int t = wid; t < ntasks;) {
        const int j = find_seg_warp<NT>(ts.pre, ts.coarse, t, lane);
        const int64_t start = ts.lo[j] + int64_t(t - ts.pre[j]) * SUB;
        const int64_t end = ts.lo[j] + ts.len[j];
        const int64_t span = end - start;
        const int nu = span >= SUB ? U : int((span + 31) >> 5);
        const AT a = s_aval[j];
        int col[U];
        BT val[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            col[u] = -1;
            if (u < nu) {
                const int64_t p = start + lane + 32 * u;
                if (p < end) {
                    col[u] = g.b_col[p];
                    val[u] = bval[p];
                }
            }
        }
        int rk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            rk[u] = (u < nu && (uint64_t)col[u] < (uint64_t)g.ncols) ? rank_of(col[u]) : -1;
            if ((unsigned)rk[u] < (unsigned)rcount) on_rank(rk[u], col[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if ((unsigned)rk[u] < (unsigned)rcount) upd(rk[u], col[u], val[u], a);
        int nt = 0;
        if (lane == 0) nt = atomicAdd(&ts.next, 1);
        t = __shfl_sync(0xffffffffu, nt, 0);
    }
}

// Shared-memory layout of the numeric rank kernel; its prefix [0, winfirst) is
// also the per-row record the symbolic pass stores:
//   wb[NW]        uint2 per bitmap word: x = the word's bits, y = rank (position in
//                 the output row) of the word's first present column
//   summ[ncell]   bit w%32 of summ[w/32] set when word w is non-zero
//   cellbase[ncell+1]  rank of the first present column of each 1024-column cell
struct RankLayout {
    size_t wb, summ, cellbase, winfirst, vals, scol, sig, total;
};

__host__ __device__ inline size_t rk_align(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline RankLayout rank_layout(int ncell, int vcap, int maxwin, size_t acc_bytes,
                                                  bool multpath) {
    RankLayout L;
    const size_t NW = size_t(ncell) * 32;
    L.wb = 0;
    L.summ = rk_align(L.wb + NW * 8);
    L.cellbase = rk_align(L.summ + size_t(ncell) * 4);
    L.winfirst = rk_align(L.cellbase + (size_t(ncell) + 1) * 4);
    L.vals = rk_align(L.winfirst + (size_t(maxwin) + 1) * 4);
    L.scol = rk_align(L.vals + size_t(vcap) * acc_bytes);
    L.sig = rk_align(L.scol + size_t(vcap) * 4);
    L.total = multpath ? rk_align(L.sig + size_t(vcap) * 8) : L.sig;
    return L;
}

// Shared-memory layout of the symbolic rank kernel: compact bitmap, summary, cell
// prefix.  (A word's rank inside its cell is a warp scan when the record is written:
// a cell is 32 words, one per lane.)
struct SymLayout {
    size_t bits, summ, cellbase, total;
};

__host__ __device__ inline SymLayout sym_layout(int ncell) {
    SymLayout L;
    const size_t NW = size_t(ncell) * 32;
    L.bits = 0;
    L.summ = rk_align(NW * 4);
    L.cellbase = rk_align(L.summ + size_t(ncell) * 4);
    L.total = rk_align(L.cellbase + (size_t(ncell) + 1) * 4);
    return L;
}

// Exclusive prefix of x over the warp's lanes.
__device__ __forceinline__ int warp_exclusive_sum(int x, int lane) {
    int y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
    }
    return y - x;
}

// Persistent-CTA row loop over a row list of global rows.  Thread 0 claims rows
// two ahead: it holds one claimed row whose list entry is already loaded and one
// whose entry is being loaded, so moving to the next row waits on neither the
// claim nor the list read.  Thread 0 resolves the row's matrix into shared memory.
struct RowClaim {
    int r1;        // claimed list position, entry loaded into g1
    int64_t g1;
    int r2;        // claimed list position, entry not loaded yet
};

__device__ __forceinline__ void claim_init(RowClaim& c, int* counter, int nlist, const int32_t* rowlist) {
    if (threadIdx.x == 0) {
        c.r1 = atomicAdd(counter, 1);
        c.g1 = c.r1 < nlist ? rowlist[c.r1] : -1;
        c.r2 = atomicAdd(counter, 1);
    }
}

// Returns the global row or -1; s_row = {global row, row in its matrix, list position}.
__device__ __forceinline__ int64_t next_row_b(RowClaim& c, int* counter, int nlist, const int32_t* rowlist,
                                              const SpgRows& R, SpgArgs* s_args, int64_t* s_row) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int r = c.r1;
        const int64_t gi = c.g1;
        c.r1 = c.r2;
        c.g1 = c.r2 < nlist ? rowlist[c.r2] : -1;
        c.r2 = atomicAdd(counter, 1);
        int64_t li = gi;
        if (gi >= 0) {
            if (R.table) {
                const int b = batch_of(R, gi);
                *s_args = R.table[b];
                li = gi - R.row_off[b];
            } else {
                *s_args = R.one;
            }
        }
        s_row[0] = gi;
        s_row[1] = li;
        s_row[2] = r;
    }
    __syncthreads();
    return s_row[0];
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_symbolic_rank(SpgRows R, int ncell_max, const int32_t* __restrict__ rowlist, const int* __restrict__ nlist_ptr,
                int* __restrict__ counter, int64_t* __restrict__ row_nnz, int* __restrict__ max_nnz,
                uint4* __restrict__ rec, int2* __restrict__ rec_meta, int sparse_max) {
    extern __shared__ uint4 smem_raw[];
    const SymLayout L = sym_layout(ncell_max);
    const RankLayout LR = rank_layout(ncell_max, 0, 0, 4, false);  // record layout
    const int NWmax = ncell_max * 32;
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem_raw);
    uint32_t* bits = reinterpret_cast<uint32_t*>(sm + L.bits);
    uint32_t* summ = reinterpret_cast<uint32_t*>(sm + L.summ);  // one summary word per cell
    int* cellbase = reinterpret_cast<int*>(sm + L.cellbase);
    const int64_t rec_bytes = int64_t(LR.winfirst);
    __shared__ TaskSmem<NT> ts;
    __shared__ SpgArgs s_args;
    __shared__ int64_t s_row[3];
    __shared__ int s_red[NT / 32 + 1];
    __shared__ int s_zb[RK_MAX_COLS / RK_CELL];  // sparse record: first slot of each cell's words
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int w = threadIdx.x; w < NWmax; w += NT) bits[w] = 0u;
    for (int c = threadIdx.x; c < ncell_max; c += NT) summ[c] = 0u;
    const int nlist = *nlist_ptr;
    RowClaim rc;
    claim_init(rc, counter, nlist, rowlist);
    int local_max = 0;
    for (;;) {
        const int64_t gi = next_row_b(rc, counter, nlist, rowlist, R, &s_args, s_row);
        if (gi < 0) break;
        const SpgArgs& g = s_args;
        const int64_t i = s_row[1];
        const int NW = g.ncell * 32;
        int64_t alo, ahi;
        row_range(g.a_ptr, i, g.nnzA, alo, ahi);
        for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
            const int ntasks = load_tasks<NT, int, false>(g, nullptr, 0, p0, ahi, 0, 0, ts, nullptr);
            walk_tasks_bits<NT>(g, ts, ntasks, bits);
            __syncthreads();
        }
        int tot;
        if (rec) {
            // summary bits: one ballot per 32 words
            for (int c = wid; c < g.ncell; c += NT / 32) {
                const unsigned m = __ballot_sync(0xffffffffu, bits[c * 32 + lane] != 0u);
                if (lane == 0) summ[c] = m;
            }
            __syncthreads();
            // ranks: the cells' exclusive prefix (a word's rank inside its cell is
            // taken by a warp scan when the record is written); the whole rank
            // structure is stored for the numeric pass
            constexpr int CPT = (RK_MAX_COLS / RK_CELL + NT - 1) / NT;
            int cnt[CPT];
            int ctot = 0;
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int c = threadIdx.x * CPT + q;
                int n = 0;
                if (c < g.ncell) {
                    uint32_t sw = summ[c];
                    while (sw) {
                        const int w = c * 32 + __ffs(sw) - 1;
                        sw &= sw - 1;
                        n += __popc(bits[w]);
                    }
                }
                cnt[q] = n;
                ctot += n;
            }
            int ex = block_exclusive_scan<NT, int>(ctot, s_red, tot);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int c = threadIdx.x * CPT + q;
                if (c < g.ncell) cellbase[c] = ex;
                ex += cnt[q];
            }
            if (threadIdx.x == 0) cellbase[g.ncell] = tot;
            __syncthreads();
            unsigned char* dst = reinterpret_cast<unsigned char*>(rec) + gi * rec_bytes;  // slot of the global row
            // light rows (one rank window in the numeric pass, few non-zero words): only
            // the non-zero words, as (bits, word << 18 | rank of the word's first column)
            bool sparse = false;
            if (tot <= sparse_max) {
                int nz = 0;
#pragma unroll
                for (int q = 0; q < CPT; ++q) {
                    const int c = threadIdx.x * CPT + q;
                    if (c < g.ncell) nz += __popc(summ[c]);
                }
                int nzt;
                int zex = block_exclusive_scan<NT, int>(nz, s_red, nzt);
                if (nzt <= RK_SPARSE_MAX_WORDS) {
                    sparse = true;
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        const int c = threadIdx.x * CPT + q;
                        if (c < g.ncell) {
                            s_zb[c] = zex;
                            zex += __popc(summ[c]);
                        }
                    }
                    __syncthreads();
                    // a warp per cell, a lane per word: the non-zero words in order
                    uint2* dsp = reinterpret_cast<uint2*>(dst);
                    for (int c = wid; c < g.ncell; c += NT / 32) {
                        const uint32_t sw = summ[c];
                        if (!sw) continue;
                        const uint32_t b = bits[c * 32 + lane];
                        const int ex = warp_exclusive_sum(__popc(b), lane);
                        if (b)
                            dsp[s_zb[c] + __popc(sw & ((1u << lane) - 1u))] =
                                make_uint2(b, (uint32_t(c * 32 + lane) << 18) | uint32_t(cellbase[c] + ex));
                    }
                    if (threadIdx.x == 0) rec_meta[gi] = make_int2(nzt, tot);
                }
            }
            if (!sparse) {
                // the dense record, in the numeric kernel's layout: (bits, rank of the
                // word) pairs, the summary and the cell prefix; a warp per cell
                uint2* dwb = reinterpret_cast<uint2*>(dst + LR.wb);
                for (int c = wid; c < ncell_max; c += NT / 32) {
                    const int w = c * 32 + lane;
                    const uint32_t b = bits[w];
                    const int ex = warp_exclusive_sum(__popc(b), lane);
                    dwb[w] = make_uint2(b, b ? uint32_t(cellbase[c] + ex) : 0u);
                }
                uint32_t* dsumm = reinterpret_cast<uint32_t*>(dst + LR.summ);
                for (int c = threadIdx.x; c < ncell_max; c += NT) dsumm[c] = summ[c];
                int* dcb = reinterpret_cast<int*>(dst + LR.cellbase);
                for (int c = threadIdx.x; c <= ncell_max; c += NT) dcb[c] = c <= g.ncell ? cellbase[c] : tot;
                if (threadIdx.x == 0) rec_meta[gi] = make_int2(-1, tot);
            }
            __syncthreads();
            for (int c = threadIdx.x; c < g.ncell; c += NT) {
                uint32_t sw = summ[c];
                summ[c] = 0u;
                while (sw) {
                    const int w = c * 32 + __ffs(sw) - 1;
                    sw &= sw - 1;
                    bits[w] = 0u;
                }
            }
        } else {
            int cnt = 0;
            for (int w = threadIdx.x; w < NW; w += NT) {
                const uint32_t b = bits[w];
                if (b) {
                    cnt += __popc(b);
                    bits[w] = 0u;
                }
            }
            for (int c = threadIdx.x; c < g.ncell; c += NT) summ[c] = 0u;
            (void)block_exclusive_scan<NT, int>(cnt, s_red, tot);
        }
        if (threadIdx.x == 0) {
            row_nnz[gi] = tot;
            local_max = max(local_max, tot);
        }
    }
    if (threadIdx.x == 0 && local_max) atomicMax(max_nnz, local_max);
}

// ctab[k*(ncell+1) + c] = number of entries of B_k with column < c * RK_CELL, for
// matrix blockIdx.y of the batch (or the single matrix).
__global__ void k_cell_offsets(SpgRows R) {
    const SpgArgs g = R.table ? R.table[blockIdx.y] : R.one;
    int32_t* ctab = const_cast<int32_t*>(g.ctab);
    if (!ctab) return;
    // a warp per row of B, lanes over the cells (coalesced writes); each lane's
    // binary search reads the row's columns, which stay in L1 across the lanes
    const int lane = threadIdx.x & 31;
    const int64_t stride = int64_t(g.ncell) + 1;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; k < g.K; k += nwarps) {
        int64_t lo, hi;
        row_range(g.b_ptr, k, g.nnzB, lo, hi);
        int32_t* t = ctab + k * stride;
        for (int c = lane; c <= g.ncell; c += 32) {
            const int64_t target = int64_t(c) << RK_CELL_SHIFT;
            int64_t x = lo, y = hi;
            while (x < y) {
                const int64_t m = (x + y) >> 1;
                if (int64_t(g.b_col[m]) < target) x = m + 1; else y = m;
            }
            t[c] = int32_t(x - lo);
        }
    }
}

// Row analysis over global rows (batch-aware): ub and log2 bins.  With single !=
// null, a row with one stored entry whose B row is not empty goes to BIN_COPY and
// its output count is final: single[gi] = ub (one product per output column).
// Eight lanes sum a row; each 8-lane group takes a chunk of `chunk` consecutive
// rows, so the matrix of a batch is looked up once per group and matrix.  Chunks
// are dealt to groups in a scattered order (group g takes chunk g * UB_SPREAD mod
// the number of chunks; UB_SPREAD is a prime above the chunk count), so that the
// heavy rows of a power-law matrix, which sit together, spread over the grid.  A
// group loads the row pointers of eight rows at once (lane j: row j of the window)
// and walks a row's entries four per lane per round (its loads issued together).  Rows with more than UB_HEAVY
// stored entries are queued and summed by the whole block at the end.
constexpr int UB_LANES = 8;
constexpr int UB_NT = 256;
constexpr int UB_HEAVY = 256;
constexpr int UB_QCAP = 128;
constexpr int UB_UNROLL = 4;
constexpr int64_t UB_SPREAD = 1000003;

__device__ __forceinline__ void ub_finish(int64_t gi, int64_t len, int64_t sum, int64_t* __restrict__ ub,
                                          int64_t* __restrict__ single, int* s_bins) {
    ub[gi] = sum;
    const bool one = single && len == 1 && sum > 0;
    if (one) single[gi] = sum;
    atomicAdd(&s_bins[one ? BIN_COPY : bin_of(sum)], 1);
}

__global__ void __launch_bounds__(UB_NT, 5) k_row_ub_b(SpgRows R, int64_t NR, int64_t chunk, int64_t nchunks,
                                                    int64_t spread, int64_t* __restrict__ ub, int* __restrict__ bin_count,
                                                    int64_t* __restrict__ single,
                                                    int32_t* __restrict__ row_mat = nullptr) {
    __shared__ int s_bins[NBINS_ALL];
    __shared__ int64_t s_q[UB_QCAP];
    __shared__ int s_qb[UB_QCAP];
    __shared__ int s_nq;
    __shared__ int64_t s_red[UB_NT / 32];
    for (int t = threadIdx.x; t < NBINS_ALL; t += blockDim.x) s_bins[t] = 0;
    if (threadIdx.x == 0) s_nq = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int sub = lane & (UB_LANES - 1);
    const int lead = lane & ~(UB_LANES - 1);
    const unsigned gmask = 0xffu << lead;
    const int64_t grp = (int64_t(blockIdx.x) * UB_NT + threadIdx.x) / UB_LANES;
    const int64_t ch = grp < nchunks ? (grp * spread) % nchunks : nchunks;
    const int64_t r0 = ch * chunk;
    const int64_t r1 = r0 + chunk < NR ? r0 + chunk : NR;
    SpgArgs g = R.one;
    int b = 0;
    int64_t rlo = 0, rhi = R.table ? -1 : NR;  // global rows of the current matrix
    for (int64_t w0 = r0; w0 < r1;) {
        if (w0 >= rhi) {
            b = batch_of(R, w0);
            rlo = R.row_off[b];
            rhi = R.row_off[b + 1];
            g = R.table[b];
        }
        // a window of up to eight rows of one matrix: lane j holds row w0 + j's range
        int64_t w1 = w0 + UB_LANES;
        if (w1 > r1) w1 = r1;
        if (w1 > rhi) w1 = rhi;
        int64_t my_lo = 0, my_hi = 0;
        if (w0 + sub < w1) {
            const int64_t i = w0 + sub - rlo;
            int64_t x = g.a_ptr[i], y = g.a_ptr[i + 1];
            x = x < 0 ? 0 : (x > g.nnzA ? g.nnzA : x);
            y = y < x ? x : (y > g.nnzA ? g.nnzA : y);
            my_lo = x;
            my_hi = y;
            if (row_mat) row_mat[w0 + sub] = b;
        }
        for (int64_t gi = w0; gi < w1; ++gi) {
            const int src = lead + int(gi - w0);
            const int64_t lo = __shfl_sync(gmask, my_lo, src);
            const int64_t hi = __shfl_sync(gmask, my_hi, src);
            if (hi - lo > UB_HEAVY) {
                int slot = 0;
                if (sub == 0) slot = atomicAdd(&s_nq, 1);
                slot = __shfl_sync(gmask, slot, lead);
                if (slot < UB_QCAP) {
                    if (sub == 0) {
                        s_q[slot] = gi;
                        s_qb[slot] = b;
                    }
                    continue;
                }
            }
            int64_t sum = 0;
            for (int64_t p = lo + sub; p < hi; p += UB_UNROLL * UB_LANES) {
                int32_t k[UB_UNROLL];
#pragma unroll
                for (int u = 0; u < UB_UNROLL; ++u) {
                    const int64_t q = p + int64_t(u) * UB_LANES;
                    k[u] = q < hi ? g.a_col[q] : -1;
                }
                int64_t bl[UB_UNROLL], bh[UB_UNROLL];
#pragma unroll
                for (int u = 0; u < UB_UNROLL; ++u) {
                    bl[u] = bh[u] = 0;
                    if ((uint64_t)k[u] < (uint64_t)g.K) row_range(g.b_ptr, k[u], g.nnzB, bl[u], bh[u]);
                }
#pragma unroll
                for (int u = 0; u < UB_UNROLL; ++u) sum += bh[u] - bl[u];
            }
#pragma unroll
            for (int o = UB_LANES / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(gmask, sum, o);
            if (sub == 0) ub_finish(gi, hi - lo, sum, ub, single, s_bins);
        }
        w0 = w1;
    }
    __syncthreads();
    const int nq = s_nq < UB_QCAP ? s_nq : UB_QCAP;
    for (int q = 0; q < nq; ++q) {
        const int64_t gi = s_q[q];
        const SpgArgs& gq = R.table ? R.table[s_qb[q]] : R.one;
        const int64_t i = gi - (R.table ? R.row_off[s_qb[q]] : 0);
        int64_t lo, hi;
        row_range(gq.a_ptr, i, gq.nnzA, lo, hi);
        int64_t sum = 0;
        for (int64_t p = lo + threadIdx.x; p < hi; p += UB_NT) {
            const int32_t k = gq.a_col[p];
            if ((uint64_t)k < (uint64_t)gq.K) {
                int64_t bl, bh;
                row_range(gq.b_ptr, k, gq.nnzB, bl, bh);
                sum += bh - bl;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) s_red[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t tot = 0;
            for (int w = 0; w < UB_NT / 32; ++w) tot += s_red[w];
            ub_finish(gi, hi - lo, tot, ub, single, s_bins);
        }
        __syncthreads();
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NBINS_ALL; t += blockDim.x)
        if (s_bins[t]) atomicAdd(&bin_count[t], s_bins[t]);
}

// Launch of k_row_ub_b: one 8-lane group per eight of the SMs' thread slots, each
// with an equal chunk of consecutive rows.
static void launch_row_ub(const stc_handle* h, const SpgRows& R, int64_t NR, int64_t* ub, int* bin_count,
                          int64_t* single, int32_t* row_mat, cudaStream_t s) {
    if (NR <= 0) return;
    // one wave: as many groups as the SMs hold at once
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_row_ub_b, UB_NT, 0) != cudaSuccess || per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    const int64_t groups_max = int64_t(h->num_sms) * per_sm * (UB_NT / UB_LANES);
    int64_t chunk = (NR + groups_max - 1) / groups_max;
    if (chunk < 1) chunk = 1;
    const int64_t nchunks = (NR + chunk - 1) / chunk;
    // a prime above the chunk count makes g -> g * spread mod nchunks a permutation
    const int64_t spread = nchunks < UB_SPREAD ? UB_SPREAD : 1;
    const int64_t blocks = (nchunks * UB_LANES + UB_NT - 1) / UB_NT;
    k_row_ub_b<<<unsigned(blocks), UB_NT, 0, s>>>(R, NR, chunk, nchunks, spread, ub, bin_count, single, row_mat);
}

// Rows with a single stored entry a = A_ik: C_i = f(a, B_k) entry by entry, in B_k's
// column order (each output column has exactly one product, so no (+) applies).
// Warp per row over rowlist[*nlist, *nlist + *ncopy).
template <int ALG>
__global__ void __launch_bounds__(256) k_copy_rows(SpgRows R, const int32_t* __restrict__ rowlist,
                                                   const int* __restrict__ nlist_ptr,
                                                   const int* __restrict__ ncopy_ptr,
                                                   const int64_t* __restrict__ c_ptr, int32_t* __restrict__ c_col,
                                                   void* __restrict__ c_val) {
    using T = Tr<ALG>;
    using AT = typename T::A;
    using BT = typename T::B;
    auto* cval = static_cast<typename T::C*>(c_val);
    const int lane = threadIdx.x & 31;
    const int first = *nlist_ptr, n = *ncopy_ptr;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < n; q += nwarps) {
        const int64_t gi = rowlist[first + q];
        SpgArgs g;
        int64_t i = gi;
        if (R.table) {
            const int b = batch_of(R, gi);
            g = R.table[b];
            i = gi - R.row_off[b];
        } else {
            g = R.one;
        }
        const int64_t p = g.a_ptr[i];
        const int32_t k = g.a_col[p];
        const AT a = static_cast<const AT*>(g.a_val)[p];
        int64_t bl, bh;
        row_range(g.b_ptr, k, g.nnzB, bl, bh);
        const int64_t o0 = c_ptr[gi] - bl;
        const BT* __restrict__ bval = static_cast<const BT*>(g.b_val);
        for (int64_t e = bl + lane; e < bh; e += 32) {
            c_col[o0 + e] = g.b_col[e] + g.col_base;
            cval[o0 + e] = T::one(a, bval[e]);
        }
    }
}

// ----------------------------------------------------------------- warp-per-row kernels
//
// Narrow outputs (at most WR_MAX_COLS columns, e.g. many small independent
// products): one warp owns one output row, with its own slice of shared memory and
// no CTA barrier.  The products of a row are walked flattened: 32 stored entries
// A_ik at a time, lane j holds entry j and its B row; an inclusive warp scan of the
// B row lengths numbers the chunk's products 0..T-1, and product q belongs to the
// first lane whose prefix exceeds q (a five-step shuffle search), so every lane
// works on a product whatever the B row lengths are.  Rows are claimed from a
// device counter, heaviest first (the order of the row list).
//
//   count pass:   bitmap of the row's columns (one bit per output column), popcount
//   numeric pass: the same bitmap, the rank of every 32-column word (prefix of
//                 popcounts, words owned lane-strided so the prefix is one warp
//                 scan per 32 words), then every product accumulated into the
//                 rank-indexed value array with the algebra's (+), columns written
//                 from the bitmap and values by rank, both coalesced.

constexpr int WR_MAX_COLS = 16384;
constexpr int WR_WORDS = WR_MAX_COLS / 32;  // 512 bitmap words per warp
constexpr int WR_ROUNDS = WR_WORDS / 32;    // 16 words per lane
constexpr int WR_U = 8;                     // products per lane in flight per step
constexpr int WR_VCAP = 2560;               // value slots per warp of the wide numeric instance
constexpr int WR_VCAP_S = 896;              // value slots per warp of the narrow numeric instance (fp32: four
                                            // 8-warp CTAs of 56 KB fit an SM)
constexpr int WR_UB_LOG2 = 15;              // rows with 2^15 products or more stay on the CTA kernels
constexpr int WR_COUNT_WARPS = 8;           // warps per CTA of the count pass
constexpr int WR_NUM_WARPS = 4;             // warps per CTA of the wide numeric instance
constexpr int WR_NUM_WARPS_S = 8;           // warps per CTA of the narrow numeric instance

template <int ALG, int VCAP>
__host__ __device__ constexpr size_t wr_warp_bytes() {
    return size_t(WR_WORDS) * 4 + size_t(WR_WORDS) * 2 + size_t(VCAP) * sizeof(typename Tr<ALG>::Acc);
}

// Matrix of global row gi: its arguments and its row inside the matrix.
__device__ __forceinline__ const SpgArgs& wr_args(const SpgRows& R, const int32_t* __restrict__ row_mat,
                                                  int64_t gi, int64_t& i) {
    if (!R.table) {
        i = gi;
        return R.one;
    }
    const int b = row_mat[gi];
    i = gi - R.row_off[b];
    return R.table[b];
}

// Per-warp table of the current chunk of (at most 32) stored entries of A: the
// end of each entry's product range, the B position of its product q (shift + q)
// and its value.
template <class AT>
struct WrChunk {
    int end[32];
    int64_t shift[32];
    AT aval[32];
};

// Walk the products of row [alo, ahi) of A: f(col[], bv[], av[]) receives WR_U
// products per lane per call (col < 0: no product in that slot).  Lane j loads
// entry j of a 32-entry chunk; an inclusive warp scan of the B row lengths numbers
// the chunk's products, and every lane follows its products' owners in the chunk
// table (owners only move forward as q grows, a step or two per 32 products).
template <bool WITH_VAL, class AT, class BT, class F>
__device__ __forceinline__ void wr_walk(const SpgArgs& g, int64_t alo, int64_t ahi, int lane, WrChunk<AT>& tab,
                                        F f) {
    const BT* __restrict__ bval = static_cast<const BT*>(g.b_val);
    for (int64_t c0 = alo; c0 < ahi; c0 += 32) {
        const int64_t p = c0 + lane;
        int len = 0;
        int64_t base = 0;
        AT av = AT();
        if (p < ahi) {
            const int32_t k = g.a_col[p];
            if ((uint64_t)k < (uint64_t)g.K) {
                int64_t bl, bh;
                row_range(g.b_ptr, k, g.nnzB, bl, bh);
                len = int(bh - bl);
                base = bl;
                if (WITH_VAL) av = static_cast<const AT*>(g.a_val)[p];
            }
        }
        int end = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, end, o);
            if (lane >= o) end += t;
        }
        const int total = __shfl_sync(0xffffffffu, end, 31);
        __syncwarp();
        tab.end[lane] = end;
        tab.shift[lane] = base - (end - len);  // B position of product q of this entry: shift + q
        if (WITH_VAL) tab.aval[lane] = av;
        __syncwarp();
        int own = 0;
        for (int q0 = 0; q0 < total; q0 += 32 * WR_U) {
            int col[WR_U];
            BT bv[WR_U];
            AT aa[WR_U];
#pragma unroll
            for (int u = 0; u < WR_U; ++u) {
                col[u] = -1;
                const int q = q0 + u * 32 + lane;
                if (q < total) {
                    while (tab.end[own] <= q) ++own;  // q < total = end[31]: stops at 31 at the latest
                    const int64_t pos = tab.shift[own] + q;
                    col[u] = g.b_col[pos];
                    if (WITH_VAL) {
                        bv[u] = bval[pos];
                        aa[u] = tab.aval[own];
                    }
                }
            }
            f(col, bv, aa);
        }
    }
}

// Set the bitmap bit of every product's column (columns outside [0, ncols) are
// skipped: they can only come from input that validation would reject).
template <class AT, class BT>
__device__ __forceinline__ void wr_bits(const SpgArgs& g, int64_t alo, int64_t ahi, int lane, uint32_t* bits,
                                        WrChunk<AT>& tab) {
    const unsigned nc = unsigned(g.ncols);
    wr_walk<false, AT, BT>(g, alo, ahi, lane, tab, [&](const int* col, const BT*, const AT*) {
        uint32_t cur[WR_U];
#pragma unroll
        for (int u = 0; u < WR_U; ++u) cur[u] = unsigned(col[u]) < nc ? bits[col[u] >> 5] : ~0u;
#pragma unroll
        for (int u = 0; u < WR_U; ++u) {
            if (unsigned(col[u]) < nc) {
                const uint32_t m = 1u << (col[u] & 31);
                if (!(cur[u] & m)) atomicOr(&bits[col[u] >> 5], m);
            }
        }
    });
}

// Count pass: row_nnz[gi] = nnz(C_i) for the listed rows [*lo_ptr, *hi_ptr)
// (lo_ptr NULL: from 0).
// bm (may be null): every row's bitmap is also stored, ceil(ncols / 32) words at
// bm[g.bm_off + i * ceil(ncols / 32)], for the numeric pass.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_wr_count(SpgRows R, const int32_t* __restrict__ row_mat, const int32_t* __restrict__ rowlist,
           const int* __restrict__ lo_ptr, const int* __restrict__ hi_ptr, int* __restrict__ counter,
           int64_t* __restrict__ row_nnz, int* __restrict__ max_nnz, uint32_t* __restrict__ bm) {
    __shared__ uint32_t s_bits[WARPS][WR_WORDS];
    __shared__ WrChunk<int> s_tab[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* bits = s_bits[wid];
#pragma unroll
    for (int t = 0; t < WR_ROUNDS; ++t) bits[t * 32 + lane] = 0u;
    __syncwarp();
    const int first = lo_ptr ? *lo_ptr : 0, last = *hi_ptr;
    int local_max = 0;
    for (;;) {
        int r = 0;
        if (lane == 0) r = first + atomicAdd(counter, 1);
        r = __shfl_sync(0xffffffffu, r, 0);
        if (r >= last) break;
        const int64_t gi = rowlist[r];
        int64_t i;
        const SpgArgs& g = wr_args(R, row_mat, gi, i);
        int64_t alo, ahi;
        row_range(g.a_ptr, i, g.nnzA, alo, ahi);
        wr_bits<int, int>(g, alo, ahi, lane, bits, s_tab[wid]);
        __syncwarp();
        int n = 0;
        const int nw = int((g.ncols + 31) >> 5), nr = (nw + 31) >> 5;  // words, rounds of 32 words
        uint32_t* dst = bm ? bm + g.bm_off + i * nw : nullptr;
        for (int t = 0; t < nr; ++t) {
            const uint32_t b = bits[t * 32 + lane];
            n += __popc(b);
            if (dst && t * 32 + lane < nw) dst[t * 32 + lane] = b;
            bits[t * 32 + lane] = 0u;
        }
        n = __reduce_add_sync(0xffffffffu, n);
        if (lane == 0) row_nnz[gi] = n;
        local_max = max(local_max, n);
        __syncwarp();
    }
    if (lane == 0 && local_max) atomicMax(max_nnz, local_max);
}

// Numeric pass over the listed rows [0, *nlist), every one with at most VCAP
// output entries: C_i written at c_ptr[gi] (columns ascending).  A row whose
// count differs from its slot raises STC_FLAG_INTERNAL and is not written.
template <int ALG, int WARPS, int VCAP>
__global__ void __launch_bounds__(WARPS * 32)
k_wr_numeric(SpgRows R, const int32_t* __restrict__ row_mat, const int32_t* __restrict__ rowlist,
             const int* __restrict__ nlist_ptr, int* __restrict__ counter, const int64_t* __restrict__ c_ptr,
             int32_t* __restrict__ c_col, void* __restrict__ c_val, int* __restrict__ flags,
             const uint32_t* __restrict__ bm) {
    static_assert(VCAP <= 65535 && WR_MAX_COLS <= 65535, "ranks are kept in 16 bits");
    using T = Tr<ALG>;
    using AT = typename T::A;
    using BT = typename T::B;
    using Acc = typename T::Acc;
    extern __shared__ uint4 smem_raw[];
    __shared__ WrChunk<AT> s_tab[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* base = reinterpret_cast<unsigned char*>(smem_raw) + size_t(wid) * wr_warp_bytes<ALG, VCAP>();
    uint32_t* bits = reinterpret_cast<uint32_t*>(base);
    uint16_t* wpre = reinterpret_cast<uint16_t*>(base + WR_WORDS * 4);
    Acc* vals = reinterpret_cast<Acc*>(base + WR_WORDS * 6);
#pragma unroll
    for (int t = 0; t < WR_ROUNDS; ++t) bits[t * 32 + lane] = 0u;
    for (int r = lane; r < VCAP; r += 32) vals[r] = T::empty();
    __syncwarp();
    auto* cval = static_cast<typename T::C*>(c_val);
    const int nlist = *nlist_ptr;
    for (;;) {
        int r = 0;
        if (lane == 0) r = atomicAdd(counter, 1);
        r = __shfl_sync(0xffffffffu, r, 0);
        if (r >= nlist) break;
        const int64_t gi = rowlist[r];
        int64_t i;
        const SpgArgs& g = wr_args(R, row_mat, gi, i);
        int64_t alo, ahi;
        row_range(g.a_ptr, i, g.nnzA, alo, ahi);
        const int64_t o0 = c_ptr[gi];
        const int64_t want = c_ptr[gi + 1] - o0;
        // only the words of the matrix's columns are used: nr rounds of 32 words
        const int nw = int((g.ncols + 31) >> 5), nr = (nw + 31) >> 5;
        // 1) bitmap: stored by the count pass (bm), else built here
        if (bm) {
            const uint32_t* src = bm + g.bm_off + i * nw;
            for (int t = 0; t < nr; ++t)
                if (t * 32 + lane < nw) bits[t * 32 + lane] = src[t * 32 + lane];
        } else {
            wr_bits<AT, BT>(g, alo, ahi, lane, bits, s_tab[wid]);
        }
        __syncwarp();
        // 2) ranks: words owned lane-strided, one warp scan per round of 32 words
        int run = 0;
        for (int t = 0; t < nr; ++t) {
            const int c = __popc(bits[t * 32 + lane]);
            int x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            wpre[t * 32 + lane] = uint16_t(run + x - c);
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        const int count = run;
        const bool ok = count == want && count <= VCAP;
        if (!ok && lane == 0) atomicOr(flags, STC_FLAG_INTERNAL);
        __syncwarp();
        if (ok) {
            // 3) values by rank
            const unsigned nc = unsigned(g.ncols);
            wr_walk<true, AT, BT>(g, alo, ahi, lane, s_tab[wid], [&](const int* col, const BT* bv, const AT* av) {
                int rk[WR_U];
#pragma unroll
                for (int u = 0; u < WR_U; ++u) {
                    rk[u] = -1;
                    if (unsigned(col[u]) < nc) {
                        const int w = col[u] >> 5;
                        rk[u] = int(wpre[w]) + __popc(bits[w] & ((1u << (col[u] & 31)) - 1u));
                    }
                }
#pragma unroll
                for (int u = 0; u < WR_U; ++u)
                    if (rk[u] >= 0) T::combine(vals, rk[u], av[u], bv[u]);
            });
            __syncwarp();
            // 4) columns from the bitmap (each lane's word covers ranks wpre[w] ..)
#pragma unroll 1
            for (int t = 0; t < nr; ++t) {
                const int w = t * 32 + lane;
                uint32_t b = bits[w];
                int64_t dst = o0 + wpre[w];
                while (b) {
                    const int bit = __ffs(b) - 1;
                    b &= b - 1;
                    c_col[dst++] = w * 32 + bit + g.col_base;
                }
            }
            for (int q = lane; q < count; q += 32) {
                cval[o0 + q] = T::out(vals[q]);
                vals[q] = T::empty();
            }
        }
        for (int t = 0; t < nr; ++t) bits[t * 32 + lane] = 0u;
        __syncwarp();
    }
}

// Rows [0, NR) with output entries, split for the numeric pass into three lists
// in row order, so that the rows of one matrix of a batch run together while its B
// stays in L2: out[0] rows with at most WR_VCAP_S output entries, out[1] at most
// WR_VCAP, out[2] the rest: rows with 2^WR_UB_LOG2 products or more (too many for
// one warp), rows of A with more than wide_len stored entries (compensated sums,
// CTA kernels only) and wider outputs.  Rows with one stored entry (the copy
// kernel's) are left out; n[0..2] sizes.  A block takes 256 consecutive rows.
__global__ void __launch_bounds__(256) k_split_by_count(SpgRows R, const int32_t* __restrict__ row_mat,
                                                        int64_t wide_len, int64_t NR,
                                                        const int64_t* __restrict__ ub,
                                                        const int64_t* __restrict__ c_ptr,
                                                        int32_t* __restrict__ out0, int32_t* __restrict__ out1,
                                                        int32_t* __restrict__ out2, int* __restrict__ n) {
    __shared__ int s_cnt[3], s_base[3];
    for (int64_t r0 = int64_t(blockIdx.x) * blockDim.x; r0 < NR; r0 += int64_t(gridDim.x) * blockDim.x) {
        if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
        __syncthreads();
        const int64_t gi = r0 + threadIdx.x;
        int cls = 3, local = 0;
        if (gi < NR) {
            const int64_t u = ub[gi];
            const int64_t c = c_ptr[gi + 1] - c_ptr[gi];
            if (u > 0 && c > 0) {
                const int b = row_mat ? row_mat[gi] : 0;
                const SpgArgs& g = R.table ? R.table[b] : R.one;
                int64_t lo, hi;
                row_range(g.a_ptr, gi - (R.table ? R.row_off[b] : 0), g.nnzA, lo, hi);
                if (hi - lo != 1) {
                    const bool heavy = bin_of(u) > WR_UB_LOG2;
                    cls = (heavy || hi - lo > wide_len) ? 2 : c <= WR_VCAP_S ? 0 : c <= WR_VCAP ? 1 : 2;
                }
            }
        }
        if (cls < 3) local = atomicAdd(&s_cnt[cls], 1);
        __syncthreads();
        if (threadIdx.x < 3) s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&n[threadIdx.x], s_cnt[threadIdx.x]) : 0;
        __syncthreads();
        if (cls < 3) (cls == 0 ? out0 : cls == 1 ? out1 : out2)[s_base[cls] + local] = int32_t(gi);
        __syncthreads();
    }
}

// Per-batch row pointers: rp[row_off[b] + b + i] = c_ptr[row_off[b] + i] - c_ptr[row_off[b]].
__global__ void k_rebase_rowptr(SpgRows R, const int64_t* __restrict__ c_ptr, int64_t* __restrict__ rp) {
    const int64_t total = R.row_off[R.nb] + R.nb;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        int lo = 0, hi = R.nb - 1;  // last b with row_off[b] + b <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (R.row_off[mid] + mid <= e) lo = mid; else hi = mid - 1;
        }
        const int64_t i = e - (R.row_off[lo] + lo);
        rp[e] = c_ptr[R.row_off[lo] + i] - c_ptr[R.row_off[lo]];
    }
}

// c_ptr at the first row of every matrix of the batch (and the total).
__global__ void k_batch_bounds(SpgRows R, const int64_t* __restrict__ c_ptr, int64_t* __restrict__ out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= R.nb; b += gridDim.x * blockDim.x)
        out[b] = c_ptr[R.row_off[b]];
}

// MASKED: the rank records describe a given output structure (a mask M): products
// whose column is not in the row's structure are skipped, entries that no product
// reaches get the additive identity, and no columns are written (c_col unused).
template <int ALG, int NT, int MINB, bool MASKED = false>
__global__ void __launch_bounds__(NT, MINB)
k_numeric_rank(SpgRows R, int ncell_max, int vcap, int maxwin,
               const int32_t* __restrict__ rowlist, const int* __restrict__ nlist_ptr,
               int* __restrict__ counter, RankOut out, int32_t* __restrict__ c_col,
               void* __restrict__ c_val, int* __restrict__ flags, const uint4* __restrict__ rec,
               const int2* __restrict__ rec_meta) {
    using T = Tr<ALG>;
    using AT = typename T::A;
    using BT = typename T::B;
    using Acc = typename T::Acc;
    // masked products skip most products at the rank lookup, so per-task overhead
    // dominates there: long tasks
    constexpr int VSUB = MASKED ? RK_SUB : value_task_entries(ALG);
    extern __shared__ uint4 smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem_raw);
    const RankLayout L = rank_layout(ncell_max, vcap, maxwin, sizeof(Acc), ALG == ALG_MULTPATH);
    uint2* wb = reinterpret_cast<uint2*>(sm + L.wb);
    uint32_t* wbx = reinterpret_cast<uint32_t*>(sm + L.wb);  // x of word w at 2w, y at 2w + 1
    uint32_t* summ = reinterpret_cast<uint32_t*>(sm + L.summ);
    int* cellbase = reinterpret_cast<int*>(sm + L.cellbase);
    int* winfirst = reinterpret_cast<int*>(sm + L.winfirst);
    Acc* vals = reinterpret_cast<Acc*>(sm + L.vals);
    int32_t* scol = reinterpret_cast<int32_t*>(sm + L.scol);  // column of each rank of the window
    double* sig = reinterpret_cast<double*>(sm + L.sig);
    __shared__ TaskSmem<NT> ts;
    __shared__ AT s_aval[NT];
    __shared__ SpgArgs s_args;
    __shared__ int64_t s_row[3];
    __shared__ int s_warp[NT / 32 + 1];
    __shared__ int s_nwin;
    __shared__ int64_t s_dst;
    __shared__ int s_fits;

    for (int w = threadIdx.x; w < ncell_max * 32; w += NT) wb[w] = make_uint2(0u, 0u);
    for (int c = threadIdx.x; c < ncell_max; c += NT) summ[c] = 0u;
    for (int r = threadIdx.x; r < vcap; r += NT) {
        vals[r] = T::empty();
        if constexpr (ALG == ALG_MULTPATH) sig[r] = 0.0;
    }
    const int nlist = *nlist_ptr;
    RowClaim rc;
    claim_init(rc, counter, nlist, rowlist);
    const int vstep = vcap - RK_CELL;  // rank span that starts a new window
    auto* cval = static_cast<typename T::C*>(c_val);
    double err_sum = 0.0;  // thread 0: this CTA's share of out.err, added once at the end

    for (;;) {
        const int64_t gi = next_row_b(rc, counter, nlist, rowlist, R, &s_args, s_row);
        if (gi < 0) break;
        const SpgArgs& g = s_args;
        const int64_t i = s_row[1];
        const int ncell = g.ncell;
        const BT* __restrict__ bval = static_cast<const BT*>(g.b_val);
        int64_t alo, ahi;
        row_range(g.a_ptr, i, g.nnzA, alo, ahi);
        // compensated fp32 sums for this row (the column buffer holds the corrections)
        const bool wide = ALG == ALG_PT_F32 && !MASKED && ahi - alo > F32_WIDE_ROW;
        const int64_t o0 = out.ptr[gi];
        const int64_t o1 = out.cap ? o0 + out.cap[gi] : out.ptr[gi + 1];

        int total;
        bool sparse = false;  // one rank window, no cell prefixes
        // a record with meta.y < 0 was not written (the row's count came from another
        // pass): the bitmap is rebuilt
        const int2 meta = rec ? rec_meta[gi] : make_int2(0, -1);
        if (meta.y >= 0) {
            // the symbolic pass stored this row's bitmap, word prefixes and cell prefixes
            // (dense), or only its non-zero words with their ranks (sparse)
            const int rec16 = int(L.winfirst / 16);
            const uint4* src = rec + gi * int64_t(rec16);  // records are slotted by global row
            if (meta.x >= 0) {
                sparse = true;
                const uint2* sp = reinterpret_cast<const uint2*>(src);
                for (int q = threadIdx.x; q < meta.x; q += NT) {
                    const uint2 e = sp[q];
                    const int w = int(e.y >> 18);
                    wb[w] = make_uint2(e.x, e.y & 0x3ffffu);
                    atomicOr(&summ[w >> 5], 1u << (w & 31));
                }
                if (threadIdx.x == 0) cellbase[0] = 0;
                total = meta.y;
                __syncthreads();
            } else {
                for (int q = threadIdx.x; q < rec16; q += NT) smem_raw[q] = src[q];
                __syncthreads();
                total = cellbase[ncell];
                __syncthreads();
            }
        } else {
        // 1) bitmap of the row's columns (all of a task's word reads before its
        //    atomics), then the summary bits by one ballot per 32 words
        for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
            const int ntasks = load_tasks<NT, AT, false>(g, nullptr, 0, p0, ahi, 0, 0, ts, nullptr);
            walk_tasks_bits<NT, RK_SUB, 2>(g, ts, ntasks, wbx);
            __syncthreads();
        }
        {
            const int lane = threadIdx.x & 31;
            for (int c = threadIdx.x >> 5; c < ncell; c += NT / 32) {
                const unsigned m = __ballot_sync(0xffffffffu, wbx[2 * (c * 32 + lane)] != 0u);
                if (lane == 0) summ[c] = m;
            }
            __syncthreads();
        }

        // 2) ranks: prefix inside each cell, cells' prefix, then absolute word ranks
        constexpr int CPT = (RK_MAX_COLS / RK_CELL + NT - 1) / NT;  // cells per thread (upper bound)
        int cnt[CPT];
        int ctot = 0;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = threadIdx.x * CPT + q;
            int n = 0;
            if (c < ncell) {
                uint32_t sw = summ[c];
                while (sw) {
                    const int w = c * 32 + __ffs(sw) - 1;
                    sw &= sw - 1;
                    wbx[2 * w + 1] = uint32_t(n);
                    n += __popc(wbx[2 * w]);
                }
            }
            cnt[q] = n;
            ctot += n;
        }
        int ex = block_exclusive_scan<NT, int>(ctot, s_warp, total);
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = threadIdx.x * CPT + q;
            if (c < ncell) {
                cellbase[c] = ex;
                uint32_t sw = summ[c];
                while (sw) {
                    const int w = c * 32 + __ffs(sw) - 1;
                    sw &= sw - 1;
                    wbx[2 * w + 1] += uint32_t(ex);
                }
            }
            ex += cnt[q];
        }
        }
        if (threadIdx.x == 0) {
            cellbase[ncell] = total;
            int64_t dst = o0;
            int ok = total <= o1 - o0;
            if (out.cap) {
                out.nnz[gi] = total;
                if (!ok && out.n_over) atomicAdd(out.n_over, 1);
                if (!ok && out.pool_used) {
                    const unsigned long long at = atomicAdd(out.pool_used, (unsigned long long)total);
                    if (int64_t(at) + total <= out.pool_cap) {
                        dst = out.pool_base + int64_t(at);
                        ok = 1;
                    }
                }
                if (!ok) out.ovf[atomicAdd(out.novf, 1)] = int32_t(gi);
                if (out.where) out.where[gi] = ok ? dst : -1;
                if (out.pred) err_sum += fabs(double(out.pred[gi]) - log2(1.0 + double(total)));
            } else if (total != int(o1 - o0)) {
                atomicOr(flags, STC_FLAG_INTERNAL);
            }
            s_dst = dst;
            s_fits = ok;
        }
        __syncthreads();
        const bool fits = s_fits != 0;
        const int64_t od = s_dst;  // where this row's entries go
        if (!sparse) {
            for (int c = threadIdx.x; c < ncell; c += NT) {
                const int wc = cellbase[c] / vstep;
                if (c == 0 || (cellbase[c - 1] / vstep) != wc) winfirst[wc] = c;
            }
        }
        if (threadIdx.x == 0) {
            const int nw = (total > 0 && fits) ? (sparse ? 1 : cellbase[ncell - 1] / vstep + 1) : 0;
            if (sparse) winfirst[0] = 0;
            winfirst[nw] = ncell;
            s_nwin = nw;
        }
        __syncthreads();
        const int nwin = s_nwin;

        // 3) values, one rank window at a time
        for (int wdw = 0; wdw < nwin; ++wdw) {
            const int cl = winfirst[wdw], ch = winfirst[wdw + 1];
            const int rb = cellbase[cl];
            const int rcount = cellbase[ch] - rb;
            const int32_t* tab = nwin > 1 ? g.ctab : nullptr;
            auto rank_of = [&](int col) -> int {
                const uint2 e = wb[col >> 5];
                if constexpr (MASKED)
                    if (!((e.x >> (col & 31)) & 1u)) return -1;  // not in the mask
                return int(e.y) + __popc(e.x & ((1u << (col & 31)) - 1u)) - rb;
            };
            bool done = false;
            if constexpr (ALG == ALG_PT_F32 && !MASKED) {
                if (wide) {
                    // compensated sums: comp (the column buffer) collects, per entry, the
                    // exact rounding error of every accumulating add (from the value the
                    // atomic add returns) and of every product (fma); the entry is the
                    // rounded acc + comp.  Columns come from the bitmap at write-out.
                    float* comp = reinterpret_cast<float*>(scol);
                    for (int r = threadIdx.x; r < rcount; r += NT) comp[r] = 0.0f;
                    __syncthreads();
                    for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
                        const int ntasks = load_tasks<NT, AT, true, VSUB>(g, tab, ncell, p0, ahi, cl, ch, ts, s_aval);
                        walk_tasks_rank<NT, AT, BT, VSUB>(
                            g, ts, ntasks, s_aval, bval, rcount, rank_of, [&](int, int) {},
                            [&](int r, int, const BT& bb, const AT aa) {
                                const float pr = __fmul_rn(aa, bb);
                                const float ep = __fmaf_rn(aa, bb, -pr);  // aa * bb - pr, exactly
                                const float old = atomicAdd(&vals[r], pr);
                                const float sm = __fadd_rn(old, pr);  // what the atomic stored
                                const float bv = __fsub_rn(sm, old);
                                const float e = __fadd_rn(__fsub_rn(old, __fsub_rn(sm, bv)), __fsub_rn(pr, bv));
                                atomicAdd(&comp[r], __fadd_rn(e, ep));
                            });
                        __syncthreads();
                    }
                    if (fits) {
                        // each non-zero word's columns, in order, from the rank of its first column
                        for (int w = cl * 32 + int(threadIdx.x); w < ch * 32; w += NT) {
                            uint32_t bits = wb[w].x;
                            if (!bits) continue;
                            int r = int(wb[w].y) - rb;
                            while (bits) {
                                c_col[od + rb + r++] = w * 32 + __ffs(bits) - 1 + g.col_base;
                                bits &= bits - 1;
                            }
                        }
                    }
                    for (int r = threadIdx.x; r < rcount; r += NT) {
                        if (fits) cval[od + rb + r] = __fadd_rn(vals[r], comp[r]);
                        vals[r] = T::empty();
                    }
                    done = true;
                }
            }
            if (!done) {
            for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
                const int ntasks = load_tasks<NT, AT, true, VSUB>(g, tab, ncell, p0, ahi, cl, ch, ts, s_aval);
                walk_tasks_rank<NT, AT, BT, VSUB>(g, ts, ntasks, s_aval, bval, rcount, rank_of,
                                            [&](int r, int col) { scol[r] = col; },
                                            [&](int r, int col, const BT& b, const AT a) {
                                                if constexpr (ALG == ALG_MULTPATH) atomicMin(&vals[r], a + b.d);
                                                else T::combine(vals, r, a, b);
                                            });
                __syncthreads();
            }
            if constexpr (ALG == ALG_MULTPATH) {
                for (int64_t p0 = alo; p0 < ahi; p0 += NT) {
                    const int ntasks = load_tasks<NT, AT, true, VSUB>(g, tab, ncell, p0, ahi, cl, ch, ts, s_aval);
                    walk_tasks_rank<NT, AT, BT, VSUB>(g, ts, ntasks, s_aval, bval, rcount, rank_of,
                                                [&](int, int) {},
                                                [&](int r, int, const BT& b, const AT a) {
                                                    if (a + b.d == vals[r]) atomicAdd(&sig[r], b.s);
                                                });
                    __syncthreads();
                }
            }
            for (int r = threadIdx.x; r < rcount; r += NT) {
                if (fits) {
                    if constexpr (!MASKED) c_col[od + rb + r] = scol[r] + g.col_base;
                    if constexpr (ALG == ALG_MULTPATH) {
                        DSig o;
                        o.d = (MASKED && vals[r] == T::empty()) ? STC_MIN_PLUS_I32_IDENTITY : vals[r];
                        o.pad = 0;
                        o.s = sig[r];
                        cval[od + rb + r] = o;
                        sig[r] = 0.0;
                    } else if constexpr (MASKED) {
                        cval[od + rb + r] = vals[r] == T::empty() ? T::identity() : T::out(vals[r]);
                    } else {
                        cval[od + rb + r] = T::out(vals[r]);
                    }
                }
                vals[r] = T::empty();
            }
            }
            __syncthreads();
        }

        // 4) clear the touched words
        for (int c = threadIdx.x; c < ncell; c += NT) {
            uint32_t s = summ[c];
            summ[c] = 0u;
            while (s) {
                const int w = c * 32 + __ffs(s) - 1;
                s &= s - 1;
                wbx[2 * w] = 0u;
            }
        }
    }
    if (threadIdx.x == 0 && err_sum != 0.0) atomicAdd(out.err, err_sum);
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
    size_t acc = alg == ALG_PT_F64 ? 8 : 4;
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

// Launch configuration of the rank kernels: narrow outputs (at most 16384
// columns, e.g. many small matrices) use small CTAs so that many rows are in
// flight per SM; wide outputs use one 1024-thread CTA per SM and a large value
// buffer (fewer rank windows per row).
struct RankCfg {
    bool small;
    int vcap, maxwin;
    size_t smem;
    int nt = 0;  // threads per CTA: 256 (small), 512 (light rows), 1024 (wide)
};

template <int ALG, int NT, int MINB, bool MASKED = false>
stc_status launch_numeric_rank(stc_handle* h, const SpgRows& R, int ncell_max, const RankCfg& cfg,
                               const int32_t* rowlist, const int* nlist, int* counter, const RankOut& out,
                               int32_t* c_col, void* c_val, int64_t NR, const uint4* rec, const int2* rec_meta, stc_stream s) {
    auto kern = k_numeric_rank<ALG, NT, MINB, MASKED>;
    STC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cfg.smem)));
    int per_sm = 0;
    STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, cfg.smem));
    if (per_sm < 1) return STC_ERR_CUDA;
    int64_t grid = int64_t(per_sm) * h->num_sms;
    if (grid > NR) grid = NR > 0 ? NR : 1;
    kern<<<unsigned(grid), NT, cfg.smem, s>>>(R, ncell_max, cfg.vcap, cfg.maxwin, rowlist, nlist, counter, out,
                                              c_col, c_val, h->d_flags, rec, rec_meta);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

template <int ALG>
stc_status run_numeric_rank(stc_handle* h, const SpgRows& R, int ncell_max, const RankCfg& cfg,
                            const int32_t* rowlist, const int* nlist, int* counter, const RankOut& out,
                            int32_t* c_col, void* c_val, int64_t NR, const uint4* rec, const int2* rec_meta, stc_stream s) {
    if (cfg.small)
        return launch_numeric_rank<ALG, 256, 4>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val,
                                                NR, rec, rec_meta, s);
    if (cfg.nt == 512)
        return launch_numeric_rank<ALG, 512, 2>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val,
                                                NR, rec, rec_meta, s);
    return launch_numeric_rank<ALG, RK_NT, 1>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val,
                                              NR, rec, rec_meta, s);
}

stc_status run_numeric_any(stc_handle* h, int alg, const SpgRows& R, int ncell_max, const RankCfg& cfg,
                           const int32_t* rowlist, const int* nlist, int* counter, const RankOut& out,
                           int32_t* c_col, void* c_val, int64_t NR, stc_stream s, const uint4* rec = nullptr,
                           const int2* rec_meta = nullptr) {
    switch (alg) {
    case ALG_PT_F32: return run_numeric_rank<ALG_PT_F32>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val, NR, rec, rec_meta, s);
    case ALG_PT_F64: return run_numeric_rank<ALG_PT_F64>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val, NR, rec, rec_meta, s);
    case ALG_MP_I32: return run_numeric_rank<ALG_MP_I32>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val, NR, rec, rec_meta, s);
    case ALG_MP_F32: return run_numeric_rank<ALG_MP_F32>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val, NR, rec, rec_meta, s);
    case ALG_BOOL: return run_numeric_rank<ALG_BOOL>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val, NR, rec, rec_meta, s);
    case ALG_MULTPATH: return run_numeric_rank<ALG_MULTPATH>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val, NR, rec, rec_meta, s);
    case ALG_PATH: return run_numeric_rank<ALG_PATH>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_col, c_val, NR, rec, rec_meta, s);
    default: return STC_ERR_ALGEBRA;
    }
}

template <int ALG>
stc_status run_numeric_masked_alg(stc_handle* h, const SpgRows& R, int ncell_max, const RankCfg& cfg,
                                  const int32_t* rowlist, const int* nlist, int* counter, const RankOut& out,
                                  void* c_val, int64_t NR, const uint4* rec, const int2* rec_meta, stc_stream s) {
    if (cfg.small)
        return launch_numeric_rank<ALG, 256, 4, true>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, nullptr,
                                                      c_val, NR, rec, rec_meta, s);
    return launch_numeric_rank<ALG, RK_NT, 1, true>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, nullptr,
                                                    c_val, NR, rec, rec_meta, s);
}

stc_status run_numeric_masked(stc_handle* h, int alg, const SpgRows& R, int ncell_max, const RankCfg& cfg,
                              const int32_t* rowlist, const int* nlist, int* counter, const RankOut& out,
                              void* c_val, int64_t NR, const uint4* rec, const int2* rec_meta, stc_stream s) {
    switch (alg) {
    case ALG_PT_F32: return run_numeric_masked_alg<ALG_PT_F32>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_val, NR, rec, rec_meta, s);
    case ALG_PT_F64: return run_numeric_masked_alg<ALG_PT_F64>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_val, NR, rec, rec_meta, s);
    case ALG_MP_I32: return run_numeric_masked_alg<ALG_MP_I32>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_val, NR, rec, rec_meta, s);
    case ALG_MP_F32: return run_numeric_masked_alg<ALG_MP_F32>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_val, NR, rec, rec_meta, s);
    case ALG_BOOL: return run_numeric_masked_alg<ALG_BOOL>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_val, NR, rec, rec_meta, s);
    case ALG_MULTPATH: return run_numeric_masked_alg<ALG_MULTPATH>(h, R, ncell_max, cfg, rowlist, nlist, counter, out, c_val, NR, rec, rec_meta, s);
    default: return STC_ERR_ALGEBRA;
    }
}

stc_status run_copy_any(stc_handle* h, int alg, const SpgRows& R, const int32_t* rowlist, const int* nlist,
                        const int* ncopy, const int64_t* c_ptr, int32_t* c_col, void* c_val, stc_stream s) {
    const unsigned grid = unsigned(h->num_sms * 8);
    switch (alg) {
    case ALG_PT_F32: k_copy_rows<ALG_PT_F32><<<grid, 256, 0, s>>>(R, rowlist, nlist, ncopy, c_ptr, c_col, c_val); break;
    case ALG_PT_F64: k_copy_rows<ALG_PT_F64><<<grid, 256, 0, s>>>(R, rowlist, nlist, ncopy, c_ptr, c_col, c_val); break;
    case ALG_MP_I32: k_copy_rows<ALG_MP_I32><<<grid, 256, 0, s>>>(R, rowlist, nlist, ncopy, c_ptr, c_col, c_val); break;
    case ALG_MP_F32: k_copy_rows<ALG_MP_F32><<<grid, 256, 0, s>>>(R, rowlist, nlist, ncopy, c_ptr, c_col, c_val); break;
    case ALG_BOOL: k_copy_rows<ALG_BOOL><<<grid, 256, 0, s>>>(R, rowlist, nlist, ncopy, c_ptr, c_col, c_val); break;
    case ALG_MULTPATH: k_copy_rows<ALG_MULTPATH><<<grid, 256, 0, s>>>(R, rowlist, nlist, ncopy, c_ptr, c_col, c_val); break;
    case ALG_PATH: k_copy_rows<ALG_PATH><<<grid, 256, 0, s>>>(R, rowlist, nlist, ncopy, c_ptr, c_col, c_val); break;
    default: return STC_ERR_ALGEBRA;
    }
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

// Algebras of the warp-per-row kernels (the others keep the CTA kernels).
bool wr_supported(int alg) {
    return alg == ALG_PT_F32 || alg == ALG_PT_F64 || alg == ALG_MP_I32 || alg == ALG_MP_F32 || alg == ALG_BOOL;
}

template <int ALG, int WARPS, int VCAP>
stc_status launch_wr_numeric(stc_handle* h, const SpgRows& R, const int32_t* row_mat, const int32_t* rowlist,
                             const int* nlist, int* counter, const int64_t* c_ptr, int32_t* c_col, void* c_val,
                             int64_t NR, const uint32_t* bm, stc_stream s) {
    auto kern = k_wr_numeric<ALG, WARPS, VCAP>;
    const size_t smem = WARPS * wr_warp_bytes<ALG, VCAP>();
    STC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    STC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      int(cudaSharedmemCarveoutMaxShared)));
    int per_sm = 0;
    STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem));
    if (per_sm < 1) return STC_ERR_CUDA;
    int64_t grid = int64_t(per_sm) * h->num_sms;
    if (grid * WARPS > NR) grid = (NR + WARPS - 1) / WARPS;
    kern<<<unsigned(grid > 0 ? grid : 1), WARPS * 32, smem, s>>>(R, row_mat, rowlist, nlist, counter, c_ptr, c_col,
                                                                c_val, h->d_flags, bm);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

// wide == false: the instance for rows of at most WR_VCAP_S entries (more warps
// per SM), else the one for rows of at most WR_VCAP.
template <int ALG>
stc_status launch_wr_numeric_any(stc_handle* h, bool wide, const SpgRows& R, const int32_t* row_mat,
                                 const int32_t* rowlist, const int* nlist, int* counter, const int64_t* c_ptr,
                                 int32_t* c_col, void* c_val, int64_t NR, const uint32_t* bm, stc_stream s) {
    if (wide)
        return launch_wr_numeric<ALG, WR_NUM_WARPS, WR_VCAP>(h, R, row_mat, rowlist, nlist, counter, c_ptr, c_col,
                                                             c_val, NR, bm, s);
    return launch_wr_numeric<ALG, WR_NUM_WARPS_S, WR_VCAP_S>(h, R, row_mat, rowlist, nlist, counter, c_ptr, c_col,
                                                             c_val, NR, bm, s);
}

stc_status run_wr_numeric(stc_handle* h, int alg, bool wide, const SpgRows& R, const int32_t* row_mat,
                          const int32_t* rowlist, const int* nlist, int* counter, const int64_t* c_ptr,
                          int32_t* c_col, void* c_val, int64_t NR, const uint32_t* bm, stc_stream s) {
    switch (alg) {
    case ALG_PT_F32: return launch_wr_numeric_any<ALG_PT_F32>(h, wide, R, row_mat, rowlist, nlist, counter, c_ptr, c_col, c_val, NR, bm, s);
    case ALG_PT_F64: return launch_wr_numeric_any<ALG_PT_F64>(h, wide, R, row_mat, rowlist, nlist, counter, c_ptr, c_col, c_val, NR, bm, s);
    case ALG_MP_I32: return launch_wr_numeric_any<ALG_MP_I32>(h, wide, R, row_mat, rowlist, nlist, counter, c_ptr, c_col, c_val, NR, bm, s);
    case ALG_MP_F32: return launch_wr_numeric_any<ALG_MP_F32>(h, wide, R, row_mat, rowlist, nlist, counter, c_ptr, c_col, c_val, NR, bm, s);
    case ALG_BOOL: return launch_wr_numeric_any<ALG_BOOL>(h, wide, R, row_mat, rowlist, nlist, counter, c_ptr, c_col, c_val, NR, bm, s);
    default: return STC_ERR_ALGEBRA;
    }
}

// light != 0: the configuration of the light-row launch (512 threads, two CTAs
// per SM sharing its shared memory, a value buffer of a few thousand ranks).
RankCfg rank_config(int alg, int64_t ncols_max, int ncell_max, bool light = false) {
    RankCfg c{};
    const size_t acc_bytes = (alg == ALG_PT_F64 || alg == ALG_PATH) ? 8 : 4;
    const bool mp = alg == ALG_MULTPATH;
    c.small = !light && ncols_max <= 16384;
    const int nt = light ? 512 : c.small ? 256 : RK_NT;
    c.nt = nt;
    // four / two / one CTA(s) per SM
    const size_t target = c.small ? 54 * 1024 : light ? 112 * 1024 : RK_SMEM_TARGET;
    const size_t static_bytes = size_t(nt) * 16 + size_t(nt) * 8 + 512 + sizeof(SpgArgs);
    for (int v = 64 * 1024; v >= 2048; v -= 1024) {
        const int mw = int(ncols_max / (v - RK_CELL)) + 2;
        RankLayout L = rank_layout(ncell_max, v, mw, acc_bytes, mp);
        if (L.total + static_bytes <= target) {
            c.vcap = v;
            c.maxwin = mw;
            c.smem = L.total;
            return c;
        }
    }
    return c;
}

// The rank path over nb matrices (nb == 1: a single SpGEMM).  Produces the
// global row pointers (NR + 1), columns and values; *bounds_h (host, nb + 1)
// receives the output offset of every matrix's first row.
stc_status spgemm_rank_impl(stc_handle* h, int alg, int nb, const SpgArgs* args_h, const int64_t* row_off_h,
                            bool validate, const stc_csr* Av, const stc_csr* Bv, int64_t** c_ptr_out,
                            int32_t** c_col_out, void** c_val_out, int64_t* nnz_out, int64_t* bounds_h,
                            int light_log2, stc_stream s) {
    *c_ptr_out = nullptr;
    *c_col_out = nullptr;
    *c_val_out = nullptr;
    *nnz_out = 0;
    const int64_t NR = row_off_h[nb];
    const size_t vbytes = stc_val_bytes(alg, 'C');
    int64_t ncols_max = 0;
    for (int b = 0; b < nb; ++b) ncols_max = args_h[b].ncols > ncols_max ? args_h[b].ncols : ncols_max;
    const int ncell_max = int((ncols_max + RK_CELL - 1) >> RK_CELL_SHIFT) > 0
                              ? int((ncols_max + RK_CELL - 1) >> RK_CELL_SHIFT) : 1;
    const RankCfg cfg = rank_config(alg, ncols_max, ncell_max);
    if (!cfg.vcap) return STC_ERR_INVALID_ARG;
    // narrow outputs: warp-per-row count and numeric passes (rows above the warp's
    // value slots go to the CTA kernel)
    const bool warp_path = ncols_max <= WR_MAX_COLS && wr_supported(alg);
    // light rows (ub < 2^light_log2) get their own launch of 512-thread CTAs, two per
    // SM, beside the wide launch; only when their whole row fits one rank window
    RankCfg lcfg{};
    int L = (!warp_path && light_log2 > 0 && light_log2 < NBINS) ? light_log2 : 0;
    if (L) {
        lcfg = rank_config(alg, ncols_max, ncell_max, true);
        if (!lcfg.vcap || (int64_t(1) << L) > int64_t(lcfg.vcap - RK_CELL)) L = 0;
    }

    int64_t* c_ptr = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(NR + 1) * 8, s));
    if (!c_ptr) return STC_ERR_OOM;
    int32_t* c_col = nullptr;
    void* c_val = nullptr;
    auto fail = [&](stc_status st) {
        stc_free_bytes(h, c_ptr, s);
        if (c_col) stc_free_bytes(h, c_col, s);
        if (c_val) stc_free_bytes(h, c_val, s);
        return st;
    };
    StcScratch sc(h, s);
    stc_mark(h, s, 0);
    if (cudaMemsetAsync(c_ptr, 0, size_t(NR + 1) * 8, s) != cudaSuccess) return fail(STC_ERR_CUDA);
    stc_status st;
    if (validate) {
        if ((st = stc_validate_many_async(h, sc, Av, nb, s)) != STC_OK) return fail(st);
        if ((st = stc_validate_many_async(h, sc, Bv, nb, s)) != STC_OK) return fail(st);
    }
    stc_mark(h, s, 1);

    SpgRows R{};
    R.nb = nb;
    SpgArgs* table_d = nullptr;
    // warp-per-row passes: every matrix's row bitmaps (ceil(ncols / 32) words a row),
    // written by the count pass and read by the numeric pass
    std::vector<SpgArgs> args_w;
    int64_t bm_words = 0;
    if (warp_path) {
        args_w.assign(args_h, args_h + nb);
        for (int b = 0; b < nb; ++b) {
            args_w[b].bm_off = bm_words;
            bm_words += args_w[b].nA * ((args_w[b].ncols + 31) / 32);
        }
        args_h = args_w.data();
    }
    if (nb == 1) {
        R.one = args_h[0];
    } else {
        table_d = sc.get<SpgArgs>(size_t(nb));
        int64_t* roff_d = sc.get<int64_t>(size_t(nb) + 1);
        if (sc.failed) return fail(STC_ERR_OOM);
        if (cudaMemcpyAsync(table_d, args_h, sizeof(SpgArgs) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(roff_d, row_off_h, sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(STC_ERR_CUDA);
        R.table = table_d;
        R.row_off = roff_d;
    }
    int64_t* ub = sc.get<int64_t>(size_t(NR));
    int32_t* rowlist = sc.get<int32_t>(size_t(NR));
    int* ints = sc.get<int>(2 * NBINS_ALL + 24);
    int64_t* bounds_d = sc.get<int64_t>(size_t(nb) + 1);
    int32_t* row_mat = (warp_path && nb > 1) ? sc.get<int32_t>(size_t(NR)) : nullptr;
    uint32_t* bm = warp_path ? sc.get<uint32_t>(size_t(bm_words) + 1) : nullptr;
    if (sc.failed) return fail(STC_ERR_OOM);
    if (cudaMemsetAsync(ints, 0, sizeof(int) * (2 * NBINS_ALL + 24), s) != cudaSuccess) return fail(STC_ERR_CUDA);
    int* bin_count = ints;
    int* cursor = ints + NBINS_ALL;
    int* nlist = ints + 2 * NBINS_ALL;
    int* counters = ints + 2 * NBINS_ALL + 1;  // [0] symbolic, [1] numeric
    int* max_nnz = ints + 2 * NBINS_ALL + 4;
    if (NR > 0) {
        launch_row_ub(h, R, NR, ub, bin_count, c_ptr + 1, row_mat, s);
        k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
        k_bin_scatter<<<unsigned((NR + 511) / 512), 512, 0, s>>>(NR, ub, c_ptr + 1, cursor, rowlist);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 3);
    }
    stc_mark(h, s, 2);
    // stored rank records (bitmap, word and cell prefixes per listed row) when they
    // fit the budget; otherwise the numeric pass rebuilds them
    const size_t rec_bytes = rank_layout(ncell_max, 0, 0, 4, false).winfirst;
    uint4* rec = nullptr;
    int2* rec_meta = nullptr;  // per record: (number of words of a sparse record or -1, row count)
    // (warp path: records only serve the heavy rows of the CTA kernels; kept when a
    // slot per row costs at most 1 GB)
    if (NR > 0 && double(NR) * double(rec_bytes) <= (warp_path ? 1e9 : RK_RECORD_BUDGET)) {
        rec = sc.get<uint4>(size_t(NR) * (rec_bytes / 16));
        rec_meta = sc.get<int2>(size_t(NR));
        if (!rec || !rec_meta) return fail(STC_ERR_OOM);
        // only the CTA symbolic pass writes records; rows counted by the warp pass
        // keep (-1, -1) and are rebuilt by the CTA numeric kernel if they go there
        if (warp_path && cudaMemsetAsync(rec_meta, 0xff, sizeof(int2) * size_t(NR), s) != cudaSuccess)
            return fail(STC_ERR_CUDA);
    }
    // ints past the bins: [0] nlist, [1..3] pass counters, [4] max row, [5..6] light split,
    // [8..10] numeric list sizes, [11..13] their counters, [14] count-pass counter,
    // [16..17] rows with >= 2^WR_UB_LOG2 products / the others
    int* wr_heavy = ints + 2 * NBINS_ALL + 16;
    if (NR > 0 && warp_path) {
        // heavy prefix of the row list on the CTA kernel, the rest one warp per row
        k_split_counts<<<1, 32, 0, s>>>(bin_count, WR_UB_LOG2, wr_heavy);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        {
            const size_t smem = sym_layout(ncell_max).total;
            auto kern = k_symbolic_rank<RK_SYM_NT, RK_SYM_MINB>;
            STC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            int per_sm = 0;
            STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RK_SYM_NT, smem));
            if (per_sm < 1) return fail(STC_ERR_CUDA);
            int64_t grid = int64_t(per_sm) * h->num_sms;
            if (grid > NR) grid = NR;
            kern<<<unsigned(grid), RK_SYM_NT, smem, s>>>(R, ncell_max, rowlist, wr_heavy, counters, c_ptr + 1,
                                                         max_nnz, rec, rec_meta, cfg.vcap - RK_CELL);
            if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
            stc_count(h);
        }
        auto kern = k_wr_count<WR_COUNT_WARPS>;
        int per_sm = 0;
        STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WR_COUNT_WARPS * 32, 0));
        if (per_sm < 1) return fail(STC_ERR_CUDA);
        int64_t grid = int64_t(per_sm) * h->num_sms;
        if (grid * WR_COUNT_WARPS > NR) grid = (NR + WR_COUNT_WARPS - 1) / WR_COUNT_WARPS;
        kern<<<unsigned(grid), WR_COUNT_WARPS * 32, 0, s>>>(R, row_mat, rowlist, wr_heavy, nlist,
                                                           ints + 2 * NBINS_ALL + 14, c_ptr + 1, max_nnz, bm);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    } else if (NR > 0) {
        const size_t smem = sym_layout(ncell_max).total;
        auto kern = k_symbolic_rank<RK_SYM_NT, RK_SYM_MINB>;
        STC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        int per_sm = 0;
        STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RK_SYM_NT, smem));
        if (per_sm < 1) return fail(STC_ERR_CUDA);
        int64_t grid = int64_t(per_sm) * h->num_sms;
        if (grid > NR) grid = NR;
        kern<<<unsigned(grid), RK_SYM_NT, smem, s>>>(R, ncell_max, rowlist, nlist, counters, c_ptr + 1, max_nnz, rec,
                                                     rec_meta, cfg.vcap - RK_CELL);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    stc_mark(h, s, 3);
    if ((st = stc_inclusive_scan_i64(h, sc, c_ptr + 1, NR, s)) != STC_OK) return fail(st);
    if (nb > 1) {
        k_batch_bounds<<<unsigned((nb + 256) / 256), 256, 0, s>>>(R, c_ptr, bounds_d);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    // the single synchronisation: nnz, the largest row, the validation flags (and batch bounds)
    int* stage_i = reinterpret_cast<int*>(&h->h_stage[1]);
    int* stage_bins = reinterpret_cast<int*>(&h->h_stage[8]);  // NBINS_ALL ints
    stage_i[0] = 0;
    stage_i[1] = 0;
    if (cudaMemcpyAsync(&h->h_stage[0], c_ptr + NR, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&stage_i[0], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&stage_i[1], max_nnz, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        ((L || warp_path) &&
         cudaMemcpyAsync(stage_bins, bin_count, sizeof(int) * NBINS_ALL, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        (nb > 1 && cudaMemcpyAsync(bounds_h, bounds_d, sizeof(int64_t) * (nb + 1), cudaMemcpyDeviceToHost, s) !=
                       cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(STC_ERR_CUDA);
    }
    int64_t n_heavy = 0, n_light = 0;
    if (L) {
        for (int b = 1; b < NBINS; ++b) (b > L ? n_heavy : n_light) += stage_bins[b];
        if (n_light == 0) L = 0;
    }
    const int64_t nnz = h->h_stage[0];
    const int flags = stage_i[0];
    const int max_row = stage_i[1];
    if (nb == 1) {
        bounds_h[0] = 0;
        bounds_h[1] = nnz;
    }
    if (flags) {
        (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
        return fail(stc_flags_to_status(flags));
    }
    if (nnz < 0) return fail(STC_ERR_CUDA);
    c_col = static_cast<int32_t*>(stc_alloc_bytes(h, size_t(nnz) * 4, s));
    c_val = stc_alloc_bytes(h, size_t(nnz) * vbytes, s);
    if (!c_col || !c_val) return fail(STC_ERR_OOM);

    // per-cell offset tables, only when some row needs several rank windows
    if (nnz > 0 && max_row >= cfg.vcap - RK_CELL) {
        std::vector<SpgArgs> args(args_h, args_h + nb);
        size_t tot = 0;
        std::vector<size_t> off(nb);
        int64_t kmax = 0;
        for (int b = 0; b < nb; ++b) {
            off[b] = tot;
            tot += size_t(args[b].K) * size_t(args[b].ncell + 1);
            kmax = args[b].K * (args[b].ncell + 1) > kmax ? args[b].K * (args[b].ncell + 1) : kmax;
        }
        int32_t* ctab = sc.get<int32_t>(tot);
        if (!ctab) return fail(STC_ERR_OOM);
        for (int b = 0; b < nb; ++b) args[b].ctab = ctab + off[b];
        if (nb == 1) {
            R.one = args[0];
        } else if (cudaMemcpyAsync(table_d, args.data(), sizeof(SpgArgs) * nb, cudaMemcpyHostToDevice, s) !=
                   cudaSuccess) {
            return fail(STC_ERR_CUDA);
        }
        int64_t bx = (kmax + 255) / 256;
        const int64_t cap = nb == 1 ? int64_t(h->num_sms) * 64 : 64;
        if (bx > cap) bx = cap;
        if (bx < 1) bx = 1;
        k_cell_offsets<<<dim3(unsigned(bx), unsigned(nb)), 256, 0, s>>>(R);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        if (nb > 1 && cudaStreamSynchronize(s) != cudaSuccess) return fail(STC_ERR_CUDA);  // args vector lifetime
    }
    stc_mark(h, s, 4);
    if (nnz > 0 && warp_path) {
        RankOut out{};
        out.ptr = c_ptr;
        int* nsplit = ints + 2 * NBINS_ALL + 8;   // [0..2] sizes of the three lists
        int* wcounter = ints + 2 * NBINS_ALL + 11;  // [0] narrow warp instance, [1] wide, [2] CTA kernel
        int64_t wr_heavy_rows = 0;
        for (int b = WR_UB_LOG2 + 1; b < NBINS; ++b) wr_heavy_rows += stage_bins[b];
        // (+,x) fp32: rows with compensated sums may exist, and only the CTA kernel has them
        const bool maybe_wide = wide_len_of(alg) != NO_WIDE_ROWS;
        if (max_row <= WR_VCAP_S && wr_heavy_rows == 0 && !maybe_wide) {
            if ((st = run_wr_numeric(h, alg, false, R, row_mat, rowlist, nlist, wcounter, c_ptr, c_col, c_val, NR,
                                     bm, s)) != STC_OK)
                return fail(st);
        } else {
            int32_t* lists = sc.get<int32_t>(3 * size_t(NR));
            if (!lists) return fail(STC_ERR_OOM);
            int64_t blocks = (NR + 255) / 256;
            if (blocks > int64_t(h->num_sms) * 8) blocks = int64_t(h->num_sms) * 8;
            k_split_by_count<<<unsigned(blocks), 256, 0, s>>>(R, row_mat, wide_len_of(alg), NR, ub, c_ptr, lists,
                                                              lists + NR, lists + 2 * NR, nsplit);
            if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
            stc_count(h);
            if (max_row > WR_VCAP || wr_heavy_rows > 0 || maybe_wide) {
                if ((st = run_numeric_any(h, alg, R, ncell_max, cfg, lists + 2 * NR, nsplit + 2, wcounter + 2, out,
                                          c_col, c_val, NR, s, rec, rec_meta)) != STC_OK)
                    return fail(st);
            }
            if (max_row > WR_VCAP_S &&
                (st = run_wr_numeric(h, alg, true, R, row_mat, lists + NR, nsplit + 1, wcounter + 1, c_ptr, c_col,
                                     c_val, NR, bm, s)) != STC_OK)
                return fail(st);
            if ((st = run_wr_numeric(h, alg, false, R, row_mat, lists, nsplit, wcounter, c_ptr, c_col, c_val, NR,
                                     bm, s)) != STC_OK)
                return fail(st);
        }
        if ((st = run_copy_any(h, alg, R, rowlist, nlist, bin_count + BIN_COPY, c_ptr, c_col, c_val, s)) != STC_OK)
            return fail(st);
    } else if (nnz > 0) {
        RankOut out{};
        out.ptr = c_ptr;
        if (L) {
            // heavy rows (the list's prefix) on this stream, light rows (its suffix)
            // on the auxiliary stream: their CTAs take the SMs the heavy launch frees
            int* split = ints + 2 * NBINS_ALL + 5;  // [0] heavy rows, [1] light rows
            k_split_counts<<<1, 32, 0, s>>>(bin_count, L, split);
            if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
            stc_count(h);
            if ((st = run_numeric_any(h, alg, R, ncell_max, cfg, rowlist, split, counters + 1, out, c_col, c_val,
                                      NR, s, rec, rec_meta)) != STC_OK)
                return fail(st);
            cudaStream_t aux;
            if ((st = stc_fork(h, s, &aux)) != STC_OK) return fail(st);
            st = run_numeric_any(h, alg, R, ncell_max, lcfg, rowlist + n_heavy, split + 1, counters + 2, out, c_col,
                                 c_val, NR, aux, rec, rec_meta);
            const stc_status sj = stc_join(h, s);
            if (st != STC_OK) return fail(st);
            if (sj != STC_OK) return fail(sj);
        } else if ((st = run_numeric_any(h, alg, R, ncell_max, cfg, rowlist, nlist, counters + 1, out, c_col,
                                         c_val, NR, s, rec, rec_meta)) != STC_OK) {
            return fail(st);
        }
        if ((st = run_copy_any(h, alg, R, rowlist, nlist, bin_count + BIN_COPY, c_ptr, c_col, c_val, s)) != STC_OK)
            return fail(st);
    }
    stc_mark(h, s, 5);
    if (nb > 1) {
        // per-matrix row pointers that start at zero
        int64_t* rp = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(NR + nb) * 8, s));
        if (!rp) return fail(STC_ERR_OOM);
        int64_t blocks = (NR + nb + 255) / 256;
        if (blocks > int64_t(h->num_sms) * 16) blocks = int64_t(h->num_sms) * 16;
        k_rebase_rowptr<<<unsigned(blocks), 256, 0, s>>>(R, c_ptr, rp);
        if (cudaGetLastError() != cudaSuccess) {
            stc_free_bytes(h, rp, s);
            return fail(STC_ERR_CUDA);
        }
        stc_count(h);
        stc_free_bytes(h, c_ptr, s);
        c_ptr = rp;
    }
    *c_ptr_out = c_ptr;
    *c_col_out = c_col;
    *c_val_out = c_val;
    *nnz_out = nnz;
    return STC_OK;
}

// Predicted capacity of every output row: min(ub, ncols) without a model (the
// upper-bound single pass), else (1 + margin) * (2^pred - 1) + 8, clipped to
// [1, min(ub, ncols)].  Also the scan input of the scratch offsets and the largest
// capacity.
// single (may be null): non-zero for rows written by the copy kernel (no scratch).
__global__ void k_capacity(int64_t NR, const int64_t* __restrict__ ub, const float* __restrict__ pred, float margin,
                           int64_t ncols, const int64_t* __restrict__ single, int64_t* __restrict__ cap,
                           int64_t* __restrict__ cap_scan, int* __restrict__ maxcap) {
    int m = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NR; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t u = ub[i];
        int64_t c = 0;
        if (u > 0 && !(single && single[i] > 0)) {
            const int64_t lim = u < ncols ? u : ncols;
            if (pred) {
                const float p = fmaxf(exp2f(pred[i]) - 1.0f, 0.0f);
                c = int64_t(ceilf((1.0f + margin) * p)) + 8;
                c = c < lim ? c : lim;
                c = c > 1 ? c : 1;
            } else {
                c = lim;
            }
        }
        cap[i] = c;
        cap_scan[i] = c;
        m = max(m, int(c < INT_MAX ? c : INT_MAX));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxcap, m);
}

// Copy every listed row that fit its capacity from the scratch to C (warp per row).
// The row's size is cnt[i] when cnt != null (c_ptr then holds destinations only),
// else c_ptr[i + 1] - c_ptr[i].
// where (may be null): the scratch offset each row was written at (slot or
// overflow pool), -1 for a row left to the exact recomputation.
template <class V>
__global__ void k_compact(const int32_t* __restrict__ rowlist, const int* __restrict__ nlist_ptr,
                          const int64_t* __restrict__ soff, const int64_t* __restrict__ cap,
                          const int64_t* __restrict__ where, const int64_t* __restrict__ c_ptr,
                          const int64_t* __restrict__ cnt, const int32_t* __restrict__ scol,
                          const V* __restrict__ sval, int32_t* __restrict__ c_col, V* __restrict__ c_val) {
    const int lane = threadIdx.x & 31;
    const int nlist = *nlist_ptr;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t r = warp; r < nlist; r += nwarps) {
        const int32_t i = rowlist[r];
        const int64_t d0 = c_ptr[i], n = cnt ? cnt[i] : c_ptr[i + 1] - d0;
        int64_t s0;
        if (where) {
            s0 = where[i];
            if (s0 < 0) continue;  // recomputed exactly
        } else {
            if (n > cap[i]) continue;
            s0 = soff[i];
        }
        for (int64_t e = lane; e < n; e += 32) {
            c_col[d0 + e] = scol[s0 + e];
            c_val[d0 + e] = sval[s0 + e];
        }
    }
}

stc_status run_compact(stc_handle* h, size_t vbytes, const int32_t* rowlist, const int* nlist, int n_rows,
                       const int64_t* soff, const int64_t* cap, const int64_t* where, const int64_t* dst,
                       const int64_t* cnt, const int32_t* scol, const void* sval, int32_t* c_col, void* c_val,
                       stc_stream s) {
    int64_t blocks = (int64_t(n_rows) * 32 + 255) / 256;
    if (blocks > int64_t(h->num_sms) * 16) blocks = int64_t(h->num_sms) * 16;
    if (blocks < 1) blocks = 1;
    const unsigned gb = unsigned(blocks);
    switch (vbytes) {
    case 1: k_compact<uint8_t><<<gb, 256, 0, s>>>(rowlist, nlist, soff, cap, where, dst, cnt, scol, static_cast<const uint8_t*>(sval), c_col, static_cast<uint8_t*>(c_val)); break;
    case 4: k_compact<uint32_t><<<gb, 256, 0, s>>>(rowlist, nlist, soff, cap, where, dst, cnt, scol, static_cast<const uint32_t*>(sval), c_col, static_cast<uint32_t*>(c_val)); break;
    case 8: k_compact<uint64_t><<<gb, 256, 0, s>>>(rowlist, nlist, soff, cap, where, dst, cnt, scol, static_cast<const uint64_t*>(sval), c_col, static_cast<uint64_t*>(c_val)); break;
    default: k_compact<uint4><<<gb, 256, 0, s>>>(rowlist, nlist, soff, cap, where, dst, cnt, scol, static_cast<const uint4*>(sval), c_col, static_cast<uint4*>(c_val)); break;
    }
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

SpgArgs make_args(const stc_csr* A, const stc_csr* B) {
    SpgArgs g{};
    g.nA = A->nrows;
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
    g.W = 0;
    g.nwin = 1;
    g.ctab = nullptr;
    g.ncell = int((B->ncols + RK_CELL - 1) >> RK_CELL_SHIFT);
    return g;
}


// ----------------------------------------------------------------- column slabs
//
// Outputs wider than RK_MAX_COLS: B is split once into slabs of RK_MAX_COLS
// columns (B_s = the entries of B with column in [s W, (s+1) W), columns shifted
// to start at 0), every slab runs the rank path's analysis and symbolic pass, one
// scan over the per-(row, slab) counts gives C's row pointers and every row's
// offset per slab, and every slab's numeric pass writes its part of each row in
// place (C_i is the concatenation of the slabs' parts, columns ascending).

constexpr int SLAB_MAX = 32;  // at most 32 slabs (8,388,608 columns) on this path

struct SlabBases {
    int64_t base[SLAB_MAX];   // first entry of slab s in the slab arrays
};

// Per B row k: bnd[k*(S+1) + t] = number of entries of B_k with column < t W.
// Warp per row; lane t-1 binary-searches boundary t.
__global__ void k_slab_bounds(const int64_t* __restrict__ b_ptr, const int32_t* __restrict__ b_col, int64_t K,
                              int64_t nnzB, int S, int32_t* __restrict__ bnd, int64_t* __restrict__ bsptr) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; k < K; k += nw) {
        int64_t lo, hi;
        row_range(b_ptr, k, nnzB, lo, hi);
        int32_t* bk = bnd + k * (S + 1);
        for (int t = lane; t <= S; t += 32) {
            int64_t pos;
            if (t == 0) {
                pos = lo;
            } else if (t == S) {
                pos = hi;
            } else {
                const int64_t target = int64_t(t) * RK_MAX_COLS;
                int64_t a = lo, b = hi;
                while (a < b) {
                    const int64_t m = (a + b) >> 1;
                    if (int64_t(b_col[m]) < target) a = m + 1; else b = m;
                }
                pos = a;
            }
            bk[t] = int32_t(pos - lo);
        }
        __syncwarp();
        for (int t = lane; t < S; t += 32) bsptr[int64_t(t) * (K + 1) + k + 1] = bk[t + 1] - bk[t];
    }
}

// Copy every B row's slab parts into the slab arrays (columns shifted to the slab).
template <class VT>
__global__ void k_slab_scatter(const int64_t* __restrict__ b_ptr, const int32_t* __restrict__ b_col,
                               const VT* __restrict__ b_val, int64_t K, int64_t nnzB, int S,
                               const int32_t* __restrict__ bnd, const int64_t* __restrict__ bsptr, SlabBases sb,
                               int32_t* __restrict__ s_col, VT* __restrict__ s_val) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; k < K; k += nw) {
        int64_t lo, hi;
        row_range(b_ptr, k, nnzB, lo, hi);
        const int32_t* bk = bnd + k * (S + 1);
        for (int t = 0; t < S; ++t) {
            const int64_t src = lo + bk[t], n = bk[t + 1] - bk[t];
            const int64_t dst = sb.base[t] + bsptr[int64_t(t) * (K + 1) + k];
            const int32_t shift = int32_t(int64_t(t) * RK_MAX_COLS);
            for (int64_t e = lane; e < n; e += 32) {
                s_col[dst + e] = b_col[src + e] - shift;
                if (s_val) s_val[dst + e] = b_val[src + e];
            }
        }
    }
}

// dst[i] += src[i].
__global__ void k_add_i64(int64_t n, const int64_t* __restrict__ src, int64_t* __restrict__ dst) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] += src[i];
}

// c_ptr[i + 1] = sum over slabs of cnt[s NR + i].
__global__ void k_slab_total(int64_t NR, int S, const int64_t* __restrict__ cnt, int64_t* __restrict__ c_ptr) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NR; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t t = 0;
        for (int q = 0; q < S; ++q) t += cnt[int64_t(q) * NR + i];
        c_ptr[i + 1] = t;
    }
}

// off[s NR + i] = c_ptr[i] + sum over slabs q < s of cnt[q NR + i].
__global__ void k_slab_offsets(int64_t NR, int S, const int64_t* __restrict__ cnt, const int64_t* __restrict__ c_ptr,
                               int64_t* __restrict__ off) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NR; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t o = c_ptr[i];
        for (int q = 0; q < S; ++q) {
            off[int64_t(q) * NR + i] = o;
            o += cnt[int64_t(q) * NR + i];
        }
    }
}

// The slabs of B: per slab the rank path's arguments (B_s, its width and column
// base), a CSR view of B_s and the launch configuration.  Reads the validation
// flags raised so far (one synchronisation).
struct Slabs {
    int S = 0;
    std::vector<SpgArgs> args;
    std::vector<stc_csr> view;
    std::vector<RankCfg> cfg;
    std::vector<int> ncell;
};

// values == false: only the structure of the slabs (B->val may be NULL).
stc_status build_slabs(stc_handle* h, StcScratch& sc, int alg, const stc_csr* A, const stc_csr* B, int S,
                       Slabs& out, stc_stream s, bool values = true) {
    const int64_t K = A->ncols;
    const size_t vbB = stc_val_bytes(alg, 'B');
    int32_t* bnd = sc.get<int32_t>(size_t(K) * size_t(S + 1) + 1);
    int64_t* bsptr = sc.get<int64_t>(size_t(S) * size_t(K + 1));
    int32_t* s_col = sc.get<int32_t>(size_t(B->nnz) + 1);
    unsigned char* s_val = values ? sc.get<unsigned char>((size_t(B->nnz) + 1) * vbB) : nullptr;
    if (sc.failed) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(bsptr, 0, sizeof(int64_t) * size_t(S) * size_t(K + 1), s));
    const unsigned gw = unsigned(h->num_sms * 16);
    stc_status st;
    if (K > 0) {
        k_slab_bounds<<<gw, 256, 0, s>>>(B->rowptr, B->col, K, B->nnz, S, bnd, bsptr);
        STC_LAUNCH_CHECK();
        stc_count(h);
        for (int t = 0; t < S; ++t)
            if ((st = stc_inclusive_scan_i64(h, sc, bsptr + size_t(t) * (K + 1) + 1, K, s)) != STC_OK) return st;
    }
    // slab sizes and the validation flags so far
    SlabBases sb{};
    int64_t* stage = h->h_stage;
    for (int t = 0; t < S; ++t) stage[t] = 0;
    for (int t = 0; t < S && K > 0; ++t)
        STC_CUDA_TRY(cudaMemcpyAsync(&stage[t], bsptr + size_t(t) * (K + 1) + K, sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, s));
    int* f = reinterpret_cast<int*>(&stage[SLAB_MAX]);
    *f = 0;
    STC_CUDA_TRY(cudaMemcpyAsync(f, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    if (*f) {
        const int flags = *f;
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(flags);
    }
    int64_t tot = 0;
    for (int t = 0; t < S; ++t) {
        sb.base[t] = tot;
        tot += stage[t];
    }
    if (tot != B->nnz) return STC_ERR_CUDA;
    if (K > 0 && B->nnz > 0) {
        switch (vbB) {
        case 1: k_slab_scatter<uint8_t><<<gw, 256, 0, s>>>(B->rowptr, B->col, static_cast<const uint8_t*>(B->val), K, B->nnz, S, bnd, bsptr, sb, s_col, reinterpret_cast<uint8_t*>(s_val)); break;
        case 4: k_slab_scatter<uint32_t><<<gw, 256, 0, s>>>(B->rowptr, B->col, static_cast<const uint32_t*>(B->val), K, B->nnz, S, bnd, bsptr, sb, s_col, reinterpret_cast<uint32_t*>(s_val)); break;
        case 8: k_slab_scatter<uint64_t><<<gw, 256, 0, s>>>(B->rowptr, B->col, static_cast<const uint64_t*>(B->val), K, B->nnz, S, bnd, bsptr, sb, s_col, reinterpret_cast<uint64_t*>(s_val)); break;
        default: k_slab_scatter<uint4><<<gw, 256, 0, s>>>(B->rowptr, B->col, static_cast<const uint4*>(B->val), K, B->nnz, S, bnd, bsptr, sb, s_col, reinterpret_cast<uint4*>(s_val)); break;
        }
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    out.S = S;
    out.args.resize(S);
    out.view.resize(S);
    out.cfg.resize(S);
    out.ncell.resize(S);
    for (int t = 0; t < S; ++t) {
        SpgArgs g = make_args(A, B);
        const int64_t w = B->ncols - int64_t(t) * RK_MAX_COLS;
        g.ncols = w < RK_MAX_COLS ? w : RK_MAX_COLS;
        g.ncell = int((g.ncols + RK_CELL - 1) >> RK_CELL_SHIFT);
        g.b_ptr = bsptr + size_t(t) * (K + 1);
        g.b_col = s_col + sb.base[t];
        g.b_val = s_val ? s_val + size_t(sb.base[t]) * vbB : nullptr;
        g.nnzB = (t + 1 < S ? sb.base[t + 1] : B->nnz) - sb.base[t];
        g.col_base = int(int64_t(t) * RK_MAX_COLS);
        out.args[t] = g;
        stc_csr v{};
        v.nrows = K;
        v.ncols = g.ncols;
        v.nnz = g.nnzB;
        v.rowptr = const_cast<int64_t*>(g.b_ptr);
        v.col = const_cast<int32_t*>(g.b_col);
        v.val = const_cast<void*>(g.b_val);
        out.view[t] = v;
        out.ncell[t] = g.ncell > 0 ? g.ncell : 1;
        out.cfg[t] = rank_config(alg, g.ncols, out.ncell[t]);
        if (!out.cfg[t].vcap) return STC_ERR_INVALID_ARG;
    }
    return STC_OK;
}

// Exact nnz(C_i) of every row of C = A B (the symbolic phase alone): row
// analysis, binning and the symbolic rank kernel without stored records, slab by
// slab (summed) for outputs wider than RK_MAX_COLS.  counts: device int64[nrows].
stc_status row_counts_impl(stc_handle* h, const stc_csr* A, const stc_csr* B, int64_t* counts, bool validate,
                           stc_stream s) {
    const int64_t NR = A->nrows;
    if (NR == 0) return STC_OK;
    STC_CUDA_TRY(cudaMemsetAsync(counts, 0, size_t(NR) * 8, s));
    StcScratch sc(h, s);
    stc_status st;
    if (validate) {
        if ((st = stc_validate_csr_async(h, A, s)) != STC_OK) return st;
        if ((st = stc_validate_csr_async(h, B, s)) != STC_OK) return st;
    }
    const int S = B->ncols > RK_MAX_COLS ? int((B->ncols + RK_MAX_COLS - 1) / RK_MAX_COLS) : 1;
    if (S > SLAB_MAX) return STC_ERR_SHAPE;
    std::vector<SpgArgs> args;
    if (S == 1) {
        args.push_back(make_args(A, B));
    } else {
        Slabs sl;
        if ((st = build_slabs(h, sc, ALG_BOOL, A, B, S, sl, s, false)) != STC_OK) return st;
        args = sl.args;
    }
    int64_t* ub = sc.get<int64_t>(size_t(NR));
    int32_t* rowlist = sc.get<int32_t>(size_t(NR));
    int64_t* part = S > 1 ? sc.get<int64_t>(size_t(NR)) : counts;
    int* ints = sc.get<int>(2 * NBINS_ALL + 8);
    if (sc.failed) return STC_ERR_OOM;
    int64_t blocks = (NR * 32 + 255) / 256;
    if (blocks > int64_t(h->num_sms) * 16) blocks = int64_t(h->num_sms) * 16;
    for (int t = 0; t < S; ++t) {
        SpgRows R{};
        R.one = args[t];
        R.nb = 1;
        const int ncell = args[t].ncell > 0 ? args[t].ncell : 1;
        STC_CUDA_TRY(cudaMemsetAsync(ints, 0, sizeof(int) * (2 * NBINS_ALL + 8), s));
        if (S > 1) STC_CUDA_TRY(cudaMemsetAsync(part, 0, size_t(NR) * 8, s));
        int* bin_count = ints;
        int* cursor = ints + NBINS_ALL;
        int* nlist = ints + 2 * NBINS_ALL;
        int* counter = ints + 2 * NBINS_ALL + 1;
        int* max_nnz = ints + 2 * NBINS_ALL + 4;
        launch_row_ub(h, R, NR, ub, bin_count, part, nullptr, s);
        k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
        k_bin_scatter<<<unsigned((NR + 511) / 512), 512, 0, s>>>(NR, ub, part, cursor, rowlist);
        STC_LAUNCH_CHECK();
        stc_count(h, 3);
        const size_t smem = sym_layout(ncell).total;
        auto kern = k_symbolic_rank<RK_SYM_NT, RK_SYM_MINB>;
        int per_sm = 0;
        STC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RK_SYM_NT, smem));
        if (per_sm < 1) return STC_ERR_CUDA;
        int64_t grid = int64_t(per_sm) * h->num_sms;
        if (grid > NR) grid = NR;
        kern<<<unsigned(grid), RK_SYM_NT, smem, s>>>(R, ncell, rowlist, nlist, counter, part, max_nnz, nullptr,
                                                     nullptr, 0);
        STC_LAUNCH_CHECK();
        stc_count(h);
        if (S > 1) {
            k_add_i64<<<unsigned(h->num_sms * 8), 256, 0, s>>>(NR, part, counts);
            STC_LAUNCH_CHECK();
            stc_count(h);
        }
    }
    return STC_OK;
}

stc_status spgemm_slab_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C, bool validate,
                            stc_stream s) {
    const int64_t NR = A->nrows, K = A->ncols;
    const int S = int((B->ncols + RK_MAX_COLS - 1) / RK_MAX_COLS);
    if (S < 2 || S > SLAB_MAX) return STC_ERR_INVALID_ARG;
    const size_t vbC = stc_val_bytes(alg, 'C');
    int64_t* c_ptr = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(NR + 1) * 8, s));
    if (!c_ptr) return STC_ERR_OOM;
    int32_t* c_col = nullptr;
    void* c_val = nullptr;
    auto fail = [&](stc_status st) {
        (void)cudaGetLastError();
        stc_free_bytes(h, c_ptr, s);
        if (c_col) stc_free_bytes(h, c_col, s);
        if (c_val) stc_free_bytes(h, c_val, s);
        return st;
    };
    StcScratch sc(h, s);
    stc_mark(h, s, 0);
    if (cudaMemsetAsync(c_ptr, 0, size_t(NR + 1) * 8, s) != cudaSuccess) return fail(STC_ERR_CUDA);
    stc_status st;
    if (validate) {
        if ((st = stc_validate_csr_async(h, A, s)) != STC_OK) return fail(st);
        if ((st = stc_validate_csr_async(h, B, s)) != STC_OK) return fail(st);
    }
    stc_mark(h, s, 1);

    // 1) slabs of B
    Slabs sl;
    if ((st = build_slabs(h, sc, alg, A, B, S, sl, s)) != STC_OK) return fail(st);
    int64_t* cnt = sc.get<int64_t>(size_t(S) * size_t(NR));
    int64_t* off = sc.get<int64_t>(size_t(S) * size_t(NR));
    int64_t* ub = sc.get<int64_t>(size_t(NR));
    int64_t* nnz_scratch = sc.get<int64_t>(size_t(NR));
    int32_t* ovf = sc.get<int32_t>(size_t(NR));
    int32_t* rowlists = sc.get<int32_t>(size_t(S) * size_t(NR));
    const int NI = 2 * NBINS_ALL + 8;
    int* ints = sc.get<int>(size_t(S) * NI + 8);
    if (sc.failed) return fail(STC_ERR_OOM);
    if (cudaMemsetAsync(cnt, 0, sizeof(int64_t) * size_t(S) * size_t(NR), s) != cudaSuccess ||
        cudaMemsetAsync(ints, 0, sizeof(int) * (size_t(S) * NI + 8), s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    int* novf = ints + size_t(S) * NI;
    const std::vector<SpgArgs>& args = sl.args;
    const std::vector<RankCfg>& cfgs = sl.cfg;
    const std::vector<int>& ncells = sl.ncell;
    size_t rec_total = 0;
    for (int t = 0; t < S; ++t) rec_total += size_t(NR) * rank_layout(ncells[t], 0, 0, 4, false).winfirst;
    stc_mark(h, s, 2);

    // 2) per slab: analysis, binning, symbolic counts (and stored rank records when
    //    all slabs' records fit the budget together)
    const bool use_rec = NR > 0 && double(rec_total) <= RK_RECORD_BUDGET;
    std::vector<uint4*> recs(S, nullptr);
    std::vector<int2*> metas(S, nullptr);
    for (int t = 0; t < S && NR > 0; ++t) {
        SpgRows R{};
        R.one = args[t];
        R.nb = 1;
        int* ti = ints + size_t(t) * NI;
        int* bin_count = ti;
        int* cursor = ti + NBINS_ALL;
        int* nlist = ti + 2 * NBINS_ALL;
        int* counters = ti + 2 * NBINS_ALL + 1;
        int* max_nnz = ti + 2 * NBINS_ALL + 4;
        int32_t* rowlist = rowlists + size_t(t) * NR;
        int64_t* cnt_t = cnt + size_t(t) * NR;
        launch_row_ub(h, R, NR, ub, bin_count, cnt_t, nullptr, s);
        k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
        k_bin_scatter<<<unsigned((NR + 511) / 512), 512, 0, s>>>(NR, ub, cnt_t, cursor, rowlist);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 3);
        if (use_rec) {
            const size_t rb = rank_layout(ncells[t], 0, 0, 4, false).winfirst;
            recs[t] = sc.get<uint4>(size_t(NR) * (rb / 16));
            metas[t] = sc.get<int2>(size_t(NR));
            if (!recs[t] || !metas[t]) return fail(STC_ERR_OOM);
        }
        const size_t smem = sym_layout(ncells[t]).total;
        auto kern = k_symbolic_rank<RK_SYM_NT, RK_SYM_MINB>;
        int per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RK_SYM_NT, smem) != cudaSuccess || per_sm < 1)
            return fail(STC_ERR_CUDA);
        int64_t grid = int64_t(per_sm) * h->num_sms;
        if (grid > NR) grid = NR;
        kern<<<unsigned(grid), RK_SYM_NT, smem, s>>>(R, ncells[t], rowlist, nlist, counters, cnt_t, max_nnz, recs[t],
                                                     metas[t], cfgs[t].vcap - RK_CELL);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    stc_mark(h, s, 3);

    // 3) row pointers and per-slab row offsets
    if (NR > 0) {
        const unsigned gb = unsigned(h->num_sms * 8);
        k_slab_total<<<gb, 256, 0, s>>>(NR, S, cnt, c_ptr);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        if ((st = stc_inclusive_scan_i64(h, sc, c_ptr + 1, NR, s)) != STC_OK) return fail(st);
        k_slab_offsets<<<gb, 256, 0, s>>>(NR, S, cnt, c_ptr, off);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 2);
    }
    int64_t nnz = 0;
    std::vector<int> max_row(S, 0);
    {
        int* mx = reinterpret_cast<int*>(&h->h_stage[SLAB_MAX + 2]);  // S ints
        int* f = reinterpret_cast<int*>(&h->h_stage[SLAB_MAX]);
        *f = 0;
        h->h_stage[SLAB_MAX + 1] = 0;
        for (int t = 0; t < S; ++t) mx[t] = 0;
        for (int t = 0; t < S && NR > 0; ++t)
            if (cudaMemcpyAsync(&mx[t], ints + size_t(t) * NI + 2 * NBINS_ALL + 4, sizeof(int), cudaMemcpyDeviceToHost,
                                s) != cudaSuccess)
                return fail(STC_ERR_CUDA);
        if (cudaMemcpyAsync(&h->h_stage[SLAB_MAX + 1], c_ptr + NR, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(f, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(STC_ERR_CUDA);
        if (*f) {
            const int flags = *f;
            (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
            return fail(stc_flags_to_status(flags));
        }
        nnz = h->h_stage[SLAB_MAX + 1];
        for (int t = 0; t < S; ++t) max_row[t] = mx[t];
    }
    if (nnz < 0) return fail(STC_ERR_CUDA);
    c_col = static_cast<int32_t*>(stc_alloc_bytes(h, size_t(nnz) * 4, s));
    c_val = stc_alloc_bytes(h, size_t(nnz) * vbC, s);
    if ((!c_col || !c_val) && nnz > 0) return fail(STC_ERR_OOM);
    stc_mark(h, s, 4);

    // 4) per slab: numeric pass into C at the slab's row offsets
    for (int t = 0; t < S && nnz > 0; ++t) {
        StcScratch sct(h, s);  // the slab's cell-offset table, released after its pass
        SpgRows R{};
        R.one = args[t];
        R.nb = 1;
        if (max_row[t] >= cfgs[t].vcap - RK_CELL) {
            int32_t* ctab = sct.get<int32_t>(size_t(K) * size_t(ncells[t] + 1));
            if (!ctab) return fail(STC_ERR_OOM);
            R.one.ctab = ctab;
            int64_t bx = (K * (ncells[t] + 1) + 255) / 256;
            if (bx > int64_t(h->num_sms) * 64) bx = int64_t(h->num_sms) * 64;
            if (bx < 1) bx = 1;
            k_cell_offsets<<<dim3(unsigned(bx), 1), 256, 0, s>>>(R);
            if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
            stc_count(h);
        }
        int* ti = ints + size_t(t) * NI;
        int64_t* cnt_t = cnt + size_t(t) * NR;
        int64_t* off_t = off + size_t(t) * NR;
        int32_t* rowlist = rowlists + size_t(t) * NR;
        RankOut out{};
        out.ptr = off_t;
        out.cap = cnt_t;        // exact sizes: no row overflows
        out.nnz = nnz_scratch;  // receives the same sizes
        out.ovf = ovf;
        out.novf = novf;
        if ((st = run_numeric_any(h, alg, R, ncells[t], cfgs[t], rowlist, ti + 2 * NBINS_ALL, ti + 2 * NBINS_ALL + 2,
                                  out, c_col, c_val, NR, s, recs[t], metas[t])) != STC_OK)
            return fail(st);
        if ((st = run_copy_any(h, alg, R, rowlist, ti + 2 * NBINS_ALL, ti + BIN_COPY, off_t, c_col, c_val, s)) !=
            STC_OK)
            return fail(st);
    }
    stc_mark(h, s, 5);
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->rowptr = c_ptr;
    C->col = c_col;
    C->val = c_val;
    C->nnz = nnz;
    return STC_OK;
}

// Learned single-pass SpGEMM (one matrix, at most RK_MAX_COLS output columns):
// row analysis, features and perceptron (or the upper bound) give every row a
// capacity; one numeric pass writes each row into scratch of that capacity and
// records its exact size; a scan gives C's row pointers; the rows that fit are
// compacted into C and the rows that overflowed are recomputed exactly into C.
stc_status spgemm_learned_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                               const float* weights, float margin, stc_learned_stats* stats, bool validate,
                               stc_stream s) {
    SpgArgs g = make_args(A, B);
    const int64_t NR = A->nrows;
    const int ncell_max = g.ncell > 0 ? g.ncell : 1;
    const RankCfg cfg = rank_config(alg, B->ncols, ncell_max);
    if (!cfg.vcap) return STC_ERR_INVALID_ARG;
    const size_t vbytes = stc_val_bytes(alg, 'C');
    int64_t* c_ptr = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(NR + 1) * 8, s));
    if (!c_ptr) return STC_ERR_OOM;
    int32_t* c_col = nullptr;
    void* c_val = nullptr;
    auto fail = [&](stc_status st) {
        stc_free_bytes(h, c_ptr, s);
        if (c_col) stc_free_bytes(h, c_col, s);
        if (c_val) stc_free_bytes(h, c_val, s);
        return st;
    };
    StcScratch sc(h, s);
    stc_mark(h, s, 0);
    if (cudaMemsetAsync(c_ptr, 0, size_t(NR + 1) * 8, s) != cudaSuccess) return fail(STC_ERR_CUDA);
    stc_status st;
    if (validate) {
        if ((st = stc_validate_csr_async(h, A, s)) != STC_OK) return fail(st);
        if ((st = stc_validate_csr_async(h, B, s)) != STC_OK) return fail(st);
    }
    stc_mark(h, s, 1);
    SpgRows R{};
    R.one = g;
    R.nb = 1;
    int64_t* ub = sc.get<int64_t>(size_t(NR));
    int32_t* rowlist = sc.get<int32_t>(size_t(NR));
    int32_t* ovf = sc.get<int32_t>(size_t(NR));
    int64_t* cap = sc.get<int64_t>(size_t(NR));
    int64_t* soff = sc.get<int64_t>(size_t(NR) + 1);
    int* ints = sc.get<int>(2 * NBINS_ALL + 16);
    double* err = sc.get<double>(1);
    float* pred = weights ? sc.get<float>(size_t(NR)) : nullptr;
    float* feat = weights ? sc.get<float>(size_t(NR) * STC_MLP_FEAT_STRIDE) : nullptr;
    if (sc.failed) return fail(STC_ERR_OOM);
    int* bin_count = ints;
    int* cursor = ints + NBINS_ALL;
    int* nlist = ints + 2 * NBINS_ALL;
    int* counters = ints + 2 * NBINS_ALL + 1;  // [0] learned pass, [1] overflow pass
    int* maxcap = ints + 2 * NBINS_ALL + 4;
    int* novf = ints + 2 * NBINS_ALL + 5;
    if (cudaMemsetAsync(ints, 0, sizeof(int) * (2 * NBINS_ALL + 16), s) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(double), s) != cudaSuccess ||
        cudaMemsetAsync(soff, 0, sizeof(int64_t), s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    if (NR > 0) {
        // rows with one stored entry: exact size ub into c_ptr + 1, written by the copy kernel
        launch_row_ub(h, R, NR, ub, bin_count, c_ptr + 1, nullptr, s);
        k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
        k_bin_scatter<<<unsigned((NR + 511) / 512), 512, 0, s>>>(NR, ub, c_ptr + 1, cursor, rowlist);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 3);
        if (weights) {
            if ((st = stc_features_impl(h, sc, A, B, feat, s)) != STC_OK) return fail(st);
            if ((st = stc_mlp_forward_tc_impl(h, weights, feat, NR, pred, s)) != STC_OK) return fail(st);
        }
        int64_t cb = (NR + 255) / 256;
        if (cb > int64_t(h->num_sms) * 8) cb = int64_t(h->num_sms) * 8;
        k_capacity<<<unsigned(cb), 256, 0, s>>>(NR, ub, pred, margin, B->ncols, c_ptr + 1, cap, soff + 1, maxcap);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        if ((st = stc_inclusive_scan_i64(h, sc, soff + 1, NR, s)) != STC_OK) return fail(st);
    }
    stc_mark(h, s, 2);
    // synchronisation 1: scratch size, largest capacity, validation flags
    int* stage_i = reinterpret_cast<int*>(&h->h_stage[1]);
    stage_i[0] = stage_i[1] = 0;
    if (cudaMemcpyAsync(&h->h_stage[0], soff + NR, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&stage_i[0], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&stage_i[1], maxcap, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(STC_ERR_CUDA);
    }
    const int64_t S_total = h->h_stage[0];
    if (stage_i[0]) {
        const int f = stage_i[0];
        (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
        return fail(stc_flags_to_status(f));
    }
    const int max_cap = stage_i[1];
    // the slots, then an overflow pool of a quarter of them for rows the model
    // under-sized (only rows that miss the pool too are recomputed)
    const int64_t pool = S_total / 4 + 4096;
    int32_t* scol = sc.get<int32_t>(size_t(S_total + pool));
    unsigned char* sval = sc.get<unsigned char>(size_t(S_total + pool) * vbytes);
    int64_t* where = sc.get<int64_t>(size_t(NR) + 1);
    unsigned long long* pool_used = sc.get<unsigned long long>(1);
    if (sc.failed) return fail(STC_ERR_OOM);
    if (cudaMemsetAsync(pool_used, 0, sizeof(unsigned long long), s) != cudaSuccess) return fail(STC_ERR_CUDA);
    if (NR > 0 && max_cap >= cfg.vcap - RK_CELL) {
        int32_t* ctab = sc.get<int32_t>(size_t(g.K) * size_t(g.ncell + 1));
        if (!ctab) return fail(STC_ERR_OOM);
        R.one.ctab = ctab;
        int64_t bx = (g.K * (g.ncell + 1) + 255) / 256;
        if (bx > int64_t(h->num_sms) * 64) bx = int64_t(h->num_sms) * 64;
        k_cell_offsets<<<dim3(unsigned(bx > 0 ? bx : 1), 1), 256, 0, s>>>(R);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    stc_mark(h, s, 3);
    if (NR > 0) {
        RankOut out{};
        out.ptr = soff;
        out.cap = cap;
        out.nnz = c_ptr + 1;
        out.ovf = ovf;
        out.novf = novf;
        out.pred = pred;
        out.err = err;
        out.pool_used = pool_used;
        out.pool_base = S_total;
        out.pool_cap = pool;
        out.where = where;
        out.n_over = novf + 1;
        if ((st = run_numeric_any(h, alg, R, ncell_max, cfg, rowlist, nlist, counters, out, scol, sval, NR, s)) !=
            STC_OK)
            return fail(st);
        if ((st = stc_inclusive_scan_i64(h, sc, c_ptr + 1, NR, s)) != STC_OK) return fail(st);
    }
    // synchronisation 2: nnz, overflowing rows, listed rows, prediction error
    int* st2 = reinterpret_cast<int*>(&h->h_stage[8]);   // [0] recomputed, [1] listed rows
    int* st_over = reinterpret_cast<int*>(&h->h_stage[10]);  // rows above their capacity
    st2[0] = st2[1] = 0;
    *st_over = 0;
    double* err_h = reinterpret_cast<double*>(&h->h_stage[9]);
    *err_h = 0.0;
    if (cudaMemcpyAsync(&h->h_stage[0], c_ptr + NR, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&st2[0], novf, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&st2[1], nlist, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(st_over, novf + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(err_h, err, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(STC_ERR_CUDA);
    }
    const int64_t nnz = h->h_stage[0];
    const int n_ovf = st2[0], n_rows = st2[1], n_over = *st_over;
    const double err_sum = *err_h;
    c_col = static_cast<int32_t*>(stc_alloc_bytes(h, size_t(nnz) * 4, s));
    c_val = stc_alloc_bytes(h, size_t(nnz) * vbytes, s);
    if (!c_col || !c_val) return fail(STC_ERR_OOM);
    stc_mark(h, s, 4);
    if (NR > 0 && nnz > 0) {
        if ((st = run_compact(h, vbytes, rowlist, nlist, n_rows, soff, cap, where, c_ptr, nullptr, scol, sval, c_col, c_val,
                              s)) != STC_OK)
            return fail(st);
        if ((st = run_copy_any(h, alg, R, rowlist, nlist, bin_count + BIN_COPY, c_ptr, c_col, c_val, s)) != STC_OK)
            return fail(st);
        if (n_ovf > 0) {
            RankOut out{};
            out.ptr = c_ptr;
            if ((st = run_numeric_any(h, alg, R, ncell_max, cfg, ovf, novf, counters + 1, out, c_col, c_val, NR, s)) !=
                STC_OK)
                return fail(st);
        }
    }
    stc_mark(h, s, 5);
    if (stats) {
        stats->rows = n_rows;
        stats->overflow_rows = n_over;
        stats->recomputed_rows = n_ovf;
        stats->scratch_entries = S_total;
        stats->nnz = nnz;
        stats->mean_abs_log2_error = (weights && n_rows > 0) ? err_sum / n_rows : -1.0;
    }
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->rowptr = c_ptr;
    C->col = c_col;
    C->val = c_val;
    C->nnz = nnz;
    return STC_OK;
}

// Learned single pass over column slabs: every slab B_s is its own learned
// product A B_s (features of A and B_s, model, capacities, one numeric pass into
// the slab's scratch that records each row's exact size and its overflows);
// then one scan over the per-(row, slab) sizes places every slab's part of every
// row in C, the rows that fit are compacted there and the overflowing
// (row, slab) parts are recomputed exactly in place.
stc_status spgemm_learned_slab_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                                    const float* weights, float margin, stc_learned_stats* stats, bool validate,
                                    stc_stream s) {
    const int64_t NR = A->nrows, K = A->ncols;
    const int S = int((B->ncols + RK_MAX_COLS - 1) / RK_MAX_COLS);
    if (S < 2 || S > SLAB_MAX) return STC_ERR_INVALID_ARG;
    const size_t vbytes = stc_val_bytes(alg, 'C');
    int64_t* c_ptr = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(NR + 1) * 8, s));
    if (!c_ptr) return STC_ERR_OOM;
    int32_t* c_col = nullptr;
    void* c_val = nullptr;
    auto fail = [&](stc_status st) {
        (void)cudaGetLastError();
        stc_free_bytes(h, c_ptr, s);
        if (c_col) stc_free_bytes(h, c_col, s);
        if (c_val) stc_free_bytes(h, c_val, s);
        return st;
    };
    StcScratch sc(h, s);
    stc_mark(h, s, 0);
    if (cudaMemsetAsync(c_ptr, 0, size_t(NR + 1) * 8, s) != cudaSuccess) return fail(STC_ERR_CUDA);
    stc_status st;
    if (validate) {
        if ((st = stc_validate_csr_async(h, A, s)) != STC_OK) return fail(st);
        if ((st = stc_validate_csr_async(h, B, s)) != STC_OK) return fail(st);
    }
    stc_mark(h, s, 1);
    Slabs sl;
    if ((st = build_slabs(h, sc, alg, A, B, S, sl, s)) != STC_OK) return fail(st);
    const int NI = 2 * NBINS_ALL + 16;
    int64_t* ub = sc.get<int64_t>(size_t(NR));
    int64_t* cnt = sc.get<int64_t>(size_t(S) * size_t(NR));
    int64_t* off = sc.get<int64_t>(size_t(S) * size_t(NR));
    int64_t* cap = sc.get<int64_t>(size_t(S) * size_t(NR));
    int64_t* soff = sc.get<int64_t>(size_t(S) * size_t(NR + 1));
    int32_t* rowlists = sc.get<int32_t>(size_t(S) * size_t(NR));
    int32_t* ovfs = sc.get<int32_t>(size_t(S) * size_t(NR));
    int64_t* nnz_scratch = sc.get<int64_t>(size_t(NR));
    int32_t* ovf_scratch = sc.get<int32_t>(size_t(NR));
    int* ints = sc.get<int>(size_t(S) * NI + 8);
    double* err = sc.get<double>(1);
    float* feat = weights ? sc.get<float>(size_t(NR) * STC_MLP_FEAT_STRIDE) : nullptr;
    if (sc.failed) return fail(STC_ERR_OOM);
    if (cudaMemsetAsync(cnt, 0, sizeof(int64_t) * size_t(S) * size_t(NR), s) != cudaSuccess ||
        cudaMemsetAsync(soff, 0, sizeof(int64_t) * size_t(S) * size_t(NR + 1), s) != cudaSuccess ||
        cudaMemsetAsync(ints, 0, sizeof(int) * (size_t(S) * NI + 8), s) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(double), s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    int* dummy_novf = ints + size_t(S) * NI;
    std::vector<int32_t*> s_cols(S, nullptr);
    std::vector<unsigned char*> s_vals(S, nullptr);
    int64_t scratch_total = 0;
    stc_mark(h, s, 2);

    // 1) per slab: analysis, features and model, capacities and scratch offsets
    float* preds = weights ? sc.get<float>(size_t(S) * size_t(NR)) : nullptr;
    if (weights && !preds) return fail(STC_ERR_OOM);
    for (int t = 0; t < S && NR > 0; ++t) {
        SpgRows R{};
        R.one = sl.args[t];
        R.nb = 1;
        int* ti = ints + size_t(t) * NI;
        int* bin_count = ti;
        int* cursor = ti + NBINS_ALL;
        int* nlist = ti + 2 * NBINS_ALL;
        int* maxcap = ti + 2 * NBINS_ALL + 4;
        int32_t* rowlist = rowlists + size_t(t) * NR;
        int64_t* cap_t = cap + size_t(t) * NR;
        int64_t* soff_t = soff + size_t(t) * (NR + 1);
        float* pred_t = weights ? preds + size_t(t) * NR : nullptr;
        launch_row_ub(h, R, NR, ub, bin_count, nullptr, nullptr, s);
        k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
        k_bin_scatter<<<unsigned((NR + 511) / 512), 512, 0, s>>>(NR, ub, nullptr, cursor, rowlist);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 3);
        if (weights) {
            if ((st = stc_features_impl(h, sc, A, &sl.view[t], feat, s)) != STC_OK) return fail(st);
            if ((st = stc_mlp_forward_tc_impl(h, weights, feat, NR, pred_t, s)) != STC_OK) return fail(st);
        }
        int64_t cb = (NR + 255) / 256;
        if (cb > int64_t(h->num_sms) * 8) cb = int64_t(h->num_sms) * 8;
        k_capacity<<<unsigned(cb), 256, 0, s>>>(NR, ub, pred_t, margin, sl.args[t].ncols, nullptr, cap_t, soff_t + 1,
                                                 maxcap);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        if ((st = stc_inclusive_scan_i64(h, sc, soff_t + 1, NR, s)) != STC_OK) return fail(st);
    }
    // one synchronisation: every slab's scratch size and largest capacity
    std::vector<int64_t> S_t(S, 0);
    std::vector<int> max_cap(S, 0);
    if (NR > 0) {
        int* mc = reinterpret_cast<int*>(&h->h_stage[SLAB_MAX]);  // S ints
        for (int t = 0; t < S; ++t) {
            h->h_stage[t] = 0;
            mc[t] = 0;
            if (cudaMemcpyAsync(&h->h_stage[t], soff + size_t(t) * (NR + 1) + NR, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaMemcpyAsync(&mc[t], ints + size_t(t) * NI + 2 * NBINS_ALL + 4, sizeof(int), cudaMemcpyDeviceToHost,
                                s) != cudaSuccess)
                return fail(STC_ERR_CUDA);
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(STC_ERR_CUDA);
        for (int t = 0; t < S; ++t) {
            S_t[t] = h->h_stage[t];
            max_cap[t] = mc[t];
        }
    }
    // per slab: the slots, then an overflow pool of a quarter of them
    std::vector<int64_t> pool_t(S, 0);
    int64_t* wheres = sc.get<int64_t>(size_t(S) * size_t(NR) + 1);
    unsigned long long* pool_used = sc.get<unsigned long long>(size_t(S));
    if (!wheres || !pool_used) return fail(STC_ERR_OOM);
    if (cudaMemsetAsync(pool_used, 0, sizeof(unsigned long long) * size_t(S), s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    for (int t = 0; t < S && NR > 0; ++t) {
        scratch_total += S_t[t];
        pool_t[t] = S_t[t] / 4 + 4096;
        s_cols[t] = sc.get<int32_t>(size_t(S_t[t] + pool_t[t]));
        s_vals[t] = sc.get<unsigned char>(size_t(S_t[t] + pool_t[t]) * vbytes);
        if (!s_cols[t] || !s_vals[t]) return fail(STC_ERR_OOM);
    }
    stc_mark(h, s, 3);

    // one numeric pass per slab into its scratch (exact sizes and overflows recorded)
    for (int t = 0; t < S && NR > 0; ++t) {
        SpgRows R{};
        R.one = sl.args[t];
        R.nb = 1;
        int* ti = ints + size_t(t) * NI;
        int* nlist = ti + 2 * NBINS_ALL;
        int* counters = ti + 2 * NBINS_ALL + 1;
        int* novf = ti + 2 * NBINS_ALL + 5;
        int32_t* rowlist = rowlists + size_t(t) * NR;
        StcScratch sct(h, s);  // the slab's cell-offset table
        if (max_cap[t] >= sl.cfg[t].vcap - RK_CELL) {
            int32_t* ctab = sct.get<int32_t>(size_t(K) * size_t(sl.ncell[t] + 1));
            if (!ctab) return fail(STC_ERR_OOM);
            R.one.ctab = ctab;
            int64_t bx = (K * (sl.ncell[t] + 1) + 255) / 256;
            if (bx > int64_t(h->num_sms) * 64) bx = int64_t(h->num_sms) * 64;
            k_cell_offsets<<<dim3(unsigned(bx > 0 ? bx : 1), 1), 256, 0, s>>>(R);
            if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
            stc_count(h);
        }
        RankOut out{};
        out.ptr = soff + size_t(t) * (NR + 1);
        out.cap = cap + size_t(t) * NR;
        out.nnz = cnt + size_t(t) * NR;
        out.ovf = ovfs + size_t(t) * NR;
        out.novf = novf;
        out.pred = weights ? preds + size_t(t) * NR : nullptr;
        out.err = err;
        out.pool_used = pool_used + t;
        out.pool_base = S_t[t];
        out.pool_cap = pool_t[t];
        out.where = wheres + size_t(t) * NR;
        out.n_over = ti + 2 * NBINS_ALL + 6;
        if ((st = run_numeric_any(h, alg, R, sl.ncell[t], sl.cfg[t], rowlist, nlist, counters, out, s_cols[t],
                                  s_vals[t], NR, s)) != STC_OK)
            return fail(st);
    }
    stc_mark(h, s, 4);

    // 2) row pointers and per-slab offsets
    if (NR > 0) {
        const unsigned gb = unsigned(h->num_sms * 8);
        k_slab_total<<<gb, 256, 0, s>>>(NR, S, cnt, c_ptr);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        if ((st = stc_inclusive_scan_i64(h, sc, c_ptr + 1, NR, s)) != STC_OK) return fail(st);
        k_slab_offsets<<<gb, 256, 0, s>>>(NR, S, cnt, c_ptr, off);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 2);
    }
    int64_t nnz = 0;
    std::vector<int> n_ovf(S, 0), n_rows(S, 0), n_over(S, 0);
    double err_sum = 0.0;
    {
        int* v = reinterpret_cast<int*>(&h->h_stage[2]);  // 2 S ints: h_stage[2 .. 2 + S)
        int* vo = reinterpret_cast<int*>(&h->h_stage[SLAB_MAX + 12]);  // S ints
        for (int t = 0; t < 2 * S; ++t) v[t] = 0;
        for (int t = 0; t < S; ++t) vo[t] = 0;
        h->h_stage[SLAB_MAX + 8] = 0;
        double* e = reinterpret_cast<double*>(&h->h_stage[SLAB_MAX + 9]);
        *e = 0.0;
        for (int t = 0; t < S && NR > 0; ++t) {
            const int* ti = ints + size_t(t) * NI;
            if (cudaMemcpyAsync(&v[2 * t], ti + 2 * NBINS_ALL + 5, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaMemcpyAsync(&v[2 * t + 1], ti + 2 * NBINS_ALL, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaMemcpyAsync(&vo[t], ti + 2 * NBINS_ALL + 6, sizeof(int), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess)
                return fail(STC_ERR_CUDA);
        }
        if (cudaMemcpyAsync(&h->h_stage[SLAB_MAX + 8], c_ptr + NR, sizeof(int64_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(e, err, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(STC_ERR_CUDA);
        nnz = h->h_stage[SLAB_MAX + 8];
        err_sum = *e;
        for (int t = 0; t < S; ++t) {
            n_ovf[t] = v[2 * t];
            n_rows[t] = v[2 * t + 1];
            n_over[t] = vo[t];
        }
    }
    if (nnz < 0) return fail(STC_ERR_CUDA);
    c_col = static_cast<int32_t*>(stc_alloc_bytes(h, size_t(nnz) * 4, s));
    c_val = stc_alloc_bytes(h, size_t(nnz) * vbytes, s);
    if ((!c_col || !c_val) && nnz > 0) return fail(STC_ERR_OOM);
    stc_mark(h, s, 5);

    // 3) per slab: compaction of the rows that fit, exact recomputation of the others
    int units = 0, overflows = 0, recomputed = 0;
    for (int t = 0; t < S && NR > 0 && nnz > 0; ++t) {
        const int* ti = ints + size_t(t) * NI;
        int64_t* cnt_t = cnt + size_t(t) * NR;
        int64_t* off_t = off + size_t(t) * NR;
        if ((st = run_compact(h, vbytes, rowlists + size_t(t) * NR, ti + 2 * NBINS_ALL, n_rows[t],
                              soff + size_t(t) * (NR + 1), cap + size_t(t) * NR, wheres + size_t(t) * NR, off_t,
                              cnt_t, s_cols[t], s_vals[t], c_col, c_val, s)) != STC_OK)
            return fail(st);
        if (n_ovf[t] > 0) {
            SpgRows R{};
            R.one = sl.args[t];
            R.nb = 1;
            RankOut out{};
            out.ptr = off_t;
            out.cap = cnt_t;  // exact sizes
            out.nnz = nnz_scratch;
            out.ovf = ovf_scratch;
            out.novf = dummy_novf;
            if ((st = run_numeric_any(h, alg, R, sl.ncell[t], sl.cfg[t], ovfs + size_t(t) * NR,
                                      ti + 2 * NBINS_ALL + 5, const_cast<int*>(ti) + 2 * NBINS_ALL + 2, out, c_col,
                                      c_val, NR, s)) != STC_OK)
                return fail(st);
        }
        units += n_rows[t];
        overflows += n_over[t];
        recomputed += n_ovf[t];
    }
    stc_mark(h, s, 6);
    if (stats) {
        stats->rows = units;
        stats->overflow_rows = overflows;
        stats->recomputed_rows = recomputed;
        stats->scratch_entries = scratch_total;
        stats->nnz = nnz;
        stats->mean_abs_log2_error = (weights && units > 0) ? err_sum / units : -1.0;
    }
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->rowptr = c_ptr;
    C->col = c_col;
    C->val = c_val;
    C->nnz = nnz;
    return STC_OK;
}
// ----------------------------------------------------------------- masked product
//
// C<M> = A (x) B with the structure of M given: rows whose mask row is empty are
// not computed; the others are listed heaviest first by their product count.  The
// symbolic kernel run on (I, M) -- the identity pattern times the mask -- writes
// every listed row's rank record from the mask row itself; the numeric kernel in
// masked form then accumulates the products that land in the mask.

// ubm[i] = 0 for an empty mask row, else max(ub[i], 1) (listed even without
// products: its entries get the identity); bins counted by ubm.
__global__ void k_mask_ub(int64_t NR, const int64_t* __restrict__ ub, const int64_t* __restrict__ m_ptr,
                          int64_t nnzM, int64_t* __restrict__ ubm, int* __restrict__ bin_count) {
    __shared__ int s_bins[NBINS];
    for (int t = threadIdx.x; t < NBINS; t += blockDim.x) s_bins[t] = 0;
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < NR; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t lo, hi;
        row_range(m_ptr, i, nnzM, lo, hi);
        const int64_t u = hi > lo ? (ub[i] > 0 ? ub[i] : 1) : 0;
        ubm[i] = u;
        atomicAdd(&s_bins[bin_of(u)], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NBINS; t += blockDim.x)
        if (s_bins[t]) atomicAdd(&bin_count[t], s_bins[t]);
}

// The identity pattern: ptr[i] = i, col[i] = i.
__global__ void k_iota(int64_t n, int64_t* __restrict__ ptr, int32_t* __restrict__ col) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += int64_t(gridDim.x) * blockDim.x) {
        ptr[i] = i;
        if (i < n) col[i] = int32_t(i);
    }
}

stc_status spgemm_masked_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, const stc_csr* M,
                              void* c_val, bool validate, stc_stream s) {
    const int64_t NR = A->nrows;
    if (B->ncols > RK_MAX_COLS) return STC_ERR_INVALID_ARG;
    SpgArgs g = make_args(A, B);
    const int ncell_max = g.ncell > 0 ? g.ncell : 1;
    const RankCfg cfg = rank_config(alg, B->ncols, ncell_max);
    if (!cfg.vcap) return STC_ERR_INVALID_ARG;
    const size_t rec_bytes = rank_layout(ncell_max, 0, 0, 4, false).winfirst;
    if (double(NR) * double(rec_bytes) > RK_RECORD_BUDGET) return STC_ERR_INVALID_ARG;
    StcScratch sc(h, s);
    stc_mark(h, s, 0);
    stc_status st;
    if (validate) {
        if ((st = stc_validate_csr_async(h, A, s)) != STC_OK) return st;
        if ((st = stc_validate_csr_async(h, B, s)) != STC_OK) return st;
        if ((st = stc_validate_csr_async(h, M, s)) != STC_OK) return st;
    }
    stc_mark(h, s, 1);
    if (NR == 0 || M->nnz == 0) return STC_OK;
    int64_t* ub = sc.get<int64_t>(size_t(NR));
    int64_t* ubm = sc.get<int64_t>(size_t(NR));
    int64_t* cnt = sc.get<int64_t>(size_t(NR));
    int32_t* rowlist = sc.get<int32_t>(size_t(NR));
    int64_t* iota_ptr = sc.get<int64_t>(size_t(NR) + 1);
    int32_t* iota_col = sc.get<int32_t>(size_t(NR));
    int* ints = sc.get<int>(3 * NBINS_ALL + 8);
    uint4* rec = sc.get<uint4>(size_t(NR) * (rec_bytes / 16));
    int2* rec_meta = sc.get<int2>(size_t(NR));
    if (sc.failed) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(ints, 0, sizeof(int) * (3 * NBINS_ALL + 8), s));
    int* bin_count = ints;
    int* cursor = ints + NBINS_ALL;
    int* nlist = ints + 2 * NBINS_ALL;
    int* counters = ints + 2 * NBINS_ALL + 1;  // [0] symbolic, [1] numeric
    int* max_nnz = ints + 2 * NBINS_ALL + 4;
    int* product_bins = ints + 2 * NBINS_ALL + 8;  // unused counts of k_row_ub_b
    SpgRows R{};
    R.one = g;
    R.nb = 1;
    const unsigned gb = unsigned(h->num_sms * 8);
    launch_row_ub(h, R, NR, ub, product_bins, nullptr, nullptr, s);
    k_mask_ub<<<gb, 256, 0, s>>>(NR, ub, M->rowptr, M->nnz, ubm, bin_count);
    k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
    k_bin_scatter<<<unsigned((NR + 511) / 512), 512, 0, s>>>(NR, ubm, nullptr, cursor, rowlist);
    k_iota<<<gb, 256, 0, s>>>(NR, iota_ptr, iota_col);
    STC_LAUNCH_CHECK();
    stc_count(h, 5);
    stc_mark(h, s, 2);
    // rank records of the mask rows: the symbolic pass over I (x) M
    SpgArgs gm = make_args(A, B);
    gm.K = NR;
    gm.nnzA = NR;
    gm.a_ptr = iota_ptr;
    gm.a_col = iota_col;
    gm.a_val = nullptr;
    gm.nnzB = M->nnz;
    gm.b_ptr = M->rowptr;
    gm.b_col = M->col;
    gm.b_val = nullptr;
    SpgRows RM{};
    RM.one = gm;
    RM.nb = 1;
    {
        const size_t smem = sym_layout(ncell_max).total;
        auto kern = k_symbolic_rank<RK_SYM_NT, RK_SYM_MINB>;
        STC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        int per_sm = 0;
        STC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RK_SYM_NT, smem));
        if (per_sm < 1) return STC_ERR_CUDA;
        int64_t grid = int64_t(per_sm) * h->num_sms;
        if (grid > NR) grid = NR;
        kern<<<unsigned(grid), RK_SYM_NT, smem, s>>>(RM, ncell_max, rowlist, nlist, counters, cnt, max_nnz, rec,
                                                     rec_meta, cfg.vcap - RK_CELL);
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    stc_mark(h, s, 3);
    // the one synchronisation: validation flags and the longest mask row
    int* stage = reinterpret_cast<int*>(&h->h_stage[0]);
    stage[0] = stage[1] = 0;
    STC_CUDA_TRY(cudaMemcpyAsync(&stage[0], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaMemcpyAsync(&stage[1], max_nnz, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    if (stage[0]) {
        const int f = stage[0];
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(f);
    }
    if (stage[1] >= cfg.vcap - RK_CELL) {
        int32_t* ctab = sc.get<int32_t>(size_t(g.K) * size_t(g.ncell + 1));
        if (!ctab) return STC_ERR_OOM;
        R.one.ctab = ctab;
        int64_t bx = (g.K * (g.ncell + 1) + 255) / 256;
        if (bx > int64_t(h->num_sms) * 64) bx = int64_t(h->num_sms) * 64;
        k_cell_offsets<<<dim3(unsigned(bx > 0 ? bx : 1), 1), 256, 0, s>>>(R);
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    stc_mark(h, s, 4);
    RankOut out{};
    out.ptr = M->rowptr;
    if ((st = run_numeric_masked(h, alg, R, ncell_max, cfg, rowlist, nlist, counters + 1, out, c_val, NR, rec,
                                 rec_meta, s)) != STC_OK)
        return st;
    stc_mark(h, s, 5);
    return STC_OK;
}

// Light-row threshold of a call: the option when set, else the handle's tuned
// value for this algebra and output width, else no light launch.
int resolve_light(stc_handle* h, int alg, int64_t ncols_max, const stc_opts* opts) {
    int L = opts ? opts->light_rows : 0;
    if (L == 0) {
        const int c = stc_log2_ceil(ncols_max > 0 ? ncols_max : 1);
        const signed char t = (alg >= 0 && alg < 6 && c < 40) ? h->tune_light[alg][c] : -128;
        L = t == -128 ? -1 : t;
    }
    return L > 0 ? L : 0;
}

int64_t ncols_max_of(const std::vector<SpgArgs>& args) {
    int64_t m = 0;
    for (const SpgArgs& g : args) m = g.ncols > m ? g.ncols : m;
    return m;
}
}  // namespace

stc_status stc_spgemm_batched_impl(stc_handle* h, int alg, int nb, const stc_csr* A, const stc_csr* B,
                                   stc_csr* C, const stc_opts* opts, stc_stream s) {
    std::vector<SpgArgs> args(nb);
    std::vector<int64_t> row_off(size_t(nb) + 1, 0);
    for (int b = 0; b < nb; ++b) {
        args[b] = make_args(&A[b], &B[b]);
        row_off[b + 1] = row_off[b] + A[b].nrows;
        C[b].nrows = A[b].nrows;
        C[b].ncols = B[b].ncols;
        C[b].nnz = 0;
        C[b].rowptr = nullptr;
        C[b].col = nullptr;
        C[b].val = nullptr;
    }
    std::vector<int64_t> bounds(size_t(nb) + 1, 0);
    int64_t* c_ptr = nullptr;
    int32_t* c_col = nullptr;
    void* c_val = nullptr;
    int64_t nnz = 0;
    stc_status st = spgemm_rank_impl(h, alg, nb, args.data(), row_off.data(), !(opts && opts->skip_validation),
                                     A, B, &c_ptr, &c_col, &c_val, &nnz, bounds.data(),
                                     resolve_light(h, alg, ncols_max_of(args), opts), s);
    if (st != STC_OK) return st;
    const size_t vbytes = stc_val_bytes(alg, 'C');
    for (int b = 0; b < nb; ++b) {
        C[b].rowptr = c_ptr + row_off[b] + b;
        C[b].col = c_col + bounds[b];
        C[b].val = static_cast<char*>(c_val) + size_t(bounds[b]) * vbytes;
        C[b].nnz = bounds[b + 1] - bounds[b];
    }
    return STC_OK;
}

// Column-window path: any output width (the dense window accumulator of W
// columns is walked once per window, with the per-window offset table of B rows).
static stc_status spgemm_window_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                                     const stc_opts* opts, stc_stream s) {
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
    stc_status st;
    if (!(opts && opts->skip_validation)) {
        if ((st = stc_validate_csr_async(h, A, s)) != STC_OK) return fail(st);
        if ((st = stc_validate_csr_async(h, B, s)) != STC_OK) return fail(st);
    }
    stc_mark(h, s, 1);
    SpgArgs g = make_args(A, B);
    const bool trivial = nA == 0 || A->nnz == 0 || B->nnz == 0 || B->ncols == 0;
    const int64_t ncp = pow2_ceil(B->ncols > 0 ? B->ncols : 1);
    int64_t W = numeric_window_max(alg);
    if (opts && opts->window_cols) W = opts->window_cols;
    if (ncp < W) W = ncp < 32 ? 32 : ncp;
    g.W = int(W);
    g.nwin = int((B->ncols + W - 1) / W);
    if (g.nwin < 1) g.nwin = 1;
    if (numeric_smem_bytes(alg, g.W) > size_t(h->smem_optin) - 24 * 1024) return fail(STC_ERR_INVALID_ARG);
    StcScratch sc(h, s);
    int32_t* rowlist = nullptr;
    int* ints = nullptr;
    if (!trivial) {
        int64_t Ws = ncp < SYM_MAX_COLS ? ncp : SYM_MAX_COLS;
        if (Ws < W) Ws = W;
        const int R = int(Ws / W);
        int64_t* ub = sc.get<int64_t>(size_t(nA));
        rowlist = sc.get<int32_t>(size_t(nA));
        ints = sc.get<int>(2 * NBINS_ALL + 8);
        if (sc.failed) return fail(STC_ERR_OOM);
        if (cudaMemsetAsync(ints, 0, sizeof(int) * (2 * NBINS_ALL + 8), s) != cudaSuccess) return fail(STC_ERR_CUDA);
        int* bin_count = ints;
        int* cursor = ints + NBINS_ALL;
        int* nlist = ints + 2 * NBINS_ALL;
        int* counters = ints + 2 * NBINS_ALL + 1;
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
        int64_t blocks = (nA * 32 + 255) / 256;
        if (blocks > int64_t(h->num_sms) * 16) blocks = int64_t(h->num_sms) * 16;
        k_row_ub<<<unsigned(blocks), 256, 0, s>>>(g, ub, bin_count);
        k_bin_offsets<<<1, 32, 0, s>>>(bin_count, cursor, nlist);
        k_bin_scatter<<<unsigned((nA + 511) / 512), 512, 0, s>>>(nA, ub, nullptr, cursor, rowlist);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 3);
        stc_mark(h, s, 2);
        size_t smem = size_t(Ws / 32) * 4;
        int grid = 0;
        auto kern = k_symbolic<SP_NT>;
        if ((st = launch_persistent(h, kern, smem, grid)) != STC_OK) return fail(st);
        if (int64_t(grid) > nA) grid = int(nA);
        kern<<<grid, SP_NT, smem, s>>>(g, R, rowlist, nlist, counters, c_ptr + 1);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        stc_mark(h, s, 3);
        if ((st = stc_inclusive_scan_i64(h, sc, c_ptr + 1, nA, s)) != STC_OK) return fail(st);
    } else {
        stc_mark(h, s, 2);
        stc_mark(h, s, 3);
    }
    int* stage_i = reinterpret_cast<int*>(&h->h_stage[1]);
    stage_i[0] = 0;
    if (cudaMemcpyAsync(&h->h_stage[0], c_ptr + nA, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&stage_i[0], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(STC_ERR_CUDA);
    }
    const int64_t nnz = h->h_stage[0];
    const int flags = stage_i[0];
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
        int* nlist = ints + 2 * NBINS_ALL;
        int* counter = ints + 2 * NBINS_ALL + 2;
        switch (alg) {
        case ALG_PT_F32: st = run_numeric<ALG_PT_F32>(h, g, rowlist, nlist, counter, c_ptr, c_col, c_val, nA, s); break;
        case ALG_PT_F64: st = run_numeric<ALG_PT_F64>(h, g, rowlist, nlist, counter, c_ptr, c_col, c_val, nA, s); break;
        case ALG_MP_I32: st = run_numeric<ALG_MP_I32>(h, g, rowlist, nlist, counter, c_ptr, c_col, c_val, nA, s); break;
        case ALG_MP_F32: st = run_numeric<ALG_MP_F32>(h, g, rowlist, nlist, counter, c_ptr, c_col, c_val, nA, s); break;
        case ALG_BOOL: st = run_numeric<ALG_BOOL>(h, g, rowlist, nlist, counter, c_ptr, c_col, c_val, nA, s); break;
        case ALG_MULTPATH: st = run_numeric<ALG_MULTPATH>(h, g, rowlist, nlist, counter, c_ptr, c_col, c_val, nA, s); break;
        default: st = STC_ERR_ALGEBRA;
        }
        if (st != STC_OK) return fail(st);
    }
    stc_mark(h, s, 5);
    C->rowptr = c_ptr;
    C->col = c_col;
    C->val = c_val;
    C->nnz = nnz;
    return STC_OK;
}

stc_status stc_spgemm_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                           const stc_opts* opts, stc_stream s) {
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->nnz = 0;
    C->rowptr = nullptr;
    C->col = nullptr;
    C->val = nullptr;
    // rank-indexed kernels whenever the row bitmap fits shared memory, unless a
    // column window width is forced (the window kernels then serve any width)
    if (B->ncols <= RK_MAX_COLS && !(opts && opts->window_cols)) {
        SpgArgs g = make_args(A, B);
        const int64_t row_off[2] = {0, A->nrows};
        int64_t bounds[2];
        int64_t* c_ptr = nullptr;
        int32_t* c_col = nullptr;
        void* c_val = nullptr;
        int64_t nnz = 0;
        stc_status st = spgemm_rank_impl(h, alg, 1, &g, row_off, !(opts && opts->skip_validation), A, B, &c_ptr,
                                         &c_col, &c_val, &nnz, bounds,
                                         resolve_light(h, alg, B->ncols, opts), s);
        if (st != STC_OK) return st;
        C->rowptr = c_ptr;
        C->col = c_col;
        C->val = c_val;
        C->nnz = nnz;
        return STC_OK;
    }
    if (!(opts && opts->window_cols) && (B->ncols + RK_MAX_COLS - 1) / RK_MAX_COLS <= SLAB_MAX)
        return spgemm_slab_impl(h, alg, A, B, C, !(opts && opts->skip_validation), s);
    return spgemm_window_impl(h, alg, A, B, C, opts, s);
}

// Time every candidate light-row threshold on this product; cache the fastest.
stc_status stc_autotune_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, int32_t* best_out,
                             int32_t* cand_out, float* ms_out, int32_t* ncand_out, stc_stream s) {
    if (B->ncols > RK_MAX_COLS) return STC_ERR_INVALID_ARG;
    const int ncell = B->ncols > 0 ? int((B->ncols + RK_CELL - 1) >> RK_CELL_SHIFT) : 1;
    const RankCfg lc = rank_config(alg, B->ncols, ncell, true);
    int lmax = 0;
    for (int L = 1; L < 30; ++L)
        if (lc.vcap && (int64_t(1) << L) <= int64_t(lc.vcap - RK_CELL)) lmax = L;
    std::vector<int> cands{-1};
    for (int L = lmax - 6 > 6 ? lmax - 6 : 6; L <= lmax; ++L) cands.push_back(L);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    STC_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return STC_ERR_CUDA;
    }
    stc_status st = STC_OK;
    int best = -1;
    float best_ms = 0.0f;
    std::vector<float> times;
    for (int cand : cands) {
        stc_opts o{};
        o.light_rows = cand;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && st == STC_OK; ++rep) {
            stc_csr C{};
            if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) st = STC_ERR_CUDA;
            if (st == STC_OK) st = stc_spgemm_impl(h, alg, A, B, &C, &o, s);
            if (st == STC_OK && rep == 1 && cudaEventRecord(e1, s) != cudaSuccess) st = STC_ERR_CUDA;
            stc_free_bytes(h, C.rowptr, s);
            stc_free_bytes(h, C.col, s);
            stc_free_bytes(h, C.val, s);
            if (st == STC_OK && rep == 1 &&
                (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                st = STC_ERR_CUDA;
        }
        if (st != STC_OK) break;
        times.push_back(ms);
        if (times.size() == 1 || ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != STC_OK) return st;
    const int c = stc_log2_ceil(B->ncols > 0 ? B->ncols : 1);
    if (c < 40) h->tune_light[alg][c] = static_cast<signed char>(best);
    if (best_out) *best_out = best;
    if (ncand_out) *ncand_out = int32_t(times.size());
    for (size_t i = 0; i < times.size() && i < 8; ++i) {
        if (cand_out) cand_out[i] = cands[i];
        if (ms_out) ms_out[i] = times[i];
    }
    return STC_OK;
}

stc_status stc_spgemm_masked_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, const stc_csr* M,
                                  void* c_val, const stc_opts* opts, stc_stream s) {
    return spgemm_masked_impl(h, alg, A, B, M, c_val, !(opts && opts->skip_validation), s);
}

stc_status stc_spgemm_learned_impl(stc_handle* h, int alg, const stc_csr* A, const stc_csr* B, stc_csr* C,
                                   const float* weights, float margin, stc_learned_stats* stats,
                                   const stc_opts* opts, stc_stream s) {
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->nnz = 0;
    C->rowptr = nullptr;
    C->col = nullptr;
    C->val = nullptr;
    if (B->ncols > RK_MAX_COLS && (B->ncols + RK_MAX_COLS - 1) / RK_MAX_COLS <= SLAB_MAX)
        return spgemm_learned_slab_impl(h, alg, A, B, C, weights, margin, stats, !(opts && opts->skip_validation), s);
    if (B->ncols > RK_MAX_COLS) {
        // beyond the slab path: the exact two-pass path (no capacity to predict)
        if (stats) {
            stats->rows = -1;
            stats->overflow_rows = 0;
            stats->recomputed_rows = 0;
            stats->scratch_entries = 0;
            stats->mean_abs_log2_error = -1.0;
        }
        stc_status st = stc_spgemm_impl(h, alg, A, B, C, opts, s);
        if (stats) stats->nnz = C->nnz;
        return st;
    }
    return spgemm_learned_impl(h, alg, A, B, C, weights, margin, stats, !(opts && opts->skip_validation), s);
}

stc_status stc_row_counts_impl(stc_handle* h, const stc_csr* A, const stc_csr* B, int64_t* counts,
                               const stc_opts* opts, stc_stream s) {
    return row_counts_impl(h, A, B, counts, !(opts && opts->skip_validation), s);
}

// ----------------------------------------------------------------- calibration
//
// The rate at which the numeric rank kernel's accumulator can absorb products:
// one CTA of 1024 threads per SM combines `iters` x 8 products per thread into a
// shared-memory array of 8192 accumulators at pseudo-random positions (a linear
// congruential sequence per thread), with the algebra's (+) exactly as the numeric
// kernel applies it (fp64 (+,x): compare-and-swap of an fma).
namespace {

constexpr int CAL_SLOTS = 8192;

template <int ALG>
__global__ void __launch_bounds__(1024, 1) k_calibrate_acc(int iters, unsigned long long* sink) {
    using T = Tr<ALG>;
    using Acc = typename T::Acc;
    __shared__ Acc acc[CAL_SLOTS];
    for (int i = threadIdx.x; i < CAL_SLOTS; i += blockDim.x) acc[i] = T::empty();
    __syncthreads();
    unsigned s = threadIdx.x * 2654435761u + blockIdx.x * 97u + 1u;
    const typename T::A a = typename T::A(1);
    const typename T::B b = typename T::B(1);
    for (int it = 0; it < iters; ++it) {
        s = s * 1664525u + 1013904223u;
#pragma unroll
        for (int u = 0; u < 8; ++u) T::combine(acc, int(((s >> 7) + unsigned(u) * 1031u) & (CAL_SLOTS - 1)), a, b);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long x = 0;
        for (int i = 0; i < 8; ++i) x += (unsigned long long)(acc[i] != T::empty());
        atomicAdd(sink, x);
    }
}

template <int ALG>
stc_status calibrate_acc(stc_handle* h, double* rate, stc_stream s) {
    StcScratch sc(h, s);
    unsigned long long* sink = sc.get<unsigned long long>(1);
    if (!sink) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(sink, 0, sizeof(unsigned long long), s));
    const int iters = 1024;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    STC_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return STC_ERR_CUDA;
    }
    float best = 0.0f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {  // the first run warms up; the fastest of the others counts
        ok = cudaEventRecord(e0, s) == cudaSuccess;
        k_calibrate_acc<ALG><<<unsigned(h->num_sms), 1024, 0, s>>>(iters, sink);
        ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.0f;
        ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        stc_count(h);
        if (ok && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || !(best > 0.0f)) {
        (void)cudaGetLastError();
        return STC_ERR_CUDA;
    }
    *rate = double(h->num_sms) * 1024.0 * iters * 8.0 / (double(best) * 1e-3);
    return STC_OK;
}

}  // namespace

stc_status stc_calibrate_accumulate_impl(stc_handle* h, int alg, double* rate, stc_stream s) {
    switch (alg) {
    case ALG_PT_F32: return calibrate_acc<ALG_PT_F32>(h, rate, s);
    case ALG_PT_F64: return calibrate_acc<ALG_PT_F64>(h, rate, s);
    case ALG_MP_I32: return calibrate_acc<ALG_MP_I32>(h, rate, s);
    case ALG_MP_F32: return calibrate_acc<ALG_MP_F32>(h, rate, s);
    case ALG_BOOL: return calibrate_acc<ALG_BOOL>(h, rate, s);
    default: return STC_ERR_ALGEBRA;
    }
}
