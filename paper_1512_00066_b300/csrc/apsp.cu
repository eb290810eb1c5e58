// All-pairs shortest paths by path doubling (Section 4.2): the closure of the
// adjacency matrix over the tropical semiring by repeated squaring.  With the
// zero diagonal added, P (x) P already contains every path of P (P_ii = 0), so
// P <- P (x) P doubles the hop count each step; after k squarings P holds the
// shortest paths of at most 2^k edges.  The loop stops when a squaring leaves P
// unchanged (structure and values), which is the closure when no cycle is
// negative; a negative diagonal entry then reports a negative cycle.
#include "stc_internal.cuh"

namespace {

// Row lengths of I + G: every row gets its diagonal entry unless it has one.
__global__ void k_diag_count(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col, int64_t nnz,
                             int64_t* __restrict__ cnt) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        int64_t a = lo, b = hi;  // first column >= i
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (int64_t(col[m]) < i) a = m + 1; else b = m;
        }
        const bool has = a < hi && int64_t(col[a]) == i;
        cnt[i] = (hi - lo) + (has ? 0 : 1);
    }
}

__device__ __forceinline__ int32_t weight_of(int32_t w) { return w; }
__device__ __forceinline__ int32_t weight_of(PathVal p) { return p.w; }

// I + G over (min,+): the diagonal entry is min(G_ii, 0); columns stay sorted.
// Warp per row.  V: int32 lengths, or paths (their weight is taken).
template <class V>
__global__ void k_diag_fill(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const V* __restrict__ val, int64_t nnz, const int64_t* __restrict__ optr,
                            int32_t* __restrict__ ocol, int32_t* __restrict__ oval) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        int64_t a = lo, b = hi;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (int64_t(col[m]) < i) a = m + 1; else b = m;
        }
        const bool has = a < hi && int64_t(col[a]) == i;
        const int64_t o = optr[i];
        for (int64_t p = lo + lane; p < hi; p += 32) {
            const int64_t q = o + (p - lo) + ((!has && p >= a) ? 1 : 0);
            ocol[q] = col[p];
            const int32_t w = weight_of(val[p]);
            oval[q] = (has && p == a) ? min(w, 0) : w;
        }
        if (!has && lane == 0) {
            ocol[o + (a - lo)] = int32_t(i);
            oval[o + (a - lo)] = 0;
        }
    }
}

// *diff != 0 when two CSRs of the same shape and nnz differ anywhere.
__global__ void k_csr_differ(int64_t n, int64_t nnz, const int64_t* __restrict__ p1, const int32_t* __restrict__ c1,
                             const int32_t* __restrict__ v1, const int64_t* __restrict__ p2,
                             const int32_t* __restrict__ c2, const int32_t* __restrict__ v2, int* __restrict__ diff) {
    int d = 0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i <= n; i += stride) d |= p1[i] != p2[i];
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz; e += stride)
        d |= (c1[e] != c2[e]) | (v1[e] != v2[e]);
    if (__syncthreads_or(d) && threadIdx.x == 0) atomicOr(diff, 1);
}

// Raises STC_FLAG_NEG_CYCLE when some diagonal entry is negative.
__global__ void k_neg_diag(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const int32_t* __restrict__ val, int64_t nnz, int* flags) {
    int bad = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        int64_t a = lo, b = hi;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (int64_t(col[m]) < i) a = m + 1; else b = m;
        }
        if (a < hi && int64_t(col[a]) == i && val[a] < 0) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, STC_FLAG_NEG_CYCLE);
}

// ----------------------------------------------------------------- Tiskin's path doubling
//
// Paths carry (w, h): weight and hops.  P starts as the edges (w, 1); for
// l = 1, 2, 4, ... < n, Pl = the entries of P with exactly l hops, and
// P <- P (+) Pl (x) P with (+) the lexicographic minimum of (w, h).  An entry of P
// is then the least weight over the paths of at most 2l hops and, among those,
// the fewest hops; a lexicographically least path of more than l hops has a
// prefix of exactly l hops that is itself least among the paths of at most l
// hops (else replacing it would give a lesser path), so it is in Pl, and its
// suffix of at most l hops is in P.  Ties broken by hops make the result
// independent of the order of reduction.

__global__ void k_to_paths(int64_t nnz, const int32_t* __restrict__ w, PathVal* __restrict__ out) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
        PathVal p;
        p.w = w[e];
        p.h = 1;
        out[e] = p;
    }
}

// Entries with exactly l hops: per-row counts (warp per row, ballots).
__global__ void k_hops_count(int64_t n, const int64_t* __restrict__ ptr, const PathVal* __restrict__ val, int64_t nnz,
                             int l, int64_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        int64_t c = 0;
        for (int64_t p0 = lo; p0 < hi; p0 += 32) {
            const bool k = p0 + lane < hi && val[p0 + lane].h == l;
            c += __popc(__ballot_sync(0xffffffffu, k));
        }
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void k_hops_fill(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const PathVal* __restrict__ val, int64_t nnz, int l, const int64_t* __restrict__ optr,
                            int32_t* __restrict__ ocol, PathVal* __restrict__ oval) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        int64_t o = optr[i];
        for (int64_t p0 = lo; p0 < hi; p0 += 32) {
            const int64_t p = p0 + lane;
            const bool k = p < hi && val[p].h == l;
            const unsigned m = __ballot_sync(0xffffffffu, k);
            if (k) {
                const int64_t q = o + __popc(m & ((1u << lane) - 1u));
                ocol[q] = col[p];
                oval[q] = val[p];
            }
            o += __popc(m);
        }
    }
}

__device__ __forceinline__ bool path_less(PathVal a, PathVal b) { return a.w < b.w || (a.w == b.w && a.h < b.h); }

// Row lengths of the union of P and Q (thread per row, merge of sorted columns).
__global__ void k_union_count(int64_t n, const int64_t* __restrict__ pp, const int32_t* __restrict__ pc, int64_t pnnz,
                              const int64_t* __restrict__ qp, const int32_t* __restrict__ qc, int64_t qnnz,
                              int64_t* __restrict__ cnt) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t a, ae, b, be;
        row_range(pp, i, pnnz, a, ae);
        row_range(qp, i, qnnz, b, be);
        int64_t c = 0;
        while (a < ae && b < be) {
            const int32_t x = pc[a], y = qc[b];
            a += x <= y;
            b += y <= x;
            ++c;
        }
        cnt[i] = c + (ae - a) + (be - b);
    }
}

// P (+) Q row by row: lexicographic minimum where both hold the column.
__global__ void k_union_fill(int64_t n, const int64_t* __restrict__ pp, const int32_t* __restrict__ pc,
                             const PathVal* __restrict__ pv, int64_t pnnz, const int64_t* __restrict__ qp,
                             const int32_t* __restrict__ qc, const PathVal* __restrict__ qv, int64_t qnnz,
                             const int64_t* __restrict__ optr, int32_t* __restrict__ ocol,
                             PathVal* __restrict__ oval) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        int64_t a, ae, b, be;
        row_range(pp, i, pnnz, a, ae);
        row_range(qp, i, qnnz, b, be);
        int64_t o = optr[i];
        while (a < ae || b < be) {
            const int32_t x = a < ae ? pc[a] : INT_MAX, y = b < be ? qc[b] : INT_MAX;
            if (x < y) {
                ocol[o] = x;
                oval[o] = pv[a++];
            } else if (y < x) {
                ocol[o] = y;
                oval[o] = qv[b++];
            } else {
                ocol[o] = x;
                oval[o] = path_less(qv[b], pv[a]) ? qv[b] : pv[a];
                ++a;
                ++b;
            }
            ++o;
        }
    }
}

// *products += sum over the entries (i, k) of L of nnz(P_k) (warp per row).
__global__ void k_count_products(int64_t n, const int64_t* __restrict__ lp, const int32_t* __restrict__ lc,
                                 int64_t lnnz, const int64_t* __restrict__ pp, unsigned long long* products) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    unsigned long long t = 0;
    for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        int64_t lo, hi;
        row_range(lp, i, lnnz, lo, hi);
        for (int64_t p = lo + lane; p < hi; p += 32) {
            const int32_t k = lc[p];
            t += (unsigned long long)(pp[k + 1] - pp[k]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0 && t) atomicAdd(products, t);
}

void free_csr(stc_handle* h, stc_csr& m, stc_stream s) {
    stc_free_bytes(h, m.rowptr, s);
    stc_free_bytes(h, m.col, s);
    stc_free_bytes(h, m.val, s);
    m.rowptr = nullptr;
    m.col = nullptr;
    m.val = nullptr;
}

}  // namespace

stc_status stc_apsp_impl(stc_handle* h, const stc_csr* G, stc_csr* P_out, int32_t* squarings_out, stc_stream s) {
    const int64_t n = G->nrows;
    *P_out = stc_csr{};
    P_out->nrows = n;
    P_out->ncols = n;
    stc_status st = stc_validate_csr_async(h, G, s);
    if (st != STC_OK) return st;
    // P0 = I + G
    stc_csr P{};
    P.nrows = n;
    P.ncols = n;
    P.rowptr = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(n + 1) * 8, s));
    if (!P.rowptr) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(P.rowptr, 0, sizeof(int64_t), s));
    const unsigned gb = unsigned(h->num_sms * 8);
    if (n > 0) {
        k_diag_count<<<gb, 256, 0, s>>>(n, G->rowptr, G->col, G->nnz, P.rowptr + 1);
        STC_LAUNCH_CHECK();
        stc_count(h);
        StcScratch sc(h, s);
        if ((st = stc_inclusive_scan_i64(h, sc, P.rowptr + 1, n, s)) != STC_OK) {
            free_csr(h, P, s);
            return st;
        }
    }
    int* ints = static_cast<int*>(stc_alloc_bytes(h, 16, s));
    if (!ints) {
        free_csr(h, P, s);
        return STC_ERR_OOM;
    }
    auto fail = [&](stc_status e) {
        (void)cudaGetLastError();
        free_csr(h, P, s);
        stc_free_bytes(h, ints, s);
        return e;
    };
    int* st_h = reinterpret_cast<int*>(&h->h_stage[2]);
    if (cudaMemcpyAsync(&h->h_stage[0], P.rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&st_h[0], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    if (st_h[0]) {
        const int f = st_h[0];
        (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
        return fail(stc_flags_to_status(f));
    }
    P.nnz = h->h_stage[0];
    P.col = static_cast<int32_t*>(stc_alloc_bytes(h, size_t(P.nnz) * 4, s));
    P.val = stc_alloc_bytes(h, size_t(P.nnz) * 4, s);
    if (!P.col || !P.val) return fail(STC_ERR_OOM);
    if (n > 0) {
        k_diag_fill<int32_t><<<gb, 256, 0, s>>>(n, G->rowptr, G->col, static_cast<const int32_t*>(G->val), G->nnz, P.rowptr,
                                       P.col, static_cast<int32_t*>(P.val));
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    // square until a squaring changes nothing (at most ceil(log2 n) + 1 squarings)
    const int max_sq = stc_log2_ceil(n > 1 ? n : 2) + 1;
    int squarings = 0;
    stc_opts o{};
    o.skip_validation = 1;  // P is built here: sorted, unique, in range
    for (; squarings < max_sq && n > 0;) {
        stc_csr Q{};
        if ((st = stc_spgemm_impl(h, ALG_MP_I32, &P, &P, &Q, &o, s)) != STC_OK) return fail(st);
        ++squarings;
        bool same = Q.nnz == P.nnz;
        if (same) {
            if (cudaMemsetAsync(ints, 0, sizeof(int), s) != cudaSuccess) {
                free_csr(h, Q, s);
                return fail(STC_ERR_CUDA);
            }
            k_csr_differ<<<gb, 256, 0, s>>>(n, P.nnz, P.rowptr, P.col, static_cast<const int32_t*>(P.val), Q.rowptr,
                                            Q.col, static_cast<const int32_t*>(Q.val), ints);
            stc_count(h);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(&st_h[1], ints, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                free_csr(h, Q, s);
                return fail(STC_ERR_CUDA);
            }
            same = st_h[1] == 0;
        }
        free_csr(h, P, s);
        P = Q;
        if (same) break;
    }
    if (n > 0) {
        k_neg_diag<<<gb, 256, 0, s>>>(n, P.rowptr, P.col, static_cast<const int32_t*>(P.val), P.nnz, h->d_flags);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    if (cudaMemcpyAsync(&st_h[0], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    if (st_h[0]) {
        const int f = st_h[0];
        (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
        return fail(stc_flags_to_status(f));
    }
    stc_free_bytes(h, ints, s);
    if (squarings_out) *squarings_out = squarings;
    *P_out = P;
    return STC_OK;
}

namespace {

// Row pointers from per-row counts already in ptr[1..n] (ptr[0] = 0): scan, then
// the total, read back (synchronises).
stc_status scan_rows(stc_handle* h, int64_t n, int64_t* ptr, int64_t* total, stc_stream s) {
    if (n > 0) {
        StcScratch sc(h, s);
        const stc_status st = stc_inclusive_scan_i64(h, sc, ptr + 1, n, s);
        if (st != STC_OK) return st;
    }
    STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[0], ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    *total = h->h_stage[0];
    return STC_OK;
}

stc_status alloc_rows(stc_handle* h, int64_t n, stc_csr& m, stc_stream s) {
    m = stc_csr{};
    m.nrows = n;
    m.ncols = n;
    m.rowptr = static_cast<int64_t*>(stc_alloc_bytes(h, size_t(n + 1) * 8, s));
    if (!m.rowptr) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(m.rowptr, 0, sizeof(int64_t), s));
    return STC_OK;
}

stc_status alloc_entries(stc_handle* h, stc_csr& m, size_t vbytes, stc_stream s) {
    m.col = static_cast<int32_t*>(stc_alloc_bytes(h, size_t(m.nnz) * 4, s));
    m.val = stc_alloc_bytes(h, size_t(m.nnz) * vbytes, s);
    return (m.col && m.val) ? STC_OK : STC_ERR_OOM;
}

}  // namespace

stc_status stc_apsp_tiskin_impl(stc_handle* h, const stc_csr* G, stc_csr* P_out, int32_t* rounds_out,
                                int64_t* products_out, stc_stream s) {
    const int64_t n = G->nrows;
    *P_out = stc_csr{};
    stc_status st = stc_validate_csr_async(h, G, s);
    if (st != STC_OK) return st;
    const unsigned gb = unsigned(h->num_sms * 8);
    stc_csr P{}, L{}, Q{}, U{}, D{};
    unsigned long long* prod = static_cast<unsigned long long*>(stc_alloc_bytes(h, 16, s));
    auto fail = [&](stc_status e) {
        (void)cudaGetLastError();
        free_csr(h, P, s);
        free_csr(h, L, s);
        free_csr(h, Q, s);
        free_csr(h, U, s);
        free_csr(h, D, s);
        stc_free_bytes(h, prod, s);
        return e;
    };
    if (!prod) return fail(STC_ERR_OOM);
    if (cudaMemsetAsync(prod, 0, 16, s) != cudaSuccess) return fail(STC_ERR_CUDA);
    // P = the edges as paths of one hop
    if ((st = alloc_rows(h, n, P, s)) != STC_OK) return fail(st);
    P.nnz = G->nnz;
    if ((st = alloc_entries(h, P, sizeof(PathVal), s)) != STC_OK) return fail(st);
    if (cudaMemcpyAsync(P.rowptr, G->rowptr, size_t(n + 1) * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        (G->nnz > 0 &&
         cudaMemcpyAsync(P.col, G->col, size_t(G->nnz) * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess))
        return fail(STC_ERR_CUDA);
    if (G->nnz > 0) {
        k_to_paths<<<gb, 256, 0, s>>>(G->nnz, static_cast<const int32_t*>(G->val), static_cast<PathVal*>(P.val));
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    int* f = reinterpret_cast<int*>(&h->h_stage[4]);
    *f = 0;
    if (cudaMemcpyAsync(f, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    if (*f) {
        const int flags = *f;
        (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
        return fail(stc_flags_to_status(flags));
    }
    stc_opts o{};
    o.skip_validation = 1;  // every operand is built here
    int rounds = 0;
    for (int64_t l = 1; l < n; l <<= 1) {
        // L = the paths of P with exactly l hops
        if ((st = alloc_rows(h, n, L, s)) != STC_OK) return fail(st);
        k_hops_count<<<gb, 256, 0, s>>>(n, P.rowptr, static_cast<const PathVal*>(P.val), P.nnz, int(l), L.rowptr + 1);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        if ((st = scan_rows(h, n, L.rowptr, &L.nnz, s)) != STC_OK) return fail(st);
        if (L.nnz == 0) {
            free_csr(h, L, s);
            break;  // no least path has l hops: none has more
        }
        if ((st = alloc_entries(h, L, sizeof(PathVal), s)) != STC_OK) return fail(st);
        k_hops_fill<<<gb, 256, 0, s>>>(n, P.rowptr, P.col, static_cast<const PathVal*>(P.val), P.nnz, int(l),
                                       L.rowptr, L.col, static_cast<PathVal*>(L.val));
        k_count_products<<<gb, 256, 0, s>>>(n, L.rowptr, L.col, L.nnz, P.rowptr, prod);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 2);
        // Q = L (x) P; P <- P (+) Q
        if ((st = stc_spgemm_impl(h, ALG_PATH, &L, &P, &Q, &o, s)) != STC_OK) return fail(st);
        free_csr(h, L, s);
        if ((st = alloc_rows(h, n, U, s)) != STC_OK) return fail(st);
        k_union_count<<<gb, 256, 0, s>>>(n, P.rowptr, P.col, P.nnz, Q.rowptr, Q.col, Q.nnz, U.rowptr + 1);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        if ((st = scan_rows(h, n, U.rowptr, &U.nnz, s)) != STC_OK) return fail(st);
        if ((st = alloc_entries(h, U, sizeof(PathVal), s)) != STC_OK) return fail(st);
        k_union_fill<<<gb, 256, 0, s>>>(n, P.rowptr, P.col, static_cast<const PathVal*>(P.val), P.nnz, Q.rowptr,
                                        Q.col, static_cast<const PathVal*>(Q.val), Q.nnz, U.rowptr, U.col,
                                        static_cast<PathVal*>(U.val));
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
        free_csr(h, P, s);
        free_csr(h, Q, s);
        P = U;
        U = stc_csr{};
        ++rounds;
    }
    // the distances, with the zero diagonal of the empty paths
    if ((st = alloc_rows(h, n, D, s)) != STC_OK) return fail(st);
    if (n > 0) {
        k_diag_count<<<gb, 256, 0, s>>>(n, P.rowptr, P.col, P.nnz, D.rowptr + 1);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h);
    }
    if ((st = scan_rows(h, n, D.rowptr, &D.nnz, s)) != STC_OK) return fail(st);
    if ((st = alloc_entries(h, D, 4, s)) != STC_OK) return fail(st);
    if (n > 0) {
        k_diag_fill<PathVal><<<gb, 256, 0, s>>>(n, P.rowptr, P.col, static_cast<const PathVal*>(P.val), P.nnz,
                                                D.rowptr, D.col, static_cast<int32_t*>(D.val));
        k_neg_diag<<<gb, 256, 0, s>>>(n, D.rowptr, D.col, static_cast<const int32_t*>(D.val), D.nnz, h->d_flags);
        if (cudaGetLastError() != cudaSuccess) return fail(STC_ERR_CUDA);
        stc_count(h, 2);
    }
    free_csr(h, P, s);
    *f = 0;
    if (cudaMemcpyAsync(f, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&h->h_stage[5], prod, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(STC_ERR_CUDA);
    if (*f) {
        const int flags = *f;
        (void)cudaMemsetAsync(h->d_flags, 0, sizeof(int), s);
        return fail(stc_flags_to_status(flags));
    }
    stc_free_bytes(h, prod, s);
    if (rounds_out) *rounds_out = rounds;
    if (products_out) *products_out = h->h_stage[5];
    D.ncols = n;
    *P_out = D;
    return STC_OK;
}
