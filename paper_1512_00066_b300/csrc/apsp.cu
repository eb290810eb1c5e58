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

// I + G over (min,+): the diagonal entry is min(G_ii, 0); columns stay sorted.
// Warp per row.
__global__ void k_diag_fill(int64_t n, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ val, int64_t nnz, const int64_t* __restrict__ optr,
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
            oval[q] = (has && p == a) ? min(val[p], 0) : val[p];
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
        k_diag_fill<<<gb, 256, 0, s>>>(n, G->rowptr, G->col, static_cast<const int32_t*>(G->val), G->nnz, P.rowptr,
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
