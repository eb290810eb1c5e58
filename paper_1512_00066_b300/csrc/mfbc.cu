// Betweenness centrality over the (distance, multiplicity) monoid, many sources
// at once (the paper points to the geodetic semiring for betweenness centrality,
// Section 4.2; the accumulation is Brandes').
//
// State is vertex-major, [v][s] for the S sources of a batch, so that relaxing
// one edge touches one contiguous S-element slice per array.
//
// Forward (shortest distances d and path counts sigma): Bellman-Ford over the
// monoid (d1,s1) (+) (d2,s2) = smaller d, or (d, s1+s2) on a tie, reached by the
// pairwise function f(w, (d, s)) = (d + w, s).  Each vertex/source pair carries the
// multiplicity it has not propagated yet (delta); a round sends (d_u + w, delta_u)
// along the out-edges of the frontier, keeps the minimum distance per target
// (atomicMin), then adds the deltas of the candidates that reach that minimum
// (atomicAdd).  A target whose distance dropped restarts its count from the new
// deltas; one whose distance held adds them.  Because (+) is additive in the
// multiplicity at a fixed distance, the deltas sent at a vertex's final distance
// sum to its final count, so the fixed point is Brandes' sigma.
//
// Backward (dependencies): c_s(v) = number of shortest-path successors.  Vertices
// with no pending successor are ready; a ready w adds sigma_v / sigma_w *
// (1 + delta_w) to every predecessor v on a shortest path (in-edge CSR) and
// decrements its count; a count reaching zero makes v ready for the next round.
// bc[v] += sum over the batch's sources s != v of delta_s(v).
#include "stc_internal.cuh"

namespace {

constexpr int MF_NT = 256;       // one thread per source of the batch
constexpr int MF_ITEM_EDGES = 1024;  // out-edges of one vertex handled by one block
constexpr int MF_INF = STC_MIN_PLUS_I32_IDENTITY;

struct MfGraph {
    int64_t n, nnz;
    const int64_t* __restrict__ ptr;
    const int32_t* __restrict__ col;
    const int32_t* __restrict__ w;  // null: unit lengths
};

struct MfState {
    int S;
    int* d;          // [n][S] distance
    int* dn;         // [n][S] distance candidate of the round; successor count backward
    double* sig;     // [n][S] path count
    double* dl;      // [n][S] multiplicity not yet propagated; dependency backward
    double* dln;     // [n][S] multiplicity gathered in the round
    int* stamp;      // [n] round stamp of list membership
    int32_t* list[2];  // frontier / touched lists
    int64_t* iprefix;  // work-item prefix over the frontier
    int* cnt;        // [0] frontier size, [1] touched size, [2] next size
};

__device__ __forceinline__ int edge_len(const MfGraph& g, int64_t p) { return g.w ? g.w[p] : 1; }

__global__ void k_mf_init(MfGraph g, MfState st, const int32_t* __restrict__ src) {
    const int S = st.S;
    const int64_t tot = g.n * S;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < tot;
         i += int64_t(gridDim.x) * blockDim.x) {
        st.d[i] = MF_INF;
        st.dn[i] = MF_INF;
        st.sig[i] = 0.0;
        st.dl[i] = 0.0;
        st.dln[i] = 0.0;
    }
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < g.n;
         v += int64_t(gridDim.x) * blockDim.x)
        st.stamp[v] = -1;
}

// Sources: distance 0, one path, one pending multiplicity; frontier = sources.
__global__ void k_mf_seed(MfGraph g, MfState st, const int32_t* __restrict__ src) {
    const int s = threadIdx.x;
    if (s < st.S) {
        const int64_t v = src[s];
        const int64_t i = v * st.S + s;
        st.d[i] = 0;
        st.dn[i] = 0;
        st.sig[i] = 1.0;
        st.dl[i] = 1.0;
        if (atomicExch(&st.stamp[v], -2) != -2) st.list[0][atomicAdd(&st.cnt[0], 1)] = int32_t(v);
    }
}

// Work items of the frontier: vertex u contributes ceil(deg(u) / MF_ITEM_EDGES).
__global__ void k_mf_items(MfGraph g, const int32_t* __restrict__ F, const int* __restrict__ nF,
                           int64_t* __restrict__ count) {
    const int n = *nF;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t lo, hi;
        row_range(g.ptr, F[i], g.nnz, lo, hi);
        count[i] = (hi - lo + MF_ITEM_EDGES - 1) / MF_ITEM_EDGES;
    }
}

// Locate work item t: frontier index j (largest with prefix[j] <= t, prefix inclusive
// of the item counts shifted: excl[j] = incl[j] - count[j]).
__device__ __forceinline__ int mf_find(const int64_t* __restrict__ incl, int n, int64_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (incl[mid] > t) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Phase A of a round: dn[v][s] = min(dn[v][s], d[u][s] + w) over frontier edges
// with pending multiplicity; every target is listed once as touched.
__global__ void __launch_bounds__(MF_NT) k_mf_relax_min(MfGraph g, MfState st, int round) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int nF = st.cnt[0];
    if (nF == 0) return;
    const int64_t nitems = st.iprefix[nF - 1];
    const int32_t* F = st.list[0];
    for (int64_t t = blockIdx.x; t < nitems; t += gridDim.x) {
        const int j = mf_find(st.iprefix, nF, t);
        const int64_t first = j > 0 ? st.iprefix[j - 1] : 0;
        const int32_t u = F[j];
        int64_t lo, hi;
        row_range(g.ptr, u, g.nnz, lo, hi);
        const int64_t e0 = lo + (t - first) * MF_ITEM_EDGES;
        const int64_t e1 = min(hi, e0 + MF_ITEM_EDGES);
        const bool act = s < S && st.dl[int64_t(u) * S + s] > 0.0;
        const int du = act ? st.d[int64_t(u) * S + s] : 0;
        if (!__syncthreads_or(act)) continue;
        for (int64_t p = e0; p < e1; ++p) {
            const int32_t v = g.col[p];
            if ((uint64_t)v >= (uint64_t)g.n) continue;
            if (act) {
                const int cand = du + edge_len(g, p);
                int* dst = &st.dn[int64_t(v) * S + s];
                if (cand < *dst) atomicMin(dst, cand);  // most candidates cannot improve
            }
            if (s == 0 && atomicExch(&st.stamp[v], round) != round)
                st.list[1][atomicAdd(&st.cnt[1], 1)] = v;
        }
    }
}

// Phase B: add the pending multiplicity of every candidate that reached the minimum.
__global__ void __launch_bounds__(MF_NT) k_mf_relax_add(MfGraph g, MfState st) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int nF = st.cnt[0];
    if (nF == 0) return;
    const int64_t nitems = st.iprefix[nF - 1];
    const int32_t* F = st.list[0];
    for (int64_t t = blockIdx.x; t < nitems; t += gridDim.x) {
        const int j = mf_find(st.iprefix, nF, t);
        const int64_t first = j > 0 ? st.iprefix[j - 1] : 0;
        const int32_t u = F[j];
        int64_t lo, hi;
        row_range(g.ptr, u, g.nnz, lo, hi);
        const int64_t e0 = lo + (t - first) * MF_ITEM_EDGES;
        const int64_t e1 = min(hi, e0 + MF_ITEM_EDGES);
        const double m = s < S ? st.dl[int64_t(u) * S + s] : 0.0;
        const bool act = m > 0.0;
        const int du = act ? st.d[int64_t(u) * S + s] : 0;
        if (!__syncthreads_or(act)) continue;
        if (!act) continue;
        for (int64_t p = e0; p < e1; ++p) {
            const int32_t v = g.col[p];
            if ((uint64_t)v >= (uint64_t)g.n) continue;
            const int64_t i = int64_t(v) * S + s;
            if (du + edge_len(g, p) == st.dn[i]) atomicAdd(&st.dln[i], m);
        }
    }
}

// The frontier has sent its multiplicities.
__global__ void __launch_bounds__(MF_NT) k_mf_clear_frontier(MfState st) {
    const int S = st.S;
    const int nF = st.cnt[0];
    for (int b = blockIdx.x; b < nF; b += gridDim.x) {
        const int32_t u = st.list[0][b];
        if (threadIdx.x < S) st.dl[int64_t(u) * S + threadIdx.x] = 0.0;
    }
}

// Apply the round to every touched vertex; those with pending multiplicity form
// the next frontier (written to list[0] after the swap done by the host driver:
// here into list[0] of the next round, passed as `next`).
__global__ void __launch_bounds__(MF_NT) k_mf_update(MfState st, int32_t* __restrict__ next,
                                                     int* __restrict__ cnt_next) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int nT = st.cnt[1];
    for (int b = blockIdx.x; b < nT; b += gridDim.x) {
        const int32_t v = st.list[1][b];
        bool act = false;
        if (s < S) {
            const int64_t i = int64_t(v) * S + s;
            const int nd = st.dn[i];
            const int od = st.d[i];
            const double m = st.dln[i];
            if (nd < od) {
                st.d[i] = nd;
                st.sig[i] = m;
                st.dl[i] = m;
                act = m > 0.0;
            } else if (m > 0.0) {
                st.sig[i] += m;
                st.dl[i] = m;
                act = true;
            }
            st.dln[i] = 0.0;
        }
        if (__syncthreads_or(act) && s == 0) next[atomicAdd(cnt_next, 1)] = v;
    }
}

// ------------------------------------------------------------------- backward

// c[v][s] = number of out-edges v -> x on a shortest path from s (into st.dn);
// vertices with a reachable source and no successor are ready.
__global__ void __launch_bounds__(MF_NT) k_mf_succ(MfGraph g, MfState st, int32_t* __restrict__ ready,
                                                   int* __restrict__ nready) {
    const int S = st.S;
    const int s = threadIdx.x;
    for (int64_t v = blockIdx.x; v < g.n; v += gridDim.x) {
        int64_t lo, hi;
        row_range(g.ptr, v, g.nnz, lo, hi);
        const int64_t i = v * S + s;
        const int dv = s < S ? st.d[i] : MF_INF;
        int c = 0;
        if (dv < MF_INF) {
            for (int64_t p = lo; p < hi; ++p) {
                const int32_t x = g.col[p];
                if ((uint64_t)x >= (uint64_t)g.n) continue;
                if (dv + edge_len(g, p) == st.d[int64_t(x) * S + s]) ++c;
            }
        }
        if (s < S) {
            st.dn[i] = dv < MF_INF ? c : -1;  // -1: unreachable or finished
            st.dl[i] = 0.0;
        }
        const bool rd = dv < MF_INF && c == 0;
        if (__syncthreads_or(rd) && s == 0) ready[atomicAdd(nready, 1)] = int32_t(v);
    }
}

// One backward round over the ready vertices (in-edge CSR gt: row w lists v -> w).
__global__ void __launch_bounds__(MF_NT) k_mf_back(MfGraph gt, MfState st, const int32_t* __restrict__ ready,
                                                   const int* __restrict__ nready, int32_t* __restrict__ next,
                                                   int* __restrict__ nnext, int round) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int nR = *nready;
    for (int b = blockIdx.x; b < nR; b += gridDim.x) {
        const int32_t w = ready[b];
        const int64_t iw = int64_t(w) * S + s;
        bool go = false;
        double coef = 0.0;
        int dw = 0;
        if (s < S && st.dn[iw] == 0) {
            go = true;
            st.dn[iw] = -1;  // processed
            coef = (1.0 + st.dl[iw]) / st.sig[iw];
            dw = st.d[iw];
        }
        if (!__syncthreads_or(go)) continue;
        int64_t lo, hi;
        row_range(gt.ptr, w, gt.nnz, lo, hi);
        if (!go) continue;
        for (int64_t p = lo; p < hi; ++p) {
            const int32_t v = gt.col[p];
            if ((uint64_t)v >= (uint64_t)gt.n) continue;
            const int64_t iv = int64_t(v) * S + s;
            if (st.d[iv] + edge_len(gt, p) == dw) {
                atomicAdd(&st.dl[iv], st.sig[iv] * coef);
                // the source whose count reaches zero lists v (once per round)
                if (atomicSub(&st.dn[iv], 1) == 1 && atomicExch(&st.stamp[v], round) != round)
                    next[atomicAdd(nnext, 1)] = v;
            }
        }
    }
}

// bc[v] += sum over sources s != v of delta_s(v).
__global__ void __launch_bounds__(MF_NT) k_mf_bc(MfState st, int64_t n, const int32_t* __restrict__ src,
                                                 double* __restrict__ bc) {
    const int S = st.S;
    const int s = threadIdx.x;
    __shared__ double red[MF_NT / 32];
    for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
        double x = 0.0;
        if (s < S && src[s] != v && st.d[v * S + s] < MF_INF) x = st.dl[v * S + s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((s & 31) == 0) red[s >> 5] = x;
        __syncthreads();
        if (s == 0) {
            double t = 0.0;
            for (int k = 0; k < MF_NT / 32; ++k) t += red[k];
            bc[v] += t;
        }
        __syncthreads();
    }
}

__global__ void k_mf_zero(double* __restrict__ x, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] = 0.0;
}

// ------------------------------------------------------------------- transpose

__global__ void k_tr_count(MfGraph g, int64_t* __restrict__ indeg) {
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < g.nnz; p += int64_t(gridDim.x) * blockDim.x) {
        const int32_t v = g.col[p];
        if ((uint64_t)v < (uint64_t)g.n) atomicAdd(reinterpret_cast<unsigned long long*>(&indeg[v + 1]), 1ull);
    }
}

// Scatter edge u -> v into row v of the transpose (order inside a row arbitrary).
__global__ void k_tr_fill(MfGraph g, const int64_t* __restrict__ tptr, int64_t* __restrict__ cursor,
                          int32_t* __restrict__ tcol, int32_t* __restrict__ tw) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t u = warp; u < g.n; u += nwarps) {
        int64_t lo, hi;
        row_range(g.ptr, u, g.nnz, lo, hi);
        for (int64_t p = lo + lane; p < hi; p += 32) {
            const int32_t v = g.col[p];
            if ((uint64_t)v >= (uint64_t)g.n) continue;
            const int64_t q = tptr[v] + int64_t(atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[v]), 1ull));
            tcol[q] = int32_t(u);
            if (tw) tw[q] = g.w[p];
        }
    }
}

// Edge lengths must be >= 1 (a zero-length cycle would break the shortest-path DAG).
__global__ void k_mf_check_len(const int32_t* __restrict__ w, int64_t nnz, int* flags) {
    int bad = 0;
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < nnz; p += int64_t(gridDim.x) * blockDim.x)
        bad |= w[p] < 1;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, STC_FLAG_INVALID);
}

unsigned grid_for(stc_handle* h, int64_t work, int per_sm) {
    int64_t cap = int64_t(h->num_sms) * per_sm;
    if (work < 1) work = 1;
    return unsigned(work < cap ? work : cap);
}

// Forward phase for one batch (sources on the device, S of them).
stc_status mf_forward(stc_handle* h, StcScratch& sc, const MfGraph& g, MfState& st, const int32_t* d_src,
                      int64_t* d_count, stc_stream s, int* rounds_out) {
    STC_CUDA_TRY(cudaMemsetAsync(st.cnt, 0, 4 * sizeof(int), s));
    k_mf_init<<<grid_for(h, g.n * st.S / 256 + 1, 16), 256, 0, s>>>(g, st, d_src);
    k_mf_seed<<<1, MF_NT, 0, s>>>(g, st, d_src);
    STC_LAUNCH_CHECK();
    stc_count(h, 2);
    int* h_cnt = reinterpret_cast<int*>(&h->h_stage[4]);
    int rounds = 0;
    for (int r = 0;; ++r) {
        // the frontier is list[0] with size cnt[0]
        STC_CUDA_TRY(cudaMemcpyAsync(h_cnt, &st.cnt[0], sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        const int nF = *h_cnt;
        if (nF == 0) break;
        if (int64_t(r) > g.n + 1) {
            int f = STC_FLAG_NEG_CYCLE;
            STC_CUDA_TRY(cudaMemcpyAsync(h->d_flags, &f, sizeof(int), cudaMemcpyHostToDevice, s));
            break;
        }
        ++rounds;
        k_mf_items<<<grid_for(h, (nF + 255) / 256, 8), 256, 0, s>>>(g, st.list[0], &st.cnt[0], d_count);
        STC_LAUNCH_CHECK();
        stc_count(h);
        stc_status e = stc_inclusive_scan_i64(h, sc, d_count, nF, s);
        if (e != STC_OK) return e;
        st.iprefix = d_count;
        STC_CUDA_TRY(cudaMemsetAsync(&st.cnt[1], 0, 2 * sizeof(int), s));
        const unsigned gb = grid_for(h, int64_t(nF) * 4, 16);
        k_mf_relax_min<<<gb, MF_NT, 0, s>>>(g, st, r);
        k_mf_relax_add<<<gb, MF_NT, 0, s>>>(g, st);
        k_mf_clear_frontier<<<grid_for(h, nF, 16), MF_NT, 0, s>>>(st);
        // next frontier into the frontier list slot after the update reads it
        k_mf_update<<<grid_for(h, int64_t(nF) * 8, 16), MF_NT, 0, s>>>(st, st.list[0], &st.cnt[2]);
        STC_LAUNCH_CHECK();
        stc_count(h, 4);
        STC_CUDA_TRY(cudaMemcpyAsync(&st.cnt[0], &st.cnt[2], sizeof(int), cudaMemcpyDeviceToDevice, s));
    }
    if (rounds_out) *rounds_out = rounds;
    return STC_OK;
}

// Length check, then read the validation flags before any round runs.
stc_status mf_check(stc_handle* h, const MfGraph& g, stc_stream s) {
    if (g.w && g.nnz > 0) {
        k_mf_check_len<<<grid_for(h, g.nnz / 256 + 1, 8), 256, 0, s>>>(g.w, g.nnz, h->d_flags);
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    int* f = reinterpret_cast<int*>(&h->h_stage[7]);
    *f = 0;
    STC_CUDA_TRY(cudaMemcpyAsync(f, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    if (*f) {
        const int flags = *f;
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(flags);
    }
    return STC_OK;
}

stc_status mf_alloc_state(StcScratch& sc, int64_t n, int S, MfState& st, int64_t** d_count) {
    const size_t ns = size_t(n) * size_t(S);
    st.S = S;
    st.d = sc.get<int>(ns);
    st.dn = sc.get<int>(ns);
    st.sig = sc.get<double>(ns);
    st.dl = sc.get<double>(ns);
    st.dln = sc.get<double>(ns);
    st.stamp = sc.get<int>(size_t(n));
    st.list[0] = sc.get<int32_t>(size_t(n));
    st.list[1] = sc.get<int32_t>(size_t(n));
    st.cnt = sc.get<int>(8);
    *d_count = sc.get<int64_t>(size_t(n));
    return sc.failed ? STC_ERR_OOM : STC_OK;
}

}  // namespace

stc_status stc_mfbc_sssp_impl(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsrc,
                              int32_t* d_out, double* sigma_out, int32_t* rounds_out, stc_stream s) {
    StcScratch sc(h, s);
    MfGraph g{G->nrows, G->nnz, G->rowptr, G->col, static_cast<const int32_t*>(G->val)};
    stc_status st = stc_validate_csr_async(h, G, s);
    if (st != STC_OK) return st;
    if ((st = mf_check(h, g, s)) != STC_OK) return st;
    MfState ms;
    int64_t* d_count = nullptr;
    if ((st = mf_alloc_state(sc, g.n, nsrc, ms, &d_count)) != STC_OK) return st;
    int32_t* d_src = sc.get<int32_t>(size_t(nsrc));
    if (!d_src) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemcpyAsync(d_src, sources, sizeof(int32_t) * nsrc, cudaMemcpyHostToDevice, s));
    if ((st = mf_forward(h, sc, g, ms, d_src, d_count, s, rounds_out)) != STC_OK) return st;
    STC_CUDA_TRY(cudaMemcpyAsync(d_out, ms.d, sizeof(int) * size_t(g.n) * nsrc, cudaMemcpyDeviceToDevice, s));
    STC_CUDA_TRY(cudaMemcpyAsync(sigma_out, ms.sig, sizeof(double) * size_t(g.n) * nsrc,
                                 cudaMemcpyDeviceToDevice, s));
    int f = 0;
    STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[6], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    f = reinterpret_cast<int*>(&h->h_stage[6])[0];
    if (f) {
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(f);
    }
    return STC_OK;
}

stc_status stc_mfbc_impl(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsrc, int32_t batch,
                         double* bc, stc_stream s) {
    StcScratch sc(h, s);
    MfGraph g{G->nrows, G->nnz, G->rowptr, G->col, static_cast<const int32_t*>(G->val)};
    stc_status st = stc_validate_csr_async(h, G, s);
    if (st != STC_OK) return st;
    if ((st = mf_check(h, g, s)) != STC_OK) return st;
    // in-edge CSR for the backward phase
    int64_t* tptr = sc.get<int64_t>(size_t(g.n) + 1);
    int64_t* cursor = sc.get<int64_t>(size_t(g.n));
    int32_t* tcol = sc.get<int32_t>(size_t(g.nnz));
    int32_t* tw = g.w ? sc.get<int32_t>(size_t(g.nnz)) : nullptr;
    if (sc.failed) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(tptr, 0, sizeof(int64_t) * (size_t(g.n) + 1), s));
    STC_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int64_t) * size_t(g.n), s));
    k_tr_count<<<grid_for(h, g.nnz / 256 + 1, 16), 256, 0, s>>>(g, tptr);
    STC_LAUNCH_CHECK();
    stc_count(h);
    if ((st = stc_inclusive_scan_i64(h, sc, tptr + 1, g.n, s)) != STC_OK) return st;
    k_tr_fill<<<grid_for(h, g.n * 32 / 256 + 1, 16), 256, 0, s>>>(g, tptr, cursor, tcol, tw);
    STC_LAUNCH_CHECK();
    stc_count(h);
    MfGraph gt{g.n, g.nnz, tptr, tcol, tw};

    MfState ms;
    int64_t* d_count = nullptr;
    if ((st = mf_alloc_state(sc, g.n, batch, ms, &d_count)) != STC_OK) return st;
    int32_t* d_src = sc.get<int32_t>(size_t(batch));
    if (!d_src) return STC_ERR_OOM;
    k_mf_zero<<<grid_for(h, g.n / 256 + 1, 16), 256, 0, s>>>(bc, g.n);
    STC_LAUNCH_CHECK();
    stc_count(h);
    int* h_cnt = reinterpret_cast<int*>(&h->h_stage[5]);
    for (int32_t b0 = 0; b0 < nsrc; b0 += batch) {
        const int S = nsrc - b0 < batch ? nsrc - b0 : batch;
        ms.S = S;
        STC_CUDA_TRY(cudaMemcpyAsync(d_src, sources + b0, sizeof(int32_t) * S, cudaMemcpyHostToDevice, s));
        if ((st = mf_forward(h, sc, g, ms, d_src, d_count, s, nullptr)) != STC_OK) return st;
        // backward: successor counts, then ready rounds (lists reuse the frontier lists)
        STC_CUDA_TRY(cudaMemsetAsync(ms.cnt, 0, 4 * sizeof(int), s));
        k_mf_succ<<<grid_for(h, g.n, 32), MF_NT, 0, s>>>(g, ms, ms.list[0], &ms.cnt[0]);
        STC_LAUNCH_CHECK();
        stc_count(h);
        for (int r = 0, cur = 0;; ++r, cur ^= 1) {
            STC_CUDA_TRY(cudaMemcpyAsync(h_cnt, &ms.cnt[cur], sizeof(int), cudaMemcpyDeviceToHost, s));
            STC_CUDA_TRY(cudaStreamSynchronize(s));
            if (*h_cnt == 0) break;
            STC_CUDA_TRY(cudaMemsetAsync(&ms.cnt[cur ^ 1], 0, sizeof(int), s));
            k_mf_back<<<grid_for(h, *h_cnt, 16), MF_NT, 0, s>>>(gt, ms, ms.list[cur], &ms.cnt[cur],
                                                                ms.list[cur ^ 1], &ms.cnt[cur ^ 1], r + (1 << 30));
            STC_LAUNCH_CHECK();
            stc_count(h);
        }
        k_mf_bc<<<grid_for(h, g.n, 32), MF_NT, 0, s>>>(ms, g.n, d_src, bc);
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[6], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    const int f = reinterpret_cast<int*>(&h->h_stage[6])[0];
    if (f) {
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(f);
    }
    return STC_OK;
}
