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
constexpr int MF_BLOCKS_PER_SM = 8;  // fixed grids of the round kernels (2048 threads per SM)

// Device counters (MfState::cnt).  Both round loops keep their round index and
// list sizes here, so a round never needs a value from the host.
enum : int {
    MF_C_READY = 0,    // [0], [1]: backward ready-list sizes (by round parity)
    MF_C_TOUCHED = 2,  // forward touched-list size
    MF_C_ITEMS = 3,    // [3], [4]: forward work-item counts (by round parity)
    MF_C_FROUND = 5,   // forward round index
    MF_C_BROUND = 6,   // backward round index
    MF_C_GO = 7,       // 1 while the last checked loop goes on (read by the host driver)
    MF_C_NUM = 8,
};

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
    int32_t* list[2];  // forward: list[1] touched vertices; backward: ready lists
    int2* items[2];    // forward frontier work items {vertex, chunk of MF_ITEM_EDGES edges}
    int* cnt;          // MF_C_* counters
};

__device__ __forceinline__ int edge_len(const MfGraph& g, int64_t p) { return g.w ? g.w[p] : 1; }

// Select a double-buffered array by parity without indexing the kernel
// parameter (a dynamic index would copy the struct to local memory).
template <class T>
__device__ __forceinline__ T* mf_pick(T* const (&a)[2], int k) { return (k & 1) ? a[1] : a[0]; }

// Work items of a frontier vertex: one per MF_ITEM_EDGES out-edges, at least one
// (the item with chunk 0 also clears the vertex's pending multiplicity).
__device__ __forceinline__ int mf_chunks(const MfGraph& g, int32_t u) {
    int64_t lo, hi;
    row_range(g.ptr, u, g.nnz, lo, hi);
    const int64_t c = (hi - lo + MF_ITEM_EDGES - 1) / MF_ITEM_EDGES;
    return c > 1 ? int(c) : 1;
}

__global__ void k_mf_init(MfGraph g, MfState st) {
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
    if (blockIdx.x == 0 && threadIdx.x < MF_C_NUM) st.cnt[threadIdx.x] = 0;
}

// Sources: distance 0, one path, one pending multiplicity; their work items form
// the frontier of round 0.
__global__ void k_mf_seed(MfGraph g, MfState st, const int32_t* __restrict__ src) {
    const int s = threadIdx.x;
    if (s < st.S) {
        const int32_t v = src[s];
        const int64_t i = int64_t(v) * st.S + s;
        st.d[i] = 0;
        st.dn[i] = 0;
        st.sig[i] = 1.0;
        st.dl[i] = 1.0;
        if (atomicExch(&st.stamp[v], -2) != -2) {
            const int nch = mf_chunks(g, v);
            const int base = atomicAdd(&st.cnt[MF_C_ITEMS], nch);
            for (int c = 0; c < nch; ++c) st.items[0][base + c] = make_int2(v, c);
        }
    }
}

// Edge range of a work item.
__device__ __forceinline__ void mf_item_edges(const MfGraph& g, int2 it, int64_t& e0, int64_t& e1) {
    int64_t lo, hi;
    row_range(g.ptr, it.x, g.nnz, lo, hi);
    e0 = lo + int64_t(it.y) * MF_ITEM_EDGES;
    e1 = min(hi, e0 + MF_ITEM_EDGES);
}

// Edges of an item are taken MF_UNR at a time: the columns, lengths and the
// targets' source slices are all loaded before any compare or atomic, so one
// group costs one round trip to L2 instead of one per edge.
constexpr int MF_UNR = 4;

// List v as touched in round r once (stamp read first: most targets are listed).
__device__ __forceinline__ void mf_touch(int* stamp, int32_t* touched, int* count, int32_t v, int r) {
    if (stamp[v] != r && atomicExch(&stamp[v], r) != r) touched[atomicAdd(count, 1)] = v;
}

// Phase A of a round: dn[v][s] = min(dn[v][s], d[u][s] + w) over frontier edges
// with pending multiplicity; every target is listed once as touched.
__global__ void __launch_bounds__(MF_NT) k_mf_relax_min(MfGraph g, MfState st) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int r = st.cnt[MF_C_FROUND];
    const int nitems = st.cnt[MF_C_ITEMS + (r & 1)];
    const int2* __restrict__ F = mf_pick(st.items, r);
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        const int2 it = F[t];
        const int32_t u = it.x;
        int64_t e0, e1;
        mf_item_edges(g, it, e0, e1);
        const bool act = s < S && st.dl[int64_t(u) * S + s] > 0.0;
        const int du = act ? st.d[int64_t(u) * S + s] : 0;
        if (!__syncthreads_or(act)) continue;
        for (int64_t p0 = e0; p0 < e1; p0 += MF_UNR) {
            int32_t v[MF_UNR];
            int w[MF_UNR], cur[MF_UNR];
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) {
                const int64_t p = p0 + k;
                v[k] = -1;
                if (p < e1) {
                    const int32_t x = g.col[p];
                    if ((uint64_t)x < (uint64_t)g.n) v[k] = x;
                    w[k] = edge_len(g, p);
                }
            }
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) cur[k] = (act && v[k] >= 0) ? st.dn[int64_t(v[k]) * S + s] : 0;
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k)
                if (act && v[k] >= 0 && du + w[k] < cur[k]) atomicMin(&st.dn[int64_t(v[k]) * S + s], du + w[k]);
            // thread k lists target k
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k)
                if (s == k && v[k] >= 0) mf_touch(st.stamp, st.list[1], &st.cnt[MF_C_TOUCHED], v[k], r);
        }
    }
}

// Batches of at most MF_WARP_UNITS_MAX sources run the relax and backward kernels
// by work units (item, group of 32 sources), one warp each, lane per source: a unit
// whose sources are all idle at the item's vertex ends after one vote, no block-wide
// barrier is needed, and a block's threads are not left idle by a small batch.  A
// warp reads 32 edges' targets and lengths at once (one per lane) and hands them
// round by shuffles.  Larger batches keep a block per item (the eight warps of an
// item share its edge loads).
constexpr int MF_WARP_UNITS_MAX = 128;
__device__ __forceinline__ int mf_groups(int S) { return (S + 31) >> 5; }

// Edges [c0, c0 + 32) of [c0, e1): lane j's target (or -1) and length.
__device__ __forceinline__ void mf_edge_chunk(const MfGraph& g, int64_t c0, int64_t e1, int lane, int32_t& v,
                                              int& w) {
    v = -1;
    w = 0;
    if (c0 + lane < e1) {
        const int32_t x = g.col[c0 + lane];
        if ((uint64_t)x < (uint64_t)g.n) v = x;
        w = edge_len(g, c0 + lane);
    }
}

// k_mf_relax_min by warp units; a target is listed (once) as touched when some
// source's candidate reaches or lowers its distance.
__global__ void __launch_bounds__(MF_NT) k_mf_relax_min_w(MfGraph g, MfState st) {
    const int S = st.S;
    const int lane = threadIdx.x & 31;
    const int ng = mf_groups(S);
    const int r = st.cnt[MF_C_FROUND];
    const int nitems = st.cnt[MF_C_ITEMS + (r & 1)];
    const int2* __restrict__ F = mf_pick(st.items, r);
    const int units = nitems * ng;
    const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
    for (int q = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); q < units; q += nwarps) {
        const int2 it = F[q / ng];
        const int s = (q % ng) * 32 + lane;
        const int32_t u = it.x;
        const bool act = s < S && st.dl[int64_t(u) * S + s] > 0.0;
        if (!__any_sync(0xffffffffu, act)) continue;
        const int du = act ? st.d[int64_t(u) * S + s] : 0;
        int64_t e0, e1;
        mf_item_edges(g, it, e0, e1);
        for (int64_t c0 = e0; c0 < e1; c0 += 32) {
            int32_t vl;
            int wl;
            mf_edge_chunk(g, c0, e1, lane, vl, wl);
            const int nc = int(e1 - c0 < 32 ? e1 - c0 : 32);
            for (int k0 = 0; k0 < nc; k0 += MF_UNR) {
                int32_t v[MF_UNR];
                int w[MF_UNR], cur[MF_UNR];
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) {
                    v[k] = __shfl_sync(0xffffffffu, vl, (k0 + k) & 31);
                    w[k] = __shfl_sync(0xffffffffu, wl, (k0 + k) & 31);
                    if (k0 + k >= nc) v[k] = -1;
                }
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) cur[k] = (act && v[k] >= 0) ? st.dn[int64_t(v[k]) * S + s] : 0;
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) {
                    const bool near = act && v[k] >= 0 && du + w[k] <= cur[k];
                    if (near && du + w[k] < cur[k]) atomicMin(&st.dn[int64_t(v[k]) * S + s], du + w[k]);
                    if (__any_sync(0xffffffffu, near) && lane == 0)
                        mf_touch(st.stamp, st.list[1], &st.cnt[MF_C_TOUCHED], v[k], r);
                }
            }
        }
    }
}

// Phases A and B in one pass for unit lengths (g.w == null): every source's
// frontier in round r is its BFS level r (all sources start together), so every
// candidate of the round is r + 1 and none can lower a target below a tie; the
// multiplicity of a candidate that ties the minimum (atomicMin's old value
// >= r + 1) is added here and k_mf_relax_add is not run.
__global__ void __launch_bounds__(MF_NT, 8) k_mf_relax_unit(MfGraph g, MfState st) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int r = st.cnt[MF_C_FROUND];
    const int nitems = st.cnt[MF_C_ITEMS + (r & 1)];
    const int2* __restrict__ F = mf_pick(st.items, r);
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        const int2 it = F[t];
        const int32_t u = it.x;
        int64_t e0, e1;
        mf_item_edges(g, it, e0, e1);
        const double m = s < S ? st.dl[int64_t(u) * S + s] : 0.0;
        const bool act = m > 0.0;
        const int cand = act ? st.d[int64_t(u) * S + s] + 1 : 0;
        if (!__syncthreads_or(act)) continue;
        for (int64_t p0 = e0; p0 < e1; p0 += MF_UNR) {
            int32_t v[MF_UNR];
            int cur[MF_UNR];
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) {
                const int64_t p = p0 + k;
                v[k] = -1;
                if (p < e1) {
                    const int32_t x = g.col[p];
                    if ((uint64_t)x < (uint64_t)g.n) v[k] = x;
                }
            }
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) cur[k] = (act && v[k] >= 0) ? st.dn[int64_t(v[k]) * S + s] : 0;
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) {
                if (act && v[k] >= 0 && cand <= cur[k]) {
                    const int64_t i = int64_t(v[k]) * S + s;
                    const int old = cand < cur[k] ? atomicMin(&st.dn[i], cand) : cand;
                    if (old >= cand) atomicAdd(&st.dln[i], m);
                }
            }
            // thread k lists target k
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k)
                if (s == k && v[k] >= 0) mf_touch(st.stamp, st.list[1], &st.cnt[MF_C_TOUCHED], v[k], r);
        }
    }
}

// Phase B: add the pending multiplicity of every candidate that reached the minimum.
__global__ void __launch_bounds__(MF_NT) k_mf_relax_add(MfGraph g, MfState st) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int r = st.cnt[MF_C_FROUND];
    const int nitems = st.cnt[MF_C_ITEMS + (r & 1)];
    const int2* __restrict__ F = mf_pick(st.items, r);
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        const int2 it = F[t];
        const int32_t u = it.x;
        int64_t e0, e1;
        mf_item_edges(g, it, e0, e1);
        const double m = s < S ? st.dl[int64_t(u) * S + s] : 0.0;
        const bool act = m > 0.0;
        const int du = act ? st.d[int64_t(u) * S + s] : 0;
        if (!__syncthreads_or(act)) continue;
        if (!act) continue;
        for (int64_t p0 = e0; p0 < e1; p0 += MF_UNR) {
            int32_t v[MF_UNR];
            int w[MF_UNR], cur[MF_UNR];
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) {
                const int64_t p = p0 + k;
                v[k] = -1;
                if (p < e1) {
                    const int32_t x = g.col[p];
                    if ((uint64_t)x < (uint64_t)g.n) v[k] = x;
                    w[k] = edge_len(g, p);
                }
            }
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) cur[k] = v[k] >= 0 ? st.dn[int64_t(v[k]) * S + s] : 0;
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k)
                if (v[k] >= 0 && du + w[k] == cur[k]) atomicAdd(&st.dln[int64_t(v[k]) * S + s], m);
        }
    }
}

// k_mf_relax_add by warp units.
__global__ void __launch_bounds__(MF_NT) k_mf_relax_add_w(MfGraph g, MfState st) {
    const int S = st.S;
    const int lane = threadIdx.x & 31;
    const int ng = mf_groups(S);
    const int r = st.cnt[MF_C_FROUND];
    const int nitems = st.cnt[MF_C_ITEMS + (r & 1)];
    const int2* __restrict__ F = mf_pick(st.items, r);
    const int units = nitems * ng;
    const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
    for (int q = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); q < units; q += nwarps) {
        const int2 it = F[q / ng];
        const int s = (q % ng) * 32 + lane;
        const int32_t u = it.x;
        const double m = s < S ? st.dl[int64_t(u) * S + s] : 0.0;
        const bool act = m > 0.0;
        if (!__any_sync(0xffffffffu, act)) continue;
        const int du = act ? st.d[int64_t(u) * S + s] : 0;
        int64_t e0, e1;
        mf_item_edges(g, it, e0, e1);
        for (int64_t c0 = e0; c0 < e1; c0 += 32) {
            int32_t vl;
            int wl;
            mf_edge_chunk(g, c0, e1, lane, vl, wl);
            const int nc = int(e1 - c0 < 32 ? e1 - c0 : 32);
            for (int k0 = 0; k0 < nc; k0 += MF_UNR) {
                int32_t v[MF_UNR];
                int w[MF_UNR], cur[MF_UNR];
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) {
                    v[k] = __shfl_sync(0xffffffffu, vl, (k0 + k) & 31);
                    w[k] = __shfl_sync(0xffffffffu, wl, (k0 + k) & 31);
                    if (k0 + k >= nc) v[k] = -1;
                }
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) cur[k] = (act && v[k] >= 0) ? st.dn[int64_t(v[k]) * S + s] : 0;
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k)
                    if (act && v[k] >= 0 && du + w[k] == cur[k]) atomicAdd(&st.dln[int64_t(v[k]) * S + s], m);
            }
        }
    }
}

// The frontier has sent its multiplicities (each vertex once: its chunk-0 item).
__global__ void __launch_bounds__(MF_NT) k_mf_clear_frontier(MfState st) {
    const int S = st.S;
    const int r = st.cnt[MF_C_FROUND];
    const int nitems = st.cnt[MF_C_ITEMS + (r & 1)];
    const int2* __restrict__ F = mf_pick(st.items, r);
    for (int t = blockIdx.x; t < nitems; t += gridDim.x) {
        const int2 it = F[t];
        if (it.y == 0 && threadIdx.x < S) st.dl[int64_t(it.x) * S + threadIdx.x] = 0.0;
    }
}

// Apply the round to every touched vertex; those left with pending multiplicity
// append their work items to the frontier of the next round.
__global__ void __launch_bounds__(MF_NT) k_mf_update(MfGraph g, MfState st) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int r = st.cnt[MF_C_FROUND];
    const int nT = st.cnt[MF_C_TOUCHED];
    int2* __restrict__ next = mf_pick(st.items, r + 1);
    int* ncnt = &st.cnt[MF_C_ITEMS + ((r + 1) & 1)];
    __shared__ int s_base, s_nch;
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
        if (!__syncthreads_or(act)) continue;
        if (s == 0) {
            s_nch = mf_chunks(g, v);
            s_base = atomicAdd(ncnt, s_nch);
        }
        __syncthreads();
        for (int c = s; c < s_nch; c += blockDim.x) next[s_base + c] = make_int2(v, c);
        __syncthreads();
    }
}

// End of a forward round (one thread): stop when the next frontier is empty (or,
// as a guard, after |V| + 2 rounds, flagged); otherwise advance the round index
// and empty the lists the next round fills.  In the graph driver the result is
// the condition of the WHILE node; the host driver reads MF_C_GO.
__global__ void k_mf_fwd_check(MfState st, int64_t n, int* flags, int in_graph, cudaGraphConditionalHandle loop) {
    const int r = st.cnt[MF_C_FROUND];
    const int nnext = st.cnt[MF_C_ITEMS + ((r + 1) & 1)];
    unsigned go = 0;
    if (nnext > 0) {
        if (int64_t(r) + 1 > n + 1) {
            atomicOr(flags, STC_FLAG_NEG_CYCLE);
        } else {
            st.cnt[MF_C_FROUND] = r + 1;
            st.cnt[MF_C_ITEMS + (r & 1)] = 0;
            st.cnt[MF_C_TOUCHED] = 0;
            go = 1;
        }
    }
    st.cnt[MF_C_GO] = int(go);
    if (in_graph) cudaGraphSetConditional(loop, go);
}

// ------------------------------------------------------------------- backward

// c[v][s] = number of out-edges v -> x on a shortest path from s (into st.dn);
// vertices with a reachable source and no successor are ready.
__global__ void __launch_bounds__(MF_NT) k_mf_succ(MfGraph g, MfState st) {
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
        if (__syncthreads_or(rd) && s == 0) st.list[0][atomicAdd(&st.cnt[MF_C_READY], 1)] = int32_t(v);
    }
}

// One backward round over the ready vertices (in-edge CSR gt: row w lists v -> w).
// Round r reads ready list r & 1 and fills the other one.
__global__ void __launch_bounds__(MF_NT) k_mf_back(MfGraph gt, MfState st) {
    const int S = st.S;
    const int s = threadIdx.x;
    const int r = st.cnt[MF_C_BROUND];
    const int cur_l = r & 1;
    const int nR = st.cnt[MF_C_READY + cur_l];
    const int32_t* __restrict__ ready = mf_pick(st.list, cur_l);
    int32_t* __restrict__ next = mf_pick(st.list, cur_l ^ 1);
    int* nnext = &st.cnt[MF_C_READY + (cur_l ^ 1)];
    const int stamp = r + (1 << 30);  // disjoint from the forward rounds' stamps
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
        for (int64_t p0 = lo; p0 < hi; p0 += MF_UNR) {
            int32_t v[MF_UNR];
            int len[MF_UNR], dv[MF_UNR];
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) {
                const int64_t p = p0 + k;
                v[k] = -1;
                if (p < hi) {
                    const int32_t x = gt.col[p];
                    if ((uint64_t)x < (uint64_t)gt.n) v[k] = x;
                    len[k] = edge_len(gt, p);
                }
            }
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) dv[k] = v[k] >= 0 ? st.d[int64_t(v[k]) * S + s] : 0;
#pragma unroll
            for (int k = 0; k < MF_UNR; ++k) {
                if (v[k] >= 0 && dv[k] + len[k] == dw) {
                    const int64_t iv = int64_t(v[k]) * S + s;
                    atomicAdd(&st.dl[iv], st.sig[iv] * coef);
                    // the source whose count reaches zero lists v (once per round)
                    if (atomicSub(&st.dn[iv], 1) == 1 && atomicExch(&st.stamp[v[k]], stamp) != stamp)
                        next[atomicAdd(nnext, 1)] = v[k];
                }
            }
        }
    }
}

// k_mf_back by warp units: a warp per (ready vertex, group of 32 sources).
__global__ void __launch_bounds__(MF_NT) k_mf_back_w(MfGraph gt, MfState st) {
    const int S = st.S;
    const int lane = threadIdx.x & 31;
    const int ng = mf_groups(S);
    const int r = st.cnt[MF_C_BROUND];
    const int cur_l = r & 1;
    const int nR = st.cnt[MF_C_READY + cur_l];
    const int32_t* __restrict__ ready = mf_pick(st.list, cur_l);
    int32_t* __restrict__ next = mf_pick(st.list, cur_l ^ 1);
    int* nnext = &st.cnt[MF_C_READY + (cur_l ^ 1)];
    const int stamp = r + (1 << 30);  // disjoint from the forward rounds' stamps
    const int units = nR * ng;
    const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
    for (int q = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); q < units; q += nwarps) {
        const int32_t w = ready[q / ng];
        const int s = (q % ng) * 32 + lane;
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
        if (!__any_sync(0xffffffffu, go)) continue;
        int64_t lo, hi;
        row_range(gt.ptr, w, gt.nnz, lo, hi);
        for (int64_t c0 = lo; c0 < hi; c0 += 32) {
            int32_t vl;
            int ll;
            mf_edge_chunk(gt, c0, hi, lane, vl, ll);
            const int nc = int(hi - c0 < 32 ? hi - c0 : 32);
            for (int k0 = 0; k0 < nc; k0 += MF_UNR) {
                int32_t v[MF_UNR];
                int len[MF_UNR], dv[MF_UNR];
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) {
                    v[k] = __shfl_sync(0xffffffffu, vl, (k0 + k) & 31);
                    len[k] = __shfl_sync(0xffffffffu, ll, (k0 + k) & 31);
                    if (k0 + k >= nc) v[k] = -1;
                }
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) dv[k] = (go && v[k] >= 0) ? st.d[int64_t(v[k]) * S + s] : 0;
#pragma unroll
                for (int k = 0; k < MF_UNR; ++k) {
                    if (go && v[k] >= 0 && dv[k] + len[k] == dw) {
                        const int64_t iv = int64_t(v[k]) * S + s;
                        atomicAdd(&st.dl[iv], st.sig[iv] * coef);
                        // the source whose count reaches zero lists v (once per round)
                        if (atomicSub(&st.dn[iv], 1) == 1 && atomicExch(&st.stamp[v[k]], stamp) != stamp)
                            next[atomicAdd(nnext, 1)] = v[k];
                    }
                }
            }
        }
    }
}

// End of a backward round (one thread), as k_mf_fwd_check.  Every vertex becomes
// ready at most once per source, so more than |V| + 1 rounds means a fault of the
// successor counts (flagged as internal).
__global__ void k_mf_back_check(MfState st, int64_t n, int* flags, int in_graph, cudaGraphConditionalHandle loop) {
    const int r = st.cnt[MF_C_BROUND];
    const int nnext = st.cnt[MF_C_READY + ((r + 1) & 1)];
    unsigned go = 0;
    if (nnext > 0) {
        if (int64_t(r) + 1 > n + 1) {
            atomicOr(flags, STC_FLAG_INTERNAL);
        } else {
            st.cnt[MF_C_BROUND] = r + 1;
            st.cnt[MF_C_READY + (r & 1)] = 0;
            go = 1;
        }
    }
    st.cnt[MF_C_GO] = int(go);
    if (in_graph) cudaGraphSetConditional(loop, go);
}

// bc[v] += sum over sources s != v of delta_s(v).
// skip (may be null): when *skip != 0 the batch's results are discarded (the
// unit-length kernels gave up and the batch is recomputed) and nothing is added.
__global__ void __launch_bounds__(MF_NT) k_mf_bc(MfState st, int64_t n, const int32_t* __restrict__ src,
                                                 double* __restrict__ bc, const int* __restrict__ skip) {
    if (skip && *skip) return;
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

// ------------------------------------------------------------------- unit lengths: bitset frontiers
//
// With unit lengths every source's search is a breadth-first search and all of a
// batch's searches advance one level per round together, so a round is described by
// per-vertex source masks (256 bits for a batch of up to 256 sources):
//   vis[v]  sources that reached v at a level <= r,
//   fm[v]   sources for which v is on level r (the frontier),
//   nxt[v]  sources reaching v in round r (built by the round, level r + 1).
// A round takes the frontier's work items one warp each, one out-edge per lane:
// cand = fm[u] & ~vis[v] are the sources for which u -> v is a shortest-path edge;
// for each of them sigma_s(v) gathers sigma_s(u) (an fp64 atomic add of integers,
// exact below 2^53) and nxt[v] collects them.  The edge costs a 32-byte mask read
// whatever the number of sources; only shortest-path (edge, source) pairs cost a
// multiplicity update.  The update step turns nxt into distances, multiplicities,
// the next frontier and its work items.  Every round's items are kept: round l's items
// are the vertices at level l for some source.
//
// Backward, level by level from the deepest: for a vertex v at level l of source s,
// delta_s(v) = sigma_s(v) * sum over out-edges v -> w with d_s(w) = l + 1 of
// (1 + delta_s(w)) / sigma_s(w).  Warp per work item of level l, eight sources per
// lane, pulling the successors' coefficients (no successor counts) where a byte
// table of BFS levels, written by the forward, says d_s(w) = l + 1; items of one
// vertex add their partial sums atomically, then each vertex's sum becomes delta
// and its coefficient.

constexpr int MU_W = 8;                  // mask words per vertex (MF_NT = 256 sources)
constexpr int MU_MAX_ROUNDS = 254;       // levels recorded (one byte each, 255 = unreached); deeper
                                         // searches use the general kernels
constexpr int MU_LS = MF_NT;             // bytes per vertex of the level table
enum : int {
    MU_C_ITEMS = 0,   // items appended by the current round's update
    MU_C_ROUND = 1,   // forward round / backward level
    MU_C_GO = 2,      // 1 while the last checked loop goes on
    MU_C_FAIL = 3,    // item buffer or round table exhausted: rerun with the general kernels
    MU_C_LAST = 4,    // deepest level reached
    MU_C_NUM = 8,
};

struct MuState {
    uint32_t* vis;
    uint32_t* nxt;
    uint32_t* fm;
    uint8_t* lvl;      // [v][MU_LS] BFS level of v from each source (255: not reached)
    int2* items;       // all rounds' work items, round r at [off[r], off[r + 1])
    int64_t item_cap;
    int* off;          // MU_MAX_ROUNDS + 2 offsets
    int* cnt;          // MU_C_* counters
};

__device__ __forceinline__ void mu_load_mask(const uint32_t* __restrict__ m, int32_t v, uint32_t (&x)[MU_W]) {
    const uint4* p = reinterpret_cast<const uint4*>(m + int64_t(v) * MU_W);
    const uint4 a = p[0], b = p[1];
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}

// Sources: level 0, one path; their vertices form round 0's items.
__global__ void k_mu_seed(MfGraph g, MfState st, MuState u, const int32_t* __restrict__ src) {
    const int s = threadIdx.x;
    if (s < st.S) {
        const int32_t v = src[s];
        const int64_t i = int64_t(v) * st.S + s;
        st.d[i] = 0;
        st.sig[i] = 1.0;
        u.lvl[int64_t(v) * MU_LS + s] = 0;
        atomicOr(&u.vis[int64_t(v) * MU_W + (s >> 5)], 1u << (s & 31));
        atomicOr(&u.fm[int64_t(v) * MU_W + (s >> 5)], 1u << (s & 31));
        if (atomicExch(&st.stamp[v], -2) != -2) {
            const int nch = mf_chunks(g, v);
            const int base = atomicAdd(&u.cnt[MU_C_ITEMS], nch);
            for (int c = 0; c < nch; ++c) u.items[base + c] = make_int2(v, c);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u.off[0] = 0;
        u.off[1] = u.cnt[MU_C_ITEMS];
        u.cnt[MU_C_ITEMS] = 0;
        u.cnt[MU_C_ROUND] = 0;
    }
}

constexpr int MU_PUSH_UNR = 4;

// One round: warp per item of the frontier, lane per out-edge.
__global__ void __launch_bounds__(256) k_mu_push(MfGraph g, MfState st, MuState u) {
    const int S = st.S;
    const int lane = threadIdx.x & 31;
    const int r = u.cnt[MU_C_ROUND];
    const int i0 = u.off[r], i1 = u.off[r + 1];
    const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
    for (int t = i0 + int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); t < i1; t += nwarps) {
        const int2 it = u.items[t];
        const int32_t x = it.x;
        int64_t e0, e1;
        mf_item_edges(g, it, e0, e1);
        uint32_t F[MU_W];
        mu_load_mask(u.fm, x, F);
        const double* __restrict__ sx = st.sig + int64_t(x) * S;
        // MU_PUSH_UNR of a lane's edges at a time: their targets' masks are loaded
        // together before any is used
        for (int64_t p0 = e0 + lane; p0 < e1; p0 += 32 * MU_PUSH_UNR) {
            int32_t v[MU_PUSH_UNR];
            uint32_t V[MU_PUSH_UNR][MU_W];
#pragma unroll
            for (int j = 0; j < MU_PUSH_UNR; ++j) {
                const int64_t p = p0 + 32 * j;
                v[j] = -1;
                if (p < e1) {
                    const int32_t y = g.col[p];
                    if ((uint64_t)y < (uint64_t)g.n) v[j] = y;
                }
            }
#pragma unroll
            for (int j = 0; j < MU_PUSH_UNR; ++j)
                if (v[j] >= 0) mu_load_mask(u.vis, v[j], V[j]);
#pragma unroll
            for (int j = 0; j < MU_PUSH_UNR; ++j) {
                if (v[j] < 0) continue;
                bool any = false;
#pragma unroll
                for (int k = 0; k < MU_W; ++k) {
                    uint32_t c = F[k] & ~V[j][k];
                    if (!c) continue;
                    any = true;
                    atomicOr(&u.nxt[int64_t(v[j]) * MU_W + k], c);
                    while (c) {
                        const int s = k * 32 + __ffs(c) - 1;
                        c &= c - 1;
                        atomicAdd(&st.dln[int64_t(v[j]) * S + s], sx[s]);
                    }
                }
                if (any) mf_touch(st.stamp, st.list[1], &st.cnt[MF_C_TOUCHED], v[j], r);
            }
        }
    }
}

// End of a round's pushes: every touched vertex turns its new sources into distance
// r + 1 and multiplicity, becomes part of the next frontier and appends its items.
__global__ void __launch_bounds__(256) k_mu_update(MfGraph g, MfState st, MuState u) {
    const int S = st.S;
    const int lane = threadIdx.x & 31;
    const int r = u.cnt[MU_C_ROUND];
    const int nT = st.cnt[MF_C_TOUCHED];
    const int base_next = u.off[r + 1];
    const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
    for (int t = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); t < nT; t += nwarps) {
        const int32_t v = st.list[1][t];
        uint32_t N[MU_W];
        mu_load_mask(u.nxt, v, N);
        __syncwarp();
        bool any = false;
#pragma unroll
        for (int k = 0; k < MU_W; ++k) {
            if (!N[k]) continue;
            any = true;
            const int s = k * 32 + lane;
            if ((N[k] >> lane) & 1u) {
                const int64_t i = int64_t(v) * S + s;
                u.lvl[int64_t(v) * MU_LS + s] = uint8_t(r + 1);
                st.d[i] = r + 1;
                st.sig[i] = st.dln[i];
                st.dln[i] = 0.0;
            }
        }
        if (lane < MU_W) {
            const int64_t q = int64_t(v) * MU_W + lane;
            u.fm[q] = N[lane];
            u.vis[q] |= N[lane];
            u.nxt[q] = 0u;
        }
        if (any && lane == 0) {
            const int nch = mf_chunks(g, v);
            const int b = atomicAdd(&u.cnt[MU_C_ITEMS], nch);
            if (int64_t(base_next) + b + nch <= u.item_cap) {
                for (int c = 0; c < nch; ++c) u.items[base_next + b + c] = make_int2(v, c);
            } else {
                u.cnt[MU_C_FAIL] = 1;
            }
        }
    }
}

// End of a forward round (one thread).
__global__ void k_mu_fwd_check(MfState st, MuState u, int in_graph, cudaGraphConditionalHandle loop) {
    const int r = u.cnt[MU_C_ROUND];
    const int n_next = u.cnt[MU_C_ITEMS];
    unsigned go = 0;
    if (n_next > 0 && !u.cnt[MU_C_FAIL]) {
        if (r + 2 > MU_MAX_ROUNDS || int64_t(u.off[r + 1]) + n_next > u.item_cap) {
            u.cnt[MU_C_FAIL] = 1;
        } else {
            u.off[r + 2] = u.off[r + 1] + n_next;
            u.cnt[MU_C_ROUND] = r + 1;
            go = 1;
        }
    }
    if (!go) u.cnt[MU_C_LAST] = r;  // levels 0 .. r hold items
    u.cnt[MU_C_ITEMS] = 0;
    st.cnt[MF_C_TOUCHED] = 0;
    u.cnt[MU_C_GO] = int(go);
    st.cnt[MF_C_GO] = int(go);
    if (in_graph) cudaGraphSetConditional(loop, go);
}

// Backward start: from the deepest level.
__global__ void k_mu_back_init(MuState u) {
    if (threadIdx.x == 0 && blockIdx.x == 0) u.cnt[MU_C_ROUND] = u.cnt[MU_C_FAIL] ? -1 : u.cnt[MU_C_LAST];
}

// Backward: a warp per work item, eight sources per lane (sources 8j .. 8j + 7 on
// lane j), the level table read eight bytes a lane: one coalesced 256-byte read per
// out-edge covers every source, and the byte compares pick the sources for which
// the edge lies on a shortest path.
constexpr int MU_PULL_UNR = 4;  // out-edges whose successors' levels are in flight together

// Bit j set where byte j of v equals x (x < 256).
__device__ __forceinline__ unsigned mu_byte_eq8(uint2 v, unsigned x) {
    const unsigned rep = x * 0x01010101u;
    const unsigned a = __vcmpeq4(v.x, rep), b = __vcmpeq4(v.y, rep);
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) m |= ((a >> (8 * j + 7)) & 1u) << j | ((b >> (8 * j + 7)) & 1u) << (j + 4);
    return m;
}

__device__ __forceinline__ uint2 mu_levels8(const MuState& u, int32_t v, int s0) {
    return *reinterpret_cast<const uint2*>(u.lvl + int64_t(v) * MU_LS + s0);
}

// Partial sums of level l's items: acc (st.dl) += sum over the item's out-edges
// v -> w with d_s(w) = l + 1 of coef_s(w) (st.dln of level l + 1).  The warp reads 32
// of the item's columns at once and shares them by shuffles.
__global__ void __launch_bounds__(256) k_mu_pull(MfGraph g, MfState st, MuState u) {
    const int S = st.S;
    const int lane = threadIdx.x & 31;
    const int l = u.cnt[MU_C_ROUND];
    if (l < 0) return;
    const int s0 = lane * 8;
    const unsigned valid = S - s0 >= 8 ? 0xffu : (S > s0 ? (1u << (S - s0)) - 1u : 0u);
    const int i0 = u.off[l], i1 = u.off[l + 1];
    const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
    for (int t = i0 + int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); t < i1; t += nwarps) {
        const int2 it = u.items[t];
        const int32_t v = it.x;
        const unsigned act = valid ? mu_byte_eq8(mu_levels8(u, v, s0), unsigned(l)) & valid : 0u;
        if (!__any_sync(0xffffffffu, act != 0u)) continue;
        int64_t e0, e1;
        mf_item_edges(g, it, e0, e1);
        double acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = 0.0;
        for (int64_t c0 = e0; c0 < e1; c0 += 32) {
            const int nc = int(e1 - c0 < 32 ? e1 - c0 : 32);
            int32_t wl = -1;
            if (lane < nc) {
                const int32_t y = g.col[c0 + lane];
                if ((uint64_t)y < (uint64_t)g.n) wl = y;
            }
            for (int k0 = 0; k0 < nc; k0 += MU_PULL_UNR) {
                int32_t w[MU_PULL_UNR];
                uint2 lw[MU_PULL_UNR];
#pragma unroll
                for (int k = 0; k < MU_PULL_UNR; ++k) {
                    w[k] = __shfl_sync(0xffffffffu, wl, (k0 + k) & 31);
                    if (k0 + k >= nc) w[k] = -1;
                }
#pragma unroll
                for (int k = 0; k < MU_PULL_UNR; ++k)
                    lw[k] = (act && w[k] >= 0) ? mu_levels8(u, w[k], s0) : make_uint2(~0u, ~0u);
#pragma unroll
                for (int k = 0; k < MU_PULL_UNR; ++k) {
                    const unsigned m = mu_byte_eq8(lw[k], unsigned(l + 1)) & act;
                    if (m) {
                        const double* cw = st.dln + int64_t(w[k]) * S + s0;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if ((m >> j) & 1u) acc[j] += cw[j];
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (((act >> j) & 1u) && acc[j] != 0.0) atomicAdd(&st.dl[int64_t(v) * S + s0 + j], acc[j]);
    }
}

// Level l's sums become delta_s(v) = sigma_s(v) * sum and coef_s(v) = (1 + delta) /
// sigma (a warp per vertex: its chunk-0 item); then the next level up.
__global__ void __launch_bounds__(256) k_mu_final(MfState st, MuState u) {
    const int S = st.S;
    const int lane = threadIdx.x & 31;
    const int l = u.cnt[MU_C_ROUND];
    if (l < 0) return;
    const int s0 = lane * 8;
    const unsigned valid = S - s0 >= 8 ? 0xffu : (S > s0 ? (1u << (S - s0)) - 1u : 0u);
    const int i0 = u.off[l], i1 = u.off[l + 1];
    const int nwarps = int((int64_t(gridDim.x) * blockDim.x) >> 5);
    for (int t = i0 + int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); t < i1; t += nwarps) {
        const int2 it = u.items[t];
        if (it.y != 0 || !valid) continue;
        const unsigned m = mu_byte_eq8(mu_levels8(u, it.x, s0), unsigned(l)) & valid;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if ((m >> j) & 1u) {
                const int64_t i = int64_t(it.x) * S + s0 + j;
                const double sg = st.sig[i];
                const double dlt = sg * st.dl[i];
                st.dl[i] = dlt;
                st.dln[i] = (1.0 + dlt) / sg;
            }
        }
    }
}

__global__ void k_mu_back_check(MfState st, MuState u, int in_graph, cudaGraphConditionalHandle loop) {
    const int l = u.cnt[MU_C_ROUND];
    const unsigned go = l > 0 ? 1u : 0u;
    u.cnt[MU_C_ROUND] = l - 1;
    st.cnt[MF_C_GO] = int(go);
    if (in_graph) cudaGraphSetConditional(loop, go);
}

unsigned grid_for(stc_handle* h, int64_t work, int per_sm) {
    int64_t cap = int64_t(h->num_sms) * per_sm;
    if (work < 1) work = 1;
    return unsigned(work < cap ? work : cap);
}

// One batch: sources on the device (S = st.S of them); bc == null runs the
// forward phase only.
struct MfBatch {
    MfGraph g, gt;
    MfState st;
    const int32_t* src;
    double* bc;
};

unsigned mf_round_grid(stc_handle* h) { return unsigned(h->num_sms * MF_BLOCKS_PER_SM); }
unsigned mf_init_grid(stc_handle* h, const MfBatch& b) { return grid_for(h, b.g.n * b.st.S / 256 + 1, 16); }

// Host driver: each round's kernels, then MF_C_GO read back (one synchronisation
// per round).
stc_status mf_run_host(stc_handle* h, const MfBatch& b, stc_stream s) {
    const MfGraph& g = b.g;
    const MfState& st = b.st;
    const unsigned rg = mf_round_grid(h);
    const cudaGraphConditionalHandle none = 0;
    int* go = reinterpret_cast<int*>(&h->h_stage[4]);
    k_mf_init<<<mf_init_grid(h, b), 256, 0, s>>>(g, st);
    k_mf_seed<<<1, MF_NT, 0, s>>>(g, st, b.src);
    STC_LAUNCH_CHECK();
    stc_count(h, 2);
    for (;;) {
        if (g.w && st.S <= MF_WARP_UNITS_MAX) {
            k_mf_relax_min_w<<<rg, MF_NT, 0, s>>>(g, st);
            k_mf_relax_add_w<<<rg, MF_NT, 0, s>>>(g, st);
        } else if (g.w) {
            k_mf_relax_min<<<rg, MF_NT, 0, s>>>(g, st);
            k_mf_relax_add<<<rg, MF_NT, 0, s>>>(g, st);
        } else {
            k_mf_relax_unit<<<rg, MF_NT, 0, s>>>(g, st);
        }
        k_mf_clear_frontier<<<rg, MF_NT, 0, s>>>(st);
        k_mf_update<<<rg, MF_NT, 0, s>>>(g, st);
        k_mf_fwd_check<<<1, 1, 0, s>>>(st, g.n, h->d_flags, 0, none);
        STC_LAUNCH_CHECK();
        stc_count(h, g.w ? 5 : 4);
        STC_CUDA_TRY(cudaMemcpyAsync(go, &st.cnt[MF_C_GO], sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        if (!*go) break;
    }
    if (!b.bc) return STC_OK;
    k_mf_succ<<<grid_for(h, g.n, 32), MF_NT, 0, s>>>(g, st);
    STC_LAUNCH_CHECK();
    stc_count(h);
    for (;;) {
        if (st.S <= MF_WARP_UNITS_MAX)
            k_mf_back_w<<<rg, MF_NT, 0, s>>>(b.gt, st);
        else
            k_mf_back<<<rg, MF_NT, 0, s>>>(b.gt, st);
        k_mf_back_check<<<1, 1, 0, s>>>(st, g.n, h->d_flags, 0, none);
        STC_LAUNCH_CHECK();
        stc_count(h, 2);
        STC_CUDA_TRY(cudaMemcpyAsync(go, &st.cnt[MF_C_GO], sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        if (!*go) break;
    }
    k_mf_bc<<<grid_for(h, g.n, 32), MF_NT, 0, s>>>(st, g.n, b.src, b.bc, nullptr);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

// Graph driver: one CUDA graph per batch shape,
//   init -> seed -> WHILE{relax_min -> relax_add (unit lengths: relax_unit) -> clear -> update -> check}
//        [-> successors -> WHILE{back -> check} -> bc],
// each WHILE condition set on the device by its check kernel, so a batch is one
// graph launch with no host round trip.  Kernel arguments (state pointers, S) are
// fixed at build time; the batch's sources are copied into `src` before a launch.
struct MfGraphExec {
    cudaStream_t stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int S = -1;
    int nodes = 0;
    explicit MfGraphExec(stc_stream s) : stream(static_cast<cudaStream_t>(s)) {}
    void reset() {
        if (exec) {
            (void)cudaStreamSynchronize(stream);  // no launch of it left in flight
            cudaGraphExecDestroy(exec);
        }
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        S = -1;
        nodes = 0;
    }
    ~MfGraphExec() { reset(); }
};

cudaError_t mf_add_kernel(cudaGraph_t gr, cudaGraphNode_t* node, const cudaGraphNode_t* dep, const void* func,
                          unsigned grid, unsigned block, void** args) {
    cudaKernelNodeParams p = {};
    p.func = const_cast<void*>(func);
    p.gridDim = dim3(grid);
    p.blockDim = dim3(block);
    p.kernelParams = args;
    return cudaGraphAddKernelNode(node, gr, dep, dep ? 1 : 0, &p);
}

cudaError_t mf_add_while(cudaGraph_t top, cudaGraphNode_t* node, const cudaGraphNode_t* dep,
                         cudaGraphConditionalHandle* cond, cudaGraph_t* body) {
    cudaError_t e = cudaGraphConditionalHandleCreate(cond, top, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = *cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(node, top, dep, nullptr, dep ? 1 : 0, &cp);
    if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
    return e;
}

#define MF_G(call)                                  \
    do {                                            \
        const cudaError_t e_ = (call);              \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

cudaError_t mf_build_graph(stc_handle* h, MfBatch b, MfGraphExec& x) {
    x.reset();
    MF_G(cudaGraphCreate(&x.graph, 0));
    const unsigned rg = mf_round_grid(h);
    int* flags = h->d_flags;
    int in_graph = 1;
    int64_t n = b.g.n;
    cudaGraphNode_t n_init, n_seed, n_fw;
    void* a_init[] = {&b.g, &b.st};
    MF_G(mf_add_kernel(x.graph, &n_init, nullptr, (const void*)k_mf_init, mf_init_grid(h, b), 256, a_init));
    void* a_seed[] = {&b.g, &b.st, &b.src};
    MF_G(mf_add_kernel(x.graph, &n_seed, &n_init, (const void*)k_mf_seed, 1, MF_NT, a_seed));
    cudaGraphConditionalHandle hf;
    cudaGraph_t fb;
    MF_G(mf_add_while(x.graph, &n_fw, &n_seed, &hf, &fb));
    {
        cudaGraphNode_t k1, k2, k3, k4, k5;
        void* a_gs[] = {&b.g, &b.st};
        void* a_st[] = {&b.st};
        void* a_chk[] = {&b.st, &n, &flags, &in_graph, &hf};
        const bool wu = b.st.S <= MF_WARP_UNITS_MAX;
        const void* relax_min = wu ? (const void*)k_mf_relax_min_w : (const void*)k_mf_relax_min;
        const void* relax_add = wu ? (const void*)k_mf_relax_add_w : (const void*)k_mf_relax_add;
        MF_G(mf_add_kernel(fb, &k1, nullptr, b.g.w ? relax_min : (const void*)k_mf_relax_unit, rg, MF_NT, a_gs));
        k2 = k1;
        if (b.g.w) MF_G(mf_add_kernel(fb, &k2, &k1, relax_add, rg, MF_NT, a_gs));
        MF_G(mf_add_kernel(fb, &k3, &k2, (const void*)k_mf_clear_frontier, rg, MF_NT, a_st));
        MF_G(mf_add_kernel(fb, &k4, &k3, (const void*)k_mf_update, rg, MF_NT, a_gs));
        MF_G(mf_add_kernel(fb, &k5, &k4, (const void*)k_mf_fwd_check, 1, 1, a_chk));
    }
    x.nodes = b.g.w ? 7 : 6;
    if (b.bc) {
        cudaGraphNode_t n_succ, n_bw, n_bc;
        void* a_succ[] = {&b.g, &b.st};
        MF_G(mf_add_kernel(x.graph, &n_succ, &n_fw, (const void*)k_mf_succ, grid_for(h, n, 32), MF_NT, a_succ));
        cudaGraphConditionalHandle hb;
        cudaGraph_t bb;
        MF_G(mf_add_while(x.graph, &n_bw, &n_succ, &hb, &bb));
        cudaGraphNode_t k1, k2;
        void* a_back[] = {&b.gt, &b.st};
        void* a_chk[] = {&b.st, &n, &flags, &in_graph, &hb};
        const void* back = b.st.S <= MF_WARP_UNITS_MAX ? (const void*)k_mf_back_w : (const void*)k_mf_back;
        MF_G(mf_add_kernel(bb, &k1, nullptr, back, rg, MF_NT, a_back));
        MF_G(mf_add_kernel(bb, &k2, &k1, (const void*)k_mf_back_check, 1, 1, a_chk));
        const int* no_skip = nullptr;
        void* a_bc[] = {&b.st, &n, &b.src, &b.bc, &no_skip};
        MF_G(mf_add_kernel(x.graph, &n_bc, &n_bw, (const void*)k_mf_bc, grid_for(h, n, 32), MF_NT, a_bc));
        x.nodes += 4;
    }
    MF_G(cudaGraphInstantiate(&x.exec, x.graph, 0));
    x.S = b.st.S;
    return cudaSuccess;
}

#undef MF_G

// Run one batch with the handle's driver (graphs are rebuilt when S changes).
stc_status mf_run(stc_handle* h, const MfBatch& b, MfGraphExec& x, stc_stream s) {
    if (h->round_driver == 0) return mf_run_host(h, b, s);
    if (x.S != b.st.S) {
        const cudaError_t e = mf_build_graph(h, b, x);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            x.reset();
            return STC_ERR_CUDA;
        }
    }
    STC_CUDA_TRY(cudaGraphLaunch(x.exec, s));
    stc_count(h, x.nodes);  // each node once (the device repeats the loop bodies)
    return STC_OK;
}

// ------------------------------------------------------------------- unit-length drivers

stc_status mu_alloc(StcScratch& sc, const MfGraph& g, MuState& u) {
    const size_t n = size_t(g.n);
    u.vis = sc.get<uint32_t>(n * MU_W);
    u.nxt = sc.get<uint32_t>(n * MU_W);
    u.fm = sc.get<uint32_t>(n * MU_W);
    u.lvl = sc.get<uint8_t>(n * MU_LS);
    // every vertex on a few levels: eight times one round's worth of items
    u.item_cap = 8 * (int64_t(g.n) + g.nnz / MF_ITEM_EDGES + 1) + 1024;
    if (u.item_cap > int64_t(INT32_MAX)) u.item_cap = INT32_MAX;
    u.items = sc.get<int2>(size_t(u.item_cap));
    u.off = sc.get<int>(size_t(MU_MAX_ROUNDS) + 2);
    u.cnt = sc.get<int>(MU_C_NUM);
    return sc.failed ? STC_ERR_OOM : STC_OK;
}

stc_status mu_clear(stc_handle* h, const MfBatch& b, const MuState& u, stc_stream s) {
    const size_t n = size_t(b.g.n);
    STC_CUDA_TRY(cudaMemsetAsync(u.vis, 0, n * MU_W * 4, s));
    STC_CUDA_TRY(cudaMemsetAsync(u.nxt, 0, n * MU_W * 4, s));
    STC_CUDA_TRY(cudaMemsetAsync(u.fm, 0, n * MU_W * 4, s));
    STC_CUDA_TRY(cudaMemsetAsync(u.lvl, 0xff, n * MU_LS, s));
    STC_CUDA_TRY(cudaMemsetAsync(u.cnt, 0, MU_C_NUM * sizeof(int), s));
    (void)h;
    return STC_OK;
}

unsigned mu_warp_grid(stc_handle* h) { return unsigned(h->num_sms * 8); }  // 256-thread CTAs, 64 warps per SM

// Host driver of the unit-length batch: each round, then MF_C_GO read back.
stc_status mu_run_host(stc_handle* h, const MfBatch& b, const MuState& u, stc_stream s) {
    const MfGraph& g = b.g;
    const MfState& st = b.st;
    const unsigned wg = mu_warp_grid(h);
    const cudaGraphConditionalHandle none = 0;
    int* go = reinterpret_cast<int*>(&h->h_stage[4]);
    stc_status e;
    if ((e = mu_clear(h, b, u, s)) != STC_OK) return e;
    k_mf_init<<<mf_init_grid(h, b), 256, 0, s>>>(g, st);
    k_mu_seed<<<1, MF_NT, 0, s>>>(g, st, u, b.src);
    STC_LAUNCH_CHECK();
    stc_count(h, 2);
    for (;;) {
        k_mu_push<<<wg, 256, 0, s>>>(g, st, u);
        k_mu_update<<<wg, 256, 0, s>>>(g, st, u);
        k_mu_fwd_check<<<1, 1, 0, s>>>(st, u, 0, none);
        STC_LAUNCH_CHECK();
        stc_count(h, 3);
        STC_CUDA_TRY(cudaMemcpyAsync(go, &u.cnt[MU_C_GO], sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        if (!*go) break;
    }
    if (!b.bc) return STC_OK;
    k_mu_back_init<<<1, 1, 0, s>>>(u);
    STC_LAUNCH_CHECK();
    stc_count(h);
    for (;;) {
        k_mu_pull<<<wg, 256, 0, s>>>(g, st, u);
        k_mu_final<<<wg, 256, 0, s>>>(st, u);
        k_mu_back_check<<<1, 1, 0, s>>>(st, u, 0, none);
        STC_LAUNCH_CHECK();
        stc_count(h, 3);
        STC_CUDA_TRY(cudaMemcpyAsync(go, &st.cnt[MF_C_GO], sizeof(int), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        if (!*go) break;
    }
    k_mf_bc<<<grid_for(h, g.n, 32), MF_NT, 0, s>>>(st, g.n, b.src, b.bc, &u.cnt[MU_C_FAIL]);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

#define MF_G(call)                                  \
    do {                                            \
        const cudaError_t e_ = (call);              \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

// Graph driver of the unit-length batch:
//   seed -> WHILE{push -> update -> check} [-> back_init -> WHILE{pull -> final -> check} -> bc]
// (the clears and k_mf_init run on the stream before each launch).
cudaError_t mu_build_graph(stc_handle* h, MfBatch b, MuState u, MfGraphExec& x) {
    x.reset();
    MF_G(cudaGraphCreate(&x.graph, 0));
    const unsigned wg = mu_warp_grid(h);
    int in_graph = 1;
    int64_t n = b.g.n;
    cudaGraphNode_t n_seed, n_fw;
    void* a_seed[] = {&b.g, &b.st, &u, &b.src};
    MF_G(mf_add_kernel(x.graph, &n_seed, nullptr, (const void*)k_mu_seed, 1, MF_NT, a_seed));
    cudaGraphConditionalHandle hf;
    cudaGraph_t fb;
    MF_G(mf_add_while(x.graph, &n_fw, &n_seed, &hf, &fb));
    {
        cudaGraphNode_t k1, k2, k3;
        void* a_gsu[] = {&b.g, &b.st, &u};
        void* a_chk[] = {&b.st, &u, &in_graph, &hf};
        MF_G(mf_add_kernel(fb, &k1, nullptr, (const void*)k_mu_push, wg, 256, a_gsu));
        MF_G(mf_add_kernel(fb, &k2, &k1, (const void*)k_mu_update, wg, 256, a_gsu));
        MF_G(mf_add_kernel(fb, &k3, &k2, (const void*)k_mu_fwd_check, 1, 1, a_chk));
    }
    x.nodes = 4;
    if (b.bc) {
        cudaGraphNode_t n_bi, n_bw, n_bc;
        void* a_u[] = {&u};
        MF_G(mf_add_kernel(x.graph, &n_bi, &n_fw, (const void*)k_mu_back_init, 1, 1, a_u));
        cudaGraphConditionalHandle hb;
        cudaGraph_t bb;
        MF_G(mf_add_while(x.graph, &n_bw, &n_bi, &hb, &bb));
        cudaGraphNode_t k1, k2, k3;
        void* a_pull[] = {&b.g, &b.st, &u};
        void* a_fin[] = {&b.st, &u};
        void* a_chk[] = {&b.st, &u, &in_graph, &hb};
        MF_G(mf_add_kernel(bb, &k1, nullptr, (const void*)k_mu_pull, wg, 256, a_pull));
        MF_G(mf_add_kernel(bb, &k2, &k1, (const void*)k_mu_final, wg, 256, a_fin));
        MF_G(mf_add_kernel(bb, &k3, &k2, (const void*)k_mu_back_check, 1, 1, a_chk));
        const int* skip = &u.cnt[MU_C_FAIL];
        void* a_bc[] = {&b.st, &n, &b.src, &b.bc, &skip};
        MF_G(mf_add_kernel(x.graph, &n_bc, &n_bw, (const void*)k_mf_bc, grid_for(h, n, 32), MF_NT, a_bc));
        x.nodes += 5;
    }
    MF_G(cudaGraphInstantiate(&x.exec, x.graph, 0));
    x.S = b.st.S;
    return cudaSuccess;
}

#undef MF_G

// One unit-length batch with the handle's driver; *fallback is set when the
// bitset kernels gave up (too many rounds or items) and the batch must be run by the
// general kernels (nothing was added to bc).  Synchronises `s`.
stc_status mu_run(stc_handle* h, const MfBatch& b, const MuState& u, MfGraphExec& x, bool* fallback, stc_stream s) {
    *fallback = false;
    stc_status e;
    if (h->round_driver == 0) {
        if ((e = mu_run_host(h, b, u, s)) != STC_OK) return e;
    } else {
        if (x.S != b.st.S) {
            const cudaError_t ce = mu_build_graph(h, b, u, x);
            if (ce != cudaSuccess) {
                (void)cudaGetLastError();
                x.reset();
                return STC_ERR_CUDA;
            }
        }
        if ((e = mu_clear(h, b, u, s)) != STC_OK) return e;
        k_mf_init<<<mf_init_grid(h, b), 256, 0, s>>>(b.g, b.st);
        STC_LAUNCH_CHECK();
        stc_count(h);
        STC_CUDA_TRY(cudaGraphLaunch(x.exec, s));
        stc_count(h, x.nodes);
    }
    int* f = reinterpret_cast<int*>(&h->h_stage[3]);
    *f = 0;
    STC_CUDA_TRY(cudaMemcpyAsync(f, &u.cnt[MU_C_FAIL], sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    *fallback = *f != 0;
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

stc_status mf_alloc_state(StcScratch& sc, const MfGraph& g, int S, MfState& st) {
    // item and list indices are int
    if (g.n + g.nnz / MF_ITEM_EDGES + 2 > int64_t(INT32_MAX)) return STC_ERR_INVALID_ARG;
    const size_t n = size_t(g.n);
    const size_t ns = n * size_t(S);
    const size_t ni = n + size_t(g.nnz / MF_ITEM_EDGES) + 1;  // each vertex once per round
    st.S = S;
    st.d = sc.get<int>(ns);
    st.dn = sc.get<int>(ns);
    st.sig = sc.get<double>(ns);
    st.dl = sc.get<double>(ns);
    st.dln = sc.get<double>(ns);
    st.stamp = sc.get<int>(n);
    st.list[0] = sc.get<int32_t>(n);
    st.list[1] = sc.get<int32_t>(n);
    st.items[0] = sc.get<int2>(ni);
    st.items[1] = sc.get<int2>(ni);
    st.cnt = sc.get<int>(MF_C_NUM);
    return sc.failed ? STC_ERR_OOM : STC_OK;
}

stc_status mf_read_flags(stc_handle* h, stc_stream s) {
    STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[6], h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    const int f = reinterpret_cast<int*>(&h->h_stage[6])[0];
    if (f) {
        STC_CUDA_TRY(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));
        return stc_flags_to_status(f);
    }
    return STC_OK;
}

}  // namespace

stc_status stc_mfbc_sssp_impl(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsrc,
                              int32_t* d_out, double* sigma_out, int32_t* rounds_out, stc_stream s) {
    StcScratch sc(h, s);
    MfGraph g{G->nrows, G->nnz, G->rowptr, G->col, static_cast<const int32_t*>(G->val)};
    stc_status st = stc_validate_csr_async(h, G, s);
    if (st != STC_OK) return st;
    if ((st = mf_check(h, g, s)) != STC_OK) return st;
    MfBatch b{g, MfGraph{0, 0, nullptr, nullptr, nullptr}, MfState{}, nullptr, nullptr};
    if ((st = mf_alloc_state(sc, g, nsrc, b.st)) != STC_OK) return st;
    int32_t* d_src = sc.get<int32_t>(size_t(nsrc));
    if (!d_src) return STC_ERR_OOM;
    b.src = d_src;
    STC_CUDA_TRY(cudaMemcpyAsync(d_src, sources, sizeof(int32_t) * nsrc, cudaMemcpyHostToDevice, s));
    MfGraphExec x(s);
    bool general = g.w != nullptr;
    if (!general) {
        // unit lengths: bitset frontiers (the general kernels when they give up)
        MuState u{};
        if ((st = mu_alloc(sc, g, u)) != STC_OK) return st;
        MfGraphExec xu(s);
        if ((st = mu_run(h, b, u, xu, &general, s)) != STC_OK) return st;
        STC_CUDA_TRY(cudaMemcpyAsync(&b.st.cnt[MF_C_FROUND], &u.cnt[MU_C_LAST], sizeof(int), cudaMemcpyDeviceToDevice,
                                     s));
    }
    if (general && (st = mf_run(h, b, x, s)) != STC_OK) return st;
    STC_CUDA_TRY(cudaMemcpyAsync(d_out, b.st.d, sizeof(int) * size_t(g.n) * nsrc, cudaMemcpyDeviceToDevice, s));
    STC_CUDA_TRY(cudaMemcpyAsync(sigma_out, b.st.sig, sizeof(double) * size_t(g.n) * nsrc,
                                 cudaMemcpyDeviceToDevice, s));
    STC_CUDA_TRY(cudaMemcpyAsync(&h->h_stage[5], &b.st.cnt[MF_C_FROUND], sizeof(int), cudaMemcpyDeviceToHost, s));
    if ((st = mf_read_flags(h, s)) != STC_OK) return st;  // synchronises
    if (rounds_out) *rounds_out = reinterpret_cast<int*>(&h->h_stage[5])[0] + 1;
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

    MfBatch b{g, MfGraph{g.n, g.nnz, tptr, tcol, tw}, MfState{}, nullptr, bc};
    if ((st = mf_alloc_state(sc, g, batch, b.st)) != STC_OK) return st;
    int32_t* d_src = sc.get<int32_t>(size_t(batch));
    if (!d_src) return STC_ERR_OOM;
    b.src = d_src;
    k_mf_zero<<<grid_for(h, g.n / 256 + 1, 16), 256, 0, s>>>(bc, g.n);
    STC_LAUNCH_CHECK();
    stc_count(h);
    MfGraphExec x(s), xu(s);
    MuState u{};
    if (!g.w && (st = mu_alloc(sc, g, u)) != STC_OK) return st;
    for (int32_t b0 = 0; b0 < nsrc; b0 += batch) {
        b.st.S = nsrc - b0 < batch ? nsrc - b0 : batch;
        STC_CUDA_TRY(cudaMemcpyAsync(d_src, sources + b0, sizeof(int32_t) * b.st.S, cudaMemcpyHostToDevice, s));
        bool general = g.w != nullptr;
        if (!general && (st = mu_run(h, b, u, xu, &general, s)) != STC_OK) return st;
        if (general && (st = mf_run(h, b, x, s)) != STC_OK) return st;
    }
    return mf_read_flags(h, s);
}
