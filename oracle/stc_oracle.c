/*
 * Plain CPU oracle for generalized sparse contraction.  TEST INFRASTRUCTURE ONLY:
 * it is loaded by the tests, by the package's smoke check and by the timed CPU
 * baseline of the benchmark, never by the product path.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it computes (Solomonik & Hoefler, "Sparse Tensor Algebra as a Parallel
 * Programming Model"):
 *
 *  - Contraction C[i,j] (+)= f(A[i,k], B[k,j]) over an algebraic structure whose
 *    additive operator is (+) (Section 3.1, Table 1) and whose pairwise function
 *    f may combine operands of different types (Section 3.3.2, functions of the
 *    form (type_C) <- (type_A, type_B); the sum uses the output's additive op).
 *    Written as Gustavson's row-by-row product with a dense accumulator over the
 *    columns of one output row: for each k of row i of A in column order, for each
 *    j of row k of B in column order, the first product lands in the accumulator
 *    and later ones are combined with (+).  The output row lists the touched
 *    columns in ascending order.
 *  - The same contraction with a dense vector or a dense column block as B.
 *  - Bellman-Ford single-source shortest paths by repeated tropical
 *    matrix-vector products, P(r)_i = min_j (A_ij + P(r-1)_j) with A_ii = 0,
 *    iterated until nothing changes, failing after |V| rounds (Section 4.2).
 *  - Dijkstra (Section 4.2 names it as the sequential alternative).
 *  - Floyd-Warshall, used to pin path doubling (Section 4.2).
 *  - Betweenness centrality by Brandes' accumulation (the paper points to the
 *    geodetic semiring and to Brandes for this, Section 4.2).
 *
 * Algebra ids (the numbering is part of the public interface of the library,
 * restated here by value):
 *   0 (+,x) fp32 operands   - accumulated in fp64, result returned in fp64
 *   1 (+,x) fp64
 *   2 (min,+) int32, additive identity INT_MAX/2 (Section 3.1)
 *   3 (min,+) fp32, additive identity +inf, f = fp32 add
 *   4 (or,and) boolean, values are bytes 0/1
 *   5 (distance, multiplicity) monoid: A holds int32 edge lengths, B and C hold
 *     {int32 d; int32 pad; double sigma}.  f(a, (d,s)) = (a + d, s);
 *     (d1,s1) (+) (d2,s2) = the smaller d, or (d, s1 + s2) on a tie.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC stc_oracle.c -o libstc_oracle.so
 */
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PT_F32 0
#define ORC_PT_F64 1
#define ORC_MP_I32 2
#define ORC_MP_F32 3
#define ORC_BOOL 4
#define ORC_MULTPATH 5

#define ORC_TROP_I32_ID (INT_MAX / 2)

typedef struct {
    int32_t d;
    int32_t pad;
    double s;
} orc_dsig;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------ SpGEMM */

/* Number of distinct output columns of each selected row: |union of cols(B_k)|,
 * k over the stored columns of row i of A.  rows == NULL selects all rows. */
void orc_spgemm_count(int64_t nrows_a, int64_t ncols_b,
                      const int64_t* a_ptr, const int32_t* a_col,
                      const int64_t* b_ptr, const int32_t* b_col,
                      const int64_t* rows, int64_t nsel, int64_t* counts) {
    if (!rows) nsel = nrows_a;
#pragma omp parallel
    {
        int64_t* seen = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncols_b > 0 ? ncols_b : 1));
        for (int64_t j = 0; j < ncols_b; ++j) seen[j] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nsel; ++t) {
            int64_t i = rows ? rows[t] : t;
            int64_t cnt = 0;
            for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p) {
                int32_t k = a_col[p];
                for (int64_t q = b_ptr[k]; q < b_ptr[k + 1]; ++q) {
                    int32_t j = b_col[q];
                    if (seen[j] != t) { seen[j] = t; ++cnt; }
                }
            }
            counts[t] = cnt;
        }
        free(seen);
    }
}

/* Fill the selected rows: out_ptr[t]..out_ptr[t+1] receives row rows[t] (or t).
 * out_val element type by algebra: 0,1 -> double; 2 -> int32; 3 -> float;
 * 4 -> uint8; 5 -> orc_dsig.  out_abs (algebras 0/1 only, may be NULL) receives
 * the sum of |a||b| over the products of each entry, in fp64. */
void orc_spgemm_fill(int alg, int64_t nrows_a, int64_t ncols_b,
                     const int64_t* a_ptr, const int32_t* a_col, const void* a_val,
                     const int64_t* b_ptr, const int32_t* b_col, const void* b_val,
                     const int64_t* rows, int64_t nsel, const int64_t* out_ptr,
                     int32_t* out_col, void* out_val, double* out_abs) {
    if (!rows) nsel = nrows_a;
#pragma omp parallel
    {
        size_t nc = (size_t)(ncols_b > 0 ? ncols_b : 1);
        int64_t* seen = (int64_t*)malloc(sizeof(int64_t) * nc);
        double* acc_d = (double*)malloc(sizeof(double) * nc);
        double* acc_abs = (double*)malloc(sizeof(double) * nc);
        int32_t* acc_i = (int32_t*)malloc(sizeof(int32_t) * nc);
        float* acc_f = (float*)malloc(sizeof(float) * nc);
        for (size_t j = 0; j < nc; ++j) seen[j] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nsel; ++t) {
            int64_t i = rows ? rows[t] : t;
            int64_t o0 = out_ptr[t];
            int64_t cnt = 0;
            for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p) {
                int32_t k = a_col[p];
                for (int64_t q = b_ptr[k]; q < b_ptr[k + 1]; ++q) {
                    int32_t j = b_col[q];
                    int first = (seen[j] != t);
                    if (first) { seen[j] = t; out_col[o0 + cnt] = j; ++cnt; }
                    switch (alg) {
                    case ORC_PT_F32: {
                        double x = (double)((const float*)a_val)[p] * (double)((const float*)b_val)[q];
                        if (first) { acc_d[j] = x; acc_abs[j] = fabs(x); }
                        else { acc_d[j] += x; acc_abs[j] += fabs(x); }
                    } break;
                    case ORC_PT_F64: {
                        double x = ((const double*)a_val)[p] * ((const double*)b_val)[q];
                        if (first) { acc_d[j] = x; acc_abs[j] = fabs(x); }
                        else { acc_d[j] += x; acc_abs[j] += fabs(x); }
                    } break;
                    case ORC_MP_I32: {
                        int32_t x = ((const int32_t*)a_val)[p] + ((const int32_t*)b_val)[q];
                        if (first || x < acc_i[j]) acc_i[j] = x;
                    } break;
                    case ORC_MP_F32: {
                        float x = ((const float*)a_val)[p] + ((const float*)b_val)[q];
                        if (first || x < acc_f[j]) acc_f[j] = x;
                    } break;
                    case ORC_BOOL: {
                        int x = ((const uint8_t*)a_val)[p] && ((const uint8_t*)b_val)[q];
                        if (first) acc_i[j] = x; else acc_i[j] = acc_i[j] || x;
                    } break;
                    case ORC_MULTPATH: {
                        const orc_dsig* bv = (const orc_dsig*)b_val;
                        int32_t d = ((const int32_t*)a_val)[p] + bv[q].d;
                        double s = bv[q].s;
                        if (first || d < acc_i[j]) { acc_i[j] = d; acc_d[j] = s; }
                        else if (d == acc_i[j]) acc_d[j] += s;
                    } break;
                    default: break;
                    }
                }
            }
            qsort(out_col + o0, (size_t)cnt, sizeof(int32_t), cmp_i32);
            for (int64_t e = 0; e < cnt; ++e) {
                int32_t j = out_col[o0 + e];
                switch (alg) {
                case ORC_PT_F32:
                case ORC_PT_F64:
                    ((double*)out_val)[o0 + e] = acc_d[j];
                    if (out_abs) out_abs[o0 + e] = acc_abs[j];
                    break;
                case ORC_MP_I32: ((int32_t*)out_val)[o0 + e] = acc_i[j]; break;
                case ORC_MP_F32: ((float*)out_val)[o0 + e] = acc_f[j]; break;
                case ORC_BOOL: ((uint8_t*)out_val)[o0 + e] = (uint8_t)acc_i[j]; break;
                case ORC_MULTPATH: {
                    orc_dsig r; r.d = acc_i[j]; r.pad = 0; r.s = acc_d[j];
                    ((orc_dsig*)out_val)[o0 + e] = r;
                } break;
                default: break;
                }
            }
        }
        free(seen); free(acc_d); free(acc_abs); free(acc_i); free(acc_f);
    }
}

/* --------------------------------------------------------- SpMM and SpMV */

/* Y[i, c] (+)= f(A[i,k], X[k, c]) over the stored k of row i, c < ncol.
 * X is row-major with leading dimension ldx (elements), Y with ldy.
 * accumulate != 0 combines with the existing Y[i,c] (y is the first operand of
 * (+)); otherwise a row with no stored entry receives the additive identity.
 * Element types as in orc_spgemm_fill except: algebra 0 reads and writes fp32
 * but accumulates in fp64 before the single final rounding; algebra 4 bytes;
 * algebra 5 A is int32, X and Y are orc_dsig.  SpMV is ncol == 1. */
void orc_spmm(int alg, int64_t nrows, const int64_t* a_ptr, const int32_t* a_col,
              const void* a_val, const void* X, int64_t ldx, int32_t ncol,
              void* Y, int64_t ldy, int accumulate) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < nrows; ++i) {
        for (int32_t c = 0; c < ncol; ++c) {
            int64_t yo = i * ldy + c;
            switch (alg) {
            case ORC_PT_F32: {
                double acc = accumulate ? (double)((float*)Y)[yo] : 0.0;
                for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p)
                    acc += (double)((const float*)a_val)[p] *
                           (double)((const float*)X)[(int64_t)a_col[p] * ldx + c];
                ((float*)Y)[yo] = (float)acc;
            } break;
            case ORC_PT_F64: {
                double acc = accumulate ? ((double*)Y)[yo] : 0.0;
                for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p)
                    acc += ((const double*)a_val)[p] *
                           ((const double*)X)[(int64_t)a_col[p] * ldx + c];
                ((double*)Y)[yo] = acc;
            } break;
            case ORC_MP_I32: {
                int32_t acc = accumulate ? ((int32_t*)Y)[yo] : ORC_TROP_I32_ID;
                for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p) {
                    int32_t x = ((const int32_t*)a_val)[p] +
                                ((const int32_t*)X)[(int64_t)a_col[p] * ldx + c];
                    if (x < acc) acc = x;
                }
                ((int32_t*)Y)[yo] = acc;
            } break;
            case ORC_MP_F32: {
                float acc = accumulate ? ((float*)Y)[yo] : INFINITY;
                for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p) {
                    float x = ((const float*)a_val)[p] +
                              ((const float*)X)[(int64_t)a_col[p] * ldx + c];
                    if (x < acc) acc = x;
                }
                ((float*)Y)[yo] = acc;
            } break;
            case ORC_BOOL: {
                int acc = accumulate ? (((uint8_t*)Y)[yo] != 0) : 0;
                for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p)
                    acc = acc || (((const uint8_t*)a_val)[p] &&
                                  ((const uint8_t*)X)[(int64_t)a_col[p] * ldx + c]);
                ((uint8_t*)Y)[yo] = (uint8_t)acc;
            } break;
            case ORC_MULTPATH: {
                orc_dsig acc;
                if (accumulate) acc = ((orc_dsig*)Y)[yo];
                else { acc.d = ORC_TROP_I32_ID; acc.pad = 0; acc.s = 0.0; }
                for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p) {
                    orc_dsig x = ((const orc_dsig*)X)[(int64_t)a_col[p] * ldx + c];
                    int32_t d = ((const int32_t*)a_val)[p] + x.d;
                    if (d < acc.d) { acc.d = d; acc.s = x.s; }
                    else if (d == acc.d) acc.s += x.s;
                }
                acc.pad = 0;
                ((orc_dsig*)Y)[yo] = acc;
            } break;
            default: break;
            }
        }
    }
}

/* ---------------------------------------------------------- Bellman-Ford */

/* Graph in out-edge CSR: row u lists the edges u -> v with lengths w (the
 * transpose of the paper's A, whose A_ij is the length of edge j -> i).
 * P(0) = (0 at source, identity elsewhere); each round computes, from the
 * previous round's vector only,
 *     P(r)_v = min( P(r-1)_v, min over edges u->v of P(r-1)_u + w_uv ),
 * the first term being the A_vv = 0 diagonal.  A vertex still at the additive
 * identity relaxes nothing (identity is absorbing for the tropical product).
 * Stops when a round changes nothing.  Returns the number of rounds that
 * changed something (0 if the source has no out-edge), or -1 when round |V|
 * still changed something: a shortest path has at most |V|-1 edges, so a
 * change in round |V| means a reachable negative cycle.
 * alg: 2 -> int32 distances, 3 -> fp32 distances.  *relax_out (may be NULL)
 * receives the number of edge relaxations evaluated. */
int64_t orc_bellman_ford(int alg, int64_t n, const int64_t* ptr, const int32_t* col,
                         const void* w, int32_t source, void* dist_out, int64_t* relax_out) {
    int64_t rounds = 0, relax = 0;
    if (alg == ORC_MP_I32) {
        int32_t* P = (int32_t*)dist_out;
        int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t v = 0; v < n; ++v) P[v] = ORC_TROP_I32_ID;
        P[source] = 0;
        for (;;) {
            memcpy(Q, P, sizeof(int32_t) * (size_t)n);
            int changed = 0;
            for (int64_t u = 0; u < n; ++u) {
                if (Q[u] == ORC_TROP_I32_ID) continue;
                relax += ptr[u + 1] - ptr[u];
                for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
                    int32_t v = col[p];
                    int32_t x = Q[u] + ((const int32_t*)w)[p];
                    if (x < P[v]) { P[v] = x; changed = 1; }
                }
            }
            if (!changed) break;
            ++rounds;
            if (rounds >= n) { rounds = -1; break; }   /* round |V| still changed */
        }
        free(Q);
    } else {
        float* P = (float*)dist_out;
        float* Q = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
        for (int64_t v = 0; v < n; ++v) P[v] = INFINITY;
        P[source] = 0.0f;
        for (;;) {
            memcpy(Q, P, sizeof(float) * (size_t)n);
            int changed = 0;
            for (int64_t u = 0; u < n; ++u) {
                if (Q[u] == INFINITY) continue;
                relax += ptr[u + 1] - ptr[u];
                for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
                    int32_t v = col[p];
                    float x = Q[u] + ((const float*)w)[p];
                    if (x < P[v]) { P[v] = x; changed = 1; }
                }
            }
            if (!changed) break;
            ++rounds;
            if (rounds >= n) { rounds = -1; break; }
        }
        free(Q);
    }
    if (relax_out) *relax_out = relax;
    return rounds;
}

/* --------------------------------------------------------------- Dijkstra */

/* Binary-heap Dijkstra with lazy deletion; non-negative lengths only.
 * alg 2: int32 distances (unreached = INT_MAX/2); alg 3: fp32 (unreached = inf).
 * Distances are formed exactly as the relaxations above: d_u + w_uv in the
 * element type, so both methods produce the minimum over paths of the same sums. */
typedef struct { double key; int32_t v; } orc_hent;

static void heap_push(orc_hent* h, int64_t* sz, orc_hent e) {
    int64_t i = (*sz)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].key <= h[i].key) break;
        orc_hent t = h[p]; h[p] = h[i]; h[i] = t; i = p;
    }
}

static orc_hent heap_pop(orc_hent* h, int64_t* sz) {
    orc_hent top = h[0];
    h[0] = h[--(*sz)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *sz && h[l].key < h[m].key) m = l;
        if (r < *sz && h[r].key < h[m].key) m = r;
        if (m == i) break;
        orc_hent t = h[m]; h[m] = h[i]; h[i] = t; i = m;
    }
    return top;
}

void orc_dijkstra(int alg, int64_t n, const int64_t* ptr, const int32_t* col,
                  const void* w, int32_t source, void* dist_out) {
    int64_t nnz = ptr[n];
    orc_hent* h = (orc_hent*)malloc(sizeof(orc_hent) * (size_t)(nnz + 2));
    uint8_t* done = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t sz = 0;
    if (alg == ORC_MP_I32) {
        int32_t* d = (int32_t*)dist_out;
        for (int64_t v = 0; v < n; ++v) d[v] = ORC_TROP_I32_ID;
        d[source] = 0;
        orc_hent e0 = {0.0, source};
        heap_push(h, &sz, e0);
        while (sz) {
            orc_hent e = heap_pop(h, &sz);
            int32_t u = e.v;
            if (done[u]) continue;
            done[u] = 1;
            for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
                int32_t v = col[p];
                int32_t x = d[u] + ((const int32_t*)w)[p];
                if (x < d[v]) { d[v] = x; orc_hent ne = {(double)x, v}; heap_push(h, &sz, ne); }
            }
        }
    } else {
        float* d = (float*)dist_out;
        for (int64_t v = 0; v < n; ++v) d[v] = INFINITY;
        d[source] = 0.0f;
        orc_hent e0 = {0.0, source};
        heap_push(h, &sz, e0);
        while (sz) {
            orc_hent e = heap_pop(h, &sz);
            int32_t u = e.v;
            if (done[u]) continue;
            done[u] = 1;
            for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
                int32_t v = col[p];
                float x = d[u] + ((const float*)w)[p];
                if (x < d[v]) { d[v] = x; orc_hent ne = {(double)x, v}; heap_push(h, &sz, ne); }
            }
        }
    }
    free(h);
    free(done);
}

/* ---------------------------------------------------------- Floyd-Warshall */

/* Dense all-pairs distances, int32, in place on an n x n row-major matrix whose
 * absent edges hold INT_MAX/2 and whose diagonal holds min(0, A_ii). */
void orc_floyd_warshall_i32(int64_t n, int32_t* D) {
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i) {
            int32_t dik = D[i * n + k];
            if (dik >= ORC_TROP_I32_ID) continue;
            for (int64_t j = 0; j < n; ++j) {
                int32_t dkj = D[k * n + j];
                if (dkj >= ORC_TROP_I32_ID) continue;
                if (dik + dkj < D[i * n + j]) D[i * n + j] = dik + dkj;
            }
        }
}

/* ------------------------------------------------------------------ Brandes */

/* Betweenness centrality summed over the given sources (Brandes 2001):
 * for each source s, single-source shortest paths with path counts sigma_s
 * (breadth-first search when weighted == 0, else Dijkstra on int32 lengths),
 * then the dependencies
 *     delta_s(v) = sum over w with d_s(v) + w_vw == d_s(w) of
 *                  sigma_s(v) / sigma_s(w) * (1 + delta_s(w)),
 * taken in non-increasing distance order, and bc[v] += delta_s(v) for v != s.
 * bc is overwritten.  Directed graph in out-edge CSR. */
void orc_brandes(int64_t n, const int64_t* ptr, const int32_t* col, const int32_t* w,
                 int weighted, const int32_t* sources, int64_t nsrc, double* bc) {
    for (int64_t v = 0; v < n; ++v) bc[v] = 0.0;
    int nt = orc_num_threads();
    double* part = (double*)calloc((size_t)nt * (size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* mybc = part + (size_t)tid * (size_t)n;
        int64_t* dist = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        double* sigma = (double*)malloc(sizeof(double) * (size_t)n);
        double* delta = (double*)malloc(sizeof(double) * (size_t)n);
        int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        int64_t nnz = ptr[n];
        orc_hent* h = (orc_hent*)malloc(sizeof(orc_hent) * (size_t)(nnz + 2));
        uint8_t* done = (uint8_t*)malloc((size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (int64_t si = 0; si < nsrc; ++si) {
            int32_t s = sources[si];
            for (int64_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v] = 0.0; delta[v] = 0.0; done[v] = 0; }
            int64_t cnt = 0;
            dist[s] = 0; sigma[s] = 1.0;
            if (!weighted) {
                int64_t head = 0;
                order[cnt++] = s;
                while (head < cnt) {
                    int32_t u = order[head++];
                    for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
                        int32_t v = col[p];
                        if (dist[v] < 0) { dist[v] = dist[u] + 1; order[cnt++] = v; }
                        if (dist[v] == dist[u] + 1) sigma[v] += sigma[u];
                    }
                }
            } else {
                int64_t sz = 0;
                orc_hent e0 = {0.0, s};
                heap_push(h, &sz, e0);
                while (sz) {
                    orc_hent e = heap_pop(h, &sz);
                    int32_t u = e.v;
                    if (done[u]) continue;
                    done[u] = 1;
                    order[cnt++] = u;   /* settled in non-decreasing distance */
                    for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
                        int32_t v = col[p];
                        int64_t x = dist[u] + w[p];
                        if (dist[v] < 0 || x < dist[v]) {
                            dist[v] = x; sigma[v] = 0.0;
                            orc_hent ne = {(double)x, v}; heap_push(h, &sz, ne);
                        }
                    }
                }
                /* path counts in settled order: every predecessor of v settles before v
                 * because lengths are >= 1 */
                for (int64_t t = 0; t < cnt; ++t) {
                    int32_t u = order[t];
                    for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
                        int32_t v = col[p];
                        if (dist[u] + w[p] == dist[v]) sigma[v] += sigma[u];
                    }
                }
            }
            for (int64_t t = cnt - 1; t >= 0; --t) {
                int32_t v = order[t];
                for (int64_t p = ptr[v]; p < ptr[v + 1]; ++p) {
                    int32_t x = col[p];
                    int64_t len = weighted ? w[p] : 1;
                    if (dist[x] >= 0 && dist[v] + len == dist[x])
                        delta[v] += sigma[v] / sigma[x] * (1.0 + delta[x]);
                }
                if (v != s) mybc[v] += delta[v];
            }
        }
        free(dist); free(sigma); free(delta); free(order); free(h); free(done);
    }
    for (int t = 0; t < nt; ++t)
        for (int64_t v = 0; v < n; ++v) bc[v] += part[(size_t)t * (size_t)n + v];
    free(part);
}

/* Single-source shortest distances and path counts (the forward half of the
 * above) for one source: dist int32 (-1 unreached), sigma fp64. */
void orc_sssp_counts(int64_t n, const int64_t* ptr, const int32_t* col, const int32_t* w,
                     int weighted, int32_t s, int32_t* dist_out, double* sigma_out) {
    int64_t nnz = ptr[n];
    int64_t* dist = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t* done = (uint8_t*)calloc((size_t)n, 1);
    orc_hent* h = (orc_hent*)malloc(sizeof(orc_hent) * (size_t)(nnz + 2));
    for (int64_t v = 0; v < n; ++v) { dist[v] = -1; sigma_out[v] = 0.0; }
    dist[s] = 0; sigma_out[s] = 1.0;
    int64_t cnt = 0, sz = 0;
    orc_hent e0 = {0.0, s};
    heap_push(h, &sz, e0);
    while (sz) {
        orc_hent e = heap_pop(h, &sz);
        int32_t u = e.v;
        if (done[u]) continue;
        done[u] = 1;
        order[cnt++] = u;
        for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
            int32_t v = col[p];
            int64_t x = dist[u] + (weighted ? w[p] : 1);
            if (dist[v] < 0 || x < dist[v]) { dist[v] = x; orc_hent ne = {(double)x, v}; heap_push(h, &sz, ne); }
        }
    }
    for (int64_t t = 0; t < cnt; ++t) {
        int32_t u = order[t];
        for (int64_t p = ptr[u]; p < ptr[u + 1]; ++p) {
            int32_t v = col[p];
            if (dist[u] + (weighted ? w[p] : 1) == dist[v]) sigma_out[v] += sigma_out[u];
        }
    }
    for (int64_t v = 0; v < n; ++v) dist_out[v] = (int32_t)dist[v];
    free(dist); free(order); free(done); free(h);
}

/* ------------------------------------------------------- learned row sizing */

/* SplitMix64 output function (Steele, Lea & Flood; Vigna's public-domain
 * reference): the 64-bit mix of x + 0x9E3779B97F4A7C15.  The one-permutation
 * min-hash below hashes column ids with it. */
uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

#define ORC_NB 32        /* min-hash buckets */
#define ORC_NF 67        /* features per row: 3 scalars + 2 per bucket */

/* Features of the selected rows of C = A B, in fp64:
 *   f[0] = log2(1 + ub),  ub = sum over stored k of row i of nnz(B_k)
 *   f[1] = log2(1 + nnz(A_i))
 *   f[2] = log2(1 + max over stored k of nnz(B_k))
 *   f[3 + 2b], f[4 + 2b] for bucket b < 32 of the one-permutation min-hash of the
 *   union U_i of the column sets of those B rows: h = splitmix64(j), bucket =
 *   h >> 59, key = low 32 bits of h; f[3+2b] = (min key) / 2^32 and f[4+2b] = 0,
 *   or 1 and 1 when no column of U_i falls in the bucket.
 * The sketch is computed directly over U_i (every product visited). */
void orc_row_features(const int64_t* a_ptr, const int32_t* a_col, const int64_t* b_ptr,
                      const int32_t* b_col, const int64_t* rows, int64_t nsel, double* feat) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nsel; ++t) {
        int64_t i = rows[t];
        double* f = feat + t * ORC_NF;
        int64_t ub = 0, mx = 0;
        uint32_t mins[ORC_NB];
        for (int b = 0; b < ORC_NB; ++b) mins[b] = 0xFFFFFFFFu;
        int seen[ORC_NB];
        for (int b = 0; b < ORC_NB; ++b) seen[b] = 0;
        for (int64_t p = a_ptr[i]; p < a_ptr[i + 1]; ++p) {
            int32_t k = a_col[p];
            int64_t len = b_ptr[k + 1] - b_ptr[k];
            ub += len;
            if (len > mx) mx = len;
            for (int64_t q = b_ptr[k]; q < b_ptr[k + 1]; ++q) {
                uint64_t h = orc_splitmix64((uint64_t)b_col[q]);
                int b = (int)(h >> 59);
                uint32_t key = (uint32_t)(h & 0xFFFFFFFFull);
                seen[b] = 1;
                if (key < mins[b]) mins[b] = key;
            }
        }
        f[0] = log2(1.0 + (double)ub);
        f[1] = log2(1.0 + (double)(a_ptr[i + 1] - a_ptr[i]));
        f[2] = log2(1.0 + (double)mx);
        for (int b = 0; b < ORC_NB; ++b) {
            f[3 + 2 * b] = seen[b] ? (double)mins[b] / 4294967296.0 : 1.0;
            f[4 + 2 * b] = seen[b] ? 0.0 : 1.0;
        }
    }
}

/* Two-hidden-layer perceptron 67 -> 64 -> 64 -> 1 with ReLU, fp64.
 * Weight vector layout (8577 values): W1[64][67], b1[64], W2[64][64], b2[64],
 * w3[64], b3.  y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3. */
#define ORC_H 64
#define ORC_NW (ORC_H * ORC_NF + ORC_H + ORC_H * ORC_H + ORC_H + ORC_H + 1)

static void mlp_one(const double* w, const double* x, double* h1, double* h2, double* y) {
    const double* W1 = w;
    const double* b1 = W1 + ORC_H * ORC_NF;
    const double* W2 = b1 + ORC_H;
    const double* b2 = W2 + ORC_H * ORC_H;
    const double* w3 = b2 + ORC_H;
    const double* b3 = w3 + ORC_H;
    for (int o = 0; o < ORC_H; ++o) {
        double a = b1[o];
        for (int i = 0; i < ORC_NF; ++i) a += W1[o * ORC_NF + i] * x[i];
        h1[o] = a > 0.0 ? a : 0.0;
    }
    double out = b3[0];
    for (int o = 0; o < ORC_H; ++o) {
        double a = b2[o];
        for (int j = 0; j < ORC_H; ++j) a += W2[o * ORC_H + j] * h1[j];
        h2[o] = a > 0.0 ? a : 0.0;
        out += w3[o] * h2[o];
    }
    *y = out;
}

int orc_mlp_num_weights(void) { return ORC_NW; }

void orc_mlp_forward(const double* w, const double* x, int64_t n, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
        double h1[ORC_H], h2[ORC_H];
        mlp_one(w, x + r * ORC_NF, h1, h2, &y[r]);
    }
}

/* Gradient of the mean squared error L = (1/n) sum_r (y_r - t_r)^2 with respect
 * to every weight (backpropagation through the two ReLU layers); *loss = L. */
void orc_mlp_grad(const double* w, const double* x, const double* t, int64_t n, double* grad,
                  double* loss) {
    for (int k = 0; k < ORC_NW; ++k) grad[k] = 0.0;
    const double* W2 = w + ORC_H * ORC_NF + ORC_H;
    const double* w3 = W2 + ORC_H * ORC_H + ORC_H;
    double* gW1 = grad;
    double* gb1 = gW1 + ORC_H * ORC_NF;
    double* gW2 = gb1 + ORC_H;
    double* gb2 = gW2 + ORC_H * ORC_H;
    double* gw3 = gb2 + ORC_H;
    double* gb3 = gw3 + ORC_H;
    double L = 0.0;
    for (int64_t r = 0; r < n; ++r) {
        const double* xr = x + r * ORC_NF;
        double h1[ORC_H], h2[ORC_H], y, d2[ORC_H], d1[ORC_H];
        mlp_one(w, xr, h1, h2, &y);
        double e = y - t[r];
        L += e * e;
        double dy = 2.0 * e / (double)n;
        gb3[0] += dy;
        for (int o = 0; o < ORC_H; ++o) {
            gw3[o] += dy * h2[o];
            d2[o] = h2[o] > 0.0 ? dy * w3[o] : 0.0;
            gb2[o] += d2[o];
            for (int j = 0; j < ORC_H; ++j) gW2[o * ORC_H + j] += d2[o] * h1[j];
        }
        for (int j = 0; j < ORC_H; ++j) {
            double a = 0.0;
            for (int o = 0; o < ORC_H; ++o) a += W2[o * ORC_H + j] * d2[o];
            d1[j] = h1[j] > 0.0 ? a : 0.0;
            gb1[j] += d1[j];
            for (int i = 0; i < ORC_NF; ++i) gW1[j * ORC_NF + i] += d1[j] * xr[i];
        }
    }
    *loss = L / (double)n;
}
