/*
 * stc.h -- generalized sparse contraction on one B300 (sm_103a), C ABI.
 *
 * The library computes contractions
 *
 *     C[i,j]  (+)=  f( A[i,k], B[k,j] )      summed over k,
 *
 * where (+) is the additive operator of an algebraic structure and f is the
 * multiplicative operator or, more generally, a pairwise function whose operand
 * types may differ from the output type.  This is the contraction of Solomonik &
 * Hoefler, "Sparse Tensor Algebra as a Parallel Programming Model": algebraic
 * structures with an additive operator, its identity and a multiplicative
 * operator (Section 3.1, Table 1); contractions written as index expressions
 * (Section 3.3.1, C["ij"] = A["ik"]*B["kj"]); pairwise functions of the form
 * (type_C) <- (type_A, type_B) whose results are summed with the output's
 * additive operator (Section 3.3.2).  Bellman-Ford is the repeated tropical
 * matrix-vector product of Section 4.2.
 *
 * Three forms are provided: sparse x sparse (SpGEMM), sparse x dense block
 * (SpMM) and sparse x dense vector (SpMV), plus Bellman-Ford single-source
 * shortest paths built on the tropical product.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers (memory of the current CUDA device)
 *    unless stated otherwise.  Inputs are owned by the caller and only read.
 *  - CSR layout: rowptr int64[nrows+1] with rowptr[0] == 0, non-decreasing and
 *    rowptr[nrows] == nnz; col int32[nnz], ascending and unique within each row,
 *    each in [0, ncols); val: nnz elements of the algebra's operand type.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream).  Calls return once the work is enqueued, except where a result size
 *    must be known on the host (documented per call): those synchronise `stream`
 *    once.
 *  - Errors never abort the process.  A bad argument is reported before any
 *    work is enqueued; malformed CSR contents detected on the device are reported
 *    by the call's single synchronisation (or by stc_check_device_status for
 *    calls without one).  After an error no output is valid.
 *  - Memory the library needs (scratch and results) is obtained from the
 *    handle's allocator: callbacks passed to stc_create, or, when those are
 *    NULL, stream-ordered cudaMallocAsync/cudaFreeAsync.
 */
#ifndef STC_H
#define STC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define STC_API __attribute__((visibility("default")))
#else
#define STC_API
#endif

typedef struct CUstream_st* stc_stream; /* same type as cudaStream_t */

typedef enum {
    STC_OK = 0,
    STC_ERR_INVALID_ARG = 1, /* NULL pointer, negative size, unknown option        */
    STC_ERR_SHAPE = 2,       /* inner dimensions disagree, rowptr not monotone,
                                rowptr[0] != 0 or rowptr[nrows] != nnz            */
    STC_ERR_UNSORTED = 3,    /* columns not strictly ascending within a row,
                                or a column outside [0, ncols)                   */
    STC_ERR_ALGEBRA = 4,     /* algebra not supported by this entry point         */
    STC_ERR_OOM = 5,         /* the allocator returned NULL                       */
    STC_ERR_CUDA = 6,        /* a CUDA runtime call failed                        */
    STC_ERR_NEG_CYCLE = 7,   /* Bellman-Ford still relaxing after |V| rounds      */
    STC_ERR_TIMEOUT = 8,     /* a bounded device-side wait gave up                */
    STC_ERR_CAPACITY = 9     /* problem larger than the fixed scratch of
                                stc_bellman_ford_noalloc                         */
} stc_status;

/*
 * Algebras (Section 3.1, Table 1; Section 3.3.2 for the mixed-type function).
 * Operand element types are given as A / B / C.
 *
 *  STC_PLUS_TIMES_F32   (+,x) field. float / float / float.  Products rounded to
 *                       fp32, summed in fp32 in an unspecified order; in SpGEMM
 *                       the entries of a row of A with more than 1024 stored
 *                       entries are summed with compensation (the exact rounding
 *                       errors of products and adds collected beside each sum),
 *                       except in the masked product and in forced column windows.
 *  STC_PLUS_TIMES_F64   (+,x) field. double / double / double.
 *  STC_MIN_PLUS_I32     tropical semiring, (+) = min, f = integer +, additive
 *                       identity INT_MAX/2 = 1073741823 (Section 3.1: half of the
 *                       largest int, so that adding two identities cannot
 *                       overflow; no overflow check is made).  int32 throughout.
 *  STC_MIN_PLUS_F32     tropical semiring in fp32, identity +inf, f = fp32 add
 *                       (round to nearest even).  float throughout.
 *  STC_OR_AND_BOOL      boolean semiring, (+) = or, f = and.  uint8 0/1.
 *  STC_MULTPATH_I32_F64 (distance, multiplicity) monoid reached through the
 *                       pairwise function f(a, (d, s)) = (a + d, s): A holds
 *                       int32 edge lengths, B and C hold stc_dsig.
 *                       (d1,s1) (+) (d2,s2) = the pair with the smaller d, or
 *                       (d, s1 + s2) when d1 == d2.  Identity (INT_MAX/2, 0).
 */
typedef enum {
    STC_PLUS_TIMES_F32 = 0,
    STC_PLUS_TIMES_F64 = 1,
    STC_MIN_PLUS_I32 = 2,
    STC_MIN_PLUS_F32 = 3,
    STC_OR_AND_BOOL = 4,
    STC_MULTPATH_I32_F64 = 5
} stc_algebra;

#define STC_MIN_PLUS_I32_IDENTITY 1073741823

/* Element of the (distance, multiplicity) monoid: 16 bytes, sigma 8-aligned. */
typedef struct {
    int32_t d;
    int32_t pad;
    double sigma;
} stc_dsig;

/* A CSR matrix.  rowptr/col/val are device pointers.  For outputs the library
 * fills every field and allocates the three arrays with the handle's allocator;
 * release them with stc_free (or the matching user free callback). */
typedef struct {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    int64_t* rowptr;
    int32_t* col;
    void* val;
} stc_csr;

/* Allocator callbacks.  alloc returns device memory of at least `bytes` bytes
 * usable in stream order on `stream`, or NULL on failure (reported as
 * STC_ERR_OOM).  free receives a pointer from alloc and the stream after whose
 * queued work the memory may be reused. */
typedef void* (*stc_alloc_fn)(size_t bytes, void* ctx, stc_stream stream);
typedef void (*stc_free_fn)(void* ptr, void* ctx, stc_stream stream);

typedef struct stc_handle stc_handle;

/* Options of the SpGEMM call.  Pass NULL for the defaults (all zero). */
typedef struct {
    int32_t skip_validation; /* 1: trust the CSR contents (no device checks)     */
    int32_t window_cols;     /* 0: automatic; else the column-window width of the
                                numeric accumulator (power of two, >= 1024)      */
    int32_t light_rows;      /* 0: the handle's tuned value (stc_autotune_spgemm),
                                or none when untuned; -1: none; L in [1, 30]:
                                output rows whose product count is below 2^L get
                                their own numeric launch of 512-thread CTAs (two
                                per SM) beside the wide one, when such a row fits
                                the smaller value buffer (else ignored).  Applies
                                to outputs of at most 2^18 columns.              */
    int32_t reserved[5];     /* must be zero                                     */
} stc_opts;

/* Create a handle bound to the current CUDA device.  alloc/free may both be
 * NULL (stream-ordered cudaMallocAsync/cudaFreeAsync) or both non-NULL.
 * ctx is passed back to the callbacks unchanged. */
STC_API stc_status stc_create(stc_handle** out, stc_alloc_fn alloc, stc_free_fn free_fn, void* ctx);

/* Release the handle and its pinned host staging buffer.  Outputs returned by
 * earlier calls stay valid and must still be released with the allocator. */
STC_API void stc_destroy(stc_handle* h);

/* Release memory returned in an output of this library (stream-ordered). */
STC_API void stc_free(stc_handle* h, void* ptr, stc_stream stream);

/* Text for a status code (static storage). */
STC_API const char* stc_status_str(stc_status s);

/* Library version as major*10000 + minor*100 + patch. */
STC_API int32_t stc_version(void);

/*
 * SpGEMM: C = A (x) B over `alg` (Section 3.3.1 contraction C["ij"] = A["ik"]*B["kj"]
 * with the structure of Section 3.1 / function of Section 3.3.2).
 *
 * A is nrows x K, B is K x ncols (A->ncols must equal B->nrows).  On success C
 * receives nrows = A->nrows, ncols = B->ncols, nnz, and newly allocated rowptr,
 * col (ascending within each row) and val arrays.  The output structure is the
 * symbolic union of the input structures: an entry is present when at least one
 * product contributes to it, whatever its value (a (+,x) sum that cancels to 0
 * or a boolean 0 stays present).
 *
 * The call runs the plain two-pass method: row analysis and binning, an exact
 * symbolic pass that counts each output row, a scan into C->rowptr, then the
 * numeric pass.  It synchronises `stream` once, after the symbolic pass, to
 * learn nnz(C) and allocate C->col / C->val.
 *
 * opts may be NULL.  Errors: STC_ERR_INVALID_ARG, STC_ERR_SHAPE,
 * STC_ERR_UNSORTED (device checks, skipped when opts->skip_validation),
 * STC_ERR_ALGEBRA, STC_ERR_OOM, STC_ERR_CUDA.
 */
STC_API stc_status stc_contract_spgemm(stc_handle* h, stc_algebra alg, const stc_csr* A, const stc_csr* B,
                               stc_csr* C, const stc_opts* opts, stc_stream stream);

/*
 * Masked SpGEMM: the contraction with a prescribed output structure (the paper
 * lists output sparsity in contractions as future work, Section 7).  C has
 * exactly the structure of M:
 *   C_ij = (+) over k of f(A_ik, B_kj)   for every stored (i, j) of M,
 * and the algebra's additive identity where no product reaches (i, j) (0 for
 * (+,x) and bool, INT_MAX/2 for (min,+) int32, +inf for (min,+) fp32, and
 * (INT_MAX/2, 0) for the multiplicity monoid).  Products outside M are not
 * accumulated; rows whose M row is empty are not computed.
 *
 * M: CSR with nrows = A->nrows, ncols = B->ncols, sorted unique columns; its val
 * is ignored (may be NULL).  c_val: device array of M->nnz values of the
 * algebra's C type, in M's entry order (overwritten); C's row pointers and
 * columns are M's.  At most 2^18 output columns, and M->nrows times the per-row
 * rank record (8 B per 32 columns plus 8 B per 1024 columns) within 24 GB
 * (STC_ERR_INVALID_ARG otherwise).  Synchronises `stream` once (validation and
 * the longest mask row); the values are complete when the stream reaches them.
 * Errors: as stc_contract_spgemm, and STC_ERR_SHAPE when M's shape differs.
 */
STC_API stc_status stc_contract_spgemm_masked(stc_handle* h, stc_algebra alg, const stc_csr* A, const stc_csr* B,
                                              const stc_csr* M, void* c_val, const stc_opts* opts,
                                              stc_stream stream);

/*
 * Batched SpGEMM: C_b = A_b (x) B_b for b < nbatch independent pairs (Section
 * 3.3.1: an index shared by all three operands names independent problems), all
 * rows of all pairs handled by the same persistent launches (one row work queue
 * across the batch) and one synchronisation for the whole batch.
 *
 * A, B: HOST arrays of nbatch CSR descriptors (device pointers inside); every
 * B_b has at most 2^18 columns.  C: HOST array of nbatch descriptors filled on
 * success.  Their arrays are views into three allocations shared by the batch:
 * C[0].rowptr, C[0].col and C[0].val are the allocation bases (release those
 * three with stc_free); C[b].rowptr is row-pointer array b (starting at 0), and
 * C[b].col / C[b].val point at matrix b's entries.  Errors as for
 * stc_contract_spgemm; nbatch in 1..65535.
 */
STC_API stc_status stc_contract_spgemm_batched(stc_handle* h, stc_algebra alg, int32_t nbatch, const stc_csr* A,
                                               const stc_csr* B, stc_csr* C, const stc_opts* opts,
                                               stc_stream stream);

/*
 * SpMM: Y = A (x) X, or Y = Y (+) (A (x) X) when accumulate != 0
 * (Section 3.3.1 contraction with a dense operand).
 *
 * X is a dense A->ncols x ncol block, row-major with leading dimension ldx
 * (elements, ldx >= ncol); Y is A->nrows x ncol with leading dimension ldy.
 * Element types: A as in the algebra; X and Y the B/C type, except that
 * STC_PLUS_TIMES_F32 reads and writes float.  Without accumulate, a row of A
 * with no stored entry yields the additive identity.  SpMV is ncol == 1.
 * Asynchronous; malformed CSR contents are reported through
 * stc_check_device_status.
 */
STC_API stc_status stc_contract_spmm(stc_handle* h, stc_algebra alg, const stc_csr* A, const void* X,
                             int64_t ldx, int32_t ncol, void* Y, int64_t ldy, int32_t accumulate,
                             stc_stream stream);

/* SpMV: y = A (x) x, or y (+)= A (x) x.  Same rules as stc_contract_spmm with ncol 1. */
STC_API stc_status stc_contract_spmv(stc_handle* h, stc_algebra alg, const stc_csr* A, const void* x,
                             void* y, int32_t accumulate, stc_stream stream);

/* Read and clear the handle's device-side error flags raised by asynchronous
 * calls (synchronises `stream`).  Returns STC_OK when none was raised. */
STC_API stc_status stc_check_device_status(stc_handle* h, stc_stream stream);

/*
 * Bellman-Ford single-source shortest paths (Section 4.2): repeated tropical
 * products P <- P (+) A (x) P with A_ii = 0 until no distance changes.
 *
 * G is the graph in OUT-EDGE CSR: row u lists the edges u -> v with lengths
 * G->val (the transpose of the paper's A, whose A_ij is the length of edge
 * j -> i).  alg is STC_MIN_PLUS_I32 (int32 lengths and distances, unreached =
 * INT_MAX/2) or STC_MIN_PLUS_F32 (float, unreached = +inf).  A vertex at the
 * additive identity relaxes nothing.  dist_out (device, G->nrows elements)
 * receives the distances; *rounds_out (host, may be NULL) the number of rounds
 * in which some distance decreased; *relaxations_out (host, may be NULL) the
 * number of edge relaxations performed (the tropical products evaluated).
 *
 * Each round relaxes only the out-edges of vertices whose distance decreased in
 * the previous round (frontier), which reaches the same fixed point as full
 * relaxation: for fp32 the minimum over paths of the left-to-right rounded path
 * sums, bit for bit.  `persistent` selects the driver: 0 launches one kernel per
 * round and reads the frontier size on the host each round; 1 runs all rounds
 * inside one cooperative launch with a bounded grid barrier and a device-side
 * convergence test; 2 launches one CUDA graph whose conditional WHILE node
 * repeats {relaxation round, termination test}, the test setting the loop
 * condition on the device (no host round trip per round).  Synchronises `stream`.
 * Errors: STC_ERR_NEG_CYCLE when round |V| still lowers a distance (a negative
 * cycle is reachable), STC_ERR_TIMEOUT when a bounded grid barrier gives up,
 * plus the argument and CSR errors above.
 */
STC_API stc_status stc_bellman_ford(stc_handle* h, stc_algebra alg, const stc_csr* G, int32_t source,
                            void* dist_out, int32_t* rounds_out, int64_t* relaxations_out,
                            int32_t persistent, stc_stream stream);

/*
 * All-pairs shortest paths by path doubling (Section 4.2): the closure of
 * I + G over (min,+) int32 by repeated squaring, P <- P (x) P, until a squaring
 * changes nothing (at most ceil(log2 n) + 1 squarings).  Work is O(n^3 log n)
 * for a dense graph (Floyd-Warshall's O(n^3) is sequential in n; this is
 * logarithmic in depth).
 *
 * G: square CSR, row u lists the edges u -> v with int32 lengths (val required;
 * negative lengths allowed).  *P_out receives the distance matrix as a CSR
 * allocated through the handle (release rowptr, col, val with stc_free): entry
 * (u, v) is the shortest u -> v distance, stored for every reachable pair
 * (the diagonal is 0); unreachable pairs are not stored.  Path sums must fit
 * int32 (no overflow check, as for the semiring itself).  *squarings_out (host,
 * may be NULL): squarings performed.  Synchronises `stream`.  Errors: CSR and
 * argument errors, STC_ERR_SHAPE for a non-square G, STC_ERR_NEG_CYCLE when a
 * diagonal entry ends negative (a negative cycle).
 */
STC_API stc_status stc_apsp_path_doubling(stc_handle* h, const stc_csr* G, stc_csr* P_out, int32_t* squarings_out,
                                          stc_stream stream);

/*
 * All-pairs shortest paths by Tiskin's path doubling (Section 4.2, the paper's
 * simplified form: the paths of exactly l hops at every step).  Paths carry
 * (weight, hops); P starts as the edges (w, 1) and, for l = 1, 2, 4, ... < n,
 * P <- P (+) Pl (x) P where Pl holds the entries of P with exactly l hops and
 * (+) takes the lexicographic minimum of (weight, hops) -- the paper keeps the
 * second operand on a weight tie, which depends on the order of reduction; the
 * hop count breaks the tie here, so the result is the same whatever the order.
 * The loop ends early when Pl is empty.  Pl shrinks as l grows, so the product
 * count is well below that of stc_apsp_path_doubling on most graphs.
 *
 * G, *P_out and the errors as for stc_apsp_path_doubling (the same distance
 * matrix, zero diagonal included).  *rounds_out (host, may be NULL): doubling
 * steps performed; *products_out (host, may be NULL): path products evaluated,
 * the sum over the steps of the entries (i, k) of Pl times nnz(P_k).
 */
STC_API stc_status stc_apsp_tiskin(stc_handle* h, const stc_csr* G, stc_csr* P_out, int32_t* rounds_out,
                                   int64_t* products_out, stc_stream stream);

/*
 * Shortest distances and path counts from up to 256 sources at once: Bellman-Ford
 * over the (distance, multiplicity) monoid of STC_MULTPATH_I32_F64 (the geodetic
 * semiring that Section 4.2 names for betweenness centrality), with each vertex
 * propagating only the multiplicity it gained since it last sent.
 *
 * G: out-edge CSR (row u lists u -> v); val = int32 lengths >= 1, or NULL for
 * unit lengths.  sources: HOST array of nsources (1..256) vertex ids.
 * d_out (device, int32 [G->nrows][nsources]) receives d_s(v) (INT_MAX/2 when v is
 * unreachable from s); sigma_out (device, fp64 [G->nrows][nsources]) the number of
 * shortest s-v paths (exact while below 2^53).  *rounds_out (host, may be NULL):
 * rounds run.  The rounds run under the handle's round driver (see
 * stc_set_round_driver); either way the call synchronises `stream` before it
 * returns.  Errors: argument/CSR errors, STC_ERR_INVALID_ARG for a length < 1 or
 * a graph with nrows + nnz / 1024 + 2 above INT32_MAX.
 */
STC_API stc_status stc_mfbc_sssp(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsources,
                                 int32_t* d_out, double* sigma_out, int32_t* rounds_out, stc_stream stream);

/*
 * Betweenness centrality summed over the given sources (Brandes' dependency
 * accumulation on the multiplicity-monoid shortest paths above):
 *   bc_out[v] = sum over s in sources, s != v, of
 *               sum over t of sigma_st(v) / sigma_st
 * Directed; no normalisation or halving.  Sources are processed in batches of
 * `batch` (1..256) columns at a time; device memory ~ 32 * G->nrows * batch bytes.
 * G, sources and lengths as for stc_mfbc_sssp; bc_out: device fp64 [G->nrows],
 * overwritten.  Runs under the handle's round driver; synchronises `stream`
 * before it returns.
 */
STC_API stc_status stc_mfbc(stc_handle* h, const stc_csr* G, const int32_t* sources, int32_t nsources,
                            int32_t batch, double* bc_out, stc_stream stream);

/*
 * Round driver of the multi-round betweenness-centrality calls above (the paper
 * runs its iterations from the host; this is a device-side form of the same loop).
 *   driver = 0: host-driven -- each round's kernels are launched from the host,
 *               which reads the loop condition back after every round (one
 *               stream synchronisation per round);
 *   driver = 1: (default) each batch is one CUDA graph launch: the forward and
 *               backward round loops are conditional WHILE nodes whose condition
 *               a one-thread check kernel sets on the device, so no round needs
 *               the host.
 * Both drivers launch the same kernels and give identical results.  Errors:
 * STC_ERR_INVALID_ARG for a null handle or another value.
 */
STC_API stc_status stc_set_round_driver(stc_handle* h, int32_t driver);

/*
 * Learned output sizing (no counterpart in the paper, which leaves SpGEMM and
 * output sparsity as future work, Section 7; it names automatically-adjusted
 * performance models as a direction there).
 *
 * Features of output row i of C = A B, STC_MLP_FEAT_STRIDE floats per row (the
 * last is zero padding):
 *   f0 = log2(1 + ub_i), ub_i = sum over stored k of row i of A of nnz(B_k)
 *   f1 = log2(1 + nnz(A_i)),  f2 = log2(1 + max over those k of nnz(B_k))
 *   f3+2b, f4+2b (b < 32): one-permutation min-hash of the union of those B rows'
 *   columns: h = SplitMix64 output of the column id, bucket = top 5 bits of h,
 *   key = low 32 bits; (min key) / 2^32 and 0, or 1 and 1 if the bucket is empty.
 * Model: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 predicting log2(1 + nnz(C_i)),
 * 67 -> 64 -> 64 -> 1.  Weights: STC_MLP_NUM_WEIGHTS fp32 values in device memory,
 * laid out W1[64][67], b1[64], W2[64][64], b2[64], w3[64], b3; they are rounded to
 * bf16 wherever the model is evaluated, sums are fp32.
 */
#define STC_MLP_INPUTS 67
#define STC_MLP_FEAT_STRIDE 68
#define STC_MLP_HIDDEN 64
#define STC_MLP_NUM_WEIGHTS 8577

/* feat (device, float [A->nrows][STC_MLP_FEAT_STRIDE]) <- features of every row of A B. */
STC_API stc_status stc_row_features(stc_handle* h, const stc_csr* A, const stc_csr* B, float* feat,
                                    stc_stream stream);

/* y[r] (device float [n]) <- model(feat[r]). */
STC_API stc_status stc_mlp_forward(stc_handle* h, const float* weights, const float* feat, int64_t n, float* y,
                                   stc_stream stream);

/* The same model on the tensor cores (tcgen05 MMAs, fp32 accumulators in tensor
 * memory): each fp32 activation enters as the sum of two bf16 halves (hi, lo), so
 * inputs keep about 16 significant bits (error <= 2^-16 of each value).  The error
 * of y is that rounding carried through the weights: about 1e-5 of |y| on feature
 * rows, more where y cancels larger intermediate sums.  feat must be 16-byte
 * aligned (STC_ERR_INVALID_ARG otherwise).  A tensor-core completion that does not arrive within about a
 * quarter of a second raises STC_FLAG_TIMEOUT (read by stc_check_device_status);
 * the kernel then releases its tensor memory and returns. */
STC_API stc_status stc_mlp_forward_tc(stc_handle* h, const float* weights, const float* feat, int64_t n, float* y,
                                      stc_stream stream);

/* grad (device float [STC_MLP_NUM_WEIGHTS]) += gradient of
 * (1/scale) * sum over the n rows r = idx[0..n) (idx NULL: rows 0..n) of
 * (y_r - target_r)^2; *loss (device float) += that sum of squares. */
STC_API stc_status stc_mlp_grad(stc_handle* h, const float* weights, const float* feat, const float* target,
                                const int32_t* idx, int64_t n, float scale, float* grad, float* loss,
                                stc_stream stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step counted from 1) on the
 * fp32 weights with moment buffers m, v; grad is consumed and cleared. */
STC_API stc_status stc_mlp_adam(stc_handle* h, float* weights, float* m, float* v, float* grad, int64_t step,
                                float lr, stc_stream stream);

/* Initialise weights (device) with He-normal layers and zero biases from `seed`. */
STC_API stc_status stc_mlp_init(float* weights, uint64_t seed, stc_stream stream);

/* Mini-batch training: `epochs` passes over the n examples (feat, target on the
 * device) in a seeded random order, mean squared error, Adam with rate lr.
 * loss_out (host, may be NULL) receives the mean loss of every epoch.
 * Synchronises `stream` once per epoch. */
STC_API stc_status stc_mlp_train(stc_handle* h, float* weights, const float* feat, const float* target, int64_t n,
                                 int32_t batch, int32_t epochs, float lr, uint64_t seed, float* loss_out,
                                 stc_stream stream);

/*
 * Exact row sizes: counts[i] = nnz(C_i) for C = A B (device int64 [A->nrows]),
 * the symbolic phase of the plain path alone (the size of the union of the
 * column sets of the B rows that row i of A selects, Section 3.3.1).  Values of
 * A and B are not read and may be NULL.  Outputs wider than 2^18 columns are
 * counted slab by slab (at most 32 slabs of 2^18 columns; STC_ERR_SHAPE above).
 * opts may be NULL (validation on).  Synchronises `stream` once (the
 * validation flags).
 */
STC_API stc_status stc_row_counts(stc_handle* h, const stc_csr* A, const stc_csr* B, int64_t* counts,
                                  const stc_opts* opts, stc_stream stream);

/*
 * Training examples of the row-size model from the product A B: feat (device,
 * float [A->nrows][STC_MLP_FEAT_STRIDE]) as stc_row_features, and the exact
 * targets target[i] = log2(1 + nnz(C_i)) (device float [A->nrows]) from the
 * symbolic phase (stc_row_counts).  Values of A and B are not read.
 * Synchronises `stream` once.
 */
STC_API stc_status stc_training_rows(stc_handle* h, const stc_csr* A, const stc_csr* B, float* feat,
                                     float* target, stc_stream stream);

/*
 * Model files.  stc_model_save writes the STC_MLP_NUM_WEIGHTS fp32 weights
 * (device) to `path`: a 32-byte header (magic "STCMLP1", inputs 67, hidden 64,
 * number of weights, the 64-bit FNV-1a checksum of the weight bytes) followed by
 * the weights as little-endian fp32.  stc_model_load reads such a file into
 * `weights` (device); a missing or unreadable file, another layout, trailing
 * bytes or a checksum mismatch give STC_ERR_INVALID_ARG and leave `weights`
 * unchanged.  Both synchronise `stream`.
 */
STC_API stc_status stc_model_save(const char* path, const float* weights, stc_stream stream);
STC_API stc_status stc_model_load(const char* path, float* weights, stc_stream stream);

typedef struct {
    int64_t rows;              /* output rows with at least one product (-1: exact path used) */
    int64_t overflow_rows;     /* rows whose predicted capacity was too small */
    int64_t scratch_entries;   /* total predicted capacity (the slots, without the overflow pool) */
    int64_t nnz;               /* nnz(C) */
    double mean_abs_log2_error; /* mean |prediction - log2(1 + nnz(C_i))| (-1 without a model) */
    int64_t recomputed_rows;   /* overflow rows that also missed the overflow pool: recomputed */
} stc_learned_stats;

/*
 * Learned single-pass SpGEMM: C = A (x) B with the same result as
 * stc_contract_spgemm (bit-identical structure), without the separate symbolic
 * pass.  Every row gets a capacity -- (1 + margin) * (2^prediction - 1) + 8 from
 * the model `weights`, clipped to [1, min(ub_i, ncols)], or min(ub_i, ncols) when
 * weights is NULL -- and one numeric pass writes it into scratch of that size
 * while counting it exactly; a row larger than its capacity goes to an overflow
 * pool after the slots (a quarter of their size); rows that fit are compacted
 * into C, rows that missed the pool too are recomputed exactly.  Outputs wider than 2^18 columns (at most 32
 * column slabs of 2^18) run the same single pass slab by slab: every slab B_s
 * is its own learned product A B_s, and stats count (row, slab) units; wider
 * outputs than that use the exact two-pass path (stats->rows = -1).
 * Synchronises `stream` twice.  stats (host, may be NULL) as above.
 */
STC_API stc_status stc_contract_spgemm_learned(stc_handle* h, stc_algebra alg, const stc_csr* A, const stc_csr* B,
                                               stc_csr* C, const float* weights, float margin,
                                               stc_learned_stats* stats, const stc_opts* opts, stc_stream stream);

/*
 * Autotuner (the single-GPU counterpart of the paper's tuning over candidate
 * decompositions with performance models, Section 5.1, and of the
 * automatically-adjusted performance models it names as future work, Section 7).
 *
 * stc_autotune_spgemm times C = A (x) B under every candidate light-row threshold
 * (see stc_opts.light_rows: none, then each L whose rows fit the light launch's
 * value buffer, ascending), each after one untimed run, with CUDA events on
 * `stream`, and stores the fastest in the handle's cache for this algebra and
 * output width (ceil(log2 B->ncols)); later calls with light_rows == 0 use it.
 * cand_out / ms_out (host, 8 entries each, may be NULL) receive the candidates
 * (-1 = none) and their times in milliseconds, *ncand_out their number, *best_out
 * the chosen threshold.  Outputs of the timing runs are released.  Errors: those
 * of stc_contract_spgemm; STC_ERR_INVALID_ARG for B->ncols > 2^18.
 *
 * stc_tune_save writes the handle's cache as text (a header naming the device
 * and its SM count, then one "algebra log2-columns threshold" line per entry);
 * stc_tune_load reads such a file into the cache, STC_ERR_INVALID_ARG when it
 * was written for another device or is malformed (the cache is then unchanged).
 */
STC_API stc_status stc_autotune_spgemm(stc_handle* h, stc_algebra alg, const stc_csr* A, const stc_csr* B,
                                       int32_t* best_out, int32_t* cand_out, float* ms_out, int32_t* ncand_out,
                                       stc_stream stream);
STC_API stc_status stc_tune_save(const stc_handle* h, const char* path);
STC_API stc_status stc_tune_load(stc_handle* h, const char* path);

/*
 * Failure-detection self test (no counterpart in the paper).  Runs the bounded
 * grid barrier of the persistent solvers in a cooperative launch of two blocks
 * that expects 2 + missing blocks (missing = 0 or 1).  With missing = 0 every
 * block passes and the call returns STC_OK; with missing = 1 no block can pass,
 * every block gives up after spin_limit polls of about 0.5 us (1 .. 2^24) and the
 * call returns STC_ERR_TIMEOUT.  Either way nothing hangs and the handle stays
 * usable.  Synchronises `stream`.
 */
STC_API stc_status stc_selftest_barrier(stc_handle* h, int32_t missing, int32_t spin_limit, stc_stream stream);

/*
 * Instrumentation (no counterpart in the paper, which reports only the share of
 * time spent in local kernels).
 *
 * stc_set_timing: when enable != 0, later calls record CUDA events on their
 * stream at phase boundaries.  stc_phase_times synchronises on the last event of
 * the most recent timed call and writes up to max_phases durations in
 * milliseconds; it returns the number of phases of that call (0 if none).
 *   SpGEMM phases: 0 validation, 1 row analysis + binning + window table,
 *                  2 symbolic, 3 scan, 4 numeric.
 *   Bellman-Ford phases: 0 validation + initialisation, 1 all relaxation rounds.
 * stc_kernel_launches: number of kernels this handle has launched so far.
 */
STC_API stc_status stc_set_timing(stc_handle* h, int32_t enable);
STC_API int32_t stc_phase_times(stc_handle* h, float* ms_out, int32_t max_phases);
STC_API int64_t stc_kernel_launches(const stc_handle* h);

/*
 * Calibration of the numeric pass's accumulator (the paper has no counterpart;
 * it measures the bound of the SpGEMM numeric phase on the running device).  One
 * CTA of 1024 threads per SM has every thread combine 8192 products into 8192
 * shared-memory accumulators at pseudo-random positions with the algebra's (+),
 * applied as the numeric kernel applies it (fp64 (+,x): compare-and-swap of an
 * fma).  *updates_per_s (host) receives the fastest of three timed runs after one
 * warm-up, in products absorbed per second.  STC_ERR_ALGEBRA for the
 * (distance, multiplicity) monoid.  Synchronises `stream`.
 */
STC_API stc_status stc_calibrate_accumulate(stc_handle* h, stc_algebra alg, double* updates_per_s,
                                            stc_stream stream);

/*
 * Allocation-free Bellman-Ford.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run -- for
 * example code inside a host callback or a real-time loop where cudaMalloc would
 * block or is forbidden, or a host process that hands out memory only from its
 * own fixed pools.  It computes exactly what stc_bellman_ford computes with
 * persistent = 1, takes no handle, and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Its working memory (frontiers, round stamps, distance keys, counters) lives in
 * one fixed array in device global memory that the library defines for every GPU
 * it is loaded on (about 16 MiB, held until the process exits).  Hence:
 *  - G->nrows may not exceed STC_NOALLOC_BF_MAX_VERTICES; larger graphs get
 *    STC_ERR_CAPACITY before any work is enqueued.
 *  - The first call on each device looks up that array's device address
 *    (cudaGetSymbolAddress) with the device current.
 *  - Every call synchronises `stream` and reads its result back into host
 *    memory, so no call may be made while a stream on the device is being
 *    captured into a CUDA graph.
 *  - Every call on a device shares the same array and leaves its contents
 *    behind; each call clears what must start at zero.  Calls whose work
 *    overlaps on the GPU (different streams or threads without ordering) race
 *    on the array and give wrong results: serialise them.
 * Arguments, results and the other errors are those of stc_bellman_ford;
 * *rounds_out (host, may be NULL).
 */
#define STC_NOALLOC_BF_MAX_VERTICES (1 << 20)
STC_API stc_status stc_bellman_ford_noalloc(stc_algebra alg, const stc_csr* G, int32_t source,
                                            void* dist_out, int32_t* rounds_out, stc_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* STC_H */
