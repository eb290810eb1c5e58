// SpMM / SpMV: Y[i, c] (+)= f(A[i,k], X[k, c]) over the stored k of row i
// (Section 3.3.1 contraction with a dense operand; structures of Section 3.1,
// pairwise function of Section 3.3.2).
//
// ncol == 1: one warp per row, lanes over the row's entries, a warp reduction
// with the algebra's additive operator.  ncol > 1: one warp per row, lanes over
// 32 consecutive columns of X (coalesced rows of X), one accumulator per lane.
#include "stc_internal.cuh"

namespace {

template <int ALG> struct MM;

template <> struct MM<ALG_PT_F32> {
    using A = float; using X = float; using Y = float; using Acc = double;
    static __device__ __forceinline__ Acc id() { return 0.0; }
    static __device__ __forceinline__ Acc f(A a, X x) { return double(a) * double(x); }
    static __device__ __forceinline__ Acc add(Acc u, Acc v) { return u + v; }
    static __device__ __forceinline__ Acc load(Y y) { return double(y); }
    static __device__ __forceinline__ Y out(Acc v) { return float(v); }
};
template <> struct MM<ALG_PT_F64> {
    using A = double; using X = double; using Y = double; using Acc = double;
    static __device__ __forceinline__ Acc id() { return 0.0; }
    static __device__ __forceinline__ Acc f(A a, X x) { return a * x; }
    static __device__ __forceinline__ Acc add(Acc u, Acc v) { return u + v; }
    static __device__ __forceinline__ Acc load(Y y) { return y; }
    static __device__ __forceinline__ Y out(Acc v) { return v; }
};
template <> struct MM<ALG_MP_I32> {
    using A = int; using X = int; using Y = int; using Acc = int;
    static __device__ __forceinline__ Acc id() { return STC_MIN_PLUS_I32_IDENTITY; }
    static __device__ __forceinline__ Acc f(A a, X x) { return a + x; }
    static __device__ __forceinline__ Acc add(Acc u, Acc v) { return u < v ? u : v; }
    static __device__ __forceinline__ Acc load(Y y) { return y; }
    static __device__ __forceinline__ Y out(Acc v) { return v; }
};
template <> struct MM<ALG_MP_F32> {
    using A = float; using X = float; using Y = float; using Acc = float;
    static __device__ __forceinline__ Acc id() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ Acc f(A a, X x) { return __fadd_rn(a, x); }
    static __device__ __forceinline__ Acc add(Acc u, Acc v) { return v < u ? v : u; }
    static __device__ __forceinline__ Acc load(Y y) { return y; }
    static __device__ __forceinline__ Y out(Acc v) { return v; }
};
template <> struct MM<ALG_BOOL> {
    using A = uint8_t; using X = uint8_t; using Y = uint8_t; using Acc = int;
    static __device__ __forceinline__ Acc id() { return 0; }
    static __device__ __forceinline__ Acc f(A a, X x) { return (a != 0) & (x != 0); }
    static __device__ __forceinline__ Acc add(Acc u, Acc v) { return u | v; }
    static __device__ __forceinline__ Acc load(Y y) { return y != 0; }
    static __device__ __forceinline__ Y out(Acc v) { return uint8_t(v); }
};
struct DS {
    int d;
    double s;
};
template <> struct MM<ALG_MULTPATH> {
    using A = int; using X = DSig; using Y = DSig; using Acc = DS;
    static __device__ __forceinline__ Acc id() { return DS{STC_MIN_PLUS_I32_IDENTITY, 0.0}; }
    static __device__ __forceinline__ Acc f(A a, X x) { return DS{a + x.d, x.s}; }
    static __device__ __forceinline__ Acc add(Acc u, Acc v) {
        if (u.d < v.d) return u;
        if (v.d < u.d) return v;
        return DS{u.d, u.s + v.s};
    }
    static __device__ __forceinline__ Acc load(Y y) { return DS{y.d, y.s}; }
    static __device__ __forceinline__ Y out(Acc v) {
        DSig r;
        r.d = v.d;
        r.pad = 0;
        r.s = v.s;
        return r;
    }
};

template <class Acc>
__device__ __forceinline__ Acc shfl_down(Acc v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
template <>
__device__ __forceinline__ DS shfl_down<DS>(DS v, int o) {
    DS r;
    r.d = __shfl_down_sync(0xffffffffu, v.d, o);
    r.s = __shfl_down_sync(0xffffffffu, v.s, o);
    return r;
}

template <int ALG>
__global__ void __launch_bounds__(256) k_spmv(int64_t nrows, int64_t ncols, int64_t nnz,
                                              const int64_t* __restrict__ ptr,
                                              const int32_t* __restrict__ col,
                                              const void* __restrict__ aval, const void* __restrict__ x,
                                              void* __restrict__ y, int accumulate) {
    using T = MM<ALG>;
    const int lane = threadIdx.x & 31;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const auto* A = static_cast<const typename T::A*>(aval);
    const auto* X = static_cast<const typename T::X*>(x);
    auto* Y = static_cast<typename T::Y*>(y);
    for (int64_t i = warp; i < nrows; i += nwarps) {
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        typename T::Acc acc = T::id();
        for (int64_t p = lo + lane; p < hi; p += 32) {
            int32_t k = col[p];
            if ((uint64_t)k < (uint64_t)ncols) acc = T::add(acc, T::f(A[p], X[k]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = T::add(acc, shfl_down(acc, o));
        if (lane == 0) {
            if (accumulate) acc = T::add(T::load(Y[i]), acc);
            Y[i] = T::out(acc);
        }
    }
}

template <int ALG>
__global__ void __launch_bounds__(256) k_spmm(int64_t nrows, int64_t ncols, int64_t nnz,
                                              const int64_t* __restrict__ ptr,
                                              const int32_t* __restrict__ col,
                                              const void* __restrict__ aval, const void* __restrict__ x,
                                              int64_t ldx, int ncol, void* __restrict__ y, int64_t ldy,
                                              int accumulate) {
    using T = MM<ALG>;
    const int lane = threadIdx.x & 31;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const auto* A = static_cast<const typename T::A*>(aval);
    const auto* X = static_cast<const typename T::X*>(x);
    auto* Y = static_cast<typename T::Y*>(y);
    for (int64_t i = warp; i < nrows; i += nwarps) {
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        for (int c0 = 0; c0 < ncol; c0 += 32) {
            const int c = c0 + lane;
            typename T::Acc acc = T::id();
            for (int64_t p = lo; p < hi; ++p) {
                int32_t k = col[p];
                if ((uint64_t)k < (uint64_t)ncols && c < ncol) acc = T::add(acc, T::f(A[p], X[int64_t(k) * ldx + c]));
            }
            if (c < ncol) {
                if (accumulate) acc = T::add(T::load(Y[i * ldy + c]), acc);
                Y[i * ldy + c] = T::out(acc);
            }
        }
    }
}

// Wide dense operands (ncol >= MM_TILE): warp units (row, tile of MM_TILE columns)
// taken tile-major, so the warps running at one time share one column tile of X
// (nrows x MM_TILE values, resident in L2); each lane holds MM_U accumulators
// (independent chains) and the row's entries are read once per tile.
constexpr int MM_U = 4;
constexpr int MM_TILE = 32 * MM_U;

template <int ALG>
__global__ void __launch_bounds__(256) k_spmm_tiled(int64_t nrows, int64_t ncols, int64_t nnz,
                                                    const int64_t* __restrict__ ptr,
                                                    const int32_t* __restrict__ col,
                                                    const void* __restrict__ aval, const void* __restrict__ x,
                                                    int64_t ldx, int ncol, void* __restrict__ y, int64_t ldy,
                                                    int accumulate) {
    using T = MM<ALG>;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const int ntiles = (ncol + MM_TILE - 1) / MM_TILE;
    const int64_t nunits = nrows * ntiles;
    const auto* A = static_cast<const typename T::A*>(aval);
    const auto* X = static_cast<const typename T::X*>(x);
    auto* Y = static_cast<typename T::Y*>(y);
    for (int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < nunits; q += nwarps) {
        const int64_t tile = q / nrows;
        const int64_t i = q - tile * nrows;
        const int c0 = int(tile) * MM_TILE + lane;
        int64_t lo, hi;
        row_range(ptr, i, nnz, lo, hi);
        typename T::Acc acc[MM_U];
#pragma unroll
        for (int u = 0; u < MM_U; ++u) acc[u] = T::id();
        for (int64_t p = lo; p < hi; ++p) {
            const int32_t k = col[p];
            if ((uint64_t)k >= (uint64_t)ncols) continue;
            const typename T::A a = A[p];
            const auto* xr = X + int64_t(k) * ldx;
            typename T::X xv[MM_U];
#pragma unroll
            for (int u = 0; u < MM_U; ++u) {
                const int c = c0 + 32 * u;
                if (c < ncol) xv[u] = xr[c];
            }
#pragma unroll
            for (int u = 0; u < MM_U; ++u)
                if (c0 + 32 * u < ncol) acc[u] = T::add(acc[u], T::f(a, xv[u]));
        }
#pragma unroll
        for (int u = 0; u < MM_U; ++u) {
            const int c = c0 + 32 * u;
            if (c < ncol) {
                typename T::Acc v = acc[u];
                if (accumulate) v = T::add(T::load(Y[i * ldy + c]), v);
                Y[i * ldy + c] = T::out(v);
            }
        }
    }
}

template <int ALG>
stc_status launch_mm(stc_handle* h, const stc_csr* A, const void* X, int64_t ldx, int32_t ncol, void* Y,
                     int64_t ldy, int32_t accumulate, stc_stream s) {
    int64_t blocks = (A->nrows * 32 + 255) / 256;
    int64_t cap = int64_t(h->num_sms) * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (ncol == 1)
        k_spmv<ALG><<<unsigned(blocks), 256, 0, s>>>(A->nrows, A->ncols, A->nnz, A->rowptr, A->col, A->val,
                                                    X, Y, accumulate);
    else if (ncol >= MM_TILE)
        k_spmm_tiled<ALG><<<unsigned(h->num_sms * 16), 256, 0, s>>>(A->nrows, A->ncols, A->nnz, A->rowptr, A->col,
                                                                     A->val, X, ldx, ncol, Y, ldy, accumulate);
    else
        k_spmm<ALG><<<unsigned(blocks), 256, 0, s>>>(A->nrows, A->ncols, A->nnz, A->rowptr, A->col, A->val,
                                                    X, ldx, ncol, Y, ldy, accumulate);
    STC_LAUNCH_CHECK();
    return STC_OK;
}

}  // namespace

stc_status stc_spmm_impl(stc_handle* h, int alg, const stc_csr* A, const void* X, int64_t ldx,
                         int32_t ncol, void* Y, int64_t ldy, int32_t accumulate, stc_stream s) {
    if (A->nrows == 0 || ncol == 0) return STC_OK;
    stc_status st = stc_validate_csr_async(h, A, s);
    if (st != STC_OK) return st;
    switch (alg) {
    case ALG_PT_F32: return launch_mm<ALG_PT_F32>(h, A, X, ldx, ncol, Y, ldy, accumulate, s);
    case ALG_PT_F64: return launch_mm<ALG_PT_F64>(h, A, X, ldx, ncol, Y, ldy, accumulate, s);
    case ALG_MP_I32: return launch_mm<ALG_MP_I32>(h, A, X, ldx, ncol, Y, ldy, accumulate, s);
    case ALG_MP_F32: return launch_mm<ALG_MP_F32>(h, A, X, ldx, ncol, Y, ldy, accumulate, s);
    case ALG_BOOL: return launch_mm<ALG_BOOL>(h, A, X, ldx, ncol, Y, ldy, accumulate, s);
    case ALG_MULTPATH: return launch_mm<ALG_MULTPATH>(h, A, X, ldx, ncol, Y, ldy, accumulate, s);
    default: return STC_ERR_ALGEBRA;
    }
}
