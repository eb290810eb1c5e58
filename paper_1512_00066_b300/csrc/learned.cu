// Learned output sizing for SpGEMM: per-row features, a small perceptron that
// predicts log2(1 + nnz(C_i)), and its training kernels (forward, backward, Adam).
//
// Features of output row i (67 values, stored with one zero of padding):
//   f0 = log2(1 + ub_i), ub_i = sum over stored k of row i of A of nnz(B_k)
//   f1 = log2(1 + nnz(A_i)),  f2 = log2(1 + max over those k of nnz(B_k))
//   f3+2b, f4+2b: bucket b < 32 of a one-permutation min-hash of the union of the
//   column sets of those B rows (SplitMix64 of the column id; bucket = top 5 bits,
//   key = low 32 bits): (min key) / 2^32 and 0, or 1 and 1 for an empty bucket.
// The min-hash of a union is the bucket-wise minimum of the parts' min-hashes, so
// a sketch per B row is computed once and row i merges nnz(A_i) of them.
//
// Perceptron 67 -> 64 -> 64 -> 1 with ReLU.  Weights are kept in fp32 (the
// trained master copy, layout W1[64][67], b1[64], W2[64][64], b2[64], w3[64], b3)
// and rounded to bf16 when used; all sums are fp32.
#include <cuda_bf16.h>

#include <cmath>
#include <random>
#include <vector>

#include <algorithm>

#include <cstdio>
#include <cstring>

#include "stc_internal.cuh"

namespace {

constexpr int NF = STC_MLP_INPUTS;     // 67
constexpr int NFP = STC_MLP_FEAT_STRIDE;  // 68
constexpr int NH = STC_MLP_HIDDEN;     // 64
constexpr int NW = STC_MLP_NUM_WEIGHTS;
constexpr int OFF_B1 = NH * NF;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH;
constexpr unsigned long long EMPTY = 1ull << 32;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// sketch[k][b] = min over columns j of B_k in bucket b of the low 32 bits of
// splitmix64(j), or 2^32 when the bucket is empty.  One warp per row: 32-bit
// minima in shared memory, the buckets hit kept as a per-lane mask and OR-reduced
// over the warp at the end.
__global__ void __launch_bounds__(256) k_sketch_rows(int64_t K, int64_t nnzB, const int64_t* __restrict__ b_ptr,
                                                     const int32_t* __restrict__ b_col,
                                                     unsigned long long* __restrict__ sketch) {
    __shared__ unsigned s[8][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t k = warp; k < K; k += nwarps) {
        s[wl][lane] = 0xFFFFFFFFu;
        __syncwarp();
        int64_t lo, hi;
        row_range(b_ptr, k, nnzB, lo, hi);
        unsigned hit = 0u;
        for (int64_t p = lo + lane; p < hi; p += 32) {
            const unsigned long long h = splitmix64((unsigned long long)(unsigned)b_col[p]);
            const unsigned b = unsigned(h >> 59), key = unsigned(h & 0xFFFFFFFFull);
            hit |= 1u << b;
            if (key < s[wl][b]) atomicMin(&s[wl][b], key);
        }
        hit = __reduce_or_sync(0xffffffffu, hit);
        __syncwarp();
        sketch[k * 32 + lane] = ((hit >> lane) & 1u) ? (unsigned long long)s[wl][lane] : EMPTY;
        __syncwarp();
    }
}

// Features of rows [0, nA) of A B (one warp per row; lane b merges bucket b).
__global__ void __launch_bounds__(256) k_features(int64_t nA, int64_t K, int64_t nnzA, const int64_t* __restrict__ a_ptr,
                                                  const int32_t* __restrict__ a_col, int64_t nnzB,
                                                  const int64_t* __restrict__ b_ptr,
                                                  const unsigned long long* __restrict__ sketch,
                                                  float* __restrict__ feat) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t i = warp; i < nA; i += nwarps) {
        int64_t lo, hi;
        row_range(a_ptr, i, nnzA, lo, hi);
        int64_t ub = 0, mx = 0;
        for (int64_t p = lo + lane; p < hi; p += 32) {
            const int32_t k = a_col[p];
            if ((uint64_t)k >= (uint64_t)K) continue;
            int64_t bl, bh;
            row_range(b_ptr, k, nnzB, bl, bh);
            ub += bh - bl;
            mx = max(mx, bh - bl);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ub += __shfl_down_sync(0xffffffffu, ub, o);
            mx = max(mx, (int64_t)__shfl_down_sync(0xffffffffu, mx, o));
        }
        // bucket-wise minimum over the row's B sketches: 32 entries of A at a time
        // (lane j reads entry j), then eight sketch loads in flight per lane
        unsigned long long m = EMPTY;
        for (int64_t p0 = lo; p0 < hi; p0 += 32) {
            const int64_t p = p0 + lane;
            int32_t kl = -1;
            if (p < hi) {
                const int32_t k = a_col[p];
                if ((uint64_t)k < (uint64_t)K) kl = k;
            }
            const int nk = int(hi - p0 < 32 ? hi - p0 : 32);
            for (int t0 = 0; t0 < nk; t0 += 8) {
                unsigned long long v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = __shfl_sync(0xffffffffu, kl, (t0 + u) & 31);
                    v[u] = (t0 + u < nk && k >= 0) ? sketch[int64_t(k) * 32 + lane] : EMPTY;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) m = v[u] < m ? v[u] : m;
            }
        }
        float* f = feat + i * NFP;
        if (lane == 0) {
            f[0] = log2f(1.0f + float(ub));
            f[1] = log2f(1.0f + float(hi - lo));
            f[2] = log2f(1.0f + float(mx));
            f[NFP - 1] = 0.0f;
        }
        const bool empty = m == EMPTY;
        f[3 + 2 * lane] = empty ? 1.0f : float(double(m) * (1.0 / 4294967296.0));
        f[4 + 2 * lane] = empty ? 1.0f : 0.0f;
    }
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// bf16-rounded copy of the weights in shared memory (NW floats).
__device__ __forceinline__ void load_weights(const float* __restrict__ w, float* sw) {
    for (int k = threadIdx.x; k < NW; k += blockDim.x) sw[k] = bf16r(w[k]);
    __syncthreads();
}

// y[r] = MLP(feat[r]); one thread per row, weights broadcast from shared memory.
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ w, const float* __restrict__ feat,
                                                     int64_t n, float* __restrict__ y) {
    extern __shared__ float sw[];
    load_weights(w, sw);
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
        const float* x = feat + r * NFP;
        float h1[NH];
#pragma unroll
        for (int o = 0; o < NH; ++o) h1[o] = sw[OFF_B1 + o];
        for (int i = 0; i < NF; ++i) {
            const float xi = x[i];
#pragma unroll
            for (int o = 0; o < NH; ++o) h1[o] = fmaf(sw[o * NF + i], xi, h1[o]);
        }
#pragma unroll
        for (int o = 0; o < NH; ++o) h1[o] = fmaxf(h1[o], 0.0f);
        float out = sw[OFF_B3];
        for (int o = 0; o < NH; ++o) {
            float a = sw[OFF_B2 + o];
#pragma unroll
            for (int j = 0; j < NH; ++j) a = fmaf(sw[OFF_W2 + o * NH + j], h1[j], a);
            out = fmaf(sw[OFF_W3 + o], fmaxf(a, 0.0f), out);
        }
        y[r] = out;
    }
}

constexpr int GR = 64;  // rows per block of the gradient kernel

// Accumulate into grad (fp32, NW) the gradient of sum_r (y_r - t_r)^2 / scale over
// rows [0, n) (index list `idx` or identity), and the loss sum into *loss.
__global__ void __launch_bounds__(GR) k_mlp_grad(const float* __restrict__ w, const float* __restrict__ feat,
                                                 const float* __restrict__ target, const int32_t* __restrict__ idx,
                                                 int64_t n, float scale, float* __restrict__ grad,
                                                 float* __restrict__ loss) {
    extern __shared__ float smem[];
    float* sw = smem;                 // NW
    float* X = sw + NW + 3;           // [GR][NF]
    float* H1 = X + GR * NF;          // [GR][NH] activations, then their gradients
    float* H2 = H1 + GR * NH;         // [GR][NH]
    float* D2 = H2 + GR * NH;         // [GR][NH]
    float* DY = D2 + GR * NH;         // [GR]
    load_weights(w, sw);
    const int t = threadIdx.x;
    for (int64_t base = int64_t(blockIdx.x) * GR; base < n; base += int64_t(gridDim.x) * GR) {
        const int64_t r = base + t;
        const bool valid = r < n;
        const int64_t row = valid ? (idx ? int64_t(idx[r]) : r) : 0;
        // forward for this thread's row
        for (int i = 0; i < NF; ++i) X[t * NF + i] = valid ? feat[row * NFP + i] : 0.0f;
        float out = sw[OFF_B3];
        for (int o = 0; o < NH; ++o) {
            float a = sw[OFF_B1 + o];
            for (int i = 0; i < NF; ++i) a = fmaf(sw[o * NF + i], X[t * NF + i], a);
            H1[t * NH + o] = fmaxf(a, 0.0f);
        }
        for (int o = 0; o < NH; ++o) {
            float a = sw[OFF_B2 + o];
            for (int j = 0; j < NH; ++j) a = fmaf(sw[OFF_W2 + o * NH + j], H1[t * NH + j], a);
            H2[t * NH + o] = fmaxf(a, 0.0f);
            out = fmaf(sw[OFF_W3 + o], H2[t * NH + o], out);
        }
        const float e = valid ? out - target[row] : 0.0f;
        const float dy = 2.0f * e / scale;
        DY[t] = dy;
        if (valid) atomicAdd(loss, e * e);
        // dL/dh2 (pre-activation) and dL/dh1 (pre-activation) for this row
        for (int o = 0; o < NH; ++o) D2[t * NH + o] = H2[t * NH + o] > 0.0f ? dy * sw[OFF_W3 + o] : 0.0f;
        __syncthreads();
        // weight gradients of the output and second layers (need H1, H2 before reuse)
        for (int o = t; o < NH; o += GR) {
            float g3 = 0.0f, gb2 = 0.0f;
            for (int q = 0; q < GR; ++q) {
                g3 = fmaf(DY[q], H2[q * NH + o], g3);
                gb2 += D2[q * NH + o];
            }
            atomicAdd(&grad[OFF_W3 + o], g3);
            atomicAdd(&grad[OFF_B2 + o], gb2);
        }
        if (t == 0) {
            float g = 0.0f;
            for (int q = 0; q < GR; ++q) g += DY[q];
            atomicAdd(&grad[OFF_B3], g);
        }
        for (int e2 = t; e2 < NH * NH; e2 += GR) {
            const int o = e2 / NH, j = e2 - o * NH;
            float g = 0.0f;
            for (int q = 0; q < GR; ++q) g = fmaf(D2[q * NH + o], H1[q * NH + j], g);
            atomicAdd(&grad[OFF_W2 + e2], g);
        }
        __syncthreads();
        // dL/dh1 pre-activation into H1 (in place: the gate is h1 > 0)
        for (int j = 0; j < NH; ++j) {
            float a = 0.0f;
            for (int o = 0; o < NH; ++o) a = fmaf(sw[OFF_W2 + o * NH + j], D2[t * NH + o], a);
            H1[t * NH + j] = H1[t * NH + j] > 0.0f ? a : 0.0f;
        }
        __syncthreads();
        for (int o = t; o < NH; o += GR) {
            float gb1 = 0.0f;
            for (int q = 0; q < GR; ++q) gb1 += H1[q * NH + o];
            atomicAdd(&grad[OFF_B1 + o], gb1);
        }
        for (int e1 = t; e1 < NH * NF; e1 += GR) {
            const int o = e1 / NF, i = e1 - o * NF;
            float g = 0.0f;
            for (int q = 0; q < GR; ++q) g = fmaf(H1[q * NH + o], X[q * NF + i], g);
            atomicAdd(&grad[e1], g);
        }
        __syncthreads();
    }
}

// Adam step on the fp32 master weights; the gradient buffer is cleared.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, float* __restrict__ grad,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NW; k += gridDim.x * blockDim.x) {
        const float g = grad[k];
        grad[k] = 0.0f;
        const float mk = b1 * m[k] + (1.0f - b1) * g;
        const float vk = b2 * v[k] + (1.0f - b2) * g * g;
        m[k] = mk;
        v[k] = vk;
        w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

// target[i] = log2(1 + cnt[i]): the quantity the model predicts, from the exact
// row counts of the symbolic phase.
__global__ void k_log2_targets(int64_t n, const int64_t* __restrict__ cnt, float* __restrict__ target) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        target[i] = float(log2(1.0 + double(cnt[i])));
}

// 64-bit FNV-1a over a byte string (Fowler, Noll and Vo's published constants):
// the integrity check of a saved model file.
uint64_t fnv1a64(const unsigned char* p, size_t n) {
    uint64_t x = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        x ^= p[i];
        x *= 0x100000001b3ull;
    }
    return x;
}

struct ModelHeader {
    char magic[8];        // "STCMLP1" and a terminating zero
    int32_t inputs, hidden, nweights, reserved;
    uint64_t checksum;    // FNV-1a of the nweights little-endian fp32 values
};
static_assert(sizeof(ModelHeader) == 32, "model file header layout");

size_t grad_smem() { return sizeof(float) * (size_t(NW) + 3 + size_t(GR) * NF + 3 * size_t(GR) * NH + GR); }

}  // namespace

stc_status stc_features_impl(stc_handle* h, StcScratch& sc, const stc_csr* A, const stc_csr* B, float* feat,
                             stc_stream s) {
    const int64_t K = B->nrows;
    unsigned long long* sk = sc.get<unsigned long long>(size_t(K > 0 ? K : 1) * 32);
    if (!sk) return STC_ERR_OOM;
    if (K > 0) {
        int64_t blocks = (K * 32 + 255) / 256;
        if (blocks > int64_t(h->num_sms) * 32) blocks = int64_t(h->num_sms) * 32;
        k_sketch_rows<<<unsigned(blocks), 256, 0, s>>>(K, B->nnz, B->rowptr, B->col, sk);
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    if (A->nrows > 0) {
        int64_t blocks = (A->nrows * 32 + 255) / 256;
        if (blocks > int64_t(h->num_sms) * 32) blocks = int64_t(h->num_sms) * 32;
        k_features<<<unsigned(blocks), 256, 0, s>>>(A->nrows, A->ncols, A->nnz, A->rowptr, A->col, B->nnz, B->rowptr,
                                                    sk, feat);
        STC_LAUNCH_CHECK();
        stc_count(h);
    }
    return STC_OK;
}

stc_status stc_mlp_forward_impl(stc_handle* h, const float* w, const float* feat, int64_t n, float* y,
                                stc_stream s) {
    if (n <= 0) return STC_OK;
    const size_t smem = sizeof(float) * NW;
    STC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int64_t blocks = (n + 127) / 128;
    if (blocks > int64_t(h->num_sms) * 8) blocks = int64_t(h->num_sms) * 8;
    k_mlp_forward<<<unsigned(blocks), 128, smem, s>>>(w, feat, n, y);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

stc_status stc_mlp_grad_impl(stc_handle* h, const float* w, const float* feat, const float* target,
                             const int32_t* idx, int64_t n, float scale, float* grad, float* loss, stc_stream s) {
    if (n <= 0) return STC_OK;
    const size_t smem = grad_smem();
    STC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int64_t blocks = (n + GR - 1) / GR;
    if (blocks > int64_t(h->num_sms) * 2) blocks = int64_t(h->num_sms) * 2;
    k_mlp_grad<<<unsigned(blocks), GR, smem, s>>>(w, feat, target, idx, n, scale, grad, loss);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

stc_status stc_mlp_adam_impl(stc_handle* h, float* w, float* m, float* v, float* grad, int64_t step, float lr,
                             stc_stream s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, float(step)), c2 = 1.0f - powf(b2, float(step));
    k_adam<<<(NW + 255) / 256, 256, 0, s>>>(w, m, v, grad, lr, b1, b2, eps, c1, c2);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

// ------------------------------------------------------------------- C ABI

extern "C" stc_status stc_row_features(stc_handle* h, const stc_csr* A, const stc_csr* B, float* feat,
                                       stc_stream stream) {
    if (!h || !feat) return STC_ERR_INVALID_ARG;
    stc_csr a = *A, b = *B;
    if (!a.val) a.val = a.col;  // values are not read
    if (!b.val) b.val = b.col;
    stc_status st = stc_check_csr_host(&a);
    if (st != STC_OK) return st;
    if ((st = stc_check_csr_host(&b)) != STC_OK) return st;
    if (A->ncols != B->nrows) return STC_ERR_SHAPE;
    StcScratch sc(h, stream);
    return stc_features_impl(h, sc, A, B, feat, stream);
}

extern "C" stc_status stc_mlp_forward(stc_handle* h, const float* weights, const float* feat, int64_t n, float* y,
                                      stc_stream stream) {
    if (!h || !weights || n < 0 || (n > 0 && (!feat || !y))) return STC_ERR_INVALID_ARG;
    return stc_mlp_forward_impl(h, weights, feat, n, y, stream);
}

extern "C" stc_status stc_mlp_grad(stc_handle* h, const float* weights, const float* feat, const float* target,
                                   const int32_t* idx, int64_t n, float scale, float* grad, float* loss,
                                   stc_stream stream) {
    if (!h || !weights || !grad || !loss || n < 0 || !(scale > 0.0f) || (n > 0 && (!feat || !target)))
        return STC_ERR_INVALID_ARG;
    return stc_mlp_grad_impl(h, weights, feat, target, idx, n, scale, grad, loss, stream);
}

extern "C" stc_status stc_mlp_adam(stc_handle* h, float* weights, float* m, float* v, float* grad, int64_t step,
                                   float lr, stc_stream stream) {
    if (!h || !weights || !m || !v || !grad || step < 1) return STC_ERR_INVALID_ARG;
    return stc_mlp_adam_impl(h, weights, m, v, grad, step, lr, stream);
}

extern "C" stc_status stc_mlp_init(float* weights, uint64_t seed, stc_stream stream) {
    if (!weights) return STC_ERR_INVALID_ARG;
    std::vector<float> w(NW, 0.0f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int rows, int cols) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / cols));
        for (int k = 0; k < rows * cols; ++k) w[off + k] = float(nd(rng));
    };
    fill(0, NH, NF);
    fill(OFF_W2, NH, NH);
    fill(OFF_W3, 1, NH);
    STC_CUDA_TRY(cudaMemcpyAsync(weights, w.data(), sizeof(float) * NW, cudaMemcpyHostToDevice, stream));
    STC_CUDA_TRY(cudaStreamSynchronize(stream));
    return STC_OK;
}

extern "C" stc_status stc_mlp_train(stc_handle* h, float* weights, const float* feat, const float* target, int64_t n,
                                    int32_t batch, int32_t epochs, float lr, uint64_t seed, float* loss_out,
                                    stc_stream s) {
    if (!h || !weights || !feat || !target || n <= 0 || n >= INT32_MAX || batch < 1 || epochs < 0)
        return STC_ERR_INVALID_ARG;
    StcScratch sc(h, s);
    float* m = sc.get<float>(NW);
    float* v = sc.get<float>(NW);
    float* grad = sc.get<float>(NW);
    float* loss = sc.get<float>(1);
    int32_t* idx = sc.get<int32_t>(size_t(n));
    if (sc.failed) return STC_ERR_OOM;
    STC_CUDA_TRY(cudaMemsetAsync(m, 0, sizeof(float) * NW, s));
    STC_CUDA_TRY(cudaMemsetAsync(v, 0, sizeof(float) * NW, s));
    STC_CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * NW, s));
    std::vector<int32_t> perm(static_cast<size_t>(n));
    for (int64_t i = 0; i < n; ++i) perm[size_t(i)] = int32_t(i);
    std::mt19937_64 rng(seed);
    int64_t step = 0;
    stc_status st;
    for (int e = 0; e < epochs; ++e) {
        std::shuffle(perm.begin(), perm.end(), rng);
        STC_CUDA_TRY(cudaMemcpyAsync(idx, perm.data(), sizeof(int32_t) * size_t(n), cudaMemcpyHostToDevice, s));
        STC_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s));
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t nb = n - b0 < batch ? n - b0 : batch;
            if ((st = stc_mlp_grad_impl(h, weights, feat, target, idx + b0, nb, float(nb), grad, loss, s)) != STC_OK)
                return st;
            if ((st = stc_mlp_adam_impl(h, weights, m, v, grad, ++step, lr, s)) != STC_OK) return st;
        }
        float lh = 0.0f;
        STC_CUDA_TRY(cudaMemcpyAsync(&lh, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        STC_CUDA_TRY(cudaStreamSynchronize(s));
        if (loss_out) loss_out[e] = lh / float(n);
    }
    STC_CUDA_TRY(cudaStreamSynchronize(s));
    return STC_OK;
}

extern "C" stc_status stc_row_counts(stc_handle* h, const stc_csr* A, const stc_csr* B, int64_t* counts,
                                     const stc_opts* opts, stc_stream stream) {
    if (!h || !A || !B || (A->nrows > 0 && !counts)) return STC_ERR_INVALID_ARG;
    stc_csr a = *A, b = *B;
    if (!a.val) a.val = a.col;  // values are not read
    if (!b.val) b.val = b.col;
    stc_status st = stc_check_csr_host(&a);
    if (st != STC_OK) return st;
    if ((st = stc_check_csr_host(&b)) != STC_OK) return st;
    if (A->ncols != B->nrows) return STC_ERR_SHAPE;
    if ((st = stc_row_counts_impl(h, &a, &b, counts, opts, stream)) != STC_OK) return st;
    return stc_check_device_status(h, stream);
}

extern "C" stc_status stc_training_rows(stc_handle* h, const stc_csr* A, const stc_csr* B, float* feat,
                                        float* target, stc_stream stream) {
    if (!h || !A || !B || (A->nrows > 0 && (!feat || !target))) return STC_ERR_INVALID_ARG;
    stc_csr a = *A, b = *B;
    if (!a.val) a.val = a.col;
    if (!b.val) b.val = b.col;
    stc_status st = stc_check_csr_host(&a);
    if (st != STC_OK) return st;
    if ((st = stc_check_csr_host(&b)) != STC_OK) return st;
    if (A->ncols != B->nrows) return STC_ERR_SHAPE;
    if (A->nrows == 0) return STC_OK;
    StcScratch sc(h, stream);
    int64_t* cnt = sc.get<int64_t>(size_t(A->nrows));
    if (!cnt) return STC_ERR_OOM;
    if ((st = stc_row_counts_impl(h, &a, &b, cnt, nullptr, stream)) != STC_OK) return st;
    if ((st = stc_features_impl(h, sc, &a, &b, feat, stream)) != STC_OK) return st;
    int64_t blocks = (A->nrows + 255) / 256;
    if (blocks > int64_t(h->num_sms) * 8) blocks = int64_t(h->num_sms) * 8;
    k_log2_targets<<<unsigned(blocks), 256, 0, stream>>>(A->nrows, cnt, target);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return stc_check_device_status(h, stream);
}

extern "C" stc_status stc_model_save(const char* path, const float* weights, stc_stream stream) {
    if (!path || !weights) return STC_ERR_INVALID_ARG;
    std::vector<float> w(NW);
    STC_CUDA_TRY(cudaMemcpyAsync(w.data(), weights, sizeof(float) * NW, cudaMemcpyDeviceToHost, stream));
    STC_CUDA_TRY(cudaStreamSynchronize(stream));
    ModelHeader hd{};
    memcpy(hd.magic, "STCMLP1", 8);
    hd.inputs = NF;
    hd.hidden = NH;
    hd.nweights = NW;
    hd.checksum = fnv1a64(reinterpret_cast<const unsigned char*>(w.data()), sizeof(float) * NW);
    FILE* f = fopen(path, "wb");
    if (!f) return STC_ERR_INVALID_ARG;
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(w.data(), sizeof(float), NW, f) == size_t(NW);
    ok = (fclose(f) == 0) && ok;
    return ok ? STC_OK : STC_ERR_INVALID_ARG;
}

extern "C" stc_status stc_model_load(const char* path, float* weights, stc_stream stream) {
    if (!path || !weights) return STC_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return STC_ERR_INVALID_ARG;
    ModelHeader hd{};
    std::vector<float> w(NW);
    bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, "STCMLP1", 8) == 0 && hd.inputs == NF &&
              hd.hidden == NH && hd.nweights == NW && fread(w.data(), sizeof(float), NW, f) == size_t(NW);
    unsigned char extra;
    ok = ok && fread(&extra, 1, 1, f) == 0;  // nothing after the weights
    fclose(f);
    if (!ok || fnv1a64(reinterpret_cast<const unsigned char*>(w.data()), sizeof(float) * NW) != hd.checksum)
        return STC_ERR_INVALID_ARG;
    STC_CUDA_TRY(cudaMemcpyAsync(weights, w.data(), sizeof(float) * NW, cudaMemcpyHostToDevice, stream));
    STC_CUDA_TRY(cudaStreamSynchronize(stream));
    return STC_OK;
}
