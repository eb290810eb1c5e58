// Row-size perceptron forward on the fifth-generation tensor cores (tcgen05).
//
// The model is the one of learned.cu: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3,
// 67 -> 64 -> 64 -> 1, weights rounded to bf16, sums in fp32.  Per tile of 128 rows
// the two hidden layers are two MMAs of M = 128, N = 64 with bf16 operands and fp32
// accumulators in tensor memory (TMEM); the 64 -> 1 output layer is a per-row dot
// product in the epilogue.  b1 is added by the first MMA: it is stored as column 67
// of W1 and the A operand's input 67 (the feature matrix's padding) is set to 1.
//
// Precision.  An fp32 activation x is split into hi = bf16(x) and lo = bf16(x - hi)
// and both halves are multiplied by the (exactly bf16) weights, so x is carried to
// about 16 significant bits (bf16 rounds to 8 bits, so |x - hi - lo| <= 2^-16 |x|),
// close to the CUDA-core kernel that multiplies fp32 features by bf16 weights.
//
// Shared-memory operand layout (no swizzle, K-major): an operand of R rows and K
// columns is stored as 8-row x 8-element core matrices of 128 contiguous bytes
// (row r of a core matrix at 16 r), the core matrices of one 8-row group
// consecutive along K.  In the matrix descriptor the leading byte offset (next core
// matrix along K) is 128 and the stride byte offset (next 8-row group) is
// 128 * K / 8.
//
// One CTA of 512 threads per SM runs four independent tile pipelines ("slots") of
// 128 threads each: slot s owns an A region in shared memory, TMEM columns
// [128 s, 128 s + 128), an mbarrier and named barrier 1 + s; thread t of a slot
// owns tile row t (= TMEM lane t).  A slot converts its tile's features into its A
// region, its thread 0 issues the MMAs and commits them to the slot's mbarrier,
// and the slot's loads of its next tile are in flight while it waits, so four
// tiles (139 KB of features) are loading per SM.  Every wait is a bounded poll; one
// that runs out sets STC_FLAG_TIMEOUT, waits (bounded) once more for the MMAs in
// flight, and the slot stops; the CTA then frees its TMEM and ends.
#include <cuda_bf16.h>

#include "stc_internal.cuh"

namespace {

constexpr int NF = STC_MLP_INPUTS;        // 67
constexpr int NFP = STC_MLP_FEAT_STRIDE;  // 68
constexpr int NH = STC_MLP_HIDDEN;        // 64
constexpr int OFF_B1 = NH * NF;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH;

constexpr int TM = 128;                 // rows per tile (MMA M)
constexpr int K1 = 80;                  // layer-1 K: 67 inputs padded to 5 MMA K-steps of 16
constexpr int K1C = K1 / 8;             // core matrices along K1
constexpr int K2C = NH / 8;             // core matrices along K2 = 64
constexpr int SLOTS = 4;                // independent tile pipelines per CTA
constexpr int SLOT_NT = 128;            // threads of a slot: thread t owns tile row t = TMEM lane t
constexpr int TC_NT = SLOTS * SLOT_NT;  // one CTA per SM
constexpr uint32_t TMEM_COLS = 512;     // slot s: D1 in columns [128 s, 128 s + 64), D2 in [128 s + 64, 128 s + 128)

// shared-memory byte offsets: weights (B operands) and vectors shared by the slots,
// then one A region per slot (X hi and lo; later H1 hi and lo)
constexpr uint32_t SM_W1 = 0;                                   // [8][K1C] core matrices
constexpr uint32_t SM_W2 = SM_W1 + (NH / 8) * K1C * 128;        // 10240: [8][K2C]
constexpr uint32_t SM_VEC = SM_W2 + (NH / 8) * K2C * 128;       // 18432: b2, w3 (fp32), b3
constexpr uint32_t SM_BAR = SM_VEC + (3 * NH + 4) * 4;          // one mbarrier per slot
constexpr uint32_t SM_TADDR = SM_BAR + 8 * SLOTS;               // TMEM base address
constexpr uint32_t SM_SLOT = 20480;                              // first slot region
constexpr uint32_t A_LO = (TM / 8) * K1C * 128;                 // 20480: X lo after X hi
constexpr uint32_t H_LO = (TM / 8) * K2C * 128;                 // 16384: H1 lo after H1 hi
constexpr uint32_t SLOT_BYTES = 2 * A_LO;                        // 40960
constexpr uint32_t SM_TOTAL = SM_SLOT + SLOTS * SLOT_BYTES;      // 184320
static_assert(SM_TADDR + 8 <= SM_SLOT, "header overlaps the slot regions");
static_assert(2 * H_LO <= SLOT_BYTES, "H1 must fit in the X region");
static_assert(SM_BAR % 8 == 0, "mbarrier alignment");

// instruction descriptor of kind::f16: fp32 D (bits 4-5 = 1), bf16 A and B
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(NH >> 3) << 17) | (uint32_t(TM >> 4) << 24);

constexpr int WAIT_POLLS = 1 << 22;  // x 64 ns sleep: about a quarter of a second

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// matrix descriptor: start address, leading and stride byte offsets (all >> 4),
// the fixed value 1 at bits 46-48, base offset 0, no swizzle
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// barrier of one slot's 128 threads (named barrier 1 + slot); returns whether
// `pred` holds in all of them
__device__ __forceinline__ bool slot_sync_and(int slot, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"(uint32_t(pred)), "r"(1 + slot), "r"(SLOT_NT)
        : "memory");
    return r != 0;
}

// bounded wait for the completion of the mbarrier phase with the given parity
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < WAIT_POLLS; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}

// the same wait polled by lane 0 of the warp alone (an mbarrier read by 32 lanes
// costs 32 shared-memory wavefronts), its result broadcast to the warp
__device__ __forceinline__ bool warp_bar_wait(uint32_t bar, uint32_t parity) {
    uint32_t got = 0;
    if ((threadIdx.x & 31) == 0) got = bar_wait(bar, parity);
    got = __shfl_sync(0xffffffffu, got, 0);
    __syncwarp();
    return got != 0;
}

// 16 consecutive fp32 columns of this thread's TMEM lane (32x32b shape: warp w
// reads lanes [32 (w % 4), 32 (w % 4) + 32)); the wait is in the same statement so
// that no register is read before the load has landed
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);  // a in the low half
    return *reinterpret_cast<const uint32_t*>(&p);
}

// hi/lo bf16 split of 8 fp32 values, stored as one 16-byte core-matrix row in each
// of the two operand copies
__device__ __forceinline__ void store_split8(unsigned char* sm, uint32_t off_hi, uint32_t off_lo, const float* x) {
    float hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        hi[q] = __bfloat162float(__float2bfloat16_rn(x[q]));
        lo[q] = x[q] - hi[q];
    }
    *reinterpret_cast<uint4*>(sm + off_hi) =
        make_uint4(pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), pack_bf16(hi[4], hi[5]), pack_bf16(hi[6], hi[7]));
    *reinterpret_cast<uint4*>(sm + off_lo) =
        make_uint4(pack_bf16(lo[0], lo[1]), pack_bf16(lo[2], lo[3]), pack_bf16(lo[4], lo[5]), pack_bf16(lo[6], lo[7]));
}

__device__ __forceinline__ uint32_t cm_off(int row, int kc, int nkc) {
    return uint32_t(((row >> 3) * nkc + kc) * 128 + (row & 7) * 16);
}

constexpr int ITEMS = TM * K1C / SLOT_NT;  // (row, core column) items of a tile per thread: 10

// Item j of thread lt (warp w = lt / 32, lane l): 16-row block b = 2 w + j / 5 and
// kind k = j % 5 -- k < 4: row 16 b + 8 (k / 2) + l / 4, core column 4 (k % 2) + l % 4;
// k = 4: row 16 b + l / 2, core column 8 + l % 2.  A warp's 16-byte stores then
// cover 8 distinct values of row % 8 (the bank group of a core-matrix row), four
// lanes each, and its loads read whole 128-byte lines of 8 rows.
__device__ __forceinline__ void item_of(int lt, int j, int& row, int& kc) {
    const int w = lt >> 5, l = lt & 31, b = 2 * w + j / 5, k = j % 5;
    if (k < 4) {
        row = 16 * b + 8 * (k >> 1) + (l >> 2);
        kc = 4 * (k & 1) + (l & 3);
    } else {
        row = 16 * b + (l >> 1);
        kc = 8 + (l & 1);
    }
}

// this thread's items of a tile's features; rows past n and inputs past the row's
// 68 floats read 0
__device__ __forceinline__ void load_x(const float* __restrict__ feat, int64_t n, int64_t tile, int64_t ntiles,
                                       int lt, float4 (&xv)[ITEMS][2]) {
    const int64_t r0 = tile * TM;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        int row, kc;
        item_of(lt, j, row, kc);
        const int64_t r = r0 + row;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (tile < ntiles && r < n && kc <= 8) {
            const float4* src = reinterpret_cast<const float4*>(feat + r * NFP + kc * 8);
            a = src[0];              // inputs 8 kc .. 8 kc + 3 (64..67 for kc = 8)
            if (kc < 8) b = src[1];  // a row holds NFP = 68 floats: no second half at kc = 8
            else a.w = 1.0f;         // input 67 (the padding) is the constant 1 that adds b1
        }
        xv[j][0] = a;
        xv[j][1] = b;
    }
}

__global__ void __launch_bounds__(TC_NT, 1) k_mlp_forward_tc(const float* __restrict__ w,
                                                             const float* __restrict__ feat, int64_t n,
                                                             float* __restrict__ y, int* __restrict__ flags) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int t = threadIdx.x, warp = t >> 5;
    const int slot = t / SLOT_NT, lt = t - slot * SLOT_NT;
    float* vec = reinterpret_cast<float*>(sm + SM_VEC);  // b2[64], w3[64], b3 (b1 is column 67 of W1)
    const float4* vec4 = reinterpret_cast<const float4*>(sm + SM_VEC);
    const uint32_t bar = smem_u32(sm + SM_BAR + 8 * slot);

    // weights, bf16-rounded, into the B operands; biases and w3 as fp32
    for (int e = t; e < NH * K1; e += TC_NT) {
        const int o = e / K1, i = e - o * K1;
        // column NF (= 67) carries b1: the A operand's input 67 is the constant 1
        const float v = i < NF ? w[o * NF + i] : i == NF ? w[OFF_B1 + o] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(sm + SM_W1 + cm_off(o, i >> 3, K1C) + (i & 7) * 2) = __float2bfloat16_rn(v);
    }
    for (int e = t; e < NH * NH; e += TC_NT) {
        const int o = e / NH, j = e - o * NH;
        *reinterpret_cast<__nv_bfloat16*>(sm + SM_W2 + cm_off(o, j >> 3, K2C) + (j & 7) * 2) =
            __float2bfloat16_rn(w[OFF_W2 + e]);
    }
    for (int e = t; e < 2 * NH + 1; e += TC_NT) {
        const float v = e < NH ? w[OFF_B2 + e] : e < 2 * NH ? w[OFF_W3 + e - NH] : w[OFF_B3];
        vec[e] = __bfloat162float(__float2bfloat16_rn(v));
    }
    if (t == 0) {
        for (int q = 0; q < SLOTS; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(sm + SM_BAR + 8 * q)), "r"(1)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sm + SM_TADDR)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(sm + SM_TADDR);
    const uint32_t d1 = tbase + uint32_t(128 * slot), d2 = d1 + NH;
    const uint32_t lane_addr = uint32_t((warp & 3) * 32) << 16;  // this warp's TMEM lanes

    const uint32_t so = SM_SLOT + uint32_t(slot) * SLOT_BYTES;  // this slot's A region
    const uint32_t a_hi = smem_u32(sm + so), a_lo = a_hi + A_LO, h_hi = a_hi, h_lo = a_hi + H_LO;
    const uint32_t w1 = smem_u32(sm + SM_W1), w2 = smem_u32(sm + SM_W2);
    const int64_t ntiles = (n + TM - 1) / TM;
    const int64_t tstep = int64_t(gridDim.x) * SLOTS;
    uint32_t phase = 0;
    bool ok = true;

    float4 xv[ITEMS][2];
    load_x(feat, n, int64_t(blockIdx.x) * SLOTS + slot, ntiles, lt, xv);
    for (int64_t tile = int64_t(blockIdx.x) * SLOTS + slot; tile < ntiles && ok; tile += tstep) {
        const int64_t r0 = tile * TM;
        // 1) the tile's features (loaded during the previous tile), split, into A
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            int row, kc;
            item_of(lt, j, row, kc);
            const float x[8] = {xv[j][0].x, xv[j][0].y, xv[j][0].z, xv[j][0].w,
                                xv[j][1].x, xv[j][1].y, xv[j][1].z, xv[j][1].w};
            const uint32_t off = so + cm_off(row, kc, K1C);
            store_split8(sm, off, off + A_LO, x);
        }
        fence_async_smem();
        fence_before_sync();
        slot_sync_and(slot, true);
        fence_after_sync();
        // 2) layer 1: D1 = Xhi W1^T + Xlo W1^T
        if (lt == 0) {
#pragma unroll
            for (int ks = 0; ks < K1 / 16; ++ks) {
                const uint64_t bd = mat_desc(w1 + ks * 256, 128, K1C * 128);
                mma_bf16(d1, mat_desc(a_hi + ks * 256, 128, K1C * 128), bd, ks > 0);
                mma_bf16(d1, mat_desc(a_lo + ks * 256, 128, K1C * 128), bd, 1);
            }
            mma_commit(bar);
        }
        // the next tile's loads are in flight during this tile's MMAs and epilogues
        load_x(feat, n, tile + tstep, ntiles, lt, xv);
        bool got = warp_bar_wait(bar, phase);
        phase ^= 1;
        fence_after_sync();
        // 3) epilogue 1: H1 = relu(D1) (D1 includes b1), split, into the layer-2 A operand
        if (got) {
#pragma unroll
            for (int c = 0; c < NH / 16; ++c) {
                float v[16];
                tmem_ld16(d1 + lane_addr + c * 16, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q], 0.0f);
                store_split8(sm, so + cm_off(lt, 2 * c, K2C), so + H_LO + cm_off(lt, 2 * c, K2C), v);
                store_split8(sm, so + cm_off(lt, 2 * c + 1, K2C), so + H_LO + cm_off(lt, 2 * c + 1, K2C), v + 8);
            }
        }
        fence_async_smem();
        fence_before_sync();
        ok = slot_sync_and(slot, got);
        fence_after_sync();
        if (!ok) break;
        // 4) layer 2: D2 = H1hi W2^T + H1lo W2^T
        if (lt == 0) {
#pragma unroll
            for (int ks = 0; ks < NH / 16; ++ks) {
                const uint64_t bd = mat_desc(w2 + ks * 256, 128, K2C * 128);
                mma_bf16(d2, mat_desc(h_hi + ks * 256, 128, K2C * 128), bd, ks > 0);
                mma_bf16(d2, mat_desc(h_lo + ks * 256, 128, K2C * 128), bd, 1);
            }
            mma_commit(bar);
        }
        got = warp_bar_wait(bar, phase);
        phase ^= 1;
        fence_after_sync();
        // 5) epilogue 2: y = w3 . relu(D2 + b2) + b3
        if (got) {
            float out = vec[2 * NH];
#pragma unroll
            for (int c = 0; c < NH / 16; ++c) {
                float v[16];
                tmem_ld16(d2 + lane_addr + c * 16, v);
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const float4 b2 = vec4[c * 4 + q4], w3 = vec4[NH / 4 + c * 4 + q4];  // broadcast reads
                    out = fmaf(w3.x, fmaxf(v[4 * q4 + 0] + b2.x, 0.0f), out);
                    out = fmaf(w3.y, fmaxf(v[4 * q4 + 1] + b2.y, 0.0f), out);
                    out = fmaf(w3.z, fmaxf(v[4 * q4 + 2] + b2.z, 0.0f), out);
                    out = fmaf(w3.w, fmaxf(v[4 * q4 + 3] + b2.w, 0.0f), out);
                }
            }
            if (r0 + lt < n) y[r0 + lt] = out;
        }
        fence_before_sync();
        ok = slot_sync_and(slot, got);
        fence_after_sync();
    }
    if (!ok && lt == 0) {
        // a commit that did not arrive: report, then give the MMAs in flight one more
        // bounded wait before the tensor memory is released
        atomicOr(flags, STC_FLAG_TIMEOUT);
        bar_wait(bar, phase ^ 1);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

}  // namespace

stc_status stc_mlp_forward_tc_impl(stc_handle* h, const float* w, const float* feat, int64_t n, float* y,
                                   stc_stream s) {
    if (n <= 0) return STC_OK;
    if ((reinterpret_cast<uintptr_t>(feat) & 15u) != 0) return STC_ERR_INVALID_ARG;  // float4 row loads
    STC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SM_TOTAL)));
    // one CTA per SM (it holds all 512 TMEM columns): grid = SMs, or fewer for
    // fewer than SLOTS tiles per SM
    const int64_t ntiles = (n + TM - 1) / TM;
    int64_t grid = (ntiles + SLOTS - 1) / SLOTS;
    if (grid > h->num_sms) grid = h->num_sms;
    k_mlp_forward_tc<<<unsigned(grid), TC_NT, SM_TOTAL, s>>>(w, feat, n, y, h->d_flags);
    STC_LAUNCH_CHECK();
    stc_count(h);
    return STC_OK;
}

extern "C" stc_status stc_mlp_forward_tc(stc_handle* h, const float* weights, const float* feat, int64_t n, float* y,
                                         stc_stream stream) {
    if (!h || !weights || n < 0 || (n > 0 && (!feat || !y))) return STC_ERR_INVALID_ARG;
    return stc_mlp_forward_tc_impl(h, weights, feat, n, y, stream);
}
