// Learned flip proposal: the scoring MLP 32 -> 128 -> 128 -> 1 (ReLU) on the
// 5th-generation tensor cores.  BF16 operands in shared memory, FP32
// accumulation in tensor memory, one elected thread issues the MMAs
// (tcgen05.mma, cta_group::1, M = N = 128, K = 16 per instruction), completion
// is signalled through an mbarrier, and the epilogue reads the accumulator
// rows with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows).
//
// Parameter blob (device, see include/tfg.h): W1 bf16 [32][128], W2 bf16
// [128][128] (row = input unit), b1, b2, w3 f32 [128] each, b3 f32.
#include <cstdint>
#include <cuda_bf16.h>

#include "tc_common.cuh"
#include "tfg_internal.h"

namespace tfg {
namespace {

constexpr int kIn = 32, kHid = 128, kTile = 128;
constexpr uint32_t kParamW1 = 0;
constexpr uint32_t kParamW2 = kParamW1 + kIn * kHid * 2;
constexpr uint32_t kParamB1 = kParamW2 + kHid * kHid * 2;
constexpr uint32_t kParamB2 = kParamB1 + kHid * 4;
constexpr uint32_t kParamW3 = kParamB2 + kHid * 4;
constexpr uint32_t kParamB3 = kParamW3 + kHid * 4;
constexpr uint32_t kParamBytes = kParamB3 + 16;

constexpr uint32_t kSmemX = 0;                       // A: tile x 32   (8 KB)
constexpr uint32_t kSmemW1T = kSmemX + kTile * kIn * 2;   // B: 128 x 32 (8 KB)
constexpr uint32_t kSmemH1 = kSmemW1T + kHid * kIn * 2;   // A: tile x 128 (32 KB)
constexpr uint32_t kSmemW2T = kSmemH1 + kTile * kHid * 2; // B: 128 x 128 (32 KB)
constexpr uint32_t kSmemVec = kSmemW2T + kHid * kHid * 2; // b1, b2, w3 (1.5 KB)
constexpr uint32_t kScoreSmem = kSmemVec + 3 * kHid * 4;

__device__ __forceinline__ void store_row_bf16(uint8_t *base, int row, int col0, int K, const float *v8) {
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = __float2bfloat16_rn(v8[q]);
    *reinterpret_cast<uint4 *>(base + tc::kmajor_offset(row, col0, K)) = *reinterpret_cast<const uint4 *>(h);
}

__global__ void __launch_bounds__(128, 1) mlp_score_kernel(const uint8_t *__restrict__ params,
                                                            const __nv_bfloat16 *__restrict__ x, int64_t n,
                                                            float *__restrict__ out, int *__restrict__ err,
                                                            uint32_t first_limit) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int timeout;
    const int tid = threadIdx.x, warp = tid >> 5;
    uint8_t *sX = smem + kSmemX, *sW1T = smem + kSmemW1T, *sH1 = smem + kSmemH1, *sW2T = smem + kSmemW2T;
    float *sB1 = reinterpret_cast<float *>(smem + kSmemVec), *sB2 = sB1 + kHid, *sW3 = sB2 + kHid;

    // weights into the K-major operand layouts: B1 = W1^T (N = hidden, K = input),
    // B2 = W2^T (N = output unit, K = hidden)
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(params + kParamW1);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(params + kParamW2);
    for (int e = tid; e < kIn * kHid; e += blockDim.x) {
        const int i = e / kHid, h = e % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(sW1T + tc::kmajor_offset(h, i, kIn)) = W1[e];
    }
    for (int e = tid; e < kHid * kHid; e += blockDim.x) {
        const int h = e / kHid, o = e % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(sW2T + tc::kmajor_offset(o, h, kHid)) = W2[e];
    }
    for (int e = tid; e < kHid; e += blockDim.x) {
        sB1[e] = reinterpret_cast<const float *>(params + kParamB1)[e];
        sB2[e] = reinterpret_cast<const float *>(params + kParamB2)[e];
        sW3[e] = reinterpret_cast<const float *>(params + kParamW3)[e];
    }
    const float b3 = *reinterpret_cast<const float *>(params + kParamB3);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tslot), kHid);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar), 1);
        timeout = 0;
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t mb = tc::smem_u32(&mbar);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTile, kHid);
    uint32_t phase = 0;

    for (int64_t tile = blockIdx.x; tile * kTile < n; tile += gridDim.x) {
        const int64_t row = tile * kTile + tid;
        // ---- features of this row into the A operand
#pragma unroll
        for (int c = 0; c < kIn / 8; ++c) {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (row < n) v = *reinterpret_cast<const uint4 *>(x + row * kIn + c * 8);
            *reinterpret_cast<uint4 *>(sX + tc::kmajor_offset(tid, c * 8, kIn)) = v;
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
#pragma unroll
            for (int kc = 0; kc < kIn / 16; ++kc)
                tc::mma_bf16(tmem, tc::make_desc(tc::smem_u32(sX) + kc * 256, 128, (kIn / 8) * 128),
                             tc::make_desc(tc::smem_u32(sW1T) + kc * 256, 128, (kIn / 8) * 128), idesc, kc > 0);
            tc::mma_commit(mb);
        }
        // the CTA's first completion wait takes first_limit polls (the test hook), later ones the default
        bool ok = tc::mbar_wait(mb, phase, tile == blockIdx.x ? first_limit : tc::kWaitLimit);
        if (__syncthreads_or(!ok)) { if (tid == 0) timeout = 1; break; }
        phase ^= 1;
        tc::fence_after_sync();
        // ---- layer-1 epilogue: h1 = relu(z1 + b1) -> bf16 A operand of layer 2
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tlane + c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = fmaxf(v[q] + sB1[c0 + q], 0.f);
#pragma unroll
            for (int q = 0; q < 32; q += 8) store_row_bf16(sH1, tid, c0 + q, kHid, v + q);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
#pragma unroll
            for (int kc = 0; kc < kHid / 16; ++kc)
                tc::mma_bf16(tmem, tc::make_desc(tc::smem_u32(sH1) + kc * 256, 128, (kHid / 8) * 128),
                             tc::make_desc(tc::smem_u32(sW2T) + kc * 256, 128, (kHid / 8) * 128), idesc, kc > 0);
            tc::mma_commit(mb);
        }
        ok = tc::mbar_wait(mb, phase);
        if (__syncthreads_or(!ok)) { if (tid == 0) timeout = 1; break; }
        phase ^= 1;
        tc::fence_after_sync();
        // ---- layer-2 epilogue and output unit: y = w3 . relu(z2 + b2) + b3
        float y = b3;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tlane + c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) y = fmaf(fmaxf(v[q] + sB2[c0 + q], 0.f), sW3[c0 + q], y);
        }
        if (row < n) out[row] = y;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    __syncthreads();
    if (timeout) {
        // the awaited phase never completed: give the MMA still in flight one more
        // bounded wait before the accumulator is released
        tc::mbar_wait(mb, phase);
        if (tid == 0) atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kHid);
}

uint32_t g_first_wait_limit = tc::kWaitLimit;

}  // namespace

void set_first_wait_limit(int64_t polls) {
    g_first_wait_limit = (polls < 0 || polls > (int64_t)tc::kWaitLimit) ? tc::kWaitLimit : (uint32_t)polls;
}

size_t mlp_param_bytes() { return kParamBytes; }

int launch_mlp_score(const void *params, const void *x, int64_t n, float *out, int *err, cudaStream_t st) {
    if (n <= 0) return 0;
    static bool attr = [] {
        cudaFuncSetAttribute(mlp_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScoreSmem);
        return true;
    }();
    (void)attr;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int grid = (int)(tiles < 2LL * sms ? tiles : 2LL * sms);
    mlp_score_kernel<<<grid, 128, kScoreSmem, st>>>(reinterpret_cast<const uint8_t *>(params),
                                                    reinterpret_cast<const __nv_bfloat16 *>(x), n, out, err,
                                                    g_first_wait_limit);
    return 0;
}

}  // namespace tfg
