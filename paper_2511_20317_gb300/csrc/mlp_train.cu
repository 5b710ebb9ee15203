// Training of the proposal MLP on the tensor cores: one fused kernel computes,
// per 128-sample tile, the forward pass, the weighted logistic loss and the
// backward pass, and accumulates the weight gradients of the CTA's tiles in
// tensor memory; an Adam kernel then updates FP32 master weights and rewrites
// the BF16 parameter blob.
//
// Products (all BF16 x BF16 -> FP32, K = 16 per tcgen05.mma):
//   Z1  = X  W1            M = sample, N = hidden, K = input
//   Z2  = H1 W2            M = sample, N = hidden, K = hidden
//   dH1 = dZ2 W2^T         M = sample, N = hidden, K = hidden
//   dW2^T += dZ2^T H1      M = hidden, N = hidden, K = sample
//   dW1^T += dZ1^T X       M = hidden, N = input,  K = sample
// The vector gradients (b1, b2, w3, b3) and the loss are FP32 warp reductions.
#include <cstdint>
#include <cuda_bf16.h>

#include "tc_common.cuh"
#include "tfg_internal.h"

namespace tfg {
namespace {

constexpr int kIn = 32, kHid = 128, kTile = 128;
constexpr int kNumParams = kIn * kHid + kHid * kHid + 3 * kHid + 1;
// parameter blob offsets (bytes), shared with the scoring kernel
constexpr uint32_t kPW1 = 0, kPW2 = kIn * kHid * 2, kPB1 = kPW2 + kHid * kHid * 2, kPB2 = kPB1 + kHid * 4,
                   kPW3 = kPB2 + kHid * 4, kPB3 = kPW3 + kHid * 4;
// FP32 parameter vector offsets (elements): W1 [32][128], W2 [128][128], b1, b2, w3, b3
constexpr int kVW1 = 0, kVW2 = kIn * kHid, kVB1 = kVW2 + kHid * kHid, kVB2 = kVB1 + kHid, kVW3 = kVB2 + kHid,
              kVB3 = kVW3 + kHid;

// shared memory regions (bytes)
constexpr int kGradPartialRows = 256;          // CTAs of a deterministic (partial-row) gradient launch, at most
constexpr uint32_t kSX = 0;                    // A  (s, i)   K = 32
constexpr uint32_t kSXT = kSX + 8192;          // B  (i, s)   K = 128
constexpr uint32_t kSW1T = kSXT + 8192;        // B  (h, i)   K = 32
constexpr uint32_t kSW2T = kSW1T + 8192;       // B  (o, h)   K = 128
constexpr uint32_t kSW2 = kSW2T + 32768;       // B  (h, o)   K = 128
constexpr uint32_t kSH1 = kSW2 + 32768;        // A  (s, h)   K = 128
constexpr uint32_t kSH1T = kSH1 + 32768;       // B  (h, s)   K = 128
constexpr uint32_t kSD2 = kSH1T + 32768;       // A  (s, o) = dZ2, then (h, s) = dZ1^T
constexpr uint32_t kSD2T = kSD2 + 32768;       // A  (o, s)   K = 128
constexpr uint32_t kSVec = kSD2T + 32768;      // b1, b2, w3, then per-warp sums gb1, gb2, gw3 [4][128], gb3, loss [4][2]
constexpr uint32_t kTrainSmem = kSVec + (3 * kHid + 3 * 4 * kHid + 8) * 4;

constexpr uint32_t kTmemCols = 512;   // [0,128) layer/ dH1 accumulator, [128,256) dW2^T, [256,288) dW1^T

__device__ __forceinline__ void st_bf16(uint8_t *base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

// Column sums of a 32 x 32 block held one row per lane: afterwards lane l
// holds the sum of column l.  Transposing butterfly: at each stage a lane
// keeps the half of its columns selected by one bit of its lane index and
// sends the other half to the partner lane (31 shuffles in total).
template <int HALF>
__device__ __forceinline__ void colsum_stage(float (&v)[32], int lane) {
    const bool up = (lane & HALF) != 0;
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
        const float send = up ? v[j] : v[j + HALF];
        const float keep = up ? v[j + HALF] : v[j];
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, HALF);
    }
}
__device__ __forceinline__ float warp_colsum32(float (&v)[32], int lane) {
    colsum_stage<16>(v, lane);
    colsum_stage<8>(v, lane);
    colsum_stage<4>(v, lane);
    colsum_stage<2>(v, lane);
    colsum_stage<1>(v, lane);
    return v[0];
}

__device__ __forceinline__ void sync_all() {
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Gradient sums: every warp keeps its own column sums (its lanes own the
// columns, so no atomics), added in warp order at the end; the CTA's totals go
// to grad by atomics (tfg_mlp_grad), or, with `partial`, to the CTA's own row
// partial[blockIdx.x][P + 1], which grad_reduce_kernel adds up in CTA order:
// the training step's gradient is then the same bits on every run.
__global__ void __launch_bounds__(128, 1) mlp_grad_kernel(const uint8_t *__restrict__ params,
                                                           const __nv_bfloat16 *__restrict__ x,
                                                           const float *__restrict__ label,
                                                           const float *__restrict__ weight, int64_t n,
                                                           float *__restrict__ grad, float *__restrict__ partial,
                                                           int *__restrict__ err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int timeout;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *sX = smem + kSX, *sXT = smem + kSXT, *sW1T = smem + kSW1T, *sW2T = smem + kSW2T, *sW2 = smem + kSW2;
    uint8_t *sH1 = smem + kSH1, *sH1T = smem + kSH1T, *sD2 = smem + kSD2, *sD2T = smem + kSD2T;
    float *sB1 = reinterpret_cast<float *>(smem + kSVec), *sB2 = sB1 + kHid, *sW3 = sB2 + kHid;
    // per-warp sums [4][128] and scalars [4][2] (gb3, loss)
    float *gB1 = sW3 + kHid, *gB2 = gB1 + 4 * kHid, *gW3 = gB2 + 4 * kHid, *gScal = gW3 + 4 * kHid;

    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(params + kPW1);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(params + kPW2);
    for (int e = tid; e < kIn * kHid; e += blockDim.x) {
        const int i = e / kHid, h = e % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(sW1T + tc::kmajor_offset(h, i, kIn)) = W1[e];
    }
    for (int e = tid; e < kHid * kHid; e += blockDim.x) {
        const int h = e / kHid, o = e % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(sW2T + tc::kmajor_offset(o, h, kHid)) = W2[e];
        *reinterpret_cast<__nv_bfloat16 *>(sW2 + tc::kmajor_offset(h, o, kHid)) = W2[e];
    }
    for (int e = tid; e < kHid; e += blockDim.x) {
        sB1[e] = reinterpret_cast<const float *>(params + kPB1)[e];
        sB2[e] = reinterpret_cast<const float *>(params + kPB2)[e];
        sW3[e] = reinterpret_cast<const float *>(params + kPW3)[e];
    }
    for (int e = tid; e < 4 * kHid; e += blockDim.x) gB1[e] = gB2[e] = gW3[e] = 0.f;
    if (tid < 8) gScal[tid] = 0.f;
    const float b3 = *reinterpret_cast<const float *>(params + kPB3);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tslot), kTmemCols);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&mbar), 1);
        timeout = 0;
    }
    sync_all();
    const uint32_t tmem = tslot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t tAcc = tmem, tDW2 = tmem + 128, tDW1 = tmem + 256;
    const uint32_t mb = tc::smem_u32(&mbar);
    constexpr uint32_t idN128 = tc::idesc_bf16_f32(128, 128), idN32 = tc::idesc_bf16_f32(128, 32);
    uint32_t phase = 0;
    bool first = true;
    float my_gb3 = 0.f, my_loss = 0.f;

#define TFG_WAIT()                                                     \
    {                                                                  \
        const bool ok_ = tc::mbar_wait(mb, phase);                     \
        if (__syncthreads_or(!ok_)) { if (tid == 0) timeout = 1; break; } \
        phase ^= 1;                                                    \
        tc::fence_after_sync();                                        \
    }

    for (int64_t tile = blockIdx.x; tile * kTile < n; tile += gridDim.x) {
        const int64_t row = tile * kTile + tid;
        const bool valid = row < n;
        // ---- inputs: X as A (s, i) and as B^T (i, s)
#pragma unroll
        for (int c = 0; c < kIn / 8; ++c) {
            uint4 v = make_uint4(0, 0, 0, 0);
            if (valid) v = *reinterpret_cast<const uint4 *>(x + row * kIn + c * 8);
            *reinterpret_cast<uint4 *>(sX + tc::kmajor_offset(tid, c * 8, kIn)) = v;
            const __nv_bfloat16 *hv = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<__nv_bfloat16 *>(sXT + tc::kmajor_offset(c * 8 + q, tid, kTile)) = hv[q];
        }
        const float lab = valid ? label[row] : 0.f;
        const float wt = valid ? weight[row] : 0.f;
        sync_all();
        if (tid == 0) {
#pragma unroll
            for (int kc = 0; kc < kIn / 16; ++kc)
                tc::mma_bf16(tAcc, tc::make_desc(tc::smem_u32(sX) + kc * 256, 128, 512),
                             tc::make_desc(tc::smem_u32(sW1T) + kc * 256, 128, 512), idN128, kc > 0);
            tc::mma_commit(mb);
        }
        TFG_WAIT();
        // ---- layer 1: h1 = relu(z1 + b1) as bf16, kept as A (s, h) and B (h, s); ReLU mask
        uint32_t mask1[4];
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tAcc + lane_base + c0, v);
            uint32_t m = 0;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const float z = v[q] + sB1[c0 + q];
                m |= (z > 0.f ? 1u : 0u) << q;
                v[q] = fmaxf(z, 0.f);
            }
            mask1[c0 / 32] = m;
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) hb[u] = __float2bfloat16_rn(v[q + u]);
                *reinterpret_cast<uint4 *>(sH1 + tc::kmajor_offset(tid, c0 + q, kHid)) =
                    *reinterpret_cast<const uint4 *>(hb);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    *reinterpret_cast<__nv_bfloat16 *>(sH1T + tc::kmajor_offset(c0 + q + u, tid, kTile)) = hb[u];
            }
        }
        sync_all();
        if (tid == 0) {
#pragma unroll
            for (int kc = 0; kc < kHid / 16; ++kc)
                tc::mma_bf16(tAcc, tc::make_desc(tc::smem_u32(sH1) + kc * 256, 128, 2048),
                             tc::make_desc(tc::smem_u32(sW2T) + kc * 256, 128, 2048), idN128, kc > 0);
            tc::mma_commit(mb);
        }
        TFG_WAIT();
        // ---- layer 2 and output: y, loss, dy
        float y = b3;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tAcc + lane_base + c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) y = fmaf(fmaxf(v[q] + sB2[c0 + q], 0.f), sW3[c0 + q], y);
        }
        const float sgn = 2.f * lab - 1.f;
        const float mrg = -sgn * y;
        const float lossv = wt * (fmaxf(mrg, 0.f) + log1pf(expf(-fabsf(mrg))));
        const float sig = 1.f / (1.f + expf(-y));
        const float dy = wt * (sig - lab);
        my_gb3 += dy;
        my_loss += lossv;
        // dz2 = dy w3 relu'(z2): kept as A (s, o) and A^T (o, s); sums for w3 and b2
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32], gw[32], gb[32];
            tc::tmem_ld32(tAcc + lane_base + c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const float z = v[q] + sB2[c0 + q];
                const float h2 = fmaxf(z, 0.f);
                const float dz = z > 0.f ? dy * sW3[c0 + q] : 0.f;
                gw[q] = dy * h2;
                gb[q] = dz;
                v[q] = dz;
            }
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) hb[u] = __float2bfloat16_rn(v[q + u]);
                *reinterpret_cast<uint4 *>(sD2 + tc::kmajor_offset(tid, c0 + q, kHid)) =
                    *reinterpret_cast<const uint4 *>(hb);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    *reinterpret_cast<__nv_bfloat16 *>(sD2T + tc::kmajor_offset(c0 + q + u, tid, kTile)) = hb[u];
            }
            const float s_w3 = warp_colsum32(gw, lane);
            const float s_b2 = warp_colsum32(gb, lane);
            gW3[warp * kHid + c0 + lane] += s_w3;
            gB2[warp * kHid + c0 + lane] += s_b2;
        }
        sync_all();
        if (tid == 0) {
#pragma unroll
            for (int kc = 0; kc < kHid / 16; ++kc)   // dH1 = dZ2 W2^T (K = output unit)
                tc::mma_bf16(tAcc, tc::make_desc(tc::smem_u32(sD2) + kc * 256, 128, 2048),
                             tc::make_desc(tc::smem_u32(sW2) + kc * 256, 128, 2048), idN128, kc > 0);
#pragma unroll
            for (int kc = 0; kc < kTile / 16; ++kc)  // dW2^T += dZ2^T H1 (K = sample)
                tc::mma_bf16(tDW2, tc::make_desc(tc::smem_u32(sD2T) + kc * 256, 128, 2048),
                             tc::make_desc(tc::smem_u32(sH1T) + kc * 256, 128, 2048), idN128, !first || kc > 0);
            tc::mma_commit(mb);
        }
        TFG_WAIT();
        // ---- dz1 = dH1 relu'(z1) as A (h, s) in the dZ2 region; sums for b1
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tAcc + lane_base + c0, v);
            const uint32_t m = mask1[c0 / 32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = ((m >> q) & 1u) ? v[q] : 0.f;
#pragma unroll
            for (int q = 0; q < 32; ++q) st_bf16(sD2, tc::kmajor_offset(c0 + q, tid, kTile), v[q]);
            const float s_b1 = warp_colsum32(v, lane);
            gB1[warp * kHid + c0 + lane] += s_b1;
        }
        sync_all();
        if (tid == 0) {
#pragma unroll
            for (int kc = 0; kc < kTile / 16; ++kc)  // dW1^T += dZ1^T X (K = sample)
                tc::mma_bf16(tDW1, tc::make_desc(tc::smem_u32(sD2) + kc * 256, 128, 2048),
                             tc::make_desc(tc::smem_u32(sXT) + kc * 256, 128, 2048), idN32, !first || kc > 0);
            tc::mma_commit(mb);
        }
        TFG_WAIT();
        first = false;
    }
#undef TFG_WAIT
    __syncthreads();
    if (timeout) {
        tc::mbar_wait(mb, phase);
        if (tid == 0) atomicExch(err, 1);
    } else if (!first) {
        // ---- flush: dW2[h][o] (TMEM lane o, column h), dW1[i][h] (lane h, column i), vectors
        float *pp = partial ? partial + (size_t)blockIdx.x * (kNumParams + 1) : nullptr;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tDW2 + lane_base + c0, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int e = kVW2 + (c0 + q) * kHid + tid;
                if (pp) pp[e] = v[q];
                else atomicAdd(&grad[e], v[q]);
            }
        }
        {
            float v[32];
            tc::tmem_ld32(tDW1 + lane_base, v);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int e = kVW1 + q * kHid + tid;
                if (pp) pp[e] = v[q];
                else atomicAdd(&grad[e], v[q]);
            }
        }
        // scalar sums: warp reduce (a fixed butterfly), one slot per warp
        for (int o = 16; o > 0; o >>= 1) {
            my_gb3 += __shfl_xor_sync(0xffffffffu, my_gb3, o);
            my_loss += __shfl_xor_sync(0xffffffffu, my_loss, o);
        }
        if (lane == 0) {
            gScal[2 * warp] = my_gb3;
            gScal[2 * warp + 1] = my_loss;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 3; ++k) {   // b1, b2, w3: the four warps' sums in warp order
            const float *gv = gB1 + k * 4 * kHid;
            const float v = ((gv[tid] + gv[kHid + tid]) + gv[2 * kHid + tid]) + gv[3 * kHid + tid];
            const int e = (k == 0 ? kVB1 : (k == 1 ? kVB2 : kVW3)) + tid;
            if (pp) pp[e] = v;
            else atomicAdd(&grad[e], v);
        }
        if (tid == 0) {
            const float sb3 = ((gScal[0] + gScal[2]) + gScal[4]) + gScal[6];
            const float sl = ((gScal[1] + gScal[3]) + gScal[5]) + gScal[7];
            if (pp) {
                pp[kVB3] = sb3;
                pp[kNumParams] = sl;   // loss follows the gradient vector
            } else {
                atomicAdd(&grad[kVB3], sb3);
                atomicAdd(&grad[kNumParams], sl);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Adam on FP32 master weights; the BF16 / FP32 parameter blob is rewritten.
// omb1 = 1 - beta1, omb2 = 1 - beta2 and the bias corrections bc1 = 1 - beta1^t,
// bc2 = 1 - beta2^t come from the host, formed in double precision (1 - beta
// formed from an FP32 beta would be off by up to 2^-24 / (1 - beta) relative).
__global__ void adam_kernel(float *master, float *m1, float *m2, const float *grad, uint8_t *blob, float lr,
                            float beta1, float omb1, float beta2, float omb2, float eps, float bc1, float bc2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNumParams) return;
    const float g = grad[e];
    const float a = beta1 * m1[e] + omb1 * g;
    const float b = beta2 * m2[e] + omb2 * g * g;
    m1[e] = a;
    m2[e] = b;
    const float p = master[e] - lr * (a / bc1) / (sqrtf(b / bc2) + eps);
    master[e] = p;
    if (e < kVB1) {
        *reinterpret_cast<__nv_bfloat16 *>(blob + (size_t)e * 2) = __float2bfloat16_rn(p);
    } else {
        reinterpret_cast<float *>(blob + kPB1)[e - kVB1] = p;
    }
}

__global__ void master_from_blob_kernel(const uint8_t *blob, float *master, float *m1, float *m2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNumParams) return;
    master[e] = e < kVB1 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(blob)[e])
                         : reinterpret_cast<const float *>(blob + kPB1)[e - kVB1];
    m1[e] = 0.f;
    m2[e] = 0.f;
}

}  // namespace

int mlp_num_params() { return kNumParams; }

// grad[e] = sum over b < parts of partial[b][e], in order of b
__global__ void grad_reduce_kernel(const float *__restrict__ partial, int parts, float *__restrict__ grad) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > kNumParams) return;
    float s = 0.f;
    for (int b = 0; b < parts; ++b) s += partial[(size_t)b * (kNumParams + 1) + e];
    grad[e] = s;
}

int grad_partial_rows() { return kGradPartialRows; }

void launch_mlp_grad(const void *params, const void *x, const float *label, const float *weight, int64_t n,
                     float *grad, int *err, cudaStream_t st, float *partial) {
    if (n <= 0) return;
    static bool attr = [] {
        cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
        return true;
    }();
    (void)attr;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n + kTile - 1) / kTile;
    int grid = (int)(tiles < sms ? tiles : sms);
    if (partial && grid > kGradPartialRows) grid = kGradPartialRows;
    mlp_grad_kernel<<<grid, 128, kTrainSmem, st>>>(reinterpret_cast<const uint8_t *>(params),
                                                   reinterpret_cast<const __nv_bfloat16 *>(x), label, weight, n,
                                                   grad, partial, err);
    if (partial) grad_reduce_kernel<<<(kNumParams + 1 + 255) / 256, 256, 0, st>>>(partial, grid, grad);
}

void launch_adam(float *master, float *m1, float *m2, const float *grad, void *blob, float lr, int step,
                 cudaStream_t st) {
    const double beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
    double p1 = 1.0, p2 = 1.0;
    for (int k = 0; k < step; ++k) { p1 *= beta1; p2 *= beta2; }
    adam_kernel<<<(kNumParams + 255) / 256, 256, 0, st>>>(
        master, m1, m2, grad, reinterpret_cast<uint8_t *>(blob), lr, (float)beta1, (float)(1.0 - beta1),
        (float)beta2, (float)(1.0 - beta2), (float)eps, (float)(1.0 - p1), (float)(1.0 - p2));
}

void launch_master_from_blob(const void *blob, float *master, float *m1, float *m2, cudaStream_t st) {
    master_from_blob_kernel<<<(kNumParams + 255) / 256, 256, 0, st>>>(reinterpret_cast<const uint8_t *>(blob),
                                                                      master, m1, m2);
}

}  // namespace tfg
