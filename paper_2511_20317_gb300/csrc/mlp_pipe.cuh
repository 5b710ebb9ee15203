// Tile pipeline of the proposal MLP 32 -> 128 -> 128 -> 1 on the tcgen05
// tensor cores, shared by the row-scoring kernel (features read from device
// memory) and the fused window-scoring kernel (features computed in place).
//
// A CTA holds the weights once (W1^T and W2^T as K-major BF16 operands, b1,
// b2, w3 in FP32) and runs NWG independent warpgroups.  Warpgroup g owns
// TMEM columns [128 g, 128 g + 128) (its accumulator), an A tile X (128 rows
// x 32 features) and an A tile H1 (128 rows x 128 hidden units) in shared
// memory, one mbarrier and one named barrier; its thread q owns tile row q,
// which is TMEM lane 32 (warp % 4) + lane, so every tcgen05.ld of a thread
// reads its own row.  Per tile:
//   producer: row q -> X                      (the Prod object)
//   MMA1  acc = X W1        (2 x K=16, one elected thread, commit -> mbarrier)
//   epi1  H1 = bf16(relu(acc + b1))            (cvt.rn.relu.bf16x2: ReLU and rounding in one)
//   MMA2  acc = H1 W2       (8 x K=16)
//   epi2  y = b3 + sum_o w3[o] relu(acc[o] + b2[o])
// The warpgroups of a CTA interleave on the tensor pipe: while one waits for
// its products, the others run their epilogues.  The producer of a tile
// prefetches the next tile's inputs before the products of the current one,
// so their latency hides behind the pipeline.
//
// Every mbarrier wait is bounded; a warpgroup whose wait gives up records
// the timeout, stops taking tiles, waits (bounded again) for its products in
// flight and sets *err before the CTA releases its tensor memory.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

#include "tc_common.cuh"

namespace tfg {
namespace mlp {

constexpr int kIn = 32, kHid = 128, kTile = 128;
// parameter blob (bytes): W1 bf16 [32][128], W2 bf16 [128][128], b1, b2, w3 f32 [128], b3 f32, pad
constexpr uint32_t kParamW1 = 0;
constexpr uint32_t kParamW2 = kParamW1 + kIn * kHid * 2;
constexpr uint32_t kParamB1 = kParamW2 + kHid * kHid * 2;
constexpr uint32_t kParamB2 = kParamB1 + kHid * 4;
constexpr uint32_t kParamW3 = kParamB2 + kHid * 4;
constexpr uint32_t kParamB3 = kParamW3 + kHid * 4;
constexpr uint32_t kParamBytes = kParamB3 + 16;

// shared memory (dynamic part): weights, vectors, then per warpgroup X and H1
constexpr uint32_t kSmW1T = 0;                              // B of MMA1: 128 (hidden) x 32 (input)
constexpr uint32_t kSmW2T = kSmW1T + kHid * kIn * 2;        // B of MMA2: 128 (out) x 128 (hidden)
constexpr uint32_t kSmVec = kSmW2T + kHid * kHid * 2;       // b1, b2, w3
constexpr uint32_t kSmWG = kSmVec + 3 * kHid * 4;           // first warpgroup area
constexpr uint32_t kSmX = 0;                                // per warpgroup: X 128 x 32
constexpr uint32_t kSmH1 = kTile * kIn * 2;                 //                H1 128 x 128
constexpr uint32_t kSmWGBytes = kSmH1 + kTile * kHid * 2;   // 40 KB
template <int NWG>
constexpr uint32_t smem_bytes() { return kSmWG + NWG * kSmWGBytes; }
template <int NWG>
constexpr uint32_t tmem_cols() { return NWG <= 1 ? 128u : (NWG <= 2 ? 256u : 512u); }

__device__ __forceinline__ uint32_t pack_relu_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// named barrier of warpgroup g (ids 1..NWG; 0 is __syncthreads)
__device__ __forceinline__ void wg_sync(int g) {
    asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory");
}
// named barrier with an OR reduction of a predicate over the warpgroup
__device__ __forceinline__ bool wg_any(int g, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %2, 0;\n\t"
        "bar.red.or.pred po, %1, 128, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}\n"
        : "=r"(r)
        : "r"(g + 1), "r"((uint32_t)p)
        : "memory");
    return r != 0;
}

// Weights and vectors of the parameter blob into the CTA's shared memory.
__device__ __forceinline__ void load_weights(const uint8_t *__restrict__ params, uint8_t *smem, int tid, int nthr) {
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(params + kParamW1);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(params + kParamW2);
    uint8_t *sW1T = smem + kSmW1T, *sW2T = smem + kSmW2T;
    // B operands are K-major: row = output unit, K = input unit
    for (int e = tid; e < kIn * kHid; e += nthr) {
        const int i = e / kHid, h = e % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(sW1T + tc::kmajor_offset(h, i, kIn)) = W1[e];
    }
    for (int e = tid; e < kHid * kHid; e += nthr) {
        const int h = e / kHid, o = e % kHid;
        *reinterpret_cast<__nv_bfloat16 *>(sW2T + tc::kmajor_offset(o, h, kHid)) = W2[e];
    }
    float *vec = reinterpret_cast<float *>(smem + kSmVec);
    for (int e = tid; e < 3 * kHid; e += nthr) vec[e] = reinterpret_cast<const float *>(params + kParamB1)[e];
}

// Store 8 consecutive features (as 4 packed bf16x2 words) of row q into an A tile.
__device__ __forceinline__ void st_row8(uint8_t *tile, int q, int col0, int K, uint4 v) {
    *reinterpret_cast<uint4 *>(tile + tc::kmajor_offset(q, col0, K)) = v;
}

// The pipeline.  Prod (one object per thread) provides
//   bool begin(int64_t tile, int q)   load tile `tile`'s input for row q (false: the tile is
//                                     skipped; the answer must be the same for the 128 rows)
//   void fill(uint8_t *sX, int q)     write row q of the tile loaded last into X
//   void emit(float y, int q)         the score of row q of the tile last filled
// and is called as begin(t), fill, begin(t + stride) (prefetch), ..., emit.
template <int NWG, class Prod>
__device__ __forceinline__ void run_tiles(const uint8_t *__restrict__ params, Prod &prod, int64_t ntiles,
                                          int *__restrict__ err, uint32_t first_limit, uint8_t *smem,
                                          uint64_t *mbar, uint32_t *tslot, int *timeout_flag) {
    const int tid = threadIdx.x, g = tid >> 7, q = tid & 127, warp = tid >> 5;
    load_weights(params, smem, tid, NWG * 128);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), tmem_cols<NWG>());
    if (q == 0) tc::mbar_init(tc::smem_u32(&mbar[g]), 1);
    if (tid == 0) *timeout_flag = 0;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t tacc = *tslot + (uint32_t)(g * 128);
    const uint32_t tlane = tacc + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t mb = tc::smem_u32(&mbar[g]);
    uint8_t *sX = smem + kSmWG + g * kSmWGBytes + kSmX;
    uint8_t *sH1 = smem + kSmWG + g * kSmWGBytes + kSmH1;
    const uint32_t aX = tc::smem_u32(sX), aH1 = tc::smem_u32(sH1);
    const uint32_t aW1 = tc::smem_u32(smem + kSmW1T), aW2 = tc::smem_u32(smem + kSmW2T);
    const float *sB1 = reinterpret_cast<const float *>(smem + kSmVec), *sB2 = sB1 + kHid, *sW3 = sB2 + kHid;
    const float b3 = *reinterpret_cast<const float *>(params + kParamB3);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTile, kHid);
    uint32_t phase = 0;
    bool timed_out = false, first_wait = true;

    const int64_t stride = (int64_t)gridDim.x * NWG;
    int64_t t = (int64_t)blockIdx.x * NWG + g;
    bool live = t < ntiles && prod.begin(t, q);
    while (t < ntiles) {
        if (!live) {   // skipped tile (uniform over the warpgroup)
            t += stride;
            live = t < ntiles && prod.begin(t, q);
            continue;
        }
        prod.fill(sX, q);
        const int64_t tn = t + stride;
        const bool live_next = tn < ntiles && prod.begin(tn, q);   // prefetch of the next tile
        tc::fence_async_smem();
        tc::fence_before_sync();
        wg_sync(g);
        tc::fence_after_sync();
        if (q == 0) {
#pragma unroll
            for (int kc = 0; kc < kIn / 16; ++kc)
                tc::mma_bf16(tacc, tc::make_desc(aX + kc * 256, 128, (kIn / 8) * 128),
                             tc::make_desc(aW1 + kc * 256, 128, (kIn / 8) * 128), idesc, kc > 0);
            tc::mma_commit(mb);
        }
        bool ok = tc::mbar_wait(mb, phase, first_wait ? first_limit : tc::kWaitLimit);
        first_wait = false;
        if (wg_any(g, !ok)) { timed_out = true; break; }
        phase ^= 1;
        tc::fence_after_sync();
        // ---- epi1: h1 = bf16(relu(z1 + b1)) -> H1 (row q)
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tlane + c0, v);
#pragma unroll
            for (int c = 0; c < 32; c += 8) {
                const float4 ba = *reinterpret_cast<const float4 *>(sB1 + c0 + c);
                const float4 bb = *reinterpret_cast<const float4 *>(sB1 + c0 + c + 4);
                uint4 h;
                h.x = pack_relu_bf16x2(v[c + 0] + ba.x, v[c + 1] + ba.y);
                h.y = pack_relu_bf16x2(v[c + 2] + ba.z, v[c + 3] + ba.w);
                h.z = pack_relu_bf16x2(v[c + 4] + bb.x, v[c + 5] + bb.y);
                h.w = pack_relu_bf16x2(v[c + 6] + bb.z, v[c + 7] + bb.w);
                st_row8(sH1, q, c0 + c, kHid, h);
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        wg_sync(g);
        tc::fence_after_sync();
        if (q == 0) {
#pragma unroll
            for (int kc = 0; kc < kHid / 16; ++kc)
                tc::mma_bf16(tacc, tc::make_desc(aH1 + kc * 256, 128, (kHid / 8) * 128),
                             tc::make_desc(aW2 + kc * 256, 128, (kHid / 8) * 128), idesc, kc > 0);
            tc::mma_commit(mb);
        }
        ok = tc::mbar_wait(mb, phase);
        if (wg_any(g, !ok)) { timed_out = true; break; }
        phase ^= 1;
        tc::fence_after_sync();
        // ---- epi2: y = b3 + w3 . relu(z2 + b2)
        float y0 = b3, y1 = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tlane + c0, v);
#pragma unroll
            for (int c = 0; c < 32; c += 4) {
                const float4 b = *reinterpret_cast<const float4 *>(sB2 + c0 + c);
                const float4 w = *reinterpret_cast<const float4 *>(sW3 + c0 + c);
                y0 = fmaf(fmaxf(v[c + 0] + b.x, 0.f), w.x, y0);
                y1 = fmaf(fmaxf(v[c + 1] + b.y, 0.f), w.y, y1);
                y0 = fmaf(fmaxf(v[c + 2] + b.z, 0.f), w.z, y0);
                y1 = fmaf(fmaxf(v[c + 3] + b.w, 0.f), w.w, y1);
            }
        }
        prod.emit(y0 + y1, q);
        // the next MMA1 overwrites the accumulator: order this thread's loads before it
        tc::fence_before_sync();
        t = tn;
        live = live_next;
    }
    if (timed_out) {
        // the awaited products may still be in flight: one more bounded wait before release
        tc::mbar_wait(mb, phase);
        if (q == 0) {
            *timeout_flag = 1;
            atomicExch(err, 1);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(*tslot, tmem_cols<NWG>());
}

}  // namespace mlp
}  // namespace tfg
