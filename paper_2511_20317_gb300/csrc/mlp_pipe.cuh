// Tile pipeline of the proposal MLP 32 -> 128 -> 128 -> 1 on the tcgen05
// tensor cores, shared by the row-scoring kernel (features read from device
// memory) and the fused window-scoring kernel (features computed in place).
//
// A CTA holds the weights once (W1^T and W2^T as K-major BF16 operands, the
// vectors in FP32) and runs NWG independent warpgroups.  Warpgroup g owns
// TMEM columns [128 g, 128 g + 128) (its accumulator), an A tile X (128 rows
// x 32 features) and an A tile H1 (128 rows x KH hidden inputs) in shared
// memory, one mbarrier and one named barrier; its thread q owns tile row q,
// which is TMEM lane 32 (warp % 4) + lane, so every tcgen05.ld of a thread
// reads its own row.  Per tile:
//   producer: row q -> X                      (the Prod object, prefetched a tile ahead)
//   MMA1  acc = X W1        (2 x K=16, one elected thread, commit -> mbarrier)
//   epi1  H1 = bf16(relu(acc + b1))            (cvt.rn.relu.bf16x2: ReLU and rounding in one)
//   MMA2  acc = H1 W2       (KH / 16 x K=16)
//   epi2  y = b3 + sum_o w3[o] relu(acc[o] + b2[o])
// The warpgroups of a CTA interleave on the tensor pipe: while one waits for
// its products, the others run their epilogues; a warpgroup itself writes
// the next tile's X while its MMA2 runs (X's only reader, MMA1, is done), so
// the next MMA1 follows epi2 at once.  TMEM loads are issued one 16-column
// chunk ahead of the arithmetic on the previous chunk.
//
// Bias folding (Prod::kFold, used where the producer controls the feature
// rows): the constant-one input f31 is joined by f29 = f30 = 1 on every
// real row, and W1^T's rows 29, 30, 31 hold s = W1[31] + b1 as three BF16
// pieces (s = hi + mid + lo to FP32 precision), so MMA1 adds the bias; H1
// gets 16 more columns (KH = 144): three of value one whose W2^T rows hold b2
// as three BF16 pieces, the rest zero, so MMA2 adds b2.  The epilogues then
// only apply ReLU (and the w3 dot product).  Features f29 and f30 are zero by
// definition, so their W1 rows never contribute otherwise; rows past a window
// (all features zero) get no bias, and their scores are not used.
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

// Shared-memory layout (dynamic part): W1^T, W2^T, the vectors, then per
// warpgroup X and H1.  KH = 128, or 144 with the folded b2.
template <bool FOLD>
struct Layout {
    static constexpr int KH = FOLD ? kHid + 16 : kHid;
    static constexpr uint32_t W1T = 0;                            // B of MMA1: 128 (hidden) x 32 (input)
    static constexpr uint32_t W2T = W1T + kHid * kIn * 2;         // B of MMA2: 128 (out) x KH
    static constexpr uint32_t Vec = W2T + kHid * KH * 2;          // b1, b2, w3 (w3 only when folded)
    static constexpr uint32_t VecBytes = (FOLD ? 1 : 3) * kHid * 4;
    static constexpr uint32_t WG = Vec + VecBytes;                // first warpgroup area
    static constexpr uint32_t X = 0;                              // per warpgroup: X 128 x 32
    static constexpr uint32_t H1 = kTile * kIn * 2;               //                H1 128 x KH
    static constexpr uint32_t WGBytes = H1 + kTile * KH * 2;
    static constexpr uint32_t bytes(int nwg) { return WG + nwg * WGBytes; }
};
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

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane, without
// waiting: the registers are valid after the next tmem_wait().
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// Wait for this thread's TMEM loads; the empty asm afterwards redefines the
// registers of the chunk that is read next, so no use of them moves above the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]));
}

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }

// Weights and vectors of the parameter blob into the CTA's shared memory.
template <bool FOLD>
__device__ __forceinline__ void load_weights(const uint8_t *__restrict__ params, uint8_t *smem, int tid, int nthr) {
    using LY = Layout<FOLD>;
    constexpr int KH = LY::KH;
    const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(params + kParamW1);
    const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(params + kParamW2);
    const float *b1 = reinterpret_cast<const float *>(params + kParamB1);
    const float *b2 = reinterpret_cast<const float *>(params + kParamB2);
    uint8_t *sW1T = smem + LY::W1T, *sW2T = smem + LY::W2T;
    // B operands are K-major: row = output unit, K = input unit
    for (int e = tid; e < kIn * kHid; e += nthr) {
        const int i = e / kHid, h = e % kHid;
        __nv_bfloat16 v = W1[e];
        if (FOLD && i >= 29) {
            // rows 29..31: W1[31] + b1 in three bf16 pieces (inputs 29..31 are one)
            const float s = __bfloat162float(W1[31 * kHid + h]) + b1[h];
            const float hi = __bfloat162float(bf(s)), mid = __bfloat162float(bf(s - hi));
            v = i == 31 ? bf(hi) : (i == 30 ? bf(mid) : bf(s - hi - mid));
        }
        *reinterpret_cast<__nv_bfloat16 *>(sW1T + tc::kmajor_offset(h, i, kIn)) = v;
    }
    for (int e = tid; e < kHid * KH; e += nthr) {
        const int o = e / KH, h = e % KH;
        __nv_bfloat16 v;
        if (h < kHid) {
            v = W2[h * kHid + o];
        } else {
            // K rows 128..130: b2 in three bf16 pieces (H1 columns 128..130 are one), then zeros
            const float s = b2[o];
            const float hi = __bfloat162float(bf(s)), mid = __bfloat162float(bf(s - hi));
            v = h == kHid ? bf(hi) : (h == kHid + 1 ? bf(mid) : (h == kHid + 2 ? bf(s - hi - mid) : bf(0.f)));
        }
        *reinterpret_cast<__nv_bfloat16 *>(sW2T + tc::kmajor_offset(o, h, KH)) = v;
    }
    float *vec = reinterpret_cast<float *>(smem + LY::Vec);
    if (FOLD) {
        for (int e = tid; e < kHid; e += nthr) vec[e] = reinterpret_cast<const float *>(params + kParamW3)[e];
    } else {
        for (int e = tid; e < 3 * kHid; e += nthr) vec[e] = b1[e];   // b1, b2, w3 are consecutive in the blob
    }
}

// Store 8 consecutive features (as 4 packed bf16x2 words) of row q into an A tile.
__device__ __forceinline__ void st_row8(uint8_t *tile, int q, int col0, int K, uint4 v) {
    *reinterpret_cast<uint4 *>(tile + tc::kmajor_offset(q, col0, K)) = v;
}

// The pipeline.  Prod (one object per thread; static bool kFold) provides
//   void begin(int64_t tile, int q)   start loading tile `tile`'s input for row q
//   void mid(int q)                   second load phase of the tile begun last (may be empty)
//   bool live()                       false: the tile begun last is skipped (the same answer for
//                                     the 128 rows; asked only when the tile is due, so that its
//                                     loads have landed)
//   int64_t fill(uint8_t *sX, int q)  write row q of the tile loaded last into X (kFold:
//                                     features 29 and 30 one on every real row); returns
//                                     the row's output index (-1: no output)
//   void emit(float y, int64_t o)     the score y of the row whose fill returned o
template <int NWG, class Prod>
__device__ __forceinline__ void run_tiles(const uint8_t *__restrict__ params, Prod &prod, int64_t ntiles,
                                          int *__restrict__ err, uint32_t first_limit, uint8_t *smem,
                                          uint64_t *mbar, uint32_t *tslot, int *timeout_flag) {
    constexpr bool FOLD = Prod::kFold;
    using LY = Layout<FOLD>;
    constexpr int KH = LY::KH;
    const int tid = threadIdx.x, g = tid >> 7, q = tid & 127, warp = tid >> 5;
    load_weights<FOLD>(params, smem, tid, NWG * 128);
    uint8_t *sX = smem + LY::WG + g * LY::WGBytes + LY::X;
    uint8_t *sH1 = smem + LY::WG + g * LY::WGBytes + LY::H1;
    if (FOLD) {
        // the constant columns 128..143 of H1 (ones, then zeros), written once
        const uint32_t one2 = 0x3F803F80u;
        st_row8(sH1, q, kHid, KH, make_uint4(one2, 0x00003F80u, 0u, 0u));
        st_row8(sH1, q, kHid + 8, KH, make_uint4(0u, 0u, 0u, 0u));
    }
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
    const uint32_t aX = tc::smem_u32(sX), aH1 = tc::smem_u32(sH1);
    const uint32_t aW1 = tc::smem_u32(smem + LY::W1T), aW2 = tc::smem_u32(smem + LY::W2T);
    const float *vec = reinterpret_cast<const float *>(smem + LY::Vec);
    const float *sB1 = vec, *sB2 = vec + kHid, *sW3 = FOLD ? vec : vec + 2 * kHid;
    const float b3 = *reinterpret_cast<const float *>(params + kParamB3);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTile, kHid);
    uint32_t phase = 0;
    bool timed_out = false, first_wait = true;

    const int64_t stride = (int64_t)gridDim.x * NWG;
    int64_t t = (int64_t)blockIdx.x * NWG + g;
    // the first live tile, its features in X
    if (t < ntiles) {
        prod.begin(t, q);
        prod.mid(q);
    }
    while (t < ntiles && !prod.live()) {   // skipped tile (uniform over the warpgroup)
        t += stride;
        if (t < ntiles) {
            prod.begin(t, q);
            prod.mid(q);
        }
    }
    int64_t out_cur = t < ntiles ? prod.fill(sX, q) : -1;
    while (t < ntiles) {
        int64_t tn = t + stride;
        if (tn < ntiles) prod.begin(tn, q);   // first load phase of the next tile
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
        // ---- epi1: h1 = bf16(relu(z1 + b1)) -> H1 (row q), TMEM chunks of 16 one ahead
        {
            uint32_t ra[16], rb[16];
            tmem_ld16_nowait(tlane, ra);
            tmem_wait(ra);
#pragma unroll
            for (int c = 0; c < kHid / 16; ++c) {
                uint32_t(&cur)[16] = (c & 1) ? rb : ra;
                uint32_t(&nxt)[16] = (c & 1) ? ra : rb;
                if (c + 1 < kHid / 16) tmem_ld16_nowait(tlane + 16 * (c + 1), nxt);
#pragma unroll
                for (int u = 0; u < 16; u += 8) {
                    float f[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        f[k] = __uint_as_float(cur[u + k]);
                        if (!FOLD) f[k] += sB1[16 * c + u + k];
                    }
                    st_row8(sH1, q, 16 * c + u, KH,
                            make_uint4(pack_relu_bf16x2(f[0], f[1]), pack_relu_bf16x2(f[2], f[3]),
                                       pack_relu_bf16x2(f[4], f[5]), pack_relu_bf16x2(f[6], f[7])));
                }
                if (c + 1 < kHid / 16) tmem_wait(nxt);
            }
        }
        if (tn < ntiles) prod.mid(q);   // second load phase of the next tile
        tc::fence_async_smem();
        tc::fence_before_sync();
        wg_sync(g);
        tc::fence_after_sync();
        if (q == 0) {
#pragma unroll
            for (int kc = 0; kc < KH / 16; ++kc)
                tc::mma_bf16(tacc, tc::make_desc(aH1 + kc * 256, 128, (KH / 8) * 128),
                             tc::make_desc(aW2 + kc * 256, 128, (KH / 8) * 128), idesc, kc > 0);
            tc::mma_commit(mb);
        }
        // while MMA2 runs: the next live tile's features into X (MMA1, its only reader, is done)
        while (tn < ntiles && !prod.live()) {
            tn += stride;
            if (tn < ntiles) {
                prod.begin(tn, q);
                prod.mid(q);
            }
        }
        const int64_t out_next = tn < ntiles ? prod.fill(sX, q) : -1;
        ok = tc::mbar_wait(mb, phase);
        if (wg_any(g, !ok)) { timed_out = true; break; }
        phase ^= 1;
        tc::fence_after_sync();
        // ---- epi2: y = b3 + w3 . relu(z2 + b2)
        float2 y2 = make_float2(b3, 0.f);
        {
            uint32_t ra[16], rb[16];
            tmem_ld16_nowait(tlane, ra);
            tmem_wait(ra);
#pragma unroll
            for (int c = 0; c < kHid / 16; ++c) {
                uint32_t(&cur)[16] = (c & 1) ? rb : ra;
                uint32_t(&nxt)[16] = (c & 1) ? ra : rb;
                if (c + 1 < kHid / 16) tmem_ld16_nowait(tlane + 16 * (c + 1), nxt);
#pragma unroll
                for (int u = 0; u < 16; u += 4) {
                    const float4 w = *reinterpret_cast<const float4 *>(sW3 + 16 * c + u);
                    float z0 = __uint_as_float(cur[u]), z1 = __uint_as_float(cur[u + 1]);
                    float z2 = __uint_as_float(cur[u + 2]), z3 = __uint_as_float(cur[u + 3]);
                    if (!FOLD) {
                        const float4 b = *reinterpret_cast<const float4 *>(sB2 + 16 * c + u);
                        const float2 s01 = __fadd2_rn(make_float2(z0, z1), make_float2(b.x, b.y));
                        const float2 s23 = __fadd2_rn(make_float2(z2, z3), make_float2(b.z, b.w));
                        z0 = s01.x; z1 = s01.y; z2 = s23.x; z3 = s23.y;
                    }
                    y2 = __ffma2_rn(make_float2(fmaxf(z0, 0.f), fmaxf(z1, 0.f)), make_float2(w.x, w.y), y2);
                    y2 = __ffma2_rn(make_float2(fmaxf(z2, 0.f), fmaxf(z3, 0.f)), make_float2(w.z, w.w), y2);
                }
                if (c + 1 < kHid / 16) tmem_wait(nxt);
            }
        }
        prod.emit(y2.x + y2.y, out_cur);
        // the next MMA1 overwrites the accumulator: order this thread's loads before it
        tc::fence_before_sync();
        out_cur = out_next;
        t = tn;
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
