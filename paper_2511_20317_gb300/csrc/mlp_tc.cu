// Learned flip proposal: the scoring MLP 32 -> 128 -> 128 -> 1 (ReLU) on the
// 5th-generation tensor cores for rows of features in device memory
// (tfg_mlp_score).  The tile pipeline (mlp_pipe.cuh) runs four warpgroups per
// CTA, one CTA per SM; each thread loads its row of the next tile while the
// current tile's products run.
//
// Parameter blob (device, see include/tfg.h): W1 bf16 [32][128], W2 bf16
// [128][128] (row = input unit), b1, b2, w3 f32 [128] each, b3 f32.
#include <cstdint>
#include <cuda_bf16.h>

#include "mlp_pipe.cuh"
#include "tfg_internal.h"

namespace tfg {
namespace {

constexpr int kWG = 4;

// Rows of features from device memory (bf16 [n][32]); rows past n are zero.
struct RowsProducer {
    static constexpr bool kFold = false;   // arbitrary rows: the biases are added in the epilogues
    const __nv_bfloat16 *x;
    int64_t n;
    float *out;
    uint4 v[4];
    int64_t row_loaded;
    __device__ __forceinline__ bool live() const { return true; }
    __device__ __forceinline__ void begin(int64_t tile, int q) {
        row_loaded = tile * mlp::kTile + q;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = make_uint4(0, 0, 0, 0);
        if (row_loaded < n) {
            const uint4 *src = reinterpret_cast<const uint4 *>(x + row_loaded * mlp::kIn);
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = src[c];
        }
    }
    __device__ __forceinline__ void mid(int) {}
    __device__ __forceinline__ int64_t fill(uint8_t *sX, int q) {
#pragma unroll
        for (int c = 0; c < 4; ++c) mlp::st_row8(sX, q, 8 * c, mlp::kIn, v[c]);
        return row_loaded < n ? row_loaded : -1;
    }
    __device__ __forceinline__ void emit(float y, int64_t o) {
        if (o >= 0) out[o] = y;
    }
};

__global__ void __launch_bounds__(kWG * 128, 1) mlp_score_kernel(const uint8_t *__restrict__ params,
                                                                const __nv_bfloat16 *__restrict__ x, int64_t n,
                                                                float *__restrict__ out, int *__restrict__ err,
                                                                uint32_t first_limit) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar[kWG];
    __shared__ uint32_t tslot;
    __shared__ int tflag;
    RowsProducer p;
    p.x = x;
    p.n = n;
    p.out = out;
    mlp::run_tiles<kWG>(params, p, (n + mlp::kTile - 1) / mlp::kTile, err, first_limit, smem, mbar, &tslot,
                        &tflag);
}

uint32_t g_first_wait_limit = tc::kWaitLimit;

}  // namespace

void set_first_wait_limit(int64_t polls) {
    g_first_wait_limit = (polls < 0 || polls > (int64_t)tc::kWaitLimit) ? tc::kWaitLimit : (uint32_t)polls;
}
uint32_t first_wait_limit() { return g_first_wait_limit; }

size_t mlp_param_bytes() { return mlp::kParamBytes; }

int score_grid(int64_t tiles, int wg) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ctas = (tiles + wg - 1) / wg;
    return (int)(ctas < sms ? ctas : sms);
}

int launch_mlp_score(const void *params, const void *x, int64_t n, float *out, int *err, cudaStream_t st) {
    if (n <= 0) return 0;
    constexpr uint32_t smem = mlp::Layout<false>::bytes(kWG);
    static bool attr = [] {
        cudaFuncSetAttribute(mlp_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return true;
    }();
    (void)attr;
    const int64_t tiles = (n + mlp::kTile - 1) / mlp::kTile;
    mlp_score_kernel<<<score_grid(tiles, kWG), kWG * 128, smem, st>>>(
        reinterpret_cast<const uint8_t *>(params), reinterpret_cast<const __nv_bfloat16 *>(x), n, out, err,
        g_first_wait_limit);
    return 0;
}

}  // namespace tfg
