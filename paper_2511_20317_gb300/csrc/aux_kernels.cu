// Auxiliary kernels around the walk: population set-up, exact verification of
// best schemes (Eq. (1)), best-walker selection and population statistics.
#include <cstdint>

#include "tfg_internal.h"
#include "pterm.cuh"

namespace tfg {
namespace {

// ---- population set-up: every walker starts from the prepared start scheme
template <class Wd>
__global__ void replicate_kernel(const SegDesc d, const Wd *__restrict__ start, int32_t r0,
                                 uint32_t id_base, int32_t fidx) {
    const int64_t w = blockIdx.x;
    if (w >= d.n_walkers) return;
    const size_t per = (size_t)d.R * d.nws;
    Wd *s = reinterpret_cast<Wd *>(d.slots) + per * w;
    Wd *b = reinterpret_cast<Wd *>(d.best) + per * w;
    for (size_t e = threadIdx.x; e < per; e += blockDim.x) {
        const Wd v = (e < (size_t)r0 * d.nws) ? start[e] : Wd(0);
        s[e] = v;
        b[e] = v;
    }
    if (threadIdx.x == 0) {
        tfg_walker_info h;
        h.r = r0; h.best_r = r0; h.r_max = d.R; h.format = fidx;
        h.t = 0; h.plateau = 0; h.best_t = 0;
        h.walker_id = id_base + (uint32_t)w;
        h.digest = 0xCBF29CE484222325ull ^ (uint64_t)h.walker_id;
        h.accepted = h.rejected = h.nocand = h.drops = h.merges = h.plus = h.reductions = 0;
        h.pad = 0;
        d.hdr[w] = h;
    }
}

// ---- Eq. (1) on one walker's best scheme per block.  Coefficients are
// unpacked into shared memory; every tensor entry (a, b, c) sums r products.
template <class Wd>
__global__ void verify_best_kernel(const SegDesc d, int64_t first, int mode,
                                   unsigned long long *failures) {
    extern __shared__ int8_t coef[];   // [r][LT]
    __shared__ int bad;
    const int64_t w = first + blockIdx.x;
    if (w >= d.n_walkers) return;
    const int m = d.m, n = d.n, p = d.p;
    const int LU = m * n, LV = n * p, LW = p * m, LT = LU + LV + LW;
    const int r = d.hdr[w].best_r;
    const int WB = (int)sizeof(Wd) * 8;
    const Wd *b = reinterpret_cast<const Wd *>(d.best) + (size_t)d.R * d.nws * w;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < r * LT; e += blockDim.x) {
        const int l = e / LT, bit = e - l * LT;
        const int q = bit / WB, o = bit - q * WB;
        int v = (int)((b[(size_t)l * d.nws + q] >> o) & 1);
        if (mode == TFG_MODE_ZT) v -= (int)((b[(size_t)l * d.nws + d.tw + q] >> o) & 1);
        coef[e] = (int8_t)v;
    }
    __syncthreads();
    const int E = LU * LV * LW;
    int mine = 0;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int a = e / (LV * LW);
        const int rem = e - a * LV * LW;
        const int bb = rem / LW;
        const int c = rem - bb * LW;
        int sum = 0;
        for (int l = 0; l < r; ++l) {
            const int8_t *row = coef + (size_t)l * LT;
            sum += (int)row[a] * (int)row[LU + bb] * (int)row[LU + LV + c];
        }
        // a = i*n + k, bb = k2*p + j, c = j2*m + i2; target 1 iff k==k2, j==j2, i==i2
        const int i = a / n, k = a - i * n;
        const int k2 = bb / p, j = bb - k2 * p;
        const int j2 = c / m, i2 = c - j2 * m;
        const int want = (k == k2 && j == j2 && i == i2) ? 1 : 0;
        const int diff = sum - want;
        if (mode == TFG_MODE_ZT ? (diff != 0) : ((diff & 1) != 0)) mine = 1;
    }
    if (mine) atomicOr(&bad, 1);
    __syncthreads();
    if (threadIdx.x == 0 && bad) atomicAdd(failures, 1ull);
}

__global__ void argmin_kernel(const SegDesc d, unsigned long long *key) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long k = ~0ull;
    if (w < d.n_walkers) k = ((unsigned long long)(uint32_t)d.hdr[w].best_r << 32) | (unsigned long long)(uint32_t)w;
    // warp minimum, then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, k, o);
        k = y < k ? y : k;
    }
    if ((threadIdx.x & 31) == 0 && k != ~0ull) atomicMin(key, k);
}

__global__ void stats_kernel(const SegDesc d, unsigned long long *sums, int *minmax,
                             unsigned long long *hist, int hist_len) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= d.n_walkers) return;
    const tfg_walker_info &h = d.hdr[w];
    atomicAdd(&sums[0], 1ull);
    atomicAdd(&sums[1], (unsigned long long)h.t);
    atomicAdd(&sums[2], (unsigned long long)h.accepted);
    atomicAdd(&sums[3], (unsigned long long)h.rejected);
    atomicAdd(&sums[4], (unsigned long long)h.nocand);
    atomicAdd(&sums[5], (unsigned long long)h.drops);
    atomicAdd(&sums[6], (unsigned long long)h.merges);
    atomicAdd(&sums[7], (unsigned long long)h.plus);
    atomicAdd(&sums[8], (unsigned long long)h.reductions);
    atomicMin(&minmax[0], h.best_r);
    atomicMax(&minmax[1], h.best_r);
    if (hist && h.best_r >= 0 && h.best_r < hist_len) atomicAdd(&hist[h.best_r], 1ull);
}

__global__ void philox_kernel(const uint32_t *ctr, int n, uint32_t k0, uint32_t k1, uint32_t *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const dev::U4 x = dev::philox10(ctr[4 * e], ctr[4 * e + 1], ctr[4 * e + 2], ctr[4 * e + 3], k0, k1);
    out[4 * e] = x.x; out[4 * e + 1] = x.y; out[4 * e + 2] = x.z; out[4 * e + 3] = x.w;
}

}  // namespace

void launch_replicate(const SegDesc &d, const void *start_words, int32_t r0, uint32_t id_base,
                      int32_t format_idx, cudaStream_t st) {
    if (d.n_walkers <= 0) return;
    if (d.word_bits == 32)
        replicate_kernel<uint32_t><<<(unsigned)d.n_walkers, 128, 0, st>>>(
            d, reinterpret_cast<const uint32_t *>(start_words), r0, id_base, format_idx);
    else
        replicate_kernel<uint64_t><<<(unsigned)d.n_walkers, 128, 0, st>>>(
            d, reinterpret_cast<const uint64_t *>(start_words), r0, id_base, format_idx);
}

void launch_verify_best(const SegDesc &d, int64_t first, int64_t count, int mode, int64_t *d_failures,
                        cudaStream_t st) {
    if (count <= 0) return;
    const size_t smem = (size_t)d.R * d.lt;
    auto *fail = reinterpret_cast<unsigned long long *>(d_failures);
    if (d.word_bits == 32) {
        cudaFuncSetAttribute(verify_best_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        verify_best_kernel<uint32_t><<<(unsigned)count, 256, smem, st>>>(d, first, mode, fail);
    } else {
        cudaFuncSetAttribute(verify_best_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        verify_best_kernel<uint64_t><<<(unsigned)count, 256, smem, st>>>(d, first, mode, fail);
    }
}

void launch_argmin_best(const SegDesc &d, unsigned long long *d_key, cudaStream_t st) {
    const int64_t blocks = (d.n_walkers + 255) / 256;
    if (blocks > 0) argmin_kernel<<<(unsigned)blocks, 256, 0, st>>>(d, d_key);
}

void launch_stats(const SegDesc &d, int64_t *d_sums, int *d_minmax, int64_t *d_hist, int hist_len,
                  cudaStream_t st) {
    const int64_t blocks = (d.n_walkers + 255) / 256;
    if (blocks > 0)
        stats_kernel<<<(unsigned)blocks, 256, 0, st>>>(d, reinterpret_cast<unsigned long long *>(d_sums), d_minmax,
                                                        reinterpret_cast<unsigned long long *>(d_hist), hist_len);
}

void launch_philox(const uint32_t *d_ctr, int n, uint32_t k0, uint32_t k1, uint32_t *d_out, cudaStream_t st) {
    if (n > 0) philox_kernel<<<(n + 127) / 128, 128, 0, st>>>(d_ctr, n, k0, k1, d_out);
}

}  // namespace tfg
