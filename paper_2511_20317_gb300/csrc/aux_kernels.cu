// Auxiliary kernels around the walk: population set-up, exact verification of
// best schemes (Eq. (1)), best-walker selection and population statistics.
#include <algorithm>
#include <cstdint>

#include "tfg_internal.h"
#include "pterm.cuh"

namespace tfg {
namespace {

// ---- population set-up: every walker starts from the prepared start scheme
template <class Wd>
__global__ void replicate_kernel(const SegDesc d, const Wd *__restrict__ start, int32_t r0,
                                 uint32_t id_base, int32_t fidx, uint32_t start_nnz) {
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
        h.best_nnz = start_nnz;
        d.hdr[w] = h;
    }
}

// ---- re-seeding: walker `first`'s live slots hold the new packed scheme;
// copy them to the live slots of walkers first+1 .. first+count-1 and to the
// best slots of all of them, and restart their records at rank r.
template <class Wd>
__global__ void reseed_kernel(const SegDesc d, int64_t first, int32_t r, uint32_t nnz) {
    const int64_t w = first + blockIdx.x;
    const size_t per = (size_t)d.R * d.nws;
    const Wd *src = reinterpret_cast<const Wd *>(d.slots) + per * first;
    Wd *s = reinterpret_cast<Wd *>(d.slots) + per * w;
    Wd *b = reinterpret_cast<Wd *>(d.best) + per * w;
    for (size_t e = threadIdx.x; e < per; e += blockDim.x) {
        const Wd v = src[e];
        if (w != first) s[e] = v;
        b[e] = v;
    }
    if (threadIdx.x == 0) {
        tfg_walker_info &h = d.hdr[w];
        h.r = r;
        h.best_r = r;
        h.plateau = 0;
        h.best_t = h.t;
        h.best_nnz = nnz;
    }
}

// ---- Eq. (1) on one walker's best scheme per block, by sparse accumulation:
// the tensor sum_l u_l (x) v_l (x) w_l is built in shared memory from the
// non-zero coefficients of each term (a few products per term instead of r
// products per tensor entry), one slab of u-indices a at a time, and every
// entry of the slab is compared with the matrix-multiplication tensor
// (1 iff a = (i,k), b = (k,j), c = (j,i)); over Z_2 the difference must be even.
template <class Wd>
struct Bits {
    static constexpr int WB = (int)sizeof(Wd) * 8;
    // calls f(bit, sign) for every non-zero coefficient with bit index in [lo, hi)
    template <class F>
    __device__ static void each(const Wd *pos, const Wd *neg, int lo, int hi, F f) {
        for (int q = lo / WB; q * WB < hi; ++q) {
            const int o0 = max(lo - q * WB, 0), o1 = min(hi - q * WB, WB);
            Wd mask = (o1 == WB) ? ~Wd(0) : ((Wd(1) << o1) - 1);
            mask &= ~((Wd(1) << o0) - 1);
            Wd nz = (pos[q] | (neg ? neg[q] : Wd(0))) & mask;
            while (nz) {
                const int o = (sizeof(Wd) == 8) ? __ffsll((long long)nz) - 1 : __ffs((int)nz) - 1;
                nz &= nz - 1;
                const int sgn = (neg && ((neg[q] >> o) & 1)) ? -1 : 1;
                f(q * WB + o, sgn);
            }
        }
    }
};

template <class Wd>
__global__ void __launch_bounds__(256) verify_best_kernel(const SegDesc d, int64_t first, int mode, int slab_rows,
                                                          unsigned long long *failures) {
    extern __shared__ __align__(16) unsigned char vsm[];
    __shared__ int bad;
    const int64_t w = first + blockIdx.x;
    if (w >= d.n_walkers) return;
    const int m = d.m, n = d.n, p = d.p;
    const int LU = m * n, LV = n * p, LW = p * m, LT = LU + LV + LW, LVW = LV * LW;
    const int r = d.hdr[w].best_r;
    Wd *terms = reinterpret_cast<Wd *>(vsm);                                       // [R][nws]
    int *slab = reinterpret_cast<int *>(vsm + (((size_t)d.R * d.nws * sizeof(Wd) + 15) & ~(size_t)15));
    const Wd *b = reinterpret_cast<const Wd *>(d.best) + (size_t)d.R * d.nws * w;
    if (threadIdx.x == 0) bad = (r < 0 || r > d.R) ? 1 : 0;
    const int rr = (r < 0 || r > d.R) ? 0 : r;
    for (int e = threadIdx.x; e < rr * d.nws; e += blockDim.x) terms[e] = b[e];
    __syncthreads();
    const bool zt = (mode == TFG_MODE_ZT);
    const int bu = d.fbase[0], bv = d.fbase[1], bw = d.fbase[2];   // factor bit offsets
    (void)LT;
    int mine = 0;
    for (int a0 = 0; a0 < LU; a0 += slab_rows) {
        const int a1 = min(LU, a0 + slab_rows);
        const int ne = (a1 - a0) * LVW;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) slab[e] = 0;
        __syncthreads();
        for (int l = threadIdx.x; l < rr; l += blockDim.x) {
            const Wd *pos = terms + (size_t)l * d.nws;
            const Wd *neg = zt ? pos + d.tw : nullptr;
            Bits<Wd>::each(pos, neg, bu + a0, bu + a1, [&](int ia, int sa) {
                Bits<Wd>::each(pos, neg, bv, bv + LV, [&](int ib, int sb) {
                    Bits<Wd>::each(pos, neg, bw, bw + LW, [&](int ic, int sc) {
                        atomicAdd(&slab[(ia - bu - a0) * LVW + (ib - bv) * LW + (ic - bw)], sa * sb * sc);
                    });
                });
            });
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const int a = a0 + e / LVW;
            const int rem = e - (a - a0) * LVW;
            const int bb = rem / LW, c = rem - bb * LW;
            const int i = a / n, k = a - i * n;
            const int k2 = bb / p, j = bb - k2 * p;
            const int j2 = c / m, i2 = c - j2 * m;
            const int diff = slab[e] - ((k == k2 && j == j2 && i == i2) ? 1 : 0);
            if (zt ? (diff != 0) : ((diff & 1) != 0)) mine = 1;
        }
        __syncthreads();
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
                      int32_t format_idx, uint32_t start_nnz, cudaStream_t st) {
    if (d.n_walkers <= 0) return;
    if (d.word_bits == 32)
        replicate_kernel<uint32_t><<<(unsigned)d.n_walkers, 128, 0, st>>>(
            d, reinterpret_cast<const uint32_t *>(start_words), r0, id_base, format_idx, start_nnz);
    else
        replicate_kernel<uint64_t><<<(unsigned)d.n_walkers, 128, 0, st>>>(
            d, reinterpret_cast<const uint64_t *>(start_words), r0, id_base, format_idx, start_nnz);
}

void launch_verify_best(const SegDesc &d, int64_t first, int64_t count, int mode, int64_t *d_failures,
                        cudaStream_t st) {
    if (count <= 0) return;
    // slab of u-indices sized to about 64 KB of int accumulators
    const int lu = d.m * d.n, lvw = (d.n * d.p) * (d.p * d.m);
    const int slab_rows = std::max(1, std::min(lu, 16384 / lvw));
    const size_t term_bytes = ((size_t)d.R * d.nws * (d.word_bits / 8) + 15) & ~(size_t)15;
    const size_t smem = term_bytes + (size_t)slab_rows * lvw * sizeof(int);
    auto *fail = reinterpret_cast<unsigned long long *>(d_failures);
    if (d.word_bits == 32) {
        cudaFuncSetAttribute(verify_best_kernel<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        verify_best_kernel<uint32_t><<<(unsigned)count, 256, smem, st>>>(d, first, mode, slab_rows, fail);
    } else {
        cudaFuncSetAttribute(verify_best_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        verify_best_kernel<uint64_t><<<(unsigned)count, 256, smem, st>>>(d, first, mode, slab_rows, fail);
    }
}

void launch_reseed(const SegDesc &d, int64_t first, int64_t count, int32_t r, uint32_t nnz, cudaStream_t st) {
    if (count <= 0) return;
    if (d.word_bits == 32) reseed_kernel<uint32_t><<<(unsigned)count, 128, 0, st>>>(d, first, r, nnz);
    else reseed_kernel<uint64_t><<<(unsigned)count, 128, 0, st>>>(d, first, r, nnz);
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
