// Internal declarations shared by the C-ABI implementation and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tfg.h"

namespace tfg {

enum Action : int { kNoCand = 0, kReject = 1, kAccept = 2 };

// Device view of one walker population ("segment").  Walker w's slots are
// words [w][R][NWT] (NWT = 6 in Z_T: pos/neg masks of u, v, w; 3 in Z_2),
// its best scheme the same shape in `best`, its record hdr[w].
struct SegDesc {
    void *slots;
    void *best;
    tfg_walker_info *hdr;
    int64_t n_walkers;
    int32_t R;            // slots per walker (r_max)
    int32_t m, n, p;      // format
    uint32_t key0, key1;  // Philox key = seed
    int64_t plateau_len;
    uint32_t refresh_thresh;
    int32_t plus_attempts;
    int32_t plus_enabled;
    int32_t pad;
};

// One (mode, word size, lanes per walker, slots per lane) variant of the walk kernel.
struct WalkVariant {
    int mode;       // TFG_MODE_ZT / TFG_MODE_Z2
    int word_bits;  // 32 or 64
    int G;          // lanes per walker
    int S;          // slots per lane
    void (*launch)(const SegDesc &d, int32_t steps, int grid, int block, cudaStream_t st);
    const void *kernel;  // for cudaFuncGetAttributes
};

// Registry of compiled variants (filled by the instantiation units).
const WalkVariant *walk_variants(int *count);

// Auxiliary kernels (aux_kernels.cu).
void launch_replicate(const SegDesc &d, const void *start_words, int32_t r0, uint32_t id_base,
                      int32_t format_idx, int word_bits, int nwt, cudaStream_t st);
void launch_verify_best(const SegDesc &d, int64_t first, int64_t count, int word_bits, int mode,
                        int64_t *d_failures, cudaStream_t st);
void launch_argmin_best(const SegDesc &d, unsigned long long *d_key, cudaStream_t st);
void launch_stats(const SegDesc &d, int64_t *d_sums /*[9]*/, int *d_minmax /*[2]*/, int64_t *d_hist,
                  int hist_len, cudaStream_t st);
void launch_philox(const uint32_t *d_ctr, int n, uint32_t k0, uint32_t k1, uint32_t *d_out, cudaStream_t st);

}  // namespace tfg
