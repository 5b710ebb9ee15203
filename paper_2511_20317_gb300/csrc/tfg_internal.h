// Internal declarations shared by the C-ABI implementation and the kernels.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/tfg.h"

namespace tfg {

enum Action : int { kNoCand = 0, kReject = 1, kAccept = 2 };

// Device view of one walker population ("segment").  A term is packed: its
// LT = mn + np + pm coefficients as TW words of +1 bits followed, in Z_T, by
// TW words of -1 bits (NWS = 2*TW words per slot; NWS = TW in Z_2).  Factor f
// starts at bit fbase[f]: u | v | w concatenated in one word (TW = 1), else
// factor-aligned in 64-bit words (TW = 3, or 6 when a factor is longer than 64).
// Walker w's slots are words [w][R][NWS], its best scheme the same shape in
// `best`, its record hdr[w].  fmask[f][q] selects factor f (u, v, w) in word q
// (q < 3; read by the kernels of the concatenated layout).
struct SegDesc {
    void *slots;
    void *best;
    tfg_walker_info *hdr;
    int64_t n_walkers;
    int32_t R;            // slots per walker (r_max)
    int32_t m, n, p;      // format
    int32_t lt, tw, nws, word_bits;
    uint64_t fmask[3][3];
    uint32_t key0, key1;  // Philox key = seed
    int64_t plateau_len;
    uint32_t refresh_thresh;
    int32_t plus_attempts;
    int32_t plus_enabled;
    int32_t pad;
    int32_t fbase[3];     // bit offset of factor u, v, w in a packed term
    int32_t walk_policy;  // 0: plateau plus transitions; 1: Algorithm 1 expansions
    uint32_t expand_thresh;
    int32_t pad3;
};

// One compiled variant of the walk kernel.
struct WalkVariant {
    int mode;       // TFG_MODE_ZT / TFG_MODE_Z2
    int word_bits;  // 32 or 64
    int tw;         // words per sign of a packed term
    int G;          // lanes per walker (1: thread-per-walker kernel)
    int S;          // slots per lane (lane groups) or slot capacity (G = 1)
    int block;      // fixed block size (G = 1), 0 = chosen by the caller
    void (*launch)(const SegDesc &d, int32_t steps, int grid, int block, cudaStream_t st);
    const void *kernel;  // for cudaFuncGetAttributes
    void (*prepare)();   // one-time kernel attribute set-up (may be null)
    int cap = 0;         // slot capacity when not given by G and S
    int fl = 0;          // > 0: formats whose factors have at most fl coefficients only (bit-sliced)
    int sq = 0;          // 1: formats whose three factors have exactly fl coefficients only
    int capacity() const { return cap ? cap : (G == 1 ? S : G * S); }
};

// Device resize (resize.cu): output terms come in at most two blocks; a block
// takes source terms (kResizeSrc), aux terms (kResizeAux) or source x aux
// pairs (kResizeProduct, source outer); maps[map_a + e] / maps[map_b + e] give
// the source / aux row index of output coefficient e (-1: zero).
enum : int32_t { kResizeSrc = 1, kResizeAux = 2, kResizeProduct = 3 };
constexpr int kResizeMaxTerms = 1024;
struct ResizeBlock {
    int32_t kind, map_a, map_b;
};
struct ResizePlan {
    ResizeBlock blk[2];
    int32_t nblk;
    int32_t lt_src, mn_src, np_src;   // source row layout (u | v | w)
    int32_t lt_out, mn_out, np_out;   // result row layout
    int32_t lt_aux, aux_rank;
    int32_t canon;       // Z_T: restore the sign normalisation
    int32_t drop_zero;   // remove terms with a zero factor
    int32_t use_best;    // source: best scheme instead of the live one
    const int16_t *maps; // device
    const int8_t *aux;   // device [aux_rank][lt_aux]
};
bool build_resize_plan(int op, int axis, int index, const tfg_format &src, const tfg_format *aux, int aux_rank,
                       tfg_format &out, ResizePlan &plan, std::vector<int16_t> &maps);
size_t resize_smem_bytes(const ResizePlan &plan);
void launch_resize(const SegDesc &src, int64_t src_first, const SegDesc &dst, int64_t dst_first, int64_t count,
                   const ResizePlan &plan, unsigned long long *d_skipped, cudaStream_t st);

// Registry of compiled variants (filled by the instantiation units).
const WalkVariant *walk_variants(int *count);

// Auxiliary kernels (aux_kernels.cu).
void launch_replicate(const SegDesc &d, const void *start_words, int32_t r0, uint32_t id_base,
                      int32_t format_idx, uint32_t start_nnz, cudaStream_t st);
void launch_reseed(const SegDesc &d, int64_t first, int64_t count, int32_t r, uint32_t nnz, cudaStream_t st);
void launch_verify_best(const SegDesc &d, int64_t first, int64_t count, int mode, int64_t *d_failures,
                        cudaStream_t st);
void launch_argmin_best(const SegDesc &d, unsigned long long *d_key, cudaStream_t st);
void launch_stats(const SegDesc &d, int64_t *d_sums /*[9]*/, int *d_minmax /*[2]*/, int64_t *d_hist,
                  int hist_len, cudaStream_t st);
using WindowLog = tfg_log_spec;
using WindowLogEntry = tfg_log_entry;
int window_cap();
int window_apply_capacity(int word_bits, int R);
// Window mode (walk_window.cu).  desc[w][k] = (descriptor, info) of window row k of
// walker w: descriptor i | X << 10 | j << 12 | (s < 0) << 22 | rho << 23, info = the term's
// candidate count (at most 64) | its position after i0 (at most 64) << 8.
void launch_window(const SegDesc &d, void *feat /*nullable*/, uint2 *desc, int *kwin, cudaStream_t st);
void launch_window_score(const SegDesc &d, const void *params, const uint2 *desc, const int *kwin, float *score,
                         int *err, cudaStream_t st);
int launch_window_apply(const SegDesc &d, const uint2 *desc, const int *kwin, const float *score, int policy,
                        uint32_t eps, int32_t *choices, const WindowLog &log, cudaStream_t st);
size_t mlp_param_bytes();
int launch_mlp_score(const void *params, const void *x, int64_t n, float *out, int *err, cudaStream_t st);
void set_first_wait_limit(int64_t polls);   // test hook of tfg_test_set_wait_limit
uint32_t first_wait_limit();                 // the current limit (polls) of a CTA's first completion wait
int score_grid(int64_t tiles, int warpgroups);   // CTAs of a tile-pipeline launch (at most one per SM)
int mlp_num_params();
// partial (optional, [grad_partial_rows()][P + 1]): per-CTA rows added in CTA order (deterministic);
// null: CTA totals added to grad by atomics (grad zeroed by the caller)
void launch_mlp_grad(const void *params, const void *x, const float *label, const float *weight, int64_t n,
                     float *grad, int *err, cudaStream_t st, float *partial = nullptr);
int grad_partial_rows();
void launch_adam(float *master, float *m1, float *m2, const float *grad, void *blob, float lr, int step,
                 cudaStream_t st);
void launch_master_from_blob(const void *blob, float *master, float *m1, float *m2, cudaStream_t st);
void launch_philox(const uint32_t *d_ctr, int n, uint32_t k0, uint32_t k1, uint32_t *d_out, cudaStream_t st);

}  // namespace tfg
