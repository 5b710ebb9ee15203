/*
 * tfg.h - C ABI of the ternary flip-graph walker library (libtfg.so).
 *
 * The library runs many independent random walks over matrix-multiplication
 * schemes (m,n,p:r) with coefficients in Z_T = {-1,0,1} (or Z_2) on one GPU
 * (sm_103a): flips with ternary-safety rejection, zero-term and merge
 * reductions, sign-symmetry normalisation, best-scheme tracking and
 * plateau-triggered plus transitions (Sections 3.3-3.6, Algorithm 1 of
 * "Fast Matrix Multiplication via Ternary Meta Flip Graphs").  The meta
 * operators of Section 3.3.2 run on the host.
 *
 * Scheme layout (every int8_t* scheme argument): rank r rows of
 * LT = m*n + n*p + p*m int8 coefficients; row l is u_l[i*n+k] (coefficient of
 * a_ik), then v_l[k*p+j] (b_kj), then w_l[j*m+i] (c_ij): the C^T convention of
 * Section 3.1, in which Eq. (1) reads
 *     sum_l u_l[i*n+k] v_l[k'*p+j] w_l[j'*m+i'] = [k=k'][j=j'][i=i'].
 * In Z_T mode coefficients are -1, 0, 1; in Z_2 mode 0, 1.  Every size
 * m*n, n*p, p*m must be <= 128: one 64-bit word per factor and sign as in
 * Section 3.5.1 up to 64 coefficients (the limit of Section 4.1), two words
 * beyond.  The window mode and the learned proposal take terms of at most 64
 * coefficients in all.
 *
 * Errors: every int-returning call returns TFG_OK (0) or a negative TFG_E*
 * code; tfg_last_error() gives a message for the calling thread.  No call
 * falls back to a CPU implementation of the walk: without a usable CUDA
 * device the device calls fail with TFG_ECUDA.
 *
 * Memory: the library allocates no device memory.  The caller provides one
 * device workspace per context (size from tfg_workspace_size), keeps it alive
 * until tfg_destroy, and owns it.  Host buffers passed in are read or written
 * during the call only, except where a call says otherwise.
 */
#ifndef TFG_H
#define TFG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---------------------------------------------------------- */
#define TFG_OK          0
#define TFG_EINVAL     -1   /* bad argument: sizes, pointers, mode, capacity */
#define TFG_ESCHEME    -2   /* coefficient outside the set, or Eq. (1) fails */
#define TFG_ENOSPC     -3   /* caller buffer too small */
#define TFG_ENOMEM     -4   /* host allocation failed / workspace too small */
#define TFG_ECUDA      -5   /* CUDA runtime error (message in tfg_last_error) */
#define TFG_ETIMEOUT   -6   /* a bounded device wait gave up */
#define TFG_EINTERNAL  -7   /* an emitted scheme failed verification */

#define TFG_MODE_ZT 0       /* coefficients in {-1, 0, 1} (Section 3.2) */
#define TFG_MODE_Z2 1       /* binary field (Section 3.5, XOR arithmetic) */

/* Format of one population: sizes of A (m x n) and B (n x p), and the mode. */
typedef struct {
    int32_t m, n, p;
    int32_t mode;           /* TFG_MODE_ZT or TFG_MODE_Z2 */
} tfg_format;

/* Walk parameters.  tfg_default_params fills the defaults. */
typedef struct {
    int64_t plateau_len;      /* L: steps without a new best rank before a plus transition (default 10000) */
    uint32_t refresh_thresh;  /* equal-rank best refresh when draw x2 < this; default 42949672 = 0.01 * 2^32
                                 (the 1% acceptance of Algorithm 1); 0 disables */
    int32_t plus_attempts;    /* plus transition tries per plateau event, Philox sub-streams 1.. (default 16) */
    int32_t plus_enabled;     /* 1: plus transitions on plateaus (default), 0: never */
    int32_t r_slack;          /* slots per walker = prepared start rank + r_slack (default 3, >= 1) */
    int32_t mapping;          /* lanes per walker G in {4,8,16,32}; 0 = autotune (default) */
    int32_t block_threads;    /* CUDA block size, multiple of 32, at most 256 (default 256), of the
                                 lane-group kernels; a thread-per-walker kernel takes it as its
                                 walkers per block when a variant with that block size is compiled
                                 for its capacity (else its compiled default; see tfg_launch_shape) */
    uint32_t walker_id_base;  /* global id of this context's first walker (sharding across GPUs) */
    int32_t use_graph;        /* tfg_walk launches one captured CUDA graph of all populations' kernels:
                                 1 chained (default), 2 forked onto one stream per population
                                 (concurrent); 0 plain launches on the context stream */
    int32_t walk_policy;      /* the step's policy (Section 3.3.1, Algorithm 1):
                                 0 (default): a plus transition after plateau_len steps without a
                                   new best rank, when r <= best + 2;
                                 1: Algorithm 1 -- a failed try_flip (no candidate, or the flip
                                   leaves Z_T) expands and ends the step; after a flip, expand
                                   when draw x3 < expand_thresh and r <= best + 2.  An expansion
                                   is plus or split with probability 1/2 each.
                                 Both need a free slot (r < r_max).
                                 2: naive additive complexity minimisation: flips and zero-term
                                   removal only (no reductions, no expansions); the best scheme is
                                   the one of least (rank, non-zero coefficients).
                                 Window mode needs policy 0 */
    uint32_t expand_thresh;   /* policy 1: floor(p_expand * 2^32) */
    int32_t reserved[2];
} tfg_params;

/* Per-walker record.  t is the number of steps taken, digest a rolling hash of
 * every step's action (sampled term, candidate, sign, rank), best_t the step at
 * which best_r last fell.  Counters are cumulative.  best_nnz: non-zero
 * coefficients of the best scheme (its naive additive complexity is best_nnz
 * - 2 best_r - m p); kept up to date by walk policy 2, the start's count
 * under the other policies. */
typedef struct {
    int32_t r, best_r, r_max, format;
    int64_t t, plateau, best_t;
    uint64_t digest;
    int64_t accepted, rejected, nocand, drops, merges, plus, reductions;
    uint32_t walker_id, best_nnz;
} tfg_walker_info;

/* Aggregate counters over all walkers of a context (or of one format). */
typedef struct {
    int64_t walkers, steps, accepted, rejected, nocand, drops, merges, plus, reductions;
    int32_t min_best_r, max_best_r;
} tfg_stats;

typedef struct tfg_ctx tfg_ctx;

void tfg_default_params(tfg_params *out);
const char *tfg_last_error(void);

/* ---- host-only scheme functions ------------------------------------------ */

/* Eq. (1), Section 3.1: exact integer reconstruction of sum_l u_l (x) v_l (x) w_l
 * against the matrix-multiplication tensor (mod 2 in Z_2 mode).
 * Returns TFG_OK when valid, TFG_ESCHEME when not, TFG_EINVAL on bad sizes. */
int tfg_verify(const tfg_format *fmt, int32_t rank, const int8_t *scheme);

/* Section 4.5: naive additive complexity nnz(U)+nnz(V)+nnz(W) - 2r - m*p. */
int tfg_additive_complexity(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int64_t *out);

/* Isotropy invariants of a scheme (section "Isotropy Invariants and Novelty
 * Verification"): for every term the ranks of its factors read as matrices
 * U_i (m x n, entry (i,k) = u[i*n+k]), V_i (n x p) and W_i (p x m, the C^T
 * order), over Q for TFG_MODE_ZT and over GF(2) for TFG_MODE_Z2; from them
 *   type_poly[a][b][c] = number of terms with ranks (a, b, c): the coefficients
 *                        of the type polynomial sum_i X^a Y^b Z^c;
 *   sym_poly[a][b][c]  = the type polynomial summed over the six permutations
 *                        of its variables (the symmetric invariant);
 *   rank_sums[3]       = sum_i rank U_i, sum_i rank V_i, sum_i rank W_i (the
 *                        exponents of the rank-sum polynomial).
 * type_poly and sym_poly are caller arrays of 12*12*12 int64, row-major [a][b][c]
 * (a factor of at most 128 entries has rank at most 11); term_ranks is [rank][3]
 * int32.  Any output pointer may be NULL.  TFG_EINVAL for a bad format, rank
 * or coefficient; the scheme is not required to satisfy Eq. (1). */
int tfg_isotropy_invariants(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t *term_ranks,
                            int64_t *type_poly, int64_t *sym_poly, int64_t *rank_sums);

/* Z_2 -> Z_T sign lifting (section "Ternary Lifting Script"): give every
 * non-zero coefficient of `scheme` -- a Z_2 scheme of format fmt (m, n, p;
 * the mode field is ignored), coefficients 0/1, Eq. (1) modulo 2 -- a sign so
 * that Eq. (1) holds over the integers, by exact search (entries covered by
 * one or two terms are linear equations over GF(2) in the sign bits; the free
 * bits are searched depth-first against the other entries; per term the first
 * non-zero of u and of v is +1).  out: caller buffer of rank rows; the result
 * has the same non-zero pattern, is sign-normalised and satisfies Eq. (1).
 * *nodes_used (may be NULL) receives the number of search nodes.
 * TFG_OK; TFG_ESCHEME when no sign assignment exists (exhaustive search);
 * TFG_ETIMEOUT when max_nodes nodes did not decide; TFG_EINVAL for a bad
 * format or rank, coefficients other than 0/1, or Eq. (1) failing mod 2. */
int tfg_lift_signs(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int64_t max_nodes, int8_t *out,
                   int64_t *nodes_used);

/* Section 3.6: per term, make the first non-zero of u and of v equal +1, w
 * absorbing the signs (in place; Z_T only, Z_2 unchanged). */
int tfg_canonicalize(const tfg_format *fmt, int32_t rank, int8_t *scheme);

/* Start preparation used by tfg_init: canonicalise, remove terms with a zero
 * factor, then apply every reduction (Section 3.3.1, terms sharing two
 * factors up to sign) until none applies.  out has room for `cap` terms;
 * *out_rank receives the new rank.  Input must pass tfg_verify. */
int tfg_prepare(const tfg_format *fmt, int32_t rank, const int8_t *scheme,
                int8_t *out, int32_t cap, int32_t *out_rank);

/* Meta operators, Section 3.3.2.  All are pure host functions writing into a
 * caller buffer of `cap` terms (TFG_ENOSPC when too small); *out_fmt and
 * *out_rank receive the result format and rank.  Outputs are sign-normalised
 * (Z_T) and verified with Eq. (1) before returning (TFG_EINTERNAL if not).
 * axis: 0 = m (rows of A and C), 1 = n (columns of A, rows of B),
 *       2 = p (columns of B and C). */

/* project: remove index `index` along `axis`, then remove terms with a zero factor. */
int tfg_project(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t axis, int32_t index,
                tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank);
/* extend: add one to a size by merging with the naive scheme of the new block
 * ((m,n,p:r) -> (m,n,p+1:r+mn) for axis 2). */
int tfg_extend(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t axis,
               tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank);
/* merge: (m,n,p1:r1) + (m,n,p2:r2) -> (m,n,p1+p2:r1+r2) for axis 2, likewise for 0, 1.
 * Scheme a's terms come first. */
int tfg_merge(const tfg_format *fmt_a, int32_t rank_a, const int8_t *scheme_a,
              const tfg_format *fmt_b, int32_t rank_b, const int8_t *scheme_b, int32_t axis,
              tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank);
/* double: merge a scheme with itself along `axis`. */
int tfg_double(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t axis,
               tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank);
/* product: tensor product (m1 m2, n1 n2, p1 p2 : r1 r2); term l1*r2 + l2, row index
 * i1*m2 + i2 and likewise for the other indices. */
int tfg_product(const tfg_format *fmt_a, int32_t rank_a, const int8_t *scheme_a,
                const tfg_format *fmt_b, int32_t rank_b, const int8_t *scheme_b,
                tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank);
/* swap sizes: perm 0..5 gives the result order of (m,n,p):
 * 0 (m,n,p), 1 (m,p,n) [the paper's swap], 2 (n,m,p), 3 (n,p,m), 4 (p,m,n), 5 (p,n,m). */
int tfg_swap_sizes(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t perm,
                   tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank);

/* ---- walker contexts (GPU) ------------------------------------------------ */

/* Device workspace bytes for a context of n_formats populations.  ranks are
 * the ranks of the prepared starts (tfg_prepare), walkers the population sizes. */
int tfg_workspace_size(int32_t n_formats, const tfg_format *fmts, const int32_t *ranks,
                       const int64_t *walkers, const tfg_params *params, size_t *bytes);

/* Create a context of n_formats walker populations (mixed formats run in one
 * call of tfg_walk).  schemes[f] is the start of population f (rank ranks[f],
 * host memory, copied); it must pass tfg_verify; it is prepared with
 * tfg_prepare, so workspace sizes must be computed from the prepared ranks.
 * Walker ids are global: params->walker_id_base + position, populations
 * contiguous in list order.  Walker w of population f draws its randomness
 * from Philox4x32-10 with key (seed_lo, seed_hi) and counter (t_lo, t_hi, id,
 * sub), so a trajectory depends only on (seed, id, step).
 * d_workspace: caller-owned device memory of >= tfg_workspace_size bytes,
 * 256-byte aligned.  cuda_stream: a cudaStream_t (NULL = legacy default
 * stream); all device work of the context is ordered on it.  The call copies
 * the starts to the device and returns after enqueueing (asynchronous). */
int tfg_init(int32_t n_formats, const tfg_format *fmts, const int32_t *ranks,
             const int8_t *const *schemes, const int64_t *walkers, uint64_t seed,
             const tfg_params *params, void *d_workspace, size_t workspace_bytes,
             void *cuda_stream, tfg_ctx **out);

/* Advance every walker by `steps` steps (Algorithm 1 with the plateau policy:
 * draw, try_flip, ternary check, zero-term removal, sign normalisation,
 * reduction cascade, best update, plus transition).  Asynchronous on the
 * context stream; errors of the launch are returned, errors of execution at
 * the next tfg_sync. */
int tfg_walk(tfg_ctx *ctx, int64_t steps);

/* Wait for the context stream; returns the first CUDA error seen, if any,
 * else TFG_ETIMEOUT when a bounded device wait of the context's work gave up
 * since the last tfg_sync (the context's status word, set by the device, read
 * here and cleared after reading; the context stays usable), else TFG_OK. */
int tfg_sync(tfg_ctx *ctx);

/* Best scheme of population `format_idx`: the walker with the lowest best rank
 * (ties: lowest walker id).  Copies it to `out` (cap terms), verifies it on
 * the device and on the host (Eq. (1); TFG_EINTERNAL on failure) and reports
 * its rank and global walker id.  Synchronous. */
int tfg_collect_best(tfg_ctx *ctx, int32_t format_idx, int8_t *out, int32_t cap,
                     int32_t *rank_out, int64_t *walker_out);

/* Verify every walker's best scheme on the device (Eq. (1), exact integers).
 * Asynchronous; *d_failures (device pointer, int64) receives the number of
 * walkers whose best scheme fails (it is zeroed first). */
int tfg_verify_all_async(tfg_ctx *ctx, int64_t *d_failures);

/* Aggregate counters of population `format_idx` (-1 = all) and, when
 * rank_hist != NULL, a histogram of best ranks: rank_hist[k] = walkers with
 * best_r == k for k < hist_len.  Synchronous. */
int tfg_stats_get(tfg_ctx *ctx, int32_t format_idx, tfg_stats *out, int64_t *rank_hist, int32_t hist_len);

/* Exploratory search (the Resize / population-synchronisation steps of the
 * paper's search loop): replace walkers [first, first + count) -- global ids,
 * all in one population -- by `scheme` (rank rows, the population's format
 * and mode).  The scheme must satisfy Eq. (1) (TFG_ESCHEME otherwise); it is
 * prepared like a start (tfg_prepare) and written to every walker's live and
 * best slots.  Each record restarts at rank = best rank = the prepared rank,
 * plateau 0, best step = its current step count, best_nnz its non-zero
 * coefficients; the walker id, step count,
 * counters and trajectory digest continue, so the walker's random stream goes
 * on.  TFG_ENOSPC when the prepared rank exceeds the population's r_max,
 * TFG_EINVAL for a bad range.  Ordered on the context stream and synchronous. */
int tfg_reseed(tfg_ctx *ctx, int64_t first, int64_t count, int32_t rank, const int8_t *scheme);

/* Resize on the device (the Resize kernel of the paper's exploratory search,
 * Section 3.4, with the meta operators of Section 3.3.2): walker
 * src_first + k (k < count; global ids, all in one population) has its live
 * scheme (use_best = 0) or its best scheme (1) transformed by one operator,
 * and the result replaces the live and best schemes of walker dst_first + k
 * (another population, whose format must be the operator's result format and
 * whose mode must be the source's).  Operators (op):
 *   TFG_RESIZE_PROJECT  axis, index: remove row/column `index` along axis
 *                       (0: rows of A and C, 1: columns of A / rows of B,
 *                       2: columns of B and C); terms with a zero factor go
 *   TFG_RESIZE_EXTEND   axis: merge with the naive scheme of the missing block
 *   TFG_RESIZE_DOUBLE   axis: merge the scheme with itself
 *   TFG_RESIZE_MERGE    axis: block concatenation with the aux scheme
 *   TFG_RESIZE_PRODUCT  Kronecker product with the aux scheme (source terms
 *                       outer, aux terms inner)
 *   TFG_RESIZE_SWAP     index = perm: the sizes reordered as
 *                       (fmt[a] for a in ((0,1,2),(0,2,1),(1,0,2),(1,2,0),(2,0,1),(2,1,0))[perm])
 * Term order follows the host meta operators (source terms, then the second
 * block); Z_T results are sign-normalised (Section 3.6).  No reduction pass is
 * run: the result is a valid scheme, reduced later by the walk.  The
 * destination record restarts like tfg_reseed (rank = best rank = the result's
 * rank, plateau 0, best step = its step count, best_nnz); walker id, step
 * count, counters and digest continue.  A walker whose result would exceed the
 * destination's r_max is left unchanged and counted in *skipped (then the
 * call returns TFG_ENOSPC).  The aux scheme (host rows, aux_fmt, the source's
 * mode) must satisfy Eq. (1).  d_scratch: caller device memory of at least
 * tfg_resize_scratch_bytes(...) bytes (maps, the aux scheme, a counter).
 * Ordered on the context stream and synchronous. */
#define TFG_RESIZE_PROJECT 0
#define TFG_RESIZE_EXTEND  1
#define TFG_RESIZE_DOUBLE  2
#define TFG_RESIZE_MERGE   3
#define TFG_RESIZE_PRODUCT 4
#define TFG_RESIZE_SWAP    5
typedef struct tfg_resize_args {
    int32_t op, axis, index, use_best;
    int64_t src_first, dst_first, count;
    tfg_format aux_fmt;          /* TFG_RESIZE_MERGE / TFG_RESIZE_PRODUCT */
    int32_t aux_rank;
    int32_t pad;
    const int8_t *aux_scheme;    /* host rows [aux_rank][LT of aux_fmt] */
} tfg_resize_args;
size_t tfg_resize_scratch_bytes(int32_t aux_rank, const tfg_format *aux_fmt, const tfg_format *out_fmt);
int tfg_resize(tfg_ctx *ctx, const tfg_resize_args *args, void *d_scratch, size_t scratch_bytes, int64_t *skipped);

/* Copy walkers [first, first+count) (context-global positions) to the host:
 * info[count]; slots and best (either may be NULL) as int8 schemes of
 * [count][r_max][LT] of that walker's population (all walkers of the range
 * must belong to one population).  Synchronous.  For parity checks and export. */
int tfg_read_walkers(tfg_ctx *ctx, int64_t first, int64_t count, tfg_walker_info *info,
                     int8_t *slots, int8_t *best, int32_t r_max_cap);

/* Shape of population f: its format, prepared start rank, r_max, walker count
 * and position of its first walker. */
int tfg_population(tfg_ctx *ctx, int32_t f, tfg_format *fmt, int32_t *r0, int32_t *r_max,
                   int64_t *walkers, int64_t *first);

/* Checkpoint: copy the whole device state (all walkers) into a host buffer of
 * cap bytes (*used receives the size; call with buf = NULL to query).  Restore
 * writes it back into a context created with the same arguments; a restored
 * walk continues bit-identically.  Synchronous. */
int tfg_checkpoint(tfg_ctx *ctx, void *buf, size_t cap, size_t *used);
int tfg_restore(tfg_ctx *ctx, const void *buf, size_t size);

/* Autotuner: the candidates of a population are its compiled kernel variants
 * -- every mapping (one thread per walker; 4, 8, 16 or 32 lanes per walker) and,
 * for each, every walkers-per-block choice (the block sizes compiled for the
 * thread-per-walker kernel of that capacity, whose shared memory per block
 * depends on it; 128 or 256 threads for the lane-group kernels).  Population
 * by population, each candidate is timed for trial_steps steps on the first
 * min(walkers, trial_walkers) walkers of every population, all populations
 * launched as tfg_walk launches them (concurrently for use_graph 2) with the
 * others at their current choice; a candidate replaces the current choice
 * when it is more than 1% faster.  The trial walkers' state is restored bit for
 * bit afterwards (host copies; no device memory is allocated); the choice
 * changes no trajectory.  lanes_out[f] (optional) receives the chosen lanes
 * per walker; tfg_launch_shape reports the whole launch shape.  Synchronous. */
int tfg_autotune(tfg_ctx *ctx, int64_t trial_steps, int64_t trial_walkers, int32_t *lanes_out);

/* Launch shape of population f's walk kernel: lanes per walker, threads per
 * block (walkers per block = block_threads / lanes) and blocks.  Any output may
 * be NULL. */
int tfg_launch_shape(tfg_ctx *ctx, int32_t f, int32_t *lanes, int32_t *block_threads, int64_t *grid);

/* Mapping chosen for population f: lanes per walker G, slots per lane S (the
 * slot capacity for one thread per walker; 0 for the warp-per-walker kernel),
 * and slice_len > 0 when the thread-per-walker kernel also keeps the slots
 * bit-sliced (one word per coefficient, bit k = slot k; formats whose factors
 * have at most slice_len coefficients), else 0; square = 1 when that kernel is
 * the instantiation for three factors of exactly slice_len coefficients
 * (offsets and masks compiled in), else 0.  Each output may be NULL. */
int tfg_mapping(tfg_ctx *ctx, int32_t f, int32_t *lanes, int32_t *slots_per_lane, int32_t *slice_len,
                int32_t *square);

/* Release the context (host memory only; the workspace stays the caller's). */
void tfg_destroy(tfg_ctx *ctx);

/* ---- learned flip proposal (not in the paper) ------------------------------ */

/* Scoring MLP 32 -> 128 -> 128 -> 1 with ReLU, BF16 weights and inputs, FP32
 * accumulation, run on the tensor cores (tcgen05).  Parameter blob layout
 * (device memory, tfg_mlp_param_bytes() bytes, 16-byte aligned):
 *   W1  bf16 [32][128]   (row = input feature)
 *   W2  bf16 [128][128]  (row = first hidden unit)
 *   b1, b2, w3  f32 [128] each;  b3  f32 (then 12 bytes of padding).
 * score = w3 . relu(W2^T relu(W1^T x + b1) + b2) + b3, with the first hidden
 * layer rounded to bf16 before the second product. */
size_t tfg_mlp_param_bytes(void);

/* Scores n candidate feature rows d_x (bf16 [n][32], device, 16-byte aligned)
 * into d_out (f32 [n], device).  Asynchronous on cuda_stream; *d_err (device
 * int32, caller-zeroed) is set to 1 if a tensor-core completion wait gave up. */
int tfg_mlp_score(const void *d_params, const uint16_t *d_x, int64_t n, float *d_out, int32_t *d_err,
                  void *cuda_stream);

/* Training of the scoring MLP on the tensor cores.  Samples: features d_x (bf16
 * [n][32]), labels d_label (f32 0/1 [n]), weights d_weight (f32 [n]); loss =
 * sum_k weight_k * log(1 + exp(-(2 label_k - 1) score_k)) (weighted logistic).
 * Parameter vector order of every gradient / state array: W1 [32][128], W2
 * [128][128], b1, b2, w3 [128] each, b3 (P = 20865 floats).  The first hidden
 * layer and the hidden-layer gradients enter the products as bf16.
 *
 * tfg_mlp_grad: d_grad (device f32 [P + 1], overwritten) receives the gradient
 * and, at [P], the loss.  Asynchronous; *d_err set to 1 if a tensor-core
 * completion wait gave up.
 * The gradient's per-CTA sums are added by atomics, so its low bits may vary
 * from run to run.
 * tfg_mlp_train_state_bytes / tfg_mlp_train_init: optimizer state (FP32 master
 * weights, Adam moments, gradient, and one gradient row per CTA of the
 * training step's gradient launch) in caller device memory, initialised from
 * the parameter blob.
 * tfg_mlp_train_step: one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step
 * counted from 1) on the samples; rewrites d_params (bf16 W1, W2, f32 rest).
 * Its gradient adds the per-CTA rows in CTA order: the same inputs give the
 * same bits on every run (on a GPU of the same SM count). */
int tfg_mlp_grad(const void *d_params, const uint16_t *d_x, const float *d_label, const float *d_weight, int64_t n,
                 float *d_grad, int32_t *d_err, void *cuda_stream);
size_t tfg_mlp_train_state_bytes(void);
int tfg_mlp_train_init(void *d_state, const void *d_params, void *cuda_stream);
int tfg_mlp_train_step(void *d_state, void *d_params, const uint16_t *d_x, const float *d_label,
                       const float *d_weight, int64_t n, float lr, int32_t step, int32_t *d_err, void *cuda_stream);

/* Window-mode walk (the step the learned proposal acts on).  Each step of a
 * walker considers a window of up to 256 try_flip candidates: starting at term
 * i0 = mulhi(x0, r), terms i0, i0+1, ... (mod r) append their candidates in
 * (factor, slot, rho) order until 256 are collected.  Candidate (X, j, s, rho)
 * of term i flips Y_i' = Y_i + Y_j and Z_j' = Z_j - s Z_i, where (Y, Z) are the
 * two factors after X in the order u, v, w, swapped when rho = 1.  Its 32
 * features (bf16 values of small integers; nnz = number of non-zero
 * coefficients):
 *   f0..f2  one-hot X (u, v, w)        f3  rho            f4  1 when s = -1
 *   f5  nnz(X_i)   f6  nnz(Y_i)   f7  nnz(Y_j)
 *   f8  nnz(Y_i + Y_j) when that sum stays in Z_T, else 0;  f9  1 when it does
 *   f10 nnz(Z_i)   f11 nnz(Z_j)
 *   f12 nnz(Z_j - s Z_i) when in Z_T, else 0;  f13  1 when it is
 *   f14 positions where Y_i and Y_j are both non-zero;  f15  the same for Z
 *   f16 1 when Y_i + Y_j is valid and zero;  f17  1 when Z_j - s Z_i is
 *   f18 the number of candidates of term i, at most 64
 *   f19 r - best_r   f20 r   f21 m   f22 n   f23 p
 *   f24 the position q of term i after i0 (i = i0 + q mod r), at most 64
 *   f25..f30 0       f31 1
 * (tfg_window_dump writes them; the learned step computes them in shared
 * memory, on the tensor-core kernel, from the window's candidate list.)
 * policy 0 (uniform): candidate mulhi(x1, K);
 * policy 1 (learned): with x3 < eps_thresh as policy 0, else the candidate of
 * highest MLP score (first on ties); d_mlp_params is the parameter blob of
 * tfg_mlp_score (device, 16-byte aligned, TFG_EINVAL otherwise).  The chosen flip then goes through the
 * same validity test, reductions and bookkeeping as tfg_walk.
 * Populations must be Z_T with m*n + n*p + p*m <= 64 and r_max <= 88.
 * d_scratch: caller device memory of tfg_window_scratch_bytes (per walker
 * the window's candidate descriptors, scores and size: 3076 bytes).  d_choices (optional, device int32
 * [steps][walkers]) receives the chosen window index of every step (-1: no
 * candidate).  log (optional): chosen features with label 1 when the step
 * lowered the rank (always kept) or 0 (kept when a Philox draw of sub-stream
 * 256 is below neg_thresh), appended at d_count (device int64, caller-zeroed)
 * up to capacity entries.  With horizon H > 1 each walker keeps a ring of the
 * features of its last H chosen candidates; a step that lowers the rank
 * appends (label 1, each with its own step) every ring entry chosen at steps
 * t - H + 1 .. t since the walker's previous such step, in step order, and
 * empties the ring; label-0 entries are this step's alone, as for H = 1 (a
 * step logged with label 0 can later be logged again with label 1).  The
 * ring persists across calls in caller memory: d_ring (device bf16
 * [walkers][H][32], 16-byte aligned) and d_ring_step (device uint32
 * [walkers][H], the step of each entry, 0xFFFFFFFF = empty, which the caller
 * writes into every word before the first call); walkers = all of the
 * context's, in its walker order.  The window of steps is taken on the low
 * 32 bits of the step counter. */
typedef struct {
    uint16_t feat[32];  /* bf16 features of the chosen candidate */
    float label;        /* 1: the step lowered the rank */
    uint32_t walker_id, step, pad;
} tfg_log_entry;

typedef struct {
    tfg_log_entry *d_entries;
    int64_t capacity;
    int64_t *d_count;
    uint32_t neg_thresh;
    int32_t horizon;        /* H: 0 or 1 = this step's features only; 2..64 = the ring */
    uint16_t *d_ring;       /* H > 1 */
    uint32_t *d_ring_step;  /* H > 1 */
} tfg_log_spec;

int tfg_window_scratch_bytes(tfg_ctx *ctx, size_t *bytes);

/* The window the next window-mode step of every walker would consider, without
 * stepping (for inspection and tests).  d_desc (device, uint32 [walkers][256][2],
 * 8-byte aligned): per window row the candidate descriptor i | X << 10 |
 * j << 12 | (s < 0) << 22 | rho << 23 and the info word min(count of term i's
 * candidates, 64) | min(q, 64) << 8; rows past the window are not written.
 * d_kwin (device, int32 [walkers]): the window sizes K.  d_feat (optional,
 * device bf16 [walkers][256][32], 16-byte aligned): the features listed
 * above, rows past K zero.  Asynchronous on the context stream. */
int tfg_window_dump(tfg_ctx *ctx, uint16_t *d_feat, uint32_t *d_desc, int32_t *d_kwin);

int tfg_walk_window(tfg_ctx *ctx, int64_t steps, int32_t policy, const void *d_mlp_params, uint32_t eps_thresh,
                    void *d_scratch, size_t scratch_bytes, int32_t *d_choices, const tfg_log_spec *log);

/* tfg_walk_window without any caller scratch: the paper has no counterpart to
 * this entry point.  It is for callers that cannot call cudaMalloc (code that
 * runs inside another framework's memory arena, or a process whose device
 * memory is reserved up front): the window's candidate descriptors, scores
 * and sizes live in a 32 MiB array that the library itself defines as static
 * device memory, which every GPU that loads the library holds until the
 * process exits.  Contexts of more than 10908 walkers (the array's capacity at
 * 3076 bytes per walker) are rejected with TFG_EINVAL and a message.  The call
 * allocates nothing: tfg_init already looked up the array's device address on
 * its device, which loads the library's module there and so reserves the
 * 32 MiB at that point at the latest (under lazy module loading; at library
 * load otherwise).  The context's device must be current (TFG_EINVAL
 * otherwise).  All calls share the one array (it keeps the last
 * call's contents; every value a step reads is written by the same step), so
 * calls whose work overlaps on the GPU, such as two contexts on different
 * streams, race on it and must be serialised by the caller.  Results equal
 * tfg_walk_window's for the same context and arguments. */
int tfg_walk_window_noalloc(tfg_ctx *ctx, int64_t steps, int32_t policy, const void *d_mlp_params,
                            uint32_t eps_thresh, int32_t *d_choices, const tfg_log_spec *log);

/* Test hook of the bounded device waits: the first tensor-core completion
 * wait of every CTA of the scoring network (tfg_mlp_score and the learned
 * window mode) polls at most `polls` times in later launches; a negative
 * value restores the default of 2^22 polls, 0 makes that wait give up at
 * once.  A CTA whose wait gave up skips its remaining tiles, waits (with the
 * default limit) for its products in flight, releases its tensor memory and
 * sets its error word: *d_err of tfg_mlp_score, or in window mode the
 * context's status word, which the next tfg_sync returns as TFG_ETIMEOUT.
 * Process-wide setting; it changes no result of a launch whose waits finish. */
void tfg_test_set_wait_limit(int64_t polls);

/* Philox4x32-10 of the device path, for tests: d_out[4k..4k+3] = Philox(d_ctr[4k..4k+3],
 * key), n counters; d_ctr and d_out are caller-owned device arrays of 4n words.
 * Synchronous on cuda_stream. */
int tfg_philox_device(const uint32_t *d_ctr, int32_t n, uint32_t key_lo, uint32_t key_hi, uint32_t *d_out,
                      void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TFG_H */
