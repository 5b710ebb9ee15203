/*
 * Reference oracle for the ternary (and binary) flip-graph random walk.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Representation: every factor vector is a plain array of int8 coefficients
 * (the "straightforward approach" of Section 3.5, deliberately the slow one),
 * every step is written out in the order of Algorithm 1 with the operators of
 * Section 3.3, and no step is blocked, fused or reordered.
 *
 * Layout of a scheme (also the layout of the C ABI): term l occupies one row of
 * LT = mn + np + pm int8 entries: u[i*n+k] (coefficient of a_ik), then
 * v[k*p+j] (b_kj), then w[j*m+i] (c_ij, the C^T convention of Section 3.1).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11), written from that description.
 *
 * Pins (tests/test_oracle_*.py): Philox known-answer vectors of the Random123
 * distribution; Brent validity of the paper's (2,2,3:11) example (Section
 * 3.1.1), of the naive scheme and of a textbook Strassen scheme; the paper's
 * sign-normalisation example (Section 3.6) reproduced exactly; the tensor
 * invariant after every single step; brute-force candidate enumeration;
 * closed-form ranks of the meta operators (Section 3.3.2).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_MODE_ZT 0
#define ORC_MODE_Z2 1

#define ORC_NOCAND 0
#define ORC_REJECT 1
#define ORC_ACCEPT 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the SC'11 paper: 10 rounds of two 32x32->64 multiplies */
/* with the Weyl key schedule.                                                */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;   /* golden ratio */
            k1 += 0xBB67AE85u;   /* sqrt(3) - 1 */
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Range reduction of a 32-bit draw onto [0, n): multiply-shift. */
static uint32_t mulhi_range(uint32_t x, uint32_t n)
{
    return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Format                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int m, n, p, mode;
    int len[3];   /* lengths of u, v, w */
    int off[3];   /* offsets of u, v, w inside a term row */
    int LT;       /* entries per term */
} orc_fmt;

static orc_fmt make_fmt(int m, int n, int p, int mode)
{
    orc_fmt f;
    f.m = m; f.n = n; f.p = p; f.mode = mode;
    f.len[0] = m * n; f.len[1] = n * p; f.len[2] = p * m;
    f.off[0] = 0; f.off[1] = f.len[0]; f.off[2] = f.len[0] + f.len[1];
    f.LT = f.len[0] + f.len[1] + f.len[2];
    return f;
}

static int8_t *factor(const orc_fmt *f, int8_t *scheme, int term, int which)
{
    return scheme + (size_t)term * f->LT + f->off[which];
}

static int coeff_in_set(int c, int mode)
{
    if (mode == ORC_MODE_Z2) return c == 0 || c == 1;
    return c >= -1 && c <= 1;
}

/* out = a + s*b, reduced mod 2 in Z_2; returns 1 when every entry stays in the
 * coefficient set (Section 3.5.2: the validity flag of addition/subtraction). */
static int vec_add(int8_t *out, const int8_t *a, const int8_t *b, int s, int L, int mode)
{
    int ok = 1;
    for (int e = 0; e < L; ++e) {
        int c = (int)a[e] + s * (int)b[e];
        if (mode == ORC_MODE_Z2) c = ((c % 2) + 2) % 2;
        if (!coeff_in_set(c, mode)) ok = 0;
        out[e] = (int8_t)c;
    }
    return ok;
}

/* 1 when a == s*b entry-wise (Z_2: s is always +1). */
static int vec_equal(const int8_t *a, const int8_t *b, int s, int L)
{
    for (int e = 0; e < L; ++e)
        if ((int)a[e] != s * (int)b[e]) return 0;
    return 1;
}

static int vec_is_zero(const int8_t *a, int L)
{
    for (int e = 0; e < L; ++e)
        if (a[e] != 0) return 0;
    return 1;
}

static void vec_negate(int8_t *a, int L)
{
    for (int e = 0; e < L; ++e) a[e] = (int8_t)(-a[e]);
}

static int first_nonzero(const int8_t *a, int L)
{
    for (int e = 0; e < L; ++e)
        if (a[e] != 0) return a[e];
    return 0;
}

/* Sign-symmetry breaking (Section 3.6), applied per term: the first non-zero
 * coefficient of u and of v is made +1; w absorbs both signs.  This is the
 * reading under which the paper's example (U,V,W) -> (U',V',W') holds. */
static void canonicalize_term(const orc_fmt *f, int8_t *scheme, int t)
{
    if (f->mode != ORC_MODE_ZT) return;
    int8_t *u = factor(f, scheme, t, 0), *v = factor(f, scheme, t, 1), *w = factor(f, scheme, t, 2);
    if (first_nonzero(u, f->len[0]) < 0) { vec_negate(u, f->len[0]); vec_negate(w, f->len[2]); }
    if (first_nonzero(v, f->len[1]) < 0) { vec_negate(v, f->len[1]); vec_negate(w, f->len[2]); }
}

void orc_canonicalize(int m, int n, int p, int mode, int r, int8_t *scheme)
{
    orc_fmt f = make_fmt(m, n, p, mode);
    for (int t = 0; t < r; ++t) canonicalize_term(&f, scheme, t);
}

/* ------------------------------------------------------------------------ */
/* Brent equations, Eq. (1), in the C^T convention: the reconstructed tensor   */
/* sum_l u_l (x) v_l (x) w_l must equal T with T[i*n+k][k*p+j][j*m+i] = 1.     */
/* Exact integer arithmetic (mod 2 for Z_2).  Returns 1 when valid.            */
/* ------------------------------------------------------------------------ */
int orc_brent_valid(int m, int n, int p, int mode, int r, const int8_t *scheme)
{
    orc_fmt f = make_fmt(m, n, p, mode);
    for (int i1 = 0; i1 < m; ++i1)
    for (int i2 = 0; i2 < n; ++i2)
    for (int j1 = 0; j1 < n; ++j1)
    for (int j2 = 0; j2 < p; ++j2)
    for (int k2 = 0; k2 < p; ++k2)
    for (int k1 = 0; k1 < m; ++k1) {
        long long sum = 0;
        for (int l = 0; l < r; ++l) {
            const int8_t *row = scheme + (size_t)l * f.LT;
            sum += (long long)row[f.off[0] + i1 * n + i2]
                 * (long long)row[f.off[1] + j1 * p + j2]
                 * (long long)row[f.off[2] + k2 * m + k1];
        }
        long long rhs = (i2 == j1 && i1 == k1 && j2 == k2) ? 1 : 0;
        if (mode == ORC_MODE_Z2) {
            if ((((sum - rhs) % 2) + 2) % 2 != 0) return 0;
        } else if (sum != rhs) {
            return 0;
        }
    }
    return 1;
}

/* Naive additive complexity (Section 4.5): nnz(U)+nnz(V)+nnz(W) - 2r - m*p. */
long long orc_additive_complexity(int m, int n, int p, int r, const int8_t *scheme)
{
    orc_fmt f = make_fmt(m, n, p, ORC_MODE_ZT);
    long long nnz = 0;
    for (size_t e = 0; e < (size_t)r * f.LT; ++e) nnz += scheme[e] != 0;
    return nnz - 2LL * r - (long long)m * p;
}

/* ------------------------------------------------------------------------ */
/* Walker state                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t plateau_len;     /* L: plateau length that triggers a plus transition */
    uint32_t refresh_thresh; /* equal-rank best refresh when x2 < this (0.01 * 2^32) */
    int32_t plus_attempts;   /* Philox sub-streams 1..plus_attempts */
    int32_t plus_enabled;
    int32_t debug_checks;    /* re-verify the invariants after every step */
    int32_t policy;          /* 0: plus transition on a plateau; 1: Algorithm 1 (expand when try_flip
                                fails, and after a flip with probability p_expand); 2: naive additive
                                complexity minimisation (flips and zero-term removal only, the best
                                scheme is the one of least (rank, non-zero coefficients)) */
    uint32_t expand_thresh;  /* policy 1: expand after a flip when x3 < floor(p_expand * 2^32) */
} orc_params;

typedef struct {
    int32_t r, best_r, r_max, best_nnz;   /* best_nnz: non-zero coefficients of the best scheme */
    int64_t t, plateau, best_t;
    uint64_t digest;
    int64_t accepted, rejected, nocand, drops, merges, plus, reductions;
    int64_t debug_failures;
    int64_t ops;             /* algorithmic word operations of the uniform steps (walk_step_ops) */
} orc_info;

typedef struct {
    const orc_fmt *f;
    const orc_params *prm;
    int8_t *slots;           /* [r_max][LT] */
    int8_t *best;            /* [r_max][LT] */
    orc_info *info;
    uint32_t walker_id;
    uint32_t key[2];
} walker;

/* Digest: a 64-bit multiply-xorshift mix of one packed record per event. */
static uint64_t digest_mix(uint64_t h, uint64_t v)
{
    h ^= v;
    h *= 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    return h;
}

uint64_t orc_digest_init(uint32_t walker_id)
{
    return 0xCBF29CE484222325ull ^ (uint64_t)walker_id;
}

/* Queue of modified terms awaiting reduction checks (at most three entries). */
typedef struct { int item[8]; int len; } queue_t;

static void q_push(queue_t *q, int v) { q->item[q->len++] = v; }
static int q_pop_front(queue_t *q)
{
    int v = q->item[0];
    for (int a = 1; a < q->len; ++a) q->item[a - 1] = q->item[a];
    q->len--;
    return v;
}
static void q_remove(queue_t *q, int v)
{
    int o = 0;
    for (int a = 0; a < q->len; ++a)
        if (q->item[a] != v) q->item[o++] = q->item[a];
    q->len = o;
}
static void q_rename(queue_t *q, int from, int to)
{
    for (int a = 0; a < q->len; ++a)
        if (q->item[a] == from) q->item[a] = to;
}

/* Remove the term in slot h: the last live term moves into the hole. */
static void drop_slot(walker *wk, int h, queue_t *q)
{
    const orc_fmt *f = wk->f;
    int last = wk->info->r - 1;
    q_remove(q, h);
    if (h != last) {
        memcpy(wk->slots + (size_t)h * f->LT, wk->slots + (size_t)last * f->LT, (size_t)f->LT);
        q_rename(q, last, h);
    }
    wk->info->r -= 1;
}

/* Reduction (Section 3.3.1) applied to "any permutation" of (u, v, w): terms t
 * and k that share the factor pair P up to signs merge into one term whose
 * third factor is F_t + sigma*F_k.  Pairs are tried in the order (u,v), (u,w),
 * (v,w); within a pair the lowest slot k != t whose merged third factor stays
 * in the coefficient set is taken.  Returns 1 when a merge happened. */
static const int PAIR_A[3] = {0, 0, 1};
static const int PAIR_B[3] = {1, 2, 2};
static const int PAIR_F[3] = {2, 1, 0};

static int try_reduce_term(walker *wk, int t, queue_t *q)
{
    const orc_fmt *f = wk->f;
    int r = wk->info->r;
    int8_t tmp[128];
    int sgn[2] = {1, -1};
    int nsg = (f->mode == ORC_MODE_Z2) ? 1 : 2;
    for (int P = 0; P < 3; ++P) {
        int A = PAIR_A[P], B = PAIR_B[P], F = PAIR_F[P];
        for (int k = 0; k < r; ++k) {
            if (k == t) continue;
            for (int ia = 0; ia < nsg; ++ia)
            for (int ib = 0; ib < nsg; ++ib) {
                int a = sgn[ia], b = sgn[ib];
                if (!vec_equal(factor(f, wk->slots, k, A), factor(f, wk->slots, t, A), a, f->len[A])) continue;
                if (!vec_equal(factor(f, wk->slots, k, B), factor(f, wk->slots, t, B), b, f->len[B])) continue;
                int sigma = a * b;
                if (!vec_add(tmp, factor(f, wk->slots, t, F), factor(f, wk->slots, k, F), sigma,
                             f->len[F], f->mode))
                    continue;
                /* merge: (A_t, B_t, F_t + sigma F_k) goes to slot min(t,k) */
                int lo = t < k ? t : k, hi = t < k ? k : t;
                if (lo != t)
                    memcpy(wk->slots + (size_t)lo * f->LT, wk->slots + (size_t)t * f->LT, (size_t)f->LT);
                memcpy(factor(f, wk->slots, lo, F), tmp, (size_t)f->len[F]);
                q_remove(q, t);
                q_remove(q, k);
                drop_slot(wk, hi, q);
                wk->info->merges += 1;
                if (vec_is_zero(factor(f, wk->slots, lo, F), f->len[F])) {
                    drop_slot(wk, lo, q);
                    wk->info->drops += 1;
                } else {
                    canonicalize_term(f, wk->slots, lo);
                    q_push(q, lo);
                }
                return 1;
            }
        }
    }
    return 0;
}

/* "Flip with reduction edge checking" (Section 3.4.1): every modified term is
 * checked against every other term until no reduction applies. */
static void reduction_cascade(walker *wk, queue_t *q)
{
    while (q->len > 0) {
        int t = q_pop_front(q);
        try_reduce_term(wk, t, q);
    }
}

/* Candidate list of try_flip for the sampled term i: every j != i and factor X
 * with X_j = s * X_i, each giving two flips (rho = 0, 1). */
typedef struct { int X, j, s, rho; } cand_t;

static int enumerate_candidates(const walker *wk, int i, cand_t *out)
{
    const orc_fmt *f = wk->f;
    int r = wk->info->r, K = 0;
    int nsg = (f->mode == ORC_MODE_Z2) ? 1 : 2;
    int sgn[2] = {1, -1};
    for (int X = 0; X < 3; ++X)
        for (int j = 0; j < r; ++j) {
            if (j == i) continue;
            for (int is = 0; is < nsg; ++is) {
                int s = sgn[is];
                if (vec_equal(factor(f, wk->slots, j, X), factor(f, wk->slots, i, X), s, f->len[X])) {
                    cand_t c0 = {X, j, s, 0}, c1 = {X, j, s, 1};
                    out[K++] = c0;
                    out[K++] = c1;
                    break;
                }
            }
        }
    return K;
}

int orc_enumerate_candidates(int m, int n, int p, int mode, int r, const int8_t *scheme, int i,
                             int32_t *out4 /* [K][4]: X, j, s, rho */)
{
    orc_fmt f = make_fmt(m, n, p, mode);
    orc_info info; memset(&info, 0, sizeof info); info.r = r;
    walker wk; memset(&wk, 0, sizeof wk);
    wk.f = &f; wk.slots = (int8_t *)scheme; wk.info = &info;
    cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (size_t)(6 * r + 6));
    int K = enumerate_candidates(&wk, i, c);
    for (int a = 0; a < K; ++a) {
        out4[4 * a + 0] = c[a].X; out4[4 * a + 1] = c[a].j;
        out4[4 * a + 2] = c[a].s; out4[4 * a + 3] = c[a].rho;
    }
    free(c);
    return K;
}

static void take_best(walker *wk)
{
    memcpy(wk->best, wk->slots, (size_t)wk->info->r * wk->f->LT);
}

/* ---- invariants for debug mode ---------------------------------------- */
static int all_canonical(const walker *wk)
{
    const orc_fmt *f = wk->f;
    if (f->mode != ORC_MODE_ZT) return 1;
    for (int t = 0; t < wk->info->r; ++t) {
        if (first_nonzero(factor(f, wk->slots, t, 0), f->len[0]) <= 0) return 0;
        if (first_nonzero(factor(f, wk->slots, t, 1), f->len[1]) <= 0) return 0;
    }
    return 1;
}

static int no_zero_factor(const walker *wk)
{
    for (int t = 0; t < wk->info->r; ++t)
        for (int X = 0; X < 3; ++X)
            if (vec_is_zero(factor(wk->f, wk->slots, t, X), wk->f->len[X])) return 0;
    return 1;
}

static int no_reducible_pair(walker *wk)
{
    const orc_fmt *f = wk->f;
    int r = wk->info->r;
    int8_t tmp[128];
    int nsg = (f->mode == ORC_MODE_Z2) ? 1 : 2;
    int sgn[2] = {1, -1};
    for (int t = 0; t < r; ++t)
        for (int k = t + 1; k < r; ++k)
            for (int P = 0; P < 3; ++P)
                for (int ia = 0; ia < nsg; ++ia)
                    for (int ib = 0; ib < nsg; ++ib) {
                        int A = PAIR_A[P], B = PAIR_B[P], F = PAIR_F[P];
                        if (!vec_equal(factor(f, wk->slots, k, A), factor(f, wk->slots, t, A), sgn[ia], f->len[A])) continue;
                        if (!vec_equal(factor(f, wk->slots, k, B), factor(f, wk->slots, t, B), sgn[ib], f->len[B])) continue;
                        if (vec_add(tmp, factor(f, wk->slots, t, F), factor(f, wk->slots, k, F), sgn[ia] * sgn[ib], f->len[F], f->mode))
                            return 0;
                    }
    return 1;
}

static void debug_check(walker *wk)
{
    const orc_fmt *f = wk->f;
    /* policy 2 has no reduction edges, so reducible pairs may remain */
    if (!orc_brent_valid(f->m, f->n, f->p, f->mode, wk->info->r, wk->slots) ||
        !all_canonical(wk) || !no_zero_factor(wk) || (wk->prm->policy != 2 && !no_reducible_pair(wk)))
        wk->info->debug_failures += 1;
}

/* Expansions (Section 3.3.1).  Roles (A,B,C) are a permutation of (u,v,w).
 * Plus: the pair (i, j) becomes three terms
 *   A_i (x) (B_i + B_j) (x) C_i  +  A_i (x) B_j (x) (C_j - C_i)  +  (A_j - A_i) (x) B_j (x) C_j;
 * each of the three new factors must be non-zero and stay in the coefficient set.
 * Split (policy 1 only): term i becomes A_j (x) B_i (x) C_i and the new term
 *   (A_i - A_j) (x) B_i (x) C_i  is appended (term j unchanged); A_i - A_j must be
 * non-zero (A_i != A_j) and stay in the coefficient set.
 * Attempt a = 1..plus_attempts draws Philox sub-stream a: i from y0, j != i from
 * y1, the role permutation from y2, and (policy 1) split when y3 >= 2^31, else
 * plus.  The new term goes to slot r.  Returns the attempt that succeeded, or 0. */
static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static int try_expand(walker *wk, uint64_t t, int *pi_out, int *pj_out, int *perm_out, int *split_out)
{
    const orc_fmt *f = wk->f;
    int r = wk->info->r;
    if (r < 2) return 0;
    for (int a = 1; a <= wk->prm->plus_attempts; ++a) {
        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), wk->walker_id, (uint32_t)a}, y[4];
        orc_philox4x32_10(ctr, wk->key, y);
        int i = (int)mulhi_range(y[0], (uint32_t)r);
        int j = (int)((i + 1 + (int)mulhi_range(y[1], (uint32_t)(r - 1))) % r);
        int pi = (int)mulhi_range(y[2], 6u);
        int split = (wk->prm->policy == 1) && (y[3] >= 0x80000000u);
        int A = PERM[pi][0], B = PERM[pi][1], C = PERM[pi][2];
        int nt = r;
        if (split) {
            int8_t na[128];
            if (!vec_add(na, factor(f, wk->slots, i, A), factor(f, wk->slots, j, A), -1, f->len[A], f->mode) ||
                vec_is_zero(na, f->len[A]))
                continue;
            /* new term r: (A_i - A_j, B_i, C_i) */
            memcpy(factor(f, wk->slots, nt, A), na, (size_t)f->len[A]);
            memcpy(factor(f, wk->slots, nt, B), factor(f, wk->slots, i, B), (size_t)f->len[B]);
            memcpy(factor(f, wk->slots, nt, C), factor(f, wk->slots, i, C), (size_t)f->len[C]);
            /* term i: (A_j, B_i, C_i) */
            memcpy(factor(f, wk->slots, i, A), factor(f, wk->slots, j, A), (size_t)f->len[A]);
            wk->info->r = r + 1;
            canonicalize_term(f, wk->slots, i);
            canonicalize_term(f, wk->slots, nt);
        } else {
            int8_t nb[128], nc[128], na[128];
            int ok = vec_add(nb, factor(f, wk->slots, i, B), factor(f, wk->slots, j, B), +1, f->len[B], f->mode);
            ok &= vec_add(nc, factor(f, wk->slots, j, C), factor(f, wk->slots, i, C), -1, f->len[C], f->mode);
            ok &= vec_add(na, factor(f, wk->slots, j, A), factor(f, wk->slots, i, A), -1, f->len[A], f->mode);
            if (!ok || vec_is_zero(nb, f->len[B]) || vec_is_zero(nc, f->len[C]) || vec_is_zero(na, f->len[A]))
                continue;
            /* new term r: (A_j - A_i, B_j, C_j) */
            memcpy(factor(f, wk->slots, nt, A), na, (size_t)f->len[A]);
            memcpy(factor(f, wk->slots, nt, B), factor(f, wk->slots, j, B), (size_t)f->len[B]);
            memcpy(factor(f, wk->slots, nt, C), factor(f, wk->slots, j, C), (size_t)f->len[C]);
            /* term j: (A_i, B_j, C_j - C_i) */
            memcpy(factor(f, wk->slots, j, A), factor(f, wk->slots, i, A), (size_t)f->len[A]);
            memcpy(factor(f, wk->slots, j, C), nc, (size_t)f->len[C]);
            /* term i: (A_i, B_i + B_j, C_i) */
            memcpy(factor(f, wk->slots, i, B), nb, (size_t)f->len[B]);
            wk->info->r = r + 1;
            canonicalize_term(f, wk->slots, i);
            canonicalize_term(f, wk->slots, j);
            canonicalize_term(f, wk->slots, nt);
        }
        *pi_out = i; *pj_out = j; *perm_out = pi; *split_out = split;
        return a;
    }
    return 0;
}

/* An expansion followed by the reduction cascade over the changed terms, and
 * its digest record; a successful one restarts the plateau.  Returns whether
 * an attempt succeeded. */
static int expand_step(walker *wk, uint64_t t)
{
    orc_info *in = wk->info;
    int pi = 0, pj = 0, perm = 0, split = 0;
    int a = try_expand(wk, t, &pi, &pj, &perm, &split);
    if (a == 0) return 0;
    in->plus += 1;
    in->plateau = 0;
    queue_t q; q.len = 0;
    q_push(&q, pi);
    if (!split) q_push(&q, pj);
    q_push(&q, in->r - 1);
    reduction_cascade(wk, &q);
    uint64_t rec2 = 0xFull | ((uint64_t)a << 4) | ((uint64_t)perm << 9) |
                    ((uint64_t)(uint32_t)pi << 12) | ((uint64_t)(uint32_t)pj << 28) |
                    ((uint64_t)(uint32_t)in->r << 44) | ((uint64_t)split << 62);
    in->digest = digest_mix(in->digest, rec2);
    return 1;
}

/* Flip (Section 3.3.1) of candidate c on sampled term i, followed by the
 * removal of zero terms, sign normalisation of the modified terms and the
 * reduction cascade.  Returns ORC_ACCEPT, or ORC_REJECT when a new factor
 * leaves the coefficient set (state unchanged). */
static int apply_flip(walker *wk, int i, cand_t c)
{
    const orc_fmt *f = wk->f;
    orc_info *in = wk->info;
    int X = c.X, j = c.j, s = c.s;
    /* (Y, Z) = the two other factors in cyclic order after X; rho swaps them */
    int Y = (X + 1) % 3, Z = (X + 2) % 3;
    if (c.rho) { int tmpf = Y; Y = Z; Z = tmpf; }
    int8_t ny[128], nz[128];
    int ok = vec_add(ny, factor(f, wk->slots, i, Y), factor(f, wk->slots, j, Y), +1, f->len[Y], f->mode);
    ok &= vec_add(nz, factor(f, wk->slots, j, Z), factor(f, wk->slots, i, Z), -s, f->len[Z], f->mode);
    if (!ok) {
        in->rejected += 1;
        return ORC_REJECT;
    }
    in->accepted += 1;
    memcpy(factor(f, wk->slots, i, Y), ny, (size_t)f->len[Y]);
    memcpy(factor(f, wk->slots, j, Z), nz, (size_t)f->len[Z]);
    queue_t q; q.len = 0;
    q_push(&q, i);
    q_push(&q, j);
    int zi = vec_is_zero(ny, f->len[Y]);
    int zj = vec_is_zero(nz, f->len[Z]);
    /* zero terms are removed, the higher slot first */
    int hi = i > j ? i : j, lo = i > j ? j : i;
    int zhi = (hi == i) ? zi : zj, zlo = (lo == i) ? zi : zj;
    if (zhi) { drop_slot(wk, hi, &q); in->drops += 1; }
    if (zlo) { drop_slot(wk, lo, &q); in->drops += 1; }
    for (int a = 0; a < q.len; ++a) canonicalize_term(f, wk->slots, q.item[a]);
    if (wk->prm->policy != 2) reduction_cascade(wk, &q);   /* policy 2: no reduction edges */
    return ORC_ACCEPT;
}

/* Test hook: apply one flip candidate (X, j, s, rho) on term i of a scheme of
 * rank r held in a buffer of capacity >= r terms; returns the action, and the
 * new rank through *r_out. */
int orc_apply_flip(int m, int n, int p, int mode, int r, int8_t *scheme, int i,
                   int X, int j, int s, int rho, int *r_out)
{
    orc_fmt f = make_fmt(m, n, p, mode);
    orc_info info; memset(&info, 0, sizeof info); info.r = r;
    orc_params prm; memset(&prm, 0, sizeof prm);   /* policy 0: the flip with its reduction cascade */
    walker wk; memset(&wk, 0, sizeof wk);
    wk.f = &f; wk.prm = &prm; wk.slots = scheme; wk.info = &info;
    cand_t c; c.X = X; c.j = j; c.s = s; c.rho = rho;
    int action = apply_flip(&wk, i, c);
    *r_out = info.r;
    return action;
}

/* Rest of a step after the flip: rank-reduction count, digest record, best
 * scheme (strictly better always, equal rank when x2 < 0.01 * 2^32), plateau,
 * and the expansion:
 *   policy 0: a plus transition when the plateau is long and the rank is close
 *             to the best (Algorithm 1's expand guard r <= best + 2);
 *   policy 1: Algorithm 1 -- a failed try_flip (no candidate, or rejected)
 *             expands and ends the iteration; after a flip, expand when
 *             x3 < p_expand * 2^32 and r <= best + 2.
 * Every expansion needs a free slot (r < r_max). */
static void finish_step(walker *wk, const uint32_t *x, int r_before, int action, int X, int rho, int s, int i,
                        int j)
{
    orc_info *in = wk->info;
    uint64_t t = (uint64_t)in->t;
    if (in->r < r_before) in->reductions += 1;

    uint64_t rec = (uint64_t)action | ((uint64_t)X << 4) | ((uint64_t)rho << 6) |
                   ((uint64_t)(s < 0) << 7) | ((uint64_t)(uint32_t)i << 8) |
                   ((uint64_t)(uint32_t)j << 24) | ((uint64_t)(uint32_t)in->r << 40);
    in->digest = digest_mix(in->digest, rec);

    if (wk->prm->policy == 2) {
        /* best = least (rank, non-zero coefficients); equal pairs refresh with x2 */
        int nz = 0;
        for (int e = 0; e < in->r * wk->f->LT; ++e) nz += wk->slots[e] != 0;
        if (in->r < in->best_r || (in->r == in->best_r && nz < in->best_nnz)) {
            take_best(wk);
            in->best_r = in->r;
            in->best_nnz = nz;
            in->best_t = (int64_t)t;
            in->plateau = 0;
        } else {
            if (in->r == in->best_r && nz == in->best_nnz && x[2] < wk->prm->refresh_thresh) take_best(wk);
            in->plateau += 1;
        }
        in->t += 1;
        if (wk->prm->debug_checks) debug_check(wk);
        return;
    }

    if (wk->prm->policy == 1 && action != ORC_ACCEPT) {
        in->plateau += 1;
        if (in->r < in->r_max) expand_step(wk, t);
        in->t += 1;
        if (wk->prm->debug_checks) debug_check(wk);
        return;
    }

    if (in->r < in->best_r) {
        take_best(wk);
        in->best_r = in->r;
        in->best_t = (int64_t)t;
        in->plateau = 0;
    } else {
        if (in->r == in->best_r && x[2] < wk->prm->refresh_thresh) take_best(wk);
        in->plateau += 1;
    }

    if (wk->prm->policy == 1) {
        if (x[3] < wk->prm->expand_thresh && in->r <= in->best_r + 2 && in->r < in->r_max) expand_step(wk, t);
    } else if (wk->prm->plus_enabled && in->plateau >= wk->prm->plateau_len &&
               in->r <= in->best_r + 2 && in->r < in->r_max) {
        expand_step(wk, t);
    }
    in->t += 1;
    if (wk->prm->debug_checks) debug_check(wk);
}

/* One step of the walk (Algorithm 1, with the plateau or the p_expand expansion policy). */
/* Algorithmic word operations of one uniform step, the count the roofline of
 * the walk is taken against: the Philox draw (10 rounds of 10 operations);
 * the try_flip comparison of term i with the r - 1 other live slots (Z_T 8
 * word tests per slot: u and v exact, two words each, w exact or negated,
 * four; Z_2 3); when a candidate was drawn, the two new factors (Z_T 18:
 * validity 3 + result 6 each; Z_2 2 XOR); after an accepted flip, the
 * reduction check of both modified terms against the other slots.  Word
 * counts are per machine word of a sign: one word for terms of at most 64
 * coefficients, three (factor-aligned) when every factor fits 64, else six.
 * r is the rank when the step began. */
static int64_t walk_step_ops(const orc_fmt *F, int r, int action)
{
    const int64_t words = F->LT <= 64 ? 1 : ((F->len[0] <= 64 && F->len[1] <= 64 && F->len[2] <= 64) ? 3 : 6);
    const int64_t search = (F->mode == ORC_MODE_ZT ? 8 : 3) * (int64_t)(r - 1);
    int64_t ops = 100 + search;
    if (action != ORC_NOCAND) ops += F->mode == ORC_MODE_ZT ? 18 : 2;
    if (action == ORC_ACCEPT) ops += 2 * search;
    return words * ops;
}

static void walk_step(walker *wk, cand_t *cbuf)
{
    orc_info *in = wk->info;
    uint64_t t = (uint64_t)in->t;
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), wk->walker_id, 0u}, x[4];
    orc_philox4x32_10(ctr, wk->key, x);

    int r_before = in->r;
    int i = (int)mulhi_range(x[0], (uint32_t)in->r);
    int K = enumerate_candidates(wk, i, cbuf);
    int action = ORC_NOCAND, X = 0, j = 0, s = 1, rho = 0;
    if (K > 0) {
        cand_t c = cbuf[mulhi_range(x[1], (uint32_t)K)];
        X = c.X; j = c.j; s = c.s; rho = c.rho;
        action = apply_flip(wk, i, c);
    } else {
        in->nocand += 1;
    }
    in->ops += walk_step_ops(wk->f, r_before, action);
    finish_step(wk, x, r_before, action, X, rho, s, i, j);
}

/* ------------------------------------------------------------------------ */
/* Window mode (the step the learned proposal acts on): the candidates of     */
/* terms i0, i0+1, ... (mod r), each term's in walk order, first W of them.   */
/* ------------------------------------------------------------------------ */
#define ORC_FEATURES 32

typedef struct { int i, X, j, s, rho, ki, q; } wcand_t;

static int build_window(const walker *wk, int i0, int W, wcand_t *out, cand_t *tmp)
{
    int r = wk->info->r, K = 0;
    for (int q = 0; q < r && K < W; ++q) {
        int i = (i0 + q) % r;
        int ki = enumerate_candidates(wk, i, tmp);
        for (int a = 0; a < ki && K < W; ++a) {
            wcand_t c = {i, tmp[a].X, tmp[a].j, tmp[a].s, tmp[a].rho, ki, q};
            out[K++] = c;
        }
    }
    return K;
}

static int nnz(const int8_t *a, int L)
{
    int c = 0;
    for (int e = 0; e < L; ++e) c += a[e] != 0;
    return c;
}

/* Features of one window candidate: one-hot factor X, rho, sign, non-zero
 * counts of X_i, Y_i, Y_j, of the sum Y_i + Y_j (0 when it leaves Z_T) and
 * its validity, the same for Z_i, Z_j and Z_j - s Z_i, positions where both
 * Y (resp. Z) factors are non-zero, whether each sum vanishes, the term's
 * candidate count and window position (both capped at 64), r - best_r, r, m,
 * n, p, and a constant 1. */
static void window_features(const walker *wk, const wcand_t *c, float *f)
{
    const orc_fmt *F = wk->f;
    int Y = (c->X + 1) % 3, Z = (c->X + 2) % 3;
    if (c->rho) { int t = Y; Y = Z; Z = t; }
    int8_t sy[128], sz[128];
    int vy = vec_add(sy, factor(F, wk->slots, c->i, Y), factor(F, wk->slots, c->j, Y), +1, F->len[Y], F->mode);
    int vz = vec_add(sz, factor(F, wk->slots, c->j, Z), factor(F, wk->slots, c->i, Z), -c->s, F->len[Z], F->mode);
    int oy = 0, oz = 0;
    for (int e = 0; e < F->len[Y]; ++e)
        oy += factor(F, wk->slots, c->i, Y)[e] != 0 && factor(F, wk->slots, c->j, Y)[e] != 0;
    for (int e = 0; e < F->len[Z]; ++e)
        oz += factor(F, wk->slots, c->i, Z)[e] != 0 && factor(F, wk->slots, c->j, Z)[e] != 0;
    for (int k = 0; k < ORC_FEATURES; ++k) f[k] = 0.f;
    f[c->X] = 1.f;
    f[3] = (float)c->rho;
    f[4] = (float)(c->s < 0);
    f[5] = (float)nnz(factor(F, wk->slots, c->i, c->X), F->len[c->X]);
    f[6] = (float)nnz(factor(F, wk->slots, c->i, Y), F->len[Y]);
    f[7] = (float)nnz(factor(F, wk->slots, c->j, Y), F->len[Y]);
    f[8] = vy ? (float)nnz(sy, F->len[Y]) : 0.f;
    f[9] = (float)vy;
    f[10] = (float)nnz(factor(F, wk->slots, c->i, Z), F->len[Z]);
    f[11] = (float)nnz(factor(F, wk->slots, c->j, Z), F->len[Z]);
    f[12] = vz ? (float)nnz(sz, F->len[Z]) : 0.f;
    f[13] = (float)vz;
    f[14] = (float)oy;
    f[15] = (float)oz;
    f[16] = (float)(vy && nnz(sy, F->len[Y]) == 0);
    f[17] = (float)(vz && nnz(sz, F->len[Z]) == 0);
    f[18] = (float)(c->ki < 64 ? c->ki : 64);
    f[19] = (float)(wk->info->r - wk->info->best_r);
    f[20] = (float)wk->info->r;
    f[21] = (float)F->m;
    f[22] = (float)F->n;
    f[23] = (float)F->p;
    f[24] = (float)(c->q < 64 ? c->q : 64);
    f[31] = 1.f;
}

/* Training log of one window-mode step (the record the learned proposal is
 * trained on): the chosen candidate's features, computed on the state before
 * the flip, with label 1 when the step lowered the rank (the reductions
 * counter advanced: a zero-term removal or a merge after the flip), else
 * label 0; label-0 records are kept only when the first word of Philox
 * sub-stream 256 of the step, (t_lo, t_hi, walker, 256), lies below
 * neg_thresh.  *label_out = -1 when the step keeps no record (no candidate,
 * or an unsampled label-0 step).  The features are stored for every step
 * with a candidate, recorded or not (the horizon log draws on them). */
typedef struct {
    int8_t *label;     /* [steps] per walker: -1, 0 or 1 */
    uint8_t *feat;     /* [steps][32] per walker */
    uint32_t neg_thresh;
} wlog_t;

/* One window-mode step.  policy 0: candidate mulhi(x1, K); otherwise the
 * candidate index is taken from *choice (a logged decision being replayed,
 * -1 when there was no candidate).  lg (may be NULL) receives the step's
 * training-log record at position `slot`. */
static void walk_step_window(walker *wk, wcand_t *wbuf, cand_t *tmp, int W, int policy, const int32_t *choice,
                             const wlog_t *lg, int64_t slot)
{
    orc_info *in = wk->info;
    uint64_t t = (uint64_t)in->t;
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), wk->walker_id, 0u}, x[4];
    orc_philox4x32_10(ctr, wk->key, x);
    int r_before = in->r;
    int64_t red_before = in->reductions;
    int i0 = (int)mulhi_range(x[0], (uint32_t)in->r);
    int K = build_window(wk, i0, W, wbuf, tmp);
    int action = ORC_NOCAND, X = 0, j = 0, s = 1, rho = 0, i = i0;
    float f[ORC_FEATURES];
    if (K > 0) {
        int c = (policy == 0) ? (int)mulhi_range(x[1], (uint32_t)K) : *choice;
        if (c < 0 || c >= K) { in->debug_failures += 1; c = 0; }
        wcand_t w = wbuf[c];
        cand_t cc = {w.X, w.j, w.s, w.rho};
        i = w.i; X = w.X; j = w.j; s = w.s; rho = w.rho;
        if (lg) window_features(wk, &w, f);
        action = apply_flip(wk, i, cc);
    } else {
        if (policy != 0 && *choice != -1) in->debug_failures += 1;
        in->nocand += 1;
    }
    finish_step(wk, x, r_before, action, X, rho, s, i, j);
    if (lg) {
        int label = -1;
        if (K > 0) {
            if (in->reductions > red_before) {
                label = 1;
            } else if (lg->neg_thresh) {
                uint32_t c2[4] = {(uint32_t)t, (uint32_t)(t >> 32), wk->walker_id, 256u}, y[4];
                orc_philox4x32_10(c2, wk->key, y);
                if (y[0] < lg->neg_thresh) label = 0;
            }
        }
        lg->label[slot] = (int8_t)label;
        for (int k = 0; k < ORC_FEATURES; ++k)
            lg->feat[(size_t)slot * ORC_FEATURES + k] = K > 0 ? (uint8_t)f[k] : 0;
    }
}

/* Window and features of a given state (rank r, best rank best_r) for i0:
 * returns K; out_feat [K][32], out_cand [K][5] = (i, X, j, s, rho). */
int orc_window_features(int m, int n, int p, int r, int best_r, const int8_t *scheme, int i0, int W,
                        float *out_feat, int32_t *out_cand)
{
    orc_fmt f = make_fmt(m, n, p, ORC_MODE_ZT);
    orc_info info; memset(&info, 0, sizeof info);
    info.r = r; info.best_r = best_r;
    walker wk; memset(&wk, 0, sizeof wk);
    wk.f = &f; wk.slots = (int8_t *)scheme; wk.info = &info;
    wcand_t *wb = (wcand_t *)malloc(sizeof(wcand_t) * (size_t)(W > 0 ? W : 1));
    cand_t *tmp = (cand_t *)malloc(sizeof(cand_t) * (size_t)(6 * r + 6));
    int K = build_window(&wk, i0, W, wb, tmp);
    for (int k = 0; k < K; ++k) {
        window_features(&wk, &wb[k], out_feat + (size_t)k * ORC_FEATURES);
        out_cand[5 * k + 0] = wb[k].i; out_cand[5 * k + 1] = wb[k].X; out_cand[5 * k + 2] = wb[k].j;
        out_cand[5 * k + 3] = wb[k].s; out_cand[5 * k + 4] = wb[k].rho;
    }
    free(wb); free(tmp);
    return K;
}

/* ------------------------------------------------------------------------ */
/* Start preparation: canonicalise every term, remove terms with a zero        */
/* factor, then run the reduction cascade over all terms in slot order.        */
/* Returns the new rank (scheme rewritten in place).                           */
/* ------------------------------------------------------------------------ */
int orc_prepare_start(int m, int n, int p, int mode, int r, int8_t *scheme)
{
    orc_fmt f = make_fmt(m, n, p, mode);
    orc_info info; memset(&info, 0, sizeof info);
    info.r = r;
    walker wk; memset(&wk, 0, sizeof wk);
    wk.f = &f; wk.slots = scheme; wk.info = &info;
    queue_t dummy; dummy.len = 0;
    for (int t = r - 1; t >= 0; --t) {
        int zero = 0;
        for (int X = 0; X < 3; ++X) zero |= vec_is_zero(factor(&f, scheme, t, X), f.len[X]);
        if (zero) drop_slot(&wk, t, &dummy);
    }
    for (int t = 0; t < info.r; ++t) canonicalize_term(&f, scheme, t);
    /* full reduction passes: every slot in order enters the cascade, repeated
     * until a whole pass merges nothing */
    int64_t before;
    do {
        before = info.merges;
        for (int t = 0; t < info.r; ++t) {
            queue_t q; q.len = 0;
            q_push(&q, t);
            reduction_cascade(&wk, &q);
        }
    } while (info.merges != before);
    return info.r;
}

/* Initialise walker records from a prepared start scheme of rank r0. */
void orc_init_walkers(int m, int n, int p, int mode, int r0, const int8_t *start, int r_max,
                      int n_walkers, const uint32_t *walker_ids,
                      int8_t *slots, int8_t *best, orc_info *info)
{
    orc_fmt f = make_fmt(m, n, p, mode);
    size_t per = (size_t)r_max * f.LT;
    for (int w = 0; w < n_walkers; ++w) {
        memset(slots + per * w, 0, per);
        memset(best + per * w, 0, per);
        memcpy(slots + per * w, start, (size_t)r0 * f.LT);
        memcpy(best + per * w, start, (size_t)r0 * f.LT);
        orc_info *in = info + w;
        memset(in, 0, sizeof *in);
        in->r = r0; in->best_r = r0; in->r_max = r_max;
        int nz = 0;
        for (int e = 0; e < r0 * f.LT; ++e) nz += start[e] != 0;
        in->best_nnz = nz;
        in->digest = orc_digest_init(walker_ids[w]);
    }
}

typedef struct {
    const orc_fmt *f;
    const orc_params *prm;
    int r_max;
    uint64_t seed;
    int64_t steps;
    int window;              /* 0: walk_step; > 0: window mode with this capacity */
    int policy;              /* window mode: 0 uniform, 1 replay choices */
    const int32_t *choices;  /* replay: [n_walkers][steps] */
    int8_t *log_label;       /* window mode, optional: [n_walkers][steps] training-log labels */
    uint8_t *log_feat;       /* [n_walkers][steps][32] */
    uint32_t neg_thresh;
    int n_walkers;
    const uint32_t *walker_ids;
    int8_t *slots, *best;
    orc_info *info;
    int next;               /* shared work counter */
    pthread_mutex_t lock;
} job_t;

static void run_walker(job_t *job, int w)
{
    const orc_fmt *f = job->f;
    size_t per = (size_t)job->r_max * f->LT;
    walker wk;
    wk.f = f; wk.prm = job->prm;
    wk.slots = job->slots + per * w;
    wk.best = job->best + per * w;
    wk.info = job->info + w;
    wk.walker_id = job->walker_ids[w];
    wk.key[0] = (uint32_t)job->seed;
    wk.key[1] = (uint32_t)(job->seed >> 32);
    cand_t *cbuf = (cand_t *)malloc(sizeof(cand_t) * (size_t)(6 * job->r_max + 6));
    if (job->window > 0) {
        wcand_t *wbuf = (wcand_t *)malloc(sizeof(wcand_t) * (size_t)job->window);
        wlog_t lg;
        if (job->log_label) {
            lg.label = job->log_label + (size_t)w * job->steps;
            lg.feat = job->log_feat + (size_t)w * job->steps * ORC_FEATURES;
            lg.neg_thresh = job->neg_thresh;
        }
        for (int64_t s = 0; s < job->steps; ++s)
            walk_step_window(&wk, wbuf, cbuf, job->window, job->policy,
                             job->choices ? job->choices + (size_t)w * job->steps + s : NULL,
                             job->log_label ? &lg : NULL, s);
        free(wbuf);
    } else {
        for (int64_t s = 0; s < job->steps; ++s) walk_step(&wk, cbuf);
    }
    free(cbuf);
}

static void *worker_main(void *arg)
{
    job_t *job = (job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int w = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (w >= job->n_walkers) break;
        run_walker(job, w);
    }
    return NULL;
}

/* Advance n_walkers walkers by `steps` steps each, one walker per thread at a
 * time over n_threads threads.  State arrays are updated in place. */
void orc_walk(int m, int n, int p, int mode, const orc_params *prm, int r_max, uint64_t seed,
              int n_walkers, const uint32_t *walker_ids, int64_t steps, int n_threads,
              int8_t *slots, int8_t *best, orc_info *info)
{
    orc_fmt f = make_fmt(m, n, p, mode);
    job_t job;
    job.f = &f; job.prm = prm; job.r_max = r_max; job.seed = seed; job.steps = steps;
    job.n_walkers = n_walkers; job.walker_ids = walker_ids;
    job.slots = slots; job.best = best; job.info = info; job.next = 0;
    job.window = 0; job.policy = 0; job.choices = NULL;
    job.log_label = NULL; job.log_feat = NULL; job.neg_thresh = 0;
    pthread_mutex_init(&job.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_walkers) n_threads = n_walkers > 0 ? n_walkers : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int a = 0; a < n_threads; ++a) pthread_create(&th[a], NULL, worker_main, &job);
    for (int a = 0; a < n_threads; ++a) pthread_join(th[a], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
}

/* Window mode: policy 0 picks uniformly over the window; policy 1 replays
 * choices [n_walkers][steps] (window index per step, -1 for no candidate).
 * log_label / log_feat (both NULL, or [n_walkers][steps] and
 * [n_walkers][steps][32]) receive each step's training-log record (see
 * wlog_t) with label-0 records sampled below neg_thresh. */
void orc_walk_window(int m, int n, int p, const orc_params *prm, int r_max, uint64_t seed, int n_walkers,
                     const uint32_t *walker_ids, int64_t steps, int n_threads, int window, int policy,
                     const int32_t *choices, int8_t *slots, int8_t *best, orc_info *info,
                     int8_t *log_label, uint8_t *log_feat, uint32_t neg_thresh)
{
    orc_fmt f = make_fmt(m, n, p, ORC_MODE_ZT);
    job_t job;
    job.f = &f; job.prm = prm; job.r_max = r_max; job.seed = seed; job.steps = steps;
    job.n_walkers = n_walkers; job.walker_ids = walker_ids;
    job.slots = slots; job.best = best; job.info = info; job.next = 0;
    job.window = window; job.policy = policy; job.choices = choices;
    job.log_label = log_feat ? log_label : NULL; job.log_feat = log_feat; job.neg_thresh = neg_thresh;
    pthread_mutex_init(&job.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_walkers) n_threads = n_walkers > 0 ? n_walkers : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int a = 0; a < n_threads; ++a) pthread_create(&th[a], NULL, worker_main, &job);
    for (int a = 0; a < n_threads; ++a) pthread_join(th[a], NULL);
    free(th);
    pthread_mutex_destroy(&job.lock);
}

int orc_info_size(void) { return (int)sizeof(orc_info); }
int orc_params_size(void) { return (int)sizeof(orc_params); }

/* ------------------------------------------------------------------------ */
/* Sign lifting by brute force (the check for the library's exact search):  */
/* every assignment of signs to the non-zero coefficients of a Z_2 scheme,  */
/* with the first non-zero of u and of v of each term fixed to +1 (flipping */
/* two factors of a term changes nothing), each checked with Eq. (1) over   */
/* the integers.  Returns 1 and the first valid signed scheme (binary       */
/* counter over the free coefficients in row order) in out, 0 when none,    */
/* -1 when there are more than max_bits free coefficients.                  */
/* ------------------------------------------------------------------------ */
int orc_lift_bruteforce(int m, int n, int p, int r, const int8_t *z2, int max_bits, int8_t *out)
{
    orc_fmt f = make_fmt(m, n, p, ORC_MODE_ZT);
    const int LT = f.LT;
    int nfree = 0;
    int *pos = (int *)malloc(sizeof(int) * (size_t)r * (size_t)LT);
    for (int t = 0; t < r; ++t) {
        int first_u = -1, first_v = -1;
        for (int e = 0; e < f.len[0]; ++e) if (z2[t * LT + e]) { first_u = e; break; }
        for (int e = 0; e < f.len[1]; ++e) if (z2[t * LT + f.len[0] + e]) { first_v = f.len[0] + e; break; }
        for (int e = 0; e < LT; ++e)
            if (z2[t * LT + e] && e != first_u && e != first_v) pos[nfree++] = t * LT + e;
    }
    if (nfree > max_bits) { free(pos); return -1; }
    int found = 0;
    for (uint64_t mask = 0; mask < (1ull << nfree) && !found; ++mask) {
        for (int e = 0; e < r * LT; ++e) out[e] = z2[e] ? 1 : 0;
        for (int b = 0; b < nfree; ++b)
            if ((mask >> b) & 1ull) out[pos[b]] = -1;
        if (orc_brent_valid(m, n, p, ORC_MODE_ZT, r, out)) found = 1;
    }
    free(pos);
    return found;
}

/* Sign lifting by plain backtracking (no linear algebra): the free signs in
 * row order, each tensor entry checked with Eq. (1) over the integers as soon
 * as its last non-zero coefficient has a sign.  Exhaustive unless the node
 * budget runs out.  Returns 1 (out = the first valid signed scheme in that
 * order), 0 (none exists), -1 (budget exhausted). */
int orc_lift_backtrack(int m, int n, int p, int r, const int8_t *z2, int64_t max_nodes, int8_t *out)
{
    orc_fmt f = make_fmt(m, n, p, ORC_MODE_ZT);
    const int LT = f.LT, LU = f.len[0], LV = f.len[1], LW = f.len[2];
    const int NC = r * LT;
    int *order = (int *)malloc(sizeof(int) * (size_t)NC);   /* coefficient index -> position, -1 fixed or zero */
    int nfree = 0;
    for (int e = 0; e < NC; ++e) order[e] = -1;
    int *free_at = (int *)malloc(sizeof(int) * (size_t)NC);
    for (int t = 0; t < r; ++t) {
        int first_u = -1, first_v = -1;
        for (int e = 0; e < LU; ++e) if (z2[t * LT + e]) { first_u = e; break; }
        for (int e = 0; e < LV; ++e) if (z2[t * LT + LU + e]) { first_v = LU + e; break; }
        for (int e = 0; e < LT; ++e)
            if (z2[t * LT + e] && e != first_u && e != first_v) { order[t * LT + e] = nfree; free_at[nfree++] = t * LT + e; }
    }
    /* entries with at least one covering term, grouped by the position of their last free coefficient */
    int nent = LU * LV * LW;
    int *ent_last = (int *)malloc(sizeof(int) * (size_t)nent);
    for (int q = 0; q < nent; ++q) {
        int a = q / (LV * LW), b = (q / LW) % LV, c = q % LW, last = -1, any = 0;
        for (int t = 0; t < r; ++t) {
            int ia = t * LT + a, ib = t * LT + LU + b, ic = t * LT + LU + LV + c;
            if (!(z2[ia] && z2[ib] && z2[ic])) continue;
            any = 1;
            if (order[ia] > last) last = order[ia];
            if (order[ib] > last) last = order[ib];
            if (order[ic] > last) last = order[ic];
        }
        ent_last[q] = any ? last : -2;
    }
    for (int e = 0; e < NC; ++e) out[e] = z2[e] ? 1 : 0;
    /* check of one entry with the current signs */
    #define ENTRY_OK(q) ({ int a_ = (q) / (LV * LW), b_ = ((q) / LW) % LV, c_ = (q) % LW; \
        int i_ = a_ / n, k_ = a_ % n, k2_ = b_ / p, j_ = b_ % p, j2_ = c_ / m, i2_ = c_ % m; \
        int want_ = (k_ == k2_ && j_ == j2_ && i_ == i2_) ? 1 : 0, sum_ = 0; \
        for (int t_ = 0; t_ < r; ++t_) sum_ += out[t_ * LT + a_] * out[t_ * LT + LU + b_] * out[t_ * LT + LU + LV + c_]; \
        sum_ == want_; })
    int result = 1;
    /* entries without free coefficients */
    for (int q = 0; q < nent; ++q)
        if (ent_last[q] == -1 && !ENTRY_OK(q)) { result = 0; break; }
    /* entries grouped by the position of their last free sign */
    int *ent_start = (int *)calloc((size_t)nfree + 2, sizeof(int));
    int *ent_list = (int *)malloc(sizeof(int) * (size_t)(nent > 0 ? nent : 1));
    for (int q = 0; q < nent; ++q) if (ent_last[q] >= 0) ent_start[ent_last[q] + 1] += 1;
    for (int d = 0; d < nfree; ++d) ent_start[d + 1] += ent_start[d];
    {
        int *fill = (int *)calloc((size_t)nfree + 1, sizeof(int));
        for (int q = 0; q < nent; ++q)
            if (ent_last[q] >= 0) ent_list[ent_start[ent_last[q]] + fill[ent_last[q]]++] = q;
        free(fill);
    }
    if (result == 1 && nfree > 0) {
        int *val = (int *)malloc(sizeof(int) * (size_t)nfree);
        for (int d = 0; d < nfree; ++d) val[d] = -1;
        int d = 0;
        int64_t nodes = 0;
        result = 0;
        while (d >= 0) {
            if (d == nfree) { result = 1; break; }
            if (val[d] >= 1) { val[d] = -1; out[free_at[d]] = 1; --d; continue; }
            val[d] += 1;
            out[free_at[d]] = val[d] ? -1 : 1;
            if (++nodes > max_nodes) { result = -1; break; }
            int ok = 1;
            for (int k = ent_start[d]; k < ent_start[d + 1] && ok; ++k)
                if (!ENTRY_OK(ent_list[k])) ok = 0;
            if (ok) ++d;
        }
        free(val);
    }
    #undef ENTRY_OK
    free(order); free(free_at); free(ent_last); free(ent_start); free(ent_list);
    return result;
}
