// Window-mode walk step (learned flip proposal, Z_T): instead of the
// candidates of one sampled term, each step considers a window of up to
// kWin candidates: starting at term i0 = mulhi(x0, r), terms i0, i0+1, ...
// (mod r) append their try_flip candidates in (factor, slot, rho) order until
// the window is full.  Per step:
//   1. window_kernel  (one warp per walker): window, candidate descriptors and
//      32 integer features per candidate (bf16 rows for the network);
//   2. the scoring MLP on the tensor cores (mlp_tc.cu) over all rows;
//   3. window_apply_kernel (one thread per walker): policy choice (uniform
//      over the window via x1, or epsilon-greedy argmax of the scores with
//      epsilon decided by x3), then the flip, reductions and bookkeeping of
//      the uniform walker; optional logging of the chosen features with the
//      label "the step lowered the rank" for training.
#include <cstdint>
#include <cuda_bf16.h>

#include "walk_solo.cuh"

namespace tfg {
namespace dev {

constexpr int kWin = 256;         // window capacity: up to 256 candidate pairs per step (two tensor-core tiles of rows)
constexpr int kFeat = 32;
constexpr int kWinMaxSlots = 128; // slots per walker supported by the window kernel

// candidate descriptor: i (10 bits) | X (2) | j (10) | sign (1) | rho (1)
__device__ __forceinline__ uint32_t pack_cand(int i, int X, int j, int sneg, int rho) {
    return (uint32_t)i | ((uint32_t)X << 10) | ((uint32_t)j << 12) | ((uint32_t)sneg << 22) | ((uint32_t)rho << 23);
}

template <class Wd>
__device__ __forceinline__ int popc_w(Wd v) {
    if constexpr (sizeof(Wd) == 4) return __popc(v);
    else return __popcll(v);
}

// Features of candidate (X, j, sign, rho) of term a = slot i (b = slot j).
template <class Wd>
__device__ __forceinline__ void cand_features(const PTerm<Wd, 1, true> &a, const PTerm<Wd, 1, true> &b,
                                              const Masks<Wd, 1> &mk, int X, int sneg, int rho, int k_i, int q,
                                              int r, int best_r, int m, int n, int p, float (&f)[kFeat]) {
    int Y = X == 0 ? 1 : (X == 1 ? 2 : 0);
    int Z = X == 0 ? 2 : (X == 1 ? 0 : 1);
    if (rho) { const int tmp = Y; Y = Z; Z = tmp; }
    const Wd MX = mk.of(X, 0), MY = mk.of(Y, 0), MZ = mk.of(Z, 0);
    const Wd ad = a.p[0] | a.n[0], bd = b.p[0] | b.n[0];
    // Y_i + Y_j
    const bool vy = (((a.p[0] & b.p[0]) | (a.n[0] & b.n[0])) & MY) == Wd(0);
    const Wd syd = (((a.p[0] | b.p[0]) & ~(a.n[0] | b.n[0])) | ((a.n[0] | b.n[0]) & ~(a.p[0] | b.p[0]))) & MY;
    // Z_j - s Z_i  (s = +1: add (a.n, a.p); s = -1: add (a.p, a.n))
    const Wd zp = sneg ? a.p[0] : a.n[0], zn = sneg ? a.n[0] : a.p[0];
    const bool vz = (((b.p[0] & zp) | (b.n[0] & zn)) & MZ) == Wd(0);
    const Wd szd = (((b.p[0] | zp) & ~(b.n[0] | zn)) | ((b.n[0] | zn) & ~(b.p[0] | zp))) & MZ;
#pragma unroll
    for (int k = 0; k < kFeat; ++k) f[k] = (k == X) ? 1.f : 0.f;   // one-hot X in f[0..2]
    f[3] = (float)rho;
    f[4] = (float)sneg;
    f[5] = (float)popc_w<Wd>(ad & MX);
    f[6] = (float)popc_w<Wd>(ad & MY);
    f[7] = (float)popc_w<Wd>(bd & MY);
    f[8] = vy ? (float)popc_w<Wd>(syd) : 0.f;
    f[9] = vy ? 1.f : 0.f;
    f[10] = (float)popc_w<Wd>(ad & MZ);
    f[11] = (float)popc_w<Wd>(bd & MZ);
    f[12] = vz ? (float)popc_w<Wd>(szd) : 0.f;
    f[13] = vz ? 1.f : 0.f;
    f[14] = (float)popc_w<Wd>(ad & bd & MY);
    f[15] = (float)popc_w<Wd>(ad & bd & MZ);
    f[16] = (vy && syd == Wd(0)) ? 1.f : 0.f;
    f[17] = (vz && szd == Wd(0)) ? 1.f : 0.f;
    f[18] = (float)(k_i < 64 ? k_i : 64);
    f[19] = (float)(r - best_r);
    f[20] = (float)r;
    f[21] = (float)m;
    f[22] = (float)n;
    f[23] = (float)p;
    f[24] = (float)(q < 64 ? q : 64);
    f[31] = 1.f;
}

// One warp per walker.  Phase 1: eight terms i0 + g (g = lane / 4, then the
// next eight while the window has room); the four lanes of a group scan
// consecutive quarters of the slots for the term's try_flip candidates, and
// every candidate's descriptor goes to its window position in shared memory
// (order: term, then factor, then slot, then rho).  Phase 2: the lanes take
// window rows l, l+32, ... and compute and store the feature rows (coalesced
// 64-byte rows).
template <class Wd>
__global__ void __launch_bounds__(128) window_kernel(const SegDesc d, __nv_bfloat16 *__restrict__ feat,
                                                     uint32_t *__restrict__ desc, int *__restrict__ kwin) {
    __shared__ __align__(16) Wd sp[4][kWinMaxSlots], sn[4][kWinMaxSlots];
    __shared__ uint32_t sdesc[4][kWin], sinfo[4][kWin];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * 4 + warp;
    if (w >= d.n_walkers) return;
    using T = PTerm<Wd, 1, true>;
    using O = Ops<Wd, 1, true>;
    Masks<Wd, 1> mk;
    mk.load(d);
    const tfg_walker_info &H = d.hdr[w];
    const int r = H.r, best_r = H.best_r;
    const U4 x = philox10((uint32_t)H.t, (uint32_t)(H.t >> 32), H.walker_id, 0u, d.key0, d.key1);
    const int i0 = (int)__umulhi(x.x, (uint32_t)r);
    const Wd *src = reinterpret_cast<const Wd *>(d.slots) + (size_t)w * d.R * 2;
    for (int k = lane; k < r; k += 32) {
        sp[warp][k] = src[(size_t)k * 2];
        sn[warp][k] = src[(size_t)k * 2 + 1];
    }
    __syncwarp();
    // ---- phase 1: candidate descriptors in window order
    const int g = lane >> 2, sub = lane & 3;
    const int chunk = (r + 3) >> 2;                  // <= 32 slots per lane
    const int jb = sub * chunk, je = min(r, jb + chunk);
    int carry = 0;
    for (int base = 0; base < r && carry < kWin; base += 8) {
        const int q = base + g;
        const bool has = q < r;
        const int i = has ? (i0 + q) % r : 0;
        T ti;
        ti.p[0] = sp[warp][i];
        ti.n[0] = sn[warp][i];
        // bit (j - jb): slot j of this lane's quarter is a candidate of factor u / v / w (w negated)
        uint32_t bu = 0, bv = 0, bw = 0, bn = 0;
        if (has) {
            for (int j = jb; j < je; ++j) {
                if (j == i) continue;
                T c;
                c.p[0] = sp[warp][j];
                c.n[0] = sn[warp][j];
                bool eu, ev, ewp, ewn;
                O::compare(c, ti, mk, eu, ev, ewp, ewn);
                const uint32_t bit = 1u << (j - jb);
                bu |= eu ? bit : 0u;
                bv |= ev ? bit : 0u;
                bw |= (ewp || ewn) ? bit : 0u;
                bn |= ewn ? bit : 0u;
            }
        }
        // per-factor counts: this lane, earlier lanes of the group, the whole term
        const uint32_t own = (uint32_t)__popc(bu) | ((uint32_t)__popc(bv) << 8) | ((uint32_t)__popc(bw) << 16);
        uint32_t gin = own;
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, gin, o, 4);
            if (sub >= o) gin += y;
        }
        const uint32_t gtot = __shfl_sync(0xffffffffu, gin, 3, 4);
        const uint32_t gex = gin - own;
        const int nU = (int)(gtot & 255u), nV = (int)((gtot >> 8) & 255u), nW = (int)(gtot >> 16);
        const int ki = 2 * (nU + nV + nW);
        // window offset of the term: counts of the earlier terms of this round
        int incl = sub == 0 ? ki : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int tpos = carry + incl - ki;
        const uint32_t info = (uint32_t)(ki < 64 ? ki : 64) | ((uint32_t)(q < 64 ? q : 64) << 8);
        // this lane's candidates: factor X, slot order, rho 0 then 1
        for (int X = 0; X < 3; ++X) {
            const int before = X == 0 ? 0 : (X == 1 ? nU : nU + nV);
            const int lex = (int)((gex >> (8 * X)) & 255u);
            int pos = tpos + 2 * (before + lex);
            uint32_t bits = X == 0 ? bu : (X == 1 ? bv : bw);
            while (bits && pos < kWin) {
                const int o = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int j = jb + o;
                const int sneg = (X == 2) ? (int)((bn >> o) & 1u) : 0;
                sdesc[warp][pos] = pack_cand(i, X, j, sneg, 0);
                sinfo[warp][pos] = info;
                if (pos + 1 < kWin) {
                    sdesc[warp][pos + 1] = pack_cand(i, X, j, sneg, 1);
                    sinfo[warp][pos + 1] = info;
                }
                pos += 2;
            }
        }
        carry += total;
    }
    const int K = carry < kWin ? carry : kWin;
    __syncwarp();
    // ---- phase 2: feature rows (rows past the window are zero: scored, never chosen)
    __nv_bfloat16 *fw = feat + (size_t)w * kWin * kFeat;
    uint32_t *dw = desc + (size_t)w * kWin;
    for (int row = lane; row < kWin; row += 32) {
        uint4 *dst = reinterpret_cast<uint4 *>(fw + (size_t)row * kFeat);
        if (row < K) {
            const uint32_t dc = sdesc[warp][row], in = sinfo[warp][row];
            const int i = (int)(dc & 1023u), X = (int)((dc >> 10) & 3u), j = (int)((dc >> 12) & 1023u);
            const int sneg = (int)((dc >> 22) & 1u), rho = (int)((dc >> 23) & 1u);
            T ti, tj;
            ti.p[0] = sp[warp][i];
            ti.n[0] = sn[warp][i];
            tj.p[0] = sp[warp][j];
            tj.n[0] = sn[warp][j];
            float f[kFeat];
            cand_features<Wd>(ti, tj, mk, X, sneg, rho, (int)(in & 255u), (int)(in >> 8), r, best_r, d.m, d.n, d.p, f);
#pragma unroll
            for (int k = 0; k < kFeat / 8; ++k) {
                uint32_t wv[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const __nv_bfloat162 b2 = __floats2bfloat162_rn(f[8 * k + 2 * h], f[8 * k + 2 * h + 1]);
                    wv[h] = *reinterpret_cast<const uint32_t *>(&b2);
                }
                dst[k] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
            dw[row] = dc;
        } else {
#pragma unroll
            for (int k = 0; k < kFeat / 8; ++k) dst[k] = make_uint4(0, 0, 0, 0);
        }
    }
    if (lane == 0) kwin[w] = K;
}

// One window-mode step per thread (walker), on the solo walker's state machine.
template <class Wd, int RMAX, int BT>
__global__ void __launch_bounds__(BT) window_apply_kernel(const SegDesc d, const uint32_t *__restrict__ desc,
                                                          const int *__restrict__ kwin,
                                                          const float *__restrict__ score, int policy,
                                                          uint32_t eps_thresh, const __nv_bfloat16 *__restrict__ feat,
                                                          int32_t *__restrict__ choices, WindowLog log) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t w = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (w >= d.n_walkers) return;
    using SW = SoloWalker<TFG_MODE_ZT, Wd, RMAX, BT>;
    using T = typename SW::T;
    SW wk;
    wk.sm = reinterpret_cast<Wd *>(smem_raw) + (size_t)threadIdx.x * 2;
    wk.load(d, w);
    Wd *bestp = reinterpret_cast<Wd *>(d.best) + (size_t)w * d.R * 2;
    const unsigned wmask = __activemask();
    const int lane = threadIdx.x & 31;
    const int nl = __popc(wmask);
    const int64_t t_step = wk.t;
    const U4 x = philox10((uint32_t)wk.t, (uint32_t)(wk.t >> 32), wk.wid, 0u, wk.key0, wk.key1);
    const int r_before = wk.r;
    const int K = kwin[w];
    int action = kNoCand, X = 0, j = 0, rho = 0, sneg = 0, c = -1;
    int i = (int)__umulhi(x.x, (uint32_t)wk.r);
    bool need_check = false;
    T ti2, tj2;
    ti2.p[0] = tj2.p[0] = 0;
    ti2.n[0] = tj2.n[0] = 0;
    if (K > 0) {
        if (policy == 0 || x.w < eps_thresh) {
            c = (int)__umulhi(x.y, (uint32_t)K);
        } else {
            const float *sc = score + (size_t)w * kWin;
            c = 0;
            float best = sc[0];
            for (int k = 1; k < K; ++k)
                if (sc[k] > best) { best = sc[k]; c = k; }
        }
        const uint32_t dc = desc[(size_t)w * kWin + c];
        i = (int)(dc & 1023u);
        X = (int)((dc >> 10) & 3u);
        j = (int)((dc >> 12) & 1023u);
        sneg = (int)((dc >> 22) & 1u);
        rho = (int)((dc >> 23) & 1u);
        const T ti = wk.ld(i);
        wk.apply_candidate(ti, i, X, j, sneg, rho, action, need_check, ti2, tj2);
    } else {
        wk.c_noc += 1;
    }
    wk.finish_step(d, wmask, lane, nl, bestp, x.z, x.w, r_before, action, X, rho, sneg, i, j, need_check, ti2, tj2);
    if (choices) choices[w] = c;
    if (log.d_entries && c >= 0) {
        const bool positive = wk.c_red > 0;   // the flip's reductions lowered the rank this step
        bool keep = positive;
        if (!positive && log.neg_thresh) {
            const U4 y = philox10((uint32_t)t_step, (uint32_t)(t_step >> 32), wk.wid, 0x100u, wk.key0, wk.key1);
            keep = y.x < log.neg_thresh;
        }
        if (keep) {
            const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(log.d_count), 1ull);
            if (slot < (unsigned long long)log.capacity) {
                WindowLogEntry *e = reinterpret_cast<WindowLogEntry *>(log.d_entries) + slot;
                const uint4 *fsrc = reinterpret_cast<const uint4 *>(feat + ((size_t)w * kWin + c) * kFeat);
#pragma unroll
                for (int k = 0; k < kFeat / 8; ++k) reinterpret_cast<uint4 *>(e->feat)[k] = fsrc[k];
                e->label = positive ? 1.f : 0.f;
                e->walker_id = wk.wid;
                e->step = (uint32_t)t_step;
                e->pad = 0;
            }
        }
    }
    wk.store(d, w);
}

}  // namespace dev

int window_cap() { return dev::kWin; }

void launch_window(const SegDesc &d, void *feat, uint32_t *desc, int *kwin, cudaStream_t st) {
    const int64_t blocks = (d.n_walkers + 3) / 4;
    if (blocks <= 0) return;
    if (d.word_bits == 32)
        dev::window_kernel<uint32_t><<<(unsigned)blocks, 128, 0, st>>>(d, reinterpret_cast<__nv_bfloat16 *>(feat),
                                                                      desc, kwin);
    else
        dev::window_kernel<uint64_t><<<(unsigned)blocks, 128, 0, st>>>(d, reinterpret_cast<__nv_bfloat16 *>(feat),
                                                                      desc, kwin);
}

template <class Wd, int RMAX>
static void apply_variant(const SegDesc &d, const uint32_t *desc, const int *kwin, const float *score, int policy,
                          uint32_t eps, const void *feat, int32_t *choices, const WindowLog &log, cudaStream_t st) {
    constexpr int BT = 128;
    constexpr size_t smem = solo_smem_bytes<TFG_MODE_ZT, Wd, RMAX, BT>();
    static bool attr = [] {
        cudaFuncSetAttribute(dev::window_apply_kernel<Wd, RMAX, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        return true;
    }();
    (void)attr;
    const int64_t blocks = (d.n_walkers + BT - 1) / BT;
    dev::window_apply_kernel<Wd, RMAX, BT><<<(unsigned)blocks, BT, smem, st>>>(
        d, desc, kwin, score, policy, eps, reinterpret_cast<const __nv_bfloat16 *>(feat), choices, log);
}

// Capacity of the apply kernel chosen for a population (0: not supported).
int window_apply_capacity(int word_bits, int R) {
    if (word_bits == 32) {
        for (int c : {12, 16, 32}) if (R <= c) return c;
    } else {
        for (int c : {48, 64, 72, 88}) if (R <= c) return c;
    }
    return 0;
}

int launch_window_apply(const SegDesc &d, const uint32_t *desc, const int *kwin, const float *score, int policy,
                        uint32_t eps, const void *feat, int32_t *choices, const WindowLog &log, cudaStream_t st) {
    if (d.n_walkers <= 0) return 0;
    const int cap = window_apply_capacity(d.word_bits, d.R);
    if (d.word_bits == 32) {
        if (cap == 12) apply_variant<uint32_t, 12>(d, desc, kwin, score, policy, eps, feat, choices, log, st);
        else if (cap == 16) apply_variant<uint32_t, 16>(d, desc, kwin, score, policy, eps, feat, choices, log, st);
        else if (cap == 32) apply_variant<uint32_t, 32>(d, desc, kwin, score, policy, eps, feat, choices, log, st);
        else return -1;
    } else {
        if (cap == 48) apply_variant<uint64_t, 48>(d, desc, kwin, score, policy, eps, feat, choices, log, st);
        else if (cap == 64) apply_variant<uint64_t, 64>(d, desc, kwin, score, policy, eps, feat, choices, log, st);
        else if (cap == 72) apply_variant<uint64_t, 72>(d, desc, kwin, score, policy, eps, feat, choices, log, st);
        else if (cap == 88) apply_variant<uint64_t, 88>(d, desc, kwin, score, policy, eps, feat, choices, log, st);
        else return -1;
    }
    return 0;
}

}  // namespace tfg
