// Window-mode walk step (learned flip proposal, Z_T): instead of the
// candidates of one sampled term, each step considers a window of up to
// kWin candidates: starting at term i0 = mulhi(x0, r), terms i0, i0+1, ...
// (mod r) append their try_flip candidates in (factor, slot, rho) order until
// the window is full.  Per step:
//   1. window_kernel  (one warp per walker): the window as candidate
//      descriptors (8 bytes per row; features only when asked for);
//   2. learned policy: window_score_kernel, the tensor-core MLP (mlp_pipe.cuh)
//      whose producer computes each row's 32 features from the descriptor and
//      the walker's slots straight into the shared-memory A tile, so no
//      feature row goes through device memory; it writes one score per row;
//   3. window_apply_kernel (one thread per walker, working on its slots in
//      place in device memory): policy choice (uniform over the window via
//      x1, or epsilon-greedy argmax of the scores with epsilon decided by
//      x3), then the flip, reductions and bookkeeping of
//      the uniform walker; optional logging of the chosen candidate's features
//      (computed from the state before the flip) with the label "the step
//      lowered the rank" for training.
#include <cstdint>
#include <cuda_bf16.h>

#include "mlp_pipe.cuh"
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

// Features of a candidate as 16 packed bf16x2 words (small integers: exact).
template <class Wd>
__device__ __forceinline__ void cand_features_bf16(const PTerm<Wd, 1, true> &a, const PTerm<Wd, 1, true> &b,
                                                   const Masks<Wd, 1> &mk, uint32_t dc, uint32_t info, int r,
                                                   int best_r, int m, int n, int p, uint32_t (&h)[kFeat / 2]) {
    const int X = (int)((dc >> 10) & 3u), sneg = (int)((dc >> 22) & 1u), rho = (int)((dc >> 23) & 1u);
    float f[kFeat];
    cand_features<Wd>(a, b, mk, X, sneg, rho, (int)(info & 255u), (int)(info >> 8), r, best_r, m, n, p, f);
#pragma unroll
    for (int k = 0; k < kFeat / 2; ++k) h[k] = mlp::pack_bf16x2(f[2 * k], f[2 * k + 1]);
}

// One warp per walker.  Phase 1: eight terms i0 + g (g = lane / 4, then the
// next eight while the window has room); the four lanes of a group scan
// consecutive quarters of the slots for the term's try_flip candidates, and
// every candidate's descriptor goes to its window position in shared memory
// (order: term, then factor, then slot, then rho).  Phase 2: the lanes write
// the window rows l, l+32, ... (descriptor and info words), and, when `feat`
// is given, their feature rows (coalesced 64-byte rows; rows past the window
// are zero).
template <class Wd>
__global__ void __launch_bounds__(128) window_kernel(const SegDesc d, __nv_bfloat16 *__restrict__ feat,
                                                     uint2 *__restrict__ desc, int *__restrict__ kwin) {
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
    // ---- phase 2: window rows (and feature rows when asked for)
    uint2 *dw = desc + (size_t)w * kWin;
    for (int row = lane; row < K; row += 32) dw[row] = make_uint2(sdesc[warp][row], sinfo[warp][row]);
    if (feat) {
        __nv_bfloat16 *fw = feat + (size_t)w * kWin * kFeat;
        for (int row = lane; row < kWin; row += 32) {
            uint4 *dst = reinterpret_cast<uint4 *>(fw + (size_t)row * kFeat);
            if (row < K) {
                const uint32_t dc = sdesc[warp][row], in = sinfo[warp][row];
                const int i = (int)(dc & 1023u), j = (int)((dc >> 12) & 1023u);
                T ti, tj;
                ti.p[0] = sp[warp][i];
                ti.n[0] = sn[warp][i];
                tj.p[0] = sp[warp][j];
                tj.n[0] = sn[warp][j];
                uint32_t h[kFeat / 2];
                cand_features_bf16<Wd>(ti, tj, mk, dc, in, r, best_r, d.m, d.n, d.p, h);
#pragma unroll
                for (int k = 0; k < kFeat / 8; ++k) dst[k] = make_uint4(h[4 * k], h[4 * k + 1], h[4 * k + 2], h[4 * k + 3]);
            } else {
#pragma unroll
                for (int k = 0; k < kFeat / 8; ++k) dst[k] = make_uint4(0, 0, 0, 0);
            }
        }
    }
    if (lane == 0) kwin[w] = K;
}

// Producer of the fused scoring kernel: tile t is half t & 1 (rows 0-127 or
// 128-255) of walker t >> 1's window; thread q computes the features of row
// 128 (t & 1) + q from its descriptor and the walker's two slots, straight
// into the A tile.  A second half with no candidate is skipped; rows past the
// window get zero features and no score.  Loads in two phases, so that no
// load waits on another while the previous tile runs: begin() the window size,
// the row's descriptor and the walker's rank (every row's descriptor word is
// read; a row past the window holds a stale or undefined one, so its slot
// indices are clamped), mid() the two slots the descriptor names; the skip
// decision (live) is taken when the tile is due.
template <class Wd>
struct WindowProducer {
    static constexpr bool kFold = true;   // the producer writes features 29, 30 = 1: biases in the MMAs
    const Wd *slots;
    const tfg_walker_info *hdr;
    int R, m, n, p;
    const uint2 *desc;
    const int *kwin;
    float *score;
    Masks<Wd, 1> mk;
    // loaded by begin() / mid()
    int64_t w;
    int row, half, K, r, best_r;
    uint2 dci;
    PTerm<Wd, 1, true> ti, tj;
    __device__ __forceinline__ void begin(int64_t tile, int q) {
        w = tile >> 1;
        half = (int)(tile & 1);
        row = half * kWin / 2 + q;
        K = kwin[w];
        dci = desc[(size_t)w * kWin + row];
        r = hdr[w].r;
        best_r = hdr[w].best_r;
    }
    __device__ __forceinline__ bool live() const { return !(half && K <= kWin / 2); }
    __device__ __forceinline__ void mid(int) {
        const int i = min((int)(dci.x & 1023u), R - 1), j = min((int)((dci.x >> 12) & 1023u), R - 1);
        const Wd *src = slots + (size_t)w * R * 2;
        ti.p[0] = src[(size_t)i * 2];
        ti.n[0] = src[(size_t)i * 2 + 1];
        tj.p[0] = src[(size_t)j * 2];
        tj.n[0] = src[(size_t)j * 2 + 1];
    }
    __device__ __forceinline__ int64_t fill(uint8_t *sX, int q) {
        uint32_t h[kFeat / 2];
        if (row < K) {
            cand_features_bf16<Wd>(ti, tj, mk, dci.x, dci.y, r, best_r, m, n, p, h);
            h[14] |= 0x3F800000u;   // feature 29 = 1 (bf16), the bias inputs of the folded MMA
            h[15] |= 0x00003F80u;   // feature 30 = 1 (feature 31 is 1 already)
        } else {
#pragma unroll
            for (int k = 0; k < kFeat / 2; ++k) h[k] = 0u;
        }
#pragma unroll
        for (int c = 0; c < kFeat / 8; ++c)
            mlp::st_row8(sX, q, 8 * c, mlp::kIn, make_uint4(h[4 * c], h[4 * c + 1], h[4 * c + 2], h[4 * c + 3]));
        return row < K ? w * kWin + row : -1;
    }
    __device__ __forceinline__ void emit(float y, int64_t o) {
        if (o >= 0) score[o] = y;
    }
};

constexpr int kScoreWG = 4;

template <class Wd>
__global__ void __launch_bounds__(kScoreWG * 128, 1)
    window_score_kernel(const SegDesc d, const uint8_t *__restrict__ params, const uint2 *__restrict__ desc,
                        const int *__restrict__ kwin, float *__restrict__ score, int *__restrict__ err,
                        uint32_t first_limit) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t mbar[kScoreWG];
    __shared__ uint32_t tslot;
    __shared__ int tflag;
    WindowProducer<Wd> pr;
    pr.slots = reinterpret_cast<const Wd *>(d.slots);
    pr.hdr = d.hdr;
    pr.R = d.R;
    pr.m = d.m;
    pr.n = d.n;
    pr.p = d.p;
    pr.desc = desc;
    pr.kwin = kwin;
    pr.score = score;
    pr.mk.load(d);
    mlp::run_tiles<kScoreWG>(params, pr, d.n_walkers * 2, err, first_limit, smem, mbar, &tslot, &tflag);
}

// Log entry `slot` := (features, label, walker id, step).
__device__ __forceinline__ void write_log_entry(const WindowLog &log, unsigned long long slot,
                                                const uint32_t (&f)[kFeat / 2], float label, uint32_t wid,
                                                uint32_t step) {
    WindowLogEntry *e = reinterpret_cast<WindowLogEntry *>(log.d_entries) + slot;
#pragma unroll
    for (int k = 0; k < kFeat / 8; ++k)
        reinterpret_cast<uint4 *>(e->feat)[k] = make_uint4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
    e->label = label;
    e->walker_id = wid;
    e->step = step;
    e->pad = 0;
}

// One window-mode step per thread (walker), on the solo walker's state machine.
template <class Wd, int RMAX, int BT>
__global__ void __launch_bounds__(BT) window_apply_kernel(const SegDesc d, const uint2 *__restrict__ desc,
                                                          const int *__restrict__ kwin,
                                                          const float *__restrict__ score, int policy,
                                                          uint32_t eps_thresh, int32_t *__restrict__ choices,
                                                          WindowLog log) {
    const int64_t w = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (w >= d.n_walkers) return;
    // one step per launch: the walker works on its slots in place in device memory
    // (staging them through shared memory cost more than the step: 255 registers,
    // 3.5 warps per SM)
    using SW = SoloWalker<TFG_MODE_ZT, Wd, RMAX, BT, 0, false, true>;
    using T = typename SW::T;
    SW wk;
    wk.sm = reinterpret_cast<Wd *>(d.slots) + (size_t)w * d.R * 2;
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
    uint32_t lf[kFeat / 2];   // logged features of the chosen candidate (state before the flip)
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
        const uint2 dci = desc[(size_t)w * kWin + c];
        const uint32_t dc = dci.x;
        i = (int)(dc & 1023u);
        X = (int)((dc >> 10) & 3u);
        j = (int)((dc >> 12) & 1023u);
        sneg = (int)((dc >> 22) & 1u);
        rho = (int)((dc >> 23) & 1u);
        const T ti = wk.ld(i);
        if (log.d_entries) cand_features_bf16<Wd>(ti, wk.ld(j), wk.mk, dc, dci.y, wk.r, wk.best_r, d.m, d.n, d.p, lf);
        wk.apply_candidate(ti, i, X, j, sneg, rho, action, need_check, ti2, tj2);
    } else {
        wk.c_noc += 1;
    }
    wk.finish_step(d, wmask, lane, nl, bestp, x.z, x.w, r_before, action, X, rho, sneg, i, j, need_check, ti2, tj2);
    if (choices) choices[w] = c;
    if (log.d_entries && c >= 0) {
        const bool positive = wk.c_red > 0;   // the flip's reductions lowered the rank this step
        const int H = log.horizon > 1 ? log.horizon : 1;
        bool keep0 = false;
        if (!positive && log.neg_thresh) {
            const U4 y = philox10((uint32_t)t_step, (uint32_t)(t_step >> 32), wk.wid, 0x100u, wk.key0, wk.key1);
            keep0 = y.x < log.neg_thresh;
        }
        if (H > 1) {
            // this step's features into ring slot t mod H; a rank-lowering step appends the
            // entries of steps t-H+1 .. t still in the ring (step order) and empties it
            uint4 *ring = reinterpret_cast<uint4 *>(log.d_ring) + (size_t)w * H * (kFeat / 8);
            uint32_t *rs = log.d_ring_step + (size_t)w * H;
            const int kt = (int)(t_step % H);
#pragma unroll
            for (int k = 0; k < kFeat / 8; ++k)
                ring[kt * (kFeat / 8) + k] = make_uint4(lf[4 * k], lf[4 * k + 1], lf[4 * k + 2], lf[4 * k + 3]);
            rs[kt] = (uint32_t)t_step;
            if (positive) {
                int n = 0;
                for (int dd = 0; dd < H && dd <= t_step; ++dd)
                    n += rs[(int)((t_step - dd) % H)] == (uint32_t)(t_step - dd);
                unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(log.d_count),
                                                    (unsigned long long)n);
                for (int dd = H - 1; dd >= 0; --dd) {
                    if (dd > t_step) continue;
                    const int k = (int)((t_step - dd) % H);
                    if (rs[k] != (uint32_t)(t_step - dd)) continue;
                    if (slot < (unsigned long long)log.capacity) {
                        uint32_t e16[kFeat / 2];
#pragma unroll
                        for (int q = 0; q < kFeat / 8; ++q) {
                            const uint4 v = ring[k * (kFeat / 8) + q];
                            e16[4 * q] = v.x; e16[4 * q + 1] = v.y; e16[4 * q + 2] = v.z; e16[4 * q + 3] = v.w;
                        }
                        write_log_entry(log, slot, e16, 1.f, wk.wid, (uint32_t)(t_step - dd));
                    }
                    ++slot;
                }
                for (int k = 0; k < H; ++k) rs[k] = 0xFFFFFFFFu;
            }
        }
        const bool keep = (H == 1 && positive) || keep0;
        if (keep) {
            const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(log.d_count), 1ull);
            if (slot < (unsigned long long)log.capacity) write_log_entry(log, slot, lf, positive ? 1.f : 0.f, wk.wid,
                                                                         (uint32_t)t_step);
        }
    }
    wk.store(d, w);
}

}  // namespace dev

int window_cap() { return dev::kWin; }

void launch_window(const SegDesc &d, void *feat, uint2 *desc, int *kwin, cudaStream_t st) {
    const int64_t blocks = (d.n_walkers + 3) / 4;
    if (blocks <= 0) return;
    if (d.word_bits == 32)
        dev::window_kernel<uint32_t><<<(unsigned)blocks, 128, 0, st>>>(d, reinterpret_cast<__nv_bfloat16 *>(feat),
                                                                      desc, kwin);
    else
        dev::window_kernel<uint64_t><<<(unsigned)blocks, 128, 0, st>>>(d, reinterpret_cast<__nv_bfloat16 *>(feat),
                                                                      desc, kwin);
}

template <class Wd>
static void score_variant(const SegDesc &d, const void *params, const uint2 *desc, const int *kwin, float *score,
                          int *err, cudaStream_t st) {
    constexpr uint32_t smem = mlp::Layout<true>::bytes(dev::kScoreWG);
    static bool attr = [] {
        cudaFuncSetAttribute(dev::window_score_kernel<Wd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return true;
    }();
    (void)attr;
    const int grid = score_grid(d.n_walkers * 2, dev::kScoreWG);
    dev::window_score_kernel<Wd><<<grid, dev::kScoreWG * 128, smem, st>>>(
        d, reinterpret_cast<const uint8_t *>(params), desc, kwin, score, err, first_wait_limit());
}

void launch_window_score(const SegDesc &d, const void *params, const uint2 *desc, const int *kwin, float *score,
                         int *err, cudaStream_t st) {
    if (d.n_walkers <= 0) return;
    if (d.word_bits == 32) score_variant<uint32_t>(d, params, desc, kwin, score, err, st);
    else score_variant<uint64_t>(d, params, desc, kwin, score, err, st);
}

template <class Wd, int RMAX>
static void apply_variant(const SegDesc &d, const uint2 *desc, const int *kwin, const float *score, int policy,
                          uint32_t eps, int32_t *choices, const WindowLog &log, cudaStream_t st) {
    constexpr int BT = 128;
    const int64_t blocks = (d.n_walkers + BT - 1) / BT;
    dev::window_apply_kernel<Wd, RMAX, BT><<<(unsigned)blocks, BT, 0, st>>>(d, desc, kwin, score, policy, eps,
                                                                           choices, log);
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

int launch_window_apply(const SegDesc &d, const uint2 *desc, const int *kwin, const float *score, int policy,
                        uint32_t eps, int32_t *choices, const WindowLog &log, cudaStream_t st) {
    if (d.n_walkers <= 0) return 0;
    const int cap = window_apply_capacity(d.word_bits, d.R);
    if (d.word_bits == 32) {
        if (cap == 12) apply_variant<uint32_t, 12>(d, desc, kwin, score, policy, eps, choices, log, st);
        else if (cap == 16) apply_variant<uint32_t, 16>(d, desc, kwin, score, policy, eps, choices, log, st);
        else if (cap == 32) apply_variant<uint32_t, 32>(d, desc, kwin, score, policy, eps, choices, log, st);
        else return -1;
    } else {
        if (cap == 48) apply_variant<uint64_t, 48>(d, desc, kwin, score, policy, eps, choices, log, st);
        else if (cap == 64) apply_variant<uint64_t, 64>(d, desc, kwin, score, policy, eps, choices, log, st);
        else if (cap == 72) apply_variant<uint64_t, 72>(d, desc, kwin, score, policy, eps, choices, log, st);
        else if (cap == 88) apply_variant<uint64_t, 88>(d, desc, kwin, score, policy, eps, choices, log, st);
        else return -1;
    }
    return 0;
}

}  // namespace tfg
