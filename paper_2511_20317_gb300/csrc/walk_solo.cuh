// Thread-per-walker flip-graph walk kernel for sm_103a.
//
// Each thread owns one walker.  The walker's live scheme sits in shared
// memory as packed terms (pterm.cuh) in a [slot][thread] layout, so that a
// warp reading "slot k" touches one contiguous 8/16-byte-per-thread row
// (conflict-free vector loads).  Every loop over the slots is unrolled to
// the compile-time capacity RMAX, which turns every shared-memory address
// into an immediate offset and every candidate-mask bit into a constant;
// slots past the live rank are predicated off.  No lane of a warp waits on
// another: the only cross-thread effects are the shared memory banks.
//
// The bit-sliced variant (template parameter FL, capacity 32) also keeps the
// slots transposed, one 32-bit word per coefficient with bit k = slot k, and
// runs the candidate search, the reduction filter and the cascade's partner
// search on those words.
//
// Step order (Algorithm 1 with the plateau policy) and every tie-break are
// identical to the lane-group kernel and to the CPU reference:
//   draw -> sample term i -> try_flip candidates ordered (factor, slot, rho)
//   -> flip + ternary validity -> zero-term removal -> sign normalisation ->
//   reduction cascade -> best/plateau -> plus transition (+ cascade).
#pragma once
#include <cstdint>
#include <type_traits>

#include "pterm.cuh"

namespace tfg {
namespace dev {

// Bit set over RMAX slots: one 32-bit word when RMAX <= 32, else words of 64
// bits (slot index compile-time in loops).
template <int RMAX>
struct SlotBits {
    using B = typename std::conditional<(RMAX <= 32), uint32_t, uint64_t>::type;
    static constexpr int WB = (int)sizeof(B) * 8;
    static constexpr int NW = (RMAX + WB - 1) / WB;
    B w[NW];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int a = 0; a < NW; ++a) w[a] = 0;
    }
    __device__ __forceinline__ static int pc(B x) {
        if constexpr (sizeof(B) == 8) return __popcll(x);
        else return __popc(x);
    }
    __device__ __forceinline__ int count() const {
        int c = 0;
#pragma unroll
        for (int a = 0; a < NW; ++a) c += pc(w[a]);
        return c;
    }
    __device__ __forceinline__ bool test(int k) const {
        B v = w[0];
#pragma unroll
        for (int a = 1; a < NW; ++a) v = (k / WB) == a ? w[a] : v;
        return (v >> (k % WB)) & 1u;
    }
    __device__ __forceinline__ void set_if(int k, bool c) {   // k compile-time in unrolled loops
        w[k / WB] |= c ? (B(1) << (k % WB)) : B(0);
    }
    // keep bits [0, r) other than bit i
    __device__ __forceinline__ void keep_live(int r, int i) {
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            const int lo = r - WB * q;
            B lm = lo >= WB ? ~B(0) : (lo > 0 ? ((B(1) << lo) - 1u) : B(0));
            if ((i / WB) == q) lm &= ~(B(1) << (i % WB));
            w[q] &= lm;
        }
    }
    // position of the n-th (0-based) set bit; the set must hold more than n bits
    __device__ __forceinline__ int nth(int n) const {
        int base = 0;
        B x = w[0];
#pragma unroll
        for (int a = 1; a < NW; ++a) {
            const int c = pc(x);
            if (n >= c && base == (a - 1) * WB) { n -= c; base = a * WB; x = w[a]; }
        }
        int pos = 0;
        uint32_t y;
        if constexpr (sizeof(B) == 8) {
            const int c = __popc((uint32_t)x);
            if (n >= c) { n -= c; pos = 32; y = (uint32_t)(x >> 32); } else { y = (uint32_t)x; }
        } else {
            y = x;
        }
        int c = __popc(y & 0xffffu);
        if (n >= c) { n -= c; pos += 16; y >>= 16; }
        c = __popc(y & 0xffu);
        if (n >= c) { n -= c; pos += 8; y >>= 8; }
        c = __popc(y & 0xfu);
        if (n >= c) { n -= c; pos += 4; y >>= 4; }
        c = __popc(y & 0x3u);
        if (n >= c) { n -= c; pos += 2; y >>= 2; }
        if (n >= (int)(y & 1u)) pos += 1;
        return base + pos;
    }
    // this set, or a's / b's by a run-time choice (no divergent branches)
    __device__ __forceinline__ static SlotBits pick(int x, const SlotBits &a, const SlotBits &b, const SlotBits &c) {
        SlotBits o;
#pragma unroll
        for (int q = 0; q < NW; ++q) o.w[q] = x == 0 ? a.w[q] : (x == 1 ? b.w[q] : c.w[q]);
        return o;
    }
};

// FL > 0: the walker also keeps its slots bit-sliced (formats whose factors
// have at most FL coefficients, capacity <= 32): for factor f and coefficient
// e a 32-bit word whose bit k is that coefficient of slot k (+1 in P, -1 in
// N).  Comparing one factor of a term with every slot then costs a few word
// operations per coefficient instead of a test per slot.  In Z_T the w
// slices hold w up to sign (its first non-zero coefficient made +1) and one
// more word the sign bits, so that the sign changes of the normalisation
// (Section 3.6) touch one word and a flip rewrites the slices of one factor.
// SQ: the three factors have exactly FL coefficients each (square formats
// (k,k,k) with k*k = FL), so factor offsets and masks are compile-time constants.
// GM: the slots stay in the walker's device-memory array (slot k at sm[k * NWS],
// sm the walker's own slots) instead of shared-memory rows -- for kernels that run
// one step per launch, where staging every slot costs more than it saves; a load
// past the walker's R slots (the unrolled scans run to RMAX) gives an empty term.
template <int MODE, class Wd, int RMAX, int BT, int FL = 0, bool SQ = false, bool GM = false>
struct SoloWalker {
    static constexpr bool ZT = (MODE == TFG_MODE_ZT);
    static constexpr int NWS = ZT ? 2 : 1;   // words per slot (TW = 1)
    static constexpr bool SL = FL > 0;
    static_assert(!SL || (RMAX <= 32 && sizeof(Wd) == 4), "slices hold 32 slots of 32-bit packed terms");
    static_assert(!SQ || (SL && 3 * FL <= 32), "square factors: three of FL coefficients in one 32-bit word");
    static_assert(!GM || !SL, "device-memory slots: no bit slices");
    static constexpr int NSL = 3 * FL;       // slices per sign
    // Z_2: the slices in registers; Z_T: (P, N) pairs in shared memory [slice][thread],
    // then the w sign word (row NSL, .x)
    uint32_t S[(SL && !ZT) ? NSL : 1];
    uint2 *ss;                               // Z_T: this thread's slice column, slice q at ss[q * BT]
    int fb1, fb2;                            // bit offsets of v and w in a packed term
    uint32_t lm0, lm1, lm2;                  // coefficient masks of u, v, w (low bits)
    // Z_T: the step's try_flip masks of factors X and Z of term i (live slots other than i)
    // and the factors Y, Z the flip changes (Y | Z << 2), for the reduction filter
    uint32_t fmX, fmZ;
    int fYZ;
    uint32_t fe1, fe3;   // Z_T: slots matching Y of the new term i / Z of the new term j (from the upkeep)
    using T = PTerm<Wd, 1, ZT>;
    using O = Ops<Wd, 1, ZT>;
    using M = Masks<Wd, 1>;

    // Shared-memory rows hold one slot of every thread of the block; a row is
    // padded by one element so that walking one thread's column across the
    // lanes of a warp (cooperative filter and snapshot) spreads over the banks.
    static constexpr int RS = GM ? NWS : (BT + 1) * NWS;   // words per row (per slot with GM)
    // walkers per round of the cooperative reduction filter (interleaved scans
    // on small capacities)
#ifndef TFG_SOLO_ROUND_WALKERS
#define TFG_SOLO_ROUND_WALKERS 2
#endif
    static constexpr int kRoundWalkers = RMAX <= 32 ? TFG_SOLO_ROUND_WALKERS : 1;
    Wd *sm;      // this thread's column: slot k at sm[k * RS] (GM: the walker's slots in device memory)
    M mk;
    int r, best_r, R;
    int64_t t, plateau, best_t;
    uint64_t dig;
    uint32_t wid, key0, key1;
    uint32_t c_acc, c_rej, c_noc, c_drp, c_mrg, c_pls, c_red;
    int qlen, q0, q1, q2;
    int policy;                 // walk policy (2: additive complexity minimisation)
    uint32_t nnz, best_nnz;     // non-zero coefficients of the live / best scheme (nnz: policy 2 only)

    __device__ __forceinline__ static uint32_t nnz_of(const T &v) {
        if constexpr (ZT) return (uint32_t)popc_word(v.p[0] | v.n[0]);
        else return (uint32_t)popc_word(v.p[0]);
    }
    __device__ __forceinline__ static int popc_word(Wd x) {
        if constexpr (sizeof(Wd) == 8) return __popcll(x);
        else return __popc(x);
    }

    __device__ __forceinline__ T ld_from(const Wd *col, int k) const {
        const Wd *a = col + (size_t)k * RS;
        T v;
        if constexpr (GM) {
            if (k >= R) {
                v.p[0] = v.n[0] = Wd(0);
                return v;
            }
        }
        if constexpr (ZT) {
            if constexpr (sizeof(Wd) == 4) {
                const uint2 q = *reinterpret_cast<const uint2 *>(a);
                v.p[0] = q.x; v.n[0] = q.y;
            } else {
                const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(a);
                v.p[0] = q.x; v.n[0] = q.y;
            }
        } else {
            v.p[0] = a[0];
            v.n[0] = 0;
        }
        return v;
    }
    __device__ __forceinline__ T ld(int k) const {
        const Wd *a = sm + (size_t)k * RS;

        T v;
        if constexpr (GM) {
            if (k >= R) {
                v.p[0] = v.n[0] = Wd(0);
                return v;
            }
        }
        if constexpr (ZT) {
            if constexpr (sizeof(Wd) == 4) {
                const uint2 q = *reinterpret_cast<const uint2 *>(a);
                v.p[0] = q.x; v.n[0] = q.y;
            } else {
                const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(a);
                v.p[0] = q.x; v.n[0] = q.y;
            }
        } else {
            v.p[0] = a[0];
            v.n[0] = 0;
        }
        return v;
    }
    __device__ __forceinline__ void st(int k, const T &v) {
        Wd *a = sm + (size_t)k * RS;
        if constexpr (ZT) {
            if constexpr (sizeof(Wd) == 4) *reinterpret_cast<uint2 *>(a) = make_uint2(v.p[0], v.n[0]);
            else *reinterpret_cast<ulonglong2 *>(a) = make_ulonglong2(v.p[0], v.n[0]);
        } else {
            a[0] = v.p[0];
        }
        if constexpr (SL) sl_put(k, v);
    }
    // store of a flipped term (factor f changed; see sl_put_flip); Z_T slices: returns the
    // slots whose factor f equals v's
    __device__ __forceinline__ uint32_t st_flip(int k, const T &v, int f) {
        Wd *a = sm + (size_t)k * RS;
        if constexpr (ZT) {
            if constexpr (sizeof(Wd) == 4) *reinterpret_cast<uint2 *>(a) = make_uint2(v.p[0], v.n[0]);
            else *reinterpret_cast<ulonglong2 *>(a) = make_ulonglong2(v.p[0], v.n[0]);
        } else {
            a[0] = v.p[0];
        }
        if constexpr (SL) return sl_put_flip(k, v, f);
        else return 0u;
    }

    // ---- bit slices (FL > 0)
    // coefficients of factor f (compile-time) of packed word x, in the low bits
    __device__ __forceinline__ uint32_t fx(uint32_t x, int f) const {
        return f == 0 ? (x & lm0) : (f == 1 ? ((x >> fb1) & lm1) : ((x >> fb2) & lm2));
    }
    // all ones when bit e (compile-time) of y is set, else zero
    __device__ __forceinline__ static uint32_t bc(uint32_t y, int e) {
        return (uint32_t)((int32_t)(y << (31 - e)) >> 31);
    }
    // factor f (run-time) of packed word x, in the low bits
    __device__ __forceinline__ uint32_t fx_rt(uint32_t x, int f) const {
        const int sh = f == 0 ? 0 : (f == 1 ? fb1 : fb2);
        const uint32_t m = f == 0 ? lm0 : (f == 1 ? lm1 : lm2);
        return (x >> sh) & m;
    }
    // the first non-zero coefficient of the factor (xp, xn) is -1
    __device__ __forceinline__ static bool lead_neg(uint32_t xp, uint32_t xn) {
        const uint32_t d = xp | xn;
        return (xn & d & (0u - d)) != 0u;
    }
    // slices of factor f (f compile-time, or run-time through base) at slot k := (xp, xn);
    // w (f = 2) up to sign, its sign bit in the sign word.  Returns the slots whose
    // factor f equals (xp, xn), from the words as they were (slot k's own bit aside,
    // the same as after the write).
    __device__ __forceinline__ uint32_t sl_write(uint2 *base, uint32_t kb, uint32_t xp, uint32_t xn) const {
        uint32_t dd = 0;
#pragma unroll
        for (int e = 0; e < FL; ++e) {
            uint2 w = base[e * BT];
            const uint32_t bp = bc(xp, e), bn = bc(xn, e);
            dd |= (w.x ^ bp) | (w.y ^ bn);
            w.x = (w.x & ~kb) | (bp & kb);
            w.y = (w.y & ~kb) | (bn & kb);
            base[e * BT] = w;
        }
        return ~dd;
    }
    __device__ __forceinline__ void sl_sign(uint32_t kb, bool neg) const {
        uint2 *g = ss + NSL * BT;
        g->x = (g->x & ~kb) | (neg ? kb : 0u);
    }
    // slot k of every slice := term v
    __device__ __forceinline__ void sl_put(int k, const T &v) {
        const uint32_t kb = 1u << k;
        if constexpr (ZT) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                uint32_t xp = fx((uint32_t)v.p[0], f), xn = fx((uint32_t)v.n[0], f);
                if (f == 2) {
                    const bool ng = lead_neg(xp, xn);
                    sl_sign(kb, ng);
                    if (ng) { const uint32_t t = xp; xp = xn; xn = t; }
                }
                sl_write(ss + f * FL * BT, kb, xp, xn);
            }
        } else {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const uint32_t xp = fx((uint32_t)v.p[0], f);
#pragma unroll
                for (int e = 0; e < FL; ++e) {
                    const int q = f * FL + e;
                    S[q] = (S[q] & ~kb) | (bc(xp, e) & kb);
                }
            }
        }
    }
    // slot k := term v that differs from the slot's previous term in factor f
    // (run-time) only, up to the sign changes of the normalisation (u and v
    // keep their own signs; w's sign is one bit).  Z_2: every slice.
    // Z_T returns the slots whose factor f equals v's (w up to sign), for the filter.
    __device__ __forceinline__ uint32_t sl_put_flip(int k, const T &v, int f) {
        if constexpr (ZT) {
            const uint32_t kb = 1u << k;
            uint32_t xp = fx_rt((uint32_t)v.p[0], f), xn = fx_rt((uint32_t)v.n[0], f);
            const uint32_t wp = fx((uint32_t)v.p[0], 2), wn = fx((uint32_t)v.n[0], 2);
            const bool ng = lead_neg(wp, wn);
            sl_sign(kb, ng);
            if (f == 2 && ng) { const uint32_t t = xp; xp = xn; xn = t; }
            return sl_write(ss + f * FL * BT, kb, xp, xn);
        } else {
            sl_put(k, v);
            return 0u;
        }
    }
    // Slots (any of the 32) whose u / v / w equal term a's: w either sign (mw)
    // and w negated (mwn, Z_T).
    __device__ __forceinline__ void sl_match(const T &a, uint32_t &mu, uint32_t &mv, uint32_t &mw,
                                             uint32_t &mwn) const {
        uint32_t du = 0, dv = 0, dw = 0;   // bit k: slot k differs
        bool wneg = false;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            uint32_t xp = fx((uint32_t)a.p[0], f);
            uint32_t xn = ZT ? fx((uint32_t)a.n[0], f) : 0u;
            if (ZT && f == 2) {
                wneg = lead_neg(xp, xn);
                if (wneg) { const uint32_t t = xp; xp = xn; xn = t; }
            }
#pragma unroll
            for (int e = 0; e < FL; ++e) {
                const int q = f * FL + e;
                uint32_t dd;
                if constexpr (ZT) {
                    const uint2 w = ss[q * BT];
                    dd = (w.x ^ bc(xp, e)) | (w.y ^ bc(xn, e));
                } else {
                    dd = S[q] ^ bc(xp, e);
                }
                if (f == 0) du |= dd;
                else if (f == 1) dv |= dd;
                else dw |= dd;
            }
        }
        mu = ~du;
        mv = ~dv;
        mw = ~dw;
        if constexpr (ZT) mwn = mw & (ss[NSL * BT].x ^ (wneg ? ~0u : 0u));
        else mwn = 0u;
    }
    // Slots (any of the 32) whose factor f (run-time) equals term a's (w up to sign); Z_T
    __device__ __forceinline__ uint32_t sl_factor_match(const T &a, int f) const {
        uint32_t xp = fx_rt((uint32_t)a.p[0], f), xn = fx_rt((uint32_t)a.n[0], f);
        if (f == 2 && lead_neg(xp, xn)) { const uint32_t t = xp; xp = xn; xn = t; }
        const uint2 *base = ss + f * FL * BT;
        uint32_t dd = 0;
#pragma unroll
        for (int e = 0; e < FL; ++e) {
            const uint2 w = base[e * BT];
            dd |= (w.x ^ bc(xp, e)) | (w.y ^ bc(xn, e));
        }
        return ~dd;
    }
    // Z_T reduction filter from the try_flip masks: the new terms are
    // i' = (X_i, Y_i + Y_j, Z_i) and j' = (X_j, Y_j, Z_j - s Z_i) with X_j = +-X_i, so a
    // third slot shares a pair with i' iff it matches two of X_i (fmX), Y_i' and Z_i
    // (fmZ), and with j' iff two of X_j (fmX again), Y_j and Z_j'.  i' and j' never
    // share a pair with each other: besides X that would need Y_i = 0, or Z_j equal to
    // 0 or to +-2 Z_i.
    __device__ __forceinline__ bool sl_pair_hit_flip(const T &a, int i, const T &b, int j) const {
        const int Y = fYZ & 3;
        (void)a;
        const uint32_t e1 = fe1, e2 = sl_factor_match(b, Y), e3 = fe3;
        const uint32_t x = fmX, z = fmZ;
        const uint32_t live = (r >= 32 ? ~0u : ((1u << r) - 1u)) & ~(1u << i) & ~(1u << j);
        return (((x & z) | (e1 & (x | z)) | (e2 & (x | e3)) | (x & e3)) & live) != 0u;
    }
    // Any live slot other than i (j) sharing a factor pair with term a (b)?
    __device__ __forceinline__ bool sl_pair_hit(const T &a, int i, const T &b, int j) const {
        uint32_t mu, mv, mw, mwn;
        sl_match(a, mu, mv, mw, mwn);
        const uint32_t pa = ((mu & mv) | (mu & mw) | (mv & mw)) & ~(1u << i);
        sl_match(b, mu, mv, mw, mwn);
        const uint32_t pb = ((mu & mv) | (mu & mw) | (mv & mw)) & ~(1u << j);
        const uint32_t live = r >= 32 ? ~0u : ((1u << r) - 1u);
        return ((pa | pb) & live) != 0u;
    }

    // ---- reduction queue (slot indices)
    __device__ __forceinline__ void q_push(int s) {
        q0 = (qlen == 0) ? s : q0;
        q1 = (qlen == 1) ? s : q1;
        q2 = (qlen == 2) ? s : q2;
        qlen += 1;
    }
    __device__ __forceinline__ int q_pop() {
        const int s = q0;
        q0 = q1; q1 = q2;
        qlen -= 1;
        return s;
    }
    __device__ __forceinline__ void q_remove(int s) {
        const bool k0 = qlen > 0 && q0 != s, k1 = qlen > 1 && q1 != s, k2 = qlen > 2 && q2 != s;
        const int n0 = k0 ? q0 : (k1 ? q1 : q2);
        const int n1 = k0 ? (k1 ? q1 : q2) : q2;
        q0 = n0; q1 = n1;
        qlen = (int)k0 + (int)k1 + (int)k2;
    }
    __device__ __forceinline__ void q_rename(int from, int to) {
        q0 = (qlen > 0 && q0 == from) ? to : q0;
        q1 = (qlen > 1 && q1 == from) ? to : q1;
        q2 = (qlen > 2 && q2 == from) ? to : q2;
    }

    // Remove slot h: the last live term moves into the hole.
    __device__ __forceinline__ void drop(int h) {
        const int last = r - 1;
        q_remove(h);
        if (h != last) {
            st(h, ld(last));
            q_rename(last, h);
        }
        r -= 1;
    }

    // validity of a_f + (neg ? -b_f : b_f)
    __device__ __forceinline__ bool sum_ok(const T &a, const T &b, Wd m, bool neg) const {
        if constexpr (ZT) {
            const Wd bp = neg ? b.n[0] : b.p[0], bn = neg ? b.p[0] : b.n[0];
            return (((a.p[0] & bp) | (a.n[0] & bn)) & m) == Wd(0);
        } else {
            return true;
        }
    }

    // Reduction of slot s with the lowest partner sharing (u,v), else (u,w),
    // else (v,w), whose merged third factor stays in the coefficient set.
    __device__ __forceinline__ void reduce_one(int s) {
        const T v = ld(s);
        int k0 = -1, k1 = -1, k2 = -1;
        bool n1 = false, n2 = false;
        if constexpr (SL) {
            // pair candidates from the slices, then the lowest one whose merged third
            // factor stays in the coefficient set
            uint32_t mu, mv, mw, mwn;
            sl_match(v, mu, mv, mw, mwn);
            const uint32_t live = (r >= 32 ? ~0u : ((1u << r) - 1u)) & ~(1u << s);
            uint32_t c0 = mu & mv & live, c1 = mu & mw & live, c2 = mv & mw & live;
#pragma unroll 1
            while (c0 && k0 < 0) {
                const int k = __ffs(c0) - 1;
                c0 &= c0 - 1u;
                if (sum_ok(v, ld(k), mk.m[2][0], false)) k0 = k;
            }
#pragma unroll 1
            while (k0 < 0 && c1 && k1 < 0) {
                const int k = __ffs(c1) - 1;
                c1 &= c1 - 1u;
                const bool ng = (mwn >> k) & 1u;
                if (sum_ok(v, ld(k), mk.m[1][0], ng)) { k1 = k; n1 = ng; }
            }
#pragma unroll 1
            while (k0 < 0 && k1 < 0 && c2 && k2 < 0) {
                const int k = __ffs(c2) - 1;
                c2 &= c2 - 1u;
                const bool ng = (mwn >> k) & 1u;
                if (sum_ok(v, ld(k), mk.m[0][0], ng)) { k2 = k; n2 = ng; }
            }
        } else {
#pragma unroll
        for (int k = 0; k < RMAX; ++k) {
            const T c = ld(k);
            const bool live = k < r && k != s;
            bool eu, ev, ewp, ewn;
            O::compare(c, v, mk, eu, ev, ewp, ewn);
            const bool ew = ewp || ewn;
            const bool m0 = live && eu && ev && sum_ok(v, c, mk.m[2][0], false);
            const bool m1 = live && eu && ew && sum_ok(v, c, mk.m[1][0], ewn);
            const bool m2 = live && ev && ew && sum_ok(v, c, mk.m[0][0], ewn);
            if (m0 && k0 < 0) k0 = k;
            if (m1 && k1 < 0) { k1 = k; n1 = ewn; }
            if (m2 && k2 < 0) { k2 = k; n2 = ewn; }
        }
        }
        if (k0 < 0 && k1 < 0 && k2 < 0) return;
        const int P = k0 >= 0 ? 0 : (k1 >= 0 ? 1 : 2);
        const int k = P == 0 ? k0 : (P == 1 ? k1 : k2);
        const bool kneg = P == 1 ? n1 : (P == 2 ? n2 : false);
        const int F = 2 - P;   // third factor: w, v, u
        const T kv = ld(k);
        T mv;
        O::add(v, kv, F, kneg, mk, mv);
        const bool zero = O::zero(mv, F, mk);
        O::canon(mv, mk);
        const int lo = s < k ? s : k;
        const int hi = s < k ? k : s;
        q_remove(k);
        st(lo, mv);
        c_mrg += 1;
        drop(hi);
        if (zero) {
            drop(lo);
            c_drp += 1;
        } else {
            q_push(lo);
        }
    }

    // Reduction cascade of every thread of the warp: the loop runs while any
    // thread still has queued terms, so the warp is converged afterwards.
    __device__ __forceinline__ void cascade_all(unsigned wmask) {
#pragma unroll 1
        while (__any_sync(wmask, qlen > 0)) {
            if (qlen > 0) reduce_one(q_pop());
        }
    }

    // Any other live slot sharing a factor pair with a (slot sa) or b (slot sb)?
    __device__ __forceinline__ bool pair_hit2(const T &a, int sa, const T &b, int sb) const {
        bool hit = false;
#pragma unroll
        for (int k = 0; k < RMAX; ++k) {
            const T c = ld(k);
            bool eu, ev, ewp, ewn;
            O::compare(c, a, mk, eu, ev, ewp, ewn);
            const bool ew = ewp || ewn;
            const bool ha = (eu && ev) || (eu && ew) || (ev && ew);
            O::compare(c, b, mk, eu, ev, ewp, ewn);
            const bool ew2 = ewp || ewn;
            const bool hb = (eu && ev) || (eu && ew2) || (ev && ew2);
            hit |= (k < r) && ((ha && k != sa) || (hb && k != sb));
        }
        return hit;
    }

    // Reduction filter of the warp's accepted flips (terms ti2 in slot i and
    // tj2 in slot j share a factor pair with another live slot?).  When few
    // threads need it, the warp checks one walker at a time, its lanes taking
    // the walker's slots lane, lane+nl, ... from shared memory; when most
    // need it, every thread scans its own slots.
    __device__ __forceinline__ bool coop_pair_hit(unsigned wmask, int lane, int nl, bool need, const T &ti2,
                                                  int i, const T &tj2, int j) const {
        // bit slices: per thread, ~2*3*FL (Z_2) / ~2*9*FL (Z_T) word operations, which
        // measured faster than the lane-cooperative test at every pending count
        if constexpr (SL) {
            if constexpr (ZT) return need && sl_pair_hit_flip(ti2, i, tj2, j);
            else return need && sl_pair_hit(ti2, i, tj2, j);
        }
        unsigned pend = __ballot_sync(wmask, need);
        if (__popc(pend) * 4 > RMAX * 3) return need && pair_hit2(ti2, i, tj2, j);
        if constexpr (GM) __syncwarp(wmask);   // other lanes' device-memory slot writes visible
        bool mine = false;
        const int packed = i | (j << 10) | (r << 20);
        if constexpr (kRoundWalkers > 1) {
            // kRoundWalkers pending walkers per round, their scans interleaved
            constexpr int WR = kRoundWalkers;
#pragma unroll 1
            while (pend) {
                int a[WR];
#pragma unroll
                for (int q = 0; q < WR; ++q) {
                    a[q] = pend ? __ffs(pend) - 1 : a[0];   // a repeated walker recomputes the same answer
                    pend &= pend - 1;
                }
                T A[WR], B[WR];
                int pk[WR];
                bool h[WR];
                const Wd *colq[WR];
#pragma unroll
                for (int q = 0; q < WR; ++q) {
                    A[q] = shfl_term(wmask, ti2, a[q]);
                    B[q] = shfl_term(wmask, tj2, a[q]);
                    pk[q] = __shfl_sync(wmask, packed, a[q]);
                    colq[q] = col_of(wmask, a[q], lane);
                    h[q] = false;
                }
                if (nl == 32) {
#pragma unroll
                    for (int kk = 0; kk < (RMAX + 31) / 32; ++kk) {
                        const int k = lane + 32 * kk;
#pragma unroll
                        for (int q = 0; q < WR; ++q) h[q] |= slot_shares_pair(colq[q], k, pk[q], A[q], B[q]);
                    }
                } else {
#pragma unroll 1
                    for (int k = lane; k < RMAX; k += nl) {
#pragma unroll
                        for (int q = 0; q < WR; ++q) h[q] |= slot_shares_pair(colq[q], k, pk[q], A[q], B[q]);
                    }
                }
#pragma unroll
                for (int q = 0; q < WR; ++q) {
                    const unsigned hv = __ballot_sync(wmask, h[q]);
                    if (lane == a[q]) mine = hv != 0u;
                }
            }
        } else {
            // one pending walker per round
#pragma unroll 1
            while (pend) {
                const int a = __ffs(pend) - 1;
                pend &= pend - 1;
                const T A = shfl_term(wmask, ti2, a), B = shfl_term(wmask, tj2, a);
                const int pa = __shfl_sync(wmask, packed, a);
                const Wd *col = col_of(wmask, a, lane);   // walker a's slots
                const int ra = pa >> 20;
                const int ia = pa & 1023, ja = (pa >> 10) & 1023;
                bool hit = false;
#pragma unroll 1
                for (int k = lane; k < ra; k += nl) {
                    const T c = ld_from(col, k);
                    bool eu, ev, ewp, ewn;
                    O::compare(c, A, mk, eu, ev, ewp, ewn);
                    bool ew = ewp || ewn;
                    const bool ha = (eu && ev) || (eu && ew) || (ev && ew);
                    O::compare(c, B, mk, eu, ev, ewp, ewn);
                    ew = ewp || ewn;
                    const bool hb = (eu && ev) || (eu && ew) || (ev && ew);
                    hit = hit || (ha && k != ia) || (hb && k != ja);
                }
                const unsigned hv = __ballot_sync(wmask, hit);
                if (lane == a) mine = hv != 0u;
            }
        }
        return mine;
    }
    // Slots of walker a (a lane of this warp): its column of the shared-memory rows,
    // or (GM) its device-memory slots, whose address lane a holds.  Warp-converged.
    __device__ __forceinline__ const Wd *col_of(unsigned wmask, int a, int lane) const {
        if constexpr (GM)
            return reinterpret_cast<const Wd *>(__shfl_sync(wmask, reinterpret_cast<unsigned long long>(sm), a));
        else
            return sm + (a - lane) * NWS;
    }
    __device__ __forceinline__ static T shfl_term(unsigned wmask, const T &v, int src) {
        T o;
        o.p[0] = __shfl_sync(wmask, v.p[0], src);
        o.n[0] = ZT ? __shfl_sync(wmask, v.n[0], src) : Wd(0);
        return o;
    }
    // Does slot k of a walker's column share a factor pair with A (its slot
    // ia) or B (slot ja)?  packed = ia | ja << 10 | r << 20; k >= r is false.
    __device__ __forceinline__ bool slot_shares_pair(const Wd *col, int k, int packed, const T &A, const T &B) const {
        const int ia = packed & 1023, ja = (packed >> 10) & 1023, ra = packed >> 20;
        if (k >= RMAX) return false;
        const T c = ld_from(col, k);
        bool eu, ev, ewp, ewn;
        O::compare(c, A, mk, eu, ev, ewp, ewn);
        bool ew = ewp || ewn;
        const bool ha = (eu && ev) || (eu && ew) || (ev && ew);
        O::compare(c, B, mk, eu, ev, ewp, ewn);
        ew = ewp || ewn;
        const bool hb = (eu && ev) || (eu && ew) || (ev && ew);
        return k < ra && ((ha && k != ia) || (hb && k != ja));
    }

    // Warp-cooperative best snapshot: lanes copy consecutive slots of each
    // requesting walker's column to its best buffer (coalesced stores).
    __device__ __forceinline__ void coop_snapshot(unsigned wmask, int lane, int nl, bool want, Wd *bestp) const {
        unsigned pend = __ballot_sync(wmask, want);
        if constexpr (GM) __syncwarp(wmask);
#pragma unroll 1
        while (pend) {
            const int a = __ffs(pend) - 1;
            pend &= pend - 1;
            const int ra = __shfl_sync(wmask, r, a);
            Wd *dst = reinterpret_cast<Wd *>(__shfl_sync(wmask, reinterpret_cast<unsigned long long>(bestp), a));
            const Wd *col = col_of(wmask, a, lane);
#pragma unroll 1
            for (int k = lane; k < ra; k += nl) {
                const T v = ld_from(col, k);
                if constexpr (ZT) {
                    if constexpr (sizeof(Wd) == 4) reinterpret_cast<uint2 *>(dst)[k] = make_uint2(v.p[0], v.n[0]);
                    else reinterpret_cast<ulonglong2 *>(dst)[k] = make_ulonglong2(v.p[0], v.n[0]);
                } else {
                    dst[k] = v.p[0];
                }
            }
        }
    }

    // Expansion (Section 3.3.1): plus (three terms from the pair) or, under
    // walk policy 1 when y3 >= 2^31, split (term i = (A_j, B_i, C_i), new term
    // (A_i - A_j, B_i, C_i)); writes the new terms, queues them for the cascade
    // and returns the digest record (0 when no attempt passed).
    __device__ __forceinline__ uint64_t plus_setup(const SegDesc &d) {
#pragma unroll 1
        for (int a = 1; a <= d.plus_attempts; ++a) {
            const U4 y = philox10((uint32_t)t, (uint32_t)(t >> 32), wid, (uint32_t)a, key0, key1);
            const int pi = (int)__umulhi(y.x, (uint32_t)r);
            const int pj = (pi + 1 + (int)__umulhi(y.y, (uint32_t)(r - 1))) % r;
            const int perm = (int)__umulhi(y.z, 6u);
            const bool split = d.walk_policy == 1 && y.w >= 0x80000000u;
            int A, B, C;
            plus_roles(perm, A, B, C);
            const T ti = ld(pi), tj = ld(pj);
            if (split) {
                T na;                                       // (A_i - A_j, B_i, C_i)
                const bool ok = O::add(ti, tj, A, true, mk, na);
                if (!ok || O::zero(na, A, mk)) continue;
                O::canon(na, mk);
                st(r, na);
                T ti2 = ti;                                 // (A_j, B_i, C_i)
                O::take(ti2, tj, A, mk);
                O::canon(ti2, mk);
                st(pi, ti2);
                r += 1;
                plateau = 0;
                c_pls += 1;
                qlen = 0;
                q_push(pi);
                q_push(r - 1);
                return plus_record(a, perm, pi, pj, 1);
            }
            T nb, nc, na;
            bool ok = O::add(ti, tj, B, false, mk, nb);      // B_i + B_j
            ok &= O::add(tj, ti, C, true, mk, nc);           // C_j - C_i
            ok &= O::add(tj, ti, A, true, mk, na);           // A_j - A_i
            ok = ok && !O::zero(nb, B, mk) && !O::zero(nc, C, mk) && !O::zero(na, A, mk);
            if (!ok) continue;
            T tn = na;                 // (A_j - A_i, B_j, C_j)
            O::canon(tn, mk);
            st(r, tn);
            T tj2 = nc;                // (A_i, B_j, C_j - C_i)
            O::take(tj2, ti, A, mk);
            O::canon(tj2, mk);
            st(pj, tj2);
            T ti2 = nb;                // (A_i, B_i + B_j, C_i)
            O::canon(ti2, mk);
            st(pi, ti2);
            r += 1;
            plateau = 0;
            c_pls += 1;
            qlen = 0;
            q_push(pi);
            q_push(pj);
            q_push(r - 1);
            return plus_record(a, perm, pi, pj);
        }
        return 0;
    }

    // ---- walker record and slots: HBM -> registers / shared memory
    __device__ __forceinline__ void load(const SegDesc &d, int64_t w) {
        const tfg_walker_info *H = d.hdr + w;
        r = H->r; best_r = H->best_r; R = d.R;
        t = H->t; plateau = H->plateau; best_t = H->best_t;
        dig = H->digest; wid = H->walker_id;
        key0 = d.key0; key1 = d.key1;
        policy = d.walk_policy;
        best_nnz = H->best_nnz;
        mk.load(d);
        if constexpr (SL && SQ) {
            constexpr uint32_t lm = (1u << FL) - 1u;
            mk.m[0][0] = (Wd)lm;
            mk.m[1][0] = (Wd)(lm << FL);
            mk.m[2][0] = (Wd)(lm << (2 * FL));
            fb1 = FL;
            fb2 = 2 * FL;
            lm0 = lm1 = lm2 = lm;
        } else if constexpr (SL) {
            fb1 = d.fbase[1];
            fb2 = d.fbase[2];
            const int l0 = d.m * d.n, l1 = d.n * d.p, l2 = d.p * d.m;
            lm0 = (1u << l0) - 1u;
            lm1 = (1u << l1) - 1u;
            lm2 = (1u << l2) - 1u;
        }
        if constexpr (SL) {
#pragma unroll
            for (int q = 0; q < NSL + 1; ++q) {
                if constexpr (ZT) ss[q * BT] = make_uint2(0u, 0u);
                else if (q < NSL) S[q] = 0u;
            }
        }
        c_acc = c_rej = c_noc = c_drp = c_mrg = c_pls = c_red = 0;
        qlen = 0; q0 = q1 = q2 = 0;
        if constexpr (!GM) load_slots(d, w);
        nnz = 0;
        if (policy == 2) {
#pragma unroll
            for (int k = 0; k < RMAX; ++k)
                if (k < r) nnz += nnz_of(ld(k));
        }
    }

    __device__ __forceinline__ void load_slots(const SegDesc &d, int64_t w) {
        const Wd *src = reinterpret_cast<const Wd *>(d.slots) + (size_t)w * R * NWS;
        auto load_slot = [&](int k) {
            T v;
            v.p[0] = (k < R) ? src[(size_t)k * NWS] : Wd(0);
            v.n[0] = (ZT && k < R) ? src[(size_t)k * NWS + (NWS - 1)] : Wd(0);
            st(k, v);
        };
        if constexpr (SL) {
            // once per launch: a rolled loop keeps the slice writes out of line
#pragma unroll 1
            for (int k = 0; k < RMAX; ++k) load_slot(k);
        } else {
#pragma unroll
            for (int k = 0; k < RMAX; ++k) load_slot(k);
        }
    }

    __device__ __forceinline__ void store(const SegDesc &d, int64_t w) {
        if constexpr (!GM) {   // GM: the slots were written in place
            Wd *dst = reinterpret_cast<Wd *>(d.slots) + (size_t)w * R * NWS;
#pragma unroll
            for (int k = 0; k < RMAX; ++k) {
                if (k < R) {
                    const T v = ld(k);
                    dst[(size_t)k * NWS] = v.p[0];
                    if constexpr (ZT) dst[(size_t)k * NWS + 1] = v.n[0];
                }
            }
        }
        tfg_walker_info *H = d.hdr + w;
        H->r = r; H->best_r = best_r;
        H->t = t; H->plateau = plateau; H->best_t = best_t;
        H->digest = dig;
        H->accepted += c_acc; H->rejected += c_rej; H->nocand += c_noc;
        H->drops += c_drp; H->merges += c_mrg; H->plus += c_pls; H->reductions += c_red;
        H->best_nnz = best_nnz;
    }

    // ---- flip of candidate (X, j, sign, rho) on term i (Section 3.3.1) with the
    // ternary validity test; on acceptance the terms are normalised and stored,
    // zero terms are removed, and need_check asks for the reduction filter.
    __device__ __forceinline__ void apply_candidate(const T &ti, int i, int X, int j, int sneg, int rho, int &action,
                                                    bool &need_check, T &ti2, T &tj2) {
        const T tj = ld(j);
        // (Y, Z) cyclic after X, rho swaps; Y_i += Y_j, Z_j -= s Z_i
        int Y = X == 0 ? 1 : (X == 1 ? 2 : 0);
        int Z = X == 0 ? 2 : (X == 1 ? 0 : 1);
        if (rho) { const int tmp = Y; Y = Z; Z = tmp; }
        bool ok = O::add(ti, tj, Y, false, mk, ti2);
        ok &= O::add(tj, ti, Z, sneg == 0, mk, tj2);
        if (!ok) {
            action = kReject;
            c_rej += 1;
            return;
        }
        action = kAccept;
        c_acc += 1;
        const bool zi = O::zero(ti2, Y, mk);
        const bool zj = O::zero(tj2, Z, mk);
        if (policy == 2) nnz += (zi ? 0u : nnz_of(ti2)) + (zj ? 0u : nnz_of(tj2)) - nnz_of(ti) - nnz_of(tj);
        O::canon(ti2, mk);
        O::canon(tj2, mk);
        const uint32_t e1 = st_flip(i, ti2, Y), e3 = st_flip(j, tj2, Z);
        if constexpr (SL && ZT) { fe1 = e1; fe3 = e3; }
        else { (void)e1; (void)e3; }
        qlen = 0;
        if (zi || zj) {
            q_push(i);
            q_push(j);
            const int hi = i > j ? i : j, lo = i > j ? j : i;
            const bool zhi = (hi == i) ? zi : zj, zlo = (lo == i) ? zi : zj;
            if (zhi) { drop(hi); c_drp += 1; }
            if (zlo) { drop(lo); c_drp += 1; }
            if (policy == 2) qlen = 0;   // no reduction edges
        } else {
            need_check = policy != 2;
        }
    }

    // ---- rest of a step, warp-converged: reduction filter and cascade, digest,
    // best / plateau bookkeeping and snapshot, plus transition and its cascade.
    __device__ __forceinline__ void finish_step(const SegDesc &d, unsigned wmask, int lane, int nl, Wd *bestp,
                                                uint32_t x2, uint32_t x3, int r_before, int action, int X, int rho,
                                                int sneg, int i, int j, bool need_check, const T &ti2,
                                                const T &tj2) {
        if (coop_pair_hit(wmask, lane, nl, need_check, ti2, i, tj2, j)) {
            q_push(i);
            q_push(j);
        }
        uint64_t rec2 = 0;
#pragma unroll 1
        for (int phase = 0; phase < 2; ++phase) {
            cascade_all(wmask);
            if (phase == 0) {
                if (r < r_before) c_red += 1;
                dig = digest_mix(dig, flip_record(action, X, rho, sneg, i, j, r));
                // walk policy 1: a failed try_flip expands and ends the step (no best update)
                const bool failed = d.walk_policy == 1 && action != kAccept;
                bool want = false;
                if (d.walk_policy == 2) {
                    // the best scheme is the one of least (rank, non-zero coefficients)
                    if (r < best_r || (r == best_r && nnz < best_nnz)) {
                        want = true;
                        best_r = r;
                        best_nnz = nnz;
                        best_t = t;
                        plateau = 0;
                    } else {
                        want = (r == best_r && nnz == best_nnz && x2 < d.refresh_thresh);
                        plateau += 1;
                    }
                } else if (failed) {
                    plateau += 1;
                } else if (r < best_r) {
                    want = true;
                    best_r = r;
                    best_t = t;
                    plateau = 0;
                } else {
                    want = (r == best_r && x2 < d.refresh_thresh);
                    plateau += 1;
                }
                coop_snapshot(wmask, lane, nl, want, bestp);
                bool expand;
                if (d.walk_policy == 2)
                    expand = false;
                else if (d.walk_policy == 1)
                    expand = failed ? (r < R && r >= 2) : (x3 < d.expand_thresh && r <= best_r + 2 && r < R && r >= 2);
                else
                    expand = d.plus_enabled && plateau >= d.plateau_len && r <= best_r + 2 && r < R && r >= 2;
                if (expand) rec2 = plus_setup(d);
            } else if (rec2) {
                dig = digest_mix(dig, rec2 | ((uint64_t)(uint32_t)r << 44));
            }
        }
        t += 1;
    }

    __device__ __forceinline__ void run(const SegDesc &d, int64_t w, int32_t steps) {
        load(d, w);
        Wd *bestp = reinterpret_cast<Wd *>(d.best) + (size_t)w * R * NWS;
        // threads past the population returned already; the live lanes of a
        // warp are 0 .. nl-1 (walkers are assigned to consecutive threads)
        const unsigned wmask = __activemask();
        const int lane = threadIdx.x & 31;
        const int nl = __popc(wmask);
#pragma unroll 1
        for (int32_t step = 0; step < steps; ++step) {
            const U4 x = philox10((uint32_t)t, (uint32_t)(t >> 32), wid, 0u, key0, key1);
            const int r_before = r;
            const int i = (int)__umulhi(x.x, (uint32_t)r);
            int action = kNoCand, X = 0, j = 0, rho = 0, sneg = 0;
            bool need_check = false;
            T ti2, tj2;
            ti2.p[0] = tj2.p[0] = 0;
            ti2.n[0] = tj2.n[0] = 0;
            {
                const T ti = ld(i);
                // ---- try_flip candidates: X_j = +-X_i, ordered (X, slot, rho)
                SlotBits<RMAX> mu, mv, mw, mwn;
                mu.clear(); mv.clear(); mw.clear();
                if constexpr (ZT) mwn.clear();
                if constexpr (SL) {
                    uint32_t a0, a1, a2, a3;
                    sl_match(ti, a0, a1, a2, a3);
                    mu.w[0] = a0; mv.w[0] = a1; mw.w[0] = a2;
                    if constexpr (ZT) mwn.w[0] = a3;
                } else {
#pragma unroll
                    for (int k = 0; k < RMAX; ++k) {
                        const T c = ld(k);
                        bool eu, ev, ewp, ewn;
                        O::compare(c, ti, mk, eu, ev, ewp, ewn);
                        mu.set_if(k, eu);
                        mv.set_if(k, ev);
                        mw.set_if(k, ewp || ewn);
                        if constexpr (ZT) mwn.set_if(k, ewn);
                    }
                }
                // keep live slots [0, r) other than i
                mu.keep_live(r, i); mv.keep_live(r, i); mw.keep_live(r, i);
                if constexpr (ZT) mwn.keep_live(r, i);
                const int nU = mu.count(), nV = mv.count(), nW = mw.count();
                const int K = 2 * (nU + nV + nW);
                if (K > 0) {
                    const int c = (int)__umulhi(x.y, (uint32_t)K);
                    rho = c & 1;
                    const int mi = c >> 1;
                    if constexpr (SlotBits<RMAX>::NW == 1) {
                        X = mi < nU ? 0 : (mi < nU + nV ? 1 : 2);
                        const int idx = mi - (X == 0 ? 0 : (X == 1 ? nU : nU + nV));
                        j = SlotBits<RMAX>::pick(X, mu, mv, mw).nth(idx);
                        sneg = (ZT && X == 2) ? (int)mwn.test(j) : 0;
                    } else {
                        if (mi < nU) { X = 0; j = mu.nth(mi); }
                        else if (mi < nU + nV) { X = 1; j = mv.nth(mi - nU); }
                        else { X = 2; j = mw.nth(mi - nU - nV); sneg = ZT ? (int)mwn.test(j) : 0; }
                    }
                    if constexpr (SL && ZT) {
                        const int Xn = X == 0 ? 1 : (X == 1 ? 2 : 0), Xnn = X == 0 ? 2 : (X == 1 ? 0 : 1);
                        const int Zf = rho ? Xn : Xnn;
                        fYZ = (rho ? Xnn : Xn) | (Zf << 2);
                        fmX = SlotBits<RMAX>::pick(X, mu, mv, mw).w[0];
                        fmZ = SlotBits<RMAX>::pick(Zf, mu, mv, mw).w[0];
                    }
                    apply_candidate(ti, i, X, j, sneg, rho, action, need_check, ti2, tj2);
                } else {
                    c_noc += 1;
                }
            }
            finish_step(d, wmask, lane, nl, bestp, x.z, x.w, r_before, action, X, rho, sneg, i, j, need_check, ti2,
                        tj2);
        }
        store(d, w);
    }
};

template <int MODE, class Wd, int RMAX, int BT, int FL = 0>
__host__ __device__ constexpr size_t solo_packed_bytes() {
    return (size_t)RMAX * (BT + 1) * ((MODE == TFG_MODE_ZT) ? 2 : 1) * sizeof(Wd);
}

template <int MODE, class Wd, int RMAX, int BT, int FL = 0, bool SQ = false>
__device__ __forceinline__ void walk_solo_body(const SegDesc &d, int32_t steps, unsigned char *smem_raw) {
    const int64_t w = (int64_t)blockIdx.x * BT + threadIdx.x;
    if (w >= d.n_walkers) return;   // no block-wide barrier is used
    SoloWalker<MODE, Wd, RMAX, BT, FL, SQ> wk;
    constexpr int NWS = (MODE == TFG_MODE_ZT) ? 2 : 1;
    wk.sm = reinterpret_cast<Wd *>(smem_raw) + (size_t)threadIdx.x * NWS;
    if constexpr (FL > 0 && MODE == TFG_MODE_ZT)
        wk.ss = reinterpret_cast<uint2 *>(smem_raw + ((solo_packed_bytes<MODE, Wd, RMAX, BT>() + 15) & ~(size_t)15)) +
                threadIdx.x;
    wk.run(d, w, steps);
}

template <int MODE, class Wd, int RMAX, int BT>
__global__ void __launch_bounds__(BT) walk_solo_kernel(const SegDesc d, const int32_t steps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    walk_solo_body<MODE, Wd, RMAX, BT>(d, steps, smem_raw);
}

// The same kernel with registers capped for four resident blocks per SM
// (measured faster for Z_T terms of one 32-bit word at capacity 32).
template <int MODE, class Wd, int RMAX, int BT>
__global__ void __launch_bounds__(BT, 4) walk_solo_kernel_occ4(const SegDesc d, const int32_t steps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    walk_solo_body<MODE, Wd, RMAX, BT>(d, steps, smem_raw);
}

// Bit-sliced variant (factors of at most FL coefficients, capacity 32).
#ifndef TFG_SLICED_ZT_MIN_BLOCKS
#define TFG_SLICED_ZT_MIN_BLOCKS 7
#endif
#ifndef TFG_SLICED_Z2_MIN_BLOCKS
#define TFG_SLICED_Z2_MIN_BLOCKS 4
#endif
template <int MODE, class Wd, int RMAX, int BT, int FL, bool SQ>
__global__ void __launch_bounds__(BT, MODE == TFG_MODE_ZT ? TFG_SLICED_ZT_MIN_BLOCKS : TFG_SLICED_Z2_MIN_BLOCKS)
    walk_solo_kernel_sliced(const SegDesc d, const int32_t steps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    walk_solo_body<MODE, Wd, RMAX, BT, FL, SQ>(d, steps, smem_raw);
}

template <int MODE, class Wd, int RMAX, int BT, int FL = 0, bool SQ = false>
constexpr auto solo_kernel() {
    if constexpr (FL > 0) return &walk_solo_kernel_sliced<MODE, Wd, RMAX, BT, FL, SQ>;
    else if constexpr (MODE == TFG_MODE_ZT && sizeof(Wd) == 4 && RMAX == 32) return &walk_solo_kernel_occ4<MODE, Wd, RMAX, BT>;
    else return &walk_solo_kernel<MODE, Wd, RMAX, BT>;
}

}  // namespace dev

template <int MODE, class Wd, int RMAX, int BT, int FL = 0>
constexpr size_t solo_smem_bytes() {
    const size_t packed = dev::solo_packed_bytes<MODE, Wd, RMAX, BT>();
    if constexpr (FL > 0 && MODE == TFG_MODE_ZT) return ((packed + 15) & ~(size_t)15) + (size_t)(3 * FL + 1) * BT * 8;
    else return packed;
}

template <int MODE, class Wd, int RMAX, int BT, int FL = 0, bool SQ = false>
void prepare_walk_solo() {
    static bool attr = [] {
        cudaFuncSetAttribute(dev::solo_kernel<MODE, Wd, RMAX, BT, FL, SQ>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)solo_smem_bytes<MODE, Wd, RMAX, BT, FL>());
        return true;
    }();
    (void)attr;
}

template <int MODE, class Wd, int RMAX, int BT, int FL = 0, bool SQ = false>
void launch_walk_solo(const SegDesc &d, int32_t steps, int grid, int /*block*/, cudaStream_t st) {
    prepare_walk_solo<MODE, Wd, RMAX, BT, FL, SQ>();
    dev::solo_kernel<MODE, Wd, RMAX, BT, FL, SQ>()<<<grid, BT, solo_smem_bytes<MODE, Wd, RMAX, BT, FL>(), st>>>(d, steps);
}

#define TFG_SOLO_VARIANT(MODE, WD, BITS, RMAX, BT) \
    WalkVariant{MODE, BITS, 1, 1, RMAX, BT, &launch_walk_solo<MODE, WD, RMAX, BT>, \
                reinterpret_cast<const void *>(dev::solo_kernel<MODE, WD, RMAX, BT>()), \
                &prepare_walk_solo<MODE, WD, RMAX, BT>}

// bit-sliced: formats whose factors have at most FL coefficients (SQ: exactly FL each)
#define TFG_SOLO_SLICED_VARIANT(MODE, WD, BITS, RMAX, BT, FL, SQ) \
    WalkVariant{MODE, BITS, 1, 1, RMAX, BT, &launch_walk_solo<MODE, WD, RMAX, BT, FL, SQ>, \
                reinterpret_cast<const void *>(dev::solo_kernel<MODE, WD, RMAX, BT, FL, SQ>()), \
                &prepare_walk_solo<MODE, WD, RMAX, BT, FL, SQ>, 0, FL, SQ ? 1 : 0}

}  // namespace tfg
