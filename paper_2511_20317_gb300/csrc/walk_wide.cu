// Wide-term flip-graph walk kernel for sm_103a: formats whose terms have more
// than 64 coefficients (m*n + n*p + p*m > 64), with factors of up to 128.
//
// Layout.  A term is factor-aligned: factor f (u, v, w) is words f*FW ..
// f*FW+FW-1 of the positive-coefficient words and the same words of the
// negative ones (Section 3.5.1's digits/signs masks, FW = 1 or 2 words of 64
// bits per factor and sign), so every operation of Section 3.5.2 works word
// by word and needs no mask.
//
// Mapping.  One warp per walker; lane l owns the slots k*32 + l (strided, so
// that runs of related terms spread over the lanes).  The walker's terms live
// in shared memory together with 32-bit signatures of each factor (hashes of
// u, v and of w up to sign, plus the sign of w).  The candidate search of
// try_flip (Algorithm 1) compares signatures only and verifies every
// signature hit against the full factor words, so the candidate list is
// exact; the chosen candidate is located in slot order by a walk over the
// per-pass ballots.  The reduction checks (Section 3.4.1) are filtered the
// same way.  All walker-uniform bookkeeping is replicated in every lane.
// The arithmetic of a flip, a merge or a plus transition works on one word
// per lane (lane q < 3*FW holds word q, of factor q / FW, of each term
// involved): additions, normalisation, signatures and stores are a handful of
// lane-parallel instructions and ballots; __syncwarp orders the shared-memory
// writes.
//
// Terms of large walkers (capacity >= 256 slots) stay in their HBM slots and
// only the signatures sit in shared memory (more walkers resident per SM).
//
// The step contract (draws, candidate order, flip, rejection, removal,
// normalisation, reduction cascade, best/plateau bookkeeping, plus
// transitions, trajectory digest) is the one of the lane-group and
// thread-per-walker kernels.
#include <cstdint>

#include "tfg_internal.h"
#include "pterm.cuh"

namespace tfg {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// FW 64-bit words per factor and sign: word h of factor f is word f*FW + h.
template <bool ZT, int FW>
struct FTerm {
    uint64_t p[3 * FW];
    uint64_t n[3 * FW];   // kept zero in Z_2
};

// x[q] for a runtime q, by selects (no local-memory indexing)
template <int N>
__device__ __forceinline__ uint64_t pick(const uint64_t (&x)[N], int q) {
    uint64_t v = x[0];
#pragma unroll
    for (int a = 1; a < N; ++a) v = (q == a) ? x[a] : v;
    return v;
}

// 32-bit signature of word h of one factor (p, n): a multiply-xor hash, upper
// half.  The signature of a factor is the XOR over its words.
__device__ __forceinline__ uint32_t fsig(uint64_t p, uint64_t n, int h) {
    const uint64_t k = h ? 0xC2B2AE3D27D4EB4Full : 0x9E3779B97F4A7C15ull;
    const uint64_t x = (p ^ (n * 0xD6E8FEB86659FD93ull)) * k;
    return (uint32_t)(x >> 32);
}

// GW: the term words stay in the walker's HBM slots (only the signatures are
// in shared memory), else they are staged in shared memory for the launch.
// PG: the walk policy is read from the descriptor (policies 1 and 2); without
// it the plateau policy is compiled in alone.
// FW: 64-bit words per factor (1: factors of at most 64 coefficients, 2: at most 128).
template <int MODE, bool GW, bool PG, int FW>
struct WideWalker {
    static_assert(FW == 1 || FW == 2, "one or two words per factor");
    static constexpr bool ZT = (MODE == TFG_MODE_ZT);
    __device__ __forceinline__ static int policy_of(const SegDesc &d) { return PG ? d.walk_policy : 0; }
    static constexpr int TW = 3 * FW;                          // words per sign
    static constexpr int NWG = ZT ? 2 * TW : TW;               // words per slot in HBM (p words [n words])
    static constexpr int NWS = ZT ? 2 * TW : (TW + 1) / 2 * 2; // words per slot in shared memory (16-byte rows)
    static constexpr unsigned FM = (1u << FW) - 1u;            // a factor's lanes / words in a ballot
    using T = FTerm<ZT, FW>;

    uint64_t *W;    // GW: HBM slots [R][NWG]; else shared [R][NWS]: Z_T (p_q n_q) pairs, Z_2 p words (padded)
    uint4 *SG;      // [32 * KM] signatures (u, v, w up to sign, sign of w)
    int lane, KM;
    int r, best_r, R;
    int64_t t, plateau, best_t;
    uint64_t dig;
    uint32_t wid, key0, key1;
    uint32_t c_acc, c_rej, c_noc, c_drp, c_mrg, c_pls, c_red;
    int qlen, q0, q1, q2;
    uint32_t nnz, best_nnz;   // non-zero coefficients of the live (walk policy 2) / best scheme

    // shared-memory word of HBM slot word g
    __device__ __forceinline__ static int smem_word(int g) { return ZT ? (g < TW ? 2 * g : 2 * (g - TW) + 1) : g; }

    // ---- full-term comparisons (hit verification)
    __device__ __forceinline__ static bool eq(const T &a, const T &b, int f) {
        bool e = true;
#pragma unroll
        for (int h = 0; h < FW; ++h) e = e && a.p[f * FW + h] == b.p[f * FW + h] && (!ZT || a.n[f * FW + h] == b.n[f * FW + h]);
        return e;
    }
    __device__ __forceinline__ static bool eqneg(const T &a, const T &b, int f) {
        bool e = ZT;
#pragma unroll
        for (int h = 0; h < FW; ++h) e = e && a.p[f * FW + h] == b.n[f * FW + h] && a.n[f * FW + h] == b.p[f * FW + h];
        return e;
    }
    __device__ __forceinline__ static bool sum_ok(const T &a, const T &b, int f, bool neg) {
        if constexpr (ZT) {
            uint64_t clash = 0ull;
#pragma unroll
            for (int h = 0; h < FW; ++h) {
                const int q = f * FW + h;
                const uint64_t bp = neg ? b.n[q] : b.p[q], bn = neg ? b.p[q] : b.n[q];
                clash |= (a.p[q] & bp) | (a.n[q] & bn);
            }
            return clash == 0ull;
        } else {
            return true;
        }
    }
    // the first non-zero coefficient of factor f is negative
    __device__ __forceinline__ static bool lead_neg(const T &a, int f) {
        bool ng = false;
#pragma unroll
        for (int h = FW - 1; h >= 0; --h) {
            const uint64_t d = a.p[f * FW + h] | a.n[f * FW + h];
            ng = d ? ((a.n[f * FW + h] & d & (0ull - d)) != 0ull) : ng;
        }
        return ng;
    }
    __device__ __forceinline__ static uint4 sig(const T &a) {
        uint4 s = make_uint4(0u, 0u, 0u, 0u);
        const bool ng = ZT && lead_neg(a, 2);
#pragma unroll
        for (int h = 0; h < FW; ++h) {
            s.x ^= fsig(a.p[h], a.n[h], h);
            s.y ^= fsig(a.p[FW + h], a.n[FW + h], h);
            const uint64_t wp = a.p[2 * FW + h], wn = a.n[2 * FW + h];
            s.z ^= fsig(ng ? wn : wp, ng ? wp : wn, h);
        }
        s.w = ng ? 1u : 0u;
        return s;
    }

    // ---- one word per lane: lane q < 3*FW holds word q (factor q / FW) of each
    // term involved; lanes 3*FW..31 mirror word 0 and never store
    struct DF { uint64_t p, n; };
    int fq;   // this lane's word (0 on lanes 3*FW..31)
    __device__ __forceinline__ bool owns(int f) const { return (lane >> (FW - 1)) == f; }   // holds a word of factor f
    __device__ __forceinline__ int fh() const { return FW == 1 ? 0 : lane & 1; }         // its word within the factor
    __device__ __forceinline__ bool fown() const { return lane < 3 * FW; }

    __device__ __forceinline__ DF dof(const T &a) const { return DF{pick(a.p, fq), pick(a.n, fq)}; }
    __device__ __forceinline__ DF dget(int s) const {
        if constexpr (GW) {
            return DF{W[(size_t)s * NWG + fq], ZT ? W[(size_t)s * NWG + TW + fq] : 0ull};
        } else if constexpr (ZT) {
            const ulonglong2 a = reinterpret_cast<const ulonglong2 *>(W + (size_t)s * NWS)[fq];
            return DF{a.x, a.y};
        } else {
            return DF{W[(size_t)s * NWS + fq], 0ull};
        }
    }
    // res = a with factor f := a_f + b_f (neg: a_f - b_f); false when a
    // coefficient leaves the coefficient set (Section 3.5.2)
    __device__ __forceinline__ bool dadd(const DF &a, const DF &b, int f, bool neg, DF &res) const {
        const bool me = owns(f);
        bool bad = false;
        if constexpr (ZT) {
            const uint64_t bp = neg ? b.n : b.p, bn = neg ? b.p : b.n;
            res.p = me ? ((a.p | bp) & ~(a.n | bn)) : a.p;
            res.n = me ? ((a.n | bn) & ~(a.p | bp)) : a.n;
            bad = me && ((a.p & bp) | (a.n & bn)) != 0ull;
        } else {
            res.p = me ? (a.p ^ b.p) : a.p;
            res.n = 0ull;
        }
        return !__any_sync(kFull, bad);
    }
    __device__ __forceinline__ bool dzero(const DF &a, int f) const {
        return ((__ballot_sync(kFull, (a.p | a.n) == 0ull) >> (f * FW)) & FM) == FM;
    }
    __device__ __forceinline__ void dtake(DF &dst, const DF &src, int f) const {
        if (owns(f)) dst = src;
    }
    // Sign flags of the leading coefficient of every factor: bit f*FW (of the
    // returned ballot) is set when factor f's first non-zero coefficient is negative.
    __device__ __forceinline__ unsigned dlead(const DF &a) const {
        const uint64_t d = a.p | a.n;
        const unsigned ng = __ballot_sync(kFull, (a.n & d & (0ull - d)) != 0ull);
        if constexpr (FW == 1) {
            return ng;
        } else {
            // a factor's second word decides only when its first word is zero
            const unsigned nz = __ballot_sync(kFull, d != 0ull);
            return (ng & nz & 0x15u) | ((ng >> 1) & ~nz & 0x15u);
        }
    }
    // Section 3.6: first non-zero of u, then of v, made +1; w absorbs the signs
    __device__ __forceinline__ void dcanon(DF &a) const {
        if constexpr (ZT) {
            const unsigned neg = dlead(a);
            const bool f0 = neg & 1u, f1 = (neg >> FW) & 1u;
            const bool sw = (owns(0) && f0) || (owns(1) && f1) || (owns(2) && f0 != f1);
            const uint64_t p = sw ? a.n : a.p, n = sw ? a.p : a.n;
            a.p = p; a.n = n;
        }
    }
    // non-zero coefficients of a term held one word per lane
    __device__ __forceinline__ uint32_t dnnz(const DF &a) const {
        const uint32_t c = fown() ? (uint32_t)__popcll(a.p | a.n) : 0u;
        return __reduce_add_sync(kFull, c);
    }
    // w of a equals -w of b
    __device__ __forceinline__ bool dwneg(const DF &a, const DF &b) const {
        return ZT && ((__ballot_sync(kFull, a.p == b.n && a.n == b.p) >> (2 * FW)) & FM) == FM;
    }
    __device__ __forceinline__ void dput(int s, const DF &a) {
        uint64_t cp = a.p, cn = a.n;
        uint32_t ng = 0u;
        if constexpr (ZT) {
            if constexpr (FW == 1) {
                const uint64_t d = a.p | a.n;
                ng = (lane == 2 && (a.n & d & (0ull - d)) != 0ull) ? 1u : 0u;   // read by lane 2 alone
            } else {
                ng = (dlead(a) >> (2 * FW)) & 1u;
            }
            if (ng && owns(2)) { cp = a.n; cn = a.p; }
        }
        uint32_t h = fsig(cp, cn, fh());
        if constexpr (FW == 2) h ^= __shfl_xor_sync(kFull, h, 1);   // the factor's two words
        if (fown()) {
            if constexpr (GW) {
                W[(size_t)s * NWG + lane] = a.p;
                if constexpr (ZT) W[(size_t)s * NWG + TW + lane] = a.n;
            } else if constexpr (ZT) {
                reinterpret_cast<ulonglong2 *>(W + (size_t)s * NWS)[lane] = make_ulonglong2(a.p, a.n);
            } else {
                W[(size_t)s * NWS + lane] = a.p;
            }
            if (fh() == 0) {
                uint32_t *g = reinterpret_cast<uint32_t *>(SG + s);
                g[lane >> (FW - 1)] = h;
                if (owns(2)) g[3] = ng;
            }
        }
        __syncwarp();
    }

    // ---- term slots
    __device__ __forceinline__ static void set_word(T &out, int g, uint64_t v) {
        if (g < TW) out.p[g] = v;
        else out.n[g - TW] = v;
    }
    __device__ __forceinline__ T get(int s) const {
        T out;
        if constexpr (!ZT) {
#pragma unroll
            for (int q = 0; q < TW; ++q) out.n[q] = 0ull;
        }
        if constexpr (GW) {
            const uint64_t *g = W + (size_t)s * NWG;
            if constexpr (NWG % 2 == 0) {
                const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(g);   // rows of 16-byte multiples
#pragma unroll
                for (int e = 0; e < NWG / 2; ++e) {
                    const ulonglong2 a = q[e];
                    set_word(out, 2 * e, a.x);
                    set_word(out, 2 * e + 1, a.y);
                }
            } else {
#pragma unroll
                for (int e = 0; e < NWG; ++e) set_word(out, e, g[e]);
            }
            return out;
        }
        const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(W + (size_t)s * NWS);
#pragma unroll
        for (int e = 0; e < NWS / 2; ++e) {
            const ulonglong2 a = src[e];
            if constexpr (ZT) {
                out.p[e] = a.x; out.n[e] = a.y;
            } else {
                out.p[2 * e] = a.x;
                if (2 * e + 1 < TW) out.p[2 * e + 1] = a.y;
            }
        }
        return out;
    }
    // factor f of slot s equals factor f of a (wneg: or its negation)
    __device__ __forceinline__ bool fmatch(int s, int f, const T &a, bool wneg) const {
        bool ep = true, en = ZT && wneg;
#pragma unroll
        for (int h = 0; h < FW; ++h) {
            const int q = f * FW + h;
            uint64_t p, n;
            if constexpr (GW) {
                p = W[(size_t)s * NWG + q];
                n = ZT ? W[(size_t)s * NWG + TW + q] : 0ull;
            } else if constexpr (ZT) {
                const ulonglong2 x = reinterpret_cast<const ulonglong2 *>(W + (size_t)s * NWS)[q];
                p = x.x; n = x.y;
            } else {
                p = W[(size_t)s * NWS + q];
                n = 0ull;
            }
            ep = ep && p == a.p[q] && n == a.n[q];
            en = en && p == a.n[q] && n == a.p[q];
        }
        return ep || en;
    }
    __device__ __forceinline__ void move(int from, int to) {
        if constexpr (GW) {
            if (lane < NWG) W[(size_t)to * NWG + lane] = W[(size_t)from * NWG + lane];
            else if (lane == NWG) SG[to] = SG[from];
            __syncwarp();
            return;
        }
        if (lane < NWS / 2) {
            const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(W + (size_t)from * NWS);
            ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(W + (size_t)to * NWS);
            dst[lane] = src[lane];
        } else if (lane == NWS / 2) {
            SG[to] = SG[from];
        }
        __syncwarp();
    }

    // ---- reduction queue (slot indices), walker-uniform
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
            move(last, h);
            q_rename(last, h);
        }
        r -= 1;
    }

    // Does any other live slot share two factors (signatures) with the terms
    // in slots sa or sb?  A superset of the reduction test: the cascade that
    // follows a positive answer checks exactly.
    __device__ __forceinline__ bool pair_filter(int sa, int sb) const {
        const uint4 A = SG[sa], B = SG[sb];
        bool hit = false;
#pragma unroll 4
        for (int k = 0; k < KM; ++k) {
            const int s = (k << 5) + lane;
            const uint4 g = SG[s];
            const int ma = (int)(g.x == A.x) + (int)(g.y == A.y) + (int)(g.z == A.z);
            const int mb = (int)(g.x == B.x) + (int)(g.y == B.y) + (int)(g.z == B.z);
            hit |= s < r && ((s != sa && ma >= 2) || (s != sb && mb >= 2));
        }
        return __any_sync(kFull, hit);
    }

    // Reduction of the term in slot s with the lowest slot sharing (u,v), else
    // (u,w), else (v,w), whose merged third factor stays ternary; the merged
    // term keeps s's pair factors and goes to the lower slot.
    __device__ __forceinline__ void reduce_one(int s) {
        const T v = get(s);
        const uint4 vs = SG[s];
        uint32_t c0 = 0, c1 = 0, c2 = 0;   // bit k: slot k*32 + lane shares the pair by signature
#pragma unroll 4
        for (int k = 0; k < KM; ++k) {
            const int slot = (k << 5) + lane;
            const uint4 g = SG[slot];
            const bool live = slot < r && slot != s;
            const bool eu = g.x == vs.x, ev = g.y == vs.y, ew = g.z == vs.z;
            c0 |= (uint32_t)(live && eu && ev) << k;
            c1 |= (uint32_t)(live && eu && ew) << k;
            c2 |= (uint32_t)(live && ev && ew) << k;
        }
        uint32_t m0 = 0, m1 = 0, m2 = 0;   // verified, with a ternary merged third factor
        uint32_t any = c0 | c1 | c2;
#pragma unroll 1
        while (any) {
            const int k = __ffs(any) - 1;
            any &= any - 1u;
            const uint32_t bit = 1u << k;
            const T u = get((k << 5) + lane);
            const bool xu = eq(u, v, 0), xv = eq(u, v, 1), xwp = eq(u, v, 2), xwn = eqneg(u, v, 2);
            if ((c0 & bit) && xu && xv && sum_ok(v, u, 2, false)) m0 |= bit;
            if ((c1 & bit) && xu && (xwp || xwn) && sum_ok(v, u, 1, xwn)) m1 |= bit;
            if ((c2 & bit) && xv && (xwp || xwn) && sum_ok(v, u, 0, xwn)) m2 |= bit;
        }
        const unsigned b0 = __ballot_sync(kFull, m0 != 0u), b1 = __ballot_sync(kFull, m1 != 0u),
                       b2 = __ballot_sync(kFull, m2 != 0u);
        if ((b0 | b1 | b2) == 0u) return;
        const int P = b0 ? 0 : (b1 ? 1 : 2);
        const uint32_t mp = P == 0 ? m0 : (P == 1 ? m1 : m2);
        // lowest slot (k*32 + lane) with a partner of pair type P
        const unsigned mine = mp ? (unsigned)(((__ffs(mp) - 1) << 5) + lane) : 0xffffffffu;
        const int k = (int)__reduce_min_sync(kFull, mine);
        const DF dv = dof(v), dk = dget(k);
        const bool kneg = (P != 0) && dwneg(dk, dv);
        const int F = 2 - P;   // third factor: w, v, u
        DF mv;
        dadd(dv, dk, F, kneg, mv);
        const bool z = dzero(mv, F);
        dcanon(mv);
        const int lo = s < k ? s : k;
        const int hi = s < k ? k : s;
        q_remove(k);
        dput(lo, mv);
        c_mrg += 1;
        drop(hi);
        if (z) {
            drop(lo);
            c_drp += 1;
        } else {
            q_push(lo);
        }
    }

    __device__ __forceinline__ void cascade() {
#pragma unroll 1
        while (qlen > 0) reduce_one(q_pop());
    }

    __device__ __forceinline__ void snapshot(uint64_t *bestp) const {
#pragma unroll 1
        for (int e = lane; e < r * NWG; e += 32) {
            if constexpr (GW) {
                bestp[e] = W[e];
            } else {
                const int s = e / NWG, g = e - s * NWG;
                bestp[e] = W[(size_t)s * NWS + smem_word(g)];
            }
        }
    }

    // Expansion (Section 3.3.1): plus (three new terms), or split under walk policy 1
    // when y3 >= 2^31; the changed terms are queued for the cascade;
    // returns the digest record (0 when no attempt passed).
    __device__ __forceinline__ uint64_t plus_setup(const SegDesc &d) {
#pragma unroll 1
        for (int a = 1; a <= d.plus_attempts; ++a) {
            const U4 y = philox10((uint32_t)t, (uint32_t)(t >> 32), wid, (uint32_t)a, key0, key1);
            const int pi = (int)__umulhi(y.x, (uint32_t)r);
            const int pj = (pi + 1 + (int)__umulhi(y.y, (uint32_t)(r - 1))) % r;
            const int perm = (int)__umulhi(y.z, 6u);
            int A, B, C;
            plus_roles(perm, A, B, C);
            const DF ti = dget(pi), tj = dget(pj);
            if (policy_of(d) == 1 && y.w >= 0x80000000u) {
                // split: term i = (A_j, B_i, C_i), new term (A_i - A_j, B_i, C_i)
                DF ns;
                const bool ok = dadd(ti, tj, A, true, ns);
                const bool z = dzero(ns, A);
                if (!ok || z) continue;
                dcanon(ns);
                dput(r, ns);
                DF ti2 = ti;
                dtake(ti2, tj, A);
                dcanon(ti2);
                dput(pi, ti2);
                r += 1;
                plateau = 0;
                c_pls += 1;
                qlen = 0;
                q_push(pi);
                q_push(r - 1);
                return plus_record(a, perm, pi, pj, 1);
            }
            DF nb, nc, na;
            bool ok = dadd(ti, tj, B, false, nb);   // B_i + B_j
            ok &= dadd(tj, ti, C, true, nc);        // C_j - C_i
            ok &= dadd(tj, ti, A, true, na);        // A_j - A_i
            const bool z = dzero(nb, B) || dzero(nc, C) || dzero(na, A);
            if (!ok || z) continue;
            dcanon(na);                // (A_j - A_i, B_j, C_j)
            dput(r, na);
            dtake(nc, ti, A);          // (A_i, B_j, C_j - C_i)
            dcanon(nc);
            dput(pj, nc);
            dcanon(nb);                // (A_i, B_i + B_j, C_i)
            dput(pi, nb);
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

    __device__ __forceinline__ void run(const SegDesc &d, int64_t w, int32_t steps, unsigned char *sm) {
        lane = threadIdx.x & 31;
        fq = lane < 3 * FW ? lane : 0;
        R = d.R;
        KM = (R + 31) >> 5;
        if constexpr (GW) {
            W = reinterpret_cast<uint64_t *>(d.slots) + (size_t)w * R * NWG;
            SG = reinterpret_cast<uint4 *>(sm);
        } else {
            W = reinterpret_cast<uint64_t *>(sm);
            SG = reinterpret_cast<uint4 *>(W + (size_t)R * NWS);
        }
        tfg_walker_info *H = d.hdr + w;
        r = H->r; best_r = H->best_r;
        t = H->t; plateau = H->plateau; best_t = H->best_t;
        dig = H->digest; wid = H->walker_id;
        key0 = d.key0; key1 = d.key1;
        best_nnz = H->best_nnz;
        c_acc = c_rej = c_noc = c_drp = c_mrg = c_pls = c_red = 0;
        qlen = 0; q0 = q1 = q2 = 0;
        const uint64_t *src = reinterpret_cast<const uint64_t *>(d.slots) + (size_t)w * R * NWG;
        uint64_t *bestp = reinterpret_cast<uint64_t *>(d.best) + (size_t)w * R * NWG;
        if constexpr (!GW) {
            // HBM rows (p0 p1 p2 [n0 n1 n2]) -> shared rows grouped by factor
#pragma unroll 1
            for (int e = lane; e < R * NWS; e += 32) {
                const int s = e / NWS, q = e - s * NWS;
                const int g = ZT ? ((q & 1) ? TW + (q >> 1) : (q >> 1)) : q;   // source word of shared word q
                W[e] = g < NWG ? src[(size_t)s * NWG + g] : 0ull;
            }
            __syncwarp();
        }
#pragma unroll 1
        for (int s = lane; s < 32 * KM; s += 32) SG[s] = s < R ? sig(get(s)) : make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        nnz = 0;
        if (policy_of(d) == 2) {
            uint32_t mine = 0;
#pragma unroll 1
            for (int s = lane; s < r; s += 32) {
                const T v = get(s);
                for (int x = 0; x < TW; ++x) mine += (uint32_t)__popcll(v.p[x] | v.n[x]);
            }
            nnz = __reduce_add_sync(kFull, mine);
        }

        uint32_t xr0 = 0, xr1 = 0, xr2 = 0, xr3 = 0;
        int kb = 32;
#pragma unroll 1
        for (int32_t step = 0; step < steps; ++step) {
            // ---- draw: lane l holds the Philox output of step (batch start + l)
            if (kb == 32) {
                const uint64_t tl = (uint64_t)t + (uint64_t)lane;
                const U4 x = philox10((uint32_t)tl, (uint32_t)(tl >> 32), wid, 0u, key0, key1);
                xr0 = x.x; xr1 = x.y; xr2 = x.z; xr3 = x.w;
                kb = 0;
            }
            const uint32_t x0 = __shfl_sync(kFull, xr0, kb), x1 = __shfl_sync(kFull, xr1, kb),
                           x2 = __shfl_sync(kFull, xr2, kb), x3 = PG ? __shfl_sync(kFull, xr3, kb) : 0u;
            kb += 1;

            const int r_before = r;
            const int i = (int)__umulhi(x0, (uint32_t)r);
            int action = kNoCand, X = 0, j = 0, rho = 0, sneg = 0;
            {
                const T ti = get(i);
                const uint4 si = SG[i];
                // ---- try_flip: candidates (X, j) with X_j = +-X_i, ordered (X, slot)
                uint32_t bu = 0, bv = 0, bw = 0;   // bit k: slot k*32 + lane is a candidate
#pragma unroll 4
                for (int k = 0; k < KM; ++k) {
                    const int s = (k << 5) + lane;
                    const uint4 g = SG[s];
                    const bool live = s < r && s != i;
                    bu |= (uint32_t)(live && g.x == si.x) << k;
                    bv |= (uint32_t)(live && g.y == si.y) << k;
                    bw |= (uint32_t)(live && g.z == si.z) << k;
                }
                uint32_t any = bu | bv | bw;   // signature hits: verify on the full words
#pragma unroll 1
                while (any) {
                    const int k = __ffs(any) - 1;
                    any &= any - 1u;
                    const uint32_t bit = 1u << k;
                    const int s = (k << 5) + lane;
                    if ((bu & bit) && !fmatch(s, 0, ti, false)) bu &= ~bit;
                    if ((bv & bit) && !fmatch(s, 1, ti, false)) bv &= ~bit;
                    if ((bw & bit) && !fmatch(s, 2, ti, true)) bw &= ~bit;
                }
                const uint32_t tot = __reduce_add_sync(kFull, (uint32_t)__popc(bu) | ((uint32_t)__popc(bv) << 10) |
                                                                  ((uint32_t)__popc(bw) << 20));
                const int nU = (int)(tot & 1023u), nV = (int)((tot >> 10) & 1023u), nW = (int)(tot >> 20);
                const int K = 2 * (nU + nV + nW);

                if (K > 0) {
                    const int c = (int)__umulhi(x1, (uint32_t)K);
                    rho = c & 1;
                    const int mi = c >> 1;
                    int idx;
                    if (mi < nU) { X = 0; idx = mi; }
                    else if (mi < nU + nV) { X = 1; idx = mi - nU; }
                    else { X = 2; idx = mi - nU - nV; }
                    // the idx-th candidate of factor X in slot order (k, then lane)
                    const uint32_t mk = X == 0 ? bu : (X == 1 ? bv : bw);
                    int k = 0;
                    unsigned b = __ballot_sync(kFull, mk & 1u);
#pragma unroll 1
                    for (; k + 1 < KM; ) {
                        const int cnt = __popc(b);
                        if (idx < cnt) break;
                        idx -= cnt;
                        ++k;
                        b = __ballot_sync(kFull, (mk >> k) & 1u);
                    }
#pragma unroll 1
                    for (int q = 0; q < idx && b; ++q) b &= b - 1u;
                    j = (k << 5) + __ffs(b) - 1;
                    const DF di = dof(ti), dj = dget(j);
                    sneg = (X == 2 && dwneg(dj, di)) ? 1 : 0;

                    // flip: (Y, Z) cyclic after X, rho swaps; Y_i += Y_j, Z_j -= s Z_i
                    int Y = X == 0 ? 1 : (X == 1 ? 2 : 0);
                    int Z = X == 0 ? 2 : (X == 1 ? 0 : 1);
                    if (rho) { const int tmp = Y; Y = Z; Z = tmp; }
                    DF ti2, tj2;
                    bool ok = dadd(di, dj, Y, false, ti2);
                    ok &= dadd(dj, di, Z, sneg == 0, tj2);
                    if (!ok) {
                        action = kReject;
                        c_rej += 1;
                    } else {
                        action = kAccept;
                        c_acc += 1;
                        const bool zi = dzero(ti2, Y);
                        const bool zj = dzero(tj2, Z);
                        if (policy_of(d) == 2)
                            nnz += (zi ? 0u : dnnz(ti2)) + (zj ? 0u : dnnz(tj2)) - dnnz(di) - dnnz(dj);
                        dcanon(ti2);
                        dcanon(tj2);
                        dput(i, ti2);
                        dput(j, tj2);
                        qlen = 0;
                        if (zi || zj) {
                            q_push(i);
                            q_push(j);
                            const int hi = i > j ? i : j, lo = i > j ? j : i;
                            const bool zhi = (hi == i) ? zi : zj, zlo = (lo == i) ? zi : zj;
                            if (zhi) { drop(hi); c_drp += 1; }
                            if (zlo) { drop(lo); c_drp += 1; }
                            if (policy_of(d) == 2) qlen = 0;   // no reduction edges
                        } else if (policy_of(d) != 2 && pair_filter(i, j)) {
                            q_push(i);
                            q_push(j);
                        }
                    }
                } else {
                    c_noc += 1;
                }
            }

            // ---- reduction cascade (flip), then bookkeeping, then plus + cascade
            bool plus_phase = false;
            uint64_t rec2 = 0;
#pragma unroll 1
            for (;;) {
                cascade();
                if (plus_phase) {
                    dig = digest_mix(dig, rec2 | ((uint64_t)(uint32_t)r << 44));
                    break;
                }
                if (r < r_before) c_red += 1;
                dig = digest_mix(dig, flip_record(action, X, rho, sneg, i, j, r));
                // walk policy 1: a failed try_flip expands and ends the step (no best update)
                const bool failed = policy_of(d) == 1 && action != kAccept;
                // best scheme: always when better, with probability 0.01 when equal
                // (policy 2: better = least (rank, non-zero coefficients))
                if (policy_of(d) == 2) {
                    if (r < best_r || (r == best_r && nnz < best_nnz)) {
                        snapshot(bestp);
                        best_r = r;
                        best_nnz = nnz;
                        best_t = t;
                        plateau = 0;
                    } else {
                        if (r == best_r && nnz == best_nnz && x2 < d.refresh_thresh) snapshot(bestp);
                        plateau += 1;
                    }
                } else if (failed) {
                    plateau += 1;
                } else if (r < best_r) {
                    snapshot(bestp);
                    best_r = r;
                    best_t = t;
                    plateau = 0;
                } else {
                    if (r == best_r && x2 < d.refresh_thresh) snapshot(bestp);
                    plateau += 1;
                }
                // expansion: plus on a plateau near the best rank (policy 0), or Algorithm 1's
                // expand after a failed try_flip / with probability p_expand (policy 1)
                bool expand;
                if (policy_of(d) == 2)
                    expand = false;
                else if (policy_of(d) == 1)
                    expand = failed ? (r < R && r >= 2) : (x3 < d.expand_thresh && r <= best_r + 2 && r < R && r >= 2);
                else
                    expand = d.plus_enabled && plateau >= d.plateau_len && r <= best_r + 2 && r < R && r >= 2;
                if (expand) {
                    rec2 = plus_setup(d);
                    if (rec2) { plus_phase = true; continue; }
                }
                break;
            }
            t += 1;
        }

        // ---- write back
        uint64_t *dst = reinterpret_cast<uint64_t *>(d.slots) + (size_t)w * R * NWG;
        if constexpr (!GW) {
#pragma unroll 1
            for (int e = lane; e < R * NWG; e += 32) {
                const int s = e / NWG, g = e - s * NWG;
                dst[e] = W[(size_t)s * NWS + smem_word(g)];
            }
        }
        if (lane == 0) {
            H->r = r; H->best_r = best_r;
            H->t = t; H->plateau = plateau; H->best_t = best_t;
            H->digest = dig;
            H->accepted += c_acc; H->rejected += c_rej; H->nocand += c_noc;
            H->drops += c_drp; H->merges += c_mrg; H->plus += c_pls; H->reductions += c_red;
            H->best_nnz = best_nnz;
        }
    }
};

template <int MODE, bool GW, int FW>
__host__ __device__ constexpr size_t wide_walker_bytes(int R) {
    return (GW ? (size_t)0 : (size_t)R * WideWalker<MODE, GW, false, FW>::NWS * 8) + (size_t)((R + 31) / 32) * 32 * 16;
}

constexpr int kWideWarps = 2;   // walkers (warps) per block

// With the term words in HBM, registers bound residency: capped for 16
// two-warp blocks per SM with one word per factor (measured +4-8% on ranks 285
// and 351), 8 with two.
template <int MODE, bool GW, bool PG, int FW>
__global__ void __launch_bounds__(32 * kWideWarps, GW ? 16 / FW : 1) walk_wide_kernel(const SegDesc d, const int32_t steps) {
    extern __shared__ __align__(16) unsigned char wide_sm[];
    const int warp = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * kWideWarps + warp;
    if (w >= d.n_walkers) return;   // whole warps exit together
    WideWalker<MODE, GW, PG, FW> wk;
    wk.run(d, w, steps, wide_sm + wide_walker_bytes<MODE, GW, FW>(d.R) * warp);
}

}  // namespace dev

namespace {

constexpr int kWideMaxSmem = 227 * 1024;

// Term words stay in HBM from this capacity on: shared-memory residency (22.8 KB
// per walker at 354 slots) limits the larger ranks.  Measured on 16384 walkers:
// rank 202 (capacity 205) 1.00e9 shared vs 0.98e9 HBM steps/s; rank 285: 0.69e9 vs
// 0.85e9; rank 351: 0.46e9 vs 0.73e9.  Two words per factor double the bytes per
// slot, so the switch comes at half the capacity.
template <int FW>
constexpr int wide_hbm_words_min_r() { return 256 / FW; }

template <int MODE, int FW>
void prepare_walk_wide() {
    static bool attr = [] {
        cudaFuncSetAttribute(dev::walk_wide_kernel<MODE, false, false, FW>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWideMaxSmem);
        cudaFuncSetAttribute(dev::walk_wide_kernel<MODE, true, false, FW>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWideMaxSmem);
        cudaFuncSetAttribute(dev::walk_wide_kernel<MODE, false, true, FW>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWideMaxSmem);
        cudaFuncSetAttribute(dev::walk_wide_kernel<MODE, true, true, FW>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWideMaxSmem);
        return true;
    }();
    (void)attr;
}

template <int MODE, bool GW, int FW>
void launch_wide_as(const SegDesc &d, int32_t steps, cudaStream_t st) {
    const size_t smem = dev::wide_walker_bytes<MODE, GW, FW>(d.R) * dev::kWideWarps;
    if (d.n_walkers <= 0 || smem > (size_t)kWideMaxSmem) return;
    const int64_t grid = (d.n_walkers + dev::kWideWarps - 1) / dev::kWideWarps;
    if (d.walk_policy == 0)
        dev::walk_wide_kernel<MODE, GW, false, FW><<<(unsigned)grid, 32 * dev::kWideWarps, smem, st>>>(d, steps);
    else
        dev::walk_wide_kernel<MODE, GW, true, FW><<<(unsigned)grid, 32 * dev::kWideWarps, smem, st>>>(d, steps);
}

template <int MODE, int FW>
void launch_walk_wide(const SegDesc &d, int32_t steps, int /*grid*/, int /*block*/, cudaStream_t st) {
    prepare_walk_wide<MODE, FW>();
    if (d.R >= wide_hbm_words_min_r<FW>()) launch_wide_as<MODE, true, FW>(d, steps, st);
    else launch_wide_as<MODE, false, FW>(d, steps, st);
}

}  // namespace

// Factor-aligned terms: 3 (factors of at most 64 coefficients) or 6 (at most
// 128) words of 64 bits per sign; capacity 1023 slots (the shared-memory need
// of two walkers per block stays under 227 KB).
const WalkVariant *walk_variants_wide(int *n) {
    static const WalkVariant v[] = {
        WalkVariant{TFG_MODE_ZT, 64, 3, 32, 0, 0, &launch_walk_wide<TFG_MODE_ZT, 1>,
                    reinterpret_cast<const void *>(&dev::walk_wide_kernel<TFG_MODE_ZT, true, false, 1>),
                    &prepare_walk_wide<TFG_MODE_ZT, 1>, 1023},
        WalkVariant{TFG_MODE_Z2, 64, 3, 32, 0, 0, &launch_walk_wide<TFG_MODE_Z2, 1>,
                    reinterpret_cast<const void *>(&dev::walk_wide_kernel<TFG_MODE_Z2, true, false, 1>),
                    &prepare_walk_wide<TFG_MODE_Z2, 1>, 1023},
        WalkVariant{TFG_MODE_ZT, 64, 6, 32, 0, 0, &launch_walk_wide<TFG_MODE_ZT, 2>,
                    reinterpret_cast<const void *>(&dev::walk_wide_kernel<TFG_MODE_ZT, true, false, 2>),
                    &prepare_walk_wide<TFG_MODE_ZT, 2>, 1023},
        WalkVariant{TFG_MODE_Z2, 64, 6, 32, 0, 0, &launch_walk_wide<TFG_MODE_Z2, 2>,
                    reinterpret_cast<const void *>(&dev::walk_wide_kernel<TFG_MODE_Z2, true, false, 2>),
                    &prepare_walk_wide<TFG_MODE_Z2, 2>, 1023},
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

}  // namespace tfg
