// Flip-graph walk kernel for sm_103a.
//
// One walker = one group of G lanes (G in {4, 8, 16, 32}); lane l of the group
// holds slots l*S .. l*S+S-1 of the walker's scheme in registers (blocked
// layout, S compile-time).  A term is NWT words: the positive and negative
// bit masks of u, v, w in Z_T ("digits"/"signs" of Section 3.5.1, stored as
// pos = digits & ~signs, neg = digits & signs), or the three masks of Z_2.
// Word bit e is coefficient e of the factor (u: i*n+k, v: k*p+j, w: j*m+i).
//
// Every step follows Algorithm 1 with the plateau policy:
//   draw (Philox4x32-10, counter (t, walker, 0)) -> sample term i ->
//   candidate search over all slots with group ballots (try_flip) ->
//   uniform choice -> flip with the ternary validity test of Section 3.5.2 ->
//   zero-term removal -> sign normalisation (Section 3.6) -> reduction
//   cascade ("flip with reduction edge checking", Section 3.4.1) ->
//   best / plateau bookkeeping (1% equal-rank refresh) -> plus transition.
// The step contract (candidate order, slot compaction, cascade order) is the
// one of the CPU reference; every branch is data-dependent integer logic, no
// floating point is involved.
#pragma once
#include <cstdint>

#include "tfg_internal.h"

namespace tfg {
namespace dev {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, Weyl key schedule.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int rd = 0; rd < 10; ++rd) {
        if (rd > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ uint64_t digest_mix(uint64_t h, uint64_t v) {
    h ^= v;
    h *= 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    return h;
}

// ---------------------------------------------------------------------------
// Lane group of G lanes inside a warp.
// ---------------------------------------------------------------------------
template <int G>
struct Group {
    unsigned mask;
    int lane;    // 0..G-1
    int base;    // first warp lane of the group
    __device__ __forceinline__ Group() {
        const int wl = threadIdx.x & 31;
        lane = wl & (G - 1);
        base = wl & ~(G - 1);
        mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
    }
    template <class T>
    __device__ __forceinline__ T shfl(T v, int src) const { return __shfl_sync(mask, v, src, G); }
    __device__ __forceinline__ unsigned ballot(bool pr) const {
        const unsigned b = __ballot_sync(mask, pr);
        return (G == 32) ? b : ((b >> base) & ((1u << G) - 1u));
    }
};

template <class Wd, int NWT>
struct Term { Wd w[NWT]; };

// ---- factor access (f is group-uniform; selects keep the term in registers)
template <class Wd, int NWT>
__device__ __forceinline__ Wd fpos(const Term<Wd, NWT> &t, int f) {
    constexpr int st = NWT / 3;
    return f == 0 ? t.w[0] : (f == 1 ? t.w[st] : t.w[2 * st]);
}
template <class Wd, int NWT>
__device__ __forceinline__ Wd fneg(const Term<Wd, NWT> &t, int f) {
    if constexpr (NWT == 6) return f == 0 ? t.w[1] : (f == 1 ? t.w[3] : t.w[5]);
    else return Wd(0);
}
template <class Wd, int NWT>
__device__ __forceinline__ void fset(Term<Wd, NWT> &t, int f, Wd p, Wd n) {
    constexpr int st = NWT / 3;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (f == q) {
            t.w[q * st] = p;
            if constexpr (NWT == 6) t.w[q * st + 1] = n;
        }
    }
}

// Section 3.6: first non-zero of u, then of v, made +1; w absorbs the sign.
template <class Wd, int NWT>
__device__ __forceinline__ void canon(Term<Wd, NWT> &t) {
    if constexpr (NWT == 6) {
        {
            const Wd d = t.w[0] | t.w[1];
            const Wd low = d & (Wd(0) - d);
            if (t.w[1] & low) {
                Wd a = t.w[0]; t.w[0] = t.w[1]; t.w[1] = a;
                a = t.w[4]; t.w[4] = t.w[5]; t.w[5] = a;
            }
        }
        {
            const Wd d = t.w[2] | t.w[3];
            const Wd low = d & (Wd(0) - d);
            if (t.w[3] & low) {
                Wd a = t.w[2]; t.w[2] = t.w[3]; t.w[3] = a;
                a = t.w[4]; t.w[4] = t.w[5]; t.w[5] = a;
            }
        }
    }
}

// Ternary a + b (Section 3.5.2 validity: no position with both +1 or both -1).
template <class Wd>
__device__ __forceinline__ bool tadd(Wd ap, Wd an, Wd bp, Wd bn, Wd &rp, Wd &rn) {
    const bool bad = ((ap & bp) | (an & bn)) != Wd(0);
    rp = (ap | bp) & ~(an | bn);
    rn = (an | bn) & ~(ap | bp);
    return !bad;
}

// ---------------------------------------------------------------------------
// Walker: state in registers plus the group-uniform bookkeeping.
// ---------------------------------------------------------------------------
template <int MODE, class Wd, int G, int S>
struct Walker {
    static constexpr bool ZT = (MODE == TFG_MODE_ZT);
    static constexpr int NWT = ZT ? 6 : 3;
    using T = Term<Wd, NWT>;

    Group<G> g;
    Wd st[S][NWT];
    int r, best_r, R;
    int64_t t, plateau, best_t;
    uint64_t dig;
    uint32_t wid, key0, key1;
    uint32_t c_acc, c_rej, c_noc, c_drp, c_mrg, c_pls, c_red;

    // Reduction queue: slots of at most three modified terms awaiting checks.
    int qlen, q0, q1, q2;

    __device__ __forceinline__ T fetch(int k) const {
        const int o = k / S, pos = k - o * S;
        T out;
#pragma unroll
        for (int w = 0; w < NWT; ++w) {
            Wd v = st[0][w];
#pragma unroll
            for (int p = 1; p < S; ++p) v = (pos == p) ? st[p][w] : v;
            out.w[w] = g.shfl(v, o);
        }
        return out;
    }

    __device__ __forceinline__ void store(const T &v, int k) {
        const int o = k / S, pos = k - o * S;
        const bool me = (g.lane == o);
#pragma unroll
        for (int p = 0; p < S; ++p) {
            if (me && pos == p) {
#pragma unroll
                for (int w = 0; w < NWT; ++w) st[p][w] = v.w[w];
            }
        }
    }

    // ---- queue helpers (registers only)
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
            const T lv = fetch(last);
            store(lv, h);
            q_rename(last, h);
        }
        r -= 1;
    }

    // Does term v (in slot s) share any factor pair with another live slot?
    // (superset filter of the reduction test; no validity check)
    __device__ __forceinline__ bool pair_hit(const T &v, int s) const {
        bool hit = false;
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
            const bool live = slot < r && slot != s;
            bool eu, ev, ew;
            if constexpr (ZT) {
                eu = st[p][0] == v.w[0] && st[p][1] == v.w[1];
                ev = st[p][2] == v.w[2] && st[p][3] == v.w[3];
                ew = (st[p][4] == v.w[4] && st[p][5] == v.w[5]) || (st[p][4] == v.w[5] && st[p][5] == v.w[4]);
            } else {
                eu = st[p][0] == v.w[0];
                ev = st[p][1] == v.w[1];
                ew = st[p][2] == v.w[2];
            }
            hit |= live && ((eu && ev) || (eu && ew) || (ev && ew));
        }
        return g.ballot(hit) != 0u;
    }

    // Reduction (Section 3.3.1, any permutation of u, v, w) of the term in slot
    // s with the lowest slot sharing the pair (u,v), else (u,w), else (v,w),
    // whose merged third factor stays ternary.  The merged term keeps s's pair
    // factors and goes to the lower of the two slots.
    __device__ __forceinline__ void reduce_one(int s) {
        const T v = fetch(s);
        uint32_t m0 = 0, m1 = 0, m2 = 0, mn = 0;
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
            const bool live = slot < r && slot != s;
            if constexpr (ZT) {
                // u and v are sign-normalised, so they match only exactly; w up to sign
                const bool eu = st[p][0] == v.w[0] && st[p][1] == v.w[1];
                const bool ev = st[p][2] == v.w[2] && st[p][3] == v.w[3];
                const bool ewp = st[p][4] == v.w[4] && st[p][5] == v.w[5];
                const bool ewn = st[p][4] == v.w[5] && st[p][5] == v.w[4];
                // third-factor validity: w_s + w_k ; v_s + sigma v_k ; u_s + sigma u_k
                const bool vw = ((v.w[4] & st[p][4]) | (v.w[5] & st[p][5])) == Wd(0);
                const Wd kvp = ewn ? st[p][3] : st[p][2], kvn = ewn ? st[p][2] : st[p][3];
                const bool vv = ((v.w[2] & kvp) | (v.w[3] & kvn)) == Wd(0);
                const Wd kup = ewn ? st[p][1] : st[p][0], kun = ewn ? st[p][0] : st[p][1];
                const bool vu = ((v.w[0] & kup) | (v.w[1] & kun)) == Wd(0);
                m0 |= (uint32_t)(live && eu && ev && vw) << p;
                m1 |= (uint32_t)(live && eu && (ewp || ewn) && vv) << p;
                m2 |= (uint32_t)(live && ev && (ewp || ewn) && vu) << p;
                mn |= (uint32_t)ewn << p;
            } else {
                const bool eu = st[p][0] == v.w[0], ev = st[p][1] == v.w[1], ew = st[p][2] == v.w[2];
                m0 |= (uint32_t)(live && eu && ev) << p;
                m1 |= (uint32_t)(live && eu && ew) << p;
                m2 |= (uint32_t)(live && ev && ew) << p;
            }
        }
        const unsigned b0 = g.ballot(m0 != 0u), b1 = g.ballot(m1 != 0u), b2 = g.ballot(m2 != 0u);
        if ((b0 | b1 | b2) == 0u) return;
        const int P = b0 ? 0 : (b1 ? 1 : 2);
        const unsigned lanes = b0 ? b0 : (b1 ? b1 : b2);
        const uint32_t mk = P == 0 ? m0 : (P == 1 ? m1 : m2);
        const int ol = __ffs(lanes) - 1;
        const int pos = mk ? __ffs(mk) - 1 : 0;  // meaningful on the owner lane
        const int kneg_l = (P == 0) ? 0 : (int)((mn >> pos) & 1u);
        const int pk = g.shfl((g.lane * S + pos) | (kneg_l << 16), ol);
        const int k = pk & 0xffff;
        const bool kneg = (pk >> 16) != 0;
        const int F = 2 - P;  // third factor: w, v, u
        const T kv = fetch(k);
        T mv = v;
        Wd rp, rn;
        if constexpr (ZT) {
            const Wd kp = kneg ? fneg(kv, F) : fpos(kv, F);
            const Wd kn = kneg ? fpos(kv, F) : fneg(kv, F);
            tadd(fpos(v, F), fneg(v, F), kp, kn, rp, rn);
        } else {
            rp = fpos(v, F) ^ fpos(kv, F);
            rn = Wd(0);
        }
        fset(mv, F, rp, rn);
        const bool zero = (rp | rn) == Wd(0);
        canon(mv);
        const int lo = s < k ? s : k;
        const int hi = s < k ? k : s;
        q_remove(k);
        store(mv, lo);
        c_mrg += 1;
        // drop hi, then lo as well when the merged term vanished
#pragma unroll 1
        for (int d = 0; d < 2; ++d) {
            if (d == 1 && !zero) break;
            drop(d == 0 ? hi : lo);
        }
        if (zero) c_drp += 1;
        else q_push(lo);
    }

    __device__ __forceinline__ void cascade() {
#pragma unroll 1
        while (qlen > 0) reduce_one(q_pop());
    }

    __device__ __forceinline__ void snapshot(Wd *bestp) const {
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
            if (slot < r) {
#pragma unroll
                for (int w = 0; w < NWT; ++w) bestp[(size_t)slot * NWT + w] = st[p][w];
            }
        }
    }

    // Plus transition (Section 3.3.1) with roles (A,B,C) a permutation of
    // (u,v,w): writes the three new terms and queues them; returns the record
    // for the digest, or 0 when no attempt passed.
    __device__ __forceinline__ uint64_t plus_setup(const SegDesc &d) {
#pragma unroll 1
        for (int a = 1; a <= d.plus_attempts; ++a) {
            const U4 y = philox10((uint32_t)t, (uint32_t)(t >> 32), wid, (uint32_t)a, key0, key1);
            const int pi = (int)__umulhi(y.x, (uint32_t)r);
            const int pj = (pi + 1 + (int)__umulhi(y.y, (uint32_t)(r - 1))) % r;
            const int perm = (int)__umulhi(y.z, 6u);
            // PERM = {u,v,w},{u,w,v},{v,u,w},{v,w,u},{w,u,v},{w,v,u}
            const int A = perm >> 1;
            const int B = (perm == 0 || perm == 5) ? 1 : ((perm == 1 || perm == 3) ? 2 : 0);
            const int C = 3 - A - B;
            const T ti = fetch(pi), tj = fetch(pj);
            Wd nbp, nbn, ncp, ncn, nap, nan_;
            bool ok;
            if constexpr (ZT) {
                ok = tadd(fpos(ti, B), fneg(ti, B), fpos(tj, B), fneg(tj, B), nbp, nbn);
                ok &= tadd(fpos(tj, C), fneg(tj, C), fneg(ti, C), fpos(ti, C), ncp, ncn);
                ok &= tadd(fpos(tj, A), fneg(tj, A), fneg(ti, A), fpos(ti, A), nap, nan_);
            } else {
                nbp = fpos(ti, B) ^ fpos(tj, B);
                ncp = fpos(tj, C) ^ fpos(ti, C);
                nap = fpos(tj, A) ^ fpos(ti, A);
                nbn = ncn = nan_ = Wd(0);
                ok = true;
            }
            ok = ok && ((nbp | nbn) != Wd(0)) && ((ncp | ncn) != Wd(0)) && ((nap | nan_) != Wd(0));
            if (!ok) continue;
            T tn = tj;
            fset(tn, A, nap, nan_);  // (A_j - A_i, B_j, C_j)
            canon(tn);
            store(tn, r);
            tn = tj;
            fset(tn, A, fpos(ti, A), fneg(ti, A));  // (A_i, B_j, C_j - C_i)
            fset(tn, C, ncp, ncn);
            canon(tn);
            store(tn, pj);
            tn = ti;
            fset(tn, B, nbp, nbn);  // (A_i, B_i + B_j, C_i)
            canon(tn);
            store(tn, pi);
            r += 1;
            plateau = 0;
            c_pls += 1;
            qlen = 0;
            q_push(pi);
            q_push(pj);
            q_push(r - 1);
            return 0xFull | ((uint64_t)a << 4) | ((uint64_t)perm << 9) | ((uint64_t)(uint32_t)pi << 12) |
                   ((uint64_t)(uint32_t)pj << 28);
        }
        return 0;
    }

    __device__ __forceinline__ void run(const SegDesc &d, int64_t w, int32_t steps) {
        tfg_walker_info *H = d.hdr + w;
        r = H->r; best_r = H->best_r; R = d.R;
        t = H->t; plateau = H->plateau; best_t = H->best_t;
        dig = H->digest; wid = H->walker_id;
        key0 = d.key0; key1 = d.key1;
        c_acc = c_rej = c_noc = c_drp = c_mrg = c_pls = c_red = 0;
        qlen = 0; q0 = q1 = q2 = 0;
        const Wd *src = reinterpret_cast<const Wd *>(d.slots) + (size_t)w * R * NWT;
        Wd *bestp = reinterpret_cast<Wd *>(d.best) + (size_t)w * R * NWT;
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
#pragma unroll
            for (int q = 0; q < NWT; ++q) st[p][q] = (slot < R) ? src[(size_t)slot * NWT + q] : Wd(0);
        }

        uint32_t xr0 = 0, xr1 = 0, xr2 = 0;
        int kb = G;
#pragma unroll 1
        for (int32_t step = 0; step < steps; ++step) {
            // ---- draw: lane l holds the Philox output of step (batch start + l)
            if (kb == G) {
                const uint64_t tl = (uint64_t)t + (uint64_t)g.lane;
                const U4 x = philox10((uint32_t)tl, (uint32_t)(tl >> 32), wid, 0u, key0, key1);
                xr0 = x.x; xr1 = x.y; xr2 = x.z;
                kb = 0;
            }
            const uint32_t x0 = g.shfl(xr0, kb), x1 = g.shfl(xr1, kb), x2 = g.shfl(xr2, kb);
            kb += 1;

            const int r_before = r;
            const int i = (int)__umulhi(x0, (uint32_t)r);
            int action = kNoCand, X = 0, j = 0, rho = 0, sneg = 0;
            {
                T ti = fetch(i);
                // ---- try_flip: candidates (X, j) with X_j = +-X_i, ordered (X, slot)
                uint32_t bu = 0, bv = 0, bw = 0, bwn = 0;
#pragma unroll
                for (int p = 0; p < S; ++p) {
                    const int slot = g.lane * S + p;
                    const bool live = slot < r && slot != i;
                    if constexpr (ZT) {
                        const bool eu = st[p][0] == ti.w[0] && st[p][1] == ti.w[1];
                        const bool ev = st[p][2] == ti.w[2] && st[p][3] == ti.w[3];
                        const bool ewp = st[p][4] == ti.w[4] && st[p][5] == ti.w[5];
                        const bool ewn = st[p][4] == ti.w[5] && st[p][5] == ti.w[4];
                        bu |= (uint32_t)(live && eu) << p;
                        bv |= (uint32_t)(live && ev) << p;
                        bw |= (uint32_t)(live && (ewp || ewn)) << p;
                        bwn |= (uint32_t)(live && ewn) << p;
                    } else {
                        bu |= (uint32_t)(live && st[p][0] == ti.w[0]) << p;
                        bv |= (uint32_t)(live && st[p][1] == ti.w[1]) << p;
                        bw |= (uint32_t)(live && st[p][2] == ti.w[2]) << p;
                    }
                }
                const uint32_t own = (uint32_t)__popc(bu) | ((uint32_t)__popc(bv) << 10) | ((uint32_t)__popc(bw) << 20);
                uint32_t incl = own;
#pragma unroll
                for (int dd = 1; dd < G; dd <<= 1) {
                    const uint32_t y = __shfl_up_sync(g.mask, incl, dd, G);
                    if (g.lane >= dd) incl += y;
                }
                const uint32_t tot = g.shfl(incl, G - 1);
                const uint32_t excl = incl - own;
                const int nU = (int)(tot & 1023u), nV = (int)((tot >> 10) & 1023u), nW = (int)(tot >> 20);
                const int K = 2 * (nU + nV + nW);

                if (K > 0) {
                    const int c = (int)__umulhi(x1, (uint32_t)K);
                    rho = c & 1;
                    const int mi = c >> 1;
                    int basec;
                    if (mi < nU) { X = 0; basec = 0; }
                    else if (mi < nU + nV) { X = 1; basec = nU; }
                    else { X = 2; basec = nU + nV; }
                    const int idx = mi - basec;
                    const int sh = 10 * X;
                    const int myex = (int)((excl >> sh) & 1023u);
                    const int mycnt = (int)((own >> sh) & 1023u);
                    const unsigned ob = g.ballot(idx >= myex && idx < myex + mycnt);
                    const int ol = __ffs(ob) - 1;
                    const uint32_t mk = X == 0 ? bu : (X == 1 ? bv : bw);
                    const int nth = idx - myex;
                    int pos = 0, cnt = 0;
#pragma unroll
                    for (int p = 0; p < S; ++p) {
                        const int b = (int)((mk >> p) & 1u);
                        if (b && cnt == nth) pos = p;
                        cnt += b;
                    }
                    const int packed = (g.lane * S + pos) | (int)(((X == 2) ? ((bwn >> pos) & 1u) : 0u) << 16);
                    const int pk = g.shfl(packed, ol);
                    j = pk & 0xffff;
                    sneg = pk >> 16;
                    T tj = fetch(j);

                    // flip: (Y, Z) cyclic after X, rho swaps; Y_i += Y_j, Z_j -= s Z_i
                    int Y = X == 0 ? 1 : (X == 1 ? 2 : 0);
                    int Z = X == 0 ? 2 : (X == 1 ? 0 : 1);
                    if (rho) { const int tmp = Y; Y = Z; Z = tmp; }
                    Wd nyp, nyn, nzp, nzn;
                    bool ok;
                    if constexpr (ZT) {
                        ok = tadd(fpos(ti, Y), fneg(ti, Y), fpos(tj, Y), fneg(tj, Y), nyp, nyn);
                        const Wd ap = sneg ? fpos(ti, Z) : fneg(ti, Z);
                        const Wd an = sneg ? fneg(ti, Z) : fpos(ti, Z);
                        ok &= tadd(fpos(tj, Z), fneg(tj, Z), ap, an, nzp, nzn);
                    } else {
                        nyp = fpos(ti, Y) ^ fpos(tj, Y);
                        nzp = fpos(tj, Z) ^ fpos(ti, Z);
                        nyn = nzn = Wd(0);
                        ok = true;
                    }
                    if (!ok) {
                        action = kReject;
                        c_rej += 1;
                    } else {
                        action = kAccept;
                        c_acc += 1;
                        fset(ti, Y, nyp, nyn);
                        fset(tj, Z, nzp, nzn);
                        const bool zi = (nyp | nyn) == Wd(0);
                        const bool zj = (nzp | nzn) == Wd(0);
                        canon(ti);
                        canon(tj);
                        store(ti, i);
                        store(tj, j);
                        qlen = 0;
                        if (zi || zj) {
                            q_push(i);
                            q_push(j);
                            const int hi = i > j ? i : j, lo = i > j ? j : i;
                            const bool zhi = (hi == i) ? zi : zj, zlo = (lo == i) ? zi : zj;
#pragma unroll 1
                            for (int dd = 0; dd < 2; ++dd) {
                                const bool z = dd == 0 ? zhi : zlo;
                                if (z) { drop(dd == 0 ? hi : lo); c_drp += 1; }
                            }
                        } else if (pair_hit(ti, i) || pair_hit(tj, j)) {
                            // the queue is only needed when a term shares a factor pair
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
                const uint64_t rec = (uint64_t)action | ((uint64_t)X << 4) | ((uint64_t)rho << 6) |
                                     ((uint64_t)sneg << 7) | ((uint64_t)(uint32_t)i << 8) |
                                     ((uint64_t)(uint32_t)j << 24) | ((uint64_t)(uint32_t)r << 40);
                dig = digest_mix(dig, rec);
                // best scheme: always when better, with probability 0.01 when equal
                if (r < best_r) {
                    snapshot(bestp);
                    best_r = r;
                    best_t = t;
                    plateau = 0;
                } else {
                    if (r == best_r && x2 < d.refresh_thresh) snapshot(bestp);
                    plateau += 1;
                }
                // plus transition on a plateau, only near the best rank
                if (d.plus_enabled && plateau >= d.plateau_len && r <= best_r + 2 && r < R && r >= 2) {
                    rec2 = plus_setup(d);
                    if (rec2) { plus_phase = true; continue; }
                }
                break;
            }
            t += 1;
        }

        // ---- write back
        Wd *dst = reinterpret_cast<Wd *>(d.slots) + (size_t)w * R * NWT;
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
            if (slot < R) {
#pragma unroll
                for (int q = 0; q < NWT; ++q) dst[(size_t)slot * NWT + q] = st[p][q];
            }
        }
        if (g.lane == 0) {
            H->r = r; H->best_r = best_r;
            H->t = t; H->plateau = plateau; H->best_t = best_t;
            H->digest = dig;
            H->accepted += c_acc; H->rejected += c_rej; H->nocand += c_noc;
            H->drops += c_drp; H->merges += c_mrg; H->plus += c_pls; H->reductions += c_red;
        }
    }
};

template <int MODE, class Wd, int G, int S>
__global__ void __launch_bounds__(256) walk_kernel(const SegDesc d, const int32_t steps) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t w = gt / G;
    if (w >= d.n_walkers) return;  // whole groups exit together (G divides 32)
    Walker<MODE, Wd, G, S> wk;
    wk.run(d, w, steps);
}

}  // namespace dev

template <int MODE, class Wd, int G, int S>
void launch_walk_variant(const SegDesc &d, int32_t steps, int grid, int block, cudaStream_t st) {
    dev::walk_kernel<MODE, Wd, G, S><<<grid, block, 0, st>>>(d, steps);
}

#define TFG_WALK_VARIANT(MODE, WD, BITS, G, S) \
    WalkVariant{MODE, BITS, G, S, &launch_walk_variant<MODE, WD, G, S>, \
                reinterpret_cast<const void *>(&dev::walk_kernel<MODE, WD, G, S>)}

}  // namespace tfg
