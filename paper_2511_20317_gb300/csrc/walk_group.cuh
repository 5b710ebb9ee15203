// Lane-group flip-graph walk kernel for sm_103a.
//
// One walker = one group of G lanes (G in {4, 8, 16, 32}); lane l of the group
// holds slots l*S .. l*S+S-1 of the walker's scheme in registers (blocked
// layout, S compile-time) as packed terms (pterm.cuh): TW words of positive
// and TW words of negative coefficient bits over the concatenated u|v|w
// index.  This mapping serves large ranks and terms longer than 64 bits;
// small formats use the thread-per-walker kernel (walk_solo.cuh).
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

#include "pterm.cuh"

namespace tfg {
namespace dev {

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

// ---------------------------------------------------------------------------
// Walker: state in registers plus the group-uniform bookkeeping.
// ---------------------------------------------------------------------------
template <int MODE, class Wd, int TW, int G, int S>
struct GroupWalker {
    static constexpr bool ZT = (MODE == TFG_MODE_ZT);
    static constexpr int NWS = (ZT ? 2 : 1) * TW;   // words per slot in HBM
    using T = PTerm<Wd, TW, ZT>;
    using O = Ops<Wd, TW, ZT>;
    using M = Masks<Wd, TW>;

    Group<G> g;
    T st[S];
    M mk;
    int r, best_r, R;
    int64_t t, plateau, best_t;
    uint64_t dig;
    uint32_t wid, key0, key1;
    uint32_t c_acc, c_rej, c_noc, c_drp, c_mrg, c_pls, c_red;
    int qlen, q0, q1, q2;   // reduction queue (slot indices)
    uint32_t nnz, best_nnz; // non-zero coefficients of the live (walk policy 2) / best scheme

    __device__ __forceinline__ static uint32_t nnz_of(const T &v) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < TW; ++w) {
            const Wd x = ZT ? (v.p[w] | v.n[w]) : v.p[w];
            c += (uint32_t)(sizeof(Wd) == 8 ? __popcll((unsigned long long)x) : __popc((unsigned)x));
        }
        return c;
    }

    __device__ __forceinline__ T fetch(int k) const {
        const int o = k / S, pos = k - o * S;
        T out;
#pragma unroll
        for (int w = 0; w < TW; ++w) {
            Wd vp = st[0].p[w], vn = st[0].n[w];
#pragma unroll
            for (int p = 1; p < S; ++p) {
                vp = (pos == p) ? st[p].p[w] : vp;
                if constexpr (ZT) vn = (pos == p) ? st[p].n[w] : vn;
            }
            out.p[w] = g.shfl(vp, o);
            out.n[w] = ZT ? g.shfl(vn, o) : Wd(0);
        }
        return out;
    }

    __device__ __forceinline__ void store(const T &v, int k) {
        const int o = k / S, pos = k - o * S;
        const bool me = (g.lane == o);
#pragma unroll
        for (int p = 0; p < S; ++p)
            if (me && pos == p) st[p] = v;
    }

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

    // Any other live slot sharing a factor pair with a (slot sa) or b (slot sb)?
    // (superset filter of the reduction test; validity is not checked)
    __device__ __forceinline__ bool pair_hit2(const T &a, int sa, const T &b, int sb) const {
        bool hit = false;
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
            bool eu, ev, ewp, ewn;
            O::compare(st[p], a, mk, eu, ev, ewp, ewn);
            const bool ew = ewp || ewn;
            const bool ha = (eu && ev) || (eu && ew) || (ev && ew);
            O::compare(st[p], b, mk, eu, ev, ewp, ewn);
            const bool ew2 = ewp || ewn;
            const bool hb = (eu && ev) || (eu && ew2) || (ev && ew2);
            hit |= (slot < r) && ((ha && slot != sa) || (hb && slot != sb));
        }
        return g.ballot(hit) != 0u;
    }

    __device__ __forceinline__ bool sum_ok(const T &a, const T &b, int f, bool neg) const {
        if constexpr (ZT) {
            Wd bad = 0;
#pragma unroll
            for (int w = 0; w < TW; ++w) {
                const Wd bp = neg ? b.n[w] : b.p[w], bn = neg ? b.p[w] : b.n[w];
                bad |= ((a.p[w] & bp) | (a.n[w] & bn)) & mk.m[f][w];
            }
            return bad == Wd(0);
        } else {
            return true;
        }
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
            bool eu, ev, ewp, ewn;
            O::compare(st[p], v, mk, eu, ev, ewp, ewn);
            const bool ew = ewp || ewn;
            m0 |= (uint32_t)(live && eu && ev && sum_ok(v, st[p], 2, false)) << p;
            m1 |= (uint32_t)(live && eu && ew && sum_ok(v, st[p], 1, ewn)) << p;
            m2 |= (uint32_t)(live && ev && ew && sum_ok(v, st[p], 0, ewn)) << p;
            mn |= (uint32_t)ewn << p;
        }
        const unsigned b0 = g.ballot(m0 != 0u), b1 = g.ballot(m1 != 0u), b2 = g.ballot(m2 != 0u);
        if ((b0 | b1 | b2) == 0u) return;
        const int P = b0 ? 0 : (b1 ? 1 : 2);
        const unsigned lanes = b0 ? b0 : (b1 ? b1 : b2);
        const uint32_t mkp = P == 0 ? m0 : (P == 1 ? m1 : m2);
        const int ol = __ffs(lanes) - 1;
        const int pos = mkp ? __ffs(mkp) - 1 : 0;  // meaningful on the owner lane
        const int kneg_l = (P == 0) ? 0 : (int)((mn >> pos) & 1u);
        const int pk = g.shfl((g.lane * S + pos) | (kneg_l << 16), ol);
        const int k = pk & 0xffff;
        const bool kneg = (pk >> 16) != 0;
        const int F = 2 - P;  // third factor: w, v, u
        const T kv = fetch(k);
        T mv;
        O::add(v, kv, F, kneg, mk, mv);
        const bool zero = O::zero(mv, F, mk);
        O::canon(mv, mk);
        const int lo = s < k ? s : k;
        const int hi = s < k ? k : s;
        q_remove(k);
        store(mv, lo);
        c_mrg += 1;
        drop(hi);
        if (zero) {
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

    __device__ __forceinline__ void snapshot(Wd *bestp) const {
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
            if (slot < r) {
#pragma unroll
                for (int w = 0; w < TW; ++w) {
                    bestp[(size_t)slot * NWS + w] = st[p].p[w];
                    if constexpr (ZT) bestp[(size_t)slot * NWS + TW + w] = st[p].n[w];
                }
            }
        }
    }

    // Expansion (Section 3.3.1): plus, or split under walk policy 1 when y3 >= 2^31;
    // writes the new terms and queues them; returns the digest record (0 when no
    // attempt passed).
    __device__ __forceinline__ uint64_t plus_setup(const SegDesc &d) {
#pragma unroll 1
        for (int a = 1; a <= d.plus_attempts; ++a) {
            const U4 y = philox10((uint32_t)t, (uint32_t)(t >> 32), wid, (uint32_t)a, key0, key1);
            const int pi = (int)__umulhi(y.x, (uint32_t)r);
            const int pj = (pi + 1 + (int)__umulhi(y.y, (uint32_t)(r - 1))) % r;
            const int perm = (int)__umulhi(y.z, 6u);
            int A, B, C;
            plus_roles(perm, A, B, C);
            const T ti = fetch(pi), tj = fetch(pj);
            if (d.walk_policy == 1 && y.w >= 0x80000000u) {
                // split: term i = (A_j, B_i, C_i), new term (A_i - A_j, B_i, C_i)
                T ns;
                const bool ok = O::add(ti, tj, A, true, mk, ns);
                if (!ok || O::zero(ns, A, mk)) continue;
                O::canon(ns, mk);
                store(ns, r);
                T ti2 = ti;
                O::take(ti2, tj, A, mk);
                O::canon(ti2, mk);
                store(ti2, pi);
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
            O::canon(na, mk);          // (A_j - A_i, B_j, C_j)
            store(na, r);
            O::take(nc, ti, A, mk);    // (A_i, B_j, C_j - C_i)
            O::canon(nc, mk);
            store(nc, pj);
            O::canon(nb, mk);          // (A_i, B_i + B_j, C_i)
            store(nb, pi);
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

    __device__ __forceinline__ void run(const SegDesc &d, int64_t w, int32_t steps) {
        tfg_walker_info *H = d.hdr + w;
        r = H->r; best_r = H->best_r; R = d.R;
        t = H->t; plateau = H->plateau; best_t = H->best_t;
        dig = H->digest; wid = H->walker_id;
        key0 = d.key0; key1 = d.key1;
        best_nnz = H->best_nnz;
        mk.load(d);
        c_acc = c_rej = c_noc = c_drp = c_mrg = c_pls = c_red = 0;
        qlen = 0; q0 = q1 = q2 = 0;
        const Wd *src = reinterpret_cast<const Wd *>(d.slots) + (size_t)w * R * NWS;
        Wd *bestp = reinterpret_cast<Wd *>(d.best) + (size_t)w * R * NWS;
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
#pragma unroll
            for (int q = 0; q < TW; ++q) {
                st[p].p[q] = (slot < R) ? src[(size_t)slot * NWS + q] : Wd(0);
                st[p].n[q] = (ZT && slot < R) ? src[(size_t)slot * NWS + TW + q] : Wd(0);
            }
        }
        nnz = 0;
        if (d.walk_policy == 2) {
            uint32_t mine = 0;
#pragma unroll
            for (int p = 0; p < S; ++p)
                if (g.lane * S + p < r) mine += nnz_of(st[p]);
#pragma unroll
            for (int o = 1; o < G; o <<= 1) mine += __shfl_xor_sync(g.mask, mine, o, G);
            nnz = mine;
        }

        uint32_t xr0 = 0, xr1 = 0, xr2 = 0, xr3 = 0;
        int kb = G;
#pragma unroll 1
        for (int32_t step = 0; step < steps; ++step) {
            // ---- draw: lane l holds the Philox output of step (batch start + l)
            if (kb == G) {
                const uint64_t tl = (uint64_t)t + (uint64_t)g.lane;
                const U4 x = philox10((uint32_t)tl, (uint32_t)(tl >> 32), wid, 0u, key0, key1);
                xr0 = x.x; xr1 = x.y; xr2 = x.z; xr3 = x.w;
                kb = 0;
            }
            const uint32_t x0 = g.shfl(xr0, kb), x1 = g.shfl(xr1, kb), x2 = g.shfl(xr2, kb), x3 = g.shfl(xr3, kb);
            kb += 1;

            const int r_before = r;
            const int i = (int)__umulhi(x0, (uint32_t)r);
            int action = kNoCand, X = 0, j = 0, rho = 0, sneg = 0;
            {
                const T ti = fetch(i);
                // ---- try_flip: candidates (X, j) with X_j = +-X_i, ordered (X, slot)
                uint32_t bu = 0, bv = 0, bw = 0, bwn = 0;
#pragma unroll
                for (int p = 0; p < S; ++p) {
                    const int slot = g.lane * S + p;
                    const bool live = slot < r && slot != i;
                    bool eu, ev, ewp, ewn;
                    O::compare(st[p], ti, mk, eu, ev, ewp, ewn);
                    bu |= (uint32_t)(live && eu) << p;
                    bv |= (uint32_t)(live && ev) << p;
                    bw |= (uint32_t)(live && (ewp || ewn)) << p;
                    bwn |= (uint32_t)(live && ewn) << p;
                }
                const uint32_t own = (uint32_t)__popc(bu) | ((uint32_t)__popc(bv) << 10) |
                                     ((uint32_t)__popc(bw) << 20);
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
                    const uint32_t mkx = X == 0 ? bu : (X == 1 ? bv : bw);
                    const int nth = idx - myex;
                    int pos = 0, cnt = 0;
#pragma unroll
                    for (int p = 0; p < S; ++p) {
                        const int b = (int)((mkx >> p) & 1u);
                        if (b && cnt == nth) pos = p;
                        cnt += b;
                    }
                    const int packed = (g.lane * S + pos) | (int)(((X == 2) ? ((bwn >> pos) & 1u) : 0u) << 16);
                    const int pk = g.shfl(packed, ol);
                    j = pk & 0xffff;
                    sneg = pk >> 16;
                    const T tj = fetch(j);

                    // flip: (Y, Z) cyclic after X, rho swaps; Y_i += Y_j, Z_j -= s Z_i
                    int Y = X == 0 ? 1 : (X == 1 ? 2 : 0);
                    int Z = X == 0 ? 2 : (X == 1 ? 0 : 1);
                    if (rho) { const int tmp = Y; Y = Z; Z = tmp; }
                    T ti2, tj2;
                    bool ok = O::add(ti, tj, Y, false, mk, ti2);
                    ok &= O::add(tj, ti, Z, sneg == 0, mk, tj2);
                    if (!ok) {
                        action = kReject;
                        c_rej += 1;
                    } else {
                        action = kAccept;
                        c_acc += 1;
                        const bool zi = O::zero(ti2, Y, mk);
                        const bool zj = O::zero(tj2, Z, mk);
                        if (d.walk_policy == 2)
                            nnz += (zi ? 0u : nnz_of(ti2)) + (zj ? 0u : nnz_of(tj2)) - nnz_of(ti) - nnz_of(tj);
                        O::canon(ti2, mk);
                        O::canon(tj2, mk);
                        store(ti2, i);
                        store(tj2, j);
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
                            if (d.walk_policy == 2) qlen = 0;   // no reduction edges
                        } else if (d.walk_policy != 2 && pair_hit2(ti2, i, tj2, j)) {
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
                dig = digest_mix(dig, flip_record(action, X, rho, sneg, i, j, r));
                // walk policy 1: a failed try_flip expands and ends the step (no best update)
                const bool failed = d.walk_policy == 1 && action != kAccept;
                // best scheme: always when better, with probability 0.01 when equal
                // (policy 2: better = least (rank, non-zero coefficients))
                if (d.walk_policy == 2) {
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
                if (d.walk_policy == 2)
                    expand = false;
                else if (d.walk_policy == 1)
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
        Wd *dst = reinterpret_cast<Wd *>(d.slots) + (size_t)w * R * NWS;
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const int slot = g.lane * S + p;
            if (slot < R) {
#pragma unroll
                for (int q = 0; q < TW; ++q) {
                    dst[(size_t)slot * NWS + q] = st[p].p[q];
                    if constexpr (ZT) dst[(size_t)slot * NWS + TW + q] = st[p].n[q];
                }
            }
        }
        if (g.lane == 0) {
            H->r = r; H->best_r = best_r;
            H->t = t; H->plateau = plateau; H->best_t = best_t;
            H->digest = dig;
            H->accepted += c_acc; H->rejected += c_rej; H->nocand += c_noc;
            H->drops += c_drp; H->merges += c_mrg; H->plus += c_pls; H->reductions += c_red;
            H->best_nnz = best_nnz;
        }
    }
};

template <int MODE, class Wd, int TW, int G, int S>
__global__ void __launch_bounds__(256) walk_group_kernel(const SegDesc d, const int32_t steps) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t w = gt / G;
    if (w >= d.n_walkers) return;  // whole groups exit together (G divides 32)
    GroupWalker<MODE, Wd, TW, G, S> wk;
    wk.run(d, w, steps);
}

}  // namespace dev

template <int MODE, class Wd, int TW, int G, int S>
void launch_walk_group(const SegDesc &d, int32_t steps, int grid, int block, cudaStream_t st) {
    dev::walk_group_kernel<MODE, Wd, TW, G, S><<<grid, block, 0, st>>>(d, steps);
}

#define TFG_GROUP_VARIANT(MODE, WD, BITS, TW, G, S) \
    WalkVariant{MODE, BITS, TW, G, S, 0, &launch_walk_group<MODE, WD, TW, G, S>, \
                reinterpret_cast<const void *>(&dev::walk_group_kernel<MODE, WD, TW, G, S>), nullptr}

}  // namespace tfg
