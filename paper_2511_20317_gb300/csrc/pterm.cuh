// Packed ternary terms for the device walkers.
//
// A term u (x) v (x) w is held as one pair of bit vectors over the
// concatenated coefficient index b = [u: 0..mn) | [v: mn..mn+np) | [w: ..LT)
// (LT = mn + np + pm): P (coefficient +1) and N (coefficient -1).  These are
// the "digits"/"signs" masks of Section 3.5.1 with digits = P|N, signs = N.
// A factor is selected with a constant mask M[X]; every operation of Section
// 3.5.2 (addition with validity flag, equality, equality up to sign) is a few
// masked word operations.  Z_2 terms keep P only (addition is XOR).
// TW words per sign hold LT bits (Wd = 32-bit when LT <= 32, else 64-bit).
#pragma once
#include <cstdint>

#include "tfg_internal.h"

namespace tfg {
namespace dev {

struct U4 { uint32_t x, y, z, w; };

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds, Weyl key schedule.
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

// Rolling trajectory digest: multiply-xorshift of one packed record per event.
__device__ __forceinline__ uint64_t digest_mix(uint64_t h, uint64_t v) {
    h ^= v;
    h *= 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    return h;
}

__device__ __forceinline__ uint64_t flip_record(int action, int X, int rho, int sneg, int i, int j, int r) {
    return (uint64_t)action | ((uint64_t)X << 4) | ((uint64_t)rho << 6) | ((uint64_t)sneg << 7) |
           ((uint64_t)(uint32_t)i << 8) | ((uint64_t)(uint32_t)j << 24) | ((uint64_t)(uint32_t)r << 40);
}

__device__ __forceinline__ uint64_t plus_record(int attempt, int perm, int i, int j, int split = 0) {
    return 0xFull | ((uint64_t)attempt << 4) | ((uint64_t)perm << 9) | ((uint64_t)(uint32_t)i << 12) |
           ((uint64_t)(uint32_t)j << 28) | ((uint64_t)split << 62);
}

// Role permutations of a plus transition: (A,B,C) over (u,v,w), index 0..5
// = uvw, uwv, vuw, vwu, wuv, wvu.
__device__ __forceinline__ void plus_roles(int perm, int &A, int &B, int &C) {
    A = perm >> 1;
    B = (perm == 0 || perm == 5) ? 1 : ((perm == 1 || perm == 3) ? 2 : 0);
    C = 3 - A - B;
}

template <class Wd, int TW, bool ZT>
struct PTerm {
    Wd p[TW];
    Wd n[TW];   // unused (kept zero) in Z_2
};

// Factor masks of one format.
template <class Wd, int TW>
struct Masks {
    Wd m[3][TW];
    __device__ __forceinline__ void load(const SegDesc &d) {
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int w = 0; w < TW; ++w) m[x][w] = (Wd)d.fmask[x][w];
    }
    // mask of factor f (f may be a runtime value)
    __device__ __forceinline__ Wd of(int f, int w) const {
        return f == 0 ? m[0][w] : (f == 1 ? m[1][w] : m[2][w]);
    }
};

template <class Wd, int TW, bool ZT>
struct Ops {
    using T = PTerm<Wd, TW, ZT>;
    using M = Masks<Wd, TW>;

    // Equality tests of every factor of a against b: exact (u, v, w) and
    // w negated.  (u and v are sign-normalised in Z_T, so they never match
    // up to a sign; only w does.)
    __device__ __forceinline__ static void compare(const T &a, const T &b, const M &mk, bool &eu, bool &ev,
                                                   bool &ewp, bool &ewn) {
        Wd du = 0, dv = 0, dw = 0, dn = 0;
#pragma unroll
        for (int w = 0; w < TW; ++w) {
            Wd d = a.p[w] ^ b.p[w];
            if constexpr (ZT) d |= a.n[w] ^ b.n[w];
            du |= d & mk.m[0][w];
            dv |= d & mk.m[1][w];
            dw |= d & mk.m[2][w];
            if constexpr (ZT) dn |= ((a.p[w] ^ b.n[w]) | (a.n[w] ^ b.p[w])) & mk.m[2][w];
        }
        eu = du == Wd(0);
        ev = dv == Wd(0);
        ewp = dw == Wd(0);
        ewn = ZT ? (dn == Wd(0)) : false;
    }

    // r = a with factor f replaced by a_f + b_f (neg: a_f - b_f).  Returns
    // false when a coefficient would leave Z_T (Section 3.5.2 validity).
    __device__ __forceinline__ static bool add(const T &a, const T &b, int f, bool neg, const M &mk, T &r) {
        Wd bad = 0;
#pragma unroll
        for (int w = 0; w < TW; ++w) {
            const Wd m = mk.of(f, w);
            if constexpr (ZT) {
                const Wd bp = neg ? b.n[w] : b.p[w];
                const Wd bn = neg ? b.p[w] : b.n[w];
                bad |= ((a.p[w] & bp) | (a.n[w] & bn)) & m;
                const Wd rp = (a.p[w] | bp) & ~(a.n[w] | bn);
                const Wd rn = (a.n[w] | bn) & ~(a.p[w] | bp);
                r.p[w] = (a.p[w] & ~m) | (rp & m);
                r.n[w] = (a.n[w] & ~m) | (rn & m);
            } else {
                r.p[w] = a.p[w] ^ (b.p[w] & m);
                r.n[w] = 0;
            }
        }
        return bad == Wd(0);
    }

    __device__ __forceinline__ static bool zero(const T &a, int f, const M &mk) {
        Wd d = 0;
#pragma unroll
        for (int w = 0; w < TW; ++w) d |= (a.p[w] | (ZT ? a.n[w] : Wd(0))) & mk.of(f, w);
        return d == Wd(0);
    }

    // dst's factor f := src's factor f
    __device__ __forceinline__ static void take(T &dst, const T &src, int f, const M &mk) {
#pragma unroll
        for (int w = 0; w < TW; ++w) {
            const Wd m = mk.of(f, w);
            dst.p[w] = (dst.p[w] & ~m) | (src.p[w] & m);
            if constexpr (ZT) dst.n[w] = (dst.n[w] & ~m) | (src.n[w] & m);
        }
    }

    // Section 3.6: the first non-zero coefficient of u, then of v, becomes +1;
    // w absorbs each sign change.
    __device__ __forceinline__ static void canon(T &a, const M &mk) {
        if constexpr (ZT) {
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                bool found = false, negative = false;
#pragma unroll
                for (int w = 0; w < TW; ++w) {
                    const Wd d = (a.p[w] | a.n[w]) & mk.m[f][w];
                    const Wd low = d & (Wd(0) - d);
                    const bool here = !found && d != Wd(0);
                    negative = here ? ((a.n[w] & low) != Wd(0)) : negative;
                    found = found || here;
                }
                if (negative) {
#pragma unroll
                    for (int w = 0; w < TW; ++w) {
                        const Wd sw = (a.p[w] ^ a.n[w]) & (mk.m[f][w] | mk.m[2][w]);
                        a.p[w] ^= sw;
                        a.n[w] ^= sw;
                    }
                }
            }
        }
    }
};

}  // namespace dev
}  // namespace tfg
