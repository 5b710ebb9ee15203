// Z_2 -> Z_T sign lifting (section "Ternary Lifting Script"): give every
// non-zero coefficient of a scheme that satisfies Eq. (1) modulo 2 a sign so
// that Eq. (1) holds over the integers, by exact search.
//
// Sign bits: coefficient c = (-1)^x.  For a tensor entry (a, b, c) let S be
// the terms whose u[a], v[b], w[c] are all non-zero and e_t = x_u + x_v + x_w
// (mod 2) the sign bit of term t's product.  Eq. (1) over the integers says
// sum_{t in S} (-1)^e_t = T(a,b,c), i.e. exactly (|S| - T) / 2 of the e_t are
// 1.  The parity of that count is a linear equation over GF(2) in the sign
// bits (|S| = 1 forces e_t = 0, |S| = 2 forces e_1 + e_2 = 1, and in general
// sum e_t = (|S| - T) / 2 mod 2); all of them are solved by elimination.  The
// exact count of entries with |S| >= 3 is checked during a depth-first search
// over the elimination's free bits (ordered so that products' signs become
// known early), with every entry's counts of known negative and positive
// products bounded as they grow.  Per term the first non-zero of u and of v
// is +1 (flipping the signs of two factors of a term changes nothing), which
// removes the sign symmetry.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "host_scheme.h"

namespace tfg {
namespace host {
namespace {

using Bits = std::vector<uint64_t>;

inline void bset(Bits &b, int i) { b[(size_t)i >> 6] |= 1ull << (i & 63); }
inline bool btest(const Bits &b, int i) { return (b[(size_t)i >> 6] >> (i & 63)) & 1ull; }
inline void bxor(Bits &a, const Bits &b) {
    for (size_t k = 0; k < a.size(); ++k) a[k] ^= b[k];
}

// An affine function over GF(2) of the free bits: constant + sum of bits in mask.
struct Affine {
    Bits mask;
    int c = 0;
};

struct Constraint {                // entries with |S| >= 3
    std::vector<int> prods;        // indices into the product list
    int want_neg;                  // number of negative products required
};

}  // namespace

int lift_signs(const tfg_format &f, int r, const int8_t *rows, int64_t max_nodes, int8_t *out,
               int64_t *nodes_used) {
    const int LU = f.m * f.n, LV = f.n * f.p, LW = f.p * f.m, LT = LU + LV + LW;
    // sign variables: one per non-zero coefficient; var[t*LT + e] = index or -1
    std::vector<int> var((size_t)r * LT, -1);
    int nv = 0;
    for (int t = 0; t < r; ++t)
        for (int e = 0; e < LT; ++e)
            if (rows[(size_t)t * LT + e] != 0) var[(size_t)t * LT + e] = nv++;
    const int W = (nv + 64) / 64;   // one extra bit: the constant column
    // fixed bits (sign symmetry): first non-zero of u and of v of every term is +1
    std::vector<int> fixed_zero;
    for (int t = 0; t < r; ++t)
        for (int x = 0; x < 2; ++x) {
            const int base = x == 0 ? 0 : LU, len = x == 0 ? LU : LV;
            for (int e = base; e < base + len; ++e)
                if (var[(size_t)t * LT + e] >= 0) { fixed_zero.push_back(var[(size_t)t * LT + e]); break; }
        }
    // products per tensor entry
    struct Prod { int t, xa, xb, xc; };
    std::vector<Prod> prods;
    std::vector<Bits> rowsys;            // linear equations: bits of vars + constant at bit nv
    std::vector<Constraint> nonlin;
    auto eq = [&](const std::vector<int> &vars, int rhs) {
        Bits row((size_t)W, 0);
        for (int v : vars) row[(size_t)v >> 6] ^= 1ull << (v & 63);
        if (rhs) bset(row, nv);
        rowsys.push_back(row);
    };
    for (int v : fixed_zero) eq({v}, 0);
    for (int a = 0; a < LU; ++a)
        for (int b = 0; b < LV; ++b)
            for (int c = 0; c < LW; ++c) {
                const int i = a / f.n, k = a % f.n, k2 = b / f.p, j = b % f.p, j2 = c / f.m, i2 = c % f.m;
                const int T = (k == k2 && j == j2 && i == i2) ? 1 : 0;
                std::vector<int> S;
                for (int t = 0; t < r; ++t)
                    if (var[(size_t)t * LT + a] >= 0 && var[(size_t)t * LT + LU + b] >= 0 &&
                        var[(size_t)t * LT + LU + LV + c] >= 0)
                        S.push_back(t);
                const int K = (int)S.size();
                if (K == 0) {
                    if (T) { set_error("not a Z_2 scheme: an entry of the tensor is not covered"); return TFG_EINVAL; }
                    continue;
                }
                if ((K - T) % 2 != 0) { set_error("not a Z_2 scheme (Eq. (1) fails modulo 2)"); return TFG_EINVAL; }
                const int want = (K - T) / 2;
                if (K == 1) {
                    const int t = S[0];
                    eq({var[(size_t)t * LT + a], var[(size_t)t * LT + LU + b], var[(size_t)t * LT + LU + LV + c]}, 0);
                } else if (K == 2) {
                    std::vector<int> vs;
                    for (int t : S)
                        for (int v : {var[(size_t)t * LT + a], var[(size_t)t * LT + LU + b],
                                      var[(size_t)t * LT + LU + LV + c]})
                            vs.push_back(v);
                    eq(vs, 1);
                } else {
                    // the parity of the number of negatives is linear: sum e_t = want (mod 2)
                    std::vector<int> vs;
                    for (int t : S)
                        for (int v : {var[(size_t)t * LT + a], var[(size_t)t * LT + LU + b],
                                      var[(size_t)t * LT + LU + LV + c]})
                            vs.push_back(v);
                    eq(vs, want & 1);
                    Constraint cs;
                    cs.want_neg = want;
                    for (int t : S) {
                        cs.prods.push_back((int)prods.size());
                        prods.push_back({t, var[(size_t)t * LT + a], var[(size_t)t * LT + LU + b],
                                         var[(size_t)t * LT + LU + LV + c]});
                    }
                    nonlin.push_back(cs);
                }
            }
    // Gauss-Jordan elimination over GF(2)
    std::vector<int> pivot_row_of(nv, -1);
    int rank_sys = 0;
    for (int col = 0; col < nv && rank_sys < (int)rowsys.size(); ++col) {
        int piv = -1;
        for (int q = rank_sys; q < (int)rowsys.size(); ++q)
            if (btest(rowsys[q], col)) { piv = q; break; }
        if (piv < 0) continue;
        std::swap(rowsys[(size_t)piv], rowsys[(size_t)rank_sys]);
        for (int q = 0; q < (int)rowsys.size(); ++q)
            if (q != rank_sys && btest(rowsys[q], col)) bxor(rowsys[q], rowsys[rank_sys]);
        pivot_row_of[col] = rank_sys;
        ++rank_sys;
    }
    for (int q = rank_sys; q < (int)rowsys.size(); ++q)
        if (btest(rowsys[q], nv)) {
            set_error("no sign assignment exists (the linear equations are inconsistent)");
            if (nodes_used) *nodes_used = 0;
            return TFG_ESCHEME;
        }
    // free variables and each variable as an affine function of them
    std::vector<int> free_vars;
    for (int v = 0; v < nv; ++v)
        if (pivot_row_of[v] < 0) free_vars.push_back(v);
    const int nf = (int)free_vars.size();
    const int FW = (nf + 64) / 64;
    std::vector<int> free_pos(nv, -1);
    for (int q = 0; q < nf; ++q) free_pos[free_vars[q]] = q;
    std::vector<Affine> val((size_t)nv);
    for (int v = 0; v < nv; ++v) {
        Affine &A = val[(size_t)v];
        A.mask.assign((size_t)FW, 0);
        if (free_pos[v] >= 0) {
            bset(A.mask, free_pos[v]);
        } else {
            const Bits &row = rowsys[(size_t)pivot_row_of[v]];
            A.c = btest(row, nv) ? 1 : 0;
            for (int q = 0; q < nf; ++q)
                if (btest(row, free_vars[q])) bset(A.mask, q);
        }
    }
    // sign bit of every product of the non-linear entries
    std::vector<Affine> pe(prods.size());
    for (size_t k = 0; k < prods.size(); ++k) {
        Affine e;
        e.mask.assign((size_t)FW, 0);
        for (int v : {prods[k].xa, prods[k].xb, prods[k].xc}) {
            bxor(e.mask, val[(size_t)v].mask);
            e.c ^= val[(size_t)v].c;
        }
        pe[k] = e;
    }
    // search order of the free bits: greedily, the bit that most advances the
    // products nearest to being fixed (weight 1 / bits left), so that products'
    // signs become known early
    std::vector<int> remaining(pe.size());
    for (size_t k = 0; k < pe.size(); ++k) {
        int c = 0;
        for (uint64_t wd : pe[k].mask) c += __builtin_popcountll(wd);
        remaining[k] = c;
    }
    std::vector<std::vector<int>> prods_of(nf);
    for (size_t k = 0; k < pe.size(); ++k)
        for (int q = 0; q < nf; ++q)
            if (btest(pe[k].mask, q)) prods_of[(size_t)q].push_back((int)k);
    std::vector<int> order_bits;                    // search position -> original free bit
    std::vector<char> taken((size_t)nf, 0);
    for (int step = 0; step < nf; ++step) {
        int best = -1;
        double best_w = -1.0;
        for (int q = 0; q < nf; ++q) {
            if (taken[(size_t)q]) continue;
            double wgt = 0.0;
            for (int k : prods_of[(size_t)q]) wgt += 1.0 / remaining[(size_t)k];
            if (wgt > best_w) { best_w = wgt; best = q; }
        }
        taken[(size_t)best] = 1;
        order_bits.push_back(best);
        for (int k : prods_of[(size_t)best]) remaining[(size_t)k] -= 1;
    }
    std::vector<int> newpos((size_t)nf);
    for (int q = 0; q < nf; ++q) newpos[(size_t)order_bits[(size_t)q]] = q;
    auto permute = [&](Affine &A) {
        Bits m2((size_t)FW, 0);
        for (int q = 0; q < nf; ++q)
            if (btest(A.mask, q)) bset(m2, newpos[(size_t)q]);
        A.mask = m2;
    };
    for (Affine &A : val) permute(A);
    for (Affine &A : pe) permute(A);
    // each product's sign is known once its last bit is set
    std::vector<std::vector<int>> det_at((size_t)nf + 1);
    std::vector<int> cons_of(pe.size(), -1);
    for (size_t q = 0; q < nonlin.size(); ++q)
        for (int k : nonlin[q].prods) cons_of[(size_t)k] = (int)q;
    for (size_t k = 0; k < pe.size(); ++k) {
        int last = -1;
        for (int b = nf - 1; b >= 0; --b)
            if (btest(pe[k].mask, b)) { last = b; break; }
        det_at[(size_t)(last + 1)].push_back((int)k);
    }
    Bits assign((size_t)FW, 0);
    auto eval = [&](const Affine &A) {
        int s2 = A.c;
        for (size_t k = 0; k < A.mask.size(); ++k) s2 ^= __builtin_parityll(A.mask[k] & assign[k]);
        return s2;
    };
    // running counts of known negative / positive products per entry; an entry
    // with K products needing N negatives fails once neg > N or pos > K - N
    std::vector<int> negc(nonlin.size(), 0), posc(nonlin.size(), 0);
    auto apply = [&](int at, int sign) {      // sign +1 adds the products fixed at `at`, -1 removes them
        bool ok = true;
        for (int k : det_at[(size_t)at]) {
            const int q = cons_of[(size_t)k];
            if (eval(pe[(size_t)k])) negc[(size_t)q] += sign; else posc[(size_t)q] += sign;
        }
        if (sign > 0)
            for (int k : det_at[(size_t)at]) {
                const int q = cons_of[(size_t)k];
                const int K = (int)nonlin[(size_t)q].prods.size(), N = nonlin[(size_t)q].want_neg;
                if (negc[(size_t)q] > N || posc[(size_t)q] > K - N) ok = false;
            }
        return ok;
    };
    int64_t nodes = 0;
    bool found = false, exhausted = true;
    if (!apply(0, +1)) {
        if (nodes_used) *nodes_used = 0;
        set_error("no sign assignment exists");
        return TFG_ESCHEME;
    }
    // iterative depth-first search over search positions 0..nf-1 (0 tried before 1)
    std::vector<int> choice((size_t)nf, -1);
    std::vector<char> applied((size_t)nf, 0);
    int depth = 0;
    while (true) {
        if (depth == nf) { found = true; break; }
        if (applied[(size_t)depth]) { apply(depth + 1, -1); applied[(size_t)depth] = 0; }
        if (choice[(size_t)depth] >= 1) {          // both values tried: backtrack
            choice[(size_t)depth] = -1;
            assign[(size_t)depth >> 6] &= ~(1ull << (depth & 63));
            if (depth == 0) break;
            --depth;
            continue;
        }
        choice[(size_t)depth] += 1;
        if (choice[(size_t)depth]) assign[(size_t)depth >> 6] |= 1ull << (depth & 63);
        else assign[(size_t)depth >> 6] &= ~(1ull << (depth & 63));
        if (++nodes > max_nodes) { exhausted = false; break; }
        applied[(size_t)depth] = 1;
        if (apply(depth + 1, +1)) ++depth;
    }
    if (nodes_used) *nodes_used = nodes;
    if (!found) {
        set_error(exhausted ? "no sign assignment exists" : "search budget exhausted");
        return exhausted ? TFG_ESCHEME : TFG_ETIMEOUT;
    }
    for (int t = 0; t < r; ++t)
        for (int e = 0; e < LT; ++e) {
            const int v = var[(size_t)t * LT + e];
            out[(size_t)t * LT + e] = (int8_t)(v < 0 ? 0 : (eval(val[(size_t)v]) ? -1 : 1));
        }
    return TFG_OK;
}

}  // namespace host
}  // namespace tfg
