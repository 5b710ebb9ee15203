// Host-side scheme functions of the C ABI: validation, Eq. (1), sign
// normalisation (Section 3.6), start preparation (Section 3.3.1 reductions)
// and the meta operators of Section 3.3.2.  Terms are held as positive /
// negative coefficient masks (one 64-bit word per factor), the representation
// of Section 3.5.1.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "host_scheme.h"

namespace tfg {
namespace host {

static thread_local std::string g_err;
void set_error(const std::string &s) { g_err = s; }
const char *last_error() { return g_err.c_str(); }

bool format_ok(const tfg_format *f) {
    if (!f) return false;
    if (f->m < 1 || f->n < 1 || f->p < 1) return false;
    if (f->m * f->n > 128 || f->n * f->p > 128 || f->p * f->m > 128) return false;
    return f->mode == TFG_MODE_ZT || f->mode == TFG_MODE_Z2;
}

int factor_len(const tfg_format &f, int x) { return x == 0 ? f.m * f.n : (x == 1 ? f.n * f.p : f.p * f.m); }
int term_len(const tfg_format &f) { return f.m * f.n + f.n * f.p + f.p * f.m; }

int parse(const tfg_format &f, int rank, const int8_t *rows, std::vector<HTerm> &out) {
    if (rank < 0 || (rank > 0 && !rows)) { set_error("bad rank or scheme pointer"); return TFG_EINVAL; }
    const int LT = term_len(f);
    out.assign((size_t)rank, HTerm{});
    for (int l = 0; l < rank; ++l) {
        int off = 0;
        for (int x = 0; x < 3; ++x) {
            const int L = factor_len(f, x);
            for (int e = 0; e < L; ++e) {
                const int c = rows[(size_t)l * LT + off + e];
                const bool ok = (f.mode == TFG_MODE_ZT) ? (c >= -1 && c <= 1) : (c == 0 || c == 1);
                if (!ok) {
                    set_error("coefficient " + std::to_string(c) + " outside the coefficient set at term " +
                              std::to_string(l));
                    return TFG_ESCHEME;
                }
                if (c > 0) out[l].p[x].set(e);
                if (c < 0) out[l].n[x].set(e);
            }
            off += L;
        }
    }
    return TFG_OK;
}

void emit(const tfg_format &f, const std::vector<HTerm> &t, int8_t *rows) {
    const int LT = term_len(f);
    for (size_t l = 0; l < t.size(); ++l) {
        int off = 0;
        for (int x = 0; x < 3; ++x) {
            const int L = factor_len(f, x);
            for (int e = 0; e < L; ++e)
                rows[l * LT + off + e] = (int8_t)((int)t[l].p[x].bit(e) - (int)t[l].n[x].bit(e));
            off += L;
        }
    }
}

// Eq. (1): accumulate every term's contribution sparsely into the tensor of
// size LU x LV x LW and compare with the matrix-multiplication tensor.
bool brent_ok(const tfg_format &f, const std::vector<HTerm> &t) {
    const int LU = f.m * f.n, LV = f.n * f.p, LW = f.p * f.m;
    std::vector<int32_t> T((size_t)LU * LV * LW, 0);
    auto coef = [](const HTerm &h, int x, int e) -> int {
        return (int)h.p[x].bit(e) - (int)h.n[x].bit(e);
    };
    for (const HTerm &h : t) {
        for (int a = 0; a < LU; ++a) {
            const int ca = coef(h, 0, a);
            if (!ca) continue;
            for (int b = 0; b < LV; ++b) {
                const int cb = coef(h, 1, b);
                if (!cb) continue;
                int32_t *row = &T[((size_t)a * LV + b) * LW];
                for (int c = 0; c < LW; ++c) {
                    const int cc = coef(h, 2, c);
                    if (cc) row[c] += ca * cb * cc;
                }
            }
        }
    }
    for (int i = 0; i < f.m; ++i)
        for (int k = 0; k < f.n; ++k)
            for (int k2 = 0; k2 < f.n; ++k2)
                for (int j = 0; j < f.p; ++j)
                    for (int j2 = 0; j2 < f.p; ++j2)
                        for (int i2 = 0; i2 < f.m; ++i2) {
                            const int a = i * f.n + k, b = k2 * f.p + j, c = j2 * f.m + i2;
                            const int want = (k == k2 && j == j2 && i == i2) ? 1 : 0;
                            const int got = T[((size_t)a * LV + b) * LW + c];
                            if (f.mode == TFG_MODE_ZT ? (got != want) : (((got - want) & 1) != 0)) return false;
                        }
    return true;
}

// Section 3.6, per term: lowest set coefficient of u, then of v, becomes +1.
void canon_term(const tfg_format &f, HTerm &h) {
    if (f.mode != TFG_MODE_ZT) return;
    for (int x = 0; x < 2; ++x) {
        const FMask low = (h.p[x] | h.n[x]).lowbit();
        if ((h.n[x] & low).any()) {
            std::swap(h.p[x], h.n[x]);
            std::swap(h.p[2], h.n[2]);
        }
    }
}

static bool zero_factor(const HTerm &h, int x) { return !(h.p[x] | h.n[x]).any(); }

// Sign relation of two factor masks: +1 equal, -1 negated, 0 neither.
static int relation(const tfg_format &f, const HTerm &a, const HTerm &b, int x) {
    if (a.p[x] == b.p[x] && a.n[x] == b.n[x]) return 1;
    if (f.mode == TFG_MODE_ZT && a.p[x] == b.n[x] && a.n[x] == b.p[x]) return -1;
    return 0;
}

// a + s*b on one factor; false when a coefficient leaves the set (Z_T).
static bool add_factor(const tfg_format &f, const HTerm &a, const HTerm &b, int x, int s, FMask &rp,
                       FMask &rn) {
    if (f.mode == TFG_MODE_Z2) { rp = a.p[x] ^ b.p[x]; rn = FMask{}; return true; }
    const FMask bp = s > 0 ? b.p[x] : b.n[x], bn = s > 0 ? b.n[x] : b.p[x];
    if (((a.p[x] & bp) | (a.n[x] & bn)).any()) return false;
    rp = (a.p[x] | bp) & ~(a.n[x] | bn);
    rn = (a.n[x] | bn) & ~(a.p[x] | bp);
    return true;
}

namespace {
struct Reducer {
    const tfg_format &f;
    std::vector<HTerm> &t;
    std::vector<int> q;
    int64_t merges = 0;

    void q_remove(int s) { q.erase(std::remove(q.begin(), q.end(), s), q.end()); }
    void q_rename(int a, int b) { for (int &v : q) if (v == a) v = b; }
    void drop(int h) {
        const int last = (int)t.size() - 1;
        q_remove(h);
        if (h != last) { t[h] = t[last]; q_rename(last, h); }
        t.pop_back();
    }
    // pairs (u,v), (u,w), (v,w); lowest partner slot with a valid merge
    bool reduce(int s) {
        static const int PA[3] = {0, 0, 1}, PB[3] = {1, 2, 2}, PF[3] = {2, 1, 0};
        for (int P = 0; P < 3; ++P) {
            for (int k = 0; k < (int)t.size(); ++k) {
                if (k == s) continue;
                const int a = relation(f, t[k], t[s], PA[P]);
                if (!a) continue;
                const int b = relation(f, t[k], t[s], PB[P]);
                if (!b) continue;
                FMask rp, rn;
                if (!add_factor(f, t[s], t[k], PF[P], a * b, rp, rn)) continue;
                HTerm mv = t[s];
                mv.p[PF[P]] = rp;
                mv.n[PF[P]] = rn;
                const int lo = std::min(s, k), hi = std::max(s, k);
                q_remove(k);
                t[lo] = mv;
                drop(hi);
                ++merges;
                if (!(rp | rn).any()) {
                    drop(lo);
                } else {
                    canon_term(f, t[lo]);
                    q.push_back(lo);
                }
                return true;
            }
        }
        return false;
    }
    void cascade() {
        while (!q.empty()) {
            const int s = q.front();
            q.erase(q.begin());
            reduce(s);
        }
    }
};
}  // namespace

void prepare(const tfg_format &f, std::vector<HTerm> &t) {
    Reducer red{f, t, {}};
    for (int s = (int)t.size() - 1; s >= 0; --s)
        if (zero_factor(t[s], 0) || zero_factor(t[s], 1) || zero_factor(t[s], 2)) red.drop(s);
    for (HTerm &h : t) canon_term(f, h);
    int64_t before;
    do {
        before = red.merges;
        for (int s = 0; s < (int)t.size(); ++s) {
            red.q.assign(1, s);
            red.cascade();
        }
    } while (red.merges != before);
}

// ---------------------------------------------------------------------------
// Meta operators on dense coefficient arrays U[l][i][k], V[l][k][j], W[l][j][i].
// ---------------------------------------------------------------------------
struct Dense {
    tfg_format f;
    int r;
    std::vector<int8_t> U, V, W;
    Dense(const tfg_format &ff, int rr) : f(ff), r(rr) {
        U.assign((size_t)rr * ff.m * ff.n, 0);
        V.assign((size_t)rr * ff.n * ff.p, 0);
        W.assign((size_t)rr * ff.p * ff.m, 0);
    }
    int8_t &u(int l, int i, int k) { return U[((size_t)l * f.m + i) * f.n + k]; }
    int8_t &v(int l, int k, int j) { return V[((size_t)l * f.n + k) * f.p + j]; }
    int8_t &w(int l, int j, int i) { return W[((size_t)l * f.p + j) * f.m + i]; }
};

static Dense to_dense(const tfg_format &f, int r, const int8_t *rows) {
    Dense d(f, r);
    const int LU = f.m * f.n, LV = f.n * f.p, LW = f.p * f.m, LT = LU + LV + LW;
    for (int l = 0; l < r; ++l) {
        std::memcpy(&d.U[(size_t)l * LU], rows + (size_t)l * LT, LU);
        std::memcpy(&d.V[(size_t)l * LV], rows + (size_t)l * LT + LU, LV);
        std::memcpy(&d.W[(size_t)l * LW], rows + (size_t)l * LT + LU + LV, LW);
    }
    return d;
}

static std::vector<int8_t> to_rows(Dense &d) {
    const int LU = d.f.m * d.f.n, LV = d.f.n * d.f.p, LW = d.f.p * d.f.m, LT = LU + LV + LW;
    std::vector<int8_t> rows((size_t)d.r * LT);
    for (int l = 0; l < d.r; ++l) {
        std::memcpy(&rows[(size_t)l * LT], &d.U[(size_t)l * LU], LU);
        std::memcpy(&rows[(size_t)l * LT + LU], &d.V[(size_t)l * LV], LV);
        std::memcpy(&rows[(size_t)l * LT + LU + LV], &d.W[(size_t)l * LW], LW);
    }
    return rows;
}

// Validate sizes, coefficients and Eq. (1) of an input scheme.
int check_input(const tfg_format *f, int rank, const int8_t *rows) {
    if (!format_ok(f)) { set_error("format sizes must be >= 1 with m*n, n*p, p*m <= 128 and a known mode"); return TFG_EINVAL; }
    std::vector<HTerm> t;
    int rc = parse(*f, rank, rows, t);
    if (rc) return rc;
    if (!brent_ok(*f, t)) { set_error("scheme does not satisfy the Brent equations"); return TFG_ESCHEME; }
    return TFG_OK;
}

// Normalise (Z_T), verify, and copy a result into the caller's buffer.
static int finish(Dense &d, tfg_format *out_fmt, int8_t *out, int cap, int *out_rank) {
    std::vector<int8_t> rows = to_rows(d);
    std::vector<HTerm> t;
    int rc = parse(d.f, d.r, rows.data(), t);
    if (rc) { set_error("internal: result coefficient outside the set"); return TFG_EINTERNAL; }
    for (HTerm &h : t) canon_term(d.f, h);
    if (!brent_ok(d.f, t)) { set_error("internal: meta operator result fails Eq. (1)"); return TFG_EINTERNAL; }
    if (out_fmt) *out_fmt = d.f;
    if (out_rank) *out_rank = d.r;
    if (d.r > cap) { set_error("output buffer holds " + std::to_string(cap) + " terms, result has " + std::to_string(d.r)); return TFG_ENOSPC; }
    if (d.r > 0 && !out) { set_error("null output buffer"); return TFG_EINVAL; }
    emit(d.f, t, out);
    return TFG_OK;
}

int project(const tfg_format *f, int r, const int8_t *rows, int axis, int index, tfg_format *of, int8_t *out,
            int cap, int *orank) {
    int rc = check_input(f, r, rows);
    if (rc) return rc;
    const int dim = axis == 0 ? f->m : (axis == 1 ? f->n : f->p);
    if (axis < 0 || axis > 2 || index < 0 || index >= dim || dim < 2) { set_error("bad axis/index for project"); return TFG_EINVAL; }
    Dense s = to_dense(*f, r, rows);
    tfg_format nf = *f;
    (axis == 0 ? nf.m : (axis == 1 ? nf.n : nf.p)) -= 1;
    // keep terms whose projected factors are all non-zero, in order
    Dense tmp(nf, r);
    int nr = 0;
    for (int l = 0; l < r; ++l) {
        bool nzu = false, nzv = false, nzw = false;
        for (int i = 0, ii = 0; i < f->m; ++i) {
            if (axis == 0 && i == index) continue;
            for (int k = 0, kk = 0; k < f->n; ++k) {
                if (axis == 1 && k == index) continue;
                tmp.u(nr, ii, kk) = s.u(l, i, k);
                nzu |= s.u(l, i, k) != 0;
                ++kk;
            }
            ++ii;
        }
        for (int k = 0, kk = 0; k < f->n; ++k) {
            if (axis == 1 && k == index) continue;
            for (int j = 0, jj = 0; j < f->p; ++j) {
                if (axis == 2 && j == index) continue;
                tmp.v(nr, kk, jj) = s.v(l, k, j);
                nzv |= s.v(l, k, j) != 0;
                ++jj;
            }
            ++kk;
        }
        for (int j = 0, jj = 0; j < f->p; ++j) {
            if (axis == 2 && j == index) continue;
            for (int i = 0, ii = 0; i < f->m; ++i) {
                if (axis == 0 && i == index) continue;
                tmp.w(nr, jj, ii) = s.w(l, j, i);
                nzw |= s.w(l, j, i) != 0;
                ++ii;
            }
            ++jj;
        }
        if (nzu && nzv && nzw) {
            ++nr;
        } else {  // clear the partially written row for reuse
            for (int i = 0; i < nf.m; ++i) for (int k = 0; k < nf.n; ++k) tmp.u(nr, i, k) = 0;
            for (int k = 0; k < nf.n; ++k) for (int j = 0; j < nf.p; ++j) tmp.v(nr, k, j) = 0;
            for (int j = 0; j < nf.p; ++j) for (int i = 0; i < nf.m; ++i) tmp.w(nr, j, i) = 0;
        }
    }
    Dense res(nf, nr);
    std::copy(tmp.U.begin(), tmp.U.begin() + (size_t)nr * nf.m * nf.n, res.U.begin());
    std::copy(tmp.V.begin(), tmp.V.begin() + (size_t)nr * nf.n * nf.p, res.V.begin());
    std::copy(tmp.W.begin(), tmp.W.begin() + (size_t)nr * nf.p * nf.m, res.W.begin());
    return finish(res, of, out, cap, orank);
}

static Dense naive_dense(const tfg_format &f) {
    Dense d(f, f.m * f.n * f.p);
    int l = 0;
    for (int i = 0; i < f.m; ++i)
        for (int k = 0; k < f.n; ++k)
            for (int j = 0; j < f.p; ++j) {
                d.u(l, i, k) = 1; d.v(l, k, j) = 1; d.w(l, j, i) = 1;
                ++l;
            }
    return d;
}

static bool merge_dense(const Dense &a, const Dense &b, int axis, Dense &res) {
    const tfg_format &fa = a.f, &fb = b.f;
    tfg_format nf = fa;
    if (axis == 0) { if (fa.n != fb.n || fa.p != fb.p) return false; nf.m = fa.m + fb.m; }
    else if (axis == 1) { if (fa.m != fb.m || fa.p != fb.p) return false; nf.n = fa.n + fb.n; }
    else { if (fa.m != fb.m || fa.n != fb.n) return false; nf.p = fa.p + fb.p; }
    if (nf.m * nf.n > 64 || nf.n * nf.p > 64 || nf.p * nf.m > 64) return false;
    res = Dense(nf, a.r + b.r);
    Dense &A = const_cast<Dense &>(a), &B = const_cast<Dense &>(b);
    for (int l = 0; l < a.r; ++l) {
        for (int i = 0; i < fa.m; ++i) for (int k = 0; k < fa.n; ++k) res.u(l, i, k) = A.u(l, i, k);
        for (int k = 0; k < fa.n; ++k) for (int j = 0; j < fa.p; ++j) res.v(l, k, j) = A.v(l, k, j);
        for (int j = 0; j < fa.p; ++j) for (int i = 0; i < fa.m; ++i) res.w(l, j, i) = A.w(l, j, i);
    }
    const int oi = axis == 0 ? fa.m : 0, ok = axis == 1 ? fa.n : 0, oj = axis == 2 ? fa.p : 0;
    for (int l = 0; l < b.r; ++l) {
        const int L = a.r + l;
        for (int i = 0; i < fb.m; ++i) for (int k = 0; k < fb.n; ++k) res.u(L, oi + i, ok + k) = B.u(l, i, k);
        for (int k = 0; k < fb.n; ++k) for (int j = 0; j < fb.p; ++j) res.v(L, ok + k, oj + j) = B.v(l, k, j);
        for (int j = 0; j < fb.p; ++j) for (int i = 0; i < fb.m; ++i) res.w(L, oj + j, oi + i) = B.w(l, j, i);
    }
    return true;
}

int merge(const tfg_format *fa, int ra, const int8_t *sa, const tfg_format *fb, int rb, const int8_t *sb, int axis,
          tfg_format *of, int8_t *out, int cap, int *orank) {
    int rc = check_input(fa, ra, sa);
    if (rc) return rc;
    rc = check_input(fb, rb, sb);
    if (rc) return rc;
    if (fa->mode != fb->mode || axis < 0 || axis > 2) { set_error("merge: modes differ or bad axis"); return TFG_EINVAL; }
    Dense a = to_dense(*fa, ra, sa), b = to_dense(*fb, rb, sb), res(*fa, 0);
    if (!merge_dense(a, b, axis, res)) { set_error("merge: sizes do not match along the other axes or exceed 64"); return TFG_EINVAL; }
    return finish(res, of, out, cap, orank);
}

int extend(const tfg_format *f, int r, const int8_t *rows, int axis, tfg_format *of, int8_t *out, int cap,
           int *orank) {
    int rc = check_input(f, r, rows);
    if (rc) return rc;
    if (axis < 0 || axis > 2) { set_error("bad axis"); return TFG_EINVAL; }
    tfg_format blk = *f;
    (axis == 0 ? blk.m : (axis == 1 ? blk.n : blk.p)) = 1;
    Dense a = to_dense(*f, r, rows), b = naive_dense(blk), res(*f, 0);
    if (!merge_dense(a, b, axis, res)) { set_error("extend: result exceeds 64 entries per factor"); return TFG_EINVAL; }
    return finish(res, of, out, cap, orank);
}

int product(const tfg_format *fa, int ra, const int8_t *sa, const tfg_format *fb, int rb, const int8_t *sb,
            tfg_format *of, int8_t *out, int cap, int *orank) {
    int rc = check_input(fa, ra, sa);
    if (rc) return rc;
    rc = check_input(fb, rb, sb);
    if (rc) return rc;
    if (fa->mode != fb->mode) { set_error("product: modes differ"); return TFG_EINVAL; }
    tfg_format nf{fa->m * fb->m, fa->n * fb->n, fa->p * fb->p, fa->mode};
    if (!format_ok(&nf)) { set_error("product: result exceeds 64 entries per factor"); return TFG_EINVAL; }
    if ((int64_t)ra * rb > (1 << 20)) { set_error("product: rank too large"); return TFG_EINVAL; }
    Dense A = to_dense(*fa, ra, sa), B = to_dense(*fb, rb, sb), res(nf, ra * rb);
    const int m2 = fb->m, n2 = fb->n, p2 = fb->p;
    for (int l1 = 0; l1 < ra; ++l1)
        for (int l2 = 0; l2 < rb; ++l2) {
            const int l = l1 * rb + l2;
            for (int i1 = 0; i1 < fa->m; ++i1) for (int i2 = 0; i2 < m2; ++i2)
                for (int k1 = 0; k1 < fa->n; ++k1) for (int k2 = 0; k2 < n2; ++k2)
                    res.u(l, i1 * m2 + i2, k1 * n2 + k2) = (int8_t)(A.u(l1, i1, k1) * B.u(l2, i2, k2));
            for (int k1 = 0; k1 < fa->n; ++k1) for (int k2 = 0; k2 < n2; ++k2)
                for (int j1 = 0; j1 < fa->p; ++j1) for (int j2 = 0; j2 < p2; ++j2)
                    res.v(l, k1 * n2 + k2, j1 * p2 + j2) = (int8_t)(A.v(l1, k1, j1) * B.v(l2, k2, j2));
            for (int j1 = 0; j1 < fa->p; ++j1) for (int j2 = 0; j2 < p2; ++j2)
                for (int i1 = 0; i1 < fa->m; ++i1) for (int i2 = 0; i2 < m2; ++i2)
                    res.w(l, j1 * p2 + j2, i1 * m2 + i2) = (int8_t)(A.w(l1, j1, i1) * B.w(l2, j2, i2));
        }
    return finish(res, of, out, cap, orank);
}

// (AB)^T = B^T A^T: (m,n,p) -> (p,n,m) with u' = v^T, v' = u^T, w' = w^T.
static Dense transpose_dense(Dense &s) {
    tfg_format nf{s.f.p, s.f.n, s.f.m, s.f.mode};
    Dense d(nf, s.r);
    for (int l = 0; l < s.r; ++l) {
        for (int k = 0; k < s.f.n; ++k) for (int j = 0; j < s.f.p; ++j) d.u(l, j, k) = s.v(l, k, j);
        for (int i = 0; i < s.f.m; ++i) for (int k = 0; k < s.f.n; ++k) d.v(l, k, i) = s.u(l, i, k);
        for (int j = 0; j < s.f.p; ++j) for (int i = 0; i < s.f.m; ++i) d.w(l, i, j) = s.w(l, j, i);
    }
    return d;
}

// Cyclic symmetry of the C^T tensor: (u, v, w) -> (v, w, u) maps (m,n,p) to (n,p,m).
static Dense cycle_dense(Dense &s) {
    tfg_format nf{s.f.n, s.f.p, s.f.m, s.f.mode};
    Dense d(nf, s.r);
    d.U = s.V;
    d.V = s.W;
    d.W = s.U;
    return d;
}

int swap_sizes(const tfg_format *f, int r, const int8_t *rows, int perm, tfg_format *of, int8_t *out, int cap,
               int *orank) {
    int rc = check_input(f, r, rows);
    if (rc) return rc;
    // perm -> (transpose?, number of cycles): result order of (m, n, p)
    // 0 (m,n,p): (0,0)  1 (m,p,n): (1,2)  2 (n,m,p): (1,1)  3 (n,p,m): (0,1)  4 (p,m,n): (0,2)  5 (p,n,m): (1,0)
    static const int TR[6] = {0, 1, 1, 0, 0, 1}, CY[6] = {0, 2, 1, 1, 2, 0};
    if (perm < 0 || perm > 5) { set_error("perm must be 0..5"); return TFG_EINVAL; }
    Dense d = to_dense(*f, r, rows);
    if (TR[perm]) d = transpose_dense(d);
    for (int c = 0; c < CY[perm]; ++c) d = cycle_dense(d);
    return finish(d, of, out, cap, orank);
}

// ---- isotropy invariants: matrix ranks of the factors
// Over Q: fraction-free (Bareiss) elimination on integers; every intermediate
// is a minor of the matrix, at most 8^4 in size for an 8 x 8 matrix of
// entries in {-1, 0, 1}.  Over GF(2): elimination on row bit masks.
int factor_rank(const tfg_format &f, const HTerm &h, int x) {
    const int rows = x == 0 ? f.m : (x == 1 ? f.n : f.p);
    const int cols = x == 0 ? f.n : (x == 1 ? f.p : f.m);
    if (f.mode == TFG_MODE_Z2) {
        std::vector<uint64_t> r((size_t)rows, 0);
        for (int a = 0; a < rows; ++a)
            for (int b = 0; b < cols; ++b)
                if (h.p[x].bit(a * cols + b)) r[(size_t)a] |= 1ull << b;
        int rank = 0;
        for (int c = 0; c < cols && rank < rows; ++c) {
            int piv = -1;
            for (int a = rank; a < rows; ++a)
                if ((r[(size_t)a] >> c) & 1) { piv = a; break; }
            if (piv < 0) continue;
            std::swap(r[(size_t)rank], r[(size_t)piv]);
            for (int a = 0; a < rows; ++a)
                if (a != rank && ((r[(size_t)a] >> c) & 1)) r[(size_t)a] ^= r[(size_t)rank];
            ++rank;
        }
        return rank;
    }
    std::vector<int64_t> M((size_t)rows * cols, 0);
    for (int a = 0; a < rows; ++a)
        for (int b = 0; b < cols; ++b) {
            const int e = a * cols + b;
            M[(size_t)a * cols + b] = (int64_t)h.p[x].bit(e) - (int64_t)h.n[x].bit(e);
        }
    int rank = 0;
    int64_t prev = 1;
    for (int c = 0; c < cols && rank < rows; ++c) {
        int piv = -1;
        for (int a = rank; a < rows; ++a)
            if (M[(size_t)a * cols + c] != 0) { piv = a; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int b = 0; b < cols; ++b) std::swap(M[(size_t)piv * cols + b], M[(size_t)rank * cols + b]);
        const int64_t pv = M[(size_t)rank * cols + c];
        for (int a = rank + 1; a < rows; ++a) {
            const int64_t f0 = M[(size_t)a * cols + c];
            for (int b = 0; b < cols; ++b)
                M[(size_t)a * cols + b] = (pv * M[(size_t)a * cols + b] - f0 * M[(size_t)rank * cols + b]) / prev;
        }
        prev = pv;
        ++rank;
    }
    return rank;
}

}  // namespace host
}  // namespace tfg
