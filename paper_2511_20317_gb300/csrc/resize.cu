// Resize on the device: one meta operator of Section 3.3.2 (project, extend,
// double, merge, product, swap of sizes) applied to many walkers' schemes at
// once, each result written into a walker of the population of the result
// format (the Resize step of the exploratory search, Section 3.4).
//
// Every operator is a coefficient re-indexing of the source term (product: of
// a source and an aux term, multiplied): the host builds, per block of output
// terms, a map from each output coefficient to a source (and aux) coefficient
// in the u | v | w row layout, and the kernel evaluates it term by term,
// restores the sign normalisation (Section 3.6), drops terms with a zero
// factor (project), and packs the terms into the destination's slot layout.
#include <cstdint>
#include <vector>

#include "tfg_internal.h"

namespace tfg {

// ---------------------------------------------------------------------------
// Host: coefficient maps.  Row layout of a term of (m, n, p): u[i*n + k] at 0,
// v[k*p + j] at m*n, w[j*m + i] at m*n + n*p.
namespace {

struct Fmt {
    int m, n, p;
    int lu() const { return m * n; }
    int lv() const { return n * p; }
    int lt() const { return m * n + n * p + p * m; }
    int iu(int i, int k) const { return i * n + k; }
    int iv(int k, int j) const { return lu() + k * p + j; }
    int iw(int j, int i) const { return lu() + lv() + j * m + i; }
};

// block concatenation along `axis`: out = (a | b); maps of a's and b's terms
void merge_maps(const Fmt &a, const Fmt &b, int axis, Fmt &o, std::vector<int16_t> &ma, std::vector<int16_t> &mb) {
    o = Fmt{a.m + (axis == 0 ? b.m : 0), a.n + (axis == 1 ? b.n : 0), a.p + (axis == 2 ? b.p : 0)};
    const int oi = axis == 0 ? a.m : 0, ok = axis == 1 ? a.n : 0, oj = axis == 2 ? a.p : 0;
    ma.assign(o.lt(), -1);
    mb.assign(o.lt(), -1);
    for (int i = 0; i < o.m; ++i)
        for (int k = 0; k < o.n; ++k) {
            if (i < a.m && k < a.n) ma[o.iu(i, k)] = (int16_t)a.iu(i, k);
            if (i >= oi && i < oi + b.m && k >= ok && k < ok + b.n) mb[o.iu(i, k)] = (int16_t)b.iu(i - oi, k - ok);
        }
    for (int k = 0; k < o.n; ++k)
        for (int j = 0; j < o.p; ++j) {
            if (k < a.n && j < a.p) ma[o.iv(k, j)] = (int16_t)a.iv(k, j);
            if (k >= ok && k < ok + b.n && j >= oj && j < oj + b.p) mb[o.iv(k, j)] = (int16_t)b.iv(k - ok, j - oj);
        }
    for (int j = 0; j < o.p; ++j)
        for (int i = 0; i < o.m; ++i) {
            if (j < a.p && i < a.m) ma[o.iw(j, i)] = (int16_t)a.iw(j, i);
            if (j >= oj && j < oj + b.p && i >= oi && i < oi + b.m) mb[o.iw(j, i)] = (int16_t)b.iw(j - oj, i - oi);
        }
}

// remove index `idx` along `axis`
void project_map(const Fmt &f, int axis, int idx, Fmt &o, std::vector<int16_t> &mp) {
    o = Fmt{f.m - (axis == 0), f.n - (axis == 1), f.p - (axis == 2)};
    auto src = [&](int x, int ax) { return (axis == ax && x >= idx) ? x + 1 : x; };
    mp.assign(o.lt(), -1);
    for (int i = 0; i < o.m; ++i)
        for (int k = 0; k < o.n; ++k) mp[o.iu(i, k)] = (int16_t)f.iu(src(i, 0), src(k, 1));
    for (int k = 0; k < o.n; ++k)
        for (int j = 0; j < o.p; ++j) mp[o.iv(k, j)] = (int16_t)f.iv(src(k, 1), src(j, 2));
    for (int j = 0; j < o.p; ++j)
        for (int i = 0; i < o.m; ++i) mp[o.iw(j, i)] = (int16_t)f.iw(src(j, 2), src(i, 0));
}

// Kronecker product: row index i = i1*m2 + i2, and so on for k and j
void product_maps(const Fmt &a, const Fmt &b, Fmt &o, std::vector<int16_t> &ma, std::vector<int16_t> &mb) {
    o = Fmt{a.m * b.m, a.n * b.n, a.p * b.p};
    ma.assign(o.lt(), -1);
    mb.assign(o.lt(), -1);
    for (int i1 = 0; i1 < a.m; ++i1)
        for (int i2 = 0; i2 < b.m; ++i2)
            for (int k1 = 0; k1 < a.n; ++k1)
                for (int k2 = 0; k2 < b.n; ++k2) {
                    const int e = o.iu(i1 * b.m + i2, k1 * b.n + k2);
                    ma[e] = (int16_t)a.iu(i1, k1);
                    mb[e] = (int16_t)b.iu(i2, k2);
                }
    for (int k1 = 0; k1 < a.n; ++k1)
        for (int k2 = 0; k2 < b.n; ++k2)
            for (int j1 = 0; j1 < a.p; ++j1)
                for (int j2 = 0; j2 < b.p; ++j2) {
                    const int e = o.iv(k1 * b.n + k2, j1 * b.p + j2);
                    ma[e] = (int16_t)a.iv(k1, j1);
                    mb[e] = (int16_t)b.iv(k2, j2);
                }
    for (int j1 = 0; j1 < a.p; ++j1)
        for (int j2 = 0; j2 < b.p; ++j2)
            for (int i1 = 0; i1 < a.m; ++i1)
                for (int i2 = 0; i2 < b.m; ++i2) {
                    const int e = o.iw(j1 * b.p + j2, i1 * b.m + i2);
                    ma[e] = (int16_t)a.iw(j1, i1);
                    mb[e] = (int16_t)b.iw(j2, i2);
                }
}

// (AB)^T = B^T A^T: (m,n,p) -> (p,n,m), u' = v^T, v' = u^T, w' = w^T
void transpose_map(const Fmt &f, Fmt &o, std::vector<int16_t> &mp) {
    o = Fmt{f.p, f.n, f.m};
    mp.assign(o.lt(), -1);
    for (int j = 0; j < f.p; ++j)
        for (int k = 0; k < f.n; ++k) mp[o.iu(j, k)] = (int16_t)f.iv(k, j);
    for (int k = 0; k < f.n; ++k)
        for (int i = 0; i < f.m; ++i) mp[o.iv(k, i)] = (int16_t)f.iu(i, k);
    // w'[j'*m' + i'] with j' < p' = m, i' < m' = p: c'_{j'i'} ... = w[i' * m + j']
    for (int jp = 0; jp < o.p; ++jp)
        for (int ip = 0; ip < o.m; ++ip) mp[o.iw(jp, ip)] = (int16_t)f.iw(ip, jp);
}

// (u, v, w) -> (v, w, u): (m,n,p) -> (n,p,m), rows unchanged
void cyclic_map(const Fmt &f, Fmt &o, std::vector<int16_t> &mp) {
    o = Fmt{f.n, f.p, f.m};
    mp.assign(o.lt(), -1);
    for (int e = 0; e < f.lv(); ++e) mp[e] = (int16_t)(f.lu() + e);
    for (int e = 0; e < f.p * f.m; ++e) mp[f.lv() + e] = (int16_t)(f.lu() + f.lv() + e);
    for (int e = 0; e < f.lu(); ++e) mp[f.lv() + f.p * f.m + e] = (int16_t)e;
}

// out[e] = first[second[e]] (second maps the output to the intermediate term)
std::vector<int16_t> compose(const std::vector<int16_t> &first, const std::vector<int16_t> &second) {
    std::vector<int16_t> r(second.size(), -1);
    for (size_t e = 0; e < second.size(); ++e) r[e] = second[e] < 0 ? (int16_t)-1 : first[second[e]];
    return r;
}

const int kSwapTargets[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// the order of the sizes after transpose^t then cyclic^c
void order_after(int t, int c, int out[3]) {
    int o[3] = {0, 1, 2};
    if (t) { const int x = o[0]; o[0] = o[2]; o[2] = x; }
    for (int q = 0; q < c; ++q) { const int x = o[0]; o[0] = o[1]; o[1] = o[2]; o[2] = x; }
    for (int q = 0; q < 3; ++q) out[q] = o[q];
}

bool swap_map(const Fmt &f, int perm, Fmt &o, std::vector<int16_t> &mp) {
    for (int t = 0; t < 2; ++t)
        for (int c = 0; c < 3; ++c) {
            int ord[3];
            order_after(t, c, ord);
            if (ord[0] != kSwapTargets[perm][0] || ord[1] != kSwapTargets[perm][1] || ord[2] != kSwapTargets[perm][2])
                continue;
            Fmt cur = f;
            std::vector<int16_t> total(f.lt());
            for (int e = 0; e < f.lt(); ++e) total[e] = (int16_t)e;
            if (t) {
                Fmt nx;
                std::vector<int16_t> m1;
                transpose_map(cur, nx, m1);
                total = compose(total, m1);
                cur = nx;
            }
            for (int q = 0; q < c; ++q) {
                Fmt nx;
                std::vector<int16_t> m1;
                cyclic_map(cur, nx, m1);
                total = compose(total, m1);
                cur = nx;
            }
            o = cur;
            mp = total;
            return true;
        }
    return false;
}

}  // namespace

// Builds the plan of one resize operator on the host (maps and blocks; the
// caller uploads maps and aux terms).  Returns false for an unsupported
// operator or argument.
bool build_resize_plan(int op, int axis, int index, const tfg_format &src, const tfg_format *aux, int aux_rank,
                       tfg_format &out, ResizePlan &plan, std::vector<int16_t> &maps) {
    const Fmt f{src.m, src.n, src.p};
    Fmt o{0, 0, 0};
    maps.clear();
    plan = ResizePlan{};
    plan.lt_src = f.lt();
    plan.mn_src = f.lu();
    plan.np_src = f.lv();
    plan.canon = src.mode == TFG_MODE_ZT;
    std::vector<int16_t> a, b;
    auto add_block = [&](int kind, const std::vector<int16_t> *ma, const std::vector<int16_t> *mb) {
        ResizeBlock &bk = plan.blk[plan.nblk++];
        bk.kind = kind;
        bk.map_a = -1;
        bk.map_b = -1;
        if (ma) { bk.map_a = (int32_t)maps.size(); maps.insert(maps.end(), ma->begin(), ma->end()); }
        if (mb) { bk.map_b = (int32_t)maps.size(); maps.insert(maps.end(), mb->begin(), mb->end()); }
    };
    const bool ax_ok = axis >= 0 && axis < 3;
    switch (op) {
    case TFG_RESIZE_PROJECT: {
        const int size = axis == 0 ? f.m : (axis == 1 ? f.n : f.p);
        if (!ax_ok || index < 0 || index >= size || size < 2) return false;
        project_map(f, axis, index, o, a);
        add_block(kResizeSrc, &a, nullptr);
        plan.drop_zero = 1;
        break;
    }
    case TFG_RESIZE_EXTEND: {
        if (!ax_ok) return false;
        const Fmt blk{axis == 0 ? 1 : f.m, axis == 1 ? 1 : f.n, axis == 2 ? 1 : f.p};
        merge_maps(f, blk, axis, o, a, b);
        add_block(kResizeSrc, &a, nullptr);
        add_block(kResizeAux, nullptr, &b);   // the naive scheme of the block, uploaded as aux
        plan.lt_aux = blk.lt();
        plan.aux_rank = blk.m * blk.n * blk.p;
        break;
    }
    case TFG_RESIZE_DOUBLE: {
        if (!ax_ok) return false;
        merge_maps(f, f, axis, o, a, b);
        add_block(kResizeSrc, &a, nullptr);
        add_block(kResizeSrc, &b, nullptr);
        break;
    }
    case TFG_RESIZE_MERGE: {
        if (!ax_ok || !aux) return false;
        const Fmt g{aux->m, aux->n, aux->p};
        const bool agree = axis == 0 ? (g.n == f.n && g.p == f.p) : axis == 1 ? (g.m == f.m && g.p == f.p)
                                                                            : (g.m == f.m && g.n == f.n);
        if (!agree) return false;
        merge_maps(f, g, axis, o, a, b);
        add_block(kResizeSrc, &a, nullptr);
        add_block(kResizeAux, nullptr, &b);
        plan.lt_aux = g.lt();
        plan.aux_rank = aux_rank;
        break;
    }
    case TFG_RESIZE_PRODUCT: {
        if (!aux) return false;
        const Fmt g{aux->m, aux->n, aux->p};
        product_maps(f, g, o, a, b);
        add_block(kResizeProduct, &a, &b);
        plan.lt_aux = g.lt();
        plan.aux_rank = aux_rank;
        break;
    }
    case TFG_RESIZE_SWAP: {
        if (index < 0 || index >= 6 || !swap_map(f, index, o, a)) return false;
        add_block(kResizeSrc, &a, nullptr);
        break;
    }
    default:
        return false;
    }
    out = tfg_format{o.m, o.n, o.p, src.mode};
    plan.lt_out = o.lt();
    plan.mn_out = o.lu();
    plan.np_out = o.lv();
    return true;
}

// ---------------------------------------------------------------------------
// Device
namespace {

constexpr int kResizeThreads = 64;

// coefficient (-1, 0, 1) at row index q of term t of a packed segment
__device__ __forceinline__ int coef_at(const SegDesc &d, const uint32_t *words, int t, int q, int mn, int np, bool zt) {
    const int f = q < mn ? 0 : (q < mn + np ? 1 : 2);
    const int e = q - (f == 0 ? 0 : (f == 1 ? mn : mn + np));
    const int64_t base = (int64_t)t * d.nws * d.word_bits;
    const int64_t bp = base + d.fbase[f] + e;
    const int pv = (words[bp >> 5] >> (bp & 31)) & 1;
    int nv = 0;
    if (zt) {
        const int64_t bn = bp + (int64_t)d.tw * d.word_bits;
        nv = (words[bn >> 5] >> (bn & 31)) & 1;
    }
    return pv - nv;
}

// output term o of the plan into row[] (lt_out int8), sign-normalised;
// returns false when a factor is zero
__device__ bool build_term(const SegDesc &s, const uint32_t *sw, int r_src, const ResizePlan &pl, int o, int8_t *row,
                           bool zt) {
    int blk = 0, loc = o;
    const int n0 = pl.blk[0].kind == kResizeAux ? pl.aux_rank : (pl.blk[0].kind == kResizeProduct ? r_src * pl.aux_rank : r_src);
    if (pl.nblk > 1 && o >= n0) { blk = 1; loc = o - n0; }
    const ResizeBlock &bk = pl.blk[blk];
    int t = -1, a = -1;
    if (bk.kind == kResizeSrc) t = loc;
    else if (bk.kind == kResizeAux) a = loc;
    else { t = loc / pl.aux_rank; a = loc - t * pl.aux_rank; }
    for (int e = 0; e < pl.lt_out; ++e) {
        int v = 1;
        if (bk.map_a >= 0) {
            const int q = pl.maps[bk.map_a + e];
            v = q < 0 ? 0 : coef_at(s, sw, t, q, pl.mn_src, pl.np_src, zt);
        }
        if (bk.map_b >= 0 && v != 0) {
            const int q = pl.maps[bk.map_b + e];
            v = q < 0 ? 0 : v * (int)pl.aux[(int64_t)a * pl.lt_aux + q];
        }
        row[e] = (int8_t)v;
    }
    // Section 3.6: first non-zero of u, then of v, made +1; w absorbs the signs
    const int lu = pl.mn_out, lv = pl.np_out;
    bool nz[3] = {false, false, false};
    for (int f = 0; f < 3; ++f) {
        const int lo = f == 0 ? 0 : (f == 1 ? lu : lu + lv), hi = f == 0 ? lu : (f == 1 ? lu + lv : pl.lt_out);
        int lead = 0;
        for (int e = lo; e < hi && lead == 0; ++e) lead = row[e];
        nz[f] = lead != 0;
        if (pl.canon && f < 2 && lead < 0) {
            for (int e = lo; e < hi; ++e) row[e] = (int8_t)-row[e];
            for (int e = lu + lv; e < pl.lt_out; ++e) row[e] = (int8_t)-row[e];
        }
    }
    return nz[0] && nz[1] && nz[2];
}

// row[] -> packed slot k of a segment (live and best)
__device__ void put_term(const SegDesc &d, uint32_t *live, uint32_t *best, int k, const int8_t *row, int mn, int np,
                         int lt, bool zt) {
    const int nw32 = d.nws * d.word_bits / 32;
    const int64_t base32 = (int64_t)k * nw32;
    uint32_t buf[24];   // at most 12 words of 64 bits per slot
    for (int q = 0; q < nw32; ++q) buf[q] = 0u;
    for (int e = 0; e < lt; ++e) {
        if (row[e] == 0) continue;
        const int f = e < mn ? 0 : (e < mn + np ? 1 : 2);
        const int ef = e - (f == 0 ? 0 : (f == 1 ? mn : mn + np));
        int64_t bit = d.fbase[f] + ef;
        if (zt && row[e] < 0) bit += (int64_t)d.tw * d.word_bits;
        buf[bit >> 5] |= 1u << (bit & 31);
    }
    for (int q = 0; q < nw32; ++q) {
        live[base32 + q] = buf[q];
        best[base32 + q] = buf[q];
    }
}

__global__ void __launch_bounds__(kResizeThreads) resize_kernel(const SegDesc src, int64_t src_first, const SegDesc dst,
                                                                int64_t dst_first, const ResizePlan pl,
                                                                unsigned long long *skipped) {
    extern __shared__ __align__(16) unsigned char rsm[];
    int *pos = reinterpret_cast<int *>(rsm);                       // [kResizeMaxTerms] output slot or -1
    int8_t *rows = reinterpret_cast<int8_t *>(pos + kResizeMaxTerms);   // [threads][lt_out]
    __shared__ int s_total, s_nnz;
    const int64_t ws = src_first + blockIdx.x, wd = dst_first + blockIdx.x;
    const bool ztm = src.tw * 2 == src.nws;   // Z_T: negative words present
    const tfg_walker_info &hs = src.hdr[ws];
    const int r_src = pl.use_best ? hs.best_r : hs.r;
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(pl.use_best ? src.best : src.slots) +
                         (size_t)ws * src.R * src.nws * (src.word_bits / 32);
    int r_raw = 0;
    for (int b = 0; b < pl.nblk; ++b)
        r_raw += pl.blk[b].kind == kResizeAux ? pl.aux_rank
                                               : (pl.blk[b].kind == kResizeProduct ? r_src * pl.aux_rank : r_src);
    if (r_src < 1 || r_src > src.R || r_raw > kResizeMaxTerms || (!pl.drop_zero && r_raw > dst.R)) {
        if (threadIdx.x == 0) atomicAdd(skipped, 1ull);
        return;
    }
    int8_t *row = rows + (size_t)threadIdx.x * pl.lt_out;
    // pass 1: which output terms stay
    for (int o = threadIdx.x; o < r_raw; o += blockDim.x) pos[o] = build_term(src, sw, r_src, pl, o, row, ztm) ? 1 : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int o = 0; o < r_raw; ++o) pos[o] = pos[o] ? c++ : -1;
        s_total = c;
        s_nnz = 0;
    }
    __syncthreads();
    const int r_new = s_total;
    if (r_new > dst.R || r_new == 0) {
        if (threadIdx.x == 0) atomicAdd(skipped, 1ull);
        return;
    }
    // pass 2: write the kept terms in order
    uint32_t *live = reinterpret_cast<uint32_t *>(dst.slots) + (size_t)wd * dst.R * dst.nws * (dst.word_bits / 32);
    uint32_t *best = reinterpret_cast<uint32_t *>(dst.best) + (size_t)wd * dst.R * dst.nws * (dst.word_bits / 32);
    int nnz = 0;
    for (int o = threadIdx.x; o < r_raw; o += blockDim.x) {
        if (pos[o] < 0) continue;
        build_term(src, sw, r_src, pl, o, row, ztm);
        for (int e = 0; e < pl.lt_out; ++e) nnz += row[e] != 0;
        put_term(dst, live, best, pos[o], row, pl.mn_out, pl.np_out, pl.lt_out, ztm);
    }
    // unused slots cleared
    const int nw32 = dst.nws * dst.word_bits / 32;
    for (int64_t q = (int64_t)r_new * nw32 + threadIdx.x; q < (int64_t)dst.R * nw32; q += blockDim.x) {
        live[q] = 0u;
        best[q] = 0u;
    }
    atomicAdd(&s_nnz, nnz);
    __syncthreads();
    if (threadIdx.x == 0) {
        tfg_walker_info &h = dst.hdr[wd];
        h.r = r_new;
        h.best_r = r_new;
        h.plateau = 0;
        h.best_t = h.t;
        h.best_nnz = (uint32_t)s_nnz;
    }
}

}  // namespace

size_t resize_smem_bytes(const ResizePlan &pl) {
    return (size_t)kResizeMaxTerms * sizeof(int) + (size_t)kResizeThreads * pl.lt_out;
}

void launch_resize(const SegDesc &src, int64_t src_first, const SegDesc &dst, int64_t dst_first, int64_t count,
                   const ResizePlan &plan, unsigned long long *d_skipped, cudaStream_t st) {
    if (count <= 0) return;
    const size_t smem = resize_smem_bytes(plan);
    cudaFuncSetAttribute(resize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    resize_kernel<<<(unsigned)count, kResizeThreads, smem, st>>>(src, src_first, dst, dst_first, plan, d_skipped);
}

}  // namespace tfg
