// C ABI of libtfg: walker contexts on one GPU plus the host scheme functions.
// Device memory is the caller's workspace; the library allocates none.
#include <algorithm>
#include <climits>
#include <mutex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "host_scheme.h"
#include "tfg_internal.h"

using tfg::host::HTerm;
using tfg::host::set_error;

namespace {

constexpr size_t kAlign = 256;
constexpr int kHistCap = 1024;
constexpr int kMaxSlots = 1023;   // per-lane match counts are packed in 10-bit fields

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Results of the small reduction kernels, at the start of the workspace.
struct Aux {
    unsigned long long argmin_key;
    int64_t sums[9];
    int32_t minmax[2];
    int64_t verify_failures;
    int32_t status;          // 1: a bounded device wait gave up (read and cleared by tfg_sync)
    int32_t status_pad;
    int64_t hist[kHistCap];
};
constexpr size_t kAuxBytes = (sizeof(Aux) + kAlign - 1) / kAlign * kAlign;

struct Segment {
    tfg_format fmt{};
    int r0 = 0, R = 0, word_bits = 32, lt = 0, tw = 1, nws = 2;
    int fbase[3] = {0, 0, 0};   // bit offset of each factor in a packed term
    int64_t n = 0, first = 0;
    size_t off_hdr = 0, off_slots = 0, off_best = 0, off_start = 0;
    const tfg::WalkVariant *var = nullptr;
    int block = 0;   // threads per block for variants whose block size the caller chooses (0: default)
    std::vector<int8_t> start_rows;
};

// Packed term geometry.  Terms of at most 64 coefficients: the coefficient
// bits of u | v | w concatenated in one word per sign (32 bits when LT <= 32).
// Longer terms: factor-aligned, factor f in word f of 64 bits per sign, or in
// words 2f and 2f+1 when a factor has more than 64 coefficients.
void set_geometry(Segment &s) {
    const int lu = s.fmt.m * s.fmt.n, lv = s.fmt.n * s.fmt.p, lw = s.fmt.p * s.fmt.m;
    s.lt = lu + lv + lw;
    if (s.lt <= 64) {
        s.word_bits = s.lt <= 32 ? 32 : 64;
        s.tw = 1;
        s.fbase[0] = 0; s.fbase[1] = lu; s.fbase[2] = lu + lv;
    } else {
        const int fw = (lu > 64 || lv > 64 || lw > 64) ? 2 : 1;
        s.word_bits = 64;
        s.tw = 3 * fw;
        for (int f = 0; f < 3; ++f) s.fbase[f] = 64 * fw * f;
    }
    s.nws = (s.fmt.mode == TFG_MODE_ZT ? 2 : 1) * s.tw;
}

// Lay out one segment at offset `off`; returns the offset past it.
size_t layout_segment(Segment &s, size_t off) {
    const size_t wb = (size_t)s.word_bits / 8;
    const size_t per = (size_t)s.R * s.nws * wb;
    s.off_hdr = off;
    off = align_up(off + (size_t)s.n * sizeof(tfg_walker_info));
    s.off_slots = off;
    off = align_up(off + (size_t)s.n * per);
    s.off_best = off;
    off = align_up(off + (size_t)s.n * per);
    s.off_start = off;
    off = align_up(off + per);
    return off;
}

int cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return TFG_ECUDA;
}

int max_factor_len(const tfg_format &f) { return std::max(f.m * f.n, std::max(f.n * f.p, f.p * f.m)); }
int min_factor_len(const tfg_format &f) { return std::min(f.m * f.n, std::min(f.n * f.p, f.p * f.m)); }

// The variant of the smallest capacity >= R for a mapping (G lanes per walker);
// at equal capacity a bit-sliced variant (fl >= the longest factor) wins, and a
// square one (every factor exactly fl) over that.
const tfg::WalkVariant *pick_variant(int mode, int bits, int tw, int G, int R, const tfg_format &fmt) {
    const int maxlen = max_factor_len(fmt), minlen = min_factor_len(fmt);
    auto score = [](const tfg::WalkVariant &x) { return (x.fl ? 1 : 0) + (x.sq ? 1 : 0); };
    int cnt = 0;
    const tfg::WalkVariant *v = tfg::walk_variants(&cnt);
    const tfg::WalkVariant *best = nullptr;
    for (int a = 0; a < cnt; ++a) {
        if (v[a].mode != mode || v[a].word_bits != bits || v[a].tw != tw || v[a].G != G) continue;
        if (v[a].capacity() < R) continue;
        if (v[a].fl && v[a].fl < maxlen) continue;
        if (v[a].sq && (minlen != v[a].fl || maxlen != v[a].fl)) continue;
        if (!best || v[a].S < best->S || (v[a].S == best->S && score(v[a]) > score(*best))) best = &v[a];
    }
    return best;
}

// The variant compiled for the same mapping and capacity as v with `block`
// threads per block, if any (else v): how tfg_params.block_threads selects the
// walkers per block of a thread-per-walker kernel.
const tfg::WalkVariant *with_block(const tfg::WalkVariant *v, int block) {
    if (!v || !v->block || v->block == block) return v;
    int cnt = 0;
    const tfg::WalkVariant *all = tfg::walk_variants(&cnt);
    for (int a = 0; a < cnt; ++a) {
        const tfg::WalkVariant &x = all[a];
        if (x.mode == v->mode && x.word_bits == v->word_bits && x.tw == v->tw && x.G == v->G &&
            x.capacity() == v->capacity() && x.fl == v->fl && x.sq == v->sq && x.block == block)
            return &x;
    }
    return v;
}

// Default mapping: one thread per walker (shared-memory slots) when such a
// variant exists for the rank; otherwise the fewest lanes per walker that keep
// at most 4 slots per lane; otherwise 32 lanes.
const tfg::WalkVariant *default_variant(int mode, int bits, int tw, int R, const tfg_format &fmt) {
    if (const tfg::WalkVariant *v = pick_variant(mode, bits, tw, 1, R, fmt)) return v;
    static const int order[4] = {4, 8, 16, 32};
    for (int G : order) {
        const tfg::WalkVariant *v = pick_variant(mode, bits, tw, G, R, fmt);
        if (v && v->S <= 4) return v;
    }
    return pick_variant(mode, bits, tw, 32, R, fmt);
}

// Window scratch of tfg_walk_window_noalloc, for callers that cannot call
// cudaMalloc: a static device array of this translation unit.  Host code only
// sees a host-side stand-in of the symbol, so its device address is looked up
// per device with cudaGetSymbolAddress.  tfg_init does that lookup for its
// device, which also loads this unit's module (and reserves the array) under
// lazy module loading, so that tfg_walk_window_noalloc itself never causes a
// device allocation.
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB, held by every GPU that loads the library
__device__ __align__(256) unsigned char g_window_scratch[kNoAllocScratchBytes];
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

int window_scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) { set_error("device index beyond 64"); return TFG_EINVAL; }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_window_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TFG_OK;
}

}  // namespace

struct tfg_ctx {
    // one captured graph per launch step count: fork to one stream per population, join
    struct Graph { int32_t steps; cudaGraphExec_t exec; };
    std::vector<Graph> graphs;
    std::vector<cudaStream_t> fork_streams;   // [0] carries the graph, [1 + f] population f
    std::vector<cudaEvent_t> fork_events;     // [f] join of population f, [P] fork, [P+1] / [P+2] in / out
    ~tfg_ctx() {
        for (Graph &g : graphs) cudaGraphExecDestroy(g.exec);
        for (cudaStream_t s : fork_streams) cudaStreamDestroy(s);
        for (cudaEvent_t e : fork_events) cudaEventDestroy(e);
    }
    std::vector<Segment> segs;
    tfg_params prm{};
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0, ws_used = 0;
    int64_t total = 0;
    int device = 0;

    tfg::SegDesc desc(const Segment &s) const {
        tfg::SegDesc d{};
        d.slots = ws + s.off_slots;
        d.best = ws + s.off_best;
        d.hdr = reinterpret_cast<tfg_walker_info *>(ws + s.off_hdr);
        d.n_walkers = s.n;
        d.R = s.R;
        d.m = s.fmt.m; d.n = s.fmt.n; d.p = s.fmt.p;
        d.lt = s.lt; d.tw = s.tw; d.nws = s.nws; d.word_bits = s.word_bits;
        const int len[3] = {s.fmt.m * s.fmt.n, s.fmt.n * s.fmt.p, s.fmt.p * s.fmt.m};
        for (int f = 0; f < 3; ++f) d.fbase[f] = s.fbase[f];
        for (int f = 0; f < 3; ++f)
            for (int q = 0; q < 3; ++q) {
                uint64_t mword = 0;
                for (int b = 0; b < s.word_bits; ++b) {
                    const int bit = q * s.word_bits + b;
                    if (bit >= s.fbase[f] && bit < s.fbase[f] + len[f]) mword |= 1ull << b;
                }
                d.fmask[f][q] = mword;
            }
        d.key0 = (uint32_t)seed;
        d.key1 = (uint32_t)(seed >> 32);
        d.plateau_len = prm.plateau_len;
        d.refresh_thresh = prm.refresh_thresh;
        d.plus_attempts = prm.plus_attempts;
        d.plus_enabled = prm.plus_enabled;
        d.walk_policy = prm.walk_policy;
        d.expand_thresh = prm.expand_thresh;
        return d;
    }
    Aux *aux() const { return reinterpret_cast<Aux *>(ws); }
};

extern "C" {

void tfg_default_params(tfg_params *out) {
    if (!out) return;
    std::memset(out, 0, sizeof *out);
    out->plateau_len = 10000;
    out->refresh_thresh = 42949672u;
    out->plus_attempts = 16;
    out->plus_enabled = 1;
    out->r_slack = 3;
    out->mapping = 0;
    out->block_threads = 256;
    out->walker_id_base = 0;
    out->use_graph = 1;
}

const char *tfg_last_error(void) { return tfg::host::last_error(); }

int tfg_verify(const tfg_format *fmt, int32_t rank, const int8_t *scheme) {
    return tfg::host::check_input(fmt, rank, scheme);
}

int tfg_additive_complexity(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int64_t *out) {
    if (!tfg::host::format_ok(fmt) || !out || rank < 0 || (rank > 0 && !scheme)) {
        set_error("bad arguments");
        return TFG_EINVAL;
    }
    const int LT = tfg::host::term_len(*fmt);
    int64_t nnz = 0;
    for (int64_t e = 0; e < (int64_t)rank * LT; ++e) nnz += scheme[e] != 0;
    *out = nnz - 2LL * rank - (int64_t)fmt->m * fmt->p;
    return TFG_OK;
}

int tfg_isotropy_invariants(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t *term_ranks,
                            int64_t *type_poly, int64_t *sym_poly, int64_t *rank_sums) {
    if (!tfg::host::format_ok(fmt)) { set_error("bad format"); return TFG_EINVAL; }
    std::vector<HTerm> t;
    int rc = tfg::host::parse(*fmt, rank, scheme, t);
    if (rc) return rc;
    constexpr int D = 12;
    if (type_poly) std::memset(type_poly, 0, sizeof(int64_t) * D * D * D);
    if (sym_poly) std::memset(sym_poly, 0, sizeof(int64_t) * D * D * D);
    int64_t sums[3] = {0, 0, 0};
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (size_t l = 0; l < t.size(); ++l) {
        int rk[3];
        for (int x = 0; x < 3; ++x) {
            rk[x] = tfg::host::factor_rank(*fmt, t[l], x);
            sums[x] += rk[x];
            if (term_ranks) term_ranks[l * 3 + x] = rk[x];
        }
        if (type_poly) type_poly[(rk[0] * D + rk[1]) * D + rk[2]] += 1;
        if (sym_poly)
            for (const auto &pm : perms) sym_poly[(rk[pm[0]] * D + rk[pm[1]]) * D + rk[pm[2]]] += 1;
    }
    if (rank_sums)
        for (int x = 0; x < 3; ++x) rank_sums[x] = sums[x];
    return TFG_OK;
}

int tfg_lift_signs(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int64_t max_nodes, int8_t *out,
                   int64_t *nodes_used) {
    if (!fmt || !out || rank < 1 || !scheme || max_nodes < 0) { set_error("bad arguments"); return TFG_EINVAL; }
    tfg_format f = *fmt;
    f.mode = TFG_MODE_Z2;
    if (!tfg::host::format_ok(&f)) { set_error("bad format"); return TFG_EINVAL; }
    const int LT = tfg::host::term_len(f);
    for (int64_t e = 0; e < (int64_t)rank * LT; ++e)
        if (scheme[e] != 0 && scheme[e] != 1) { set_error("coefficients of a Z_2 scheme must be 0 or 1"); return TFG_EINVAL; }
    int rc = tfg::host::check_input(&f, rank, scheme);
    if (rc == TFG_ESCHEME) { set_error("not a Z_2 scheme (Eq. (1) fails modulo 2)"); return TFG_EINVAL; }
    if (rc) return rc;
    std::vector<int8_t> res((size_t)rank * LT);
    rc = tfg::host::lift_signs(f, rank, scheme, max_nodes, res.data(), nodes_used);
    if (rc) return rc;
    tfg_format ft = f;
    ft.mode = TFG_MODE_ZT;
    std::vector<HTerm> t;
    if (tfg::host::parse(ft, rank, res.data(), t) != TFG_OK || !tfg::host::brent_ok(ft, t)) {
        set_error("internal: lifted scheme fails Eq. (1)");
        return TFG_EINTERNAL;
    }
    for (HTerm &h : t) tfg::host::canon_term(ft, h);
    tfg::host::emit(ft, t, out);
    return TFG_OK;
}

int tfg_canonicalize(const tfg_format *fmt, int32_t rank, int8_t *scheme) {
    if (!tfg::host::format_ok(fmt)) { set_error("bad format"); return TFG_EINVAL; }
    std::vector<HTerm> t;
    int rc = tfg::host::parse(*fmt, rank, scheme, t);
    if (rc) return rc;
    for (HTerm &h : t) tfg::host::canon_term(*fmt, h);
    tfg::host::emit(*fmt, t, scheme);
    return TFG_OK;
}

int tfg_prepare(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int8_t *out, int32_t cap,
                int32_t *out_rank) {
    int rc = tfg::host::check_input(fmt, rank, scheme);
    if (rc) return rc;
    std::vector<HTerm> t;
    tfg::host::parse(*fmt, rank, scheme, t);
    tfg::host::prepare(*fmt, t);
    if (out_rank) *out_rank = (int32_t)t.size();
    if ((int)t.size() > cap) { set_error("output buffer too small"); return TFG_ENOSPC; }
    if (!t.empty() && !out) { set_error("null output"); return TFG_EINVAL; }
    tfg::host::emit(*fmt, t, out);
    return TFG_OK;
}

int tfg_project(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t axis, int32_t index,
                tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank) {
    return tfg::host::project(fmt, rank, scheme, axis, index, out_fmt, out, cap, out_rank);
}
int tfg_extend(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t axis, tfg_format *out_fmt,
               int8_t *out, int32_t cap, int32_t *out_rank) {
    return tfg::host::extend(fmt, rank, scheme, axis, out_fmt, out, cap, out_rank);
}
int tfg_merge(const tfg_format *fa, int32_t ra, const int8_t *sa, const tfg_format *fb, int32_t rb,
              const int8_t *sb, int32_t axis, tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank) {
    return tfg::host::merge(fa, ra, sa, fb, rb, sb, axis, out_fmt, out, cap, out_rank);
}
int tfg_double(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t axis, tfg_format *out_fmt,
               int8_t *out, int32_t cap, int32_t *out_rank) {
    return tfg::host::merge(fmt, rank, scheme, fmt, rank, scheme, axis, out_fmt, out, cap, out_rank);
}
int tfg_product(const tfg_format *fa, int32_t ra, const int8_t *sa, const tfg_format *fb, int32_t rb,
                const int8_t *sb, tfg_format *out_fmt, int8_t *out, int32_t cap, int32_t *out_rank) {
    return tfg::host::product(fa, ra, sa, fb, rb, sb, out_fmt, out, cap, out_rank);
}
int tfg_swap_sizes(const tfg_format *fmt, int32_t rank, const int8_t *scheme, int32_t perm, tfg_format *out_fmt,
                   int8_t *out, int32_t cap, int32_t *out_rank) {
    return tfg::host::swap_sizes(fmt, rank, scheme, perm, out_fmt, out, cap, out_rank);
}

static int check_params(const tfg_params &p) {
    if (p.plateau_len < 1 || p.plus_attempts < 0 || p.r_slack < 1 || p.block_threads < 32 ||
        p.block_threads % 32 != 0 || p.block_threads > 256) {
        set_error("bad parameters (plateau_len >= 1, r_slack >= 1, block_threads a multiple of 32 <= 256)");
        return TFG_EINVAL;
    }
    if (p.use_graph < 0 || p.use_graph > 2) {
        set_error("use_graph must be 0 (plain launches), 1 (chained graph) or 2 (forked graph)");
        return TFG_EINVAL;
    }
    if (p.walk_policy < 0 || p.walk_policy > 2) {
        set_error("walk_policy must be 0 (plateau plus transitions), 1 (Algorithm 1 expansions) or 2 (additive "
                  "complexity minimisation)");
        return TFG_EINVAL;
    }
    if (p.mapping != 0 && p.mapping != 1 && p.mapping != 4 && p.mapping != 8 && p.mapping != 16 && p.mapping != 32) {
        set_error("mapping must be 0 (auto), 1 (thread per walker), 4, 8, 16 or 32");
        return TFG_EINVAL;
    }
    return TFG_OK;
}

static int plan_segments(int32_t n_formats, const tfg_format *fmts, const int32_t *ranks, const int64_t *walkers,
                         const tfg_params &prm, std::vector<Segment> &segs, size_t *bytes) {
    if (n_formats < 1 || !fmts || !ranks || !walkers) { set_error("need at least one population"); return TFG_EINVAL; }
    segs.assign((size_t)n_formats, Segment{});
    size_t off = kAuxBytes;
    int64_t first = 0;
    for (int f = 0; f < n_formats; ++f) {
        Segment &s = segs[f];
        if (!tfg::host::format_ok(&fmts[f])) { set_error("bad format " + std::to_string(f)); return TFG_EINVAL; }
        if (ranks[f] < 1 || walkers[f] < 0) { set_error("bad rank or walker count"); return TFG_EINVAL; }
        s.fmt = fmts[f];
        s.r0 = ranks[f];
        s.R = ranks[f] + prm.r_slack;
        if (s.R > kMaxSlots) { set_error("rank + slack exceeds the supported 1023 slots"); return TFG_EINVAL; }
        set_geometry(s);
        s.n = walkers[f];
        s.first = first;
        first += s.n;
        if (first > (int64_t)UINT32_MAX) { set_error("more than 2^32 walkers"); return TFG_EINVAL; }
        off = layout_segment(s, off);
        s.var = prm.mapping ? pick_variant(s.fmt.mode, s.word_bits, s.tw, prm.mapping, s.R, s.fmt)
                            : default_variant(s.fmt.mode, s.word_bits, s.tw, s.R, s.fmt);
        s.var = with_block(s.var, prm.block_threads);
        if (!s.var) { set_error("no compiled kernel variant for this format/rank/mapping"); return TFG_EINVAL; }
    }
    *bytes = off;
    return TFG_OK;
}

int tfg_workspace_size(int32_t n_formats, const tfg_format *fmts, const int32_t *ranks, const int64_t *walkers,
                       const tfg_params *params, size_t *bytes) {
    tfg_params prm;
    if (params) prm = *params; else tfg_default_params(&prm);
    int rc = check_params(prm);
    if (rc) return rc;
    if (!bytes) { set_error("null bytes"); return TFG_EINVAL; }
    std::vector<Segment> segs;
    return plan_segments(n_formats, fmts, ranks, walkers, prm, segs, bytes);
}

// Host term (a coefficient mask per factor and sign) -> packed slot words.
static void pack_terms(const Segment &s, const std::vector<HTerm> &t, std::vector<uint8_t> &buf) {
    const size_t wb = (size_t)s.word_bits / 8;
    buf.assign((size_t)s.R * s.nws * wb, 0);
    const int *off = s.fbase;
    const int len[3] = {s.fmt.m * s.fmt.n, s.fmt.n * s.fmt.p, s.fmt.p * s.fmt.m};
    const int signs = s.fmt.mode == TFG_MODE_ZT ? 2 : 1;
    for (size_t l = 0; l < t.size(); ++l)
        for (int sg = 0; sg < signs; ++sg) {
            std::vector<uint64_t> words((size_t)s.tw, 0);
            for (int x = 0; x < 3; ++x) {
                const tfg::host::FMask &m = sg == 0 ? t[l].p[x] : t[l].n[x];
                for (int e = 0; e < len[x]; ++e)
                    if (m.bit(e)) {
                        const int bit = off[x] + e;
                        words[bit / s.word_bits] |= 1ull << (bit % s.word_bits);
                    }
            }
            for (int q = 0; q < s.tw; ++q) {
                const size_t idx = l * s.nws + (size_t)sg * s.tw + q;
                if (wb == 4) {
                    const uint32_t v = (uint32_t)words[q];
                    std::memcpy(&buf[idx * 4], &v, 4);
                } else {
                    std::memcpy(&buf[idx * 8], &words[q], 8);
                }
            }
        }
}

static void unpack_terms(const Segment &s, const uint8_t *words, int r, int8_t *rows) {
    const size_t wb = (size_t)s.word_bits / 8;
    const int *off = s.fbase;
    const int len[3] = {s.fmt.m * s.fmt.n, s.fmt.n * s.fmt.p, s.fmt.p * s.fmt.m};
    const int signs = s.fmt.mode == TFG_MODE_ZT ? 2 : 1;
    std::vector<HTerm> t((size_t)r);
    for (int l = 0; l < r; ++l)
        for (int sg = 0; sg < signs; ++sg) {
            std::vector<uint64_t> w((size_t)s.tw, 0);
            for (int q = 0; q < s.tw; ++q) {
                const size_t idx = (size_t)l * s.nws + (size_t)sg * s.tw + q;
                if (wb == 4) { uint32_t v32; std::memcpy(&v32, words + idx * 4, 4); w[q] = v32; }
                else std::memcpy(&w[q], words + idx * 8, 8);
            }
            for (int x = 0; x < 3; ++x) {
                tfg::host::FMask m;
                for (int e = 0; e < len[x]; ++e) {
                    const int bit = off[x] + e;
                    if ((w[bit / s.word_bits] >> (bit % s.word_bits)) & 1) m.set(e);
                }
                (sg == 0 ? t[l].p[x] : t[l].n[x]) = m;
            }
        }
    tfg::host::emit(s.fmt, t, rows);
}

int tfg_init(int32_t n_formats, const tfg_format *fmts, const int32_t *ranks, const int8_t *const *schemes,
             const int64_t *walkers, uint64_t seed, const tfg_params *params, void *d_workspace,
             size_t workspace_bytes, void *cuda_stream, tfg_ctx **out) {
    if (!out) { set_error("null out"); return TFG_EINVAL; }
    *out = nullptr;
    tfg_params prm;
    if (params) prm = *params; else tfg_default_params(&prm);
    int rc = check_params(prm);
    if (rc) return rc;
    if (n_formats < 1 || !fmts || !ranks || !schemes || !walkers) { set_error("null arguments"); return TFG_EINVAL; }
    if (!d_workspace || ((uintptr_t)d_workspace % kAlign) != 0) { set_error("workspace must be 256-byte aligned device memory"); return TFG_EINVAL; }

    // validate and prepare every start on the host
    std::vector<std::vector<HTerm>> starts((size_t)n_formats);
    std::vector<int32_t> r0((size_t)n_formats);
    for (int f = 0; f < n_formats; ++f) {
        rc = tfg::host::check_input(&fmts[f], ranks[f], schemes[f]);
        if (rc) return rc;
        tfg::host::parse(fmts[f], ranks[f], schemes[f], starts[f]);
        tfg::host::prepare(fmts[f], starts[f]);
        r0[f] = (int32_t)starts[f].size();
        if (r0[f] < 1) { set_error("prepared start is empty"); return TFG_ESCHEME; }
    }
    auto *ctx = new tfg_ctx();
    ctx->prm = prm;
    ctx->seed = seed;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    ctx->ws = reinterpret_cast<char *>(d_workspace);
    ctx->ws_bytes = workspace_bytes;
    rc = plan_segments(n_formats, fmts, r0.data(), walkers, prm, ctx->segs, &ctx->ws_used);
    if (rc) { delete ctx; return rc; }
    if (ctx->ws_used > workspace_bytes) {
        set_error("workspace holds " + std::to_string(workspace_bytes) + " bytes, need " + std::to_string(ctx->ws_used));
        delete ctx;
        return TFG_ENOMEM;
    }
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "cudaGetDevice"); }
    {
        void *scratch = nullptr;   // load the static window scratch on this device now (see above)
        rc = window_scratch_address(ctx->device, &scratch);
        if (rc) { delete ctx; return rc; }
    }
    e = cudaMemsetAsync(&ctx->aux()->status, 0, sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "clear status"); }
    for (int f = 0; f < n_formats; ++f) {
        Segment &s = ctx->segs[f];
        s.first = (f == 0) ? 0 : ctx->segs[f - 1].first + ctx->segs[f - 1].n;
        s.start_rows.resize((size_t)r0[f] * tfg::host::term_len(s.fmt));
        tfg::host::emit(s.fmt, starts[f], s.start_rows.data());
        std::vector<uint8_t> buf;
        pack_terms(s, starts[f], buf);
        e = cudaMemcpyAsync(ctx->ws + s.off_start, buf.data(), buf.size(), cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "copy start"); }
        uint32_t nnz = 0;
        for (int8_t c : s.start_rows) nnz += c != 0;
        tfg::launch_replicate(ctx->desc(s), ctx->ws + s.off_start, s.r0, prm.walker_id_base + (uint32_t)s.first, f,
                              nnz, ctx->stream);
        e = cudaGetLastError();
        if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "replicate launch"); }
    }
    ctx->total = ctx->segs.back().first + ctx->segs.back().n;
    *out = ctx;
    return TFG_OK;
}

static int block_of(const tfg_ctx *ctx, const Segment &s) {
    return s.var->block ? s.var->block : (s.block ? s.block : ctx->prm.block_threads);
}

static void launch_segment(tfg_ctx *ctx, const Segment &s, int32_t steps, cudaStream_t st) {
    const int b = block_of(ctx, s);
    const int64_t threads = s.n * s.var->G;
    const int64_t grid = (threads + b - 1) / b;
    s.var->launch(ctx->desc(s), steps, (int)grid, b, st);
}

// Streams and events of the forked launch: [0] the origin, [1 + f] population f.
static int ensure_fork_resources(tfg_ctx *ctx) {
    const size_t P = ctx->segs.size();
    cudaError_t e = cudaSuccess;
    while (ctx->fork_streams.size() < P + 1 && e == cudaSuccess) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) ctx->fork_streams.push_back(s);
    }
    while (ctx->fork_events.size() < P + 3 && e == cudaSuccess) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) ctx->fork_events.push_back(ev);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fork streams");
    return TFG_OK;
}

// Capture (once per step count) a graph of every population's walk kernel:
// chained on one stream (use_graph 1), or forked into one stream per
// population and joined (use_graph 2).
// The capture origin is a private stream (the caller's stream may be the
// legacy default stream, which cannot be captured).
static int walk_graph(tfg_ctx *ctx, int32_t steps, cudaGraphExec_t *out) {
    for (const tfg_ctx::Graph &g : ctx->graphs)
        if (g.steps == steps) { *out = g.exec; return TFG_OK; }
    const size_t P = ctx->segs.size();
    int rc = ensure_fork_resources(ctx);
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    for (const Segment &s : ctx->segs)
        if (s.var->prepare) s.var->prepare();   // kernel attributes are set outside the capture
    cudaStream_t origin = ctx->fork_streams[0];
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    if (ctx->prm.use_graph == 2) {
        // forked: every population on its own branch, all concurrent
        cudaEventRecord(ctx->fork_events[P], origin);
        for (size_t f = 0; f < P; ++f) {
            cudaStream_t sf = ctx->fork_streams[1 + f];
            cudaStreamWaitEvent(sf, ctx->fork_events[P], 0);
            if (ctx->segs[f].n > 0) launch_segment(ctx, ctx->segs[f], steps, sf);
            cudaEventRecord(ctx->fork_events[f], sf);
            cudaStreamWaitEvent(origin, ctx->fork_events[f], 0);
        }
    } else {
        // chained: the populations one after another inside the one graph
        for (size_t f = 0; f < P; ++f)
            if (ctx->segs[f].n > 0) launch_segment(ctx, ctx->segs[f], steps, origin);
    }
    e = cudaStreamEndCapture(origin, &graph);
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    ctx->graphs.push_back({steps, exec});
    *out = exec;
    return TFG_OK;
}

int tfg_walk(tfg_ctx *ctx, int64_t steps) {
    if (!ctx || steps < 0) { set_error("bad arguments"); return TFG_EINVAL; }
    while (steps > 0) {
        const int32_t chunk = (int32_t)std::min<int64_t>(steps, 1 << 30);
        if (ctx->prm.use_graph) {
            cudaGraphExec_t exec = nullptr;
            int rc = walk_graph(ctx, chunk, &exec);
            if (rc) return rc;
            const size_t P = ctx->segs.size();
            cudaStream_t origin = ctx->fork_streams[0];
            // order the graph after the context stream's work, and that stream after the graph
            cudaError_t e = cudaEventRecord(ctx->fork_events[P + 1], ctx->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ctx->fork_events[P + 1], 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, origin);
            if (e == cudaSuccess) e = cudaEventRecord(ctx->fork_events[P + 2], origin);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->fork_events[P + 2], 0);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        } else {
            for (const Segment &s : ctx->segs)
                if (s.n > 0) launch_segment(ctx, s, chunk, ctx->stream);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "walk launch");
        }
        steps -= chunk;
    }
    return TFG_OK;
}

int tfg_autotune(tfg_ctx *ctx, int64_t trial_steps, int64_t trial_walkers, int32_t *lanes_out) {
    if (!ctx || trial_steps < 1 || trial_walkers < 1) { set_error("bad arguments"); return TFG_EINVAL; }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    // timing events, released on every return path
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    e = cudaEventCreate(&ev.a);
    if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
    if (e != cudaSuccess) return cuda_fail(e, "autotune events");
    const size_t P = ctx->segs.size();
    int nvar = 0;
    const tfg::WalkVariant *all = tfg::walk_variants(&nvar);

    // the trial walkers (the first min(walkers, trial_walkers) of each population), saved on the host
    struct Saved { std::vector<char> hdr, sl, be; int64_t nt = 0; size_t per = 0; };
    std::vector<Saved> saved(P);
    for (size_t f = 0; f < P; ++f) {
        Segment &s = ctx->segs[f];
        Saved &sv = saved[f];
        sv.nt = std::min<int64_t>(s.n, trial_walkers);
        sv.per = (size_t)s.R * s.nws * (s.word_bits / 8);
        sv.hdr.resize(sizeof(tfg_walker_info) * sv.nt);
        sv.sl.resize(sv.per * sv.nt);
        sv.be.resize(sv.per * sv.nt);
        e = cudaMemcpy(sv.hdr.data(), ctx->ws + s.off_hdr, sv.hdr.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sv.sl.data(), ctx->ws + s.off_slots, sv.sl.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sv.be.data(), ctx->ws + s.off_best, sv.be.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "autotune save");
    }
    // candidates of every population: every mapping (lanes per walker) at its smallest
    // capacity, and for each every walkers-per-block choice (the block sizes compiled for a
    // thread-per-walker kernel of that capacity, whose shared memory per block depends on it;
    // 128 or 256 threads for the lane-group kernels)
    struct Choice { const tfg::WalkVariant *var; int block; };
    std::vector<std::vector<Choice>> cand(P);
    static const int lanes[5] = {1, 4, 8, 16, 32};
    for (size_t f = 0; f < P; ++f) {
        const Segment &s = ctx->segs[f];
        for (int G : lanes) {
            const tfg::WalkVariant *base = pick_variant(s.fmt.mode, s.word_bits, s.tw, G, s.R, s.fmt);
            if (!base) continue;
            for (int a = 0; a < nvar; ++a) {
                const tfg::WalkVariant &v = all[a];
                if (v.mode != base->mode || v.word_bits != base->word_bits || v.tw != base->tw || v.G != base->G ||
                    v.capacity() != base->capacity() || v.fl != base->fl || v.sq != base->sq)
                    continue;
                if (v.block) cand[f].push_back({&v, 0});
                else { cand[f].push_back({&v, 128}); cand[f].push_back({&v, 256}); }
            }
        }
    }
    // Put the trial walkers back into their saved state (before every timed trial, so
    // that every candidate is timed from the same point of the walk: the cost of a step
    // changes along a trajectory).
    auto restore_state = [&]() -> cudaError_t {
        cudaError_t r = cudaSuccess;
        for (size_t f = 0; f < P && r == cudaSuccess; ++f) {
            const Segment &s = ctx->segs[f];
            const Saved &sv = saved[f];
            r = cudaMemcpy(ctx->ws + s.off_hdr, sv.hdr.data(), sv.hdr.size(), cudaMemcpyHostToDevice);
            if (r == cudaSuccess) r = cudaMemcpy(ctx->ws + s.off_slots, sv.sl.data(), sv.sl.size(), cudaMemcpyHostToDevice);
            if (r == cudaSuccess) r = cudaMemcpy(ctx->ws + s.off_best, sv.be.data(), sv.be.size(), cudaMemcpyHostToDevice);
        }
        return r;
    };
    // One timed trial: `steps` steps of the trial walkers through tfg_walk itself (the
    // graph rebuilt for the current choices), so a trial is timed in the launch shape the
    // walk uses: milliseconds, or < 0 on error.  The populations are cut to their trial
    // walkers meanwhile.
    std::vector<int64_t> full_n(P);
    for (size_t f = 0; f < P; ++f) { full_n[f] = ctx->segs[f].n; ctx->segs[f].n = saved[f].nt; }
    auto restore_n = [&] { for (size_t f = 0; f < P; ++f) ctx->segs[f].n = full_n[f]; };
    auto trial = [&](int32_t steps) -> float {
        for (tfg_ctx::Graph &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
        ctx->graphs.clear();
        cudaEventRecord(ev.a, ctx->stream);
        if (tfg_walk(ctx, steps) != TFG_OK) return -1.f;
        cudaEventRecord(ev.b, ctx->stream);
        if (cudaEventSynchronize(ev.b) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev.a, ev.b);
        return ms;
    };
    // coordinate descent: population by population, every candidate timed with the other
    // populations at their current choice; a candidate replaces the current choice only
    // when it is more than 1% faster
    for (size_t f = 0; f < P; ++f) {
        Segment &s = ctx->segs[f];
        if (full_n[f] == 0 || cand[f].empty()) continue;
        const Choice cur{s.var, s.block};
        float base_ms = -1.f;
        if (trial((int32_t)std::min<int64_t>(trial_steps, 64)) < 0.f || restore_state() != cudaSuccess ||
            (base_ms = trial((int32_t)trial_steps)) < 0.f) {
            restore_n();
            return cuda_fail(cudaGetLastError(), "autotune trial");
        }
        Choice best = cur;
        float best_ms = base_ms;
        for (const Choice &c : cand[f]) {
            if (c.var == cur.var && c.block == cur.block) continue;
            s.var = c.var;
            s.block = c.block;
            float ms = trial((int32_t)std::min<int64_t>(trial_steps, 64));   // warm-up (first launch of a kernel)
            if (ms >= 0.f && restore_state() != cudaSuccess) ms = -1.f;
            if (ms >= 0.f) ms = trial((int32_t)trial_steps);
            if (ms < 0.f) {
                s.var = cur.var;
                s.block = cur.block;
                restore_n();
                return cuda_fail(cudaGetLastError(), "autotune trial");
            }
            if (ms < best_ms) { best_ms = ms; best = c; }
        }
        if (!(best_ms < 0.99f * base_ms)) best = cur;
        s.var = best.var;
        s.block = best.block;
        if (lanes_out) lanes_out[f] = best.var->G;
    }
    restore_n();
    // restore the trial walkers bit for bit
    for (size_t f = 0; f < P; ++f)
        if (lanes_out && (ctx->segs[f].n == 0 || cand[f].empty())) lanes_out[f] = ctx->segs[f].var->G;
    e = restore_state();
    if (e != cudaSuccess) return cuda_fail(e, "autotune restore");
    for (tfg_ctx::Graph &g : ctx->graphs) cudaGraphExecDestroy(g.exec);   // variants changed
    ctx->graphs.clear();
    return TFG_OK;
}

int tfg_launch_shape(tfg_ctx *ctx, int32_t f, int32_t *lanes, int32_t *block_threads, int64_t *grid) {
    if (!ctx || f < 0 || f >= (int)ctx->segs.size()) { set_error("bad population index"); return TFG_EINVAL; }
    const Segment &s = ctx->segs[f];
    const int b = block_of(ctx, s);
    if (lanes) *lanes = s.var->G;
    if (block_threads) *block_threads = b;
    if (grid) *grid = (s.n * s.var->G + b - 1) / b;
    return TFG_OK;
}

// The status word of the context: a device wait that gave up since the last
// check sets it; it is read here and cleared only after it has been read.
static int take_status(tfg_ctx *ctx) {
    int32_t status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, &ctx->aux()->status, sizeof status, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "read status");
    if (status == 0) return TFG_OK;
    e = cudaMemsetAsync(&ctx->aux()->status, 0, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
    set_error("a bounded device wait gave up (tensor-core completion of the proposal network): the scores of "
              "the window step it served are not valid");
    return TFG_ETIMEOUT;
}

int tfg_sync(tfg_ctx *ctx) {
    if (!ctx) { set_error("null ctx"); return TFG_EINVAL; }
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "device error");
    return take_status(ctx);
}

int tfg_population(tfg_ctx *ctx, int32_t f, tfg_format *fmt, int32_t *r0, int32_t *r_max, int64_t *walkers,
                   int64_t *first) {
    if (!ctx || f < 0 || f >= (int)ctx->segs.size()) { set_error("bad population index"); return TFG_EINVAL; }
    const Segment &s = ctx->segs[f];
    if (fmt) *fmt = s.fmt;
    if (r0) *r0 = s.r0;
    if (r_max) *r_max = s.R;
    if (walkers) *walkers = s.n;
    if (first) *first = s.first;
    return TFG_OK;
}

int tfg_mapping(tfg_ctx *ctx, int32_t f, int32_t *lanes, int32_t *slots_per_lane, int32_t *slice_len,
                int32_t *square) {
    if (!ctx || f < 0 || f >= (int)ctx->segs.size()) { set_error("bad population index"); return TFG_EINVAL; }
    if (lanes) *lanes = ctx->segs[f].var->G;
    if (slots_per_lane) *slots_per_lane = ctx->segs[f].var->S;
    if (slice_len) *slice_len = ctx->segs[f].var->fl;
    if (square) *square = ctx->segs[f].var->sq;
    return TFG_OK;
}

int tfg_verify_all_async(tfg_ctx *ctx, int64_t *d_failures) {
    if (!ctx || !d_failures) { set_error("bad arguments"); return TFG_EINVAL; }
    cudaError_t e = cudaMemsetAsync(d_failures, 0, sizeof(int64_t), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    for (const Segment &s : ctx->segs)
        tfg::launch_verify_best(ctx->desc(s), 0, s.n, s.fmt.mode, d_failures, ctx->stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "verify launch");
    return TFG_OK;
}

int tfg_collect_best(tfg_ctx *ctx, int32_t format_idx, int8_t *out, int32_t cap, int32_t *rank_out,
                     int64_t *walker_out) {
    if (!ctx || format_idx < 0 || format_idx >= (int)ctx->segs.size()) { set_error("bad population index"); return TFG_EINVAL; }
    const Segment &s = ctx->segs[format_idx];
    if (s.n == 0) { set_error("empty population"); return TFG_EINVAL; }
    Aux *aux = ctx->aux();
    cudaError_t e = cudaMemsetAsync(&aux->argmin_key, 0xff, sizeof(aux->argmin_key), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    const tfg::SegDesc d = ctx->desc(s);
    tfg::launch_argmin_best(d, &aux->argmin_key, ctx->stream);
    unsigned long long key = 0;
    e = cudaMemcpyAsync(&key, &aux->argmin_key, sizeof key, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy key");
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "argmin");
    const int64_t w = (int64_t)(key & 0xffffffffull);
    const int r = (int)(key >> 32);
    // device check of the chosen walker's best scheme
    e = cudaMemsetAsync(&aux->verify_failures, 0, sizeof(int64_t), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    tfg::launch_verify_best(d, w, 1, s.fmt.mode, &aux->verify_failures, ctx->stream);
    const size_t per = (size_t)s.R * s.nws * (s.word_bits / 8);
    std::vector<uint8_t> words(per);
    int64_t dev_fail = 0;
    e = cudaMemcpyAsync(words.data(), ctx->ws + s.off_best + per * w, per, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&dev_fail, &aux->verify_failures, sizeof dev_fail, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "collect best");
    std::vector<int8_t> rows((size_t)r * tfg::host::term_len(s.fmt));
    unpack_terms(s, words.data(), r, rows.data());
    std::vector<HTerm> t;
    const bool host_ok = tfg::host::parse(s.fmt, r, rows.data(), t) == TFG_OK && tfg::host::brent_ok(s.fmt, t);
    if (rank_out) *rank_out = r;
    if (walker_out) *walker_out = (int64_t)ctx->prm.walker_id_base + s.first + w;
    if (!host_ok || dev_fail != 0) {
        set_error("best scheme failed verification (host " + std::string(host_ok ? "ok" : "FAIL") + ", device " +
                  std::string(dev_fail ? "FAIL" : "ok") + ")");
        return TFG_EINTERNAL;
    }
    if (r > cap) { set_error("output buffer too small"); return TFG_ENOSPC; }
    if (out) std::memcpy(out, rows.data(), rows.size());
    return TFG_OK;
}

int tfg_stats_get(tfg_ctx *ctx, int32_t format_idx, tfg_stats *out, int64_t *rank_hist, int32_t hist_len) {
    if (!ctx || !out || format_idx < -1 || format_idx >= (int)ctx->segs.size()) { set_error("bad arguments"); return TFG_EINVAL; }
    if (rank_hist && (hist_len < 1 || hist_len > kHistCap)) { set_error("hist_len must be 1..1024"); return TFG_EINVAL; }
    Aux *aux = ctx->aux();
    cudaError_t e = cudaMemsetAsync(aux->sums, 0, sizeof(aux->sums), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&aux->minmax[0], 0x7f, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&aux->minmax[1], 0x80, sizeof(int32_t), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(aux->hist, 0, sizeof(aux->hist), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    for (int f = 0; f < (int)ctx->segs.size(); ++f) {
        if (format_idx >= 0 && f != format_idx) continue;
        tfg::launch_stats(ctx->desc(ctx->segs[f]), aux->sums, aux->minmax, aux->hist, kHistCap, ctx->stream);
    }
    Aux host;
    e = cudaMemcpyAsync(&host, aux, sizeof(Aux), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stats");
    out->walkers = host.sums[0];
    out->steps = host.sums[1];
    out->accepted = host.sums[2];
    out->rejected = host.sums[3];
    out->nocand = host.sums[4];
    out->drops = host.sums[5];
    out->merges = host.sums[6];
    out->plus = host.sums[7];
    out->reductions = host.sums[8];
    out->min_best_r = host.minmax[0];
    out->max_best_r = host.minmax[1];
    if (rank_hist) std::memcpy(rank_hist, host.hist, sizeof(int64_t) * hist_len);
    return TFG_OK;
}

int tfg_reseed(tfg_ctx *ctx, int64_t first, int64_t count, int32_t rank, const int8_t *scheme) {
    if (!ctx || first < 0 || count < 1 || first + count > ctx->total) { set_error("walker range out of bounds"); return TFG_EINVAL; }
    const Segment *sp = nullptr;
    for (const Segment &s : ctx->segs)
        if (first >= s.first && first + count <= s.first + s.n) sp = &s;
    if (!sp) { set_error("walker range spans several populations"); return TFG_EINVAL; }
    const Segment &s = *sp;
    int rc = tfg::host::check_input(&s.fmt, rank, scheme);
    if (rc) return rc;
    std::vector<HTerm> t;
    rc = tfg::host::parse(s.fmt, rank, scheme, t);
    if (rc) return rc;
    tfg::host::prepare(s.fmt, t);
    if ((int)t.size() > s.R) { set_error("prepared rank exceeds the population's r_max"); return TFG_ENOSPC; }
    if (t.empty()) { set_error("empty scheme"); return TFG_EINVAL; }
    std::vector<uint8_t> buf;
    pack_terms(s, t, buf);
    const size_t per = buf.size();
    const int64_t lo = first - s.first;
    // stage the packed scheme in the first walker's live slots, then copy on the device
    cudaError_t e = cudaMemcpyAsync(ctx->ws + s.off_slots + per * lo, buf.data(), per, cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reseed copy");
    tfg::SegDesc d = ctx->desc(s);
    uint32_t nnz = 0;
    for (const HTerm &h : t)
        for (int x = 0; x < 3; ++x) nnz += (uint32_t)(h.p[x] | h.n[x]).popcount();
    tfg::launch_reseed(d, lo, count, (int32_t)t.size(), nnz, ctx->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reseed");
    return TFG_OK;
}

// ---- device resize (resize.cu): scratch = [skip counter][maps int16][aux int8]
static size_t resize_maps_bytes(const tfg_format &out) {
    return ((size_t)2 * tfg::host::term_len(out) * sizeof(int16_t) + 15) & ~(size_t)15;
}

size_t tfg_resize_scratch_bytes(int32_t aux_rank, const tfg_format *aux_fmt, const tfg_format *out_fmt) {
    if (!out_fmt || out_fmt->m < 1 || out_fmt->n < 1 || out_fmt->p < 1) return 0;
    const tfg_format &o = *out_fmt;
    // the naive block of an extension has at most max(mn, np, pm) terms of at most LT(out) coefficients
    const size_t naive = (size_t)std::max(o.m * o.n, std::max(o.n * o.p, o.p * o.m)) * tfg::host::term_len(o);
    const size_t aux = aux_fmt && aux_rank > 0 ? (size_t)aux_rank * tfg::host::term_len(*aux_fmt) : 0;
    return 16 + resize_maps_bytes(o) + std::max(naive, aux);
}

int tfg_resize(tfg_ctx *ctx, const tfg_resize_args *a, void *d_scratch, size_t scratch_bytes, int64_t *skipped) {
    if (skipped) *skipped = 0;
    if (!ctx || !a || !d_scratch) { set_error("null argument"); return TFG_EINVAL; }
    if (a->count < 1 || a->src_first < 0 || a->dst_first < 0 || a->src_first + a->count > ctx->total ||
        a->dst_first + a->count > ctx->total) {
        set_error("walker range out of bounds");
        return TFG_EINVAL;
    }
    const Segment *sp = nullptr, *dp = nullptr;
    for (const Segment &s : ctx->segs) {
        if (a->src_first >= s.first && a->src_first + a->count <= s.first + s.n) sp = &s;
        if (a->dst_first >= s.first && a->dst_first + a->count <= s.first + s.n) dp = &s;
    }
    if (!sp || !dp) { set_error("a walker range spans several populations"); return TFG_EINVAL; }
    if (sp == dp && a->src_first < a->dst_first + a->count && a->dst_first < a->src_first + a->count) {
        set_error("source and destination walkers overlap");
        return TFG_EINVAL;
    }
    if (sp->fmt.mode != dp->fmt.mode) { set_error("source and destination modes differ"); return TFG_EINVAL; }
    if (a->use_best != 0 && a->use_best != 1) { set_error("use_best must be 0 or 1"); return TFG_EINVAL; }
    const bool with_aux = a->op == TFG_RESIZE_MERGE || a->op == TFG_RESIZE_PRODUCT;
    tfg_format aux_fmt = a->aux_fmt;
    if (with_aux) {
        if (!a->aux_scheme || a->aux_rank < 1) { set_error("the operator needs an aux scheme"); return TFG_EINVAL; }
        if (aux_fmt.mode != sp->fmt.mode) { set_error("aux mode differs from the populations'"); return TFG_EINVAL; }
        int rc = tfg::host::check_input(&aux_fmt, a->aux_rank, a->aux_scheme);
        if (rc) return rc;
    }
    tfg::ResizePlan plan;
    std::vector<int16_t> maps;
    tfg_format out{};
    if (!tfg::build_resize_plan(a->op, a->axis, a->index, sp->fmt, with_aux ? &aux_fmt : nullptr, a->aux_rank, out,
                                plan, maps)) {
        set_error("unsupported resize operator or argument for the source format");
        return TFG_EINVAL;
    }
    if (out.m != dp->fmt.m || out.n != dp->fmt.n || out.p != dp->fmt.p) {
        set_error("the result format (" + std::to_string(out.m) + "," + std::to_string(out.n) + "," +
                  std::to_string(out.p) + ") is not the destination population's");
        return TFG_EINVAL;
    }
    if (!tfg::host::format_ok(&out)) { set_error("result format too large"); return TFG_EINVAL; }
    // aux rows: the caller's scheme, or the naive scheme of an extension's block (terms in (i, k, j) order)
    std::vector<int8_t> aux_rows;
    if (with_aux) {
        aux_rows.assign(a->aux_scheme, a->aux_scheme + (size_t)a->aux_rank * tfg::host::term_len(aux_fmt));
    } else if (a->op == TFG_RESIZE_EXTEND) {
        const int bm = a->axis == 0 ? 1 : sp->fmt.m, bn = a->axis == 1 ? 1 : sp->fmt.n, bp = a->axis == 2 ? 1 : sp->fmt.p;
        const int lt = bm * bn + bn * bp + bp * bm;
        for (int i = 0; i < bm; ++i)
            for (int k = 0; k < bn; ++k)
                for (int j = 0; j < bp; ++j) {
                    std::vector<int8_t> row((size_t)lt, 0);
                    row[(size_t)i * bn + k] = 1;
                    row[(size_t)bm * bn + k * bp + j] = 1;
                    row[(size_t)bm * bn + bn * bp + j * bm + i] = 1;
                    aux_rows.insert(aux_rows.end(), row.begin(), row.end());
                }
    }
    const size_t need = tfg_resize_scratch_bytes(a->aux_rank, with_aux ? &aux_fmt : nullptr, &out);
    if (scratch_bytes < need || aux_rows.size() + 16 + resize_maps_bytes(out) > scratch_bytes) {
        set_error("scratch holds " + std::to_string(scratch_bytes) + " bytes, the resize needs " + std::to_string(need));
        return TFG_ENOSPC;
    }
    if (maps.size() * sizeof(int16_t) > resize_maps_bytes(out)) { set_error("internal: map table"); return TFG_EINTERNAL; }
    char *sc = static_cast<char *>(d_scratch);
    auto *d_skip = reinterpret_cast<unsigned long long *>(sc);
    plan.maps = reinterpret_cast<const int16_t *>(sc + 16);
    plan.aux = reinterpret_cast<const int8_t *>(sc + 16 + resize_maps_bytes(out));
    plan.use_best = a->use_best;
    cudaError_t e = cudaMemsetAsync(d_skip, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sc + 16, maps.data(), maps.size() * sizeof(int16_t), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && !aux_rows.empty())
        e = cudaMemcpyAsync(sc + 16 + resize_maps_bytes(out), aux_rows.data(), aux_rows.size(), cudaMemcpyHostToDevice,
                            ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "resize staging");
    tfg::launch_resize(ctx->desc(*sp), a->src_first - sp->first, ctx->desc(*dp), a->dst_first - dp->first, a->count,
                       plan, d_skip, ctx->stream);
    e = cudaGetLastError();
    unsigned long long sk = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sk, d_skip, sizeof(sk), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "resize");
    if (skipped) *skipped = (int64_t)sk;
    if (sk) { set_error(std::to_string(sk) + " walkers left unchanged: result above the destination's r_max"); return TFG_ENOSPC; }
    return TFG_OK;
}

int tfg_read_walkers(tfg_ctx *ctx, int64_t first, int64_t count, tfg_walker_info *info, int8_t *slots, int8_t *best,
                     int32_t r_max_cap) {
    if (!ctx || first < 0 || count < 0 || first + count > ctx->total) { set_error("walker range out of bounds"); return TFG_EINVAL; }
    if (count == 0) return TFG_OK;
    const Segment *sp = nullptr;
    for (const Segment &s : ctx->segs)
        if (first >= s.first && first + count <= s.first + s.n) sp = &s;
    if (!sp) { set_error("walker range spans several populations"); return TFG_EINVAL; }
    const Segment &s = *sp;
    if ((slots || best) && r_max_cap < s.R) { set_error("r_max_cap smaller than the population's r_max"); return TFG_ENOSPC; }
    const int64_t lo = first - s.first;
    const size_t per = (size_t)s.R * s.nws * (s.word_bits / 8);
    const int LT = tfg::host::term_len(s.fmt);
    std::vector<tfg_walker_info> hdr((size_t)count);
    cudaError_t e = cudaMemcpyAsync(hdr.data(), ctx->ws + s.off_hdr + sizeof(tfg_walker_info) * lo,
                                    sizeof(tfg_walker_info) * count, cudaMemcpyDeviceToHost, ctx->stream);
    std::vector<uint8_t> ws, wb;
    if (e == cudaSuccess && slots) {
        ws.resize(per * count);
        e = cudaMemcpyAsync(ws.data(), ctx->ws + s.off_slots + per * lo, per * count, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess && best) {
        wb.resize(per * count);
        e = cudaMemcpyAsync(wb.data(), ctx->ws + s.off_best + per * lo, per * count, cudaMemcpyDeviceToHost, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "read walkers");
    if (info) std::memcpy(info, hdr.data(), sizeof(tfg_walker_info) * count);
    for (int64_t a = 0; a < count; ++a) {
        if (slots) {
            int8_t *dst = slots + (size_t)a * r_max_cap * LT;
            std::memset(dst, 0, (size_t)r_max_cap * LT);
            unpack_terms(s, ws.data() + per * a, std::min(hdr[a].r, s.R), dst);
        }
        if (best) {
            int8_t *dst = best + (size_t)a * r_max_cap * LT;
            std::memset(dst, 0, (size_t)r_max_cap * LT);
            unpack_terms(s, wb.data() + per * a, std::min(hdr[a].best_r, s.R), dst);
        }
    }
    return TFG_OK;
}

int tfg_checkpoint(tfg_ctx *ctx, void *buf, size_t cap, size_t *used) {
    if (!ctx || !used) { set_error("bad arguments"); return TFG_EINVAL; }
    const size_t n = ctx->ws_used - kAuxBytes;
    *used = n;
    if (!buf) return TFG_OK;
    if (cap < n) { set_error("checkpoint buffer too small"); return TFG_ENOSPC; }
    cudaError_t e = cudaMemcpyAsync(buf, ctx->ws + kAuxBytes, n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint");
    return TFG_OK;
}

int tfg_restore(tfg_ctx *ctx, const void *buf, size_t size) {
    if (!ctx || !buf) { set_error("bad arguments"); return TFG_EINVAL; }
    if (size != ctx->ws_used - kAuxBytes) { set_error("checkpoint size does not match this context"); return TFG_EINVAL; }
    cudaError_t e = cudaMemcpyAsync(ctx->ws + kAuxBytes, buf, size, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "restore");
    return TFG_OK;
}

void tfg_destroy(tfg_ctx *ctx) { delete ctx; }

size_t tfg_mlp_param_bytes(void) { return tfg::mlp_param_bytes(); }

int tfg_mlp_score(const void *d_params, const uint16_t *d_x, int64_t n, float *d_out, int32_t *d_err,
                  void *cuda_stream) {
    if (n < 0 || (n > 0 && (!d_params || !d_x || !d_out || !d_err))) { set_error("bad arguments"); return TFG_EINVAL; }
    if (((uintptr_t)d_x % 16) != 0 || ((uintptr_t)d_params % 16) != 0) { set_error("inputs must be 16-byte aligned"); return TFG_EINVAL; }
    tfg::launch_mlp_score(d_params, d_x, n, d_out, d_err, reinterpret_cast<cudaStream_t>(cuda_stream));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mlp score launch");
    return TFG_OK;
}

// optimizer state: master weights, Adam moments (P each), the gradient (P + 1, then padding to 4 floats),
// then the per-CTA gradient rows of the deterministic gradient launch
static size_t train_partial_offset() { return (size_t)4 * tfg::mlp_num_params() + 4; }
size_t tfg_mlp_train_state_bytes(void) {
    return (train_partial_offset() + (size_t)tfg::grad_partial_rows() * (tfg::mlp_num_params() + 1)) * sizeof(float);
}

int tfg_mlp_grad(const void *d_params, const uint16_t *d_x, const float *d_label, const float *d_weight, int64_t n,
                 float *d_grad, int32_t *d_err, void *cuda_stream) {
    if (n < 0 || !d_params || !d_grad || !d_err || (n > 0 && (!d_x || !d_label || !d_weight))) {
        set_error("bad arguments");
        return TFG_EINVAL;
    }
    if (((uintptr_t)d_x % 16) != 0) { set_error("features must be 16-byte aligned"); return TFG_EINVAL; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(d_grad, 0, sizeof(float) * (tfg::mlp_num_params() + 1), st);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    tfg::launch_mlp_grad(d_params, d_x, d_label, d_weight, n, d_grad, d_err, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mlp grad launch");
    return TFG_OK;
}

int tfg_mlp_train_init(void *d_state, const void *d_params, void *cuda_stream) {
    if (!d_state || !d_params) { set_error("bad arguments"); return TFG_EINVAL; }
    const int P = tfg::mlp_num_params();
    float *s = reinterpret_cast<float *>(d_state);
    tfg::launch_master_from_blob(d_params, s, s + P, s + 2 * P, reinterpret_cast<cudaStream_t>(cuda_stream));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "train init launch");
    return TFG_OK;
}

int tfg_mlp_train_step(void *d_state, void *d_params, const uint16_t *d_x, const float *d_label,
                       const float *d_weight, int64_t n, float lr, int32_t step, int32_t *d_err, void *cuda_stream) {
    if (!d_state || !d_params || step < 1) { set_error("bad arguments (step counts from 1)"); return TFG_EINVAL; }
    const int P = tfg::mlp_num_params();
    float *s = reinterpret_cast<float *>(d_state);
    if (n < 0 || !d_err || (n > 0 && (!d_x || !d_label || !d_weight))) { set_error("bad arguments"); return TFG_EINVAL; }
    if (((uintptr_t)d_x % 16) != 0) { set_error("features must be 16-byte aligned"); return TFG_EINVAL; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(s + 3 * P, 0, sizeof(float) * (P + 1), st);
        if (e != cudaSuccess) return cuda_fail(e, "memset");
    }
    // the gradient from per-CTA rows added in CTA order: the same bits on every run
    tfg::launch_mlp_grad(d_params, d_x, d_label, d_weight, n, s + 3 * P, d_err, st, s + train_partial_offset());
    tfg::launch_adam(s, s + P, s + 2 * P, s + 3 * P, d_params, lr, step, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adam launch");
    return TFG_OK;
}

// per walker: W window rows of (descriptor, info) words and a score, then the window size
static size_t window_row_bytes() { return (size_t)tfg::window_cap() * (8 + 4); }

int tfg_window_scratch_bytes(tfg_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) { set_error("bad arguments"); return TFG_EINVAL; }
    *bytes = align_up((size_t)ctx->total * window_row_bytes() + (size_t)ctx->total * 4);
    return TFG_OK;
}

// Window mode applies to Z_T populations whose terms fit one word per sign and
// whose slot capacity the apply kernel supports.
static int check_window_ctx(const tfg_ctx *ctx, int64_t steps, int32_t policy, const void *d_mlp_params) {
    if (!ctx || steps < 0 || (policy != 0 && policy != 1) || (policy == 1 && !d_mlp_params)) {
        set_error("bad arguments");
        return TFG_EINVAL;
    }
    if (policy == 1 && (uintptr_t)d_mlp_params % 16) { set_error("network parameters must be 16-byte aligned"); return TFG_EINVAL; }
    if (ctx->prm.walk_policy != 0) { set_error("window mode needs walk_policy 0"); return TFG_EINVAL; }
    for (const Segment &s : ctx->segs) {
        if (s.fmt.mode != TFG_MODE_ZT || s.tw != 1 || s.R > 128 ||
            tfg::window_apply_capacity(s.word_bits, s.R) == 0) {
            set_error("window mode needs Z_T populations with m*n+n*p+p*m <= 64 and r_max <= 88");
            return TFG_EINVAL;
        }
    }
    return TFG_OK;
}

// The window-mode steps on the context stream, with the scratch at `base`
// (features, descriptors, scores, window sizes; tfg_window_scratch_bytes).
// A tensor-core wait of the network that gives up sets the context's status
// word, which tfg_sync reports as TFG_ETIMEOUT.
static int window_steps(tfg_ctx *ctx, int64_t steps, int32_t policy, const void *d_mlp_params, uint32_t eps_thresh,
                        char *base, int32_t *d_choices, const tfg_log_spec *log) {
    const int W = tfg::window_cap();
    const int64_t N = ctx->total;
    auto *desc = reinterpret_cast<uint2 *>(base);
    auto *score = reinterpret_cast<float *>(base + (size_t)N * W * 8);
    auto *kwin = reinterpret_cast<int *>(base + (size_t)N * W * 12);
    tfg_log_spec lg{};
    if (log) lg = *log;
    if (lg.d_entries && lg.horizon > 1) {
        if (lg.horizon > 64 || !lg.d_ring || !lg.d_ring_step || (uintptr_t)lg.d_ring % 16 ||
            (uintptr_t)lg.d_ring_step % 4) {
            set_error("log horizon: 2..64 with a 16-byte aligned ring and its step words");
            return TFG_EINVAL;
        }
    } else {
        lg.horizon = 1;
    }
    const int H = lg.horizon;
    int32_t *status = &ctx->aux()->status;
    for (int64_t st = 0; st < steps; ++st) {
        for (const Segment &s : ctx->segs)
            tfg::launch_window(ctx->desc(s), nullptr, desc + (size_t)s.first * W, kwin + s.first, ctx->stream);
        if (policy == 1)
            for (const Segment &s : ctx->segs)
                tfg::launch_window_score(ctx->desc(s), d_mlp_params, desc + (size_t)s.first * W, kwin + s.first,
                                         score + (size_t)s.first * W, status, ctx->stream);
        for (const Segment &s : ctx->segs) {
            int32_t *ch = d_choices ? d_choices + (size_t)st * N + s.first : nullptr;
            tfg_log_spec ls = lg;   // the segment's walkers' rings
            if (H > 1) {
                ls.d_ring = lg.d_ring + (size_t)s.first * H * 32;
                ls.d_ring_step = lg.d_ring_step + (size_t)s.first * H;
            }
            tfg::launch_window_apply(ctx->desc(s), desc + (size_t)s.first * W, kwin + s.first,
                                     score + (size_t)s.first * W, policy, eps_thresh, ch, ls, ctx->stream);
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "window step launch");
    }
    return TFG_OK;
}

int tfg_window_dump(tfg_ctx *ctx, uint16_t *d_feat, uint32_t *d_desc, int32_t *d_kwin) {
    int rc = check_window_ctx(ctx, 0, 0, nullptr);
    if (rc) return rc;
    if (!d_desc || !d_kwin) { set_error("bad arguments: null descriptor or window-size array"); return TFG_EINVAL; }
    if ((d_feat && (uintptr_t)d_feat % 16) || (uintptr_t)d_desc % 8) {
        set_error("features must be 16-byte aligned, descriptors 8-byte aligned");
        return TFG_EINVAL;
    }
    const int W = tfg::window_cap();
    for (const Segment &s : ctx->segs)
        tfg::launch_window(ctx->desc(s), d_feat ? d_feat + (size_t)s.first * W * 32 : nullptr,
                           reinterpret_cast<uint2 *>(d_desc) + (size_t)s.first * W, d_kwin + s.first, ctx->stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "window dump launch");
    return TFG_OK;
}

int tfg_walk_window(tfg_ctx *ctx, int64_t steps, int32_t policy, const void *d_mlp_params, uint32_t eps_thresh,
                    void *d_scratch, size_t scratch_bytes, int32_t *d_choices, const tfg_log_spec *log) {
    int rc = check_window_ctx(ctx, steps, policy, d_mlp_params);
    if (rc) return rc;
    if (!d_scratch) { set_error("bad arguments: null scratch"); return TFG_EINVAL; }
    size_t need = 0;
    tfg_window_scratch_bytes(ctx, &need);
    if (scratch_bytes < need) { set_error("window scratch too small"); return TFG_ENOMEM; }
    if ((uintptr_t)d_scratch % 16) { set_error("scratch must be 16-byte aligned"); return TFG_EINVAL; }
    return window_steps(ctx, steps, policy, d_mlp_params, eps_thresh, reinterpret_cast<char *>(d_scratch), d_choices,
                        log);
}

// tfg_walk_window for callers that cannot call cudaMalloc: the scratch is the
// library's static array g_window_scratch (see above), so the call allocates
// nothing.  Every value a step reads from the scratch is written earlier in
// the same step (features and window sizes by the window kernel, scores by
// the network), so what an earlier call left there needs no clearing.
int tfg_walk_window_noalloc(tfg_ctx *ctx, int64_t steps, int32_t policy, const void *d_mlp_params,
                            uint32_t eps_thresh, int32_t *d_choices, const tfg_log_spec *log) {
    int rc = check_window_ctx(ctx, steps, policy, d_mlp_params);
    if (rc) return rc;
    size_t need = 0;
    tfg_window_scratch_bytes(ctx, &need);
    if (need > kNoAllocScratchBytes) {
        set_error("tfg_walk_window_noalloc: " + std::to_string(ctx->total) + " walkers need " + std::to_string(need) +
                  " scratch bytes, the static scratch holds " + std::to_string(kNoAllocScratchBytes) +
                  " (at most " + std::to_string(kNoAllocScratchBytes / (window_row_bytes() + 4)) + " walkers)");
        return TFG_EINVAL;
    }
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != ctx->device) {
        set_error("tfg_walk_window_noalloc: device " + std::to_string(dev) + " is current, the context lives on device " +
                  std::to_string(ctx->device) + "; make the context's device current");
        return TFG_EINVAL;
    }
    void *scratch = nullptr;
    rc = window_scratch_address(dev, &scratch);
    if (rc) return rc;
    return window_steps(ctx, steps, policy, d_mlp_params, eps_thresh, reinterpret_cast<char *>(scratch), d_choices,
                        log);
}

void tfg_test_set_wait_limit(int64_t polls) { tfg::set_first_wait_limit(polls); }

int tfg_philox_device(const uint32_t *d_ctr, int32_t n, uint32_t key_lo, uint32_t key_hi, uint32_t *d_out,
                      void *cuda_stream) {
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) { set_error("bad arguments"); return TFG_EINVAL; }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    tfg::launch_philox(d_ctr, n, key_lo, key_hi, d_out, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "philox");
    return TFG_OK;
}

}  // extern "C"

