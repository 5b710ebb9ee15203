// Host-side scheme representation used by the C ABI implementation.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tfg.h"

namespace tfg {
namespace host {

// Coefficient bits of one factor of at most 128 entries: entry e is bit e % 64
// of word e / 64.
struct FMask {
    uint64_t w[2] = {0, 0};
    bool bit(int e) const { return (w[e >> 6] >> (e & 63)) & 1ull; }
    void set(int e) { w[e >> 6] |= 1ull << (e & 63); }
    bool any() const { return (w[0] | w[1]) != 0; }
    int popcount() const { return __builtin_popcountll(w[0]) + __builtin_popcountll(w[1]); }
    FMask operator|(const FMask &o) const { return FMask{{w[0] | o.w[0], w[1] | o.w[1]}}; }
    FMask operator&(const FMask &o) const { return FMask{{w[0] & o.w[0], w[1] & o.w[1]}}; }
    FMask operator^(const FMask &o) const { return FMask{{w[0] ^ o.w[0], w[1] ^ o.w[1]}}; }
    FMask operator~() const { return FMask{{~w[0], ~w[1]}}; }
    bool operator==(const FMask &o) const { return w[0] == o.w[0] && w[1] == o.w[1]; }
    bool operator!=(const FMask &o) const { return !(*this == o); }
    // the lowest set bit alone
    FMask lowbit() const {
        if (w[0]) return FMask{{w[0] & (~w[0] + 1), 0}};
        return FMask{{0, w[1] & (~w[1] + 1)}};
    }
};

// One term: positive and negative coefficient masks of u, v, w (Z_2: p only).
struct HTerm {
    FMask p[3];
    FMask n[3];
};

void set_error(const std::string &s);
const char *last_error();

bool format_ok(const tfg_format *f);   // sizes >= 1, each factor at most 128 entries
int factor_len(const tfg_format &f, int x);
int term_len(const tfg_format &f);
int parse(const tfg_format &f, int rank, const int8_t *rows, std::vector<HTerm> &out);
void emit(const tfg_format &f, const std::vector<HTerm> &t, int8_t *rows);
bool brent_ok(const tfg_format &f, const std::vector<HTerm> &t);
void canon_term(const tfg_format &f, HTerm &h);
void prepare(const tfg_format &f, std::vector<HTerm> &t);
int check_input(const tfg_format *f, int rank, const int8_t *rows);

int project(const tfg_format *f, int r, const int8_t *rows, int axis, int index, tfg_format *of, int8_t *out,
            int cap, int *orank);
int merge(const tfg_format *fa, int ra, const int8_t *sa, const tfg_format *fb, int rb, const int8_t *sb, int axis,
          tfg_format *of, int8_t *out, int cap, int *orank);
int extend(const tfg_format *f, int r, const int8_t *rows, int axis, tfg_format *of, int8_t *out, int cap,
           int *orank);
int product(const tfg_format *fa, int ra, const int8_t *sa, const tfg_format *fb, int rb, const int8_t *sb,
            tfg_format *of, int8_t *out, int cap, int *orank);
int swap_sizes(const tfg_format *f, int r, const int8_t *rows, int perm, tfg_format *of, int8_t *out, int cap,
               int *orank);

// Rank of factor x of a term read as a matrix (u: m x n, v: n x p, w: p x m),
// over Q (Z_T) or GF(2) (Z_2).
int factor_rank(const tfg_format &f, const HTerm &h, int x);

// Z_2 -> Z_T sign lifting (lift.cpp): rows hold a Z_2 scheme (0/1); out gets the
// signed scheme.  TFG_OK, TFG_ESCHEME (no assignment exists), TFG_ETIMEOUT, TFG_EINVAL.
int lift_signs(const tfg_format &f, int r, const int8_t *rows, int64_t max_nodes, int8_t *out, int64_t *nodes_used);

}  // namespace host
}  // namespace tfg
