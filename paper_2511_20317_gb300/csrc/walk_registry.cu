// Registry of the compiled walk-kernel variants.
#include <vector>

#include "tfg_internal.h"

namespace tfg {
#define TFG_DECL(name) const WalkVariant *name(int *n);
TFG_DECL(walk_variants_zt32_g4)
TFG_DECL(walk_variants_zt32_g8)
TFG_DECL(walk_variants_zt32_g16)
TFG_DECL(walk_variants_zt32_g32)
TFG_DECL(walk_variants_z232_g4)
TFG_DECL(walk_variants_z232_g8)
TFG_DECL(walk_variants_z232_g16)
TFG_DECL(walk_variants_z232_g32)
#undef TFG_DECL

const WalkVariant *walk_variants(int *count) {
    static std::vector<WalkVariant> all = [] {
        std::vector<WalkVariant> v;
        const WalkVariant *(*parts[])(int *) = {
            walk_variants_zt32_g4, walk_variants_zt32_g8, walk_variants_zt32_g16, walk_variants_zt32_g32,
            walk_variants_z232_g4, walk_variants_z232_g8, walk_variants_z232_g16, walk_variants_z232_g32,
        };
        for (auto part : parts) {
            int n = 0;
            const WalkVariant *p = part(&n);
            v.insert(v.end(), p, p + n);
        }
        return v;
    }();
    *count = (int)all.size();
    return all.data();
}
}  // namespace tfg
