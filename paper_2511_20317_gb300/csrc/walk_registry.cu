// Registry of the compiled walk-kernel variants.
#include <vector>

#include "tfg_internal.h"

namespace tfg {
const WalkVariant *walk_variants_group_zt32(int *n);
const WalkVariant *walk_variants_group_z232(int *n);
const WalkVariant *walk_variants_group_64(int *n);
const WalkVariant *walk_variants_wide(int *n);
const WalkVariant *walk_variants_solo_zt32(int *n);
const WalkVariant *walk_variants_solo_z232(int *n);
const WalkVariant *walk_variants_solo_zt64(int *n);
const WalkVariant *walk_variants_solo_z264(int *n);
const WalkVariant *walk_variants_solo_zt64_alt(int *n);

const WalkVariant *walk_variants(int *count) {
    static std::vector<WalkVariant> all = [] {
        std::vector<WalkVariant> v;
        const WalkVariant *(*parts[])(int *) = {
            walk_variants_group_zt32,
            walk_variants_group_z232,
            walk_variants_group_64,
            walk_variants_wide,
            walk_variants_solo_zt32,
            walk_variants_solo_z232,
            walk_variants_solo_zt64,
            walk_variants_solo_z264,
            walk_variants_solo_zt64_alt,   // after the defaults: pick_variant takes the first match
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
