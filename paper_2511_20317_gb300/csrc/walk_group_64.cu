// Lane-group walk kernel variants for 64-bit terms (m*n + n*p + p*m <= 64).
#include "walk_group.cuh"

namespace tfg {
const WalkVariant *walk_variants_group_64(int *n) {
    static const WalkVariant v[] = {
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 8, 4),
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 8, 8),
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 8, 12),
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 16, 4),
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 16, 6),
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 32, 2),
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 32, 3),
        TFG_GROUP_VARIANT(TFG_MODE_ZT, uint64_t, 64, 1, 32, 4),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 8, 4),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 8, 8),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 8, 12),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 16, 4),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 16, 6),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 32, 2),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 32, 3),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint64_t, 64, 1, 32, 4),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
