// Lane-group walk kernel variants (z232).
#include "walk_group.cuh"

namespace tfg {
const WalkVariant *walk_variants_group_z232(int *n) {
    static const WalkVariant v[] = {
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 4, 2),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 4, 3),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 4, 4),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 4, 8),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 8, 1),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 8, 2),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 8, 3),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 8, 4),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 8, 8),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 16, 1),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 16, 2),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 16, 4),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 32, 1),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 32, 2),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 32, 3),
        TFG_GROUP_VARIANT(TFG_MODE_Z2, uint32_t, 32, 1, 32, 4),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
