// Walk kernel variants: mode Z2, 32-bit words, 8 lanes per walker.
#include "walk_kernel.cuh"

namespace tfg {
const WalkVariant *walk_variants_z232_g8(int *n) {
    static const WalkVariant v[] = {
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 8, 1),
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 8, 2),
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 8, 3),
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 8, 4),
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 8, 8),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
