// Walk kernel variants: mode Z2, 32-bit words, 4 lanes per walker.
#include "walk_kernel.cuh"

namespace tfg {
const WalkVariant *walk_variants_z232_g4(int *n) {
    static const WalkVariant v[] = {
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 4, 2),
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 4, 3),
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 4, 4),
        TFG_WALK_VARIANT(TFG_MODE_Z2, uint32_t, 32, 4, 8),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
