// Walk kernel variants: mode ZT, 32-bit words, 16 lanes per walker.
#include "walk_kernel.cuh"

namespace tfg {
const WalkVariant *walk_variants_zt32_g16(int *n) {
    static const WalkVariant v[] = {
        TFG_WALK_VARIANT(TFG_MODE_ZT, uint32_t, 32, 16, 1),
        TFG_WALK_VARIANT(TFG_MODE_ZT, uint32_t, 32, 16, 2),
        TFG_WALK_VARIANT(TFG_MODE_ZT, uint32_t, 32, 16, 4),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
