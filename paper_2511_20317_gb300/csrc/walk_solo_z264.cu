// Thread-per-walker walk kernel variants (z264), 128 threads per block.
#include "walk_solo.cuh"

namespace tfg {
const WalkVariant *walk_variants_solo_z264(int *n) {
    static const WalkVariant v[] = {
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 16, 128),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 32, 128),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 48, 128),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 64, 128),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 72, 128),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 88, 128),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
