// Thread-per-walker walk kernel variants (zt32), 128 threads per block.
#include "walk_solo.cuh"

#ifndef TFG_SLICED_ZT_BLOCK
#define TFG_SLICED_ZT_BLOCK 64   // threads per block of the bit-sliced kernel (shared-memory slices)
#endif

namespace tfg {
const WalkVariant *walk_variants_solo_zt32(int *n) {
    static const WalkVariant v[] = {
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint32_t, 32, 12, 128),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint32_t, 32, 16, 128),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint32_t, 32, 24, 128),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint32_t, 32, 32, 128),
        TFG_SOLO_SLICED_VARIANT(TFG_MODE_ZT, uint32_t, 32, 32, TFG_SLICED_ZT_BLOCK, 9, false),
        TFG_SOLO_SLICED_VARIANT(TFG_MODE_ZT, uint32_t, 32, 32, TFG_SLICED_ZT_BLOCK, 9, true),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
