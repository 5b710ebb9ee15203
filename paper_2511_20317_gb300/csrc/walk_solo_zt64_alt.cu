// Thread-per-walker walk kernel variants (zt64): alternative block sizes.
#include "walk_solo.cuh"

namespace tfg {
// Other walkers-per-block choices of the kernels of walk_solo_zt64.cu, for the
// autotuner (the registry lists those defaults first, so a context starts with them): each
// changes how many walkers the shared memory of an SM holds (capacity 48 at
// 96 threads: three blocks, 9 warps; 88 at 160 threads: one block, 5 warps).
const WalkVariant *walk_variants_solo_zt64_alt(int *n) {
    static const WalkVariant v[] = {
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 48, 96),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 64, 128),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 72, 128),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 88, 160),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
