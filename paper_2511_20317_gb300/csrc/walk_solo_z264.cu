// Thread-per-walker walk kernel variants (z264), 128 threads per block.
#include "walk_solo.cuh"

// threads per block of the larger capacities (shared memory per block = capacity x
// (threads + 1) x 16 bytes in Z_T decides how many blocks fit on an SM)
#ifndef TFG_SOLO64_BT48
#define TFG_SOLO64_BT48 128
#endif
#ifndef TFG_SOLO64_BT64
#define TFG_SOLO64_BT64 128
#endif
#ifndef TFG_SOLO64_BT72
#define TFG_SOLO64_BT72 128
#endif
#ifndef TFG_SOLO64_BT88
#define TFG_SOLO64_BT88 128
#endif

namespace tfg {
const WalkVariant *walk_variants_solo_z264(int *n) {
    static const WalkVariant v[] = {
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 16, 128),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 32, 128),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 48, TFG_SOLO64_BT48),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 64, TFG_SOLO64_BT64),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 72, TFG_SOLO64_BT72),
        TFG_SOLO_VARIANT(TFG_MODE_Z2, uint64_t, 64, 88, TFG_SOLO64_BT88),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}
}  // namespace tfg
