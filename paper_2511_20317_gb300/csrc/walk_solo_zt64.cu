// Thread-per-walker walk kernel variants (zt64).
#include "walk_solo.cuh"

// threads per block of the larger capacities (shared memory per block = capacity x
// (threads + 1) x 16 bytes in Z_T decides how many blocks fit on an SM): 64 threads
// let three blocks of capacity 64 or 72 reside instead of one of 128 (measured
// (3,4,5) 2.68e9 -> 3.45e9, (4,4,4) 2.67e9 -> 3.14e9 steps/s)
#ifndef TFG_SOLO64_BT48
#define TFG_SOLO64_BT48 128
#endif
#ifndef TFG_SOLO64_BT64
#define TFG_SOLO64_BT64 64
#endif
#ifndef TFG_SOLO64_BT72
#define TFG_SOLO64_BT72 64
#endif
#ifndef TFG_SOLO64_BT88
#define TFG_SOLO64_BT88 128
#endif

namespace tfg {
const WalkVariant *walk_variants_solo_zt64(int *n) {
    static const WalkVariant v[] = {
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 16, 128),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 32, 128),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 48, TFG_SOLO64_BT48),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 64, TFG_SOLO64_BT64),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 72, TFG_SOLO64_BT72),
        TFG_SOLO_VARIANT(TFG_MODE_ZT, uint64_t, 64, 88, TFG_SOLO64_BT88),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

}  // namespace tfg
