// dev_util.h -- small device helpers shared by the kernels (internal).
#pragma once

#include <cstdint>

namespace dmk {

// cell indices (ix, iy, iz) of a Morton code (bit 3b + d = bit b of axis d)
__device__ __forceinline__ void morton_decode_d(uint64_t m, int &ix, int &iy, int &iz) {
    auto compact = [](uint64_t x) -> int {
        x &= 0x1249249249249249ull;
        x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
        x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
        x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
        x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
        x = (x ^ (x >> 32)) & 0x1fffffull;
        return (int)x;
    };
    ix = compact(m);
    iy = compact(m >> 1);
    iz = compact(m >> 2);
}

// cell indices of a box key at level l: the key's low 3 l bits are the Morton
// code of the cell (the bits above them number the system of a batch)
__device__ __forceinline__ void box_decode_d(uint64_t key, int l, int &ix, int &iy, int &iz) {
    morton_decode_d(key & ((1ull << (3 * l)) - 1ull), ix, iy, iz);
}

}  // namespace dmk
