// Morton (Z-order) keys of integer octree coordinates, x in bit 0 of each group of
// `dim` bits (host code: mesh construction, transfer operators, coarse meshes).
#pragma once

#include <stdint.h>

static inline uint64_t part1by1(uint64_t x) {
    x &= 0xffffffffull;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

static inline uint64_t part1by2(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Morton key, x in bit 0 of each group of `dim` bits.
static inline uint64_t morton(int dim, const int64_t* c) {
    if (dim == 2) return part1by1((uint64_t)c[0]) | (part1by1((uint64_t)c[1]) << 1);
    return part1by2((uint64_t)c[0]) | (part1by2((uint64_t)c[1]) << 1) | (part1by2((uint64_t)c[2]) << 2);
}

