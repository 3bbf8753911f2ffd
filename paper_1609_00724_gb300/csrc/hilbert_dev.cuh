// Hilbert curve on the device (Sec. "Adaptive refinements" of
// arXiv:1609.00724): Skilling (2004) "transpose" method in nd = 2 or 3
// dimensions with `bits` bits per axis; the curve starts at the origin. The
// key interleaves the transposed words most significant bit first, axis 0
// taking the highest bit of each group.
#pragma once
#include <stdint.h>

namespace qsl {

__device__ __forceinline__ uint64_t hilbert_key_dev(const uint32_t* coords, int nd, int bits) {
  uint32_t X0 = coords[0], X1 = coords[1], X2 = nd == 3 ? coords[2] : 0u;
  if (bits > 0) {
    // undo reflections and exchanges from the top level down
    for (uint32_t q = 1u << (bits - 1); q > 1; q >>= 1) {
      uint32_t p = q - 1;
      // i = 0
      if (X0 & q) X0 ^= p;
      // i = 1
      if (X1 & q) {
        X0 ^= p;
      } else {
        uint32_t t = (X0 ^ X1) & p;
        X0 ^= t;
        X1 ^= t;
      }
      if (nd == 3) {
        if (X2 & q) {
          X0 ^= p;
        } else {
          uint32_t t = (X0 ^ X2) & p;
          X0 ^= t;
          X2 ^= t;
        }
      }
    }
    // Gray code
    X1 ^= X0;
    if (nd == 3) X2 ^= X1;
    uint32_t last = nd == 3 ? X2 : X1;
    uint32_t t = 0;
    for (uint32_t q = 1u << (bits - 1); q > 1; q >>= 1)
      if (last & q) t ^= q - 1;
    X0 ^= t;
    X1 ^= t;
    if (nd == 3) X2 ^= t;
  }
  uint64_t key = 0;
  for (int b = bits - 1; b >= 0; --b) {
    key = (key << 1) | ((X0 >> b) & 1u);
    key = (key << 1) | ((X1 >> b) & 1u);
    if (nd == 3) key = (key << 1) | ((X2 >> b) & 1u);
  }
  return key;
}

__device__ __forceinline__ void hilbert_coords_dev(uint64_t key, int nd, int bits, uint32_t* coords) {
  uint32_t X0 = 0, X1 = 0, X2 = 0;
  int pos = nd * bits - 1;
  for (int b = bits - 1; b >= 0; --b) {
    X0 |= (uint32_t)((key >> pos) & 1u) << b;
    --pos;
    X1 |= (uint32_t)((key >> pos) & 1u) << b;
    --pos;
    if (nd == 3) {
      X2 |= (uint32_t)((key >> pos) & 1u) << b;
      --pos;
    }
  }
  if (bits > 0) {
    // Gray decode
    uint32_t last = nd == 3 ? X2 : X1;
    uint32_t t = last >> 1;
    if (nd == 3) X2 ^= X1;
    X1 ^= X0;
    X0 ^= t;
    // redo exchanges and reflections from the bottom level up
    for (int lev = 1; lev < bits; ++lev) {
      uint32_t q = 1u << lev, p = q - 1;
      if (nd == 3) {
        if (X2 & q) {
          X0 ^= p;
        } else {
          uint32_t u = (X0 ^ X2) & p;
          X0 ^= u;
          X2 ^= u;
        }
      }
      if (X1 & q) {
        X0 ^= p;
      } else {
        uint32_t u = (X0 ^ X1) & p;
        X0 ^= u;
        X1 ^= u;
      }
      if (X0 & q) X0 ^= p;
    }
  }
  coords[0] = X0;
  coords[1] = X1;
  if (nd == 3) coords[2] = X2;
}

}  // namespace qsl
