// Storage of the blocks the H^2 product streams, and unpacking of their
// 16-byte rows.
//
// An M x K block (row-major in the paper's notation) is padded to
// K_pad = K rounded up to a multiple of 8 with zero columns and cut into
// tiles of at most 64 rows x 64 columns: row slices a0 = 0, 64, ... and,
// inside a slice, column chunks k0 = 0, 64, ...  Each tile is contiguous:
// tile (a0, k0) with ms = min(64, M - a0) rows starts at element
// a0 * K_pad + ms * k0, and holds its columns as panels of P consecutive
// entries per row (16 bytes: P = 2 double, 4 float, 8 bfloat16), entry
// (a, kk) of the tile at (kk / P) * ms * P + a * P + kk % P.  One tile is one
// work segment of the product and moves with one contiguous copy; a row of a
// panel is one 16-byte shared-memory load.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace gca {

__host__ __device__ constexpr int pad8(int k) { return (k + 7) & ~7; }

template <typename T>
struct Panel {
  static constexpr int P = 16 / (int)sizeof(T);
};

__device__ __forceinline__ void unpack(const uint4& u, float (&v)[4]) {
  v[0] = __uint_as_float(u.x);
  v[1] = __uint_as_float(u.y);
  v[2] = __uint_as_float(u.z);
  v[3] = __uint_as_float(u.w);
}

// bfloat16 -> float is exact: the bfloat16 bits are the high half of the float
__device__ __forceinline__ void unpack(const uint4& u, float (&v)[8]) {
  const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    v[2 * i] = __uint_as_float(w[i] << 16);
    v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

__device__ __forceinline__ void unpack(const uint4& u, double (&v)[2]) {
  v[0] = __hiloint2double((int)u.y, (int)u.x);
  v[1] = __hiloint2double((int)u.w, (int)u.z);
}

}  // namespace gca
