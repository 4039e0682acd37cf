// Panel layout of the stored blocks and the two register-tiled micro-kernels
// every H^2 product stage is made of.
//
// Panel layout.  An M x K block (row-major in the paper's notation) is
// stored as K_pad / P column panels, each M rows of P consecutive entries
// (16 bytes: P = 4 float, 8 bfloat16, 2 double), K_pad = K rounded up to a
// multiple of 8 with zero columns.  Entry (a, k) sits at
//     (k / P) * M * P + a * P + k % P.
// A warp reading rows a..a+31 of one panel reads 512 contiguous bytes, so
// both micro-kernels stream blocks straight from HBM fully coalesced.
//
//   fwd_block   acc[c] += sum_k A[a, k] X[k, c]   thread owns row a
//   trn_block   acc[c] += sum_a A[a, k] X[a, c]   thread owns column k
//
// X is a shared-memory tile with RC right-hand sides per row (broadcast to
// the warp); the accumulator type TA is float (float / bfloat16 storage) or
// double.
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

template <typename TA>
__device__ __forceinline__ TA to_acc(float v) { return (TA)v; }
__device__ __forceinline__ float elem(const float* p) { return __ldg(p); }
__device__ __forceinline__ float elem(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ double elem(const double* p) { return __ldg(p); }

// acc[c] += sum_{k < Kp} A[a, k] * Xs[k * RC + c] for the thread's row a.
// A: panel layout, M rows; rows a >= M contribute nothing (caller skips).
template <typename T, typename TA, int RC>
__device__ __forceinline__ void fwd_block(const T* __restrict__ A, int M, int Kp,
                                          const TA* __restrict__ Xs, int a, TA (&acc)[RC]) {
  constexpr int P = Panel<T>::P;
  const int np = Kp / P;
  const uint4* A4 = reinterpret_cast<const uint4*>(A) + a;
  int p = 0;
  for (; p + 2 <= np; p += 2) {
    const uint4 u0 = __ldcs(A4 + (int64_t)p * M);
    const uint4 u1 = __ldcs(A4 + (int64_t)(p + 1) * M);
    TA v0[P], v1[P];
    unpack(u0, v0);
    unpack(u1, v1);
#pragma unroll
    for (int kk = 0; kk < P; ++kk) {
      const TA* xr = Xs + (p * P + kk) * RC;
#pragma unroll
      for (int c = 0; c < RC; ++c) acc[c] = fma(v0[kk], xr[c], acc[c]);
    }
#pragma unroll
    for (int kk = 0; kk < P; ++kk) {
      const TA* xr = Xs + ((p + 1) * P + kk) * RC;
#pragma unroll
      for (int c = 0; c < RC; ++c) acc[c] = fma(v1[kk], xr[c], acc[c]);
    }
  }
  if (p < np) {
    const uint4 u0 = __ldcs(A4 + (int64_t)p * M);
    TA v0[P];
    unpack(u0, v0);
#pragma unroll
    for (int kk = 0; kk < P; ++kk) {
      const TA* xr = Xs + (p * P + kk) * RC;
#pragma unroll
      for (int c = 0; c < RC; ++c) acc[c] = fma(v0[kk], xr[c], acc[c]);
    }
  }
}

// Deep variant for warp work items: issues G panel loads before using any of
// them, so that one warp keeps G x 512 bytes in flight.  Xs rows must be
// zero beyond K (up to Kp).
template <typename T, typename TA, int RC, int G>
__device__ __forceinline__ void fwd_block_deep(const T* __restrict__ A, int M, int Kp,
                                               const TA* __restrict__ Xs, int a, bool valid,
                                               TA (&acc)[RC]) {
  constexpr int P = Panel<T>::P;
  const int np = Kp / P;
  const uint4* A4 = reinterpret_cast<const uint4*>(A) + a;
  for (int p0 = 0; p0 < np; p0 += G) {
    uint4 u[G];
#pragma unroll
    for (int g = 0; g < G; ++g)
      u[g] = (valid && p0 + g < np) ? __ldcs(A4 + (int64_t)(p0 + g) * M) : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (p0 + g >= np) break;
      TA v[P];
      unpack(u[g], v);
#pragma unroll
      for (int kk = 0; kk < P; ++kk) {
        const TA* xr = Xs + ((p0 + g) * P + kk) * RC;
#pragma unroll
        for (int c = 0; c < RC; ++c) acc[c] = fma(v[kk], xr[c], acc[c]);
      }
    }
  }
}

// acc[c] += sum_{a < M} A[a, k] * Xs[a * RC + c] for the thread's column k.
template <typename T, typename TA, int RC>
__device__ __forceinline__ void trn_block(const T* __restrict__ A, int M, const TA* __restrict__ Xs,
                                          int k, TA (&acc)[RC]) {
  constexpr int P = Panel<T>::P;
  const T* col = A + (int64_t)(k / P) * M * P + (k % P);
  int a = 0;
  for (; a + 4 <= M; a += 4) {
    const TA v0 = (TA)elem(col + (int64_t)a * P);
    const TA v1 = (TA)elem(col + (int64_t)(a + 1) * P);
    const TA v2 = (TA)elem(col + (int64_t)(a + 2) * P);
    const TA v3 = (TA)elem(col + (int64_t)(a + 3) * P);
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      TA s = acc[c];
      s = fma(v0, Xs[a * RC + c], s);
      s = fma(v1, Xs[(a + 1) * RC + c], s);
      s = fma(v2, Xs[(a + 2) * RC + c], s);
      s = fma(v3, Xs[(a + 3) * RC + c], s);
      acc[c] = s;
    }
  }
  for (; a < M; ++a) {
    const TA v0 = (TA)elem(col + (int64_t)a * P);
#pragma unroll
    for (int c = 0; c < RC; ++c) acc[c] = fma(v0, Xs[a * RC + c], acc[c]);
  }
}

// Stage rows [0, rows) of a row-major [*][R] vector block (columns c0 ..
// c0 + RC) into Xs[row * RC + c], zero-filling rows [rows, rows_pad) and
// columns beyond R.
template <typename TV, typename TA, int RC>
__device__ __forceinline__ void stage(const TV* __restrict__ X, int rows, int rows_pad, int R, int c0,
                                      TA* __restrict__ Xs) {
  for (int i = threadIdx.x; i < rows_pad * RC; i += blockDim.x) {
    const int r = i / RC, c = i % RC;
    Xs[i] = (r < rows && c0 + c < R) ? (TA)X[(int64_t)r * R + c0 + c] : (TA)0;
  }
}

}  // namespace gca
