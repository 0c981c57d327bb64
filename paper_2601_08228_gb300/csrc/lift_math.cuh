// Register-level lazy-Haar lifting of one tube group (Sec. II-A).
//
// The lazy choice P_j = I, U_j = I/2 has support 2^L: the G = 2^L consecutive
// tube entries of group g (slices g*G .. g*G+G-1) transform independently of
// every other group.  Each routine below maps one group held in registers;
// the kernels gather / scatter the group from / to global memory.
//
// Local Mallat order inside a group: [s_L | d_L | d_{L-1} (2) | ... | d_1 (G/2)],
// i.e. d_j occupies local indices [G >> j, G >> (j-1)).  Local index t of group
// g lives in global slice mallat_slice(t, g, p, L) of the Mallat-ordered tensor
// (Eq. 1): s_L at slice g, and the d_j coefficient k of group g at
// p/2^j + g*2^(L-j) + k.
#pragma once

#include <stdint.h>

namespace wp {

__host__ __device__ constexpr int ilog2_floor(int t) { return t <= 1 ? 0 : 1 + ilog2_floor(t >> 1); }

template <int L>
__device__ __forceinline__ int64_t mallat_slice(int t, int64_t g, int64_t p) {
  if (t == 0) return g;
  const int hb = ilog2_floor(t);       // t in [2^hb, 2^(hb+1)) -> level j = L - hb
  return (p >> (L - hb)) + g * (int64_t(1) << hb) + (t - (1 << hb));
}

// Forward W_[L] of one group (Algorithm 1 forward loop, 1-based pairs):
// d = x[2k-1] - x[2k], s = x[2k] + d/2.  x spatial order -> y local Mallat.
template <int L>
__device__ __forceinline__ void lift_group(const float* x, float* y) {
  constexpr int G = 1 << L;
  float s[G];
#pragma unroll
  for (int i = 0; i < G; ++i) s[i] = x[i];
#pragma unroll
  for (int j = 1; j <= L; ++j) {
    const int half = G >> j;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float a = s[2 * k], b = s[2 * k + 1];
      const float d = a - b;
      y[half + k] = d;
      s[k] = fmaf(0.5f, d, b);         // 0.5*d is exact: same as b + d/2
    }
  }
  y[0] = s[0];
}

// Inverse W_[L]^{-1} of one group (Eq. 3, Algorithm 1 inverse loop):
// x[2k] = s - d/2, x[2k-1] = d + x[2k], coarsest level first.
template <int L>
__device__ __forceinline__ void ilift_group(const float* y, float* x) {
  constexpr int G = 1 << L;
  float s[G];
  s[0] = y[0];
#pragma unroll
  for (int j = L; j >= 1; --j) {
    const int half = G >> j;
#pragma unroll
    for (int k = half - 1; k >= 0; --k) {
      const float d = y[half + k];
      const float even = fmaf(-0.5f, d, s[k]);
      s[2 * k] = d + even;
      s[2 * k + 1] = even;
    }
  }
#pragma unroll
  for (int i = 0; i < G; ++i) x[i] = s[i];
}

// W^T of one group: transposes of the forward level maps, coarsest first:
// g_a = g_s/2 + g_d, g_b = g_s/2 - g_d.  Local Mallat -> spatial.
template <int L>
__device__ __forceinline__ void lift_adjoint_group(const float* g, float* h) {
  constexpr int G = 1 << L;
  float s[G];
  s[0] = g[0];
#pragma unroll
  for (int j = L; j >= 1; --j) {
    const int half = G >> j;
#pragma unroll
    for (int k = half - 1; k >= 0; --k) {
      const float gd = g[half + k];
      const float gs = s[k];
      s[2 * k] = fmaf(0.5f, gs, gd);
      s[2 * k + 1] = fmaf(0.5f, gs, -gd);
    }
  }
#pragma unroll
  for (int i = 0; i < G; ++i) h[i] = s[i];
}

// W^{-T} of one group: transposes of the inverse level maps, finest first:
// g_s = g_a + g_b, g_d = (g_a - g_b)/2.  Spatial -> local Mallat.
template <int L>
__device__ __forceinline__ void ilift_adjoint_group(const float* h, float* g) {
  constexpr int G = 1 << L;
  float s[G];
#pragma unroll
  for (int i = 0; i < G; ++i) s[i] = h[i];
#pragma unroll
  for (int j = 1; j <= L; ++j) {
    const int half = G >> j;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float a = s[2 * k], b = s[2 * k + 1];
      g[half + k] = 0.5f * (a - b);
      s[k] = a + b;
    }
  }
  g[0] = s[0];
}

}  // namespace wp
