// Definitions shared by the batched one-sided Jacobi kernels (jacobi.cu,
// jacobi_block.cu): launch arguments, the round-robin pair map, cluster
// barrier and the multi-value warp reduction.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace wp {

namespace cg = cooperative_groups;

constexpr int JAC_THREADS = 512;
constexpr int kStrictSweeps = 20;

struct JacobiArgs {
  const float* X;      // slices (p, n1, n2)
  int n1, n2;
  int trans;           // 1: working columns are the rows of the slice
  int m_len, n_vec, n_pad, rpc;
  int slice0;          // first slice handled by this launch
  int r;
  float* vec_out;      // (p, m_len, r): leading r unit vectors, slice-indexed
  float* sig_out;      // (p, r): leading r singular values, descending
  float tol;
  int max_sweeps;
  int* status;
  unsigned long long* stats;   // [0] += sweeps of each slice, [1] = max sweeps
};

__device__ __forceinline__ void pair_of(int i, int k, int n, int& a, int& b) {
  // circle method: position 0 fixed, positions 1..n-1 rotate by k
  auto elem = [&](int pos) {
    int q = pos - 1 + k;
    q -= (q >= n - 1) ? (n - 1) : 0;
    return pos == 0 ? 0 : 1 + q;
  };
  a = elem(i);
  b = elem(n - 1 - i);
}

template <int CL>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (CL > 1) cg::this_cluster().sync();
  else __syncthreads();
}

template <int CL>
__device__ __forceinline__ float gather(const float* part, int buf, int n_pad, int i) {
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < CL; ++q) s += part[(size_t(buf) * CL + q) * n_pad + i];
  return s;
}

// Sum PPW per-lane values over the 32 lanes of a warp with a multi-value
// butterfly: after the call, lane l holds the warp total of value
// (l >> (5 - log2 PPW)).  log2(PPW) + (5 - log2 PPW) shuffle stages, 2 PPW - 1
// + (5 - log2 PPW) shuffles in all (9 for PPW = 8, instead of 40).
template <int PPW>
__device__ __forceinline__ float multi_reduce(float (&v)[PPW], int lane) {
  int c = PPW;
  int d = 16;
#pragma unroll
  for (int step = 0; (1 << step) < PPW; ++step) {
    c >>= 1;
    const bool upper = (lane & d) != 0;
#pragma unroll
    for (int i = 0; i < PPW / 2; ++i) {
      if (i < c) {
        const float send = upper ? v[i] : v[i + c];
        const float keep = upper ? v[i + c] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, d);
      }
    }
    d >>= 1;
  }
  float t = v[0];
#pragma unroll
  for (; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
  return t;
}

// Launch the block-cyclic register-resident kernel (jacobi_block.cu) when the
// slice shape suits it; WP_ERR_UNSUPPORTED otherwise (the caller then uses
// the shared-memory kernel).
int jacobi_block_launch(const JacobiArgs& a, int nslices, cudaStream_t st);

// Column-split register-resident kernel on 2-CTA clusters (jacobi_cols.cu):
// working matrices of at most 256 rows and 192..256 columns.
bool jacobi_cols_fits(int m_len, int n_vec);
bool jacobi_cols_enabled();
int jacobi_cols_launch(const JacobiArgs& a, int nslices, cudaStream_t st);

}  // namespace wp
