// Plain FP32 SIMT batched GEMM for the face-product Delta (Def. 2.1,
// Algorithm 1 middle loop): C[b] = op(A[b]) op(B[b]) for every frontal slice b.
//
// Row-major storage.  op(A[b]) is M x K: A[b] is M x K, or K x M if transA.
// op(B[b]) is K x N: B[b] is K x N, or N x K if transB.  C[b] is M x N.
//
// 128 x 128 x 8 CTA tile, 256 threads, 8 x 8 outputs per thread (two 4 x 4
// quadrants so that shared-memory reads are conflict-free float4 broadcasts),
// register-staged double buffering of the shared-memory tiles.  Ragged edges
// are zero-filled on load and masked on store.

#include "common.cuh"

namespace wp {

constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_batched_kernel(
    const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C, int M, int N,
    int K, int64_t sA, int64_t sB, int64_t sC, int batch) {
  __shared__ __align__(16) float As[2][SG_BK][SG_BM];
  __shared__ __align__(16) float Bs[2][SG_BK][SG_BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * SG_BM, n0 = blockIdx.x * SG_BN;

  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* Ab = A + int64_t(b) * sA;
    const float* Bb = B + int64_t(b) * sB;
    float* Cb = C + int64_t(b) * sC;

    // per-thread load coordinates (4 elements of A and 4 of B per k-tile)
    float ra[4], rb[4];
    auto load_a = [&](int k0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int m, k;
        if (!TA) { m = tid / 2; k = (tid % 2) * 4 + i; }     // k contiguous in memory
        else { k = tid / 32; m = (tid % 32) * 4 + i; }       // m contiguous in memory
        const int gm = m0 + m, gk = k0 + k;
        float v = 0.f;
        if (gm < M && gk < K) v = TA ? Ab[int64_t(gk) * M + gm] : Ab[int64_t(gm) * K + gk];
        ra[i] = v;
      }
    };
    auto store_a = [&](int buf) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int m, k;
        if (!TA) { m = tid / 2; k = (tid % 2) * 4 + i; }
        else { k = tid / 32; m = (tid % 32) * 4 + i; }
        As[buf][k][m] = ra[i];
      }
    };
    auto load_b = [&](int k0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int n, k;
        if (!TB) { k = tid / 32; n = (tid % 32) * 4 + i; }   // n contiguous in memory
        else { n = tid / 2; k = (tid % 2) * 4 + i; }         // k contiguous in memory
        const int gn = n0 + n, gk = k0 + k;
        float v = 0.f;
        if (gn < N && gk < K) v = TB ? Bb[int64_t(gn) * K + gk] : Bb[int64_t(gk) * N + gn];
        rb[i] = v;
      }
    };
    auto store_b = [&](int buf) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int n, k;
        if (!TB) { k = tid / 32; n = (tid % 32) * 4 + i; }
        else { n = tid / 2; k = (tid % 2) * 4 + i; }
        Bs[buf][k][n] = rb[i];
      }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int ktiles = (K + SG_BK - 1) / SG_BK;
    load_a(0);
    load_b(0);
    store_a(0);
    store_b(0);
    __syncthreads();
    for (int kt = 0; kt < ktiles; ++kt) {
      const int cur = kt & 1;
      if (kt + 1 < ktiles) {
        load_a((kt + 1) * SG_BK);
        load_b((kt + 1) * SG_BK);
      }
#pragma unroll
      for (int k = 0; k < SG_BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (kt + 1 < ktiles) {
        store_a(cur ^ 1);
        store_b(cur ^ 1);
      }
      __syncthreads();
    }

    const bool vec_ok = (N % 4 == 0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      if (gm >= M) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int gn = n0 + h * 64 + tx * 4;
        float* dst = Cb + int64_t(gm) * N + gn;
        if (vec_ok && gn + 3 < N) {
          *reinterpret_cast<float4*>(dst) =
              make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (gn + j < N) dst[j] = acc[i][h * 4 + j];
        }
      }
    }
    __syncthreads();
  }
}

int sgemm_batched(const float* A, const float* B, float* C, int M, int N, int K, bool transA,
                  bool transB, int batch, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return WP_OK;
  if (K <= 0) {
    WP_CUDA_TRY(cudaMemsetAsync(C, 0, size_t(M) * N * batch * sizeof(float), st));
    return WP_OK;
  }
  const int64_t sA = int64_t(M) * K, sB = int64_t(K) * N, sC = int64_t(M) * N;
  dim3 grid((N + SG_BN - 1) / SG_BN, (M + SG_BM - 1) / SG_BM, std::min(batch, 65535));
  if (grid.y > 65535) return WP_ERR_SHAPE;
  WP_PROFILE("sgemm_fp32", st);
  if (!transA && !transB) sgemm_batched_kernel<false, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch);
  else if (!transA && transB) sgemm_batched_kernel<false, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch);
  else if (transA && !transB) sgemm_batched_kernel<true, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch);
  else sgemm_batched_kernel<true, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch);
  return launch_status();
}

}  // namespace wp
