// Plain FP32 SIMT batched GEMM for the face-product Delta (Def. 2.1,
// Algorithm 1 middle loop): C[b] = op(A[b]) op(B[b]) for every frontal slice b.
//
// Row-major storage.  op(A[b]) is M x K: A[b] is M x K, or K x M if transA.
// op(B[b]) is K x N: B[b] is K x N, or N x K if transB.  C[b] is M x N.
//
// 128 x 128 x 16 CTA tile, 256 threads, 8 x 8 outputs per thread,
// register-staged double buffering of the shared-memory tiles.  Ragged edges
// are zero-filled on load and masked on store.

#include "common.cuh"

namespace wp {

constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 16;

// Eight consecutive elements base[row * ld + c0 .. c0 + 7] (zero outside
// row_ext x c_ext); 16-byte loads when `vec` (c_ext % 4 == 0, 16-byte base).
__device__ __forceinline__ void sg_load8(const float* __restrict__ base, int64_t ld, int row, int row_ext, int c0,
                                         int c_ext, bool vec, float (&r)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) r[i] = 0.f;
  if (row >= row_ext) return;
  const float* src = base + int64_t(row) * ld + c0;
  if (vec) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (c0 + 4 * h < c_ext) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(src + 4 * h));
        r[4 * h] = v.x; r[4 * h + 1] = v.y; r[4 * h + 2] = v.z; r[4 * h + 3] = v.w;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (c0 + i < c_ext) r[i] = __ldg(src + i);
  }
}

// 128 x 128 x 16 CTA tile, 256 threads, 8 x 8 outputs per thread (two 4 x 4
// quadrants: conflict-free float4 shared reads), tiles staged k-major in
// shared memory, the next k-tile's global loads (8 consecutive elements of
// A and of B per thread, 16-byte vectors where the storage allows) in
// registers while the current one is multiplied.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256, 2) sgemm_batched_kernel(
    const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C, int M, int N,
    int K, int64_t sA, int64_t sB, int64_t sC, int batch, int va, int vb) {
  __shared__ __align__(16) float As[2][SG_BK][SG_BM];
  __shared__ __align__(16) float Bs[2][SG_BK][SG_BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * SG_BM, n0 = blockIdx.x * SG_BN;
  // load roles: along the contiguous dimension, 8 elements per thread; for
  // k-contiguous operands the 32 lanes of a warp take 32 rows (conflict-free
  // transposing shared stores)
  const int a_row = TA ? (tid >> 4) : (tid & 127), a_c = TA ? (tid & 15) * 8 : (tid >> 7) * 8;
  const int b_row = TB ? (tid & 127) : (tid >> 4), b_c = TB ? (tid >> 7) * 8 : (tid & 15) * 8;

  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* Ab = A + int64_t(b) * sA;
    const float* Bb = B + int64_t(b) * sB;
    float* Cb = C + int64_t(b) * sC;
    float ra[8], rb[8];
    auto load = [&](int k0) {
      if (TA) sg_load8(Ab, M, k0 + a_row, K, m0 + a_c, M, va, ra);     // stored K x M
      else sg_load8(Ab, K, m0 + a_row, M, k0 + a_c, K, va, ra);        // stored M x K
      if (TB) sg_load8(Bb, K, n0 + b_row, N, k0 + b_c, K, vb, rb);     // stored N x K
      else sg_load8(Bb, N, k0 + b_row, K, n0 + b_c, N, vb, rb);        // stored K x N
    };
    auto store = [&](int buf) {
      if (TA) {
        *reinterpret_cast<float4*>(&As[buf][a_row][a_c]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
        *reinterpret_cast<float4*>(&As[buf][a_row][a_c + 4]) = make_float4(ra[4], ra[5], ra[6], ra[7]);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) As[buf][a_c + i][a_row] = ra[i];
      }
      if (TB) {
#pragma unroll
        for (int i = 0; i < 8; ++i) Bs[buf][b_c + i][b_row] = rb[i];
      } else {
        *reinterpret_cast<float4*>(&Bs[buf][b_row][b_c]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
        *reinterpret_cast<float4*>(&Bs[buf][b_row][b_c + 4]) = make_float4(rb[4], rb[5], rb[6], rb[7]);
      }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int ktiles = (K + SG_BK - 1) / SG_BK;
    load(0);
    store(0);
    __syncthreads();
    for (int kt = 0; kt < ktiles; ++kt) {
      const int cur = kt & 1;
      if (kt + 1 < ktiles) load((kt + 1) * SG_BK);
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
      if (kt + 1 < ktiles) store(cur ^ 1);
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
  // 16-byte loads where each operand's contiguous dimension is a multiple of 4
  const int va = aligned16(A) && ((transA ? M : K) % 4 == 0);
  const int vb = aligned16(B) && ((transB ? K : N) % 4 == 0);
  WP_PROFILE("sgemm_fp32", st);
  if (!transA && !transB)
    sgemm_batched_kernel<false, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch, va, vb);
  else if (!transA && transB)
    sgemm_batched_kernel<false, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch, va, vb);
  else if (transA && !transB)
    sgemm_batched_kernel<true, false><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch, va, vb);
  else
    sgemm_batched_kernel<true, true><<<grid, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch, va, vb);
  return launch_status();
}

}  // namespace wp
