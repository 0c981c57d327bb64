// Plain FP32 SIMT batched GEMM for the face-product Delta (Def. 2.1,
// Algorithm 1 middle loop): C[b] = op(A[b]) op(B[b]) for every frontal slice b.
//
// Row-major storage.  op(A[b]) is M x K: A[b] is M x K, or K x M if transA.
// op(B[b]) is K x N: B[b] is K x N, or N x K if transB.  C[b] is M x N.
//
// 128 x 128 x 16 CTA tile, 256 threads, 8 x 8 outputs per thread,
// register-staged double buffering of the shared-memory tiles.  Ragged edges
// are zero-filled on load and masked on store.  Three thin variants take the
// rank-r products of the w-svd rebuild (K <= 32; M <= 32 with A transposed;
// N <= 32), which are bound by their memory traffic, not their FMAs.

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

// Thin inner dimension (K <= 32: the rank-r products of the w-svd rebuild,
// C = U T): the whole K extent of a 64-row panel of A and of a 128-column
// panel of op(B) sits in shared memory at once, each of the 256 threads
// computes 4 x 8 outputs with K FMAs each (in k order, as the tiled kernel
// does), and the CTA writes its 64 x 128 tile: the product is bound by
// writing C, so tiles are small (many CTAs) and there is no k loop to
// pipeline.  A is stored M x K; op(B) is K x N, stored K x N or N x K (TB).
constexpr int TH_BM = 64, TH_BN = 128, TH_KMAX = 32;

template <bool TB>
__global__ void __launch_bounds__(256, 4) sgemm_thin_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                        float* __restrict__ C, int M, int N, int K, int64_t sA,
                                                        int64_t sB, int64_t sC, int batch) {
  __shared__ __align__(16) float As[TH_KMAX][TH_BM];
  __shared__ __align__(16) float Bs[TH_KMAX][TH_BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * TH_BM, n0 = blockIdx.x * TH_BN;
  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* Ab = A + int64_t(b) * sA;
    const float* Bb = B + int64_t(b) * sB;
    float* Cb = C + int64_t(b) * sC;
    for (int idx = tid; idx < TH_BM * K; idx += 256) {   // A panel, k-major in shared memory
      const int i = idx % TH_BM, k = idx / TH_BM;         // consecutive threads: consecutive rows
      As[k][i] = (m0 + i < M) ? __ldg(Ab + int64_t(m0 + i) * K + k) : 0.f;
    }
    for (int idx = tid; idx < TH_BN * K; idx += 256) {   // op(B) panel
      int k, j;
      if (TB) {
        j = idx / K;
        k = idx % K;
      } else {
        k = idx / TH_BN;
        j = idx % TH_BN;
      }
      Bs[k][j] = (n0 + j < N) ? __ldg(TB ? Bb + int64_t(n0 + j) * K + k : Bb + int64_t(k) * N + n0 + j) : 0.f;
    }
    __syncthreads();
    float acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    for (int k = 0; k < K; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[k][64 + tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    const bool vec_ok = (N % 4 == 0) && (reinterpret_cast<uintptr_t>(Cb) & 15u) == 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty * 4 + i;
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
    __syncthreads();   // the panels are reloaded for the next slice
  }
}

// Thin outer dimension with A transposed (M <= 32 rows of C, A stored
// K x M, op(B) = B stored K x N: the products T = U^T A of the w-svd
// rebuild): one CTA per 128 columns of C holds all M rows, runs through K in
// chunks of 32 staged in shared memory, and each thread computes 4 rows x
// 4 columns (in k order, as the tiled kernel does); the 128 x 128 tiles of
// the tiled kernel would be mostly padding here.
constexpr int TM_N = 128, TM_KC = 32, TM_MMAX = 32;

__global__ void __launch_bounds__(256, 4) sgemm_thinm_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                            float* __restrict__ C, int M, int N, int K, int64_t sA,
                                                            int64_t sB, int64_t sC, int batch) {
  __shared__ __align__(16) float As[TM_KC][TM_MMAX];
  __shared__ __align__(16) float Bs[TM_KC][TM_N];
  const int tid = threadIdx.x, tx = tid % 32, ty = tid / 32;   // rows ty + 8 i, columns 4 tx .. 4 tx + 3
  const int n0 = blockIdx.x * TM_N;
  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* Ab = A + int64_t(b) * sA;
    const float* Bb = B + int64_t(b) * sB;
    float* Cb = C + int64_t(b) * sC;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += TM_KC) {
      for (int idx = tid; idx < TM_KC * TM_MMAX; idx += 256) {
        const int k = idx / TM_MMAX, m = idx % TM_MMAX;
        As[k][m] = (k0 + k < K && m < M) ? __ldg(Ab + int64_t(k0 + k) * M + m) : 0.f;
      }
      for (int idx = tid; idx < TM_KC * TM_N; idx += 256) {
        const int k = idx / TM_N, j = idx % TM_N;
        Bs[k][j] = (k0 + k < K && n0 + j < N) ? __ldg(Bb + int64_t(k0 + k) * N + n0 + j) : 0.f;
      }
      __syncthreads();
      const int kc = K - k0 < TM_KC ? K - k0 : TM_KC;
      for (int k = 0; k < kc; ++k) {
        const float4 bv = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float av = As[k][ty + 8 * i];   // one address per warp: a broadcast
          acc[i][0] = fmaf(av, bv.x, acc[i][0]);
          acc[i][1] = fmaf(av, bv.y, acc[i][1]);
          acc[i][2] = fmaf(av, bv.z, acc[i][2]);
          acc[i][3] = fmaf(av, bv.w, acc[i][3]);
        }
      }
      __syncthreads();
    }
    const bool vec_ok = (N % 4 == 0) && (reinterpret_cast<uintptr_t>(Cb) & 15u) == 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = ty + 8 * i, gn = n0 + tx * 4;
      if (gm >= M) continue;
      float* dst = Cb + int64_t(gm) * N + gn;
      if (vec_ok && gn + 3 < N) {
        *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (gn + j < N) dst[j] = acc[i][j];
      }
    }
  }
}

// Thin N (N <= 32 columns of C, A stored M x K, B stored K x N: the
// products T = A V of the w-svd rebuild): one CTA per 128 rows of C holds
// all N columns, runs through K in chunks of 32 staged in shared memory (A
// read as 16-byte vectors along K), and each thread computes 4 rows x 4
// columns in k order.
constexpr int TN_M = 128, TN_KC = 32, TN_NMAX = 32;

__global__ void __launch_bounds__(256, 4) sgemm_thinn_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                            float* __restrict__ C, int M, int N, int K, int64_t sA,
                                                            int64_t sB, int64_t sC, int batch, int va) {
  __shared__ __align__(16) float As[TN_KC][TN_M];
  __shared__ __align__(16) float Bs[TN_KC][TN_NMAX];
  const int tid = threadIdx.x, tx = tid % 8, ty = tid / 8;   // columns 4 tx .., rows 4 ty ..
  const int m0 = blockIdx.y * TN_M;
  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* Ab = A + int64_t(b) * sA;
    const float* Bb = B + int64_t(b) * sB;
    float* Cb = C + int64_t(b) * sC;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += TN_KC) {
      // A chunk: thread takes 4 consecutive k of one row (consecutive threads: consecutive rows)
      for (int idx = tid; idx < TN_M * (TN_KC / 4); idx += 256) {
        const int i = idx % TN_M, kq = idx / TN_M, k = k0 + 4 * kq;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (m0 + i < M) {
          const float* src = Ab + int64_t(m0 + i) * K + k;
          if (va && k + 3 < K) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(src));
            v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (k + e < K) v[e] = __ldg(src + e);
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) As[4 * kq + e][i] = v[e];
      }
      for (int idx = tid; idx < TN_KC * TN_NMAX; idx += 256) {
        const int k = idx / TN_NMAX, j = idx % TN_NMAX;
        Bs[k][j] = (k0 + k < K && j < N) ? __ldg(Bb + int64_t(k0 + k) * N + j) : 0.f;
      }
      __syncthreads();
      const int kc = K - k0 < TN_KC ? K - k0 : TN_KC;
      for (int k = 0; k < kc; ++k) {
        const float4 av = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
        const float4 bv = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
        const float a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc[i][0] = fmaf(a4[i], bv.x, acc[i][0]);
          acc[i][1] = fmaf(a4[i], bv.y, acc[i][1]);
          acc[i][2] = fmaf(a4[i], bv.z, acc[i][2]);
          acc[i][3] = fmaf(a4[i], bv.w, acc[i][3]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty * 4 + i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = tx * 4 + j;
        if (gn < N) Cb[int64_t(gm) * N + gn] = acc[i][j];
      }
    }
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
  if (!transA && K <= TH_KMAX && (M + TH_BM - 1) / TH_BM <= 65535) {
    const dim3 tg((N + TH_BN - 1) / TH_BN, (M + TH_BM - 1) / TH_BM, std::min(batch, 65535));
    WP_PROFILE("sgemm_fp32_thin", st);
    if (transB) sgemm_thin_kernel<true><<<tg, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch);
    else sgemm_thin_kernel<false><<<tg, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch);
    return launch_status();
  }
  if (!transA && !transB && N <= TN_NMAX && K > TH_KMAX && (M + TN_M - 1) / TN_M <= 65535) {
    const dim3 tg(1, (M + TN_M - 1) / TN_M, std::min(batch, 65535));
    const int va4 = aligned16(A) && (K % 4 == 0);
    WP_PROFILE("sgemm_fp32_thin", st);
    sgemm_thinn_kernel<<<tg, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch, va4);
    return launch_status();
  }
  if (transA && !transB && M <= TM_MMAX) {
    const dim3 tg((N + TM_N - 1) / TM_N, 1, std::min(batch, 65535));
    WP_PROFILE("sgemm_fp32_thin", st);
    sgemm_thinm_kernel<<<tg, 256, 0, st>>>(A, B, C, M, N, K, sA, sB, sC, batch);
    return launch_status();
  }
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
