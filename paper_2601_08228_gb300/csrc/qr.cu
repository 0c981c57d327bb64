// Householder QR (the triangular factor R only) of every slice's working
// matrix, the preconditioner of the one-sided Jacobi SVD (jacobi.cu).
//
// For a working matrix X (m x n, m >= n: the slice, or its transpose when
// it is wide) with X = Q R, the singular values of X are those of R, and
// the one-sided Jacobi method applied to the columns of R^T converges in
// markedly fewer sweeps than applied to X (R's rows come graded and nearly
// orthogonal; Drmac and Veselic, "New fast and accurate Jacobi SVD algorithm",
// SIAM J. Matrix Anal. Appl. 29, 2008).  Its converged columns R^T V = U_R S
// give the right singular vectors of X (U_R) and its singular values; Q is
// never formed.
//
// Working matrices of at most 256 x 256 go to the register-resident cluster
// kernel of qr_cols.cu instead.  Larger ones: one CTA per slice.  The working
// matrix is copied column-major into a work
// buffer (each column contiguous, L2-resident) and factored in panels of
// QR_B columns: one warp factors the panel in shared memory with Householder
// reflections H_c = I - tau_c v_c v_c^T (v_c[c] = 1; beta_c = -sign(alpha)
// |x| so that H_c x = beta_c e_c), the CTA builds the compact-WY factor T of
// H_0 ... H_{kb-1} = I - V T V^T (T upper triangular, T[c][c] = tau_c,
// T[0:c, c] = -tau_c T[0:c, 0:c] V^T v_c), and all warps apply
// Q^T = I - V T^T V^T to the trailing columns, one column per warp at a time.
// R is written column-major -- R^T row-major, lower triangle, zeros above --
// so that the Jacobi kernels take the columns of R^T as the working columns.

#include "common.cuh"
#include "internal.cuh"
#include "jacobi_common.cuh"

namespace wp {

constexpr int QR_B = 16;
constexpr int QR_CB = 2;             // trailing columns per warp at a time (one V load serves both)
constexpr int QR_RPL = 8;            // rows per lane of a trailing-update chunk (256 rows)
static_assert(QR_CB * QR_B == 32, "y' = T^T y: one (column, l) pair per lane");
// CTA sizes: 512 threads when every slice has an SM of its own (the
// per-slice critical path is shortest), 256 when the slices outnumber the
// SMs (two slices per SM overlap one's barrier waits with the other's work:
// 192 slices of 256 x 256 take 0.96 ms instead of 1.25 ms)
constexpr int QR_MAX_THREADS = 512;
constexpr int QR_MAX_M = 1024;       // panel of QR_B x m floats in shared memory (64 KB)

__device__ __forceinline__ float qr_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// X: slices (p, n1, n2); the working matrix of slice s is X_s (trans = 0,
// m = n1 rows, n = n2 columns) or X_s^T (trans = 1, m = n2, n = n1).
// W: (nslices, n, m) column-major work; Rt: (nslices, n, n), R^T row-major.
template <int QR_THREADS>
__global__ void __launch_bounds__(QR_THREADS, 65536 / (QR_THREADS * 128)) qr_r_kernel(
    const float* __restrict__ X, int n1, int n2, int trans, int m, int n, float* __restrict__ W,
    float* __restrict__ Rt) {
  extern __shared__ __align__(16) float qsm[];
  float* V = qsm;                                   // [QR_B][m] panel (rows relative to k0)
  float* T = V + QR_B * m;                          // [QR_B][QR_B] (T[row * QR_B + col])
  float* tau = T + QR_B * QR_B;                     // [QR_B]
  float* beta = tau + QR_B;                         // [QR_B]
  float* ybuf = beta + QR_B;                        // [1 + warps * QR_CB][QR_B]: z of the T build, y per warp
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  constexpr int NW = QR_THREADS / 32;
  const int64_t s = blockIdx.x;
  const float* Xs = X + s * int64_t(n1) * n2;
  float* Ws = W + s * int64_t(n) * m;
  float* Rs = Rt + s * int64_t(n) * n;

  // working matrix -> W (column-major); R <- 0
  if (trans) {
    for (int64_t idx = threadIdx.x; idx < int64_t(n) * m; idx += QR_THREADS) Ws[idx] = Xs[idx];   // rows of X_s
  } else {
    // 32 x 32 tiles transposed through one staging tile per warp (no CTA
    // barrier: every warp's tiles are independent)
    float* tile = qsm + warp * (32 * 33);
    const int tr = (m + 31) / 32, tc = (n + 31) / 32;
    for (int t = warp; t < tr * tc; t += NW) {
      const int r0 = (t / tc) * 32, c0 = (t % tc) * 32;
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i)
        v[i] = (r0 + i < m && c0 + lane < n) ? __ldg(Xs + int64_t(r0 + i) * n2 + c0 + lane) : 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) tile[i * 33 + lane] = v[i];
      __syncwarp();
#pragma unroll 4
      for (int j = 0; j < 32; ++j)
        if (r0 + lane < m && c0 + j < n) Ws[int64_t(c0 + j) * m + r0 + lane] = tile[lane * 33 + j];
      __syncwarp();
    }
  }
  for (int64_t idx = threadIdx.x; idx < int64_t(n) * n; idx += QR_THREADS) Rs[idx] = 0.f;
  __syncthreads();

  for (int k0 = 0; k0 < n; k0 += QR_B) {
    const int kb = min(QR_B, n - k0), rows = m - k0;
    // the panel; rows kb .. QR_B of V zero (a partial last panel), so that the
    // trailing update may read all QR_B of them
    for (int idx = threadIdx.x; idx < QR_B * rows; idx += QR_THREADS) {
      const int j = idx / rows, i = idx % rows;
      V[j * m + i] = j < kb ? Ws[int64_t(k0 + j) * m + k0 + i] : 0.f;
    }
    __syncthreads();
    // ---- panel factorisation (the panel in shared memory) ----
    // Column j of the panel belongs to warp j % NW, which alone updates it;
    // the owner of column c computes reflector c right after applying
    // reflector c - 1 to it, so one CTA barrier per reflector suffices.
    for (int c = 0; c < kb; ++c) {
      float* x = V + c * m;
      if (warp == c % NW) {
        const float alpha = x[c];
        float s2 = 0.f;
        for (int i = c + 1 + lane; i < rows; i += 32) s2 = fmaf(x[i], x[i], s2);
        s2 = qr_warp_sum(s2);
        float t = 0.f, b = alpha;
        if (s2 > 0.f) {
          const float nrm = sqrtf(fmaf(alpha, alpha, s2));
          b = alpha >= 0.f ? -nrm : nrm;
          t = (b - alpha) / b;
          const float scale = 1.f / (alpha - b);
          for (int i = c + 1 + lane; i < rows; i += 32) x[i] *= scale;
        }
        __syncwarp();
        if (lane == 0) {
          tau[c] = t;
          beta[c] = b;
          x[c] = 1.f;
        }
      }
      __syncthreads();
      // H_c applied to the later columns, each by its owner
      for (int j = warp; j < kb; j += NW) {
        if (j <= c) continue;
        float* y = V + j * m;
        float w = 0.f;
        for (int i = c + lane; i < rows; i += 32) w = fmaf(x[i], y[i], w);
        w = qr_warp_sum(w) * tau[c];
        for (int i = c + lane; i < rows; i += 32) y[i] = fmaf(-w, x[i], y[i]);
        __syncwarp();
      }
    }
    __syncthreads();
    if (warp == 0) {
      // R entries of the panel block, then V with explicit zeros above the unit diagonal
      for (int idx = lane; idx < kb * kb; idx += 32) {
        const int c = idx / kb, j = idx % kb;
        if (c <= j) Rs[int64_t(k0 + j) * n + k0 + c] = (c == j) ? beta[c] : V[j * m + c];   // R[k0+c][k0+j]
      }
      __syncwarp();
      for (int idx = lane; idx < kb * kb; idx += 32) {
        const int j = idx / kb, i = idx % kb;
        if (i < j) V[j * m + i] = 0.f;
      }
      __syncwarp();
    }
    __syncthreads();
    // ---- T of the panel: T[c][c] = tau_c, T[0:c, c] = -tau_c T[0:c, 0:c] (V^T v_c)[0:c] ----
    // the strictly upper Gram entries G[l][c] = v_l . v_c (c > l; v_c is zero
    // above row c) by all warps, then the recurrence by one warp (lane l owns
    // row l of T): two CTA barriers per panel
    for (int e = warp; e < QR_B * QR_B; e += NW) {
      const int l = e / QR_B, c = e % QR_B;
      if (l < c && c < kb) {
        float z = 0.f;
        for (int i = c + lane; i < rows; i += 32) z = fmaf(V[l * m + i], V[c * m + i], z);
        z = qr_warp_sum(z);
        if (lane == 0) T[l * QR_B + c] = z;   // G, overwritten by T below
      }
    }
    __syncthreads();
    if (warp == 0) {
      float trow[QR_B];                     // row `lane` of T (lanes >= QR_B idle)
#pragma unroll
      for (int c = 0; c < QR_B; ++c) trow[c] = 0.f;
#pragma unroll
      for (int c = 0; c < QR_B; ++c) {
        if (c < kb) {
          // T[l][c] = -tau_c sum_{q=l}^{c-1} T[l][q] G[q][c] for l < c; T[c][c] = tau_c
          float acc = 0.f;
#pragma unroll
          for (int q = 0; q < QR_B; ++q)
            if (q < c && lane < QR_B && q >= lane) acc = fmaf(trow[q], T[q * QR_B + c], acc);
          if (lane < c) trow[c] = -tau[c] * acc;
          else if (lane == c) trow[c] = tau[c];
        }
      }
      __syncwarp();
      if (lane < QR_B)
#pragma unroll
        for (int c = 0; c < QR_B; ++c) T[lane * QR_B + c] = (lane < kb && c < kb) ? trow[c] : 0.f;
    }
    __syncthreads();
    // ---- trailing columns: C <- (I - V T^T V^T) C, QR_CB columns per warp ----
    float* yw = ybuf + QR_B + warp * (QR_CB * QR_B);   // this warp's y (then y') values
    for (int j0 = k0 + kb + warp * QR_CB; j0 < n; j0 += NW * QR_CB) {
      const int ncol = min(QR_CB, n - j0);
      float* C[QR_CB];
#pragma unroll
      for (int q = 0; q < QR_CB; ++q) C[q] = Ws + int64_t(j0 + (q < ncol ? q : 0)) * m + k0;
      float acc[QR_CB][QR_B];
#pragma unroll
      for (int q = 0; q < QR_CB; ++q)
#pragma unroll
        for (int l = 0; l < QR_B; ++l) acc[q][l] = 0.f;
      // rows in chunks of 32 QR_RPL: every load of a chunk is issued before
      // any is used (one L2 round trip per chunk, not per row); a single
      // chunk (rows <= 256) stays in registers for the update below
      float cv[QR_CB][QR_RPL];
      for (int c0 = 0; c0 < rows; c0 += 32 * QR_RPL) {
#pragma unroll
        for (int q = 0; q < QR_CB; ++q)
#pragma unroll
          for (int r = 0; r < QR_RPL; ++r) {
            const int i = c0 + lane + 32 * r;
            cv[q][r] = i < rows ? __ldcg(C[q] + i) : 0.f;
          }
#pragma unroll
        for (int r = 0; r < QR_RPL; ++r) {
          const int i = c0 + lane + 32 * r;
          if (i < rows) {
            float v[QR_B];
#pragma unroll
            for (int l = 0; l < QR_B; ++l) v[l] = V[l * m + i];   // zero beyond kb
#pragma unroll
            for (int q = 0; q < QR_CB; ++q)
#pragma unroll
              for (int l = 0; l < QR_B; ++l) acc[q][l] = fmaf(v[l], cv[q][r], acc[q][l]);
          }
        }
      }
      // y[q][l]: lane pair (2l, 2l+1) holds the total of value l after the transposing reduction
#pragma unroll
      for (int q = 0; q < QR_CB; ++q) {
        const float y = multi_reduce<QR_B>(acc[q], lane);
        if ((lane & 1) == 0) yw[q * QR_B + (lane >> 1)] = y;
      }
      __syncwarp();
      // y' = T^T y, one (column, l) per lane: every lane reads y before any lane overwrites it
      {
        const int q = lane / QR_B, l = lane % QR_B;
        float a2 = 0.f;
        for (int t2 = 0; t2 <= l; ++t2) a2 = fmaf(T[t2 * QR_B + l], yw[q * QR_B + t2], a2);
        __syncwarp();
        yw[lane] = a2;
        __syncwarp();
      }
      float yp[QR_CB][QR_B];
#pragma unroll
      for (int q = 0; q < QR_CB; ++q)
#pragma unroll
        for (int l = 0; l < QR_B; ++l) yp[q][l] = yw[q * QR_B + l];
      __syncwarp();
      const bool one_chunk = rows <= 32 * QR_RPL;
      for (int c0 = 0; c0 < rows; c0 += 32 * QR_RPL) {
        if (!one_chunk) {
#pragma unroll
          for (int q = 0; q < QR_CB; ++q)
#pragma unroll
            for (int r = 0; r < QR_RPL; ++r) {
              const int i = c0 + lane + 32 * r;
              cv[q][r] = i < rows ? __ldcg(C[q] + i) : 0.f;
            }
        }
#pragma unroll
        for (int r = 0; r < QR_RPL; ++r) {
          const int i = c0 + lane + 32 * r;
          if (i >= rows) continue;
          float v[QR_B];
#pragma unroll
          for (int l = 0; l < QR_B; ++l) v[l] = V[l * m + i];
#pragma unroll
          for (int q = 0; q < QR_CB; ++q) {
            if (q >= ncol) continue;
            float c = cv[q][r];
#pragma unroll
            for (int l = 0; l < QR_B; ++l) c = fmaf(-v[l], yp[q][l], c);
            if (i < kb) Rs[int64_t(j0 + q) * n + k0 + i] = c;   // R[k0+i][j0+q]
            else C[q][i] = c;
          }
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }
}

bool qr_supported(int m_len, int n_vec) { return m_len >= n_vec && m_len <= QR_MAX_M && n_vec >= 1; }

size_t qr_work_bytes(int m_len, int n_vec, int nslices) {
  Sizer s;
  s.take<float>(size_t(nslices) * n_vec * m_len);   // W
  s.take<float>(size_t(nslices) * n_vec * n_vec);   // R
  return s.bytes();
}

// R of the working matrices of slices [0, nslices) of X into the work
// buffer; returns the address of R^T (row-major (nslices, n_vec, n_vec)).
int qr_r(const float* X, int n1, int n2, int nslices, void* work, size_t work_bytes, float** R_out, cudaStream_t st) {
  const int trans = n1 < n2 ? 1 : 0;
  const int m = trans ? n2 : n1, n = trans ? n1 : n2;
  if (!qr_supported(m, n)) return WP_ERR_UNSUPPORTED;
  Carver cv(work, work_bytes);
  float* W = cv.take<float>(size_t(nslices) * n * m);
  float* R = cv.take<float>(size_t(nslices) * n * n);
  if (!cv.ok) return WP_ERR_WORKSPACE;
  // working matrices of at most 256 x 256: factored in registers on a cluster
  // (qr_cols.cu); W is not used then
  if (qr_cols_fits(m, n)) {
    WP_TRY(qr_cols_launch(X, n1, n2, nslices, R, st));
    *R_out = R;
    return WP_OK;
  }
  // panel, T, tau, beta, z + per-warp y; at least the per-warp 32 x 33 staging tiles
  auto floats = [](int mm, int threads) {
    return std::max<size_t>(size_t(QR_B) * mm + QR_B * QR_B + 2 * QR_B + ((threads / 32) * QR_CB + 1) * QR_B,
                            size_t(threads / 32) * 32 * 33);
  };
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(qr_r_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(floats(QR_MAX_M, 256) * sizeof(float))));
    WP_CUDA_TRY(cudaFuncSetAttribute(qr_r_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(floats(QR_MAX_M, 512) * sizeof(float))));
    attr = true;
  }
  WP_PROFILE("qr_r", st);
  if (nslices > sm_count())
    qr_r_kernel<256><<<unsigned(nslices), 256, floats(m, 256) * sizeof(float), st>>>(X, n1, n2, trans, m, n, W, R);
  else
    qr_r_kernel<512><<<unsigned(nslices), 512, floats(m, 512) * sizeof(float), st>>>(X, n1, n2, trans, m, n, W, R);
  WP_TRY(launch_status());
  *R_out = R;
  return WP_OK;
}

}  // namespace wp
