// Householder QR (R only) of working matrices of at most 256 x 256 held in
// registers across a cluster: the preconditioner of the one-sided Jacobi SVD
// (jacobi.cu), the same factorisation as qr_r_kernel (qr.cu) -- reflections
// H_c = I - tau_c v_c v_c^T with v_c[c] = 1, beta_c = -sign(alpha) |x| --
// applied in panels of four columns with the compact-WY form
// H_k0 ... H_k0+3 = I - V T V^T.
//
// Layout.  A cluster of CL CTAs of 16 warps holds one slice: the working
// matrix X (m x n, m >= n) in 4-column blocks, block b in warp b mod (16 CL)
// of the cluster (slot b / (16 CL) of that warp), each lane holding rows
// lane + 32 q, q < 8, of the block's columns.  Per panel b: the warp owning
// block b factors it in registers (each reflector's norm and each column
// update a warp butterfly; no barrier), builds T (4 x 4) from the Gram
// entries of the panel's v's, and writes V (explicit zeros above the unit
// diagonal) and T into every CTA's shared memory (DSMEM stores into the
// peers'); one cluster barrier publishes them; then every warp applies
// Q^T = I - V T^T V^T to its blocks to the right of the panel (Y = V^T C by
// per-lane partial sums and one 16-value butterfly, Y' = T^T Y, C -= V Y').
// Panel buffers alternate, so the owner of panel b + 2 writes a buffer that
// every warp finished reading before the barrier of panel b + 1.  Compared
// with qr_r_kernel (one CTA per slice, the matrix in L2, one CTA barrier
// per reflector), the slice stays on chip and a panel costs one barrier.
// R is written transposed (R^T row-major), as qr_r_kernel writes it.

#include "common.cuh"
#include "internal.cuh"
#include "jacobi_common.cuh"

namespace wp {
namespace qrc {

constexpr int NW = 16;           // warps per CTA
constexpr int THREADS = NW * 32;
constexpr int RPL = 8;           // rows per lane: 256 rows
constexpr int PB = 4;            // panel (block) width
constexpr int kMaxDim = 32 * RPL;
constexpr int VBUF = PB * RPL * 32 + 16;   // V (4 x 256, float4 layout) + T (4 x 4)

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rows 4h..4h+3 (of a lane's 8) of column c at float offset ((c 2 + h) 32 + lane) 4.
__device__ __forceinline__ int voff(int c, int h, int lane) { return ((c * (RPL / 4) + h) * 32 + lane) * 4; }

// X: slices (p, n1, n2); the working matrix of slice s is X_s (trans = 0,
// m = n1, n = n2) or X_s^T (trans = 1, m = n2, n = n1).  Rt: (nslices, n, n),
// R^T row-major.
template <int CL>
__global__ void __launch_bounds__(THREADS, 1) qr_cols_kernel(const float* __restrict__ Xg, int n1, int n2, int trans,
                                                              int m, int n, float* __restrict__ Rt) {
  constexpr int NWT = NW * CL;                    // warps per cluster
  constexpr int SLOTS = (64 + NWT - 1) / NWT;     // blocks per warp (64 blocks at most)
  __shared__ __align__(16) float vbuf[2][VBUF];   // panel buffers: V, then T at [PB * RPL * 32]
  __shared__ __align__(16) float ysh[NW][16];     // per-warp Y exchange
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  const int wg = rank * NW + warp;                // warp number in the cluster
  const int64_t s = blockIdx.x / CL;
  const float* A = Xg + s * int64_t(n1) * n2;
  const int nbk = (n + PB - 1) / PB;

  // ---- load this warp's blocks (zero beyond m rows and n columns)
  float X[SLOTS][PB][RPL];
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int b = wg + sl * NWT;
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      const int c = b * PB + j;
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int i = lane + 32 * q;
        float v = 0.f;
        if (b < nbk && c < n && i < m) v = trans ? __ldg(A + int64_t(c) * n2 + i) : __ldg(A + int64_t(i) * n2 + c);
        X[sl][j][q] = v;
      }
    }
  }
  float* ysw = ysh[warp];

  for (int b = 0; b < nbk; ++b) {
    float* vb = vbuf[b & 1];
    const int k0 = b * PB;
    if (wg == b % NWT) {
      // ---- factor the panel (block b, slot b / NWT) in registers
      float tau[PB];
      auto factor = [&](float (&P)[PB][RPL]) {
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          const int k = k0 + c, kq = k >> 5, kl = k & 31;
          float xk = 0.f, s2 = 0.f;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            if (q == kq) xk = P[c][q];
            if (i > k) s2 = fmaf(P[c][q], P[c][q], s2);
          }
          const float alpha = __shfl_sync(0xffffffffu, xk, kl);
          s2 = warp_sum(s2);
          float t = 0.f, beta = alpha, scl = 0.f;
          if (s2 > 0.f) {
            const float nrm = sqrtf(fmaf(alpha, alpha, s2));
            beta = alpha >= 0.f ? -nrm : nrm;
            t = (beta - alpha) / beta;
            scl = 1.f / (alpha - beta);
          }
          tau[c] = t;
          // v: 1 at row k, x / (alpha - beta) below, 0 above
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int i = lane + 32 * q;
            if (i > k) P[c][q] *= scl;
          }
          // H_c applied to the panel's later columns
#pragma unroll
          for (int c2 = c + 1; c2 < PB; ++c2) {
            float d = 0.f;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
              const int i = lane + 32 * q;
              const float v = i > k ? P[c][q] : (i == k ? 1.f : 0.f);
              d = fmaf(v, P[c2][q], d);
            }
            const float w = warp_sum(d) * t;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
              const int i = lane + 32 * q;
              const float v = i > k ? P[c][q] : (i == k ? 1.f : 0.f);
              P[c2][q] = fmaf(-w, v, P[c2][q]);
            }
          }
          // R diagonal in place of alpha
#pragma unroll
          for (int q = 0; q < RPL; ++q)
            if (q == kq && lane == kl) P[c][q] = beta;
        }
        // Gram entries G[l][c] = v_l . v_c (l < c): rows >= k0 + c, where
        // v_c is 1 at row k0 + c and v_l is its stored value (rows > k0 + l)
        float G[PB][PB];
#pragma unroll
        for (int c = 1; c < PB; ++c) {
          const int k = k0 + c;
#pragma unroll
          for (int l = 0; l < c; ++l) {
            float d = 0.f;
#pragma unroll
            for (int q = 0; q < RPL; ++q) {
              const int i = lane + 32 * q;
              const float vc = i > k ? P[c][q] : (i == k ? 1.f : 0.f);
              d = fmaf(i >= k ? P[l][q] : 0.f, vc, d);
            }
            G[l][c] = warp_sum(d);
          }
        }
        // T[c][c] = tau_c, T[l][c] = -tau_c sum_{q=l}^{c-1} T[l][q] G[q][c]
        float T[PB][PB];
#pragma unroll
        for (int c = 0; c < PB; ++c) {
#pragma unroll
          for (int l = 0; l < PB; ++l) T[l][c] = 0.f;
          T[c][c] = tau[c];
#pragma unroll
          for (int l = 0; l < c; ++l) {
            float acc = 0.f;
#pragma unroll
            for (int q = l; q < c; ++q) acc = fmaf(T[l][q], G[q][c], acc);
            T[l][c] = -tau[c] * acc;
          }
        }
        // publish V and T to every CTA of the cluster
#pragma unroll
        for (int r2 = 0; r2 < CL; ++r2) {
          float* dst = cluster.map_shared_rank(vb, r2);
#pragma unroll
          for (int c = 0; c < PB; ++c) {
            const int k = k0 + c;
#pragma unroll
            for (int h = 0; h < RPL / 4; ++h) {
              float v4[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int q = 4 * h + e, i = lane + 32 * q;
                v4[e] = i > k ? P[c][q] : (i == k ? 1.f : 0.f);
              }
              *reinterpret_cast<float4*>(dst + voff(c, h, lane)) = make_float4(v4[0], v4[1], v4[2], v4[3]);
            }
          }
          float te = 0.f;   // T entry `lane` (compile-time register indices)
#pragma unroll
          for (int e = 0; e < PB * PB; ++e)
            if (lane == e) te = T[e / PB][e % PB];
          if (lane < PB * PB) dst[PB * RPL * 32 + lane] = te;
        }
        // the block keeps R: zero below the diagonal
#pragma unroll
        for (int c = 0; c < PB; ++c)
#pragma unroll
          for (int q = 0; q < RPL; ++q)
            if (lane + 32 * q > k0 + c) P[c][q] = 0.f;
      };
      const int sl_own = b / NWT;
#pragma unroll
      for (int sl = 0; sl < SLOTS; ++sl)
        if (sl == sl_own) factor(X[sl]);
    }
    cluster.sync();
    // ---- C <- (I - V T^T V^T) C for this warp's blocks right of the panel
    const float* Tm = vb + PB * RPL * 32;
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) {
      const int bs = wg + sl * NWT;
      if (bs <= b || bs >= nbk) continue;
      float y[PB * PB];
#pragma unroll
      for (int e = 0; e < PB * PB; ++e) y[e] = 0.f;
#pragma unroll
      for (int h = 0; h < RPL / 4; ++h) {
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(vb + voff(c, h, lane));
#pragma unroll
          for (int j = 0; j < PB; ++j) {
            float a2 = y[c * PB + j];
            a2 = fmaf(v.x, X[sl][j][4 * h], a2);
            a2 = fmaf(v.y, X[sl][j][4 * h + 1], a2);
            a2 = fmaf(v.z, X[sl][j][4 * h + 2], a2);
            a2 = fmaf(v.w, X[sl][j][4 * h + 3], a2);
            y[c * PB + j] = a2;
          }
        }
      }
      // totals: lane pair (2e, 2e + 1) holds Y entry e
      const float tot = multi_reduce<PB * PB>(y, lane);
      __syncwarp();
      if ((lane & 1) == 0) ysw[lane >> 1] = tot;
      __syncwarp();
      // Y' = T^T Y (Y and T read from shared memory)
      float Yp[PB][PB];
#pragma unroll
      for (int c = 0; c < PB; ++c)
#pragma unroll
        for (int j = 0; j < PB; ++j) {
          float a2 = 0.f;
#pragma unroll
          for (int l = 0; l <= c; ++l) a2 = fmaf(Tm[l * PB + c], ysw[l * PB + j], a2);
          Yp[c][j] = a2;
        }
#pragma unroll
      for (int h = 0; h < RPL / 4; ++h) {
#pragma unroll
        for (int c = 0; c < PB; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(vb + voff(c, h, lane));
#pragma unroll
          for (int j = 0; j < PB; ++j) {
            X[sl][j][4 * h] = fmaf(-v.x, Yp[c][j], X[sl][j][4 * h]);
            X[sl][j][4 * h + 1] = fmaf(-v.y, Yp[c][j], X[sl][j][4 * h + 1]);
            X[sl][j][4 * h + 2] = fmaf(-v.z, Yp[c][j], X[sl][j][4 * h + 2]);
            X[sl][j][4 * h + 3] = fmaf(-v.w, Yp[c][j], X[sl][j][4 * h + 3]);
          }
        }
      }
      __syncwarp();   // ysw is reused by the next block
    }
  }
  // ---- R^T: row c of Rt is column c of R (rows 0..c; zeros below)
  float* Rs = Rt + s * int64_t(n) * n;
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int b = wg + sl * NWT;
    if (b >= nbk) continue;
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      const int c = b * PB + j;
      if (c >= n) continue;
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int i = lane + 32 * q;
        if (i < n) Rs[int64_t(c) * n + i] = X[sl][j][q];
      }
    }
  }
  // no CTA may leave while a peer can still write its panel buffers
  cluster.sync();
}

template <int CL>
int launch(const float* X, int n1, int n2, int trans, int m, int n, int nslices, float* R, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(nslices * CL), 1, 1);
  cfg.blockDim = dim3(THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = CL;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  WP_PROFILE("qr_r", st);
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, qr_cols_kernel<CL>, X, n1, n2, trans, m, n, R));
  return launch_status();
}

}  // namespace qrc

bool qr_cols_fits(int m_len, int n_vec) { return m_len >= n_vec && m_len <= qrc::kMaxDim && n_vec >= 1; }

// 4-CTA clusters when every slice fits in one wave of them (a shorter
// per-slice time), 2-CTA clusters otherwise.
int qr_cols_launch(const float* X, int n1, int n2, int nslices, float* R, cudaStream_t st) {
  const int trans = n1 < n2 ? 1 : 0;
  const int m = trans ? n2 : n1, n = trans ? n1 : n2;
  if (!qr_cols_fits(m, n)) return WP_ERR_UNSUPPORTED;
  if (4 * nslices <= sm_count()) return qrc::launch<4>(X, n1, n2, trans, m, n, nslices, R, st);
  return qrc::launch<2>(X, n1, n2, trans, m, n, nslices, R, st);
}

}  // namespace wp
