// One-sided Jacobi SVD for slices too large for a thread-block cluster's
// shared memory (Algorithm 2's facewise SVD and Def. 2.6's pseudo-inverse of
// the wavelet-domain slices, e.g. the 610 x 610 and 1476 x 1476 blur
// operators of the deblurring experiments of Sec. IV-C).
//
// The working columns of every slice (the slice itself when n1 >= n2, its
// transpose otherwise; m_len rows, n_pad columns) live in a global-memory
// work buffer, column-major, so a block of B consecutive columns is one
// contiguous run of B * m_len floats.  A sweep is a round-robin tournament
// over the nb = n_pad / B column blocks: nb - 1 rounds of nb / 2 disjoint
// block pairs.  A work item is one block pair of one slice: a CTA copies the
// two blocks into shared memory, meets every column of one block with every
// column of the other (B sub-rounds of B disjoint column pairs, one warp per
// pair) -- and, in the first round of a sweep, every block also meets
// itself, so every column pair meets once per sweep -- and writes the blocks
// back.  The rotation of a pair is the one of the other Jacobi kernels
// (jacobi.cu): alpha = |x|^2, beta = |y|^2, gamma = x . y computed afresh
// from the columns, zeta = (beta - alpha) / (2 gamma), t = sign(zeta) /
// (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t, rotated when
// |gamma| > tol sqrt(alpha beta); columns below (m_len eps)^2 max |x|^2 are
// numerically zero and never rotated.  A sweep in which no pair's cosine
// |gamma| / sqrt(alpha beta) reaches sqrt(tol) ends the iteration of that
// slice (quadratic convergence: the next sweep would leave cosines of order
// tol).
//
// The kernel is persistent and launched cooperatively (all CTAs resident):
// the CTAs take the work items of a round in turn and meet at a grid-wide
// barrier between rounds.  The barrier's wait is bounded (2 s); on expiry
// the kernel records WP_ERR_TIMEOUT, raises an abort flag that every CTA
// checks, and returns.  Data written by other CTAs of the same launch (the
// columns, norms, flags) is read through L2 only (ld.global.cg).

#include "common.cuh"
#include "internal.cuh"
#include "jacobi_common.cuh"
#include "tc_ptx.cuh"

namespace wp {
namespace jglobal {

struct Args {
  JacobiArgs a;
  int nslices;
  int nb;                // column blocks (even); n_pad = nb * B
  int n_pad;
  float* W;              // [nslices][n_pad][m_len] working columns
  float* norms;          // [nslices][n_pad] squared column norms
  unsigned* nmax;        // [nslices] largest squared norm of the sweep (float bits)
  int* big;              // [nslices] a pair above the stopping bound in this sweep
  int* done;             // [nslices] sweeps the slice needed (0: still rotating)
  int* left;             // [1] slices still rotating after the last sweep
  unsigned* bar;         // [2] grid barrier: arrivals, generation
  int* abort;            // [1] a barrier wait expired
};

// Bounded grid-wide barrier (all CTAs resident: cooperative launch).
__device__ bool grid_barrier(const Args& g) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = __ldcg(g.abort) == 0;
    if (ok) {
      volatile unsigned* gen = g.bar + 1;
      const unsigned my_gen = *gen;
      __threadfence();
      if (atomicAdd(g.bar, 1u) == gridDim.x - 1) {
        atomicExch(g.bar, 0u);
        __threadfence();
        atomicAdd(g.bar + 1, 1u);
      } else {
        const uint64_t t0 = ptx::globaltimer();
        while (*gen == my_gen) {
          if (__ldcg(g.abort) != 0) { ok = 0; break; }
          if (ptx::globaltimer() - t0 > ptx::kWaitLimitNs) {
            report_device_error(g.a.status, WP_ERR_TIMEOUT);
            atomicExch(g.abort, 1);
            ok = 0;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rotate the column pair (x, y) (shared memory, m rows) if it is not yet
// orthogonal; true when its cosine exceeds the stopping bound.
__device__ __forceinline__ bool rotate_pair(float* x, float* y, int m, float tol, float negl, int lane) {
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int r = lane; r < m; r += 32) {
    const float u = x[r], v = y[r];
    al = fmaf(u, u, al);
    be = fmaf(v, v, be);
    ga = fmaf(u, v, ga);
  }
  al = warp_sum(al);
  be = warp_sum(be);
  ga = warp_sum(ga);
  if (!(al > negl && be > negl) || ga == 0.f) return false;
  const float ab = al * be;
  const bool big = ga * ga > tol * ab;
  if (fabsf(ga) <= tol * sqrtf(ab)) return big;
  const float zeta = __fdividef(be - al, 2.f * ga);
  const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
  // correctly rounded square root and division: a few-ulp reciprocal square
  // root would bias every rotation the same way, and a column of an n x n
  // slice takes about 12 n rotations (1.5e-4 of shrinkage measured at n = 640)
  const float c = 1.f / sqrtf(fmaf(t, t, 1.f));
  const float s = c * t;
  for (int r = lane; r < m; r += 32) {
    const float u = x[r], v = y[r];
    x[r] = fmaf(c, u, -s * v);
    y[r] = fmaf(s, u, c * v);
  }
  return big;
}

// Block id at position pos of round k of the circle tournament on nb players.
__device__ __forceinline__ int circle(int pos, int k, int nb) {
  return pos == 0 ? 0 : 1 + (pos - 1 + k) % (nb - 1);
}

template <int B>
__global__ void __launch_bounds__(B * 32) jacobi_global_kernel(Args g) {
  extern __shared__ __align__(16) float sm[];     // [2B][m_len]; the 32 x 33 staging tile at load
  const JacobiArgs& a = g.a;
  const int m = a.m_len, n_pad = g.n_pad, nb = g.nb, ns = g.nslices;
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  const int nthreads = B * 32;

  // ---- working columns: W[s][c][R] = X_s[R][c] (or X_s[c][R] when transposed), zero padded
  {
    const int tr = (m + 31) / 32, tc = n_pad / 32;     // n_pad is a multiple of 32
    const int64_t tiles = int64_t(ns) * tr * tc;
    float* tile = sm;                                  // [32][33]
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
      const int s = int(t / (int64_t(tr) * tc));
      const int rem = int(t - int64_t(s) * tr * tc);
      const int R0 = (rem / tc) * 32, c0 = (rem % tc) * 32;
      const float* X = a.X + int64_t(a.slice0 + s) * a.n1 * a.n2;
      float* Ws = g.W + int64_t(s) * n_pad * m;
      for (int idx = threadIdx.x; idx < 32 * 32; idx += nthreads) {
        const int i = idx / 32, j = idx % 32;
        if (!a.trans) {
          // tile row i = slice row R0 + i, lane j = column c0 + j (coalesced along the slice row)
          const int R = R0 + i, c = c0 + j;
          tile[i * 33 + j] = (R < m && c < a.n_vec) ? X[int64_t(R) * a.n2 + c] : 0.f;
        } else {
          // the slice's row c is working column c: copy along it
          const int c = c0 + i, R = R0 + j;
          if (R < m) Ws[int64_t(c) * m + R] = (c < a.n_vec) ? X[int64_t(c) * a.n2 + R] : 0.f;
        }
      }
      __syncthreads();
      if (!a.trans) {
        for (int idx = threadIdx.x; idx < 32 * 32; idx += nthreads) {
          const int j = idx / 32, i = idx % 32;        // column c0 + j, rows R0 + i (coalesced along W)
          const int R = R0 + i;
          if (R < m) Ws[int64_t(c0 + j) * m + R] = tile[i * 33 + j];
        }
      }
      __syncthreads();
    }
  }
  if (!grid_barrier(g)) return;

  // squared norms of the columns of slice-columns [first, ...), stride, and
  // the slice maxima (atomicMax on the bit patterns of non-negative floats)
  auto norms_pass = [&](bool all) {
    const int64_t cols = int64_t(ns) * n_pad;
    for (int64_t wc = int64_t(blockIdx.x) * B + warp; wc < cols; wc += int64_t(gridDim.x) * B) {
      const int s = int(wc / n_pad);
      if (!all && __ldcg(g.done + s) != 0) continue;
      const float* col = g.W + wc * m;
      float acc = 0.f;
      for (int r = lane; r < m; r += 32) {
        const float v = __ldcg(col + r);
        acc = fmaf(v, v, acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        g.norms[wc] = acc;
        atomicMax(g.nmax + s, __float_as_uint(acc));
      }
    }
  };

  const float meps = float(m) * 1.1920929e-7f;
  __shared__ int s_big;
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    const float tol = sweep < kStrictSweeps ? a.tol : 8.f * a.tol;
    norms_pass(false);
    if (!grid_barrier(g)) return;
    for (int k = 0; k < nb - 1; ++k) {
      const int64_t items = int64_t(ns) * (nb / 2);
      for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int s = int(it / (nb / 2)), i = int(it % (nb / 2));
        if (__ldcg(g.done + s) != 0) continue;
        const float nmx = __uint_as_float(__ldcg(g.nmax + s));
        if (!(nmx > 0.f)) continue;                    // an all-zero slice: nothing to rotate
        const float negl = nmx * meps * meps;
        const int P = circle(i, k, nb), Q = circle(nb - 1 - i, k, nb);
        float* gp = g.W + (int64_t(s) * n_pad + int64_t(P) * B) * m;
        float* gq = g.W + (int64_t(s) * n_pad + int64_t(Q) * B) * m;
        const int len = B * m;
        const bool v4 = (m % 4) == 0;
        if (v4) {
          for (int idx = threadIdx.x; idx < len / 4; idx += nthreads) {
            reinterpret_cast<float4*>(sm)[idx] = __ldcg(reinterpret_cast<const float4*>(gp) + idx);
            reinterpret_cast<float4*>(sm + len)[idx] = __ldcg(reinterpret_cast<const float4*>(gq) + idx);
          }
        } else {
          for (int idx = threadIdx.x; idx < len; idx += nthreads) {
            sm[idx] = __ldcg(gp + idx);
            sm[len + idx] = __ldcg(gq + idx);
          }
        }
        if (threadIdx.x == 0) s_big = 0;
        __syncthreads();
        int big = 0;
        if (k == 0) {
          // every block meets itself: warps [0, B/2) on P, [B/2, B) on Q
          const int half = B / 2, j = warp % half;
          float* blk = sm + (warp < half ? 0 : len);
          for (int S = 0; S < B - 1; ++S) {
            const int ca = circle(j, S, B), cb = circle(B - 1 - j, S, B);
            big |= rotate_pair(blk + ca * m, blk + cb * m, m, tol, negl, lane);
            __syncthreads();
          }
        }
        // column j of P meets column (j + S) mod B of Q
        for (int S = 0; S < B; ++S) {
          big |= rotate_pair(sm + warp * m, sm + len + ((warp + S) % B) * m, m, tol, negl, lane);
          __syncthreads();
        }
        if (big && lane == 0) atomicOr(&s_big, 1);
        if (v4) {
          for (int idx = threadIdx.x; idx < len / 4; idx += nthreads) {
            reinterpret_cast<float4*>(gp)[idx] = reinterpret_cast<const float4*>(sm)[idx];
            reinterpret_cast<float4*>(gq)[idx] = reinterpret_cast<const float4*>(sm + len)[idx];
          }
        } else {
          for (int idx = threadIdx.x; idx < len; idx += nthreads) {
            gp[idx] = sm[idx];
            gq[idx] = sm[len + idx];
          }
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_big) atomicOr(g.big + s, 1);
      }
      if (!grid_barrier(g)) return;
    }
    // sweep bookkeeping (CTA 0), then one more barrier so every CTA sees it
    if (blockIdx.x == 0) {
      int left = 0;
      for (int s = threadIdx.x; s < ns; s += nthreads) {
        if (__ldcg(g.done + s) == 0) {
          if (__ldcg(g.big + s) == 0) g.done[s] = sweep + 1;
          else ++left;
        }
        g.big[s] = 0;
        g.nmax[s] = 0u;
      }
      left = __syncthreads_count(left > 0);
      if (threadIdx.x == 0) *g.left = left;
    }
    if (!grid_barrier(g)) return;
    if (__ldcg(g.left) == 0) break;
  }

  // ---- exact norms, then the leading r unit columns in descending order
  norms_pass(true);
  if (!grid_barrier(g)) return;
  const int64_t cols = int64_t(ns) * a.n_vec;
  for (int64_t wc = int64_t(blockIdx.x) * B + warp; wc < cols; wc += int64_t(gridDim.x) * B) {
    const int s = int(wc / a.n_vec), c = int(wc % a.n_vec);
    const float* nrm = g.norms + int64_t(s) * n_pad;
    const float sc = __ldcg(nrm + c);
    int pos = 0;
    for (int q = lane; q < a.n_vec; q += 32) {
      const float sq = __ldcg(nrm + q);
      pos += (sq > sc) || (sq == sc && q < c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pos += __shfl_xor_sync(0xffffffffu, pos, o);
    if (pos >= a.r) continue;
    const int slice = a.slice0 + s;
    const float sg = sqrtf(sc);
    const float inv = sg > 0.f ? 1.f / sg : 0.f;
    const float* col = g.W + (int64_t(s) * n_pad + c) * m;
    float* vo = a.vec_out + int64_t(slice) * m * a.r;
    for (int R = lane; R < m; R += 32) vo[int64_t(R) * a.r + pos] = __ldcg(col + R) * inv;
    if (lane == 0) a.sig_out[int64_t(slice) * a.r + pos] = sg;
  }
  if (blockIdx.x == 0) {
    for (int s = threadIdx.x; s < ns; s += nthreads) {
      const int d = __ldcg(g.done + s);
      if (d == 0) report_device_error(a.status, WP_ERR_NOT_CONVERGED);
      if (a.stats) {
        const unsigned long long sw = (unsigned long long)(d ? d : a.max_sweeps);
        atomicAdd(&a.stats[0], sw);
        atomicMax(&a.stats[1], sw);
      }
    }
  }
}

}  // namespace jglobal

// Column block width for m_len rows: two blocks of B columns in at most
// 200 KB of shared memory.
static int global_block_width(int m_len) {
  const size_t cap = 200 * 1024;
  for (int B : {16, 8, 4})
    if (size_t(2) * B * m_len * sizeof(float) <= cap) return B;
  return 0;
}

// Padded column count: a multiple of 32 (the load tiles), hence of 2B (an
// even number of blocks) for B <= 16.
static int global_npad(int n_vec) { return std::max(32, (n_vec + 31) / 32 * 32); }

static void global_layout(int m_len, int n_vec, int nslices, Sizer& s) {
  const int np = global_npad(n_vec);
  s.take<float>(size_t(nslices) * np * m_len);   // W
  s.take<float>(size_t(nslices) * np);           // norms
  s.take<int>(size_t(nslices) * 4);              // nmax, big, done (+ spare)
  s.take<int>(8);                                // left, barrier, abort
}

size_t jacobi_global_work_bytes(int n1, int n2, int nslices) {
  const int m_len = std::max(n1, n2), n_vec = std::min(n1, n2);
  const int B = global_block_width(m_len);
  if (B == 0 || nslices <= 0) return 0;
  Sizer s;
  global_layout(m_len, n_vec, nslices, s);
  return s.bytes();
}

bool jacobi_global_supported(int n1, int n2) { return global_block_width(std::max(n1, n2)) > 0; }

template <int B>
static int launch_global(jglobal::Args& g, cudaStream_t st) {
  auto kern = jglobal::jacobi_global_kernel<B>;
  const size_t smem = std::max<size_t>(size_t(2) * B * g.a.m_len * sizeof(float), 32 * 33 * sizeof(float));
  WP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  int per_sm = 0;
  WP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B * 32, smem));
  if (per_sm < 1) return WP_ERR_UNSUPPORTED;
  const int64_t items = int64_t(g.nslices) * (g.nb / 2);
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(per_sm) * sm_count(), items)));
  void* args[] = {&g};
  WP_PROFILE("jacobi_svd_global", st);
  WP_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), dim3(unsigned(grid)), dim3(B * 32), args,
                                          smem, st));
  return launch_status();
}

int jacobi_global_launch(const JacobiArgs& a, int nslices, void* work, size_t work_bytes, cudaStream_t st) {
  const int B = global_block_width(a.m_len);
  if (B == 0) return WP_ERR_UNSUPPORTED;
  Sizer need;
  const int n_pad = global_npad(a.n_vec);
  global_layout(a.m_len, a.n_vec, nslices, need);
  if (!work || work_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(work, work_bytes);
  jglobal::Args g{};
  g.a = a;
  g.nslices = nslices;
  g.n_pad = n_pad;
  g.nb = n_pad / B;
  g.W = cv.take<float>(size_t(nslices) * n_pad * a.m_len);
  g.norms = cv.take<float>(size_t(nslices) * n_pad);
  int* ctl = cv.take<int>(size_t(nslices) * 4);
  int* misc = cv.take<int>(8);
  if (!cv.ok) return WP_ERR_WORKSPACE;
  g.nmax = reinterpret_cast<unsigned*>(ctl);
  g.big = ctl + nslices;
  g.done = ctl + 2 * size_t(nslices);
  g.left = misc;
  g.bar = reinterpret_cast<unsigned*>(misc + 2);
  g.abort = misc + 4;
  WP_CUDA_TRY(cudaMemsetAsync(ctl, 0, size_t(nslices) * 4 * sizeof(int), st));
  WP_CUDA_TRY(cudaMemsetAsync(misc, 0, 8 * sizeof(int), st));
  switch (B) {
    case 16: return launch_global<16>(g, st);
    case 8: return launch_global<8>(g, st);
    default: return launch_global<4>(g, st);
  }
}

}  // namespace wp
