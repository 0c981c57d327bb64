// One-sided Jacobi SVD of one small slice (at most 64 x 64) on one CTA of
// NW warps with lane-group pairs: the same rotation, thresholds, stopping
// rule and outputs as the block-cyclic kernel (jacobi_block.cuh), for the
// batched launch (batched.cu).
//
// Layout.  Columns in blocks of 4, the block tournament of the block-cyclic
// kernel over n_pad / 4 positions (warp w holds a top and a bottom block).
// Inside a warp each 8-lane group owns one column pair of a round: group g
// holds the top block's column g and, in column round S, the bottom
// block's column (g + S) mod 4, rows sub + 8 q (q < 8) of both.  A pair's
// dot product is one 8-lane butterfly and each group applies its own
// rotation; between rounds the bottom columns move one group down (8
// register shuffles per lane: the columns are short).  The 6 pairs inside a
// block (a sweep's first rounds) are done by both groups of a pair with the
// partner's column read through shuffles.  Block moves go through shared
// memory between two CTA barriers, as in the block-cyclic kernel with one
// CTA.  Compared with that kernel on these slices (4 pairs per warp summed
// over all 32 lanes, 2 rows per lane, then a rotation broadcast), a round
// has a shorter dependency chain and fewer instructions.
#pragma once

#include "jacobi_block.cuh"

namespace wp {
namespace jgroup {

constexpr int PPW = 4;            // columns per block
constexpr int GL = 8;             // lanes per group
constexpr int QB = 8;             // rows per lane: rows sub + 8 q, 64 rows
constexpr int kRows = GL * QB;    // 64
constexpr int BLK = PPW * QB * GL;   // floats per block
constexpr int kPitch = kRows + 1;

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// Shared memory: norms[64] | order[64] | rank_of[64] | red[NW] |
// mnorm[2 NW][4] | mscale[2 NW][4] | (16-byte aligned) mailboxes
// [2 NW][BLK], which first stage the slice (64 columns of pitch 65).
template <int NW>
struct Lay {
  static constexpr size_t norms = 0, order = 64 * 4, rank_of = 128 * 4, red = 192 * 4;
  static constexpr size_t mnorm = red + NW * 4, mscale = mnorm + 2 * NW * PPW * 4;
  static constexpr size_t mail = al16(mscale + 2 * NW * PPW * 4);
  static constexpr size_t mail_floats = (2 * NW * BLK > 64 * kPitch) ? 2 * NW * BLK : 64 * kPitch;
  static constexpr size_t total = al16(mail + mail_floats * 4);
};

// a.m_len <= 64, a.n_pad = n_vec rounded up to 8 (<= 8 NW).  Writes the
// leading r unit vectors to vo (m_len x r, row-major, any memory space).
// Every thread of the CTA calls it; ends with a CTA barrier.
template <int NW>
__device__ __forceinline__ void group_jacobi_slice(const JacobiArgs& a, const float* A, float* vo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using L = Lay<NW>;
  float* norms = reinterpret_cast<float*>(smem_raw + L::norms);
  int* order = reinterpret_cast<int*>(smem_raw + L::order);
  int* rank_of = reinterpret_cast<int*>(smem_raw + L::rank_of);
  float* red = reinterpret_cast<float*>(smem_raw + L::red);
  float* mnorm = reinterpret_cast<float*>(smem_raw + L::mnorm);
  float* mscale = reinterpret_cast<float*>(smem_raw + L::mscale);
  float* mail = reinterpret_cast<float*>(smem_raw + L::mail);
  constexpr int NTH = NW * 32;
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  const int g = lane / GL, sub = lane % GL;
  const int n_pad = a.n_pad, nb = n_pad / PPW, nw = nb / 2;
  const bool active = warp < nw;
  const int topc = warp * PPW, botc = (nb - 1 - warp) * PPW;

  // stage the working matrix column-major (pitch 65), zero-padded
  for (int idx = threadIdx.x; idx < n_pad * kRows; idx += NTH) {
    int c, R;
    if (a.trans) {
      c = idx / kRows;
      R = idx % kRows;
    } else {
      R = idx / n_pad;
      c = idx % n_pad;
    }
    float v = 0.f;
    if (c < a.n_vec && R < a.m_len) v = a.trans ? A[int64_t(c) * a.n2 + R] : A[int64_t(R) * a.n2 + c];
    mail[c * kPitch + R] = v;
  }
  __syncthreads();
  float Tc[QB], Bc[QB];
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    Tc[q] = active ? mail[(topc + g) * kPitch + sub + GL * q] : 0.f;
    Bc[q] = active ? mail[(botc + g) * kPitch + sub + GL * q] : 0.f;
  }
  __syncthreads();   // staging reads done before the mailboxes are reused

  float nT = 0.f, nB = 0.f, dT = 1.f, dB = 1.f;
  auto gsum = [&](float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
  };
  auto fold = [&]() {
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      Tc[q] *= dT;
      Bc[q] *= dB;
    }
    dT = dB = 1.f;
  };
  auto exact_norms = [&]() {
    float st = 0.f, sb = 0.f;
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      st = fmaf(Tc[q], Tc[q], st);
      sb = fmaf(Bc[q], Bc[q], sb);
    }
    nT = gsum(st);
    nB = gsum(sb);
  };
  int big = 0;
  float tol2s = 0.f;
  auto angle = [&](float gam, float al, float be, float negl, float tol2, float& c, float& s, float& t) {
    const float ab = al * be;
    if (al > negl && be > negl && gam * gam > tol2s * ab) big = 1;
    if (al > negl && be > negl && gam * gam > tol2 * ab) {
      const float zeta = __fdividef(be - al, 2.f * gam);
      const float az = fminf(fabsf(zeta), 1e18f);
      const float h = fmaf(az, az, 1.f);
      t = copysignf(__fdividef(1.f, az + h * rsqrtf(h)), zeta);
      c = rsqrtf(fmaf(t, t, 1.f));
      s = c * t;
      return true;
    }
    c = 1.f;
    s = 0.f;
    t = 0.f;
    return false;
  };
  // a pair inside a block: the group's column X and group p's column of
  // the same block; both groups compute the same rotation (the lower group
  // index is the pair's first column), c = 1, s = 0 when not rotated
  auto rotate_within = [&](float (&X)[QB], float& nrm, int p, float negl, float tol2) {
    const int src = p * GL + sub;
    const bool first = g < p;
    float e = 0.f, xp[QB];
#pragma unroll
    for (int q = 0; q < QB; ++q) {
      xp[q] = __shfl_sync(0xffffffffu, X[q], src);
      e = fmaf(X[q], xp[q], e);
    }
    const float gam = gsum(e);
    const float np = __shfl_sync(0xffffffffu, nrm, src);
    float c, s, t;
    if (angle(gam, first ? nrm : np, first ? np : nrm, negl, tol2, c, s, t)) nrm = fmaf(first ? -t : t, gam, nrm);
    const float cs = first ? -s : s;
#pragma unroll
    for (int q = 0; q < QB; ++q) X[q] = fmaf(c, X[q], cs * xp[q]);
  };
  // block transfer: rows sub + 8 (4h .. 4h + 3) of group g's column at
  // float offset ((g QB/4 + h) 8 + sub) 4 of the block
  auto boff = [&](int h) { return ((g * (QB / 4) + h) * GL + sub) * 4; };
  auto post = [&](const float (&X)[QB], float nrm, float d, int slot) {
    float* dst = mail + size_t(slot) * BLK;
#pragma unroll
    for (int h = 0; h < QB / 4; ++h)
      *reinterpret_cast<float4*>(dst + boff(h)) = make_float4(X[4 * h], X[4 * h + 1], X[4 * h + 2], X[4 * h + 3]);
    if (sub == 0) {
      mnorm[slot * PPW + g] = nrm;
      mscale[slot * PPW + g] = d;
    }
  };
  auto fetch = [&](float (&X)[QB], float& nrm, float& d, int slot) {
    const float* src = mail + size_t(slot) * BLK;
#pragma unroll
    for (int h = 0; h < QB / 4; ++h) {
      const float4 v = *reinterpret_cast<const float4*>(src + boff(h));
      X[4 * h] = v.x;
      X[4 * h + 1] = v.y;
      X[4 * h + 2] = v.z;
      X[4 * h + 3] = v.w;
    }
    nrm = mnorm[slot * PPW + g];
    d = mscale[slot * PPW + g];
  };

  bool converged = false;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    sweeps_done = sweep + 1;
    const float tol_eff = sweep < kStrictSweeps ? a.tol : 8.f * a.tol;
    const float tol2 = tol_eff * tol_eff;
    if (active) {
      fold();
      exact_norms();
    }
    float mx = active ? fmaxf(nT, nB) : 0.f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    float nmax = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) nmax = fmaxf(nmax, red[w]);
    const float meps = float(a.m_len) * 1.1920929e-7f;
    const float negl = nmax * meps * meps;
    tol2s = tol_eff;
    big = 0;

    if (active) {
      jblock::static_for<PPW - 1>([&](auto K_) {
        constexpr int K = decltype(K_)::value;
        const int p = jblock::circ<PPW>(PPW - 1 - jblock::circ_pos<PPW>(g, K), K);
        rotate_within(Tc, nT, p, negl, tol2);
        rotate_within(Bc, nB, p, negl, tol2);
      });
    }

    for (int o = 0; o < nb - 1; ++o) {
      if (active) {
#pragma unroll
        for (int S = 0; S < PPW; ++S) {
          float e0 = 0.f, e1 = 0.f;
#pragma unroll
          for (int q = 0; q < QB; q += 2) {
            e0 = fmaf(Tc[q], Bc[q], e0);
            e1 = fmaf(Tc[q + 1], Bc[q + 1], e1);
          }
          const float gam = gsum(e0 + e1) * (dT * dB);
          const float rba = __fdividef(dB, dT), rab = __fdividef(dT, dB);
          float c, s, t, ta = 0.f, tb = 0.f;
          if (angle(gam, nT, nB, negl, tol2, c, s, t)) {
            nT = fmaf(-t, gam, nT);
            nB = fmaf(t, gam, nB);
            ta = t * rba;
            tb = t * rab;
            dT *= c;
            dB *= c;
          }
          if (__any_sync(0xffffffffu, ta != 0.f)) {
#pragma unroll
            for (int q = 0; q < QB; ++q) {
              const float u = Tc[q], v = Bc[q];
              Tc[q] = fmaf(-ta, v, u);
              Bc[q] = fmaf(tb, u, v);
            }
          }
          // the bottom column moves one group down
          const int from = (lane + GL) & 31;
#pragma unroll
          for (int q = 0; q < QB; ++q) Bc[q] = __shfl_sync(0xffffffffu, Bc[q], from);
          nB = __shfl_sync(0xffffffffu, nB, from);
          dB = __shfl_sync(0xffffffffu, dB, from);
        }
        if (__any_sync(0xffffffffu, dT < 1.f / 1024.f || dB < 1.f / 1024.f)) fold();
      }
      // block move: positions 1..nb-1 advance by one (position 0 stays)
      __syncthreads();
      if (active && nw > 1) {
        if (warp >= 1 && warp <= nw - 2) post(Tc, nT, dT, 2 * warp);
        post(Bc, nB, dB, 2 * warp + 1);
      }
      __syncthreads();
      if (active && nw > 1) {
        if (warp == nw - 1) {
#pragma unroll
          for (int q = 0; q < QB; ++q) Bc[q] = Tc[q];
          nB = nT;
          dB = dT;
        } else {
          fetch(Bc, nB, dB, 2 * (warp + 1) + 1);
        }
        if (warp >= 1) fetch(Tc, nT, dT, warp == 1 ? 1 : 2 * (warp - 1));
      }
    }
    if (!__syncthreads_or(big)) {
      converged = true;
      break;
    }
  }
  if (!converged && threadIdx.x == 0) report_device_error(a.status, WP_ERR_NOT_CONVERGED);
  if (threadIdx.x == 0 && a.stats) {
    atomicAdd(&a.stats[0], (unsigned long long)sweeps_done);
    atomicMax(&a.stats[1], (unsigned long long)sweeps_done);
  }

  if (active) {
    fold();
    exact_norms();
    if (sub == 0) {
      norms[topc + g] = nT;
      norms[botc + g] = nB;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n_pad; c += NTH) {
    int pos = a.r;
    if (c < a.n_vec) {
      const float sc = norms[c];
      pos = 0;
      for (int q = 0; q < a.n_vec; ++q) {
        const float sq = norms[q];
        pos += (sq > sc) || (sq == sc && q < c);
      }
      if (pos < a.r) order[pos] = c;
    }
    rank_of[c] = pos < a.r ? pos : -1;
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int c = (side ? botc : topc) + g;
      const int kq = rank_of[c];
      if (kq >= 0) {
        const float sg = sqrtf(norms[c]);
        const float inv = sg > 0.f ? 1.f / sg : 0.f;
#pragma unroll
        for (int q = 0; q < QB; ++q) {
          const int R = sub + GL * q;
          if (R < a.m_len) vo[R * a.r + kq] = (side ? Bc[q] : Tc[q]) * inv;
        }
      }
    }
  }
  __syncthreads();
}

}  // namespace jgroup
}  // namespace wp
