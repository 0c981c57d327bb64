// Block-cyclic, register-resident one-sided Jacobi SVD of wavelet-domain
// frontal slices (Algorithm 2: the facewise "svd" of every A_{d_j}[:, :, k]
// and A_{s_L}[:, :, k]); same rotation, thresholds, outputs and error
// reporting as the kernels in jacobi.cu.
//
// Ordering.  The n_pad working columns form nb = n_pad / PPW blocks of PPW
// columns.  A sweep is one round-robin tournament over the blocks (circle
// method, block position 0 fixed): in each of its nb - 1 block rounds warp w
// holds the blocks at positions w ("top") and nb - 1 - w ("bottom") and meets
// every top column with every bottom column in PPW column rounds (round s
// pairs top column j with bottom column (j + s) mod PPW).  Before the first
// block round every block meets itself (PPW - 1 rounds of the circle method
// inside the block).  Every column pair therefore meets exactly once per
// sweep, in n_pad - 1 rounds of n_pad / 2 disjoint rotations.  After loop
// unrolling every register index is a compile-time constant, so no column
// moves between registers; whole blocks move between warps through shared
// memory once every PPW rounds, and after nb - 1 block rounds every block is
// back where the sweep started.
//
// Cluster reduction.  The rows of a slice are split over a cluster of CL
// CTAs (rows of the working matrix in registers: RPL per lane).  Warp w of
// every CTA owns the same pairs; each round it sends its PPW partial dot
// products to warp w of every peer CTA with st.async, which completes
// transaction bytes on that warp's mbarrier (two buffers, alternating by
// round), and adds the CL partials in rank order -- bit-identical totals,
// hence identical rotation decisions, on every CTA.  Within a block round no
// CTA-wide barrier is taken: warps advance independently.

#include "jacobi_block.cuh"

namespace wp {

namespace jblock {
extern template int launch_block_ppw<1>(const JacobiArgs&, int, int, int, cudaStream_t);
extern template int launch_block_ppw<2>(const JacobiArgs&, int, int, int, cudaStream_t);
extern template int launch_block_ppw<4>(const JacobiArgs&, int, int, int, cudaStream_t);
extern template int launch_block_ppw<8>(const JacobiArgs&, int, int, int, cudaStream_t);
}  // namespace jblock

// Shape selection: PPW (columns per block) the smallest power of two with
// at most 16 warps of two blocks; the smallest cluster whose per-CTA rows
// fit in 32 RPL register rows (2 PPW RPL <= 64), doubled while the grid
// still fits in one wave (few slices: spread their rows over more SMs).
int jacobi_block_launch(const JacobiArgs& a0, int nslices, cudaStream_t st) {
  if (a0.n_pad <= 32) return WP_ERR_UNSUPPORTED;
  int ppw = 2;
  while (ppw < 16 && 2 * ppw * jblock::kBlockWarps < a0.n_pad) ppw *= 2;
  if (2 * ppw * jblock::kBlockWarps < a0.n_pad) return WP_ERR_UNSUPPORTED;
  const int rpl_max = std::min(4, 32 / ppw);
  int CL = 1;
  while (CL <= 8 && (a0.m_len + CL - 1) / CL > 32 * rpl_max) CL *= 2;
  if (CL > 8) return WP_ERR_UNSUPPORTED;
  // shapes the column-split kernel takes (no per-round cluster exchange):
  // it picks its own cluster sizes
  if (CL == 2 && jacobi_cols_enabled() && jacobi_cols_fits(a0.m_len, a0.n_vec))
    return jacobi_cols_launch(a0, nslices, st);
  while (CL < 8 && 2 * CL * nslices <= sm_count()) CL *= 2;
  JacobiArgs a = a0;
  a.n_pad = (a0.n_pad + 2 * ppw - 1) / (2 * ppw) * (2 * ppw);
  a.rpc = (a.m_len + CL - 1) / CL;
  int rpl = 1;
  while (32 * rpl < a.rpc) rpl *= 2;
  switch (CL) {
    case 1: return jblock::launch_block_ppw<1>(a, nslices, ppw, rpl, st);
    case 2: return jblock::launch_block_ppw<2>(a, nslices, ppw, rpl, st);
    case 4: return jblock::launch_block_ppw<4>(a, nslices, ppw, rpl, st);
    default: return jblock::launch_block_ppw<8>(a, nslices, ppw, rpl, st);
  }
}

}  // namespace wp
