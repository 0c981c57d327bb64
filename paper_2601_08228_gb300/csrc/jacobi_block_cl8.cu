// Cluster size 8 instances of the block-cyclic Jacobi kernel.
#include "jacobi_block.cuh"

WP_JACOBI_BLOCK_INSTANTIATE(8)
