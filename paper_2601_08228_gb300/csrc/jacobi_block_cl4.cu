// Cluster size 4 instances of the block-cyclic Jacobi kernel.
#include "jacobi_block.cuh"

WP_JACOBI_BLOCK_INSTANTIATE(4)
