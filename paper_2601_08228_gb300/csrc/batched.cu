// Batched launch over many uneven tensors (placeholder until the persistent kernel lands).
#include "common.cuh"

extern "C" int wp_batched_workspace(const wp_batch_item*, int, size_t*) { return WP_ERR_UNSUPPORTED; }
extern "C" int wp_batched(const wp_batch_item*, int, void*, size_t, void*) { return WP_ERR_UNSUPPORTED; }
