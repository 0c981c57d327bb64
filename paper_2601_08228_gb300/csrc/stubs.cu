// Entry points not implemented yet.
#include "common.cuh"

extern "C" int wp_wsvd_workspace(int64_t, int64_t, int64_t, int, int, size_t*) { return WP_ERR_UNSUPPORTED; }
extern "C" int wp_wsvd(const float*, float*, float*, float*, float*, int64_t, int64_t, int64_t, int, int, int, int, void*, size_t, void*) { return WP_ERR_UNSUPPORTED; }
extern "C" int wp_wpinv_workspace(int64_t, int64_t, int64_t, int, size_t*) { return WP_ERR_UNSUPPORTED; }
extern "C" int wp_wpinv(const float*, float*, int64_t, int64_t, int64_t, int, double, int, void*, size_t, void*) { return WP_ERR_UNSUPPORTED; }
extern "C" int wp_batched_workspace(const wp_batch_item*, int, size_t*) { return WP_ERR_UNSUPPORTED; }
extern "C" int wp_batched(const wp_batch_item*, int, void*, size_t, void*) { return WP_ERR_UNSUPPORTED; }
