/*
 * wprod.h -- C ABI of libwprod.so, the GB300 (sm_103a) w-product library.
 *
 * Implements the hot path of "Second-Generation Wavelet-inspired Tensor
 * Product with Applications in Hyperspectral Imaging" (arXiv 2601.08228):
 * the L-level lazy-Haar lifting transform along mode 3 (Sec. II-A, Eq. 1-3),
 * the facewise products of the wavelet-domain frontal slices (Def. 2.1,
 * Algorithm 1), facewise truncated SVDs (Algorithm 2, Thm 2.5, sp-w-svd of
 * Sec. IV-B), the Moore-Penrose inverse (Def. 2.6, Thm 2.6), the backward
 * pass of the w-product and a batched launch over many uneven tensors.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Tensors.  A third-order tensor A in R^{n1 x n2 x p} is a contiguous float32
 *   array in DEVICE memory, slice-major: shape (p, n1, n2), row-major, so the
 *   frontal slice A(:, :, k) is the dense n1 x n2 row-major matrix at offset
 *   (k-1) * n1 * n2.  Tube length p must be a multiple of 2^L (p = 2^L m,
 *   Sec. II-A); L = 0 is accepted and makes the w-product a plain batched
 *   matrix product.
 * Wavelet domain.  Transformed tensors use the Mallat coefficient order of
 *   Eq. (1) along mode 3: slices [0, m) hold s_L, [m, 2m) hold d_L, and
 *   [p / 2^j, p / 2^(j-1)) hold d_j.
 * Lifting convention.  Algorithm 1 with 1-based tube positions:
 *   d_j[k] = s_{j-1}[2k-1] - s_{j-1}[2k],  s_j[k] = s_{j-1}[2k] + d_j[k] / 2.
 * Ownership.  The caller owns every buffer.  Work buffers are passed in as
 *   `ws` / `ws_bytes` (device memory, 256-byte aligned); query the size with
 *   the matching *_workspace() call.  The library never allocates device
 *   memory on these paths.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Every call only enqueues work on it and returns; no call
 *   synchronises unless stated.
 * Aliasing.  Outputs must not overlap inputs (WP_ERR_ALIAS).
 * Alignment.  Every tensor pointer must be 16-byte aligned (WP_ERR_ALIGN).
 * Errors.  Arguments are validated on the host before anything is launched;
 *   a failing call launches nothing and returns a wp_status code.  Faults
 *   detected inside kernels (an expired bounded wait, a Jacobi sweep limit)
 *   are recorded in a per-device status word that wp_get_device_error()
 *   returns and clears.  Nothing calls abort() and no kernel traps.
 * Device reset.  The library keeps per-device addresses of its own device
 *   variables (status word, counters, scratch array) from the first call on
 *   each device.  cudaDeviceReset() destroys them: calls after a reset in the
 *   same process are not supported.
 */
#ifndef WPROD_H
#define WPROD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define WP_API __attribute__((visibility("default")))
#else
#define WP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WP_OK = 0,
  WP_ERR_NULL = 1,          /* a required pointer is NULL                      */
  WP_ERR_SHAPE = 2,         /* a dimension is < 1 or too large                 */
  WP_ERR_LEVELS = 3,        /* L < 0, L > WP_MAX_LEVELS or p % 2^L != 0        */
  WP_ERR_RANK = 4,          /* r < 1 or r > min(rows, cols)                    */
  WP_ERR_PREC = 5,          /* unknown precision mode                          */
  WP_ERR_ALIGN = 6,         /* a pointer is not 16-byte aligned                */
  WP_ERR_WORKSPACE = 7,     /* ws is NULL or ws_bytes too small                */
  WP_ERR_NOT_CONVERGED = 8, /* Jacobi SVD hit its sweep limit (device word)    */
  WP_ERR_TIMEOUT = 9,       /* a bounded device-side wait expired (device word)*/
  WP_ERR_CUDA = 10,         /* a CUDA runtime call failed                      */
  WP_ERR_ALIAS = 11,        /* an output overlaps an input                     */
  WP_ERR_UNSUPPORTED = 12   /* valid request this build does not implement     */
} wp_status;

/* Facewise-product arithmetic (Sec. "precision" of the library):
 *  FP32      plain FP32 SIMT products (the reference path of the library)
 *  BF16      one BF16 x BF16 tcgen05 product per slice, FP32 accumulation
 *  BF16X3    split precision: x = hi + lo with hi, lo BF16; computes
 *            hi*hi + hi*lo + lo*hi on tcgen05 tensor cores, FP32 accumulation
 *  FP8       E4M3 operands scaled per wavelet-domain slice, tcgen05, FP32
 *            accumulation, scales folded into the epilogue                  */
typedef enum { WP_PREC_FP32 = 0, WP_PREC_BF16 = 1, WP_PREC_BF16X3 = 2, WP_PREC_FP8 = 3 } wp_prec;

#define WP_MAX_LEVELS 10

/* Human-readable name of a wp_status value (static string, never NULL). */
WP_API const char* wp_status_string(int status);

/* Library version: major * 10000 + minor * 100 + patch. */
WP_API int wp_version(void);

/* Number of kernels this library has launched in the calling process so far
 * (a host-side counter incremented at every launch site). */
WP_API uint64_t wp_launch_count(void);

/* Per-kernel timing.  wp_profile_begin() clears the table and enables it:
 * from then on every kernel launch is bracketed by two CUDA events recorded
 * on the stream it is launched on.  wp_profile_end() disables recording,
 * synchronises the device and totals the elapsed times per kernel name;
 * wp_profile_count() / wp_profile_get() read the totals (name copied into
 * `name`, NUL-terminated, at most name_len bytes).  Do not enable it while a
 * stream is being captured into a CUDA graph.  wp_profile_only(name) limits
 * the recording to launches of that kernel name (NULL or "": every launch),
 * so that the events do not separate the other launches of a timed region
 * (a recorded event between two kernels ends the overlap that programmatic
 * stream serialisation gives them). */
WP_API int wp_profile_begin(void);
WP_API int wp_profile_only(const char* name);
WP_API int wp_profile_end(void);
WP_API int wp_profile_count(void);
WP_API int wp_profile_get(int index, char* name, int name_len, int64_t* launches,
                          double* total_ms);

/* Jacobi SVD counters since the last call (synchronises the device, then
 * clears them): the sum over slices of the sweeps each needed, and the
 * largest sweep count of any slice. */
WP_API int wp_jacobi_stats(int64_t* total_sweeps, int* max_sweeps);

/* Sweep limit of the one-sided Jacobi SVD used by wp_wsvd, wp_wpinv,
 * wp_deblur_pinv and wp_batched_run (Algorithm 2 takes its facewise SVDs
 * from a library routine; the iteration limit is this library's own).
 * Default 40; 1 <= max_sweeps <= 1000, else WP_ERR_SHAPE and no change.
 * Applies to launches enqueued after the call (a CUDA graph keeps the limit
 * it was captured with).  A slice still rotating after the last allowed
 * sweep keeps its partial result and sets WP_ERR_NOT_CONVERGED in the device
 * status word (wp_get_device_error).  Process-wide; not synchronised with
 * calls in flight on other host threads. */
WP_API int wp_set_jacobi_max_sweeps(int max_sweeps);

/* QR preconditioning of the facewise Jacobi SVD of wp_wsvd (on = 1, the
 * default; 0 = off; else WP_ERR_SHAPE).  wp_wpinv and wp_deblur_pinv always
 * use the plain Jacobi: a pseudo-inverse needs every singular value down to
 * its cut-off (max(m, n) eps sigma_max), and at that level the columns of
 * R^T fall below the Jacobi's numerically-zero threshold.  For
 * slices with 32 <= min(n1, n2) and max(n1, n2) <= 1024 the working matrix X
 * (the slice, or its transpose when it is wide) is first factored X = Q R by
 * Householder reflections, and the one-sided Jacobi method runs on the
 * columns of R^T, which converges in fewer sweeps; its converged columns
 * give the singular values and the singular vectors of X's short side,
 * from which the rank-r reconstruction, the factors and the pseudo-inverse
 * follow as before (Q is never formed).  Same results within the stated
 * tolerances; the workspace queries include the QR's work buffer.
 * Process-wide; applies to calls made after it (query workspaces after it). */
WP_API int wp_set_jacobi_precondition(int on);

/* Kernel choice for facewise Jacobi SVDs whose working matrix (the longer
 * side as rows) has at most 256 rows and 192..256 columns and that would run
 * on 2-CTA clusters: on = 1 (the default) takes the column-split kernel
 * (each CTA holds whole columns), 0 the row-split block kernel (each CTA
 * holds half of every column).  Both compute the same one-sided Jacobi SVD
 * (same rotation, thresholds and stopping rule; a different pair order, so
 * results agree to rounding).  0 or 1, else WP_ERR_SHAPE.  Process-wide. */
WP_API int wp_set_jacobi_column_split(int on);

/* Cluster size of the column-split Jacobi kernel: 0 (the default) picks it
 * per call -- one wave of 4- or 3-CTA clusters when every slice fits in it;
 * else a wave of 3-CTA clusters with the few slices beyond it on 2-CTA
 * clusters in the SMs it leaves; else full waves of 2-CTA clusters with the
 * remaining slices beside them on 3-CTA clusters when they fit one wave of
 * those.  Two such parts run side by side: the second on a library-owned
 * stream of the device, forked from and joined back to the call's stream
 * with events (both are captured when the call's stream is); calls from
 * several host threads on one device share that stream, so their second
 * parts run one after another (the enqueueing is serialised by a lock).
 * 2, 3 or 4 puts every launch on clusters of that size, on the call's
 * stream.  Else WP_ERR_SHAPE.  Process-wide. */
WP_API int wp_set_jacobi_cluster_size(int cl);

/* Number of clusters of `cl` CTAs (2, 3 or 4, else WP_ERR_SHAPE) of the
 * column-split Jacobi kernel that can be resident at once on the current
 * device, into *clusters (0 if the occupancy query fails); WP_ERR_NULL if
 * clusters is null. */
WP_API int wp_jacobi_cluster_capacity(int cl, int* clusters);

/* Synchronise `stream`, then return and clear the device status word of the
 * current device (WP_OK if no kernel reported a fault since the last call).
 * Returns WP_ERR_CUDA if the synchronisation itself fails. */
WP_API int wp_get_device_error(void* stream);

/* Test of the failure-detection path of the bounded device-side waits (the
 * paper has no counterpart).  Launches one kernel that waits, with the given
 * limit, on a barrier that nothing ever completes: which = 0 uses the
 * CTA-scope wait of the tensor-core kernels, which = 1 the cluster-scope wait
 * of the Jacobi kernels.  The wait expires after limit_ns nanoseconds
 * (1e3 <= limit_ns <= 1e8, else WP_ERR_SHAPE and nothing is launched), sets
 * WP_ERR_TIMEOUT in the device status word and the kernel returns normally:
 * nothing is in flight on the barrier, so the context stays usable.  Read
 * the result with wp_get_device_error(). */
WP_API int wp_selftest_bounded_wait(int which, int64_t limit_ns, void* stream);

/* ---- a1 / a4: lifting along mode 3 (Sec. II-A, Eq. 1-3, Algorithm 1) ---- */

/* y = W_[L](x): forward lazy-Haar lifting of every mode-3 tube, all L levels
 * in one pass (Eq. 1, Algorithm 1 forward loop).  x, y: (p, n1, n2) device
 * float32; y is written in Mallat order.  0 <= L <= WP_MAX_LEVELS. */
WP_API int wp_lift_forward(const float* x, float* y, int64_t n1, int64_t n2, int64_t p, int L,
                    void* stream);

/* x = W_[L]^{-1}(y): inverse lifting (Eq. 3, Algorithm 1 inverse loop).
 * y in Mallat order, x spatial; both (p, n1, n2). */
WP_API int wp_lift_inverse(const float* y, float* x, int64_t n1, int64_t n2, int64_t p, int L,
                    void* stream);

/* Adjoint transforms (the transform is not orthogonal, Remark 2.1).
 * of_inverse = 0: h = W^T g     (g Mallat order -> h spatial)
 * of_inverse = 1: h = W^{-T} g  (g spatial -> h Mallat order)              */
WP_API int wp_lift_adjoint(const float* g, float* h, int64_t n1, int64_t n2, int64_t p, int L,
                    int of_inverse, void* stream);

/* ---- a2: face-product Delta of wavelet-domain slices (Def. 2.1) ---------- */

/* Ch[k] = op(Ah[k]) op(Bh[k]) for k = 0..p-1.  op(Ah[k]) is n1 x n2: Ah is
 * (p, n1, n2), or (p, n2, n1) when transA.  op(Bh[k]) is n2 x n4: Bh is
 * (p, n2, n4), or (p, n4, n2) when transB.  Ch is (p, n1, n4). */
WP_API int wp_facewise_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int prec,
                          size_t* bytes);
WP_API int wp_facewise(const float* Ah, const float* Bh, float* Ch, int64_t n1, int64_t n2,
                int64_t n4, int64_t p, int transA, int transB, int prec, void* ws,
                size_t ws_bytes, void* stream);

/* ---- a1 + a2 + a4: the w-product (Def. 2.1, Algorithm 1) ---------------- */

/* C = op(A) *w op(B) = W^{-1}( W(op A) Delta W(op B) ), op as in
 * wp_facewise; C is (p, n1, n4) spatial.  BF16 / BF16X3 without transposes
 * run one of the three tensor-core w-product kernels described with the
 * plan cache below (the stored variant, else a rule of thumb); the size
 * wp_wprod_workspace returns covers all of them (the kernel that lifts the
 * operands in its producer warps uses none). */
WP_API int wp_wprod_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                       size_t* bytes);
WP_API int wp_wprod(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
             int64_t p, int L, int transA, int transB, int prec, void* ws, size_t ws_bytes,
             void* stream);

/* ---- general predict / update operators (Eq. 2-3, Example 2.1, Remark 3.1) */

/* One level's lifting operators.  Level j splits its input f (length n) into
 * odd[k] = f[2k] and even[k] = f[2k+1] (0-based storage of Algorithm 1's
 * 1-based odd / even positions) and computes (Eq. 2)
 *     d_j = odd - P_j(even),    s_j = even + U_j(d_j)
 * with stencil operators (Op y)[k] = sum_{t < taps} c_t y[k + offset + t],
 * 0 <= taps <= 4 (taps = 0: the zero operator), under half-sample symmetric
 * extension at both ends of the length-n/2 sequence: y[-1-i] = y[i],
 * y[n/2 + i] = y[n/2 - 1 - i]; every tap must reach less than n/2 positions
 * from k (else WP_ERR_SHAPE).  P = {0, 1, {1}}, U = {0, 1, {0.5}} is the
 * lazy-Haar transform of wp_lift_forward; Example 2.1's interpolating
 * predict is P = {-1, 2, {0.5, 0.5}} with U = 0. */
typedef struct {
  int32_t predict_offset;
  int32_t predict_taps;
  float predict[4];
  int32_t update_offset;
  int32_t update_taps;
  float update[4];
} wp_lift_ops;

/* Transform every mode-3 tube of x (p, n1, n2) with the L levels' operators
 * ops[0..L) (host array): op = 0 forward W (Mallat order out, Eq. 1),
 * 1 inverse W^{-1} (Eq. 3; Mallat order in), 2 the adjoint W^T (Mallat order
 * in), 3 W^{-T} (Mallat order out).  All levels in one pass over HBM; one
 * thread per tube holds the whole tube in shared memory, so p <= 800
 * (WP_ERR_UNSUPPORTED beyond).  x and y must not overlap. */
WP_API int wp_glift(const float* x, float* y, int64_t n1, int64_t n2, int64_t p, int L,
                    const wp_lift_ops* ops, int op, void* stream);

/* C = W^{-1}( W(A) Delta W(B) ) (Def. 2.1) with the general operators:
 * A (p, n1, n2), B (p, n2, n4), C (p, n1, n4); face-products in `prec`. */
WP_API int wp_gwprod_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                               size_t* bytes);
WP_API int wp_gwprod(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
                     int64_t p, int L, const wp_lift_ops* ops, int prec, void* ws, size_t ws_bytes,
                     void* stream);

/* Backward of wp_gwprod by the adjoint route (the transform is not
 * orthogonal): G_hat = W^{-T} G, dA = W^T (G_hat Delta B_hat^T),
 * dB = W^T (A_hat^T Delta G_hat); dA or dB may be NULL. */
WP_API int wp_gwprod_backward_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                                        size_t* bytes);
WP_API int wp_gwprod_backward(const float* A, const float* B, const float* G, float* dA, float* dB,
                              int64_t n1, int64_t n2, int64_t n4, int64_t p, int L,
                              const wp_lift_ops* ops, int prec, void* ws, size_t ws_bytes,
                              void* stream);

/* ---- autotuner and plan cache of the tensor-core w-product -------------- */

/* The BF16 / BF16X3 w-product without transposes (1 <= L <= 5) has three
 * kernels: (1) one CTA per 128 x (512 / 2^L) tile of all 2^L slices of a
 * tube group, whose epilogue applies the inverse lift (Eq. 3) across the 2^L
 * tensor-memory accumulators, so the wavelet-domain product never reaches
 * HBM; (2) a persistent wide-tile GEMM into the wavelet-domain product, then
 * a separate inverse lift; (3) the tile of (1) whose own producer warps
 * apply the forward lift (Eq. 2) and the BF16 split to the spatial operands,
 * so that W(A) and W(B) do not reach HBM either (L <= 3, n2 and n4 multiples
 * of 4, A, B and C 16-byte aligned; elsewhere a stored variant 3 falls back
 * to the rule for (1) and (2)).  All compute the same product (Algorithm 1);
 * the fastest depends on the shape.  wp_wprod takes the variant stored for
 * the shape in a process-wide plan cache keyed by (n1, n2, n4, p, L, prec),
 * else a rule of thumb measured on GB300.
 *
 * wp_wprod_tune: times the variants on the caller's tensors (one warm-up
 * call, then the mean of three back-to-back calls each, CUDA events on
 * `stream`), stores the fastest in the cache and returns it in *variant
 * (1 fused epilogue, 2 persistent GEMM + inverse lift, 3 lifted operands +
 * fused epilogue) and its time in *best_ms (if not NULL).  C holds the product on return.  Synchronises
 * `stream`; do not call it while the stream is being captured.  For
 * arguments with a single kernel (FP32, FP8, transposes, L = 0 or L > 5) it
 * runs wp_wprod once and returns WP_OK with *variant = 0.
 * wp_plan_set: stores variant 1, 2 or 3 for the key; <= 0 removes the entry.
 * wp_plan_get: *variant = the cached value, 0 if none.
 * wp_plan_clear: empties the cache.
 * wp_plan_save / wp_plan_load: write / read the cache as a text file of one
 *   JSON object per line ({"op": "wprod", "n1": .., "n2": .., "n4": .., "p":
 *   .., "L": .., "prec": .., "variant": .., "ms": ..}); load adds the file's
 *   entries to the cache (*entries = how many, if not NULL) and returns
 *   WP_ERR_SHAPE for an unreadable file or a malformed line (the entries
 *   before it are kept). */
WP_API int wp_wprod_tune(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
                         int64_t p, int L, int prec, void* ws, size_t ws_bytes, void* stream,
                         int* variant, double* best_ms);
WP_API int wp_plan_set(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec, int variant);
WP_API int wp_plan_get(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec, int* variant);
WP_API int wp_plan_clear(void);
WP_API int wp_plan_save(const char* path);
WP_API int wp_plan_load(const char* path, int* entries);

/* ---- w-product of host-resident tensors ---------------------------------- */

/* C = A *w B (Def. 2.1, Algorithm 1; no transposes) for A (p, n1, n2),
 * B (p, n2, n4) and C (p, n1, n4) in HOST memory.  The slices are taken in
 * chunks of `chunk_slices` consecutive slices, a multiple of 2^L so that every
 * chunk holds whole tube groups (the transform never mixes two groups, so
 * each chunk's product is the product of its slices): chunk k + 1 is copied
 * to the device while chunk k is multiplied (wp_wprod) and chunk k - 1 is
 * copied back, on three library-owned streams that start after the work
 * already queued on `stream`; `stream` then waits for the last copy back.
 * The result equals wp_wprod's on the same slices.  chunk_slices = 0 picks
 * one tube group for the first and the last chunk (a short copy before the
 * first product and after the last) and about p / 4 slices for the others.
 *   - Page-locked host buffers let the copies overlap; pageable ones work
 *     but each copy then blocks the host.
 *   - ws: device memory of wp_wprod_host_workspace() bytes (three chunks of
 *     A, B and C, and one chunk's wp_wprod workspace), 256-byte aligned.
 *   - All calls on one device share the three streams and their events:
 *     calls from several host threads on one device must be serialised.
 * Errors: as wp_wprod (shapes, levels, precision, workspace), WP_ERR_NULL
 * for a null buffer, WP_ERR_SHAPE for a chunk that is not a multiple of 2^L,
 * WP_ERR_CUDA when a copy or stream operation fails. */
WP_API int wp_wprod_host_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                                   int64_t chunk_slices, size_t* bytes);
WP_API int wp_wprod_host(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
                         int64_t p, int L, int prec, int64_t chunk_slices, void* ws, size_t ws_bytes,
                         void* stream);

/* ---- w-product without a caller-supplied workspace ---------------------- */

/* Size in bytes of the library-owned scratch array used by wp_wprod_noalloc. */
#define WP_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Same result as wp_wprod, for callers that cannot allocate device memory
 * for a workspace: plain C hosts without a device allocator, or plug-ins
 * whose host application owns every device allocation.  The paper has no
 * counterpart to this call; it only changes where the scratch space lives.
 *
 * The scratch space is one fixed array of WP_NOALLOC_SCRATCH_BYTES bytes in
 * device global memory, created when the library is loaded and held by every
 * GPU that loads it until the process exits.  The call allocates nothing;
 * the caller still owns and passes A, B and C.
 *   - Requests whose wp_wprod_workspace() size exceeds the array return
 *     WP_ERR_WORKSPACE and launch nothing.
 *   - The first call on each device looks up the array's device address on
 *     that device (the device current at the time of the call) and keeps it
 *     for the rest of the process.  Make that first call before any stream
 *     capture.  cudaDeviceReset() invalidates the kept address (as it does
 *     every device address the library keeps, see "Device reset" above):
 *     do not call this entry point after a device reset.
 *   - All calls share the one array.  Calls whose kernels overlap on the GPU
 *     (different streams, or different host threads on one device) race on
 *     it and give wrong results: serialise them, e.g. on one stream.
 *   - The array keeps whatever the last call left in it; every byte a call
 *     reads is written earlier in that same call, so no clearing is needed. */
WP_API int wp_wprod_noalloc(const float* A, const float* B, float* C, int64_t n1, int64_t n2,
                            int64_t n4, int64_t p, int L, int transA, int transB, int prec,
                            void* stream);

/* ---- a6: backward of C = A *w B (adjoint route) ------------------------- */

/* Given G = dLoss/dC (p, n1, n4), computes
 *   G_hat = W^{-T} G,  dA = W^T (G_hat Delta B_hat^T),  dB = W^T (A_hat^T Delta G_hat)
 * with A_hat = W(A), B_hat = W(B) recomputed (not stored by the forward).
 * A (p, n1, n2), B (p, n2, n4); dA (p, n1, n2) and dB (p, n2, n4) may each
 * be NULL to skip that gradient. */
WP_API int wp_wprod_backward_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L,
                                int prec, size_t* bytes);
WP_API int wp_wprod_backward(const float* A, const float* B, const float* G, float* dA, float* dB,
                      int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                      void* ws, size_t ws_bytes, void* stream);

/* ---- deblurring step driven by the backward (Sec. IV-C) ----------------- */

/* One gradient step on f(X) = ||K *w X - Y||_F^2 + lam ||X||_F^2, the
 * least-squares form of the deblurring model of Sec. IV-C with one blur
 * operator:  X <- X - eta (2 K^T *w (K *w X - Y) + 2 lam X).  K^T *w R is
 * evaluated by the w-product backward (adjoint route).  K (p, n1, n1),
 * Y and X (p, n1, n2); X is updated in place.  If `loss` is not NULL (device
 * pointer to one double), f(X) at the start of the step is ADDED to *loss.
 * No host synchronisation and no allocation: a loop of steps can be
 * captured in a CUDA graph. */
WP_API int wp_deblur_workspace(int64_t n1, int64_t n2, int64_t p, int L, int prec, size_t* bytes);
WP_API int wp_deblur_step(const float* K, const float* Y, float* X, int64_t n1, int64_t n2, int64_t p,
                          int L, float lam, float eta, int prec, double* loss, void* ws, size_t ws_bytes,
                          void* stream);

/* ---- two-sided pseudo-inverse deblurring (Sec. IV-C) -------------------- */

/* X = A_V^dagger *w B *w (A_H^T)^dagger, the least-squares reconstruction of
 * a cube blurred as B = A_V *w X *w A_H^T.  A_V (p, n1, n1), A_H (p, n2, n2),
 * B and X (p, n1, n2), all device float32, slice-major.  The two
 * pseudo-inverses are wp_wpinv (cut-off `rtol`, `refine_iters` refinement
 * steps); (A_H^T)^dagger is applied as (A_H^dagger)^T, and the two
 * w-products run in precision `prec`.  X must not overlap the inputs.
 * Limits are those of wp_wpinv for n1 x n1 and n2 x n2 slices (the Jacobi
 * kernels hold a slice on one CTA cluster: up to about 568 x 568;
 * WP_ERR_UNSUPPORTED beyond). */
WP_API int wp_deblur_pinv_workspace(int64_t n1, int64_t n2, int64_t p, int L, int prec, size_t* bytes);
WP_API int wp_deblur_pinv(const float* AV, const float* AH, const float* B, float* X, int64_t n1, int64_t n2,
                          int64_t p, int L, double rtol, int refine_iters, int prec, void* ws, size_t ws_bytes,
                          void* stream);

/* ---- a3: truncated w-svd and sp-w-svd (Algorithm 2, Thm 2.5, Sec. IV-B) -- */

/* C_r = rank-r w-svd of A (p, n1, n2): per wavelet-domain slice a one-sided
 * Jacobi SVD, keep the r leading triplets, inverse-transform.  sparse = 1
 * gives sp-w-svd: only the s_L and d_L slices (Mallat rows [0, 2m)) are
 * truncated, the finer details d_1..d_{L-1} are set to zero.
 * Optional factor outputs (NULL to skip): U (p, n1, r), S (p, r), V (p, n2, r)
 * -- singular vectors as columns, singular values in descending order.  With
 * factors_in_wavelet_domain = 1 they are the per-slice factors in Mallat
 * order; with 0 they are mapped to the spatial domain with W^{-1} (Thm 2.5).
 * Singular vectors are determined up to sign.
 * Size limit: a slice's working matrix (max(n1, n2) rows, min(n1, n2)
 * columns) is held on one thread-block cluster (in registers or shared
 * memory) when it fits one, and otherwise in a global-memory work buffer
 * (part of the workspace) with two column blocks of the long side staged
 * in shared memory: up to 6400 rows; longer ones return WP_ERR_UNSUPPORTED
 * (the same limits hold for wp_wpinv).
 * Range: column norms and dot products are FP32 sums of products, so
 * slices whose entries all lie below about 1e-19 or above about 1e19 in
 * magnitude (squares under- or overflowing FP32) lose their small or large
 * columns; scale such tensors first (the SVD of cA is c times that of A). */
WP_API int wp_wsvd_workspace(int64_t n1, int64_t n2, int64_t p, int L, int r, size_t* bytes);
WP_API int wp_wsvd(const float* A, float* C_r, float* U, float* S, float* V, int64_t n1, int64_t n2,
            int64_t p, int L, int r, int sparse, int factors_in_wavelet_domain, void* ws,
            size_t ws_bytes, void* stream);

/* ---- a5: Moore-Penrose inverse (Def. 2.6, Thm 2.6) --------------------- */

/* X = A^dagger for A (p, m, n); X is (p, n, m).  Per wavelet slice
 * pinv = V Sigma^+ U^T from the Jacobi SVD, keeping sigma_i > rtol sigma_max
 * (rtol < 0 selects max(m, n) * FLT_EPSILON), then `refine_iters` steps of
 * X <- X + X (I - A X) with the residual I - A X evaluated as compensated
 * dot products (twice working precision, Dot2 of Ogita, Rump and Oishi), then
 * W^{-1}. */
WP_API int wp_wpinv_workspace(int64_t m, int64_t n, int64_t p, int L, size_t* bytes);
WP_API int wp_wpinv(const float* A, float* X, int64_t m, int64_t n, int64_t p, int L, double rtol,
             int refine_iters, void* ws, size_t ws_bytes, void* stream);

/* ---- a7: batched launch over many uneven tensors ------------------------ */

/* One item: C = A *w B (Def. 2.1) and C_r = rank-r w-svd of A
 * (Algorithm 2), for A (p, n1, n2), B (p, n2, n4), C (p, n1, n4),
 * C_r (p, n1, n2); all device pointers, slice-major as everywhere. */
typedef struct {
  const float* A;
  const float* B;
  float* C;
  float* C_r;
  int32_t n1, n2, n4, p, L, r;
} wp_batch_item;

/* Plan of a batched launch, filled by wp_batched_plan and passed unchanged
 * to wp_batched_run.  Offsets are bytes into the workspace. */
typedef struct {
  int32_t count;
  int32_t n_lift_fwd, n_lift_inv;
  int32_t gemm_threads, svd_threads;   /* CTA sizes (autotuned when tune = 1) */
  int32_t svd_vec_floats;              /* max over items of max(n1, n2) * r */
  int64_t n_units;                     /* wavelet-domain slices over all items */
  int64_t n_units_narrow;              /* the first n_units_narrow of them have min(n1, n2) <= 32, */
  int64_t n_units_mid;                 /* the next n_units_mid 32 < min(n1, n2) <= 48 */
  int64_t lift_fwd_blocks, lift_inv_blocks;
  uint64_t items_off, lift_fwd_off, lift_inv_off, units_off;
  int32_t svd_group;                   /* 1: lane-group Jacobi kernel for every slice class, 0: block-cyclic
                                          (autotuned when tune = 1; 1 otherwise) */
  int32_t reserved;
} wp_batch_plan;

/* `items` is a HOST array of `count` descriptors (device pointers inside).
 * Limits: 1 <= n1, n2, n4 <= 64, 0 <= L <= 5, p % 2^L == 0,
 * 1 <= r <= min(n1, n2).  wp_batched_plan writes the work lists into the
 * workspace (host-to-device copies, then a synchronisation of `stream`) and,
 * with tune = 1, times candidate CTA sizes for the face-product and Jacobi
 * phases on the planned work (this runs those phases; outputs are not
 * final until wp_batched_run).  wp_batched_run launches the four phases
 * (lifting, face-products, Jacobi SVD with rank-r rebuild, inverse lifting;
 * the Jacobi phase as up to three launches, one per slice-width class of the
 * plan).  The face-products run on a library-owned second stream of the
 * device (created on the first call), forked from `stream` after the lifting
 * and joined back before the inverse lifting, so they overlap the Jacobi
 * phase; calls on one device therefore share that stream and must not run
 * concurrently from several host threads.  The call neither allocates,
 * copies nor synchronises, so it can be captured in a CUDA graph (the fork
 * and join become graph dependencies; wp_batched_plan creates the second
 * stream beforehand) and replayed while the workspace and the items'
 * buffers live. */
WP_API int wp_batched_workspace(const wp_batch_item* items, int count, size_t* bytes);
WP_API int wp_batched_plan(const wp_batch_item* items, int count, int tune, void* ws, size_t ws_bytes,
                           wp_batch_plan* plan, void* stream);
WP_API int wp_batched_run(const wp_batch_plan* plan, void* ws, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* WPROD_H */
