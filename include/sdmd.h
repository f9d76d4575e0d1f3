/*
 * sdmd.h -- C ABI of libsdmd, a streaming method-of-snapshots DMD engine for
 * one NVIDIA GB300 (sm_103a). Implements the streaming SVD and exact DMD of
 * Pendergrass, Kutz & Brunton, "Streaming GPU Singular Value and Dynamic Mode
 * Decompositions" (arXiv 1612.07875).
 *
 * Model. A handle holds a window of the m most recent snapshots x_t (each a
 * vector of n values) in a device-resident ring buffer, and the window's
 * inner-product matrix G = X^H X (m x m) indexed by ring slot. Each push
 * computes the one new row/column of G (m dot products over n) and drops the
 * oldest snapshot by advancing the ring head instead of moving data
 * (Sec. 3.1, Eq. 12a-b; Algorithm 1). sdmd_modes then reads X^H X and X^H X'
 * as two blocks of the same G, solves the small eigenproblems in FP64 on the
 * device and forms the exact DMD modes Phi = X' V Sigma^-1 W (Sec. 2.2,
 * Eqs. 7-9; Algorithm 2).
 *
 * Conventions for every entry point:
 *  - Return value is an sdmd_status; nothing throws across the ABI. On error
 *    sdmd_last_error() gives a message (thread-local, valid until the next
 *    call on the same thread).
 *  - `stream` is a cudaStream_t (CUstream) passed as void*; NULL means the
 *    legacy default stream. All device work is enqueued on it and the call
 *    returns without waiting, except where stated.
 *  - Buffer arguments may be device pointers (cudaMalloc / managed) or host
 *    pointers (pinned or pageable); the kind is detected per call. Host
 *    inputs are copied with cudaMemcpyAsync on `stream` (a pageable source is
 *    copied before the call returns). Outputs to device or pinned host memory
 *    are written in stream order; outputs to pageable host memory make the
 *    call wait for `stream` to finish. Buffers must stay valid until the
 *    stream reaches the work that uses them.
 *  - The library owns the ring buffer, G and its workspaces (device memory
 *    allocated in sdmd_create, freed in sdmd_destroy). The caller owns every
 *    pointer it passes.
 *  - Calls on one handle must be issued in one stream order (one stream, or
 *    streams the caller orders with events); a handle is not thread-safe.
 *  - The handle is bound to the CUDA device that was current at create time;
 *    each call makes that device current and restores the caller's device.
 */
#ifndef SDMD_H
#define SDMD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SDMD_API __attribute__((visibility("default")))
#else
#define SDMD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdmd_s *sdmd_t;

/* Snapshot element types. */
enum {
    SDMD_F32 = 0,        /* dense float32 snapshots; G accumulated in FP64      */
    SDMD_U8 = 1,         /* dense uint8 (e.g. video pixels); G exact in int64   */
    SDMD_C64 = 2,        /* dense complex64 (interleaved re, im); G complex128  */
    SDMD_C64_SPARSE = 3  /* sparse complex64 coefficients of an orthonormal
                            transform (sdmd_create_sparse); G complex128      */
};

/* Status codes. */
enum {
    SDMD_OK = 0,
    SDMD_ERR_ARG = -1,        /* invalid argument (size, pointer, dtype, r)    */
    SDMD_ERR_OOM = -2,        /* device allocation failed                      */
    SDMD_ERR_NOT_READY = -3,  /* window too short for the request              */
    SDMD_ERR_CUDA = -4,       /* a CUDA runtime call or kernel launch failed   */
    SDMD_ERR_TIMEOUT = -5,    /* a bounded device wait gave up                 */
    SDMD_ERR_RANK = -6,       /* numerically singular system                   */
    SDMD_ERR_UNSUPPORTED = -7 /* operation not available for this handle type  */
};

/* Largest window (number of resident snapshots) a handle may hold. */
#define SDMD_MAX_M 256
/* Largest number of DMD frames in flight in a pipelined handle. */
#define SDMD_MAX_DEPTH 16

/*
 * sdmd_create -- allocate a streaming window.
 *   n      number of values per snapshot (the paper's n, Eq. 1), 1 <= n <= 2^34.
 *   m      window length: number of resident snapshots, 2 <= m <= SDMD_MAX_M.
 *          G is m x m; DMD uses the c-1 snapshot pairs of the c <= m resident
 *          snapshots (X = oldest c-1, X' = newest c-1; Algorithm 2).
 *   dtype  SDMD_F32, SDMD_U8 or SDMD_C64 (sparse handles: sdmd_create_sparse).
 *   out    receives the handle (host pointer).
 * Device memory: m * round_up(n * sizeof(elem), 4096) bytes of ring plus
 * O(m^2) of G and workspaces. Ring padding is zero and never written, so
 * vector kernels may read whole 4 KiB units. Returns SDMD_ERR_OOM if any
 * allocation fails (nothing is leaked). Synchronous.
 */
SDMD_API int sdmd_create(int64_t n, int32_t m, int32_t dtype, sdmd_t *out);

/*
 * sdmd_create_ex -- as sdmd_create, with `depth` DMD frames in flight for
 * sdmd_step (1 <= depth <= SDMD_MAX_DEPTH; 1 = no pipelining). A pipelined
 * handle keeps m + depth snapshots in its ring (so the X' of frames still
 * being decomposed is not overwritten), one workspace and CUDA stream per
 * frame in flight.
 */
SDMD_API int sdmd_create_ex(int64_t n, int32_t m, int32_t dtype, int32_t depth, sdmd_t *out);

/*
 * sdmd_create_sparse -- allocate a streaming window of Fourier-sparse
 * snapshots (Sec. 3.5: the SVD and DMD are invariant under unitary
 * transforms, so the coefficients of an orthonormal FFT give the Gram of the
 * physical fields by Parseval's identity).
 *   n        length of the dense coefficient vector (e.g. 1024 * 1024),
 *            1 <= n < 2^31.
 *   m        window length, 2 <= m <= SDMD_MAX_M.
 *   nnz_max  largest number of nonzero coefficients of one snapshot.
 * Device memory: m * nnz_max * 12 bytes of ring, an n * 12-byte lookup
 * table, and O(m^2) for G (complex128). Synchronous.
 */
SDMD_API int sdmd_create_sparse(int64_t n, int32_t m, int32_t nnz_max, sdmd_t *out);

/* sdmd_destroy -- wait for the handle's device work and free it. NULL is OK. */
SDMD_API int sdmd_destroy(sdmd_t h);

/*
 * sdmd_push -- append one snapshot (streaming Gram update, Sec. 3.1, Eq. 12b;
 * Algorithm 1's else branch).
 *   x   n elements of the handle's dtype, contiguous; host or device pointer.
 * Copies x into ring slot `head`, computes g_j = <x_j, x> for every resident
 * slot j (including x itself) and writes g into row and column `head` of G
 * (the symmetric insert), then advances head. The oldest snapshot is
 * overwritten, not moved. Before the window is full nothing is evicted
 * (ramp-up, Sec. 5). FP32: products in FP32 over short runs, sums in FP64,
 * fixed reduction order (deterministic for a given n and GPU). U8: exact.
 */
SDMD_API int sdmd_push(sdmd_t h, const void *x, void *stream);

/*
 * sdmd_push_sparse -- append one sparse snapshot (sparse handles only).
 *   nnz   number of coefficients, 0 <= nnz <= nnz_max.
 *   idx   nnz distinct int32 indices in [0, n) (host or device pointer).
 *   vals  nnz complex64 values (interleaved re, im floats), same order.
 * Computes g_j = sum over indices present in both of conj(x_j[k]) x_new[k]
 * for every resident snapshot j (Sec. 3.1, Eq. 12b on the coefficients),
 * products in FP32 and sums in FP64 in a fixed order, and writes row and
 * column `head` of the Hermitian G. Host index arrays are checked (range,
 * strictly increasing) and rejected with SDMD_ERR_ARG; device index arrays
 * are range-checked by the kernel, which skips offending entries and makes
 * sdmd_status report SDMD_ERR_ARG.
 */
SDMD_API int sdmd_push_sparse(sdmd_t h, int32_t nnz, const int32_t *idx, const void *vals, void *stream);

/*
 * sdmd_rebuild -- recompute the whole Gram of the resident window from the
 * ring buffer (Algorithm 1's first-step branch, G = X^T X; Sec. 2.1 Eq. 3),
 * e.g. to resynchronise G after the ring was modified outside the library.
 * uint8 windows (with SDMD_OPT_REBUILD_TENSOR, the default): on the tensor
 * cores, exact int64, so equal to the streamed G -- one pass over the window
 * up to 127 snapshots; larger windows in groups of 64 target snapshots, each
 * paired with the older ones in blocks of up to 127 - 64 rows. FP32 windows with SDMD_OPT_F32_BF16X3 = 1: the
 * tensor cores in BF16x3 split precision, one pass per block of 64 target
 * columns (|G_ij - <x_i, x_j>| <= 1e-6 sum_p |x_ip x_jp|); windows of at
 * most 16 snapshots in one CUDA-core pass with FP32 products (the same
 * bound, as for sdmd_push_batch). Otherwise one
 * Gram-row pass per resident snapshot, in time order, so every entry is
 * computed with the same reduction as when it was streamed: the result
 * equals the streamed G bit for bit (c passes).
 */
SDMD_API int sdmd_rebuild(sdmd_t h, void *stream);

/*
 * sdmd_push_batch -- append k snapshots at once (1 <= k <= m): the
 * multi-column catch-up of a stream that fell behind. Snapshot j is at
 * X + j * ld elements (ld >= n), host or device memory; each must stay valid
 * until the stream reaches the call. The resulting G equals that of k
 * sdmd_push calls. uint8 windows (with SDMD_OPT_REBUILD_TENSOR): the k new
 * rows and columns of G on the tensor cores (exact int64; one pass over a
 * window of up to 127 snapshots, else per group of 64 new snapshots about
 * one pass per 127 - (group size) older ones) instead of k passes; FP32
 * windows with SDMD_OPT_F32_BF16X3 = 1 (or 2) and k >= 2: the k new rows and
 * columns in one pass over the window -- for k <= 16 on the CUDA cores (FP32
 * products accumulated in FP32 per 64 positions, compensated sums, FP64 over
 * CTAs: the pass is bound by the window's reads), for larger k in BF16x3 on
 * the tensor cores, one pass per 64 new snapshots -- equal to k pushes within
 * the bound given at sdmd_rebuild; other handles: k sdmd_push calls.
 * SDMD_ERR_ARG for a bad k,
 * ld or pointer.
 */
SDMD_API int sdmd_push_batch(sdmd_t h, int32_t k, const void *X, int64_t ld, void *stream);

/*
 * sdmd_push_many -- append one snapshot to each of `count` distinct handles
 * (1 <= count <= SDMD_MAX_BATCH; dense handles of any n, window and element
 * type, one device) with all their Gram rows in one kernel launch: the
 * batching of many streams. xs[i] is handle hs[i]'s snapshot (host or device
 * memory). Each handle's G equals, bit for bit, what sdmd_push gives (same
 * chunking, per-lane sums and reduction order). All handles must be used on
 * `stream`.
 */
#define SDMD_MAX_BATCH 64
SDMD_API int sdmd_push_many(const sdmd_t *hs, const void *const *xs, int32_t count, void *stream);

/*
 * Serving many streams on one GPU (the library's request loop). A server
 * admits streams by device-memory footprint (ring, G, workspaces and a queue
 * of 4 frames): sdmd_server_open admits a stream at once if it fits within
 * the budget after every stream waiting before it, else it waits in arrival
 * order and is admitted when sdmd_server_close frees memory. sdmd_server_submit
 * queues a frame (copied, host or device source; SDMD_ERR_NOT_READY when the
 * stream is not active or its queue is full). sdmd_server_tick pushes the
 * oldest queued frame of every active stream with one sdmd_push_many launch
 * per 64 streams, waits for it, and records each frame's latency (tick
 * completion minus arrival: the host clock at submit, or `arrival_ms` when
 * >= 0, in the same steady millisecond clock). Every stream's G is bit-identical
 * to pushing its frames alone. One host thread drives a server; its GPU work
 * runs on its own stream (sdmd_server_stream), which the caller uses for
 * sdmd_modes and the other calls on served handles (sdmd_server_handle).
 */
typedef struct sdmd_server_s *sdmd_server_t;
enum { SDMD_STREAM_WAITING = 0, SDMD_STREAM_ACTIVE = 1, SDMD_STREAM_CLOSED = 2 };
SDMD_API int sdmd_server_create(int64_t hbm_budget, sdmd_server_t *out);
SDMD_API int sdmd_server_destroy(sdmd_server_t s);
SDMD_API int sdmd_server_stream(sdmd_server_t s, void **stream);
/* SDMD_ERR_ARG if the stream alone exceeds the budget or a size is invalid */
SDMD_API int sdmd_server_open(sdmd_server_t s, int64_t n, int32_t m, int32_t dtype, int32_t *sid);
/* SDMD_STREAM_* of stream `sid` */
SDMD_API int sdmd_server_state(sdmd_server_t s, int32_t sid);
SDMD_API int sdmd_server_handle(sdmd_server_t s, int32_t sid, sdmd_t *h);
SDMD_API int sdmd_server_submit(sdmd_server_t s, int32_t sid, const void *x, double arrival_ms);
SDMD_API int sdmd_server_tick(sdmd_server_t s, int32_t *frames_done);
SDMD_API int sdmd_server_close(sdmd_server_t s, int32_t sid);
SDMD_API int sdmd_server_stats(sdmd_server_t s, double *p50_ms, double *p99_ms, int64_t *frames);
/* device bytes held by active streams (-1 for a NULL server) */
SDMD_API int64_t sdmd_server_used_bytes(sdmd_server_t s);
/* on (default): each tick's batch is one CUDA graph launch (copy nodes and
 * the batched kernel node), built once per set of streams and updated in
 * place on later ticks; off: copies and a kernel launch on the stream */
SDMD_API int sdmd_server_set_graphs(sdmd_server_t s, int32_t on);
/* graphs built and updated in place so far (host pointers, may be NULL) */
SDMD_API int sdmd_server_graph_stats(sdmd_server_t s, int64_t *builds, int64_t *updates);
/* sdmd_autotune on every active stream holding a snapshot (server stream) */
SDMD_API int sdmd_server_autotune(sdmd_server_t s);
/* forget the latencies and frame count gathered so far (e.g. after warm-up) */
SDMD_API int sdmd_server_reset_stats(sdmd_server_t s);
/* the clock that arrival_ms and the latencies use: milliseconds of a
 * monotonic host clock (arbitrary origin, shared by all servers) */
SDMD_API double sdmd_server_clock_ms(void);

/* sdmd_count -- number of snapshots pushed so far (host pointer). Host-side
 * bookkeeping only; does not touch the device. */
SDMD_API int sdmd_count(sdmd_t h, int64_t *count);

/*
 * sdmd_gram -- copy the window's Gram in time order (test and inspection
 * hook). G receives c x c row-major values, c = min(count, m), oldest
 * snapshot first: double for SDMD_F32, int64_t for SDMD_U8, complex128
 * (interleaved re, im doubles; G[i][j] = <x_i, x_j> = x_i^H x_j) for the
 * complex handles.
 */
SDMD_API int sdmd_gram(sdmd_t h, void *G, void *stream);

/*
 * sdmd_modes -- exact DMD of the current window (Sec. 2.2, Eqs. 7-9;
 * Algorithm 2), all small algebra in FP64 on the device:
 *   G_X = G[0:c-1, 0:c-1], G_XY = G[0:c-1, 1:c]  (X^H X and X^H X', read as
 *        blocks of the one time-ordered G; no second set of dot products)
 *   G_X V = V Lambda_G, sorted descending, sigma = sqrt(Lambda_G), truncated
 *        to r and to the numerical rank (Gram eigenvalues above
 *        lambda_1 * 64 * (c-1) * 2^-52)
 *   vsi = V Sigma^-1; A~ = vsi^T G_XY vsi; A~ W = W Lambda (unit-norm columns)
 *   Phi = X' vsi W   (X' read in place from the ring)
 *   r       requested number of modes, 1 <= r <= m-1. While the window is
 *           ramping up (c-1 < r) the modes beyond c-1 come out as zero.
 *   phi     n x r complex64, column-major (mode k at phi + 2*k*n floats,
 *           interleaved re, im), or NULL to skip forming Phi. Columns at or
 *           beyond the kept rank are zero.
 *   lambda  r complex128 (interleaved re, im doubles) ordered by descending
 *           |lambda| then by angle; entries beyond the kept rank are zero.
 *   r_out   receives the kept rank (int32), or NULL.
 * phi must be device memory (SDMD_ERR_ARG otherwise); lambda and r_out may
 * be device or host memory. Complex handles (SDMD_C64, SDMD_C64_SPARSE):
 * the same small algebra with complex V (FP64 Jacobi for the Hermitian G_X,
 * A~ = vsi^H G_XY vsi), lambda / sigma / amplitudes as above; dense complex
 * handles form Phi = X' M with complex X' (CUDA cores, FP32 complex
 * products); Fourier-sparse handles take phi = NULL (SDMD_ERR_UNSUPPORTED
 * otherwise) and form their modes in coefficient space with
 * sdmd_fourier_modes. Needs c >= 3
 * snapshots (else SDMD_ERR_NOT_READY). The eigensolvers have iteration caps; if one is
 * reached the call still completes and sdmd_status reports SDMD_ERR_RANK.
 */
SDMD_API int sdmd_modes(sdmd_t h, int32_t r, void *phi, void *lambda, int32_t *r_out, void *stream);

/*
 * sdmd_step -- pipelined streaming DMD: push x (as sdmd_push), then compute
 * the exact DMD of the new window (as sdmd_modes) on an internal stream so
 * that it overlaps with the following pushes. The eigensolvers, Phi and the
 * output copies run on the internal stream of one of `depth` frame contexts;
 * the eigensolvers read the window's entries of G in place (later pushes
 * write only their own slots' rows and columns). `stream` only waits for a
 * context when its workspace, the ring slots it reads or their rows of G are
 * about to be reused (depth pushes later); sdmd_rebuild waits for every
 * context's eigensolver.
 * Results of this call (phi, lambda, r_out) are complete once `stream`
 * passes sdmd_sync, or the sdmd_step call `depth` calls later. phi must be
 * a distinct device buffer per frame in flight; lambda / r_out must be
 * device or pinned host memory. Until 3 snapshots are resident only the
 * push happens. Real dense handles only; all pushes and steps of a handle
 * must use one stream. With depth 1 this is sdmd_push + sdmd_modes.
 */
SDMD_API int sdmd_step(sdmd_t h, const void *x, int32_t r, void *phi, void *lambda, int32_t *r_out,
                       void *stream);

/*
 * sdmd_autotune -- pick the Gram-row schedule of this handle by measurement:
 * the newest snapshot's row over the current window is timed (CUDA events,
 * 3 runs after a warm-up) with 1, 2, 3, 4 and 6 chunks per SM (chunks of 4 to
 * 24 KiB taken from a counter by persistent CTAs) and the fastest is kept for
 * later pushes (and for sdmd_push_many). The row is recomputed with the kept
 * schedule at the end. uint8 rows are exact under every schedule; float rows
 * change only in rounding (the reduction order follows the chunks).
 * chunk_bytes / us (host, may be NULL) receive the kept chunk size and its
 * time per row. Waits for the stream, and first for the eigensolvers of
 * sdmd_step frames still in flight (they read that row). Dense handles with
 * at least one snapshot (SDMD_ERR_NOT_READY otherwise).
 */
SDMD_API int sdmd_autotune(sdmd_t h, int64_t *chunk_bytes, double *us, void *stream);

/* sdmd_sync -- make `stream` wait for every sdmd_step frame still in flight. */
SDMD_API int sdmd_sync(sdmd_t h, void *stream);

/*
 * sdmd_svd -- singular values and right singular vectors of X from the last
 * sdmd_modes call (Sec. 2.1, Eqs. 3-4; Algorithm 1). sigma receives r doubles
 * (descending; zero beyond the kept rank), V receives (c-1) x r doubles,
 * column-major (vector k at V + k*(c-1)); complex handles: (c-1) x r
 * complex128 (interleaved re, im; vector k at V + 2*k*(c-1)). Either may be
 * NULL. r must equal the r of that sdmd_modes call.
 */
SDMD_API int sdmd_svd(sdmd_t h, int32_t r, double *sigma, double *V, void *stream);

/*
 * sdmd_amplitudes -- DMD mode amplitudes b of the last sdmd_modes call, from
 * the POD coefficients of x_1 (Sec. 3.3, Eq. 14a-e: b = (W Lambda)^-1 alpha_1,
 * alpha_1 = Sigma V^H e_1, x_1 the oldest snapshot of X), in the order of that
 * call's lambda. b receives r complex128 (interleaved re, im; zero beyond the
 * kept rank), host or device memory; bg_index (host, may be NULL) receives the
 * background mode argmin_k |log lambda_k| (Algorithm 3, principal log), -1 if
 * no mode was kept; with bg_index the call waits for the stream.
 * SDMD_ERR_NOT_READY if no sdmd_modes call has run since the last push (the
 * frames of sdmd_step keep their results per frame and do not count).
 */
SDMD_API int sdmd_amplitudes(sdmd_t h, void *b, int32_t *bg_index, void *stream);

/* What sdmd_reconstruct returns. */
enum {
    SDMD_RECON_MODES = 0,       /* sum_k b_k phi_k lambda_k^t over the kept modes */
    SDMD_RECON_BACKGROUND = 1,  /* b_i phi_i lambda_i^t, i = background mode (Algorithm 3) */
    SDMD_RECON_FOREGROUND = 2,  /* x_t minus its background (Eq. 11's sparse part) */
    SDMD_RECON_BACKGROUND_SLOW = 3, /* sum over the slow modes, |log lambda_k| <= tol
                                       (several background modes; sdmd_reconstruct_ex) */
    SDMD_RECON_FOREGROUND_SLOW = 4  /* x_t minus the slow-mode background */
};

/*
 * sdmd_reconstruct -- the window's DMD reconstruction at time index t from
 * the last sdmd_modes call (Sec. 2.2, Eq. 11; Algorithm 3): t = 0 is x_1, the
 * oldest snapshot of X, and t = c-1 the newest resident snapshot; larger t
 * extrapolates. Computed as X' Re(M c), c_k = b_k lambda_k^t, without forming
 * Phi (the snapshots are real). out receives n float32 values (real part),
 * device memory, 16-byte aligned. SDMD_RECON_FOREGROUND needs 0 <= t <= c-1.
 * Real dense handles (SDMD_F32, SDMD_U8; SDMD_ERR_UNSUPPORTED otherwise);
 * SDMD_ERR_NOT_READY if no sdmd_modes call has run since the last push
 * (sdmd_step frames do not count); SDMD_ERR_ARG for a bad t, `what` or
 * pointer.
 */
SDMD_API int sdmd_reconstruct(sdmd_t h, int64_t t, int32_t what, float *out, void *stream);

/*
 * sdmd_reconstruct_ex -- sdmd_reconstruct with a tolerance for the slow-mode
 * variants: SDMD_RECON_BACKGROUND_SLOW sums b_k phi_k lambda_k^t over every
 * kept mode with |log lambda_k| <= tol (principal log; the background of
 * Eq. 11 spanned by several slow modes instead of Algorithm 3's single
 * argmin), SDMD_RECON_FOREGROUND_SLOW is x_t minus that sum. tol >= 0; it is
 * ignored by the other variants. Errors as sdmd_reconstruct.
 */
SDMD_API int sdmd_reconstruct_ex(sdmd_t h, int64_t t, int32_t what, double tol, float *out, void *stream);

/*
 * sdmd_fourier_modes -- DMD modes of a Fourier-sparse window without leaving
 * coefficient space (Sec. 3.5; Eq. 9 with X' in Fourier coefficients):
 * Phi-hat = X'-hat M from the last sdmd_modes call, which is nonzero only on
 * the union of the supports of X' (the c-1 newest resident snapshots). The
 * compressed result: idx receives the union's coefficient indices in
 * increasing order (int32), phi the matching rows of Phi-hat, complex64
 * column-major with leading dimension cap (mode k at phi + 2*k*cap floats).
 * *count (host) receives the union size. cap = 0 (idx and phi may be NULL)
 * only counts; if the union exceeds cap the outputs are incomplete and the
 * call returns SDMD_ERR_ARG with *count set. idx and phi are device memory.
 * Waits for the stream. Fourier-sparse handles only (SDMD_ERR_UNSUPPORTED);
 * SDMD_ERR_NOT_READY if no sdmd_modes call has run since the last push; r
 * must equal that call's r.
 */
SDMD_API int sdmd_fourier_modes(sdmd_t h, int32_t r, int32_t *idx, void *phi, int64_t cap, int64_t *count,
                                void *stream);

/*
 * sdmd_pod_modes -- the POD (left singular) vectors of X from the last
 * sdmd_modes call: U = X V Sigma^-1 (Sec. 2.1, Eq. 4), the SVD-only output of
 * the method of snapshots, formed in one pass over X (the oldest c-1
 * resident snapshots). U receives n x r float32, column-major (vector k at
 * U + k*n), device memory, 4-byte aligned; columns beyond the kept rank are
 * zero. r must equal the r of that sdmd_modes call. Real dense handles;
 * SDMD_ERR_NOT_READY if no sdmd_modes call has run since the last push.
 */
SDMD_API int sdmd_pod_modes(sdmd_t h, int32_t r, float *U, void *stream);

/*
 * sdmd_status -- waits for `stream`, then reports the device-side status
 * word of the handle (SDMD_OK, or SDMD_ERR_RANK / SDMD_ERR_TIMEOUT /
 * SDMD_ERR_ARG (sparse index out of range) raised by a kernel since the last
 * sdmd_status call) and clears it.
 */
SDMD_API int sdmd_status(sdmd_t h, void *stream);

/* Options (sdmd_set_option). */
enum {
    SDMD_OPT_PHI_TENSOR = 1 /* 1 (default): Phi of uint8 handles on the tensor
                               cores (tcgen05, fp16 operands: pixels exact,
                               M = V Sigma^-1 W as three power-of-two-scaled
                               fp16 terms, FP32 accumulation), the modes
                               of a pass fitted to r (r <= 10: one pass of
                               10 modes); 2: the same arithmetic in passes
                               of 16 modes whatever r (results are
                               identical); 0: CUDA-core FP32 kernel */
    ,
    SDMD_OPT_REBUILD_TENSOR = 2 /* 1 (default): sdmd_rebuild and sdmd_push_batch
                                   of uint8 windows on the tensor cores
                                   (centred fp16 pixels, exact int64 G); 0:
                                   one Gram-row pass per snapshot
                                   (bit-identical to streaming for every
                                   dtype) */
    ,
    SDMD_OPT_F32_BF16X3 = 3 /* 0 (default): FP32 windows keep FP32 products
                               with FP64 sums everywhere; 1: sdmd_rebuild and
                               sdmd_push_batch (k >= 2) of FP32 windows on the
                               tensor cores in BF16x3 split precision (each
                               value as three bf16 terms, the six products
                               b_i c_j with i + j <= 2, FP32 accumulation per
                               64 positions, compensated sums; bound
                               1e-6 sum_p |x_ip x_jp|); 2: the same with two
                               bf16 terms and the three products with
                               i + j <= 1 (about 2^-16 per product). Either
                               value runs catch-ups of at most 16 snapshots
                               (and rebuilds of windows of at most 16) on the
                               CUDA cores with FP32 products instead, within
                               the three-term bound */
    ,
    SDMD_OPT_F32_FP64 = 4   /* 0 (default): Gram rows of FP32 windows with FP32
                               products and FP64 sums; 1: FP64 products (exact
                               for FP32 inputs) and FP64 sums, the reference
                               precision (GB300 runs FP64 at a small fraction
                               of FP32: several times slower) */
    ,
    SDMD_OPT_HOST_EARLY_READ = 5 /* 0 (default): a snapshot in host memory is
                               read in stream order, like a device one; 1: a
                               snapshot in pinned (page-locked) host memory
                               given to sdmd_push / sdmd_step is copied as
                               soon as the call is made, on the handle's own
                               copy stream into one of two device staging
                               slots, so the transfer overlaps the kernels
                               queued before the call; the stream then waits
                               for it and moves it into the ring. The host
                               buffer must hold the snapshot when the call is
                               made (not only when the stream reaches it) and
                               must not change until the stream passes the
                               push. Costs 2 x n x element size of device
                               memory. Dense handles only (sparse:
                               SDMD_ERR_UNSUPPORTED). */
};

/* sdmd_set_option -- set a handle option (SDMD_OPT_*). Host-side only. */
SDMD_API int sdmd_set_option(sdmd_t h, int32_t option, int64_t value);

/* Kernel classes for tracing. */
enum {
    SDMD_K_INGEST = 0,    /* snapshot copy into its ring slot (a memcpy)       */
    SDMD_K_GRAM_ROW = 1,  /* Gram-row multi-dot + symmetric insert            */
    SDMD_K_MODES = 2,     /* FP64 eigensolvers / small products (one CTA)     */
    SDMD_K_PHI = 3,       /* Phi = X' (V Sigma^-1 W)                          */
    SDMD_K_FRAME = 4,     /* one sdmd_step frame: call start to outputs done  */
    SDMD_K_FUSED = 5,     /* Phi of an earlier frame + this snapshot's Gram row in one pass */
    SDMD_K_COUNT = 6
};

/*
 * sdmd_trace -- enable (1) or disable (0) per-launch timing on a handle. While
 * enabled, every device operation of the handle is bracketed by a pair of
 * CUDA events recorded on the stream it is enqueued on. Host-side only; adds
 * no device work besides the event records.
 */
SDMD_API int sdmd_trace(sdmd_t h, int32_t enable);

/*
 * sdmd_trace_read -- for kernel class `kernel` (SDMD_K_*), waits for the
 * recorded events and returns the number of traced launches and their total
 * device time in milliseconds since the previous read (or since tracing was
 * enabled), then resets that class's counters.
 */
SDMD_API int sdmd_trace_read(sdmd_t h, int32_t kernel, int64_t *launches, double *total_ms);

/*
 * sdmd_trace_times -- like sdmd_trace_read, but returns the individual
 * durations (ms) of up to `cap` traced launches of class `kernel` in `ms`
 * and their number in `count` (host pointers); resets that class.
 */
SDMD_API int sdmd_trace_times(sdmd_t h, int32_t kernel, double *ms, int32_t cap, int32_t *count);

/*
 * sdmd_modes_phase_cycles -- SM clock counter (clock64) at the phase
 * boundaries of the last FP64 modes kernel, for profiling: [0] start,
 * [1] gather, [2] tridiagonalisation, [3] bisection, [4] inverse iteration,
 * [5] back-transform, [6] A~, [7] eig(A~), [8] end. Copies `count` (<= 16)
 * values to host memory and waits for `stream`.
 */
SDMD_API int sdmd_modes_phase_cycles(sdmd_t h, int64_t *cycles, int32_t count, void *stream);

/*
 * sdmd_modes_many -- the small algebra of exact DMD (as sdmd_modes, Sec. 2.2,
 * Eqs. 7-8; Algorithm 2: eig of G_X, rank, sigma, V, A~, eig(A~), the
 * amplitudes) for `count` <= 64 real dense handles in one launch, one CTA per
 * handle, each on its own G and workspace: the eigenvalues, rank and every
 * later sdmd_svd / sdmd_amplitudes / sdmd_reconstruct of a handle are the
 * same bits as after sdmd_modes(hs[i], r[i], NULL, ...). Serves many streams
 * whose frames arrive together (the serving loop), where one-CTA launches
 * per stream would queue behind each other.
 *   hs      count handles (distinct, one device, >= 3 snapshots each)
 *   r       count requested ranks, 1 <= r[i] <= m_i - 1 (host)
 *   lambda  NULL, or count pointers (host array) to r[i] complex128 each,
 *           device or pinned host memory (an entry may be NULL)
 *   r_out   NULL, or count int32 kept ranks (device or pinned host)
 * No Phi: use sdmd_pod_modes / sdmd_reconstruct, or sdmd_modes per handle.
 * Errors as sdmd_modes; SDMD_ERR_UNSUPPORTED for complex handles.
 */
SDMD_API int sdmd_modes_many(const sdmd_t *hs, int32_t count, const int32_t *r, void *const *lambda,
                             int32_t *r_out, void *stream);

/*
 * sdmd_newest_row / sdmd_set_newest_row -- read or overwrite the newest
 * snapshot's row of the window's G (and, for the set, its column: the
 * conjugate), in time order: entry q is <x_q, x_new> for the q-th oldest
 * resident snapshot, the last entry <x_new, x_new>. Element type as
 * sdmd_gram (int64, double or complex128), c entries (c = resident
 * snapshots). `row` may be device or host memory; pageable host memory makes
 * the call wait for the stream.
 * These are the exchange points of the row-slab split of one stream over
 * several GPUs (Sec. 3.1, Eq. 12a-b: every entry of the new row is a sum
 * over the n positions, so it splits over position ranges). Each rank holds
 * positions [lo, hi) of every snapshot in a handle of n = hi - lo, pushes
 * its part of x_new (sdmd_push computes the partial row over its positions
 * and inserts it), reads that partial row with sdmd_newest_row, sums the
 * ranks' partial rows (one all-reduce of c values; exact for int64), and
 * writes the sum back with sdmd_set_newest_row. Every rank then holds the
 * full window's G; sdmd_modes on each gives the same eigenvalues and the
 * rows lo .. hi - 1 of Phi. SDMD_ERR_NOT_READY before the first push.
 */
SDMD_API int sdmd_newest_row(sdmd_t h, void *row, void *stream);
SDMD_API int sdmd_set_newest_row(sdmd_t h, const void *row, void *stream);

/*
 * sdmd_gram_row_static -- one Gram row, g[j] = <x_j, y> for j < c, computed
 * without allocating any device memory. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code whose
 * device memory is owned by another allocator (a framework's caching pool or
 * a serving runtime that hands out only pre-registered buffers), real-time
 * loops that must not take cudaMalloc's device-wide synchronisation or its
 * unbounded latency, and plugins whose host application forbids device
 * allocations. It needs no handle: the caller passes every input and output.
 *   dtype  SDMD_F32 (g: c doubles) or SDMD_U8 (g: c int64, exact).
 *   X      device pointer to c snapshots of n elements; snapshot j starts at
 *          element j * ld. X and y 16-byte aligned, ld * sizeof(elem) a
 *          multiple of 16, ld >= n.
 *   c      1 <= c <= SDMD_GRAM_ROW_STATIC_MAX_C; larger c is rejected with
 *          SDMD_ERR_ARG.
 *   y      device pointer to n elements (may alias one of the x_j).
 *   g      device pointer to the c outputs.
 * Scratch: a fixed 1 MiB + 256 B array in device global memory, compiled
 * into the library (every GPU that loads the library holds it until process
 * exit). The first call on each device looks up that array's address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * All calls share the one array and the ticket in it is reset to zero at the
 * start of each call: calls that overlap on the GPU (on different streams,
 * or from several threads) race and must be serialised by the caller.
 * FP32 results use a different summation order than sdmd_push (equal to
 * rounding); U8 results are exact.
 * `stream` must belong to the current device (SDMD_ERR_ARG otherwise): the
 * kernel runs there with that device's scratch address. The address is
 * looked up once per device ordinal and kept for the life of the process, so
 * calls after cudaDeviceReset (a new primary context) are not supported.
 */
#define SDMD_GRAM_ROW_STATIC_MAX_C 256
SDMD_API int sdmd_gram_row_static(int32_t dtype, const void *X, int64_t ld, int32_t c, const void *y,
                                  int64_t n, void *g, void *stream);

/* sdmd_last_error -- message for the last failed call on this thread. */
SDMD_API const char *sdmd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SDMD_H */
