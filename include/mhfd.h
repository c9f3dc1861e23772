/*
 * mhfd.h - C ABI of the GB300 (sm_103a) multi-scale histologic feature
 * detector (MHFD, arXiv 2108.12050).
 *
 * The detector computes, for one grey-level image I (H x W, row pitch in
 * bytes, uint8 / uint16 / float32, resident in device memory):
 *
 *   1. the histogram stretch of §3 (Algorithm 1, first step): lo/hi are the
 *      k-th smallest and (N-1-k)-th smallest pixel values, k = floor(clip*N),
 *      N = H*W, and I' = clamp((I - lo)/(hi - lo), 0, 1);
 *   2. the Gaussian scale-space stack of §2.2 over the linear ladder
 *      t_i = t_min + (i-1)(t_max - t_min)/n, i = 1..n+1: each level is the
 *      separable convolution of I' with the sampled Gaussian of variance t_i^2,
 *      truncated at R_i = ceil(truncate * t_i), normalised, reflect boundary;
 *   3. the DoG responses of Eq. 2: D_i = t_i (L_{i+1} - L_i), i = 1..n;
 *   4. local maxima (Eq. 3): either the paper's rule (M = max_i D_i, first
 *      argmax i_hat; keep when M > threshold and M equals its 3x3 max-pool,
 *      out-of-image neighbours ignored) or 3x3x3 scale-space maxima;
 *   5. greedy overlap pruning of the blobs (radius sqrt(2) t_i): visited by
 *      radius, then response (both descending), then row-major position; a
 *      blob is dropped when a kept blob covers more than `overlap` of the
 *      smaller circle; overlap >= 1 keeps every candidate;
 *   6. the focus score of §3 / Algorithm 1: the number of features kept.
 *
 * Every step runs in this library's own CUDA kernels on the caller's stream;
 * there is no CPU fallback.  All calls return an int status: MHFD_OK (0), a
 * negative error code, or the positive warning MHFD_WARN_OVERFLOW.  The text of
 * the last error of the calling thread is available from mhfd_last_error().
 */
#ifndef MHFD_H
#define MHFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MHFD_OK 0
#define MHFD_WARN_OVERFLOW 1        /* candidate list truncated; true count reported */
#define MHFD_ERR_INVALID_ARG (-1)   /* bad size, pointer, ladder or parameter */
#define MHFD_ERR_UNSUPPORTED (-2)   /* ladder too wide for the on-chip tile, or a
                                       variant the entry point does not serve */
#define MHFD_ERR_OOM (-3)           /* device or pinned allocation failed */
#define MHFD_ERR_CUDA (-4)          /* a CUDA runtime/driver call failed */
#define MHFD_ERR_TIMEOUT (-5)       /* a bounded device-side wait gave up */
#define MHFD_ERR_JIT (-6)           /* run-time compilation of the kernel failed */
#define MHFD_ERR_CHECK (-7)         /* debug build (MHFD_DEBUG_CHECKS=1): a bounds check
                                       failed; the access was skipped */

typedef enum { MHFD_U8 = 0, MHFD_U16 = 1, MHFD_F32 = 2 } mhfd_dtype;
typedef enum { MHFD_NMS_PAPER = 0, MHFD_NMS_LOCAL26 = 1 } mhfd_nms;
/* Response: the DoG of Eq. 2, or the scale-normalised Laplacian t_i^2 grad^2 L
 * of §2.2 that the DoG approximates (5-point stencil on each level t_1..t_n;
 * the fused kernel folds the second differences into derived taps; it lacks
 * the DoG's factor dt, so thresholds scale by 1/dt). */
typedef enum { MHFD_RESPONSE_DOG = 0, MHFD_RESPONSE_LOG = 1 } mhfd_response;
/* Boundary of the blur: reflect, or periodic (the circular convolution of the
 * paper's Fourier formulation, §3). */
typedef enum { MHFD_BOUNDARY_REFLECT = 0, MHFD_BOUNDARY_PERIODIC = 1 } mhfd_boundary;

typedef struct mhfd_detector mhfd_detector;  /* opaque, owned by the library */

/* Detector configuration (Algorithm 1's inputs n, min_t, max_t plus the
 * threshold, pruning and stretch parameters).  Fill with
 * mhfd_default_params() and override fields. */
typedef struct {
    int32_t n;              /* DoG layers; n+1 Gaussian scales; 1 <= n <= 63 */
    double t_min, t_max;    /* ladder ends, 0 < t_min < t_max */
    const double *sigmas;   /* optional explicit ladder of n+1 increasing scales
                               (host memory, read during create); overrides
                               t_min/t_max when non-NULL */
    float threshold;        /* a feature needs response > threshold (finite) */
    float overlap;          /* prune fraction in [0, 1]; >= 1 disables pruning */
    int32_t nms;            /* mhfd_nms */
    float truncate;         /* kernel radius R = ceil(truncate * t); > 0 */
    double clip_frac;       /* stretch saturation per end, 0 <= clip < 0.5 */
    int64_t max_candidates; /* capacity of the candidate and blob lists */
    int32_t device;         /* CUDA device ordinal; -1 = the current device */
    int32_t keep_candidates;/* 1: also expose the pre-prune candidate list */
    int32_t tile_override;  /* 0 = built-in tile choice; k > 0 = row k-1 of
                               mhfd_tile_configs() (autotuner use) */
    int32_t tile_shape[6];  /* explicit fused-kernel geometry when
                               tile_shape[0] > 0, overriding tile_override:
                               strip width incl. the 2 NMS border columns
                               (multiple of 4), tile height incl. 2 border
                               rows, rows per step (2..16), threads per
                               block (multiple of 32), level groups,
                               horizontal item kind (0 or 1: one row of four
                               outputs; 2: two rows of four, packed two-lane
                               FMAs over the row pair, needs an even number
                               of rows per step; 3: one row of two outputs,
                               twice the items per step); the same six
                               fields as mhfd_tile_configs.
                               INVALID_ARG when out of range, UNSUPPORTED
                               when it does not fit in shared memory */
    int32_t timing;         /* 1: record CUDA events around the kernels of each
                               detection (read with mhfd_last_timing) */
    int32_t response;       /* mhfd_response; every entry point but the soft
                               score (DoG only) supports both */
    int32_t boundary;       /* mhfd_boundary; every entry point but the soft
                               score (reflect only) supports both */
    int32_t tensor_cores;   /* detection of uint8 images and of uint16
                               images whose stretch range hi - lo is at most
                               4095 runs on the tensor cores (tcgen05, fp16
                               operands that hold the window exactly and the
                               taps as two parts, f32 accumulation); other
                               images take the FFMA kernel (same results
                               within the FP32 tolerance).
                               1 (default): detection with the DoG response
                               runs both blur passes as products (the
                               two-pass kernel: tiles of 126 output rows,
                               the V rows split into fp16 hi + lo parts for
                               the horizontal product; the 26-neighbour rule
                               tested one layer at a time, up to n = 16);
                               tile_shape[0] > 0 then sets its strip width
                               (a multiple of 16, at most 128, incl. the 2
                               NMS border columns).  The LoG response, the
                               26-neighbour rule beyond 16 layers and
                               ladders too wide for the two-pass kernel take
                               the vertical-pass kernel of 2.
                               2: the vertical blur on the tensor cores, the
                               horizontal on FFMA (the vertical-pass kernel:
                               the paper rule with either response, the
                               26-neighbour rule with the DoG response);
                               tile_shape / tile_override then describe it
                               (four rows per step, at least 128 threads).
                               0: FFMA only. */
} mhfd_params;

/* A detected feature.  scale_idx is the 0-based DoG layer i-1; sigma = t_i,
 * radius = sqrt(2) t_i. */
typedef struct {
    int32_t x, y, scale_idx;
    float sigma, radius, response;
} mhfd_blob;

/* Results of one detection, valid until the next detect on the detector. */
typedef struct {
    const mhfd_blob *blobs;       /* kept features (detector-owned pinned host
                                     memory), in tile order */
    int64_t n_blobs;
    const mhfd_blob *candidates;  /* pre-prune list if keep_candidates, else NULL */
    int64_t n_candidates;         /* candidates stored (<= max_candidates) */
    int64_t n_candidates_true;    /* candidates found (> stored on overflow) */
    float focus_score;            /* = n_blobs, the paper's criterion */
    float mean_response;          /* mean response of the kept features */
    int32_t per_scale[64];        /* kept features per scale index */
    float lo, hi;                 /* stretch bounds (in input units) */
    int32_t status;               /* MHFD_OK or MHFD_WARN_OVERFLOW */
} mhfd_result;

/* Writes the default parameters: n = 10, t in [1, 10], threshold 0.1,
 * overlap 0.5, paper NMS, truncate 4, clip 0.00175, 1<<20 candidates,
 * current device. */
void mhfd_default_params(mhfd_params *p);

/* Creates a detector.  Validates the parameters, builds the ladder and the
 * kernel taps, and compiles (or loads from the on-disk cache) the fused
 * kernel specialised for the ladder's radii; this may take seconds the first
 * time a ladder is used.  *out receives the handle.  Device scratch grows on
 * first use with a larger image.  Errors: INVALID_ARG, UNSUPPORTED, JIT,
 * CUDA, OOM. */
int mhfd_create_detector(const mhfd_params *p, mhfd_detector **out);

/* Releases every resource of the detector (synchronises its last work). */
int mhfd_destroy_detector(mhfd_detector *det);

/* Enqueues one detection on `stream` (a cudaStream_t; NULL = legacy default
 * stream).  d_img is device memory owned by the caller, H rows of W pixels
 * of `dtype`, rows `pitch_bytes` apart (>= W * element size), and must stay
 * alive and unchanged until the stream work completes.  Nothing is
 * synchronised on the host.  Results are read with mhfd_result_wait.
 * One detector must not be used from two streams at once.
 * Errors: INVALID_ARG (H, W < 1; pitch too small; NULL image), CUDA, OOM. */
int mhfd_detect(mhfd_detector *det, const void *d_img, int32_t dtype, int32_t H, int32_t W,
                size_t pitch_bytes, void *stream);

/* Blocks until the last detection enqueued on `det` has finished, copies its
 * blob list (exactly n_blobs entries; and the candidate list when kept) from
 * device memory into the detector's pinned host buffers and fills *out.
 * Returns the detection's status (MHFD_OK or MHFD_WARN_OVERFLOW) or an
 * error. */
int mhfd_result_wait(mhfd_detector *det, mhfd_result *out);

/* Batch of n images (uneven sizes, mixed dtypes) in one go: per-image
 * stretch selects run together (one launch per radix pass), ONE persistent
 * launch of the fused kernel takes every tile of every image from a device
 * work queue, then each image is gathered, pruned and compacted.  The whole
 * sequence is captured in a CUDA graph the first time a batch shape (sizes,
 * dtypes, pitches) is seen and replayed for later batches of that shape (the
 * image pointers may change).  Arrays of n entries are host memory; d_imgs[j]
 * is device memory, alive until the work completes.  Results of image j are
 * bit-identical to a single mhfd_detect of it.  Read them with
 * mhfd_result_wait_batch.  With params.timing set no graph is used.
 * Errors: INVALID_ARG (per-image checks as mhfd_detect), CUDA, OOM. */
int mhfd_detect_batch(mhfd_detector *det, int32_t n, const void *const *d_imgs,
                      const int32_t *dtypes, const int32_t *H, const int32_t *W,
                      const size_t *pitch_bytes, void *stream);

/* Waits for the last batch and fills outs[0..n-1] (n must equal the batch
 * size).  Blob lists point into detector-owned pinned memory valid until the
 * next batch; candidate lists are not kept for batches.  Returns MHFD_OK,
 * MHFD_WARN_OVERFLOW if any image overflowed, or an error. */
int mhfd_result_wait_batch(mhfd_detector *det, mhfd_result *outs, int32_t n);

/* 2 if the detector's narrow-range detections run the two-pass
 * tensor-core kernel, 1 if they run the vertical-pass tensor-core kernel,
 * 0 if FFMA only (see params.tensor_cores), negative on error.  Host only. */
int mhfd_uses_tensor_cores(mhfd_detector *det);

/* 1 if the last batch ran from a captured CUDA graph, 0 if its kernels were
 * launched directly. */
int mhfd_batch_uses_graph(mhfd_detector *det);

/* Differentiable soft focus score of one image, with the stretch bounds of
 * §3 held fixed (detached):
 *   S = sum_i w_i mean_{x,y} sigmoid((D_i(x,y) - tau) / temperature),
 * D_i the DoG responses of Eq. 2 over the detector's ladder.  d_w: n floats
 * (device).  Writes *d_S and d_mean_sig[i] = mean sigmoid of layer i (device).
 * If d_dimg is not NULL (device, H x W float32) the backward pass also runs,
 * for the upstream gradient grad_s: d_dimg = grad_s dS/dI in input units (the
 * exact transpose of the DoG, of both reflect-boundary blur passes and of the
 * clamp, which passes gradient only strictly between lo and hi) and, if d_dw
 * is not NULL, d_dw[i] = grad_s * mean sigmoid of layer i.  The Gaussian
 * levels are recomputed on every call (nothing is kept between calls).
 * Without d_dimg only the forward runs, in the fused kernel (per-block FP64
 * layer sums, reduced in a fixed order); with it, the fused kernel writes the
 * D planes, and the adjoint blurs each level's gradient plane with that
 * level's own kernel (the reflect blur is self-adjoint).  Both are
 * deterministic.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, UNSUPPORTED (the LoG or
 * periodic variants), CUDA, OOM, JIT. */
int mhfd_soft_score(mhfd_detector *det, const void *d_img, int32_t dtype, int32_t H, int32_t W,
                    size_t pitch_bytes, const float *d_w, float tau, float temperature,
                    float grad_s, void *stream, float *d_S, float *d_mean_sig, float *d_dimg,
                    float *d_dw);

/* Non-blocking: 1 if the last detection (or batch) enqueued on `det` has
 * finished on the GPU, 0 if it is still running, or an error. */
int mhfd_result_ready(mhfd_detector *det);

/* End-to-end convenience: h_img is HOST memory (pinned or pageable); the
 * image is copied to detector-owned device memory on `stream`, detected and
 * the results are waited for and written to *out.  Same errors as above. */
int mhfd_detect_host(mhfd_detector *det, const void *h_img, int32_t dtype, int32_t H, int32_t W,
                     size_t pitch_bytes, void *stream, mhfd_result *out);

/* Asynchronous form of mhfd_detect_host: enqueues the copy of the host image
 * into detector-owned device memory and the detection on `stream` and
 * returns; read the results with mhfd_result_wait.  h_img must stay valid
 * and unchanged until then; with pinned host memory the copy overlaps work
 * already running on other streams (for example the detection of the
 * previous image by another detector).  Same errors as mhfd_detect. */
int mhfd_detect_host_async(mhfd_detector *det, const void *h_img, int32_t dtype, int32_t H,
                           int32_t W, size_t pitch_bytes, void *stream);

/* Same detection as mhfd_detect, computed by the unfused "plain" pipeline:
 * one blur kernel pair per Gaussian level writing every L_i to device
 * memory, then a DoG/argmax kernel, an NMS kernel and the same pruning.  It
 * is the comparison baseline of the fused kernel.  Results through
 * mhfd_result_wait. */
int mhfd_detect_plain(mhfd_detector *det, const void *d_img, int32_t dtype, int32_t H, int32_t W,
                      size_t pitch_bytes, void *stream);

/* Test and inspection entry point: runs the fused kernel in its stack-storing
 * variant and writes the responses D (n planes of H x W float32, plane i =
 * layer i), the per-pixel maximum M (H x W float32) and its first argmax
 * (H x W int32) to caller-owned device buffers (any of them may be NULL).
 * Also leaves a full detection for mhfd_result_wait. */
int mhfd_debug_stack(mhfd_detector *det, const void *d_img, int32_t dtype, int32_t H, int32_t W,
                     size_t pitch_bytes, void *stream, float *d_D, float *d_M, int32_t *d_arg);

/* Runs only the overlap prune (step 5) on a caller-supplied candidate list
 * in device memory: d_x, d_y, d_i (int32 scale index < n), d_resp (float32),
 * n_cand entries, positions inside an H x W image (entries outside are
 * clamped into it).  d_keep (uint8, device) receives 1 for kept candidates.
 * Asynchronous on `stream`. */
int mhfd_prune(mhfd_detector *det, const int32_t *d_x, const int32_t *d_y, const int32_t *d_i,
               const float *d_resp, int64_t n_cand, int32_t H, int32_t W, uint8_t *d_keep,
               void *stream);

/* Allocation-free variant of mhfd_prune.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory, such as
 * code running in a host callback or a real-time thread that must not block
 * on the allocator's implicit synchronisation, or a framework that owns every
 * device allocation.  It needs no detector and calls no cudaMalloc/cudaFree:
 * its working memory is one fixed file-scope device array of about 6.6 MB
 * that every GPU which loads this library holds until the process exits.
 * radius: host array of n_levels (1..64) blob radii, one per scale index
 * (sqrt(2) t_i for the detector's ladder); overlap as in mhfd_params;
 * d_x, d_y, d_i, d_resp, n_cand, H, W, d_keep as in mhfd_prune (entries
 * outside the image or the ladder are clamped into it).  Limits: n_cand <=
 * 65536 and ceil(W/c)*ceil(H/c) <= 65536 with c = ceil(2 max(radius)) + 1;
 * larger calls return MHFD_ERR_INVALID_ARG and do nothing.  Asynchronous on
 * `stream`.  d_keep receives 1 (kept), 0 (dropped) or 2 (unresolved): the
 * settle loop's wait is bounded (2^24 sweeps or 2 s of device time; the
 * environment variable MHFD_PRUNE_MAX_SWEEPS sets a smaller sweep bound),
 * and when the bound runs out the candidates it has not settled get 2 - the
 * result is then incomplete (the detector's prune reports the same event as
 * MHFD_ERR_TIMEOUT).  All calls share the one array (each clears what must
 * start at zero), so calls whose work overlaps on the GPU race: serialise
 * them.  The first call on a device looks up the array's device address
 * with that device current (and `stream` must belong to that device); make
 * it before any stream capture.  The address is kept for the life of the
 * process: cudaDeviceReset after the first call is not supported. */
int mhfd_prune_noalloc(const double *radius, int32_t n_levels, float overlap, const int32_t *d_x,
                       const int32_t *d_y, const int32_t *d_i, const float *d_resp,
                       int64_t n_cand, int32_t H, int32_t W, uint8_t *d_keep, void *stream);

/* Device memory of a detector, for callers that budget HBM (the serving
 * loop admits requests by it; not in the paper).  *fixed_bytes receives the
 * bytes mhfd_create_detector allocated (candidate list and prune buffers
 * sized by params.max_candidates, ladder tables; for the 26-neighbour rule
 * on the two-pass kernel, a response scratch of SMs x n x 128 x strip
 * width floats); *image_bytes the bytes a
 * fused detection (mhfd_detect) of an H x W image adds: tile counters,
 * candidate staging (about 2 B per pixel) and the prune grid.  Those grow to
 * the largest image detected and stay until mhfd_destroy_detector.  The
 * image itself is the caller's; H = W = 0 gives *image_bytes = 0.  The plain
 * path, batches, the soft score and mhfd_detect_host allocate more.  Host
 * only.  Errors: INVALID_ARG. */
int mhfd_device_bytes(mhfd_detector *det, int32_t H, int32_t W, int64_t *fixed_bytes,
                      int64_t *image_bytes);

/* Gives back the device memory a detector grew for the images it has seen:
 * waits for its work to finish, then frees the per-image scratch (tile
 * counters, candidate staging, prune grid, plain-path planes, the device
 * copy of host images, soft-score planes) and any captured batch graph,
 * keeping what mhfd_create_detector allocated (mhfd_device_bytes' fixed
 * bytes).  The next detection grows the scratch again.  Results already
 * read stay valid; a detection enqueued but not yet waited for cannot be
 * read after this call.  Errors: INVALID_ARG, CUDA. */
int mhfd_trim(mhfd_detector *det);

/* Tile configurations the fused kernel can be specialised with for the
 * ladder of `p` (autotuner menu): returns their count; if `desc` is not NULL
 * writes up to `cap` rows of six int32 (strip width and tile height, both
 * including the one-pixel NMS border, rows per step, threads per block,
 * level groups, horizontal item kind).
 * Row k is selected by params.tile_override = k + 1.  Host only. */
int mhfd_tile_configs(const mhfd_params *p, int32_t *desc, int32_t cap);

/* The configuration mhfd_create_detector would use for `p` (same six
 * fields as above).  Host only. */
int mhfd_chosen_tile(const mhfd_params *p, int32_t *desc6);

/* Compiles the fused kernel for the ladder and tile of `p` (store = 0: the
 * detection kernel of params.nms; 1: the stack-storing variant of
 * mhfd_debug_stack; 2: the soft-score forward of mhfd_soft_score; 3: the
 * single-level blurs of its adjoint) into the on-disk kernel cache
 * without using a GPU, so that a later mhfd_create_detector starts at once.
 * The cache directory is $MHFD_JIT_CACHE, else `_jit_cache` next to the
 * library.  Errors: INVALID_ARG, UNSUPPORTED, JIT. */
int mhfd_precompile(const mhfd_params *p, int32_t store);

/* Kernel timing of the last mhfd_detect / mhfd_detect_plain on `det` (waits
 * for it): writes the device time in milliseconds of the fused kernel (or of
 * the plain path's blur/DoG/NMS kernels) and of the whole detection, measured
 * with CUDA events recorded on the launching stream.  Needs params.timing. */
int mhfd_last_timing(mhfd_detector *det, float *ms_detect_kernel, float *ms_total);

/* Measures the FP32 FFMA issue peak of the current device with a register-
 * only probe kernel: returns FFMA lane-operations per second (one FFMA = 1)
 * in *ops_per_s, timed with CUDA events on `stream`. */
int mhfd_probe_ffma_peak(void *stream, double *ops_per_s);

/* Last error message of the calling thread ("" if none). */
const char *mhfd_last_error(void);

/* Library version string. */
const char *mhfd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MHFD_H */
