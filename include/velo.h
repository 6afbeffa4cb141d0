/* velo.h -- C ABI of the B300 (sm_103a) event-batched VELO-like pixel tracking library.
 *
 * What it computes.  The paper's first trigger stage reconstructs every
 * collision event on GPUs at the full input rate (Sec. "Introduction",
 * Sec. "Data flow overview"), with a simplified pattern recognition and a
 * parameterised Kalman filter applied only to the pixel-tracker (VELO)
 * segment of each track (Sec. "HLT1 details and results").  The paper gives
 * no algorithm; this library implements one concrete definition of it:
 *   pixel words -> 8-connected clusters per module (hits)
 *   -> search by triplet seeding + forward extension across modules
 *   -> straight-line least-squares fit + simplified Kalman filter
 *   -> chi2/ndf cut -> tracks in canonical order.
 * Every floating-point decision is binary32 with one rounding per operation
 * in a fixed order and no fused multiply-add, so results are reproducible
 * bit for bit on any IEEE-754 machine that runs the same steps.
 *
 * Conventions.
 *   - All functions return VELO_OK (0) or a positive VELO_E* code; no function
 *     aborts, traps or prints.  velo_strerror() names a code.
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     "host" pointers are ordinary (preferably pinned) host memory.
 *   - Every buffer is caller-owned unless a function says it allocates.
 *   - Asynchronous functions enqueue work on the given cudaStream_t (passed
 *     as void*; NULL = the legacy default stream) and return without waiting;
 *     results are valid once the stream has reached that point.
 *   - The library keeps no global state and never synchronises a stream it
 *     was not asked to (the *_host entry points synchronise their own
 *     stream before returning).
 */
#ifndef VELO_H
#define VELO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VELO_STATE_STRIDE 20          /* floats per track state, layout below */
#define VELO_N_FEATURES 12            /* candidate features (learned ghost rejection) */
#define VELO_MLP_HIDDEN 32
#define VELO_MLP_WEIGHTS 1505         /* trainable: W1[32][12] b1[32] W2[32][32] b2[32] W3[32] b3 */
#define VELO_MLP_FLOATS 1529          /* model blob: mean[12] inv_std[12] + the weights */
#define VELO_MAX_MODULES 32u          /* geometry limit (5-bit module field) */
#define VELO_MAX_MODULE_CLUSTERS 65535u /* per module per event; beyond it the event fails */

/* Return codes. */
enum {
  VELO_OK = 0,
  VELO_EINVAL = 1,     /* bad argument: NULL where a pointer is required, bad geometry or params */
  VELO_ECAPACITY = 2,  /* a caller buffer or workspace is smaller than velo_query_sizes asked for */
  VELO_ECUDA = 3,      /* a CUDA runtime call failed (the CUDA error is not cleared) */
  /* 4 is not used: a bounded device-side loop that gives up fails its event
     (VELO_EVT_TIMEOUT), not the call */
  VELO_ENOMEM = 5      /* a library allocation failed (only the allocating entry points) */
};

/* Per-event status codes written to velo_output_t.status. */
enum {
  VELO_EVT_OK = 0,
  VELO_EVT_BADWORD = 1,  /* a pixel word has bit 31 set, q = 0, or module/row/col outside the geometry */
  VELO_EVT_OVERFLOW = 2, /* a module has more than VELO_MAX_MODULE_CLUSTERS clusters */
  VELO_EVT_TIMEOUT = 3   /* the clustering's lock-free union-find gave up after its bounded link
                            attempts (velo_tuning_t.union_link_attempts; not expected at the default) */
};
/* A failed event contributes no cluster and no track; the other events are unaffected. */

/* Detector geometry: planar pixel modules perpendicular to the beam (z). */
typedef struct velo_geometry {
  uint32_t n_modules;     /* 3 .. VELO_MAX_MODULES */
  const float* module_z;  /* host [n_modules], strictly ascending, mm */
  float pitch_mm;         /* square pixel pitch */
  uint32_t n_rows, n_cols;/* pixel grid per module, each <= 2048 */
  float x0_mm, y0_mm;     /* lower edge of the grid: pixel (row, col) spans
                             x in [x0 + pitch*col, x0 + pitch*(col+1)) */
} velo_geometry_t;

/* Reconstruction parameters (velo_params_default fills the standard values). */
typedef struct velo_params {
  float win_seed;          /* pseudo-angle half window for seeding, in [0, 1] (full turn = 4) */
  float win_fwd;           /* pseudo-angle half window for extension, in [0, 1] */
  float max_slope;         /* seeds need |tx|, |ty| <= max_slope */
  float max_scatter_seed;  /* mm^2: squared 2D distance of the middle hit to the outer-hit line */
  float max_scatter_fwd;   /* mm^2: squared 2D distance of a hit to the extrapolated track */
  uint32_t max_skipped;    /* modules a track may miss in a row before it terminates */
  float sigma_meas;        /* mm, hit resolution used by both fits */
  float ms_theta;          /* rad per module; 0 -> the cut uses the straight-line chi2,
                              > 0 -> the Kalman chi2 with slope noise ms_theta^2 per module */
  float chi2ndf_max;       /* keep a track if chi2/ndf <= chi2ndf_max */
  float chi2ndf_max_3hit;  /* ... and a 3-hit track only if also <= chi2ndf_max_3hit */
  /* Learned ghost rejection (the paper has no learned component; this is the
   * project's extension): when use_mlp is 1 a 12 -> 32 -> 32 -> 1 network
   * scores every candidate on bfloat16 tensor cores (float32 accumulation) and
   * "logit >= mlp_logit_min" replaces the 3-hit rule; chi2ndf_max still applies.
   * mlp: device pointer to a VELO_MLP_FLOATS float32 blob
   * (mean[12], inv_std[12], W1[32][12], b1[32], W2[32][32], b2[32], W3[32], b3). */
  uint32_t use_mlp;
  float mlp_logit_min;
  const float* mlp;
} velo_params_t;

/* A batch of events in CSR form.  Pixel word layout (any order inside an event):
 *   bit 31 = 0 | q (4 bits, 1..15) << 27 | module (5) << 22 | row (11) << 11 | col (11) */
typedef struct velo_events {
  uint64_t n_events;
  uint64_t n_pixels;              /* == event_offsets[n_events] */
  const uint64_t* event_offsets;  /* [n_events + 1], event_offsets[0] == 0, non-decreasing */
  const uint32_t* pixels;         /* [n_pixels] */
} velo_events_t;

/* Output buffers (all caller-owned; capacities from velo_query_sizes).
 * Cluster ids are event-local: the rank of a cluster in the event when the
 * clusters are ordered by (module, smallest row*2048+col of their pixels).
 * Tracks of an event are ordered by their smallest cluster id; a track's hit
 * list holds its cluster ids ascending (= upstream to downstream).
 * Track state layout (VELO_STATE_STRIDE floats per track):
 *   0 x, 1 y, 2 tx, 3 ty   straight-line least squares, at the first hit's z
 *   4 z_first              z of the first (most upstream) hit
 *   5 z_beam               z of the fitted line's closest approach to the z axis
 *   6 chi2_lsq, 7 chi2_kf  straight-line chi2 and Kalman chi2 (sum of r^2/S)
 *   8 kf_x, 9 kf_y, 10 kf_tx, 11 kf_ty   Kalman state at the first hit
 *  12 C_xx, 13 C_xtx, 14 C_txtx          Kalman covariance, x projection
 *  15 C_yy, 16 C_yty, 17 C_tyty          Kalman covariance, y projection
 *  18 ndf = 2 n_hits - 4, 19 the network's logit when use_mlp, else 0
 * Candidate features (VELO_N_FEATURES floats per track, optional output):
 *   n_hits, chi2/ndf (of the cut), tx, ty, z_first, z_last, modules skipped,
 *   mean and RMS of the x residuals, mean and RMS of the y residuals,
 *   largest |residual| (residuals of the straight-line fit, mm). */
typedef struct velo_output {
  int32_t* status;              /* [n_events] VELO_EVT_* */
  uint64_t* cluster_offsets;    /* [n_events + 1] into cluster_x/y/z */
  float* cluster_x;             /* [cap_clusters] mm */
  float* cluster_y;             /* [cap_clusters] mm */
  float* cluster_z;             /* [cap_clusters] mm */
  uint32_t* pixel_cluster;      /* optional (NULL = not written) [n_pixels]: event-local cluster id
                                   of every input word, 0xFFFFFFFF in failed events */
  uint64_t* track_offsets;      /* [n_events + 1] into the track arrays */
  uint64_t* track_hit_offsets;  /* [cap_tracks + 1] into track_hits (global positions) */
  uint32_t* track_hits;         /* [cap_track_hits] event-local cluster ids */
  float* track_states;          /* [cap_tracks * VELO_STATE_STRIDE] */
  uint64_t* totals;             /* [4]: n_clusters, n_tracks, n_track_hits, n_failed_events */
  float* track_features;        /* optional (NULL = not written) [cap_tracks * VELO_N_FEATURES] */
  /* Capacities of the arrays above (0 = the bounds velo_query_sizes gives,
   * which always suffice).  A batch whose totals exceed a capacity writes no
   * cluster and no track: the caller sees totals[0..2] above its capacities
   * and retries with larger buffers or a smaller batch. */
  uint64_t cap_clusters, cap_tracks, cap_track_hits;
} velo_output_t;

/* Capacities that always suffice for a batch of n_events events holding
 * n_pixels pixel words, and the device workspace velo_reconstruct_into needs. */
typedef struct velo_sizes {
  uint64_t cap_clusters;     /* = n_pixels (a cluster has >= 1 pixel) */
  uint64_t cap_tracks;       /* = n_pixels / 3 (disjoint tracks of >= 3 hits) */
  uint64_t cap_track_hits;   /* = n_pixels */
  uint64_t workspace_bytes;  /* device scratch, 256-byte aligned start required */
} velo_sizes_t;

/* Fill *p with the standard parameters (win 0.04, slope 0.3, scatter 0.01 /
 * 0.02 mm^2, 1 skipped module, sigma 0.0159 mm, 0.5 mrad, cuts 10 and 2).
 * Passage: Sec. "HLT1 details and results" names the pattern recognition,
 * the parameterised Kalman filter and the track-quality cut these values
 * steer; the paper prints none of the values (they are this library's,
 * tuned on simulated events).  VELO_EINVAL for a NULL p. */
int velo_params_default(velo_params_t* p);

/* Sizes for a batch (host arithmetic only; no device call). */
int velo_query_sizes(uint64_t n_events, uint64_t n_pixels, velo_sizes_t* out);

/* Reconstruct a device-resident batch into caller-owned device buffers.
 * Passage: Sec. "HLT1 details and results" (simplified pattern recognition
 * and a parameterised Kalman filter on the pixel-tracker segment of each
 * track) for what is computed; Sec. "Data flow overview" (every event
 * reconstructed, events independent) for the batching.
 * events->event_offsets/pixels and every output pointer are device pointers;
 * geometry->module_z is a host pointer (copied into the launch arguments).
 * workspace: device, >= sizes.workspace_bytes, 256-byte aligned, contents
 * ignored on entry and undefined on exit.  Allocates nothing and never
 * synchronises: everything runs on `stream` (a cudaStream_t).  Offsets that
 * are not monotone or do not end at n_pixels are detected on the device and
 * make every event fail with VELO_EVT_BADWORD. */
int velo_reconstruct_into(const velo_events_t* events, const velo_geometry_t* geometry,
                          const velo_params_t* params, const velo_output_t* out, void* workspace,
                          uint64_t workspace_bytes, void* stream);

/* velo_reconstruct_into plus timing marks: stage_events holds 5 cudaEvent_t
 * handles created by the caller (cast to void*), recorded on `stream` before
 * the clustering kernel, after it, after the pattern-recognition kernels,
 * after the fit kernel (which in the fused form, velo_tuning_t.fused_output,
 * also writes the offsets and the output) and after the offsets-scan and
 * output kernels (none in the fused form).  NULL records nothing.  The marks
 * add no work and no synchronisation. */
int velo_reconstruct_into_marked(const velo_events_t* events, const velo_geometry_t* geometry,
                                 const velo_params_t* params, const velo_output_t* out, void* workspace,
                                 uint64_t workspace_bytes, void* stream, void* const* stage_events);

/* Block shapes of the persistent kernels (events of any size are spread over
 * the SMs by work queues; these choose how).  Any valid setting gives the same
 * results bit for bit; speed depends on the workload (autotuned by the Python
 * layer).  velo_tuning_default: 1024 / largest tier / 256 / all resident / 0 /
 * 0 / 2^20; start from it (a zeroed struct is rejected with VELO_EINVAL). */
typedef struct velo_tuning {
  uint32_t cluster_threads;      /* 512 (two CTAs per SM) or 1024 (one) */
  uint32_t cluster_smem_pixels;  /* words per event sorted in shared memory, 0 = the most that fits;
                                    larger events run on their global-memory slice */
  uint32_t track_threads;        /* 128 or 256 */
  uint32_t ctas_per_sm;          /* grid of the clustering and output kernels: 0 = every CTA that fits,
                                    persistent; k = at most k per SM, persistent; VELO_CTAS_PER_EVENT =
                                    one CTA per event, scheduled by the hardware as CTAs finish (the
                                    tracking kernel always runs one CTA per event) */
  uint32_t wide_cluster;         /* CTAs (a thread-block cluster of 1024-thread CTAs) tracking each event of
                                    20000 clusters or more: 0 = the largest the device can place (16, else
                                    8), or 8 or 16 (VELO_EINVAL if the device cannot place it) */
  uint32_t fused_output;         /* 1 = the fit kernel also writes the event offsets (decoupled
                                    look-back) and the compact output, one launch instead of three,
                                    when no capacity can be exceeded and no features are asked for;
                                    0 = separate fit, offsets-scan and output kernels (faster on
                                    pile-up-5.5 batches) */
  uint32_t union_link_attempts;  /* most link attempts of one union in the clustering's lock-free
                                    union-find before it gives up and its event fails with
                                    VELO_EVT_TIMEOUT (an attempt retries only after losing a race to
                                    another union, so the default 2^20 is never reached); 0 = a
                                    union that still has to link two trees gives up at once (a test
                                    setting: it fails exactly the events that need such a union) */
} velo_tuning_t;
#define VELO_CTAS_PER_EVENT 0xFFFFFFFFu
int velo_tuning_default(velo_tuning_t* t);
/* velo_reconstruct_into_marked with explicit block shapes (NULL = defaults). */
int velo_reconstruct_into_tuned(const velo_events_t* events, const velo_geometry_t* geometry,
                                const velo_params_t* params, const velo_output_t* out, void* workspace,
                                uint64_t workspace_bytes, void* stream, void* const* stage_events,
                                const velo_tuning_t* tuning);

/* The same with library-owned results (the form of the call that returns
 * "tracks"; passage as velo_reconstruct_into): allocates the output buffers and the workspace on `stream`
 * with cudaMallocAsync and returns an opaque handle in *result.  The handle
 * is valid immediately; its contents once `stream` reaches this point. */
typedef struct velo_result velo_result_t;
typedef struct velo_result_view {
  uint64_t n_events, n_pixels;
  uint64_t cap_clusters, cap_tracks, cap_track_hits;
  velo_output_t out;  /* device pointers owned by the result */
} velo_result_view_t;
int velo_reconstruct(const velo_events_t* events, const velo_geometry_t* geometry,
                     const velo_params_t* params, velo_result_t** result, void* stream);
/* The device pointers and capacities of a result (the tracks and clusters of
 * Sec. "HLT1 details and results" in the velo_output_t layout above), owned
 * by the result: valid until velo_result_free.  VELO_EINVAL for NULL. */
int velo_result_view(const velo_result_t* result, velo_result_view_t* view);
/* Frees the result's buffers on its stream (stream-ordered; no host wait).
 * NULL is ignored.  No counterpart in the paper (memory ownership only). */
void velo_result_free(velo_result_t* result);

/* Host-buffer form, for callers whose events sit in host memory: a context
 * owns device buffers for up to max_events / max_pixels and its own streams
 * (allocated once, by velo_context_create).  velo_reconstruct_host
 * reconstructs a batch whose inputs and results live in HOST memory
 * (results in caller-owned buffers of the capacities from velo_query_sizes,
 * laid out exactly as velo_reconstruct_into's).  It cuts the batch into
 * chunks of whole events, each reconstructed by velo_reconstruct_into in
 * its own region of the context's buffers, so that the copies of one chunk
 * overlap with the kernels of the others; the events are independent
 * (Sec. "Data flow overview"), so the results do not depend on the
 * chunking.  The chunks' offsets are moved to batch-wide values on the
 * host.  Work starts after what `stream` holds at the call; the call
 * returns once every result is in the host buffers.  Page-locked host
 * buffers are needed for the overlap (pageable ones work, with the copies
 * serialised).  Only the used part of each output is copied back; cluster_x,
 * cluster_y and cluster_z may be NULL (the clusters are still found and
 * tracked, their coordinates are not copied back: tracks-only results).  Offsets
 * that the device form rejects are passed to it unchanged, in one chunk, so
 * every event then fails as there.  The capacities in host_out behave as in
 * velo_reconstruct_into: a batch whose totals exceed one copies no cluster
 * and no track (status, per-event offsets, pixel labels and totals are
 * still written), so nothing is written past a capacity; capacities below
 * velo_query_sizes' bounds make the call wait for every chunk's totals
 * before it copies results out (less overlap).  velo_context_set_pipeline
 * sets the most chunks per call: 0 = automatic (about 10.5M pixel words per
 * chunk when cluster coordinates are copied back, about 12.6M for
 * tracks-only results, at most 12 chunks), 1 = one chunk (copy in, compute,
 * copy out, no overlap), at most 64; VELO_EINVAL otherwise. */
typedef struct velo_context velo_context_t;
int velo_context_create(uint64_t max_events, uint64_t max_pixels, velo_context_t** ctx);
void velo_context_destroy(velo_context_t* ctx);
int velo_context_set_pipeline(velo_context_t* ctx, uint32_t max_chunks);
int velo_reconstruct_host(velo_context_t* ctx, const velo_events_t* host_events,
                          const velo_geometry_t* geometry, const velo_params_t* params,
                          const velo_output_t* host_out, void* stream);

/* Allocation-free form, for callers that cannot allocate device memory
 * while they reconstruct: a trigger node whose device memory is fixed at
 * start-up, or code running inside another framework's callbacks, where a
 * cudaMalloc could block or re-enter that framework's allocator.  The paper
 * has no counterpart of this entry point.
 * Same as velo_reconstruct_into, but the scratch is a file-scope __device__
 * array of VELO_STATIC_SCRATCH_BYTES inside the library (every device that
 * loads the library holds it until the process exits); the caller passes
 * device inputs and outputs exactly as for velo_reconstruct_into.  A batch
 * whose scratch need (velo_query_sizes' workspace_bytes) exceeds
 * VELO_STATIC_SCRATCH_BYTES -- about 620k pixel words, some 50 pile-up-5.5
 * events -- is rejected with VELO_ECAPACITY before any device work.  Calls
 * no cudaMalloc, cudaFree or allocating routine.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, that device
 * current): make that first call before any stream capture.  Every call
 * shares the one array, which keeps the previous call's contents (nothing
 * needs clearing: the kernels initialise what they read); calls that overlap
 * on the GPU race on it. */
#define VELO_STATIC_SCRATCH_BYTES (64ull << 20)
int velo_reconstruct_static(const velo_events_t* events, const velo_geometry_t* geometry,
                            const velo_params_t* params, const velo_output_t* out, void* stream);

/* ---- Training and evaluation of the ghost-rejection network (device pointers,
 * asynchronous on `stream`).  Inputs x are normalised features
 * ((f - mean) * inv_std) [n * 12], labels y in {0, 1} [n]; weights w are the
 * VELO_MLP_WEIGHTS trainable floats in blob order.  Gradients are summed over
 * the batch in a fixed order (deterministic). */

/* Logits of n feature vectors (raw features [n * 12], the model blob):
 * mode 0 = the reconstruction's bfloat16 tensor-core path, mode 1 = float32
 * on CUDA cores (no bfloat16 rounding). */
int velo_mlp_infer(const float* features, uint64_t n, const float* mlp, float* logits, int mode, void* stream);
/* Device scratch velo_mlp_loss_grad needs for a batch of n samples. */
int velo_mlp_workspace_size(uint64_t n, uint64_t* bytes);
/* Mean binary cross-entropy of sigmoid(logit) (float32, written to *loss) and
 * its gradient with respect to w (grad[VELO_MLP_WEIGHTS]). */
int velo_mlp_loss_grad(const float* x, const float* y, uint64_t n, const float* w, float* grad, float* loss,
                       void* workspace, uint64_t workspace_bytes, void* stream);
/* One Adam step on w with moments m, v (all [n_weights]); step counts from 1. */
int velo_mlp_adam_step(float* w, const float* grad, float* m, float* v, uint32_t n_weights, float lr, float beta1,
                       float beta2, float eps, uint32_t step, void* stream);

/* ---- Forward tracking: pixel-tracker tracks traced to a downstream tracker
 *
 * The first stage traces pixel-tracker tracks forwards: straight to the
 * middle of the magnet, where the field is taken as one change of angle, then
 * straight to the fibre tracker, keeping a track when enough hits with a low
 * enough chi2 are found (Sec. "HLT1 details and results").  The paper gives
 * neither the geometry nor the algorithm; this library reads it on a
 * downstream tracker of VELO_FWD_LAYERS planar layers measuring (x, y) and a
 * kick plane at z_mag (kick kappa q / p to tx, none to ty), every step in
 * binary32 in a fixed order (the CPU oracle defines the same steps):
 *   0. the track's line through its two most downstream clusters a, b:
 *      tx = (x_a - x_b) / (z_a - z_b), ty likewise;
 *   1. xm = x_a + tx (z_mag - z_a), ym likewise: the line at the kick plane;
 *   2. candidates: hits c of layers 0 and 1 with
 *      |x_c - (xm + tx dz)| <= (kappa / p_min) dz + tol_x, |y_c - (ym + ty dz)|
 *      <= win_y, dz = z_layer - z_mag;
 *   3. slope t = (x_c - xm) / dz; in layers 0-3 the nearest hit in x to
 *      xm + t dz_L (ties: smaller id) within tol_x (and tol_y in y); at least
 *      2 of them, whose least-squares line predicts layers 4-11 (nearest hit
 *      within tol_x_far);
 *   4. n >= min_hits: least-squares lines x = a + b (z - z_layer0),
 *      y = ay + by (z - z_layer0), chi2 = sum (((x - a) - b dz) / sigma_x)^2;
 *   5. match at the kick plane d_x = a + b (z_mag - z_layer0) - xm, d_y
 *      likewise, D = d_x^2 + d_y^2;
 *   6. among candidates with chi2 / (n - 2) <= chi2ndf_max and
 *      D <= tol_match^2: most hits, then smallest D, then smallest candidate
 *      id; q/p = (b - tx) / kappa.
 * Tracks are searched independently (a hit may serve several tracks). */
#define VELO_FWD_LAYERS 12u
#define VELO_FWD_STATE 6u /* q/p, chi2/ndf, b (slope behind the magnet), a (x at layer 0), d_x, d_y */

typedef struct velo_downstream {
  float z_mag;                    /* mm */
  float z_layers[VELO_FWD_LAYERS];/* mm, ascending; layers 0-3 form the first station */
  float kappa;                    /* GeV/c * rad: kick = kappa * q / p */
} velo_downstream_t;

typedef struct velo_forward_params {
  float p_min;        /* GeV/c: smallest momentum whose kick is searched */
  float win_y;        /* mm: candidate window in y */
  float tol_x, tol_y; /* mm: hit windows around a candidate's prediction */
  float tol_x_far;    /* mm: in x in layers 4-11 */
  float sigma_x;      /* mm: for the chi2 */
  float tol_match;    /* mm: distance of the lines at the kick plane */
  float chi2ndf_max;
  uint32_t min_hits;
} velo_forward_params_t;

/* Downstream hits in CSR form, DEVICE pointers: hits of event e at
 * [event_offsets[e], event_offsets[e+1]) in any order; a hit's id is its
 * index inside its event.  Hits with layer >= VELO_FWD_LAYERS, or an x
 * or y that is not finite, are never taken (a window test holds only for a
 * distance that is a number within the tolerance). */
typedef struct velo_downstream_hits {
  uint64_t n_events;
  uint64_t n_hits;
  const uint64_t* event_offsets; /* [n_events + 1] */
  const uint32_t* layer;         /* [n_hits] */
  const float* x;                /* [n_hits] mm */
  const float* y;                /* [n_hits] mm */
} velo_downstream_hits_t;

/* Per pixel-tracker track (the batch-global track index of the result),
 * DEVICE pointers, capacity cap_tracks (tracks beyond it are not written). */
typedef struct velo_forward_output {
  uint32_t* n_found;  /* [cap_tracks] hits found, 0 = no downstream track */
  uint32_t* hits;     /* [cap_tracks * VELO_FWD_LAYERS] event-local hit ids, 0xFFFFFFFF = none */
  float* state;       /* [cap_tracks * VELO_FWD_STATE] */
  uint64_t cap_tracks;
} velo_forward_output_t;

int velo_forward_params_default(velo_forward_params_t* params);
/* Device scratch velo_forward needs for a batch of n_events / n_hits. */
int velo_forward_workspace_size(uint64_t n_events, uint64_t n_hits, uint64_t* bytes);
/* Forward tracking of the tracks of a reconstruction result `tracks` (the
 * device outputs of velo_reconstruct_into on the same events, in order;
 * cluster_offsets, cluster_x/y/z, track_offsets, track_hit_offsets,
 * track_hits and totals are read), on `stream`, asynchronously.  Workspace:
 * 256-byte aligned, >= velo_forward_workspace_size.  VELO_EINVAL for a NULL
 * or inconsistent argument (a parameter or z that is not finite, z_layers not
 * ascending behind z_mag, min_hits outside [3, 12], a non-positive p_min,
 * sigma_x or kappa), VELO_ECAPACITY for a small workspace.  Event offsets
 * that do not start at 0, decrease, end past n_hits or give an event 2^29
 * hits or more leave every track without a downstream track (n 0, no hits, state
 * 0); a track of fewer than two hits never has one; a result whose totals
 * exceed its capacities (no track lists written) makes velo_forward write
 * nothing. */
int velo_forward(const velo_downstream_hits_t* hits, const velo_output_t* tracks, const velo_downstream_t* geometry,
                 const velo_forward_params_t* params, const velo_forward_output_t* out, void* workspace,
                 uint64_t workspace_bytes, void* stream);

/* Measurement helper, not part of the method: the FP32 multiply-add rate of
 * the current device (flops/s, 2 per FMA), from a kernel of independent FMA
 * chains on every SM timed with CUDA events on `stream` (best of three
 * launches after one warm-up; synchronises `stream`).  The reconstruction
 * has no dense contraction, so this plain-ALU ceiling is its second
 * roofline after HBM bandwidth.  VELO_EINVAL for a NULL output, VELO_ECUDA
 * if a CUDA call fails. */
int velo_measure_fp32_peak(double* flops_per_s, void* stream);

/* Name of a VELO_* return code (a static string; unknown codes get a generic
 * name, never NULL).  No counterpart in the paper (error reporting only). */
const char* velo_strerror(int code);

/* Library version (major * 10000 + minor * 100 + patch). */
int velo_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VELO_H */
