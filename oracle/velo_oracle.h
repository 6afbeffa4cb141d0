/* CPU oracle for event-batched VELO-like pixel tracking -- TEST INFRASTRUCTURE.
 *
 * This library defines the result that the CUDA path must reproduce.  It is
 * plain, slow and written to be checked by eye against the method's
 * definition; it shares no code, header, helper or constant with the CUDA
 * library.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it.
 *
 * The paper states the problem only in words: the first trigger stage
 * reconstructs every collision event on GPUs (Sec. "Introduction"), with a
 * simplified pattern recognition and a parameterised Kalman filter applied
 * to the pixel-tracker segment of a track only (Sec. "HLT1 details and
 * results").  It gives no algorithm, so the steps below are this project's
 * reading of that statement; every reading is listed with the algorithm
 * definition in the design notes.
 *
 * Arithmetic contract: IEEE-754 binary32 for every floating-point quantity
 * that decides anything, one rounding per + - * / in the written order, no
 * fused multiply-add (built with -ffp-contract=off), no transcendental
 * function.  The double-precision entry points exist only for pins.
 */
#ifndef VELO_ORACLE_H
#define VELO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VO_STATE_STRIDE 20
#define VO_N_FEATURES 12
/* Ghost-rejection network blob (float32): mean[12], inv_std[12], W1[32][12],
 * b1[32], W2[32][32], b2[32], W3[32], b3 -- 1529 floats. */
#define VO_MLP_HIDDEN 32
#define VO_MLP_FLOATS 1529
#define VO_MAX_MODULE_CLUSTERS 65535u
#define VO_MAX_MODULES 32u

enum { VO_EVT_OK = 0, VO_EVT_BADWORD = 1, VO_EVT_OVERFLOW = 2 };

typedef struct vo_geometry {
  uint32_t n_modules;     /* <= 32 */
  const float* module_z;  /* host [n_modules], strictly ascending */
  float pitch_mm;
  uint32_t n_rows, n_cols;
  float x0_mm, y0_mm;     /* lower edge of the pixel grid */
} vo_geometry_t;

typedef struct vo_params {
  float win_seed;          /* pseudo-angle half window, seeding */
  float win_fwd;           /* pseudo-angle half window, extension */
  float max_slope;         /* |tx|, |ty| bound for a seed */
  float max_scatter_seed;  /* mm^2 */
  float max_scatter_fwd;   /* mm^2 */
  uint32_t max_skipped;    /* consecutive modules a track may miss */
  float sigma_meas;        /* mm */
  float ms_theta;          /* rad; 0 -> the cut uses the straight-line chi2 */
  float chi2ndf_max;
  float chi2ndf_max_3hit;
  uint32_t use_mlp;        /* 1: the network's logit >= mlp_logit_min replaces the 3-hit rule */
  float mlp_logit_min;
  const float* mlp;        /* host, VO_MLP_FLOATS, used when use_mlp */
} vo_params_t;

/* Pseudo-angle ("diamond angle") in [0, 4), monotone in phi. */
float vo_pseudo_angle(float x, float y);

/* Clustering of one event.  words[n] in any order.  Writes up to n clusters
 * (x, y, z in cluster-id order), the module of every cluster, and the
 * cluster id of every input word.  Returns a VO_EVT_* status; on failure no
 * cluster is written, *n_clusters = 0 and pixel_cluster[] = 0xFFFFFFFF. */
int vo_cluster_event(const uint32_t* words, uint64_t n, const vo_geometry_t* geo, float* cx, float* cy,
                     float* cz, uint32_t* cmodule, uint32_t* pixel_cluster, uint64_t* n_clusters);

/* Pattern recognition + fit + cut on one event's hits, given in cluster-id
 * order (module[] ascending).  Tracks are returned in canonical order in
 * caller buffers of capacity cap_tracks (tracks) and n_hits (hit ids):
 * hit_offsets[n_tracks+1], hit ids ascending within each track, states
 * [n_tracks * VO_STATE_STRIDE].  Returns 0, or -1 if a buffer is too small. */
int vo_track_event(uint64_t n_hits, const uint32_t* module, const float* x, const float* y,
                   const vo_geometry_t* geo, const vo_params_t* p, uint64_t cap_tracks,
                   uint64_t* n_tracks, uint64_t* hit_offsets, uint32_t* hit_ids, float* states);

/* Straight-line least squares and simplified Kalman filter of one track
 * (hits in ascending z).  state[VO_STATE_STRIDE] as documented in the .cpp. */
void vo_fit_f32(uint32_t n, const float* x, const float* y, const float* z, float sigma, float ms_theta,
                float* state);
void vo_fit_f64(uint32_t n, const double* x, const double* y, const double* z, double sigma,
                double ms_theta, double* state);

/* The 12 candidate features of one track (hits ascending in z, their module
 * indices, the fitted state from vo_fit_f32, the cut's chi2/ndf): n_hits,
 * chi2/ndf, tx, ty, z_first, z_last, modules skipped, mean and RMS of the x
 * residuals, mean and RMS of the y residuals, largest |residual|. */
void vo_features(uint32_t n, const float* x, const float* y, const float* z, const uint32_t* module,
                 const float* state, float chi2ndf, float* features);
/* The network's logit for one feature vector: inputs, weights and the first
 * hidden layer rounded to bfloat16 (round to nearest even), sums in float32
 * in index order, bias added after the sum, ReLU; the second hidden layer stays
 * float32; logit = sum_j W3[j] h2[j] (j ascending) + b3. */
float vo_mlp_logit(const float* mlp, const float* features);

/* Whole batch (the oracle form of velo_reconstruct): events in CSR form on
 * the host.  Returns an opaque handle; read it with vo_batch_sizes and
 * vo_batch_copy, release with vo_batch_free.  n_threads <= 0: all cores. */
void* vo_reconstruct(uint64_t n_events, const uint64_t* event_offsets, const uint32_t* pixels,
                     const vo_geometry_t* geo, const vo_params_t* p, int n_threads);
void vo_batch_sizes(void* h, uint64_t* n_clusters, uint64_t* n_tracks, uint64_t* n_track_hits);
/* Any pointer may be NULL.  status[E], cluster_offsets[E+1], cluster_x/y/z[C],
 * pixel_cluster[P], track_offsets[E+1], track_hit_offsets[T+1] (global),
 * track_hits[H] (event-local cluster ids), track_states[T*20] (state[19] = the
 * network's logit when use_mlp, else 0), track_features[T*12]. */
void vo_batch_copy(void* h, int32_t* status, uint64_t* cluster_offsets, float* cx, float* cy, float* cz,
                   uint32_t* pixel_cluster, uint64_t* track_offsets, uint64_t* track_hit_offsets,
                   uint32_t* track_hits, float* track_states, float* track_features);
void vo_batch_free(void* h);

#ifdef __cplusplus
}
#endif
#endif
