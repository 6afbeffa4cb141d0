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
 * reading of that statement.
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

/* ---- Forward tracking (pixel-tracker tracks traced to a downstream tracker)
 *
 * The paper traces pixel-tracker tracks forwards: straight to the middle of
 * the magnet, where the field acts as one change of angle, then straight to
 * the fibre tracker, keeping a track when enough hits with a low enough chi2
 * are found (Sec. "HLT1 details and results").  It gives no geometry and no
 * algorithm; this is the project's reading, on an invented downstream
 * geometry (12 layers measuring (x, y), a kick plane at z_mag, a kick
 * kappa q / p to tx only), every step in binary32 in the written order.
 * Per pixel-tracker track:
 *   0. the line through its two most downstream hits a (last) and b:
 *      tx = (x_a - x_b) / (z_a - z_b), ty likewise, from (x_a, y_a, z_a);
 *   1. xm = x_a + tx (z_mag - z_a), ym = y_a + ty (z_mag - z_a);
 *   2. candidates: every hit c of the two first layers r (r = 0, 1) with
 *      |x_c - (xm + tx dz_r)| <= (kappa / p_min) dz_r + tol_x and
 *      |y_c - (ym + ty dz_r)| <= win_y, dz_r = z_r - z_mag;
 *   3. a candidate gives the slope behind the magnet t = (x_c - xm) / dz_r;
 *      in each layer L of the first station (0-3) it takes the hit nearest
 *      to xm + t dz_L in x (ties: the smaller id) with
 *      |x - (xm + t dz_L)| <= tol_x and |y - (ym + ty dz_L)| <= tol_y; with
 *      fewer than 2 such hits the candidate is dropped; the straight line
 *      through them (least squares as in 4.) then predicts the layers of the
 *      other stations, where the nearest hit within tol_x_far (and tol_y) is
 *      taken;
 *   4. a candidate with n >= min_hits hits is fitted by the straight lines
 *      x = a + b (z - z_0) and y = ay + by (z - z_0) (least squares, sums in
 *      layer order S0, Sz, Szz, Sx, Sxz, dz = z_L - z_0) with
 *      chi2 = sum (((x - a) - b dz) / sigma_x)^2 over n - 2;
 *   5. behind a single kick the lines meet the pixel-tracker line at the
 *      kick plane: d_x = (a + b (z_mag - z_0)) - xm, d_y likewise with ym,
 *      D = d_x^2 + d_y^2;
 *   6. among candidates with chi2/ndf <= chi2ndf_max and D <= tol_match^2
 *      the one with the most hits, then the smallest D, then the smallest
 *      candidate id wins; its q/p = (b - tx) / kappa.
 * Outputs per track: n (0 = none), hit ids per layer (0xFFFFFFFF = none),
 * state[VO_FWD_STATE] = q/p, chi2/ndf, b, a, d_x, d_y. */
#define VO_FWD_LAYERS 12
#define VO_FWD_STATE 6
typedef struct vo_downstream {
  float z_mag;
  float z_layers[VO_FWD_LAYERS];
  float kappa;
} vo_downstream_t;
typedef struct vo_fwd_params {
  float p_min;        /* GeV/c: smallest momentum whose kick is searched */
  float win_y;        /* mm, candidate window in y */
  float tol_x, tol_y; /* mm, hit collection windows around a candidate's prediction */
  float tol_x_far;    /* mm, in x in the stations after the first */
  float sigma_x;      /* mm, for the chi2 */
  float tol_match;    /* mm, distance of the lines at the kick plane */
  float chi2ndf_max;
  uint32_t min_hits;
} vo_fwd_params_t;
/* One event: downstream hits (layer, x, y) in any order, ids = their
 * indices; pixel-tracker tracks as hit lists (track_hit_offsets[n_tracks+1]
 * into track_hits: event-local cluster ids ascending; a track of fewer than
 * two gets no downstream track) over the event's clusters (x, y, z by id).
 * A window test holds only for a distance that is a number within its
 * tolerance, so hits with a coordinate that is not finite are never taken.
 * Writes n_found[t], hits[t * 12 + L], state[t * VO_FWD_STATE + k]. */
void vo_forward_event(uint64_t n_hits, const uint32_t* layer, const float* x, const float* y, uint64_t n_tracks,
                      const uint64_t* track_hit_offsets, const uint32_t* track_hits, const float* cluster_x,
                      const float* cluster_y, const float* cluster_z, const vo_downstream_t* geo,
                      const vo_fwd_params_t* p, uint32_t* n_found, uint32_t* hits, float* state);

#ifdef __cplusplus
}
#endif
#endif
