// Internal launch arguments and workspace layout of the VELO tracking library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "velo.h"

namespace velo {

// Block shapes (the tunable ones are chosen per call, see velo_tuning_t).
constexpr int kOutputThreads = 256;
// CTAs of the output kernel that share one heavy-ion-like event (its work
// queue holds that many parts of each listed event, then the other events)
constexpr uint32_t kOutputParts = 32;
constexpr int kScanThreads = 1024;
constexpr uint32_t kSmemPerSm = 228u * 1024u;    // shared memory of one SM
constexpr uint32_t kSmemPerBlock = 227u * 1024u; // largest dynamic allocation of one CTA

// Events of at most this many words sum their integer charges in 32 bits
// (15 * 4095 * 23552 < 2^32); larger ones use 64 bits.
constexpr uint32_t kNarrowPixels = 23552;
constexpr uint32_t kModOffStride = 33;  // per-event module offsets, n_modules + 1 <= 33
// Events with at least this many clusters (heavy-ion-like: some 2000 tracks
// and more) are tracked by clusters of CTAs (k_track_wide), listed by the
// clustering kernel in wide_list (count in queue[3]).
constexpr uint32_t kWideClusters = 20000;
// Events of at least this many pixel words (heavy-ion-like) are clustered
// module by module, one thread-block cluster of CTAs per event
// (k_cluster_wide), listed by k_validate_offsets in heavy_list.
constexpr uint32_t kHeavyWords = 1u << 16;
// The tracking kernel takes the events of at least this many clusters first
// (listed at the front of `order` by the clustering kernel, the others from
// the back), so that the last CTAs to start are small events.
constexpr uint32_t kLargeEvent = 8192;

// Per-track metadata word: n_hits (8 bits) | active (1 bit) << 8 |
// module of the last (most upstream) hit << 16 | module of the one before << 24.
constexpr uint32_t kTrkActive = 1u << 8;

// Device scratch, carved out of the caller's workspace.  Arrays marked
// "pixel-indexed" give each event the slice [event_offsets[e], +n_e); arrays
// marked "track-indexed" the slice [event_offsets[e] / 3, + n_e / 3): an
// event has at most n_e clusters and n_e / 3 tracks, so slices never overlap.
struct Workspace {
  uint32_t* flag;            // [1] offsets invalid
  uint32_t* queue;           // [8] work-queue counters of the persistent kernels; [3] wide_list count,
                             // [4] / [5] events listed at the front / back of order
  uint32_t* wide_list;       // [E] events of kWideClusters clusters or more (any order)
  uint32_t* heavy_list;      // [E] events of kHeavyWords words or more (queue[7] of them, any order)
  uint32_t* order;           // [E] events in the tracking kernel's order: kLargeEvent clusters or more first
  uint32_t* ev_nclusters;    // [E]
  uint32_t* ev_modoff;       // [E * 33] cluster-id (= sorted position) offsets per module
  uint32_t* ev_ntracks_all;  // [E] tracks built (kept or not)
  uint32_t* ev_ntracks;      // [E] tracks kept
  uint32_t* ev_nhits;        // [E] hits on kept tracks
  uint64_t* ev_hitbase;      // [E] first global position of the event's track hits
  uint32_t* sa;              // pixel-indexed u32: sort ping-pong / seed h0
  uint32_t* sb;              // pixel-indexed u32: sort ping-pong / seed h2
  uint32_t* sc;              // pixel-indexed u32: hit-sort values / prev link
  uint32_t* sd;              // pixel-indexed u32: hit-sort values / first_of
  unsigned long long* acc;   // pixel-indexed x3: centroid sums / claims, seed keys, seeding u terms
  float2* cl_xy;             // pixel-indexed: cluster (x, y) in id order (clustering -> output)
  float4* hit;               // pixel-indexed: hits sorted by (module, key, id), one 16-byte record
                             // each: x, y, pseudo-angle key, cluster id (its bits)
  uint32_t* h_pos;           // pixel-indexed: sorted position of each cluster id
  uint8_t* used;             // pixel-indexed
  uint32_t* trk_meta;        // track-indexed
  uint32_t* trk_a;           // last hit position
  uint32_t* trk_b;           // hit position before it
  uint32_t* trk_pick;        // extension candidate of this step
  unsigned long long* trk_pick_key;
  uint32_t* trk_rank;        // canonical rank among kept tracks, kNone if dropped
  uint32_t* trk_hoff;        // first hit of the track among the event's kept hits
  float* trk_logit;          // the network's logit (learned rejection)
  float* trk_state;          // VELO_STATE_STRIDE floats per track: the fit's state, written by k_fit
  uint32_t* lb_flag;         // [E] look-back record state of the fused fit: 0 none, 1 aggregate, 2 prefix
  unsigned long long* lb_val;// [E * 8] the event's counts (clusters, kept tracks, hits, failed), then
                             // the inclusive prefix of those counts over the events up to it
};

struct Geo {
  uint32_t n_modules, n_rows, n_cols;
  float pitch, x0, y0;
  float z[VELO_MAX_MODULES];
};

struct Par {
  float win_seed, win_fwd, max_slope, max_scatter_seed, max_scatter_fwd;
  uint32_t max_skipped;
  float sigma, ms_theta, chi2ndf_max, chi2ndf_max_3hit;
  uint32_t use_mlp;
  float mlp_logit_min;
  const float* mlp;
};

struct Launch {
  uint64_t n_events, n_pixels;
  uint32_t cluster_tier;  // words per event kept in shared memory by the clustering kernel
  uint32_t union_link_attempts;  // bound of each union's link attempts (velo_tuning_t)
  const uint64_t* off;
  const uint32_t* pix;
  Geo geo;
  Par par;
  Workspace ws;
  velo_output_t out;
};

// byte size of the workspace for E events and P pixels
uint64_t workspace_bytes(uint64_t E, uint64_t P);
// carve a workspace; returns false if too small
bool carve_workspace(void* base, uint64_t bytes, uint64_t E, uint64_t P, Workspace* ws);

// kernels and their launchers (persistent grids; velo_capi.cu sizes them)
__global__ void k_validate_offsets(Launch L);
__global__ void k_scan(Launch L);
int launch_cluster(const Launch& L, int nt, uint32_t grid, cudaStream_t s);  // k_cluster, then k_cluster_wide
int launch_track(const Launch& L, int nt, uint32_t grid, uint32_t wide_cluster, cudaStream_t s);
int launch_fit(const Launch& L, bool fused, cudaStream_t s);  // k_fit_out, or k_fit (k_scan and k_output follow)
int launch_output(const Launch& L, uint32_t grid, cudaStream_t s);
uint32_t cluster_smem_bytes(int nt, uint32_t tier);
uint32_t cluster_max_tier(int nt);
uint32_t cluster_wide_tier();  // the shared-memory tier of the heavy-event clustering
int cluster_blocks_per_sm(int nt, uint32_t tier);
int track_blocks_per_sm(int nt);
int output_blocks_per_sm(bool features);

// host helpers (velo_capi.cu): raise a kernel's dynamic shared-memory limit
// once per device (slot = a small id per kernel instance; occupancy with
// slot < 0 leaves the limit alone), resident CTAs per SM
bool set_max_smem_once(const void* func, int slot, uint32_t bytes = kSmemPerBlock);
int occupancy(const void* func, int threads, uint32_t smem, int slot);
int device_sm_count();  // SMs of the current device (148 if it cannot be read)
bool allow_large_clusters_once(const void* func, int slot);  // thread-block clusters of up to 16 CTAs

}  // namespace velo
