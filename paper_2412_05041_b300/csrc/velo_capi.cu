// Host side of the C ABI declared in include/velo.h: argument validation,
// workspace layout, the launch sequence, and the allocating conveniences.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "velo_internal.cuh"

namespace velo {

namespace {

struct Carver {
  uint8_t* base;
  uint64_t off = 0;
  template <class T>
  T* take(uint64_t count) {
    off = (off + 255ull) & ~255ull;
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

void carve(Carver& c, uint64_t E, uint64_t P, Workspace* ws) {
  const uint64_t T = P / 3 + 1;
  ws->flag = c.take<uint32_t>(4);
  ws->queue = c.take<uint32_t>(8);
  ws->wide_list = c.take<uint32_t>(E);
  ws->heavy_list = c.take<uint32_t>(E);
  ws->order = c.take<uint32_t>(E);
  ws->ev_nclusters = c.take<uint32_t>(E);
  ws->ev_modoff = c.take<uint32_t>(E * kModOffStride);
  ws->ev_ntracks_all = c.take<uint32_t>(E);
  ws->ev_ntracks = c.take<uint32_t>(E);
  ws->ev_nhits = c.take<uint32_t>(E);
  ws->ev_hitbase = c.take<uint64_t>(E);
  ws->sa = c.take<uint32_t>(P);
  ws->sb = c.take<uint32_t>(P);
  ws->sc = c.take<uint32_t>(P);
  ws->sd = c.take<uint32_t>(P);
  ws->acc = c.take<unsigned long long>(3 * P);
  ws->cl_xy = c.take<float2>(P);
  ws->hit = c.take<float4>(P);
  ws->h_pos = c.take<uint32_t>(P);
  ws->used = c.take<uint8_t>(P);
  ws->trk_meta = c.take<uint32_t>(T);
  ws->trk_a = c.take<uint32_t>(T);
  ws->trk_b = c.take<uint32_t>(T);
  ws->trk_pick = c.take<uint32_t>(T);
  ws->trk_pick_key = c.take<unsigned long long>(T);
  ws->trk_rank = c.take<uint32_t>(T);
  ws->trk_hoff = c.take<uint32_t>(T);
  ws->trk_logit = c.take<float>(T);
  ws->trk_state = c.take<float>(T * VELO_STATE_STRIDE);
  ws->lb_flag = c.take<uint32_t>(E);
  ws->lb_val = c.take<unsigned long long>(8 * E);
}

bool geometry_ok(const velo_geometry_t* g) {
  if (!g || !g->module_z) return false;
  if (g->n_modules < 3 || g->n_modules > VELO_MAX_MODULES) return false;
  if (g->n_rows < 1 || g->n_rows > 2048 || g->n_cols < 1 || g->n_cols > 2048) return false;
  if (!(g->pitch_mm > 0.0f) || !std::isfinite(g->pitch_mm) || !std::isfinite(g->x0_mm) || !std::isfinite(g->y0_mm))
    return false;
  for (uint32_t m = 0; m < g->n_modules; ++m) {
    if (!std::isfinite(g->module_z[m])) return false;
    if (m && !(g->module_z[m] > g->module_z[m - 1])) return false;
  }
  return true;
}

bool params_ok(const velo_params_t* p) {
  if (!p) return false;
  auto fin = [](float v) { return std::isfinite(v); };
  if (!fin(p->win_seed) || p->win_seed < 0.0f || p->win_seed > 1.0f) return false;
  if (!fin(p->win_fwd) || p->win_fwd < 0.0f || p->win_fwd > 1.0f) return false;
  if (!fin(p->max_slope) || p->max_slope < 0.0f) return false;
  if (!fin(p->max_scatter_seed) || p->max_scatter_seed < 0.0f) return false;
  if (!fin(p->max_scatter_fwd) || p->max_scatter_fwd < 0.0f) return false;
  if (p->max_skipped >= VELO_MAX_MODULES) return false;
  if (!fin(p->sigma_meas) || !(p->sigma_meas > 0.0f)) return false;
  if (!fin(p->ms_theta) || p->ms_theta < 0.0f) return false;
  if (!fin(p->chi2ndf_max) || !fin(p->chi2ndf_max_3hit)) return false;
  if (p->use_mlp > 1 || (p->use_mlp && (!p->mlp || !fin(p->mlp_logit_min)))) return false;
  return true;
}

bool output_ok(const velo_output_t* o) {
  return o && o->status && o->cluster_offsets && o->cluster_x && o->cluster_y && o->cluster_z && o->track_offsets &&
         o->track_hit_offsets && o->track_hits && o->track_states && o->totals;
}

Geo make_geo(const velo_geometry_t* g) {
  Geo G;
  std::memset(&G, 0, sizeof(G));
  G.n_modules = g->n_modules;
  G.n_rows = g->n_rows;
  G.n_cols = g->n_cols;
  G.pitch = g->pitch_mm;
  G.x0 = g->x0_mm;
  G.y0 = g->y0_mm;
  for (uint32_t m = 0; m < g->n_modules; ++m) G.z[m] = g->module_z[m];
  return G;
}

Par make_par(const velo_params_t* p) {
  Par P;
  P.win_seed = p->win_seed;
  P.win_fwd = p->win_fwd;
  P.max_slope = p->max_slope;
  P.max_scatter_seed = p->max_scatter_seed;
  P.max_scatter_fwd = p->max_scatter_fwd;
  P.max_skipped = p->max_skipped;
  P.sigma = p->sigma_meas;
  P.ms_theta = p->ms_theta;
  P.chi2ndf_max = p->chi2ndf_max;
  P.chi2ndf_max_3hit = p->chi2ndf_max_3hit;
  P.use_mlp = p->use_mlp;
  P.mlp_logit_min = p->mlp_logit_min;
  P.mlp = p->mlp;
  return P;
}

constexpr int kMaxDev = 64;
std::mutex g_mu;
uint32_t g_smem_set[kMaxDev] = {};  // bit per kernel slot: dynamic shared-memory limit raised
uint32_t g_cluster_set[kMaxDev] = {};  // bit per kernel slot: clusters above 8 CTAs allowed
struct OccKey {
  int dev;
  const void* func;
  uint32_t smem;
  int occ;
};
OccKey g_occ[256];
int g_nocc = 0;
int g_sms[kMaxDev] = {};

int current_device() {
  int d = 0;
  return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}

int sm_count() {
  const int d = current_device();
  if (d < 0 || d >= kMaxDev) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_sms[d]) cudaDeviceGetAttribute(&g_sms[d], cudaDevAttrMultiProcessorCount, d);
  return g_sms[d];
}

}  // namespace

int device_sm_count() {
  const int n = sm_count();
  return n > 0 ? n : 148;
}

bool set_max_smem_once(const void* func, int slot, uint32_t bytes) {
  const int d = current_device();
  if (d < 0 || d >= kMaxDev) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_smem_set[d] & (1u << slot)) return true;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();  // do not leave the failure as the sticky last error
    return false;
  }
  g_smem_set[d] |= 1u << slot;
  return true;
}

bool allow_large_clusters_once(const void* func, int slot) {
  const int d = current_device();
  if (d < 0 || d >= kMaxDev) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_cluster_set[d] & (1u << slot)) return true;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  g_cluster_set[d] |= 1u << slot;
  return true;
}

int occupancy(const void* func, int threads, uint32_t smem, int slot) {
  const int d = current_device();
  if (d < 0 || d >= kMaxDev) return 0;
  if (slot >= 0 && !set_max_smem_once(func, slot)) return 0;  // slot < 0: static shared memory only
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < g_nocc; ++i)
    if (g_occ[i].dev == d && g_occ[i].func == func && g_occ[i].smem == smem) return g_occ[i].occ;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, func, threads, smem) != cudaSuccess) occ = 0;
  if (g_nocc < 256) g_occ[g_nocc++] = {d, func, smem, occ};
  return occ;
}

uint64_t workspace_bytes(uint64_t E, uint64_t P) {
  Carver c{nullptr};
  Workspace ws;
  carve(c, E, P, &ws);
  return (c.off + 255ull) & ~255ull;
}

bool carve_workspace(void* base, uint64_t bytes, uint64_t E, uint64_t P, Workspace* ws) {
  if (workspace_bytes(E, P) > bytes) return false;
  Carver c{reinterpret_cast<uint8_t*>(base)};
  carve(c, E, P, ws);
  return true;
}

}  // namespace velo

using namespace velo;

struct velo_result {
  uint64_t n_events, n_pixels;
  velo_sizes_t sizes;
  velo_output_t out;
  void* workspace;
  cudaStream_t stream;
};

extern "C" {

int velo_version(void) { return 100; }

const char* velo_strerror(int code) {
  switch (code) {
    case VELO_OK: return "ok";
    case VELO_EINVAL: return "invalid argument";
    case VELO_ECAPACITY: return "buffer or workspace too small";
    case VELO_ECUDA: return "CUDA runtime error";
    case VELO_ENOMEM: return "allocation failed";
    default: return "unknown error";
  }
}

int velo_params_default(velo_params_t* p) {
  if (!p) return VELO_EINVAL;
  p->win_seed = 0.04f;
  p->win_fwd = 0.04f;
  p->max_slope = 0.3f;
  p->max_scatter_seed = 0.01f;
  p->max_scatter_fwd = 0.02f;
  p->max_skipped = 1;
  p->sigma_meas = 0.0159f;
  p->ms_theta = 5e-4f;
  p->chi2ndf_max = 10.0f;
  p->chi2ndf_max_3hit = 2.0f;
  p->use_mlp = 0;
  p->mlp_logit_min = 0.0f;
  p->mlp = nullptr;
  return VELO_OK;
}

int velo_query_sizes(uint64_t n_events, uint64_t n_pixels, velo_sizes_t* out) {
  if (!out || n_events >= (1ull << 31) || n_pixels >= (1ull << 40)) return VELO_EINVAL;
  out->cap_clusters = n_pixels;
  out->cap_tracks = n_pixels / 3;
  out->cap_track_hits = n_pixels;
  out->workspace_bytes = workspace_bytes(n_events, n_pixels);
  return VELO_OK;
}

int velo_reconstruct_into(const velo_events_t* events, const velo_geometry_t* geometry, const velo_params_t* params,
                          const velo_output_t* out, void* workspace, uint64_t workspace_bytes_, void* stream) {
  return velo_reconstruct_into_marked(events, geometry, params, out, workspace, workspace_bytes_, stream, nullptr);
}

int velo_reconstruct_into_marked(const velo_events_t* events, const velo_geometry_t* geometry,
                                 const velo_params_t* params, const velo_output_t* out, void* workspace,
                                 uint64_t workspace_bytes_, void* stream, void* const* marks) {
  return velo_reconstruct_into_tuned(events, geometry, params, out, workspace, workspace_bytes_, stream, marks,
                                     nullptr);
}

int velo_tuning_default(velo_tuning_t* t) {
  if (!t) return VELO_EINVAL;
  t->cluster_threads = 1024;
  t->cluster_smem_pixels = 0;
  t->track_threads = 256;
  t->ctas_per_sm = 0;
  t->wide_cluster = 0;
  t->fused_output = 0;
  t->union_link_attempts = 1u << 20;
  return VELO_OK;
}

int velo_reconstruct_into_tuned(const velo_events_t* events, const velo_geometry_t* geometry,
                                const velo_params_t* params, const velo_output_t* out, void* workspace,
                                uint64_t workspace_bytes_, void* stream, void* const* marks,
                                const velo_tuning_t* tuning) {
  if (!events || !events->event_offsets || (events->n_pixels && !events->pixels)) return VELO_EINVAL;
  if (events->n_events >= (1ull << 31) || events->n_pixels >= (1ull << 40)) return VELO_EINVAL;
  if (!geometry_ok(geometry) || !params_ok(params) || !output_ok(out)) return VELO_EINVAL;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return VELO_EINVAL;
  velo_tuning_t tu;
  velo_tuning_default(&tu);
  if (tuning) tu = *tuning;
  if ((tu.cluster_threads != 512 && tu.cluster_threads != 1024) ||
      (tu.track_threads != 128 && tu.track_threads != 256) ||
      (tu.wide_cluster != 0 && tu.wide_cluster != 8 && tu.wide_cluster != 16) || tu.fused_output > 1u)
    return VELO_EINVAL;
  const uint32_t max_tier = cluster_max_tier((int)tu.cluster_threads);
  const uint32_t tier = tu.cluster_smem_pixels ? tu.cluster_smem_pixels : max_tier;
  if (tier > max_tier || tier < 256) return VELO_EINVAL;
  Launch L;
  std::memset(&L, 0, sizeof(L));
  L.n_events = events->n_events;
  L.n_pixels = events->n_pixels;
  L.off = events->event_offsets;
  L.pix = events->pixels;
  L.geo = make_geo(geometry);
  L.par = make_par(params);
  L.out = *out;
  L.cluster_tier = tier;
  L.union_link_attempts = tu.union_link_attempts;
  if (!carve_workspace(workspace, workspace_bytes_, L.n_events, L.n_pixels, &L.ws)) return VELO_ECAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t E = L.n_events;
  const int sms = sm_count();
  if (sms <= 0) return VELO_ECUDA;
  // persistent grid, never more CTAs than work items (`items`: the events,
  // unless stated)
  auto grid = [&](int per_sm, uint64_t items = 0) -> uint32_t {
    if (tu.ctas_per_sm == VELO_CTAS_PER_EVENT) return (uint32_t)E;  // one CTA per event, hardware-scheduled
    if (tu.ctas_per_sm) per_sm = per_sm > 0 ? (int)std::min<uint32_t>((uint32_t)per_sm, tu.ctas_per_sm) : 0;
    const uint64_t g = (uint64_t)(per_sm > 0 ? per_sm : 1) * (uint64_t)sms;
    return (uint32_t)std::min<uint64_t>(g, items ? items : E);
  };
  auto mark = [&](int i) {
    if (marks && marks[i]) cudaEventRecord(reinterpret_cast<cudaEvent_t>(marks[i]), s);
  };
  k_validate_offsets<<<1, kScanThreads, 0, s>>>(L);
  mark(0);
  int rc = VELO_OK;
  if (E) rc = launch_cluster(L, (int)tu.cluster_threads, grid(cluster_blocks_per_sm((int)tu.cluster_threads, tier)), s);
  if (rc != VELO_OK) return rc;
  mark(1);
  if (E) rc = launch_track(L, (int)tu.track_threads, (uint32_t)E, tu.wide_cluster, s);  // one CTA per event
  if (rc != VELO_OK) return rc;
  mark(2);
  // In the fused form the fit writes the compact output itself (offsets by
  // a decoupled look-back), unless the candidate features are asked for or
  // the output could exceed a capacity the caller set (then nothing may be
  // written, so the totals must be known first: the separate scan and output
  // kernels).
  const uint64_t P = L.n_pixels;
  const bool fits_always = (!out->cap_clusters || out->cap_clusters >= P) &&
                           (!out->cap_tracks || out->cap_tracks >= P / 3) &&
                           (!out->cap_track_hits || out->cap_track_hits >= P);
  const bool fused = tu.fused_output && E && !out->track_features && fits_always;
  if (E) rc = launch_fit(L, fused, s);
  if (rc != VELO_OK) return rc;
  mark(3);
  if (!fused) {
    k_scan<<<1, kScanThreads, 0, s>>>(L);
    // (up to kOutputParts work items per event: parts of heavy-ion-like events)
    if (E) rc = launch_output(L, grid(output_blocks_per_sm(L.out.track_features != nullptr), E * kOutputParts), s);
    if (rc != VELO_OK) return rc;
  }
  mark(4);
  return cudaGetLastError() == cudaSuccess ? VELO_OK : VELO_ECUDA;
}

int velo_reconstruct(const velo_events_t* events, const velo_geometry_t* geometry, const velo_params_t* params,
                     velo_result_t** result, void* stream) {
  if (!result || !events) return VELO_EINVAL;
  *result = nullptr;
  velo_sizes_t sz;
  if (velo_query_sizes(events->n_events, events->n_pixels, &sz) != VELO_OK) return VELO_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  velo_result* r = new velo_result;
  std::memset(r, 0, sizeof(*r));
  r->n_events = events->n_events;
  r->n_pixels = events->n_pixels;
  r->sizes = sz;
  r->stream = s;
  const uint64_t E = events->n_events;
  bool ok = true;
  auto alloc = [&](void** p, uint64_t bytes) {
    if (cudaMallocAsync(p, bytes ? bytes : 256, s) != cudaSuccess) ok = false;
  };
  alloc((void**)&r->out.status, 4 * E);
  alloc((void**)&r->out.cluster_offsets, 8 * (E + 1));
  alloc((void**)&r->out.cluster_x, 4 * sz.cap_clusters);
  alloc((void**)&r->out.cluster_y, 4 * sz.cap_clusters);
  alloc((void**)&r->out.cluster_z, 4 * sz.cap_clusters);
  alloc((void**)&r->out.pixel_cluster, 4 * events->n_pixels);
  alloc((void**)&r->out.track_offsets, 8 * (E + 1));
  alloc((void**)&r->out.track_hit_offsets, 8 * (sz.cap_tracks + 1));
  alloc((void**)&r->out.track_hits, 4 * sz.cap_track_hits);
  alloc((void**)&r->out.track_states, 4ull * VELO_STATE_STRIDE * (sz.cap_tracks ? sz.cap_tracks : 1));
  alloc((void**)&r->out.totals, 8 * 4);
  alloc(&r->workspace, sz.workspace_bytes);
  if (!ok) {
    velo_result_free(r);
    cudaGetLastError();
    return VELO_ENOMEM;
  }
  const int rc = velo_reconstruct_into(events, geometry, params, &r->out, r->workspace, sz.workspace_bytes, stream);
  if (rc != VELO_OK) {
    velo_result_free(r);
    return rc;
  }
  *result = r;
  return VELO_OK;
}

int velo_result_view(const velo_result_t* r, velo_result_view_t* v) {
  if (!r || !v) return VELO_EINVAL;
  v->n_events = r->n_events;
  v->n_pixels = r->n_pixels;
  v->cap_clusters = r->sizes.cap_clusters;
  v->cap_tracks = r->sizes.cap_tracks;
  v->cap_track_hits = r->sizes.cap_track_hits;
  v->out = r->out;
  return VELO_OK;
}

void velo_result_free(velo_result_t* r) {
  if (!r) return;
  void* ptrs[] = {r->out.status,    r->out.cluster_offsets, r->out.cluster_x,         r->out.cluster_y,
                  r->out.cluster_z, r->out.pixel_cluster,   r->out.track_offsets,     r->out.track_hit_offsets,
                  r->out.track_hits, r->out.track_states,   r->out.totals,            r->workspace};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, r->stream);
  delete r;
}


}  // extern "C"
