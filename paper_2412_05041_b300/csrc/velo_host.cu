// Host-buffer form of the C ABI (velo_context_*, velo_reconstruct_host).
//
// The events of the first stage are independent (Sec. "Data flow overview"),
// so a batch in host memory can be cut into chunks of whole events, each
// reconstructed by the plain device call: a chunk's results are those of its
// events in any batch.  The copies of one chunk then overlap with the
// kernels of the others.
//
// One buffer set of the batch's full size is cut into disjoint regions, one
// per chunk (its words, offsets, outputs and workspace), so no chunk waits
// for another's buffers and every copy in and every kernel is enqueued at
// once:
//   copy-in stream    the chunks' offsets (rebased to 0, pinned staging) and
//                     words, in order;
//   compute streams   two, alternating: chunk c waits for its words and
//                     for the clustering of chunk c - 1, runs the
//                     reconstruction and copies its totals, status,
//                     per-event offsets (and labels) out;
//   copy-out stream   the host waits for each chunk's totals in order and
//                     enqueues the copies of its clusters and tracks, at the
//                     batch-wide bases of the chunks before it; once they
//                     landed, the chunk's offsets are moved by those bases.
// Offsets that the device call would reject (not starting at 0, decreasing,
// not ending at n_pixels, an event of 2^30 words or more) are passed through
// unchanged in one chunk, so that every event fails exactly as it does there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "velo.h"

namespace {

constexpr uint32_t kMaxChunks = 64;
// automatic chunking: about this many pixel words per chunk, at most kAutoMaxChunks chunks.  On 10k
// pile-up-5.5 events (125M words, half-size first and last chunks) tracks-only results measured best
// at 10 chunks (18.7 ms against 19.0 at 6, 8 and 12, 21.2 at 16), full results (three times the
// bytes out) at 12 (25.1 ms against 25.6 at 10, 26.1 at 8 and 26.6 at 20)
constexpr uint32_t kAutoMaxChunks = 12;
constexpr uint64_t kAutoChunkWords = 12ull << 20;          // tracks only
constexpr uint64_t kAutoChunkWordsClusters = 10ull << 20;  // with cluster coordinates
// chunk k's kernels start once chunk k-1's clustering is done (stage mark 1):
// chunk k's clustering then fills the SMs that chunk k-1's tracking tail
// leaves idle, but never competes with chunk k-1's clustering, so chunks
// finish in order and their copies out start early.
constexpr int kStageMark = 1;
constexpr uint64_t kChunkSlack = 64ull << 10;      // workspace alignment slack per chunk (bytes)

struct Chunk {
  uint64_t e0 = 0, e1 = 0, p0 = 0, p1 = 0;
  uint64_t ws_off = 0;                      // byte offset of its workspace region
  uint64_t nc = 0, nt = 0, nh = 0, nf = 0;  // its totals
  uint64_t bc = 0, bt = 0, bh = 0;          // batch-wide bases of its clusters, tracks, track hits
  // disjoint regions of the buffer set: events at e0 + c (one extra offset
  // entry per chunk), words / clusters / track hits at p0, tracks at p0/3 + c
  uint64_t eo(uint32_t c) const { return e0 + c; }
  uint64_t to(uint32_t c) const { return p0 / 3 + c; }
};

bool offsets_valid(const uint64_t* off, uint64_t E, uint64_t P) {
  if (off[0] != 0 || off[E] != P) return false;
  for (uint64_t e = 0; e < E; ++e)
    if (off[e + 1] < off[e] || off[e + 1] - off[e] >= (1ull << 30)) return false;
  return true;
}

}  // namespace

struct velo_context {
  uint64_t max_events, max_pixels;
  uint64_t ws_bytes;
  uint32_t max_chunks;  // 0 = automatic
  uint64_t* d_off;      // max_events + 1 + kMaxChunks
  uint32_t* d_pix;
  velo_output_t d_out;  // regions per chunk (see Chunk)
  uint64_t* d_tot;      // 4 per chunk
  void* workspace;
  uint64_t* h_off;  // pinned staging of the rebased offsets
  uint64_t* h_tot;  // pinned: 4 per chunk
  cudaStream_t s_in, s_comp[2], s_out;
  cudaEvent_t ev_start, ev_in[kMaxChunks], ev_stage[kMaxChunks], ev_tot[kMaxChunks], ev_done[kMaxChunks];
};

extern "C" {

void velo_context_destroy(velo_context_t* c) {
  if (!c) return;
  cudaStream_t ss[] = {c->s_in, c->s_comp[0], c->s_comp[1], c->s_out};
  for (cudaStream_t s : ss)
    if (s) cudaStreamSynchronize(s);
  void* dev[] = {c->d_off,
                 c->d_pix,
                 c->d_out.status,
                 c->d_out.cluster_offsets,
                 c->d_out.cluster_x,
                 c->d_out.cluster_y,
                 c->d_out.cluster_z,
                 c->d_out.pixel_cluster,
                 c->d_out.track_offsets,
                 c->d_out.track_hit_offsets,
                 c->d_out.track_hits,
                 c->d_out.track_states,
                 c->d_out.track_features,
                 c->d_tot,
                 c->workspace};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (c->h_off) cudaFreeHost(c->h_off);
  if (c->h_tot) cudaFreeHost(c->h_tot);
  if (c->ev_start) cudaEventDestroy(c->ev_start);
  for (uint32_t k = 0; k < kMaxChunks; ++k) {
    if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
    if (c->ev_stage[k]) cudaEventDestroy(c->ev_stage[k]);
    if (c->ev_tot[k]) cudaEventDestroy(c->ev_tot[k]);
    if (c->ev_done[k]) cudaEventDestroy(c->ev_done[k]);
  }
  for (cudaStream_t s : ss)
    if (s) cudaStreamDestroy(s);
  delete c;
}

int velo_context_create(uint64_t max_events, uint64_t max_pixels, velo_context_t** ctx) {
  if (!ctx) return VELO_EINVAL;
  *ctx = nullptr;
  velo_sizes_t sz;
  if (velo_query_sizes(max_events, max_pixels, &sz) != VELO_OK) return VELO_EINVAL;
  velo_context* c = new velo_context;
  std::memset(c, 0, sizeof(*c));
  c->max_events = max_events;
  c->max_pixels = max_pixels;
  c->ws_bytes = sz.workspace_bytes + kMaxChunks * kChunkSlack;
  bool ok = true;
  auto alloc = [&](void** p, uint64_t bytes) {
    if (cudaMalloc(p, bytes ? bytes : 256) != cudaSuccess) ok = false;
  };
  const uint64_t E = max_events, EK = max_events + 1 + kMaxChunks, T = max_pixels / 3 + kMaxChunks;
  alloc((void**)&c->d_off, 8 * EK);
  alloc((void**)&c->d_pix, 4 * max_pixels);
  alloc((void**)&c->d_out.status, 4 * E);
  alloc((void**)&c->d_out.cluster_offsets, 8 * EK);
  alloc((void**)&c->d_out.cluster_x, 4 * max_pixels);
  alloc((void**)&c->d_out.cluster_y, 4 * max_pixels);
  alloc((void**)&c->d_out.cluster_z, 4 * max_pixels);
  alloc((void**)&c->d_out.pixel_cluster, 4 * max_pixels);
  alloc((void**)&c->d_out.track_offsets, 8 * EK);
  alloc((void**)&c->d_out.track_hit_offsets, 8 * (T + 1));
  alloc((void**)&c->d_out.track_hits, 4 * max_pixels);
  alloc((void**)&c->d_out.track_states, 4ull * VELO_STATE_STRIDE * T);
  alloc((void**)&c->d_out.track_features, 4ull * VELO_N_FEATURES * T);
  alloc((void**)&c->d_tot, 8 * 4 * kMaxChunks);
  alloc(&c->workspace, c->ws_bytes);
  if (cudaMallocHost((void**)&c->h_off, 8 * EK) != cudaSuccess) ok = false;
  if (cudaMallocHost((void**)&c->h_tot, 8 * 4 * kMaxChunks) != cudaSuccess) ok = false;
  if (cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking) != cudaSuccess) ok = false;
  if (cudaStreamCreateWithFlags(&c->s_comp[0], cudaStreamNonBlocking) != cudaSuccess) ok = false;
  if (cudaStreamCreateWithFlags(&c->s_comp[1], cudaStreamNonBlocking) != cudaSuccess) ok = false;
  if (cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking) != cudaSuccess) ok = false;
  if (cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) != cudaSuccess) ok = false;
  for (uint32_t k = 0; k < kMaxChunks; ++k) {
    if (cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (cudaEventCreateWithFlags(&c->ev_stage[k], cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (cudaEventCreateWithFlags(&c->ev_tot[k], cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming) != cudaSuccess) ok = false;
  }
  if (!ok) {
    velo_context_destroy(c);
    cudaGetLastError();
    return VELO_ENOMEM;
  }
  *ctx = c;
  return VELO_OK;
}

int velo_context_set_pipeline(velo_context_t* c, uint32_t max_chunks) {
  if (!c || max_chunks > kMaxChunks) return VELO_EINVAL;
  c->max_chunks = max_chunks;
  return VELO_OK;
}

int velo_reconstruct_host(velo_context_t* c, const velo_events_t* ev, const velo_geometry_t* geometry,
                          const velo_params_t* params, const velo_output_t* ho, void* stream) {
  if (!c || !ev || !ev->event_offsets || (ev->n_pixels && !ev->pixels)) return VELO_EINVAL;
  if (!ho || !ho->status || !ho->cluster_offsets || !ho->track_offsets || !ho->track_hit_offsets || !ho->track_hits ||
      !ho->track_states || !ho->totals)
    return VELO_EINVAL;
  if (ev->n_events > c->max_events || ev->n_pixels > c->max_pixels) return VELO_ECAPACITY;
  const uint64_t E = ev->n_events, P = ev->n_pixels;
  const uint64_t* off = ev->event_offsets;

  // ---- chunks of whole events (the middle ones of about equal word counts), their workspace regions
  const bool valid = offsets_valid(off, E, P);
  uint32_t K = c->max_chunks;
  if (K == 0) {
    const uint64_t per = ho->cluster_x || ho->cluster_y || ho->cluster_z ? kAutoChunkWordsClusters : kAutoChunkWords;
    K = (uint32_t)std::min<uint64_t>(kAutoMaxChunks, std::max<uint64_t>(1, (P + per - 1) / per));
  }
  if (!valid) K = 1;
  K = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(K, E));
  Chunk ch[kMaxChunks];
  for (;;) {
    uint64_t ws = 0;
    for (uint32_t k = 0; k < K; ++k) {
      Chunk& q = ch[k];
      q = Chunk();
      q.e0 = k ? ch[k - 1].e1 : 0;
      q.e1 = E;
      if (k + 1 < K) {
        // word shares 1 : 2 : ... : 2 : 1 (K >= 3): a short first chunk starts the
        // kernels early, a short last chunk leaves little to copy out at the end
        const uint64_t parts = K >= 3 ? 2ull * K - 2 : K, upto = K >= 3 ? 2ull * k + 1 : k + 1;
        const uint64_t target = (P * upto + parts - 1) / parts;
        uint64_t e1 = (uint64_t)(std::lower_bound(off, off + E + 1, target) - off);
        e1 = std::max(e1, q.e0 + 1);                   // at least one event
        q.e1 = std::min(e1, E - (uint64_t)(K - 1 - k));  // and one for every later chunk
      }
      q.p0 = valid ? off[q.e0] : 0;
      q.p1 = valid ? off[q.e1] : P;
      velo_sizes_t s;
      if (velo_query_sizes(q.e1 - q.e0, q.p1 - q.p0, &s) != VELO_OK) return VELO_EINVAL;
      q.ws_off = ws;
      ws += (s.workspace_bytes + 255ull) & ~255ull;
    }
    if (ws <= c->ws_bytes || K == 1) break;
    K = 1;  // not reached with the context's slack; one chunk always fits
  }

  // ---- everything on the device is enqueued at once, after what `stream` holds
  bool ok = cudaEventRecord(c->ev_start, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess;
  cudaStream_t all[] = {c->s_in, c->s_comp[0], c->s_comp[1], c->s_out};
  for (cudaStream_t s : all) ok &= cudaStreamWaitEvent(s, c->ev_start, 0) == cudaSuccess;
  auto d2h = [&](void* dst, const void* src, uint64_t bytes, cudaStream_t s) {
    if (bytes && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) ok = false;
  };
  auto h2d = [&](void* dst, const void* src, uint64_t bytes, cudaStream_t s) {
    if (bytes && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) ok = false;
  };
  auto region = [&](uint32_t k) {  // chunk k's outputs
    const Chunk& q = ch[k];
    velo_output_t d = c->d_out;
    d.status += q.e0;
    d.cluster_offsets += q.eo(k);
    d.cluster_x += q.p0;
    d.cluster_y += q.p0;
    d.cluster_z += q.p0;
    d.pixel_cluster = ho->pixel_cluster ? d.pixel_cluster + q.p0 : nullptr;
    d.track_offsets += q.eo(k);
    d.track_hit_offsets += q.to(k);
    d.track_hits += q.p0;
    d.track_states += VELO_STATE_STRIDE * q.to(k);
    d.track_features = ho->track_features ? d.track_features + VELO_N_FEATURES * q.to(k) : nullptr;
    d.totals = c->d_tot + 4 * k;
    d.cap_clusters = d.cap_tracks = d.cap_track_hits = 0;  // the chunk's own (velo_query_sizes) capacities
    return d;
  };

  for (uint32_t k = 0; k < K; ++k) {
    const Chunk& q = ch[k];
    const uint64_t Ec = q.e1 - q.e0;
    uint64_t* ho_off = c->h_off + q.eo(k);
    for (uint64_t i = 0; i <= Ec; ++i) ho_off[i] = valid ? off[q.e0 + i] - q.p0 : off[i];
    h2d(c->d_off + q.eo(k), ho_off, 8 * (Ec + 1), c->s_in);
    h2d(c->d_pix + q.p0, ev->pixels + q.p0, 4 * (q.p1 - q.p0), c->s_in);
    ok &= cudaEventRecord(c->ev_in[k], c->s_in) == cudaSuccess;
  }
  int rc = VELO_OK;
  for (uint32_t k = 0; k < K && rc == VELO_OK; ++k) {
    const Chunk& q = ch[k];
    const uint64_t Ec = q.e1 - q.e0, Pc = q.p1 - q.p0;
    cudaStream_t s = c->s_comp[k & 1];
    ok &= cudaStreamWaitEvent(s, c->ev_in[k], 0) == cudaSuccess;
    if (k) ok &= cudaStreamWaitEvent(s, c->ev_stage[k - 1], 0) == cudaSuccess;
    const velo_events_t dev = {Ec, Pc, c->d_off + q.eo(k), c->d_pix + q.p0};
    const velo_output_t d = region(k);
    void* marks[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    marks[kStageMark] = c->ev_stage[k];
    rc = velo_reconstruct_into_marked(&dev, geometry, params, &d, static_cast<uint8_t*>(c->workspace) + q.ws_off,
                                      c->ws_bytes - q.ws_off, s, marks);
    if (rc != VELO_OK) break;
    d2h(c->h_tot + 4 * k, d.totals, 32, s);
    d2h(ho->status + q.e0, d.status, 4 * Ec, s);
    d2h(ho->cluster_offsets + q.e0 + 1, d.cluster_offsets + 1, 8 * Ec, s);  // entry 0 is the base
    d2h(ho->track_offsets + q.e0 + 1, d.track_offsets + 1, 8 * Ec, s);
    if (ho->pixel_cluster) d2h(ho->pixel_cluster + q.p0, d.pixel_cluster, 4 * Pc, s);
    ok &= cudaEventRecord(c->ev_tot[k], s) == cudaSuccess;
  }

  // ---- the host takes the chunks' totals in order and copies their results out.
  // Capacities below the bounds of velo_query_sizes may not hold the batch:
  // then every chunk's totals are awaited first, and a batch that does not fit
  // copies no cluster and no track (as the device form writes none), only its
  // status, per-event offsets, labels and totals.
  const bool may_overflow = (ho->cap_clusters && ho->cap_clusters < P) ||
                            (ho->cap_tracks && ho->cap_tracks < P / 3) ||
                            (ho->cap_track_hits && ho->cap_track_hits < P);
  bool copy = true;
  if (may_overflow && rc == VELO_OK && ok) {
    uint64_t nc = 0, nt = 0, nh = 0;
    for (uint32_t k = 0; k < K && ok; ++k) {
      if (cudaEventSynchronize(c->ev_tot[k]) != cudaSuccess) ok = false;
      nc += c->h_tot[4 * k];
      nt += c->h_tot[4 * k + 1];
      nh += c->h_tot[4 * k + 2];
    }
    copy = (!ho->cap_clusters || nc <= ho->cap_clusters) && (!ho->cap_tracks || nt <= ho->cap_tracks) &&
           (!ho->cap_track_hits || nh <= ho->cap_track_hits);
  }
  uint64_t run_c = 0, run_t = 0, run_h = 0, run_f = 0;
  auto fixup = [&](const Chunk& q, uint32_t k) {
    if (cudaEventSynchronize(c->ev_done[k]) != cudaSuccess) {
      ok = false;
      return;
    }
    if (q.bc | q.bt)
      for (uint64_t e = q.e0 + 1; e <= q.e1; ++e) {
        ho->cluster_offsets[e] += q.bc;
        ho->track_offsets[e] += q.bt;
      }
    if (q.bh && copy)
      for (uint64_t t = q.bt + 1; t <= q.bt + q.nt; ++t) ho->track_hit_offsets[t] += q.bh;
  };
  ho->cluster_offsets[0] = 0;
  ho->track_offsets[0] = 0;
  ho->track_hit_offsets[0] = 0;
  if (rc == VELO_OK && ok) {
    for (uint32_t k = 0; k < K && ok; ++k) {
      Chunk& q = ch[k];
      if (cudaEventSynchronize(c->ev_tot[k]) != cudaSuccess) {
        ok = false;
        break;
      }
      const uint64_t* t = c->h_tot + 4 * k;
      q.nc = t[0];
      q.nt = t[1];
      q.nh = t[2];
      q.nf = t[3];
      q.bc = run_c;
      q.bt = run_t;
      q.bh = run_h;
      run_c += q.nc;
      run_t += q.nt;
      run_h += q.nh;
      run_f += q.nf;
      const velo_output_t d = region(k);
      cudaStream_t s = c->s_out;
      if (!copy) {
        ok &= cudaEventRecord(c->ev_done[k], s) == cudaSuccess;
        if (k) fixup(ch[k - 1], k - 1);
        continue;
      }
      if (ho->cluster_x) d2h(ho->cluster_x + q.bc, d.cluster_x, 4 * q.nc, s);
      if (ho->cluster_y) d2h(ho->cluster_y + q.bc, d.cluster_y, 4 * q.nc, s);
      if (ho->cluster_z) d2h(ho->cluster_z + q.bc, d.cluster_z, 4 * q.nc, s);
      d2h(ho->track_hit_offsets + q.bt + 1, d.track_hit_offsets + 1, 8 * q.nt, s);
      d2h(ho->track_hits + q.bh, d.track_hits, 4 * q.nh, s);
      d2h(ho->track_states + VELO_STATE_STRIDE * q.bt, d.track_states, 4ull * VELO_STATE_STRIDE * q.nt, s);
      if (ho->track_features)
        d2h(ho->track_features + VELO_N_FEATURES * q.bt, d.track_features, 4ull * VELO_N_FEATURES * q.nt, s);
      ok &= cudaEventRecord(c->ev_done[k], s) == cudaSuccess;
      if (k) fixup(ch[k - 1], k - 1);  // overlaps with the copies of chunk k
    }
    if (ok) fixup(ch[K - 1], K - 1);
  }
  for (cudaStream_t s : all)
    if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
  if (rc != VELO_OK) return rc;
  if (!ok) return VELO_ECUDA;
  ho->totals[0] = run_c;
  ho->totals[1] = run_t;
  ho->totals[2] = run_h;
  ho->totals[3] = run_f;
  return VELO_OK;
}

}  // extern "C"
