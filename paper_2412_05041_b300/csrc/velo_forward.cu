// Forward tracking: pixel-tracker tracks traced through one magnet kick to
// the downstream layers (velo_forward; the steps are stated in velo.h).
//
// The first stage traces pixel-tracker tracks forwards, straight to the
// middle of the magnet, one change of angle there, straight to the fibre
// tracker (Sec. "HLT1 details and results").  One CTA per event:
//   1. the event's downstream hits are sorted by (layer, x) -- four stable
//      radix passes over the order-preserving bits of x, one over the layer
//      -- and gathered into sorted x, y arrays with per-layer offsets;
//   2. every thread takes tracks of the event: the line through the track's
//      two most downstream clusters, the candidates of layers 0 and 1, the
//      hits each candidate collects (bisection of a layer's sorted x for a
//      superset of the window, then the exact binary32 tests), the fits and
//      the choice of the best candidate.
// All arithmetic is binary32 in the order the oracle uses (-fmad=false and
// the __f*_rn intrinsics); every choice is a minimum under a strict total
// order, so the search order does not matter.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "velo_device.cuh"
#include "velo_fit.cuh"
#include "velo_internal.cuh"

namespace velo {

namespace {

constexpr int kFwdThreads = 256;
constexpr uint32_t kFwdL = VELO_FWD_LAYERS;

// x range [xp - tol - m, xp + tol + m] bisected in a layer's sorted x: m =
// 0.05 mm + 10^-6 (|xp| + tol) is more than ten times the rounding of the
// bounds and of the exact test |x - xp| <= tol, so the range holds every hit
// the exact test (which decides) accepts
__device__ __forceinline__ void fwd_range(float xp, float tol, float* lo, float* hi) {
  const float m = fa(fm(fa(fabsf(xp), tol), 1e-6f), 0.05f);
  *lo = fs(fs(xp, tol), m);
  *hi = fa(fa(xp, tol), m);
}

struct FwdWork {
  uint32_t* flag;            // kFwdBadOffsets | kFwdNoTracks
  uint32_t *ka, *kb;         // sort keys (ordered x bits) and their ping-pong copy
  uint32_t *va, *vb;         // hit ids
  float *sx, *sy;            // x, y in sorted order
};

struct Fwd {
  velo_downstream_hits_t h;
  velo_output_t t;
  velo_downstream_t g;
  velo_forward_params_t p;
  velo_forward_output_t o;
  FwdWork w;
};

uint64_t fwd_carve(uint8_t* base, uint64_t n_hits, FwdWork* w) {
  uint64_t off = 0;
  auto take = [&](uint64_t bytes) -> uint8_t* {
    off = (off + 255ull) & ~255ull;
    uint8_t* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const uint64_t H = n_hits ? n_hits : 1;
  w->flag = reinterpret_cast<uint32_t*>(take(4));
  w->ka = reinterpret_cast<uint32_t*>(take(4 * H));
  w->kb = reinterpret_cast<uint32_t*>(take(4 * H));
  w->va = reinterpret_cast<uint32_t*>(take(4 * H));
  w->vb = reinterpret_cast<uint32_t*>(take(4 * H));
  w->sx = reinterpret_cast<float*>(take(4 * H));
  w->sy = reinterpret_cast<float*>(take(4 * H));
  return (off + 255ull) & ~255ull;
}

__device__ __forceinline__ uint32_t ordered_bits(float v) {  // monotone in v
  const uint32_t u = __float_as_uint(v);
  return u ^ ((u >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}

// flag bits: the hit offsets are invalid / the pixel-tracker result did not
// fit its buffers (its track lists were not written)
constexpr uint32_t kFwdBadOffsets = 1u, kFwdNoTracks = 2u;

// One CTA: the event offsets start at 0, never decrease, end at n_hits and
// give no event 2^31 hits or more; the pixel-tracker totals fit its capacities.
__global__ void __launch_bounds__(1024) k_fwd_validate(Fwd F) {
  const uint64_t E = F.h.n_events;
  int bad = 0;
  if (threadIdx.x == 0) bad |= (F.h.event_offsets[0] != 0ull) | (F.h.event_offsets[E] != F.h.n_hits);
  for (uint64_t e = threadIdx.x; e < E; e += blockDim.x) {
    const uint64_t a = F.h.event_offsets[e], b = F.h.event_offsets[e + 1];
    bad |= (b < a) | (b - a >= (1ull << 31));
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    const velo_output_t& o = F.t;
    const bool fits = (!o.cap_clusters || o.totals[0] <= o.cap_clusters) && (!o.cap_tracks || o.totals[1] <= o.cap_tracks) &&
                      (!o.cap_track_hits || o.totals[2] <= o.cap_track_hits);
    *F.w.flag = (bad ? kFwdBadOffsets : 0u) | (fits ? 0u : kFwdNoTracks);
  }
}

// sort bucket of a hit: its layer, or kFwdL (never searched) for a layer
// number >= kFwdL or an x that is not finite
__device__ __forceinline__ uint32_t fwd_bucket(const uint32_t* lay, const float* x, uint32_t id) {
  return isfinite(x[id]) ? min(lay[id], kFwdL) : kFwdL;
}

struct FwdSmem {
  uint32_t cnt[radix_counters(kFwdThreads)];
  uint32_t tmp[64];
  uint32_t loff[kFwdL + 1];  // first sorted position of each layer; [kFwdL] = end of the valid layers
  float zl[kFwdL];
};

// The hits of one layer sorted by x: positions [lo, hi) of sx.
struct LayerView {
  const float* sx;
  const float* sy;
  const uint32_t* id;
  uint32_t lo, hi;
};

// nearest hit in x to xp (ties: the smaller id) with |x - xp| <= tol and
// |y - yp| <= tol_y; returns its sorted position or kNone
__device__ __forceinline__ uint32_t fwd_nearest(const LayerView& V, float xp, float yp, float tol, float tol_y) {
  float lo_x, hi_x;
  fwd_range(xp, tol, &lo_x, &hi_x);
  uint32_t pos = lower_bound_by(V.lo, V.hi, [&](uint32_t i) { return V.sx[i] < lo_x; });
  uint32_t best = kNone, best_id = 0;
  float bd = 0.0f;
  for (; pos < V.hi && V.sx[pos] <= hi_x; ++pos) {
    const float d = fabsf(fs(V.sx[pos], xp));
    if (!(d <= tol) || !(fabsf(fs(V.sy[pos], yp)) <= tol_y)) continue;
    const uint32_t id = V.id[pos];
    if (best == kNone || d < bd || (d == bd && id < best_id)) {
      best = pos;
      best_id = id;
      bd = d;
    }
  }
  return best;
}

// least-squares line v = a + b (z - z_0) through the found hits of layers [l0, l1)
__device__ __forceinline__ void fwd_line(const uint32_t* hl, const float* v, const float* zl, int l0, int l1, float* a,
                                         float* b) {
  float S0 = 0.0f, Sz = 0.0f, Szz = 0.0f, Sx = 0.0f, Sxz = 0.0f;
  for (int L = l0; L < l1; ++L) {
    if (hl[L] == kNone) continue;
    const float dz = fs(zl[L], zl[0]);
    const float xv = v[hl[L]];
    S0 = fa(S0, 1.0f);
    Sz = fa(Sz, dz);
    Szz = fa(Szz, fm(dz, dz));
    Sx = fa(Sx, xv);
    Sxz = fa(Sxz, fm(xv, dz));
  }
  const float det = fs(fm(S0, Szz), fm(Sz, Sz));
  const float bb = fd(fs(fm(S0, Sxz), fm(Sz, Sx)), det);
  *b = bb;
  *a = fd(fs(Sx, fm(bb, Sz)), S0);
}

__device__ void fwd_track(const Fwd& F, const FwdSmem& S, uint64_t e, uint64_t tg, uint64_t h0) {
  const velo_forward_params_t& P = F.p;
  const float zmag = F.g.z_mag, kappa = F.g.kappa;
  const float* zl = S.zl;
  // 0. the line through the two most downstream clusters (ids ascend with z)
  const uint64_t c0 = F.t.cluster_offsets[e];
  const uint64_t he = F.t.track_hit_offsets[tg + 1];
  if (he < F.t.track_hit_offsets[tg] + 2) {  // fewer than two hits: no line, no downstream track
    F.o.n_found[tg] = 0u;
    for (int L = 0; L < (int)kFwdL; ++L) F.o.hits[tg * kFwdL + L] = kNone;
    for (int k = 0; k < (int)VELO_FWD_STATE; ++k) F.o.state[tg * VELO_FWD_STATE + k] = 0.0f;
    return;
  }
  const uint64_t ha = c0 + F.t.track_hits[he - 1], hb = c0 + F.t.track_hits[he - 2];
  const float x0 = F.t.cluster_x[ha], y0 = F.t.cluster_y[ha], z0 = F.t.cluster_z[ha];
  const float dzab = fs(z0, F.t.cluster_z[hb]);
  const float tx = fd(fs(x0, F.t.cluster_x[hb]), dzab), ty = fd(fs(y0, F.t.cluster_y[hb]), dzab);
  // 1. the line at the kick plane
  const float dzm = fs(zmag, z0);
  const float xm = fa(x0, fm(tx, dzm)), ym = fa(y0, fm(ty, dzm));
  const float tm2 = fm(P.tol_match, P.tol_match);
  const float* sx = F.w.sx + h0;
  const float* sy = F.w.sy + h0;
  const uint32_t* sid = F.w.vb + h0;
  auto layer = [&](int L) { return LayerView{sx, sy, sid, S.loff[L], S.loff[L + 1]}; };

  bool have = false;
  uint32_t b_n = 0, b_c = 0;
  float b_r = 0.0f, b_b = 0.0f, b_a = 0.0f, b_d = 0.0f, b_dy = 0.0f, b_ad = 0.0f;
  uint32_t b_hits[kFwdL];
  for (int r = 0; r < 2; ++r) {
    // 2. candidates in layers 0 and 1
    const float dzr = fs(zl[r], zmag);
    const float xr = fa(xm, fm(tx, dzr)), yr = fa(ym, fm(ty, dzr));
    const float wx = fa(fm(fd(kappa, P.p_min), dzr), P.tol_x);
    const LayerView R = layer(r);
    float lo_x, hi_x;
    fwd_range(xr, wx, &lo_x, &hi_x);
    for (uint32_t pc = lower_bound_by(R.lo, R.hi, [&](uint32_t i) { return sx[i] < lo_x; }); pc < R.hi && sx[pc] <= hi_x;
         ++pc) {
      const float xc = sx[pc];
      if (!(fabsf(fs(xc, xr)) <= wx) || !(fabsf(fs(sy[pc], yr)) <= P.win_y)) continue;
      const uint32_t c = sid[pc];
      // 3. the first station from the kick line, the others from the line through it
      const float tk = fd(fs(xc, xm), dzr);
      uint32_t hl[kFwdL];
      uint32_t n1 = 0;
      for (int L = 0; L < 4; ++L) {
        const float dzl = fs(zl[L], zmag);
        hl[L] = fwd_nearest(layer(L), fa(xm, fm(tk, dzl)), fa(ym, fm(ty, dzl)), P.tol_x, P.tol_y);
        n1 += hl[L] != kNone ? 1u : 0u;
      }
      if (n1 < 2) continue;
      float a1, b1;
      fwd_line(hl, sx, zl, 0, 4, &a1, &b1);
      uint32_t n = n1;
      for (int L = 4; L < (int)kFwdL; ++L) {
        const float dzl = fs(zl[L], zmag);
        hl[L] = fwd_nearest(layer(L), fa(a1, fm(b1, fs(zl[L], zl[0]))), fa(ym, fm(ty, dzl)), P.tol_x_far, P.tol_y);
        n += hl[L] != kNone ? 1u : 0u;
      }
      if (n < P.min_hits) continue;
      // 4. the lines through all of them and the chi2 in x
      float a, b;
      fwd_line(hl, sx, zl, 0, kFwdL, &a, &b);
      float chi2 = 0.0f;
      for (int L = 0; L < (int)kFwdL; ++L) {
        if (hl[L] == kNone) continue;
        const float res = fd(fs(fs(sx[hl[L]], a), fm(b, fs(zl[L], zl[0]))), P.sigma_x);
        chi2 = fa(chi2, fm(res, res));
      }
      const float rchi = fd(chi2, (float)(n - 2));
      if (!(rchi <= P.chi2ndf_max)) continue;
      // 5. the match at the kick plane
      const float d = fs(fa(a, fm(b, fs(zmag, zl[0]))), xm);
      float ya, yb;
      fwd_line(hl, sy, zl, 0, kFwdL, &ya, &yb);
      const float dy = fs(fa(ya, fm(yb, fs(zmag, zl[0]))), ym);
      const float ad = fa(fm(d, d), fm(dy, dy));
      if (!(ad <= tm2)) continue;
      // 6. most hits, then the smallest distance, then the smallest candidate id
      const bool better = !have || n > b_n || (n == b_n && (ad < b_ad || (ad == b_ad && c < b_c)));
      if (!better) continue;
      have = true;
      b_n = n;
      b_c = c;
      b_r = rchi;
      b_b = b;
      b_a = a;
      b_d = d;
      b_dy = dy;
      b_ad = ad;
      for (int L = 0; L < (int)kFwdL; ++L) b_hits[L] = hl[L] != kNone ? sid[hl[L]] : kNone;
    }
  }
  F.o.n_found[tg] = have ? b_n : 0u;
  for (int L = 0; L < (int)kFwdL; ++L) F.o.hits[tg * kFwdL + L] = have ? b_hits[L] : kNone;
  float* so = F.o.state + tg * VELO_FWD_STATE;
  so[0] = have ? fd(fs(b_b, tx), kappa) : 0.0f;
  so[1] = have ? b_r : 0.0f;
  so[2] = have ? b_b : 0.0f;
  so[3] = have ? b_a : 0.0f;
  so[4] = have ? b_d : 0.0f;
  so[5] = have ? b_dy : 0.0f;
}

__global__ void __launch_bounds__(kFwdThreads) k_forward(Fwd F) {
  __shared__ FwdSmem S;
  const uint64_t e = blockIdx.x;
  const uint32_t tid = threadIdx.x;
  const uint64_t t0 = F.t.track_offsets[e], t1 = F.t.track_offsets[e + 1];
  const uint64_t cap = F.o.cap_tracks;
  const uint32_t flag = *(const volatile uint32_t*)F.w.flag;
  if (flag & kFwdNoTracks) return;  // no track lists to read: nothing is written
  if (flag & kFwdBadOffsets) {      // hits rejected: no track has a downstream track
    for (uint64_t t = t0 + tid; t < t1 && t < cap; t += kFwdThreads) {
      F.o.n_found[t] = 0u;
      for (int L = 0; L < (int)kFwdL; ++L) F.o.hits[t * kFwdL + L] = kNone;
      for (int k = 0; k < (int)VELO_FWD_STATE; ++k) F.o.state[t * VELO_FWD_STATE + k] = 0.0f;
    }
    return;
  }
  const uint64_t h0 = F.h.event_offsets[e];
  const uint32_t n = (uint32_t)(F.h.event_offsets[e + 1] - h0);
  const FwdWork& W = F.w;
  if (tid < kFwdL) S.zl[tid] = F.g.z_layers[tid];
  // 1. sort by (layer, x): four passes over the ordered bits of x, one over the layer
  for (uint32_t i = tid; i < n; i += kFwdThreads) {
    W.ka[h0 + i] = ordered_bits(F.h.x[h0 + i]);
    W.va[h0 + i] = i;
  }
  __syncthreads();
  const uint32_t* lay = F.h.layer + h0;
  radix_pass<kFwdThreads, true>(W.ka + h0, W.kb + h0, W.va + h0, W.vb + h0, n,
                                [](uint32_t k, uint32_t) { return k & 255u; }, S.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.kb + h0, W.ka + h0, W.vb + h0, W.va + h0, n,
                                [](uint32_t k, uint32_t) { return (k >> 8) & 255u; }, S.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.ka + h0, W.kb + h0, W.va + h0, W.vb + h0, n,
                                [](uint32_t k, uint32_t) { return (k >> 16) & 255u; }, S.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.kb + h0, W.ka + h0, W.vb + h0, W.va + h0, n,
                                [](uint32_t k, uint32_t) { return k >> 24; }, S.cnt, S.tmp);
  const float* xin = F.h.x + h0;
  radix_pass<kFwdThreads, true>(W.ka + h0, W.kb + h0, W.va + h0, W.vb + h0, n,
                                [lay, xin](uint32_t, uint32_t id) { return fwd_bucket(lay, xin, id); }, S.cnt, S.tmp);
  // sorted x, y, and the first position of every layer (a layer's slots from
  // its predecessor's layer (exclusive) to its own get the position)
  for (uint32_t q = tid; q <= kFwdL; q += kFwdThreads) S.loff[q] = n;
  __syncthreads();
  for (uint32_t pos = tid; pos < n; pos += kFwdThreads) {
    const uint32_t id = W.vb[h0 + pos];
    W.sx[h0 + pos] = F.h.x[h0 + id];
    W.sy[h0 + pos] = F.h.y[h0 + id];
    const uint32_t L = fwd_bucket(lay, xin, id), Lp = pos ? fwd_bucket(lay, xin, W.vb[h0 + pos - 1]) + 1u : 0u;
    for (uint32_t q = Lp; q <= L; ++q) S.loff[q] = pos;
  }
  __syncthreads();
  // 2. the tracks of the event
  for (uint64_t t = t0 + tid; t < t1; t += kFwdThreads)
    if (t < cap) fwd_track(F, S, e, t, h0);
}

}  // namespace

}  // namespace velo

using namespace velo;

extern "C" {

int velo_forward_params_default(velo_forward_params_t* p) {
  if (!p) return VELO_EINVAL;
  p->p_min = 3.0f;
  p->win_y = 40.0f;
  p->tol_x = 8.0f;
  p->tol_y = 40.0f;
  p->tol_x_far = 3.0f;
  p->sigma_x = 0.08f;
  p->tol_match = 25.0f;
  p->chi2ndf_max = 4.0f;
  p->min_hits = 9;
  return VELO_OK;
}

int velo_forward_workspace_size(uint64_t n_events, uint64_t n_hits, uint64_t* bytes) {
  if (!bytes) return VELO_EINVAL;
  (void)n_events;
  FwdWork w;
  *bytes = fwd_carve(nullptr, n_hits, &w);
  return VELO_OK;
}

int velo_forward(const velo_downstream_hits_t* hits, const velo_output_t* tracks, const velo_downstream_t* geometry,
                 const velo_forward_params_t* params, const velo_forward_output_t* out, void* workspace,
                 uint64_t workspace_bytes, void* stream) {
  if (!hits || !tracks || !geometry || !params || !out || !workspace) return VELO_EINVAL;
  if (!hits->event_offsets || (hits->n_hits && (!hits->layer || !hits->x || !hits->y))) return VELO_EINVAL;
  if (!tracks->cluster_offsets || !tracks->cluster_x || !tracks->cluster_y || !tracks->cluster_z ||
      !tracks->track_offsets || !tracks->track_hit_offsets || !tracks->track_hits || !tracks->totals)
    return VELO_EINVAL;
  if (!out->n_found || !out->hits || !out->state) return VELO_EINVAL;
  if (hits->n_events >= (1ull << 31) || hits->n_hits >= (1ull << 40)) return VELO_EINVAL;
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return VELO_EINVAL;
  const velo_forward_params_t& p = *params;
  const float fin[] = {p.p_min, p.win_y, p.tol_x, p.tol_y, p.tol_x_far, p.sigma_x, p.tol_match, p.chi2ndf_max,
                       geometry->z_mag, geometry->kappa, geometry->kappa / p.p_min};
  for (float v : fin)
    if (!std::isfinite(v)) return VELO_EINVAL;
  if (!(p.p_min > 0.0f) || !(p.sigma_x > 0.0f) || p.min_hits < 3 || p.min_hits > VELO_FWD_LAYERS ||
      !(geometry->kappa > 0.0f))
    return VELO_EINVAL;
  for (uint32_t L = 0; L < VELO_FWD_LAYERS; ++L)
    if (!std::isfinite(geometry->z_layers[L]) || !(geometry->z_layers[L] > geometry->z_mag) ||
        (L && !(geometry->z_layers[L] > geometry->z_layers[L - 1])))
      return VELO_EINVAL;
  Fwd F;
  std::memset(&F, 0, sizeof(F));
  F.h = *hits;
  F.t = *tracks;
  F.g = *geometry;
  F.p = *params;
  F.o = *out;
  if (fwd_carve(static_cast<uint8_t*>(workspace), hits->n_hits, &F.w) > workspace_bytes) return VELO_ECAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_fwd_validate<<<1, 1024, 0, s>>>(F);
  if (hits->n_events) k_forward<<<(uint32_t)hits->n_events, kFwdThreads, 0, s>>>(F);
  return cudaGetLastError() == cudaSuccess ? VELO_OK : VELO_ECUDA;
}

}  // extern "C"
