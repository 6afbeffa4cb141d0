// Forward tracking: pixel-tracker tracks traced through one magnet kick to
// the downstream layers (velo_forward; the steps are stated in velo.h).
//
// The first stage traces pixel-tracker tracks forwards, straight to the
// middle of the magnet, one change of angle there, straight to the fibre
// tracker (Sec. "HLT1 details and results").  One CTA per event:
//   1. the span of x in every layer (and of y in layers 0 and 1) cut into
//      equal buckets; the event's downstream hits sorted by (layer, x bucket)
//      -- two stable counting passes -- and gathered into x, y arrays
//      (shared memory when the event fits, else its slice of the workspace)
//      with per-layer offsets and the first position of every bucket, then
//      by x inside every bucket (so by x in every layer); layers 0 and 1 also
//      by (layer, y bucket);
//   2. the tracks of the event, up to one per thread at a time: one thread
//      per track finds its line and the ranges of its candidate windows in
//      layers 0 and 1; a scan flattens the (track, candidate) pairs and the
//      threads share them out evenly -- the exact window test, the first
//      station and a bound on the match distance; the survivors' far
//      stations, fits and cuts, each offering its rank key (hits, distance,
//      id) to its track by a 64-bit atomicMin;
//   3. one thread per track recomputes its winning candidate and writes it.
// The work of an event grows about as the square of its hit count, so events
// of up to kFwdSmallHits hits run on 256-thread CTAs, four per SM, one event
// each; larger events on 1024-thread CTAs, one per SM, looping over a list
// of them that the validation kernel builds (shared memory up to
// kFwdBigHits hits, the workspace beyond).
// All arithmetic is binary32 in the order the oracle uses (-fmad=false and
// the __f*_rn intrinsics); every choice is a minimum under a strict total
// order, so the search order does not matter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "velo_device.cuh"
#include "velo_fit.cuh"
#include "velo_internal.cuh"

namespace velo {

namespace {

constexpr uint32_t kFwdL = VELO_FWD_LAYERS;

// x range [xp - tol - m, xp + tol + m] searched in a layer's sorted x: m =
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
  uint32_t *yka, *ykb;       // layers 0 and 1 by y: keys (ordered y bits)
  uint32_t *yva, *yvb;       // and (layer, x)-sorted positions
  uint32_t* nlist;           // [2]: events in list_big, list_huge
  uint32_t *list_big, *list_huge;  // events of more than kFwdSmallHits / kFwdBigHits hits
};

struct Fwd {
  velo_downstream_hits_t h;
  velo_output_t t;
  velo_downstream_t g;
  velo_forward_params_t p;
  velo_forward_output_t o;
  FwdWork w;
  float lam;  // largest sum |w_i| of the final x fit's weights at the kick plane (any admissible hit set)
};

uint64_t fwd_carve(uint8_t* base, uint64_t n_events, uint64_t n_hits, FwdWork* w) {
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
  w->yka = reinterpret_cast<uint32_t*>(take(4 * H));
  w->ykb = reinterpret_cast<uint32_t*>(take(4 * H));
  w->yva = reinterpret_cast<uint32_t*>(take(4 * H));
  w->yvb = reinterpret_cast<uint32_t*>(take(4 * H));
  const uint64_t E = n_events ? n_events : 1;
  w->nlist = reinterpret_cast<uint32_t*>(take(8));
  w->list_big = reinterpret_cast<uint32_t*>(take(4 * E));
  w->list_huge = reinterpret_cast<uint32_t*>(take(4 * E));
  return (off + 255ull) & ~255ull;
}

__device__ __forceinline__ uint32_t ordered_bits(float v) {  // monotone in v
  const uint32_t u = __float_as_uint(v);
  return u ^ ((u >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}

__device__ __forceinline__ float from_ordered_bits(uint32_t o) {
  return __uint_as_float(o ^ ((o >> 31) ? 0x80000000u : 0xFFFFFFFFu));
}


// flag bits: the hit offsets are invalid / the pixel-tracker result did not
// fit its buffers (its track lists were not written)
constexpr uint32_t kFwdBadOffsets = 1u, kFwdNoTracks = 2u;
constexpr uint32_t kFwdIdBits = 29;        // hit ids in a rank key: events hold fewer than 2^29 hits
constexpr uint32_t kFwdSmallHits = 4864;   // events up to this size: 256-thread CTAs, hits in shared memory
constexpr uint32_t kFwdBigHits = 16384;    // up to this size: 1024-thread CTAs, hits in shared memory
constexpr uint32_t kFwdRows = kFwdL + 2;   // bucket tables: x of every layer, y of layers 0 and 1

// One CTA: the event offsets start at 0, never decrease, end at n_hits and
// give no event 2^29 hits or more; the pixel-tracker totals fit its
// capacities.  With valid offsets, the lists of events above kFwdSmallHits
// and above kFwdBigHits hits (any order).
__global__ void __launch_bounds__(1024) k_fwd_validate(Fwd F) {
  __shared__ uint32_t nl[2];
  const uint64_t E = F.h.n_events;
  if (threadIdx.x < 2) nl[threadIdx.x] = 0u;
  int bad = 0;
  if (threadIdx.x == 0) bad |= (F.h.event_offsets[0] != 0ull) | (F.h.event_offsets[E] != F.h.n_hits);
  for (uint64_t e = threadIdx.x; e < E; e += blockDim.x) {
    const uint64_t a = F.h.event_offsets[e], b = F.h.event_offsets[e + 1];
    bad |= (b < a) | (b - a >= (1ull << kFwdIdBits));
  }
  bad = __syncthreads_or(bad);
  if (!bad)
    for (uint64_t e = threadIdx.x; e < E; e += blockDim.x) {
      const uint64_t n = F.h.event_offsets[e + 1] - F.h.event_offsets[e];
      if (n > kFwdBigHits) F.w.list_huge[atomicAdd(&nl[1], 1u)] = (uint32_t)e;
      else if (n > kFwdSmallHits) F.w.list_big[atomicAdd(&nl[0], 1u)] = (uint32_t)e;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    const velo_output_t& o = F.t;
    const bool fits = (!o.cap_clusters || o.totals[0] <= o.cap_clusters) && (!o.cap_tracks || o.totals[1] <= o.cap_tracks) &&
                      (!o.cap_track_hits || o.totals[2] <= o.cap_track_hits);
    *F.w.flag = (bad ? kFwdBadOffsets : 0u) | (fits ? 0u : kFwdNoTracks);
    F.w.nlist[0] = nl[0];
    F.w.nlist[1] = nl[1];
  }
}

// sort bucket of a hit: its layer, or kFwdL (never searched) for a layer
// number >= kFwdL or an x that is not finite
__device__ __forceinline__ uint32_t fwd_layer_of(const uint32_t* lay, const float* x, uint32_t id) {
  return isfinite(x[id]) ? min(lay[id], kFwdL) : kFwdL;
}

// Shared memory of a CTA of NT threads holding up to HC hits (HC = 0: the
// hits stay in the workspace).
template <int NT, uint32_t HC>
struct FwdSmem {
  static constexpr bool SM = HC > 0;
  static constexpr uint32_t NB = SM ? 256u : 128u;  // buckets per table (16-bit entries when SM)
  union {
    uint32_t cnt[radix_counters(NT)];  // radix counters of the (layer, x) sort
    float xy[2 * (SM ? HC : 1u)];      // then x, y in sorted order
  } u;
  union {
    uint32_t cnt[radix_counters(NT)];  // radix counters of the y sort
    struct {                           // then the tracks of the current chunk
      float4 trk[NT];                  // xm, ym, tx, ty
      uint32_t rlo[NT][2];             // first entries of the candidate ranges in the y order
      uint32_t rn0[NT];                // length of the layer-0 range
      uint32_t poff[NT + 1];           // first pair of each track
      unsigned long long best[NT];
    } c;
  } u2;
  // row q < kFwdL: first position of each x bucket of layer q (+ the layer's
  // end); rows kFwdL + r: first entry of each y bucket of layer r in the
  // (layer, y bucket) order of layers 0 and 1
  union {
    uint16_t s[kFwdRows][256 + 1];
    uint32_t g[kFwdRows][128 + 1];
  } tab;
  float vmin[kFwdRows], vinv[kFwdRows];  // bucket of v in row q: (v - vmin) * vinv, clamped
  uint32_t loff[kFwdL + 1];  // first position of each layer; [kFwdL] = end of the searched layers
  float dzm[kFwdL], dz0[kFwdL];  // z_L - z_mag, z_L - z_0
  float zm0, reach;              // z_mag - z_0; max(|z_mag - z_0|, z_11 - z_0)
  float wx[2];                   // candidate half-widths in x, layers 0 and 1
  uint32_t tmp[64];
  uint32_t nsv;                  // survivors of the current round
};

using FwdSmall = FwdSmem<256, kFwdSmallHits>;
using FwdBig = FwdSmem<1024, kFwdBigHits>;
using FwdHuge = FwdSmem<1024, 0>;
// 228 KB of shared memory per SM, 1 KB of it reserved per CTA: four small
// CTAs per SM, one big
static_assert(sizeof(FwdSmall) + 1024 <= 228 * 1024 / 4, "shared memory for four CTAs per SM");
static_assert(sizeof(FwdBig) <= 227 * 1024, "shared memory of one CTA");
static_assert(kFwdBigHits <= 65535u, "16-bit bucket tables");

template <class S>
__device__ __forceinline__ uint32_t fwd_bucket(float v, float vmin, float inv) {
  const float t = fm(fs(v, vmin), inv);  // monotone in v; NaN goes to bucket 0
  if (!(t >= 0.0f)) return 0u;
  if (t >= (float)S::NB) return S::NB - 1u;
  return (uint32_t)t;
}

template <class S>
__device__ __forceinline__ uint32_t tab_get(const S& sm, uint32_t row, uint32_t b) {
  if constexpr (S::SM) return sm.tab.s[row][b];
  else return sm.tab.g[row][b];
}

template <class S>
__device__ __forceinline__ void tab_set(S& sm, uint32_t row, uint32_t b, uint32_t v) {
  if constexpr (S::SM) sm.tab.s[row][b] = (uint16_t)v;
  else sm.tab.g[row][b] = v;
}

// first entry of row q at or after which every value >= v lies
template <class S>
__device__ __forceinline__ uint32_t tab_first(const S& sm, uint32_t row, float v) {
  return tab_get(sm, row, fwd_bucket<S>(v, sm.vmin[row], sm.vinv[row]));
}

// first entry of row q before which every value <= v lies
template <class S>
__device__ __forceinline__ uint32_t tab_past(const S& sm, uint32_t row, float v) {
  return tab_get(sm, row, fwd_bucket<S>(v, sm.vmin[row], sm.vinv[row]) + 1u);
}

// scale of row q's buckets over a sorted range [vmin, vmax]
template <class S>
__device__ __forceinline__ void fwd_bucket_scale(S& sm, uint32_t row, bool any, float vmin, float vmax) {
  const float span = fs(vmax, vmin);
  const float iv = any && span > 0.0f ? fd((float)S::NB, span) : 0.0f;
  sm.vmin[row] = any ? vmin : 0.0f;
  sm.vinv[row] = isfinite(iv) ? iv : 0.0f;
}

// the sorted hits of one event
template <class S>
struct FwdEvent {
  const float* sx;      // x in sorted order (shared memory when S::SM, else global)
  const float* sy;
  const uint32_t* sid;  // hit id of each sorted position (global)
  const S* sm;
};

// nearest hit in x to xp (ties: the smaller id) with |x - xp| <= tol and
// |y - yp| <= tol_y in layer L; returns its sorted position or kNone
template <class S>
__device__ __forceinline__ uint32_t fwd_nearest(const FwdEvent<S>& V, int L, float xp, float yp, float tol,
                                                float tol_y) {
  float lo_x, hi_x;
  fwd_range(xp, tol, &lo_x, &hi_x);
  const uint32_t end = V.sm->loff[L + 1];
  uint32_t pos = tab_first(*V.sm, L, lo_x);  // every hit with x >= lo_x lies at or after it
  while (pos < end && V.sx[pos] < lo_x) ++pos;
  uint32_t best = kNone;
  float bd = 0.0f;
  for (; pos < end && V.sx[pos] <= hi_x; ++pos) {
    const float d = fabsf(fs(V.sx[pos], xp));
    if (!(d <= tol) || !(fabsf(fs(V.sy[pos], yp)) <= tol_y)) continue;
    if (best == kNone || d < bd || (d == bd && V.sid[pos] < V.sid[best])) {
      best = pos;
      bd = d;
    }
  }
  return best;
}

// least-squares line v = a + b (z - z_0) through the found hits of layers [l0, l1)
__device__ __forceinline__ void fwd_line(const uint32_t* hl, const float* v, const float* dz0, int l0, int l1,
                                         float* a, float* b) {
  float S0 = 0.0f, Sz = 0.0f, Szz = 0.0f, Sx = 0.0f, Sxz = 0.0f;
#pragma unroll
  for (int L = l0; L < l1; ++L) {
    if (hl[L] == kNone) continue;
    const float dz = dz0[L];
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

struct FwdCand {
  uint32_t n;
  float rchi, a, b, d, dy, ad;
  uint32_t hl[kFwdL];  // sorted positions, kNone = no hit
};

// Step 3's first station for the candidate at sorted position pc of layer r
// of a track whose line reaches the kick plane at (xm, ym) with slope ty:
// its hits hl[0..3] and the line (a1, b1) through them; false with fewer
// than two
template <class S>
__device__ __forceinline__ bool fwd_station1(const FwdEvent<S>& V, const Fwd& F, float xm, float ym, float ty, int r,
                                             uint32_t pc, uint32_t* hl, float* a1, float* b1) {
  const velo_forward_params_t& P = F.p;
  const S& sm = *V.sm;
  const float tk = fd(fs(V.sx[pc], xm), sm.dzm[r]);
  uint32_t n1 = 0;
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    hl[L] = fwd_nearest(V, L, fa(xm, fm(tk, sm.dzm[L])), fa(ym, fm(ty, sm.dzm[L])), P.tol_x, P.tol_y);
    n1 += hl[L] != kNone ? 1u : 0u;
  }
  if (n1 < 2) return false;
  fwd_line(hl, V.sx, sm.dz0, 0, 4, a1, b1);
  return true;
}

// steps 3 (the other stations) to 5 given the first station's hits C.hl[0..3]
// and line (a1, b1): false when a cut drops the candidate
template <class S>
__device__ __forceinline__ bool fwd_far(const FwdEvent<S>& V, const Fwd& F, float xm, float ym, float ty, float a1,
                                        float b1, FwdCand& C) {
  const velo_forward_params_t& P = F.p;
  const S& sm = *V.sm;
  uint32_t n = 0;
#pragma unroll
  for (int L = 0; L < 4; ++L) n += C.hl[L] != kNone ? 1u : 0u;
#pragma unroll
  for (int L = 4; L < (int)kFwdL; ++L) {
    C.hl[L] = fwd_nearest(V, L, fa(a1, fm(b1, sm.dz0[L])), fa(ym, fm(ty, sm.dzm[L])), P.tol_x_far, P.tol_y);
    n += C.hl[L] != kNone ? 1u : 0u;
  }
  if (n < P.min_hits) return false;
  float a, b;
  fwd_line(C.hl, V.sx, sm.dz0, 0, kFwdL, &a, &b);
  float chi2 = 0.0f;
#pragma unroll
  for (int L = 0; L < (int)kFwdL; ++L) {
    if (C.hl[L] == kNone) continue;
    const float res = fd(fs(fs(V.sx[C.hl[L]], a), fm(b, sm.dz0[L])), P.sigma_x);
    chi2 = fa(chi2, fm(res, res));
  }
  const float rchi = fd(chi2, (float)(n - 2));
  if (!(rchi <= P.chi2ndf_max)) return false;
  const float d = fs(fa(a, fm(b, sm.zm0)), xm);
  float ya, yb;
  fwd_line(C.hl, V.sy, sm.dz0, 0, kFwdL, &ya, &yb);
  const float dy = fs(fa(ya, fm(yb, sm.zm0)), ym);
  const float ad = fa(fm(d, d), fm(dy, dy));
  if (!(ad <= fm(P.tol_match, P.tol_match))) return false;
  C.n = n;
  C.rchi = rchi;
  C.a = a;
  C.b = b;
  C.d = d;
  C.dy = dy;
  C.ad = ad;
  return true;
}

// steps 3-5 for the candidate at sorted position pc of layer r: false when a
// cut drops it
template <class S>
__device__ __forceinline__ bool fwd_candidate(const FwdEvent<S>& V, const Fwd& F, float xm, float ym, float ty, int r,
                                              uint32_t pc, FwdCand& C) {
  float a1, b1;
  if (!fwd_station1(V, F, xm, ym, ty, r, pc, C.hl, &a1, &b1)) return false;
  return fwd_far(V, F, xm, ym, ty, a1, b1, C);
}

// A necessary condition for the candidate with first-station hits hl[0..3]
// and line L1 = (a1, b1) to pass the match cut.  The final x line is the
// least-squares line of the first-station hits and the far hits; written as
// L1 plus the least-squares line of the hits' offsets e_i from L1, its
// distance at the kick plane is d1 + sum w_i e_i, with d1 that of L1, w_i the
// fit's weights at the kick plane and |e_i| at most E = max(first-station
// residuals, tol_x_far).  So |d| <= tol_match needs |d1| <= tol_match + lam E,
// lam the largest sum |w_i| over the hit sets a candidate can end with (host
// arithmetic); the allowance 1 mm + 2e-3 M (M the size of the coordinates
// involved) covers the binary32 rounding of both lines, its worst case being
// some 1e-4 M.
template <class S>
__device__ __forceinline__ bool fwd_may_match(const FwdEvent<S>& V, const Fwd& F, float xm, const uint32_t* hl,
                                              float a1, float b1) {
  const S& sm = *V.sm;
  float E = F.p.tol_x_far;
#pragma unroll
  for (int L = 0; L < 4; ++L)
    if (hl[L] != kNone) E = fmaxf(E, fabsf(fs(V.sx[hl[L]], fa(a1, fm(b1, sm.dz0[L])))));
  const float M = fa(fa(fa(fabsf(a1), fm(fabsf(b1), sm.reach)), fabsf(xm)), E);
  const float d1 = fs(fa(a1, fm(b1, sm.zm0)), xm);
  return fabsf(d1) <= fa(fa(F.p.tol_match, fm(F.lam, E)), fa(1.0f, fm(2e-3f, M)));
}

// rank key: more hits, then the smaller distance (non-negative binary32
// orders as its bits), then the smaller candidate id -- the smallest key wins
__device__ __forceinline__ unsigned long long fwd_key(uint32_t n, float ad, uint32_t c) {
  return ((unsigned long long)(kFwdL - n) << 60) | ((unsigned long long)__float_as_uint(ad) << kFwdIdBits) | c;
}

__device__ __forceinline__ void fwd_write_none(const Fwd& F, uint64_t t) {
  F.o.n_found[t] = 0u;
  for (int L = 0; L < (int)kFwdL; ++L) F.o.hits[t * kFwdL + L] = kNone;
  for (int k = 0; k < (int)VELO_FWD_STATE; ++k) F.o.state[t * VELO_FWD_STATE + k] = 0.0f;
}

// Steps 1 to 3 of event e on a CTA of NT threads (S: its shared memory).
template <int NT, class S>
__device__ __forceinline__ void fwd_event(const Fwd& F, S& sm, uint64_t e) {
  const uint32_t tid = threadIdx.x;
  const uint64_t cap = F.o.cap_tracks;
  const FwdWork& W = F.w;
  const uint64_t t0 = F.t.track_offsets[e], t1 = F.t.track_offsets[e + 1];
  const uint64_t h0 = F.h.event_offsets[e];
  const uint32_t n = (uint32_t)(F.h.event_offsets[e + 1] - h0);
  const uint32_t* lay = F.h.layer + h0;
  const float* xin = F.h.x + h0;
  const float* yin = F.h.y + h0;
  constexpr uint32_t NB = S::NB;
  constexpr uint32_t NW = NT / 32;
  const float zmag = F.g.z_mag;
  // 1. the span of x in every layer and of y in layers 0 and 1 (finite values
  // of searched hits): ordered-bit minima and maxima per warp, then over the
  // warps; the buckets of each table divide its span evenly
  uint32_t* mm = sm.u2.cnt;  // [NW][kFwdRows][min, max]
  for (uint32_t i = tid; i < NW * kFwdRows * 2; i += NT) mm[i] = (i & 1u) ? 0u : ~0u;
  __syncthreads();
  for (uint32_t i = tid; i < n; i += NT) {
    const uint32_t L = fwd_layer_of(lay, xin, i);
    if (L >= kFwdL) continue;
    uint32_t* m = mm + (warp_id() * kFwdRows + L) * 2;
    const uint32_t o = ordered_bits(xin[i]);
    atomicMin(m, o);
    atomicMax(m + 1, o);
    const float y = yin[i];
    if (L < 2 && isfinite(y)) {
      uint32_t* my = mm + (warp_id() * kFwdRows + kFwdL + L) * 2;
      const uint32_t oy = ordered_bits(y);
      atomicMin(my, oy);
      atomicMax(my + 1, oy);
    }
  }
  __syncthreads();
  if (tid < kFwdRows) {
    uint32_t lo = ~0u, hi = 0u;
    for (uint32_t w = 0; w < NW; ++w) {
      lo = min(lo, mm[(w * kFwdRows + tid) * 2]);
      hi = max(hi, mm[(w * kFwdRows + tid) * 2 + 1]);
    }
    const bool any = lo <= hi;
    fwd_bucket_scale(sm, tid, any, any ? from_ordered_bits(lo) : 0.0f, any ? from_ordered_bits(hi) : 0.0f);
  } else if (tid >= 32 && tid < 32 + kFwdL) {
    const float z = F.g.z_layers[tid - 32];
    sm.dzm[tid - 32] = fs(z, zmag);
    sm.dz0[tid - 32] = fs(z, F.g.z_layers[0]);
  } else if (tid == 64) {
    sm.zm0 = fs(zmag, F.g.z_layers[0]);
    sm.reach = fmaxf(fabsf(sm.zm0), fs(F.g.z_layers[kFwdL - 1], F.g.z_layers[0]));
  } else if (tid >= 96 && tid < 98) {
    sm.wx[tid - 96] = fa(fm(fd(F.g.kappa, F.p.p_min), fs(F.g.z_layers[tid - 96], zmag)), F.p.tol_x);
  }
  __syncthreads();
  // 2. counting sort by (layer, x bucket): a stable pass over the bucket, one
  // over the layer (kFwdL: not searched); the order inside a bucket is the
  // ids' (searches scan whole buckets, the exact tests decide)
  for (uint32_t i = tid; i < n; i += NT) {
    const uint32_t L = fwd_layer_of(lay, xin, i);
    W.ka[h0 + i] = (L < kFwdL ? fwd_bucket<S>(xin[i], sm.vmin[L], sm.vinv[L]) : 0u) | L << 8;
    W.va[h0 + i] = i;
  }
  __syncthreads();
  radix_pass<NT, true>(W.ka + h0, W.kb + h0, W.va + h0, W.vb + h0, n, [](uint32_t k, uint32_t) { return k & 255u; },
                       sm.u.cnt, sm.tmp);
  radix_pass<NT, true>(W.kb + h0, W.ka + h0, W.vb + h0, W.va + h0, n, [](uint32_t k, uint32_t) { return k >> 8; },
                       sm.u.cnt, sm.tmp);
  // sorted x, y, the sorted position of every id (into vb, free after the
  // sort), the first position of every layer (a layer's slots after its
  // predecessor's layer get the position)
  const uint32_t* skey = W.ka + h0;  // (layer, bucket) of every sorted position
  float* sx = S::SM ? sm.u.xy : W.sx + h0;
  float* sy = S::SM ? sm.u.xy + n : W.sy + h0;
  uint32_t* sid = W.va + h0;
  uint32_t* pos_of = W.vb + h0;
  for (uint32_t q = tid; q <= kFwdL; q += NT) sm.loff[q] = n;
  __syncthreads();
  for (uint32_t pos = tid; pos < n; pos += NT) {
    const uint32_t id = sid[pos];
    sx[pos] = xin[id];
    sy[pos] = yin[id];
    const uint32_t L = skey[pos] >> 8, Lp = pos ? (skey[pos - 1] >> 8) + 1u : 0u;
    for (uint32_t q = Lp; q <= L; ++q) sm.loff[q] = pos;
  }
  __syncthreads();
  // the x tables from the sorted keys: entry b of a row is the first position
  // whose bucket is b or more (the layer's end past its last hit)
  for (uint32_t i = tid; i < kFwdL * (NB + 1); i += NT) {
    const uint32_t q = i / (NB + 1);
    tab_set(sm, q, i % (NB + 1), sm.loff[q + 1]);
  }
  __syncthreads();
  for (uint32_t pos = tid; pos < sm.loff[kFwdL]; pos += NT) {
    const uint32_t L = skey[pos] >> 8, b = skey[pos] & 255u;
    const uint32_t bp = pos > sm.loff[L] ? (skey[pos - 1] & 255u) + 1u : 0u;
    for (uint32_t q = bp; q <= b; ++q) tab_set(sm, L, q, pos);
  }
  __syncthreads();
  // x order inside every bucket (insertion sort: a bucket holds a few hits),
  // so that every layer is sorted by x; then the position of every id
  for (uint32_t q = tid; q < kFwdL * NB; q += NT) {
    const uint32_t L = q / NB, b = q % NB;
    const uint32_t lo = tab_get(sm, L, b), hi = tab_get(sm, L, b + 1);
    for (uint32_t i = lo + 1; i < hi; ++i) {
      const float xv = sx[i], yv = sy[i];
      const uint32_t idv = sid[i];
      uint32_t k = i;
      for (; k > lo && sx[k - 1] > xv; --k) {
        sx[k] = sx[k - 1];
        sy[k] = sy[k - 1];
        sid[k] = sid[k - 1];
      }
      sx[k] = xv;
      sy[k] = yv;
      sid[k] = idv;
    }
  }
  __syncthreads();
  for (uint32_t pos = tid; pos < n; pos += NT) pos_of[sid[pos]] = pos;
  // 3. layers 0 and 1 by (layer, y bucket), the same way: ypos holds their
  // (layer, x)-sorted positions, layer 0's at [0, l1), layer 1's at [l1, n01)
  const uint32_t n01 = sm.loff[2], l1 = sm.loff[1];
  for (uint32_t pos = tid; pos < n01; pos += NT) {
    const uint32_t r = pos >= l1 ? 1u : 0u;
    W.yka[h0 + pos] = fwd_bucket<S>(sy[pos], sm.vmin[kFwdL + r], sm.vinv[kFwdL + r]) | r << 8;
    W.yva[h0 + pos] = pos;
  }
  __syncthreads();
  radix_pass<NT, true>(W.yka + h0, W.ykb + h0, W.yva + h0, W.yvb + h0, n01,
                       [](uint32_t k, uint32_t) { return k & 255u; }, sm.u2.cnt, sm.tmp);
  radix_pass<NT, true>(W.ykb + h0, W.yka + h0, W.yvb + h0, W.yva + h0, n01, [](uint32_t k, uint32_t) { return k >> 8; },
                       sm.u2.cnt, sm.tmp);
  const uint32_t* ypos = W.yva + h0;
  const uint32_t* ykey = W.yka + h0;
  // 4. the y tables the same way (the order inside a y bucket does not
  // matter: candidate ranges are whole buckets, the exact tests decide)
  for (uint32_t i = tid; i < 2 * (NB + 1); i += NT) {
    const uint32_t r = i / (NB + 1);
    tab_set(sm, kFwdL + r, i % (NB + 1), r ? n01 : l1);
  }
  __syncthreads();
  for (uint32_t i = tid; i < n01; i += NT) {
    const uint32_t r = ykey[i] >> 8, b = ykey[i] & 255u;
    const uint32_t bp = i > (r ? l1 : 0u) ? (ykey[i - 1] & 255u) + 1u : 0u;
    for (uint32_t q = bp; q <= b; ++q) tab_set(sm, kFwdL + r, q, i);
  }
  __syncthreads();
  const FwdEvent<S> V{sx, sy, sid, &sm};
  // 2.-3. the tracks, NT at a time
  for (uint64_t tc = t0; tc < t1; tc += NT) {
    const uint64_t t = tc + tid;
    uint32_t cnt = 0;
    bool live = false;
    if (t < t1 && t < cap) {
      const uint64_t hs = F.t.track_hit_offsets[t], he = F.t.track_hit_offsets[t + 1];
      if (he >= hs + 2) {
        // 0.-1. the line through the two most downstream clusters, at the kick plane
        const uint64_t c0 = F.t.cluster_offsets[e];
        const uint64_t ha = c0 + F.t.track_hits[he - 1], hb = c0 + F.t.track_hits[he - 2];
        const float x0 = F.t.cluster_x[ha], y0 = F.t.cluster_y[ha], z0 = F.t.cluster_z[ha];
        const float dzab = fs(z0, F.t.cluster_z[hb]);
        const float tx = fd(fs(x0, F.t.cluster_x[hb]), dzab), ty = fd(fs(y0, F.t.cluster_y[hb]), dzab);
        const float dzm = fs(zmag, z0);
        const float xm = fa(x0, fm(tx, dzm)), ym = fa(y0, fm(ty, dzm));
        sm.u2.c.trk[tid] = make_float4(xm, ym, tx, ty);
        live = true;
        // 2. ranges of the y order holding the candidate windows of layers 0 and 1
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          float lo_y, hi_y;
          fwd_range(fa(ym, fm(ty, sm.dzm[r])), F.p.win_y, &lo_y, &hi_y);
          const uint32_t lo = tab_first(sm, kFwdL + r, lo_y);
          const uint32_t hi = tab_past(sm, kFwdL + r, hi_y);
          sm.u2.c.rlo[tid][r] = lo;
          const uint32_t len = hi > lo ? hi - lo : 0u;
          if (r == 0) sm.u2.c.rn0[tid] = len;
          cnt += len;
        }
      } else {
        fwd_write_none(F, t);
      }
    }
    sm.u2.c.best[tid] = ~0ull;
    uint32_t total;
    const uint32_t first = block_exclusive_scan<NT, uint32_t>(cnt, &total, sm.tmp);
    sm.u2.c.poff[tid] = first;
    if (tid == 0) sm.u2.c.poff[NT] = total;
    __syncthreads();
    // the (track, candidate) pairs, shared out evenly, n at a time: the
    // window test, the first station and the bound, the survivors listed in
    // the event's workspace entries that are dead by now (at most one per
    // pair, so at most n); then the survivors' far stations, fits and cuts.
    // With positions of 16 bits (hits in shared memory) a survivor keeps its
    // first station too.
    const uint32_t R = max(1u, n);
    uint32_t* sv_pj = W.yvb + h0;  // position, | track in the chunk << 16 when S::SM
    uint32_t* sv_j = W.ka + h0;    // track in the chunk (hits in the workspace)
    uint32_t* sv_h01 = W.ka + h0;  // first-station positions, 16 bits each (0xFFFF: none)
    uint32_t* sv_h23 = W.kb + h0;
    uint32_t* sv_a1 = W.yka + h0;  // and line
    uint32_t* sv_b1 = W.ykb + h0;
    for (uint32_t q0 = 0; q0 < total; q0 += R) {
      if (tid == 0) sm.nsv = 0;
      __syncthreads();
      for (uint32_t q = q0 + tid; q < min(total, q0 + R); q += NT) {
        uint32_t lo = 0, hi = NT;  // the track j with poff[j] <= q < poff[j + 1]
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (sm.u2.c.poff[mid] <= q) lo = mid;
          else hi = mid;
        }
        const uint32_t j = lo, k = q - sm.u2.c.poff[j];
        const int r = k < sm.u2.c.rn0[j] ? 0 : 1;
        const uint32_t pc = ypos[sm.u2.c.rlo[j][r] + (r ? k - sm.u2.c.rn0[j] : k)];
        const float4 tr = sm.u2.c.trk[j];
        if (!(fabsf(fs(sx[pc], fa(tr.x, fm(tr.z, sm.dzm[r])))) <= sm.wx[r]) ||
            !(fabsf(fs(sy[pc], fa(tr.y, fm(tr.w, sm.dzm[r])))) <= F.p.win_y))
          continue;
        uint32_t hl[4];
        float a1, b1;
        if (!fwd_station1(V, F, tr.x, tr.y, tr.w, r, pc, hl, &a1, &b1)) continue;
        if (!fwd_may_match(V, F, tr.x, hl, a1, b1)) continue;
        const uint32_t slot = atomicAdd(&sm.nsv, 1u);
        if constexpr (S::SM) {
          sv_pj[slot] = pc | j << 16;
          sv_h01[slot] = (hl[0] & 0xFFFFu) | hl[1] << 16;
          sv_h23[slot] = (hl[2] & 0xFFFFu) | hl[3] << 16;
          sv_a1[slot] = __float_as_uint(a1);
          sv_b1[slot] = __float_as_uint(b1);
        } else {
          sv_pj[slot] = pc;
          sv_j[slot] = j;
        }
      }
      __syncthreads();
      const uint32_t nsv = sm.nsv;
      for (uint32_t i = tid; i < nsv; i += NT) {
        const uint32_t pc = S::SM ? sv_pj[i] & 0xFFFFu : sv_pj[i], j = S::SM ? sv_pj[i] >> 16 : sv_j[i];
        const float4 tr = sm.u2.c.trk[j];
        FwdCand C;
        bool ok;
        if constexpr (S::SM) {
          const uint32_t p01 = sv_h01[i], p23 = sv_h23[i];
          const uint32_t p[4] = {p01 & 0xFFFFu, p01 >> 16, p23 & 0xFFFFu, p23 >> 16};
#pragma unroll
          for (int L = 0; L < 4; ++L) C.hl[L] = p[L] == 0xFFFFu ? kNone : p[L];
          ok = fwd_far(V, F, tr.x, tr.y, tr.w, __uint_as_float(sv_a1[i]), __uint_as_float(sv_b1[i]), C);
        } else {
          ok = fwd_candidate(V, F, tr.x, tr.y, tr.w, pc < sm.loff[1] ? 0 : 1, pc, C);
        }
        if (ok) atomicMin(&sm.u2.c.best[j], fwd_key(C.n, C.ad, sid[pc]));
      }
      __syncthreads();
    }
    // 3. the winner of every track, recomputed and written
    if (live) {
      const unsigned long long key = sm.u2.c.best[tid];
      if (key == ~0ull) {
        fwd_write_none(F, t);
      } else {
        const uint32_t pc = pos_of[(uint32_t)(key & ((1ull << kFwdIdBits) - 1ull))];
        const float4 tr = sm.u2.c.trk[tid];
        FwdCand C;
        fwd_candidate(V, F, tr.x, tr.y, tr.w, pc < sm.loff[1] ? 0 : 1, pc, C);
        F.o.n_found[t] = C.n;
#pragma unroll
        for (int L = 0; L < (int)kFwdL; ++L) F.o.hits[t * kFwdL + L] = C.hl[L] != kNone ? sid[C.hl[L]] : kNone;
        float* so = F.o.state + t * VELO_FWD_STATE;
        so[0] = fd(fs(C.b, tr.z), F.g.kappa);
        so[1] = C.rchi;
        so[2] = C.b;
        so[3] = C.a;
        so[4] = C.d;
        so[5] = C.dy;
      }
    }
    __syncthreads();
  }
}

// One 256-thread CTA per event; events of more than kFwdSmallHits hits are
// left to k_forward_list (so are all when the result or the offsets are
// rejected, except for writing the empty answers).
__global__ void __launch_bounds__(256, 4) k_forward_small(Fwd F) {
  extern __shared__ __align__(16) uint8_t fwd_smem_raw[];
  FwdSmall& sm = *reinterpret_cast<FwdSmall*>(fwd_smem_raw);
  const uint64_t e = blockIdx.x;
  const uint32_t flag = *(const volatile uint32_t*)F.w.flag;
  if (flag & kFwdNoTracks) return;  // no track lists to read: nothing is written
  if (flag & kFwdBadOffsets) {      // hits rejected: no track has a downstream track
    const uint64_t t0 = F.t.track_offsets[e], t1 = F.t.track_offsets[e + 1];
    for (uint64_t t = t0 + threadIdx.x; t < t1 && t < F.o.cap_tracks; t += 256) fwd_write_none(F, t);
    return;
  }
  if (F.h.event_offsets[e + 1] - F.h.event_offsets[e] > kFwdSmallHits) return;
  fwd_event<256>(F, sm, e);
}

// 1024-thread CTAs over the list of events above kFwdSmallHits hits (HUGE =
// false: up to kFwdBigHits, hits in shared memory) or above kFwdBigHits
// (HUGE = true: hits in the workspace); the lists are empty when the
// offsets or the result are rejected.
template <bool HUGE>
__global__ void __launch_bounds__(1024, 1) k_forward_list(Fwd F) {
  using S = typename std::conditional<HUGE, FwdHuge, FwdBig>::type;
  extern __shared__ __align__(16) uint8_t fwd_smem_raw[];
  S& sm = *reinterpret_cast<S*>(fwd_smem_raw);
  if (*(const volatile uint32_t*)F.w.flag & kFwdNoTracks) return;
  const uint32_t count = F.w.nlist[HUGE ? 1 : 0];
  const uint32_t* list = HUGE ? F.w.list_huge : F.w.list_big;
  for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
    fwd_event<1024>(F, sm, list[i]);
    __syncthreads();
  }
}

}  // namespace

}  // namespace velo

using namespace velo;

namespace {

// Largest sum over the hits of |w_i|, w_i the weights of the least-squares
// line's value at the kick plane, over every set of layers a candidate can
// end with (at least min_hits layers, two or more of them in the first
// station); in double, rounded up.  The last answer is kept.
float fwd_lambda(const velo_downstream_t& g, uint32_t min_hits) {
  static std::mutex mu;
  static velo_downstream_t last_g;
  static uint32_t last_min = 0;
  static float last = -1.0f;
  std::lock_guard<std::mutex> lk(mu);
  if (last >= 0.0f && last_min == min_hits && std::memcmp(&last_g, &g, sizeof(g)) == 0) return last;
  double best = 0.0;
  for (uint32_t m = 0; m < (1u << VELO_FWD_LAYERS); ++m) {
    if ((uint32_t)__builtin_popcount(m) < min_hits || __builtin_popcount(m & 15u) < 2) continue;
    double n = 0.0, zb = 0.0;
    for (uint32_t L = 0; L < VELO_FWD_LAYERS; ++L)
      if (m >> L & 1u) {
        n += 1.0;
        zb += (double)g.z_layers[L] - g.z_layers[0];
      }
    zb /= n;
    double sxx = 0.0;
    for (uint32_t L = 0; L < VELO_FWD_LAYERS; ++L)
      if (m >> L & 1u) {
        const double dz = (double)g.z_layers[L] - g.z_layers[0] - zb;
        sxx += dz * dz;
      }
    const double zq = (double)g.z_mag - g.z_layers[0] - zb;
    double sum = 0.0;
    for (uint32_t L = 0; L < VELO_FWD_LAYERS; ++L)
      if (m >> L & 1u) sum += std::fabs(1.0 / n + zq * ((double)g.z_layers[L] - g.z_layers[0] - zb) / sxx);
    best = std::max(best, sum);
  }
  last = std::nextafter((float)(best * (1.0 + 1e-6)), INFINITY);
  last_g = g;
  last_min = min_hits;
  return last;
}

int fwd_sm_count() {
  static std::mutex mu;
  static int cached[64] = {};
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (!cached[d] && cudaDeviceGetAttribute(&cached[d], cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
    cudaGetLastError();
    cached[d] = 148;
  }
  return cached[d];
}

}  // namespace

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
  FwdWork w;
  *bytes = fwd_carve(nullptr, n_events, n_hits, &w);
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
  F.lam = fwd_lambda(*geometry, p.min_hits);
  F.h = *hits;
  F.t = *tracks;
  F.g = *geometry;
  F.p = *params;
  F.o = *out;
  if (fwd_carve(static_cast<uint8_t*>(workspace), hits->n_events, hits->n_hits, &F.w) > workspace_bytes)
    return VELO_ECAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!set_max_smem_once(reinterpret_cast<const void*>(k_forward_small), 2) ||
      !set_max_smem_once(reinterpret_cast<const void*>(k_forward_list<false>), 3) ||
      !set_max_smem_once(reinterpret_cast<const void*>(k_forward_list<true>), 4))
    return VELO_ECUDA;
  k_fwd_validate<<<1, 1024, 0, s>>>(F);
  if (hits->n_events) {
    // the large events first (one 1024-thread CTA per SM), then the rest
    const uint32_t ctas = (uint32_t)std::min<uint64_t>(fwd_sm_count(), hits->n_events);
    if (hits->n_hits > kFwdSmallHits) k_forward_list<false><<<ctas, 1024, sizeof(FwdBig), s>>>(F);
    if (hits->n_hits > kFwdBigHits) k_forward_list<true><<<ctas, 1024, sizeof(FwdHuge), s>>>(F);
    k_forward_small<<<(uint32_t)hits->n_events, 256, sizeof(FwdSmall), s>>>(F);
  }
  return cudaGetLastError() == cudaSuccess ? VELO_OK : VELO_ECUDA;
}

}  // extern "C"
