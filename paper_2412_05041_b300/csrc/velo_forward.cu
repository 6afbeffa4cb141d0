// Forward tracking: pixel-tracker tracks traced through one magnet kick to
// the downstream layers (velo_forward; the steps are stated in velo.h).
//
// The first stage traces pixel-tracker tracks forwards, straight to the
// middle of the magnet, one change of angle there, straight to the fibre
// tracker (Sec. "HLT1 details and results").  One CTA per event:
//   1. the event's downstream hits are sorted by (layer, x) -- four stable
//      radix passes over the order-preserving bits of x, one over the layer
//      -- and gathered into sorted x, y arrays (shared memory when the event
//      fits, else its slice of the workspace), with per-layer offsets and a
//      bucket index per layer (first position of each of its x buckets),
//      layers 0 and 1 also in y order with a bucket index over y;
//   2. the tracks of the event, up to kFwdThreads at a time: one thread per
//      track finds its line and the position ranges of its candidate windows
//      in layers 0 and 1; a scan flattens the (track, candidate) pairs and
//      the threads share them out evenly -- each runs the exact window test
//      and, for a candidate inside it, the hit collection, fits and cuts, and
//      offers the candidate's rank key (hits, distance, id) to its track by a
//      64-bit atomicMin;
//   3. one thread per track recomputes its winning candidate and writes it.
// All arithmetic is binary32 in the order the oracle uses (-fmad=false and
// the __f*_rn intrinsics); every choice is a minimum under a strict total
// order, so the search order does not matter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "velo_device.cuh"
#include "velo_fit.cuh"
#include "velo_internal.cuh"

namespace velo {

namespace {

constexpr int kFwdThreads = 256;
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
  w->yka = reinterpret_cast<uint32_t*>(take(4 * H));
  w->ykb = reinterpret_cast<uint32_t*>(take(4 * H));
  w->yva = reinterpret_cast<uint32_t*>(take(4 * H));
  w->yvb = reinterpret_cast<uint32_t*>(take(4 * H));
  return (off + 255ull) & ~255ull;
}

__device__ __forceinline__ uint32_t ordered_bits(float v) {  // monotone in v
  const uint32_t u = __float_as_uint(v);
  return u ^ ((u >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}


// flag bits: the hit offsets are invalid / the pixel-tracker result did not
// fit its buffers (its track lists were not written)
constexpr uint32_t kFwdBadOffsets = 1u, kFwdNoTracks = 2u;
constexpr uint32_t kFwdIdBits = 29;      // hit ids in a rank key: events hold fewer than 2^29 hits
constexpr uint32_t kFwdSmemHits = 4096;  // events up to this size keep x, y in shared memory
constexpr uint32_t kFwdSurv = 1280;      // pairs per round (each leaves at most one survivor)
constexpr int kFwdCtasPerSm = 4;
constexpr uint32_t kFwdRows = kFwdL + 2;  // bucket tables: x of every layer, y of layers 0 and 1

// buckets per table: 256 of 16-bit positions for events in shared memory
// (positions < kFwdSmemHits), 128 of 32-bit positions otherwise
__host__ __device__ constexpr uint32_t fwd_nb(bool sm) { return sm ? 256u : 128u; }

// One CTA: the event offsets start at 0, never decrease, end at n_hits and
// give no event 2^29 hits or more; the pixel-tracker totals fit its capacities.
__global__ void __launch_bounds__(1024) k_fwd_validate(Fwd F) {
  const uint64_t E = F.h.n_events;
  int bad = 0;
  if (threadIdx.x == 0) bad |= (F.h.event_offsets[0] != 0ull) | (F.h.event_offsets[E] != F.h.n_hits);
  for (uint64_t e = threadIdx.x; e < E; e += blockDim.x) {
    const uint64_t a = F.h.event_offsets[e], b = F.h.event_offsets[e + 1];
    bad |= (b < a) | (b - a >= (1ull << kFwdIdBits));
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
__device__ __forceinline__ uint32_t fwd_layer_of(const uint32_t* lay, const float* x, uint32_t id) {
  return isfinite(x[id]) ? min(lay[id], kFwdL) : kFwdL;
}

struct FwdSmem {
  union {
    uint32_t cnt[radix_counters(kFwdThreads)];  // radix counters of the (layer, x) sort
    float xy[2 * kFwdSmemHits];                 // then x, y in sorted order (events that fit)
  } u;
  union {
    uint32_t cnt[radix_counters(kFwdThreads)];  // radix counters of the y sort
    struct {                                    // then the tracks of the current chunk
      float4 trk[kFwdThreads];                  // xm, ym, tx, ty
      uint32_t rlo[kFwdThreads][2];             // first entries of the candidate ranges in the y order
      uint32_t rn0[kFwdThreads];                // length of the layer-0 range
      uint32_t poff[kFwdThreads + 1];           // first pair of each track
      unsigned long long best[kFwdThreads];
    } c;
  } u2;
  // row q < kFwdL: first position of each x bucket of layer q (+ the layer's
  // end); rows kFwdL + r: first entry of each y bucket of layer r in the y order
  union {
    uint16_t s[kFwdRows][fwd_nb(true) + 1];
    uint32_t g[kFwdRows][fwd_nb(false) + 1];
  } tab;
  float vmin[kFwdRows], vinv[kFwdRows];  // bucket of v in row q: (v - vmin) * vinv, clamped
  uint32_t loff[kFwdL + 1];  // first position of each layer; [kFwdL] = end of the searched layers
  // layers 0 and 1 by y (candidate search): ypos holds (layer, x)-sorted
  // positions in (layer, finite y, y) order; yoff[2 r] .. yoff[2 r + 1] are
  // layer r's hits with a finite y
  uint32_t yoff[5];
  float dzm[kFwdL], dz0[kFwdL];  // z_L - z_mag, z_L - z_0
  float zm0, reach;              // z_mag - z_0; max(|z_mag - z_0|, z_11 - z_0)
  float wx[2];                   // candidate half-widths in x, layers 0 and 1
  uint32_t tmp[64];
  uint32_t nsv;                  // survivors of the current round
  uint32_t sv_pc[kFwdSurv];      // their sorted positions
  uint8_t sv_j[kFwdSurv];        // and tracks in the chunk
};

// four CTAs per SM: 228 KB of shared memory per SM, 1 KB of it reserved per CTA
static_assert(sizeof(FwdSmem) + 1024 <= 228 * 1024 / kFwdCtasPerSm, "shared memory for four CTAs per SM");
static_assert(kFwdSmemHits <= 65535u, "16-bit bucket tables");

template <bool SM>
__device__ __forceinline__ uint32_t fwd_bucket(float v, float vmin, float inv) {
  constexpr uint32_t NB = fwd_nb(SM);
  const float t = fm(fs(v, vmin), inv);  // monotone in v; NaN goes to bucket 0
  if (!(t >= 0.0f)) return 0u;
  if (t >= (float)NB) return NB - 1u;
  return (uint32_t)t;
}

template <bool SM>
__device__ __forceinline__ uint32_t tab_get(const FwdSmem& S, uint32_t row, uint32_t b) {
  if constexpr (SM) return S.tab.s[row][b];
  else return S.tab.g[row][b];
}

template <bool SM>
__device__ __forceinline__ void tab_set(FwdSmem& S, uint32_t row, uint32_t b, uint32_t v) {
  if constexpr (SM) S.tab.s[row][b] = (uint16_t)v;
  else S.tab.g[row][b] = v;
}

// first entry of row q at or after which every value >= v lies
template <bool SM>
__device__ __forceinline__ uint32_t tab_first(const FwdSmem& S, uint32_t row, float v) {
  return tab_get<SM>(S, row, fwd_bucket<SM>(v, S.vmin[row], S.vinv[row]));
}

// first entry of row q before which every value <= v lies
template <bool SM>
__device__ __forceinline__ uint32_t tab_past(const FwdSmem& S, uint32_t row, float v) {
  return tab_get<SM>(S, row, fwd_bucket<SM>(v, S.vmin[row], S.vinv[row]) + 1u);
}

// scale of row q's buckets over a sorted range [vmin, vmax]
template <bool SM>
__device__ __forceinline__ void fwd_bucket_scale(FwdSmem& S, uint32_t row, bool any, float vmin, float vmax) {
  const float span = fs(vmax, vmin);
  const float iv = any && span > 0.0f ? fd((float)fwd_nb(SM), span) : 0.0f;
  S.vmin[row] = any ? vmin : 0.0f;
  S.vinv[row] = isfinite(iv) ? iv : 0.0f;
}

// the sorted hits of one event
template <bool SM>
struct FwdEvent {
  const float* sx;      // x in sorted order (shared memory when SM, else global)
  const float* sy;
  const uint32_t* sid;  // hit id of each sorted position (global)
  const FwdSmem* S;
};

// nearest hit in x to xp (ties: the smaller id) with |x - xp| <= tol and
// |y - yp| <= tol_y in layer L; returns its sorted position or kNone
template <bool SM>
__device__ __forceinline__ uint32_t fwd_nearest(const FwdEvent<SM>& V, int L, float xp, float yp, float tol,
                                                float tol_y) {
  float lo_x, hi_x;
  fwd_range(xp, tol, &lo_x, &hi_x);
  const uint32_t end = V.S->loff[L + 1];
  uint32_t pos = tab_first<SM>(*V.S, L, lo_x);
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

// steps 3-5 for the candidate at sorted position pc of layer r of a track
// whose line reaches the kick plane at (xm, ym) with slope ty: false when a
// cut drops it
template <bool SM>
__device__ __forceinline__ bool fwd_candidate(const FwdEvent<SM>& V, const Fwd& F, float xm, float ym, float ty,
                                              int r, uint32_t pc, FwdCand& C) {
  const velo_forward_params_t& P = F.p;
  const FwdSmem& S = *V.S;
  const float tk = fd(fs(V.sx[pc], xm), S.dzm[r]);
  uint32_t n1 = 0;
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    C.hl[L] = fwd_nearest<SM>(V, L, fa(xm, fm(tk, S.dzm[L])), fa(ym, fm(ty, S.dzm[L])), P.tol_x, P.tol_y);
    n1 += C.hl[L] != kNone ? 1u : 0u;
  }
  if (n1 < 2) return false;
  float a1, b1;
  fwd_line(C.hl, V.sx, S.dz0, 0, 4, &a1, &b1);
  uint32_t n = n1;
#pragma unroll
  for (int L = 4; L < (int)kFwdL; ++L) {
    C.hl[L] = fwd_nearest<SM>(V, L, fa(a1, fm(b1, S.dz0[L])), fa(ym, fm(ty, S.dzm[L])), P.tol_x_far, P.tol_y);
    n += C.hl[L] != kNone ? 1u : 0u;
  }
  if (n < P.min_hits) return false;
  float a, b;
  fwd_line(C.hl, V.sx, S.dz0, 0, kFwdL, &a, &b);
  float chi2 = 0.0f;
#pragma unroll
  for (int L = 0; L < (int)kFwdL; ++L) {
    if (C.hl[L] == kNone) continue;
    const float res = fd(fs(fs(V.sx[C.hl[L]], a), fm(b, S.dz0[L])), P.sigma_x);
    chi2 = fa(chi2, fm(res, res));
  }
  const float rchi = fd(chi2, (float)(n - 2));
  if (!(rchi <= P.chi2ndf_max)) return false;
  const float d = fs(fa(a, fm(b, S.zm0)), xm);
  float ya, yb;
  fwd_line(C.hl, V.sy, S.dz0, 0, kFwdL, &ya, &yb);
  const float dy = fs(fa(ya, fm(yb, S.zm0)), ym);
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

// Step 3's first station for the candidate at sorted position pc of layer r,
// and a necessary condition for passing the match cut: false when the
// candidate certainly fails a cut.  The final x line is the least-squares
// line of the first-station hits and the far hits; written as the
// first-station line L1 (a1, b1) plus the least-squares line of the hits'
// offsets e_i from L1, its distance at the kick plane is d1 + sum w_i e_i,
// with d1 that of L1, w_i the fit's weights at the kick plane and |e_i| at
// most E = max(first-station residuals, tol_x_far).  So |d| <= tol_match
// needs |d1| <= tol_match + lam E, lam the largest sum |w_i| over the hit
// sets a candidate can end with (host arithmetic); the allowance
// 1 mm + 2e-3 M (M the size of the coordinates involved) covers the binary32
// rounding of both lines, its worst case being some 1e-4 M.
template <bool SM>
__device__ __forceinline__ bool fwd_first_station(const FwdEvent<SM>& V, const Fwd& F, float xm, float ym, float ty,
                                                  int r, uint32_t pc) {
  const velo_forward_params_t& P = F.p;
  const FwdSmem& S = *V.S;
  const float tk = fd(fs(V.sx[pc], xm), S.dzm[r]);
  uint32_t hl[4];
  uint32_t n1 = 0;
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    hl[L] = fwd_nearest<SM>(V, L, fa(xm, fm(tk, S.dzm[L])), fa(ym, fm(ty, S.dzm[L])), P.tol_x, P.tol_y);
    n1 += hl[L] != kNone ? 1u : 0u;
  }
  if (n1 < 2) return false;
  float a1, b1;
  fwd_line(hl, V.sx, S.dz0, 0, 4, &a1, &b1);
  float E = P.tol_x_far;
#pragma unroll
  for (int L = 0; L < 4; ++L)
    if (hl[L] != kNone) E = fmaxf(E, fabsf(fs(V.sx[hl[L]], fa(a1, fm(b1, S.dz0[L])))));
  const float M = fa(fa(fa(fabsf(a1), fm(fabsf(b1), S.reach)), fabsf(xm)), E);
  const float d1 = fs(fa(a1, fm(b1, S.zm0)), xm);
  return fabsf(d1) <= fa(fa(P.tol_match, fm(F.lam, E)), fa(1.0f, fm(2e-3f, M)));
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

// Steps 1 (after the sort by (layer, x)) to 3 of one event.
template <bool SM>
__device__ __forceinline__ void fwd_event(const Fwd& F, FwdSmem& S, uint64_t e, uint64_t t0, uint64_t t1, uint64_t h0,
                                          uint32_t n) {
  const uint32_t tid = threadIdx.x;
  const uint64_t cap = F.o.cap_tracks;
  const FwdWork& W = F.w;
  const uint32_t* lay = F.h.layer + h0;
  const float* xin = F.h.x + h0;
  const float* yin = F.h.y + h0;
  // sorted x, y, the sorted position of every id (into va, free after the
  // sort), the first position of every layer (a layer's slots after its
  // predecessor's layer get the position)
  float* sx = SM ? S.u.xy : W.sx + h0;
  float* sy = SM ? S.u.xy + kFwdSmemHits : W.sy + h0;
  const uint32_t* sid = W.vb + h0;
  uint32_t* pos_of = W.va + h0;
  for (uint32_t q = tid; q <= kFwdL; q += kFwdThreads) S.loff[q] = n;
  __syncthreads();
  for (uint32_t pos = tid; pos < n; pos += kFwdThreads) {
    const uint32_t id = sid[pos];
    sx[pos] = xin[id];
    sy[pos] = yin[id];
    pos_of[id] = pos;
    const uint32_t L = fwd_layer_of(lay, xin, id), Lp = pos ? fwd_layer_of(lay, xin, sid[pos - 1]) + 1u : 0u;
    for (uint32_t q = Lp; q <= L; ++q) S.loff[q] = pos;
  }
  __syncthreads();
  // layers 0 and 1 sorted by y: four passes over the ordered bits of y, one
  // over (layer, y not finite)
  const uint32_t n01 = S.loff[2];
  for (uint32_t pos = tid; pos < n01; pos += kFwdThreads) {
    W.yka[h0 + pos] = ordered_bits(sy[pos]);
    W.yva[h0 + pos] = pos;
  }
  __syncthreads();
  const uint32_t l1 = S.loff[1];
  auto ydig = [sy, l1](uint32_t, uint32_t pos) { return (pos >= l1 ? 2u : 0u) + (isfinite(sy[pos]) ? 0u : 1u); };
  radix_pass<kFwdThreads, true>(W.yka + h0, W.ykb + h0, W.yva + h0, W.yvb + h0, n01,
                                [](uint32_t k, uint32_t) { return k & 255u; }, S.u2.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.ykb + h0, W.yka + h0, W.yvb + h0, W.yva + h0, n01,
                                [](uint32_t k, uint32_t) { return (k >> 8) & 255u; }, S.u2.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.yka + h0, W.ykb + h0, W.yva + h0, W.yvb + h0, n01,
                                [](uint32_t k, uint32_t) { return (k >> 16) & 255u; }, S.u2.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.ykb + h0, W.yka + h0, W.yvb + h0, W.yva + h0, n01,
                                [](uint32_t k, uint32_t) { return k >> 24; }, S.u2.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.yka + h0, W.ykb + h0, W.yva + h0, W.yvb + h0, n01, ydig, S.u2.cnt, S.tmp);
  const uint32_t* ypos = W.yvb + h0;
  for (uint32_t q = tid; q < 5; q += kFwdThreads) S.yoff[q] = n01;
  __syncthreads();
  for (uint32_t i = tid; i < n01; i += kFwdThreads) {
    const uint32_t g = ydig(0u, ypos[i]), gp = i ? ydig(0u, ypos[i - 1]) + 1u : 0u;
    for (uint32_t q = gp; q <= g; ++q) S.yoff[q] = i;
  }
  __syncthreads();
  // bucket tables: x of every layer over its span, y of layers 0 and 1 over theirs
  constexpr uint32_t NB = fwd_nb(SM);
  const float zmag = F.g.z_mag;
  if (tid < kFwdL) {
    const uint32_t lo = S.loff[tid], hi = S.loff[tid + 1];
    fwd_bucket_scale<SM>(S, tid, hi > lo, hi > lo ? sx[lo] : 0.0f, hi > lo ? sx[hi - 1] : 0.0f);
    const float z = F.g.z_layers[tid];
    S.dzm[tid] = fs(z, zmag);
    S.dz0[tid] = fs(z, F.g.z_layers[0]);
  } else if (tid >= 32 && tid < 34) {
    const uint32_t r = tid - 32, lo = S.yoff[2 * r], hi = S.yoff[2 * r + 1];
    fwd_bucket_scale<SM>(S, kFwdL + r, hi > lo, hi > lo ? sy[ypos[lo]] : 0.0f, hi > lo ? sy[ypos[hi - 1]] : 0.0f);
  } else if (tid == 64) {
    S.zm0 = fs(zmag, F.g.z_layers[0]);
    S.reach = fmaxf(fabsf(S.zm0), fs(F.g.z_layers[kFwdL - 1], F.g.z_layers[0]));
  } else if (tid >= 96 && tid < 98) {
    S.wx[tid - 96] = fa(fm(fd(F.g.kappa, F.p.p_min), fs(F.g.z_layers[tid - 96], zmag)), F.p.tol_x);
  }
  for (uint32_t i = tid; i < kFwdRows * (NB + 1); i += kFwdThreads) {
    const uint32_t q = i / (NB + 1);  // entries past a row's last value: the row's end
    tab_set<SM>(S, q, i % (NB + 1), q < kFwdL ? S.loff[q + 1] : S.yoff[2 * (q - kFwdL) + 1]);
  }
  __syncthreads();
  for (uint32_t pos = tid; pos < S.loff[kFwdL]; pos += kFwdThreads) {
    uint32_t L = 0;
    while (S.loff[L + 1] <= pos) ++L;
    const uint32_t b = fwd_bucket<SM>(sx[pos], S.vmin[L], S.vinv[L]);
    const uint32_t bp = pos > S.loff[L] ? fwd_bucket<SM>(sx[pos - 1], S.vmin[L], S.vinv[L]) + 1u : 0u;
    for (uint32_t q = bp; q <= b; ++q) tab_set<SM>(S, L, q, pos);
  }
  for (uint32_t r = 0; r < 2; ++r)
    for (uint32_t i = S.yoff[2 * r] + tid; i < S.yoff[2 * r + 1]; i += kFwdThreads) {
      const uint32_t q = kFwdL + r;
      const uint32_t b = fwd_bucket<SM>(sy[ypos[i]], S.vmin[q], S.vinv[q]);
      const uint32_t bp = i > S.yoff[2 * r] ? fwd_bucket<SM>(sy[ypos[i - 1]], S.vmin[q], S.vinv[q]) + 1u : 0u;
      for (uint32_t b2 = bp; b2 <= b; ++b2) tab_set<SM>(S, q, b2, i);
    }
  __syncthreads();
  const FwdEvent<SM> V{sx, sy, sid, &S};
  // 2.-3. the tracks, kFwdThreads at a time
  for (uint64_t tc = t0; tc < t1; tc += kFwdThreads) {
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
        S.u2.c.trk[tid] = make_float4(xm, ym, tx, ty);
        live = true;
        // 2. ranges of the y order holding the candidate windows of layers 0 and 1
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          float lo_y, hi_y;
          fwd_range(fa(ym, fm(ty, S.dzm[r])), F.p.win_y, &lo_y, &hi_y);
          const uint32_t lo = tab_first<SM>(S, kFwdL + r, lo_y);
          const uint32_t hi = tab_past<SM>(S, kFwdL + r, hi_y);
          S.u2.c.rlo[tid][r] = lo;
          const uint32_t len = hi > lo ? hi - lo : 0u;
          if (r == 0) S.u2.c.rn0[tid] = len;
          cnt += len;
        }
      } else {
        fwd_write_none(F, t);
      }
    }
    S.u2.c.best[tid] = ~0ull;
    uint32_t total;
    const uint32_t first = block_exclusive_scan<kFwdThreads, uint32_t>(cnt, &total, S.tmp);
    S.u2.c.poff[tid] = first;
    if (tid == 0) S.u2.c.poff[kFwdThreads] = total;
    __syncthreads();
    // the (track, candidate) pairs, shared out evenly, kFwdSurv at a time:
    // the window test, the first station and the bound, the survivors listed;
    // then the survivors' far stations, fits and cuts
    for (uint32_t q0 = 0; q0 < total; q0 += kFwdSurv) {
      if (tid == 0) S.nsv = 0;
      __syncthreads();
      for (uint32_t q = q0 + tid; q < min(total, q0 + kFwdSurv); q += kFwdThreads) {
        uint32_t lo = 0, hi = kFwdThreads;  // the track j with poff[j] <= q < poff[j + 1]
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (S.u2.c.poff[mid] <= q) lo = mid;
          else hi = mid;
        }
        const uint32_t j = lo, k = q - S.u2.c.poff[j];
        const int r = k < S.u2.c.rn0[j] ? 0 : 1;
        const uint32_t pc = ypos[S.u2.c.rlo[j][r] + (r ? k - S.u2.c.rn0[j] : k)];
        const float4 tr = S.u2.c.trk[j];
        if (!(fabsf(fs(sx[pc], fa(tr.x, fm(tr.z, S.dzm[r])))) <= S.wx[r]) ||
            !(fabsf(fs(sy[pc], fa(tr.y, fm(tr.w, S.dzm[r])))) <= F.p.win_y))
          continue;
        if (!fwd_first_station<SM>(V, F, tr.x, tr.y, tr.w, r, pc)) continue;
        const uint32_t slot = atomicAdd(&S.nsv, 1u);
        S.sv_pc[slot] = pc;
        S.sv_j[slot] = (uint8_t)j;
      }
      __syncthreads();
      const uint32_t nsv = S.nsv;
      for (uint32_t i = tid; i < nsv; i += kFwdThreads) {
        const uint32_t pc = S.sv_pc[i], j = S.sv_j[i];
        const float4 tr = S.u2.c.trk[j];
        FwdCand C;
        if (fwd_candidate<SM>(V, F, tr.x, tr.y, tr.w, pc < S.loff[1] ? 0 : 1, pc, C))
          atomicMin(&S.u2.c.best[j], fwd_key(C.n, C.ad, sid[pc]));
      }
      __syncthreads();
    }
    // 3. the winner of every track, recomputed and written
    if (live) {
      const unsigned long long key = S.u2.c.best[tid];
      if (key == ~0ull) {
        fwd_write_none(F, t);
      } else {
        const uint32_t pc = pos_of[(uint32_t)(key & ((1ull << kFwdIdBits) - 1ull))];
        const float4 tr = S.u2.c.trk[tid];
        FwdCand C;
        fwd_candidate<SM>(V, F, tr.x, tr.y, tr.w, pc < S.loff[1] ? 0 : 1, pc, C);
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

// One CTA per event; the instance with SM = true takes the events whose hits
// fit in shared memory, the other the rest (a CTA of the wrong instance
// returns at once).
template <bool SM>
__global__ void __launch_bounds__(kFwdThreads, kFwdCtasPerSm) k_forward(Fwd F) {
  extern __shared__ __align__(16) uint8_t fwd_smem_raw[];
  FwdSmem& S = *reinterpret_cast<FwdSmem*>(fwd_smem_raw);
  const uint64_t e = blockIdx.x;
  const uint32_t tid = threadIdx.x;
  const uint32_t flag = *(const volatile uint32_t*)F.w.flag;
  if (flag & kFwdNoTracks) return;  // no track lists to read: nothing is written
  const uint64_t t0 = F.t.track_offsets[e], t1 = F.t.track_offsets[e + 1];
  if (flag & kFwdBadOffsets) {      // hits rejected: no track has a downstream track
    if (SM)
      for (uint64_t t = t0 + tid; t < t1 && t < F.o.cap_tracks; t += kFwdThreads) fwd_write_none(F, t);
    return;
  }
  const uint64_t h0 = F.h.event_offsets[e];
  const uint32_t n = (uint32_t)(F.h.event_offsets[e + 1] - h0);
  if ((n <= kFwdSmemHits) != SM) return;
  const FwdWork& W = F.w;
  // 1. sort by (layer, x): four passes over the ordered bits of x, one over the layer
  for (uint32_t i = tid; i < n; i += kFwdThreads) {
    W.ka[h0 + i] = ordered_bits(F.h.x[h0 + i]);
    W.va[h0 + i] = i;
  }
  __syncthreads();
  const uint32_t* lay = F.h.layer + h0;
  const float* xin = F.h.x + h0;
  radix_pass<kFwdThreads, true>(W.ka + h0, W.kb + h0, W.va + h0, W.vb + h0, n,
                                [](uint32_t k, uint32_t) { return k & 255u; }, S.u.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.kb + h0, W.ka + h0, W.vb + h0, W.va + h0, n,
                                [](uint32_t k, uint32_t) { return (k >> 8) & 255u; }, S.u.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.ka + h0, W.kb + h0, W.va + h0, W.vb + h0, n,
                                [](uint32_t k, uint32_t) { return (k >> 16) & 255u; }, S.u.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.kb + h0, W.ka + h0, W.vb + h0, W.va + h0, n,
                                [](uint32_t k, uint32_t) { return k >> 24; }, S.u.cnt, S.tmp);
  radix_pass<kFwdThreads, true>(W.ka + h0, W.kb + h0, W.va + h0, W.vb + h0, n,
                                [lay, xin](uint32_t, uint32_t id) { return fwd_layer_of(lay, xin, id); }, S.u.cnt,
                                S.tmp);
  fwd_event<SM>(F, S, e, t0, t1, h0, n);
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
  F.lam = fwd_lambda(*geometry, p.min_hits);
  F.h = *hits;
  F.t = *tracks;
  F.g = *geometry;
  F.p = *params;
  F.o = *out;
  if (fwd_carve(static_cast<uint8_t*>(workspace), hits->n_hits, &F.w) > workspace_bytes) return VELO_ECAPACITY;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!set_max_smem_once(reinterpret_cast<const void*>(k_forward<true>), 2) ||
      !set_max_smem_once(reinterpret_cast<const void*>(k_forward<false>), 3))
    return VELO_ECUDA;
  k_fwd_validate<<<1, 1024, 0, s>>>(F);
  if (hits->n_events) {
    k_forward<true><<<(uint32_t)hits->n_events, kFwdThreads, sizeof(FwdSmem), s>>>(F);
    k_forward<false><<<(uint32_t)hits->n_events, kFwdThreads, sizeof(FwdSmem), s>>>(F);
  }
  return cudaGetLastError() == cudaSuccess ? VELO_OK : VELO_ECUDA;
}

}  // extern "C"
