// Pattern recognition, fit and output kernels.
//
// The first stage's "simplified pattern recognition" (Sec. "HLT1 details and
// results") is realised as search by triplet + forward extension, run per
// event from the most downstream module to the most upstream one.  At step m
// (m = M-2 .. 0):
//   extension  every active track whose last hit sits on module l > m and
//              that has missed at most max_skipped modules extrapolates the
//              line through its last two hits to module m and takes the
//              unused hit within the pseudo-angle window and the scatter cut
//              with the smallest (d^2, id); several tracks on one hit -> the
//              smallest (bits(d^2), track index) wins (64-bit atomicMin, so
//              the outcome does not depend on thread order);
//   seeding    (m >= 1) every unused hit h1 on m takes the (h0 on m+1 unused,
//              h2 on m-1) pair inside the windows, slope and scatter cuts with
//              the smallest (s, id0, id2) -- the pairs of all h1 are spread
//              evenly over the block as (h1, h0) work items; a seed claims h0
//              and h2 with (bits(s), id1) and survives if it holds both claims;
//              survivors become tracks in the order of h1 (block scan).
// Then every track is fitted (straight line + simplified Kalman), cut on
// chi2/ndf (or, in the learned form, scored by the ghost-rejection network on
// tensor cores), and ranked canonically by its smallest cluster id.
//
// One CTA of NT threads (128 or 256) per event;
// the event's hits stay in the global workspace (sorted by module,
// pseudo-angle key, id; L1/L2 resident), the per-step claims and used flags too.
#include "velo_device.cuh"
#include "velo_fit.cuh"
#include "velo_internal.cuh"
#include "velo_mlp.cuh"

#include <cooperative_groups.h>
#include <cstddef>
#include <mutex>

namespace velo {

namespace {

// middle hits per seeding chunk (a multiple of the block size)
template <int NT>
__host__ __device__ constexpr uint32_t seed_chunk() {
  return NT > 512 ? (uint32_t)NT : 512u;
}

// Events with at least kWideClusters clusters (heavy-ion-like) are tracked
// by clusters of CTAs of kWideThreads threads, the others by the tuned block
// size.
constexpr int kWideThreads = 1024;
// CTAs (a thread-block cluster) per heavy event: every CTA runs the module
// loop; the parallel loops of a step are shared out over the cluster's
// threads and a cluster barrier orders their global-memory results.  16 (a
// non-portable size) where the device can place such a cluster, else the
// portable 8; the kernel reads the size at run time.
constexpr uint32_t kWideClusterMax = 16, kWideClusterPortable = 8;
// Heavy events seed through a grid of the h2 module's hits in the plane of
// their u terms (the per-hit half of the seeding's pre-test, u = (1 - a')
// (x2, y2)): kGridSide^2 cells over the sensor, for modules of up to kGridCap
// hits; the next step's extension into that module reads the same grid.
// Every CTA of the cluster keeps its own copy in the dynamic shared memory of
// k_track_wide: the u terms in cell order (2 f32), the cell starts (u16: a
// module has at most kGridCap hits; counted two to a 32-bit word), the
// hits' module-local indices in cell order (u16), and the used flags of the
// h0 and h1 modules (1 bit each), so that the triplet loop reads none of them
// from another SM through L2.
constexpr uint32_t kGridSide = 128, kGridCells = kGridSide * kGridSide, kGridCap = 8192;
constexpr uint32_t kGridOffAt = kGridCap * 8u, kGridIdAt = kGridOffAt + (kGridCells + 2u) * 2u,
                   kGridUsedAt = kGridIdAt + kGridCap * 2u, kGridUsed1At = kGridUsedAt + kGridCap / 8u,
                   kGridNextAt = kGridUsed1At + kGridCap / 8u, kGridBytes = kGridNextAt + 16u;
static_assert(kGridIdAt % 4 == 0 && kGridUsedAt % 4 == 0, "grid arrays aligned");

template <uint32_t C>
struct SeedArrays {
  uint2 r0[C];                // h0 window: two module-local index ranges, 16-bit ends packed
  uint2 r2[C];                // h2 window
  uint32_t ioff[C];           // first work item of each middle hit
  unsigned long long best[C]; // smallest (bits(s), id0, id2) key of each middle hit
};

// module-local ranges (< 2^16: a module holds at most VELO_MAX_MODULE_CLUSTERS hits)
__device__ __forceinline__ uint2 pack_ranges(const Ranges& r, uint32_t lo) {
  return make_uint2((r.a0 - lo) | (r.a1 - lo) << 16, (r.b0 - lo) | (r.b1 - lo) << 16);
}
__device__ __forceinline__ Ranges unpack_ranges(uint2 v, uint32_t lo) {
  return Ranges{lo + (v.x & 0xFFFFu), lo + (v.x >> 16), lo + (v.y & 0xFFFFu), lo + (v.y >> 16)};
}

template <int NT>
struct TrackSmem {
  uint16_t ktab[3][kKeyBuckets + 1];  // bucketed key index of the modules a step reads, module j in j % 3
  uint32_t mod_off[kModOffStride];
  float z[VELO_MAX_MODULES];
  alignas(16) uint32_t tmp[64];  // (also read as 64-bit scan words)
  SeedArrays<seed_chunk<NT>()> sd;
};
static_assert(offsetof(TrackSmem<256>, tmp) % 8 == 0 && offsetof(TrackSmem<128>, tmp) % 8 == 0,
              "the scan buffer holds 64-bit words");

constexpr int kFitThreads = 256;
constexpr int kFitWideThreads = 1024;  // the fit of the heavy-ion-like events (thousands of tracks)
// Events of up to this many tracks have their kept tracks ranked in shared
// memory by the fit (a count of smaller first ids); larger ones through the
// id -> track map over all the event's ids.
constexpr uint32_t kRankCap = 1024;
static_assert(VELO_STATE_STRIDE % 4 == 0, "states move in 16-byte pieces");

template <int NT>
struct FitSmem {
  uint32_t hit_fill;  // hit ids of the event's tracks staged so far (on a cluster: rank 0's)
  unsigned long long cta_counts;  // (on a cluster) this CTA's kept tracks << 32 | their hits
  uint32_t n_kept;                // (kRankCap tracks or fewer) kept tracks so far
  uint32_t rkey[kRankCap];        // their first cluster id << 11 | track index
  uint16_t rtrk[kRankCap];        // the track of each rank
  uint8_t rnh[kRankCap];          // its hits
  uint32_t mod_off[kModOffStride];
  float z[VELO_MAX_MODULES];
  unsigned long long tmp64[64];
  MlpWeights mlp;
  MlpTiles tiles[NT / 32];
};

// the caller's output buffers hold the batch (capacity 0 = as velo_query_sizes)
__device__ __forceinline__ bool output_fits(const velo_output_t& o, uint64_t nc, uint64_t nt, uint64_t nh) {
  return (!o.cap_clusters || nc <= o.cap_clusters) && (!o.cap_tracks || nt <= o.cap_tracks) &&
         (!o.cap_track_hits || nh <= o.cap_track_hits);
}

__device__ __forceinline__ uint32_t fbits(float f) { return __float_as_uint(f); }

__device__ __forceinline__ uint32_t module_of_pos(const uint32_t* mod_off, uint32_t M, uint32_t pos) {
  uint32_t lo = 0, hi = M;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (mod_off[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}

// hits of track t, ascending in z (upstream first), into x/y/z (+ modules,
// cluster ids when asked); returns n
__device__ __forceinline__ uint32_t gather_track(const Workspace& W, uint64_t p0, uint64_t tb, uint32_t t,
                                                 const uint32_t* mod_off, const float* mz, uint32_t M, float* xs,
                                                 float* ys, float* zs, uint32_t* mods, uint32_t* ids) {
  const uint32_t n = W.trk_meta[tb + t] & 255u;
  uint32_t p = W.trk_a[tb + t];
  for (uint32_t j = 0; j < n; ++j) {
    const uint32_t m = module_of_pos(mod_off, M, p);
    const float4 h = W.hit[p0 + p];
    xs[j] = h.x;
    ys[j] = h.y;
    zs[j] = mz[m];
    mods[j] = m;
    if (ids) ids[j] = __float_as_uint(h.w);
    p = W.sc[p0 + p];  // link to the next hit downstream
  }
  return n;
}

// Windows with more candidates than this are narrowed by position first
// (dense events); below it the bound costs more than it saves.
constexpr uint32_t kNarrowAbove = 16;

// Candidate ranges narrowed by position.  A hit that can pass a cut of
// radius `reach` (mm) around the point (xc, yc) lies within reach of it, so
// its azimuth differs by at most asin(reach / r) <= (pi/2) reach / r from the
// point's (r = |(xc, yc)| > reach), and its pseudo-angle -- whose slope in the
// azimuth is between 1/2 and 1 -- by no more.  When that bound is tighter than
// the window `win`, the ranges around the point's own key replace
// the window's; the exact window and cut tests still run on every candidate,
// so only hits that would fail them are skipped.
__device__ __forceinline__ Ranges narrowed_ranges(const KeyIndex& I, float win, const Ranges& wide, float xc, float yc,
                                                  float reach) {
  const float r = sqrtf(xc * xc + yc * yc);
  if (!(r > 2.0f * reach)) return wide;
  const float half = 1.5708f * reach / r * 1.01f + 1e-4f;
  if (!(half < win)) return wide;
  return window_ranges(I, pseudo_angle(xc, yc), half);
}

// A claim on a hit at module step m: the step in the top five bits, then the
// claim's value (the bits of a non-negative binary32, which order as the
// values) and a 28-bit index (a track index or cluster id: below 2^21, as an
// event holds at most 32 x 65535 clusters).  Steps run downwards, so a claim of
// step m is smaller than any left by an earlier step and the claims need no
// reset between steps; within a step the order is the method's (value, index).
__device__ __forceinline__ unsigned long long step_key(uint32_t m, uint32_t value_bits, uint32_t index) {
  return (unsigned long long)m << 59 | (unsigned long long)value_bits << 28 | index;
}

// chi2/ndf of the cut: straight-line chi2 without scattering, Kalman chi2 with it
__device__ __forceinline__ float cut_chi2ndf(uint32_t n, const float* st, float theta) {
  return fd(theta == 0.0f ? st[6] : st[7], (float)(2 * n - 4));
}

}  // namespace

// Loads of workspace values another CTA of the cluster may have written
// (WIDE): from L2, past this SM's L1, which is not kept coherent with the
// other SMs' writes.
template <bool L2ONLY, class T>
__device__ __forceinline__ T ldx(const T* p) {
  if constexpr (L2ONLY) return __ldcg(p);
  else return *p;
}

// WIDE: this instance tracks the events of kWideClusters clusters or more
// (and only those); the other instance every other event.
template <int NT, bool WIDE>
__device__ __forceinline__ void track_one(const Launch& L, const uint64_t e, TrackSmem<NT>& S, uint8_t* gsm) {
  const Workspace& W = L.ws;
  const uint32_t tid = threadIdx.x;
  const Par P = L.par;  // by value: kept in registers, not re-read through a reference
  const uint32_t M = L.geo.n_modules;
  // the threads that share the event: this CTA, or (WIDE) its cluster
  uint32_t CS = 1, rank = 0;
  if constexpr (WIDE) {
    CS = cooperative_groups::this_cluster().num_blocks();
    rank = cooperative_groups::this_cluster().block_rank();
  }
  const uint32_t gt = rank * NT + tid, GT = CS * NT;
  // (WIDE) the cluster barrier releases each CTA's writes and acquires the
  // others' at cluster scope; reads of the other CTAs' workspace values go
  // through L2 (ldx)
  auto bar = [&]() {
    if constexpr (WIDE) cooperative_groups::this_cluster().sync();
    else __syncthreads();
  };
  // largest |x| or |y| of a hit (centroids lie on the sensor: x0 .. x0 + pitch n_cols)
  const float coord_max = fmaxf(fmaxf(fabsf(L.geo.x0), fabsf(L.geo.x0 + L.geo.pitch * (float)L.geo.n_cols)),
                                fmaxf(fabsf(L.geo.y0), fabsf(L.geo.y0 + L.geo.pitch * (float)L.geo.n_rows)));

  if (*(const volatile uint32_t*)W.flag != 0u || L.out.status[e] != VELO_EVT_OK) {
    if (!WIDE && tid == 0) {
      W.ev_ntracks_all[e] = 0;
      W.ev_ntracks[e] = 0;
      W.ev_nhits[e] = 0;
    }
    return;
  }
  if ((W.ev_nclusters[e] >= kWideClusters) != WIDE) return;
  const uint64_t p0 = L.off[e];
  const uint64_t tb = p0 / 3;
  const uint32_t H = W.ev_nclusters[e];
  const uint32_t track_cap = (uint32_t)((L.off[e + 1] - p0) / 3);
  if (tid < kModOffStride) S.mod_off[tid] = W.ev_modoff[e * kModOffStride + tid];
  if (tid < VELO_MAX_MODULES) S.z[tid] = L.geo.z[tid];

  const float4* hit = W.hit + p0;  // x, y, key, id bits
  uint8_t* used = W.used + p0;
  uint32_t* prev = W.sc + p0;
  uint32_t* first_of = W.sd + p0;
  uint32_t* seed_h0 = W.sa + p0;
  uint32_t* seed_h2 = W.sb + p0;
  unsigned long long* claim = W.acc + p0;
  unsigned long long* seedkey = W.acc + L.n_pixels + p0;
  uint32_t* meta = W.trk_meta + tb;
  uint32_t* ta = W.trk_a + tb;
  uint32_t* tbk = W.trk_b + tb;
  uint32_t* pick = W.trk_pick + tb;
  unsigned long long* pick_key = W.trk_pick_key + tb;

  for (uint32_t i = gt; i < H; i += GT) {
    used[i] = 0;
    if (WIDE) first_of[i] = kNone;  // (see the end: only events of many tracks need it)
    claim[i] = ~0ull;  // claims carry their step (step_key): no reset between steps
  }
  bar();  // mod_off
  // bucketed key index of module j into slot j % 3, without a barrier: every
  // entry is written once -- each hit fills the buckets from its predecessor's
  // (exclusive) to its own, the last hit the ones after its own with the count
  auto index_module = [&](uint32_t j) {
    const uint32_t lo = S.mod_off[j], n = S.mod_off[j + 1] - lo;
    uint16_t* tab = S.ktab[j % 3u];
    if (n == 0u) {
      for (uint32_t q = tid; q <= kKeyBuckets; q += NT) tab[q] = 0;
      return;
    }
    for (uint32_t i = tid; i < n; i += NT) {
      const uint32_t b = key_bucket(hit[lo + i].z), b0 = i ? key_bucket(hit[lo + i - 1].z) + 1u : 0u;
      for (uint32_t q = b0; q <= b; ++q) tab[q] = (uint16_t)i;
      if (i + 1u == n)
        for (uint32_t q = b + 1u; q <= kKeyBuckets; ++q) tab[q] = (uint16_t)n;
    }
  };
  index_module(M - 1);
  index_module(M - 2);
  __syncthreads();

  // (heavy events) the grid in the dynamic shared memory, built at step m
  // for the seeding's h2 module m - 1 and read again by the extension into
  // that module at step m - 1 (grid_m: the grid holds module m's hits).  A
  // hit's cell and a query box's cells come from one monotone function of
  // the coordinate, so every u inside a box lies in the box's cells.
  float2* gu = WIDE ? reinterpret_cast<float2*>(gsm) : nullptr;
  uint16_t* goff = WIDE ? reinterpret_cast<uint16_t*>(gsm + kGridOffAt) : nullptr;
  // adds 1 to goff[c] (two entries to a 32-bit word; no entry exceeds
  // kGridCap, so no carry crosses) and returns its old value
  auto goff_inc = [&](uint32_t c) -> uint32_t {
    const uint32_t sh = (c & 1u) * 16u;
    return (atomicAdd(reinterpret_cast<uint32_t*>(goff) + (c >> 1), 1u << sh) >> sh) & 0xFFFFu;
  };
  uint16_t* gid = WIDE ? reinterpret_cast<uint16_t*>(gsm + kGridIdAt) : nullptr;
  bool grid_m = false;
  float g_lo = 0.0f, g_inv = 0.0f, g_oma = 0.0f;
  auto gcell = [&](float v) -> uint32_t {
    const float t = fm(fs(v, g_lo), g_inv);
    return !(t > 0.0f) ? 0u : (t >= (float)kGridSide ? kGridSide - 1u : (uint32_t)t);
  };

  uint32_t n_tr = 0;
  for (int m = (int)M - 2; m >= 0; --m) {
    if (m >= 1) index_module((uint32_t)m - 1u);  // its slot held module m + 2, done with at step m + 1
    // ---- extension into module m (against the used flags of the step start);
    // a hit within the cut lies within sqrt(max_scatter_fwd) of the prediction
    const float fwd_reach = sqrtf(P.max_scatter_fwd) * 1.01f + 1e-3f;
    const float zm = S.z[m];
    const uint32_t mlo = S.mod_off[m], mhi = S.mod_off[m + 1];
    for (uint32_t t = gt; t < n_tr; t += GT) {
      const uint32_t mt = ldx<WIDE>(meta + t);
      uint32_t pk = kNone;
      if (mt & kTrkActive) {
        const int la = (int)((mt >> 16) & 255u), lb = (int)(mt >> 24);
        if (la - m - 1 > (int)P.max_skipped) {
          meta[t] = mt & ~kTrkActive;
        } else if (la > m) {
          const uint32_t a = ldx<WIDE>(ta + t), b = ldx<WIDE>(tbk + t);
          const float4 A = hit[a], B = hit[b];
          const float xa = A.x, ya = A.y, ka = A.z, xb = B.x, yb = B.y;
          const float za = S.z[la], zb = S.z[lb];
          const float dzab = fs(za, zb);
          const float tx = fd(fs(xa, xb), dzab), ty = fd(fs(ya, yb), dzab);
          const float dzm = fs(zm, za);
          const float xp = fa(xa, fm(tx, dzm)), yp = fa(ya, fm(ty, dzm));
          unsigned long long best = ~0ull;
          bool searched = false;
          if constexpr (WIDE) {
            if (grid_m) {
              // the hits of the grid cells around the prediction, scaled to the
              // grid's plane: a hit within the cut lies within |1 - a'| fwd_reach
              // of it there (+ the roundings of the two products, far below
              // the margin of bx); the exact tests decide as below
              const float ucx = fm(g_oma, xp), ucy = fm(g_oma, yp);
              const float bx = fabsf(g_oma) * fwd_reach * 1.001f + 1e-4f, bx2 = bx * bx;
              const uint32_t cx0 = gcell(fs(ucx, bx)), cx1 = gcell(fa(ucx, bx));
              for (uint32_t cy = gcell(fs(ucy, bx)), cy1 = gcell(fa(ucy, bx)); cy <= cy1; ++cy) {
                const uint32_t s1 = goff[cy * kGridSide + cx1 + 1u];  // cells cx0 .. cx1 of the row are adjacent
                for (uint32_t sl = goff[cy * kGridSide + cx0]; sl < s1; ++sl) {
                  const float2 u = gu[sl];
                  const float ex = fs(u.x, ucx), ey = fs(u.y, ucy);
                  if (fa(fm(ex, ex), fm(ey, ey)) > bx2) continue;
                  const uint32_t pos = mlo + gid[sl];
                  const float4 h = hit[pos];
                  const float dx = fs(xp, h.x), dy = fs(yp, h.y);
                  const float d2 = fa(fm(dx, dx), fm(dy, dy));
                  if (d2 > P.max_scatter_fwd) continue;
                  if (ldx<WIDE>(used + pos)) continue;
                  if (dmod4(h.z, ka) > P.win_fwd) continue;
                  const unsigned long long cand = (unsigned long long)fbits(d2) << 32 | fbits(h.w);
                  if (cand < best) {
                    best = cand;
                    pk = pos;
                  }
                }
              }
              searched = true;
            }
          }
          if (!searched) {
            const KeyIndex Im{mlo, S.ktab[m % 3]};
            Ranges R = window_ranges(Im, ka, P.win_fwd);
            if ((R.a1 - R.a0) + (R.b1 - R.b0) > kNarrowAbove) R = narrowed_ranges(Im, P.win_fwd, R, xp, yp, fwd_reach);
            for (int part = 0; part < 2; ++part) {
              const uint32_t s = part ? R.b0 : R.a0, en = part ? R.b1 : R.a1;
              for (uint32_t pos = s; pos < en; ++pos) {  // the cut first: few candidates pass it
                const float4 h = hit[pos];
                const float dx = fs(xp, h.x), dy = fs(yp, h.y);
                const float d2 = fa(fm(dx, dx), fm(dy, dy));
                if (d2 > P.max_scatter_fwd) continue;
                if (ldx<WIDE>(used + pos)) continue;
                if (dmod4(h.z, ka) > P.win_fwd) continue;
                const unsigned long long cand = (unsigned long long)fbits(d2) << 32 | fbits(h.w);
                if (cand < best) {
                  best = cand;
                  pk = pos;
                }
              }
            }
          }
          if (pk != kNone) {
            const unsigned long long key = step_key((uint32_t)m, (uint32_t)(best >> 32), t);
            pick_key[t] = key;
            atomicMin(claim + pk, key);
          }
        }
      }
      pick[t] = pk;
    }
    bar();
    for (uint32_t t = gt; t < n_tr; t += GT) {
      const uint32_t pk = pick[t];
      if (pk == kNone || ldx<WIDE>(claim + pk) != pick_key[t]) continue;
      const uint32_t mt = meta[t];
      const uint32_t n = mt & 255u, la = (mt >> 16) & 255u;
      prev[pk] = ta[t];
      tbk[t] = ta[t];
      ta[t] = pk;
      meta[t] = (n + 1u) | kTrkActive | ((uint32_t)m << 16) | (la << 24);
      used[pk] = 1;
    }
    bar();
    if (m == 0) break;

    // ---- seeding with the middle hit on m.  The (h0, h2) pairs of all middle
    // hits are spread evenly over the block: one work item per (h1, h0
    // candidate), each looping over h1's h2 window, in chunks of kChunk
    // middle hits; per h1 the smallest pair key wins (shared 64-bit atomicMin).
    const uint32_t lo0 = S.mod_off[m + 1], hi0 = S.mod_off[m + 2];
    const uint32_t lo2 = S.mod_off[m - 1], hi2 = mlo;
    const float z0 = S.z[m + 1], z2 = S.z[m - 1];
    const float dz02 = fs(z0, z2), dz12 = fs(zm, z2);
    // The seed's point at z1 is x2 + (x0 - x2) dz12/dz02 = (1 - a) x2 + a x0, so a
    // h2 that passes the scatter cut lies within seed_reach of
    // ((x1, y1) - a (x0, y0)) / (1 - a): its distance to that point is the seed
    // point's distance to h1 divided by (1 - a), so at most sqrt(max) / (1 - a).
    const float alpha = dz12 / dz02, one_m_alpha = 1.0f - alpha;
    const bool seed_narrow = one_m_alpha > 0.05f && one_m_alpha < 0.95f;
    const float seed_reach = seed_narrow ? sqrtf(P.max_scatter_seed) / one_m_alpha * 1.01f + 1e-3f : 0.0f;
    // Division-free pre-test of the scatter cut.  The seed's residual at z1 is
    // D = (1 - a) x2 + a x0 - x1 with a = dz12 / dz02; the pre-test uses
    // a' = rcp(dz02) dz12 and dx' = (1 - a') x2 + (a' x0 - x1), the first term
    // computed once per hit of module m - 1 and the second once per (h1, h0).
    // With u = 2^-24, S the slope cut, X the largest |coordinate| of a hit on
    // the sensor and r = sqrt(scatter cut): |a' - a| <= 2u a, so for a triplet
    // that passes the exact slope cut the a' error moves D by at most
    // 2u S dz12, and the roundings of the pre-test by at most 5u X + u r;
    // the exact chain (quotient, product with dz12, two sums) stays within
    // 5u S dz12 + 2u (X + r) + 2u r of D.  So for a triplet that passes the
    // exact cuts |dx' - dx|, |dy' - dy| <= 8u (S |dz12| + 2 X + 2 r + 1) =: err
    // and dx'^2 + dy'^2 is below (r + 1.5 err)^2 (with margin for the roundoff
    // of the test itself).  A candidate is dropped early only when it exceeds
    // that bound, i.e. when the exact arithmetic (still run, with the window
    // test, for every other candidate) rejects it too: the result is unchanged.
    const float rcp_dz02 = __frcp_rn(dz02);
    const float pre_err =
        8.0f * 5.9604645e-8f * (P.max_slope * fabsf(dz12) + 2.0f * coord_max + 2.0f * sqrtf(P.max_scatter_seed) + 1.0f);
    const float pre_r = sqrtf(P.max_scatter_seed) * (1.0f + 1e-6f) + 1.5f * pre_err;
    const float pre_sc = pre_r * pre_r * (1.0f + 1e-5f);
    const float ap = fm(rcp_dz02, dz12), oma = fs(1.0f, ap);
    // (1 - a') x2, (1 - a') y2 of the hits of module m - 1, in the third slice of
    // the clustering's charge-sum scratch (dead after the clustering; the
    // first two hold the claims and the seed keys)
    float2* uxy = reinterpret_cast<float2*>(W.acc + 2 * L.n_pixels) + p0;
    // (heavy events) the grid of module m - 1's hits by their u terms
    bool grid = false;
    if constexpr (WIDE) {
      grid = hi2 - lo2 <= kGridCap && hi0 - lo0 <= kGridCap && mhi - mlo <= kGridCap && fabsf(oma) > 0.05f;
      if (grid) {
        static_assert(kGridCells % (2 * NT) == 0, "the cell scan gives every thread the same number of words");
        constexpr uint32_t PG = kGridCells / NT;  // cells per thread in the scan (an even number)
        const uint32_t n2 = hi2 - lo2;
        const float half = fabsf(oma) * coord_max * 1.01f + 1e-3f;
        g_oma = oma;
        g_lo = -half;
        g_inv = (float)kGridSide / (2.0f * half);
        for (uint32_t w = tid; w < kGridCells / 2u + 1u; w += NT) reinterpret_cast<uint32_t*>(goff)[w] = 0u;
        __syncthreads();
        for (uint32_t i = tid; i < n2; i += NT) {  // counts of cell c at c + 1
          const float4 h = hit[lo2 + i];
          goff_inc(1u + gcell(fm(oma, h.y)) * kGridSide + gcell(fm(oma, h.x)));
        }
        __syncthreads();
        uint32_t cnt[PG], sum = 0;
#pragma unroll
        for (uint32_t k = 0; k < PG; k += 2) {
          const uint32_t w = reinterpret_cast<const uint32_t*>(goff)[(tid * PG + k) >> 1];
          cnt[k] = w & 0xFFFFu;
          cnt[k + 1] = w >> 16;
          sum += cnt[k] + cnt[k + 1];
        }
        uint32_t total;
        uint32_t run = block_exclusive_scan<NT, uint32_t>(sum, &total, S.tmp);
#pragma unroll
        for (uint32_t k = 0; k < PG; ++k) {  // goff[c + 1] = the first slot of cell c
          goff[tid * PG + k] = (uint16_t)run;
          run += cnt[k];
        }
        if (tid == 0) goff[kGridCells] = (uint16_t)total;
        __syncthreads();
        // (afterwards goff[c + 1] is the end of cell c, so cell c is [goff[c], goff[c + 1]))
        for (uint32_t i = tid; i < n2; i += NT) {
          const float4 h = hit[lo2 + i];
          const float2 u = make_float2(fm(oma, h.x), fm(oma, h.y));
          const uint32_t at = goff_inc(1u + gcell(u.y) * kGridSide + gcell(u.x));
          gu[at] = u;
          gid[at] = (uint16_t)i;
        }
      }
      grid_m = grid;  // module m - 1 is the next step's module m
    }
    if (grid) {
      // (heavy events) one warp of the cluster per middle hit, its lanes over
      // the h0 window.  For an h0 the pre-test accepts only u terms within
      // sqrt(pre_sc) (+ the roundings of u + c0 and of the squares, far below
      // the margin of `box`) of -c0, so the h2 candidates are the hits of the
      // grid cells of that box; the exact chain then decides as above.  The
      // warp's smallest (bits(s), id0, id2) key is the seed of h1 (the same
      // minimum as a search over the whole window), claimed at once.
      // used flags of module m + 1 (final since step m + 1) and of module m
      // (final since the extension's)
      uint32_t* sused = reinterpret_cast<uint32_t*>(gsm + kGridUsedAt);
      uint32_t* s1used = reinterpret_cast<uint32_t*>(gsm + kGridUsed1At);
      for (uint32_t base = 0; base < hi0 - lo0; base += NT) {
        const uint32_t q = base + tid;
        const uint32_t bal = __ballot_sync(kFull, q < hi0 - lo0 && ldx<WIDE>(used + lo0 + q));
        if (lane_id() == 0 && base + warp_id() * 32u < hi0 - lo0) sused[(base >> 5) + warp_id()] = bal;
      }
      for (uint32_t base = 0; base < mhi - mlo; base += NT) {
        const uint32_t q = base + tid;
        const uint32_t bal = __ballot_sync(kFull, q < mhi - mlo && ldx<WIDE>(used + mlo + q));
        if (lane_id() == 0 && base + warp_id() * 32u < mhi - mlo) s1used[(base >> 5) + warp_id()] = bal;
      }
      // the CTA of rank r takes the middle hits mlo + r + j CS, its warps the
      // next j from a counter as they finish (the work per middle hit varies)
      uint32_t* next = reinterpret_cast<uint32_t*>(gsm + kGridNextAt);
      if (tid == 0) *next = 0u;
      __syncthreads();
      const float box = sqrtf(pre_sc) * 1.001f + 1e-4f;
      const uint32_t lane = lane_id();
      const KeyIndex I0{lo0, S.ktab[(m + 1) % 3]};
      for (;;) {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(next, 1u);
        const uint32_t p1 = mlo + rank + __shfl_sync(kFull, j, 0) * CS;  // (warp-uniform)
        if (p1 >= mhi) break;
        unsigned long long best = ~0ull, skey = ~0ull;
        uint32_t b0 = 0, b2 = 0;
        if (!((s1used[(p1 - mlo) >> 5] >> ((p1 - mlo) & 31u)) & 1u)) {
          const float4 H1 = hit[p1];
          uint32_t bq = 0;  // (q0 - lo0) | (q2 - lo2) << 16 of this lane's best
          const float k1 = H1.z, x1 = H1.x, y1 = H1.y;
          const Ranges R0 = window_ranges(I0, k1, P.win_seed);
          const uint32_t na = R0.a1 - R0.a0, nw = na + (R0.b1 - R0.b0);
          for (uint32_t kk = lane; kk < nw; kk += 32) {
            const uint32_t q0 = kk < na ? R0.a0 + kk : R0.b0 + (kk - na);
            if ((sused[(q0 - lo0) >> 5] >> ((q0 - lo0) & 31u)) & 1u) continue;
            const float4 H0 = hit[q0];
            if (dmod4(H0.z, k1) > P.win_seed) continue;
            const float x0 = H0.x, y0 = H0.y;
            const unsigned long long lid0 = fbits(H0.w) - lo0;
            const float c0x = fs(fm(ap, x0), x1), c0y = fs(fm(ap, y0), y1);
            const uint32_t cx0 = gcell(-c0x - box), cx1 = gcell(box - c0x);
            for (uint32_t cy = gcell(-c0y - box), cy1 = gcell(box - c0y); cy <= cy1; ++cy) {
              const uint32_t s1 = goff[cy * kGridSide + cx1 + 1u];  // cells cx0 .. cx1 of the row are adjacent
              for (uint32_t sl = goff[cy * kGridSide + cx0]; sl < s1; ++sl) {
                const float2 u = gu[sl];
                const float ex = fa(u.x, c0x), ey = fa(u.y, c0y);
                if (fa(fm(ex, ex), fm(ey, ey)) > pre_sc) continue;
                const uint32_t q2 = lo2 + gid[sl];
                const float4 H2 = hit[q2];
                if (dmod4(H2.z, k1) > P.win_seed) continue;
                const float x2 = H2.x, y2 = H2.y;
                const float tx = fd(fs(x0, x2), dz02), ty = fd(fs(y0, y2), dz02);
                if (fabsf(tx) > P.max_slope || fabsf(ty) > P.max_slope) continue;
                const float xp = fa(x2, fm(tx, dz12)), yp = fa(y2, fm(ty, dz12));
                const float dx = fs(xp, x1), dy = fs(yp, y1);
                const float sc = fa(fm(dx, dx), fm(dy, dy));
                if (sc > P.max_scatter_seed) continue;
                const unsigned long long cand =
                    (unsigned long long)fbits(sc) << 32 | lid0 << 16 | (unsigned long long)(fbits(H2.w) - lo2);
                if (cand < best) {
                  best = cand;
                  bq = (q0 - lo0) | (q2 - lo2) << 16;
                }
              }
            }
          }
          unsigned long long wbest = best;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(kFull, wbest, o);
            wbest = v < wbest ? v : wbest;
          }
          // the positions of h0 and h2 from the one lane that found the pair
          const uint32_t own = __ballot_sync(kFull, best == wbest && wbest != ~0ull);
          bq = __shfl_sync(kFull, bq, own ? __ffs(own) - 1 : 0);
          if (own) {
            b0 = lo0 + (bq & 0xFFFFu);
            b2 = lo2 + (bq >> 16);
            skey = step_key((uint32_t)m, (uint32_t)(wbest >> 32), fbits(H1.w));
          }
        }
        if (lane == 0) {
          if (skey != ~0ull) {
            seed_h0[p1] = b0;
            seed_h2[p1] = b2;
            atomicMin(claim + b0, skey);
            atomicMin(claim + b2, skey);
          }
          seedkey[p1] = skey;
        }
      }
      bar();
    } else {
      for (uint32_t q = lo2 + gt; q < hi2; q += GT) {
        const float4 h = hit[q];
        uxy[q] = make_float2(fm(oma, h.x), fm(oma, h.y));
      }
    }
    constexpr uint32_t kChunk = seed_chunk<NT>();
    constexpr int PER = kChunk / NT;
    // a module of one chunk (nearly always): every thread keeps the seeds of
    // its middle hits (tid + k NT) in registers from the claims to the
    // survivors, instead of the seed arrays in global memory
    const bool one_chunk = !WIDE && mhi - mlo <= kChunk;
    unsigned long long rkey[PER];
    uint32_t rb0[PER], rb2[PER];
    for (uint32_t cbase = grid ? mhi : mlo; cbase < mhi; cbase += kChunk) {  // (the grid's seeds are made)
      const uint32_t cn = min(kChunk, mhi - cbase);
      uint32_t cnt[PER], sum = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {  // thread tid owns middle hits PER*tid .. PER*tid+PER-1
        const uint32_t i = tid * PER + k;
        uint32_t c = 0;
        if (i < cn) {
          const uint32_t p1 = cbase + i;
          if (WIDE) {
            if (rank == 0) seedkey[p1] = ~0ull;  // the cluster's per-h1 minimum lives in global memory
          } else {
            S.sd.best[i] = ~0ull;
          }
          if (!ldx<WIDE>(used + p1)) {
            const float k1 = hit[p1].z;
            const Ranges R0 = window_ranges(KeyIndex{lo0, S.ktab[(m + 1) % 3]}, k1, P.win_seed);
            S.sd.r0[i] = pack_ranges(R0, lo0);
            S.sd.r2[i] = pack_ranges(window_ranges(KeyIndex{lo2, S.ktab[(m - 1) % 3]}, k1, P.win_seed), lo2);
            c = (R0.a1 - R0.a0) + (R0.b1 - R0.b0);
          }
        }
        cnt[k] = c;
        sum += c;
      }
      uint32_t n_items;
      uint32_t run = block_exclusive_scan<NT, uint32_t>(sum, &n_items, S.tmp);
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const uint32_t i = tid * PER + k;
        if (i < cn) S.sd.ioff[i] = run;
        run += cnt[k];
      }
      bar();  // (WIDE) the u terms and the reset minima of every CTA
      for (uint32_t j = gt; j < n_items; j += GT) {
        // middle hit of item j: the last i with ioff[i] <= j (empty entries
        // share the offset of the next one, so that i owns item j)
        const uint32_t i = lower_bound_by(0u, cn, [&](uint32_t x) { return S.sd.ioff[x] <= j; }) - 1u;
        const uint32_t p1 = cbase + i;
        const Ranges R0 = unpack_ranges(S.sd.r0[i], lo0);
        const uint32_t kk = j - S.sd.ioff[i], na = R0.a1 - R0.a0;
        const uint32_t q0 = kk < na ? R0.a0 + kk : R0.b0 + (kk - na);
        if (ldx<WIDE>(used + q0)) continue;
        const float4 H0 = hit[q0], H1 = hit[p1];
        const float k1 = H1.z;
        if (dmod4(H0.z, k1) > P.win_seed) continue;
        const float x1 = H1.x, y1 = H1.y, x0 = H0.x, y0 = H0.y;
        const unsigned long long lid0 = fbits(H0.w) - lo0;
        Ranges R2 = unpack_ranges(S.sd.r2[i], lo2);
        const float c0x = fs(fm(ap, x0), x1), c0y = fs(fm(ap, y0), y1);
        unsigned long long best = ~0ull;
        auto try_h2 = [&](uint32_t q2) {
          const float2 u = ldx<WIDE>(uxy + q2);
          const float ex = fa(u.x, c0x), ey = fa(u.y, c0y);
          if (fa(fm(ex, ex), fm(ey, ey)) > pre_sc) return;
          const float4 H2 = hit[q2];
          if (dmod4(H2.z, k1) > P.win_seed) return;
          const float x2 = H2.x, y2 = H2.y;
          const float dx02 = fs(x0, x2), dy02 = fs(y0, y2);
          const float tx = fd(dx02, dz02), ty = fd(dy02, dz02);
          if (fabsf(tx) > P.max_slope || fabsf(ty) > P.max_slope) return;
          const float xp = fa(x2, fm(tx, dz12)), yp = fa(y2, fm(ty, dz12));
          const float dx = fs(xp, x1), dy = fs(yp, y1);
          const float sc = fa(fm(dx, dx), fm(dy, dy));
          if (sc > P.max_scatter_seed) return;
          const unsigned long long cand =
              (unsigned long long)fbits(sc) << 32 | lid0 << 16 | (unsigned long long)(fbits(H2.w) - lo2);
          best = cand < best ? cand : best;
        };
        if (seed_narrow && (R2.a1 - R2.a0) + (R2.b1 - R2.b0) > kNarrowAbove)
          R2 = narrowed_ranges(KeyIndex{lo2, S.ktab[(m - 1) % 3]}, P.win_seed, R2,
                               (x1 - alpha * x0) / one_m_alpha, (y1 - alpha * y0) / one_m_alpha, seed_reach);
        for (int part2 = 0; part2 < 2; ++part2) {
          const uint32_t s2 = part2 ? R2.b0 : R2.a0, e2 = part2 ? R2.b1 : R2.a1;
          for (uint32_t q2 = s2; q2 < e2; ++q2) try_h2(q2);
        }
        if (best != ~0ull) atomicMin(WIDE ? &seedkey[p1] : &S.sd.best[i], best);
      }
      bar();
      if (one_chunk) {  // seeds claim their h0 and h2
#pragma unroll
        for (int k = 0; k < PER; ++k) {
          const uint32_t i = tid + (uint32_t)k * NT;
          rkey[k] = ~0ull;
          rb0[k] = rb2[k] = 0;
          const unsigned long long key = i < cn ? S.sd.best[i] : ~0ull;
          if (key != ~0ull) {
            rb0[k] = W.h_pos[p0 + lo0 + (uint32_t)((key >> 16) & 0xFFFFu)];
            rb2[k] = W.h_pos[p0 + lo2 + (uint32_t)(key & 0xFFFFu)];
            rkey[k] = step_key((uint32_t)m, (uint32_t)(key >> 32), fbits(hit[cbase + i].w));
            atomicMin(claim + rb0[k], rkey[k]);
            atomicMin(claim + rb2[k], rkey[k]);
          }
        }
      } else {
        for (uint32_t i = gt; i < cn; i += GT) {  // seeds claim their h0 and h2
          const uint32_t p1 = cbase + i;
          const unsigned long long key = WIDE ? ldx<WIDE>(seedkey + p1) : S.sd.best[i];
          unsigned long long skey = ~0ull;
          if (key != ~0ull) {
            const uint32_t b0 = W.h_pos[p0 + lo0 + (uint32_t)((key >> 16) & 0xFFFFu)];
            const uint32_t b2 = W.h_pos[p0 + lo2 + (uint32_t)(key & 0xFFFFu)];
            skey = step_key((uint32_t)m, (uint32_t)(key >> 32), fbits(hit[p1].w));
            seed_h0[p1] = b0;
            seed_h2[p1] = b2;
            atomicMin(claim + b0, skey);
            atomicMin(claim + b2, skey);
          }
          seedkey[p1] = skey;
        }
      }
      bar();
    }
    if (one_chunk) {
      // surviving seeds become tracks in the order of h1: middle hit tid + k NT
      // is ranked by the survivors of the blocks before k and of the lower
      // threads in block k (one scan of the counts, 16 bits per block)
      bool surv[PER];
      unsigned long long v = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        surv[k] = rkey[k] != ~0ull && claim[rb0[k]] == rkey[k] && claim[rb2[k]] == rkey[k];
        v |= (unsigned long long)(surv[k] ? 1u : 0u) << (16 * k);
      }
      unsigned long long tot;
      const unsigned long long ex =
          block_exclusive_scan<NT, unsigned long long>(v, &tot, reinterpret_cast<unsigned long long*>(S.tmp));
      uint32_t before = 0;
#pragma unroll
      for (int k = 0; k < PER; ++k) {
        const uint32_t r = before + (uint32_t)((ex >> (16 * k)) & 0xFFFFu);
        if (surv[k] && n_tr + r < track_cap) {  // (the slice bound, as below)
          const uint32_t t = n_tr + r, p1 = mlo + tid + (uint32_t)k * NT;
          ta[t] = rb2[k];
          tbk[t] = p1;
          meta[t] = 3u | kTrkActive | ((uint32_t)(m - 1) << 16) | ((uint32_t)m << 24);
          prev[rb2[k]] = p1;
          prev[p1] = rb0[k];
          prev[rb0[k]] = kNone;
          used[rb0[k]] = 1;
          used[p1] = 1;
          used[rb2[k]] = 1;
        }
        before += (uint32_t)((tot >> (16 * k)) & 0xFFFFu);
      }
      n_tr = min(n_tr + before, track_cap);
      bar();
      continue;
    }
    // surviving seeds become tracks in the order of h1: two consecutive
    // middle hits per thread, one block scan per 2 NT of them
    for (uint32_t base = mlo; base < mhi; base += 2u * NT) {
      bool surv[2];
      uint32_t b0[2], b2[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint32_t p1 = base + 2u * tid + (uint32_t)k;
        surv[k] = false;
        b0[k] = b2[k] = 0;
        if (p1 < mhi) {
          const unsigned long long skey = ldx<WIDE>(seedkey + p1);
          if (skey != ~0ull) {
            b0[k] = ldx<WIDE>(seed_h0 + p1);
            b2[k] = ldx<WIDE>(seed_h2 + p1);
            surv[k] = ldx<WIDE>(claim + b0[k]) == skey && ldx<WIDE>(claim + b2[k]) == skey;
          }
        }
      }
      uint32_t tot;
      uint32_t r = block_exclusive_scan<NT, uint32_t>((surv[0] ? 1u : 0u) + (surv[1] ? 1u : 0u), &tot, S.tmp);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (!surv[k]) continue;
        // tracks hold >= 3 hits each and never share one, so n_tr <= H / 3 <= the
        // event's track slice (n / 3); the test only guards the slice bound.  Every
        // CTA of a cluster counts the same survivors; the first one writes them.
        if (n_tr + r < track_cap && rank == 0) {
          const uint32_t t = n_tr + r, p1 = base + 2u * tid + (uint32_t)k;
          ta[t] = b2[k];
          tbk[t] = p1;
          meta[t] = 3u | kTrkActive | ((uint32_t)(m - 1) << 16) | ((uint32_t)m << 24);
          prev[b2[k]] = p1;
          prev[p1] = b0[k];
          prev[b0[k]] = kNone;
          used[b0[k]] = 1;
          used[p1] = 1;
          used[b2[k]] = 1;
        }
        ++r;
      }
      n_tr = min(n_tr + tot, track_cap);
    }
    bar();
  }

  if (rank == 0 && tid == 0) W.ev_ntracks_all[e] = n_tr;
  // the fit ranks the kept tracks of an event of up to kRankCap tracks in
  // shared memory; above that it reads the id -> track map, reset here
  if (!WIDE && n_tr > kRankCap)
    for (uint32_t i = tid; i < H; i += NT) first_of[i] = kNone;
}


// One CTA per event, scheduled by the hardware as CTAs finish (this kernel
// measured 20 % faster this way than as a persistent loop over a work queue: the
// loop raised its register pressure), which balances uneven events as well.
// The module loop is latency-bound, so resident warps pay more than
// registers: with the fit in a kernel of its own (k_fit), 8 CTAs of 256
// threads per SM (32 registers, a few bytes spilled) measured 8 % faster
// than 6 (40 registers), which was 6 % faster than 5 and 8 % faster than 4.
// CTA b tracks event order[b]: the large events start first.
template <int NT>
__global__ void __launch_bounds__(NT, 2048 / NT) k_track(Launch L) {
  __shared__ TrackSmem<NT> S;
  track_one<NT, false>(L, L.ws.order[blockIdx.x], S, nullptr);
}

// The heavy events: one wave of clusters of CTAs of kWideThreads threads
// (cluster size chosen at the launch) takes the events of kWideClusters clusters or more
// from the list the clustering kernel made, one cluster per event.
__global__ void __launch_bounds__(kWideThreads, 1) k_track_wide(Launch L) {
  __shared__ TrackSmem<kWideThreads> S;
  extern __shared__ __align__(16) uint8_t grid_raw[];
  const uint32_t count = *(const volatile uint32_t*)(L.ws.queue + 3);
  const uint32_t cs = cooperative_groups::this_cluster().num_blocks();
  for (uint32_t i = blockIdx.x / cs; i < count; i += gridDim.x / cs) {
    track_one<kWideThreads, true>(L, L.ws.wide_list[i], S, grid_raw);
    cooperative_groups::this_cluster().sync();  // shared memory and the workspace are reused by the next event
  }
}

// Fit, cut and canonical rank of the tracks of event e (one CTA per event):
// every track is fitted (straight line + simplified Kalman), kept by its
// chi2/ndf (or scored by the ghost-rejection network on tensor cores), and
// the kept ones are ranked by their smallest cluster id.  A kernel of its
// own, so that the module loop runs with fewer registers and more CTAs.
// CL: a thread-block cluster shares the event (its CTAs take every CS-th
// round of tracks and a CS-th of the ids; rank 0 holds the staging counter).
template <int NT, bool CL = false>
__device__ __forceinline__ void fit_event(const Launch& L, const uint64_t e, FitSmem<NT>& S) {
  constexpr int kFitThreads = NT;
  const Workspace& W = L.ws;
  const uint32_t tid = threadIdx.x;
  uint32_t CS = 1, crank = 0;
  if constexpr (CL) {
    CS = cooperative_groups::this_cluster().num_blocks();
    crank = cooperative_groups::this_cluster().block_rank();
  }
  auto sync_event = [&]() {  // (CL: a cluster barrier also orders the CTAs' global writes)
    if constexpr (CL) cooperative_groups::this_cluster().sync();
    else __syncthreads();
  };
  const Par P = L.par;
  const uint32_t M = L.geo.n_modules;
  if (P.use_mlp) mlp_load(P.mlp, S.mlp, tid, kFitThreads);  // network constants
  if (*(const volatile uint32_t*)W.flag != 0u || L.out.status[e] != VELO_EVT_OK) {
    if (tid == 0) {
      W.ev_ntracks[e] = 0;
      W.ev_nhits[e] = 0;
    }
    return;
  }
  const uint64_t p0 = L.off[e];
  const uint64_t tb = p0 / 3;
  const uint32_t H = W.ev_nclusters[e];
  const uint32_t n_tr = W.ev_ntracks_all[e];
  if (tid < kModOffStride) S.mod_off[tid] = W.ev_modoff[e * kModOffStride + tid];
  if (tid < VELO_MAX_MODULES) S.z[tid] = L.geo.z[tid];
  if (tid == 0) {
    S.hit_fill = 0;
    S.n_kept = 0;
  }
  sync_event();
  // (events of up to kRankCap tracks) ranks in shared memory
  const bool ranks_here = !CL && n_tr <= kRankCap;
  uint32_t* fill = &S.hit_fill;
  if constexpr (CL) fill = cooperative_groups::this_cluster().map_shared_rank(&S.hit_fill, 0);
  const float4* hit = W.hit + p0;
  uint32_t* first_of = W.sd + p0;
  // for k_output: every track's state and its hit ids (in z order) at a slot of
  // the event's word slice of sa (dead after the module loop; the tracks hold
  // at most n hits), the slot's start in trk_pick
  uint32_t* hit_stage = W.sa + p0;
  const uint32_t* meta = W.trk_meta + tb;
  const uint32_t* ta = W.trk_a + tb;

  // ---- fit, cut, canonical rank (by smallest cluster id) of every track
  uint32_t* rank = W.trk_rank + tb;
  uint32_t* hoff = W.trk_hoff + tb;
  // every thread takes part in every round (the learned rule scores a warp's
  // 32 candidates with warp-wide tensor-core instructions)
  for (uint32_t base = crank * kFitThreads; base < n_tr; base += CS * kFitThreads) {
    const uint32_t t = base + tid;
    const bool valid = t < n_tr;
    float xs[VELO_MAX_MODULES], ys[VELO_MAX_MODULES], zs[VELO_MAX_MODULES], st[VELO_STATE_STRIDE];
    float f[VELO_N_FEATURES];
    uint32_t mods[VELO_MAX_MODULES], ids[VELO_MAX_MODULES];
    uint32_t n = 0;
    bool keep = false;
    if (valid) {
      n = gather_track(W, p0, tb, t, S.mod_off, S.z, M, xs, ys, zs, mods, ids);
      fit_track(n, xs, ys, zs, P.sigma, P.ms_theta, st);
      keep = keep_track(n, st, P.ms_theta, P.chi2ndf_max, P.chi2ndf_max_3hit);
    }
    if (P.use_mlp) {
      const float r = valid ? cut_chi2ndf(n, st, P.ms_theta) : 0.0f;
      if (valid) candidate_features(n, xs, ys, zs, mods, st, r, f);
      else
        for (int k = 0; k < VELO_N_FEATURES; ++k) f[k] = 0.0f;
      const float logit = mlp_logit_warp(f, S.mlp, S.tiles[tid >> 5]);
      if (valid) {
        W.trk_logit[tb + t] = logit;
        keep = r <= P.chi2ndf_max && logit >= P.mlp_logit_min;
      }
    }
    if (valid) {
      rank[t] = kNone;
      if (keep) {
        const uint32_t fid = fbits(hit[ta[t]].w);  // the track's smallest cluster id (< 2^21), t < 2^11
        if (ranks_here) S.rkey[atomicAdd(&S.n_kept, 1u)] = fid << 11 | t;
        else first_of[fid] = t;
        if (P.use_mlp) st[19] = W.trk_logit[tb + t];
        float4* so = reinterpret_cast<float4*>(W.trk_state + (tb + t) * VELO_STATE_STRIDE);  // 16-byte aligned
#pragma unroll
        for (int k = 0; k < VELO_STATE_STRIDE / 4; ++k)
          so[k] = make_float4(st[4 * k], st[4 * k + 1], st[4 * k + 2], st[4 * k + 3]);
        const uint32_t slot = atomicAdd(fill, n);
        W.trk_pick[tb + t] = slot;
        for (uint32_t j = 0; j < n; ++j) hit_stage[slot + j] = ids[j];
      }
    }
  }
  sync_event();
  if (ranks_here) {
    // Ranks: kept tracks in the order of their first cluster id (distinct:
    // tracks share no hit), each the count of smaller keys; hit offsets by a
    // block scan of the hit counts in rank order.
    const uint32_t nk = S.n_kept;
    for (uint32_t k = tid; k < nk; k += kFitThreads) {
      const uint32_t key = S.rkey[k];
      uint32_t r = 0;
      for (uint32_t j = 0; j < nk; ++j) r += S.rkey[j] < key ? 1u : 0u;
      const uint32_t t = key & 2047u;
      rank[t] = r;
      S.rtrk[r] = (uint16_t)t;
      S.rnh[r] = (uint8_t)(meta[t] & 255u);
    }
    __syncthreads();
    static_assert(kRankCap % kFitThreads == 0, "the rank scan gives every thread the same number of ranks");
    constexpr uint32_t PR = kRankCap / kFitThreads;
    uint32_t v[PR], sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < PR; ++k) {
      const uint32_t r = tid * PR + k;
      v[k] = r < nk ? S.rnh[r] : 0u;
      sum += v[k];
    }
    uint32_t nh_all;
    uint32_t run = block_exclusive_scan<kFitThreads, uint32_t>(sum, &nh_all, reinterpret_cast<uint32_t*>(S.tmp64));
#pragma unroll
    for (uint32_t k = 0; k < PR; ++k) {
      const uint32_t r = tid * PR + k;
      if (r < nk) hoff[S.rtrk[r]] = run;
      run += v[k];
    }
    if (tid == 0) {
      W.ev_ntracks[e] = nk;
      W.ev_nhits[e] = nh_all;
    }
    return;
  }
  // Ranks: kept tracks in the order of their first cluster id.  Every warp
  // takes a contiguous chunk of the ids (of the CTA's CS-th of them), 32 at
  // a time (coalesced): ballots and a warp scan count its tracks and their
  // hits, one block scan over the warps gives each chunk its first rank and
  // first hit (on a cluster, after the counts of the lower ranks' ids).
  constexpr uint32_t NW = kFitThreads / 32;
  const uint32_t lane = lane_id(), wid = warp_id();
  const uint32_t c_lo = (uint32_t)((uint64_t)H * crank / CS), c_hi = (uint32_t)((uint64_t)H * (crank + 1) / CS);
  const uint32_t cw = ((c_hi - c_lo + NW - 1) / NW + 31u) & ~31u;
  const uint32_t wlo = min(c_hi, c_lo + wid * cw), whi = min(c_hi, wlo + cw);
  // (CL: first_of was written by other SMs; read past this SM's L1)
  auto first_at = [&](uint32_t id) -> uint32_t {
    if constexpr (CL) return __ldcg(first_of + id);
    else return first_of[id];
  };
  uint32_t wtr = 0, wht = 0;
  for (uint32_t b0 = wlo; b0 < whi; b0 += 32) {
    const uint32_t id = b0 + lane;
    const uint32_t t = id < whi ? first_at(id) : kNone;
    wtr += __popc(__ballot_sync(kFull, t != kNone));
    wht += __reduce_add_sync(kFull, t != kNone ? meta[t] & 255u : 0u);
  }
  unsigned long long tot;
  const unsigned long long ex = block_exclusive_scan<kFitThreads, unsigned long long>(
      lane == 0 ? ((unsigned long long)wtr << 32) | wht : 0ull, &tot, S.tmp64);
  unsigned long long below = 0;  // (CL) the counts of the lower ranks' ids
  if constexpr (CL) {
    if (tid == 0) S.cta_counts = tot;
    cooperative_groups::this_cluster().sync();
    if (wid == 0) {
      unsigned long long v = lane < crank ? *cooperative_groups::this_cluster().map_shared_rank(&S.cta_counts, lane) : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if (lane == 0) S.tmp64[NW] = v;  // (past the block scan's words)
    }
    __syncthreads();
    below = S.tmp64[NW];
  }
  const unsigned long long ex0 = __shfl_sync(kFull, ex, 0) + below;
  uint32_t rr = (uint32_t)(ex0 >> 32), rh = (uint32_t)ex0;
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t b0 = wlo; b0 < whi; b0 += 32) {
    const uint32_t id = b0 + lane;
    const uint32_t t = id < whi ? first_at(id) : kNone;
    const uint32_t nh = t != kNone ? meta[t] & 255u : 0u;
    uint32_t x = nh;  // inclusive warp scan of the hit counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    const uint32_t bal = __ballot_sync(kFull, t != kNone);
    if (t != kNone) {
      rank[t] = rr + __popc(bal & lt);
      hoff[t] = rh + x - nh;
    }
    rr += __popc(bal);
    rh += __shfl_sync(kFull, x, 31);
  }
  if (tid == 0 && crank + 1 == CS) {
    W.ev_ntracks[e] = (uint32_t)((below + tot) >> 32);
    W.ev_nhits[e] = (uint32_t)(below + tot);
  }
}

// The fit of the separate form (one CTA per event; k_scan and k_output
// follow); the heavy-ion-like events (those k_track_wide tracked) are left
// to k_fit_wide.
__global__ void __launch_bounds__(kFitThreads, 6) k_fit(Launch L) {
  __shared__ FitSmem<kFitThreads> S;
  const uint64_t e = blockIdx.x;
  if (*(const volatile uint32_t*)L.ws.flag == 0u && L.out.status[e] == VELO_EVT_OK &&
      L.ws.ev_nclusters[e] >= kWideClusters)
    return;
  fit_event<kFitThreads>(L, e, S);
}

// The fit of the heavy-ion-like events: one thread-block cluster of
// 1024-thread CTAs per listed event (the clusters take the events of the list
// in turn).
__global__ void __launch_bounds__(kFitWideThreads, 1) k_fit_wide(Launch L) {
  extern __shared__ __align__(16) uint8_t fit_raw[];
  FitSmem<kFitWideThreads>& S = *reinterpret_cast<FitSmem<kFitWideThreads>*>(fit_raw);
  const uint32_t count = *(const volatile uint32_t*)(L.ws.queue + 3);
  const uint32_t cs = cooperative_groups::this_cluster().num_blocks();
  for (uint32_t i = blockIdx.x / cs; i < count; i += gridDim.x / cs) {
    fit_event<kFitWideThreads, true>(L, L.ws.wide_list[i], S);
    cooperative_groups::this_cluster().sync();  // the shared records are reused by the next event
  }
}

// Compaction: clusters and kept tracks of event e into the caller's CSR
// arrays (offsets from k_scan).  Without features the states and hit ids are
// the ones k_fit staged; with them (FEAT) every kept track is gathered and
// fitted again for its features.
// Part `part` of `parts` of event e (its clusters and tracks in as many
// equal ranges): a heavy-ion-like event is written by several CTAs.
template <bool FEAT>
__device__ __forceinline__ void output_one(const Launch& L, const uint64_t e, uint32_t* mod_off, float* mz,
                                           uint32_t part, uint32_t parts) {
  constexpr int NT = kOutputThreads;
  constexpr int U = 4;  // cluster words in flight per thread
  const Workspace& W = L.ws;
  const uint32_t tid = threadIdx.x;
  const uint32_t M = L.geo.n_modules;
  if (*(const volatile uint32_t*)W.flag != 0u || L.out.status[e] != VELO_EVT_OK) return;
  const uint64_t p0 = L.off[e];
  const uint64_t tb = p0 / 3;
  if (tid < kModOffStride) mod_off[tid] = W.ev_modoff[e * kModOffStride + tid];
  if (tid < VELO_MAX_MODULES) mz[tid] = L.geo.z[tid];
  __syncthreads();
  const uint32_t Hall = W.ev_nclusters[e];  // this part's clusters: [id_lo, H)
  const uint32_t id_lo = (uint32_t)((uint64_t)Hall * part / parts), H = (uint32_t)((uint64_t)Hall * (part + 1) / parts);
  const uint64_t co = L.out.cluster_offsets[e];
  // clusters in id order (coalesced loads and stores): the clustering's
  // (x, y) by id, untouched by the tracking; the loads of U ids are issued
  // before their stores.  The module offsets hold for ids as for positions
  // (the hit sort keeps every module's clusters together).
  for (uint32_t id0 = id_lo + tid; id0 < H; id0 += U * NT) {
    float x[U], y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t id = id0 + u * NT;
      if (id < H) {
        const float2 c = W.cl_xy[p0 + id];
        x[u] = c.x;
        y[u] = c.y;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t id = id0 + u * NT;
      if (id < H) {
        L.out.cluster_x[co + id] = x[u];
        L.out.cluster_y[co + id] = y[u];
        L.out.cluster_z[co + id] = mz[module_of_pos(mod_off, M, id)];
      }
    }
  }
  const uint32_t nt_all = W.ev_ntracks_all[e];  // this part's tracks: [t0, nt)
  const uint32_t t0 = (uint32_t)((uint64_t)nt_all * part / parts), nt = (uint32_t)((uint64_t)nt_all * (part + 1) / parts);
  const uint64_t to = L.out.track_offsets[e];
  const uint64_t hb = W.ev_hitbase[e];
  if constexpr (!FEAT) {  // states and hit ids as k_fit staged them
    // states in 16-byte pieces when the caller's array allows it (the
    // workspace copy always does)
    const bool v4 = (reinterpret_cast<uintptr_t>(L.out.track_states) & 15u) == 0u;
    for (uint32_t t = t0 + tid; t < nt; t += NT) {
      const uint32_t r = W.trk_rank[tb + t];
      if (r == kNone) continue;
      const uint32_t n = W.trk_meta[tb + t] & 255u, slot = W.trk_pick[tb + t];
      const uint64_t dst = to + r;
      const uint64_t h0 = hb + W.trk_hoff[tb + t];
      L.out.track_hit_offsets[dst] = h0;
      for (uint32_t j = 0; j < n; ++j) L.out.track_hits[h0 + j] = W.sa[p0 + slot + j];
      const float* si = W.trk_state + (tb + t) * VELO_STATE_STRIDE;
      float* o = L.out.track_states + dst * VELO_STATE_STRIDE;
      if (v4) {
#pragma unroll
        for (int k = 0; k < VELO_STATE_STRIDE / 4; ++k)
          reinterpret_cast<float4*>(o)[k] = reinterpret_cast<const float4*>(si)[k];
      } else {
#pragma unroll
        for (int k = 0; k < VELO_STATE_STRIDE; ++k) o[k] = si[k];
      }
    }
  } else {
    for (uint32_t t = t0 + tid; t < nt; t += NT) {  // with the features: gathered and fitted again
      const uint32_t r = W.trk_rank[tb + t];
      if (r == kNone) continue;
      float xs[VELO_MAX_MODULES], ys[VELO_MAX_MODULES], zs[VELO_MAX_MODULES], st[VELO_STATE_STRIDE];
      uint32_t ids[VELO_MAX_MODULES], mods[VELO_MAX_MODULES];
      const uint32_t n = gather_track(W, p0, tb, t, mod_off, mz, M, xs, ys, zs, mods, ids);
      fit_track(n, xs, ys, zs, L.par.sigma, L.par.ms_theta, st);
      if (L.par.use_mlp) st[19] = W.trk_logit[tb + t];
      const uint64_t dst = to + r;
      float f[VELO_N_FEATURES];
      candidate_features(n, xs, ys, zs, mods, st, cut_chi2ndf(n, st, L.par.ms_theta), f);
      float* of = L.out.track_features + dst * VELO_N_FEATURES;
#pragma unroll
      for (int k = 0; k < VELO_N_FEATURES; ++k) of[k] = f[k];
      const uint64_t h0 = hb + W.trk_hoff[tb + t];
      L.out.track_hit_offsets[dst] = h0;
      for (uint32_t j = 0; j < n; ++j) L.out.track_hits[h0 + j] = ids[j];
      float* o = L.out.track_states + dst * VELO_STATE_STRIDE;
#pragma unroll
      for (int k = 0; k < VELO_STATE_STRIDE; ++k) o[k] = st[k];
    }
  }
}

// Persistent: work items from the queue -- first kOutputParts parts of each
// heavy-ion-like event (those the clustering listed), then every other event
// whole.  The plain form is small (six CTAs per SM keep more loads in
// flight); the form with features carries the fit's arrays.
template <bool FEAT>
__global__ void __launch_bounds__(kOutputThreads, FEAT ? 1 : 6) k_output(Launch L) {
  __shared__ uint32_t mod_off[kModOffStride];
  __shared__ float mz[VELO_MAX_MODULES];
  __shared__ uint32_t next;
  // nothing is written when the batch does not fit the caller's buffers
  if (!output_fits(L.out, L.out.totals[0], L.out.totals[1], L.out.totals[2])) return;
  const uint32_t n_parts = *(const volatile uint32_t*)(L.ws.queue + 3) * kOutputParts;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(L.ws.queue + 2, 1u);
    __syncthreads();
    const uint32_t item = next;
    __syncthreads();
    uint32_t e, part = 0, parts = 1;
    if (item < n_parts) {
      e = L.ws.wide_list[item / kOutputParts];
      part = item % kOutputParts;
      parts = kOutputParts;
    } else {
      e = item - n_parts;
      if (e >= L.n_events) break;
      // (a listed event has this many clusters; one that failed writes nothing)
      if (L.ws.ev_nclusters[e] >= kWideClusters && *(const volatile uint32_t*)L.ws.flag == 0u &&
          L.out.status[e] == VELO_EVT_OK)
        continue;
    }
    output_one<FEAT>(L, e, mod_off, mz, part, parts);
    __syncthreads();
  }
}

// Fit, offsets and output in one kernel (the fused form, for batches whose
// output cannot exceed the caller's capacities).  Every CTA takes the next
// event from a ticket counter, so the events before it have all started;
// it fits the event's tracks (as k_fit), publishes the event's counts
// (clusters, kept tracks, their hits, failed) and finds the counts of all
// the events before it by a decoupled look-back: one warp reads the records
// of the 32 events before its window at once, adding aggregates until it
// meets an event that already published its inclusive prefix.  It then
// publishes its own inclusive prefix, writes its event's offsets and its
// clusters and tracks straight into the caller's CSR arrays (as k_output),
// and the last event writes the closing offsets and the totals.  Every wait
// on another event's record is bounded; a wait that gives up (not expected:
// the events waited for are running) fails this event with
// VELO_EVT_TIMEOUT instead of hanging, and its record never holds a prefix.
__global__ void __launch_bounds__(kFitThreads, 4) k_fit_out(Launch L) {
  __shared__ FitSmem<kFitThreads> S;
  __shared__ uint32_t ticket;
  __shared__ unsigned long long prefix[4];
  __shared__ bool gave_up;
  const Workspace& W = L.ws;
  const uint32_t tid = threadIdx.x, lane = lane_id();
  if (tid == 0) {
    ticket = atomicAdd(W.queue + 6, 1u);
    gave_up = false;
  }
  __syncthreads();
  const uint64_t e = ticket;
  fit_event<kFitThreads>(L, e, S);
  __syncthreads();
  unsigned long long* rec = W.lb_val + 8 * e;  // aggregate [0, 4), inclusive prefix [4, 8)
  if (tid == 0) {
    const bool failed = *(const volatile uint32_t*)W.flag != 0u || L.out.status[e] != VELO_EVT_OK;
    rec[0] = failed ? 0ull : W.ev_nclusters[e];
    rec[1] = W.ev_ntracks[e];
    rec[2] = W.ev_nhits[e];
    rec[3] = failed ? 1ull : 0ull;
    __threadfence();
    atomicExch(W.lb_flag + e, 1u);
  }
  if (tid < 32) {
    constexpr uint32_t kSpinLimit = 1u << 22;  // x 64 ns: a wait gives up after about a quarter second
    unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
    int64_t j = (int64_t)e - 1;  // the window of events j, j - 1, ..., j - 31 (lane l reads j - l)
    bool done = j < 0, bad = false;
    while (!done) {
      const int64_t q = j - (int64_t)lane;
      uint32_t fl = 2u;  // before event 0: an empty inclusive prefix
      if (q >= 0) {
        uint32_t it = 0;
        while ((fl = *(const volatile uint32_t*)(W.lb_flag + q)) == 0u && ++it < kSpinLimit) __nanosleep(64);
      }
      if (__any_sync(kFull, fl == 0u)) {
        bad = true;
        break;
      }
      __threadfence();  // the records' values after their flags
      const uint32_t incl = __ballot_sync(kFull, fl == 2u);
      const uint32_t stop = incl ? (uint32_t)__ffs(incl) - 1u : 31u;  // the lanes up to it contribute
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        unsigned long long v = 0ull;
        if (q >= 0 && lane <= stop) v = *(const volatile unsigned long long*)(W.lb_val + 8 * q + (fl == 2u ? 4 : 0) + k);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        acc[k] += v;
      }
      done = incl != 0u;
      j -= 32;
    }
    if (lane == 0) {
      if (bad) {
        gave_up = true;
      } else {
        for (int k = 0; k < 4; ++k) {
          prefix[k] = acc[k];
          rec[4 + k] = acc[k] + rec[k];
        }
        __threadfence();
        atomicExch(W.lb_flag + e, 2u);
      }
    }
  }
  __syncthreads();
  if (gave_up) {
    if (tid == 0) L.out.status[e] = VELO_EVT_TIMEOUT;
    return;
  }
  if (tid == 0) {
    L.out.cluster_offsets[e] = prefix[0];
    L.out.track_offsets[e] = prefix[1];
    W.ev_hitbase[e] = prefix[2];
    if (e + 1 == L.n_events) {  // the closing offsets and the totals
      const unsigned long long tc = rec[4], tt = rec[5], th = rec[6], tf = rec[7];
      L.out.cluster_offsets[e + 1] = tc;
      L.out.track_offsets[e + 1] = tt;
      L.out.track_hit_offsets[tt] = th;
      L.out.totals[0] = tc;
      L.out.totals[1] = tt;
      L.out.totals[2] = th;
      L.out.totals[3] = tf;
    }
  }
  __syncthreads();
  output_one<false>(L, e, S.mod_off, S.z, 0, 1);
}

// One CTA: event offsets into the output CSR arrays and the batch totals.
__global__ void __launch_bounds__(kScanThreads) k_scan(Launch L) {
  constexpr int NT = kScanThreads;
  __shared__ unsigned long long tmp[64];
  const Workspace& W = L.ws;
  const uint64_t E = L.n_events;
  unsigned long long rc = 0, rt = 0, rh = 0, rf = 0;
  for (uint64_t base = 0; base < E; base += NT) {
    const uint64_t e = base + threadIdx.x;
    unsigned long long c = 0, t = 0, h = 0, f = 0;
    if (e < E) {
      c = W.ev_nclusters[e];
      t = W.ev_ntracks[e];
      h = W.ev_nhits[e];
      f = L.out.status[e] != VELO_EVT_OK;
    }
    unsigned long long tc, tt, th, tf;
    const unsigned long long xc = block_exclusive_scan<NT, unsigned long long>(c, &tc, tmp);
    const unsigned long long xt = block_exclusive_scan<NT, unsigned long long>(t, &tt, tmp);
    const unsigned long long xh = block_exclusive_scan<NT, unsigned long long>(h, &th, tmp);
    block_exclusive_scan<NT, unsigned long long>(f, &tf, tmp);
    if (e < E) {
      L.out.cluster_offsets[e] = rc + xc;
      L.out.track_offsets[e] = rt + xt;
      W.ev_hitbase[e] = rh + xh;
    }
    rc += tc;
    rt += tt;
    rh += th;
    rf += tf;
  }
  if (threadIdx.x == 0) {
    L.out.cluster_offsets[E] = rc;
    L.out.track_offsets[E] = rt;
    if (output_fits(L.out, rc, rt, rh)) L.out.track_hit_offsets[rt] = rh;
    L.out.totals[0] = rc;
    L.out.totals[1] = rt;
    L.out.totals[2] = rh;
    L.out.totals[3] = rf;
  }
}

// One CTA: the event offsets must start at 0, never decrease, end at
// n_pixels and give no event 2^30 words or more; otherwise every event fails.
__global__ void __launch_bounds__(kScanThreads) k_validate_offsets(Launch L) {
  const uint64_t E = L.n_events;
  int bad = 0;
  if (threadIdx.x == 0) bad |= (L.off[0] != 0ull) | (L.off[E] != L.n_pixels);
  for (uint64_t e = threadIdx.x; e < E; e += blockDim.x) {
    const uint64_t a = L.off[e], b = L.off[e + 1];
    bad |= (b < a) | (b - a >= (1ull << 30));
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    *L.ws.flag = bad ? 1u : 0u;
    for (int q = 0; q < 8; ++q) L.ws.queue[q] = 0u;  // the persistent kernels' work queues, the fit tickets
  }
  for (uint64_t e = threadIdx.x; e < E; e += blockDim.x) L.ws.lb_flag[e] = 0u;  // the fused fit's look-back
  __syncthreads();
  if (!bad)  // the heavy-ion-like events, for the module-by-module clustering
    for (uint64_t e = threadIdx.x; e < E; e += blockDim.x)
      if (L.off[e + 1] - L.off[e] >= kHeavyWords) L.ws.heavy_list[atomicAdd(L.ws.queue + 7, 1u)] = (uint32_t)e;
  if (bad) {
    for (uint64_t e = threadIdx.x; e < E; e += blockDim.x) L.out.status[e] = VELO_EVT_BADWORD;
    if (L.out.pixel_cluster)
      for (uint64_t i = threadIdx.x; i < L.n_pixels; i += blockDim.x) L.out.pixel_cluster[i] = kNone;
  }
}

// Cluster size of k_track_wide on the current device (once per device): 16
// if one such cluster of 1024-thread CTAs with their shared memory can be
// resident, else 8; 0 if the kernel's attributes cannot be set.
uint32_t wide_cluster_size() {
  static std::mutex mu;
  static uint32_t size[64] = {};
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (size[d]) return size[d];
  const void* f = reinterpret_cast<const void*>(k_track_wide);
  if (!set_max_smem_once(f, 5, kGridBytes)) return 0;
  uint32_t cs = kWideClusterPortable;
  if (allow_large_clusters_once(f, 0)) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kWideClusterMax;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(kWideClusterMax);
    cfg.blockDim = dim3(kWideThreads);
    cfg.dynamicSmemBytes = kGridBytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_track_wide, &cfg) == cudaSuccess && n >= 1) cs = kWideClusterMax;
    cudaGetLastError();
  }
  size[d] = cs;
  return cs;
}

int launch_track(const Launch& L, int nt, uint32_t grid, uint32_t wide_cluster, cudaStream_t s) {
  switch (nt) {
    case 128: k_track<128><<<grid, 128, 0, s>>>(L); break;
    case 256: k_track<256><<<grid, 256, 0, s>>>(L); break;
    default: return VELO_EINVAL;
  }
  const uint32_t cs_max = wide_cluster_size();
  if (!cs_max) return VELO_ECUDA;
  if (wide_cluster > cs_max) return VELO_EINVAL;  // the device cannot place such a cluster
  const uint32_t cs = wide_cluster ? wide_cluster : cs_max;
  // one wave: a cluster per cs SMs (one 1024-thread CTA per SM)
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(std::max<uint32_t>(1u, (uint32_t)device_sm_count() / cs) * cs);
  cfg.blockDim = dim3(kWideThreads);
  cfg.dynamicSmemBytes = kGridBytes;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_track_wide, L) != cudaSuccess) return VELO_ECUDA;
  return VELO_OK;
}

// Cluster size of k_fit_wide on the current device (once per device): the
// largest of 16, 8, 4, 2 that the device can place, else 1; 0 if the
// kernel's attributes cannot be set.
uint32_t fit_wide_cluster_size() {
  static std::mutex mu;
  static uint32_t size[64] = {};
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (size[d]) return size[d];
  const void* f = reinterpret_cast<const void*>(k_fit_wide);
  const uint32_t smem = (uint32_t)sizeof(FitSmem<kFitWideThreads>);
  if (!set_max_smem_once(f, 7, smem)) return 0;
  const bool large = allow_large_clusters_once(f, 2);
  uint32_t cs = 1;
  for (uint32_t c = kWideClusterMax; c > 1; c /= 2) {
    if (c > kWideClusterPortable && !large) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kFitWideThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, k_fit_wide, &cfg) == cudaSuccess && n >= 1;
    cudaGetLastError();
    if (ok) {
      cs = c;
      break;
    }
  }
  size[d] = cs;
  return cs;
}

int launch_fit(const Launch& L, bool fused, cudaStream_t s) {
  const uint32_t grid = (uint32_t)L.n_events;  // one CTA per event
  if (fused) {
    k_fit_out<<<grid, kFitThreads, 0, s>>>(L);
    return VELO_OK;
  }
  k_fit<<<grid, kFitThreads, 0, s>>>(L);
  const uint32_t cs = fit_wide_cluster_size();
  if (!cs) return VELO_ECUDA;
  // one wave: a cluster per cs SMs (one 1024-thread CTA per SM)
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(std::max<uint32_t>(1u, (uint32_t)device_sm_count() / cs) * cs);
  cfg.blockDim = dim3(kFitWideThreads);
  cfg.dynamicSmemBytes = (uint32_t)sizeof(FitSmem<kFitWideThreads>);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_fit_wide, L) != cudaSuccess) return VELO_ECUDA;
  return VELO_OK;
}

int track_blocks_per_sm(int nt) {
  switch (nt) {
    case 128: return occupancy(reinterpret_cast<const void*>(k_track<128>), 128, 0, -1);
    case 256: return occupancy(reinterpret_cast<const void*>(k_track<256>), 256, 0, -1);
    default: return 0;
  }
}

int launch_output(const Launch& L, uint32_t grid, cudaStream_t s) {
  if (L.out.track_features) k_output<true><<<grid, kOutputThreads, 0, s>>>(L);
  else k_output<false><<<grid, kOutputThreads, 0, s>>>(L);
  return VELO_OK;
}

int output_blocks_per_sm(bool features) {
  return features ? occupancy(reinterpret_cast<const void*>(k_output<true>), kOutputThreads, 0, -1)
                  : occupancy(reinterpret_cast<const void*>(k_output<false>), kOutputThreads, 0, -1);
}

}  // namespace velo
