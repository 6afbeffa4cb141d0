// Device helpers of the VELO tracking kernels (sm_103a).
//
// Everything here is either integer work or binary32 arithmetic written in
// the one order the method fixes; the library is compiled with -fmad=false so
// that no multiply-add pair is contracted into an FMA.
#pragma once

#include <stdint.h>

namespace velo {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kKeyMask = 0x7FFFFFFu;  // (module, row, col) bits of a pixel word

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t warp_id() { return threadIdx.x >> 5; }

// ---------------------------------------------------------------- scans
// Exclusive block-wide scan of one value per thread.  tmp: >= NT/32 + 1 words
// of shared memory, reused on return.  *total receives the block sum.
template <int NT, class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* tmp) {
  constexpr int NW = NT / 32;
  const uint32_t lane = lane_id(), w = warp_id();
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) tmp[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < (uint32_t)NW ? tmp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(kFull, s, o);
      if (lane >= (uint32_t)o) s += y;
    }
    if (lane < (uint32_t)NW) tmp[lane] = s;
  }
  __syncthreads();
  T base = w ? tmp[w - 1] : T(0);
  *total = tmp[NW - 1];
  __syncthreads();
  return base + x - v;
}

// ---------------------------------------------------------------- radix sort
// Lanes of the warp whose value d (< 2^BITS) equals this lane's: one ballot
// per bit (on this GPU cheaper than the match instruction).
template <int BITS>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d) {
  uint32_t m = kFull;
#pragma unroll
  for (int bit = 0; bit < BITS; ++bit) {
    const uint32_t set = (d >> bit) & 1u;
    const uint32_t bb = __ballot_sync(kFull, set);
    m &= set ? bb : ~bb;
  }
  return m;
}

// One stable LSD pass of a block-wide radix sort with 8-bit digits.
// The n elements are cut into one contiguous chunk per warp; every warp
// histograms its chunk into its own row of cnt (NW rows of 257 counters in
// shared memory, shared atomics; the pad word makes both the per-warp
// access, lanes on different digits, and the scan's access, one digit across
// warps, hit 32 different banks), one exclusive scan in (digit, warp) order
// gives each (digit, warp) its first output slot, and every warp then
// scatters its chunk in index order: among the lanes of one step with equal
// digits the lowest lane reads and advances the digit's slot and broadcasts
// it, and each lane adds its rank among those lanes, so equal digits keep
// their relative order.  a/b (and va/vb, of any unsigned type) may live in
// shared or global memory.  cnt: radix_counters(NT) words.
constexpr uint32_t kRadixRow = 257;  // 256 digit counters + 1 pad word per warp
__host__ __device__ constexpr uint32_t radix_counters(int nt) { return kRadixRow * (uint32_t)(nt / 32); }

template <int NT, bool HAS_VAL, class K, class V, class DigitF>
__device__ void radix_pass(const K* a, K* b, const V* va, V* vb, uint32_t n, DigitF digit, uint32_t* cnt,
                           uint32_t* tmp) {
  constexpr int NW = NT / 32;
  constexpr uint32_t NB = 256;
  const uint32_t lane = lane_id(), w = warp_id();
  uint32_t* row = cnt + w * kRadixRow;  // this warp's counters
  for (uint32_t i = threadIdx.x; i < kRadixRow * NW; i += NT) cnt[i] = 0;
  __syncthreads();
  const uint32_t chunk = (n + NW - 1) / NW;
  const uint32_t s = min(n, w * chunk), e = min(n, s + chunk);
  for (uint32_t i = s + lane; i < e; i += 32) atomicAdd(row + digit(a[i], HAS_VAL ? (uint32_t)va[i] : 0u), 1u);
  __syncthreads();
  // exclusive scan of the 256*NW counters in (digit, warp) order; thread t
  // owns the 8 consecutive entries j = 8t .. 8t+7 (digit j / NW, warp j % NW)
  constexpr int PER = NB * NW / NT;
  uint32_t loc[PER], sum = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const uint32_t jj = threadIdx.x * PER + j;
    loc[j] = cnt[(jj % NW) * kRadixRow + jj / NW];
    sum += loc[j];
  }
  uint32_t tot;
  uint32_t run = block_exclusive_scan<NT, uint32_t>(sum, &tot, tmp);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const uint32_t jj = threadIdx.x * PER + j;
    cnt[(jj % NW) * kRadixRow + jj / NW] = run;
    run += loc[j];
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t base = s; base < e; base += 32) {
    const uint32_t i = base + lane;
    const bool valid = i < e;
    K k = K(0);
    V v = V(0);
    uint32_t d = NB;
    if (valid) {
      k = a[i];
      if (HAS_VAL) v = va[i];
      d = digit(k, (uint32_t)v);
    }
    // full steps (warp-uniform) have no idle lane, whose digit NB needs a ninth bit
    const uint32_t peers = base + 32u <= e ? warp_peers<8>(d) : warp_peers<9>(d);
    const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
    uint32_t first = 0;
    if (valid && lane == leader) {
      first = row[d];
      row[d] = first + __popc(peers);
    }
    first = __shfl_sync(kFull, first, leader);
    if (valid) {
      const uint32_t pos = first + __popc(peers & lt);
      b[pos] = k;
      if (HAS_VAL) vb[pos] = v;
    }
    __syncwarp();  // the counter updates are seen by the next step's leaders
  }
  __syncthreads();
}

// ---------------------------------------------------------------- searches
// first index in [lo, hi) with key(a[i]) >= v (a sorted by key)
template <class F>
__device__ __forceinline__ uint32_t lower_bound_by(uint32_t lo, uint32_t hi, F key_less_than_v) {
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (key_less_than_v(mid)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- geometry
// Pseudo-angle ("diamond angle") in [0, 4), monotone in phi: one division,
// no transcendental function (so CPU and GPU agree bit for bit).
__device__ __forceinline__ float pseudo_angle(float x, float y) {
  float k;
  if (y >= 0.0f) {
    if (x >= 0.0f) {
      const float d = __fadd_rn(x, y);
      k = d > 0.0f ? __fdiv_rn(y, d) : 0.0f;
    } else {
      k = __fadd_rn(1.0f, __fdiv_rn(-x, __fsub_rn(y, x)));
    }
  } else {
    if (x < 0.0f) {
      k = __fadd_rn(2.0f, __fdiv_rn(-y, __fsub_rn(-x, y)));
    } else {
      k = __fadd_rn(3.0f, __fdiv_rn(x, __fsub_rn(x, y)));
    }
  }
  return __fadd_rn(k, 0.0f);  // -0 -> +0
}

// |a - b| on the circle of circumference 4
__device__ __forceinline__ float dmod4(float a, float b) {
  float d = fabsf(__fsub_rn(a, b));
  if (d > 2.0f) d = __fsub_rn(4.0f, d);
  return d;
}

// Candidate index ranges of a module's sorted keys that contain every key
// within half-width w of k on the circle [0, 4).  The ranges are a superset
// (margin 1e-5 >> rounding of k +- w); callers apply the exact dmod4 test to
// every candidate.
struct Ranges {
  uint32_t a0, a1, b0, b1;  // [a0, a1) and [b0, b1)
};

// Bucketed index of one module's sorted keys: bucket b holds the keys in
// [b/S, (b+1)/S), S = kKeyBuckets / 4 (the last one also a key rounded up to
// 4), tab[b] is the first module-local index of a key in bucket b or later,
// tab[kKeyBuckets] the count.  The buckets are fine (about half a hit each in
// a pile-up-5.5 module), so a window is searched as the whole buckets it
// touches, from the table alone: a key >= v lies in v's bucket or later, so
// at or after tab[bucket(v)], and a key <= v before tab[bucket(v) + 1].  The
// ranges are therefore supersets of the window (callers test every candidate
// exactly), and finding them reads no key.
#ifndef VELO_KEY_BUCKETS
#define VELO_KEY_BUCKETS 512
#endif
constexpr uint32_t kKeyBuckets = VELO_KEY_BUCKETS;
__device__ __forceinline__ uint32_t key_bucket(float v) {
  const float t = v * (float)(kKeyBuckets / 4);  // exact: a power of two
  return t <= 0.0f ? 0u : (t >= (float)(kKeyBuckets - 1) ? kKeyBuckets - 1 : (uint32_t)t);
}

struct KeyIndex {
  uint32_t lo;          // first position of the module
  const uint16_t* tab;  // kKeyBuckets + 1 module-local indices
};

__device__ __forceinline__ Ranges window_ranges(const KeyIndex& I, float k, float w) {
  const float eps = 1e-5f;
  const float a = k - w - eps, b = k + w + eps;
  const uint32_t lo = I.lo, hi = I.lo + I.tab[kKeyBuckets];
  auto first = [&](float v) { return lo + I.tab[key_bucket(v)]; };     // every key >= v is at or after it
  auto past = [&](float v) { return lo + I.tab[key_bucket(v) + 1]; };  // every key <= v is before it
  Ranges r;
  if (a < 0.0f) {
    r.a0 = lo;
    r.a1 = past(b);
    r.b0 = max(first(a + 4.0f), r.a1);
    r.b1 = hi;
  } else if (b >= 4.0f) {
    r.a0 = lo;
    r.a1 = past(b - 4.0f);
    r.b0 = max(first(a), r.a1);
    r.b1 = hi;
  } else {
    r.a0 = first(a);
    r.a1 = past(b);
    r.b0 = r.b1 = r.a1;
  }
  return r;
}

}  // namespace velo
