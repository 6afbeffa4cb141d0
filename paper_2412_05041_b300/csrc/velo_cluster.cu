// Clustering kernel: pixel words of one event -> clusters (hits).
//
// The first stage reconstructs every event from the raw detector data
// (Sec. "Data flow overview"); for the pixel tracker this starts with
// clustering.  One CTA per event at a time (1024 threads and one CTA per SM,
// or 512 threads and two; persistent, events from a work queue):
//   1. load and validate the event's words (coalesced, 4 B per thread);
//   2. sort by the 27-bit (module, row, col) key in shared memory: one
//      counting pass by (module, row) (2 radix passes where the counters do
//      not fit), then each row by insertion;
//   3. union-find over 8-connected neighbours found in the sorted array
//      (they sit just before a word): every word links to its smallest
//      earlier neighbour, and the few whose earlier neighbours are not
//      adjacent to one another unite with atomicMin, so every root ends as
//      the smallest sorted position of its component, i.e. its smallest
//      (module, row, col);
//   4. cluster id = exclusive scan of root flags (canonical, order-free);
//   5. integer charge sums per cluster with atomics (exact, so the order of
//      the additions does not matter) and the binary32 centroid;
//   6. pseudo-angle key and the sort of the hits by (module, key, id): in
//      shared memory one counting pass by (module, top 8 key bits) and an
//      insertion sort of every bucket (about one hit); else a stable block
//      radix sort, 3 passes over (module, 19-bit fixed-point key), then the
//      rare runs of equal fixed-point keys by insertion.
// Events larger than the shared-memory tier run the same code on their
// slice of the global workspace (generic pointers).
#include <type_traits>

#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "velo_device.cuh"
#include "velo_internal.cuh"

namespace velo {

namespace {

template <int NT>
struct ClusterSmem {
  uint32_t cnt[radix_counters(NT)];
  uint32_t tmp[64];
  uint32_t mod_count[VELO_MAX_MODULES];  // first cluster id of each module (kNone: no word)
  uint32_t mod_off[kModOffStride];
  uint32_t flag;
  uint32_t next;  // event taken from the work queue
  uint32_t pad[2];
};

constexpr uint32_t kRootFlag = 0x80000000u;
constexpr uint32_t kRowSortMax = 32;  // longest row sorted by insertion (else the full radix sort)
// key buckets per module of the counting hit sort: 2^8 (about one hit each
// at pile-up 5.5)
constexpr uint32_t kHitBucketBits = 8;
// Events of at least this many words (kept in the workspace) index the first
// sorted position of every (module, row): 32 modules x 2048 rows.
constexpr uint32_t kRowTable = 1u << 16;
// Sub-events (modules of heavy events) of at least this many words use a row
// table of their one module (2048 entries in their own word range).
constexpr uint32_t kSubRowTable = 4096;

__device__ __forceinline__ uint32_t vload(const uint32_t* p) { return *(const volatile uint32_t*)p; }

// Root of a, halving the path on the way: every node passed is linked to its
// grandparent.  parent[x] < x for every non-root and every write lowers a
// parent to a node of the same component (atomicMin, as the unions write),
// so the walk ends at the root within a steps and the forest stays one.
__device__ __forceinline__ uint32_t uf_find(uint32_t* parent, uint32_t a) {
  for (;;) {
    const uint32_t p = vload(parent + a);
    if (p == a) return a;
    const uint32_t gp = vload(parent + p);
    if (gp == p) return p;
    atomicMin(parent + a, gp);
    a = gp;
  }
}

// Link the larger root under the smaller.  A link attempt that loses a race
// (another union lowered the root first) retries from the new root; after
// `attempts` attempts the union gives up and returns false (never expected
// with the default bound of 2^20; the event then fails with
// VELO_EVT_TIMEOUT instead of looping).  With attempts = 0 every union that
// still has to link two trees gives up.
__device__ __forceinline__ bool uf_unite(uint32_t* parent, uint32_t a, uint32_t b, uint32_t attempts) {
  for (uint32_t it = 0;; ++it) {
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a == b) return true;
    if (it >= attempts) return false;
    if (a < b) {
      const uint32_t t = a;
      a = b;
      b = t;
    }
    const uint32_t old = atomicMin(parent + a, b);
    if (old == a) return true;
    a = old;
  }
}

// 19-bit fixed-point value of a pseudo-angle key in [0, 4] (a key can round
// up to 4): never decreases as the key grows (scaling by 2^17 is exact).
__device__ __forceinline__ uint32_t hit_key_fixed(float key) {
  const float t = key * 131072.0f;
  return t >= 524287.0f ? 524287u : (uint32_t)t;
}

__device__ __forceinline__ bool word_valid(uint32_t w, const Geo& g) {
  return (w >> 31) == 0u && ((w >> 27) & 15u) != 0u && ((w >> 22) & 31u) < g.n_modules &&
         ((w >> 11) & 2047u) < g.n_rows && (w & 2047u) < g.n_cols;
}

__device__ __forceinline__ uint32_t module_of(const uint32_t* mod_off, uint32_t n_modules, uint32_t id) {
  // largest m with mod_off[m] <= id
  uint32_t lo = 0, hi = n_modules;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (mod_off[mid] <= id) lo = mid;
    else hi = mid;
  }
  return lo;
}

// A sub-event: one module of a heavy event, clustered by one CTA of the
// heavy-event kernel (k_cluster_wide) in shared memory.  Its words come from
// the module-grouped copy of the event, with their positions in the event's
// input; its clusters take the event-wide ids id_base + local id and its hits
// the event-wide positions id_base + local position.  The event's own records
// (status, module offsets, counts, lists) are left to the heavy kernel, and a
// failure only raises *fail (the heavy kernel then fails the event).
struct Sub {
  bool on = false;
  const uint32_t* words = nullptr;  // the module's words
  const uint32_t* index = nullptr;  // their positions in the event's input
  uint64_t ev_p0 = 0;               // the event's first word
  uint32_t id_base = 0;             // event-wide id of the module's first cluster
  uint32_t* fail = nullptr;         // VELO_EVT_* code of a failure, 0 if none
  uint32_t* big = nullptr;          // set when the clusters are too many for the shared hit sort
};

__device__ void fail_event(const Launch& L, uint64_t e, int32_t code, bool offsets_ok, uint64_t p0, uint32_t n) {
  if (threadIdx.x == 0) {
    L.out.status[e] = code;
    L.ws.ev_nclusters[e] = 0;
  }
  if (threadIdx.x < kModOffStride) L.ws.ev_modoff[e * kModOffStride + threadIdx.x] = 0;
  if (offsets_ok && L.out.pixel_cluster)
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) L.out.pixel_cluster[p0 + i] = kNone;
}

}  // namespace

// Phases 2-5 on the event's n pixel words in A (B: the second buffer), in
// shared memory when PS (so that the sorts, the union-find and its atomics
// compile to shared-memory instructions), else in the event's global slice.
// Returns the cluster count, or kNone after failing the event; *sums gets
// the 32-bit charge sums (3 per cluster) when they were kept in 32 bits.
template <int NT, bool PS>
__device__ __forceinline__ uint32_t pixel_phases(const Launch& L, const uint64_t e, ClusterSmem<NT>& S,
                                                 uint32_t* region, const uint32_t tier, const uint64_t p0,
                                                 const uint32_t n, uint32_t** sums, const Sub& sub) {
  const Workspace& W = L.ws;
  const uint32_t tid = threadIdx.x;
  const uint32_t M = L.geo.n_modules;
  uint32_t* A = PS ? region : W.sa + p0;
  uint32_t* B = PS ? region + n : W.sb + p0;

  // 2. sort by (module, row, col).  In shared memory, when 16-bit counters
  // per group fit after the two word arrays -- a group is a (module, row), or
  // a (module, row pair) for larger events -- by one counting pass: counts,
  // their exclusive scan, and a scatter whose atomics give the words of a
  // group their places in arbitrary order (A -> B) and leave every group's
  // end in its counter; then every word takes its place in (row, column)
  // order inside its group by counting the group's words that precede it
  // (a smaller key, or an equal key at an earlier place: B -> A).  Groups
  // hold a few words in a pile-up event.  Otherwise by two stable LSD passes
  // by (module, row) and an insertion sort of every row by the thread that
  // owns its first word; a row of more than kRowSortMax words sends the whole
  // array to the full sort by the key (4 passes).  (Events of kRowTable
  // words or more -- dense modules, long rows -- take the full sort at once.)
  // Words with equal keys (duplicates) may end in any order among
  // themselves, and nothing that follows depends on it: they share one
  // cluster, their charges add without order, and every label is found by
  // key.
  bool long_row = !PS && n >= kRowTable;
  bool counted = false;
  if constexpr (PS) {
    const uint32_t nrow = L.geo.n_rows;
    const uint32_t Mg = sub.on ? 1u : M;  // a sub-event's words all lie on one module
    bool fits = false;
    uint32_t gshift = 11, ngrp = nrow, cw = 0;  // group = key >> gshift: (module, row), else (module, row pair)
    for (int pass = 0; pass < 2 && !fits; ++pass) {
      gshift = 11u + (uint32_t)pass;
      ngrp = (nrow + (uint32_t)pass) >> pass;
      cw = (Mg * ngrp + 1u) / 2u;  // u32 words of 16-bit counter pairs
      fits = n < 65536u && 2u * n + cw <= 2u * tier;
    }
    if (fits) {
      counted = true;
      uint32_t* C = region + 2 * n;
      const uint32_t rmask = 2047u >> (gshift - 11u);
      auto group = [&](uint32_t w) { return (sub.on ? 0u : (w >> 22) & 31u) * ngrp + ((w >> gshift) & rmask); };
      for (uint32_t q = tid; q < cw; q += NT) C[q] = 0u;
      __syncthreads();
      for (uint32_t i = tid; i < n; i += NT) {
        const uint32_t b = group(A[i]);
        atomicAdd(C + (b >> 1), 1u << ((b & 1u) << 4));
      }
      __syncthreads();
      // exclusive scan of the counts in group order: a chunk of an odd
      // number of words per thread (no bank conflicts), one block scan
      const uint32_t per = ((cw + NT - 1) / NT) | 1u;
      const uint32_t q0 = min(cw, tid * per), q1 = min(cw, q0 + per);
      uint32_t sum = 0;
      for (uint32_t q = q0; q < q1; ++q) {
        const uint32_t v = C[q];
        sum += (v & 0xFFFFu) + (v >> 16);
      }
      uint32_t total;
      uint32_t run = block_exclusive_scan<NT, uint32_t>(sum, &total, S.tmp);
      for (uint32_t q = q0; q < q1; ++q) {  // prefixes < n < 2^16
        const uint32_t v = C[q], lo = run, hi = run + (v & 0xFFFFu);
        run = hi + (v >> 16);
        C[q] = lo | hi << 16;
      }
      __syncthreads();
      for (uint32_t i = tid; i < n; i += NT) {
        const uint32_t w = A[i], b = group(w), sh = (b & 1u) << 4;
        B[(atomicAdd(C + (b >> 1), 1u << sh) >> sh) & 0xFFFFu] = w;
      }
      __syncthreads();
      // every counter now holds its group's end (start + count, < n < 2^16)
      auto group_end = [&](uint32_t b) { return (C[b >> 1] >> ((b & 1u) << 4)) & 0xFFFFu; };
      for (uint32_t p = tid; p < n; p += NT) {
        const uint32_t w = B[p], k = w & kKeyMask, b = group(w);
        const uint32_t s0 = b ? group_end(b - 1u) : 0u, s1 = group_end(b);
        uint32_t r = s0;
        for (uint32_t q = s0; q < s1; ++q) {
          const uint32_t kq = B[q] & kKeyMask;
          r += kq < k || (kq == k && q < p);
        }
        A[r] = w;
      }
      __syncthreads();
    }
  }
  if (!long_row && !counted) {
    radix_pass<NT, false>(A, B, (const uint32_t*)nullptr, (uint32_t*)nullptr, n,
                          [](uint32_t k, uint32_t) { return ((k & kKeyMask) >> 11) & 255u; }, S.cnt, S.tmp);
    radix_pass<NT, false>(B, A, (const uint32_t*)nullptr, (uint32_t*)nullptr, n,
                          [](uint32_t k, uint32_t) { return (k & kKeyMask) >> 19; }, S.cnt, S.tmp);
  }
  // After the LSD passes every row's words are contiguous, in any column
  // order.  The thread that holds a row's first word (the word before it lies
  // in another row) puts the row in column order by insertion when it has
  // more than one word.  Rows only permute inside themselves, and a word's
  // row never changes, so the row tests of the other threads read the same
  // rows while a row is being sorted.
  if (!counted && (PS || n < kRowTable)) {
    for (uint32_t pos = tid; pos < n; pos += NT) {
      const uint32_t mr = (A[pos] & kKeyMask) >> 11;
      if (pos > 0 && ((A[pos - 1] & kKeyMask) >> 11) == mr) continue;   // not the row's first word
      if (pos + 1 >= n || ((A[pos + 1] & kKeyMask) >> 11) != mr) continue;  // a row of one word
      uint32_t end = pos + 2;
      while (end < n && end - pos <= kRowSortMax && ((A[end] & kKeyMask) >> 11) == mr) ++end;
      if (end - pos > kRowSortMax) {
        long_row = true;
        continue;
      }
      for (uint32_t a = pos + 1; a < end; ++a) {
        const uint32_t wa = A[a], ka = wa & kKeyMask;
        uint32_t b = a;
        for (; b > pos && (A[b - 1] & kKeyMask) > ka; --b) A[b] = A[b - 1];
        A[b] = wa;
      }
    }
  }
  if (__syncthreads_or(long_row)) {
    radix_pass<NT, false>(A, B, (const uint32_t*)nullptr, (uint32_t*)nullptr, n,
                          [](uint32_t k, uint32_t) { return (k & kKeyMask) & 255u; }, S.cnt, S.tmp);
    radix_pass<NT, false>(B, A, (const uint32_t*)nullptr, (uint32_t*)nullptr, n,
                          [](uint32_t k, uint32_t) { return ((k & kKeyMask) >> 8) & 255u; }, S.cnt, S.tmp);
    radix_pass<NT, false>(A, B, (const uint32_t*)nullptr, (uint32_t*)nullptr, n,
                          [](uint32_t k, uint32_t) { return ((k & kKeyMask) >> 16) & 255u; }, S.cnt, S.tmp);
    radix_pass<NT, false>(B, A, (const uint32_t*)nullptr, (uint32_t*)nullptr, n,
                          [](uint32_t k, uint32_t) { return (k & kKeyMask) >> 24; }, S.cnt, S.tmp);
  }

  // 3. union-find over 8-connected neighbours.  Every earlier neighbour of
  // word i has a key in [lo_all, k]: duplicates (k), the left neighbour
  // (k - 1) and, if r > 0, the previous row's columns c-1 .. c+1 ([lo_k,
  // hi_k]).  Those keys sit just before i in the sorted array, so a backward
  // scan that stops below lo_all sees all of them; the words of a sparse
  // event are a few rows apart, so it usually stops within a few steps.
  // Pass a links every word, without atomics, to its smallest earlier
  // neighbour (parent < child: a forest).  That is all a word needs when its
  // earlier neighbours are connected among themselves: each edge between two
  // of them is taken care of by the later one (by induction on the sorted
  // position, every word ends in one component with all its earlier
  // neighbours).  Among the left (L), up-left (UL), up (U) and up-right (UR)
  // positions only L-UR and UL-UR are not adjacent, so the earlier
  // neighbours fail to be connected only when UR is there without U but with
  // L or UL (a duplicate of the word itself touches them all).  Those words,
  // and words whose scan ran past 16 steps, are flagged in bit 31 of their
  // word (never set in a valid word; every reader masks it) and, in pass b,
  // united with each of their earlier neighbours (the full search past 16
  // steps), linking the larger root under the smaller with atomicMin.  Every
  // root of pass a has no earlier neighbour, and each union keeps the smaller
  // root, so every component ends with its smallest sorted position, i.e. its
  // smallest (module, row, col), as root -- whatever the thread order.
  bool ok = true;
  if ((!PS && n >= kRowTable) || (sub.on && n >= kSubRowTable)) {
    // Large events (words in the workspace) and large sub-events (the dense
    // modules of heavy events): a table of the first sorted position of every
    // (module, row) -- in the hit-sort scratch, free until then; a sub-event's
    // rows of its one module, module * 2048 + row at rt[row] -- gives the
    // previous row's words directly, so every word finds all its earlier
    // neighbours (duplicates and the left neighbour just before it, the
    // previous row by bisection of that row) and only the V-shaped ones are
    // united in pass b.
    const uint32_t rbase = sub.on ? ((A[0] & kKeyMask) >> 22) << 11 : 0u;
    const uint32_t rsize = sub.on ? 2048u : kRowTable;
    uint32_t* rt = W.sc + p0;  // rt[mr - rbase] for mr = module * 2048 + row
    auto row_start = [&](uint32_t mr) { return rt[mr - rbase]; };
    for (uint32_t q = tid; q < rsize; q += NT) rt[q] = n;
    __syncthreads();
    for (uint32_t pos = tid; pos < n; pos += NT) {
      const uint32_t mr = (A[pos] & kKeyMask) >> 11, mp = pos ? ((A[pos - 1] & kKeyMask) >> 11) + 1u : rbase;
      for (uint32_t q = mp; q <= mr; ++q) rt[q - rbase] = pos;
    }
    __syncthreads();
    for (uint32_t i = tid; i < n; i += NT) {
      const uint32_t k = A[i] & kKeyMask;
      const uint32_t c = k & 2047u, r = (k >> 11) & 2047u;
      bool dup = false, left = false, up_left = false, up = false, up_right = false;
      uint32_t nb_min = i;
      for (int64_t j = (int64_t)i - 1; j >= 0; --j) {  // duplicates, then the left neighbour's copies
        const uint32_t kj = A[j] & kKeyMask;
        if (kj == k) dup = true;
        else if (c > 0u && kj == k - 1u) left = true;
        else break;
        nb_min = (uint32_t)j;
      }
      if (r > 0u) {
        const uint32_t lo_k = k - 2048u - (c > 0u ? 1u : 0u), hi_k = k - 2048u + (c + 1u < L.geo.n_cols ? 1u : 0u);
        const uint32_t mr = k >> 11;
        uint32_t j = lower_bound_by(row_start(mr - 1u), row_start(mr), [&](uint32_t x) { return (A[x] & kKeyMask) < lo_k; });
        if (j < row_start(mr) && (A[j] & kKeyMask) <= hi_k) nb_min = j;  // the smallest earlier neighbour
        for (; j < row_start(mr); ++j) {
          const uint32_t pc = A[j] & 2047u;  // previous-row column c-1, c or c+1
          if ((A[j] & kKeyMask) > hi_k) break;
          up_left |= pc + 1u == c;
          up |= pc == c;
          up_right |= pc == c + 1u;
        }
      }
      B[i] = nb_min;
      if (up_right && !up && (left || up_left) && !dup) A[i] |= 0x80000000u;
    }
    __syncthreads();
    for (uint32_t i = tid; i < n; i += NT) {
      if (!(A[i] >> 31)) continue;
      const uint32_t k = A[i] & kKeyMask;
      const uint32_t c = k & 2047u, r = (k >> 11) & 2047u;
      for (int64_t j = (int64_t)i - 1; j >= 0; --j) {
        const uint32_t kj = A[j] & kKeyMask;
        if (kj != k && !(c > 0u && kj == k - 1u)) break;
        ok &= uf_unite(B, i, (uint32_t)j, L.union_link_attempts);
      }
      if (r > 0u) {
        const uint32_t lo_k = k - 2048u - (c > 0u ? 1u : 0u), hi_k = k - 2048u + (c + 1u < L.geo.n_cols ? 1u : 0u);
        const uint32_t mr = k >> 11;
        uint32_t j = lower_bound_by(row_start(mr - 1u), row_start(mr), [&](uint32_t x) { return (A[x] & kKeyMask) < lo_k; });
        for (; j < row_start(mr) && (A[j] & kKeyMask) <= hi_k; ++j) ok &= uf_unite(B, i, j, L.union_link_attempts);
      }
    }
  } else {
    // Every earlier word j in reach has d = k - key(j) <= span = k - lo_all;
    // d = 0 is a duplicate, 1 the left neighbour (c > 0), 2047 / 2048 / 2049
    // the previous row's columns c+1 (c+1 < n_cols), c, c-1 (c > 0): bits 0-4
    // of `seen` (a previous row is in reach only when r > 0).
    for (uint32_t i = tid; i < n; i += NT) {
      const uint32_t k = A[i] & kKeyMask;
      const uint32_t c = k & 2047u, r = (k >> 11) & 2047u;
      const uint32_t span = r > 0u ? 2048u + (c > 0u ? 1u : 0u) : (c > 0u ? 1u : 0u);
      const uint32_t allow = 9u | (c > 0u ? 18u : 0u) | (c + 1u < L.geo.n_cols ? 4u : 0u);
      bool done = false;
      uint32_t seen = 0, nb_min = i, j = i;
      for (int steps = 0; steps < 16; ++steps) {
        if (j == 0u) {
          done = true;
          break;
        }
        --j;
        const uint32_t d = k - (A[j] & kKeyMask);
        if (d > span) {
          done = true;
          break;
        }
        const uint32_t bit = (d <= 1u ? 1u << d : (d - 2047u <= 2u ? 4u << (d - 2047u) : 0u)) & allow;
        if (bit) nb_min = j;  // scanning down: the last one found is the smallest
        seen |= bit;
      }
      B[i] = nb_min;
      // the V shape: up-right without up, with left or up-left, no duplicate
      if (!done || ((seen & 29u) == 4u + (seen & 16u) && (seen & 18u) != 0u)) A[i] |= 0x80000000u;
    }
    __syncthreads();
    for (uint32_t i = tid; i < n; i += NT) {
      if (!(A[i] >> 31)) continue;
      const uint32_t k = A[i] & kKeyMask;
      const uint32_t c = k & 2047u, r = (k >> 11) & 2047u;
      const uint32_t lo_k = r > 0u ? k - 2048u - (c > 0u ? 1u : 0u) : 0u;
      const uint32_t hi_k = r > 0u ? k - 2048u + (c + 1u < L.geo.n_cols ? 1u : 0u) : 0u;
      const uint32_t lo_all = r > 0u ? lo_k : (c > 0u ? k - 1u : k);
      bool done = false;
      int64_t j = (int64_t)i - 1;
      for (int steps = 0; steps < 16; ++steps, --j) {
        if (j < 0) {
          done = true;
          break;
        }
        const uint32_t kj = A[j] & kKeyMask;
        if (kj < lo_all) {
          done = true;
          break;
        }
        if (kj == k || (c > 0u && kj == k - 1u) || (r > 0u && kj >= lo_k && kj <= hi_k))
          ok &= uf_unite(B, i, (uint32_t)j, L.union_link_attempts);
      }
      if (!done) {  // past 16 steps (unions are idempotent: a neighbour seen twice is harmless)
        // duplicates of k and the left neighbour (k - 1) are the words just before i
        for (int64_t jj = (int64_t)i - 1; jj >= 0; --jj) {
          const uint32_t kj = A[jj] & kKeyMask;
          if (kj == k || (c > 0u && kj == k - 1u)) ok &= uf_unite(B, i, (uint32_t)jj, L.union_link_attempts);
          else break;
        }
        if (r > 0u) {  // previous row, columns c-1 .. c+1 of the same module
          uint32_t jj = lower_bound_by(0u, i, [&](uint32_t x) { return (A[x] & kKeyMask) < lo_k; });
          for (; jj < i && (A[jj] & kKeyMask) <= hi_k; ++jj) ok &= uf_unite(B, i, jj, L.union_link_attempts);
        }
      }
    }
  }
  if (!ok) S.flag = 2u;
  __syncthreads();
  if (S.flag) {  // a union gave up after its bounded link attempts
    if (sub.on) {
      if (tid == 0) atomicMax(sub.fail, (uint32_t)VELO_EVT_TIMEOUT);
      return kNone;
    }
    fail_event(L, e, VELO_EVT_TIMEOUT, true, p0, n);
    return kNone;
  }
  // every word to its root (the walks halve their paths with atomicMin, so a
  // word whose root is already written keeps it: the root is the smallest)
  for (uint32_t i = tid; i < n; i += NT) B[i] = uf_find(B, i);
  __syncthreads();

  // 4. cluster ids: rank of each root among the roots.  Every warp takes a
  // contiguous chunk, 32 words at a time (coalesced): a ballot counts its
  // roots, a block scan over the warps gives each chunk its first rank, a
  // second ballot pass numbers the roots.  Then every word takes its root's
  // rank; the first word of a module is a root (no earlier neighbour there),
  // so its rank is the module's first cluster id.
  constexpr uint32_t NW = NT / 32;
  const uint32_t lane = lane_id(), wid = warp_id();
  const uint32_t cw = ((n + NW - 1) / NW + 31u) & ~31u;
  const uint32_t wlo = min(n, wid * cw), whi = min(n, wlo + cw);
  uint32_t wroots = 0;
  for (uint32_t base = wlo; base < whi; base += 32) {
    const uint32_t i = base + lane;
    wroots += __popc(__ballot_sync(kFull, i < whi && B[i] == i));
  }
  uint32_t n_clusters;
  uint32_t rank = block_exclusive_scan<NT, uint32_t>(lane == 0 ? wroots : 0u, &n_clusters, S.tmp);
  rank = __shfl_sync(kFull, rank, 0);
  // where the charge sums of phase 5 go (known now that n_clusters is): with
  // at most kNarrowPixels words, sum q(2c+1) <= 15 * 4095 * 23552 < 2^32, so
  // 32-bit sums (and a 32-bit division) are exact; larger events use 64 bits.
  // The 32-bit sums go to shared memory after the two pixel arrays (free
  // since the row sort) when they fit there and clear of the hit sort's keys
  // and first ids ([0, 2.5 n_c) words), which the centroid pass writes while
  // it reads the sums.  Their layout: a 64-bit word per cluster holding the
  // charge sum (< 15 * 23552 < 2^27, above it the cluster's module in bits
  // 27-31) in its high half and the row sum sum q(2r+1) (< 2^32, so no carry
  // ever reaches the high half) in its low half -- one atomic adds both --
  // then a 32-bit column sum per cluster: 3 n_c words from an 8-byte aligned
  // start.  Every root starts its cluster's sums with its module.
  const bool narrow = n <= kNarrowPixels;
  unsigned long long* acc = W.acc + 3 * p0;
  const bool sums_smem = PS && narrow && 2u * n + 3u * n_clusters + 1u <= 2u * tier && 5u * n_clusters <= 4u * n;
  uint32_t* acc32 = reinterpret_cast<uint32_t*>(acc);  // global: in this event's slice (8-byte aligned)
  if (sums_smem) {
    uintptr_t a = reinterpret_cast<uintptr_t>(region + 2 * n);
    acc32 = reinterpret_cast<uint32_t*>(a + (a & 4u));  // the next 8-byte boundary
  }
  unsigned long long* qy64 = reinterpret_cast<unsigned long long*>(acc32);  // (charge | module, row sum)
  uint32_t* qx32 = acc32 + 2 * n_clusters;                                    // column sums
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t base = wlo; base < whi; base += 32) {
    const uint32_t i = base + lane;
    const bool root = i < whi && B[i] == i;
    const uint32_t bal = __ballot_sync(kFull, root);
    if (root) {
      const uint32_t id = rank + __popc(bal & lt);
      B[i] = id | kRootFlag;
      if (narrow) {
        qy64[id] = (unsigned long long)(((A[i] >> 22) & 31u) << 27) << 32;
        qx32[id] = 0u;
      }
    }
    rank += __popc(bal);
  }
  __syncthreads();
  for (uint32_t i = tid; i < n; i += NT) {
    const uint32_t v = B[i];
    const uint32_t id = (v & kRootFlag) ? (v & ~kRootFlag) : (vload(B + v) & ~kRootFlag);
    B[i] = id;
    const uint32_t m = (A[i] >> 22) & 31u;
    if (i == 0 || m != ((A[i - 1] >> 22) & 31u)) S.mod_count[m] = id;  // the module's first cluster id
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t o = n_clusters;
    S.mod_off[M] = o;
    for (int m = (int)M - 1; m >= 0; --m) {
      const uint32_t f = S.mod_count[m];
      if (f != kNone) {
        if (o - f > VELO_MAX_MODULE_CLUSTERS) S.flag = 3u;
        o = f;
      }
      S.mod_off[m] = o;  // an empty module starts where the next one does
    }
  }
  __syncthreads();
  if (S.flag) {
    if (sub.on) {
      if (tid == 0) atomicMax(sub.fail, (uint32_t)VELO_EVT_OVERFLOW);
      return kNone;
    }
    fail_event(L, e, VELO_EVT_OVERFLOW, true, p0, n);
    return kNone;
  }

  // optional per-word labels in input order (a sub-event's at its words' event positions)
  if (L.out.pixel_cluster) {
    for (uint32_t i = tid; i < n; i += NT) {
      const uint32_t k = (sub.on ? sub.words[i] : __ldg(L.pix + p0 + i)) & kKeyMask;
      const uint32_t j = lower_bound_by(0u, n, [&](uint32_t x) { return (A[x] & kKeyMask) < k; });
      const uint32_t label = j < n ? sub.id_base + B[j] : kNone;  // j < n always: the word is in A
      L.out.pixel_cluster[sub.on ? sub.ev_p0 + sub.index[i] : p0 + i] = label;
    }
  }

  // 5. integer charge sums per cluster (32-bit ones started by the roots in
  // phase 4), then the binary32 centroid.
  *sums = acc32;
  if (!narrow) {
    for (uint32_t i = tid; i < 3 * n_clusters; i += NT) acc[i] = 0ull;
    __syncthreads();
  }
  for (uint32_t i = tid; i < n; i += NT) {
    const uint32_t w = A[i];
    const uint32_t q = (w >> 27) & 15u, c = w & 2047u, r = (w >> 11) & 2047u;
    if (narrow) {
      const uint32_t id = B[i];
      atomicAdd(qy64 + id, (unsigned long long)q << 32 | (unsigned long long)(q * (2u * r + 1u)));
      atomicAdd(qx32 + id, q * (2u * c + 1u));
    } else {
      unsigned long long* a3 = acc + 3ull * B[i];
      atomicAdd(a3 + 0, (unsigned long long)q);
      atomicAdd(a3 + 1, (unsigned long long)(q * (2u * c + 1u)));
      atomicAdd(a3 + 2, (unsigned long long)(q * (2u * r + 1u)));
    }
  }
  __syncthreads();
  return n_clusters;
}

// Centroids, pseudo-angle keys and the hit sort of the event's n_clusters
// clusters (charge sums: acc32 when 32-bit, else the 64-bit workspace
// sums), through shared memory when HS.
template <int NT, bool HS>
__device__ __forceinline__ void hit_phases(const Launch& L, const uint64_t e, ClusterSmem<NT>& S, uint32_t* region,
                                           const uint32_t tier, const uint64_t p0, const uint32_t n,
                                           const uint32_t n_clusters, const uint32_t* acc32, const Sub& sub) {
  const Workspace& W = L.ws;
  const uint32_t tid = threadIdx.x;
  const uint32_t M = L.geo.n_modules;
  const bool narrow = n <= kNarrowPixels;
  const unsigned long long* acc = W.acc + 3 * p0;
  // the pixel arrays are dead from here on.  In shared memory (HS) the hit
  // sort keeps its keys (32-bit) and cluster ids (16-bit: fewer than 2^16
  // clusters here) with their ping-pong copies, 12 bytes per cluster; the
  // cluster x, y and pseudo-angle key, read once at the end, go to global
  // scratch (cl_xy, and sc, unused by the shared tier; in the global tier
  // h_pos, written only at the end).
  using V = typename std::conditional<HS, uint16_t, uint32_t>::type;
  uint32_t* KA = HS ? region : W.sa + p0;
  uint32_t* KB = HS ? region + n_clusters : W.sb + p0;
  V* VA = HS ? reinterpret_cast<V*>(region + 2 * n_clusters) : reinterpret_cast<V*>(W.sc + p0);
  V* VB = HS ? reinterpret_cast<V*>(region + 2 * n_clusters) + n_clusters : reinterpret_cast<V*>(W.sd + p0);
  float2* cxy = sub.on ? W.cl_xy + sub.ev_p0 + sub.id_base : W.cl_xy + p0;  // by (local) id
  float* ck = reinterpret_cast<float*>(HS ? W.sc + p0 : W.h_pos + p0);
  const Geo& g = L.geo;
  const uint32_t* mo = S.mod_off;
  // In shared memory, when 16-bit counters of 2^kHitBucketBits key buckets
  // per module fit at the region's end (clear of the charge sums, which the
  // centroid pass reads), the hit sort is one counting pass by (module, top
  // key bits) and an insertion sort of every bucket -- about one hit each
  // -- by (key, id).
  const uint32_t cwh = (M << kHitBucketBits) / 2u;  // u32 words of 16-bit counter pairs
  const uint32_t c0 = 2u * tier - cwh;
  const bool counted = HS && n_clusters < 65536u && 2u * tier >= cwh && c0 >= 3u * n_clusters &&
                       (acc32 < region || acc32 >= region + 2u * tier || c0 >= 2u * n + 3u * n_clusters + 1u);
  uint32_t* C = region + c0;
  if (counted) {
    for (uint32_t q = tid; q < cwh; q += NT) C[q] = 0u;
    __syncthreads();
  }
  for (uint32_t id = tid; id < n_clusters; id += NT) {
    float u, v;
    uint32_t mod;
    if (narrow) {
      const unsigned long long qy = reinterpret_cast<const unsigned long long*>(acc32)[id];
      const uint32_t s0 = (uint32_t)(qy >> 32), sny = (uint32_t)qy, snx = acc32[2 * n_clusters + id];
      const uint32_t sq = s0 & 0x7FFFFFFu;
      mod = s0 >> 27;
      const uint32_t D = 2u * sq;
      const float Df = __uint2float_rn(D);
      u = __fadd_rn(__uint2float_rn(snx / D), __fdiv_rn(__uint2float_rn(snx % D), Df));
      v = __fadd_rn(__uint2float_rn(sny / D), __fdiv_rn(__uint2float_rn(sny % D), Df));
    } else {
      const unsigned long long sq = acc[3 * id], snx = acc[3 * id + 1], sny = acc[3 * id + 2];
      mod = module_of(mo, M, id);
      const unsigned long long D = 2ull * sq;
      const float Df = __ull2float_rn(D);
      u = __fadd_rn(__ull2float_rn(snx / D), __fdiv_rn(__ull2float_rn(snx % D), Df));
      v = __fadd_rn(__ull2float_rn(sny / D), __fdiv_rn(__ull2float_rn(sny % D), Df));
    }
    const float x = __fadd_rn(g.x0, __fmul_rn(g.pitch, u));
    const float y = __fadd_rn(g.y0, __fmul_rn(g.pitch, v));
    const float key = pseudo_angle(x, y);
    cxy[id] = make_float2(x, y);
    if (counted) {  // key bits and bucket (< 2^16) of every cluster
      const uint32_t b = mod << kHitBucketBits | hit_key_fixed(key) >> (19 - kHitBucketBits);
      KA[id] = __float_as_uint(key);
      VA[id] = (V)b;
      atomicAdd(C + (b >> 1), 1u << ((b & 1u) << 4));
    } else {
      ck[id] = key;
      KA[id] = mod << 19 | hit_key_fixed(key);
      VA[id] = (V)id;
    }
  }
  __syncthreads();
  if (counted) {
    // exclusive scan of the bucket counts (a chunk of an odd number of words
    // per thread, one block scan), the scatter of (key, id) into KB, VB, and
    // every bucket [end of the previous one, its end) in (key, id) order
    const uint32_t per = ((cwh + NT - 1) / NT) | 1u;
    const uint32_t q0 = min(cwh, tid * per), q1 = min(cwh, q0 + per);
    uint32_t sum = 0;
    for (uint32_t q = q0; q < q1; ++q) {
      const uint32_t v = C[q];
      sum += (v & 0xFFFFu) + (v >> 16);
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<NT, uint32_t>(sum, &total, S.tmp);
    for (uint32_t q = q0; q < q1; ++q) {  // prefixes < n_clusters < 2^16
      const uint32_t v = C[q], lo = run, hi = run + (v & 0xFFFFu);
      run = hi + (v >> 16);
      C[q] = lo | hi << 16;
    }
    __syncthreads();
    for (uint32_t id = tid; id < n_clusters; id += NT) {
      const uint32_t b = VA[id], sh = (b & 1u) << 4;
      const uint32_t slot = (atomicAdd(C + (b >> 1), 1u << sh) >> sh) & 0xFFFFu;
      KB[slot] = KA[id];
      VB[slot] = (V)id;
    }
    __syncthreads();
    for (uint32_t b = tid; b < 2u * cwh; b += NT) {  // C now holds every bucket's end
      const uint32_t end = (C[b >> 1] >> ((b & 1u) << 4)) & 0xFFFFu;
      const uint32_t beg = b ? (C[(b - 1) >> 1] >> (((b - 1) & 1u) << 4)) & 0xFFFFu : 0u;
      for (uint32_t a = beg + 1; a < end; ++a) {
        const uint32_t ka = KB[a];
        const V va = VB[a];
        uint32_t q = a;
        for (; q > beg && (KB[q - 1] > ka || (KB[q - 1] == ka && VB[q - 1] > va)); --q) {
          KB[q] = KB[q - 1];
          VB[q] = VB[q - 1];
        }
        KB[q] = ka;
        VB[q] = va;
      }
    }
    __syncthreads();
  } else {
    // 6. hits sorted by (module, key, id).  The ids enter in ascending order,
    // and three stable LSD passes sort them by (module, fixed-point key): the
    // fixed-point value never decreases with the key, so only hits of one
    // module with equal fixed-point keys can still be out of (key, id) order;
    // those runs (rare: a few per event) are put in order by insertion.
    radix_pass<NT, true>(KA, KB, VA, VB, n_clusters, [](uint32_t k, uint32_t) { return k & 255u; }, S.cnt, S.tmp);
    radix_pass<NT, true>(KB, KA, VB, VA, n_clusters, [](uint32_t k, uint32_t) { return (k >> 8) & 255u; }, S.cnt,
                         S.tmp);
    radix_pass<NT, true>(KA, KB, VA, VB, n_clusters, [](uint32_t k, uint32_t) { return k >> 16; }, S.cnt, S.tmp);
    for (uint32_t pos = tid; pos < n_clusters; pos += NT) {
      const uint32_t c = KB[pos];
      if ((pos > 0 && KB[pos - 1] == c) || pos + 1 >= n_clusters || KB[pos + 1] != c) continue;
      uint32_t end = pos + 2;  // this thread owns the run [pos, end)
      while (end < n_clusters && KB[end] == c) ++end;
      for (uint32_t a = pos + 1; a < end; ++a) {
        const uint32_t id = VB[a];
        const unsigned long long kv = (unsigned long long)__float_as_uint(ck[id]) << 32 | id;
        uint32_t b = a;
        for (; b > pos; --b) {
          const uint32_t o = VB[b - 1];
          if (((unsigned long long)__float_as_uint(ck[o]) << 32 | o) <= kv) break;
          VB[b] = (V)o;
        }
        VB[b] = (V)id;
      }
    }
    __syncthreads();
    // the keys in sorted order through KA (dead after the last pass)
    for (uint32_t pos = tid; pos < n_clusters; pos += NT) KA[pos] = __float_as_uint(ck[VB[pos]]);
    __syncthreads();
  }
  const uint32_t* KS = counted ? KB : KA;  // the keys (bits) in sorted order
  for (uint32_t pos = tid; pos < n_clusters; pos += NT) {
    const uint32_t id = VB[pos];
    const float2 c = cxy[id];
    const uint64_t base = sub.on ? sub.ev_p0 + sub.id_base : p0;  // a sub-event's hits at their event-wide places
    W.hit[base + pos] = make_float4(c.x, c.y, __uint_as_float(KS[pos]), __uint_as_float(sub.id_base + id));
    W.h_pos[base + id] = sub.id_base + pos;
  }
  if (sub.on) return;  // the heavy kernel writes the event's records
  if (tid <= M) W.ev_modoff[e * kModOffStride + tid] = S.mod_off[tid];
  if (tid == 0) {
    W.ev_nclusters[e] = n_clusters;
    L.out.status[e] = VELO_EVT_OK;
    if (n_clusters >= kWideClusters) W.wide_list[atomicAdd(W.queue + 3, 1u)] = (uint32_t)e;
  }
}

// The clustering of event e by one CTA of NT threads; `tier` = most words
// kept in shared memory (the region holds 2 * tier words).
// (With sub.on: module m of a heavy event, whose words lie at [p0, p0 + n) of
// the event's word slices: the sub-event's scratch.)
template <int NT>
__device__ __forceinline__ uint32_t cluster_one(const Launch& L, const uint64_t e, ClusterSmem<NT>& S, uint32_t* region,
                                            const uint32_t tier, const Sub& sub = Sub(), uint64_t sub_p0 = 0,
                                            uint32_t sub_n = 0) {
  const Workspace& W = L.ws;
  const uint32_t tid = threadIdx.x;

  const bool offsets_ok = sub.on || *(const volatile uint32_t*)W.flag == 0u;
  uint64_t p0 = 0, p1 = 0;
  if (sub.on) {
    p0 = sub_p0;
    p1 = sub_p0 + sub_n;
  } else if (offsets_ok) {
    p0 = L.off[e];
    p1 = L.off[e + 1];
  }
  const uint32_t n = (uint32_t)(p1 - p0);
  if (tid == 0) S.flag = offsets_ok ? 0u : 1u;
  if (tid < VELO_MAX_MODULES) S.mod_count[tid] = kNone;
  // the words of event e + gridDim.x (taken, most likely, in the next round
  // by some CTA) into L2 meanwhile, one 128-byte line per thread at a time
  // (the offsets are valid: every range lies inside the pixel array)
  if (!sub.on && offsets_ok && e + gridDim.x < L.n_events) {
    const uint64_t q0 = L.off[e + gridDim.x], q1 = L.off[e + gridDim.x + 1];
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(L.pix + q0) & ~uintptr_t(127);
    const uintptr_t a1 = reinterpret_cast<uintptr_t>(L.pix + q1);
    for (uintptr_t a = a0 + 128u * tid; a < a1; a += 128u * NT) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
  }
  __syncthreads();

  // 1. load + validate
  const bool smem_tier = n <= tier;
  uint32_t* A = smem_tier ? region : W.sa + p0;
  if (offsets_ok) {
    bool bad = false;
#pragma unroll 4
    for (uint32_t i = tid; i < n; i += NT) {
      const uint32_t w = sub.on ? sub.words[i] : __ldg(L.pix + p0 + i);
      bad |= !word_valid(w, L.geo);
      A[i] = w;
    }
    if (bad) S.flag = 1u;
  }
  __syncthreads();
  if (S.flag) {
    if (sub.on) {  // the heavy kernel validated the words (not expected)
      if (tid == 0) atomicMax(sub.fail, (uint32_t)VELO_EVT_BADWORD);
      return kNone;
    }
    fail_event(L, e, VELO_EVT_BADWORD, offsets_ok, p0, n);
    return kNone;
  }
  uint32_t* sums = nullptr;
  const uint32_t n_clusters = smem_tier ? pixel_phases<NT, true>(L, e, S, region, tier, p0, n, &sums, sub)
                                        : pixel_phases<NT, false>(L, e, S, region, tier, p0, n, &sums, sub);
  if (n_clusters == kNone) return n_clusters;
  if (sub.on && 3u * n_clusters > 2u * tier) {  // (the heavy kernel then clusters the event on one CTA)
    if (tid == 0) atomicOr(sub.big, 1u);
    return n_clusters;
  }
  if (3u * n_clusters <= 2u * tier) hit_phases<NT, true>(L, e, S, region, tier, p0, n, n_clusters, sums, sub);
  else hit_phases<NT, false>(L, e, S, region, tier, p0, n, n_clusters, sums, sub);
  return n_clusters;
}

// Persistent: every CTA takes events from the work queue until it is empty,
// so events of uneven size spread over the SMs as they finish.
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_cluster(Launch L) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  ClusterSmem<NT>& S = *reinterpret_cast<ClusterSmem<NT>*>(smem_raw);
  uint32_t* region = reinterpret_cast<uint32_t*>(smem_raw + sizeof(ClusterSmem<NT>));
  for (;;) {
    if (threadIdx.x == 0) S.next = atomicAdd(L.ws.queue + 0, 1u);
    __syncthreads();
    const uint32_t e = S.next;
    __syncthreads();
    if (e >= L.n_events) break;
    // heavy-ion-like events are left to k_cluster_wide (listed when the offsets are valid)
    if (*(const volatile uint32_t*)L.ws.flag == 0u && L.off[e + 1] - L.off[e] >= kHeavyWords) continue;
    cluster_one<NT>(L, e, S, region, L.cluster_tier);
    if (threadIdx.x == 0) {  // the event's place in the tracking order (its count was written by this thread)
      const bool large = L.ws.ev_nclusters[e] >= kLargeEvent;
      const uint32_t at =
          large ? atomicAdd(L.ws.queue + 4, 1u) : (uint32_t)L.n_events - 1u - atomicAdd(L.ws.queue + 5, 1u);
      L.ws.order[at] = e;
    }
    __syncthreads();
  }
}

// Cross-CTA records of k_cluster_wide: every CTA's own, read by the others
// through distributed shared memory; the event-wide ones live in rank 0's.
struct WideShared {
  uint32_t cnt[VELO_MAX_MODULES];    // words of each module in this CTA's slice of the event
  uint32_t base[VELO_MAX_MODULES];   // where this CTA's words of each module go in the grouped copy
  uint32_t mo[kModOffStride];        // module word offsets of the grouped copy
  uint32_t cb[kModOffStride];        // module cluster offsets (first event-wide id of each module)
  uint32_t order[VELO_MAX_MODULES];  // the non-empty modules, most words first
  uint32_t n_jobs;                   // how many
  uint32_t next;                     // this CTA's current module job
  // rank 0 only:
  uint32_t nclu[VELO_MAX_MODULES];   // clusters of each module
  uint32_t job;                      // the next module job
  uint32_t bad;                      // a word of the event is invalid
  uint32_t fail;                     // a module's failure (VELO_EVT_*), 0 if none
  uint32_t big;                      // a module has too many clusters for the shared hit sort
};

// Heavy-ion-like events (kHeavyWords words or more), one thread-block
// cluster of CTAs of 1024 threads per event.  Clusters never span modules,
// so every module is a sub-event of about a C2 event's size that one CTA
// clusters in shared memory with the ordinary code:
//  1. every CTA counts (and validates) the words of its slice of the event
//     by module; the module offsets follow, and every CTA scatters its words
//     into a module-grouped copy of the event (words in sa, their input
//     positions in sb);
//  2. the CTAs take modules from a cluster-wide counter (most words first)
//     and cluster each one, writing its labels, centroids and hit records at
//     provisional event-wide places (ids and positions from its first word's
//     place in the grouped copy);
//  3. the module cluster offsets give every module its first event-wide id,
//     and the records move down to their final places (ids and positions
//     lowered; the labels in place);
//  4. rank 0 writes the event's records (status, module offsets, counts,
//     lists).
// A module larger than the shared-memory tier, or with too many clusters
// for the shared-memory hit sort, sends the whole event to rank 0 alone
// (the ordinary one-CTA path from the input words).
constexpr uint32_t kClusterWideMax = 16, kClusterWidePortable = 8;

__global__ void __launch_bounds__(1024, 1) k_cluster_wide(Launch L, uint32_t tier) {
  constexpr int NT = 1024;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  ClusterSmem<NT>& S = *reinterpret_cast<ClusterSmem<NT>*>(smem_raw);
  uint32_t* region = reinterpret_cast<uint32_t*>(smem_raw + sizeof(ClusterSmem<NT>));
  __shared__ WideShared X;
  const Workspace& W = L.ws;
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t CS = cl.num_blocks(), rank = cl.block_rank(), tid = threadIdx.x;
  WideShared* X0 = cl.map_shared_rank(&X, 0);
  const uint32_t M = L.geo.n_modules;
  const uint32_t count = *(const volatile uint32_t*)(W.queue + 7);
  const uint32_t wid = warp_id();
  for (uint32_t q = blockIdx.x / CS; q < count; q += gridDim.x / CS) {
    const uint64_t e = W.heavy_list[q];
    const uint64_t p0 = L.off[e];
    const uint32_t n = (uint32_t)(L.off[e + 1] - p0);
    // ---- 1. per-module word counts of this CTA's slice (per-warp counters), validation
    const uint32_t s0 = (uint32_t)((uint64_t)n * rank / CS), s1 = (uint32_t)((uint64_t)n * (rank + 1) / CS);
    S.cnt[tid] = 0u;  // 32 warps x 32 modules
    if (rank == 0 && tid == 0) {
      X.job = 0u;
      X.bad = X.fail = X.big = 0u;
    }
    __syncthreads();
    bool bad = false;
    for (uint32_t i = s0 + tid; i < s1; i += NT) {
      const uint32_t w = __ldg(L.pix + p0 + i);
      if (word_valid(w, L.geo)) atomicAdd(&S.cnt[wid * 32u + ((w >> 22) & 31u)], 1u);
      else bad = true;
    }
    if (bad) atomicOr(&X0->bad, 1u);
    __syncthreads();
    if (tid < 32) {
      uint32_t c = 0;
      for (uint32_t w = 0; w < NT / 32; ++w) c += S.cnt[w * 32u + tid];
      X.cnt[tid] = c;
    }
    cl.sync();  // every CTA's counts, the bad-word flag
    const bool ev_bad = *(volatile uint32_t*)&X0->bad != 0u;
    if (!ev_bad) {
      if (tid < 32) {  // module totals and this CTA's share before it
        uint32_t tot = 0, mine = 0;
        for (uint32_t r = 0; r < CS; ++r) {
          const uint32_t c = cl.map_shared_rank(&X, r)->cnt[tid];
          tot += c;
          if (r < rank) mine += c;
        }
        X.base[tid] = mine;
        X.cb[tid] = tot;  // (module word totals until the offsets are taken)
      }
      __syncthreads();
      if (tid == 0) {
        uint32_t o = 0;
        for (uint32_t m = 0; m < VELO_MAX_MODULES; ++m) {
          X.mo[m] = o;
          X.base[m] += o;
          o += X.cb[m];
        }
        X.mo[VELO_MAX_MODULES] = o;
        // the non-empty modules, most words first (a selection over at most 32)
        uint32_t k = 0;
        for (uint32_t m = 0; m < M; ++m)
          if (X.cb[m]) X.order[k++] = m;
        for (uint32_t a = 0; a < k; ++a)
          for (uint32_t b = a + 1; b < k; ++b)
            if (X.cb[X.order[b]] > X.cb[X.order[a]]) {
              const uint32_t t = X.order[a];
              X.order[a] = X.order[b];
              X.order[b] = t;
            }
        X.n_jobs = k;
      }
      __syncthreads();
      for (uint32_t i = s0 + tid; i < s1; i += NT) {  // the module-grouped copy
        const uint32_t w = __ldg(L.pix + p0 + i);
        const uint32_t pos = atomicAdd(&X.base[(w >> 22) & 31u], 1u);
        W.sa[p0 + pos] = w;
        W.sb[p0 + pos] = i;
      }
    }
    cl.sync();  // the grouped copy is complete
    uint32_t big = 0;  // a module too large for the shared-memory tier
    if (!ev_bad)
      for (uint32_t m = 0; m < M; ++m) big |= X.mo[m + 1] - X.mo[m] > tier;
    if (!ev_bad && !big) {
      // ---- 2. one pass over the modules, each at provisional event-wide
      // places: its first cluster id (and first hit position) is its first
      // word's place in the grouped copy, mo[m] >= its final cb[m]
      for (;;) {
        if (tid == 0) X.next = atomicAdd(&X0->job, 1u);
        __syncthreads();
        const uint32_t j = X.next;
        __syncthreads();
        if (j >= X.n_jobs) break;
        const uint32_t m = X.order[j];
        Sub sub;
        sub.on = true;
        sub.words = W.sa + p0 + X.mo[m];
        sub.index = W.sb + p0 + X.mo[m];
        sub.ev_p0 = p0;
        sub.id_base = X.mo[m];
        sub.fail = &X0->fail;
        sub.big = &X0->big;
        const uint32_t nc = cluster_one<NT>(L, e, S, region, tier, sub, p0 + X.mo[m], X.mo[m + 1] - X.mo[m]);
        if (tid == 0) X0->nclu[m] = nc;
        __syncthreads();
      }
      cl.sync();  // every module's count and results
      if (tid == 0) {  // module cluster offsets; too many clusters for the hit sort -> one CTA
        uint32_t o = 0;
        for (uint32_t m = 0; m < VELO_MAX_MODULES; ++m) {
          const uint32_t c = m < M && X.mo[m + 1] > X.mo[m] ? X0->nclu[m] : 0u;
          X.cb[m] = o;
          if (c != kNone) o += c;
        }
        X.cb[VELO_MAX_MODULES] = o;
        X.next = *(volatile uint32_t*)&X0->big;
      }
      __syncthreads();
      big = X.next;
      if (!big && !*(volatile uint32_t*)&X0->fail) {  // (every CTA sees the same)
        // ---- 3. the records to their final places: the cluster (x, y) and
        // the hit records and id -> position map of module m move from
        // [mo[m], mo[m] + c) to [cb[m], cb[m] + c) with their ids and
        // positions lowered by mo[m] - cb[m].  Every move goes down (cb[m] <=
        // mo[m]), so in rounds of rising final places, each read before a
        // cluster barrier and written after it, no write reaches a record
        // that a later round still reads.  The labels are lowered in place.
        const uint32_t nct = X.cb[VELO_MAX_MODULES];
        auto module_of_final = [&](uint32_t f) {  // the last non-empty m with cb[m] <= f
          uint32_t lo = 0, hi = M;
          while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (X.cb[mid] <= f) lo = mid;
            else hi = mid;
          }
          return lo;
        };
        for (uint32_t f0 = 0; f0 < nct; f0 += CS * NT) {
          const uint32_t f = f0 + rank * NT + tid;
          float2 xy = make_float2(0.0f, 0.0f);
          float4 h = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          uint32_t hp = 0, d = 0;
          if (f < nct) {
            const uint32_t m = module_of_final(f);
            d = X.mo[m] - X.cb[m];
            xy = __ldcg(W.cl_xy + p0 + f + d);
            h = __ldcg(W.hit + p0 + f + d);
            hp = __ldcg(W.h_pos + p0 + f + d);
          }
          cl.sync();
          if (f < nct) {
            W.cl_xy[p0 + f] = xy;
            W.hit[p0 + f] = make_float4(h.x, h.y, h.z, __uint_as_float(__float_as_uint(h.w) - d));
            W.h_pos[p0 + f] = hp - d;
          }
        }
        if (L.out.pixel_cluster) {
          auto module_of_provisional = [&](uint32_t v) {  // the last m with mo[m] <= v
            uint32_t lo = 0, hi = M;
            while (hi - lo > 1) {
              const uint32_t mid = (lo + hi) >> 1;
              if (X.mo[mid] <= v) lo = mid;
              else hi = mid;
            }
            return lo;
          };
          for (uint32_t i = rank * NT + tid; i < n; i += CS * NT) {
            const uint32_t v = __ldcg(L.out.pixel_cluster + p0 + i);
            const uint32_t m = module_of_provisional(v);
            L.out.pixel_cluster[p0 + i] = v - (X.mo[m] - X.cb[m]);
          }
        }
      }
    }
    // ---- 4. the event's records (rank 0)
    if (rank == 0) {
      const uint32_t fail = ev_bad ? (uint32_t)VELO_EVT_BADWORD : *(volatile uint32_t*)&X0->fail;
      if (fail) {
        fail_event(L, e, (int32_t)fail, true, p0, n);
      } else if (big) {
        cluster_one<NT>(L, e, S, region, tier);  // the whole event here, from its input words
      } else {
        const uint32_t nc = X.cb[VELO_MAX_MODULES];
        if (tid <= M) W.ev_modoff[e * kModOffStride + tid] = X.cb[tid];
        if (tid == 0) {
          W.ev_nclusters[e] = nc;
          L.out.status[e] = VELO_EVT_OK;
          if (nc >= kWideClusters) W.wide_list[atomicAdd(W.queue + 3, 1u)] = (uint32_t)e;
        }
      }
      if (tid == 0) W.order[atomicAdd(W.queue + 4, 1u)] = (uint32_t)e;  // tracked first
    }
    cl.sync();  // the shared records are reused by the next event
  }
}

// CTAs per heavy event for k_cluster_wide on the current device (once per
// device): the largest of 16, 8, 4, 2 for which such a cluster of
// 1024-thread CTAs with their shared memory can be placed, else 1; 0 if the
// kernel's attributes cannot be set.
uint32_t cluster_wide_size(uint32_t smem) {
  static std::mutex mu;
  static uint32_t size[64] = {};
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (size[d]) return size[d];
  const void* f = reinterpret_cast<const void*>(k_cluster_wide);
  if (!set_max_smem_once(f, 6, smem)) return 0;
  const bool large = allow_large_clusters_once(f, 1);
  uint32_t cs = 1;  // the largest cluster (16, 8, 4, 2) the device can place, else single CTAs
  for (uint32_t c = kClusterWideMax; c > 1; c /= 2) {
    if (c > kClusterWidePortable && !large) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, k_cluster_wide, &cfg) == cudaSuccess && n >= 1;
    cudaGetLastError();
    if (ok) {
      cs = c;
      break;
    }
  }
  size[d] = cs;
  return cs;
}

uint32_t cluster_smem_bytes(int nt, uint32_t tier) {
  const uint32_t head = nt == 512 ? (uint32_t)sizeof(ClusterSmem<512>) : (uint32_t)sizeof(ClusterSmem<1024>);
  return head + 2u * tier * 4u;
}

uint32_t cluster_max_tier(int nt) {
  const uint32_t head = cluster_smem_bytes(nt, 0);
  const uint32_t cap = nt == 512 ? kSmemPerSm / 2 - 1024 : kSmemPerBlock;  // two CTAs per SM at 512 threads
  return ((cap - head) / 8u) & ~255u;
}

int launch_cluster(const Launch& L, int nt, uint32_t grid, cudaStream_t s) {
  const uint32_t smem = cluster_smem_bytes(nt, L.cluster_tier);
  if (nt == 512) {
    if (!set_max_smem_once(reinterpret_cast<const void*>(k_cluster<512>), 0)) return VELO_ECUDA;
    k_cluster<512><<<grid, 512, smem, s>>>(L);
  } else {
    if (!set_max_smem_once(reinterpret_cast<const void*>(k_cluster<1024>), 1)) return VELO_ECUDA;
    k_cluster<1024><<<grid, 1024, smem, s>>>(L);
  }
  // the heavy-ion-like events: one wave of thread-block clusters (one
  // 1024-thread CTA per SM), each taking events from the list
  const uint32_t wtier = cluster_wide_tier();
  const uint32_t wsmem = cluster_smem_bytes(1024, wtier);
  const uint32_t cs = cluster_wide_size(wsmem);
  if (!cs) return VELO_ECUDA;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(std::max<uint32_t>(1u, (uint32_t)device_sm_count() / cs) * cs);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = wsmem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_cluster_wide, L, wtier) != cudaSuccess) return VELO_ECUDA;
  return VELO_OK;
}

// The shared-memory tier of k_cluster_wide: the largest at 1024 threads that
// leaves room for its static cross-CTA records.
uint32_t cluster_wide_tier() {
  const uint32_t head = cluster_smem_bytes(1024, 0) + (uint32_t)sizeof(WideShared);
  return ((kSmemPerBlock - head) / 8u) & ~255u;
}

int cluster_blocks_per_sm(int nt, uint32_t tier) {
  return occupancy(nt == 512 ? reinterpret_cast<const void*>(k_cluster<512>)
                             : reinterpret_cast<const void*>(k_cluster<1024>),
                   nt, cluster_smem_bytes(nt, tier), nt == 512 ? 0 : 1);
}

}  // namespace velo
