// CPU oracle for event-batched VELO-like pixel tracking -- TEST INFRASTRUCTURE.
//
// Plain, slow, obviously-correct restatement of the method.  The paper
// (Sec. "HLT1 details and results") says only that the first trigger stage
// runs a simplified pattern recognition and a parameterised Kalman filter on
// the pixel-tracker (VELO) segment of each track, on every event (Sec.
// "Introduction", Sec. "Data flow overview").  The algorithm below is this
// project's definition of that statement, step by step:
//   1. pixel words and their validation
//   2. clustering: 8-connected components per module, canonical ids, centroid
//   3. pseudo-angle key and per-module hit order
//   4. triplet seeding                      (run at step m after 5)
//   5. forward extension                    (run first at step m)
//   6. step order and used flags
//   7. termination and the 3-hit rule
//   8. straight-line fit and simplified Kalman filter
//   9. chi2/ndf cut (optionally with the learned ghost rejection)
//  10. canonical output order
// Arithmetic: binary32, one rounding per operation in the written order,
// no FMA contraction (compiled with -ffp-contract=off), no transcendental
// function anywhere.  Nothing here is blocked, fused or reordered: window
// candidates are found by scanning every hit of the target module.

#include "velo_oracle.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- step 1
// word = q << 27 | module << 22 | row << 11 | col; bit 31 must be clear,
// q in 1..15, module/row/col inside the geometry.
inline uint32_t w_q(uint32_t w) { return (w >> 27) & 15u; }
inline uint32_t w_module(uint32_t w) { return (w >> 22) & 31u; }
inline uint32_t w_row(uint32_t w) { return (w >> 11) & 2047u; }
inline uint32_t w_col(uint32_t w) { return w & 2047u; }
inline uint32_t w_key(uint32_t w) { return w & 0x7FFFFFFu; }  // (module, row, col)

bool word_valid(uint32_t w, const vo_geometry_t* g) {
  if (w >> 31) return false;
  if (w_q(w) == 0) return false;
  if (w_module(w) >= g->n_modules) return false;
  if (w_row(w) >= g->n_rows) return false;
  if (w_col(w) >= g->n_cols) return false;
  return true;
}

// ---------------------------------------------------------------- step 3
float pseudo_angle(float x, float y) {
  float k;
  if (y >= 0.0f) {
    if (x >= 0.0f) {
      float d = x + y;
      k = d > 0.0f ? y / d : 0.0f;
    } else {
      k = 1.0f + (-x) / (y - x);
    }
  } else {
    if (x < 0.0f) {
      k = 2.0f + (-y) / ((-x) - y);
    } else {
      k = 3.0f + x / (x - y);
    }
  }
  return k + 0.0f;  // -0 -> +0
}

// |a - b| on the circle of circumference 4
float dmod4(float a, float b) {
  float d = std::fabs(a - b);
  if (d > 2.0f) d = 4.0f - d;
  return d;
}

inline uint32_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// ---------------------------------------------------------------- step 2
struct UnionFind {
  std::vector<uint32_t> parent;
  explicit UnionFind(size_t n) : parent(n) {
    for (size_t i = 0; i < n; ++i) parent[i] = (uint32_t)i;
  }
  uint32_t find(uint32_t a) {
    while (parent[a] != a) a = parent[a];
    return a;
  }
  void unite(uint32_t a, uint32_t b) {  // the smaller index becomes the root
    a = find(a);
    b = find(b);
    if (a == b) return;
    if (a < b) parent[b] = a;
    else parent[a] = b;
  }
};

struct ClusterOut {
  std::vector<float> x, y, z;
  std::vector<uint32_t> module;
  std::vector<uint32_t> pixel_cluster;  // per input word
  int status = VO_EVT_OK;
};

void cluster_event(const uint32_t* words, uint64_t n, const vo_geometry_t* g, ClusterOut& out) {
  out.x.clear(); out.y.clear(); out.z.clear(); out.module.clear();
  out.pixel_cluster.assign(n, 0xFFFFFFFFu);
  out.status = VO_EVT_OK;
  for (uint64_t i = 0; i < n; ++i)
    if (!word_valid(words[i], g)) { out.status = VO_EVT_BADWORD; return; }
  // positions sorted by (module, row, col)
  std::vector<uint32_t> order(n);
  for (uint64_t i = 0; i < n; ++i) order[i] = (uint32_t)i;
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t a, uint32_t b) { return w_key(words[a]) < w_key(words[b]); });
  std::vector<uint32_t> skey(n);
  for (uint64_t i = 0; i < n; ++i) skey[i] = w_key(words[order[i]]);
  // 8-connectivity inside a module: every pixel at |drow| <= 1, |dcol| <= 1
  // (same cell included: duplicate words join the same cluster)
  UnionFind uf(n);
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t k = skey[i];
    int m = (int)(k >> 22), r = (int)((k >> 11) & 2047u), c = (int)(k & 2047u);
    for (int dr = -1; dr <= 1; ++dr)
      for (int dc = -1; dc <= 1; ++dc) {
        int rr = r + dr, cc = c + dc;
        if (rr < 0 || cc < 0 || rr >= (int)g->n_rows || cc >= (int)g->n_cols) continue;
        uint32_t kk = (uint32_t)m << 22 | (uint32_t)rr << 11 | (uint32_t)cc;
        auto range = std::equal_range(skey.begin(), skey.end(), kk);
        for (auto it = range.first; it != range.second; ++it) uf.unite((uint32_t)i, (uint32_t)(it - skey.begin()));
      }
  }
  // roots are the smallest sorted position of their component, i.e. the pixel
  // with the smallest (module, row*2048+col): cluster id = rank of the root.
  std::vector<uint32_t> cid(n, 0xFFFFFFFFu);
  uint32_t nc = 0;
  for (uint64_t i = 0; i < n; ++i)
    if (uf.find((uint32_t)i) == i) cid[i] = nc++;
  std::vector<int64_t> sq(nc, 0), snx(nc, 0), sny(nc, 0);
  std::vector<uint32_t> cmod(nc, 0);
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t id = cid[uf.find((uint32_t)i)];
    uint32_t w = words[order[i]];
    int64_t q = w_q(w);
    sq[id] += q;
    snx[id] += q * (int64_t)(2 * w_col(w) + 1);
    sny[id] += q * (int64_t)(2 * w_row(w) + 1);
    cmod[id] = w_module(w);
    out.pixel_cluster[order[i]] = id;
  }
  // capacity contract: at most VO_MAX_MODULE_CLUSTERS clusters per module
  std::vector<uint32_t> per_module(g->n_modules, 0);
  for (uint32_t id = 0; id < nc; ++id)
    if (++per_module[cmod[id]] > VO_MAX_MODULE_CLUSTERS) {
      out.status = VO_EVT_OVERFLOW;
      out.pixel_cluster.assign(n, 0xFFFFFFFFu);
      return;
    }
  // centroid in pixel units: u = Nx / D with Nx = sum q (2 col + 1), D = 2 sum q;
  // integer quotient (exact) plus one division of the remainder, one add.
  out.x.resize(nc); out.y.resize(nc); out.z.resize(nc); out.module = cmod;
  for (uint32_t id = 0; id < nc; ++id) {
    int64_t D = 2 * sq[id];
    float u = (float)(snx[id] / D) + (float)(snx[id] % D) / (float)D;
    float v = (float)(sny[id] / D) + (float)(sny[id] % D) / (float)D;
    out.x[id] = g->x0_mm + g->pitch_mm * u;
    out.y[id] = g->y0_mm + g->pitch_mm * v;
    out.z[id] = g->module_z[cmod[id]];
  }
}

// ---------------------------------------------------------------- step 8
// state layout (VO_STATE_STRIDE floats):
//  0 x, 1 y, 2 tx, 3 ty        straight-line least squares at z_first
//  4 z_first, 5 z_beam         z of the first hit; closest approach to the z axis
//  6 chi2_lsq, 7 chi2_kf
//  8 kf_x, 9 kf_y, 10 kf_tx, 11 kf_ty   Kalman state at z_first
// 12 C_xx, 13 C_xtx, 14 C_txtx  Kalman covariance, x projection
// 15 C_yy, 16 C_yty, 17 C_tyty  Kalman covariance, y projection
// 18 ndf = 2n - 4, 19 learned score (0 for the plain method)
template <class R>
struct LineFit {
  R pos, slope, chi2;
};

template <class R>
void lsq_fit(uint32_t n, const R* z, const R* xs, const R* ys, R sigma, R out[7]) {
  // sums in the order S0 = n, Sz, Szz, Sx, Sxz (then Sy, Syz), hits ascending in z
  R z0 = z[0];
  R S0 = (R)n, Sz = 0, Szz = 0, Sx = 0, Sxz = 0, Sy = 0, Syz = 0;
  for (uint32_t i = 0; i < n; ++i) {
    R dz = z[i] - z0;
    Sz = Sz + dz;
    Szz = Szz + dz * dz;
    Sx = Sx + xs[i];
    Sxz = Sxz + xs[i] * dz;
    Sy = Sy + ys[i];
    Syz = Syz + ys[i] * dz;
  }
  R det = S0 * Szz - Sz * Sz;
  R tx = (S0 * Sxz - Sz * Sx) / det;
  R x = (Sx - tx * Sz) / S0;
  R ty = (S0 * Syz - Sz * Sy) / det;
  R y = (Sy - ty * Sz) / S0;
  R chi2 = 0;
  for (uint32_t i = 0; i < n; ++i) {
    R dz = z[i] - z0;
    R rx = ((xs[i] - x) - tx * dz) / sigma;
    chi2 = chi2 + rx * rx;
    R ry = ((ys[i] - y) - ty * dz) / sigma;
    chi2 = chi2 + ry * ry;
  }
  R num = x * tx + y * ty;
  R den = tx * tx + ty * ty;
  R zb = den > 0 ? z0 - num / den : z0;
  out[0] = x; out[1] = y; out[2] = tx; out[3] = ty; out[4] = z0; out[5] = zb; out[6] = chi2;
}

// One projection, downstream -> upstream.  Start at the second-to-last hit
// from the last two hits (no prior): X = m[n-2], T = (m[n-2] - m[n-1]) / dz0,
// C = [[s2, s2/dz0], [s2/dz0, 2 s2/dz0^2 + q]] with dz0 = z[n-2] - z[n-1],
// s2 = sigma^2, q = theta^2 (the slope kick between those two hits).  Then
// for every earlier hit: predict with F = [[1, dz], [0, 1]], Q = diag(0, q);
// update with H = [1, 0], R = s2.  chi2 = sum of r^2 / S over the updates.
template <class R>
void kalman_1d(uint32_t n, const R* z, const R* m, R sigma, R theta, R out[5], R* chi2_out) {
  R s2 = sigma * sigma, q = theta * theta;
  R dz0 = z[n - 2] - z[n - 1];
  R X = m[n - 2];
  R T = (m[n - 2] - m[n - 1]) / dz0;
  R C00 = s2;
  R C01 = s2 / dz0;
  R C11 = (s2 + s2) / (dz0 * dz0) + q;
  R chi2 = 0;
  for (int i = (int)n - 3; i >= 0; --i) {
    R dz = z[i] - z[i + 1];
    // predict
    X = X + T * dz;
    R t1 = C11 * dz;
    C00 = C00 + dz * ((C01 + C01) + t1);
    C01 = C01 + t1;
    C11 = C11 + q;
    // update
    R r = m[i] - X;
    R S = C00 + s2;
    R K0 = C00 / S, K1 = C01 / S;
    X = X + K0 * r;
    T = T + K1 * r;
    C11 = C11 - K1 * C01;
    C01 = C01 - K0 * C01;
    C00 = C00 - K0 * C00;
    chi2 = chi2 + (r * r) / S;
  }
  out[0] = X; out[1] = T; out[2] = C00; out[3] = C01; out[4] = C11;
  *chi2_out = chi2;
}

template <class R>
void fit_track(uint32_t n, const R* x, const R* y, const R* z, R sigma, R theta, R* st) {
  R l[7];
  lsq_fit<R>(n, z, x, y, sigma, l);
  R kx[5], ky[5], cx2, cy2;
  kalman_1d<R>(n, z, x, sigma, theta, kx, &cx2);
  kalman_1d<R>(n, z, y, sigma, theta, ky, &cy2);
  for (int i = 0; i < 7; ++i) st[i] = l[i];
  st[7] = cx2 + cy2;
  st[8] = kx[0]; st[9] = ky[0]; st[10] = kx[1]; st[11] = ky[1];
  st[12] = kx[2]; st[13] = kx[3]; st[14] = kx[4];
  st[15] = ky[2]; st[16] = ky[3]; st[17] = ky[4];
  st[18] = (R)(2 * n - 4);
  st[19] = 0;
}

// ---------------------------------------------------------------- learned ghost rejection
// Candidate features (binary32, fixed order).  Residuals are the straight-line
// fit's: r_i = (x_i - x) - tx dz_i, as in its chi2.
void features(uint32_t n, const float* x, const float* y, const float* z, const uint32_t* module, const float* st,
              float chi2ndf, float* f) {
  f[0] = (float)n;
  f[1] = chi2ndf;
  f[2] = st[2];
  f[3] = st[3];
  f[4] = z[0];
  f[5] = z[n - 1];
  f[6] = (float)((int)(module[n - 1] - module[0] + 1) - (int)n);
  float sx = 0.0f, sxx = 0.0f, sy = 0.0f, syy = 0.0f, mx = 0.0f;
  for (uint32_t i = 0; i < n; ++i) {
    float dz = z[i] - z[0];
    float rx = (x[i] - st[0]) - st[2] * dz;
    float ry = (y[i] - st[1]) - st[3] * dz;
    sx = sx + rx;
    sxx = sxx + rx * rx;
    sy = sy + ry;
    syy = syy + ry * ry;
    mx = std::fmax(mx, std::fmax(std::fabs(rx), std::fabs(ry)));
  }
  float fn = (float)n;
  f[7] = sx / fn;
  f[8] = std::sqrt(sxx / fn);  // IEEE square root: correctly rounded
  f[9] = sy / fn;
  f[10] = std::sqrt(syy / fn);
  f[11] = mx;
}

float bf16(float v) {  // round to nearest even, to bfloat16 (finite inputs)
  uint32_t u;
  std::memcpy(&u, &v, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  std::memcpy(&v, &u, 4);
  return v;
}

float mlp_logit(const float* w, const float* f) {
  const int H = VO_MLP_HIDDEN, F = VO_N_FEATURES;
  const float* mean = w;
  const float* istd = w + F;
  const float* W1 = w + 2 * F;
  const float* b1 = W1 + H * F;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float b3 = W3[H];
  float xin[VO_N_FEATURES], h1[VO_MLP_HIDDEN], h2[VO_MLP_HIDDEN];
  for (int k = 0; k < F; ++k) xin[k] = bf16((f[k] - mean[k]) * istd[k]);
  for (int j = 0; j < H; ++j) {
    float a = 0.0f;
    for (int k = 0; k < F; ++k) a = a + bf16(W1[j * F + k]) * xin[k];
    a = a + b1[j];
    h1[j] = bf16(a > 0.0f ? a : 0.0f);
  }
  for (int j = 0; j < H; ++j) {
    float a = 0.0f;
    for (int k = 0; k < H; ++k) a = a + bf16(W2[j * H + k]) * h1[k];
    a = a + b2[j];
    h2[j] = a > 0.0f ? a : 0.0f;
  }
  float z = 0.0f;
  for (int j = 0; j < H; ++j) z = z + W3[j] * h2[j];
  return z + b3;
}

// ---------------------------------------------------------------- steps 4-7, 9, 10
struct Hits {
  uint32_t n = 0;
  std::vector<uint32_t> module;
  std::vector<float> x, y, z, key;
  std::vector<std::vector<uint32_t>> by_module;  // ids sorted by (key, id)
};

struct Track {
  std::vector<uint32_t> hits;  // build order: downstream first
  bool active = true;
};

struct TrackOut {
  std::vector<std::vector<uint32_t>> hits;  // ascending ids, canonical order
  std::vector<float> states;
  std::vector<float> features;
};

void track_event(const Hits& H, const vo_geometry_t* g, const vo_params_t* p, TrackOut& out) {
  const int M = (int)g->n_modules;
  const float* Z = g->module_z;
  std::vector<uint8_t> used(H.n, 0);
  std::vector<Track> tracks;
  for (int m = M - 2; m >= 0; --m) {
    // 5. extension into module m against the used flags at the start of the step
    std::vector<uint8_t> used0 = used;
    std::vector<uint64_t> claim(H.n, ~0ull);
    struct Pick { uint32_t t, h; uint64_t key; };
    std::vector<Pick> picks;
    for (uint32_t t = 0; t < tracks.size(); ++t) {
      Track& T = tracks[t];
      if (!T.active) continue;
      uint32_t a = T.hits[T.hits.size() - 1], b = T.hits[T.hits.size() - 2];
      int l = (int)H.module[a];
      if (l - m - 1 > (int)p->max_skipped) { T.active = false; continue; }
      if (l <= m) continue;
      float tx = (H.x[a] - H.x[b]) / (H.z[a] - H.z[b]);
      float ty = (H.y[a] - H.y[b]) / (H.z[a] - H.z[b]);
      float xp = H.x[a] + tx * (Z[m] - H.z[a]);
      float yp = H.y[a] + ty * (Z[m] - H.z[a]);
      bool found = false;
      float bd2 = 0.0f;
      uint32_t bh = 0;
      for (uint32_t h : H.by_module[m]) {
        if (used0[h]) continue;
        if (dmod4(H.key[h], H.key[a]) > p->win_fwd) continue;
        float dx = xp - H.x[h], dy = yp - H.y[h];
        float d2 = dx * dx + dy * dy;
        if (d2 > p->max_scatter_fwd) continue;
        if (!found || d2 < bd2 || (d2 == bd2 && h < bh)) { found = true; bd2 = d2; bh = h; }
      }
      if (found) {
        uint64_t k = (uint64_t)fbits(bd2) << 32 | t;
        claim[bh] = std::min(claim[bh], k);
        picks.push_back({t, bh, k});
      }
    }
    for (const Pick& pk : picks)
      if (claim[pk.h] == pk.key) {  // the smallest (d2, track index) takes the hit
        tracks[pk.t].hits.push_back(pk.h);
        used[pk.h] = 1;
      }
    if (m == 0) break;  // module 0 receives extension only
    // 4. seeding with the middle hit on m, h0 on m+1 (unused), h2 on m-1
    struct Seed { uint32_t h0, h1, h2; float s; };
    std::vector<Seed> seeds;
    for (uint32_t h1 : H.by_module[m]) {  // sorted order of module m
      if (used[h1]) continue;
      bool found = false;
      Seed best{0, h1, 0, 0.0f};
      for (uint32_t h0 : H.by_module[m + 1]) {
        if (used[h0]) continue;
        if (dmod4(H.key[h0], H.key[h1]) > p->win_seed) continue;
        for (uint32_t h2 : H.by_module[m - 1]) {
          if (dmod4(H.key[h2], H.key[h1]) > p->win_seed) continue;
          float dz02 = H.z[h0] - H.z[h2];
          float tx = (H.x[h0] - H.x[h2]) / dz02;
          float ty = (H.y[h0] - H.y[h2]) / dz02;
          if (std::fabs(tx) > p->max_slope || std::fabs(ty) > p->max_slope) continue;
          float dz12 = H.z[h1] - H.z[h2];
          float xp = H.x[h2] + tx * dz12;
          float yp = H.y[h2] + ty * dz12;
          float dx = xp - H.x[h1], dy = yp - H.y[h1];
          float s = dx * dx + dy * dy;
          if (s > p->max_scatter_seed) continue;
          bool better = !found || s < best.s || (s == best.s && (h0 < best.h0 || (h0 == best.h0 && h2 < best.h2)));
          if (better) { found = true; best = {h0, h1, h2, s}; }
        }
      }
      if (found) seeds.push_back(best);
    }
    // conflicts: a seed claims h0 and h2 with (bits(s), id1); the smallest claim wins
    // each hit, and a seed survives only if it holds both of its claims.
    std::vector<uint64_t> sclaim(H.n, ~0ull);
    for (const Seed& s : seeds) {
      uint64_t k = (uint64_t)fbits(s.s) << 32 | s.h1;
      sclaim[s.h0] = std::min(sclaim[s.h0], k);
      sclaim[s.h2] = std::min(sclaim[s.h2], k);
    }
    for (const Seed& s : seeds) {  // in sorted order of h1: new track indices
      uint64_t k = (uint64_t)fbits(s.s) << 32 | s.h1;
      if (sclaim[s.h0] != k || sclaim[s.h2] != k) continue;
      used[s.h0] = used[s.h1] = used[s.h2] = 1;
      Track T;
      T.hits = {s.h0, s.h1, s.h2};
      tracks.push_back(T);
    }
  }
  // 7-9. every track terminates; fit; 3-hit rule; chi2/ndf cut
  struct Kept { std::vector<uint32_t> hits; std::vector<float> st, f; };
  std::vector<Kept> kept;
  for (const Track& T : tracks) {
    uint32_t n = (uint32_t)T.hits.size();
    std::vector<uint32_t> asc(T.hits.rbegin(), T.hits.rend());  // ascending z == ascending id
    std::vector<float> xs(n), ys(n), zs(n);
    std::vector<uint32_t> ms(n);
    for (uint32_t i = 0; i < n; ++i) {
      xs[i] = H.x[asc[i]]; ys[i] = H.y[asc[i]]; zs[i] = H.z[asc[i]]; ms[i] = H.module[asc[i]];
    }
    std::vector<float> st(VO_STATE_STRIDE), f(VO_N_FEATURES);
    fit_track<float>(n, xs.data(), ys.data(), zs.data(), p->sigma_meas, p->ms_theta, st.data());
    float chi2 = p->ms_theta == 0.0f ? st[6] : st[7];
    float ndf = (float)(2 * n - 4);
    float r = chi2 / ndf;
    features(n, xs.data(), ys.data(), zs.data(), ms.data(), st.data(), r, f.data());
    if (p->use_mlp) {
      // learned rejection: the network's logit replaces the 3-hit rule
      st[19] = mlp_logit(p->mlp, f.data());
      if (!(st[19] >= p->mlp_logit_min)) continue;
    } else {
      // hits are never shared between tracks (every claim is exclusive), so
      // "no hit in another candidate" always holds for a 3-hit track.
      if (n == 3 && !(r <= p->chi2ndf_max_3hit)) continue;
    }
    if (!(r <= p->chi2ndf_max)) continue;
    kept.push_back({asc, st, f});
  }
  // 10. canonical order: lexicographic by the ascending hit-id list
  std::sort(kept.begin(), kept.end(), [](const Kept& a, const Kept& b) { return a.hits < b.hits; });
  out.hits.clear();
  out.states.clear();
  out.features.clear();
  for (auto& k : kept) {
    out.hits.push_back(k.hits);
    out.states.insert(out.states.end(), k.st.begin(), k.st.end());
    out.features.insert(out.features.end(), k.f.begin(), k.f.end());
  }
}

void build_hits(uint64_t n, const uint32_t* module, const float* x, const float* y, const vo_geometry_t* g,
                Hits& H) {
  H.n = (uint32_t)n;
  H.module.assign(module, module + n);
  H.x.assign(x, x + n);
  H.y.assign(y, y + n);
  H.z.resize(n);
  H.key.resize(n);
  for (uint64_t i = 0; i < n; ++i) {
    H.z[i] = g->module_z[module[i]];
    H.key[i] = pseudo_angle(x[i], y[i]);
  }
  H.by_module.assign(g->n_modules, {});
  for (uint32_t i = 0; i < n; ++i) H.by_module[module[i]].push_back(i);
  for (auto& v : H.by_module)
    std::sort(v.begin(), v.end(), [&](uint32_t a, uint32_t b) {
      if (H.key[a] != H.key[b]) return H.key[a] < H.key[b];
      return a < b;
    });
}

struct EventResult {
  ClusterOut cl;
  TrackOut tr;
};

struct Batch {
  std::vector<EventResult> ev;
};

}  // namespace

extern "C" {

float vo_pseudo_angle(float x, float y) { return pseudo_angle(x, y); }

int vo_cluster_event(const uint32_t* words, uint64_t n, const vo_geometry_t* geo, float* cx, float* cy,
                     float* cz, uint32_t* cmodule, uint32_t* pixel_cluster, uint64_t* n_clusters) {
  ClusterOut c;
  cluster_event(words, n, geo, c);
  size_t nc = c.x.size();
  for (size_t i = 0; i < nc; ++i) {
    if (cx) cx[i] = c.x[i];
    if (cy) cy[i] = c.y[i];
    if (cz) cz[i] = c.z[i];
    if (cmodule) cmodule[i] = c.module[i];
  }
  if (pixel_cluster) std::memcpy(pixel_cluster, c.pixel_cluster.data(), n * 4);
  *n_clusters = nc;
  return c.status;
}

int vo_track_event(uint64_t n_hits, const uint32_t* module, const float* x, const float* y,
                   const vo_geometry_t* geo, const vo_params_t* p, uint64_t cap_tracks, uint64_t* n_tracks,
                   uint64_t* hit_offsets, uint32_t* hit_ids, float* states) {
  Hits H;
  build_hits(n_hits, module, x, y, geo, H);
  TrackOut T;
  track_event(H, geo, p, T);
  if (T.hits.size() > cap_tracks) return -1;
  *n_tracks = T.hits.size();
  uint64_t o = 0;
  for (size_t t = 0; t < T.hits.size(); ++t) {
    hit_offsets[t] = o;
    for (uint32_t h : T.hits[t]) hit_ids[o++] = h;
  }
  hit_offsets[T.hits.size()] = o;
  std::memcpy(states, T.states.data(), T.states.size() * 4);
  return 0;
}

void vo_fit_f32(uint32_t n, const float* x, const float* y, const float* z, float sigma, float ms_theta,
                float* state) {
  fit_track<float>(n, x, y, z, sigma, ms_theta, state);
}

void vo_fit_f64(uint32_t n, const double* x, const double* y, const double* z, double sigma, double ms_theta,
                double* state) {
  fit_track<double>(n, x, y, z, sigma, ms_theta, state);
}

void* vo_reconstruct(uint64_t n_events, const uint64_t* off, const uint32_t* pixels, const vo_geometry_t* geo,
                     const vo_params_t* p, int n_threads) {
  Batch* B = new Batch;
  B->ev.resize(n_events);
  int nt = n_threads > 0 ? n_threads : (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  std::atomic<uint64_t> next(0);
  auto work = [&]() {
    for (;;) {
      uint64_t e = next.fetch_add(1);
      if (e >= n_events) break;
      EventResult& R = B->ev[e];
      cluster_event(pixels + off[e], off[e + 1] - off[e], geo, R.cl);
      if (R.cl.status != VO_EVT_OK) continue;
      Hits H;
      build_hits(R.cl.x.size(), R.cl.module.data(), R.cl.x.data(), R.cl.y.data(), geo, H);
      track_event(H, geo, p, R.tr);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return B;
}

void vo_batch_sizes(void* h, uint64_t* n_clusters, uint64_t* n_tracks, uint64_t* n_track_hits) {
  Batch* B = (Batch*)h;
  uint64_t c = 0, t = 0, k = 0;
  for (auto& e : B->ev) {
    c += e.cl.x.size();
    t += e.tr.hits.size();
    for (auto& v : e.tr.hits) k += v.size();
  }
  *n_clusters = c;
  *n_tracks = t;
  *n_track_hits = k;
}

void vo_batch_copy(void* h, int32_t* status, uint64_t* cluster_offsets, float* cx, float* cy, float* cz,
                   uint32_t* pixel_cluster, uint64_t* track_offsets, uint64_t* track_hit_offsets,
                   uint32_t* track_hits, float* track_states, float* track_features) {
  Batch* B = (Batch*)h;
  uint64_t c = 0, t = 0, k = 0, p = 0;
  for (size_t e = 0; e < B->ev.size(); ++e) {
    const EventResult& R = B->ev[e];
    if (status) status[e] = R.cl.status;
    if (cluster_offsets) cluster_offsets[e] = c;
    if (track_offsets) track_offsets[e] = t;
    for (size_t i = 0; i < R.cl.x.size(); ++i, ++c) {
      if (cx) cx[c] = R.cl.x[i];
      if (cy) cy[c] = R.cl.y[i];
      if (cz) cz[c] = R.cl.z[i];
    }
    if (pixel_cluster) {
      if (!R.cl.pixel_cluster.empty())
        std::memcpy(pixel_cluster + p, R.cl.pixel_cluster.data(), R.cl.pixel_cluster.size() * 4);
    }
    p += R.cl.pixel_cluster.size();
    for (size_t i = 0; i < R.tr.hits.size(); ++i, ++t) {
      if (track_hit_offsets) track_hit_offsets[t] = k;
      for (uint32_t hid : R.tr.hits[i]) {
        if (track_hits) track_hits[k] = hid;
        ++k;
      }
      if (track_states) std::memcpy(track_states + t * VO_STATE_STRIDE, R.tr.states.data() + i * VO_STATE_STRIDE, VO_STATE_STRIDE * 4);
      if (track_features)
        std::memcpy(track_features + t * VO_N_FEATURES, R.tr.features.data() + i * VO_N_FEATURES, VO_N_FEATURES * 4);
    }
  }
  if (cluster_offsets) cluster_offsets[B->ev.size()] = c;
  if (track_offsets) track_offsets[B->ev.size()] = t;
  if (track_hit_offsets) track_hit_offsets[t] = k;
}

void vo_batch_free(void* h) { delete (Batch*)h; }

void vo_features(uint32_t n, const float* x, const float* y, const float* z, const uint32_t* module,
                 const float* state, float chi2ndf, float* f) {
  features(n, x, y, z, module, state, chi2ndf, f);
}

float vo_mlp_logit(const float* mlp, const float* f) { return mlp_logit(mlp, f); }

// Forward tracking of one event, the steps in the order the header states.
void vo_forward_event(uint64_t n_hits, const uint32_t* layer, const float* x, const float* y, uint64_t n_tracks,
                      const uint64_t* track_hit_offsets, const uint32_t* track_hits, const float* cluster_x,
                      const float* cluster_y, const float* cluster_z, const vo_downstream_t* geo,
                      const vo_fwd_params_t* p, uint32_t* n_found, uint32_t* hits, float* state) {
  const int NL = VO_FWD_LAYERS;
  for (uint64_t t = 0; t < n_tracks; ++t) {
    n_found[t] = 0u;
    for (int L = 0; L < NL; ++L) hits[t * NL + L] = 0xFFFFFFFFu;
    for (int k = 0; k < VO_FWD_STATE; ++k) state[t * VO_FWD_STATE + k] = 0.0f;
    if (track_hit_offsets[t + 1] < track_hit_offsets[t] + 2) continue;  // no line through fewer than two hits
    // 0. the line through the two most downstream hits (ids ascend with z)
    const uint32_t ha = track_hits[track_hit_offsets[t + 1] - 1], hb = track_hits[track_hit_offsets[t + 1] - 2];
    const float x0 = cluster_x[ha], y0 = cluster_y[ha], z0 = cluster_z[ha];
    const float dzab = z0 - cluster_z[hb];
    const float tx = (x0 - cluster_x[hb]) / dzab, ty = (y0 - cluster_y[hb]) / dzab;
    // 1. the straight line at the kick plane
    const float dzm = geo->z_mag - z0;
    const float xm = x0 + tx * dzm, ym = y0 + ty * dzm;
    bool have = false;
    uint32_t b_n = 0, b_c = 0;
    float b_r = 0.0f, b_b = 0.0f, b_a = 0.0f, b_d = 0.0f, b_dy = 0.0f, b_ad = 0.0f;
    uint32_t b_hits[VO_FWD_LAYERS];
    for (int r = 0; r < 2; ++r) {
      // 2. candidates in the first two layers
      const float dzr = geo->z_layers[r] - geo->z_mag;
      const float xr = xm + tx * dzr, yr = ym + ty * dzr;
      const float wx = (geo->kappa / p->p_min) * dzr + p->tol_x;
      for (uint64_t c = 0; c < n_hits; ++c) {
        if (layer[c] != (uint32_t)r) continue;
        // a distance that is not a number never lies within a window
        if (!(std::fabs(x[c] - xr) <= wx) || !(std::fabs(y[c] - yr) <= p->win_y)) continue;
        // 3. the slope behind the magnet; the first station from it, the
        // others from the line through the first station's hits
        const float tk = (x[c] - xm) / dzr;
        uint32_t hl[VO_FWD_LAYERS];
        auto nearest = [&](int L, float xp, float yp, float tol) -> uint32_t {
          bool f = false;
          float bd = 0.0f;
          uint32_t bh = 0xFFFFFFFFu;
          for (uint64_t h = 0; h < n_hits; ++h) {
            if (layer[h] != (uint32_t)L) continue;
            const float d = std::fabs(x[h] - xp);
            if (!(d <= tol) || !(std::fabs(y[h] - yp) <= p->tol_y)) continue;
            if (!f || d < bd || (d == bd && h < bh)) { f = true; bd = d; bh = (uint32_t)h; }
          }
          return bh;
        };
        // least-squares line x = a + b (z - z_0) through the found hits of layers [l0, l1)
        auto line = [&](int l0, int l1, float* a_out, float* b_out) -> uint32_t {
          float S0 = 0.0f, Sz = 0.0f, Szz = 0.0f, Sx = 0.0f, Sxz = 0.0f;
          uint32_t k = 0;
          for (int L = l0; L < l1; ++L) {
            if (hl[L] == 0xFFFFFFFFu) continue;
            const float dz = geo->z_layers[L] - geo->z_layers[0];
            S0 = S0 + 1.0f;
            Sz = Sz + dz;
            Szz = Szz + dz * dz;
            Sx = Sx + x[hl[L]];
            Sxz = Sxz + x[hl[L]] * dz;
            ++k;
          }
          const float det = S0 * Szz - Sz * Sz;
          const float bb = (S0 * Sxz - Sz * Sx) / det;
          *b_out = bb;
          *a_out = (Sx - bb * Sz) / S0;
          return k;
        };
        uint32_t n1 = 0;
        for (int L = 0; L < 4; ++L) {
          const float dzl = geo->z_layers[L] - geo->z_mag;
          hl[L] = nearest(L, xm + tk * dzl, ym + ty * dzl, p->tol_x);
          n1 += hl[L] != 0xFFFFFFFFu ? 1u : 0u;
        }
        if (n1 < 2) continue;
        float a1, b1;
        line(0, 4, &a1, &b1);
        uint32_t n = n1;
        for (int L = 4; L < NL; ++L) {
          const float dzl = geo->z_layers[L] - geo->z_mag;
          hl[L] = nearest(L, a1 + b1 * (geo->z_layers[L] - geo->z_layers[0]), ym + ty * dzl, p->tol_x_far);
          n += hl[L] != 0xFFFFFFFFu ? 1u : 0u;
        }
        if (n < p->min_hits) continue;
        // 4. straight line through all of them and its chi2
        float a, b;
        line(0, NL, &a, &b);
        float chi2 = 0.0f;
        for (int L = 0; L < NL; ++L) {
          if (hl[L] == 0xFFFFFFFFu) continue;
          const float dz = geo->z_layers[L] - geo->z_layers[0];
          const float res = ((x[hl[L]] - a) - b * dz) / p->sigma_x;
          chi2 = chi2 + res * res;
        }
        const float rchi = chi2 / (float)(n - 2);
        if (!(rchi <= p->chi2ndf_max)) continue;
        // 4-5. the y line and the match at the kick plane, in x and in y (y is not bent)
        const float d = (a + b * (geo->z_mag - geo->z_layers[0])) - xm;
        float Y0 = 0.0f, Yz = 0.0f, Yzz = 0.0f, Yy = 0.0f, Yyz = 0.0f;
        for (int L = 0; L < NL; ++L) {
          if (hl[L] == 0xFFFFFFFFu) continue;
          const float dz = geo->z_layers[L] - geo->z_layers[0];
          Y0 = Y0 + 1.0f;
          Yz = Yz + dz;
          Yzz = Yzz + dz * dz;
          Yy = Yy + y[hl[L]];
          Yyz = Yyz + y[hl[L]] * dz;
        }
        const float ydet = Y0 * Yzz - Yz * Yz;
        const float yb = (Y0 * Yyz - Yz * Yy) / ydet;
        const float ya = (Yy - yb * Yz) / Y0;
        const float dy = (ya + yb * (geo->z_mag - geo->z_layers[0])) - ym;
        const float ad = d * d + dy * dy;
        if (!(ad <= p->tol_match * p->tol_match)) continue;
        // 6. most hits, then the smallest distance, then the smallest candidate id
        const bool better = !have || n > b_n || (n == b_n && (ad < b_ad || (ad == b_ad && c < b_c)));
        if (!better) continue;
        have = true;
        b_n = n;
        b_c = (uint32_t)c;
        b_r = rchi;
        b_b = b;
        b_a = a;
        b_d = d;
        b_dy = dy;
        b_ad = ad;
        for (int L = 0; L < NL; ++L) b_hits[L] = hl[L];
      }
    }
    n_found[t] = have ? b_n : 0u;
    for (int L = 0; L < NL; ++L) hits[t * NL + L] = have ? b_hits[L] : 0xFFFFFFFFu;
    float* so = state + t * VO_FWD_STATE;
    so[0] = have ? (b_b - tx) / geo->kappa : 0.0f;
    so[1] = have ? b_r : 0.0f;
    so[2] = have ? b_b : 0.0f;
    so[3] = have ? b_a : 0.0f;
    so[4] = have ? b_d : 0.0f;
    so[5] = have ? b_dy : 0.0f;
  }
}

}  // extern "C"
