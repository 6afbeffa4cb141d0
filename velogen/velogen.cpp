// Seeded synthetic event generator for VELO-like pixel tracking.
//
// This module only produces input data (pixel words) and Monte-Carlo truth.
// It holds none of the reconstruction arithmetic: both the CPU oracle and the
// CUDA path consume its output, and neither depends on how it was produced.
//
// Physics model (the paper gives the detector only in words, Sec. "Detector":
// a pixel tracker around the interaction region, pp collisions at pile-up ~5,
// Sec. "Introduction"; the numbers below are the synthetic workload's):
//   * primary vertices: x, y ~ N(0, sigma_xy), z ~ N(0, sigma_z);
//   * straight tracks from each vertex with eta ~ U[eta_min, eta_max],
//     phi ~ U[0, 2 pi), optionally kinked at every module plane by
//     independent N(0, ms_theta) kicks to tx and ty;
//   * each (particle, module) crossing is kept with probability hit_eff and
//     deposited on the 2x2 pixels nearest to the crossing point with bilinear
//     weights w, charge q = round-half-even(15 w), q = 0 dropped, deposits on
//     one pixel add and saturate at 15, pixels outside the sensitive annulus
//     (judged at the pixel centre) dropped;
//   * noise: every sensitive cell of every module fires with probability
//     noise_prob (drawn as Poisson(noise_prob * n_sensitive) cells placed
//     uniformly), charge ~ U{1..15};
//   * pixel truth = the particle with the largest deposit on that pixel
//     (noise = -1; ties go to the smaller id).
// Every event draws from its own SplitMix64 stream seeded by (seed, event
// index), so any event regenerates alone and the output does not depend on
// the thread count.
//
// Pixel word: q << 27 | module << 22 | row << 11 | col.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

extern "C" {

typedef struct velogen_config {
  uint64_t seed;
  int32_t fixed_pvs;      // > 0: exactly this many primary vertices per event
  int32_t fixed_tracks;   // > 0: exactly this many tracks per vertex
  double pv_mu;           // else n_PV ~ Poisson(pv_mu)
  double heavy_frac;      // fraction of events with n_PV ~ Poisson(pv_mu_heavy)
  double pv_mu_heavy;
  double hi_frac;         // fraction of heavy-ion-like events (1 PV, U{hi_min..hi_max} tracks)
  int32_t hi_min_tracks;
  int32_t hi_max_tracks;
  double tracks_mu;       // tracks per PV ~ Poisson(tracks_mu) unless fixed_tracks > 0
  double eta_min, eta_max;
  double pv_sigma_xy, pv_sigma_z;
  double ms_theta;        // multiple-scattering kick sigma per module plane [rad]
  double hit_eff;         // probability to keep a (particle, module) deposit
  double noise_prob;      // per sensitive cell per module
  int32_t shuffle;        // shuffle the words inside each event
  int32_t n_threads;      // <= 0: hardware concurrency
} velogen_config_t;

typedef struct velogen_geometry {
  int32_t n_modules;
  int32_t n_rows, n_cols;
  double module_z[32];
  double pitch;
  double x0, y0;          // lower edge of the pixel grid [mm]
  double r_min, r_max;    // sensitive annulus, judged at the pixel centre [mm]
} velogen_geometry_t;

// Per particle record (float64 x 15):
//   pv, x0, y0, z0, tx, ty, eta, phi, n_modules_with_pixels, heavy_ion_event,
//   and the line it leaves the pixel tracker on (after the last kink):
//   x, y, z, tx, ty there (the vertex and first direction if it crossed no module)
enum { VELOGEN_PARTICLE_FIELDS = 15 };

}  // extern "C"

namespace {

inline uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed) {}
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    return splitmix64_mix(s);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)
  double uniform_open() {  // (0,1)
    double u;
    do { u = uniform(); } while (u <= 0.0);
    return u;
  }
  double normal() {  // Box-Muller, one value per call
    double u1 = uniform_open(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  uint32_t below(uint32_t n) { return (uint32_t)(uniform() * n); }
  int64_t poisson(double mu) {  // Knuth; fine for the means used here (< 700)
    if (mu <= 0) return 0;
    double L = std::exp(-mu), p = 1.0;
    int64_t k = 0;
    do { ++k; p *= uniform(); } while (p > L);
    return k - 1;
  }
};

inline uint64_t event_seed(uint64_t seed, uint64_t e) {
  return splitmix64_mix(seed ^ splitmix64_mix(e + 0x632BE59BD9B4E019ull));
}

struct Deposit {
  uint32_t key;    // module << 22 | row << 11 | col
  int32_t particle;
  uint32_t q;
};

struct EventOut {
  std::vector<uint32_t> words;
  std::vector<int32_t> truth;
  std::vector<double> particles;
};

struct Gen {
  velogen_config_t c;
  velogen_geometry_t g;
  uint64_t n_sensitive = 0;
  std::vector<uint8_t> sensitive;  // n_rows * n_cols

  bool cell_sensitive(int r, int col) const {
    double xc = g.x0 + g.pitch * (col + 0.5), yc = g.y0 + g.pitch * (r + 0.5);
    double rr = std::sqrt(xc * xc + yc * yc);
    return rr >= g.r_min && rr <= g.r_max;
  }

  void init() {
    sensitive.assign((size_t)g.n_rows * g.n_cols, 0);
    n_sensitive = 0;
    for (int r = 0; r < g.n_rows; ++r)
      for (int col = 0; col < g.n_cols; ++col)
        if (cell_sensitive(r, col)) {
          sensitive[(size_t)r * g.n_cols + col] = 1;
          ++n_sensitive;
        }
  }

  void deposit(std::vector<Deposit>& d, int m, double x, double y, int32_t pid) const {
    double u = (x - g.x0) / g.pitch - 0.5, v = (y - g.y0) / g.pitch - 0.5;
    double cu = std::floor(u), cv = std::floor(v);
    double fu = u - cu, fv = v - cv;
    long c0 = (long)cu, r0 = (long)cv;
    const double w[4] = {(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv};
    const long dc[4] = {0, 1, 0, 1}, dr[4] = {0, 0, 1, 1};
    for (int i = 0; i < 4; ++i) {
      long col = c0 + dc[i], row = r0 + dr[i];
      if (col < 0 || row < 0 || col >= g.n_cols || row >= g.n_rows) continue;
      if (!sensitive[(size_t)row * g.n_cols + col]) continue;
      double qd = std::nearbyint(15.0 * w[i]);  // round half to even
      if (qd <= 0) continue;
      d.push_back({(uint32_t)m << 22 | (uint32_t)row << 11 | (uint32_t)col, pid, (uint32_t)qd});
    }
  }

  void event(uint64_t e, EventOut& out, bool want_truth) const {
    Rng rng(event_seed(c.seed, e));
    std::vector<Deposit> dep;
    std::vector<double>& parts = out.particles;
    parts.clear();
    bool hi = c.hi_frac > 0 && rng.uniform() < c.hi_frac;
    bool heavy = c.heavy_frac > 0 && rng.uniform() < c.heavy_frac;
    int64_t n_pv;
    if (hi) n_pv = 1;
    else if (c.fixed_pvs > 0) n_pv = c.fixed_pvs;
    else n_pv = rng.poisson(heavy ? c.pv_mu_heavy : c.pv_mu);
    int32_t pid = 0;
    for (int64_t v = 0; v < n_pv; ++v) {
      double vx = c.pv_sigma_xy * rng.normal();
      double vy = c.pv_sigma_xy * rng.normal();
      double vz = c.pv_sigma_z * rng.normal();
      int64_t nt;
      if (hi) nt = c.hi_min_tracks + (int64_t)rng.below((uint32_t)(c.hi_max_tracks - c.hi_min_tracks + 1));
      else if (c.fixed_tracks > 0) nt = c.fixed_tracks;
      else nt = rng.poisson(c.tracks_mu);
      for (int64_t t = 0; t < nt; ++t, ++pid) {
        double eta = c.eta_min + (c.eta_max - c.eta_min) * rng.uniform();
        double phi = 6.283185307179586 * rng.uniform();
        double theta = 2.0 * std::atan(std::exp(-eta));
        double tn = std::tan(theta);
        double tx0 = tn * std::cos(phi), ty0 = tn * std::sin(phi);
        double tx = tx0, ty = ty0, x = vx, y = vy, z = vz;
        int n_mod_dep = 0;
        for (int m = 0; m < g.n_modules; ++m) {
          double zm = g.module_z[m];
          if (zm <= vz) continue;
          x += tx * (zm - z);
          y += ty * (zm - z);
          z = zm;
          bool keep = rng.uniform() < c.hit_eff;
          if (keep) {
            size_t before = dep.size();
            deposit(dep, m, x, y, pid);
            if (dep.size() > before) ++n_mod_dep;
          }
          if (c.ms_theta > 0) {
            tx += c.ms_theta * rng.normal();
            ty += c.ms_theta * rng.normal();
          }
        }
        if (want_truth) {
          double rec[VELOGEN_PARTICLE_FIELDS] = {(double)v, vx, vy, vz, tx0, ty0, eta, phi,
                                                 (double)n_mod_dep, hi ? 1.0 : 0.0, x, y, z, tx, ty};
          parts.insert(parts.end(), rec, rec + VELOGEN_PARTICLE_FIELDS);
        }
      }
    }
    if (c.noise_prob > 0) {
      double mu = c.noise_prob * (double)n_sensitive;
      for (int m = 0; m < g.n_modules; ++m) {
        int64_t nn = rng.poisson(mu);
        for (int64_t i = 0; i < nn; ++i) {
          uint32_t row, col;
          do {
            row = rng.below((uint32_t)g.n_rows);
            col = rng.below((uint32_t)g.n_cols);
          } while (!sensitive[(size_t)row * g.n_cols + col]);
          uint32_t q = 1 + rng.below(15);
          dep.push_back({(uint32_t)m << 22 | row << 11 | col, -1, q});
        }
      }
    }
    // merge deposits on the same pixel
    std::sort(dep.begin(), dep.end(), [](const Deposit& a, const Deposit& b) {
      if (a.key != b.key) return a.key < b.key;
      return a.particle < b.particle;
    });
    out.words.clear();
    out.truth.clear();
    size_t i = 0;
    while (i < dep.size()) {
      size_t j = i;
      uint32_t qsum = 0;
      // per-contributor totals (deposits of one particle on one pixel add first)
      int32_t best_p = 0;
      uint32_t best_q = 0;
      bool have = false;
      while (j < dep.size() && dep[j].key == dep[i].key) {
        size_t k = j;
        uint32_t qp = 0;
        while (k < dep.size() && dep[k].key == dep[i].key && dep[k].particle == dep[j].particle) qp += dep[k++].q;
        qsum += qp;
        if (!have || qp > best_q) { best_q = qp; best_p = dep[j].particle; have = true; }
        j = k;
      }
      uint32_t q = qsum > 15 ? 15 : qsum;
      out.words.push_back(q << 27 | dep[i].key);
      out.truth.push_back(best_p);
      i = j;
    }
    if (c.shuffle) {
      for (size_t k = out.words.size(); k > 1; --k) {
        size_t r = (size_t)(rng.uniform() * (double)k);
        std::swap(out.words[k - 1], out.words[r]);
        std::swap(out.truth[k - 1], out.truth[r]);
      }
    }
    if (!want_truth) out.truth.clear();
  }
};

struct Handle {
  std::vector<EventOut> ev;
  bool truth;
};

}  // namespace

extern "C" {

void* velogen_run(const velogen_config_t* cfg, const velogen_geometry_t* geo, uint64_t first_event,
                  uint64_t n_events, int want_truth) {
  if (!cfg || !geo || geo->n_modules <= 0 || geo->n_modules > 32) return nullptr;
  Gen gen;
  gen.c = *cfg;
  gen.g = *geo;
  gen.init();
  Handle* h = new Handle;
  h->truth = want_truth != 0;
  h->ev.resize(n_events);
  int nt = cfg->n_threads > 0 ? cfg->n_threads : (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if ((uint64_t)nt > n_events) nt = (int)(n_events ? n_events : 1);
  std::atomic<uint64_t> next(0);
  auto work = [&]() {
    for (;;) {
      uint64_t i = next.fetch_add(1);
      if (i >= n_events) break;
      gen.event(first_event + i, h->ev[i], h->truth);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  return h;
}

int velogen_sizes(void* hv, uint64_t* n_events, uint64_t* n_pixels, uint64_t* n_particles) {
  Handle* h = (Handle*)hv;
  if (!h) return -1;
  uint64_t p = 0, q = 0;
  for (auto& e : h->ev) {
    p += e.words.size();
    q += e.particles.size() / VELOGEN_PARTICLE_FIELDS;
  }
  if (n_events) *n_events = h->ev.size();
  if (n_pixels) *n_pixels = p;
  if (n_particles) *n_particles = q;
  return 0;
}

// Copies the generated batch out. Any output pointer may be NULL.
//   offsets[n_events+1], pixels[n_pixels], pixel_truth[n_pixels],
//   particle_offsets[n_events+1], particles[n_particles * VELOGEN_PARTICLE_FIELDS]
int velogen_copy(void* hv, uint64_t* offsets, uint32_t* pixels, int32_t* pixel_truth,
                 uint64_t* particle_offsets, double* particles) {
  Handle* h = (Handle*)hv;
  if (!h) return -1;
  if ((pixel_truth || particles || particle_offsets) && !h->truth) return -2;
  uint64_t p = 0, q = 0;
  for (size_t e = 0; e < h->ev.size(); ++e) {
    const EventOut& E = h->ev[e];
    if (offsets) offsets[e] = p;
    if (particle_offsets) particle_offsets[e] = q;
    if (pixels && !E.words.empty()) std::memcpy(pixels + p, E.words.data(), E.words.size() * 4);
    if (pixel_truth && !E.truth.empty()) std::memcpy(pixel_truth + p, E.truth.data(), E.truth.size() * 4);
    if (particles && !E.particles.empty())
      std::memcpy(particles + q * VELOGEN_PARTICLE_FIELDS, E.particles.data(), E.particles.size() * 8);
    p += E.words.size();
    q += E.particles.size() / VELOGEN_PARTICLE_FIELDS;
  }
  if (offsets) offsets[h->ev.size()] = p;
  if (particle_offsets) particle_offsets[h->ev.size()] = q;
  return 0;
}

void velogen_free(void* hv) { delete (Handle*)hv; }

uint64_t velogen_n_sensitive(const velogen_geometry_t* geo) {
  Gen gen;
  gen.g = *geo;
  gen.init();
  return gen.n_sensitive;
}

}  // extern "C"
