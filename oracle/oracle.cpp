// CPU oracle for Monte Carlo photon propagation through layered ice.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, double-precision
// statement of what the GPU path must compute.  Only the tests, the smoke
// check and the benchmark's CPU-baseline leg load it; the library's product
// path never does.  It shares no code, header, table or helper with the CUDA
// library: it reads the same input arrays and nothing else.
//
// What it follows.  The paper (Sec. 2, "Old Simulation Chain") describes the
// photon propagation step in a few sentences: the ice is divided into 10 m
// layers, each with its own scattering and absorption coefficient; for every
// photon a Monte Carlo draw gives the distance to the next scatter, a new
// direction is picked from the scattering physics, and this repeats until the
// photon meets a detector module (DOM) or is absorbed.  Photons are
// independent ("embarrassingly parallel", Sec. 2).  Everything numeric beyond
// that skeleton is a stated reading:
//   * random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11,
//     "Parallel Random Numbers: As Easy as 1, 2, 3"), key (seed lo, seed hi),
//     counter (photon id lo, photon id hi, block, event id lo); block 0 =
//     birth, block n >= 1 = step n;
//   * u = ((x >> 8) | 1) * 2^-24, exact in binary32 and binary64, in (0, 1);
//   * step lengths: exponential in optical depth, the scattering coefficient
//     b = b_e / (1 - g) (b_e is the effective coefficient), absorption
//     optical depth tau_a drawn once at birth and consumed along the path;
//   * scattering angle: Henyey-Greenstein inversion (Henyey & Greenstein,
//     ApJ 93, 1941), direction update by the MCML rotation formulas (Wang,
//     Jacques & Zheng, Comput. Methods Programs Biomed. 47, 1995);
//   * a DOM is a sphere; the first sphere met along the step wins, ties to
//     the lowest DOM index; a hit counts as one (acceptance not modelled);
//   * the world is a vertical cylinder: DOM extent plus a margin; leaving it
//     is "escaped";
//   * a step cap: reaching it counts as absorbed and as "truncated".
//
// Parity pins (the tests that tie this file to something other than itself)
// are in tests/test_oracle_*.py.
//
// Broad phase.  first_hit() tests every DOM (brute force) when asked to; by
// default it first drops DOMs whose axis-aligned bounding box cannot overlap
// the step's bounding box.  That filter only removes spheres the segment
// cannot touch, so the result is the brute-force result; a test checks the
// two agree on random segments.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

const double kInf = std::numeric_limits<double>::infinity();
const double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------ Philox --
// Philox4x32 with 10 rounds, from its definition in Salmon et al. (SC'11):
// one round maps counter words (c0, c1, c2, c3) under key (k0, k1) to
//   (hi(B*c2) ^ c1 ^ k0,  lo(B*c2),  hi(A*c0) ^ c3 ^ k1,  lo(A*c0))
// with A = 0xD2511F53, B = 0xCD9E8D57; between rounds the key is bumped by the
// Weyl constants (0x9E3779B9, 0xBB67AE85).
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t pa = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t pb = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi_a = (uint32_t)(pa >> 32), lo_a = (uint32_t)pa;
    const uint32_t hi_b = (uint32_t)(pb >> 32), lo_b = (uint32_t)pb;
    const uint32_t n0 = hi_b ^ c[1] ^ k0;
    const uint32_t n2 = hi_a ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo_b;
    c[2] = n2;
    c[3] = lo_a;
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

// uint32 -> uniform in (0, 1): the top 24 bits with the lowest forced to one,
// scaled by 2^-24; every value is an odd multiple of 2^-24.
double u01(uint32_t x) { return (double)((x >> 8) | 1u) * 0x1p-24; }

// --------------------------------------------------------------- Geometry --

struct Ice {
  int L = 0;
  double z_top = 0;   // z of the top of layer 0 (depth_top)
  double dz = 10;     // layer thickness (Sec. 2: 10 m)
  double g = 0.9;     // HG mean cosine
  std::vector<double> b, a;  // geometric scattering / absorption per layer (1/m)
  // z of boundary k: top of layer k (k = 0..L)
  double zb(int k) const { return z_top - (double)k * dz; }
};

struct World {
  double R = 0, zlo = 0, zhi = 0;
};

struct Cluster {        // DOMs of one string, with their joint bounding box
  double lo[3], hi[3];
  std::vector<int> doms;  // ascending DOM index
};

struct Geom {
  int n = 0;
  double r = 0;
  std::vector<double> x, y, z;
  std::vector<Cluster> clusters;
};

}  // namespace

extern "C" {

// Inputs to the oracle.  Geometry and ice arrays are the same float32 arrays
// the library receives; the oracle widens them to double.
struct orc_params {
  uint64_t seed;
  uint32_t max_steps;
  int32_t scatter_coeff_is_effective;  // 1: b = b_e / (1 - g); 0: b = b_e
  double g;
  double world_margin;
  double depth_of_z0;                  // z = depth_of_z0 - depth
  int32_t n_dom;
  int32_t brute_force;                 // 1: no bounding-box filter in first_hit
  double dom_radius;
  const float* dom_xyz;                // [n_dom][3]
  const int32_t* string_id;            // [n_dom] or NULL (one cluster)
  int32_t n_layers;
  int32_t n_threads;                   // 0: all hardware threads
  double depth_top;
  double layer_dz;
  const float* b_e;                    // [n_layers]
  const float* a;                      // [n_layers]
};

}  // extern "C"

namespace {

struct Model {
  Ice ice;
  World world;
  Geom geom;
  uint64_t seed = 0;
  uint32_t max_steps = 100000;
  bool brute = false;
};

void build_model(const orc_params* P, Model* M) {
  M->seed = P->seed;
  M->max_steps = P->max_steps;
  M->brute = P->brute_force != 0;
  // Ice: Sec. 2 -- vertical layers of 10 m, each with its own scattering and
  // absorption coefficient.  Layer i spans depth [top + i dz, top + (i+1) dz).
  Ice& ice = M->ice;
  ice.L = P->n_layers;
  ice.dz = P->layer_dz;
  ice.g = P->g;
  ice.z_top = P->depth_of_z0 - P->depth_top;
  ice.b.resize(ice.L);
  ice.a.resize(ice.L);
  for (int i = 0; i < ice.L; ++i) {
    const double be = (double)P->b_e[i];
    ice.b[i] = P->scatter_coeff_is_effective ? be / (1.0 - P->g) : be;
    ice.a[i] = (double)P->a[i];
  }
  // Geometry: DOM spheres (Sec. 1: 5160 DOMs between 1450 m and 2450 m).
  Geom& G = M->geom;
  G.n = P->n_dom;
  G.r = P->dom_radius;
  G.x.resize(G.n);
  G.y.resize(G.n);
  G.z.resize(G.n);
  double rmax = 0, zmin = 0, zmax = 0;
  for (int k = 0; k < G.n; ++k) {
    G.x[k] = P->dom_xyz[3 * k + 0];
    G.y[k] = P->dom_xyz[3 * k + 1];
    G.z[k] = P->dom_xyz[3 * k + 2];
    rmax = std::max(rmax, std::sqrt(G.x[k] * G.x[k] + G.y[k] * G.y[k]));
    if (k == 0 || G.z[k] < zmin) zmin = G.z[k];
    if (k == 0 || G.z[k] > zmax) zmax = G.z[k];
  }
  // World: a vertical cylinder about the z axis, DOM extent plus the margin.
  M->world.R = rmax + P->world_margin;
  M->world.zlo = zmin - P->world_margin;
  M->world.zhi = zmax + P->world_margin;
  // Clusters for the bounding-box filter: one per string id.
  std::vector<int> ids(G.n, 0);
  if (P->string_id)
    for (int k = 0; k < G.n; ++k) ids[k] = P->string_id[k];
  std::vector<int> order(G.n);
  for (int k = 0; k < G.n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return ids[p] < ids[q]; });
  for (int idx = 0; idx < G.n;) {
    int j = idx;
    Cluster c;
    for (int d = 0; d < 3; ++d) {
      c.lo[d] = kInf;
      c.hi[d] = -kInf;
    }
    while (j < G.n && ids[order[j]] == ids[order[idx]]) {
      const int k = order[j];
      const double p[3] = {G.x[k], G.y[k], G.z[k]};
      for (int d = 0; d < 3; ++d) {
        c.lo[d] = std::min(c.lo[d], p[d] - G.r);
        c.hi[d] = std::max(c.hi[d], p[d] + G.r);
      }
      c.doms.push_back(k);
      ++j;
    }
    std::sort(c.doms.begin(), c.doms.end());
    G.clusters.push_back(c);
    idx = j;
  }
}

// Layer of a point at height z moving with vertical direction component w:
// floor((z_top - z) / dz), except that a point exactly on a boundary and
// moving up belongs to the layer above; clamped to the table (depths outside
// it take the edge layer's properties).
int layer_at(const Ice& ice, double z, double w) {
  const double f = (ice.z_top - z) / ice.dz;
  if (!(f >= 0.0)) return 0;                   // above the table
  if (f >= (double)ice.L) return ice.L - 1;    // below the table
  const double fl = std::floor(f);
  int i = (int)fl;
  if (w > 0.0 && f == fl) i -= 1;
  return std::max(0, std::min(ice.L - 1, i));
}

// One step's walk through the layers (Sec. 2: "distance to the next scatter"
// drawn by Monte Carlo in layered ice).  The step consumes the scattering
// optical depth tau_s with the local b_i and the photon's remaining absorption
// optical depth tau_a with the local a_i; it ends at the scatter point or at
// the absorption point, whichever comes first (a tie is absorption).  Layer
// boundaries are crossed on the way; the photon's layer index is carried.
struct WalkResult {
  double S;          // geometric length of the step (m)
  bool absorb;       // the step ends by absorption
  int layer;         // layer at the end of the step
  double tau_a;      // absorption optical depth left
  int64_t crossings;
  double race;       // |da - ds| in the last layer (m): how close scatter and
                     // absorption came (a diagnostic, not used by the method)
};

WalkResult walk(const Ice& ice, double z, double w, int layer, double tau_s, double tau_a) {
  WalkResult r{0.0, false, layer, tau_a, 0, kInf};
  double zc = z;
  for (;;) {
    const int i = r.layer;
    const double bi = ice.b[i], ai = ice.a[i];
    double ell = kInf;  // distance to the boundary ahead (none in the edge layers)
    if (w < 0.0 && i < ice.L - 1) ell = (ice.zb(i + 1) - zc) / w;
    else if (w > 0.0 && i > 0) ell = (ice.zb(i) - zc) / w;
    if (ell < 0.0) ell = 0.0;
    const double ds = bi > 0.0 ? tau_s / bi : kInf;
    const double da = ai > 0.0 ? r.tau_a / ai : kInf;
    if (da <= ell || ds <= ell) r.race = std::fabs(da - ds);
    if (da <= ds && da <= ell) {
      r.S += da;
      r.tau_a = 0.0;
      r.absorb = true;
      return r;
    }
    if (ds <= ell) {
      r.S += ds;
      r.tau_a = std::max(0.0, r.tau_a - ai * ds);
      return r;
    }
    r.S += ell;
    tau_s = std::max(0.0, tau_s - bi * ell);
    r.tau_a = std::max(0.0, r.tau_a - ai * ell);
    zc = (w < 0.0) ? ice.zb(i + 1) : ice.zb(i);
    r.layer += (w < 0.0) ? 1 : -1;
    r.crossings += 1;
  }
}

// Distance along d from p to where the photon leaves the world cylinder;
// 0 when p is already outside.
double world_exit(const World& W, const double p[3], const double d[3]) {
  const double c = p[0] * p[0] + p[1] * p[1] - W.R * W.R;
  if (c > 0.0 || p[2] < W.zlo || p[2] > W.zhi) return 0.0;
  double tz = kInf;
  if (d[2] > 0.0) tz = (W.zhi - p[2]) / d[2];
  else if (d[2] < 0.0) tz = (W.zlo - p[2]) / d[2];
  double tr = kInf;
  const double a = d[0] * d[0] + d[1] * d[1];
  if (a > 0.0) {
    const double b = p[0] * d[0] + p[1] * d[1];
    const double sq = std::sqrt(std::max(0.0, b * b - a * c));
    tr = (b > 0.0) ? (-c) / (b + sq) : (sq - b) / a;
  }
  return std::min(tz, tr);
}

// Sec. 2: propagation repeats "until the photon intersects a detector".  A DOM
// is a sphere of radius r about its centre c.  With m = p - c, beta = m.d,
// gamma = |m|^2 - r^2: a start inside the sphere is a hit at t = 0; otherwise
// the entry point t = -beta - sqrt(beta^2 - gamma) must lie in [0, S].
bool sphere_hit(double px, double py, double pz, const double d[3], double cx, double cy,
                double cz, double r, double S, double* t) {
  const double mx = px - cx, my = py - cy, mz = pz - cz;
  const double beta = mx * d[0] + my * d[1] + mz * d[2];
  const double gamma = mx * mx + my * my + mz * mz - r * r;
  if (gamma <= 0.0) {
    *t = 0.0;
    return true;
  }
  const double disc = beta * beta - gamma;
  if (disc < 0.0) return false;
  const double tt = -beta - std::sqrt(disc);
  if (tt < 0.0 || tt > S) return false;
  *t = tt;
  return true;
}

// First DOM met on the segment [p, p + S d]: smallest t, ties to the lowest
// DOM index.  Returns the DOM index or -1.
int first_hit(const Geom& G, bool brute, const double p[3], const double d[3], double S,
              double* t_out) {
  int best = -1;
  double bt = kInf;
  auto consider = [&](int k) {
    double t;
    if (sphere_hit(p[0], p[1], p[2], d, G.x[k], G.y[k], G.z[k], G.r, S, &t)) {
      if (t < bt || (t == bt && k < best)) {
        bt = t;
        best = k;
      }
    }
  };
  if (brute) {
    for (int k = 0; k < G.n; ++k) consider(k);
  } else {
    const double eps = 1e-9 * (1.0 + std::fabs(S));
    double lo[3], hi[3];
    for (int q = 0; q < 3; ++q) {
      const double e = p[q] + S * d[q];
      lo[q] = std::min(p[q], e) - eps;
      hi[q] = std::max(p[q], e) + eps;
    }
    for (const Cluster& c : G.clusters) {
      if (c.hi[0] < lo[0] || c.lo[0] > hi[0] || c.hi[1] < lo[1] || c.lo[1] > hi[1] ||
          c.hi[2] < lo[2] || c.lo[2] > hi[2])
        continue;
      for (int k : c.doms) {
        if (G.x[k] + G.r < lo[0] || G.x[k] - G.r > hi[0] || G.y[k] + G.r < lo[1] ||
            G.y[k] - G.r > hi[1] || G.z[k] + G.r < lo[2] || G.z[k] - G.r > hi[2])
          continue;
        consider(k);
      }
    }
  }
  *t_out = bt;
  return best;
}

// Henyey-Greenstein: cosine of the scattering angle from one uniform u by
// inverting the HG cumulative distribution; g = 0 is isotropic.
double hg_mu(double g, double u) {
  if (g == 0.0) return 2.0 * u - 1.0;
  const double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
  const double mu = (1.0 + g * g - t * t) / (2.0 * g);
  return std::max(-1.0, std::min(1.0, mu));
}

// New direction at polar cosine mu and azimuth phi about d (MCML formulas);
// near the poles (|d_z| > 0.99999) the frame is the lab frame.  The result is
// renormalised.
void rotate(const double d[3], double mu, double phi, double out[3]) {
  const double st = std::sqrt(std::max(0.0, 1.0 - mu * mu));
  const double cp = std::cos(phi), sp = std::sin(phi);
  if (std::fabs(d[2]) > 0.99999) {
    out[0] = st * cp;
    out[1] = st * sp;
    out[2] = (d[2] >= 0.0) ? mu : -mu;
  } else {
    const double tmp = std::sqrt(1.0 - d[2] * d[2]);
    out[0] = st * (d[0] * d[2] * cp - d[1] * sp) / tmp + d[0] * mu;
    out[1] = st * (d[1] * d[2] * cp + d[0] * sp) / tmp + d[1] * mu;
    out[2] = -st * cp * tmp + d[2] * mu;
  }
  const double n = std::sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
  out[0] /= n;
  out[1] /= n;
  out[2] /= n;
}

struct Source {
  double p[3], d[3], len;
  uint32_t type;
};

Source read_source(const float* f, const uint32_t* type, int64_t s) {
  Source S;
  for (int q = 0; q < 3; ++q) {
    S.p[q] = f[7 * s + q];
    S.d[q] = f[7 * s + 3 + q];
  }
  const double n = std::sqrt(S.d[0] * S.d[0] + S.d[1] * S.d[1] + S.d[2] * S.d[2]);
  if (n > 0.0)
    for (int q = 0; q < 3; ++q) S.d[q] /= n;
  S.len = f[7 * s + 6];
  S.type = type[s];
  return S;
}

const double kCherenkovCos = std::cos(41.0 * kPi / 180.0);

enum { OUT_ABSORBED = -1, OUT_ESCAPED = -2, OUT_TRUNCATED = -3 };

struct PhotonStats {
  int64_t steps = 0, scatters = 0, crossings = 0;
  double path = 0.0, cos_sum = 0.0;
};

// One photon from birth to its end.  Returns the DOM index it hits, or
// OUT_ABSORBED / OUT_ESCAPED / OUT_TRUNCATED.  trace (optional) receives the
// birth point and direction and the first n_trace scatter points.
// Distance (m) from the decision boundaries of the DOM test on [p, p + S d]:
// for every sphere, | closest approach of the segment to its centre - r |.
double dom_margin(const Geom& G, const double p[3], const double d[3], double S) {
  double m = kInf;
  for (int k = 0; k < G.n; ++k) {
    const double v[3] = {G.x[k] - p[0], G.y[k] - p[1], G.z[k] - p[2]};
    double t = v[0] * d[0] + v[1] * d[1] + v[2] * d[2];
    t = std::max(0.0, std::min(S, t));
    const double q[3] = {p[0] + t * d[0] - G.x[k], p[1] + t * d[1] - G.y[k],
                         p[2] + t * d[2] - G.z[k]};
    m = std::min(m, std::fabs(std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - G.r));
  }
  return m;
}

int simulate_photon(const Model& M, uint32_t event_lo, uint64_t pid, const Source& src,
                    PhotonStats* st, double* birth6, double* trace, int n_trace,
                    double* margin = nullptr, double* emit_offset = nullptr,
                    double* hit_dir = nullptr) {
  const uint32_t key[2] = {(uint32_t)M.seed, (uint32_t)(M.seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), 0u, event_lo};
  uint32_t x[4];
  // Birth (block 0): point along the emitting segment, direction, and the
  // absorption optical depth the photon carries.
  philox4x32_10(ctr, key, x);
  double pos[3], dir[3];
  const double t0 = u01(x[0]) * src.len;
  if (emit_offset) *emit_offset = t0;
  for (int q = 0; q < 3; ++q) pos[q] = src.p[q] + t0 * src.d[q];
  if (src.type == 1) {
    rotate(src.d, kCherenkovCos, 2.0 * kPi * u01(x[2]), dir);
  } else {
    const double mu = 2.0 * u01(x[1]) - 1.0;
    const double phi = 2.0 * kPi * u01(x[2]);
    const double s = std::sqrt(std::max(0.0, 1.0 - mu * mu));
    dir[0] = s * std::cos(phi);
    dir[1] = s * std::sin(phi);
    dir[2] = mu;
  }
  double tau_a = -std::log(u01(x[3]));
  if (birth6) {
    for (int q = 0; q < 3; ++q) {
      birth6[q] = pos[q];
      birth6[3 + q] = dir[q];
    }
  }
  int layer = layer_at(M.ice, pos[2], dir[2]);
  for (uint32_t n = 1; n <= M.max_steps; ++n) {
    ctr[2] = n;
    philox4x32_10(ctr, key, x);
    st->steps += 1;
    const double tau_s = -std::log(u01(x[0]));
    const WalkResult w = walk(M.ice, pos[2], dir[2], layer, tau_s, tau_a);
    st->crossings += w.crossings;
    const double tw = world_exit(M.world, pos, dir);
    const double S_test = std::min(w.S, tw);
    double th = kInf;
    const int k = first_hit(M.geom, M.brute, pos, dir, S_test, &th);
    if (margin && (int)n <= n_trace) {
      // diagnostic: how close this step's discrete decisions came to flipping
      double mg = std::min(w.race, dom_margin(M.geom, pos, dir, S_test));
      if (std::isfinite(tw) && std::isfinite(w.S)) mg = std::min(mg, std::fabs(tw - w.S));
      if (std::fabs(std::fabs(dir[2]) - 0.99999) < 1e-6) mg = 0.0;  // rotation frame choice
      margin[n - 1] = mg;
    }
    if (k >= 0 && th < tw) {
      st->path += th;
      if (hit_dir)
        for (int q = 0; q < 3; ++q) hit_dir[q] = dir[q];
      return k;
    }
    if (tw <= w.S) {
      st->path += tw;
      return OUT_ESCAPED;
    }
    st->path += w.S;
    if (w.absorb) return OUT_ABSORBED;
    // Scatter (Sec. 2: a new angle from the physics of scattering).
    for (int q = 0; q < 3; ++q) pos[q] += w.S * dir[q];
    const double mu = hg_mu(M.ice.g, u01(x[1]));
    const double phi = 2.0 * kPi * u01(x[2]);
    double nd[3];
    rotate(dir, mu, phi, nd);
    st->cos_sum += dir[0] * nd[0] + dir[1] * nd[1] + dir[2] * nd[2];
    st->scatters += 1;
    for (int q = 0; q < 3; ++q) dir[q] = nd[q];
    layer = w.layer;
    tau_a = w.tau_a;
    if (trace && (int)n <= n_trace)
      for (int q = 0; q < 3; ++q) trace[3 * (n - 1) + q] = pos[q];
  }
  return OUT_TRUNCATED;
}

// Exclusive prefix sum of the sources' photon counts: photon j of source s in
// an event has photon id offset[s] + j (photon ids are per event).
std::vector<uint64_t> photon_offsets(const uint64_t* n_ph, int64_t b, int64_t e) {
  std::vector<uint64_t> off(e - b + 1, 0);
  for (int64_t s = b; s < e; ++s) off[s - b + 1] = off[s - b] + n_ph[s];
  return off;
}

int resolve_threads(int n) {
  if (n > 0) return n;
  const unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

}  // namespace

extern "C" {

// ---- primitives (exported for the pins) -----------------------------------

void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

void orc_u01(const uint32_t* x, double* u, int64_t n) {
  for (int64_t i = 0; i < n; ++i) u[i] = u01(x[i]);
}

void orc_hg(double g, const double* u, double* mu, int64_t n) {
  for (int64_t i = 0; i < n; ++i) mu[i] = hg_mu(g, u[i]);
}

void orc_rotate(const double* d, const double* mu, const double* phi, double* out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) rotate(d + 3 * i, mu[i], phi[i], out + 3 * i);
}

void orc_layer_at(const orc_params* P, const double* z, const double* w, int32_t* layer,
                  int64_t n) {
  Model M;
  build_model(P, &M);
  for (int64_t i = 0; i < n; ++i) layer[i] = layer_at(M.ice, z[i], w[i]);
}

// Walk from height z with vertical direction w (starting layer by layer_at).
void orc_walk(const orc_params* P, const double* z, const double* w, const double* tau_s,
              const double* tau_a, double* S, int32_t* absorb, int32_t* layer_end,
              double* tau_a_end, int64_t n) {
  Model M;
  build_model(P, &M);
  for (int64_t i = 0; i < n; ++i) {
    const int l0 = layer_at(M.ice, z[i], w[i]);
    const WalkResult r = walk(M.ice, z[i], w[i], l0, tau_s[i], tau_a[i]);
    S[i] = r.S;
    absorb[i] = r.absorb ? 1 : 0;
    layer_end[i] = r.layer;
    tau_a_end[i] = r.tau_a;
  }
}

void orc_world_exit(const orc_params* P, const double* p, const double* d, double* t,
                    int64_t n) {
  Model M;
  build_model(P, &M);
  for (int64_t i = 0; i < n; ++i) t[i] = world_exit(M.world, p + 3 * i, d + 3 * i);
}

void orc_world(const orc_params* P, double* out3) {
  Model M;
  build_model(P, &M);
  out3[0] = M.world.R;
  out3[1] = M.world.zlo;
  out3[2] = M.world.zhi;
}

void orc_first_hit(const orc_params* P, const double* p, const double* d, const double* S,
                   int32_t* dom, double* t, int64_t n) {
  Model M;
  build_model(P, &M);
  for (int64_t i = 0; i < n; ++i) dom[i] = first_hit(M.geom, M.brute, p + 3 * i, d + 3 * i, S[i], t + i);
}

// ---- whole propagation -----------------------------------------------------

// Propagates every photon of every event.  Event e owns sources
// [src_begin[e], src_begin[e+1]).  Outputs (all zeroed here):
//   hits   [n_events][n_dom]  photons that ended on each DOM
//   counts [n_events][4]      absorbed (incl. truncated), escaped, truncated, steps
//   stats  [4]                scatters, crossings, path length sum, cos sum
// Returns 0, or -1 on bad arguments.
int orc_propagate(const orc_params* P, int32_t n_events, const uint64_t* event_ids,
                  const int64_t* src_begin, const float* src_f, const uint32_t* src_type,
                  const uint64_t* src_n, uint64_t* hits, uint64_t* counts, double* stats) {
  if (!P || n_events < 0 || P->n_layers < 1) return -1;
  Model M;
  build_model(P, &M);
  const int n_dom = M.geom.n;
  std::memset(hits, 0, sizeof(uint64_t) * (size_t)n_events * (size_t)n_dom);
  std::memset(counts, 0, sizeof(uint64_t) * (size_t)n_events * 4);
  for (int q = 0; q < 4; ++q) stats[q] = 0.0;

  // Work items: (event, source, photon range) of at most 4096 photons.
  struct Item {
    int32_t e;
    int64_t s;
    uint64_t j0, j1, id0;
  };
  std::vector<Item> items;
  for (int32_t e = 0; e < n_events; ++e) {
    const std::vector<uint64_t> off = photon_offsets(src_n, src_begin[e], src_begin[e + 1]);
    for (int64_t s = src_begin[e]; s < src_begin[e + 1]; ++s) {
      const uint64_t n = src_n[s];
      for (uint64_t j = 0; j < n; j += 4096)
        items.push_back({e, s, j, std::min(n, j + 4096), off[s - src_begin[e]]});
    }
  }
  std::vector<std::atomic<uint64_t>> hit_acc((size_t)n_events * n_dom);
  for (auto& h : hit_acc) h.store(0);
  std::vector<std::atomic<uint64_t>> cnt_acc((size_t)n_events * 4);
  for (auto& c : cnt_acc) c.store(0);
  std::atomic<size_t> next(0);
  const int T = resolve_threads(P->n_threads);
  std::vector<PhotonStats> tstats(T);
  auto worker = [&](int tid) {
    PhotonStats& ps = tstats[tid];
    for (;;) {
      const size_t it = next.fetch_add(1);
      if (it >= items.size()) break;
      const Item& I = items[it];
      const Source src = read_source(src_f, src_type, I.s);
      const uint32_t ev = (uint32_t)event_ids[I.e];
      uint64_t c_abs = 0, c_esc = 0, c_trunc = 0;
      const int64_t steps0 = ps.steps;
      for (uint64_t j = I.j0; j < I.j1; ++j) {
        const int out = simulate_photon(M, ev, I.id0 + j, src, &ps, nullptr, nullptr, 0);
        if (out >= 0) hit_acc[(size_t)I.e * n_dom + out].fetch_add(1, std::memory_order_relaxed);
        else if (out == OUT_ESCAPED) ++c_esc;
        else if (out == OUT_ABSORBED) ++c_abs;
        else {
          ++c_abs;
          ++c_trunc;
        }
      }
      cnt_acc[(size_t)I.e * 4 + 0].fetch_add(c_abs);
      cnt_acc[(size_t)I.e * 4 + 1].fetch_add(c_esc);
      cnt_acc[(size_t)I.e * 4 + 2].fetch_add(c_trunc);
      cnt_acc[(size_t)I.e * 4 + 3].fetch_add((uint64_t)(ps.steps - steps0));
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) pool.emplace_back(worker, t);
  for (auto& th : pool) th.join();
  for (size_t i = 0; i < hit_acc.size(); ++i) hits[i] = hit_acc[i].load();
  for (size_t i = 0; i < cnt_acc.size(); ++i) counts[i] = cnt_acc[i].load();
  for (const PhotonStats& ps : tstats) {
    stats[0] += (double)ps.scatters;
    stats[1] += (double)ps.crossings;
    stats[2] += ps.path;
    stats[3] += ps.cos_sum;
  }
  return 0;
}

// Compact hit records of one event (paper Sec. 4: the producing particle's
// ID, the hit time and the weight), one per photon that ends on a DOM, in
// photon order: DOM, source index, time = (emission offset along the segment
// + group_index x path length) / c in ns, the weight and the photon's id.  The
// weight is the probability that the hit makes a photoelectron (paper Sec. 2
// names it a function of the photon's position, direction, time and
// wavelength and gives none): here the caller's polynomial accept[0..n_accept)
// in eta, the z component of the photon's direction at the DOM, clamped to
// [0, 1]; 1 when n_accept = 0.  At most max_records are written (weight may
// be NULL); *n_records receives the number of hits.
int orc_hit_records(const orc_params* P, uint64_t event_id, int64_t n_src, const float* src_f,
                    const uint32_t* src_type, const uint64_t* src_n, double group_index,
                    int32_t n_accept, const double* accept, int64_t max_records, uint32_t* dom,
                    uint32_t* source, double* time_ns, double* weight, uint64_t* photon,
                    int64_t* n_records) {
  if (!P || n_src < 0 || max_records < 0 || !(group_index >= 1.0) || n_accept < 0 ||
      (n_accept > 0 && !accept))
    return -1;
  Model M;
  build_model(P, &M);
  const double c = 0.299792458;  // m / ns
  const std::vector<uint64_t> off = photon_offsets(src_n, 0, n_src);
  int64_t n = 0;
  PhotonStats ps;
  for (int64_t s = 0; s < n_src; ++s) {
    const Source src = read_source(src_f, src_type, s);
    for (uint64_t j = 0; j < src_n[s]; ++j) {
      const double path0 = ps.path;
      double t_emit = 0.0, hd[3] = {0.0, 0.0, 0.0};
      const uint64_t pid = off[s] + j;
      const int out = simulate_photon(M, (uint32_t)event_id, pid, src, &ps, nullptr, nullptr, 0,
                                      nullptr, &t_emit, hd);
      if (out < 0) continue;
      if (n < max_records) {
        dom[n] = (uint32_t)out;
        source[n] = (uint32_t)s;
        time_ns[n] = (t_emit + group_index * (ps.path - path0)) / c;
        photon[n] = pid;
        // weight: the caller's acceptance polynomial in the z component of the
        // photon's direction at the DOM, clamped to [0, 1]; 1 without one
        double w = 1.0;
        if (n_accept > 0) {
          w = 0.0;
          double eta_i = 1.0;
          for (int32_t i = 0; i < n_accept; ++i) {
            w += accept[i] * eta_i;
            eta_i *= hd[2];
          }
          w = std::min(1.0, std::max(0.0, w));
        }
        if (weight) weight[n] = w;
      }
      ++n;
    }
  }
  *n_records = n;
  return 0;
}

// Follows chosen photons of one event.  photon_ids are per-event ids.
// Outputs: outcome[n] (DOM index, -1 absorbed, -2 escaped, -3 truncated),
// n_steps[n], birth[n][6] (point, direction), trace[n][n_trace][3] scatter
// points (NaN past the photon's last scatter).
// margins[n][n_trace] (optional): for each of the first n_trace steps, the
// distance in metres of that step's decisions from a flip (scatter/absorb race,
// sphere grazing, world exit); NaN past the photon's end.
int orc_trace(const orc_params* P, uint64_t event_id, int64_t n_src, const float* src_f,
              const uint32_t* src_type, const uint64_t* src_n, const uint64_t* photon_ids,
              int64_t n, int32_t n_trace, int32_t* outcome, int64_t* n_steps, double* birth,
              double* trace, double* margins) {
  if (!P || n < 0 || n_trace < 0) return -1;
  Model M;
  build_model(P, &M);
  const std::vector<uint64_t> off = photon_offsets(src_n, 0, n_src);
  const int T = resolve_threads(P->n_threads);
  std::atomic<int64_t> next(0);
  int bad = 0;
  auto worker = [&]() {
    for (;;) {
      const int64_t i = next.fetch_add(1);
      if (i >= n) break;
      const uint64_t pid = photon_ids[i];
      // source containing this photon id: last s with off[s] <= pid
      const int64_t s = (int64_t)(std::upper_bound(off.begin(), off.end() - 1, pid) - off.begin()) - 1;
      double* tr = trace + (size_t)i * n_trace * 3;
      for (int q = 0; q < 3 * n_trace; ++q) tr[q] = std::nan("");
      double* mg = margins ? margins + (size_t)i * n_trace : nullptr;
      for (int q = 0; mg && q < n_trace; ++q) mg[q] = std::nan("");
      if (s < 0 || pid >= off[n_src]) {
        outcome[i] = -4;
        n_steps[i] = 0;
        bad = 1;
        continue;
      }
      PhotonStats ps;
      const Source src = read_source(src_f, src_type, s);
      outcome[i] = simulate_photon(M, (uint32_t)event_id, pid, src, &ps, birth + 6 * i, tr, n_trace,
                                   mg);
      n_steps[i] = ps.steps;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  return bad ? -1 : 0;
}

}  // extern "C"
