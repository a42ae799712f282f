// Surrogate pair features, shared by the feature kernel and the fused
// inference kernel.
#pragma once

#include <cuda_bf16.h>

#include "mlp_internal.h"

namespace mlp {

// Continuous layer coordinate of height z and its (clamped) layer index.
__device__ __forceinline__ int feat_layer(const FeatGeom& fg, float u) {
  int i = (int)floorf(u);
  return i < 0 ? 0 : (i > fg.L - 1 ? fg.L - 1 : i);
}

// Surrogate inputs of a (source, DOM) pair.  p = segment midpoint, d = unit
// direction, e = DOM - p, r = |e|, c = d.e / max(r, 1 mm), delta = acos(c) -
// theta_c (angle from the Cherenkov cone), rho = r sin(delta) (distance from
// the cone's surface), u = (z_top - z) / dz (layer coordinate):
//   0-2 p / 500 m, 3 polar angle / pi, 4 azimuth / pi, 5-7 e / 100 m,
//   8 b_e(p) x 10, 9 a(p) x 50, 10-12 d, 13 r / 100 m, 14 c,
//   15 ln(1 + r / 1 m) / 5, 16 2 delta, 17 rho / 10 m, 18 exp(-|rho| / 2 m),
//   19 b_e(DOM) x 10, 20 a(DOM) x 50, 21-22 the means of b_e and a along the
//   line (the integral of the layer profile, edge layers extended) x 10, x 50,
//   23 r x mean a, 24 r x mean b_e / 10, 25-27 exp(-r / 10, 30, 100 m),
//   28 DOM z / 500 m, 29 e_z / max(r, 1 mm), 30 1 / (1 + r / 5 m),
//   31 r sin(acos c) / 100 m.
// What the features take from the source alone (shared by all its pairs).
struct __align__(16) SrcPrep {
  float px, py, pz;  // segment midpoint
  float dx, dy, dz;  // unit direction
  float us;          // layer coordinate of the midpoint
  float bs, as;      // effective scattering and absorption there
  float f3, f4;      // polar angle / pi, azimuth / pi
  int is;            // layer index of the midpoint
};
static_assert(sizeof(SrcPrep) == 48, "three 16-byte loads");

__device__ __forceinline__ SrcPrep source_prep(const FeatGeom& fg, const pp_source& s) {
  SrcPrep P;
  float dx = s.dx, dy = s.dy, dz = s.dz;
  const float nn = sqrtf(dx * dx + dy * dy + dz * dz);
  if (nn > 0.0f) {
    dx /= nn;
    dy /= nn;
    dz /= nn;
  }
  const float h = 0.5f * s.length;
  P.px = s.x + h * dx;
  P.py = s.y + h * dy;
  P.pz = s.z + h * dz;
  P.dx = dx;
  P.dy = dy;
  P.dz = dz;
  P.us = (fg.z_top - P.pz) / fg.dz;
  P.is = feat_layer(fg, P.us);
  const float4 Ls = fg.layer[P.is];
  P.bs = Ls.x * fg.be_over_b;
  P.as = Ls.y;
  const float inv_pi = 0.318309886183791f;
  P.f3 = acosf(fminf(1.0f, fmaxf(-1.0f, dz))) * inv_pi;
  P.f4 = atan2f(dy, dx) * inv_pi;
  return P;
}

// Features kPart * 16 .. + 15 of the pair from its source's part and the DOM
// centre c (two halves, so that two threads can share a row's work).
template <int kPart>
__device__ __forceinline__ void pair_features_half(const FeatGeom& fg, const SrcPrep& P, float4 c,
                                                   __nv_bfloat16* out) {
  const float px = P.px, py = P.py, pz = P.pz, dx = P.dx, dy = P.dy, dz = P.dz;
  const float ex = c.x - px, ey = c.y - py, ez = c.z - pz;
  const float r = sqrtf(ex * ex + ey * ey + ez * ez);
  const float rr = fmaxf(r, 1e-3f);
  const float cs = __fdividef(dx * ex + dy * ey + dz * ez, rr);
  // Every input is rounded to BF16 (8 significant bits), so the scalings use
  // constant reciprocals and the exponentials, logarithm and sine the SFU
  // forms (errors of order 1e-6 relative, far below one BF16 step).
  float f[kIn / 2];
  if (kPart == 0) {
    f[0] = px * (1.0f / 500.0f);
    f[1] = py * (1.0f / 500.0f);
    f[2] = pz * (1.0f / 500.0f);
    f[3] = P.f3;
    f[4] = P.f4;
    f[5] = ex * (1.0f / 100.0f);
    f[6] = ey * (1.0f / 100.0f);
    f[7] = ez * (1.0f / 100.0f);
    f[8] = P.bs * 10.0f;
    f[9] = P.as * 50.0f;
    f[10] = dx;
    f[11] = dy;
    f[12] = dz;
    f[13] = r * (1.0f / 100.0f);
    f[14] = cs;
    f[15] = __logf(1.0f + r) * (1.0f / 5.0f);
  } else {
    const float th = acosf(fminf(1.0f, fmaxf(-1.0f, cs)));
    const float delta = th - fg.theta_c;
    const float rho = r * __sinf(delta);
    // point values and line means of the layer profile
    const float us = P.us, ud = (fg.z_top - c.z) / fg.dz;
    const int is = P.is, id = feat_layer(fg, ud);
    const float4 Ld = fg.layer[id];
    const float bs = P.bs, as = P.as;
    const float bd = Ld.x * fg.be_over_b, ad = Ld.y;
    float mb = bs, ma = as;
    if (is != id) {
      const float2 cs_ = fg.cum[is], cd = fg.cum[id];
      const float fs = us - (float)is, fd = ud - (float)id;
      const float du = ud - us;
      mb = ((cd.x - cs_.x) + fd * bd - fs * bs) / du;
      ma = ((cd.y - cs_.y) + fd * ad - fs * as) / du;
    }
    f[0] = 2.0f * delta;
    f[1] = rho * (1.0f / 10.0f);
    f[2] = __expf(-0.5f * fabsf(rho));
    f[3] = bd * 10.0f;
    f[4] = ad * 50.0f;
    f[5] = mb * 10.0f;
    f[6] = ma * 50.0f;
    f[7] = r * ma;
    f[8] = r * mb * (1.0f / 10.0f);
    f[9] = __expf(r * (-1.0f / 10.0f));
    f[10] = __expf(r * (-1.0f / 30.0f));
    f[11] = __expf(r * (-1.0f / 100.0f));
    f[12] = c.z * (1.0f / 500.0f);
    f[13] = __fdividef(ez, rr);
    f[14] = __fdividef(1.0f, fmaf(r, 1.0f / 5.0f, 1.0f));
    f[15] = r * sqrtf(fmaxf(0.0f, 1.0f - cs * cs)) * (1.0f / 100.0f);
  }
#pragma unroll
  for (int i = 0; i < kIn / 2; ++i) out[i] = __float2bfloat16_rn(f[i]);
}

// All 32 features of the pair.
__device__ __forceinline__ void pair_features(const FeatGeom& fg, const SrcPrep& P, float4 c,
                                              __nv_bfloat16* out) {
  pair_features_half<0>(fg, P, c, out);
  pair_features_half<1>(fg, P, c, out + kIn / 2);
}

__device__ __forceinline__ void pair_features(const FeatGeom& fg, const pp_source& s, float4 c,
                                              __nv_bfloat16* out) {
  pair_features(fg, source_prep(fg, s), c, out);
}

}  // namespace mlp
