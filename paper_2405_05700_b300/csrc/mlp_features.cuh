// Surrogate pair features, shared by the feature kernel and the fused
// inference kernel.
#pragma once

#include <cuda_bf16.h>

#include "mlp_internal.h"

namespace mlp {

// Surrogate inputs of a (source, DOM) pair.  The ten named inputs: source
// position (/500 m), direction polar and azimuth angles (/pi), DOM position
// relative to the source (/100 m), effective scattering and absorption at the
// source's layer (x10, x50); six derived: the unit direction, the distance
// (/100 m), the cosine between the direction and the line to the DOM, and
// ln(1 + distance / 1 m) / 5.  The source point is the segment's midpoint.
__device__ __forceinline__ void pair_features(const FeatGeom& fg, const pp_source& s, float4 c,
                                              __nv_bfloat16* out) {
  float dx = s.dx, dy = s.dy, dz = s.dz;
  const float nn = sqrtf(dx * dx + dy * dy + dz * dz);
  if (nn > 0.0f) {
    dx /= nn;
    dy /= nn;
    dz /= nn;
  }
  const float h = 0.5f * s.length;
  const float px = s.x + h * dx, py = s.y + h * dy, pz = s.z + h * dz;
  const float ex = c.x - px, ey = c.y - py, ez = c.z - pz;
  const float r = sqrtf(ex * ex + ey * ey + ez * ez);
  int li = (int)floorf((fg.z_top - pz) / fg.dz);
  li = li < 0 ? 0 : (li > fg.L - 1 ? fg.L - 1 : li);
  const float4 L = fg.layer[li];
  float f[kIn];
  f[0] = px / 500.0f;
  f[1] = py / 500.0f;
  f[2] = pz / 500.0f;
  f[3] = acosf(fminf(1.0f, fmaxf(-1.0f, dz))) / 3.14159265358979f;
  f[4] = atan2f(dy, dx) / 3.14159265358979f;
  f[5] = ex / 100.0f;
  f[6] = ey / 100.0f;
  f[7] = ez / 100.0f;
  f[8] = L.x * fg.be_over_b * 10.0f;
  f[9] = L.y * 50.0f;
  f[10] = dx;
  f[11] = dy;
  f[12] = dz;
  f[13] = r / 100.0f;
  f[14] = (dx * ex + dy * ey + dz * ez) / fmaxf(r, 1e-3f);
  f[15] = log1pf(r) / 5.0f;
#pragma unroll
  for (int i = 0; i < kIn; ++i) out[i] = __float2bfloat16_rn(f[i]);
}

}  // namespace mlp
