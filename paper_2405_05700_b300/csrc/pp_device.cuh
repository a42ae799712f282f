// Device code of one photon's life: birth, steps through layered ice, DOM hit
// test, world escape, scattering.  Everything here runs in FP32 (random words
// in uint32) and is shared by every kernel that moves photons, so that the
// plain, persistent and trace kernels follow identical trajectories.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pp_internal.h"

namespace ppk {

#define PP_INF (__int_as_float(0x7f800000))

// ---------------------------------------------------------------- Philox --
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// on counter words 0 and 2, the high halves xor-ed into the other words with
// the round's key, the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t kx, uint32_t ky) {
  // one 32 x 32 -> 64-bit product each (high and low halves together)
  const unsigned long long p0 = 0xD2511F53ull * c.x;
  const unsigned long long p1 = 0xCD9E8D57ull * c.z;
  return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ kx, (uint32_t)p1,
                    (uint32_t)(p0 >> 32) ^ c.w ^ ky, (uint32_t)p0);
}

// Any counter and key (the generator as such, for its check against the
// oracle).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    c = philox_round(c, k.x, k.y);
  }
  return c;
}

// The photons' streams: key (seed lo, seed hi) with its schedule from the
// run's parameters, counter (photon id lo, photon id hi, block, event id lo).
// Block 0 is the birth, block n >= 1 step n.
__device__ __forceinline__ uint4 photon_block(const RunDev& R, uint32_t pid_lo, uint32_t pid_hi,
                                              uint32_t block, uint32_t ev_lo) {
  uint4 c = make_uint4(pid_lo, pid_hi, block, ev_lo);
#pragma unroll
  for (int r = 0; r < 10; ++r) c = philox_round(c, R.key_x[r], R.key_y[r]);
  return c;
}

// Two FP32 operations in one instruction (PTX mul.rn.f32x2 / fma.rn.f32x2,
// sm_100 and later), each lane-half rounded to nearest exactly as FMUL / FFMA
// is: the pairs below give the results of the scalar code, in half the
// instructions, on a kernel bound by instruction issue.
__device__ __forceinline__ unsigned long long pack_f2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}

__device__ __forceinline__ float2 unpack_f2(unsigned long long r) {
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(r));
  return d;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(pack_f2(a.x, a.y)), "l"(pack_f2(b.x, b.y)), "l"(pack_f2(c.x, c.y)));
  return unpack_f2(d);
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pack_f2(a.x, a.y)), "l"(pack_f2(b.x, b.y)));
  return unpack_f2(d);
}

// uint32 -> (0, 1): top 24 bits with the lowest forced to 1, times 2^-24
// (exact in FP32).  With j = x >> 9 that is (2j + 1) 2^-24, formed without an
// int-to-float conversion as (1 + j 2^-23) - (1 - 2^-24): both operands and
// the difference are exact in FP32, so the subtraction is exact.
__device__ __forceinline__ float u01f(uint32_t x) {
  return __uint_as_float(0x3F800000u | (x >> 9)) - __uint_as_float(0x3F7FFFFFu);
}

// Hot-path arithmetic: hardware approximations (PTX sqrt.approx / MUFU
// instructions behind the CUDA intrinsics), accurate to a few ulp -- far
// inside the 1e-4 position tolerance against the FP64 oracle.
__device__ __forceinline__ float fast_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The other special functions of the step, as the PTX .approx instructions
// with .ftz: every operand on the step is a normal number (directions,
// distances and optical depths), where flushing subnormals changes no result,
// and the .ftz forms need no subnormal handling -- and no branch -- around
// the hardware operation.  Same results, 4 % less time for the batched kernel.
__device__ __forceinline__ float fast_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float fast_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// -ln u for u in (0, 1): -log2(u) ln 2
__device__ __forceinline__ float neg_log(float u) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(u));
  return y * -0.693147180559945309f;
}

// (sin, cos) of 2 pi u for u in (0, 1): evaluated at pi (2u - 1), which lies
// in (-pi, pi) where the hardware sine/cosine are accurate, and negated
// (sin(x + pi) = -sin x, cos(x + pi) = -cos x).
__device__ __forceinline__ void sincos_2pi(float u, float& s, float& c) {
  const float xx = 3.14159265358979f * fmaf(2.0f, u, -1.0f);  // sin / cos.approx.ftz
  float sx, cx;
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(sx) : "f"(xx));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(cx) : "f"(xx));
  s = -sx;
  c = -cx;
}

// --------------------------------------------------------- shared tables --
struct Tables {
  const float4* layer;   // [L]
  const float4* str;     // [n_str]
  const int2* range;     // [n_str]
  const uint8_t* clear;  // [nx*ny]
};

__device__ __forceinline__ Tables stage_tables(unsigned char* smem, const IceDev& I,
                                               const GeomDev& G) {
  float4* lay = reinterpret_cast<float4*>(smem);
  float4* str = lay + I.L;
  int2* rng = reinterpret_cast<int2*>(str + G.n_str);
  uint8_t* clr = reinterpret_cast<uint8_t*>(rng + G.n_str);
  for (int i = threadIdx.x; i < I.L; i += blockDim.x) lay[i] = I.layer[i];
  for (int i = threadIdx.x; i < G.n_str; i += blockDim.x) {
    str[i] = G.str[i];
    rng[i] = G.str_range[i];
  }
  const int ncell = G.nx * G.ny;
  const int nvec = ncell >> 4;
  const uint4* csrc = reinterpret_cast<const uint4*>(G.clear);
  uint4* cdst = reinterpret_cast<uint4*>(clr);
  if ((reinterpret_cast<uintptr_t>(clr) & 15) == 0) {
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) cdst[i] = csrc[i];
    for (int i = (nvec << 4) + threadIdx.x; i < ncell; i += blockDim.x) clr[i] = G.clear[i];
  } else {
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) clr[i] = G.clear[i];
  }
  return Tables{lay, str, rng, clr};
}

// ------------------------------------------------------------ geometry --
// Layer of a point at height z moving with vertical component w (same rule as
// the ice description: a point on a boundary belongs to the layer it moves
// into; depths outside the table take the edge layer).
__device__ __forceinline__ int layer_at(const IceDev& I, float z, float w) {
  const float f = (I.z_top - z) / I.dz;
  if (!(f >= 0.0f)) return 0;
  if (f >= (float)I.L) return I.L - 1;
  const float fl = floorf(f);
  int i = (int)fl;
  if (w > 0.0f && f == fl) i -= 1;
  return max(0, min(I.L - 1, i));
}

// Paper Sec. 2: ice in layers of given scattering and absorption; the
// distance to the next scatter is a Monte Carlo draw.  The step consumes tau_s
// with the local scattering coefficient and the photon's remaining tau_a with
// the local absorption coefficient, crossing layer boundaries as it goes; it
// ends at the scatter point or the absorption point (tie: absorption).  On
// return tau_a holds what is left after a scatter; after an absorption its
// value is unspecified (the photon ends there).
//
// Layers are 10 m and steps ~2 m, so a step crosses at most one boundary in
// all but ~0.5 % of its crossings; but some lane of a warp crosses in ~90 %
// of the warp's steps, and a loop pass for those few lanes cost the whole
// warp.  So the current layer and the next one are evaluated together,
// without branches (the next as if the boundary were crossed; its value is
// discarded when it is not), and only a step that leaves the next layer as
// well continues in the loop.  Each quantity is formed by the same operations
// as in a layer-by-layer loop, so the results are those of the loop.
__device__ __forceinline__ float walk(const float4* __restrict__ lay, const IceDev& I, float z,
                                      float w, int& layer, float tau_s, float& tau_a,
                                      bool& absorb, uint32_t& crossings) {
  const float inv_w = fast_rcp(w);
  const bool down = w < 0.0f;
  // layer 1: the current one; the boundary ahead (none at the table's edge,
  // or when level)
  const float4 L1 = lay[layer];
  const int l2 = layer + (down ? 1 : -1);
  const bool has1 = down ? (layer < I.L - 1) : (w > 0.0f && layer > 0);
  const float4 L2 = lay[has1 ? l2 : layer];
  const float zb1 = fmaf(-(float)(down ? layer + 1 : layer), I.dz, I.z_top);
  const float ell1 = fmaxf(has1 ? (zb1 - z) * inv_w : PP_INF, 0.0f);
  const float2 q1 = mul2(make_float2(tau_s, tau_a), make_float2(L1.z, L1.w));
  // the layer table holds 1/b = inf (1/a = inf) for a layer without scattering
  // (absorption); tau * inf is inf, or NaN for tau = 0, which fminf maps to inf
  const float ds1 = fminf(q1.x, PP_INF);
  const float da1 = fminf(q1.y, PP_INF);
  const bool ab1 = da1 <= fminf(ds1, ell1);
  const bool cross1 = !ab1 && !(ds1 <= ell1);
  // layer 2: what remains of the depths after crossing layer 1
  const float2 r2 = fma2(make_float2(-L1.x, -L1.y), make_float2(ell1, ell1),
                         make_float2(tau_s, tau_a));
  const float ts2 = fmaxf(0.0f, r2.x);
  const float ta2 = fmaxf(0.0f, r2.y);
  const bool has2 = down ? (l2 < I.L - 1) : (w > 0.0f && l2 > 0);
  const float zb2 = fmaf(-(float)(down ? l2 + 1 : l2), I.dz, I.z_top);
  const float ell2 = fmaxf(has2 ? (zb2 - zb1) * inv_w : PP_INF, 0.0f);
  const float2 q2 = mul2(make_float2(ts2, ta2), make_float2(L2.z, L2.w));
  const float ds2 = fminf(q2.x, PP_INF);
  const float da2 = fminf(q2.y, PP_INF);
  const bool ab2 = da2 <= fminf(ds2, ell2);
  const bool cross2 = !ab2 && !(ds2 <= ell2);
  if (!(cross1 && cross2)) {
    absorb = cross1 ? ab2 : ab1;
    const float d1 = ab1 ? da1 : ds1;
    const float d2 = ab2 ? da2 : ds2;
    // tau_a after a scatter (an absorbed photon's tau_a is never read again)
    const float taf1 = fmaxf(0.0f, fmaf(-L1.y, ds1, tau_a));
    const float taf2 = fmaxf(0.0f, fmaf(-L2.y, ds2, ta2));
    tau_a = cross1 ? taf2 : taf1;
    crossings += cross1 ? 1u : 0u;
    layer = cross1 ? l2 : layer;
    return cross1 ? ell1 + d2 : d1;
  }
  // rare: beyond the second layer, one layer per pass.  (Written out again
  // rather than shared with the two layers above: that form compiled to a
  // 0.5 % slower kernel.)
  crossings += 2;
  float S = ell1 + ell2;
  tau_s = fmaxf(0.0f, fmaf(-L2.x, ell2, ts2));
  tau_a = fmaxf(0.0f, fmaf(-L2.y, ell2, ta2));
  float zc = zb2;
  layer = l2 + (down ? 1 : -1);
  for (;;) {
    const float4 L = lay[layer];
    const bool has = down ? (layer < I.L - 1) : (w > 0.0f && layer > 0);
    const float zb = fmaf(-(float)(down ? layer + 1 : layer), I.dz, I.z_top);
    float ell = has ? (zb - zc) * inv_w : PP_INF;
    ell = fmaxf(ell, 0.0f);
    const float ds = (L.x > 0.0f) ? tau_s * L.z : PP_INF;
    const float da = (L.y > 0.0f) ? tau_a * L.w : PP_INF;
    if (da <= ds && da <= ell) {
      absorb = true;
      tau_a = 0.0f;
      return S + da;
    }
    if (ds <= ell) {
      absorb = false;
      tau_a = fmaxf(0.0f, fmaf(-L.y, ds, tau_a));
      return S + ds;
    }
    S += ell;
    crossings += 1;
    tau_s = fmaxf(0.0f, fmaf(-L.x, ell, tau_s));
    tau_a = fmaxf(0.0f, fmaf(-L.y, ell, tau_a));
    zc = zb;  // the boundary crossed
    layer += down ? 1 : -1;
  }
}

// Distance to the exit of the world cylinder along d; 0 when already outside.
__device__ __forceinline__ float world_exit(const GeomDev& G, float px, float py, float pz,
                                            float dx, float dy, float dz) {
  const float c = fmaf(px, px, fmaf(py, py, -G.R2));
  if (c > 0.0f || pz < G.zlo || pz > G.zhi) return 0.0f;
  float tz = PP_INF;
  if (dz > 0.0f) tz = __fdividef(G.zhi - pz, dz);
  else if (dz < 0.0f) tz = __fdividef(G.zlo - pz, dz);
  float tr = PP_INF;
  const float a = fmaf(dx, dx, dy * dy);
  if (a > 0.0f) {
    const float b = fmaf(px, dx, py * dy);
    const float sq = fast_sqrt(fmaxf(0.0f, fmaf(b, b, -a * c)));
    tr = (b > 0.0f) ? __fdividef(-c, b + sq) : __fdividef(sq - b, a);
  }
  return fminf(tz, tr);
}

// Radius of a ball about p that lies inside the world cylinder (less a 1 cm
// margin for FP32 error); negative outside.
__device__ __forceinline__ float world_inner(const GeomDev& G, float px, float py, float pz) {
  const float rho = fast_sqrt(fmaf(px, px, py * py));
  return fminf(G.R - rho, fminf(pz - G.zlo, G.zhi - pz)) - 0.01f;
}

// Sphere of radius r about c met on [p, p + S d]: entry distance, 0 when the
// start is inside.  Uses r^2 - |m - (m.d) d|^2 for the discriminant (the
// same quantity as (m.d)^2 - |m|^2 + r^2, with less cancellation).
__device__ __forceinline__ bool sphere_hit(float4 c, float r2, float px, float py, float pz,
                                           float dx, float dy, float dz, float S, float& t) {
  const float mx = px - c.x, my = py - c.y, mz = pz - c.z;
  const float beta = fmaf(mx, dx, fmaf(my, dy, mz * dz));
  const float gamma = fmaf(mx, mx, fmaf(my, my, fmaf(mz, mz, -r2)));
  if (gamma <= 0.0f) {
    t = 0.0f;
    return true;
  }
  if (beta >= 0.0f) return false;
  const float hx = fmaf(-beta, dx, mx), hy = fmaf(-beta, dy, my), hz = fmaf(-beta, dz, mz);
  const float disc = r2 - fmaf(hx, hx, fmaf(hy, hy, hz * hz));
  if (disc < 0.0f) return false;
  const float tt = -beta - sqrtf(disc);
  if (tt < 0.0f || tt > S) return false;
  t = tt;
  return true;
}

__device__ __forceinline__ void consider_dom(const GeomDev& G, int k, float px, float py,
                                             float pz, float dx, float dy, float dz, float S,
                                             int& best, float& bt) {
  float t;
  if (sphere_hit(__ldg(G.dom + k), G.r2, px, py, pz, dx, dy, dz, S, t)) {
    if (t < bt || (t == bt && k < best)) {
      bt = t;
      best = k;
    }
  }
}

// Candidate DOMs of one string: the part of the segment inside the string's
// bounding cylinder gives a z window; the string's DOMs in that window (by
// binary search on their sorted z) get the exact sphere test.
__device__ __forceinline__ void test_string(const GeomDev& G, const Tables& T, int s, float px,
                                            float py, float pz, float dx, float dy, float dz,
                                            float S, float dxy2, int& best, float& bt) {
  const float4 st = T.str[s];
  const float ox = px - st.x, oy = py - st.y;
  float t0 = 0.0f, t1 = S;
  const float c2 = fmaf(ox, ox, fmaf(oy, oy, -st.z * st.z));
  if (dxy2 > 1e-12f) {
    const float b2 = fmaf(ox, dx, oy * dy);
    const float disc = fmaf(b2, b2, -dxy2 * c2);
    if (disc < 0.0f) return;
    const float sq = sqrtf(disc);
    const float inv = 1.0f / dxy2;
    t0 = fmaxf(0.0f, (-b2 - sq) * inv);
    t1 = fminf(S, (-b2 + sq) * inv);
    if (t0 > t1) return;
  } else if (c2 > 0.0f) {
    return;
  }
  const float za = fmaf(t0, dz, pz), zb = fmaf(t1, dz, pz);
  const float zl = fminf(za, zb) - G.zpad, zh = fmaxf(za, zb) + G.zpad;
  const int2 rg = T.range[s];
  int lo = rg.x, hi = rg.x + rg.y;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(G.sdom_z + mid) < zl) lo = mid + 1;
    else hi = mid;
  }
  const int end = rg.x + rg.y;
  for (int q = lo; q < end; ++q) {
    if (__ldg(G.sdom_z + q) > zh) break;
    consider_dom(G, __ldg(G.sdom_idx + q), px, py, pz, dx, dy, dz, S, best, bt);
  }
}

// First DOM met on [p, p + S d] (smallest t, ties to the lowest index).
// Fast path: a step shorter (horizontally) than its cell's clearance cannot
// reach any string.  Next, the clearance of the start point itself: strings
// missing from the cell's list lie more than `halo` beyond their cylinders'
// radius from every point of the cell, so the point's clearance is at least
// min(halo, distance to each listed string's cylinder), less a 1 cm margin
// for FP32 rounding; a step shorter than that cannot reach a string either.
// Otherwise the cell's string list (steps up to `halo` long) or every string
// is searched.
// clear_out (optional) receives the larger of the two clearances: no
// horizontal displacement shorter than it reaches a string.
// A detector without DOMs needs no special case: its grid has no strings,
// the full clearance everywhere and empty cell lists.
__device__ __forceinline__ int first_hit_grid(const GeomDev& G, const Tables& T, float px,
                                              float py, float pz, float dx, float dy, float dz,
                                              float S, float& t_out, uint32_t& slow,
                                              float* clear_out = nullptr) {
  t_out = PP_INF;
  const float dxy2 = fmaf(dx, dx, dy * dy);
  const float L2 = S * S * dxy2;  // squared horizontal length of the step
  const int ix = min(max(__float2int_rd((px - G.gx0) * G.inv_cell), 0), G.nx - 1);
  const int iy = min(max(__float2int_rd((py - G.gy0) * G.inv_cell), 0), G.ny - 1);
  const int cell = iy * G.nx + ix;
  float clr = (float)T.clear[cell] * G.clear_unit;
  if (L2 < clr * clr) {
    if (clear_out) *clear_out = clr;
    return -1;
  }
  const uint32_t b = __ldg(G.cell_off + cell), e = __ldg(G.cell_off + cell + 1);
  float pc = G.halo;
  for (uint32_t j = b; j < e; ++j) {
    const float4 st = T.str[__ldg(G.cell_list + j)];
    const float ox = px - st.x, oy = py - st.y;
    pc = fminf(pc, fast_sqrt(fmaf(ox, ox, oy * oy)) - st.z);
  }
  clr = fmaxf(clr, pc - 0.01f);
  if (clear_out) *clear_out = clr;
  if (L2 < clr * clr) return -1;
  slow += 1;
  const float Lxy = fast_sqrt(L2);
  int best = -1;
  float bt = PP_INF;
  if (Lxy <= G.halo) {
    for (uint32_t j = b; j < e; ++j)
      test_string(G, T, (int)__ldg(G.cell_list + j), px, py, pz, dx, dy, dz, S, dxy2, best, bt);
  } else {
    for (int s = 0; s < G.n_str; ++s)
      test_string(G, T, s, px, py, pz, dx, dy, dz, S, dxy2, best, bt);
  }
  t_out = bt;
  return best;
}

__device__ __forceinline__ int first_hit_brute(const GeomDev& G, float px, float py, float pz,
                                               float dx, float dy, float dz, float S,
                                               float& t_out) {
  int best = -1;
  float bt = PP_INF;
  for (int k = 0; k < G.n_dom; ++k) consider_dom(G, k, px, py, pz, dx, dy, dz, S, best, bt);
  t_out = bt;
  return best;
}

// ---------------------------------------------------------- scattering --
// Henyey-Greenstein scattering angle by inversion of its cumulative
// distribution: mu = (1 + g^2 - t^2) / (2g), t = (1 - g^2) / (1 - g + 2gu).
// Strong forward scattering puts mu within 1e-5 of 1 for a percent of the
// draws, where FP32 loses 1 - mu to rounding; so 1 - mu and 1 + mu come from
// the algebraically equal, cancellation-free forms
//   1 - mu = (1-g)(1-u)(t + 1 - g) / (1 - g + 2gu)
//   1 + mu = (1+g) u (1 + g + t) / (1 - g + 2gu)
// (1 - u is exact in FP32), and sin(theta) = sqrt((1 - mu)(1 + mu)).  The
// same forms cover g = 0 (isotropic): t = 1, 1 - mu = 2(1 - u), 1 + mu = 2u,
// so no branch is taken on g (a uniform branch on the step cost 1 % of the
// batched kernel's time).
__device__ __forceinline__ void hg_angle(const IceDev& I, float u, float& mu, float& st) {
  const float den = fmaf(I.c3, u, I.c2);        // 1 - g + 2gu
  const float inv = fast_rcp(den);
  const float t = I.c1 * inv;
  // (1 - mu, 1 + mu) = (c2 (1 - u) (t + c2) inv, (2 - c2) u ((2 - c2) + t) inv),
  // the products taken left to right
  const float2 p1 = mul2(make_float2(I.c2, 2.0f - I.c2), make_float2(1.0f - u, u));
  const float2 p2 = mul2(p1, make_float2(t + I.c2, (2.0f - I.c2) + t));
  const float2 p3 = mul2(p2, make_float2(inv, inv));
  const float omm = p3.x, opm = p3.y;
  // both forms are positive (1 - g, 1 - u, t, u and 1 - g + 2gu are), so mu
  // lies in [-1, 1] and (1 - mu)(1 + mu) >= 0 without clamps
  mu = (omm < opm) ? 1.0f - omm : opm - 1.0f;
  st = fast_sqrt(omm * opm);
}

// New direction at polar cosine mu (sine st), azimuth 2 pi u_phi about
// (dx, dy, dz): the MCML rotation (Wang, Jacques & Zheng 1995), lab frame near
// the poles.  Not renormalised: for |d|^2 = 1 + 2e the result has
// |d'|^2 = 1 + 2e (mu^2 + st^2 cos^2 phi) up to one step's rounding, so a
// length error never grows (it shrinks by (1 + <mu^2>) / 2 = 0.94 per step
// on average for g = 0.9) and stays at a few 1e-7, far inside the 1e-4
// tolerance of every consumer of d; the lab frame is unit by construction.
__device__ __forceinline__ void rotate(float& dx, float& dy, float& dz, float mu, float st,
                                       float u_phi) {
  float sp, cp;
  sincos_2pi(u_phi, sp, cp);
  // 1 - dz^2 of a unit vector, taken as dx^2 + dy^2: an FP32 direction is
  // unit only to ~1e-7, and near the poles 1 - dz^2 would carry that error
  // into a frame of size ~1e-4.  Both forms are evaluated and the lab frame
  // is selected near the poles (a select, not a branch: the general form's
  // value there, possibly not finite, is discarded)
  const float q = fmaf(dx, dx, dy * dy);
  const float it = fast_rsqrt(q);
  const float tmp = q * it;
  const bool pole = fabsf(dz) > 0.99999f;
  // g_xy = st (d_xy d_z cos phi + (-d_y, d_x) sin phi) / sqrt(q) + d_xy mu, in pairs
  const float2 a2 = mul2(make_float2(dx, dy), make_float2(dz, dz));
  const float2 b2 = mul2(make_float2(-dy, dx), make_float2(sp, sp));
  const float2 c2 = fma2(a2, make_float2(cp, cp), b2);
  const float2 e2 = mul2(make_float2(st, st), c2);
  const float2 m2 = mul2(make_float2(dx, dy), make_float2(mu, mu));
  const float2 g2 = fma2(e2, make_float2(it, it), m2);
  const float gx = g2.x, gy = g2.y;
  const float2 zz2 = mul2(make_float2(-st, dz), make_float2(cp, mu));
  const float gz = fmaf(zz2.x, tmp, zz2.y);
  const float ox = pole ? st * cp : gx;
  const float oy = pole ? st * sp : gy;
  dx = ox;
  dy = oy;
  dz = pole ? ((dz >= 0.0f) ? mu : -mu) : gz;
}

// ------------------------------------------------------------- photon --
struct Photon {
  float px, py, pz, dx, dy, dz, tau_a;
  int layer;
  uint32_t n;          // steps taken
  uint32_t pid_lo, pid_hi, ev_lo;
  int ev;              // event slot for the tallies
  // hit records only (dead code elsewhere): emission offset along the
  // segment, path length so far, emitting source
  float t_emit, path;
  int src;
  // conservative budget (negative: unknown): no horizontal move shorter than
  // cb reaches a string.  It shrinks by each step's horizontal length, so
  // most steps skip the cell-grid test.
  float cb;
};

// a2: birth from Philox block 0 -- point on the emitting segment, direction
// (isotropic, or on the Cherenkov cone about the segment), and the absorption
// optical depth the photon carries.  Returns false for a malformed source.
__device__ __forceinline__ bool birth(Photon& ph, const pp_source& s, const IceDev& I,
                                      const RunDev& R) {
  const uint4 x = photon_block(R, ph.pid_lo, ph.pid_hi, 0u, ph.ev_lo);
  float sdx = s.dx, sdy = s.dy, sdz = s.dz;
  const float nn = fmaf(sdx, sdx, fmaf(sdy, sdy, sdz * sdz));
  if (nn > 0.0f) {
    const float inv = rsqrtf(nn);
    sdx *= inv;
    sdy *= inv;
    sdz *= inv;
  }
  const float t0 = u01f(x.x) * s.length;
  ph.t_emit = t0;
  ph.path = 0.0f;
  ph.px = fmaf(t0, sdx, s.x);
  ph.py = fmaf(t0, sdy, s.y);
  ph.pz = fmaf(t0, sdz, s.z);
  if (s.type == PP_SRC_CHERENKOV) {
    ph.dx = sdx;
    ph.dy = sdy;
    ph.dz = sdz;
    rotate(ph.dx, ph.dy, ph.dz, R.cos_cherenkov, R.sin_cherenkov, u01f(x.z));
  } else {
    // mu = 2u - 1, so (1 - mu)(1 + mu) = 4u(1 - u) without cancellation
    const float u = u01f(x.y);
    const float mu = fmaf(2.0f, u, -1.0f);
    const float st = 2.0f * fast_sqrt(u * (1.0f - u));
    float sp, cp;
    sincos_2pi(u01f(x.z), sp, cp);
    ph.dx = st * cp;
    ph.dy = st * sp;
    ph.dz = mu;
  }
  ph.tau_a = neg_log(u01f(x.w));
  ph.n = 0;
  ph.cb = -1.0f;
  const bool ok = s.type <= PP_SRC_CASCADE && isfinite(ph.px) && isfinite(ph.py) &&
                  isfinite(ph.pz) && nn > 0.0f && s.length >= 0.0f;
  ph.layer = ok ? layer_at(I, ph.pz, ph.dz) : 0;
  return ok;
}

// a3..a7: one step.  Returns kScattered after a scatter, else the outcome.
__device__ __forceinline__ int photon_step(Photon& ph, const IceDev& I, const GeomDev& G,
                                           const Tables& T, const RunDev& R,
                                           uint32_t& crossings, uint32_t& slow) {
  ph.n += 1;
  const uint4 x = photon_block(R, ph.pid_lo, ph.pid_hi, ph.n, ph.ev_lo);
  const float tau_s = neg_log(u01f(x.x));
  int layer = ph.layer;
  float tau_a = ph.tau_a;
  bool absorb;
  const float S = walk(T.layer, I, ph.pz, ph.dz, layer, tau_s, tau_a, absorb, crossings);
  // world exit: +inf while the step provably stays inside (shorter than the
  // radius of a ball about the start that lies in the world), which gives
  // the same decisions as the exact distance (only "t_exit > S" matters
  // then); the 1 cm margin exceeds the FP32 error of the test.  The ball is
  // measured on every step: a few converged instructions cost less than a
  // budget carried across steps, whose re-measures some lane of the warp
  // needed in most steps
  float tw = PP_INF;
  if (!(S + 0.01f < world_inner(G, ph.px, ph.py, ph.pz)))
    tw = world_exit(G, ph.px, ph.py, ph.pz, ph.dx, ph.dy, ph.dz);
  const float St = fminf(S, tw);
  // DOM test, skipped while the step's horizontal length is inside the budget
  const float lxy = St * fast_sqrt(fmaf(ph.dx, ph.dx, ph.dy * ph.dy));
  float th = PP_INF;
  int k = -1;
  if (!(lxy < ph.cb))
    k = first_hit_grid(G, T, ph.px, ph.py, ph.pz, ph.dx, ph.dy, ph.dz, St, th, slow, &ph.cb);
  if (k >= 0 && th < tw) {
    ph.path += th;
    return k;
  }
  if (tw <= S) return kEscaped;
  if (absorb) return kAbsorbed;
  ph.path += S;
  ph.cb -= lxy + 1e-4f;
  ph.px = fmaf(S, ph.dx, ph.px);
  ph.py = fmaf(S, ph.dy, ph.py);
  ph.pz = fmaf(S, ph.dz, ph.pz);
  float mu, st;
  hg_angle(I, u01f(x.y), mu, st);
  rotate(ph.dx, ph.dy, ph.dz, mu, st, u01f(x.z));
  ph.layer = layer;
  ph.tau_a = tau_a;
  if (ph.n >= R.max_steps) return kTruncated;
  return kScattered;
}

// Loads of the work description's read-only arrays.  kCg: through L2 only
// (ld.global.cg), for memory the host may have rewritten while the kernel
// runs (the serving arenas, reused by later requests), where a line left in
// an SM's L1 could be stale; otherwise the read-only path.
template <bool kCg, class T>
__device__ __forceinline__ T ld_work(const T* p) {
  if (kCg) return __ldcg(p);
  return __ldg(p);
}

// Source containing batch photon index g: the last s with off[s] <= g, found
// inside the range the photon-chunk table gives for g's chunk.
template <bool kCg = false>
__device__ __forceinline__ int find_source(const WorkDev& W, uint32_t chunk_log2, uint64_t g) {
  const uint64_t c = g >> chunk_log2;
  int lo = (int)ld_work<kCg>(W.chunk_src + c), hi = (int)ld_work<kCg>(W.chunk_src + c + 1);
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ld_work<kCg>(W.off + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Fills the photon's identity (event slot, Philox key word, event-local id)
// from its source s and its index within that source.
__device__ __forceinline__ void identify(const WorkDev& W, int s, uint64_t in_src, uint64_t g,
                                         Photon& ph) {
  uint64_t pid = g;
  if (W.aux) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(W.aux) + s);
    pid = ((uint64_t)a.y << 32 | a.x) + in_src;
    ph.ev_lo = a.z;
    ph.ev = (int)a.w;
  } else {
    ph.ev = 0;
    ph.ev_lo = W.single_event_lo;
  }
  ph.pid_lo = (uint32_t)pid;
  ph.pid_hi = (uint32_t)(pid >> 32);
}

// One photon's identity from its batch index alone.  Returns the source.
__device__ __forceinline__ int locate(const WorkDev& W, uint32_t chunk_log2, uint64_t g,
                                      Photon& ph) {
  const int s = find_source(W, chunk_log2, g);
  identify(W, s, g - __ldg(W.off + s), g, ph);
  return s;
}

// Sources of a warp's claim of consecutive batch photons g0 .. g0 + 31 (lane
// with rank r takes g0 + r): one warp-uniform search for g0's source s0, one
// coalesced load of the 32 boundaries off[s0 + 1 .. s0 + 32], and per lane a
// 5-step shuffle search for how many of them lie at or below its photon.
// Returns the lane's source; in_src receives the photon's index inside it.
// Must be called by all 32 lanes; `rank` only matters for lanes that use it.
template <bool kCg = false>
__device__ __forceinline__ int locate_claim(const WorkDev& W, uint32_t chunk_log2, uint64_t g0,
                                            uint32_t rank, uint64_t total, uint64_t& in_src) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int s0 = find_source<kCg>(W, chunk_log2, g0);
  const uint64_t off0 = ld_work<kCg>(W.off + s0);
  const int sj = s0 + 1 + lane;
  const uint64_t bj = (sj <= W.n_src) ? ld_work<kCg>(W.off + sj) : ~0ull;
  const uint64_t dj = bj - g0;  // > 0: boundary after source s0 + lane, relative to g0
  const uint32_t kj = dj > 0xffffffffull ? 0xffffffffu : (uint32_t)dj;
  int pos = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const uint32_t kv = __shfl_sync(full, kj, pos + step - 1);
    if (kv <= rank) pos += step;
  }
  if (__shfl_sync(full, kj, 31) <= rank && pos == 31) pos = 32;
  const uint32_t kprev = __shfl_sync(full, kj, pos > 0 ? (pos < 32 ? pos - 1 : 31) : 0);
  if (pos == 32) {  // more than 32 sources in the claim (empty sources): plain search
    const uint64_t g = g0 + rank;
    if (g >= total) {  // past the end: a lane with nothing to claim
      in_src = 0;
      return s0;
    }
    const int s = find_source<kCg>(W, chunk_log2, g);
    in_src = g - ld_work<kCg>(W.off + s);
    return s;
  }
  in_src = (pos == 0) ? (g0 - off0) + rank : (uint64_t)(rank - kprev);
  return s0 + pos;
}

// a6: integer tallies.
__device__ __forceinline__ void tally(const WorkDev& W, int n_dom, const Photon& ph, int out) {
  unsigned long long* cnt = W.counts + (size_t)ph.ev * 4;
  if (out >= 0) {
    atomicAdd(W.hits + (size_t)ph.ev * n_dom + out, 1ull);
  } else if (out == kEscaped) {
    atomicAdd(cnt + 1, 1ull);
  } else {
    atomicAdd(cnt + 0, 1ull);
    if (out == kTruncated) atomicAdd(cnt + 2, 1ull);
  }
  atomicAdd(cnt + 3, (unsigned long long)ph.n);
}

// Compact hit record (paper Sec. 4: the producing particle's ID, the hit time
// and the weight): appended at an atomic cursor; past the capacity only the
// count grows.
__device__ __forceinline__ void record_hit(const WorkDev& W, const RunDev& R, const Photon& ph,
                                           int dom) {
  const unsigned long long i = atomicAdd(W.n_records, 1ull);
  if (i < W.max_records) {
    pp_hit h;
    h.dom = (uint32_t)dom;
    h.source = (uint32_t)ph.src;
    h.time_ns = fmaf(ph.path, R.ns_per_m_path, ph.t_emit * R.ns_per_m_emit);
    // acceptance: the caller's polynomial in the direction's z (Horner), in [0, 1]
    float w = 1.0f;
    if (R.n_accept > 0) {
      w = R.accept[R.n_accept - 1];
      for (int i = R.n_accept - 2; i >= 0; --i) w = fmaf(w, ph.dz, R.accept[i]);
      w = __saturatef(w);
    }
    h.weight = w;
    W.records[i] = h;
  }
}

// Per-lane tallies of the lane's current event: the absorbed / escaped /
// truncated / step counts of successive photons of one event are summed in
// registers and added to the event's counters only when the lane moves to
// another event (and at exit).  A batch of one huge event would otherwise send
// every photon's atomics to the same three addresses.
struct LaneTally {
  int ev = -1;
  uint32_t absorbed = 0, escaped = 0, truncated = 0;
  unsigned long long steps = 0;
};

__device__ __forceinline__ void flush(const WorkDev& W, LaneTally& t) {
  if (t.ev >= 0) {
    unsigned long long* cnt = W.counts + (size_t)t.ev * 4;
    if (t.absorbed) atomicAdd(cnt + 0, (unsigned long long)t.absorbed);
    if (t.escaped) atomicAdd(cnt + 1, (unsigned long long)t.escaped);
    if (t.truncated) atomicAdd(cnt + 2, (unsigned long long)t.truncated);
    if (t.steps) atomicAdd(cnt + 3, t.steps);
  }
  t.absorbed = t.escaped = t.truncated = 0;
  t.steps = 0;
}

__device__ __forceinline__ void tally(const WorkDev& W, int n_dom, const Photon& ph, int out,
                                      LaneTally& t) {
  if (ph.ev != t.ev) {
    flush(W, t);
    t.ev = ph.ev;
  }
  if (out >= 0) {
    atomicAdd(W.hits + (size_t)ph.ev * n_dom + out, 1ull);
  } else if (out == kEscaped) {
    t.escaped += 1;
  } else {
    t.absorbed += 1;
    if (out == kTruncated) t.truncated += 1;
  }
  t.steps += ph.n;
}

}  // namespace ppk
