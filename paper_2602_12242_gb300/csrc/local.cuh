// Device helpers shared by the local-field kernels (local.cu) and the
// adjoint kernels (adjoint.cu): float3 arithmetic, the local field terms at
// one cell (exchange, DMI with the chiral ghost cells, anisotropy, Zeeman,
// plus the demag field read from the convolution) and the LLG right-hand side.
#pragma once

#include "common.cuh"

namespace mx {

struct Terms {
  float3 demag, exch, dmi, anis, zee;
};

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// All field terms at cell (i, j, k).
template <bool DMI>
__device__ __forceinline__ void local_terms(const float4* __restrict__ m, const float4* __restrict__ hd,
                                            const Grid& g, const LocalCoef& c, int i, int j, int k, long idx,
                                            float3 mc, float inv_ms, Terms& t) {
  const long sx = 1, sy = g.nx, sz = (long)g.nx * g.ny;
  float3 xm, xp, ym, yp, zm, zp;
  // chiral ghosts (kdx, kdy are zero when DMI is off)
  xp = (i + 1 < g.nx) ? f3(__ldg(&m[idx + sx])) : make_float3(mc.x - c.kdx * mc.z, mc.y, mc.z + c.kdx * mc.x);
  xm = (i > 0) ? f3(__ldg(&m[idx - sx])) : make_float3(mc.x + c.kdx * mc.z, mc.y, mc.z - c.kdx * mc.x);
  yp = (j + 1 < g.ny) ? f3(__ldg(&m[idx + sy])) : make_float3(mc.x, mc.y - c.kdy * mc.z, mc.z + c.kdy * mc.y);
  ym = (j > 0) ? f3(__ldg(&m[idx - sy])) : make_float3(mc.x, mc.y + c.kdy * mc.z, mc.z - c.kdy * mc.y);
  zp = (k + 1 < g.nz) ? f3(__ldg(&m[idx + sz])) : mc;
  zm = (k > 0) ? f3(__ldg(&m[idx - sz])) : mc;
  const float3 two = 2.f * mc;
  const float3 lap = c.inv_dx2 * (xp + xm - two) + c.inv_dy2 * (yp + ym - two) + c.inv_dz2 * (zp + zm - two);
  t.exch = (c.cA * inv_ms) * lap;
  if (DMI) {
    const float3 ddx = c.inv_2dx * (xp - xm);
    const float3 ddy = c.inv_2dy * (yp - ym);
    t.dmi = (c.cD * inv_ms) * make_float3(ddx.z, ddy.z, -(ddx.x + ddy.y));
  } else {
    t.dmi = make_float3(0.f, 0.f, 0.f);
  }
  const float3 e = c.axis_map ? f3(__ldg(&c.axis_map[idx])) : make_float3(c.ax, c.ay, c.az);
  const float cK = c.ku_map ? (__ldg(&c.ku_map[idx]) * (float)(2.0 / kMu0)) : c.cK;
  t.anis = (cK * inv_ms * dot3(mc, e)) * e;
  t.zee = make_float3(c.hx, c.hy, c.hz);
  t.demag = hd ? f3(__ldg(&hd[idx])) : make_float3(0.f, 0.f, 0.f);
}

__device__ __forceinline__ float3 llg(const LocalCoef& c, float3 mc, float3 H) {
  const float3 mxH = cross3(mc, H);
  const float3 mxmxH = cross3(mc, mxH);
  const float3 p = c.precession ? mxH : make_float3(0.f, 0.f, 0.f);
  return c.llg * (p + c.alpha * mxmxH);
}

__device__ __forceinline__ float3 unit(float3 v) {
  const float r = rnorm3df(v.x, v.y, v.z);
  return r * v;
}


// normalise v; r receives |v|
__device__ __forceinline__ float3 unit_norm(float3 v, float& r) {
  r = norm3df(v.x, v.y, v.z);
  const float inv = rnorm3df(v.x, v.y, v.z);
  return inv * v;
}

}  // namespace mx
