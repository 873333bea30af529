// Device helpers shared by the local-field kernels (local.cu) and the
// adjoint kernels (adjoint.cu): float3 arithmetic, the local field terms at
// one cell (exchange, DMI with the chiral ghost cells, anisotropy, Zeeman,
// plus the demag field read from the convolution) and the LLG right-hand side.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

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

// The six face neighbours of cell (i, j, k), with the ghost cells of the
// boundary condition where a neighbour is missing: the chiral ghost
// m_b - h (D/2A)(e_z x n) x m_b on x and y faces (kdx, kdy are zero when DMI
// is off, which leaves the Neumann ghost m_b), m_b on z faces.
__device__ __forceinline__ void neighbours(const float4* __restrict__ m, const Grid& g, const LocalCoef& c, int i,
                                           int j, int k, long idx, float3 mc, float3& xp, float3& xm, float3& yp,
                                           float3& ym, float3& zp, float3& zm) {
  const long sx = 1, sy = g.nx, sz = (long)g.nx * g.ny;
  xp = (i + 1 < g.nx) ? f3(__ldg(&m[idx + sx])) : make_float3(mc.x - c.kdx * mc.z, mc.y, mc.z + c.kdx * mc.x);
  xm = (i > 0) ? f3(__ldg(&m[idx - sx])) : make_float3(mc.x + c.kdx * mc.z, mc.y, mc.z - c.kdx * mc.x);
  yp = (j + 1 < g.ny) ? f3(__ldg(&m[idx + sy])) : make_float3(mc.x, mc.y - c.kdy * mc.z, mc.z + c.kdy * mc.y);
  ym = (j > 0) ? f3(__ldg(&m[idx - sy])) : make_float3(mc.x, mc.y + c.kdy * mc.z, mc.z - c.kdy * mc.y);
  zp = (k + 1 < g.nz) ? f3(__ldg(&m[idx + sz])) : mc;
  zm = (k > 0) ? f3(__ldg(&m[idx - sz])) : mc;
}

// All field terms at cell (i, j, k); the demag term is the given value hdv,
// the easy axis e and the anisotropy coefficient cK = 2 Ku / mu0 are given.
template <bool DMI>
__device__ __forceinline__ void local_terms_ek(const float4* __restrict__ m, float3 hdv, const Grid& g,
                                               const LocalCoef& c, int i, int j, int k, long idx, float3 mc,
                                               float inv_ms, float3 e, float cK, Terms& t) {
  float3 xm, xp, ym, yp, zm, zp;
  neighbours(m, g, c, i, j, k, idx, mc, xp, xm, yp, ym, zp, zm);
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
  t.anis = (cK * inv_ms * dot3(mc, e)) * e;
  t.zee = make_float3(c.hx, c.hy, c.hz);
  t.demag = hdv;
}

__device__ __forceinline__ float3 easy_axis(const LocalCoef& c, long idx) {
  return c.axis_map ? f3(__ldg(&c.axis_map[idx])) : make_float3(c.ax, c.ay, c.az);
}
__device__ __forceinline__ float aniso_coef(const LocalCoef& c, long idx) {
  return c.ku_map ? (__ldg(&c.ku_map[idx]) * (float)(2.0 / kMu0)) : c.cK;
}

// All field terms at cell (i, j, k); the demag term is the given value hdv.
template <bool DMI>
__device__ __forceinline__ void local_terms_v(const float4* __restrict__ m, float3 hdv, const Grid& g,
                                              const LocalCoef& c, int i, int j, int k, long idx, float3 mc,
                                              float inv_ms, Terms& t) {
  local_terms_ek<DMI>(m, hdv, g, c, i, j, k, idx, mc, inv_ms, easy_axis(c, idx), aniso_coef(c, idx), t);
}

// All field terms at cell (i, j, k), the demag term read from hd (zero if hd is null).
template <bool DMI>
__device__ __forceinline__ void local_terms(const float4* __restrict__ m, const float4* __restrict__ hd,
                                            const Grid& g, const LocalCoef& c, int i, int j, int k, long idx,
                                            float3 mc, float inv_ms, Terms& t) {
  local_terms_v<DMI>(m, hd ? f3(__ldg(&hd[idx])) : make_float3(0.f, 0.f, 0.f), g, c, i, j, k, idx, mc, inv_ms, t);
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

// What the local stage of MODE reads at the cell itself (the neighbours
// are read while the fields are formed).
struct CellIn {
  float3 m, m0, acc, e;
  float ms, cK;
};

template <int MODE>
__device__ __forceinline__ CellIn load_cell(const StageIO& io, const LocalCoef& c, long idx) {
  CellIn v;
  v.m = f3(io.m[idx]);
  v.ms = c.ms_map ? __ldg(&c.ms_map[idx]) : c.Ms;
  v.e = easy_axis(c, idx);
  v.cK = aniso_coef(c, idx);
  if (MODE == LM_RK4_S1 || MODE == LM_RK4_S2 || MODE == LM_RK4_S3) {
    v.m0 = f3(io.m0[idx]);
    v.acc = f3(io.acc[idx]);
  } else {
    v.m0 = v.acc = make_float3(0.f, 0.f, 0.f);
  }
  return v;
}

// One cell of the fused local stage from its loaded inputs v: H_eff (demag
// term hdv), the LLG right-hand side and the stage update of MODE
// (LocalMode), written to io.out.
template <int MODE, bool DMI>
__device__ __forceinline__ void local_cell_in(const StageIO& io, const Grid& g, const LocalCoef& c, int i, int j,
                                              int k, long idx, float3 hdv, const CellIn& v, int* flag) {
  const float3 mc = v.m;
  const float inv_ms = 1.f / v.ms;
  Terms t;
  local_terms_ek<DMI>(io.m, hdv, g, c, i, j, k, idx, mc, inv_ms, v.e, v.cK, t);
  float3 out;
  float wout = 0.f;  // |u| of a renormalised stage output (used by the adjoint)
  if (MODE == LM_HEFF) {
    out = make_float3(0.f, 0.f, 0.f);
    if (io.terms & MX_TERM_DEMAG) out = out + t.demag;
    if (io.terms & MX_TERM_EXCH) out = out + t.exch;
    if (io.terms & MX_TERM_ANIS) out = out + t.anis;
    if (io.terms & MX_TERM_DMI) out = out + t.dmi;
    if (io.terms & MX_TERM_ZEEMAN) out = out + t.zee;
  } else {
    const float3 H = t.demag + t.exch + t.anis + t.dmi + t.zee;
    const float3 kk = llg(c, mc, H);
    if (MODE == LM_RHS) {
      out = kk;
    } else if (MODE == LM_EULER) {
      out = unit_norm(mc + io.dt * kk, wout);
    } else if (MODE == LM_RK4_S0) {
      io.acc[idx] = make_float4(kk.x, kk.y, kk.z, 0.f);
      out = unit_norm(mc + (0.5f * io.dt) * kk, wout);
    } else {
      const float3 m0 = v.m0;
      const float3 a = v.acc;
      if (MODE == LM_RK4_S3) {
        out = unit_norm(m0 + (io.dt * (1.f / 6.f)) * (a + kk), wout);
      } else {
        io.acc[idx] = make_float4(a.x + 2.f * kk.x, a.y + 2.f * kk.y, a.z + 2.f * kk.z, 0.f);
        out = unit_norm(m0 + ((MODE == LM_RK4_S1 ? 0.5f : 1.f) * io.dt) * kk, wout);
      }
    }
  }
  if (!(isfinite(out.x) && isfinite(out.y) && isfinite(out.z))) atomicOr(flag, kFlagNonfinite);
  io.out[idx] = make_float4(out.x, out.y, out.z, wout);
}

// The same with the inputs loaded here.
template <int MODE, bool DMI>
__device__ __forceinline__ void local_cell_v(const StageIO& io, const Grid& g, const LocalCoef& c, int i, int j,
                                             int k, long idx, float3 hdv, int* flag) {
  local_cell_in<MODE, DMI>(io, g, c, i, j, k, idx, hdv, load_cell<MODE>(io, c, idx), flag);
}

// The same with the demag term read from io.hd (zero if io.hd is null).
template <int MODE, bool DMI>
__device__ __forceinline__ void local_cell(const StageIO& io, const Grid& g, const LocalCoef& c, int i, int j, int k,
                                           long idx, int* flag) {
  local_cell_v<MODE, DMI>(io, g, c, i, j, k, idx, io.hd ? f3(__ldg(&io.hd[idx])) : make_float3(0.f, 0.f, 0.f), flag);
}

}  // namespace mx
