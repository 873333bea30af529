// Explicit-explicit multirate infinitesimal (MRI) step (Sec. II-C, III-C).
//
// Fast part of the LLG right-hand side: the one driven by the exchange field
// (stencil only); slow part: demag + anisotropy + DMI + Zeeman.  Both levels
// use the three-stage third-order explicit method of Knoth and Wolke,
//   A = [[0,0,0],[1/3,0,0],[-3/16,15/16,0]], b = [1/6,3/10,8/15],
//   c = [0,1/3,3/4].
// Slow stages Y_1 = m and, for i = 2, 3, 4 (c_4 = 1, row 4 of A = b), the
// end of an interval of length (c_i - c_{i-1}) h of
//   v' = f_fast(v) + r_i,  v(0) = Y_{i-1},
//   r_i = sum_{j<i} (a_ij - a_{i-1,j}) f_slow(Y_j) / (c_i - c_{i-1}),
// integrated with ceil((c_i - c_{i-1}) / ratio) equal Knoth-Wolke steps;
// m_new = Y_4.  Every fast stage input and fast step result is renormalised
// (Sec. II-B).  One step: three demag convolutions and three slow kernels,
// 12 x 3 fast kernels at ratio 0.1; everything in place on m except the
// slow right-hand sides F_1..F_3 and two stage buffers.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"
#include "local.cuh"

namespace mx {

namespace {
constexpr double kA21 = 1.0 / 3.0, kA31 = -3.0 / 16.0, kA32 = 15.0 / 16.0;
constexpr double kB1 = 1.0 / 6.0, kB2 = 3.0 / 10.0, kB3 = 8.0 / 15.0;
constexpr double kC[4] = {0.0, 1.0 / 3.0, 3.0 / 4.0, 1.0};
constexpr double kAext[4][3] = {{0.0, 0.0, 0.0}, {kA21, 0.0, 0.0}, {kA31, kA32, 0.0}, {kB1, kB2, kB3}};
}  // namespace

// F = f_slow(m): LLG right-hand side of demag + anisotropy + DMI + Zeeman.
template <bool DMI>
__global__ void __launch_bounds__(256) mri_slow_kernel(const float4* __restrict__ m, const float4* __restrict__ hd,
                                                       Grid g, LocalCoef c, float4* __restrict__ F, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long idx = ((long)k * g.ny + j) * g.nx + i;
  const float3 mc = f3(m[idx]);
  const float ms = c.ms_map ? __ldg(&c.ms_map[idx]) : c.Ms;
  Terms t;
  local_terms<DMI>(m, hd, g, c, i, j, k, idx, mc, 1.f / ms, t);
  const float3 f = llg(c, mc, t.demag + t.anis + t.dmi + t.zee);
  if (!(isfinite(f.x) && isfinite(f.y) && isfinite(f.z))) atomicOr(flag, kFlagNonfinite);
  F[idx] = make_float4(f.x, f.y, f.z, 0.f);
}

// Forcing r and the fast step's stage data.
struct FastIO {
  const float4* __restrict__ u;  // stage input (stencil acts on it)
  float4* __restrict__ v;        // fast step start; the step result replaces it (stage 2)
  float4* __restrict__ acc;      // stage 0: k1; stage 1 on: b1 k1 + b2 k2
  float4* __restrict__ out;      // stages 0, 1: next stage input
  const float4* __restrict__ F0;
  const float4* __restrict__ F1;
  const float4* __restrict__ F2;
  float w0, w1, w2;  // r = w0 F0 + w1 F1 + w2 F2
  float h;           // fast step
};

// One Knoth-Wolke stage of v' = f_fast(v) + r (STAGE 0, 1, 2).
template <int STAGE>
__global__ void __launch_bounds__(256) mri_fast_kernel(FastIO io, Grid g, LocalCoef c, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long idx = ((long)k * g.ny + j) * g.nx + i;
  const float3 uc = f3(io.u[idx]);
  const float ms = c.ms_map ? __ldg(&c.ms_map[idx]) : c.Ms;
  float3 xp, xm, yp, ym, zp, zm;
  neighbours(io.u, g, c, i, j, k, idx, uc, xp, xm, yp, ym, zp, zm);
  const float3 two = 2.f * uc;
  const float3 lap = c.inv_dx2 * (xp + xm - two) + c.inv_dy2 * (yp + ym - two) + c.inv_dz2 * (zp + zm - two);
  float3 kk = llg(c, uc, (c.cA / ms) * lap);
  if (io.w0 != 0.f) kk = kk + io.w0 * f3(__ldg(&io.F0[idx]));
  if (io.w1 != 0.f) kk = kk + io.w1 * f3(__ldg(&io.F1[idx]));
  if (io.w2 != 0.f) kk = kk + io.w2 * f3(__ldg(&io.F2[idx]));
  const float3 v = STAGE == 0 ? uc : f3(io.v[idx]);
  float3 res;
  float wout = 0.f;
  if (STAGE == 0) {
    io.acc[idx] = make_float4(kk.x, kk.y, kk.z, 0.f);
    res = unit_norm(v + (float)(kA21)*io.h * kk, wout);
    io.out[idx] = make_float4(res.x, res.y, res.z, wout);
  } else if (STAGE == 1) {
    const float3 k1 = f3(io.acc[idx]);
    res = unit_norm(v + io.h * ((float)kA31 * k1 + (float)kA32 * kk), wout);
    io.out[idx] = make_float4(res.x, res.y, res.z, wout);
    const float3 s = (float)kB1 * k1 + (float)kB2 * kk;
    io.acc[idx] = make_float4(s.x, s.y, s.z, 0.f);
  } else {
    const float3 s = f3(io.acc[idx]);
    res = unit_norm(v + io.h * (s + (float)kB3 * kk), wout);
    io.v[idx] = make_float4(res.x, res.y, res.z, wout);
  }
  if (!(isfinite(res.x) && isfinite(res.y) && isfinite(res.z))) atomicOr(flag, kFlagNonfinite);
}

int mri_fast_steps(double interval, double ratio) {
  const int n = (int)ceil(interval / ratio - 1e-9);
  return n < 1 ? 1 : n;
}

static void local_grid(const Grid& g, dim3& grid, dim3& block) {
  block = dim3(32, 8, 1);
  if (g.nx < 32) block = dim3(g.nx <= 8 ? 8 : (g.nx <= 16 ? 16 : 32), 256 / (g.nx <= 8 ? 8 : (g.nx <= 16 ? 16 : 32)), 1);
  grid = dim3((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
}

mx_status mri_reserve(mx_ctx* ctx) {
  if (ctx->mri_f) return MX_OK;
  if (cudaMalloc(&ctx->mri_f, sizeof(float4) * 3 * ctx->g.ncell) != cudaSuccess) {
    cudaGetLastError();
    ctx->mri_f = nullptr;
    set_error("mx_rk_step: cannot allocate the MRI slow right-hand sides");
    return MX_ERR_OOM;
  }
  return MX_OK;
}

// One MRI step of size dt on m (in place); stage buffers sa, sb, acc.
mx_status mri_step(mx_ctx* ctx, float4* m, double dt, cudaStream_t st) {
  MX_TRY(mri_reserve(ctx));
  const Grid& g = ctx->g;
  const LocalCoef c = local_coef(ctx);
  const bool demag = ctx->p.demag != 0;
  const double ratio = ctx->p.mri_fast_ratio > 0.0 ? ctx->p.mri_fast_ratio : 0.1;
  dim3 grid, block;
  local_grid(g, grid, block);
  float4* F[3] = {ctx->mri_f, ctx->mri_f + g.ncell, ctx->mri_f + 2 * g.ncell};
  for (int i = 1; i <= 3; ++i) {
    // slow right-hand side of Y_{i-1} (= m now)
    if (demag) MX_TRY(demag_field(ctx, m, ctx->hd, st));
    {
      ProfScope ps(ctx, KID_MRI_SLOW, st);
      if (c.dmi)
        mri_slow_kernel<true><<<grid, block, 0, st>>>(m, demag ? ctx->hd : nullptr, g, c, F[i - 1], ctx->flag);
      else
        mri_slow_kernel<false><<<grid, block, 0, st>>>(m, demag ? ctx->hd : nullptr, g, c, F[i - 1], ctx->flag);
      MX_TRY(launch_check("mri_slow_kernel"));
    }
    const double dc = kC[i] - kC[i - 1];
    double w[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < i; ++j) w[j] = (kAext[i][j] - kAext[i - 1][j]) / dc;
    const int n = mri_fast_steps(dc, ratio);
    FastIO io{};
    io.v = m;
    io.acc = ctx->acc;
    io.F0 = F[0];
    io.F1 = F[1];
    io.F2 = F[2];
    io.w0 = (float)w[0];
    io.w1 = (float)w[1];
    io.w2 = (float)w[2];
    io.h = (float)(dc * dt / n);
    ProfScope ps(ctx, KID_MRI_FAST, st);
    for (int q = 0; q < n; ++q) {
      io.u = m;
      io.out = ctx->sa;
      mri_fast_kernel<0><<<grid, block, 0, st>>>(io, g, c, ctx->flag);
      io.u = ctx->sa;
      io.out = ctx->sb;
      mri_fast_kernel<1><<<grid, block, 0, st>>>(io, g, c, ctx->flag);
      io.u = ctx->sb;
      io.out = nullptr;
      mri_fast_kernel<2><<<grid, block, 0, st>>>(io, g, c, ctx->flag);
      MX_TRY(launch_check("mri_fast_kernel"));
    }
  }
  return MX_OK;
}

}  // namespace mx
