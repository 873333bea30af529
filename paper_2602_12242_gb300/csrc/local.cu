// Fused local kernel: exchange / DMI / anisotropy / Zeeman fields, the demag
// field read from the convolution, the LLG right-hand side and the RK stage
// update with renormalisation, one thread per cell with float4 access.
//
//   exchange  H = 2A/(mu0 Ms_i) sum_d (m_{i+d} + m_{i-d} - 2 m_i)/h_d^2
//             (Sec. II-A exchange term, second-order central differences of
//             Sec. II-B)
//   DMI       H = 2D/(mu0 Ms_i) (d_x m_z, d_y m_z, -(d_x m_x + d_y m_y)),
//             central differences in x and y (Sec. II-A interfacial form)
//   boundary  a missing neighbour across the face with outward normal n is
//             the ghost m_b - h (D/2A) (e_z x n) x m_b, the discrete form of
//             dm/dx_k = -(D/2A)(e_z x e_k) x m (Sec. II-A, II-B); with DMI off
//             (or on z faces) this is m_b, the Neumann condition
//   anisotropy H = 2 Ku/(mu0 Ms_i) (m.e) e
//   LLG       dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)]  (Eq. 1)
//   RK4       k_s at stage s; acc = k1 + 2k2 + 2k3; stage inputs
//             normalize(m0 + c dt k), result normalize(m0 + dt/6 (acc + k4))
//             (renormalisation after every stage, Sec. II-B)
#include "common.cuh"
#include "kernels.cuh"
#include "local.cuh"

namespace mx {

template <int MODE, bool DMI>
__global__ void __launch_bounds__(256) local_kernel(StageIO io, Grid g, LocalCoef c, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  pdl_wait();
  if (i >= g.nx || j >= g.ny) return;
  const long idx = ((long)k * g.ny + j) * g.nx + i;
  local_cell<MODE, DMI>(io, g, c, i, j, k, idx, flag);
}

__global__ void normalize_kernel(float4* m, long n, int* flag) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const float4 v = m[idx];
  const float r = rnorm3df(v.x, v.y, v.z);
  const float4 o = make_float4(v.x * r, v.y * r, v.z * r, 0.f);
  if (!(isfinite(o.x) && isfinite(o.y) && isfinite(o.z))) atomicOr(flag, kFlagNonfinite);
  m[idx] = o;
}

__global__ void copy_kernel(float4* __restrict__ dst, const float4* __restrict__ src, long n) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) dst[idx] = src[idx];
}

// Energies: [demag, exch, anis, dmi, zeeman], FP64 block sums then atomics.
template <bool DMI>
__global__ void __launch_bounds__(256) energy_kernel(const float4* __restrict__ m, const float4* __restrict__ hd,
                                                     Grid g, LocalCoef c, double V, double Ku, double* e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double acc[5] = {0, 0, 0, 0, 0};
  if (i < g.nx && j < g.ny) {
    const long idx = ((long)k * g.ny + j) * g.nx + i;
    const float3 mc = f3(m[idx]);
    const float ms = c.ms_map ? c.ms_map[idx] : c.Ms;
    Terms t;
    local_terms<DMI>(m, hd, g, c, i, j, k, idx, mc, 1.f / ms, t);
    const double q = -0.5 * kMu0 * V * (double)ms;
    acc[0] = q * (double)dot3(mc, t.demag);
    acc[1] = q * (double)dot3(mc, t.exch);
    const float3 e3 = c.axis_map ? f3(c.axis_map[idx]) : make_float3(c.ax, c.ay, c.az);
    const double ku = c.ku_map ? (double)c.ku_map[idx] : Ku;
    const double me = (double)dot3(mc, e3);
    acc[2] = V * ku * (1.0 - me * me);
    acc[3] = q * (double)dot3(mc, t.dmi);
    acc[4] = 2.0 * q * (double)dot3(mc, t.zee);
  }
  __shared__ double red[5][8];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  for (int q = 0; q < 5; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (tid < 5) {
    double s = 0.0;
    const int nw = (blockDim.x * blockDim.y + 31) / 32;
    for (int w = 0; w < nw; ++w) s += red[tid][w];
    atomicAdd(&e[tid], s);
  }
}

LocalCoef local_coef(const mx_ctx* ctx) { return local_coef_from(ctx->p, ctx->ms_map, ctx->ku_map, ctx->axis_map); }

LocalCoef local_coef_from(const mx_params& p, const float* ms_map, const float* ku_map, const float4* axis_map) {
  LocalCoef c;
  c.inv_dx2 = (float)(1.0 / (p.dx * p.dx));
  c.inv_dy2 = (float)(1.0 / (p.dy * p.dy));
  c.inv_dz2 = (float)(1.0 / (p.dz * p.dz));
  c.inv_2dx = (float)(0.5 / p.dx);
  c.inv_2dy = (float)(0.5 / p.dy);
  const bool dmi = p.dmi_interfacial && p.D != 0.0 && p.A > 0.0;
  const double kappa = dmi ? p.D / (2.0 * p.A) : 0.0;
  c.kdx = (float)(p.dx * kappa);
  c.kdy = (float)(p.dy * kappa);
  c.cA = (float)(2.0 * p.A / kMu0);
  c.cD = (float)(2.0 * p.D / kMu0);
  c.cK = (float)(2.0 * p.Ku / kMu0);
  c.Ms = (float)p.Ms;
  double ax = p.ku_axis[0], ay = p.ku_axis[1], az = p.ku_axis[2];
  double an = sqrt(ax * ax + ay * ay + az * az);
  if (an > 0) { ax /= an; ay /= an; az /= an; }
  c.ax = (float)ax; c.ay = (float)ay; c.az = (float)az;
  c.hx = (float)p.h_bias[0];
  c.hy = (float)p.h_bias[1];
  c.hz = (float)p.h_bias[2];
  c.llg = (float)(-p.gamma / (1.0 + p.alpha * p.alpha));
  c.alpha = (float)p.alpha;
  c.dmi = dmi ? 1 : 0;
  c.precession = p.precession ? 1 : 0;
  c.ms_map = ms_map;
  c.ku_map = ku_map;
  c.axis_map = axis_map;
  return c;
}

template <int MODE>
static void launch_local(bool dmi, dim3 grid, dim3 block, cudaStream_t st, const StageIO& io, const Grid& g,
                         const LocalCoef& c, int* flag) {
  if (dmi)
    launch_pdl(local_kernel<MODE, true>, grid, block, 0, st, io, g, c, flag);
  else
    launch_pdl(local_kernel<MODE, false>, grid, block, 0, st, io, g, c, flag);
}

static void local_dims(const Grid& g, dim3& grid, dim3& block) {
  block = dim3(32, 8, 1);
  if (g.nx < 32) block = dim3(g.nx <= 8 ? 8 : (g.nx <= 16 ? 16 : 32), 256 / (g.nx <= 8 ? 8 : (g.nx <= 16 ? 16 : 32)), 1);
  grid = dim3((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
}

mx_status local_stage(mx_ctx* ctx, int mode, const StageIO& io, cudaStream_t st) {
  const Grid& g = ctx->g;
  const LocalCoef c = local_coef(ctx);
  dim3 grid, block;
  local_dims(g, grid, block);
  const bool dmi = c.dmi != 0;
  ProfScope ps(ctx, KID_LOCAL, st);
  switch (mode) {
    case LM_HEFF: launch_local<LM_HEFF>(dmi, grid, block, st, io, g, c, ctx->flag); break;
    case LM_RHS: launch_local<LM_RHS>(dmi, grid, block, st, io, g, c, ctx->flag); break;
    case LM_RK4_S0: launch_local<LM_RK4_S0>(dmi, grid, block, st, io, g, c, ctx->flag); break;
    case LM_RK4_S1: launch_local<LM_RK4_S1>(dmi, grid, block, st, io, g, c, ctx->flag); break;
    case LM_RK4_S2: launch_local<LM_RK4_S2>(dmi, grid, block, st, io, g, c, ctx->flag); break;
    case LM_RK4_S3: launch_local<LM_RK4_S3>(dmi, grid, block, st, io, g, c, ctx->flag); break;
    case LM_EULER: launch_local<LM_EULER>(dmi, grid, block, st, io, g, c, ctx->flag); break;
    default: set_error("local_stage: bad mode"); return MX_ERR_INVALID_ARG;
  }
  return launch_check("local_kernel");
}

mx_status normalize_field(mx_ctx* ctx, float4* m, cudaStream_t st) {
  const long n = ctx->g.ncell;
  ProfScope ps(ctx, KID_NORMALIZE, st);
  normalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, n, ctx->flag);
  return launch_check("normalize_kernel");
}

mx_status copy_field(mx_ctx* ctx, float4* dst, const float4* src, cudaStream_t st) {
  const long n = ctx->g.ncell;
  ProfScope ps(ctx, KID_COPY, st);
  copy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst, src, n);
  return launch_check("copy_kernel");
}

// Exchange energy A V sum |grad m|^2 with second-order central differences
// (m_+ - m_-)/(2h) over the field's ghost cells; FP64 block sums, one atomic
// per block.
__global__ void __launch_bounds__(256) exch_central_kernel(const float4* __restrict__ m, Grid g, LocalCoef c,
                                                           double AV, double inv4dx2, double inv4dy2,
                                                           double inv4dz2, double* e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double acc = 0.0;
  if (i < g.nx && j < g.ny) {
    const long idx = ((long)k * g.ny + j) * g.nx + i;
    const float3 mc = f3(m[idx]);
    float3 xp, xm, yp, ym, zp, zm;
    neighbours(m, g, c, i, j, k, idx, mc, xp, xm, yp, ym, zp, zm);
    const float3 dx = xp - xm, dy = yp - ym, dz = zp - zm;
    acc = AV * (inv4dx2 * (double)dot3(dx, dx) + inv4dy2 * (double)dot3(dy, dy) + inv4dz2 * (double)dot3(dz, dz));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[8];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  if ((t & 31) == 0) red[t >> 5] = acc;
  __syncthreads();
  if (t == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x * blockDim.y) / 32; ++w) sum += red[w];
    atomicAdd(e, sum);
  }
}

mx_status exchange_energy_central(mx_ctx* ctx, const float4* m, double* e_dev, cudaStream_t st) {
  const Grid& g = ctx->g;
  const LocalCoef c = local_coef(ctx);
  dim3 grid, block;
  local_dims(g, grid, block);
  const mx_params& p = ctx->p;
  exch_central_kernel<<<grid, block, 0, st>>>(m, g, c, p.A * p.dx * p.dy * p.dz, 0.25 / (p.dx * p.dx),
                                              0.25 / (p.dy * p.dy), 0.25 / (p.dz * p.dz), e_dev);
  return launch_check("exch_central_kernel");
}

mx_status energy_terms(mx_ctx* ctx, const float4* m, const float4* hd, double* e_dev, cudaStream_t st) {
  const Grid& g = ctx->g;
  const LocalCoef c = local_coef(ctx);
  dim3 grid, block;
  local_dims(g, grid, block);
  const double V = ctx->p.dx * ctx->p.dy * ctx->p.dz;
  if (c.dmi)
    energy_kernel<true><<<grid, block, 0, st>>>(m, hd, g, c, V, ctx->p.Ku, e_dev);
  else
    energy_kernel<false><<<grid, block, 0, st>>>(m, hd, g, c, V, ctx->p.Ku, e_dev);
  return launch_check("energy_kernel");
}

}  // namespace mx
