// Compile-time-sized x passes of the demag convolution (the same arithmetic as demag.cu's generic
// kernels, Sec. II-B: zero-padded FFT convolution with the tensor spectrum),
// built from the register FFTs of regfft.cuh.
//
//   xf<E,S>    r2c along x: M = Px/2 = E*S complex points per row (the real
//              row packed as z[n] = x[2n] + i x[2n+1]) plus the split step.
//   xi<E,S>    c2r along x, cells i < nx written as float4.
#include "common.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "local.cuh"
#include "regfft.cuh"
#include "xrows.cuh"

namespace mx {

template <int E, int S, int R, int NT>
__global__ void __launch_bounds__(NT) xf_kernel(const float4* __restrict__ m, Grid g, float ms,
                                                const float* __restrict__ ms_map, float2* __restrict__ w1,
                                                const float2* __restrict__ twM, const float2* __restrict__ twP) {
  extern __shared__ float2 sm[];
  pdl_wait();
  xf_rows<E, S, R, NT, false>(sm, m, g, ms, ms_map, w1, blockIdx.x * R, twM, twP);
}

// ---------------------------------------------------------------------------
// x inverse (c2r).
// ---------------------------------------------------------------------------
template <int E, int S, int R, int NT>
__global__ void __launch_bounds__(NT) xi_kernel(const float2* __restrict__ w1, Grid g, float4* __restrict__ hd,
                                                const float2* __restrict__ twM, const float2* __restrict__ twP) {
  extern __shared__ float2 sm[];
  const int nrows = g.ny * g.nz;
  const int row0 = blockIdx.x * R;
  pdl_wait();
  xi_rows<E, S, R, NT>(sm, w1, g, row0, twM, twP);
  for (int e = threadIdx.x; e < R * g.nx; e += NT) {
    const int r = e / g.nx, i = e % g.nx;
    const int row = row0 + r;
    if (row >= nrows) continue;
    const float3 h = xi_cell<E, S>(sm, r, i);
    hd[(long)row * g.nx + i] = make_float4(h.x, h.y, h.z, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Row kernel of the RK4 step: the inverse x pass of rows row0 .. row0 + R - 1,
// the local stage of `mode` on their cells (demag term from shared memory),
// and, with `xf_next`, the forward x pass of the stage output io.out for the
// next stage, so that between the y/z passes of two stages there is one
// kernel and H_demag never goes to global memory.  io.out of the block's rows
// is written by this block only and read back after a block barrier.
// ---------------------------------------------------------------------------
template <int MODE, bool DMI, int E, int S, int R, int NT>
__device__ __forceinline__ void xr_cells(const float2* sm, const StageIO& io, const Grid& g, const LocalCoef& c,
                                         int row0, float4* __restrict__ hd_out, int* flag) {
  // KC cells per thread and round with every cell's own loads issued first
  constexpr int KC = (R * E * S + NT - 1) / NT < 3 ? (R * E * S + NT - 1) / NT : 3;
  const int nrows = g.ny * g.nz;
  const int total = min(R, nrows - row0) * g.nx;
  for (int e0 = threadIdx.x; e0 < total; e0 += KC * NT) {
    CellIn v[KC];
    long idx[KC];
#pragma unroll
    for (int u = 0; u < KC; ++u) {
      const int e = min(e0 + u * NT, total - 1);
      idx[u] = (long)row0 * g.nx + e;
      v[u] = load_cell<MODE>(io, c, idx[u]);
    }
#pragma unroll
    for (int u = 0; u < KC; ++u) {
      const int e = e0 + u * NT;
      if (e >= total) break;
      const int r = e / g.nx, i = e - r * g.nx;
      const int row = row0 + r;
      const int z = row / g.ny, y = row - z * g.ny;
      const float3 h = xi_cell<E, S>(sm, r, i);
      if (hd_out) hd_out[idx[u]] = make_float4(h.x, h.y, h.z, 0.f);
      local_cell_in<MODE, DMI>(io, g, c, i, y, z, idx[u], h, v[u], flag);
    }
  }
}

template <int E, int S, int R, int NT, bool DMI>
__global__ void __launch_bounds__(NT) xr_kernel(float2* __restrict__ w1, Grid g, float ms,
                                                const float* __restrict__ ms_map, const float2* __restrict__ twM,
                                                const float2* __restrict__ twP, StageIO io, LocalCoef c, int mode,
                                                int xf_next, float4* __restrict__ hd_out, int* flag) {
  extern __shared__ float2 sm[];
  const int row0 = blockIdx.x * R;
  pdl_wait();
  xi_rows<E, S, R, NT>(sm, w1, g, row0, twM, twP);
  switch (mode) {
    case LM_RK4_S0: xr_cells<LM_RK4_S0, DMI, E, S, R, NT>(sm, io, g, c, row0, hd_out, flag); break;
    case LM_RK4_S1: xr_cells<LM_RK4_S1, DMI, E, S, R, NT>(sm, io, g, c, row0, hd_out, flag); break;
    case LM_RK4_S2: xr_cells<LM_RK4_S2, DMI, E, S, R, NT>(sm, io, g, c, row0, hd_out, flag); break;
    default: xr_cells<LM_RK4_S3, DMI, E, S, R, NT>(sm, io, g, c, row0, hd_out, flag); break;
  }
  if (!xf_next) return;
  __syncthreads();  // the block's io.out rows are written; the c2r lines are read
  xf_rows<E, S, R, NT, true>(sm, io.out, g, ms, ms_map, w1, row0, twM, twP);
}

// ---------------------------------------------------------------------------
// y transform + tensor multiply + inverse y of a one-z-plane spectrum
// (Pz == 1, so no z transform and N_xz = N_yz = 0), T kx columns per block,
// small-grid layout w1[c][y][kx].  The Py-point transform of the zero-padded
// column (inputs y < ny <= Py/2) splits into its even outputs, a Py/2-point
// FFT of x, and its odd outputs, a Py/2-point FFT of x W_Py^y; the inverse
// restricted to y < ny is even + W_Py^-y odd.  Lines (c, t, half) of LH =
// Py/2 points run the register line FFT, S threads each.
// ---------------------------------------------------------------------------
template <int E, int S, int T, int NT>
__global__ void __launch_bounds__(NT) yz2d_kernel(float2* __restrict__ w1, Grid g, const float* __restrict__ nhat,
                                                  const float2* __restrict__ twH,
                                                  const float2* __restrict__ twPy) {
  constexpr int LH = E * S;
  constexpr int PITCH = LineFft<E, S>::kPitch;
  constexpr int NF = 6 * T * S;  // threads of the FFT phases (whole warps, or S == 1)
  static_assert(NT >= NF && NT % 32 == 0 && (NF % 32 == 0 || S == 1), "yz2d thread count");
  extern __shared__ __align__(16) float2 sm[];
  float2* twS = sm + 6 * T * PITCH;  // W_LH^(s k) at [k S + s]
  float2* twS2 = twS + LH;           // W_Py^y, y < LH
  const int kx0 = blockIdx.x * T;
  const int tid = threadIdx.x;
  const int ny = g.ny;
  const long wc = (long)g.ny * g.Hx;  // component stride of w1 (one z plane)
  for (int q = tid; q < LH; q += NT) {
    twS[q] = __ldg(&twH[(q % S) * (q / S)]);
    twS2[q] = __ldg(&twPy[q]);
  }
  // this thread's tensor entries for the multiply below (constants, so read
  // while the previous kernel may still run)
  constexpr int NMUL = T * 2 * LH, KM = (NMUL + NT - 1) / NT;
  const long no = (long)g.Hx * g.Oy * g.Oz;
  float4 nt[KM];
#pragma unroll
  for (int u = 0; u < KM; ++u) {
    const int e = tid + u * NT;
    const int j = e % LH, h = (e / LH) % 2, t = e / (2 * LH);
    const int kx = kx0 + t;
    nt[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < NMUL && kx < g.Hx) {
      const int ky = 2 * j + h;
      const bool fy = ky > (g.Py >> 1);
      const long o = (long)(fy ? g.Py - ky : ky) * g.Hx + kx;
      nt[u] = make_float4(__ldg(&nhat[o]), __ldg(&nhat[no + o]), __ldg(&nhat[2 * no + o]),
                          (fy ? -1.f : 1.f) * __ldg(&nhat[3 * no + o]));
    }
  }
  pdl_wait();  // the tables are constants; w1 is the previous kernel's
  __syncthreads();
  // line (c, t, h) at ((c T + t) 2 + h) PITCH; every load of a thread in flight at once
  {
    constexpr int NE = 3 * T * LH, KB = (NE + NT - 1) / NT;
    float2 v[KB];
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int e = tid + u * NT;
      const int t = e % T, y = (e / T) % LH, c = e / (T * LH);
      const int kx = kx0 + t;
      v[u] = (e < NE && y < ny && kx < g.Hx) ? w1[c * wc + (long)y * g.Hx + kx] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < KB; ++u) {
      const int e = tid + u * NT;
      if (e >= NE) break;
      const int t = e % T, y = (e / T) % LH, c = e / (T * LH);
      float2* L = sm + ((c * T + t) * 2) * PITCH;
      L[y] = v[u];
      L[PITCH + y] = cmul(v[u], twS2[y]);
    }
  }
  __syncthreads();
  if (tid < NF) line_fft<E, S, false, true, true>(sm + (tid / S) * PITCH, tid % S, twS);
  __syncthreads();
#pragma unroll
  for (int u = 0; u < KM; ++u) {
    const int e = tid + u * NT;
    const int j = e % LH, h = (e / LH) % 2, t = e / (2 * LH);
    const int kx = kx0 + t;
    if (e >= NMUL || kx >= g.Hx) continue;
    const float nxx = nt[u].x, nyy = nt[u].y, nzz = nt[u].z, nxy = nt[u].w;
    float2* px = sm + ((0 * T + t) * 2 + h) * PITCH + j;
    float2* py = sm + ((1 * T + t) * 2 + h) * PITCH + j;
    float2* pz = sm + ((2 * T + t) * 2 + h) * PITCH + j;
    const float2 mx = *px, my = *py, mz = *pz;
    *px = make_float2(nxx * mx.x + nxy * my.x, nxx * mx.y + nxy * my.y);
    *py = make_float2(nxy * mx.x + nyy * my.x, nxy * mx.y + nyy * my.y);
    *pz = make_float2(nzz * mz.x, nzz * mz.y);
  }
  __syncthreads();
  if (tid < NF) line_fft<E, S, true, true, true>(sm + (tid / S) * PITCH, tid % S, twS);
  __syncthreads();
  for (int e = tid; e < 3 * T * ny; e += NT) {
    const int t = e % T, y = (e / T) % ny, c = e / (T * ny);
    const int kx = kx0 + t;
    if (kx >= g.Hx) continue;
    const float2* L = sm + ((c * T + t) * 2) * PITCH;
    w1[c * wc + (long)y * g.Hx + kx] = cadd(L[y], cmul(L[PITCH + y], cconj(twS2[y])));
  }
}

// 384 threads per block at least: most of them only load, multiply and store
template <int E, int S, int T>
static mx_status yz2d_run(mx_ctx* ctx, cudaStream_t st, bool setup) {
  constexpr int NT = 6 * T * S > 384 ? 6 * T * S : 384;
  const size_t sm = sizeof(float2) * (6 * T * LineFft<E, S>::kPitch + 2 * E * S);
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(yz2d_kernel<E, S, T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  launch_pdl(yz2d_kernel<E, S, T, NT>, dim3((ctx->g.Hx + T - 1) / T), dim3(NT), sm, st, ctx->w1, ctx->g,
             ctx->nhat, ctx->tw_yh, ctx->tw_y);
  return launch_check("yz2d_kernel");
}

static mx_status yz2d_dispatch(mx_ctx* ctx, cudaStream_t st, bool setup) {
  switch (ctx->g.Py / 2) {
    case 512: return yz2d_run<32, 16, 2>(ctx, st, setup);
    case 256: return yz2d_run<16, 16, 2>(ctx, st, setup);
    case 128: return yz2d_run<16, 8, 2>(ctx, st, setup);
    case 64: return yz2d_run<8, 8, 2>(ctx, st, setup);
    case 32: return yz2d_run<32, 1, 8>(ctx, st, setup);
    case 16: return yz2d_run<16, 1, 8>(ctx, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

mx_status yz2d_pass(mx_ctx* ctx, cudaStream_t st) { return yz2d_dispatch(ctx, st, false); }

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
template <int E, int S, int R> static size_t x_smem() {
  return sizeof(float2) * XfShape<S, R>::lines * LineFft<E, S>::kPitch;
}
template <int E, int S, int R, int NT>
static mx_status run_xf(mx_ctx* ctx, const float4* m, cudaStream_t st, bool setup) {
  const size_t sm = x_smem<E, S, R>();
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(xf_kernel<E, S, R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nrows = g.ny * g.nz;
  launch_pdl(xf_kernel<E, S, R, NT>, dim3((nrows + R - 1) / R), dim3(NT), sm, st, m, g, (float)ctx->p.Ms,
             ctx->ms_map, ctx->w1, ctx->tw_m, ctx->tw_x);
  return launch_check("xf_kernel");
}

template <int E, int S, int R, int NT>
static mx_status run_xi(mx_ctx* ctx, float4* hd, cudaStream_t st, bool setup) {
  const size_t sm = x_smem<E, S, R>();
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(xi_kernel<E, S, R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nrows = g.ny * g.nz;
  launch_pdl(xi_kernel<E, S, R, NT>, dim3((nrows + R - 1) / R), dim3(NT), sm, st, ctx->w1, g, hd, ctx->tw_m,
             ctx->tw_x);
  return launch_check("xi_kernel");
}

template <int E, int S, int R, int NT>
static mx_status run_xr(mx_ctx* ctx, int mode, const StageIO& io, bool xf_next, float4* hd_out, cudaStream_t st,
                        bool setup) {
  const size_t sm = x_smem<E, S, R>();
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(xr_kernel<E, S, R, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm));
    MX_CUDA_TRY(cudaFuncSetAttribute(xr_kernel<E, S, R, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nrows = g.ny * g.nz;
  const LocalCoef c = local_coef(ctx);
  const dim3 grid((nrows + R - 1) / R);
  if (c.dmi)
    launch_pdl(xr_kernel<E, S, R, NT, true>, grid, dim3(NT), sm, st, ctx->w1, g, (float)ctx->p.Ms, ctx->ms_map,
               ctx->tw_m, ctx->tw_x, io, c, mode, xf_next ? 1 : 0, hd_out, ctx->flag);
  else
    launch_pdl(xr_kernel<E, S, R, NT, false>, grid, dim3(NT), sm, st, ctx->w1, g, (float)ctx->p.Ms, ctx->ms_map,
               ctx->tw_m, ctx->tw_x, io, c, mode, xf_next ? 1 : 0, hd_out, ctx->flag);
  return launch_check("xr_kernel");
}

// x pass for M = Px/2 (returns MX_ERR_UNSUPPORTED when no specialisation fits).
// Each size has a many-rows-per-block variant and a few-rows one; grids whose
// row count would give fewer than two blocks per SM with the first take the
// second (set-up prepares both).  The few-rows variant runs kFewRowsNT
// threads, most of which only load and store.

template <int E, int S, int RB, int RS>
static mx_status x_pass_rs(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup) {
  constexpr int NB = XfShape<S, RB>::NF;
  constexpr int NS = XfShape<S, RS>::NF > kFewRowsNT ? XfShape<S, RS>::NF : kFewRowsNT;
  if (setup) {
    mx_status s = run_xi<E, S, RB, NB>(ctx, hd, st, true);
    if (s == MX_OK) s = run_xf<E, S, RB, NB>(ctx, m, st, true);
    if (s == MX_OK) s = run_xi<E, S, RS, NS>(ctx, hd, st, true);
    if (s == MX_OK) s = run_xf<E, S, RS, NS>(ctx, m, st, true);
    return s;
  }
  if (!few_rows(ctx->g))
    return inverse ? run_xi<E, S, RB, NB>(ctx, hd, st, false) : run_xf<E, S, RB, NB>(ctx, m, st, false);
  return inverse ? run_xi<E, S, RS, NS>(ctx, hd, st, false) : run_xf<E, S, RS, NS>(ctx, m, st, false);
}

// The row kernel exists for the few-row blocks only (grids whose x passes
// have fewer blocks than two per SM, where the step is bound by its kernel
// boundaries); MX_ERR_UNSUPPORTED for the others.
struct XrLaunch {
  mx_ctx* ctx;
  int mode;
  const StageIO* io;
  bool xf_next;
  float4* hd_out;
  cudaStream_t st;
  bool setup;
  template <int E, int S, int R, int NT> mx_status run() {
    return run_xr<E, S, R, NT>(ctx, mode, *io, xf_next, hd_out, st, setup);
  }
};

static mx_status xr_pass(mx_ctx* ctx, int mode, const StageIO& io, bool xf_next, float4* hd_out, cudaStream_t st,
                         bool setup) {
  if (!few_rows(ctx->g)) return MX_ERR_UNSUPPORTED;
  XrLaunch L{ctx, mode, &io, xf_next, hd_out, st, setup};
  return few_rows_dispatch(ctx->g.Px / 2, L);
}

static mx_status x_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup) {
  switch (ctx->g.Px / 2) {
    case 1024: return x_pass_rs<32, 32, 2, 1>(ctx, m, hd, inverse, st, setup);
    case 512: return x_pass_rs<32, 16, 4, 1>(ctx, m, hd, inverse, st, setup);
    case 256: return x_pass_rs<16, 16, 4, 1>(ctx, m, hd, inverse, st, setup);
    case 128: return x_pass_rs<16, 8, 8, 1>(ctx, m, hd, inverse, st, setup);
    case 64: return x_pass_rs<8, 8, 8, 2>(ctx, m, hd, inverse, st, setup);
    case 32: return x_pass_rs<32, 1, 32, 4>(ctx, m, hd, inverse, st, setup);
    case 16: return x_pass_rs<16, 1, 32, 4>(ctx, m, hd, inverse, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

mx_status fast_setup(mx_ctx* ctx) {
  MX_TRY(upload_w32());
  ctx->fast_x = ctx->p.demag_path != MX_DEMAG_GENERIC &&
                x_pass(ctx, nullptr, nullptr, false, nullptr, true) == MX_OK &&
                x_pass(ctx, nullptr, nullptr, true, nullptr, true) == MX_OK;
  ctx->yz2d = ctx->fused_yz && ctx->g.Pz == 1 && yz2d_dispatch(ctx, nullptr, true) == MX_OK;
  StageIO none{};
  ctx->xrow = ctx->fast_x && xr_pass(ctx, LM_RK4_S0, none, false, nullptr, nullptr, true) == MX_OK;
  clear_error();
  return MX_OK;
}

mx_status fast_row_stage(mx_ctx* ctx, int mode, const StageIO& io, bool xf_next, float4* hd_out, cudaStream_t st) {
  if (mode < LM_RK4_S0 || mode > LM_RK4_S3) {
    set_error("fast_row_stage: bad mode");
    return MX_ERR_INVALID_ARG;
  }
  return xr_pass(ctx, mode, io, xf_next, hd_out, st, false);
}

mx_status fast_x_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st) {
  return x_pass(ctx, m, hd, inverse, st, false);
}

}  // namespace mx
