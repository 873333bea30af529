// Compile-time-sized demag passes (the same arithmetic as demag.cu's generic
// kernels, Sec. II-B: zero-padded FFT convolution with the tensor spectrum),
// built from the register FFTs of regfft.cuh.
//
//   xf<E,S>    r2c along x: M = Px/2 = E*S complex points per row (the real
//              row packed as z[n] = x[2n] + i x[2n+1]) plus the split step.
//   yc<E,S,I>  FFT along y of a tile of T consecutive kx columns; the tile is
//              transposed into shared memory so that each column is one line
//              handled by one warp (or part of one).
//   zc<P>      FFT along z, 3x3 tensor multiply, inverse FFT along z, all in
//              registers.  With only the first P/2 inputs non-zero, the even
//              and odd outputs are two P/2-point FFTs (of x and of x W_P^n); one
//              thread does the even half and its neighbour lane the odd half,
//              and the two inverse halves are added through a lane shuffle.
//   xi<E,S>    c2r along x, cells i < nx written as float4.
#include "common.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "regfft.cuh"

namespace mx {

// tensor multiply shared with the generic kernels (demag.cu)
__device__ __forceinline__ void tmul(float2& mx, float2& my, float2& mz, const float* __restrict__ nhat, const Grid& g,
                                     int kx, int ky, int kz) {
  const bool fy = ky > (g.Py >> 1), fz = kz > (g.Pz >> 1);
  const int qy = fy ? g.Py - ky : ky, qz = fz ? g.Pz - kz : kz;
  const long no = (long)g.Hx * g.Oy * g.Oz;
  const long o = ((long)qz * g.Oy + qy) * g.Hx + kx;
  const float nxx = __ldg(&nhat[o]), nyy = __ldg(&nhat[no + o]), nzz = __ldg(&nhat[2 * no + o]);
  const float nxy = (fy ? -1.f : 1.f) * __ldg(&nhat[3 * no + o]);
  float nxz = 0.f, nyz = 0.f;
  if (g.Pz > 1) {
    nxz = (fz ? -1.f : 1.f) * __ldg(&nhat[4 * no + o]);
    nyz = ((fy != fz) ? -1.f : 1.f) * __ldg(&nhat[5 * no + o]);
  }
  const float2 hx = make_float2(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
  const float2 hy = make_float2(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
  const float2 hz = make_float2(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
  mx = hx;
  my = hy;
  mz = hz;
}

// ---------------------------------------------------------------------------
// x forward (r2c), R rows per block, 3R lines of M = E*S points.
// ---------------------------------------------------------------------------
template <int E, int S, int R>
__global__ void __launch_bounds__(3 * R * S) xf_kernel(const float4* __restrict__ m, Grid g, float ms,
                                                       const float* __restrict__ ms_map, float2* __restrict__ w1,
                                                       const float2* __restrict__ twM, const float2* __restrict__ twP) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch;
  constexpr int NT = 3 * R * S;
  extern __shared__ float2 sm[];
  const int nrows = g.ny * g.nz;
  const int row0 = blockIdx.x * R;
  const int tid = threadIdx.x;
  for (int e = tid; e < R * M; e += NT) {
    const int r = e / M, n = e % M;
    const int row = row0 + r;
    float2 zx = make_float2(0.f, 0.f), zy = zx, zz = zx;
    if (row < nrows) {
      const long cell = (long)row * g.nx;
      const int i0 = 2 * n, i1 = i0 + 1;
      if (i0 < g.nx) {
        const float4 a = __ldg(&m[cell + i0]);
        const float s = ms_map ? __ldg(&ms_map[cell + i0]) : ms;
        zx.x = s * a.x; zy.x = s * a.y; zz.x = s * a.z;
      }
      if (i1 < g.nx) {
        const float4 b = __ldg(&m[cell + i1]);
        const float s = ms_map ? __ldg(&ms_map[cell + i1]) : ms;
        zx.y = s * b.x; zy.y = s * b.y; zz.y = s * b.z;
      }
    }
    sm[(3 * r + 0) * P + n] = zx;
    sm[(3 * r + 1) * P + n] = zy;
    sm[(3 * r + 2) * P + n] = zz;
  }
  __syncthreads();
  line_fft<E, S, false>(sm + (tid / S) * P, tid % S, twM);
  __syncthreads();
  const long cs = (long)g.nz * g.ny * g.Hx;
  for (int e = tid; e < 3 * R * (M + 1); e += NT) {
    const int line = e / (M + 1), k = e % (M + 1);
    const int r = line / 3, c = line % 3;
    const int row = row0 + r;
    if (row >= nrows) continue;
    const float2* L = sm + line * P;
    const float2 zk = L[k == M ? 0 : k];
    const float2 zc = cconj(L[k == 0 ? 0 : M - k]);
    const float2 Ev = cscale(cadd(zk, zc), 0.5f);
    const float2 D = csub(zk, zc);
    const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);
    w1[c * cs + (long)row * g.Hx + k] = cadd(Ev, cmul(__ldg(&twP[k]), O));
  }
}

// ---------------------------------------------------------------------------
// x inverse (c2r).
// ---------------------------------------------------------------------------
template <int E, int S, int R>
__global__ void __launch_bounds__(3 * R * S) xi_kernel(const float2* __restrict__ w1, Grid g, float4* __restrict__ hd,
                                                       const float2* __restrict__ twM, const float2* __restrict__ twP) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch;
  constexpr int NT = 3 * R * S;
  extern __shared__ float2 sm[];
  const int nrows = g.ny * g.nz;
  const int row0 = blockIdx.x * R;
  const int tid = threadIdx.x;
  const long cs = (long)g.nz * g.ny * g.Hx;
  for (int e = tid; e < 3 * R * M; e += NT) {
    const int line = e / M, k = e % M;
    const int r = line / 3, c = line % 3;
    const int row = row0 + r;
    float2 z = make_float2(0.f, 0.f);
    if (row < nrows) {
      const float2* X = w1 + c * cs + (long)row * g.Hx;
      const float2 a = __ldg(&X[k]);
      const float2 b = cconj(__ldg(&X[M - k]));
      const float2 Sv = cadd(a, b);
      const float2 t = cmul(cconj(__ldg(&twP[k])), csub(a, b));
      z = make_float2(Sv.x - t.y, Sv.y + t.x);
    }
    sm[line * P + k] = z;
  }
  __syncthreads();
  line_fft<E, S, true>(sm + (tid / S) * P, tid % S, twM);
  __syncthreads();
  for (int e = tid; e < R * g.nx; e += NT) {
    const int r = e / g.nx, i = e % g.nx;
    const int row = row0 + r;
    if (row >= nrows) continue;
    const float2* L = sm + (3 * r) * P;
    const int n = i >> 1;
    const bool odd = i & 1;
    const float hx = odd ? L[n].y : L[n].x;
    const float hy = odd ? L[P + n].y : L[P + n].x;
    const float hz = odd ? L[2 * P + n].y : L[2 * P + n].x;
    hd[(long)row * g.nx + i] = make_float4(hx, hy, hz, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Column FFT along y: T columns per block, one line (column) per S threads.
// src rows [0, nin) are read (the rest are zero), dst rows [0, nout) written.
// ---------------------------------------------------------------------------
template <int E, int S, int T> struct YcShape {
  static constexpr int L = E * S;
  static constexpr int R = (32 / T) > 0 ? 32 / T : 1;  // rows per warp in the transposing copy
  static constexpr int base = LineFft<E, S>::kPitch;
  static constexpr int pitch = base + (((R - base % 16) % 16) + 16) % 16;
};

template <int E, int S, int T, bool INV>
__global__ void __launch_bounds__(T * S) yc_kernel(const float2* __restrict__ src, float2* __restrict__ dst, Grid g,
                                                   int nin, int nout, const float2* __restrict__ twL) {
  constexpr int L = E * S;
  constexpr int P = YcShape<E, S, T>::pitch;
  constexpr int NT = T * S;
  extern __shared__ float2 sm[];
  const int ntile = (g.Hx + T - 1) / T;
  const int kx0 = (blockIdx.x % ntile) * T;
  const int ck = blockIdx.x / ntile;  // c * nz + k
  const int tid = threadIdx.x;
  const float2* s0 = src + (long)ck * nin * g.Hx + kx0;
  for (int e = tid; e < L * T; e += NT) {
    const int y = e / T, c = e % T;
    float2 v = make_float2(0.f, 0.f);
    if (y < nin && kx0 + c < g.Hx) v = __ldg(&s0[(long)y * g.Hx + c]);
    sm[c * P + y] = v;
  }
  __syncthreads();
  line_fft<E, S, INV>(sm + (tid / S) * P, tid % S, twL);
  __syncthreads();
  float2* d0 = dst + (long)ck * nout * g.Hx + kx0;
  for (int e = tid; e < nout * T; e += NT) {
    const int y = e / T, c = e % T;
    if (kx0 + c < g.Hx) d0[(long)y * g.Hx + c] = sm[c * P + y];
  }
}

// ---------------------------------------------------------------------------
// z FFT + tensor multiply + inverse z, registers only.  Two lanes per
// (kx, ky) column: lane parity h selects the even (h = 0) or odd (h = 1)
// output frequencies kz = 2q + h.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(256) zc_kernel(float2* __restrict__ w2, Grid g, const float* __restrict__ nhat,
                                                 const float2* __restrict__ twz) {
  constexpr int H = P / 2;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long col = gid >> 1;
  const int h = (int)(gid & 1);
  const long ncol = (long)g.Py * g.Hx;
  const bool live = col < ncol;
  const int kx = live ? (int)(col % g.Hx) : 0;
  const int ky = live ? (int)(col / g.Hx) : 0;
  const long zs = (long)g.Py * g.Hx;        // stride between z planes
  const long cs = (long)g.nz * zs;          // stride between components
  const long base = (long)ky * g.Hx + kx;
  float2 v[3][H];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int n = 0; n < H; ++n) {
      float2 x = make_float2(0.f, 0.f);
      if (live && n < g.nz) x = w2[c * cs + n * zs + base];
      if (h) x = cmul(x, __ldg(&twz[n]));
      v[c][n] = x;
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) RegFft<H, false>::run(v[c]);
  if (live) {
#pragma unroll
    for (int q = 0; q < H; ++q) tmul(v[0][q], v[1][q], v[2][q], nhat, g, kx, ky, 2 * q + h);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) RegFft<H, true>::run(v[c]);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int n = 0; n < H; ++n) {
      float2 x = v[c][n];
      if (h) x = cmul(x, cconj(__ldg(&twz[n])));
      float2 o;
      o.x = __shfl_xor_sync(0xffffffffu, x.x, 1);
      o.y = __shfl_xor_sync(0xffffffffu, x.y, 1);
      x = cadd(x, o);
      if (live && n < g.nz && (n & 1) == h) w2[c * cs + n * zs + base] = x;
    }
}

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------
template <int E, int S> static size_t x_smem(int R) { return sizeof(float2) * 3 * R * LineFft<E, S>::kPitch; }
template <int E, int S, int T> static size_t y_smem() { return sizeof(float2) * T * YcShape<E, S, T>::pitch; }

template <int E, int S, int R>
static mx_status run_xf(mx_ctx* ctx, const float4* m, cudaStream_t st, bool setup) {
  const size_t sm = x_smem<E, S>(R);
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(xf_kernel<E, S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nrows = g.ny * g.nz;
  xf_kernel<E, S, R><<<(nrows + R - 1) / R, 3 * R * S, sm, st>>>(m, g, (float)ctx->p.Ms, ctx->ms_map, ctx->w1,
                                                                 ctx->tw_m, ctx->tw_x);
  return launch_check("xf_kernel");
}

template <int E, int S, int R>
static mx_status run_xi(mx_ctx* ctx, float4* hd, cudaStream_t st, bool setup) {
  const size_t sm = x_smem<E, S>(R);
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(xi_kernel<E, S, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nrows = g.ny * g.nz;
  xi_kernel<E, S, R><<<(nrows + R - 1) / R, 3 * R * S, sm, st>>>(ctx->w1, g, hd, ctx->tw_m, ctx->tw_x);
  return launch_check("xi_kernel");
}

template <int E, int S, int T>
static mx_status run_yc(mx_ctx* ctx, bool inv, cudaStream_t st, bool setup) {
  const size_t sm = y_smem<E, S, T>();
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(yc_kernel<E, S, T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    MX_CUDA_TRY(cudaFuncSetAttribute(yc_kernel<E, S, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nblk = 3 * g.nz * ((g.Hx + T - 1) / T);
  if (!inv)
    yc_kernel<E, S, T, false><<<nblk, T * S, sm, st>>>(ctx->w1, ctx->w2, g, g.ny, g.Py, ctx->tw_y);
  else
    yc_kernel<E, S, T, true><<<nblk, T * S, sm, st>>>(ctx->w2, ctx->w1, g, g.Py, g.ny, ctx->tw_y);
  return launch_check("yc_kernel");
}

template <int P>
static mx_status run_zc(mx_ctx* ctx, cudaStream_t st) {
  const Grid& g = ctx->g;
  const long threads = 2L * g.Py * g.Hx;
  zc_kernel<P><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(ctx->w2, g, ctx->nhat, ctx->tw_z);
  return launch_check("zc_kernel");
}

// x pass for M = Px/2 (returns MX_ERR_UNSUPPORTED when no specialisation fits)
static mx_status x_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup) {
  const int M = ctx->g.Px / 2;
#define MX_X(E_, S_, R_)                                                               \
  return inverse ? run_xi<E_, S_, R_>(ctx, hd, st, setup) : run_xf<E_, S_, R_>(ctx, m, st, setup)
  switch (M) {
    case 1024: MX_X(32, 32, 2);
    case 512: MX_X(32, 16, 4);
    case 256: MX_X(16, 16, 4);
    case 128: MX_X(16, 8, 8);
    case 64: MX_X(8, 8, 8);
    case 32: MX_X(32, 1, 32);
    case 16: MX_X(16, 1, 32);
    default: break;
  }
#undef MX_X
  return MX_ERR_UNSUPPORTED;
}

static mx_status y_pass(mx_ctx* ctx, bool inverse, cudaStream_t st, bool setup) {
  switch (ctx->g.Py) {
    case 1024: return run_yc<32, 32, 8>(ctx, inverse, st, setup);
    case 512: return run_yc<32, 16, 16>(ctx, inverse, st, setup);
    case 256: return run_yc<16, 16, 16>(ctx, inverse, st, setup);
    case 128: return run_yc<16, 8, 32>(ctx, inverse, st, setup);
    case 64: return run_yc<8, 8, 32>(ctx, inverse, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

static mx_status z_pass(mx_ctx* ctx, cudaStream_t st) {
  switch (ctx->g.Pz) {
    case 32: return run_zc<32>(ctx, st);
    case 16: return run_zc<16>(ctx, st);
    case 8: return run_zc<8>(ctx, st);
    case 4: return run_zc<4>(ctx, st);
    case 2: return run_zc<2>(ctx, st);
    default: return MX_ERR_UNSUPPORTED;
  }
}

mx_status fast_setup(mx_ctx* ctx) {
  MX_TRY(upload_w32());
  ctx->fast_x = x_pass(ctx, nullptr, nullptr, false, nullptr, true) == MX_OK &&
                x_pass(ctx, nullptr, nullptr, true, nullptr, true) == MX_OK;
  ctx->fast_yz = !ctx->fused_yz && y_pass(ctx, false, nullptr, true) == MX_OK && ctx->g.Pz >= 2 &&
                 ctx->g.Pz <= 32;
  clear_error();
  return MX_OK;
}

mx_status fast_x_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st) {
  return x_pass(ctx, m, hd, inverse, st, false);
}

mx_status fast_yz_passes(mx_ctx* ctx, cudaStream_t st) {
  {
    ProfScope ps(ctx, KID_Y_FWD, st);
    MX_TRY(y_pass(ctx, false, st, false));
  }
  {
    ProfScope ps(ctx, KID_Z_MUL, st);
    MX_TRY(z_pass(ctx, st));
  }
  {
    ProfScope ps(ctx, KID_Y_INV, st);
    MX_TRY(y_pass(ctx, true, st, false));
  }
  return MX_OK;
}

}  // namespace mx
