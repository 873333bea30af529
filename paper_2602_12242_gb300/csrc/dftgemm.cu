// Split-BF16 DFT-as-GEMM first radix stage of the x transforms (precision
// option MX_FFT_SPLIT_BF16 of the per-kx-plane demag path).
//
// A line of M = 32 S points is transformed in two steps (regfft.cuh): 32-point
// DFTs over the stride-S subsequences x[s + S n], twiddles W_M^(s k1), then
// S-point FFTs.  Here the first step is a real GEMM on the tensor cores:
//   [Re Y; Im Y] (64 x V) = [[Re F, -Im F], [Im F, Re F]] (64 x 64) [Re X; Im X] (64 x V)
// for the V = 3 R S subsequences of a block, F the 32-point DFT matrix.  Both
// operands are split into BF16 parts, a = a_hi + a_lo with a_hi = bf16(a) and
// a_lo = bf16(a - a_hi), and the product is a_hi b_hi + a_hi b_lo + a_lo b_hi
// accumulated in FP32 (the dropped a_lo b_lo and the 16-bit representation
// bound the relative error near 2^-16).  The twiddles, the second step and
// the real-to-complex split stay in FP32.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "mma.cuh"
#include "regfft.cuh"

namespace mx {

constexpr int kDftPitch = 72;  // bf16 elements per row of the A and X tiles (64 + 8 pad)

// The block's V = 192 subsequences: line l = v / S, s = v % S.
template <int S> struct DftShape {
  static constexpr int E = 32;
  static constexpr int M = E * S;
  static constexpr int R = 64 / S;          // rows per block (3R lines, 3RS = 192 vectors)
  static constexpr int NT = 3 * R * S;      // threads
  static constexpr int V = 3 * R * S;       // vectors
  static constexpr int P = LineFft<E, S>::kPitch + 1;
  static constexpr size_t smem_lines = sizeof(float2) * 3 * R * P;
  static constexpr size_t smem_a = sizeof(bf16_t) * 2 * 64 * kDftPitch;
  static constexpr size_t smem_x = sizeof(bf16_t) * 2 * V * kDftPitch;
  static constexpr size_t smem = smem_lines + smem_a + smem_x;
};

// Step 1 by split-BF16 GEMM on the block's lines; writes the twiddled rows
// k1 * (S + 1) + s that line_fft_step2 reads.  A (hi, lo) for the direction is
// in global memory: 2 x [64][64] bf16.
template <int S, bool INV>
__device__ __forceinline__ void dft_stage1(float2* lines, bf16_t* sa, bf16_t* sx, const bf16_t* __restrict__ agl,
                                           const float2* __restrict__ twM) {
  typedef DftShape<S> D;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // A hi/lo into shared memory
  for (int e = tid; e < 2 * 64 * 8; e += D::NT) {
    const int part = e / (64 * 8), row = (e / 8) % 64, ch = e % 8;
    cp_async16(smem_u32(sa + (part * 64 + row) * kDftPitch + ch * 8), agl + (part * 64 + row) * 64 + ch * 8, true);
  }
  // X hi/lo: vector v, k = n (re) and 32 + n (im)
  bf16_t* xh = sx;
  bf16_t* xl = sx + D::V * kDftPitch;
  for (int e = tid; e < D::V * 32; e += D::NT) {
    const int v = e % D::V, n = e / D::V;
    const int l = v / S, s = v % S;
    const float2 x = lines[l * D::P + s + S * n];
    const bf16_t rh = f2bf(x.x), ih = f2bf(x.y);
    xh[v * kDftPitch + n] = rh;
    xh[v * kDftPitch + 32 + n] = ih;
    xl[v * kDftPitch + n] = f2bf(x.x - bf2f(rh));
    xl[v * kDftPitch + 32 + n] = f2bf(x.y - bf2f(ih));
  }
  cp_async_wait_all();
  __syncthreads();
  // warp w: vectors [32 w, 32 w + 32) = 4 n tiles, all 4 m tiles
  float acc[4][4][4];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
  const bf16_t* ah = sa;
  const bf16_t* al = sa + 64 * kDftPitch;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    uint32_t bh[4][2], bl[4][2];
#pragma unroll
    for (int np = 0; np < 2; ++np) {
      const int vrow = warp * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
      const int kof = ks * 16 + ((lane >> 3) & 1) * 8;
      ldsm_x4(smem_u32(xh + vrow * kDftPitch + kof), bh[2 * np][0], bh[2 * np][1], bh[2 * np + 1][0],
              bh[2 * np + 1][1]);
      ldsm_x4(smem_u32(xl + vrow * kDftPitch + kof), bl[2 * np][0], bl[2 * np][1], bl[2 * np + 1][0],
              bl[2 * np + 1][1]);
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      const int arow = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
      const int akof = ks * 16 + (lane >> 4) * 8;
      uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
      ldsm_x4(smem_u32(ah + arow * kDftPitch + akof), h0, h1, h2, h3);
      ldsm_x4(smem_u32(al + arow * kDftPitch + akof), l0, l1, l2, l3);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        mma16816(acc[mt][nt], h0, h1, h2, h3, bh[nt][0], bh[nt][1]);
        mma16816(acc[mt][nt], h0, h1, h2, h3, bl[nt][0], bl[nt][1]);
        mma16816(acc[mt][nt], l0, l1, l2, l3, bh[nt][0], bh[nt][1]);
      }
    }
  }
  __syncthreads();  // every thread has read its line inputs from X (copied); lines may be overwritten
  // rows 16 mt + g (+8): k1 (mt 0, 1 real; mt 2, 3 imaginary), cols: vectors
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k1 = mt * 16 + g + (r >= 2 ? 8 : 0);
        const int v = warp * 32 + nt * 8 + 2 * q + (r & 1);
        const int l = v / S, s = v % S;
        float2 y = make_float2(acc[mt][nt][r], acc[mt + 2][nt][r]);
        if (k1 > 0) {
          float2 w = __ldg(&twM[s * k1]);
          if (INV) w.y = -w.y;
          y = cmul(y, w);
        }
        lines[l * D::P + k1 * (S + 1) + s] = y;
      }
  __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(DftShape<S>::NT) xfk_dft_kernel(const float4* __restrict__ m, Grid g, float ms,
                                                                  const float* __restrict__ ms_map,
                                                                  float2* __restrict__ w1, const bf16_t* __restrict__ agl,
                                                                  const float2* __restrict__ twM,
                                                                  const float2* __restrict__ twP) {
  typedef DftShape<S> D;
  constexpr int M = D::M, P = D::P, R = D::R, NT = D::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = (float2*)smraw;
  bf16_t* sa = (bf16_t*)(smraw + D::smem_lines);
  bf16_t* sx = (bf16_t*)(smraw + D::smem_lines + D::smem_a);
  const int ychunks = (g.ny + R - 1) / R;
  const int z = blockIdx.x / ychunks;
  const int y0 = (blockIdx.x % ychunks) * R;
  const int tid = threadIdx.x;
  for (int e = tid; e < R * M; e += NT) {
    const int r = e / M, n = e % M;
    const int y = y0 + r;
    float2 zx = make_float2(0.f, 0.f), zy = zx, zz = zx;
    if (y < g.ny) {
      const long cell = ((long)z * g.ny + y) * g.nx;
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
  dft_stage1<S, false>(sm, sa, sx, agl, twM);
  line_fft_step2<32, S, false>(sm + (tid / S) * P, tid % S);
  __syncthreads();
  const long plane = 3L * g.nz * g.ny;
  for (int e = tid; e < 3 * R * (M + 1); e += NT) {
    const int r = e % R;
    const int c = (e / R) % 3;
    const int k = e / (3 * R);
    const int y = y0 + r;
    if (y >= g.ny) continue;
    const float2* L = sm + (3 * r + c) * P;
    const float2 zk = L[k == M ? 0 : k];
    const float2 zc = cconj(L[k == 0 ? 0 : M - k]);
    const float2 Ev = cscale(cadd(zk, zc), 0.5f);
    const float2 Dd = csub(zk, zc);
    const float2 O = make_float2(0.5f * Dd.y, -0.5f * Dd.x);
    w1[(long)k * plane + ((long)c * g.nz + z) * g.ny + y] = cadd(Ev, cmul(__ldg(&twP[k]), O));
  }
}

template <int S>
__global__ void __launch_bounds__(DftShape<S>::NT) xik_dft_kernel(const float2* __restrict__ w2, Grid g,
                                                                  float4* __restrict__ hd, const bf16_t* __restrict__ agl,
                                                                  const float2* __restrict__ twM,
                                                                  const float2* __restrict__ twP) {
  typedef DftShape<S> D;
  constexpr int M = D::M, P = D::P, R = D::R, NT = D::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = (float2*)smraw;
  bf16_t* sa = (bf16_t*)(smraw + D::smem_lines);
  bf16_t* sx = (bf16_t*)(smraw + D::smem_lines + D::smem_a);
  const int ychunks = (g.ny + R - 1) / R;
  const int z = blockIdx.x / ychunks;
  const int y0 = (blockIdx.x % ychunks) * R;
  const int tid = threadIdx.x;
  const long plane = 3L * g.nz * g.ny;
  for (int e = tid; e < 3 * R * M; e += NT) {
    const int r = e % R;
    const int c = (e / R) % 3;
    const int k = e / (3 * R);
    const int y = y0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (y < g.ny) {
      const long o = ((long)c * g.nz + z) * g.ny + y;
      const float2 a = __ldg(&w2[(long)k * plane + o]);
      const float2 b = cconj(__ldg(&w2[(long)(M - k) * plane + o]));
      const float2 Sv = cadd(a, b);
      const float2 t = cmul(cconj(__ldg(&twP[k])), csub(a, b));
      v = make_float2(Sv.x - t.y, Sv.y + t.x);
    }
    sm[(3 * r + c) * P + k] = v;
  }
  __syncthreads();
  dft_stage1<S, true>(sm, sa, sx, agl + 2 * 64 * 64, twM);
  line_fft_step2<32, S, true>(sm + (tid / S) * P, tid % S);
  __syncthreads();
  for (int e = tid; e < R * g.nx; e += NT) {
    const int r = e / g.nx, i = e % g.nx;
    const int y = y0 + r;
    if (y >= g.ny) continue;
    const float2* L = sm + (3 * r) * P;
    const int n = i >> 1;
    const bool odd = i & 1;
    const float hx = odd ? L[n].y : L[n].x;
    const float hy = odd ? L[P + n].y : L[P + n].x;
    const float hz = odd ? L[2 * P + n].y : L[2 * P + n].x;
    hd[((long)z * g.ny + y) * g.nx + i] = make_float4(hx, hy, hz, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// float -> bfloat16 bits, round to nearest, ties to even (finite inputs)
static uint16_t host_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
static float host_bf16_to_float(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// [fwd hi, fwd lo, inv hi, inv lo], each [64][64]: rows (Re k, Im k), cols (Re n, Im n)
mx_status dft_gemm_setup(mx_ctx* ctx) {
  std::vector<uint16_t> a(4 * 64 * 64);
  for (int dir = 0; dir < 2; ++dir) {
    const double sgn = dir == 0 ? -1.0 : 1.0;
    for (int k = 0; k < 32; ++k)
      for (int n = 0; n < 32; ++n) {
        const double ang = sgn * 2.0 * kPi * (double)((k * n) % 32) / 32.0;
        const double c = cos(ang), s = sin(ang);
        const double blk[2][2] = {{c, -s}, {s, c}};  // [out re/im][in re/im]
        for (int oi = 0; oi < 2; ++oi)
          for (int ii = 0; ii < 2; ++ii) {
            const float v = (float)blk[oi][ii];
            const uint16_t hi = host_bf16(v);
            const uint16_t lo = host_bf16((float)((double)v - (double)host_bf16_to_float(hi)));
            const int row = oi * 32 + k, col = ii * 32 + n;
            a[(dir * 2 + 0) * 4096 + row * 64 + col] = hi;
            a[(dir * 2 + 1) * 4096 + row * 64 + col] = lo;
          }
      }
  }
  if (!ctx->dft_a) MX_CUDA_TRY(cudaMalloc(&ctx->dft_a, sizeof(uint16_t) * a.size()));
  MX_CUDA_TRY(cudaMemcpy(ctx->dft_a, a.data(), sizeof(uint16_t) * a.size(), cudaMemcpyHostToDevice));
  return MX_OK;
}

template <int S>
static mx_status dft_run(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup) {
  typedef DftShape<S> D;
  if (setup) {
    MX_TRY(upload_w32());  // this unit's copy of the W_32 table (second-step RegFft)
    MX_CUDA_TRY(cudaFuncSetAttribute(xfk_dft_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D::smem));
    MX_CUDA_TRY(cudaFuncSetAttribute(xik_dft_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D::smem));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nblk = g.nz * ((g.ny + D::R - 1) / D::R);
  const bf16_t* A = (const bf16_t*)ctx->dft_a;
  if (!inverse) {
    xfk_dft_kernel<S><<<nblk, D::NT, D::smem, st>>>(m, g, (float)ctx->p.Ms, ctx->ms_map, ctx->w1, A, ctx->tw_m,
                                                    ctx->tw_x);
    return launch_check("xfk_dft_kernel");
  }
  xik_dft_kernel<S><<<nblk, D::NT, D::smem, st>>>(ctx->w2, g, hd, A, ctx->tw_m, ctx->tw_x);
  return launch_check("xik_dft_kernel");
}

// x passes of the plane path with the GEMM first stage; M = Px/2 = 32 S.
mx_status dft_x_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup) {
  switch (ctx->g.Px / 2) {
    case 512: return dft_run<16>(ctx, m, hd, inverse, st, setup);
    case 1024: return dft_run<32>(ctx, m, hd, inverse, st, setup);
    default:
      set_error("split-BF16 DFT stage needs Px/2 = 512 or 1024 (nx in 257..1024)");
      return MX_ERR_UNSUPPORTED;
  }
}

}  // namespace mx
