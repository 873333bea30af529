// Split-BF16 DFT-as-GEMM first radix stage of the x transforms (precision
// option MX_FFT_SPLIT_BF16 of the per-kx-plane demag path), on the tcgen05
// tensor cores with the accumulator in tensor memory.
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
#include "bulk.cuh"
#include "mma.cuh"
#include "regfft.cuh"
#include "tc05.cuh"

namespace mx {

// Operands in the canonical K-major layout without swizzle (tc05.cuh): the
// element (row, k) of a 16-bit matrix with 64 columns of K sits at byte
// (row / 8) * 1024 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2, so core
// matrices adjacent along K are 128 bytes apart (LBO) and 8-row groups 1024
// bytes apart (SBO).
__host__ __device__ constexpr uint32_t dft_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// The block's V = 192 subsequences: line l = v / S, s = v % S.  On the tensor
// cores the GEMM is D (V x 64) = X (V x 64) F^T, vectors along M in two
// 128-row tiles (rows 192..255 of the second are scratch), F (64 x 64) the
// B operand; D lives in tensor memory, 64 FP32 columns per tile.
template <int S> struct DftShape {
  static constexpr int E = 32;
  static constexpr int M = E * S;
  static constexpr int R = 64 / S;          // rows per block (3R lines, 3RS = 192 vectors)
  static constexpr int NT = 3 * R * S;      // threads
  static constexpr int V = 3 * R * S;       // vectors
  static constexpr int VP = 256;            // vectors padded to two M = 128 tiles
  static constexpr int P = LineFft<E, S>::kPitch + 1;
  static constexpr size_t smem_lines = sizeof(float2) * 3 * R * P;
  static constexpr size_t smem_a = 2 * 64 * 64 * 2;      // F hi, lo
  static constexpr size_t smem_x = 2 * VP * 64 * 2;      // X hi, lo
  static constexpr size_t smem = smem_lines + smem_a + smem_x;
  static_assert(V == 192 && NT == 192 && smem_lines % 16 == 0, "DFT stage shape");
};

// Step 1 by split-BF16 GEMM on the block's lines; writes the twiddled rows
// k1 * (S + 1) + s that line_fft_step2 reads.  F (hi, lo) for the direction
// is in global memory: 2 x [64][64] bf16, row = output (Re k, Im k), column
// = input (Re n, Im n).  sa, sx: 16-byte aligned shared buffers; bar, tb:
// the block's mbarrier and tensor-memory base (128 columns, allocated by the
// caller); flag receives kFlagTimeout if the MMAs do not complete in time.
template <int S, bool INV>
__device__ __forceinline__ void dft_stage1(float2* lines, unsigned char* sa, unsigned char* sx,
                                           const bf16_t* __restrict__ agl, const float2* __restrict__ twM,
                                           uint64_t* bar, uint32_t tb, int* flag) {
  typedef DftShape<S> D;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // F hi/lo into shared memory: 16-byte chunk (part, row, ch) = 8 consecutive k
  for (int e = tid; e < 2 * 64 * 8; e += D::NT) {
    const int part = e / (64 * 8), row = (e / 8) % 64, ch = e % 8;
    cp_async16(smem_u32(sa + part * 8192 + dft_off(row, 8 * ch)), agl + (part * 64 + row) * 64 + ch * 8, true);
  }
  // X hi/lo: vector v, k = n (re) and 32 + n (im); a work item is 8
  // consecutive n of one vector, stored as four 16-byte rows of core matrices
  unsigned char* xh = sx;
  unsigned char* xl = sx + D::VP * 128;
  for (int e = tid; e < D::V * 4; e += D::NT) {
    const int v = e % D::V, c = e / D::V;
    const int l = v / S, s = v % S;
    const float2* src = lines + l * D::P + s + S * 8 * c;
    uint32_t rh[4], ih[4], rl[4], il[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 x0 = src[S * (2 * q)], x1 = src[S * (2 * q + 1)];
      const bf16_t r0 = f2bf(x0.x), r1 = f2bf(x1.x), i0 = f2bf(x0.y), i1 = f2bf(x1.y);
      rh[q] = (uint32_t)r0 | ((uint32_t)r1 << 16);
      ih[q] = (uint32_t)i0 | ((uint32_t)i1 << 16);
      rl[q] = pack2(x0.x - bf2f(r0), x1.x - bf2f(r1));
      il[q] = pack2(x0.y - bf2f(i0), x1.y - bf2f(i1));
    }
    *(uint4*)(xh + dft_off(v, 8 * c)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
    *(uint4*)(xh + dft_off(v, 32 + 8 * c)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
    *(uint4*)(xl + dft_off(v, 8 * c)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
    *(uint4*)(xl + dft_off(v, 32 + 8 * c)) = make_uint4(il[0], il[1], il[2], il[3]);
  }
  cp_async_wait_all();
  fence_proxy_async_smem();  // the operands are read by the tensor core (async proxy)
  tc_fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after_sync();
    constexpr uint32_t idesc = tc_idesc_bf16(128, 64);
    const uint32_t a0 = smem_u32(sa), x0 = smem_u32(sx);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      // hi.hi, lo.hi (X part), hi.lo (F part)
#pragma unroll
      for (int pr = 0; pr < 3; ++pr) {
        const uint32_t xb = x0 + (pr == 1 ? D::VP * 128 : 0) + t * 128 * 128;
        const uint32_t fb = a0 + (pr == 2 ? 8192 : 0);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          tc_mma_bf16(tb + t * 64, tc_sdesc(xb + ks * 256, 128, 1024), tc_sdesc(fb + ks * 256, 128, 1024), idesc,
                      pr > 0 || ks > 0);
      }
    }
    tc_commit(bar);
  }
  if (!mbar_wait(bar, 0)) atomicOr(flag, kFlagTimeout);
  tc_fence_after_sync();
  // row v of D: tile warp / 4, lanes of this warp's quarter; 64 columns =
  // (Re k1, Im k1) for k1 < 32.  The lines' inputs were copied into X above.
  const int t = warp >> 2;
  const int v = t * 128 + 32 * (warp & 3) + lane;
  float d[64];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float q[8];
    tmem_ld8(tb + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(t * 64 + 8 * j), q);
#pragma unroll
    for (int i = 0; i < 8; ++i) d[8 * j + i] = q[i];
  }
  if (v < D::V) {
    const int l = v / S, s = v % S;
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) {
      float2 y = make_float2(d[k1], d[32 + k1]);
      if (k1 > 0) {
        float2 w = __ldg(&twM[s * k1]);
        if (INV) w.y = -w.y;
        y = cmul(y, w);
      }
      lines[l * D::P + k1 * (S + 1) + s] = y;
    }
  }
  tc_fence_before_sync();
  __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(DftShape<S>::NT) xfk_dft_kernel(const float4* __restrict__ m, Grid g, float ms,
                                                                  const float* __restrict__ ms_map,
                                                                  float2* __restrict__ w1, const bf16_t* __restrict__ agl,
                                                                  const float2* __restrict__ twM,
                                                                  const float2* __restrict__ twP, int* flag) {
  typedef DftShape<S> D;
  constexpr int M = D::M, P = D::P, R = D::R, NT = D::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  float2* sm = (float2*)smraw;
  unsigned char* sa = smraw + D::smem_lines;
  unsigned char* sx = smraw + D::smem_lines + D::smem_a;
  if (threadIdx.x < 32) tmem_alloc(&tbase, 128);
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  pdl_wait();
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
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tb = tbase;
  dft_stage1<S, false>(sm, sa, sx, agl, twM, &bar, tb, flag);
  if (threadIdx.x < 32) {
    tc_fence_after_sync();
    tmem_dealloc(tb, 128);
  }
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
                                                                  const float2* __restrict__ twP, int* flag) {
  typedef DftShape<S> D;
  constexpr int M = D::M, P = D::P, R = D::R, NT = D::NT;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  float2* sm = (float2*)smraw;
  unsigned char* sa = smraw + D::smem_lines;
  unsigned char* sx = smraw + D::smem_lines + D::smem_a;
  if (threadIdx.x < 32) tmem_alloc(&tbase, 128);
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  pdl_wait();
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
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tb = tbase;
  dft_stage1<S, true>(sm, sa, sx, agl + 2 * 64 * 64, twM, &bar, tb, flag);
  if (threadIdx.x < 32) {
    tc_fence_after_sync();
    tmem_dealloc(tb, 128);
  }
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
    launch_pdl(xfk_dft_kernel<S>, dim3(nblk), dim3(D::NT), D::smem, st, m, g, (float)ctx->p.Ms, ctx->ms_map,
               ctx->w1, A, ctx->tw_m, ctx->tw_x, ctx->flag);
    return launch_check("xfk_dft_kernel");
  }
  launch_pdl(xik_dft_kernel<S>, dim3(nblk), dim3(D::NT), D::smem, st, ctx->w2, g, hd, A, ctx->tw_m, ctx->tw_x,
             ctx->flag);
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
