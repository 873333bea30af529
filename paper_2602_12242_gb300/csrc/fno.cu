// Fourier-neural-operator demag surrogate of a film (Sec. II-D): lifting
// 3 -> 32 channels, four spectral layers keeping K modes per dimension, a
// 32 -> 128 -> 3 projection; forward, SmoothL1 loss, backward and Adam.
//
//   v_0     = P x + p                               x: normalised m
//   v_{l+1} = act_l(K_l v_l + W_l v_l + w_l)        GELU for l < 3, identity for l = 3
//   K_l v   = irfft2(R_l . rfft2(v) on the kept modes)
//             kept: ky in [0, K) u [H-K, H), kx in [0, K);  Y_o = sum_i X_i R_l[mode][i][o]
//   y       = Q2 gelu(Q1 v_4 + q1) + q2
// H = ny (rows), W = nx (columns); activations are FP32, channels-last
// [b][y][x][32].  Only 2K x K of the H x (W/2+1) Fourier modes are used, so
// the transforms are truncated DFTs, not FFTs: a row pass (W real samples ->
// K complex outputs per channel), a column pass (H -> 2K), the per-mode
// 32 x 32 complex channel mix over the whole batch, then the same two passes
// backwards; the last one is fused with the pointwise W_l v_l + w_l and the
// activation.
//
// Backward.  With g = dL/d(K v) and X_g its truncated rfft2, the filter
// gradient is dR[mode][i][o] = c_kx / (H W) * sum_b conj(X[b][i]) X_g[b][o]
// (c_0 = 1, c_kx = 2: the half spectrum stands for its mirror) and the input
// gradient is the same spectral convolution of g with the conjugate-transposed
// filters R'[mode][o][i] = conj(R[mode][i][o]) (so every pass is reused).
// Pointwise weight gradients are sums over cells of outer products.
#include <math.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace mx {

constexpr int kFC = 32;    // channel width
constexpr int kFH = 128;   // projection hidden width
constexpr int kFL = 4;     // spectral layers
constexpr int kFMaxK = 16; // largest K (block of 32 x 2K threads)
constexpr int kFMaxN = 1024;

__device__ __forceinline__ float fgelu(float y) { return 0.5f * y * (1.f + erff(y * 0.70710678118654752f)); }
__device__ __forceinline__ float fgelu_grad(float y) {
  return 0.5f * (1.f + erff(y * 0.70710678118654752f)) + y * 0.39894228040143268f * expf(-0.5f * y * y);
}

// v0[cell][c] = p[c] + sum_k P[c][k] x[k],  x = (m - mean) / std; x0 keeps x (float4).
__global__ void fno_lift_kernel(const float4* __restrict__ m, long ncells, float3 mean, float3 inv_std,
                                const float* __restrict__ P, const float* __restrict__ p, float4* __restrict__ x0,
                                float* __restrict__ v0) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells * kFC) return;
  const long cell = t / kFC;
  const int c = (int)(t % kFC);
  const float4 a = m[cell];
  const float x = (a.x - mean.x) * inv_std.x, y = (a.y - mean.y) * inv_std.y, z = (a.z - mean.z) * inv_std.z;
  v0[t] = p[c] + P[c * 3] * x + P[c * 3 + 1] * y + P[c * 3 + 2] * z;
  if (x0 && c == 0) x0[cell] = make_float4(x, y, z, 0.f);
}

// Row pass: A[row][kx][c] = sum_x v[row][x][c] e^{-2 pi i kx x / W}, kx < K.
// One block per row of one sample; thread (c, kx).
__global__ void fno_dft_x_kernel(const float* __restrict__ v, float2* __restrict__ A, int W, int K,
                                 const float2* __restrict__ twW) {
  extern __shared__ float fsm[];
  float* row = fsm;                           // [W][32]
  float2* tw = (float2*)(fsm + W * kFC);      // [W]
  const long r = blockIdx.x;
  const float4* src = (const float4*)(v + r * W * kFC);
  for (int q = threadIdx.x; q < W * kFC / 4; q += blockDim.x) ((float4*)row)[q] = src[q];
  for (int q = threadIdx.x; q < W; q += blockDim.x) tw[q] = twW[q];
  __syncthreads();
  const int c = threadIdx.x & 31, kx = threadIdx.x >> 5;
  float re = 0.f, im = 0.f;
  int ph = 0;
  for (int x = 0; x < W; ++x) {
    const float a = row[x * kFC + c];
    const float2 w = tw[ph];
    re = fmaf(a, w.x, re);
    im = fmaf(a, w.y, im);
    ph += kx;
    if (ph >= W) ph -= W;
  }
  A[(r * K + kx) * kFC + c] = make_float2(re, im);
}

// Column pass: X[m][kx][b][c] = sum_y A[b][y][kx][c] e^{-2 pi i ky y / H}, m < 2K,
// ky = m (m < K) or H - 2K + m.  One block per (kx, b); thread (c, m).
__global__ void fno_dft_y_kernel(const float2* __restrict__ A, float2* __restrict__ X, int B, int H, int K,
                                 const float2* __restrict__ twH) {
  __shared__ float2 col[64][kFC];
  const int kx = blockIdx.x, b = blockIdx.y;
  const int c = threadIdx.x & 31, m = threadIdx.x >> 5;
  const int ky = m < K ? m : H - 2 * K + m;
  float re = 0.f, im = 0.f;
  int ph = 0;
  for (int y0 = 0; y0 < H; y0 += 64) {
    const int ny = min(64, H - y0);
    __syncthreads();
    for (int q = threadIdx.x; q < ny * kFC; q += blockDim.x) {
      const int yy = q / kFC, cc = q % kFC;
      col[yy][cc] = A[(((long)b * H + y0 + yy) * K + kx) * kFC + cc];
    }
    __syncthreads();
    for (int yy = 0; yy < ny; ++yy) {
      const float2 a = col[yy][c];
      const float2 w = __ldg(&twH[ph]);
      re = fmaf(a.x, w.x, fmaf(-a.y, w.y, re));
      im = fmaf(a.x, w.y, fmaf(a.y, w.x, im));
      ph += ky;
      if (ph >= H) ph -= H;
    }
  }
  X[(((long)m * K + kx) * B + b) * kFC + c] = make_float2(re, im);
}

// Channel mix per kept mode over the batch: Y[mode][b][o] = sum_i X[mode][b][i] F[i][o]
// with F = R[mode] (forward) or F[o'][i'] = conj(R[mode][i'][o']) (ADJ).
template <bool ADJ>
__global__ void __launch_bounds__(256) fno_mix_kernel(const float2* __restrict__ X, float2* __restrict__ Y,
                                                       const float* __restrict__ R, int B) {
  __shared__ float2 F[kFC][kFC];
  const int mode = blockIdx.x;
  const float2* Rm = (const float2*)(R + (long)mode * kFC * kFC * 2);
  for (int q = threadIdx.x; q < kFC * kFC; q += blockDim.x) {
    const int i = q / kFC, o = q % kFC;  // R[mode][i][o]
    const float2 r = Rm[q];
    if (ADJ)
      F[o][i] = make_float2(r.x, -r.y);
    else
      F[i][o] = r;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float2* Xm = X + (long)mode * B * kFC;
  float2* Ym = Y + (long)mode * B * kFC;
  for (int b = warp; b < B; b += blockDim.x >> 5) {
    const float2 xv = Xm[(long)b * kFC + lane];
    float re = 0.f, im = 0.f;
#pragma unroll 8
    for (int i = 0; i < kFC; ++i) {
      const float xr = __shfl_sync(0xffffffffu, xv.x, i), xi = __shfl_sync(0xffffffffu, xv.y, i);
      const float2 f = F[i][lane];
      re = fmaf(xr, f.x, fmaf(-xi, f.y, re));
      im = fmaf(xr, f.y, fmaf(xi, f.x, im));
    }
    Ym[(long)b * kFC + lane] = make_float2(re, im);
  }
}

// Inverse column pass: A[b][y][kx][o] = sum_m Y[m][kx][b][o] e^{+2 pi i ky y / H}.
// Block (kx, b, 32-row chunk); warp w takes rows y0 + w, y0 + w + 8, ...
__global__ void __launch_bounds__(256) fno_idft_y_kernel(const float2* __restrict__ Y, float2* __restrict__ A, int B,
                                                         int H, int K, const float2* __restrict__ twH) {
  __shared__ float2 col[2 * kFMaxK][kFC];
  const int kx = blockIdx.x, b = blockIdx.y, y0 = blockIdx.z * 32;
  for (int q = threadIdx.x; q < 2 * K * kFC; q += blockDim.x) {
    const int m = q / kFC, o = q % kFC;
    col[m][o] = Y[(((long)m * K + kx) * B + b) * kFC + o];
  }
  __syncthreads();
  const int o = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int y = y0 + w; y < min(H, y0 + 32); y += 8) {
    float re = 0.f, im = 0.f;
    for (int m = 0; m < 2 * K; ++m) {
      const int ky = m < K ? m : H - 2 * K + m;
      const float2 t = __ldg(&twH[(int)(((long)ky * y) % H)]);  // e^{-i theta}; use its conjugate
      const float2 a = col[m][o];
      re = fmaf(a.x, t.x, fmaf(a.y, t.y, re));
      im = fmaf(a.y, t.x, fmaf(-a.x, t.y, im));
    }
    A[(((long)b * H + y) * K + kx) * kFC + o] = make_float2(re, im);
  }
}

// Inverse row pass fused with the pointwise part.  For output channel o of cell x:
//   s = (1/(H W)) [Re A[0][o] + 2 sum_{kx>=1} Re(A[kx][o] e^{+2 pi i kx x / W})]
// FWD: u = s + sum_i Wl[o][i] vin[x][i] + wl[o];  pre = u (if stored); out = act(u)
// BWD: u = s + sum_i Wl[i][o] vin[x][i]  (vin = dL/du of this layer, o = input channel);
//      out = u * gelu'(gpre[x][o]) when gpre is given (the layer below's pre-activation)
template <bool BWD>
__global__ void __launch_bounds__(256) fno_idft_x_kernel(const float2* __restrict__ A, const float* __restrict__ vin,
                                                         const float* __restrict__ Wl, const float* __restrict__ wl,
                                                         float* __restrict__ pre, float* __restrict__ out,
                                                         const float* __restrict__ gpre, int W, int K, float scale,
                                                         int gelu_out, const float2* __restrict__ twW) {
  extern __shared__ float fsm[];
  float* Ws = fsm;                               // [32][32]: Ws[j][lane] multiplies vin[j]
  float2* As = (float2*)(fsm + kFC * kFC);       // [K][32]
  float2* tw = As + kFMaxK * kFC;                // [W]
  const long r = blockIdx.x;
  for (int q = threadIdx.x; q < kFC * kFC; q += blockDim.x) {
    const int j = q / kFC, l = q % kFC;
    Ws[q] = BWD ? Wl[j * kFC + l] : Wl[l * kFC + j];
  }
  for (int q = threadIdx.x; q < K * kFC; q += blockDim.x) {
    const float2 a = A[r * K * kFC + q];
    const float ck = (q / kFC) == 0 ? scale : 2.f * scale;
    As[q] = make_float2(a.x * ck, a.y * ck);
  }
  for (int q = threadIdx.x; q < W; q += blockDim.x) tw[q] = twW[q];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float bias = (!BWD && wl) ? wl[lane] : 0.f;
  for (int x = warp; x < W; x += 8) {
    const long cell = r * W + x;
    const float xin = vin[cell * kFC + lane];
    float u = bias;
#pragma unroll 8
    for (int j = 0; j < kFC; ++j) u = fmaf(Ws[j * kFC + lane], __shfl_sync(0xffffffffu, xin, j), u);
    float s = As[lane].x;
    int ph = x;
    for (int kx = 1; kx < K; ++kx) {
      const float2 t = tw[ph];  // e^{-i theta}: Re(a e^{+i theta}) = a.x t.x + a.y t.y
      const float2 a = As[kx * kFC + lane];
      s = fmaf(a.x, t.x, fmaf(a.y, t.y, s));
      ph += x;
      if (ph >= W) ph -= W;
    }
    u += s;
    if (BWD) {
      if (gpre) u *= fgelu_grad(gpre[cell * kFC + lane]);
      out[cell * kFC + lane] = u;
    } else {
      if (pre) pre[cell * kFC + lane] = u;
      out[cell * kFC + lane] = gelu_out ? fgelu(u) : u;
    }
  }
}

// Projection q = Q2 gelu(Q1 v + q1) + q2 per cell (one thread per cell).
// INFER: h = q * std + mean (float4); else pred = q, and z1 (pre-GELU hidden)
// is stored hidden-major, z1[j * ncells + cell], so a warp's stores coalesce.
template <bool INFER>
__global__ void __launch_bounds__(128) fno_proj_kernel(const float* __restrict__ v, long ncells,
                                                       const float* __restrict__ Q1, const float* __restrict__ q1,
                                                       const float* __restrict__ Q2, const float* __restrict__ q2,
                                                       float* __restrict__ z1, float4* __restrict__ out, float3 mean,
                                                       float3 sd) {
  __shared__ float sQ1[kFH][kFC + 1];
  __shared__ float sq1[kFH];
  __shared__ float sQ2[3][kFH];
  for (int q = threadIdx.x; q < kFH * kFC; q += blockDim.x) sQ1[q / kFC][q % kFC] = Q1[q];
  for (int q = threadIdx.x; q < kFH; q += blockDim.x) sq1[q] = q1[q];
  for (int q = threadIdx.x; q < 3 * kFH; q += blockDim.x) sQ2[q / kFH][q % kFH] = Q2[q];
  __syncthreads();
  const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncells) return;
  float a[kFC];
  const float4* src = (const float4*)(v + cell * kFC);
#pragma unroll
  for (int q = 0; q < kFC / 4; ++q) {
    const float4 t = src[q];
    a[4 * q] = t.x;
    a[4 * q + 1] = t.y;
    a[4 * q + 2] = t.z;
    a[4 * q + 3] = t.w;
  }
  float o0 = q2[0], o1 = q2[1], o2 = q2[2];
  for (int j = 0; j < kFH; ++j) {
    float z = sq1[j];
#pragma unroll
    for (int i = 0; i < kFC; ++i) z = fmaf(sQ1[j][i], a[i], z);
    if (!INFER) z1[(long)j * ncells + cell] = z;
    const float h = fgelu(z);
    o0 = fmaf(sQ2[0][j], h, o0);
    o1 = fmaf(sQ2[1][j], h, o1);
    o2 = fmaf(sQ2[2][j], h, o2);
  }
  if (INFER)
    out[cell] = make_float4(o0 * sd.x + mean.x, o1 * sd.y + mean.y, o2 * sd.z + mean.z, 0.f);
  else
    out[cell] = make_float4(o0, o1, o2, 0.f);
}

// SmoothL1 (beta 1) of pred against the normalised target; g = dL/dpred.
__global__ void fno_loss_kernel(const float4* __restrict__ pred, const float4* __restrict__ h_target, long ncells,
                                float3 mean, float3 inv_std, float inv_count, float4* __restrict__ g,
                                float* __restrict__ loss) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (c < ncells) {
    const float4 p = pred[c];
    const float4 t = h_target[c];
    const float d[3] = {p.x - (t.x - mean.x) * inv_std.x, p.y - (t.y - mean.y) * inv_std.y,
                        p.z - (t.z - mean.z) * inv_std.z};
    float gg[3];
    for (int k = 0; k < 3; ++k) {
      const float a = fabsf(d[k]);
      l += a < 1.f ? 0.5f * d[k] * d[k] : a - 0.5f;
      gg[k] = fminf(fmaxf(d[k], -1.f), 1.f) * inv_count;
    }
    g[c] = make_float4(gg[0], gg[1], gg[2], 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l * inv_count);
}

// Projection backward per cell: dz1[j] = gelu'(z1[j]) sum_k Q2[k][j] g[k];
// dv[i] = sum_j Q1[j][i] dz1[j] (the last spectral layer has no activation).
// z1 and dz1 are hidden-major ([j][cell]).
__global__ void __launch_bounds__(128) fno_proj_bwd_kernel(const float4* __restrict__ g, const float* __restrict__ z1,
                                                           long ncells, const float* __restrict__ Q1,
                                                           const float* __restrict__ Q2, float* __restrict__ dz1,
                                                           float* __restrict__ dv) {
  __shared__ float sQ1[kFH][kFC + 1];
  __shared__ float sQ2[3][kFH];
  for (int q = threadIdx.x; q < kFH * kFC; q += blockDim.x) sQ1[q / kFC][q % kFC] = Q1[q];
  for (int q = threadIdx.x; q < 3 * kFH; q += blockDim.x) sQ2[q / kFH][q % kFH] = Q2[q];
  __syncthreads();
  const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncells) return;
  const float4 gc = g[cell];
  float d[kFC];
#pragma unroll
  for (int i = 0; i < kFC; ++i) d[i] = 0.f;
  for (int j = 0; j < kFH; ++j) {
    const float z = z1[(long)j * ncells + cell];
    const float dz = fgelu_grad(z) * (sQ2[0][j] * gc.x + sQ2[1][j] * gc.y + sQ2[2][j] * gc.z);
    dz1[(long)j * ncells + cell] = dz;
#pragma unroll
    for (int i = 0; i < kFC; ++i) d[i] = fmaf(sQ1[j][i], dz, d[i]);
  }
  float4* dst = (float4*)(dv + cell * kFC);
#pragma unroll
  for (int q = 0; q < kFC / 4; ++q) dst[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
}

// Pointwise weight gradient over cells: dW[m][n] += sum_c A[c][m] f(Bv[c][n]),
// db[m] += sum_c A[c][m]; f = gelu when gelu_b.  A has M used columns of row
// stride lda; Bv has N columns of row stride ldb, or (ldb = 0) is stored
// column-major, Bv[n * ncells + c].  Each block sums a chunk of cells, then adds
// its partial sums with FP32 atomics (the general form; the 128 x 32 and
// 32 x 32 cases take the register-tiled kernel below).
constexpr int kWgTile = 32;
__global__ void __launch_bounds__(256) fno_wgrad_kernel(const float* __restrict__ Av, int M, int lda,
                                                        const float* __restrict__ Bv, int N, int ldb, int gelu_b,
                                                        long ncells, long chunk, float* __restrict__ dW,
                                                        float* __restrict__ db) {
  extern __shared__ float fsm[];
  float* As = fsm;                  // [tile][M]
  float* Bs = fsm + kWgTile * M;    // [tile][N + 1] (last column: 1, for the bias)
  const int NB = N + 1;
  const int nout = M * NB;
  constexpr int kPer = 17;          // outputs per thread (M * (N + 1) <= 256 * 17)
  float acc[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) acc[k] = 0.f;
  const long c0 = (long)blockIdx.x * chunk;
  const long c1 = min(ncells, c0 + chunk);
  for (long t0 = c0; t0 < c1; t0 += kWgTile) {
    const int nt = (int)min((long)kWgTile, c1 - t0);
    __syncthreads();
    for (int q = threadIdx.x; q < kWgTile * M; q += blockDim.x) {
      const int c = q / M, mm = q % M;
      As[q] = c < nt ? Av[(t0 + c) * lda + mm] : 0.f;
    }
    for (int q = threadIdx.x; q < kWgTile * NB; q += blockDim.x) {
      const int c = q / NB, nn = q % NB;
      float b = 0.f;
      if (c < nt) {
        if (nn == N) {
          b = 1.f;
        } else {
          b = ldb ? Bv[(t0 + c) * ldb + nn] : Bv[(long)nn * ncells + t0 + c];
          if (gelu_b) b = fgelu(b);
        }
      }
      Bs[q] = b;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int o = threadIdx.x + k * 256;
      if (o < nout) {
        const int mm = o / NB, nn = o % NB;
        float s = acc[k];
        for (int c = 0; c < kWgTile; ++c) s = fmaf(As[c * M + mm], Bs[c * NB + nn], s);
        acc[k] = s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int o = threadIdx.x + k * 256;
    if (o < nout) {
      const int mm = o / NB, nn = o % NB;
      if (nn == N)
        atomicAdd(&db[mm], acc[k]);
      else
        atomicAdd(&dW[mm * N + nn], acc[k]);
    }
  }
}

// The same sum for M = 128 or 32 rows and N = 32 columns (B with row stride
// N; A with row stride M, or column-major A[m * ncells + c] when A_CM), as a
// register-tiled product: thread (tm, tn) owns rows tm*TM.. and columns
// tn*TN.. and reads TM + TN values per cell for TM*TN FMAs.
template <int M, int N, int TM, int TN, bool A_CM>
__global__ void __launch_bounds__(256) fno_wgrad_tiled_kernel(const float* __restrict__ Av,
                                                              const float* __restrict__ Bv, long ncells, long chunk,
                                                              float* __restrict__ dW, float* __restrict__ db) {
  static_assert((M / TM) * (N / TN) == 256, "one output tile per thread");
  __shared__ __align__(16) float As[kWgTile][M];
  __shared__ __align__(16) float Bs[kWgTile][N];
  const int tm = threadIdx.x % (M / TM), tn = threadIdx.x / (M / TM);
  const int m0 = tm * TM, n0 = tn * TN;
  float acc[TM][TN], bacc[TM];
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    bacc[a] = 0.f;
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.f;
  }
  const long c0 = (long)blockIdx.x * chunk;
  const long c1 = min(ncells, c0 + chunk);
  for (long t0 = c0; t0 < c1; t0 += kWgTile) {
    const int nt = (int)min((long)kWgTile, c1 - t0);
    __syncthreads();
    if (A_CM) {
      // lanes take consecutive cells of one row m (coalesced reads)
      for (int q = threadIdx.x; q < kWgTile * M; q += 256) {
        const int c = q % kWgTile, mm = q / kWgTile;
        As[c][mm] = c < nt ? Av[(long)mm * ncells + t0 + c] : 0.f;
      }
    } else {
      for (int q = threadIdx.x; q < kWgTile * M / 4; q += 256) {
        const int c = q / (M / 4);
        ((float4*)&As[0][0])[q] = c < nt ? ((const float4*)(Av + t0 * M))[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    for (int q = threadIdx.x; q < kWgTile * N / 4; q += 256) {
      const int c = q / (N / 4);
      ((float4*)&Bs[0][0])[q] = c < nt ? ((const float4*)(Bv + t0 * N))[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < kWgTile; ++c) {
      float a[TM], b[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) a[q] = As[c][m0 + q];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = Bs[c][n0 + q];
#pragma unroll
      for (int x = 0; x < TM; ++x) {
        bacc[x] += a[x];
#pragma unroll
        for (int y = 0; y < TN; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
      }
    }
  }
#pragma unroll
  for (int x = 0; x < TM; ++x) {
#pragma unroll
    for (int y = 0; y < TN; ++y) atomicAdd(&dW[(m0 + x) * N + n0 + y], acc[x][y]);
    if (tn == 0) atomicAdd(&db[m0 + x], bacc[x]);
  }
}

// Filter gradient per kept mode: dR[mode][i][o] = s_kx sum_b conj(X[mode][b][i]) Xg[mode][b][o],
// s_kx = (kx == 0 ? 1 : 2) / (H W).  One block of 32 x 32 threads per mode.
__global__ void __launch_bounds__(1024) fno_rgrad_kernel(const float2* __restrict__ X, const float2* __restrict__ Xg,
                                                         float* __restrict__ dR, int B, int K, float scale) {
  __shared__ float2 xs[kFC][kFC];
  __shared__ float2 gs[kFC][kFC];
  const int mode = blockIdx.x, kx = mode % K;
  const int i = threadIdx.x >> 5, o = threadIdx.x & 31;
  const float2* Xm = X + (long)mode * B * kFC;
  const float2* Gm = Xg + (long)mode * B * kFC;
  float re = 0.f, im = 0.f;
  for (int b0 = 0; b0 < B; b0 += kFC) {
    const int nb = min(kFC, B - b0);
    __syncthreads();
    if (i < nb) {
      xs[i][o] = Xm[(long)(b0 + i) * kFC + o];
      gs[i][o] = Gm[(long)(b0 + i) * kFC + o];
    }
    __syncthreads();
    for (int b = 0; b < nb; ++b) {
      const float2 a = xs[b][i], g = gs[b][o];
      re = fmaf(a.x, g.x, fmaf(a.y, g.y, re));  // conj(a) g
      im = fmaf(a.x, g.y, fmaf(-a.y, g.x, im));
    }
  }
  const float s = kx == 0 ? scale : 2.f * scale;
  float2* out = (float2*)(dR + (long)mode * kFC * kFC * 2);
  out[i * kFC + o] = make_float2(re * s, im * s);
}

}  // namespace mx

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct mx_fno {
  int nx, ny, K, max_batch;
  long cells;  // per sample
  long np;
  float* params = nullptr;
  float* grad = nullptr;
  float* am = nullptr;
  float* av = nullptr;
  int adam_t = 0;
  float2* twW = nullptr;
  float2* twH = nullptr;
  float4* x0 = nullptr;
  float* v[mx::kFL + 1] = {};
  float* pre[mx::kFL - 1] = {};
  float2* A = nullptr;
  float2* X[mx::kFL] = {};
  float2* Y = nullptr;
  float2* Xg = nullptr;
  float* z1 = nullptr;
  float* dz1 = nullptr;
  float* du[2] = {};
  float4* pred = nullptr;
  float4* g = nullptr;
  float* loss = nullptr;
  float stats[12] = {0, 0, 0, 1, 1, 1, 0, 0, 0, 1, 1, 1};
};

namespace mx {

struct FnoOffsets {
  long P, p, R[kFL], W[kFL], w[kFL], Q1, q1, Q2, q2, total;
};

static FnoOffsets fno_offsets(int K) {
  FnoOffsets f;
  long o = 0;
  f.P = o; o += kFC * 3;
  f.p = o; o += kFC;
  for (int l = 0; l < kFL; ++l) {
    f.R[l] = o; o += 2L * K * K * kFC * kFC * 2;
    f.W[l] = o; o += kFC * kFC;
    f.w[l] = o; o += kFC;
  }
  f.Q1 = o; o += kFH * kFC;
  f.q1 = o; o += kFH;
  f.Q2 = o; o += 3 * kFH;
  f.q2 = o; o += 3;
  f.total = o;
  return f;
}

static size_t dft_x_smem(int W) { return (size_t)W * kFC * sizeof(float) + (size_t)W * sizeof(float2); }
static size_t idft_x_smem(int W) {
  return (size_t)kFC * kFC * sizeof(float) + (size_t)kFMaxK * kFC * sizeof(float2) + (size_t)W * sizeof(float2);
}

// One spectral layer's transforms: v (real, [rows][W][32]) -> X (kept modes).
static mx_status fno_forward_transform(mx_fno* n, const float* v, float2* X, int B, cudaStream_t st) {
  const int W = n->nx, H = n->ny, K = n->K;
  fno_dft_x_kernel<<<(unsigned)(B * H), kFC * K, dft_x_smem(W), st>>>(v, n->A, W, K, n->twW);
  MX_TRY(launch_check("fno_dft_x_kernel"));
  fno_dft_y_kernel<<<dim3(K, B), kFC * 2 * K, 0, st>>>(n->A, X, B, H, K, n->twH);
  return launch_check("fno_dft_y_kernel");
}

// Y (kept modes) -> A (rows x K), the input of the fused inverse row pass.
static mx_status fno_inverse_columns(mx_fno* n, const float2* Y, int B, cudaStream_t st) {
  const int H = n->ny, K = n->K;
  fno_idft_y_kernel<<<dim3(K, B, (H + 31) / 32), 256, 0, st>>>(Y, n->A, B, H, K, n->twH);
  return launch_check("fno_idft_y_kernel");
}

static mx_status fno_forward(mx_fno* n, const float4* m, int B, bool train, float4* h_out, cudaStream_t st) {
  const FnoOffsets f = fno_offsets(n->K);
  const float* P = n->params;
  const long nc = n->cells * B;
  const float* s = n->stats;
  const int W = n->nx, H = n->ny, K = n->K;
  fno_lift_kernel<<<(unsigned)((nc * kFC + 255) / 256), 256, 0, st>>>(
      m, nc, make_float3(s[0], s[1], s[2]), make_float3(1.f / s[3], 1.f / s[4], 1.f / s[5]), P + f.P, P + f.p,
      train ? n->x0 : nullptr, n->v[0]);
  MX_TRY(launch_check("fno_lift_kernel"));
  const float scale = 1.f / ((float)H * (float)W);
  for (int l = 0; l < kFL; ++l) {
    // inference keeps one spectrum buffer and ping-pongs v[0] / v[1]
    const float* vin = train ? n->v[l] : n->v[l & 1];
    float* vout = train ? n->v[l + 1] : n->v[(l + 1) & 1];
    float2* X = train ? n->X[l] : n->X[0];
    MX_TRY(fno_forward_transform(n, vin, X, B, st));
    fno_mix_kernel<false><<<2 * K * K, 256, 0, st>>>(X, n->Y, P + f.R[l], B);
    MX_TRY(launch_check("fno_mix_kernel"));
    MX_TRY(fno_inverse_columns(n, n->Y, B, st));
    fno_idft_x_kernel<false><<<(unsigned)(B * H), 256, idft_x_smem(W), st>>>(
        n->A, vin, P + f.W[l], P + f.w[l], (train && l < kFL - 1) ? n->pre[l] : nullptr, vout, nullptr, W, K,
        scale, l < kFL - 1 ? 1 : 0, n->twW);
    MX_TRY(launch_check("fno_idft_x_kernel"));
  }
  const float* v4 = train ? n->v[kFL] : n->v[kFL & 1];
  const unsigned pg = (unsigned)((nc + 127) / 128);
  if (train) {
    fno_proj_kernel<false><<<pg, 128, 0, st>>>(v4, nc, P + f.Q1, P + f.q1, P + f.Q2, P + f.q2, n->z1, n->pred,
                                               make_float3(0, 0, 0), make_float3(1, 1, 1));
  } else {
    fno_proj_kernel<true><<<pg, 128, 0, st>>>(v4, nc, P + f.Q1, P + f.q1, P + f.Q2, P + f.q2, nullptr, h_out,
                                              make_float3(s[6], s[7], s[8]), make_float3(s[9], s[10], s[11]));
  }
  return launch_check("fno_proj_kernel");
}

static mx_status fno_wgrad(const float* A, int M, int lda, const float* Bv, int N, int ldb, bool gelu_b, long nc,
                           float* dW, float* db, cudaStream_t st) {
  // about two blocks per SM, each summing a whole number of 32-cell tiles
  long chunk = (nc + 2 * 152 - 1) / (2 * 152);
  chunk = ((chunk + kWgTile - 1) / kWgTile) * kWgTile;
  const unsigned grid = (unsigned)((nc + chunk - 1) / chunk);
  // lda = 0: A column-major (A[m * nc + c]); ldb = 0: B column-major
  if (!gelu_b && ldb == N && N == kFC && M == kFH && lda == 0) {
    fno_wgrad_tiled_kernel<kFH, kFC, 4, 4, true><<<grid, 256, 0, st>>>(A, Bv, nc, chunk, dW, db);
    return launch_check("fno_wgrad_tiled_kernel");
  }
  if (!gelu_b && ldb == N && N == kFC && M == kFC && lda == M) {
    fno_wgrad_tiled_kernel<kFC, kFC, 2, 2, false><<<grid, 256, 0, st>>>(A, Bv, nc, chunk, dW, db);
    return launch_check("fno_wgrad_tiled_kernel");
  }
  if (lda == 0) {
    set_error("fno_wgrad: column-major A is only supported for the 128 x 32 case");
    return MX_ERR_INVALID_ARG;
  }
  if (M * (N + 1) > 256 * 17) {  // outputs per thread of the general kernel
    set_error("fno_wgrad: more than 256 x 17 outputs");
    return MX_ERR_INVALID_ARG;
  }
  const size_t sm = (size_t)kWgTile * (M + N + 1) * sizeof(float);
  fno_wgrad_kernel<<<grid, 256, sm, st>>>(A, M, lda, Bv, N, ldb, gelu_b ? 1 : 0, nc, chunk, dW, db);
  return launch_check("fno_wgrad_kernel");
}

static mx_status fno_backward(mx_fno* n, int B, cudaStream_t st) {
  const FnoOffsets f = fno_offsets(n->K);
  const float* P = n->params;
  float* G = n->grad;
  const long nc = n->cells * B;
  const int W = n->nx, H = n->ny, K = n->K;
  const float scale = 1.f / ((float)H * (float)W);
  const unsigned pg = (unsigned)((nc + 127) / 128);
  // projection: dz1, dv4 (= dL/du_3), then dQ1/dq1 and dQ2/dq2
  fno_proj_bwd_kernel<<<pg, 128, 0, st>>>(n->g, n->z1, nc, P + f.Q1, P + f.Q2, n->dz1, n->du[0]);
  MX_TRY(launch_check("fno_proj_bwd_kernel"));
  MX_TRY(fno_wgrad(n->dz1, kFH, 0, n->v[kFL], kFC, kFC, false, nc, G + f.Q1, G + f.q1, st));
  MX_TRY(fno_wgrad((const float*)n->g, 3, 4, n->z1, kFH, 0, true, nc, G + f.Q2, G + f.q2, st));
  int cur = 0;
  for (int l = kFL - 1; l >= 0; --l) {
    const float* du = n->du[cur];
    float* dnext = n->du[cur ^ 1];
    // pointwise weights of layer l
    MX_TRY(fno_wgrad(du, kFC, kFC, n->v[l], kFC, kFC, false, nc, G + f.W[l], G + f.w[l], st));
    // spectral: X_g, filter gradient, adjoint mix, inverse passes fused with W_l^T du
    MX_TRY(fno_forward_transform(n, du, n->Xg, B, st));
    fno_rgrad_kernel<<<2 * K * K, 1024, 0, st>>>(n->X[l], n->Xg, G + f.R[l], B, K, scale);
    MX_TRY(launch_check("fno_rgrad_kernel"));
    fno_mix_kernel<true><<<2 * K * K, 256, 0, st>>>(n->Xg, n->Y, P + f.R[l], B);
    MX_TRY(launch_check("fno_mix_kernel"));
    MX_TRY(fno_inverse_columns(n, n->Y, B, st));
    fno_idft_x_kernel<true><<<(unsigned)(B * H), 256, idft_x_smem(W), st>>>(
        n->A, du, P + f.W[l], nullptr, nullptr, dnext, l > 0 ? n->pre[l - 1] : nullptr, W, K, scale, 0, n->twW);
    MX_TRY(launch_check("fno_idft_x_kernel"));
    cur ^= 1;
  }
  // lifting layer (no activation): dP, dp from dL/dv_0 and the normalised input
  return fno_wgrad(n->du[cur], kFC, kFC, (const float*)n->x0, 3, 4, false, nc, G + f.P, G + f.p, st);
}

bool fno_matches(const mx_fno* n, const Grid& g) { return n->nx == g.nx && n->ny == g.ny && g.nz == 1; }

mx_status fno_demag(mx_fno* n, const float4* m, float4* h, cudaStream_t st) {
  return fno_forward(n, m, 1, false, h, st);
}

}  // namespace mx

using namespace mx;

extern "C" {

int mx_fno_num_params(int modes) {
  if (modes < 1 || modes > kFMaxK) return -1;
  return (int)fno_offsets(modes).total;
}

mx_status mx_fno_destroy(mx_fno* n) {
  if (!n) return MX_OK;
  std::vector<void*> ptrs = {n->params, n->grad, n->am, n->av, n->twW, n->twH, n->x0, n->A, n->Y, n->Xg,
                             n->z1, n->dz1, n->du[0], n->du[1], n->pred, n->g, n->loss};
  for (int l = 0; l <= kFL; ++l) ptrs.push_back(n->v[l]);
  for (int l = 0; l < kFL - 1; ++l) ptrs.push_back(n->pre[l]);
  for (int l = 0; l < kFL; ++l) ptrs.push_back(n->X[l]);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete n;
  return MX_OK;
}

mx_status mx_fno_create(mx_fno** out, int nx, int ny, int modes, int max_batch) {
  clear_error();
  // the column passes put the batch on the grid's y axis (at most 65535 blocks)
  if (!out || modes < 1 || modes > kFMaxK || nx < 2 * modes || ny < 2 * modes || nx > kFMaxN || ny > kFMaxN ||
      max_batch < 1 || max_batch > 65535) {
    set_error("mx_fno_create: need out != NULL, 1 <= modes <= 16, 2*modes <= nx, ny <= 1024 and "
              "1 <= max_batch <= 65535");
    return MX_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mx_fno* n = new mx_fno();
  n->nx = nx;
  n->ny = ny;
  n->K = modes;
  n->max_batch = max_batch;
  n->cells = (long)nx * ny;
  n->np = fno_offsets(modes).total;
  const long nc = n->cells * max_batch;
  const long nspec = 2L * modes * modes * max_batch * kFC;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  };
  alloc((void**)&n->params, sizeof(float) * n->np);
  alloc((void**)&n->grad, sizeof(float) * n->np);
  alloc((void**)&n->am, sizeof(float) * n->np);
  alloc((void**)&n->av, sizeof(float) * n->np);
  alloc((void**)&n->twW, sizeof(float2) * nx);
  alloc((void**)&n->twH, sizeof(float2) * ny);
  alloc((void**)&n->x0, sizeof(float4) * nc);
  for (int l = 0; l <= kFL; ++l) alloc((void**)&n->v[l], sizeof(float) * nc * kFC);
  for (int l = 0; l < kFL - 1; ++l) alloc((void**)&n->pre[l], sizeof(float) * nc * kFC);
  alloc((void**)&n->A, sizeof(float2) * (size_t)max_batch * ny * modes * kFC);
  for (int l = 0; l < kFL; ++l) alloc((void**)&n->X[l], sizeof(float2) * nspec);
  alloc((void**)&n->Y, sizeof(float2) * nspec);
  alloc((void**)&n->Xg, sizeof(float2) * nspec);
  alloc((void**)&n->z1, sizeof(float) * nc * kFH);
  alloc((void**)&n->dz1, sizeof(float) * nc * kFH);
  alloc((void**)&n->du[0], sizeof(float) * nc * kFC);
  alloc((void**)&n->du[1], sizeof(float) * nc * kFC);
  alloc((void**)&n->pred, sizeof(float4) * nc);
  alloc((void**)&n->g, sizeof(float4) * nc);
  alloc((void**)&n->loss, sizeof(float));
  if (!ok) {
    mx_fno_destroy(n);
    set_error("mx_fno_create: device allocation failed");
    return MX_ERR_OOM;
  }
  // twiddles e^{-2 pi i t / N}, in double on the host
  std::vector<float2> tw((size_t)(nx > ny ? nx : ny));
  auto fill = [&](int N) {
    for (int t = 0; t < N; ++t) {
      const double a = 2.0 * kPi * (double)t / (double)N;
      tw[t] = make_float2((float)cos(a), (float)-sin(a));
    }
  };
  bool okc = true;
  fill(nx);
  okc = okc && cudaMemcpy(n->twW, tw.data(), sizeof(float2) * nx, cudaMemcpyHostToDevice) == cudaSuccess;
  fill(ny);
  okc = okc && cudaMemcpy(n->twH, tw.data(), sizeof(float2) * ny, cudaMemcpyHostToDevice) == cudaSuccess;
  okc = okc && cudaMemset(n->params, 0, sizeof(float) * n->np) == cudaSuccess;
  okc = okc && cudaMemset(n->am, 0, sizeof(float) * n->np) == cudaSuccess;
  okc = okc && cudaMemset(n->av, 0, sizeof(float) * n->np) == cudaSuccess;
  okc = okc && cudaFuncSetAttribute(fno_dft_x_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)dft_x_smem(kFMaxN)) == cudaSuccess;
  okc = okc && cudaFuncSetAttribute(fno_idft_x_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)idft_x_smem(kFMaxN)) == cudaSuccess;
  okc = okc && cudaFuncSetAttribute(fno_idft_x_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)idft_x_smem(kFMaxN)) == cudaSuccess;
  if (!okc) {
    cudaGetLastError();
    mx_fno_destroy(n);
    set_error("mx_fno_create: device set-up failed");
    return MX_ERR_CUDA;
  }
  *out = n;
  return MX_OK;
}

mx_status mx_fno_set_params(mx_fno* n, const float* params, mx_stream_t stream) {
  if (!n || !params) {
    set_error("mx_fno_set_params: NULL argument");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MX_CUDA_TRY(cudaMemcpyAsync(n->params, params, sizeof(float) * n->np, cudaMemcpyDeviceToDevice, st));
  MX_CUDA_TRY(cudaMemsetAsync(n->am, 0, sizeof(float) * n->np, st));
  MX_CUDA_TRY(cudaMemsetAsync(n->av, 0, sizeof(float) * n->np, st));
  n->adam_t = 0;
  return MX_OK;
}

mx_status mx_fno_get_params(const mx_fno* n, float* params, mx_stream_t stream) {
  if (!n || !params) {
    set_error("mx_fno_get_params: NULL argument");
    return MX_ERR_INVALID_ARG;
  }
  MX_CUDA_TRY(cudaMemcpyAsync(params, n->params, sizeof(float) * n->np, cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return MX_OK;
}

mx_status mx_fno_set_normalizer(mx_fno* n, const double stats[12]) {
  if (!n || !stats) {
    set_error("mx_fno_set_normalizer: NULL argument");
    return MX_ERR_INVALID_ARG;
  }
  for (int q = 0; q < 12; ++q) {
    if (!isfinite(stats[q]) || ((q % 6) >= 3 && !(stats[q] > 0))) {
      set_error("mx_fno_set_normalizer: standard deviations must be > 0 and every entry finite");
      return MX_ERR_INVALID_ARG;
    }
  }
  for (int q = 0; q < 12; ++q) n->stats[q] = (float)stats[q];
  return MX_OK;
}

static mx_status fno_check(const mx_fno* n, const float* m, int batch, const char* what) {
  if (!n || !m || batch < 1 || batch > n->max_batch || (((uintptr_t)m) & 15)) {
    set_error(std::string(what) + ": bad network, pointer or batch (1..max_batch)");
    return MX_ERR_INVALID_ARG;
  }
  return MX_OK;
}

mx_status mx_fno_forward(mx_fno* n, const float* m, float* h, int batch, mx_stream_t stream) {
  MX_TRY(fno_check(n, m, batch, "mx_fno_forward"));
  if (!h || (((uintptr_t)h) & 15)) {
    set_error("mx_fno_forward: h must be a 16-byte aligned device pointer");
    return MX_ERR_INVALID_ARG;
  }
  return fno_forward(n, (const float4*)m, batch, false, (float4*)h, (cudaStream_t)stream);
}

mx_status mx_fno_loss_grad(mx_fno* n, const float* m, const float* h_target, int batch, float* loss_out,
                           float* grad_out, mx_stream_t stream) {
  MX_TRY(fno_check(n, m, batch, "mx_fno_loss_grad"));
  if (!h_target || (((uintptr_t)h_target) & 15)) {
    set_error("mx_fno_loss_grad: h_target must be a 16-byte aligned device pointer");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MX_TRY(fno_forward(n, (const float4*)m, batch, true, nullptr, st));
  const long nc = n->cells * batch;
  MX_CUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(float), st));
  MX_CUDA_TRY(cudaMemsetAsync(n->grad, 0, sizeof(float) * n->np, st));
  const float* s = n->stats;
  fno_loss_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
      n->pred, (const float4*)h_target, nc, make_float3(s[6], s[7], s[8]),
      make_float3(1.f / s[9], 1.f / s[10], 1.f / s[11]), 1.f / (3.f * (float)nc), n->g, n->loss);
  MX_TRY(launch_check("fno_loss_kernel"));
  MX_TRY(fno_backward(n, batch, st));
  if (loss_out) MX_CUDA_TRY(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (grad_out)
    MX_CUDA_TRY(cudaMemcpyAsync(grad_out, n->grad, sizeof(float) * n->np, cudaMemcpyDeviceToDevice, st));
  return MX_OK;
}

mx_status mx_fno_adam_step(mx_fno* n, double lr, double weight_decay, mx_stream_t stream) {
  if (!n || !(lr > 0) || !(weight_decay >= 0)) {
    set_error("mx_fno_adam_step: need a network, lr > 0 and weight_decay >= 0");
    return MX_ERR_INVALID_ARG;
  }
  n->adam_t += 1;
  return adam_update(n->params, n->grad, n->am, n->av, n->np, lr, weight_decay, n->adam_t, (cudaStream_t)stream);
}

}  // extern "C"
