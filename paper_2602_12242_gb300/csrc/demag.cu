// Demagnetising field by zero-padded FFT convolution (Sec. II-B), FP32.
//
//   H_d = IFFT3( Nhat . FFT3( pad(Ms m) ) ), cropped to the n-region,
// with Nhat the tensor spectrum already scaled by -1/(Px Py Pz).
//
// Passes (spectra are float2, layout [c][k][y][kx], kx fastest, kx < Hx):
//   x_fwd   real-to-complex along x of the padded rows, M = Ms m folded in
//           (length-Px real FFT done as a length-Px/2 complex FFT of the
//           even/odd interleave plus a split step);           m  -> w1
//   yz      (plane fits on chip) one kernel per tile of kx columns: forward
//           y FFT of the n_z planes, forward z FFT, 3x3 tensor multiply,
//           inverse z, inverse y, keep the n_y rows and n_z planes; w1 -> w1
//   y_fwd / z_mul / y_inv  (large planes) the same as three passes
//           through w2 = [c][k][Py][kx];            w1 -> w2 -> w2 -> w1
//   x_inv   complex-to-real along x, keep the n_x cells;       w1 -> H_d
#include "common.cuh"
#include "fft.cuh"
#include "kernels.cuh"

namespace mx {

constexpr int kNT = 256;   // threads per block of every FP32 FFT kernel
constexpr int kEPT = 32;   // complex elements per thread in a pass
constexpr int kCap = kNT * kEPT;

// ---------------------------------------------------------------------------
// x forward: rows (j, k); `rows` rows per block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kNT) x_fwd_kernel(const float4* __restrict__ m, Grid g, float ms,
                                                    const float* __restrict__ ms_map, float2* __restrict__ w1,
                                                    const float2* __restrict__ twx, int rows) {
  extern __shared__ float2 sm[];
  const int nrows_tot = g.ny * g.nz;
  const int row0 = blockIdx.x * rows;
  const int nr = min(rows, nrows_tot - row0);
  const long cstride = (long)g.nz * g.ny * g.Hx;  // component stride in w1
  if (g.Px == 1) {
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const int row = row0 + r;
      const long cell = (long)row * g.nx;
      const float s = ms_map ? ms_map[cell] : ms;
      const float4 v = m[cell];
      w1[0 * cstride + row] = make_float2(s * v.x, 0.f);
      w1[1 * cstride + row] = make_float2(s * v.y, 0.f);
      w1[2 * cstride + row] = make_float2(s * v.z, 0.f);
    }
    return;
  }
  const int M = g.Px / 2;
  // line (r, c) at (r * 3 + c) * M
  for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
    const int r = e / M, n = e % M;
    const long cell = (long)(row0 + r) * g.nx;
    const int i0 = 2 * n, i1 = 2 * n + 1;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    float sa = 0.f, sb = 0.f;
    if (i0 < g.nx) { a = m[cell + i0]; sa = ms_map ? ms_map[cell + i0] : ms; }
    if (i1 < g.nx) { b = m[cell + i1]; sb = ms_map ? ms_map[cell + i1] : ms; }
    float2* L = sm + (r * 3) * M;
    L[n] = make_float2(sa * a.x, sb * b.x);
    L[M + n] = make_float2(sa * a.y, sb * b.y);
    L[2 * M + n] = make_float2(sa * a.z, sb * b.z);
  }
  __syncthreads();
  block_fft<false, float2, kEPT, kNT>(sm, M, 3 * nr, lines1(M), 1, twx, 2);
  // split: X[k] = E[k] + W_Px^k O[k], k = 0..M
  for (int e = threadIdx.x; e < nr * 3 * (M + 1); e += blockDim.x) {
    const int line = e / (M + 1), k = e % (M + 1);
    const float2* L = sm + line * M;
    const float2 zk = L[k == M ? 0 : k];
    const float2 zc = cconj(L[k == 0 ? 0 : M - k]);
    const float2 E = cscale(cadd(zk, zc), 0.5f);
    const float2 D = csub(zk, zc);                       // 2i O
    const float2 O = make_float2(0.5f * D.y, -0.5f * D.x);  // D / (2i)
    const float2 w = __ldg(&twx[k]);
    const float2 X = cadd(E, cmul(w, O));
    const int r = line / 3, c = line % 3;
    const int row = row0 + r;  // row = j + ny k
    w1[c * cstride + (long)row * g.Hx + k] = X;
  }
}

// ---------------------------------------------------------------------------
// x inverse: complex-to-real, cells i < nx written to hd (float4).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kNT) x_inv_kernel(const float2* __restrict__ w1, Grid g, float4* __restrict__ hd,
                                                    const float2* __restrict__ twx, int rows) {
  extern __shared__ float2 sm[];
  const int nrows_tot = g.ny * g.nz;
  const int row0 = blockIdx.x * rows;
  const int nr = min(rows, nrows_tot - row0);
  const long cstride = (long)g.nz * g.ny * g.Hx;
  if (g.Px == 1) {
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      const int row = row0 + r;
      hd[row] = make_float4(w1[row].x, w1[cstride + row].x, w1[2 * cstride + row].x, 0.f);
    }
    return;
  }
  const int M = g.Px / 2;
  // Z[k] = (X[k] + conj X[M-k]) + i W_Px^{-k} (X[k] - conj X[M-k]), k < M
  for (int e = threadIdx.x; e < nr * 3 * M; e += blockDim.x) {
    const int line = e / M, k = e % M;
    const int r = line / 3, c = line % 3;
    const float2* X = w1 + c * cstride + (long)(row0 + r) * g.Hx;
    const float2 a = X[k];
    const float2 b = cconj(X[M - k]);
    const float2 S = cadd(a, b);
    const float2 D = csub(a, b);
    const float2 w = cconj(__ldg(&twx[k]));
    const float2 t = cmul(w, D);
    sm[line * M + k] = make_float2(S.x - t.y, S.y + t.x);  // S + i t
  }
  __syncthreads();
  block_fft<true, float2, kEPT, kNT>(sm, M, 3 * nr, lines1(M), 1, twx, 2);
  for (int e = threadIdx.x; e < nr * g.nx; e += blockDim.x) {
    const int r = e / g.nx, i = e % g.nx;
    const float2* L = sm + (r * 3) * M;
    const int n = i >> 1;
    const bool odd = i & 1;
    const float hx = odd ? L[n].y : L[n].x;
    const float hy = odd ? L[M + n].y : L[M + n].x;
    const float hz = odd ? L[2 * M + n].y : L[2 * M + n].x;
    hd[(long)(row0 + r) * g.nx + i] = make_float4(hx, hy, hz, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Spectral tensor multiply at (kx, ky, kz): the octant store is folded with
// each component's parity (xy odd in ky; xz odd in kz; yz odd in both).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tensor_mul(float2& mx, float2& my, float2& mz, const float* __restrict__ nhat,
                                           const Grid& g, int kx, int ky, int kz, bool has_z) {
  const bool fy = ky > (g.Py >> 1), fz = kz > (g.Pz >> 1);
  const int qy = fy ? g.Py - ky : ky, qz = fz ? g.Pz - kz : kz;
  const long no = (long)g.Hx * g.Oy * g.Oz;
  const long o = ((long)qz * g.Oy + qy) * g.Hx + kx;
  const float nxx = __ldg(&nhat[o]), nyy = __ldg(&nhat[no + o]), nzz = __ldg(&nhat[2 * no + o]);
  const float nxy = (fy ? -1.f : 1.f) * __ldg(&nhat[3 * no + o]);
  float nxz = 0.f, nyz = 0.f;
  if (has_z) {
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
// Fused y/z pass for planes that fit in shared memory: one block per tile of
// T kx columns holds [c][Pz][Py][T].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kNT) yz_fused_kernel(float2* __restrict__ w1, Grid g,
                                                       const float* __restrict__ nhat, const float2* __restrict__ twy,
                                                       const float2* __restrict__ twz, int T) {
  extern __shared__ float2 sm[];
  const int kx0 = blockIdx.x * T;
  const int nt = min(T, g.Hx - kx0);
  const int plane = g.Py * T;          // one z plane of one component
  const int cst = g.Pz * plane;        // component stride in shared memory
  const long wc = (long)g.nz * g.ny * g.Hx;
  // load the n_z x n_y region, zero the padding
  for (int e = threadIdx.x; e < 3 * cst; e += blockDim.x) {
    const int t = e % T;
    const int y = (e / T) % g.Py;
    const int z = (e / plane) % g.Pz;
    const int c = e / cst;
    float2 v = make_float2(0.f, 0.f);
    if (t < nt && y < g.ny && z < g.nz) v = w1[c * wc + ((long)z * g.ny + y) * g.Hx + kx0 + t];
    sm[e] = v;
  }
  __syncthreads();
  const Lines ylines{T, 1, g.nz, plane, cst};
  const Lines zlines{T, 1, g.Py, T, cst};
  block_fft<false, float2, kEPT, kNT>(sm, g.Py, 3 * g.nz * T, ylines, T, twy, 1);
  block_fft<false, float2, kEPT, kNT>(sm, g.Pz, 3 * g.Py * T, zlines, plane, twz, 1);
  const bool has_z = g.Pz > 1;
  for (int e = threadIdx.x; e < cst; e += blockDim.x) {
    const int t = e % T;
    if (t >= nt) continue;
    const int ky = (e / T) % g.Py;
    const int kz = e / plane;
    tensor_mul(sm[e], sm[cst + e], sm[2 * cst + e], nhat, g, kx0 + t, ky, kz, has_z);
  }
  __syncthreads();
  block_fft<true, float2, kEPT, kNT>(sm, g.Pz, 3 * g.Py * T, zlines, plane, twz, 1);
  block_fft<true, float2, kEPT, kNT>(sm, g.Py, 3 * g.nz * T, ylines, T, twy, 1);
  for (int e = threadIdx.x; e < 3 * cst; e += blockDim.x) {
    const int t = e % T;
    const int y = (e / T) % g.Py;
    const int z = (e / plane) % g.Pz;
    const int c = e / cst;
    if (t < nt && y < g.ny && z < g.nz) w1[c * wc + ((long)z * g.ny + y) * g.Hx + kx0 + t] = sm[e];
  }
}

// ---------------------------------------------------------------------------
// Unfused path: y forward (w1 -> w2), z + multiply + inverse z (w2 in place),
// y inverse (w2 -> w1).  Blocks over (c, k, kx tile) or (ky, kx tile).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kNT) y_fwd_kernel(const float2* __restrict__ w1, float2* __restrict__ w2, Grid g,
                                                    const float2* __restrict__ twy, int T) {
  extern __shared__ float2 sm[];
  const int ntile = (g.Hx + T - 1) / T;
  const int kx0 = (blockIdx.x % ntile) * T;
  const int ck = blockIdx.x / ntile;  // c * nz + k
  const int nt = min(T, g.Hx - kx0);
  const float2* src = w1 + (long)ck * g.ny * g.Hx + kx0;
  for (int e = threadIdx.x; e < g.Py * T; e += blockDim.x) {
    const int t = e % T, y = e / T;
    sm[e] = (t < nt && y < g.ny) ? src[(long)y * g.Hx + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  block_fft<false, float2, kEPT, kNT>(sm, g.Py, T, lines1(1), T, twy, 1);
  float2* dst = w2 + (long)ck * g.Py * g.Hx + kx0;
  for (int e = threadIdx.x; e < g.Py * T; e += blockDim.x) {
    const int t = e % T, y = e / T;
    if (t < nt) dst[(long)y * g.Hx + t] = sm[e];
  }
}

__global__ void __launch_bounds__(kNT) z_mul_kernel(float2* __restrict__ w2, Grid g, const float* __restrict__ nhat,
                                                    const float2* __restrict__ twz, int T) {
  extern __shared__ float2 sm[];
  const int ntile = (g.Hx + T - 1) / T;
  const int kx0 = (blockIdx.x % ntile) * T;
  // ky and Py - ky read the same folded tensor rows: order the blocks so the
  // two land next to each other (q even -> q/2, q odd -> Py - 1 - q/2)
  const int q = blockIdx.x / ntile;
  const int ky = (q % 2 == 0) ? q / 2 : g.Py - 1 - q / 2;
  const int nt = min(T, g.Hx - kx0);
  const int cst = g.Pz * T;
  const long wc = (long)g.nz * g.Py * g.Hx;
  for (int e = threadIdx.x; e < 3 * cst; e += blockDim.x) {
    const int t = e % T, z = (e / T) % g.Pz, c = e / cst;
    sm[e] = (t < nt && z < g.nz) ? w2[c * wc + ((long)z * g.Py + ky) * g.Hx + kx0 + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const Lines zl{T, 1, 3, cst, 0};
  block_fft<false, float2, kEPT, kNT>(sm, g.Pz, 3 * T, zl, T, twz, 1);
  const bool has_z = g.Pz > 1;
  for (int e = threadIdx.x; e < cst; e += blockDim.x) {
    const int t = e % T;
    if (t >= nt) continue;
    tensor_mul(sm[e], sm[cst + e], sm[2 * cst + e], nhat, g, kx0 + t, ky, e / T, has_z);
  }
  __syncthreads();
  block_fft<true, float2, kEPT, kNT>(sm, g.Pz, 3 * T, zl, T, twz, 1);
  for (int e = threadIdx.x; e < 3 * cst; e += blockDim.x) {
    const int t = e % T, z = (e / T) % g.Pz, c = e / cst;
    if (t < nt && z < g.nz) w2[c * wc + ((long)z * g.Py + ky) * g.Hx + kx0 + t] = sm[e];
  }
}

__global__ void __launch_bounds__(kNT) y_inv_kernel(const float2* __restrict__ w2, float2* __restrict__ w1, Grid g,
                                                    const float2* __restrict__ twy, int T) {
  extern __shared__ float2 sm[];
  const int ntile = (g.Hx + T - 1) / T;
  const int kx0 = (blockIdx.x % ntile) * T;
  const int ck = blockIdx.x / ntile;
  const int nt = min(T, g.Hx - kx0);
  const float2* src = w2 + (long)ck * g.Py * g.Hx + kx0;
  for (int e = threadIdx.x; e < g.Py * T; e += blockDim.x) {
    const int t = e % T, y = e / T;
    sm[e] = (t < nt) ? src[(long)y * g.Hx + t] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  block_fft<true, float2, kEPT, kNT>(sm, g.Py, T, lines1(1), T, twy, 1);
  float2* dst = w1 + (long)ck * g.ny * g.Hx + kx0;
  for (int e = threadIdx.x; e < g.ny * T; e += blockDim.x) {
    const int t = e % T, y = e / T;
    if (t < nt) dst[(long)y * g.Hx + t] = sm[e];
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static int x_rows(const Grid& g) {
  const int M = g.Px > 1 ? g.Px / 2 : 1;
  int r = kCap / (3 * M);
  if (r < 1) r = 1;
  if (r > 32) r = 32;
  return r;
}

static int col_tile(int L) {
  int t = kCap / L;
  if (t > 64) t = 64;
  return t < 1 ? 1 : t;
}

mx_status demag_setup(mx_ctx* ctx) {
  const Grid& g = ctx->g;
  // fused y/z plane: 3 Py Pz T elements within one block's FFT capacity and
  // at most 96 KB of shared memory
  int T = kCap / (3 * g.Py * g.Pz);
  while (T > 1 && (size_t)3 * g.Py * g.Pz * T * sizeof(float2) > 96 * 1024) --T;
  if (T > 16) T = 16;
  // fewer columns per block while that leaves fewer than two blocks per SM
  while (T > 1 && (g.Hx + T - 1) / T < 2 * 152) T /= 2;
  ctx->fused_yz = ctx->p.demag_path == MX_DEMAG_AUTO && (T >= 1) && (3L * g.Py * g.Pz <= kCap) &&
                  (size_t)3 * g.Py * g.Pz * sizeof(float2) <= 96 * 1024;
  ctx->yz_tile = T < 1 ? 1 : T;
  const int big = 200 * 1024;
  MX_CUDA_TRY(cudaFuncSetAttribute(x_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  MX_CUDA_TRY(cudaFuncSetAttribute(x_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  MX_CUDA_TRY(cudaFuncSetAttribute(yz_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  MX_CUDA_TRY(cudaFuncSetAttribute(y_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  MX_CUDA_TRY(cudaFuncSetAttribute(z_mul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  MX_CUDA_TRY(cudaFuncSetAttribute(y_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return MX_OK;
}

mx_status demag_yz(mx_ctx* ctx, cudaStream_t st) {
  const Grid& g = ctx->g;
  if (ctx->yz2d) {
    ProfScope ps(ctx, KID_YZ, st);
    MX_TRY(yz2d_pass(ctx, st));
  } else if (ctx->fused_yz) {
    const int T = ctx->yz_tile;
    const size_t s = sizeof(float2) * 3 * g.Py * g.Pz * T;
    ProfScope ps(ctx, KID_YZ, st);
    yz_fused_kernel<<<(g.Hx + T - 1) / T, kNT, s, st>>>(ctx->w1, g, ctx->nhat, ctx->tw_y, ctx->tw_z, T);
    MX_TRY(launch_check("yz_fused_kernel"));
  } else {
    const int Ty = col_tile(g.Py);
    const int nty = (g.Hx + Ty - 1) / Ty;
    {
      ProfScope ps(ctx, KID_Y_FWD, st);
      y_fwd_kernel<<<3 * g.nz * nty, kNT, sizeof(float2) * g.Py * Ty, st>>>(ctx->w1, ctx->w2, g, ctx->tw_y, Ty);
      MX_TRY(launch_check("y_fwd_kernel"));
    }
    const int Tz = col_tile(3 * g.Pz);
    const int ntz = (g.Hx + Tz - 1) / Tz;
    {
      ProfScope ps(ctx, KID_Z_MUL, st);
      z_mul_kernel<<<g.Py * ntz, kNT, sizeof(float2) * 3 * g.Pz * Tz, st>>>(ctx->w2, g, ctx->nhat, ctx->tw_z, Tz);
      MX_TRY(launch_check("z_mul_kernel"));
    }
    {
      ProfScope ps(ctx, KID_Y_INV, st);
      y_inv_kernel<<<3 * g.nz * nty, kNT, sizeof(float2) * g.Py * Ty, st>>>(ctx->w2, ctx->w1, g, ctx->tw_y, Ty);
      MX_TRY(launch_check("y_inv_kernel"));
    }
  }
  return MX_OK;
}

mx_status demag_field(mx_ctx* ctx, const float4* m, float4* hd, cudaStream_t st) {
  if (ctx->surrogate) return cnn_demag(ctx->surrogate, m, hd, st);
  if (ctx->fno) return fno_demag(ctx->fno, m, hd, st);
  if (ctx->plane) return plane_field(ctx, m, hd, st);
  const Grid& g = ctx->g;
  const int rows = x_rows(g);
  const int nrows = g.ny * g.nz;
  const int M = g.Px > 1 ? g.Px / 2 : 1;
  const size_t xs = sizeof(float2) * 3 * rows * M;
  {
    ProfScope ps(ctx, KID_X_FWD, st);
    if (ctx->fast_x) {
      MX_TRY(fast_x_pass(ctx, m, nullptr, false, st));
    } else {
      x_fwd_kernel<<<(nrows + rows - 1) / rows, kNT, xs, st>>>(m, g, (float)ctx->p.Ms, ctx->ms_map, ctx->w1,
                                                               ctx->tw_x, rows);
      MX_TRY(launch_check("x_fwd_kernel"));
    }
  }
  MX_TRY(demag_yz(ctx, st));
  {
    ProfScope ps(ctx, KID_X_INV, st);
    if (ctx->fast_x) {
      MX_TRY(fast_x_pass(ctx, nullptr, hd, true, st));
    } else {
      x_inv_kernel<<<(nrows + rows - 1) / rows, kNT, xs, st>>>(ctx->w1, g, hd, ctx->tw_x, rows);
      MX_TRY(launch_check("x_inv_kernel"));
    }
  }
  return MX_OK;
}

}  // namespace mx
