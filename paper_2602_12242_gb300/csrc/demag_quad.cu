// Demag convolution on large grids: the y and z passes of one kx plane on a
// cluster of four CTAs (Sec. II-B: zero-padded FFT convolution of M with the
// tensor spectrum; the arithmetic of the other schedules in another order).
//
// Input and output are the kx-major spectra of the x passes, w[kx][c][z][y]
// (ny values per row).  The tensor octant is in the oct4 layout
// [kx][qz][qy mod 4][qy / 4][comp] (plane_octant_index).
//
// Forward y.  A column is zero for y >= Py/2, so with L4 = Py/4 the outputs of
// residue h (ky = 4k + h) are an L4-point FFT of the folded column
//   f_h[y] = W_Py^(h y) (x[y] + (-i)^h x[y + L4]),   y < L4.
// Each CTA loads a quarter of the plane's lines once and stores all four
// folds x[y] + (-i)^j x[y + L4] into CTA j's shared memory (distributed
// shared memory), so the plane crosses L2 once.  CTA h (its rank) then
// transforms every line (c, z) in two register steps (E-point FFTs over n of
// y = s + S n, then S-point FFTs over s).  The fold's twiddle is split
// between the steps: W_4E^(h n) before step 1, and W_Py^(s (4 k1 + h)) (which
// includes the usual W_L4^(s k1)) between them.
//
// z stage.  For each of its L4 columns, the Pz-point transform of the
// nz <= Pz/2 non-zero planes splits into even kz (a Pz/2-point FFT of x) and
// odd kz (a Pz/2-point FFT of x W_Pz^z).  A warp takes 32 columns of one
// parity, multiplies by the 3x3 tensor (real; N_xy odd in ky, N_xz odd in kz,
// N_yz odd in both) and transforms back; the inverse z transform is the even
// half plus W_Pz^(-z) times the odd half, summed in shared memory by the two
// warps of the column block, which synchronise on a barrier of their own.
// The CTA's tensor entries are prefetched into L2 at the start.
//
// Inverse y.  With u_h[y] = W_Py^(-h y) IFFT_L4(Y_h)[y] (that twiddle again
// split across the two steps), the output for y < Py/2 is a radix-4
// combination over the cluster:
//   out[y] = sum_h u_h[y],   out[y + L4] = sum_h i^h u_h[y].
// CTA j forms it for a quarter of the plane's lines, reading the other CTAs'
// u_h through distributed shared memory, and stores it.
//
// Two CTAs fit on an SM (about 108 KB of shared memory and at most 128
// registers per thread each for the bulk grid), so one CTA's loads and
// barriers overlap the other's arithmetic.
#include <math.h>

#include "cluster.cuh"
#include "common.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "regfft.cuh"

namespace mx {

constexpr int kQuadNT = 256;  // threads per CTA

// Step 2 of the inverse line transform with the per-output twiddle
// conj(twB[k2]): the twiddled E x S matrix is in rows k1 * (S + 1); thread s
// does S-point inverse FFTs over s for k1 = s + S j and writes x[k1 + E k2].
template <int E, int S>
__device__ __forceinline__ void quad_inv_step2(float2* line, int s, const float2* __restrict__ twB) {
  float2 v[E];
  constexpr int J = E / S;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k1 = s + S * j;
#pragma unroll
    for (int t = 0; t < S; ++t) v[j * S + t] = line[k1 * (S + 1) + t];
    RegFft<S, true>::run(&v[j * S]);
#pragma unroll
    for (int t = 1; t < S; ++t) v[j * S + t] = cmul(v[j * S + t], cconj(twB[t]));
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k1 = s + S * j;
#pragma unroll
    for (int t = 0; t < S; ++t) line[k1 + E * t] = v[j * S + t];
  }
  __syncwarp();
}

// (a, b, c) <- N (a, b, c) for the symmetric 3x3 tensor N, complex vectors.
__device__ __forceinline__ void tensor_apply(float2& a, float2& b, float2& c, float nxx, float nyy, float nzz,
                                             float nxy, float nxz, float nyz) {
  const float2 mx = a, my = b, mz = c;
  a = make_float2(fmaf(nxz, mz.x, fmaf(nxy, my.x, nxx * mx.x)), fmaf(nxz, mz.y, fmaf(nxy, my.y, nxx * mx.y)));
  b = make_float2(fmaf(nyz, mz.x, fmaf(nyy, my.x, nxy * mx.x)), fmaf(nyz, mz.y, fmaf(nyy, my.y, nxy * mx.y)));
  c = make_float2(fmaf(nzz, mz.x, fmaf(nyz, my.x, nxz * mx.x)), fmaf(nzz, mz.y, fmaf(nyz, my.y, nxz * mx.y)));
}

// Tensor multiply of one column's half spectrum, kz parity PAR: y[.][q] holds
// kz = 2 q + PAR; kz and its mirror P - kz share one octant entry (the mirror
// with N_xz and N_yz negated).  tq: the column's entry at qz = 0, qzs floats
// per step of qz; sy = -1 where ky > Py/2 (N_xy and N_yz are odd in ky).
template <int P, int PAR>
__device__ __forceinline__ void quad_z_multiply(float2 (&y)[3][P / 2], const float* __restrict__ tq, long qzs,
                                                float sy) {
  constexpr int Q = P / 2;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int kz = 2 * q + PAR;
    if (kz > P / 2) continue;  // done with its mirror
    const float2* t = reinterpret_cast<const float2*>(tq + kz * qzs);
    const float2 t01 = __ldg(t), t23 = __ldg(t + 1), t45 = __ldg(t + 2);
    const float nxy = sy * t23.y, nyz = sy * t45.y;
    tensor_apply(y[0][q], y[1][q], y[2][q], t01.x, t01.y, t23.x, nxy, t45.x, nyz);
    if (kz != 0 && kz != P / 2) {
      const int qm = Q - q - PAR;  // 2 qm + PAR = P - kz
      tensor_apply(y[0][qm], y[1][qm], y[2][qm], t01.x, t01.y, t23.x, nxy, -t45.x, -nyz);
    }
  }
}

// One column, kz parity p (uniform across the warp): half-length forward
// transform of the nz planes of each component (times W_P^z first for odd
// kz), the tensor multiply and the inverse half transform (times W_P^-z after
// it for odd kz); y[c][n] is this parity's share of output plane n.  col: the
// column's element in line 0 of the plane.
template <int P>
__device__ __forceinline__ void quad_z_column(const float2* col, int pitch, int nz, const float* __restrict__ tq,
                                              long qzs, float sy, int p, float2 (&y)[3][P / 2]) {
  constexpr int Q = P / 2;
  constexpr int TS = 32 / P;  // W_P^n = c_w32[n TS]
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int n = 0; n < Q; ++n) y[c][n] = n < nz ? col[(c * nz + n) * pitch] : make_float2(0.f, 0.f);
  if (p) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 1; n < Q; ++n) y[c][n] = cmul(y[c][n], c_w32[n * TS]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) RegFft<Q, false>::run(y[c]);
  if (p)
    quad_z_multiply<P, 1>(y, tq, qzs, sy);
  else
    quad_z_multiply<P, 0>(y, tq, qzs, sy);
#pragma unroll
  for (int c = 0; c < 3; ++c) RegFft<Q, true>::run(y[c]);
  if (p) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 1; n < Q; ++n) y[c][n] = cmul(y[c][n], cconj(c_w32[n * TS]));
  }
}

// barrier `id` (1..15) over `count` threads (whole warps)
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int E, int S, int P>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(kQuadNT, 2)
    yzq_kernel(const float2* __restrict__ w1, float2* __restrict__ w2, Grid g, const float* __restrict__ nhk,
               const float2* __restrict__ twPy) {
  constexpr int L4 = E * S;
  constexpr int PITCH = LineFft<E, S>::kPitch;
  constexpr int NT = kQuadNT;
  constexpr int Q = P / 2;
  extern __shared__ __align__(16) float2 sm[];
  pdl_wait();                // w1 is the previous kernel's
  cluster_arrive_relaxed();  // this CTA has started (waited for before the first remote store)
  const int h = (int)cluster_rank();
  const int kx = blockIdx.x >> 2;
  const int tid = threadIdx.x;
  const int nz = g.nz, ny = g.ny, Py = g.Py;
  const int nlines = 3 * nz;
  const long kxoff = (long)kx * nlines * ny;
  float2* plane = sm;                  // [3 nz][PITCH]
  float2* dummy = plane + nlines * PITCH;  // scratch line for idle thread groups
  float2* twF = dummy + PITCH;         // [k1 S + s]: W_Py^(s (4 k1 + h))
  float2* twI = twF + L4;              // [k1 S + s]: W_Py^(k1 (4 s + h))
  float2* twA = twI + L4;              // [n]: W_Py^(h n S) = W_4E^(h n)
  float2* twB = twA + E;               // [k2]: W_Py^(h k2 E) = W_4S^(h k2)

  // folds: CTA h loads a quarter of the plane's lines (both halves of each
  // column) and stores x[y] + (-i)^j x[y + L4] into line slot y of CTA j
  const int LQ = (nlines + 3) >> 2;
  const int lb = min(nlines, h * LQ), le = min(nlines, lb + LQ);
  // twiddle-table entries of this thread, loaded with the first fold loads
  constexpr int NTW = (L4 + NT - 1) / NT;
  float2 tf[NTW], ti[NTW];
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    const int q = tid + j * NT;
    const int k1 = q / S, s = q % S;
    tf[j] = q < L4 ? __ldg(&twPy[s * (4 * k1 + h)]) : make_float2(0.f, 0.f);
    ti[j] = q < L4 ? __ldg(&twPy[k1 * (4 * s + h)]) : make_float2(0.f, 0.f);
  }
  const float2 ta = tid < E ? __ldg(&twPy[h * tid * S]) : make_float2(0.f, 0.f);
  const float2 tb = tid < S ? __ldg(&twPy[h * tid * E]) : make_float2(0.f, 0.f);
  {
    const int cnt = (le - lb) * L4;
    constexpr int kB = 12;  // column pairs per thread in flight (all of them for the bulk grid)
    for (int base = 0; base < cnt; base += NT * kB) {
      float2 a[kB], b[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int e = base + tid + u * NT;
        const int line = lb + e / L4, y = e % L4;
        const float2* src = w1 + kxoff + (long)line * ny;
        a[u] = (e < cnt && y < ny) ? __ldg(src + y) : make_float2(0.f, 0.f);
        b[u] = (e < cnt && y + L4 < ny) ? __ldg(src + y + L4) : make_float2(0.f, 0.f);
      }
      if (base == 0) cluster_wait();  // every CTA of the cluster has started
      float2* dst0 = const_cast<float2*>(cluster_map(plane, 0u));
      float2* dst1 = const_cast<float2*>(cluster_map(plane, 1u));
      float2* dst2 = const_cast<float2*>(cluster_map(plane, 2u));
      float2* dst3 = const_cast<float2*>(cluster_map(plane, 3u));
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int e = base + tid + u * NT;
        if (e >= cnt) break;
        const int o = (lb + e / L4) * PITCH + e % L4;
        dst0[o] = cadd(a[u], b[u]);
        dst1[o] = make_float2(a[u].x + b[u].y, a[u].y - b[u].x);
        dst2[o] = csub(a[u], b[u]);
        dst3[o] = make_float2(a[u].x - b[u].y, a[u].y + b[u].x);
      }
    }
    if (cnt == 0) cluster_wait();
  }
  cluster_arrive_release();  // this CTA's folds are stored

  // while the other CTAs finish theirs: the twiddle tables, and the tensor
  // entries of this CTA's columns (qy = 4k + h and Py - 4k - h, classes h and
  // -h mod 4) into L2, so the z stage's loads do not wait on HBM
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    const int q = tid + j * NT;
    if (q < L4) {
      twF[q] = tf[j];
      twI[q] = ti[j];
    }
  }
  if (tid < E) twA[tid] = ta;
  if (tid < S) twB[tid] = tb;
  {
    const int o4 = plane_oct4_rows(g);
    const long cls_bytes = (long)o4 * 6 * sizeof(float);
    const char* nk = reinterpret_cast<const char*>(nhk + (long)kx * g.Oz * 4 * o4 * 6);
    const int c2 = (4 - h) & 3;
    const int ncls = c2 == h ? 1 : 2;
    const int lines_per = (int)((cls_bytes + 127) / 128);
    for (int q = tid; q < g.Oz * ncls * lines_per; q += NT) {
      const int qz = q / (ncls * lines_per), r = q % (ncls * lines_per);
      const int cls = r < lines_per ? h : c2;
      // (the last line of a class starts inside it)
      const char* a = nk + ((long)qz * 4 + cls) * cls_bytes + min((long)(r % lines_per) * 128, cls_bytes - 4);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
  }
  __syncthreads();          // tables
  cluster_wait_acquire();   // every CTA's folds

  constexpr int LPR = NT / S;  // lines per round, S threads per line
  const int s = tid % S;

  // forward y of every line: W_4E^(h n) before step 1, W_Py^(s (4 k1 + h)) between the steps
  for (int l0 = 0; l0 < nlines; l0 += LPR) {
    const int l = l0 + tid / S;
    float2* line = l < nlines ? plane + l * PITCH : dummy;
    float2 v[E];
#pragma unroll
    for (int n = 0; n < E; ++n) v[n] = n ? cmul(line[s + S * n], twA[n]) : line[s];
    RegFft<E, false>::run(v);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) line[k1 * (S + 1) + s] = cmul(v[k1], twF[k1 * S + s]);
    __syncwarp();
    line_fft_step2<E, S, false>(line, s);
  }
  __syncthreads();

  // z stage: warp w takes 32 columns of one parity per round; the two warps
  // of a column block (w and w + HW) meet at their own named barrier
  {
    constexpr int CB = L4 / 32;       // column blocks
    constexpr int HW = NT / 64;       // warps per parity
    static_assert(HW + 1 <= 16, "named barrier ids");
    const int warp = tid >> 5, lane = tid & 31;
    const int bar = 1 + warp % HW;
    const int o4 = plane_oct4_rows(g);
    const long qzs = 4L * o4 * 6;
    const float* nk = nhk + (long)kx * g.Oz * qzs;
    for (int cb0 = 0; cb0 < CB; cb0 += HW) {
      const int cb = cb0 + warp % HW;
      if (cb >= CB) break;  // both warps of the pair leave together
      // the odd half costs more (twiddles, the final add): a warp takes the
      // even and the odd half in alternate rounds
      const int p = (warp / HW) ^ ((cb0 / HW) & 1);
      const int col = 32 * cb + lane;
      const int ky = 4 * col + h;
      const bool fy = ky > (Py >> 1);
      const int qy = fy ? Py - ky : ky;
      const float* tq = nk + ((long)(qy & 3) * o4 + (qy >> 2)) * 6;
      float2* cp = plane + col;
      float2 y[3][Q];
      quad_z_column<P>(cp, PITCH, nz, tq, qzs, fy ? -1.f : 1.f, p, y);
      named_sync(bar, 64);  // both parities have read these columns
      if (p == 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int n = 0; n < Q; ++n)
            if (n < nz) cp[(c * nz + n) * PITCH] = y[c][n];
      }
      named_sync(bar, 64);
      if (p == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int n = 0; n < Q; ++n)
            if (n < nz) {
              float2* o = cp + (c * nz + n) * PITCH;
              *o = cadd(*o, y[c][n]);
            }
      }
    }
  }
  __syncthreads();

  // inverse y: u_h in natural order in each line
  for (int l0 = 0; l0 < nlines; l0 += LPR) {
    const int l = l0 + tid / S;
    float2* line = l < nlines ? plane + l * PITCH : dummy;
    float2 v[E];
#pragma unroll
    for (int n = 0; n < E; ++n) v[n] = line[s + S * n];
    RegFft<E, true>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1) v[k1] = cmul(v[k1], cconj(twI[k1 * S + s]));
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) line[k1 * (S + 1) + s] = v[k1];
    __syncwarp();
    quad_inv_step2<E, S>(line, s, twB);
  }

  // radix-4 combination over the cluster for lines [lb, le)
  cluster_sync_all();
  {
    // the other CTAs' partials through distributed shared memory, this CTA's own directly
    const float2* u0 = h == 0 ? plane : cluster_map(plane, 0u);
    const float2* u1 = h == 1 ? plane : cluster_map(plane, 1u);
    const float2* u2 = h == 2 ? plane : cluster_map(plane, 2u);
    const float2* u3 = h == 3 ? plane : cluster_map(plane, 3u);
    const int cnt = (le - lb) * L4;
    float2* dst = w2 + kxoff;
    constexpr int kB = L4 >= 256 ? 6 : 4;  // outputs per thread in flight
    // uniform trip count: the arrive below is executed once by every thread,
    // after its last read of another CTA's shared memory
    for (int base = 0; base < cnt; base += NT * kB) {
      float2 a[kB][4];
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const int e = base + tid + b * NT;
        if (e < cnt) {
          const int o = (lb + e / L4) * PITCH + e % L4;
          a[b][0] = u0[o];
          a[b][1] = u1[o];
          a[b][2] = u2[o];
          a[b][3] = u3[o];
        }
      }
      if (base + NT * kB >= cnt) cluster_arrive_release();
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const int e = base + tid + b * NT;
        if (e >= cnt) break;
        const int line = lb + e / L4, y = e % L4;
        const float2 s02 = cadd(a[b][0], a[b][2]), d02 = csub(a[b][0], a[b][2]);
        const float2 s13 = cadd(a[b][1], a[b][3]), d13 = csub(a[b][1], a[b][3]);
        float2* row = dst + (long)line * ny;
        if (y < ny) row[y] = cadd(s02, s13);
        if (y + L4 < ny) row[y + L4] = make_float2(d02.x - d13.y, d02.y + d13.x);
      }
    }
    if (cnt == 0) cluster_arrive_release();
  }
  // no CTA leaves while another may still read its shared memory
  cluster_wait();
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int E, int S> static size_t yzq_smem(int nz) {
  return sizeof(float2) * ((size_t)(3 * nz + 1) * LineFft<E, S>::kPitch + 2 * E * S + E + S);
}

template <int E, int S, int P>
static mx_status yzq_run(mx_ctx* ctx, cudaStream_t st, bool setup) {
  const size_t sm = yzq_smem<E, S>(ctx->g.nz);
  if (setup) {
    if (sm > 227 * 1024) return MX_ERR_UNSUPPORTED;
    MX_CUDA_TRY(cudaFuncSetAttribute(yzq_kernel<E, S, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  launch_pdl(yzq_kernel<E, S, P>, dim3(4 * ctx->g.Hx), dim3(kQuadNT), sm, st, ctx->w1, ctx->w2, ctx->g, ctx->nhat,
             ctx->tw_y);
  return launch_check("yzq_kernel");
}

template <int E, int S>
static mx_status yzq_pz(mx_ctx* ctx, cudaStream_t st, bool setup) {
  switch (ctx->g.Pz) {
    case 32: return yzq_run<E, S, 32>(ctx, st, setup);
    case 16: return yzq_run<E, S, 16>(ctx, st, setup);
    case 8: return yzq_run<E, S, 8>(ctx, st, setup);
    case 4: return yzq_run<E, S, 4>(ctx, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

mx_status quad_pass(mx_ctx* ctx, cudaStream_t st, bool setup) {
  if (setup) MX_TRY(upload_w32());
  switch (ctx->g.Py / 4) {
    case 512: return yzq_pz<32, 16>(ctx, st, setup);
    case 256: return yzq_pz<16, 16>(ctx, st, setup);
    case 128: return yzq_pz<16, 8>(ctx, st, setup);
    case 64: return yzq_pz<8, 8>(ctx, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

}  // namespace mx
