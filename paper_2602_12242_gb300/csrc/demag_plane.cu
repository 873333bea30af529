// Demag convolution for large grids with one kernel per kx plane (Sec. II-B:
// zero-padded FFT convolution with the tensor spectrum; the arithmetic is the
// same as demag.cu, only the schedule differs).
//
// Spectra use a kx-major layout, w[kx][c][z][y] (y fastest), so a kx plane is
// contiguous.  The tensor octant is kx-major too, [kx][qz][qy mod 2][qy / 2][comp]
// (plane_octant_index).
//
//   xfk  r2c along x for R consecutive rows (same z); the spectrum is
//        transposed in shared memory so the kx-major stores are coalesced.
//   yzh  a cluster of two CTAs per kx: the y transform of the zero-padded
//        column (only the first ny <= Py/2 inputs non-zero) splits into its
//        even outputs, an Py/2-point FFT of x, and its odd outputs, an
//        Py/2-point FFT of x W_Py^y.  CTA h holds half h, [c][z][Py/2], in
//        shared memory (bulk row copies in): forward y FFT, then per ky the z
//        FFT, the 3x3 tensor multiply and the inverse z FFT (four lanes per
//        column, one residue class kz mod 4 each), then the inverse y FFT.
//        The inverse y transform restricted to y < ny is the sum of the two
//        halves' inverses, the odd one times W_Py^-y: each CTA sums half of
//        the plane's rows with the other CTA's rows (distributed shared
//        memory) and bulk-stores them.
//   xik  c2r along x for R consecutive rows, reading the kx-major spectrum.
#include <math.h>

#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "kernels.cuh"
#include "bulk.cuh"
#include "cluster.cuh"
#include "local.cuh"
#include "regfft.cuh"

namespace mx {

constexpr int kRows = 8;      // rows per block in xfk / xik
constexpr int kPlaneNT = 384; // threads per yzh block (48 lines of 16 threads in two passes)

// Line pitch of the yzh plane in float2: the line FFT's footprint plus 2, so
// that the pitch in 4-byte words is 4 mod 8 and the z stage's four lanes per
// column (rows n, n + Q/2, n + Q, n + 3Q/2) write to two bank halves instead
// of one.
template <int E, int S> struct YzhPitch {
  static constexpr int value = LineFft<E, S>::kPitch + 2;
};

// ---------------------------------------------------------------------------
// x forward into the kx-major spectrum.
// ---------------------------------------------------------------------------
template <int E, int S>
__global__ void __launch_bounds__(3 * kRows * S, S >= 32 ? 1 : 2) xfk_kernel(const float4* __restrict__ m, Grid g, float ms,
                                                            const float* __restrict__ ms_map, float2* __restrict__ w1,
                                                            const float2* __restrict__ twM,
                                                            const float2* __restrict__ twP) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch + 1;
  constexpr int NT = 3 * kRows * S;
  extern __shared__ float2 sm[];
  const int ychunks = (g.ny + kRows - 1) / kRows;
  const int nblk = g.nz * ychunks;
  const int tid = threadIdx.x;
  pdl_wait();
  // Persistent blocks: block b of rows (z, y0 .. y0 + kRows - 1) for
  // b = blockIdx.x, blockIdx.x + gridDim.x, ...; the next block's rows are
  // prefetched into L2 while this block's spectrum is written out.
  // Ms m as packed pairs z[n] = M[2n] + i M[2n+1]; nx <= M, so only n < M/2
  // can be non-zero.
  constexpr int HALF = M / 2;
  constexpr int NLD = (kRows * HALF + NT - 1) / NT;
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    float4 va[NLD], vb[NLD];
    {
      const int z = b / ychunks, y0 = (b % ychunks) * kRows;
#pragma unroll
      for (int j = 0; j < NLD; ++j) {
        const int e = tid + j * NT;
        const int r = e / HALF, n = e % HALF;
        const int y = y0 + r;
        const bool in = e < kRows * HALF && y < g.ny;
        const long cell = ((long)z * g.ny + (in ? y : 0)) * g.nx + 2 * n;
        va[j] = (in && 2 * n < g.nx) ? __ldg(&m[cell]) : make_float4(0.f, 0.f, 0.f, 0.f);
        vb[j] = (in && 2 * n + 1 < g.nx) ? __ldg(&m[cell + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    const int z = b / ychunks, y0 = (b % ychunks) * kRows;
    float sa[NLD], sb[NLD];
#pragma unroll
    for (int j = 0; j < NLD; ++j) sa[j] = sb[j] = ms;
    if (ms_map) {
#pragma unroll
      for (int j = 0; j < NLD; ++j) {
        const int e = tid + j * NT;
        const int r = e / HALF, n = e % HALF;
        const int y = y0 + r;
        const bool in = e < kRows * HALF && y < g.ny;
        const long cell = ((long)z * g.ny + (in ? y : 0)) * g.nx + 2 * n;
        if (in && 2 * n < g.nx) sa[j] = __ldg(&ms_map[cell]);
        if (in && 2 * n + 1 < g.nx) sb[j] = __ldg(&ms_map[cell + 1]);
      }
    }
#pragma unroll
    for (int j = 0; j < NLD; ++j) {
      const int e = tid + j * NT;
      if (e >= kRows * HALF) break;
      const int r = e / HALF, n = e % HALF;
      sm[(3 * r + 0) * P + n] = make_float2(sa[j] * va[j].x, sb[j] * vb[j].x);
      sm[(3 * r + 1) * P + n] = make_float2(sa[j] * va[j].y, sb[j] * vb[j].y);
      sm[(3 * r + 2) * P + n] = make_float2(sa[j] * va[j].z, sb[j] * vb[j].z);
    }
    for (int e = tid; e < 3 * kRows * HALF; e += NT) sm[(e / HALF) * P + HALF + e % HALF] = make_float2(0.f, 0.f);
    __syncthreads();
    line_fft<E, S, false, false, true>(sm + (tid / S) * P, tid % S, twM);
    __syncthreads();
    {
      // the next block's rows (kRows rows of nx float4, contiguous per row) into L2
      const int bn = b + gridDim.x;
      if (bn < nblk) {
        const int zn = bn / ychunks, yn = (bn % ychunks) * kRows;
        const int lines_per_row = (g.nx * 16 + 127) / 128;
        for (int q = tid; q < kRows * lines_per_row; q += NT) {
          const int r = q / lines_per_row, k = q % lines_per_row;
          if (yn + r < g.ny) {
            const char* a = reinterpret_cast<const char*>(m + ((long)zn * g.ny + yn + r) * g.nx) +
                            min(k * 128, g.nx * 16 - 16);
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
          }
        }
      }
    }
    // r2c output from the packed transform Z: pairs (k, M - k), 0 < k < M/2,
    // with E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / 2i and
    // T = W_2M^k O give X[k] = E + T and X[M-k] = conj(E - T); k = 0 gives
    // X[0] = Re Z[0] + Im Z[0] and X[M] = Re Z[0] - Im Z[0]; X[M/2] = conj Z[M/2].
    // Each thread keeps one line (row r fastest, so eight lanes store 64
    // contiguous bytes of the kx-major spectrum).
    constexpr int NL = 3 * kRows;
    static_assert(NT % NL == 0, "xfk thread count");
    const int li = tid % NL;
    const int r = li % kRows, c = li / kRows;
    const int y = y0 + r;
    if (y < g.ny) {
      const long plane = 3L * g.nz * g.ny;  // one kx
      const float2* L = sm + (3 * r + c) * P;
      float2* dst = w1 + ((long)c * g.nz + z) * g.ny + y;
#pragma unroll 4
      for (int k = tid / NL; k <= M / 2; k += NT / NL) {
        const float2 a = L[k];
        if (k == 0) {
          dst[0] = make_float2(a.x + a.y, 0.f);
          dst[(long)M * plane] = make_float2(a.x - a.y, 0.f);
        } else if (k == M / 2) {
          dst[(long)k * plane] = cconj(a);
        } else {
          const float2 bv = L[M - k];
          const float2 Ev = make_float2(0.5f * (a.x + bv.x), 0.5f * (a.y - bv.y));
          const float2 O = make_float2(0.5f * (a.y + bv.y), -0.5f * (a.x - bv.x));
          const float2 T = cmul(__ldg(&twP[k]), O);
          dst[(long)k * plane] = cadd(Ev, T);
          dst[(long)(M - k) * plane] = cconj(csub(Ev, T));
        }
      }
    }
    __syncthreads();  // the lines are read before the next block overwrites them
  }
}

// ---------------------------------------------------------------------------
// x inverse from the kx-major spectrum.
// ---------------------------------------------------------------------------
// The c2r transforms of rows (z, y0 .. y0 + kRows - 1), all three components,
// into shared memory: afterwards element n of line 3 r + c holds H_c of cells
// 2n (real part) and 2n + 1 (imaginary part) of row y0 + r.
template <int E, int S>
__device__ __forceinline__ void xik_lines(float2* sm, const float2* __restrict__ w2, const Grid& g, int z, int y0,
                                          const float2* __restrict__ twM, const float2* __restrict__ twP) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch + 1;
  constexpr int NT = 3 * kRows * S;
  const int tid = threadIdx.x;
  // c2r input from the half spectrum X: pairs (k, M - k) with S = X[k] +
  // conj X[M-k] and t = conj(W_2M^k) (X[k] - conj X[M-k]) give
  // Z[k] = S + i t and Z[M-k] = conj(S - i t); k = 0 gives Z[0] (from X[0]
  // and X[M]) and k = M/2 gives Z[M/2] = 2 conj X[M/2].  One line per
  // thread, row r fastest (eight lanes load 64 contiguous bytes).
  constexpr int NL = 3 * kRows;
  static_assert(NT % NL == 0, "xik thread count");
  {
    const long plane = 3L * g.nz * g.ny;  // one kx
    const int li = tid % NL;
    const int r = li % kRows, c = li / kRows;
    const int y = y0 + r;
    float2* L = sm + (3 * r + c) * P;
    const float2* src = w2 + ((long)c * g.nz + z) * g.ny + (y < g.ny ? y : 0);
    // k = k0 + (NT / NL) j <= M/2, in batches of kB pairs with every load in flight
    constexpr int KS = NT / NL;
    constexpr int J = M / 2 / KS + 1;
    constexpr int kB = 8;
    const int k0 = tid / NL;
#pragma unroll
    for (int j0 = 0; j0 < J; j0 += kB) {
      float2 a[kB], b[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int k = k0 + KS * (j0 + u);
        a[u] = b[u] = make_float2(0.f, 0.f);
        if (j0 + u < J && k <= M / 2 && y < g.ny) {
          a[u] = __ldg(&src[(long)k * plane]);
          b[u] = cconj(__ldg(&src[(long)(M - k) * plane]));
        }
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int k = k0 + KS * (j0 + u);
        if (j0 + u >= J || k > M / 2) break;
        const float2 Sv = cadd(a[u], b[u]);
        const float2 t = cmul(cconj(__ldg(&twP[k])), csub(a[u], b[u]));
        L[k] = make_float2(Sv.x - t.y, Sv.y + t.x);
        if (k > 0 && k < M / 2) L[M - k] = make_float2(Sv.x + t.y, t.x - Sv.y);
      }
    }
  }
  __syncthreads();
  line_fft<E, S, true, false, true>(sm + (tid / S) * P, tid % S, twM);
  __syncthreads();
}

template <int E, int S>
__global__ void __launch_bounds__(3 * kRows * S, S >= 32 ? 1 : 2) xik_kernel(const float2* __restrict__ w2, Grid g,
                                                            float4* __restrict__ hd, const float2* __restrict__ twM,
                                                            const float2* __restrict__ twP) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch + 1;
  constexpr int NT = 3 * kRows * S;
  extern __shared__ float2 sm[];
  const int ychunks = (g.ny + kRows - 1) / kRows;
  const int z = blockIdx.x / ychunks;
  const int y0 = (blockIdx.x % ychunks) * kRows;
  pdl_wait();
  xik_lines<E, S>(sm, w2, g, z, y0, twM, twP);
  // cells 2n and 2n + 1 of row r are the real and imaginary parts of element n
  for (int e = threadIdx.x; e < kRows * (M / 2); e += NT) {
    const int r = e / (M / 2), n = e % (M / 2);
    const int y = y0 + r, i = 2 * n;
    if (y >= g.ny || i >= g.nx) continue;
    const float2* L = sm + (3 * r) * P;
    const float2 hx = L[n], hy = L[P + n], hz = L[2 * P + n];
    float4* row = hd + ((long)z * g.ny + y) * g.nx;
    row[i] = make_float4(hx.x, hy.x, hz.x, 0.f);
    if (i + 1 < g.nx) row[i + 1] = make_float4(hx.y, hy.y, hz.y, 0.f);
  }
}

// The inverse x pass fused with the local stage: the c2r transforms of a
// block's rows stay in shared memory, and each cell of those rows takes its
// demag term from there for the local fields, the LLG right-hand side and
// the stage update of `mode` (an RK4 stage or the Euler step), so H_demag
// never goes to global memory.
template <int MODE, bool DMI>
__device__ __forceinline__ void xil_cells(const float2* sm, int P, int NT, const StageIO& io, const Grid& g,
                                          const LocalCoef& c, int z, int y0, int* flag) {
  const int rows = min(kRows, g.ny - y0);
  for (int e = threadIdx.x; e < rows * g.nx; e += NT) {
    const int r = e / g.nx, i = e - r * g.nx;
    const float2* L = sm + 3 * r * P + (i >> 1);
    const float2 hx = L[0], hy = L[P], hz = L[2 * P];
    const float3 hdv = (i & 1) ? make_float3(hx.y, hy.y, hz.y) : make_float3(hx.x, hy.x, hz.x);
    const int y = y0 + r;
    local_cell_v<MODE, DMI>(io, g, c, i, y, z, ((long)z * g.ny + y) * g.nx + i, hdv, flag);
  }
}

template <int E, int S, bool DMI>
__global__ void __launch_bounds__(3 * kRows * S, S >= 32 ? 1 : 2) xil_kernel(const float2* __restrict__ w2, Grid g,
                                                            const float2* __restrict__ twM,
                                                            const float2* __restrict__ twP, StageIO io, LocalCoef c,
                                                            int mode, int* flag) {
  constexpr int P = LineFft<E, S>::kPitch + 1;
  constexpr int NT = 3 * kRows * S;
  extern __shared__ float2 sm[];
  const int ychunks = (g.ny + kRows - 1) / kRows;
  const int z = blockIdx.x / ychunks;
  const int y0 = (blockIdx.x % ychunks) * kRows;
  pdl_wait();
  xik_lines<E, S>(sm, w2, g, z, y0, twM, twP);
  switch (mode) {
    case LM_RK4_S0: xil_cells<LM_RK4_S0, DMI>(sm, P, NT, io, g, c, z, y0, flag); break;
    case LM_RK4_S1: xil_cells<LM_RK4_S1, DMI>(sm, P, NT, io, g, c, z, y0, flag); break;
    case LM_RK4_S2: xil_cells<LM_RK4_S2, DMI>(sm, P, NT, io, g, c, z, y0, flag); break;
    case LM_RK4_S3: xil_cells<LM_RK4_S3, DMI>(sm, P, NT, io, g, c, z, y0, flag); break;
    default: xil_cells<LM_EULER, DMI>(sm, P, NT, io, g, c, z, y0, flag); break;
  }
}

// ---------------------------------------------------------------------------
// Per-kx plane: y FFT halves, z FFT + multiply + inverse z, inverse y.
//
// A cluster of two CTAs takes one kx plane: CTA h (its rank in the cluster)
// computes the ky = 2 kyh + h half of the y spectrum (h = 1 multiplies the
// input by W_Py^y first), the z stage of those columns and the inverse
// Py/2-point y FFT.  The output is the sum of both halves (the odd half with
// the conjugate twiddle), formed through distributed shared memory: CTA h
// finishes lines [h L0, ...) of the plane with the other CTA's rows.
// ---------------------------------------------------------------------------
template <int E, int S, int P>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPlaneNT, 1)
    yzh_kernel(const float2* __restrict__ w1, float2* __restrict__ w2, Grid g, const float* __restrict__ nhk,
               const float2* __restrict__ twPy, const float2* __restrict__ twH, const float2* __restrict__ twz,
               int* flag, int arm_only) {
  constexpr int LH = E * S;                       // Py / 2
  constexpr int PITCH = YzhPitch<E, S>::value;
  constexpr int Q = P / 4;                        // points per residue class of kz
  constexpr int NT = kPlaneNT;
  extern __shared__ __align__(16) float2 sm[];
  __shared__ __align__(8) uint64_t bar;           // completion of the bulk plane load
  const int h = (int)cluster_rank();
  const int kx = blockIdx.x >> 1;
  const int tid = threadIdx.x;
  const int nz = g.nz, ny = g.ny;
  const int nlines = 3 * nz;
  const long kxoff = (long)kx * nlines * ny;
  float2* dummy = sm + nlines * PITCH;            // scratch line for idle groups
  float2* twS = dummy + PITCH;                    // W_LH^(s k) at [k S + s], in shared memory
  const int oyh = (g.Oy + 1) >> 1;
  const float* nk = nhk + plane_octant_index(g, kx, 0, 0, 0);
  float2* twZ = twS + LH;                         // W_P^(r n) at [r (2Q + 1) + n], r < 4, n < 2Q
  float2* twS2 = twZ + 68;                        // W_Py^y, y < Py/2
  for (int q = tid; q < LH; q += NT) {
    twS[q] = __ldg(&twH[(q % S) * (q / S)]);  // (S - 1)(E - 1) < LH
    twS2[q] = __ldg(&twPy[q]);
  }
  // rows of 2Q + 1 entries: the four lanes of a column read four banks
  for (int q = tid; q < 8 * Q; q += NT) twZ[(q / (2 * Q)) * (2 * Q + 1) + q % (2 * Q)] = __ldg(&twz[((q / (2 * Q)) * (q % (2 * Q))) % P]);
  // Rows of w1/w2 are ny float2 at 8 ny-byte strides: with ny even every row
  // starts on a 16-byte boundary and has a 16-byte multiple size, so the plane
  // moves by bulk copies (one per row); the line pitch keeps the shared rows
  // 16-byte aligned too.  Odd ny takes the per-element path.
  const bool bulk = (ny & 1) == 0;
  const uint32_t row_bytes = (uint32_t)ny * sizeof(float2);
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();

  if (bulk) {
    if (tid == 0) {
      mbar_arrive_expect_tx(&bar, (uint32_t)nlines * row_bytes);
      // arm_only (mx_inject_wait_timeout): the barrier expects the plane's
      // bytes but no copy is issued, so it never completes, the bounded wait
      // below runs out and sets kFlagTimeout, and no copy is ever in flight
      if (!arm_only)
        for (int line = 0; line < nlines; ++line)
          bulk_load(sm + line * PITCH, w1 + kxoff + (long)line * ny, row_bytes, &bar);
    }
    for (int e = tid; e < nlines * (LH - ny); e += NT) {
      const int line = e / (LH - ny), y = ny + e % (LH - ny);
      sm[line * PITCH + y] = make_float2(0.f, 0.f);
    }
    if (!mbar_wait(&bar, 0)) atomicOr(flag, kFlagTimeout);
    if (h) {
      for (int e = tid; e < nlines * ny; e += NT) {
        const int line = e / ny, y = e % ny;
        sm[line * PITCH + y] = cmul(sm[line * PITCH + y], twS2[y]);
      }
    }
  } else {
    // batches of kB independent loads per thread keep many requests in flight
    constexpr int kB = 4;
    for (int e0 = tid; e0 < nlines * LH; e0 += NT * kB) {
      float2 v[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int e = e0 + u * NT;
        const int line = e / LH, y = e % LH;
        v[u] = make_float2(0.f, 0.f);
        if (e < nlines * LH && y < ny) v[u] = __ldg(&w1[kxoff + (long)line * ny + y]);
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int e = e0 + u * NT;
        if (e >= nlines * LH) break;
        const int line = e / LH, y = e % LH;
        sm[line * PITCH + y] = (h && y < ny) ? cmul(v[u], twS2[y]) : v[u];
      }
    }
  }
  __syncthreads();
  for (int l0 = 0; l0 < nlines; l0 += NT / S) {
    const int l = l0 + tid / S;
    line_fft<E, S, false, true, true>(l < nlines ? sm + l * PITCH : dummy, tid % S, twS);
  }
  __syncthreads();
  // z stage: 4 lanes per ky column, lane r owns kz = 4q + r
  for (int task = tid; task < 4 * LH; task += NT) {
    const int kyh = task >> 2, r = task & 3;
    const float2* wz = twZ + r * (2 * Q + 1);
    const int ky = 2 * kyh + h;
    const bool fy = ky > (g.Py >> 1);
    const int qy = fy ? g.Py - ky : ky;
    // tensor values of this lane's kz = 4q + r, loaded first so that they
    // arrive while the forward z FFTs run
    float tn[Q][6];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int kz = 4 * q + r;
      const bool fz = kz > (P >> 1);
      const int qz = fz ? P - kz : kz;
      // the six components of (qz, qy) are contiguous (8-byte aligned)
      const float2* t = reinterpret_cast<const float2*>(nk + (((long)qz * 2 + h) * oyh + (qy >> 1)) * 6);
      const float2 t01 = __ldg(t), t23 = __ldg(t + 1), t45 = __ldg(t + 2);
      tn[q][0] = t01.x;
      tn[q][1] = t01.y;
      tn[q][2] = t23.x;
      tn[q][3] = fy ? -t23.y : t23.y;
      tn[q][4] = fz ? -t45.x : t45.x;
      tn[q][5] = (fy != fz) ? -t45.y : t45.y;
    }
    float2 Z[3][Q];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < Q; ++n) {
        float2 a = make_float2(0.f, 0.f), b = a;
        if (n < nz) a = sm[(c * nz + n) * PITCH + kyh];
        if (n + Q < nz) b = sm[(c * nz + n + Q) * PITCH + kyh];
        // y_r[n] = x[n] W_P^(r n) + x[n + Q] W_P^(r (n + Q))
        Z[c][n] = cadd(cmul(a, wz[n]), cmul(b, wz[n + Q]));
      }
#pragma unroll
    for (int c = 0; c < 3; ++c) RegFft<Q, false>::run(Z[c]);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const float nxx = tn[q][0], nyy = tn[q][1], nzz = tn[q][2];
      const float nxy = tn[q][3], nxz = tn[q][4], nyz = tn[q][5];
      const float2 mx = Z[0][q], my = Z[1][q], mz = Z[2][q];
      Z[0][q] = make_float2(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
      Z[1][q] = make_float2(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
      Z[2][q] = make_float2(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) RegFft<Q, true>::run(Z[c]);
    // x[n] = sum_r W_P^(-r n) u_r[n mod Q] for n < 2Q, summed over the 4 lanes.
    // With t_r[m] = W_P^(-r m) u_r[m] (m < Q) and W_P^(-r Q) = i^r:
    //   x[m] = t0 + t1 + t2 + t3,  x[m + Q] = (t0 - t2) + i (t1 - t3).
    // Round 1 (xor 2): lanes 0, 1 form t_r + t_(r+2); lanes 2, 3 form
    // t_(r-2) - t_r (lane 3 then times i).  Round 2 (xor 1) sums the pairs
    // and leaves each lane a quarter of the outputs.
    const int hb = (r >> 1) * Q;
    const float sgn = (r >> 1) ? -1.f : 1.f;
    const bool times_i = r == 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 sacc[Q];
#pragma unroll
      for (int n = 0; n < Q; ++n) {
        const float2 t = cmul(Z[c][n], cconj(wz[n]));
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, t.x, 2);
        o.y = __shfl_xor_sync(0xffffffffu, t.y, 2);
        const float2 v = make_float2(fmaf(sgn, t.x, o.x), fmaf(sgn, t.y, o.y));
        sacc[n] = times_i ? make_float2(-v.y, v.x) : v;
      }
      if constexpr (Q >= 2) {
#pragma unroll
        for (int n = 0; n < Q / 2; ++n) {
          const float2 keep = (r & 1) ? sacc[n + Q / 2] : sacc[n];
          const float2 give = (r & 1) ? sacc[n] : sacc[n + Q / 2];
          float2 o;
          o.x = __shfl_xor_sync(0xffffffffu, give.x, 1);
          o.y = __shfl_xor_sync(0xffffffffu, give.y, 1);
          const int idx = hb + (r & 1) * (Q / 2) + n;
          if (idx < nz) sm[(c * nz + idx) * PITCH + kyh] = cadd(keep, o);
        }
      } else {
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, sacc[0].x, 1);
        o.y = __shfl_xor_sync(0xffffffffu, sacc[0].y, 1);
        if ((r & 1) == 0 && hb < nz) sm[(c * nz + hb) * PITCH + kyh] = cadd(sacc[0], o);
      }
    }
  }
  __syncthreads();
  for (int l0 = 0; l0 < nlines; l0 += NT / S) {
    const int l = l0 + tid / S;
    line_fft<E, S, true, true, true>(l < nlines ? sm + l * PITCH : dummy, tid % S, twS);
  }
  // both halves' inverse-y rows are in shared memory
  cluster_sync_all();
  const float2* other = cluster_map(sm, (unsigned)(h ^ 1));
  const int L0 = (nlines + 1) >> 1;
  const int lb = h ? L0 : 0, le = h ? nlines : L0;
  {
    constexpr int kB = 4;  // independent remote loads in flight per thread
    const int cnt = (le - lb) * ny;
    for (int e0 = tid; e0 < cnt; e0 += NT * kB) {
      float2 rv[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int e = e0 + u * NT;
        if (e < cnt) rv[u] = other[(lb + e / ny) * PITCH + e % ny];
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int e = e0 + u * NT;
        if (e >= cnt) break;
        const int line = lb + e / ny, y = e % ny;
        const float2 tw = cconj(twS2[y]);
        const float2 own = sm[line * PITCH + y];
        // even half + W_Py^(-y) x odd half
        sm[line * PITCH + y] = h ? cadd(cmul(own, tw), rv[u]) : cadd(own, cmul(rv[u], tw));
      }
    }
  }
  if (bulk) {
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      for (int line = lb; line < le; ++line) bulk_store(w2 + kxoff + (long)line * ny, sm + line * PITCH, row_bytes);
      bulk_commit();
    }
  } else {
    __syncthreads();
    for (int e = tid; e < (le - lb) * ny; e += NT) {
      const int line = lb + e / ny, y = e % ny;
      w2[kxoff + (long)line * ny + y] = sm[line * PITCH + y];
    }
  }
  // the other CTA has finished reading this CTA's rows; this CTA's bulk
  // stores have read them before it exits
  cluster_sync_all();
  if (bulk && tid == 0) bulk_wait_read_all();
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int E, int S> static size_t xk_smem() { return sizeof(float2) * 3 * kRows * (LineFft<E, S>::kPitch + 1); }
template <int E, int S> static size_t yzh_smem(int nz) {
  return sizeof(float2) * ((3 * nz + 1) * YzhPitch<E, S>::value + 2 * E * S + 68);
}

template <int E, int S>
static mx_status xk_run(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup) {
  const size_t sm = xk_smem<E, S>();
  if (setup) {
    MX_CUDA_TRY(cudaFuncSetAttribute(xfk_kernel<E, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    MX_CUDA_TRY(cudaFuncSetAttribute(xik_kernel<E, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    MX_CUDA_TRY(cudaFuncSetAttribute(xil_kernel<E, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    MX_CUDA_TRY(cudaFuncSetAttribute(xil_kernel<E, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0, nsm = 0;
    MX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xfk_kernel<E, S>, 3 * kRows * S, sm));
    MX_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    ctx->xfk_grid = (per_sm > 0 ? per_sm : 1) * nsm;
    constexpr int M = E * S;
    std::vector<float2> t(M);
    for (int k = 0; k < E; ++k)
      for (int s = 0; s < S; ++s) {
        const double a = -2.0 * kPi * (double)(s * k) / (double)M;
        t[k * S + s] = make_float2((float)cos(a), (float)sin(a));
      }
    if (!ctx->tw_mk) MX_CUDA_TRY(cudaMalloc(&ctx->tw_mk, sizeof(float2) * M));
    MX_CUDA_TRY(cudaMemcpy(ctx->tw_mk, t.data(), sizeof(float2) * M, cudaMemcpyHostToDevice));
    return MX_OK;
  }
  const Grid& g = ctx->g;
  const int nblk = g.nz * ((g.ny + kRows - 1) / kRows);
  if (!inverse) {
    // persistent: as many blocks as fit on the device at once
    const int grid = nblk < ctx->xfk_grid ? nblk : ctx->xfk_grid;
    launch_pdl(xfk_kernel<E, S>, dim3(grid), dim3(3 * kRows * S), sm, st, m, g, (float)ctx->p.Ms, ctx->ms_map,
               ctx->w1, ctx->tw_mk, ctx->tw_x);
    return launch_check("xfk_kernel");
  }
  launch_pdl(xik_kernel<E, S>, dim3(nblk), dim3(3 * kRows * S), sm, st, ctx->w2, g, hd, ctx->tw_mk, ctx->tw_x);
  return launch_check("xik_kernel");
}

template <int E, int S>
static mx_status xl_run(mx_ctx* ctx, int mode, const StageIO& io, cudaStream_t st) {
  const Grid& g = ctx->g;
  const int nblk = g.nz * ((g.ny + kRows - 1) / kRows);
  const LocalCoef c = local_coef(ctx);
  if (c.dmi)
    launch_pdl(xil_kernel<E, S, true>, dim3(nblk), dim3(3 * kRows * S), xk_smem<E, S>(), st, ctx->w2, g, ctx->tw_mk,
               ctx->tw_x, io, c, mode, ctx->flag);
  else
    launch_pdl(xil_kernel<E, S, false>, dim3(nblk), dim3(3 * kRows * S), xk_smem<E, S>(), st, ctx->w2, g,
               ctx->tw_mk, ctx->tw_x, io, c, mode, ctx->flag);
  return launch_check("xil_kernel");
}

static mx_status xl_pass(mx_ctx* ctx, int mode, const StageIO& io, cudaStream_t st) {
  switch (ctx->g.Px / 2) {
    case 1024: return xl_run<32, 32>(ctx, mode, io, st);
    case 512: return xl_run<32, 16>(ctx, mode, io, st);
    case 256: return xl_run<16, 16>(ctx, mode, io, st);
    case 128: return xl_run<16, 8>(ctx, mode, io, st);
    case 64: return xl_run<8, 8>(ctx, mode, io, st);
    default: return MX_ERR_UNSUPPORTED;
  }
}

template <int E, int S, int P>
static mx_status yzh_run(mx_ctx* ctx, cudaStream_t st, bool setup) {
  const Grid& g = ctx->g;
  const size_t sm = yzh_smem<E, S>(g.nz);
  if (setup) {
    if (sm > 227 * 1024) return MX_ERR_UNSUPPORTED;
    MX_CUDA_TRY(cudaFuncSetAttribute(yzh_kernel<E, S, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return MX_OK;
  }
  yzh_kernel<E, S, P><<<2 * g.Hx, kPlaneNT, sm, st>>>(ctx->w1, ctx->w2, g, ctx->nhat, ctx->tw_y, ctx->tw_yh, ctx->tw_z,
                                                   ctx->flag, ctx->inject_wait_timeout ? 1 : 0);
  return launch_check("yzh_kernel");
}

static mx_status xk_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup) {
  switch (ctx->g.Px / 2) {
    case 1024: return xk_run<32, 32>(ctx, m, hd, inverse, st, setup);
    case 512: return xk_run<32, 16>(ctx, m, hd, inverse, st, setup);
    case 256: return xk_run<16, 16>(ctx, m, hd, inverse, st, setup);
    case 128: return xk_run<16, 8>(ctx, m, hd, inverse, st, setup);
    case 64: return xk_run<8, 8>(ctx, m, hd, inverse, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

template <int E, int S>
static mx_status yzh_pz(mx_ctx* ctx, cudaStream_t st, bool setup) {
  switch (ctx->g.Pz) {
    case 32: return yzh_run<E, S, 32>(ctx, st, setup);
    case 16: return yzh_run<E, S, 16>(ctx, st, setup);
    case 8: return yzh_run<E, S, 8>(ctx, st, setup);
    case 4: return yzh_run<E, S, 4>(ctx, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

static mx_status yzh_pass(mx_ctx* ctx, cudaStream_t st, bool setup) {
  switch (ctx->g.Py / 2) {
    case 1024: return yzh_pz<32, 32>(ctx, st, setup);
    case 512: return yzh_pz<32, 16>(ctx, st, setup);
    case 256: return yzh_pz<16, 16>(ctx, st, setup);
    case 128: return yzh_pz<16, 8>(ctx, st, setup);
    case 64: return yzh_pz<8, 8>(ctx, st, setup);
    case 32: return yzh_pz<32, 1>(ctx, st, setup);
    case 16: return yzh_pz<16, 1>(ctx, st, setup);
    default: return MX_ERR_UNSUPPORTED;
  }
}

mx_status plane_setup(mx_ctx* ctx) {
  MX_TRY(upload_w32());
  const int path = ctx->p.demag_path;
  const bool xk = path != MX_DEMAG_GENERIC && !ctx->fused_yz &&
                  xk_pass(ctx, nullptr, nullptr, false, nullptr, true) == MX_OK;
  // the four-CTA y/z kernel where it fits, else the two-CTA one
  // (MX_DEMAG_PLANE_PAIR forces the two-CTA kernel)
  ctx->quad = xk && path != MX_DEMAG_PLANE_PAIR && quad_pass(ctx, nullptr, true) == MX_OK;
  ctx->plane = ctx->quad || (xk && yzh_pass(ctx, nullptr, true) == MX_OK);
  ctx->g.oct4 = ctx->quad ? 1 : 0;
  ctx->xlocal = ctx->plane && path == MX_DEMAG_PLANE_XLOCAL;
  clear_error();
  if ((path == MX_DEMAG_PLANE || path == MX_DEMAG_PLANE_PAIR || path == MX_DEMAG_PLANE_XLOCAL) && !ctx->plane) {
    set_error("mx_create: the per-kx plane demag kernel does not support this grid");
    return MX_ERR_UNSUPPORTED;
  }
  if (ctx->xlocal && ctx->p.fft_mode != MX_FFT_FP32) {
    set_error("mx_create: MX_DEMAG_PLANE_XLOCAL needs fft_mode MX_FFT_FP32");
    return MX_ERR_UNSUPPORTED;
  }
  if (ctx->p.fft_mode == MX_FFT_SPLIT_BF16) {
    if (!ctx->plane) {
      set_error("mx_create: MX_FFT_SPLIT_BF16 needs the per-kx plane demag path");
      return MX_ERR_UNSUPPORTED;
    }
    MX_TRY(dft_x_pass(ctx, nullptr, nullptr, false, nullptr, true));
    MX_TRY(dft_gemm_setup(ctx));
  }
  return MX_OK;
}

mx_status plane_field(mx_ctx* ctx, const float4* m, float4* hd, cudaStream_t st) {
  const bool dft = ctx->p.fft_mode == MX_FFT_SPLIT_BF16;
  {
    ProfScope ps(ctx, KID_X_FWD, st);
    MX_TRY(dft ? dft_x_pass(ctx, m, nullptr, false, st, false) : xk_pass(ctx, m, nullptr, false, st, false));
  }
  {
    ProfScope ps(ctx, KID_YZ, st);
    MX_TRY(ctx->quad ? quad_pass(ctx, st, false) : yzh_pass(ctx, st, false));
  }
  {
    ProfScope ps(ctx, KID_X_INV, st);
    MX_TRY(dft ? dft_x_pass(ctx, nullptr, hd, true, st, false) : xk_pass(ctx, nullptr, hd, true, st, false));
  }
  return MX_OK;
}

mx_status plane_stage_xlocal(mx_ctx* ctx, int mode, const StageIO& io, cudaStream_t st) {
  if (mode < LM_RK4_S0 || mode > LM_EULER) {
    set_error("plane_stage_xlocal: bad mode");
    return MX_ERR_INVALID_ARG;
  }
  {
    ProfScope ps(ctx, KID_X_FWD, st);
    MX_TRY(xk_pass(ctx, io.m, nullptr, false, st, false));
  }
  {
    ProfScope ps(ctx, KID_YZ, st);
    MX_TRY(ctx->quad ? quad_pass(ctx, st, false) : yzh_pass(ctx, st, false));
  }
  ProfScope ps(ctx, KID_X_INV_LOCAL, st);
  return xl_pass(ctx, mode, io, st);
}

// plane-path octant (plane_octant_index) -> [comp][qz][qy][kx]
__global__ void octant_to_cmajor_kernel(const float* __restrict__ src, float* __restrict__ dst, Grid g) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long no = (long)g.Hx * g.Oy * g.Oz;
  if (idx >= 6 * no) return;
  const int kx = (int)(idx % g.Hx);
  const int qy = (int)((idx / g.Hx) % g.Oy);
  const int qz = (int)((idx / ((long)g.Hx * g.Oy)) % g.Oz);
  const int comp = (int)(idx / no);
  dst[idx] = src[plane_octant_index(g, kx, comp, qz, qy)];
}

mx_status plane_spectrum_out(mx_ctx* ctx, float* out, cudaStream_t st) {
  const long n = 6L * ctx->g.Hx * ctx->g.Oy * ctx->g.Oz;
  octant_to_cmajor_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctx->nhat, out, ctx->g);
  return launch_check("octant_to_cmajor_kernel");
}

}  // namespace mx
