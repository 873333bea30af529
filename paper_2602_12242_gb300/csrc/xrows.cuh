// Row pieces of the compile-time-sized x transforms (demag_fast.cu, and the
// row kernels of the RK4 step and of the adjoint's reverse sweep): r2c of
// Ms m rows into the spectrum w1[c][row][kx], c2r of spectrum rows into
// shared memory, and the few-row block configuration of each size.  The same
// arithmetic as demag.cu's generic x kernels (Sec. II-B: zero-padded FFT
// convolution), on the register or Stockham line transforms.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "regfft.cuh"

namespace mx {

// Threads of a few-row x block (most of them only load and store).
constexpr int kFewRowsNT = 192;

// Threads of the x kernels' FFT phase: the 3R lines of S threads, rounded up
// to whole warps (the extra threads transform scratch lines).  The load and
// store phases use all NT >= that many threads, so that a block with few
// rows still has many memory requests in flight.
template <int S, int R> struct XfShape {
  static constexpr int NF = (3 * R * S + 31) / 32 * 32;
  static constexpr int lines = NF / S;  // shared-memory lines, scratch included
};

// The 3R line transforms of M = E*S points of an x kernel's block, in place
// in shared memory (line l at l * P), ending with a block barrier.  Where
// every thread can take whole radix-8 butterflies (3RM / NT >= 8 elements
// each) all NT threads run the Stockham passes of block_fft (short chains per
// thread, a barrier per pass); otherwise the NF threads of the lines run the
// two-step register transform (twM[q] = W_M^q either way).
template <int E, int S, int R, int NT, bool INV>
__device__ __forceinline__ void x_line_ffts(float2* sm, const float2* __restrict__ twM) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch;
  constexpr int EPT = 3 * R * M / NT;
  if constexpr ((3 * R * M) % NT == 0 && EPT >= 8) {
    block_fft<INV, float2, EPT, NT>(sm, M, 3 * R, lines1(P), 1, twM, 1);
  } else {
    if ((int)threadIdx.x < XfShape<S, R>::NF) line_fft<E, S, INV>(sm + (threadIdx.x / S) * P, threadIdx.x % S, twM);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// x forward (r2c), R rows per block, 3R lines of M = E*S points.
// ---------------------------------------------------------------------------
// Rows row0 .. row0 + R - 1 of Ms m (the real row packed as z[n] = x[2n] +
// i x[2n+1]) through the line FFT and the split step into w1.  COHERENT reads
// m with plain loads (m written earlier in the same kernel), else through the
// read-only path.
template <int E, int S, int R, int NT, bool COHERENT>
__device__ __forceinline__ void xf_rows(float2* sm, const float4* __restrict__ m, const Grid& g, float ms,
                                        const float* __restrict__ ms_map, float2* __restrict__ w1, int row0,
                                        const float2* __restrict__ twM, const float2* __restrict__ twP) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch;
  constexpr int NF = XfShape<S, R>::NF;
  static_assert(NT >= NF && NT % 32 == 0, "xf thread count");
  const int nrows = g.ny * g.nz;
  const int tid = threadIdx.x;
  // batches of kB cell pairs per thread: 2 kB independent loads in flight
  constexpr int kB = (R * M + NT - 1) / NT < 4 ? (R * M + NT - 1) / NT : 4;
  for (int e0 = tid; e0 < R * M; e0 += NT * kB) {
    float4 a[kB], b[kB];
    float sa[kB], sb[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * NT;
      const int r = e / M, n = e % M;
      const int row = row0 + r;
      a[u] = b[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      sa[u] = sb[u] = ms;
      if (e < R * M && row < nrows) {
        const long cell = (long)row * g.nx;
        const int i0 = 2 * n, i1 = i0 + 1;
        if (i0 < g.nx) {
          a[u] = COHERENT ? m[cell + i0] : __ldg(&m[cell + i0]);
          if (ms_map) sa[u] = __ldg(&ms_map[cell + i0]);
        }
        if (i1 < g.nx) {
          b[u] = COHERENT ? m[cell + i1] : __ldg(&m[cell + i1]);
          if (ms_map) sb[u] = __ldg(&ms_map[cell + i1]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * NT;
      if (e >= R * M) break;
      const int r = e / M, n = e % M;
      // zero outside the grid (a, b are zero there)
      sm[(3 * r + 0) * P + n] = make_float2(sa[u] * a[u].x, sb[u] * b[u].x);
      sm[(3 * r + 1) * P + n] = make_float2(sa[u] * a[u].y, sb[u] * b[u].y);
      sm[(3 * r + 2) * P + n] = make_float2(sa[u] * a[u].z, sb[u] * b[u].z);
    }
  }
  __syncthreads();
  x_line_ffts<E, S, R, NT, false>(sm, twM);
  const long cs = (long)g.nz * g.ny * g.Hx;
  // batches of kB outputs per thread: the twiddle loads of a batch go out together
  constexpr int kBo = (3 * R * (M + 1) + NT - 1) / NT <= 9 ? (3 * R * (M + 1) + NT - 1) / NT : 4;
  for (int e0 = tid; e0 < 3 * R * (M + 1); e0 += NT * kBo) {
    float2 tw[kBo];
#pragma unroll
    for (int u = 0; u < kBo; ++u) {
      const int e = e0 + u * NT;
      tw[u] = e < 3 * R * (M + 1) ? __ldg(&twP[e % (M + 1)]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < kBo; ++u) {
      const int e = e0 + u * NT;
      if (e >= 3 * R * (M + 1)) break;
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
      w1[c * cs + (long)row * g.Hx + k] = cadd(Ev, cmul(tw[u], O));
    }
  }
}

// The c2r transforms of rows row0 .. row0 + R - 1 into shared memory:
// afterwards element n of line 3 r + c holds H_c of cells 2n (real part) and
// 2n + 1 (imaginary part) of row row0 + r.
template <int E, int S, int R, int NT>
__device__ __forceinline__ void xi_rows(float2* sm, const float2* __restrict__ w1, const Grid& g, int row0,
                                        const float2* __restrict__ twM, const float2* __restrict__ twP) {
  constexpr int M = E * S;
  constexpr int P = LineFft<E, S>::kPitch;
  constexpr int NF = XfShape<S, R>::NF;
  static_assert(NT >= NF && NT % 32 == 0, "xi thread count");
  const int nrows = g.ny * g.nz;
  const int tid = threadIdx.x;
  const long cs = (long)g.nz * g.ny * g.Hx;
  // batches of kB elements per thread: 2 kB independent loads in flight
  constexpr int kB = (3 * R * M + NT - 1) / NT <= 8 ? (3 * R * M + NT - 1) / NT : 4;
  for (int e0 = tid; e0 < 3 * R * M; e0 += NT * kB) {
    float2 A[kB], Bv[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * NT;
      const int line = e / M, k = e % M;
      const int r = line / 3, c = line % 3;
      A[u] = Bv[u] = make_float2(0.f, 0.f);
      if (e < 3 * R * M && row0 + r < nrows) {
        const float2* X = w1 + c * cs + (long)(row0 + r) * g.Hx;
        A[u] = __ldg(&X[k]);
        Bv[u] = __ldg(&X[M - k]);
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * NT;
      if (e >= 3 * R * M) break;
      const int k = e % M;
      const float2 a = A[u], b = cconj(Bv[u]);
      const float2 Sv = cadd(a, b);
      const float2 t = cmul(cconj(__ldg(&twP[k])), csub(a, b));
      sm[(e / M) * P + k] = make_float2(Sv.x - t.y, Sv.y + t.x);
    }
  }
  __syncthreads();
  x_line_ffts<E, S, R, NT, true>(sm, twM);
}

// H_demag of cell i of row r from the c2r lines
template <int E, int S>
__device__ __forceinline__ float3 xi_cell(const float2* sm, int r, int i) {
  constexpr int P = LineFft<E, S>::kPitch;
  const float2* L = sm + (3 * r) * P + (i >> 1);
  const float2 hx = L[0], hy = L[P], hz = L[2 * P];
  return (i & 1) ? make_float3(hx.y, hy.y, hz.y) : make_float3(hx.x, hy.x, hz.x);
}

// x blocks of a grid: many rows per block (many_rows(M) of them) unless that
// gives fewer than kMinBlocks blocks; then the few-row blocks below.
constexpr int kMinBlocks = 2 * 152;
inline int many_rows(int half) {
  switch (half) {
    case 1024: return 2;
    case 512:
    case 256: return 4;
    case 128:
    case 64: return 8;
    default: return 32;
  }
}
inline bool few_rows(const Grid& g) {
  const int rb = many_rows(g.Px / 2);
  return (g.ny * g.nz + rb - 1) / rb < kMinBlocks;
}

// Threads of the few-row block with R rows of S-thread lines.
template <int S, int R> constexpr int few_rows_nt() {
  return XfShape<S, R>::NF > kFewRowsNT ? XfShape<S, R>::NF : kFewRowsNT;
}

// Calls f.template run<E, S, R, NT>() for the few-row x configuration of
// M = Px/2 (E x S points per line, R rows per block); MX_ERR_UNSUPPORTED for
// sizes without one.
template <class F> mx_status few_rows_dispatch(int half, F& f) {
  switch (half) {
    case 1024: return f.template run<32, 32, 1, few_rows_nt<32, 1>()>();
    case 512: return f.template run<32, 16, 1, few_rows_nt<16, 1>()>();
    case 256: return f.template run<16, 16, 1, few_rows_nt<16, 1>()>();
    case 128: return f.template run<16, 8, 1, few_rows_nt<8, 1>()>();
    case 64: return f.template run<8, 8, 2, few_rows_nt<8, 2>()>();
    case 32: return f.template run<32, 1, 4, few_rows_nt<1, 4>()>();
    case 16: return f.template run<16, 1, 4, few_rows_nt<1, 4>()>();
    default: return MX_ERR_UNSUPPORTED;
  }
}

}  // namespace mx
