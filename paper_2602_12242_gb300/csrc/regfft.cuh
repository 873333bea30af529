// Register-resident FFTs with compile-time sizes.
//
// RegFft<N>: an N-point DFT (N <= 32) on an array held in registers, radix-2
// decimation in time down to hand-written 8/4/2-point kernels; every index is
// a compile-time constant after unrolling.  Twiddles W_32^k come from a
// constant-memory table (uniform across the warp).
//
// line_fft<E, S>: an L = E*S point FFT of one line in shared memory computed
// by S threads of one warp (S divides 32) in two register steps:
//   1. thread s takes x[s + S n], n < E, does an E-point FFT over n and
//      multiplies output k1 by W_L^(s k1);
//   2. the E x S matrix goes through shared memory (rows padded to S+1 to
//      avoid bank conflicts); thread s then does S-point FFTs over s for
//      E/S values of k1, giving X[k1 + E k2].
// Only __syncwarp is needed: a line never leaves its warp.
#pragma once

#include <math.h>

#include "common.cuh"
#include "fft.cuh"

namespace mx {

// W_32^k = exp(-2 pi i k / 32); one copy per translation unit that includes
// this header, filled by upload_w32() from that unit.
static __constant__ float2 c_w32[32];

static inline mx_status upload_w32() {
  float2 w[32];
  for (int k = 0; k < 32; ++k) {
    const double a = -2.0 * kPi * k / 32.0;
    w[k] = make_float2((float)cos(a), (float)sin(a));
  }
  MX_CUDA_TRY(cudaMemcpyToSymbol(c_w32, w, sizeof(w)));
  return MX_OK;
}

template <int N, bool INV> struct RegFft {
  __device__ __forceinline__ static void run(float2* v) {
    float2 e[N / 2], o[N / 2];
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    RegFft<N / 2, INV>::run(e);
    RegFft<N / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) {
      float2 t = o[k];
      if (k > 0) {
        float2 w = c_w32[k * (32 / N)];
        if (INV) w.y = -w.y;
        t = cmul(t, w);
      }
      v[k] = cadd(e[k], t);
      v[k + N / 2] = csub(e[k], t);
    }
  }
};
// 16 points as 4 x 4: four 4-point DFTs over n1 of x[4 n1 + n2], the twiddles
// W_16^(n2 k1), four 4-point DFTs over n2; output k1 + 4 k2.  W_16^4 = -i and
// W_16^(2, 6) = (+-1 - i)/sqrt 2 take no general complex multiply.
template <bool INV> struct RegFft<16, INV> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) a[n2][n1] = v[4 * n1 + n2];
      Dft<4, INV, float2>::run(a[n2]);
    }
    const float c = (float)kSqrtHalf;
    auto w1 = [](float2 x) {  // W_16^1
      float2 w = c_w32[2];
      if (INV) w.y = -w.y;
      return cmul(x, w);
    };
    auto w3 = [](float2 x) {  // W_16^3
      float2 w = c_w32[6];
      if (INV) w.y = -w.y;
      return cmul(x, w);
    };
    auto w2 = [c](float2 x) {  // W_16^2 = W_8^1
      return INV ? make_float2(c * (x.x - x.y), c * (x.x + x.y)) : make_float2(c * (x.x + x.y), c * (x.y - x.x));
    };
    auto w6 = [c](float2 x) {  // W_16^6 = W_8^3
      return INV ? make_float2(-c * (x.x + x.y), c * (x.x - x.y)) : make_float2(c * (x.y - x.x), -c * (x.x + x.y));
    };
    a[1][1] = w1(a[1][1]);
    a[1][2] = w2(a[1][2]);
    a[1][3] = w3(a[1][3]);
    a[2][1] = w2(a[2][1]);
    a[2][2] = cmul_mi<INV>(a[2][2]);
    a[2][3] = w6(a[2][3]);
    a[3][1] = w3(a[3][1]);
    a[3][2] = w6(a[3][2]);
    {
      const float2 t = w1(a[3][3]);  // W_16^9 = -W_16^1
      a[3][3] = make_float2(-t.x, -t.y);
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      float2 b[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
      Dft<4, INV, float2>::run(b);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
    }
  }
};
template <bool INV> struct RegFft<8, INV> {
  __device__ __forceinline__ static void run(float2* v) { Dft<8, INV, float2>::run(v); }
};
template <bool INV> struct RegFft<4, INV> {
  __device__ __forceinline__ static void run(float2* v) { Dft<4, INV, float2>::run(v); }
};
template <bool INV> struct RegFft<2, INV> {
  __device__ __forceinline__ static void run(float2* v) { Dft<2, INV, float2>::run(v); }
};
template <bool INV> struct RegFft<1, INV> {
  __device__ __forceinline__ static void run(float2*) {}
};

// Shared-memory footprint (complex elements) of one line for line_fft<E, S>.
template <int E, int S> struct LineFft {
  static constexpr int L = E * S;
  static constexpr int kPitch = (S > 1) ? E * (S + 1) : E;
};

// Second step of line_fft: the twiddled E x S matrix is in rows k1 * (S + 1);
// thread s does S-point FFTs over s for k1 = s + S j and writes X[k1 + E k2]
// in natural order.
template <int E, int S, bool INV>
__device__ __forceinline__ void line_fft_step2(float2* line, int s) {
  float2 v[E];
  constexpr int J = E / S;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int k1 = s + S * j;
#pragma unroll
    for (int t = 0; t < S; ++t) v[j * S + t] = line[k1 * (S + 1) + t];
    RegFft<S, INV>::run(&v[j * S]);
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

// In-place FFT of `line` (natural order in and out).  `s` in [0, S); the S
// threads of a line are consecutive lanes of one warp.
// TW_KS: twL is the product table twL[k * S + s] = W_L^(s k) (k < E, s < S),
// which the S threads of a line read at consecutive addresses (no shared
// memory bank conflicts, coalesced global loads); otherwise twL[q] = W_L^q.
template <int E, int S, bool INV, bool TW_SHARED = false, bool TW_KS = false>
__device__ __forceinline__ void line_fft(float2* line, int s, const float2* __restrict__ twL) {
  static_assert(E >= S && (E % S) == 0 && S <= 32, "line_fft shape");
  float2 v[E];
#pragma unroll
  for (int n = 0; n < E; ++n) v[n] = line[s + S * n];
  RegFft<E, INV>::run(v);
  if (S == 1) {
#pragma unroll
    for (int n = 0; n < E; ++n) line[n] = v[n];
    return;
  }
#pragma unroll
  for (int k = 1; k < E; ++k) {
    const int ti = TW_KS ? k * S + s : s * k;
    float2 w = TW_SHARED ? twL[ti] : __ldg(&twL[ti]);
    if (INV) w.y = -w.y;
    v[k] = cmul(v[k], w);
  }
  __syncwarp();
  // row k1 of the E x S matrix at k1 * (S + 1)
#pragma unroll
  for (int k = 0; k < E; ++k) line[k * (S + 1) + s] = v[k];
  __syncwarp();
  line_fft_step2<E, S, INV>(line, s);
}

}  // namespace mx
