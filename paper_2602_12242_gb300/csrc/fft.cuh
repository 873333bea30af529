// Block-level FFT on data staged in shared memory.
//
// Radix-8/4/2 Stockham passes (self-sorting, so the result is in natural
// order).  In pass p with sub-transform length Ns (the product of the radices
// of the earlier passes) and radix R, butterfly group j of a line reads the R
// elements j + r L/R, multiplies element r by W_{Ns R}^{r (j mod Ns)}, applies
// an R-point DFT in registers and writes element r to
// (j div Ns) Ns R + (j mod Ns) + r Ns.  Every thread first loads all of its
// groups into registers, the block synchronises, and then the groups are
// written back in place, so no second buffer is needed.
//
// Twiddles come from a table of W_L^q = exp(-2 pi i q / L) computed in FP64 on
// the host and rounded once to the element type.
#pragma once

#include "common.cuh"

namespace mx {

constexpr double kSqrtHalf = 0.70710678118654752440;

// R-point DFT in registers; forward sign exp(-2 pi i n k / R), inverse +.
template <int R, bool INV, typename C> struct Dft;

template <bool INV, typename C> struct Dft<1, INV, C> {
  __device__ __forceinline__ static void run(C*) {}
};

template <bool INV, typename C> struct Dft<2, INV, C> {
  __device__ __forceinline__ static void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV, typename C> struct Dft<4, INV, C> {
  __device__ __forceinline__ static void run(C* v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = cmul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV, typename C> struct Dft<8, INV, C> {
  __device__ __forceinline__ static void run(C* v) {
    typedef typename real_of<C>::type T;
    const T c = (T)kSqrtHalf;
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV, C>::run(e);
    Dft<4, INV, C>::run(o);
    // o[k] *= W_8^k
    C o1 = INV ? mkc<C>(c * (o[1].x - o[1].y), c * (o[1].x + o[1].y))
               : mkc<C>(c * (o[1].x + o[1].y), c * (o[1].y - o[1].x));
    C o2 = cmul_mi<INV>(o[2]);
    C o3 = INV ? mkc<C>(-c * (o[3].x + o[3].y), c * (o[3].x - o[3].y))
               : mkc<C>(c * (o[3].y - o[3].x), -c * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// Where line l starts in shared memory: l = a + n1 (b + n2 c) with
// a < n1, b < n2  ->  a s1 + b s2 + c s3.
struct Lines {
  int n1, s1, n2, s2, s3;
  __device__ __forceinline__ int base(int l) const {
    int a = l % n1;
    int b = l / n1;
    return a * s1 + (b % n2) * s2 + (b / n2) * s3;
  }
};

__host__ __device__ inline Lines lines1(int stride) { return Lines{1 << 30, stride, 1, 0, 0}; }

template <int R, bool INV, typename C, int EPT, int NT>
__device__ __forceinline__ void fft_pass(C* s, int L, int Ns, int nlines, const Lines& ln, int es,
                                         bool elems_fast, const C* __restrict__ tw, int tws) {
  constexpr int G = EPT / R;
  const int LR = L / R;
  const int total = nlines * LR;
  const int tstep = (L / (Ns * R)) * tws;  // table stride of W_{Ns R}
  C v[G * R];
  int bb[G], jj[G];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    int g = threadIdx.x + q * NT;
    jj[q] = -1;
    if (g < total) {
      int line, j;
      if (elems_fast) {
        j = g % LR;
        line = g / LR;
      } else {
        line = g % nlines;
        j = g / nlines;
      }
      int b = ln.base(line);
      bb[q] = b;
      jj[q] = j;
      int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = s[b + (j + r * LR) * es];
        if (r > 0 && Ns > 1) {
          C w = __ldg(&tw[r * k * tstep]);
          if (INV) w.y = -w.y;
          x = cmul(x, w);
        }
        v[q * R + r] = x;
      }
      Dft<R, INV, C>::run(&v[q * R]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < G; ++q) {
    if (jj[q] >= 0) {
      int j = jj[q];
      int k = j & (Ns - 1);
      int o = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[bb[q] + (o + r * Ns) * es] = v[q * R + r];
    }
  }
  __syncthreads();
}

// nlines FFTs of length L (a power of two, 1..4096) on shared memory s.
// Element e of line l is s[ln.base(l) + e * es].  Requires
// nlines * L <= NT * EPT.  tw[q * tws] = W_L^q.  Unnormalised both ways.
template <bool INV, typename C, int EPT, int NT>
__device__ void block_fft(C* s, int L, int nlines, const Lines& ln, int es, const C* __restrict__ tw,
                          int tws) {
  const bool elems_fast = (es == 1);
  int Ns = 1;
  while (Ns < L) {
    int rem = L / Ns;
    if (rem >= 8) {
      fft_pass<8, INV, C, EPT, NT>(s, L, Ns, nlines, ln, es, elems_fast, tw, tws);
      Ns *= 8;
    } else if (rem == 4) {
      fft_pass<4, INV, C, EPT, NT>(s, L, Ns, nlines, ln, es, elems_fast, tw, tws);
      Ns *= 4;
    } else {
      fft_pass<2, INV, C, EPT, NT>(s, L, Ns, nlines, ln, es, elems_fast, tw, tws);
      Ns *= 2;
    }
  }
}

inline int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

}  // namespace mx
