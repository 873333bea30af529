// Demag kernel build (Sec. II-B: the demagnetisation tensor of Newell,
// Williams & Dunlop on the zero-padded grid of Nakatani et al. / Hayashi et
// al., then its FFT).  Runs once per geometry; everything here is FP64.
//
// Tensor convention: H_i = -sum_j N_ij(r - r') M_j(r'), so a cube's
// self-factors are 1/3.  N(R) is the field of a uniformly magnetised cell
// averaged over another cell R away:
//   N_ij(R) = -1/(4 pi V) Int_{[-h,h]^3} L(u) d_i d_j (1/|R + u|) du,
//   L(u) = prod_k (h_k - |u_k|).
// Near the source it is evaluated with Newell's closed form (auxiliary
// functions f, g and the (-1, 2, -1)^3 second-difference stencil); the
// stencil cancels catastrophically with distance (relative error about
// eps (R/h)^6), so beyond 6 smallest cell edges the integral above is
// evaluated directly with Gauss-Legendre rules on each half of each axis.
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <vector>

#include "common.cuh"
#include "fft.cuh"

namespace mx {

// ---------------------------------------------------------------------------
// Gauss-Legendre rules for n in {3,4,6,8,12,16}, nodes on [0,1] and weights
// summing to 1, in constant memory.  Computed on the host by Newton's method
// from Tricomi's initial estimates of the roots of P_n.
// ---------------------------------------------------------------------------
constexpr int kNumRules = 6;
__constant__ int c_rule_n[kNumRules];
__constant__ int c_rule_off[kNumRules];
__constant__ double c_gl_x[64];
__constant__ double c_gl_w[64];

static void legendre_rule(int n, double* x01, double* w01) {
  for (int i = 1; i <= n; ++i) {
    double th = kPi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
    double t = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
    double der = 1.0;
    for (int it = 0; it < 60; ++it) {
      // P_n(t) and P_n'(t) by the three-term recurrence
      double pm1 = 1.0, p = t;
      for (int k = 2; k <= n; ++k) {
        double pn = (2.0 * k - 1.0) / k * t * p - (k - 1.0) / k * pm1;
        pm1 = p;
        p = pn;
      }
      der = n * (pm1 - t * p) / (1.0 - t * t);
      double step = p / der;
      t -= step;
      if (fabs(step) <= 1e-17) break;
    }
    double w = 2.0 / ((1.0 - t * t) * der * der);
    x01[i - 1] = 0.5 * (1.0 + t);
    w01[i - 1] = 0.5 * w;
  }
}

static bool g_rules_ready[64] = {false};

static mx_status upload_rules() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && g_rules_ready[dev]) return MX_OK;
  const int ns[kNumRules] = {3, 4, 6, 8, 12, 16};
  int off[kNumRules];
  double x[64], w[64];
  int o = 0;
  for (int r = 0; r < kNumRules; ++r) {
    off[r] = o;
    legendre_rule(ns[r], x + o, w + o);
    o += ns[r];
  }
  MX_CUDA_TRY(cudaMemcpyToSymbol(c_rule_n, ns, sizeof(ns)));
  MX_CUDA_TRY(cudaMemcpyToSymbol(c_rule_off, off, sizeof(off)));
  MX_CUDA_TRY(cudaMemcpyToSymbol(c_gl_x, x, sizeof(double) * o));
  MX_CUDA_TRY(cudaMemcpyToSymbol(c_gl_w, w, sizeof(double) * o));
  if (dev < 64) g_rules_ready[dev] = true;
  return MX_OK;
}

// ---------------------------------------------------------------------------
// Newell's auxiliary functions.  A term whose polynomial factor is zero
// contributes zero (its transcendental factor may be singular there).
// ---------------------------------------------------------------------------
__device__ double aux_f(double x, double y, double z) {
  const double xx = x * x, yy = y * y, zz = z * z;
  const double r = sqrt(xx + yy + zz);
  if (r == 0.0) return 0.0;
  double acc = (2.0 * xx - yy - zz) * r * (1.0 / 6.0);
  const double a = 0.5 * y * (zz - xx);
  if (a != 0.0) acc += a * asinh(y / sqrt(xx + zz));
  const double b = 0.5 * z * (yy - xx);
  if (b != 0.0) acc += b * asinh(z / sqrt(xx + yy));
  const double c = x * y * z;
  if (c != 0.0) acc -= c * atan((y * z) / (x * r));
  return acc;
}

__device__ double aux_g(double x, double y, double z) {
  const double xx = x * x, yy = y * y, zz = z * z;
  const double r = sqrt(xx + yy + zz);
  if (r == 0.0) return 0.0;
  double acc = -x * y * r * (1.0 / 3.0);
  const double xyz = x * y * z;
  if (xyz != 0.0) acc += xyz * asinh(z / sqrt(xx + yy));
  const double a = y * (3.0 * zz - yy) * (1.0 / 6.0);
  if (a != 0.0) acc += a * asinh(x / sqrt(yy + zz));
  const double b = x * (3.0 * zz - xx) * (1.0 / 6.0);
  if (b != 0.0) acc += b * asinh(y / sqrt(xx + zz));
  const double c = zz * z * (1.0 / 6.0);
  if (c != 0.0) acc -= c * atan((x * y) / (z * r));
  const double d = 0.5 * z * yy;
  if (d != 0.0) acc -= d * atan((x * z) / (y * r));
  const double e = 0.5 * z * xx;
  if (e != 0.0) acc -= e * atan((y * z) / (x * r));
  return acc;
}

// Stencil sum_{a,b,c} w_a w_b w_c F(X + a hx, ...), w = (-1, 2, -1), / (4 pi V).
template <bool OFFDIAG>
__device__ double stencil27(double X, double Y, double Z, double hx, double hy, double hz) {
  double s = 0.0;
  for (int c = -1; c <= 1; ++c) {
    const double wc = (c == 0) ? 2.0 : -1.0;
    for (int b = -1; b <= 1; ++b) {
      const double wb = (b == 0) ? 2.0 : -1.0;
      for (int a = -1; a <= 1; ++a) {
        const double wa = (a == 0) ? 2.0 : -1.0;
        const double u = X + a * hx, v = Y + b * hy, w = Z + c * hz;
        s += wa * wb * wc * (OFFDIAG ? aux_g(u, v, w) : aux_f(u, v, w));
      }
    }
  }
  return s / (4.0 * kPi * hx * hy * hz);
}

__device__ void closed_form(double X, double Y, double Z, double hx, double hy, double hz, double* t) {
  t[0] = stencil27<false>(X, Y, Z, hx, hy, hz);
  t[1] = stencil27<false>(Y, X, Z, hy, hx, hz);
  t[2] = stencil27<false>(Z, Y, X, hz, hy, hx);
  t[3] = stencil27<true>(X, Y, Z, hx, hy, hz);
  t[4] = stencil27<true>(X, Z, Y, hx, hz, hy);
  t[5] = stencil27<true>(Y, Z, X, hy, hz, hx);
}

// Direct quadrature of the defining integral with rule index ri.
__device__ void quadrature(double X, double Y, double Z, double hx, double hy, double hz, int ri, double* t) {
  const int n = c_rule_n[ri], o = c_rule_off[ri];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  // u_k runs over Gauss nodes of [0, h] and their mirror in [-h, 0];
  // the tent weight (h - |u|) is folded into the node weight.
  for (int ic = 0; ic < 2 * n; ++ic) {
    const double gz = c_gl_x[o + (ic % n)];
    const double uz = (ic < n ? 1.0 : -1.0) * hz * gz;
    const double wz = c_gl_w[o + (ic % n)] * hz * (hz - fabs(uz));
    const double rz = Z + uz;
    for (int ib = 0; ib < 2 * n; ++ib) {
      const double gy = c_gl_x[o + (ib % n)];
      const double uy = (ib < n ? 1.0 : -1.0) * hy * gy;
      const double wy = c_gl_w[o + (ib % n)] * hy * (hy - fabs(uy));
      const double ry = Y + uy;
      const double wzy = wz * wy;
      for (int ia = 0; ia < 2 * n; ++ia) {
        const double gx = c_gl_x[o + (ia % n)];
        const double ux = (ia < n ? 1.0 : -1.0) * hx * gx;
        const double wx = c_gl_w[o + (ia % n)] * hx * (hx - fabs(ux));
        const double rx = X + ux;
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double inv = rsqrt(r2);
        const double inv2 = inv * inv;
        const double q = wzy * wx * inv * inv2 * inv2;  // weight / r^5
        const double q3 = 3.0 * q;
        acc[0] += q3 * rx * rx - q * r2;
        acc[1] += q3 * ry * ry - q * r2;
        acc[2] += q3 * rz * rz - q * r2;
        acc[3] += q3 * rx * ry;
        acc[4] += q3 * rx * rz;
        acc[5] += q3 * ry * rz;
      }
    }
  }
  const double s = -1.0 / (4.0 * kPi * hx * hy * hz);
  for (int k = 0; k < 6; ++k) t[k] = acc[k] * s;
}

// Rule choice from the gap between the singular point -R and the box
// [-h, h]^3, in units of the largest cell edge.
__device__ int rule_for_gap(double gap) {
  if (gap >= 64.0) return 0;   // n = 3
  if (gap >= 24.0) return 1;   // n = 4
  if (gap >= 10.0) return 2;   // n = 6
  if (gap >= 4.0) return 3;    // n = 8
  if (gap >= 2.0) return 4;    // n = 12
  return 5;                    // n = 16
}

__global__ void tensor_octant_kernel(int nx, int ny, int nz, double hx, double hy, double hz, double* out) {
  const long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nc = (long)nx * ny * nz;
  if (cell >= nc) return;
  const int i = (int)(cell % nx);
  const int j = (int)((cell / nx) % ny);
  const int k = (int)(cell / ((long)nx * ny));
  const double X = i * hx, Y = j * hy, Z = k * hz;
  const double hmin = fmin(hx, fmin(hy, hz));
  const double hmax = fmax(hx, fmax(hy, hz));
  const double R = sqrt(X * X + Y * Y + Z * Z);
  const double ex = fmax(X - hx, 0.0), ey = fmax(Y - hy, 0.0), ez = fmax(Z - hz, 0.0);
  const double gap = sqrt(ex * ex + ey * ey + ez * ez) / hmax;
  double t[6];
  if (R < 6.0 * hmin || gap < 1.0)
    closed_form(X, Y, Z, hx, hy, hz, t);
  else
    quadrature(X, Y, Z, hx, hy, hz, rule_for_gap(gap), t);
  for (int c = 0; c < 6; ++c) out[c * nc + cell] = t[c];
}

// Place component c of the octant on the padded grid (complex, imag 0):
// padded index x holds offset X = x (x < nx) or x - Px (x > Px - nx), using
// the component's parity for negative offsets; other points are zero.
__global__ void scatter_padded_kernel(const double* oct, int comp, Grid g, double2* buf) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long np = (long)g.Px * g.Py * g.Pz;
  if (idx >= np) return;
  const int x = (int)(idx % g.Px);
  const int y = (int)((idx / g.Px) % g.Py);
  const int z = (int)(idx / ((long)g.Px * g.Py));
  int X = (x < g.nx) ? x : ((x > g.Px - g.nx) ? x - g.Px : INT32_MAX);
  int Y = (y < g.ny) ? y : ((y > g.Py - g.ny) ? y - g.Py : INT32_MAX);
  int Z = (z < g.nz) ? z : ((z > g.Pz - g.nz) ? z - g.Pz : INT32_MAX);
  double v = 0.0;
  if (X != INT32_MAX && Y != INT32_MAX && Z != INT32_MAX) {
    // parity: xx,yy,zz even; xy odd in X,Y; xz odd in X,Z; yz odd in Y,Z
    const bool oddx = (comp == 3 || comp == 4), oddy = (comp == 3 || comp == 5), oddz = (comp == 4 || comp == 5);
    double sgn = 1.0;
    if (oddx && X < 0) sgn = -sgn;
    if (oddy && Y < 0) sgn = -sgn;
    if (oddz && Z < 0) sgn = -sgn;
    const long o = ((long)abs(Z) * g.ny + abs(Y)) * g.nx + abs(X);
    v = sgn * oct[(long)comp * g.nx * g.ny * g.nz + o];
  }
  buf[idx] = make_double2(v, 0.0);
}

// Forward FFT along one axis of a complex FP64 array viewed as
// [outer][L][inner].  inner == 1: a block transforms `rows` contiguous lines;
// otherwise a block transforms `cols` consecutive inner columns of one outer
// index.
constexpr int kF64Threads = 256, kF64Ept = 16;

__global__ void __launch_bounds__(kF64Threads) fft_axis_f64_kernel(double2* data, int L, long inner, long outer,
                                                                   int tile, const double2* __restrict__ tw) {
  extern __shared__ double2 sm64[];
  if (inner == 1) {
    const long row0 = (long)blockIdx.x * tile;
    const int nrows = (int)min((long)tile, outer - row0);
    for (int e = threadIdx.x; e < nrows * L; e += blockDim.x) sm64[e] = data[row0 * L + e];
    __syncthreads();
    block_fft<false, double2, kF64Ept, kF64Threads>(sm64, L, nrows, lines1(L), 1, tw, 1);
    for (int e = threadIdx.x; e < nrows * L; e += blockDim.x) data[row0 * L + e] = sm64[e];
  } else {
    const long tiles_per_outer = (inner + tile - 1) / tile;
    const long ob = blockIdx.x / tiles_per_outer;
    const long c0 = (blockIdx.x % tiles_per_outer) * tile;
    const int ncol = (int)min((long)tile, inner - c0);
    double2* base = data + ob * L * inner + c0;
    for (int e = threadIdx.x; e < ncol * L; e += blockDim.x) {
      const int l = e / ncol, c = e % ncol;
      sm64[l * ncol + c] = base[(long)l * inner + c];
    }
    __syncthreads();
    block_fft<false, double2, kF64Ept, kF64Threads>(sm64, L, ncol, lines1(1), ncol, tw, 1);
    for (int e = threadIdx.x; e < ncol * L; e += blockDim.x) {
      const int l = e / ncol, c = e % ncol;
      base[(long)l * inner + c] = sm64[l * ncol + c];
    }
  }
}

// Keep the real part of the octant kx <= Px/2, ky <= Py/2, kz <= Pz/2,
// scaled by -1/(Px Py Pz), in FP32.  Also record max |imag| / max |real| of
// the whole spectrum (a check that the symmetric tensor's spectrum is real).
__global__ void extract_octant_kernel(const double2* buf, int comp, Grid g, float* nhat, int kxmajor,
                                      unsigned long long* max_re, unsigned long long* max_im) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long no = (long)g.Hx * g.Oy * g.Oz;
  if (idx >= no) return;
  const int kx = (int)(idx % g.Hx);
  const int ky = (int)((idx / g.Hx) % g.Oy);
  const int kz = (int)(idx / ((long)g.Hx * g.Oy));
  const double2 v = buf[((long)kz * g.Py + ky) * g.Px + kx];
  const double scale = -1.0 / ((double)g.Px * g.Py * g.Pz);
  const long dst = kxmajor ? plane_octant_index(g, kx, comp, kz, ky) : (long)comp * no + idx;
  nhat[dst] = (float)(v.x * scale);
  // warp maxima first, then one atomic per warp
  unsigned long long re = (unsigned long long)__double_as_longlong(fabs(v.x));
  unsigned long long im = (unsigned long long)__double_as_longlong(fabs(v.y));
  const unsigned mask = __activemask();
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long r2 = __shfl_down_sync(mask, re, o);
    const unsigned long long i2 = __shfl_down_sync(mask, im, o);
    if ((threadIdx.x & 31) + o < 32 && ((mask >> ((threadIdx.x & 31) + o)) & 1)) {
      re = r2 > re ? r2 : re;
      im = i2 > im ? i2 : im;
    }
  }
  if ((threadIdx.x & 31) == (__ffs(mask) - 1)) {
    atomicMax(max_re, re);
    atomicMax(max_im, im);
  }
}

static mx_status fft3_f64(double2* buf, const Grid& g, const double2* twx, const double2* twy,
                          const double2* twz, cudaStream_t st) {
  const int cap = kF64Threads * kF64Ept;
  const size_t smem = sizeof(double2) * cap;
  MX_CUDA_TRY(cudaFuncSetAttribute(fft_axis_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  struct Ax { int L; long inner, outer; const double2* tw; } ax[3] = {
      {g.Px, 1, (long)g.Py * g.Pz, twx}, {g.Py, g.Px, g.Pz, twy}, {g.Pz, (long)g.Px * g.Py, 1, twz}};
  for (int a = 0; a < 3; ++a) {
    if (ax[a].L == 1) continue;
    const int tile = cap / ax[a].L;
    long blocks;
    if (ax[a].inner == 1)
      blocks = (ax[a].outer + tile - 1) / tile;
    else
      blocks = ax[a].outer * ((ax[a].inner + tile - 1) / tile);
    fft_axis_f64_kernel<<<(unsigned)blocks, kF64Threads, smem, st>>>(buf, ax[a].L, ax[a].inner, ax[a].outer, tile,
                                                                      ax[a].tw);
    MX_TRY(launch_check("fft_axis_f64_kernel"));
  }
  return MX_OK;
}

static std::vector<double2> twiddles64(int L) {
  std::vector<double2> t(L);
  for (int q = 0; q < L; ++q) {
    const double a = -2.0 * kPi * q / L;
    t[q] = make_double2(cos(a), sin(a));
  }
  return t;
}

mx_status build_demag_kernel(mx_ctx* ctx, cudaStream_t st) {
  const Grid& g = ctx->g;
  MX_TRY(upload_rules());
  const long nc = g.ncell;
  if (!ctx->t_real) MX_CUDA_TRY(cudaMalloc(&ctx->t_real, sizeof(double) * 6 * nc));
  tensor_octant_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, st>>>(g.nx, g.ny, g.nz, ctx->p.dx, ctx->p.dy,
                                                                     ctx->p.dz, ctx->t_real);
  MX_TRY(launch_check("tensor_octant_kernel"));

  const long np = (long)g.Px * g.Py * g.Pz;
  double2 *buf = nullptr, *tw = nullptr;
  unsigned long long* mx = nullptr;
  mx_status status = MX_OK;
  std::vector<double2> hx = twiddles64(g.Px), hy = twiddles64(g.Py), hz = twiddles64(g.Pz);
  if (cudaMalloc(&buf, sizeof(double2) * np) != cudaSuccess ||
      cudaMalloc(&tw, sizeof(double2) * (g.Px + g.Py + g.Pz)) != cudaSuccess ||
      cudaMalloc(&mx, sizeof(unsigned long long) * 2) != cudaSuccess) {
    cudaGetLastError();
    set_error("mx_build_demag_kernel: FP64 scratch allocation failed");
    status = MX_ERR_OOM;
  }
  if (status == MX_OK) {
    cudaMemcpyAsync(tw, hx.data(), sizeof(double2) * g.Px, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(tw + g.Px, hy.data(), sizeof(double2) * g.Py, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(tw + g.Px + g.Py, hz.data(), sizeof(double2) * g.Pz, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 2, st);
    const int ncomp = 6;
    for (int c = 0; c < ncomp && status == MX_OK; ++c) {
      scatter_padded_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(ctx->t_real, c, g, buf);
      status = launch_check("scatter_padded_kernel");
      if (status == MX_OK) status = fft3_f64(buf, g, tw, tw + g.Px, tw + g.Px + g.Py, st);
      if (status == MX_OK) {
        const long no = (long)g.Hx * g.Oy * g.Oz;
        extract_octant_kernel<<<(unsigned)((no + 255) / 256), 256, 0, st>>>(buf, c, g, ctx->nhat, ctx->plane ? 1 : 0,
                                                                             mx, mx + 1);
        status = launch_check("extract_octant_kernel");
      }
    }
  }
  if (status == MX_OK) {
    unsigned long long h[2];
    if (cudaMemcpyAsync(h, mx, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_error(std::string("mx_build_demag_kernel: ") + cudaGetErrorString(cudaGetLastError()));
      status = MX_ERR_CUDA;
    } else {
      double re, im;
      memcpy(&re, &h[0], 8);
      memcpy(&im, &h[1], 8);
      ctx->spectrum_imag_ratio = (re > 0) ? im / re : 0.0;
    }
  } else {
    cudaStreamSynchronize(st);
  }
  cudaFree(buf);
  cudaFree(tw);
  cudaFree(mx);
  if (status == MX_OK) ctx->built = true;
  return status;
}

}  // namespace mx
