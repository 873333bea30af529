// Shared definitions of libmx: context layout, error reporting, complex helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/mx.h"

namespace mx {

constexpr double kPi = 3.14159265358979323846;
constexpr double kMu0 = 4e-7 * kPi;  // vacuum permeability [T m/A]
constexpr int kMaxPad = 4096;         // largest padded length per axis

// ---------------------------------------------------------------------------
// Error reporting: a per-thread message plus a status code.
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
void clear_error();

#define MX_CUDA_TRY(expr)                                                         \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ::mx::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));        \
      return MX_ERR_CUDA;                                                         \
    }                                                                             \
  } while (0)

#define MX_TRY(expr)                       \
  do {                                     \
    mx_status s_ = (expr);                 \
    if (s_ != MX_OK) return s_;            \
  } while (0)

// Check the launch that was just enqueued.
inline mx_status launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return MX_ERR_CUDA;
  }
  return MX_OK;
}

// Programmatic dependent launch.  A kernel launched by launch_pdl may be
// scheduled while the kernel before it in the stream is still running; it
// calls pdl_wait() before its first access to memory that kernel writes or
// reads (the wait returns once that kernel has completed and its writes are
// visible; without a programmatic dependency it returns at once).
// pdl_trigger() lets the next launch_pdl kernel be scheduled as soon as every
// CTA of this one has executed it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);  // errors reach launch_check
}

// ---------------------------------------------------------------------------
// Complex arithmetic on float2 / double2.
// ---------------------------------------------------------------------------
template <typename C> struct real_of;
template <> struct real_of<float2> { typedef float type; };
template <> struct real_of<double2> { typedef double type; };

template <typename C> __host__ __device__ __forceinline__ C mkc(typename real_of<C>::type r, typename real_of<C>::type i) {
  C c; c.x = r; c.y = i; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mkc<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mkc<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mkc<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, typename real_of<C>::type s) { return mkc<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C cmul_mi(C a) {
  return INV ? mkc<C>(-a.y, a.x) : mkc<C>(a.y, -a.x);
}

// ---------------------------------------------------------------------------
// Derived per-context constants passed to kernels by value.
// ---------------------------------------------------------------------------
// Bits of the context's device status flag (read and cleared by mx_sync).
constexpr int kFlagNonfinite = 1;  // a kernel produced a non-finite value
constexpr int kFlagTimeout = 2;    // a bounded wait on a bulk copy ran out

struct Grid {
  int nx, ny, nz;      // cells
  int Px, Py, Pz;      // padded lengths
  int Hx;              // Px/2 + 1 (half spectrum along x); 1 when Px == 1
  int Oy, Oz;          // Py/2 + 1, Pz/2 + 1 (octant extents of the spectrum)
  long ncell;
  int oct4;            // plane-path tensor octant split by qy mod 4 (else by qy mod 2)
};

// Tensor octant layouts of the per-kx plane path (6 comps innermost, so one
// (qz, qy) is three float2 loads):
//   oct4 == 0: [kx][qz][qy mod 2][qy / 2][comp], the even-ky and odd-ky halves
//              of a plane (two-CTA plane kernel) each read contiguous rows;
//   oct4 == 1: [kx][qz][qy mod 4][qy / 4][comp], Py/8 + 1 entries per class, so
//              each CTA of the four-CTA plane kernel (one residue of ky mod 4)
//              reads contiguous rows.
__host__ __device__ __forceinline__ int plane_oct4_rows(const Grid& g) { return (g.Py >> 3) + 1; }
__host__ __device__ __forceinline__ long plane_octant_index(const Grid& g, int kx, int comp, int qz, int qy) {
  if (g.oct4) return ((((long)kx * g.Oz + qz) * 4 + (qy & 3)) * plane_oct4_rows(g) + (qy >> 2)) * 6 + comp;
  const int oyh = (g.Oy + 1) >> 1;
  return ((((long)kx * g.Oz + qz) * 2 + (qy & 1)) * oyh + (qy >> 1)) * 6 + comp;
}
// floats to allocate for either layout
__host__ __device__ __forceinline__ long plane_octant_size(const Grid& g) {
  const long two = (long)g.Hx * g.Oz * 2 * ((g.Oy + 1) >> 1) * 6;
  const long four = (long)g.Hx * g.Oz * 4 * plane_oct4_rows(g) * 6;
  return two > four ? two : four;
}

struct LocalCoef {
  float inv_dx2, inv_dy2, inv_dz2;   // 1/h^2
  float inv_2dx, inv_2dy;            // 1/(2h) for central differences
  float kdx, kdy;                    // h * D/(2A): chiral ghost strength
  float cA;                          // 2A/mu0      (divide by Ms_i)
  float cD;                          // 2D/mu0      (divide by Ms_i)
  float cK;                          // 2Ku/mu0     (scalar Ku; divide by Ms_i)
  float Ms;                          // scalar Ms
  float ax, ay, az;                  // scalar easy axis (unit)
  float hx, hy, hz;                  // bias
  float llg;                         // -gamma0/(1+alpha^2)
  float alpha;
  int dmi, precession;
  const float* ms_map;               // may be null
  const float* ku_map;               // may be null (then cK)
  const float4* axis_map;            // may be null (then ax, ay, az)
};

struct Profiler;
struct AdjWork;

}  // namespace mx

// The context (opaque to callers).
struct mx_ctx {
  mx_params p;
  int device;
  mx::Grid g;

  // material maps (context copies)
  float* ms_map = nullptr;
  float* ku_map = nullptr;
  float4* axis_map = nullptr;

  // demag
  bool built = false;
  float* nhat = nullptr;          // tensor octant: [comp][qz][qy][kx], or plane_octant_index() on the plane path
  float2* w1 = nullptr;           // 3 x nz x ny x Hx   (after the x pass)
  float2* w2 = nullptr;           // 3 x nz x Py x Hx   (after the y pass; unfused path)
  float2* tw_x = nullptr;         // W_Px^k, k < Px
  float2* tw_y = nullptr;         // W_Py^k, k < Py
  float2* tw_z = nullptr;         // W_Pz^k, k < Pz
  bool fused_yz = false;          // y/z passes in one kernel (plane fits on chip)
  bool fast_x = false;            // compile-time-sized x passes available
  bool yz2d = false;              // single-z-plane y kernel (Pz == 1) for the fused y/z pass
  float2* tw_m = nullptr;         // W_M^k, k < M = Px/2
  float2* tw_mk = nullptr;        // W_M^(s k) at [k * S + s] for the plane path's x line FFTs (M = E S)
  float2* tw_yh = nullptr;        // W_{Py/2}^k, k < Py/2
  bool plane = false;             // per-kx plane kernel (kx-major spectra and tensor)
  bool quad = false;              // plane path uses the four-CTA y/z kernel (else the two-CTA one)
  int xfk_grid = 1;               // persistent grid of the plane path's x forward kernel
  bool xlocal = false;            // inverse x pass fused into the RK/Euler local stage
  bool xrow = false;              // few-row grids: inverse x, local stage and next forward x in one kernel
  bool inject_wait_timeout = false;  // mx_inject_wait_timeout: the two-CTA kernel's bulk-copy wait runs out
  void* dft_a = nullptr;          // split-BF16 DFT matrices (MX_FFT_SPLIT_BF16)
  int yz_tile = 1;                // kx columns per block in the fused kernel
  double* t_real = nullptr;       // FP64 real-space tensor octant (kept for checking)
  double spectrum_imag_ratio = 0; // max|Im| / max|Re| of the FP64 tensor spectrum

  // stage buffers
  float4* hd = nullptr;           // demag field
  float4* sa = nullptr;           // stage input A
  float4* sb = nullptr;           // stage input B
  float4* acc = nullptr;          // RK accumulator
  int* flag = nullptr;            // non-finite flag
  double* ered = nullptr;         // energy accumulators (5)

  // CUDA graph cache for mx_rk_step
  cudaGraphExec_t graph = nullptr;
  const float* graph_m = nullptr;
  double graph_dt = 0.0;
  int graph_method = -1;
  cudaStream_t cap_stream = nullptr;

  // profiling hook (events around each launch when non-null)
  mx::Profiler* prof = nullptr;

  // adjoint workspaces (mx_adjoint_reserve)
  mx::AdjWork* adj = nullptr;

  // learned demag backend (mx_set_demag_surrogate / mx_set_demag_fno; at
  // most one is set); both NULL: FFT convolution
  struct mx_cnn* surrogate = nullptr;
  struct mx_fno* fno = nullptr;
  float4* mri_f = nullptr;        // MRI slow right-hand sides F_1..F_3 (allocated at first use)
  double* red2 = nullptr;         // 2 FP64 accumulators for mx_rel_l2
};
