// Energy entry point that allocates no device memory (mx_energy_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs inside a device-memory
// budget owned by another framework (which hands it every buffer it may
// touch), or a latency-critical loop where an allocation's implicit
// synchronisation would stall other work on the device.  For them this entry
// point takes its inputs and its output buffer from the caller and keeps its
// only scratch -- one row of five FP64 partial sums per 256-cell block -- in a
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address.  The device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on that device's first call.
#include <mutex>
#include <string>

#include "common.cuh"
#include "kernels.cuh"
#include "local.cuh"

namespace mx {

// One partial-sum row (5 doubles) per block of 256 cells: 16384 blocks cover
// 4,194,304 cells and take 640 KiB.
constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 16384;
constexpr long kNoallocMaxCells = (long)kNoallocThreads * kNoallocMaxBlocks;

static __device__ __align__(256) double g_noalloc_partials[5 * kNoallocMaxBlocks];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device.
static mx_status noalloc_scratch(double** out) {
  int dev = 0;
  MX_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("mx_energy_noalloc: device ordinal out of range");
    return MX_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      set_error(std::string("mx_energy_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return MX_ERR_CUDA;
    }
    g_noalloc_addr[dev] = (double*)p;
  }
  *out = g_noalloc_addr[dev];
  return MX_OK;
}

// Per-block sums of [demag, exch, anis, dmi, zeeman] written to partials.
template <bool DMI>
__global__ void __launch_bounds__(kNoallocThreads) energy_partials_kernel(const float4* __restrict__ m,
                                                                          const float4* __restrict__ hd, Grid g,
                                                                          LocalCoef c, double V, double Ku,
                                                                          double* __restrict__ partials) {
  const long idx = (long)blockIdx.x * kNoallocThreads + threadIdx.x;
  double acc[5] = {0, 0, 0, 0, 0};
  if (idx < g.ncell) {
    const int i = (int)(idx % g.nx);
    const int j = (int)((idx / g.nx) % g.ny);
    const int k = (int)(idx / ((long)g.nx * g.ny));
    const float3 mc = f3(m[idx]);
    const float ms = c.ms_map ? c.ms_map[idx] : c.Ms;
    Terms t;
    local_terms<DMI>(m, hd, g, c, i, j, k, idx, mc, 1.f / ms, t);
    const double q = -0.5 * kMu0 * V * (double)ms;
    acc[0] = q * (double)dot3(mc, t.demag);
    acc[1] = q * (double)dot3(mc, t.exch);
    const float3 e3 = c.axis_map ? f3(c.axis_map[idx]) : make_float3(c.ax, c.ay, c.az);
    const double ku = c.ku_map ? (double)c.ku_map[idx] : Ku;
    const double me = (double)dot3(mc, e3);
    acc[2] = V * ku * (1.0 - me * me);
    acc[3] = q * (double)dot3(mc, t.dmi);
    acc[4] = 2.0 * q * (double)dot3(mc, t.zee);
  }
  __shared__ double red[5][kNoallocThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 5; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < kNoallocThreads / 32; ++w) s += red[threadIdx.x][w];
    partials[(long)blockIdx.x * 5 + threadIdx.x] = s;
  }
}

// e_out[q] = sum over the first nblocks rows of partials, in a fixed order.
__global__ void __launch_bounds__(kNoallocThreads) energy_reduce_kernel(const double* __restrict__ partials,
                                                                        int nblocks, double* __restrict__ e_out) {
  __shared__ double red[5][kNoallocThreads];
  for (int q = 0; q < 5; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kNoallocThreads) s += partials[(long)b * 5 + q];
    red[q][threadIdx.x] = s;
  }
  __syncthreads();
  for (int w = kNoallocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 5) e_out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace mx

using namespace mx;

extern "C" mx_status mx_energy_noalloc(const mx_params* p, const float* m, const float* h_demag,
                                       const float* ms_map, const float* ku_map, const float* axis_map,
                                       double* e_out, mx_stream_t stream) {
  clear_error();
  if (!p || !m || !e_out) {
    set_error("mx_energy_noalloc: p, m and e_out must not be NULL");
    return MX_ERR_INVALID_ARG;
  }
  if ((((uintptr_t)m) & 15) || (h_demag && (((uintptr_t)h_demag) & 15)) || (axis_map && (((uintptr_t)axis_map) & 15)) ||
      (ms_map && (((uintptr_t)ms_map) & 3)) || (ku_map && (((uintptr_t)ku_map) & 3)) || (((uintptr_t)e_out) & 7)) {
    set_error("mx_energy_noalloc: m, h_demag and axis_map must be 16-byte aligned, ms_map and ku_map 4-byte, "
              "e_out 8-byte aligned");
    return MX_ERR_INVALID_ARG;
  }
  // the same per-axis limit as mx_create, checked before the cell count is formed
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 2048 || p->ny > 2048 || p->nz > 2048) {
    set_error("mx_energy_noalloc: grid must be 1..2048 cells per axis");
    return MX_ERR_UNSUPPORTED;
  }
  if (!(p->dx > 0 && p->dy > 0 && p->dz > 0) || !(p->Ms > 0) || !(p->A >= 0)) {
    set_error("mx_energy_noalloc: need dx, dy, dz, Ms > 0 and A >= 0");
    return MX_ERR_INVALID_ARG;
  }
  const long ncell = (long)p->nx * p->ny * p->nz;
  if (ncell > kNoallocMaxCells) {
    set_error("mx_energy_noalloc: " + std::to_string(ncell) + " cells exceed the limit of " +
              std::to_string(kNoallocMaxCells) + " cells of the fixed-size scratch; use mx_energy");
    return MX_ERR_UNSUPPORTED;
  }
  double* partials = nullptr;
  MX_TRY(noalloc_scratch(&partials));
  Grid g{};
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz;
  g.ncell = ncell;
  const LocalCoef c = local_coef_from(*p, ms_map, ku_map, (const float4*)axis_map);
  const double V = p->dx * p->dy * p->dz;
  const int nblocks = (int)((ncell + kNoallocThreads - 1) / kNoallocThreads);
  cudaStream_t st = (cudaStream_t)stream;
  if (c.dmi)
    energy_partials_kernel<true><<<nblocks, kNoallocThreads, 0, st>>>((const float4*)m, (const float4*)h_demag, g,
                                                                      c, V, p->Ku, partials);
  else
    energy_partials_kernel<false><<<nblocks, kNoallocThreads, 0, st>>>((const float4*)m, (const float4*)h_demag, g,
                                                                       c, V, p->Ku, partials);
  MX_TRY(launch_check("energy_partials_kernel"));
  energy_reduce_kernel<<<1, kNoallocThreads, 0, st>>>(partials, nblocks, e_out);
  return launch_check("energy_reduce_kernel");
}
