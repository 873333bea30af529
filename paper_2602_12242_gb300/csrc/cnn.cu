// Learned demag surrogate: a 3D conv net 3 -> 32 -> 64 -> 32 -> 3 (3x3x3
// kernels, zero padding 1, exact-erf GELU after the first three layers) that
// maps the normalised magnetisation to the normalised demag field, trained
// with SmoothL1 loss and Adam with L2 weight decay (the paper's ML module,
// Sec. II-D: a network trained offline on (M, H_demag) pairs from the FFT
// solver, per-channel Gaussian normaliser, Adam lr 1e-3, weight decay 1e-4).
//
// Activations are BF16, channels-last [b][z][y][x][C] with C padded to a
// multiple of 16 (first input: 3 -> 16); weights are FP32 masters with BF16
// copies for the tensor cores.  Every convolution is an implicit GEMM on the
// tcgen05 tensor cores (BF16 in, FP32 accumulator in tensor memory): a block
// takes 8 x 16 x 1 tiles of output cells (M = 128) with a (10 x 18 x 3) halo
// of input cells staged with cp.async; all 27 taps of the layer's weights
// stay in shared memory.  The weight gradient runs on tcgen05 too, with
// MN-major operands (wgrad_tc_kernel).
//   forward     out = conv(a, W) + b, stored pre-activation y and a = gelu(y)
//   backward-x  dA_{l-1} = conv(dY_l, W'), W'[tap][ci][co] = W[26 - tap][co][ci],
//               times gelu'(y_{l-1}) in the epilogue -> dY_{l-1}
//   backward-W  dW[tap] = sum over cells of dY (x) x_shifted(tap), one block per
//               (dz, ddy, chunk of tiles) with its three taps in tensor memory,
//               FP32 atomics into the gradient
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "bulk.cuh"
#include "mma.cuh"
#include "tc05.cuh"

namespace mx {

constexpr int kTX = 16, kTY = 8;             // output tile (cells)
constexpr int kHX = kTX + 2, kHY = kTY + 2;  // halo
constexpr int kHalo = kHX * kHY * 3;
constexpr int kCnnThreads = 256;
static const int kCh[5] = {3, 32, 64, 32, 3};
static const int kCinPad[4] = {16, 32, 64, 32};
static const int kCoutPad[4] = {32, 64, 32, 8};

__device__ __forceinline__ float gelu_f(float y) { return 0.5f * y * (1.f + erff(y * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float y) {
  return 0.5f * (1.f + erff(y * 0.70710678118654752f)) + y * 0.39894228040143268f * expf(-0.5f * y * y);
}

struct ConvDims {
  int nx, ny, nz, batch;
  int tiles_x, tiles_y, ntiles;  // tiles per (b, z) plane and total
};

__host__ __device__ inline void tile_coords(const ConvDims& d, int t, int& b, int& z, int& y0, int& x0) {
  const int tx = t % d.tiles_x;
  int r = t / d.tiles_x;
  const int ty = r % d.tiles_y;
  r /= d.tiles_y;
  z = r % d.nz;
  b = r / d.nz;
  y0 = ty * kTY;
  x0 = tx * kTX;
}

enum ConvMode { CM_HIDDEN = 0, CM_LAST = 1, CM_BWD = 2 };

// ---------------------------------------------------------------------------
// Convolution: in [cells][CIN] (bf16), weights wk [27][COUT][CIN] (bf16), on
// the tcgen05 tensor cores, one persistent block per SM looping over tiles.
//   CM_HIDDEN: ypre = acc + b (bf16), out = gelu(acc + b) (bf16), [cells][COUT]
//   CM_LAST:   outf = acc + b (fp32) channels 0..2 of a float4 record per cell
//   CM_BWD:    out = acc * gelu'(ypre) (bf16), [cells][COUT]  (ypre read)  A block (persistent, one
// per SM) takes an 8 (x) x 16 (y) x 1 tile of output cells, M = 128 rows
// (row = 8 y + x); N = COUT (16 for the last layer, whose padding rows are
// zero weights); K = 27 taps x CIN.  Shared memory holds every operand in the
// canonical K-major layout without swizzle:
//   weights [tap][CIN/8][N][8]   B of tap t, K chunk c: 8-row groups (8 output
//                                channels) 128 B apart, K chunks N x 16 B apart
//   halo    [CIN/8][540][8]      (3 x 18 x 10 cells): A of tap (dz, dy, dx) starts
//                                at cell (dz, dy, dx); consecutive x are 16 B
//                                apart, so each output row y (8 cells) is one
//                                8-row group and groups are 10 x 16 B apart
// One thread issues the 27 CIN/16 MMAs of a tile into a TMEM accumulator
// (128 lanes x N columns, FP32) and commits them to an mbarrier; after the
// (bounded) wait, warp w reads lanes 32 (w mod 4) .. +31, columns of half
// w / 4, for the epilogue.
// ---------------------------------------------------------------------------
constexpr int kTXc = 8, kTYc = 16;
constexpr int kHXc = kTXc + 2, kHYc = kTYc + 2;
constexpr int kHaloC = kHXc * kHYc * 3;

template <int CIN, int COUT> struct ConvTc {
  static constexpr int NP = COUT < 16 ? 16 : COUT;  // MMA N
  static constexpr int KC = CIN / 8;
  static constexpr size_t w_bytes = sizeof(bf16_t) * 8 * 27 * KC * NP;
  static constexpr size_t h_bytes = sizeof(bf16_t) * 8 * KC * kHaloC;
  // two halo buffers where they fit next to the weights (227 KB)
  static constexpr int NB = (w_bytes + 2 * h_bytes <= 227 * 1024) ? 2 : 1;
  static constexpr size_t smem = w_bytes + NB * h_bytes;
  // two accumulators of NP columns, allocated as a power of two >= 32
  static constexpr uint32_t TCOLS = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : (2 * NP <= 128 ? 128 : 256));
};

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(kCnnThreads, 1) conv_tc_kernel(const bf16_t* __restrict__ in,
                                                                  const bf16_t* __restrict__ wk,
                                                                  const float* __restrict__ bias,
                                                                  bf16_t* __restrict__ out, bf16_t* __restrict__ ypre,
                                                                  float4* __restrict__ outf, ConvDims d, int* flag) {
  typedef ConvTc<CIN, COUT> T;
  constexpr int NP = T::NP, KC = T::KC, NH = NP / 2, NB = T::NB;
  const int cta = (int)blockIdx.x, ncta = (int)gridDim.x;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tbase;
  bf16_t* sw = (bf16_t*)smraw;  // [27][KC][NP][8]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < 27 * KC * NP; e += kCnnThreads) {
    const int co = e % NP, kc = (e / NP) % KC, tap = e / (NP * KC);
    const bool ok = co < COUT;
    cp_async16(smem_u32(sw + (long)e * 8), wk + ((long)tap * COUT + (ok ? co : 0)) * CIN + kc * 8, ok);
  }
  if (warp == 0) tmem_alloc(&tbase, T::TCOLS);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  const uint32_t sw_a = smem_u32(sw);
  const uint32_t sh_a0 = sw_a + (uint32_t)T::w_bytes;
  constexpr uint32_t idesc = tc_idesc_bf16(128, NP);
  const int tiles_x = (d.nx + kTXc - 1) / kTXc, tiles_y = (d.ny + kTYc - 1) / kTYc;
  const int ntiles = tiles_x * tiles_y * d.nz * d.batch;
  const int nmine = cta < ntiles ? (ntiles - 1 - cta) / ncta + 1 : 0;
  const long plane = (long)d.nx * d.ny;
  // this thread's accumulator row: cell (cx, cy) of the tile; lane quarter, column half
  const int row = 32 * (warp & 3) + lane;
  const int cx = row & 7, cy = row >> 3;
  const int cb = (warp >> 2) * NH;
  auto coords = [&](int k, int& b, int& z, int& y0, int& x0) {
    const int t = cta + k * ncta;
    const int tx = t % tiles_x;
    int r = t / tiles_x;
    const int ty = r % tiles_y;
    r /= tiles_y;
    z = r % d.nz;
    b = r / d.nz;
    x0 = tx * kTXc;
    y0 = ty * kTYc;
  };
  // halo of tile k into buffer k % NB: issue the cp.async copies as one group
  // (halo_ready waits for them and makes them visible to the tensor core)
  auto load_halo = [&](int k) {
    int b, z, y0, x0;
    coords(k, b, z, y0, x0);
    bf16_t* sh = (bf16_t*)(smraw + T::w_bytes + (k % NB) * T::h_bytes);
    for (int e = tid; e < kHaloC * KC; e += kCnnThreads) {
      const int hc = e % kHaloC, kc = e / kHaloC;
      const int hx = hc % kHXc, hy = (hc / kHXc) % kHYc, hz = hc / (kHXc * kHYc);
      const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z + hz - 1;
      const bool ok = gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny && gz >= 0 && gz < d.nz;
      const long cell = ok ? ((long)b * d.nz + gz) * plane + (long)gy * d.nx + gx : 0;
      cp_async16(smem_u32(sh + (long)e * 8), in + cell * CIN + kc * 8, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  auto halo_ready = [&]() {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    fence_proxy_async_smem();
  };
  // the 27 CIN/16 MMAs of tile k into accumulator k & 1 (one thread)
  auto issue = [&](int k) {
    const uint32_t sh_a = sh_a0 + (uint32_t)((k % NB) * T::h_bytes);
    const uint32_t dt = tbase + (uint32_t)((k & 1) * NP);
    tc_fence_after_sync();
#pragma unroll 1
    for (int tap = 0; tap < 27; ++tap) {
      const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
      const uint32_t aoff = (uint32_t)(((dz * kHYc + dy) * kHXc + dx) * 16);
#pragma unroll
      for (int ks = 0; ks < CIN / 16; ++ks) {
        const uint64_t ad = tc_sdesc(sh_a + (uint32_t)(2 * ks * kHaloC * 16) + aoff, kHaloC * 16, kHXc * 16);
        const uint64_t bd = tc_sdesc(sw_a + (uint32_t)((tap * KC + 2 * ks) * NP * 16), NP * 16, 128);
        tc_mma_bf16(dt, ad, bd, idesc, tap > 0 || ks > 0);
      }
    }
    tc_commit(&bar[k & 1]);
  };
  uint32_t par[2] = {0u, 0u};
  auto wait_mma = [&](int k) {
    if (!mbar_wait(&bar[k & 1], par[k & 1])) atomicOr(flag, kFlagTimeout);
    par[k & 1] ^= 1u;
    tc_fence_after_sync();
  };
  cp_async_wait_all();  // weights
  if (nmine > 0) {
    load_halo(0);
    halo_ready();
  }
  tc_fence_before_sync();
  __syncthreads();
  if (nmine > 0 && tid == 0) issue(0);
  if (NB == 2 && nmine > 1) load_halo(1);  // buffer 1 is free: prefetch
  for (int k = 0; k < nmine; ++k) {
    if (NB == 2) {
      if (k + 1 < nmine) {
        halo_ready();  // tile k + 1's halo (prefetched) is in buffer (k + 1) % 2
        tc_fence_before_sync();
        __syncthreads();
        if (tid == 0) issue(k + 1);
      }
      wait_mma(k);  // buffer k % 2 and accumulator k & 1 are done with
      if (k + 2 < nmine) load_halo(k + 2);  // lands during the epilogue
    } else {
      wait_mma(k);  // the only halo buffer is free once tile k's MMAs are done
      if (k + 1 < nmine) {
        load_halo(k + 1);
        halo_ready();
        tc_fence_before_sync();
        __syncthreads();
        if (tid == 0) issue(k + 1);
      }
    }
    // epilogue of tile k (overlaps the MMAs of tile k + 1)
    float v[NH];
#pragma unroll
    for (int q = 0; q < NH / 8; ++q) {
      float t8[8];
      tmem_ld8(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((k & 1) * NP + cb + 8 * q), t8);
#pragma unroll
      for (int i = 0; i < 8; ++i) v[8 * q + i] = t8[i];
    }
    int b, z, y0, x0;
    coords(k, b, z, y0, x0);
    const int gx = x0 + cx, gy = y0 + cy;
    if (gx < d.nx && gy < d.ny) {
      const long cell = ((long)b * d.nz + z) * plane + (long)gy * d.nx + gx;
      // eight channels per 16-byte store
#pragma unroll
      for (int c = 0; c < NH; c += 8) {
        const int cg = cb + c;  // channel of v[c]
        if (cg >= COUT) break;
        if (MODE == CM_HIDDEN) {
          uint32_t yp[4], o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float v0 = v[c + 2 * j] + bias[cg + 2 * j], v1 = v[c + 2 * j + 1] + bias[cg + 2 * j + 1];
            yp[j] = pack2(v0, v1);
            o[j] = pack2(gelu_f(v0), gelu_f(v1));
          }
          *(uint4*)(ypre + cell * COUT + cg) = make_uint4(yp[0], yp[1], yp[2], yp[3]);
          *(uint4*)(out + cell * COUT + cg) = make_uint4(o[0], o[1], o[2], o[3]);
        } else if (MODE == CM_BWD) {
          const uint4 y4 = *(const uint4*)(ypre + cell * COUT + cg);
          const uint32_t yw[4] = {y4.x, y4.y, y4.z, y4.w};
          uint32_t o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float y0f = bf2f((bf16_t)(yw[j] & 0xffff)), y1f = bf2f((bf16_t)(yw[j] >> 16));
            o[j] = pack2(v[c + 2 * j] * gelu_grad(y0f), v[c + 2 * j + 1] * gelu_grad(y1f));
          }
          *(uint4*)(out + cell * COUT + cg) = make_uint4(o[0], o[1], o[2], o[3]);
        } else {
          float* o = (float*)(outf + cell);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (cg + j < 3) o[cg + j] = v[c + j] + bias[cg + j];
        }
      }
    }
    tc_fence_before_sync();
    __syncthreads();  // accumulator k & 1 and halo buffer k % NB may be reused
  }
  if (warp == 0) {
    tc_fence_after_sync();
    tmem_dealloc(tbase, T::TCOLS);
  }
}

// ---------------------------------------------------------------------------
// Weight gradient of one layer on the tcgen05 tensor cores:
//   dW[tap][co][ci] += sum_cells dY[cell][co] * x[cell + off(tap)][ci].
// Block (range of 16 x 8 output tiles, dz, ddy) owns the three taps
// (dz, ddy, ddx = 0..2).  Per tile and tile row cy, three MMAs
// D_ddx (co x ci) += dY^T (co x the 16 cells of row cy) X_ddx (those cells
// shifted by the tap x ci), M = 128 (co, rows >= COUT zero), N = CIN, K = 16,
// accumulated in tensor memory over all of the block's tiles.  Both operands
// are MN-major (channels contiguous, one 16-byte row of 8 channels per cell,
// core matrices adjacent along K 128 B apart, 8-channel groups SBO apart), so
// they are 16-byte copies of the [cell][channel] activations: dY of the tile
// (row q = cell cy * 16 + cx) and the tile's band of x rows for this ddy
// (8 rows of 18 cells, row r * 18 + hx); the operand of (cy, ddx) starts at
// row cy * 16 of dY and row cy * 18 + ddx of the band.
// ---------------------------------------------------------------------------
template <int CIN, int COUT> struct WgradShape {
  static constexpr int HXp = kTX + 2;                    // band row: 18 cells
  static constexpr int NROW = kTY * HXp;                 // 144 band cells
  static constexpr uint32_t A_SBO = kTX * kTY * 16 + 16;  // 128 cells + 16 B pad (bank spread)
  static constexpr uint32_t B_SBO = NROW * 16 + 16;
  static constexpr uint32_t A_BYTES = 16 * A_SBO;
  static constexpr uint32_t BUF = A_BYTES + (CIN / 8) * B_SBO;  // one tile's operands
  static constexpr size_t smem = BUF;
  static constexpr int TCOLS = 3 * CIN <= 64 ? 64 : (3 * CIN <= 128 ? 128 : 256);
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kCnnThreads, 1) wgrad_tc_kernel(const bf16_t* __restrict__ x,
                                                                  const bf16_t* __restrict__ dy,
                                                                  float* __restrict__ dw, ConvDims d, int cin_real,
                                                                  int cout_real, int tiles_per_block, int* flag) {
  typedef WgradShape<CIN, COUT> W;
  static_assert(COUT % 8 == 0 && COUT <= 128 && CIN % 16 == 0 && 3 * CIN <= 256, "wgrad shape");
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int dz = blockIdx.y / 3, ddy = blockIdx.y % 3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // dY^T (16 channel groups, those >= COUT/8 stay zero) then the x band
  for (int i = tid; i < (int)(W::smem / 16); i += kCnnThreads) ((uint4*)smraw)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tmem_alloc(&tbase, W::TCOLS);
  if (tid == 0) mbar_init(&bar, 1);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tb = tbase;
  const long plane = (long)d.nx * d.ny;
  const int t0 = blockIdx.x * tiles_per_block;
  const int n = max(0, min(d.ntiles, t0 + tiles_per_block) - t0);
  constexpr uint32_t idesc = tc_idesc_bf16(128, CIN) | (1u << 15) | (1u << 16);  // A and B MN-major
  // the copies of tile k, as one cp.async group
  auto stage = [&](int k) {
    unsigned char* sA = smraw;
    unsigned char* sB = sA + W::A_BYTES;
    int b, z, y0, x0;
    tile_coords(d, t0 + k, b, z, y0, x0);
    const int gz = z + dz - 1;
    // band cell (r, hx) -> x cell (gz, y0 + r + ddy - 1, x0 + hx - 1); chunk fastest (coalesced reads)
    for (int e = tid; e < W::NROW * (CIN / 8); e += kCnnThreads) {
      const int ch = e % (CIN / 8), c = e / (CIN / 8);
      const int gx = x0 + c % W::HXp - 1, gy = y0 + c / W::HXp + ddy - 1;
      const bool ok = gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny && gz >= 0 && gz < d.nz;
      const long cell = ok ? ((long)b * d.nz + gz) * plane + (long)gy * d.nx + gx : 0;
      cp_async16(smem_u32(sB + ch * W::B_SBO + c * 16), x + cell * CIN + ch * 8, ok);
    }
    // dY of the tile's output cells (zero outside the grid, so those cells add nothing)
    for (int e = tid; e < kTX * kTY * (COUT / 8); e += kCnnThreads) {
      const int ch = e % (COUT / 8), q = e / (COUT / 8);
      const int ox = x0 + q % kTX, oy = y0 + q / kTX;
      const bool ok = ox < d.nx && oy < d.ny;
      const long cell = ok ? ((long)b * d.nz + z) * plane + (long)oy * d.nx + ox : 0;
      cp_async16(smem_u32(sA + ch * W::A_SBO + q * 16), dy + cell * COUT + ch * 8, ok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // Per tile: copies, then the 24 MMAs of one issuing thread; the next
  // tile's copies wait for them (a second operand buffer, measured, was
  // slower: two buffers of 103 KB leave fewer blocks per SM).
  uint32_t par = 0u;
  for (int k = 0; k < n; ++k) {
    stage(k);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after_sync();
      const uint32_t a0 = smem_u32(smraw), b0 = a0 + W::A_BYTES;
#pragma unroll
      for (int cy = 0; cy < kTY; ++cy)
#pragma unroll
        for (int ddx = 0; ddx < 3; ++ddx)
          tc_mma_bf16(tb + ddx * CIN, tc_sdesc(a0 + cy * kTX * 16, 128, W::A_SBO),
                      tc_sdesc(b0 + (cy * W::HXp + ddx) * 16, 128, W::B_SBO), idesc, k > 0 || cy > 0);
      tc_commit(&bar);
    }
    if (!mbar_wait(&bar, par)) atomicOr(flag, kFlagTimeout);
    par ^= 1u;
    tc_fence_after_sync();
  }
  // accumulators: lane = co (warps 0..3), column ddx * CIN + ci
  if (n > 0 && warp < 4) {
    const int co = 32 * warp + lane;
#pragma unroll
    for (int ddx = 0; ddx < 3; ++ddx) {
      const int tap = dz * 9 + ddy * 3 + ddx;
#pragma unroll
      for (int j = 0; j < CIN / 8; ++j) {
        float v[8];
        tmem_ld8(tb + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ddx * CIN + 8 * j), v);
        if (co < cout_real) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int ci = 8 * j + i;
            if (ci < cin_real) atomicAdd(&dw[((long)co * cin_real + ci) * 27 + tap], v[i]);
          }
        }
      }
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after_sync();
    tmem_dealloc(tb, W::TCOLS);
  }
}

// bias gradient: db[co] += sum over cells of dY[cell][co]
__global__ void bgrad_kernel(const bf16_t* __restrict__ dy, int cpad, int creal, long ncells, float* __restrict__ db) {
  const int co = threadIdx.x % 64;
  const int lane_grp = threadIdx.x / 64;  // 4 groups
  if (co >= creal) return;
  float s = 0.f;
  for (long c = (long)blockIdx.x * 4 + lane_grp; c < ncells; c += (long)gridDim.x * 4) s += bf2f(dy[c * cpad + co]);
  atomicAdd(&db[co], s);
}

// input normalisation: m float4 -> x0 bf16 [cells][16]
__global__ void normalize_in_kernel(const float4* __restrict__ m, bf16_t* __restrict__ x0, long ncells, float3 mean,
                                    float3 inv_std) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const float4 v = m[c];
  uint4 lo, hi;
  lo.x = pack2((v.x - mean.x) * inv_std.x, (v.y - mean.y) * inv_std.y);
  lo.y = pack2((v.z - mean.z) * inv_std.z, 0.f);
  lo.z = lo.w = 0u;
  hi.x = hi.y = hi.z = hi.w = 0u;
  uint4* o = (uint4*)(x0 + c * 16);
  o[0] = lo;
  o[1] = hi;
}

// output: normalised prediction (float4) -> H = pred * std + mean
__global__ void denormalize_out_kernel(const float4* __restrict__ pred, float4* __restrict__ h, long ncells,
                                       float3 mean, float3 std) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const float4 p = pred[c];
  h[c] = make_float4(p.x * std.x + mean.x, p.y * std.y + mean.y, p.z * std.z + mean.z, 0.f);
}

// SmoothL1 (beta 1) of pred against the normalised target; dY4 [cells][16] bf16
__global__ void loss_kernel(const float4* __restrict__ pred, const float4* __restrict__ h_target, long ncells,
                            float3 mean, float3 inv_std, float inv_count, bf16_t* __restrict__ dy4,
                            float* __restrict__ loss) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (c < ncells) {
    const float4 p = pred[c];
    const float4 t = h_target[c];
    const float d0 = p.x - (t.x - mean.x) * inv_std.x;
    const float d1 = p.y - (t.y - mean.y) * inv_std.y;
    const float d2 = p.z - (t.z - mean.z) * inv_std.z;
    const float ds[3] = {d0, d1, d2};
    float g[3];
    for (int k = 0; k < 3; ++k) {
      const float a = fabsf(ds[k]);
      l += a < 1.f ? 0.5f * ds[k] * ds[k] : a - 0.5f;
      g[k] = fminf(fmaxf(ds[k], -1.f), 1.f) * inv_count;
    }
    uint4 lo, hi;
    lo.x = pack2(g[0], g[1]);
    lo.y = pack2(g[2], 0.f);
    lo.z = lo.w = 0u;
    hi.x = hi.y = hi.z = hi.w = 0u;
    uint4* o = (uint4*)(dy4 + c * 16);
    o[0] = lo;
    o[1] = hi;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l * inv_count);
}

// FP32 master weights -> bf16 [27][COUT_PAD][CIN_PAD] (forward) and the
// flipped, transposed copy [27][CIN_PAD'][COUT_PAD'] for the backward pass.
__global__ void pack_weights_kernel(const float* __restrict__ W, int cin, int cout, bf16_t* __restrict__ fwd,
                                    int cin_pad, int cout_pad, bf16_t* __restrict__ bwd, int bwd_in_pad,
                                    int bwd_out_pad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = 27 * cout_pad * cin_pad;
  if (e < nf) {
    const int ci = e % cin_pad, co = (e / cin_pad) % cout_pad, tap = e / (cin_pad * cout_pad);
    const float v = (ci < cin && co < cout) ? W[((long)co * cin + ci) * 27 + tap] : 0.f;
    fwd[e] = f2bf(v);
  }
  if (bwd) {
    const int nb = 27 * bwd_out_pad * bwd_in_pad;
    if (e < nb) {
      // backward conv: input channels = this layer's cout, output channels = cin
      const int co = e % bwd_in_pad, ci = (e / bwd_in_pad) % bwd_out_pad, tapb = e / (bwd_in_pad * bwd_out_pad);
      const int tap = 26 - tapb;
      const float v = (ci < cin && co < cout) ? W[((long)co * cin + ci) * 27 + tap] : 0.f;
      bwd[e] = f2bf(v);
    }
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long n, float lr, float wd, float b1, float b2, float c1, float c2,
                            float eps) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] + wd * p[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

mx_status adam_update(float* p, const float* g, float* m, float* v, long n, double lr, double wd, int t,
                      cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, (float)lr, (float)wd, (float)b1,
                                                           (float)b2, (float)c1, (float)c2, 1e-8f);
  return launch_check("adam_kernel");
}

}  // namespace mx

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using mx::bf16_t;

struct mx_cnn {
  int nx, ny, nz, max_batch;
  long cells;
  float* params = nullptr;  // FP32 masters, oracle order (W1, b1, ..., W4, b4)
  float* grad = nullptr;
  float* am = nullptr;
  float* av = nullptr;
  int adam_t = 0;
  bf16_t* wf[4] = {nullptr, nullptr, nullptr, nullptr};
  bf16_t* wb[4] = {nullptr, nullptr, nullptr, nullptr};
  bf16_t *x0 = nullptr, *a1 = nullptr, *y1 = nullptr, *a2 = nullptr, *y2 = nullptr, *a3 = nullptr, *y3 = nullptr;
  bf16_t *dy4 = nullptr, *dy3 = nullptr, *dy2 = nullptr, *dy1 = nullptr;
  float4* pred = nullptr;
  float* loss = nullptr;
  int* flag = nullptr;  // device status bits (kFlagTimeout), read by mx_cnn_sync / mx_sync
  float stats[12] = {0, 0, 0, 1, 1, 1, 0, 0, 0, 1, 1, 1};
};

namespace mx {

static long layer_w_off(int l) {
  long o = 0;
  for (int q = 0; q < l; ++q) o += (long)kCh[q] * kCh[q + 1] * 27 + kCh[q + 1];
  return o;
}
static long num_params_total() { return layer_w_off(4); }

static ConvDims conv_dims(const mx_cnn* n, int batch) {
  ConvDims d;
  d.nx = n->nx;
  d.ny = n->ny;
  d.nz = n->nz;
  d.batch = batch;
  d.tiles_x = (n->nx + kTX - 1) / kTX;
  d.tiles_y = (n->ny + kTY - 1) / kTY;
  d.ntiles = d.tiles_x * d.tiles_y * n->nz * batch;
  return d;
}

static int g_num_sms = 0;

template <int CIN, int COUT, int MODE>
static mx_status conv_launch(const bf16_t* in, const bf16_t* w, const float* b, bf16_t* out, bf16_t* ypre,
                             float4* outf, const ConvDims& d, int* flag, int ntiles, cudaStream_t st) {
  const size_t sm = ConvTc<CIN, COUT>::smem;
  static bool attr = false;
  if (!attr) {
    MX_CUDA_TRY(cudaFuncSetAttribute(conv_tc_kernel<CIN, COUT, MODE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    attr = true;
  }
  const int ctas = ntiles < g_num_sms ? ntiles : g_num_sms;
  conv_tc_kernel<CIN, COUT, MODE><<<ctas, kCnnThreads, sm, st>>>(in, w, b, out, ypre, outf, d, flag);
  return launch_check("conv_tc_kernel");
}

template <int CIN, int COUT, int MODE>
static mx_status conv_run(const bf16_t* in, const bf16_t* w, const float* b, bf16_t* out, bf16_t* ypre, float4* outf,
                          const ConvDims& d, int* flag, cudaStream_t st) {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  const int ntiles = ((d.nx + kTXc - 1) / kTXc) * ((d.ny + kTYc - 1) / kTYc) * d.nz * d.batch;
  return conv_launch<CIN, COUT, MODE>(in, w, b, out, ypre, outf, d, flag, ntiles, st);
}

template <int CIN, int COUT>
static mx_status wgrad_run(const bf16_t* x, const bf16_t* dy, float* dw, const ConvDims& d, int cin_real,
                           int cout_real, int* flag, cudaStream_t st) {
  typedef WgradShape<CIN, COUT> W;
  static bool attr = false;
  if (!attr) {
    MX_CUDA_TRY(cudaFuncSetAttribute(wgrad_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)W::smem));
    attr = true;
  }
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  // about six blocks per SM over the nine (dz, ddy) tap rows: blocks that
  // wait for tensor memory or for their MMAs overlap the others' copies
  // (measured: 5.00 ms per batch-64 loss + gradient at 64x64x4 against 5.89
  // with two blocks per SM and 5.66 with the earlier mma.sync kernel)
  int tpb = (int)(((long)d.ntiles * 9 + 6 * g_num_sms - 1) / (6 * g_num_sms));
  if (tpb < 1) tpb = 1;
  dim3 grid((d.ntiles + tpb - 1) / tpb, 9);
  wgrad_tc_kernel<CIN, COUT><<<grid, kCnnThreads, W::smem, st>>>(x, dy, dw, d, cin_real, cout_real, tpb, flag);
  return launch_check("wgrad_tc_kernel");
}

static mx_status pack_all(mx_cnn* n, cudaStream_t st) {
  // forward packs [27][coutpad][cinpad]; backward packs for layers 2..4
  const int bw_in[4] = {0, 64, 32, 16};   // backward conv input channels (this layer's cout, padded)
  const int bw_out[4] = {0, 32, 64, 32};  // backward conv output channels (this layer's cin)
  for (int l = 0; l < 4; ++l) {
    const int cin = kCh[l], cout = kCh[l + 1];
    const int nf = 27 * kCoutPad[l] * kCinPad[l];
    const int nb = l > 0 ? 27 * bw_in[l] * bw_out[l] : 0;
    const int ne = nf > nb ? nf : nb;
    pack_weights_kernel<<<(ne + 255) / 256, 256, 0, st>>>(n->params + layer_w_off(l), cin, cout, n->wf[l], kCinPad[l],
                                                          kCoutPad[l], l > 0 ? n->wb[l] : nullptr, bw_in[l], bw_out[l]);
    MX_TRY(launch_check("pack_weights_kernel"));
  }
  return MX_OK;
}

static mx_status cnn_forward_to_pred(mx_cnn* n, const float4* m, int batch, cudaStream_t st) {
  const long nc = n->cells * batch;
  const float* s = n->stats;
  normalize_in_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
      m, n->x0, nc, make_float3(s[0], s[1], s[2]), make_float3(1.f / s[3], 1.f / s[4], 1.f / s[5]));
  MX_TRY(launch_check("normalize_in_kernel"));
  const ConvDims d = conv_dims(n, batch);
  const float* P = n->params;
  MX_TRY((conv_run<16, 32, CM_HIDDEN>(n->x0, n->wf[0], P + layer_w_off(0) + 32 * 3 * 27, n->a1, n->y1, nullptr, d, n->flag, st)));
  MX_TRY((conv_run<32, 64, CM_HIDDEN>(n->a1, n->wf[1], P + layer_w_off(1) + 64 * 32 * 27, n->a2, n->y2, nullptr, d, n->flag, st)));
  MX_TRY((conv_run<64, 32, CM_HIDDEN>(n->a2, n->wf[2], P + layer_w_off(2) + 32 * 64 * 27, n->a3, n->y3, nullptr, d, n->flag, st)));
  MX_TRY((conv_run<32, 8, CM_LAST>(n->a3, n->wf[3], P + layer_w_off(3) + 3 * 32 * 27, nullptr, nullptr, n->pred, d, n->flag, st)));
  return MX_OK;
}

bool cnn_matches(const mx_cnn* n, const Grid& g) { return n->nx == g.nx && n->ny == g.ny && n->nz == g.nz; }

mx_status cnn_demag(mx_cnn* n, const float4* m, float4* h, cudaStream_t st) {
  MX_TRY(cnn_forward_to_pred(n, m, 1, st));
  const float* s = n->stats;
  denormalize_out_kernel<<<(unsigned)((n->cells + 255) / 256), 256, 0, st>>>(
      n->pred, h, n->cells, make_float3(s[6], s[7], s[8]), make_float3(s[9], s[10], s[11]));
  return launch_check("denormalize_out_kernel");
}

// Reads and clears the net's device status flag (synchronises `stream`).
mx_status cnn_take_flag(mx_cnn* n, cudaStream_t st, int* flag_out) {
  int f = 0;
  MX_CUDA_TRY(cudaMemcpyAsync(&f, n->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  MX_CUDA_TRY(cudaStreamSynchronize(st));
  if (f) {
    MX_CUDA_TRY(cudaMemsetAsync(n->flag, 0, sizeof(int), st));
    MX_CUDA_TRY(cudaStreamSynchronize(st));
  }
  *flag_out = f;
  return MX_OK;
}

}  // namespace mx

using namespace mx;

extern "C" {

int mx_cnn_num_params(void) { return (int)num_params_total(); }

mx_status mx_cnn_destroy(mx_cnn* n) {
  if (!n) return MX_OK;
  void* ptrs[] = {n->params, n->grad, n->am, n->av, n->wf[0], n->wf[1], n->wf[2], n->wf[3], n->wb[1], n->wb[2],
                  n->wb[3], n->x0, n->a1, n->y1, n->a2, n->y2, n->a3, n->y3, n->dy4, n->dy3, n->dy2, n->dy1,
                  n->pred, n->loss, n->flag};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete n;
  return MX_OK;
}

mx_status mx_cnn_create(mx_cnn** out, int nx, int ny, int nz, int max_batch) {
  clear_error();
  if (!out || nx < 1 || ny < 1 || nz < 1 || max_batch < 1) {
    set_error("mx_cnn_create: need out != NULL and nx, ny, nz, max_batch >= 1");
    return MX_ERR_INVALID_ARG;
  }
  *out = nullptr;
  mx_cnn* n = new mx_cnn();
  n->nx = nx;
  n->ny = ny;
  n->nz = nz;
  n->max_batch = max_batch;
  n->cells = (long)nx * ny * nz;
  const long nc = n->cells * max_batch;
  const long np = num_params_total();
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  };
  alloc((void**)&n->params, sizeof(float) * np);
  alloc((void**)&n->grad, sizeof(float) * np);
  alloc((void**)&n->am, sizeof(float) * np);
  alloc((void**)&n->av, sizeof(float) * np);
  const int bw_in[4] = {0, 64, 32, 16}, bw_out[4] = {0, 32, 64, 32};
  for (int l = 0; l < 4; ++l) {
    alloc((void**)&n->wf[l], sizeof(bf16_t) * 27 * kCoutPad[l] * kCinPad[l]);
    if (l > 0) alloc((void**)&n->wb[l], sizeof(bf16_t) * 27 * bw_in[l] * bw_out[l]);
  }
  alloc((void**)&n->x0, sizeof(bf16_t) * nc * 16);
  alloc((void**)&n->a1, sizeof(bf16_t) * nc * 32);
  alloc((void**)&n->y1, sizeof(bf16_t) * nc * 32);
  alloc((void**)&n->a2, sizeof(bf16_t) * nc * 64);
  alloc((void**)&n->y2, sizeof(bf16_t) * nc * 64);
  alloc((void**)&n->a3, sizeof(bf16_t) * nc * 32);
  alloc((void**)&n->y3, sizeof(bf16_t) * nc * 32);
  alloc((void**)&n->dy4, sizeof(bf16_t) * nc * 16);
  alloc((void**)&n->dy3, sizeof(bf16_t) * nc * 32);
  alloc((void**)&n->dy2, sizeof(bf16_t) * nc * 64);
  alloc((void**)&n->dy1, sizeof(bf16_t) * nc * 32);
  alloc((void**)&n->pred, sizeof(float4) * nc);
  alloc((void**)&n->loss, sizeof(float));
  alloc((void**)&n->flag, sizeof(int));
  if (!ok) {
    mx_cnn_destroy(n);
    set_error("mx_cnn_create: device allocation failed");
    return MX_ERR_OOM;
  }
  if (cudaMemset(n->params, 0, sizeof(float) * np) != cudaSuccess || cudaMemset(n->flag, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(n->am, 0, sizeof(float) * np) != cudaSuccess ||
      cudaMemset(n->av, 0, sizeof(float) * np) != cudaSuccess) {
    mx_cnn_destroy(n);
    set_error("mx_cnn_create: memset failed");
    return MX_ERR_CUDA;
  }
  *out = n;
  return MX_OK;
}

mx_status mx_cnn_sync(mx_cnn* n, mx_stream_t stream) {
  clear_error();
  if (!n) {
    set_error("mx_cnn_sync: NULL net");
    return MX_ERR_INVALID_ARG;
  }
  int f = 0;
  MX_TRY(cnn_take_flag(n, (cudaStream_t)stream, &f));
  if (f & kFlagTimeout) {
    set_error("mx_cnn_sync: a bounded wait for the tensor cores ran out");
    return MX_ERR_TIMEOUT;
  }
  return MX_OK;
}

mx_status mx_cnn_set_params(mx_cnn* n, const float* params, mx_stream_t stream) {
  if (!n || !params) {
    set_error("mx_cnn_set_params: NULL argument");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MX_CUDA_TRY(cudaMemcpyAsync(n->params, params, sizeof(float) * num_params_total(), cudaMemcpyDeviceToDevice, st));
  MX_CUDA_TRY(cudaMemsetAsync(n->am, 0, sizeof(float) * num_params_total(), st));
  MX_CUDA_TRY(cudaMemsetAsync(n->av, 0, sizeof(float) * num_params_total(), st));
  n->adam_t = 0;
  return pack_all(n, st);
}

mx_status mx_cnn_get_params(const mx_cnn* n, float* params, mx_stream_t stream) {
  if (!n || !params) {
    set_error("mx_cnn_get_params: NULL argument");
    return MX_ERR_INVALID_ARG;
  }
  MX_CUDA_TRY(cudaMemcpyAsync(params, n->params, sizeof(float) * num_params_total(), cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return MX_OK;
}

mx_status mx_cnn_set_normalizer(mx_cnn* n, const double stats[12]) {
  if (!n || !stats) {
    set_error("mx_cnn_set_normalizer: NULL argument");
    return MX_ERR_INVALID_ARG;
  }
  for (int q = 0; q < 12; ++q) {
    if (!isfinite(stats[q]) || ((q % 6) >= 3 && !(stats[q] > 0))) {
      set_error("mx_cnn_set_normalizer: standard deviations must be > 0 and every entry finite");
      return MX_ERR_INVALID_ARG;
    }
    n->stats[q] = (float)stats[q];
  }
  return MX_OK;
}

static mx_status check_batch(const mx_cnn* n, const float* m, int batch, const char* what) {
  if (!n || !m || batch < 1 || batch > n->max_batch || (((uintptr_t)m) & 15)) {
    set_error(std::string(what) + ": bad network, pointer or batch (1..max_batch)");
    return MX_ERR_INVALID_ARG;
  }
  return MX_OK;
}

mx_status mx_cnn_forward(mx_cnn* n, const float* m, float* h, int batch, mx_stream_t stream) {
  MX_TRY(check_batch(n, m, batch, "mx_cnn_forward"));
  if (!h || (((uintptr_t)h) & 15)) {
    set_error("mx_cnn_forward: h must be a 16-byte aligned device pointer");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MX_TRY(cnn_forward_to_pred(n, (const float4*)m, batch, st));
  const float* s = n->stats;
  const long nc = n->cells * batch;
  denormalize_out_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
      n->pred, (float4*)h, nc, make_float3(s[6], s[7], s[8]), make_float3(s[9], s[10], s[11]));
  return launch_check("denormalize_out_kernel");
}

mx_status mx_cnn_loss_grad(mx_cnn* n, const float* m, const float* h_target, int batch, float* loss_out,
                           float* grad_out, mx_stream_t stream) {
  MX_TRY(check_batch(n, m, batch, "mx_cnn_loss_grad"));
  if (!h_target || (((uintptr_t)h_target) & 15)) {
    set_error("mx_cnn_loss_grad: h_target must be a 16-byte aligned device pointer");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MX_TRY(cnn_forward_to_pred(n, (const float4*)m, batch, st));
  const long nc = n->cells * batch;
  const long np = num_params_total();
  MX_CUDA_TRY(cudaMemsetAsync(n->loss, 0, sizeof(float), st));
  MX_CUDA_TRY(cudaMemsetAsync(n->grad, 0, sizeof(float) * np, st));
  const float* s = n->stats;
  loss_kernel<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(
      n->pred, (const float4*)h_target, nc, make_float3(s[6], s[7], s[8]),
      make_float3(1.f / s[9], 1.f / s[10], 1.f / s[11]), 1.f / (3.f * (float)nc), n->dy4, n->loss);
  MX_TRY(launch_check("loss_kernel"));
  const ConvDims d = conv_dims(n, batch);
  float* G = n->grad;
  const unsigned bgrid = (unsigned)((nc + 1023) / 1024 < 1024 ? (nc + 1023) / 1024 : 1024);
  // layer 4: weights, bias, then dY3 = conv(dY4, W4') * gelu'(y3)
  MX_TRY((wgrad_run<32, 16>(n->a3, n->dy4, G + layer_w_off(3), d, 32, 3, n->flag, st)));
  bgrad_kernel<<<bgrid, 256, 0, st>>>(n->dy4, 16, 3, nc, G + layer_w_off(3) + 3 * 32 * 27);
  MX_TRY(launch_check("bgrad_kernel"));
  MX_TRY((conv_run<16, 32, CM_BWD>(n->dy4, n->wb[3], nullptr, n->dy3, n->y3, nullptr, d, n->flag, st)));
  // layer 3
  MX_TRY((wgrad_run<64, 32>(n->a2, n->dy3, G + layer_w_off(2), d, 64, 32, n->flag, st)));
  bgrad_kernel<<<bgrid, 256, 0, st>>>(n->dy3, 32, 32, nc, G + layer_w_off(2) + 32 * 64 * 27);
  MX_TRY(launch_check("bgrad_kernel"));
  MX_TRY((conv_run<32, 64, CM_BWD>(n->dy3, n->wb[2], nullptr, n->dy2, n->y2, nullptr, d, n->flag, st)));
  // layer 2
  MX_TRY((wgrad_run<32, 64>(n->a1, n->dy2, G + layer_w_off(1), d, 32, 64, n->flag, st)));
  bgrad_kernel<<<bgrid, 256, 0, st>>>(n->dy2, 64, 64, nc, G + layer_w_off(1) + 64 * 32 * 27);
  MX_TRY(launch_check("bgrad_kernel"));
  MX_TRY((conv_run<64, 32, CM_BWD>(n->dy2, n->wb[1], nullptr, n->dy1, n->y1, nullptr, d, n->flag, st)));
  // layer 1
  MX_TRY((wgrad_run<16, 32>(n->x0, n->dy1, G + layer_w_off(0), d, 3, 32, n->flag, st)));
  bgrad_kernel<<<bgrid, 256, 0, st>>>(n->dy1, 32, 32, nc, G + layer_w_off(0) + 32 * 3 * 27);
  MX_TRY(launch_check("bgrad_kernel"));
  if (loss_out) MX_CUDA_TRY(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (grad_out) MX_CUDA_TRY(cudaMemcpyAsync(grad_out, n->grad, sizeof(float) * np, cudaMemcpyDeviceToDevice, st));
  return MX_OK;
}

mx_status mx_cnn_adam_step(mx_cnn* n, double lr, double weight_decay, mx_stream_t stream) {
  if (!n || !(lr > 0) || !(weight_decay >= 0)) {
    set_error("mx_cnn_adam_step: need a network, lr > 0 and weight_decay >= 0");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  n->adam_t += 1;
  MX_TRY(adam_update(n->params, n->grad, n->am, n->av, num_params_total(), lr, weight_decay, n->adam_t, st));
  return pack_all(n, st);
}

}  // extern "C"
