// Discrete adjoint of the RK4 step (gradient of an objective of the final
// magnetisation with respect to the raw initial field and the per-cell Ms).
//
// One RK4 step (every stage input renormalised, Sec. II-B):
//   k1 = f(m0); u1 = m0 + dt/2 k1; m1 = N(u1); k2 = f(m1); u2 = m0 + dt/2 k2;
//   m2 = N(u2); k3 = f(m2); u3 = m0 + dt k3; m3 = N(u3); k4 = f(m3);
//   u4 = m0 + dt/6 (k1 + 2 k2 + 2 k3 + k4); m_new = N(u4),
// with N(u) = u/|u| and f(m) = c [m x H + alpha m x (m x H)] (Eq. 1),
// c = -gamma0/(1+alpha^2), H = L m + h_bias.  L (demag, exchange, DMI with the
// chiral ghosts, anisotropy) is linear and Ms-weighted symmetric, so
// L^T g = Ms (L (g / Ms)).  Reverse sweep for a cotangent lam of m_new:
//   lam_u4 = J_N(u4)^T lam; lam_m0 = lam_u4; lam_k4 = dt/6 lam_u4;
//   stage s = 3, 2, 1: lam_ms = f'(m_s)^T lam_ks, lam_us = J_N(u_s)^T lam_ms,
//     lam_m0 += lam_us, lam_k(s) = (dt/3 or dt/6) lam_u4 + (dt or dt/2) lam_us;
//   stage 0: lam_m0 += f'(m0)^T lam_k1.
// J_N(u)^T l = (l - n (n.l)) / |u| with n = N(u); |u| travels in the w slot of
// every renormalised stage output.  For a stage with state m and cotangent v:
//   g_m = c [H x v + alpha (v (m.H) + H (v.m) - 2 m (v.H))]
//   g_H = c [v x m + alpha (m (v.m) - v |m|^2)]
//   f'(m)^T v = g_m + Ms (L (g_H / Ms))
//   dJ/dMs_i += m_i . (demag field of g_H)_i - (g_H/Ms)_i . (L_local m)_i
// (the demag field of M = Ms (g_H/Ms) is what the convolution returns for
// input g_H / Ms).  The forward keeps a checkpoint every C steps; the reverse
// sweep recomputes each segment's states and each step's stage states.
#include <string>

#include "common.cuh"
#include "kernels.cuh"
#include "local.cuh"
#include "xrows.cuh"

namespace mx {

struct AdjWork {
  int nsteps = 0, every = 0, nckpt = 0;
  float4* ckpt = nullptr;   // nckpt states
  float4* seg = nullptr;    // every + 1 states
  float4* st = nullptr;     // 3 stage states m1, m2, m3
  float4* hd4 = nullptr;    // demag fields of m0, m1, m2, m3
  float4* raw = nullptr;    // raw initial field
  float4* lam_acc = nullptr;
  float4* lam_u4 = nullptr;
  float4* lam_k = nullptr;
  float4* wbuf = nullptr;   // g_H / Ms
  float4* gm = nullptr;     // g_m
  float4* hdw = nullptr;    // demag field of wbuf
  double* dms = nullptr;
  bool recorded = false;
  double dt = 0.0;
  // Stored segments: the recompute of a segment keeps every step's three
  // stage states and four demag fields, so the reverse step does not
  // recompute them (used while they take at most kAdjStoreBytes).
  float4* segst = nullptr;  // every x 3 stage states
  float4* seghd = nullptr;  // every x 4 demag fields
  float4* wbuf2 = nullptr;  // second (w, g_m) pair of the fused reverse kernels
  float4* gm2 = nullptr;
  // graphs of one full segment (forward, recompute, reverse), for graph_dt
  cudaGraphExec_t g_fwd = nullptr, g_rec = nullptr, g_rev = nullptr;
  double graph_dt = 0.0;
  bool last_stored = false;  // the recorded forward left the last segment stored
};

constexpr double kAdjStoreBytes = 4.0e9;

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// Per-cell pieces of the reverse stage, shared by the separate and the fused kernels.
//
// prep: for state m (stencil), its demag field hd and the cotangent v of
// its stage rate, g_m = c [H x v + alpha (v (m.H) + H (v.m) - 2 m (v.H))] and
// w = g_H / Ms with g_H = c [v x m + alpha (m (v.m) - v |m|^2)].
template <bool DMI>
__device__ __forceinline__ void prep_cell(const float4* __restrict__ m, const float4* __restrict__ hd, const Grid& g,
                                          const LocalCoef& c, int i, int j, int k, long idx, float3 v,
                                          float4* __restrict__ wbuf, float4* __restrict__ gm) {
  const float3 mc = f3(m[idx]);
  const float ms = c.ms_map ? __ldg(&c.ms_map[idx]) : c.Ms;
  Terms t;
  local_terms<DMI>(m, hd, g, c, i, j, k, idx, mc, 1.f / ms, t);
  const float3 H = t.demag + t.exch + t.anis + t.dmi + t.zee;
  const float mH = dot3(mc, H), vm = dot3(v, mc), vH = dot3(v, H), mm = dot3(mc, mc);
  float3 gmv = c.alpha * (mH * v + vm * H - (2.f * vH) * mc);
  float3 gh = c.alpha * (vm * mc - mm * v);
  if (c.precession) {
    gmv = gmv + cross3(H, v);
    gh = gh + cross3(v, mc);
  }
  gmv = c.llg * gmv;
  gh = (c.llg / ms) * gh;
  gm[idx] = make_float4(gmv.x, gmv.y, gmv.z, 0.f);
  wbuf[idx] = make_float4(gh.x, gh.y, gh.z, 0.f);
}

// finish: lam_m = g_m + Ms (L w) (w's stencil and hdw, the demag field of
// w); the Ms gradient term; the stage's share of lam_acc; returns the next
// stage rate's cotangent (STAGE 3, 2, 1) or zero (STAGE 0).
template <bool DMI, int STAGE>
__device__ __forceinline__ float3 finish_cell_v(const float4* __restrict__ m, const float4* __restrict__ wbuf,
                                                float3 hdwv, const float4* __restrict__ gm,
                                                const float4* __restrict__ lam_u4, float4* __restrict__ lam_acc,
                                                double* __restrict__ dms, const Grid& g, const LocalCoef& c, float dt,
                                                int i, int j, int k, long idx) {
  const float ms = c.ms_map ? __ldg(&c.ms_map[idx]) : c.Ms;
  const float inv_ms = 1.f / ms;
  // L applied to w = g_H / Ms: demag from the convolution, local terms here
  LocalCoef cl = c;
  cl.hx = cl.hy = cl.hz = 0.f;  // the bias is not part of the linear operator
  const float3 wc = f3(wbuf[idx]);
  Terms tw;
  local_terms_v<DMI>(wbuf, hdwv, g, cl, i, j, k, idx, wc, inv_ms, tw);
  const float3 Lw = tw.demag + tw.exch + tw.anis + tw.dmi;
  const float4 m4 = m[idx];
  const float3 mc = f3(m4);
  const float3 lam_m = f3(gm[idx]) + ms * Lw;
  // Ms gradient: m . (demag of g_H) - w . (L_local m)
  if (dms) {
    Terms tm;
    local_terms<DMI>(m, nullptr, g, cl, i, j, k, idx, mc, inv_ms, tm);
    const float3 Lm = tm.exch + tm.anis + tm.dmi;
    dms[idx] += (double)dot3(mc, tw.demag) - (double)dot3(wc, Lm);
  }
  if (STAGE == 0) {
    const float4 a = lam_acc[idx];
    lam_acc[idx] = make_float4(a.x + lam_m.x, a.y + lam_m.y, a.z + lam_m.z, 0.f);
    return make_float3(0.f, 0.f, 0.f);
  }
  // J_N(u_s)^T lam_m with n = m (unit), |u_s| in m.w
  const float3 lu = (1.f / m4.w) * (lam_m - dot3(mc, lam_m) * mc);
  const float4 a = lam_acc[idx];
  lam_acc[idx] = make_float4(a.x + lu.x, a.y + lu.y, a.z + lu.z, 0.f);
  const float3 u4 = f3(lam_u4[idx]);
  const float cu4 = (STAGE == 1) ? dt / 6.f : dt / 3.f;
  const float cus = (STAGE == 3) ? dt : 0.5f * dt;
  return cu4 * u4 + cus * lu;
}

// The same with the demag field of w read from hdw (zero if hdw is null).
template <bool DMI, int STAGE>
__device__ __forceinline__ float3 finish_cell(const float4* __restrict__ m, const float4* __restrict__ wbuf,
                                              const float4* __restrict__ hdw, const float4* __restrict__ gm,
                                              const float4* __restrict__ lam_u4, float4* __restrict__ lam_acc,
                                              double* __restrict__ dms, const Grid& g, const LocalCoef& c, float dt,
                                              int i, int j, int k, long idx) {
  return finish_cell_v<DMI, STAGE>(m, wbuf, hdw ? f3(__ldg(&hdw[idx])) : make_float3(0.f, 0.f, 0.f), gm, lam_u4,
                                   lam_acc, dms, g, c, dt, i, j, k, idx);
}

template <bool DMI>
__global__ void __launch_bounds__(256) adj_prep_kernel(const float4* __restrict__ m, const float4* __restrict__ hd,
                                                       const float4* __restrict__ lam_k, Grid g, LocalCoef c,
                                                       float4* __restrict__ wbuf, float4* __restrict__ gm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long idx = ((long)k * g.ny + j) * g.nx + i;
  prep_cell<DMI>(m, hd, g, c, i, j, k, idx, f3(lam_k[idx]), wbuf, gm);
}

// STAGE 3, 2, 1: renormalised stage input; STAGE 0: the step's start state.
template <bool DMI, int STAGE>
__global__ void __launch_bounds__(256) adj_finish_kernel(const float4* __restrict__ m, const float4* __restrict__ wbuf,
                                                         const float4* __restrict__ hdw,
                                                         const float4* __restrict__ gm,
                                                         const float4* __restrict__ lam_u4,
                                                         float4* __restrict__ lam_acc, float4* __restrict__ lam_k,
                                                         double* __restrict__ dms, Grid g, LocalCoef c, float dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long idx = ((long)k * g.ny + j) * g.nx + i;
  const float3 nk = finish_cell<DMI, STAGE>(m, wbuf, hdw, gm, lam_u4, lam_acc, dms, g, c, dt, i, j, k, idx);
  if (STAGE > 0) lam_k[idx] = make_float4(nk.x, nk.y, nk.z, 0.f);
}

// Fused: begin of the reverse step (lam_u4 = J_N(u4)^T lam, lam_acc = lam_u4,
// stage-4 cotangent dt/6 lam_u4) and prep of the last stage state m3.
template <bool DMI>
__global__ void __launch_bounds__(256) adj_begin_prep_kernel(const float4* __restrict__ mnew,
                                                             const float4* __restrict__ m3,
                                                             const float4* __restrict__ hd3,
                                                             float4* __restrict__ lam_acc, float4* __restrict__ lam_u4,
                                                             float4* __restrict__ wbuf, float4* __restrict__ gm,
                                                             Grid g, LocalCoef c, float dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long idx = ((long)k * g.ny + j) * g.nx + i;
  const float4 n4 = mnew[idx];
  const float3 nc = f3(n4);
  const float3 l = f3(lam_acc[idx]);
  const float3 lu = (1.f / n4.w) * (l - dot3(nc, l) * nc);
  lam_u4[idx] = make_float4(lu.x, lu.y, lu.z, 0.f);
  lam_acc[idx] = make_float4(lu.x, lu.y, lu.z, 0.f);
  prep_cell<DMI>(m3, hd3, g, c, i, j, k, idx, (dt / 6.f) * lu, wbuf, gm);
}

// Fused: finish of stage STAGE (3, 2, 1) and prep of stage STAGE - 1, whose
// cotangent is the value just computed at the same cell.  w and g_m of the
// next stage go to the other buffer pair, because finish reads w's stencil.
template <bool DMI, int STAGE>
__global__ void __launch_bounds__(256) adj_finish_prep_kernel(
    const float4* __restrict__ m, const float4* __restrict__ wbuf, const float4* __restrict__ hdw,
    const float4* __restrict__ gm, const float4* __restrict__ lam_u4, float4* __restrict__ lam_acc,
    double* __restrict__ dms, const float4* __restrict__ m_prev, const float4* __restrict__ hd_prev,
    float4* __restrict__ wbuf_out, float4* __restrict__ gm_out, Grid g, LocalCoef c, float dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long idx = ((long)k * g.ny + j) * g.nx + i;
  const float3 nk = finish_cell<DMI, STAGE>(m, wbuf, hdw, gm, lam_u4, lam_acc, dms, g, c, dt, i, j, k, idx);
  prep_cell<DMI>(m_prev, hd_prev, g, c, i, j, k, idx, nk, wbuf_out, gm_out);
}

// ---------------------------------------------------------------------------
// Row kernels of the reverse sweep on few-row grids (as the forward step's
// row kernels): per stage, the y/z passes of w's spectrum and one kernel that
// takes the c2r transforms of its block's rows (the demag field of w, kept in
// shared memory), finishes the stage and prepares the one before at every
// cell of those rows, and leaves the forward x pass of the new w in w1.  The
// new w and g_m go to the other buffer pair, and the block reads its own rows
// of the new w back after a block barrier.
// ---------------------------------------------------------------------------
struct AdjRowArgs {
  const float4* mnew;     // step result (begin only)
  const float4* m;        // state of the stage being finished
  const float4* wbuf;     // its w (stencil) and g_m
  const float4* gm;
  float4* lam_u4;
  float4* lam_acc;
  double* dms;
  const float4* m_prev;   // state and demag field of the stage being prepared
  const float4* hd_prev;
  float4* wbuf_out;       // its w and g_m
  float4* gm_out;
};

// begin of a reverse step at one cell (lam_u4 = J_N(u4)^T lam_acc with u4's
// norm in mnew.w, lam_acc = lam_u4) and the prep of its last stage
template <bool DMI>
__device__ __forceinline__ void adj_begin_cell(const AdjRowArgs& a, const float4* __restrict__ mnew, const Grid& g,
                                               const LocalCoef& c, float dt, int i, int y, int z, long idx) {
  const float4 n4 = mnew[idx];
  const float3 nc = f3(n4);
  const float3 l = f3(a.lam_acc[idx]);
  const float3 lu = (1.f / n4.w) * (l - dot3(nc, l) * nc);
  a.lam_u4[idx] = make_float4(lu.x, lu.y, lu.z, 0.f);
  a.lam_acc[idx] = make_float4(lu.x, lu.y, lu.z, 0.f);
  prep_cell<DMI>(a.m_prev, a.hd_prev, g, c, i, y, z, idx, (dt / 6.f) * lu, a.wbuf_out, a.gm_out);
}

template <bool DMI, int R, int NT>
__device__ __forceinline__ void adj_row_begin_cells(const AdjRowArgs& a, const Grid& g, const LocalCoef& c, float dt,
                                                    int row0) {
  const int total = min(R, g.ny * g.nz - row0) * g.nx;
  for (int e = threadIdx.x; e < total; e += NT) {
    const int r = e / g.nx, i = e - r * g.nx;
    const int row = row0 + r;
    const int z = row / g.ny, y = row - z * g.ny;
    adj_begin_cell<DMI>(a, a.mnew, g, c, dt, i, y, z, (long)row * g.nx + i);
  }
}

// STAGE 0 with CHAIN: after the finish, the begin of the step before at the
// same cell (its result is this step's start state a.m) with the prep of its
// last stage (a.m_prev, a.hd_prev -> a.wbuf_out, a.gm_out).
template <bool DMI, int STAGE, int E, int S, int R, int NT, bool CHAIN = false>
__device__ __forceinline__ void adj_row_cells(const float2* sm, const AdjRowArgs& a, const Grid& g,
                                              const LocalCoef& c, float dt, int row0) {
  const int total = min(R, g.ny * g.nz - row0) * g.nx;
  for (int e = threadIdx.x; e < total; e += NT) {
    const int r = e / g.nx, i = e - r * g.nx;
    const int row = row0 + r;
    const int z = row / g.ny, y = row - z * g.ny;
    const long idx = (long)row * g.nx + i;
    const float3 nk = finish_cell_v<DMI, STAGE>(a.m, a.wbuf, xi_cell<E, S>(sm, r, i), a.gm, a.lam_u4, a.lam_acc,
                                                a.dms, g, c, dt, i, y, z, idx);
    if (STAGE > 0) prep_cell<DMI>(a.m_prev, a.hd_prev, g, c, i, y, z, idx, nk, a.wbuf_out, a.gm_out);
    if (STAGE == 0 && CHAIN) adj_begin_cell<DMI>(a, a.m, g, c, dt, i, y, z, idx);
  }
}

template <int E, int S, int R, int NT, bool DMI>
__global__ void __launch_bounds__(NT) adj_row_begin_kernel(float2* __restrict__ w1, Grid g, float ms,
                                                           const float* __restrict__ ms_map,
                                                           const float2* __restrict__ twM,
                                                           const float2* __restrict__ twP, AdjRowArgs a, LocalCoef c,
                                                           float dt) {
  extern __shared__ float2 sm[];
  const int row0 = blockIdx.x * R;
  pdl_wait();
  adj_row_begin_cells<DMI, R, NT>(a, g, c, dt, row0);
  __syncthreads();
  xf_rows<E, S, R, NT, true>(sm, a.wbuf_out, g, ms, ms_map, w1, row0, twM, twP);
}

template <int E, int S, int R, int NT, bool DMI>
__global__ void __launch_bounds__(NT) adj_row_kernel(float2* __restrict__ w1, Grid g, float ms,
                                                     const float* __restrict__ ms_map, const float2* __restrict__ twM,
                                                     const float2* __restrict__ twP, AdjRowArgs a, LocalCoef c,
                                                     float dt, int stage, int chain) {
  extern __shared__ float2 sm[];
  const int row0 = blockIdx.x * R;
  pdl_wait();
  xi_rows<E, S, R, NT>(sm, w1, g, row0, twM, twP);
  switch (stage) {
    case 3: adj_row_cells<DMI, 3, E, S, R, NT>(sm, a, g, c, dt, row0); break;
    case 2: adj_row_cells<DMI, 2, E, S, R, NT>(sm, a, g, c, dt, row0); break;
    case 1: adj_row_cells<DMI, 1, E, S, R, NT>(sm, a, g, c, dt, row0); break;
    default:
      if (!chain) {
        adj_row_cells<DMI, 0, E, S, R, NT>(sm, a, g, c, dt, row0);
        return;
      }
      adj_row_cells<DMI, 0, E, S, R, NT, true>(sm, a, g, c, dt, row0);
      break;
  }
  __syncthreads();  // the block's rows of the new w are written; the c2r lines are read
  xf_rows<E, S, R, NT, true>(sm, a.wbuf_out, g, ms, ms_map, w1, row0, twM, twP);
}

// Launches the begin kernel (begin) or the stage kernel of `stage` for the
// grid's few-row x configuration.
struct AdjRowLaunch {
  mx_ctx* ctx;
  const AdjRowArgs* a;
  float dt;
  int stage;
  bool begin;
  bool chain;
  cudaStream_t st;
  template <int E, int S, int R, int NT> mx_status run() {
    const size_t sm = sizeof(float2) * XfShape<S, R>::lines * LineFft<E, S>::kPitch;
    static_assert(sizeof(float2) * XfShape<S, R>::lines * LineFft<E, S>::kPitch <= 48 * 1024,
                  "row kernel shared memory");
    const Grid& g = ctx->g;
    const LocalCoef c = local_coef(ctx);
    const dim3 grid((g.ny * g.nz + R - 1) / R);
    if (begin) {
      auto k = c.dmi ? adj_row_begin_kernel<E, S, R, NT, true> : adj_row_begin_kernel<E, S, R, NT, false>;
      launch_pdl(k, grid, dim3(NT), sm, st, ctx->w1, g, (float)ctx->p.Ms, ctx->ms_map, ctx->tw_m, ctx->tw_x, *a,
                 c, dt);
      return launch_check("adj_row_begin_kernel");
    }
    auto k = c.dmi ? adj_row_kernel<E, S, R, NT, true> : adj_row_kernel<E, S, R, NT, false>;
    launch_pdl(k, grid, dim3(NT), sm, st, ctx->w1, g, (float)ctx->p.Ms, ctx->ms_map, ctx->tw_m, ctx->tw_x, *a, c,
               dt, stage, chain ? 1 : 0);
    return launch_check("adj_row_kernel");
  }
};

// lam_u4 = J_N(u4)^T lam (m_new carries |u4| in w); lam_acc = lam_u4; lam_k = dt/6 lam_u4
__global__ void adj_begin_kernel(const float4* __restrict__ mnew, float4* __restrict__ lam_acc,
                                 float4* __restrict__ lam_u4, float4* __restrict__ lam_k, long n, float dt) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const float4 m4 = mnew[idx];
  const float3 mc = f3(m4);
  const float3 l = f3(lam_acc[idx]);
  const float3 lu = (1.f / m4.w) * (l - dot3(mc, l) * mc);
  lam_u4[idx] = make_float4(lu.x, lu.y, lu.z, 0.f);
  lam_acc[idx] = make_float4(lu.x, lu.y, lu.z, 0.f);
  lam_k[idx] = make_float4(dt / 6.f * lu.x, dt / 6.f * lu.y, dt / 6.f * lu.z, 0.f);
}

// grad of the raw field: J_N(raw)^T lam; Ms gradient to float
__global__ void adj_end_kernel(const float4* __restrict__ raw, const float4* __restrict__ lam, float4* __restrict__ g,
                               const double* __restrict__ dms, float* __restrict__ gms, long n) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const float3 r = f3(raw[idx]);
  const float nr = norm3df(r.x, r.y, r.z);
  const float3 u = (1.f / nr) * r;
  const float3 l = f3(lam[idx]);
  const float3 o = (1.f / nr) * (l - dot3(u, l) * u);
  g[idx] = make_float4(o.x, o.y, o.z, 0.f);
  if (gms) gms[idx] = (float)dms[idx];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static void adj_dims(const Grid& g, dim3& grid, dim3& block) {
  block = dim3(32, 8, 1);
  if (g.nx < 32) block = dim3(g.nx <= 8 ? 8 : (g.nx <= 16 ? 16 : 32), 256 / (g.nx <= 8 ? 8 : (g.nx <= 16 ? 16 : 32)), 1);
  grid = dim3((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, g.nz);
}

bool adjoint_recorded(const mx_ctx* ctx) { return ctx->adj && ctx->adj->recorded; }

static void drop_graphs(AdjWork* w) {
  for (cudaGraphExec_t* gp : {&w->g_fwd, &w->g_rec, &w->g_rev}) {
    if (*gp) cudaGraphExecDestroy(*gp);
    *gp = nullptr;
  }
}

void adjoint_invalidate_graphs(mx_ctx* ctx) {
  if (ctx->adj) drop_graphs(ctx->adj);
}

void adjoint_free(mx_ctx* ctx) {
  AdjWork* w = ctx->adj;
  if (!w) return;
  drop_graphs(w);
  void* ptrs[] = {w->ckpt, w->seg, w->st, w->hd4, w->raw, w->lam_acc, w->lam_u4, w->lam_k, w->wbuf, w->gm, w->hdw,
                  w->dms, w->segst, w->seghd, w->wbuf2, w->gm2};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete w;
  ctx->adj = nullptr;
}

mx_status adjoint_reserve(mx_ctx* ctx, int nsteps, int every) {
  if (nsteps < 1 || every < 1) {
    set_error("mx_adjoint_reserve: need nsteps >= 1 and checkpoint_every >= 1");
    return MX_ERR_INVALID_ARG;
  }
  adjoint_free(ctx);
  // this unit's copy of the W_32 table used by the register FFTs of the
  // reverse sweep's row kernels
  MX_TRY(upload_w32());
  AdjWork* w = new AdjWork();
  ctx->adj = w;
  w->nsteps = nsteps;
  w->every = every < nsteps ? every : nsteps;
  w->nckpt = (nsteps + w->every - 1) / w->every;
  const long nc = ctx->g.ncell;
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  };
  alloc((void**)&w->ckpt, sizeof(float4) * nc * w->nckpt);
  alloc((void**)&w->seg, sizeof(float4) * nc * (w->every + 1));
  alloc((void**)&w->st, sizeof(float4) * nc * 3);
  alloc((void**)&w->hd4, sizeof(float4) * nc * 4);
  alloc((void**)&w->raw, sizeof(float4) * nc);
  alloc((void**)&w->lam_acc, sizeof(float4) * nc);
  alloc((void**)&w->lam_u4, sizeof(float4) * nc);
  alloc((void**)&w->lam_k, sizeof(float4) * nc);
  alloc((void**)&w->wbuf, sizeof(float4) * nc);
  alloc((void**)&w->gm, sizeof(float4) * nc);
  alloc((void**)&w->hdw, sizeof(float4) * nc);
  alloc((void**)&w->dms, sizeof(double) * nc);
  if (7.0 * w->every * nc * sizeof(float4) <= kAdjStoreBytes) {
    alloc((void**)&w->segst, sizeof(float4) * nc * 3 * w->every);
    alloc((void**)&w->seghd, sizeof(float4) * nc * 4 * w->every);
    alloc((void**)&w->wbuf2, sizeof(float4) * nc);
    alloc((void**)&w->gm2, sizeof(float4) * nc);
  }
  if (!ok) {
    adjoint_free(ctx);
    set_error("mx_adjoint_reserve: device allocation failed");
    return MX_ERR_OOM;
  }
  return MX_OK;
}

// Capture what `enqueue` puts on a stream into an executable graph.
template <typename F>
static mx_status capture_graph(mx_ctx* ctx, cudaGraphExec_t* out, F enqueue) {
  cudaGraph_t graph = nullptr;
  MX_CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  const mx_status s = enqueue(ctx->cap_stream);
  const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
  if (s != MX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) {
    set_error(std::string("adjoint: capture failed: ") + cudaGetErrorString(e));
    return MX_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    *out = nullptr;
    set_error(std::string("adjoint: instantiate failed: ") + cudaGetErrorString(ei));
    return MX_ERR_CUDA;
  }
  return MX_OK;
}

static bool graphs_usable(const mx_ctx* ctx) { return ctx->prof == nullptr; }

// Stored segments.  Step i of the segment takes seg[i] to seg[i + 1]; its
// stage states are segst[i][0..2] and the demag fields of seg[i] and the
// three stage states seghd[i][0..3].
// With row kernels (row_steps) each stage is the y/z passes plus one row
// kernel that also writes the stage state's demag field; step i = 0 runs the
// forward x pass of seg[0] first, and each step leaves that of seg[i + 1].
static mx_status stored_recompute_step(mx_ctx* ctx, AdjWork* w, int i, float dt, bool demag, cudaStream_t st) {
  const long nc = ctx->g.ncell;
  const float4* m = w->seg + (long)i * nc;
  float4* S = w->segst + (long)i * 3 * nc;
  float4* Hd = w->seghd + (long)i * 4 * nc;
  const float4* states[4] = {m, S, S + nc, S + 2 * nc};
  float4* outs[4] = {S, S + nc, S + 2 * nc, w->seg + (long)(i + 1) * nc};
  const int modes[4] = {LM_RK4_S0, LM_RK4_S1, LM_RK4_S2, LM_RK4_S3};
  if (demag && row_steps(ctx, MX_RK4)) {
    if (i == 0) MX_TRY(fast_x_pass(ctx, m, nullptr, false, st));
    for (int q = 0; q < 4; ++q) {
      StageIO io{states[q], nullptr, m, ctx->acc, outs[q], dt, MX_TERM_ALL};
      MX_TRY(demag_yz(ctx, st));
      MX_TRY(fast_row_stage(ctx, modes[q], io, true, Hd + q * nc, st));
    }
    return MX_OK;
  }
  for (int q = 0; q < 4; ++q) {
    if (demag) MX_TRY(demag_field(ctx, states[q], Hd + q * nc, st));
    StageIO io{states[q], demag ? Hd + q * nc : nullptr, m, ctx->acc, outs[q], dt, MX_TERM_ALL};
    MX_TRY(local_stage(ctx, modes[q], io, st));
  }
  return MX_OK;
}

mx_status adjoint_forward(mx_ctx* ctx, const float4* m0_raw, float4* m_final, double dt, cudaStream_t st) {
  AdjWork* w = ctx->adj;
  const long nc = ctx->g.ncell;
  const size_t bytes = sizeof(float4) * nc;
  if (w->graph_dt != dt) {
    drop_graphs(w);
    w->graph_dt = dt;
  }
  MX_CUDA_TRY(cudaMemcpyAsync(w->raw, m0_raw, bytes, cudaMemcpyDeviceToDevice, st));
  float4* cur = w->seg;  // working state
  MX_CUDA_TRY(cudaMemcpyAsync(cur, m0_raw, bytes, cudaMemcpyDeviceToDevice, st));
  MX_TRY(normalize_field(ctx, cur, st));
  const bool use_graph = graphs_usable(ctx);
  const bool demag = ctx->p.demag != 0;
  if (use_graph && !w->g_fwd && w->nsteps >= w->every) {
    MX_TRY(capture_graph(ctx, &w->g_fwd, [&](cudaStream_t cs) -> mx_status {
      // consecutive steps on cur: each leaves the next one's forward x pass
      for (int s = 0; s < w->every; ++s) MX_TRY(rk4_step_direct(ctx, cur, dt, cs, s == 0, true));
      return MX_OK;
    }));
  }
  if (use_graph && w->segst && !w->g_rec && w->nsteps >= w->every) {
    MX_TRY(capture_graph(ctx, &w->g_rec, [&](cudaStream_t cs) -> mx_status {
      for (int i = 0; i < w->every; ++i) MX_TRY(stored_recompute_step(ctx, w, i, (float)dt, demag, cs));
      return MX_OK;
    }));
  }
  const float4* fin = cur;
  for (int kseg = 0; kseg < w->nckpt; ++kseg) {
    const int s0 = kseg * w->every;
    const int len = (s0 + w->every < w->nsteps) ? w->every : w->nsteps - s0;
    MX_CUDA_TRY(cudaMemcpyAsync(w->ckpt + (long)kseg * nc, cur, bytes, cudaMemcpyDeviceToDevice, st));
    if (w->segst && kseg == w->nckpt - 1) {
      // the last segment keeps its states and stage states: the reverse sweep
      // starts on it without recomputing it
      if (use_graph && len == w->every && w->g_rec) {
        MX_CUDA_TRY(cudaGraphLaunch(w->g_rec, st));
      } else {
        for (int i = 0; i < len; ++i) MX_TRY(stored_recompute_step(ctx, w, i, (float)dt, demag, st));
      }
      fin = w->seg + (long)len * nc;
    } else if (use_graph && len == w->every && w->g_fwd) {
      MX_CUDA_TRY(cudaGraphLaunch(w->g_fwd, st));
    } else {
      for (int s = 0; s < len; ++s) MX_TRY(rk4_step_direct(ctx, cur, dt, st, s == 0, true));
    }
  }
  w->last_stored = w->segst != nullptr;
  MX_CUDA_TRY(cudaMemcpyAsync(m_final, fin, bytes, cudaMemcpyDeviceToDevice, st));
  w->recorded = true;
  w->dt = dt;
  return MX_OK;
}

// With row kernels, `first` runs the begin of step i on its own and `chain`
// (i > 0 within a stored segment) folds the begin of step i - 1 into the
// last kernel of step i, so the next call is made with first = false.
template <bool DMI>
static mx_status stored_reverse_step_t(mx_ctx* ctx, AdjWork* w, int i, float dt, bool demag, cudaStream_t st,
                                       bool first, bool chain) {
  const Grid& g = ctx->g;
  const long nc = g.ncell;
  const LocalCoef c = local_coef(ctx);
  dim3 grid, block;
  adj_dims(g, grid, block);
  const float4* m = w->seg + (long)i * nc;
  const float4* mnew = m + nc;
  const float4* S = w->segst + (long)i * 3 * nc;
  const float4* Hd = w->seghd + (long)i * 4 * nc;
  const float4* states[4] = {m, S, S + nc, S + 2 * nc};
  float4* wb[2] = {w->wbuf, w->wbuf2};
  float4* gmb[2] = {w->gm, w->gm2};
  // demag fields of the stage states are zero without demag (hd4 cleared)
  const float4* hd[4];
  for (int q = 0; q < 4; ++q) hd[q] = demag ? Hd + q * nc : w->hd4;
  if (demag && row_steps(ctx, MX_RK4)) {
    // row kernels: begin + prep of stage 3, then per stage the y/z passes of
    // w's spectrum and the finish (+ prep of the stage before) row kernel
    AdjRowArgs a{mnew, nullptr, nullptr, nullptr, w->lam_u4, w->lam_acc, w->dms, states[3], hd[3], wb[0], gmb[0]};
    if (first) {
      AdjRowLaunch L{ctx, &a, dt, 0, true, false, st};
      MX_TRY(few_rows_dispatch(g.Px / 2, L));
    }
    int b = 0;
    for (int q = 3; q >= 0; --q) {
      MX_TRY(demag_yz(ctx, st));
      a.m = states[q];
      a.wbuf = wb[b];
      a.gm = gmb[b];
      a.m_prev = q > 0 ? states[q - 1] : nullptr;
      a.hd_prev = q > 0 ? hd[q - 1] : nullptr;
      a.wbuf_out = wb[b ^ 1];
      a.gm_out = gmb[b ^ 1];
      if (q == 0 && chain) {
        // the begin of step i - 1: its last stage state and demag field, and
        // its w and g_m into the first buffer pair
        const float4* Sp = w->segst + (long)(i - 1) * 3 * nc;
        a.m_prev = Sp + 2 * nc;
        a.hd_prev = demag ? w->seghd + (long)(i - 1) * 4 * nc + 3 * nc : w->hd4;
        a.wbuf_out = wb[0];
        a.gm_out = gmb[0];
      }
      AdjRowLaunch Lq{ctx, &a, dt, q, false, q == 0 && chain, st};
      MX_TRY(few_rows_dispatch(g.Px / 2, Lq));
      b ^= 1;
    }
    return MX_OK;
  }
  adj_begin_prep_kernel<DMI><<<grid, block, 0, st>>>(mnew, states[3], hd[3], w->lam_acc, w->lam_u4, wb[0], gmb[0],
                                                     g, c, dt);
  MX_TRY(launch_check("adj_begin_prep_kernel"));
  int b = 0;
  for (int q = 3; q >= 0; --q) {
    if (demag) MX_TRY(demag_field(ctx, wb[b], w->hdw, st));
    switch (q) {
      case 3:
        adj_finish_prep_kernel<DMI, 3><<<grid, block, 0, st>>>(states[3], wb[b], w->hdw, gmb[b], w->lam_u4,
                                                               w->lam_acc, w->dms, states[2], hd[2], wb[b ^ 1],
                                                               gmb[b ^ 1], g, c, dt);
        break;
      case 2:
        adj_finish_prep_kernel<DMI, 2><<<grid, block, 0, st>>>(states[2], wb[b], w->hdw, gmb[b], w->lam_u4,
                                                               w->lam_acc, w->dms, states[1], hd[1], wb[b ^ 1],
                                                               gmb[b ^ 1], g, c, dt);
        break;
      case 1:
        adj_finish_prep_kernel<DMI, 1><<<grid, block, 0, st>>>(states[1], wb[b], w->hdw, gmb[b], w->lam_u4,
                                                               w->lam_acc, w->dms, states[0], hd[0], wb[b ^ 1],
                                                               gmb[b ^ 1], g, c, dt);
        break;
      default:
        adj_finish_kernel<DMI, 0><<<grid, block, 0, st>>>(states[0], wb[b], w->hdw, gmb[b], w->lam_u4, w->lam_acc,
                                                          w->lam_k, w->dms, g, c, dt);
        break;
    }
    MX_TRY(launch_check("adj_finish_prep_kernel"));
    b ^= 1;
  }
  return MX_OK;
}

static mx_status stored_reverse_step(mx_ctx* ctx, AdjWork* w, int i, int len, float dt, bool demag, bool dmi,
                                     cudaStream_t st) {
  const bool first = i == len - 1, chain = i > 0;
  return dmi ? stored_reverse_step_t<true>(ctx, w, i, dt, demag, st, first, chain)
             : stored_reverse_step_t<false>(ctx, w, i, dt, demag, st, first, chain);
}

template <int STAGE>
static void launch_finish(bool dmi, dim3 grid, dim3 block, cudaStream_t st, AdjWork* w, const float4* m,
                          const Grid& g, const LocalCoef& c, float dt, bool want_ms) {
  double* dms = want_ms ? w->dms : nullptr;
  if (dmi)
    adj_finish_kernel<true, STAGE><<<grid, block, 0, st>>>(m, w->wbuf, w->hdw, w->gm, w->lam_u4, w->lam_acc,
                                                           w->lam_k, dms, g, c, dt);
  else
    adj_finish_kernel<false, STAGE><<<grid, block, 0, st>>>(m, w->wbuf, w->hdw, w->gm, w->lam_u4, w->lam_acc,
                                                            w->lam_k, dms, g, c, dt);
}

mx_status adjoint_backward(mx_ctx* ctx, const float4* lam_final, float4* grad_m0, float* grad_ms, cudaStream_t st) {
  AdjWork* w = ctx->adj;
  const Grid& g = ctx->g;
  const long nc = g.ncell;
  const size_t bytes = sizeof(float4) * nc;
  const float dt = (float)w->dt;
  const LocalCoef c = local_coef(ctx);
  const bool dmi = c.dmi != 0;
  const bool demag = ctx->p.demag != 0;
  dim3 grid, block;
  adj_dims(g, grid, block);
  const unsigned nb = (unsigned)((nc + 255) / 256);
  MX_CUDA_TRY(cudaMemcpyAsync(w->lam_acc, lam_final, bytes, cudaMemcpyDeviceToDevice, st));
  MX_CUDA_TRY(cudaMemsetAsync(w->dms, 0, sizeof(double) * nc, st));
  if (!demag) {
    MX_CUDA_TRY(cudaMemsetAsync(w->hd4, 0, 4 * bytes, st));
    MX_CUDA_TRY(cudaMemsetAsync(w->hdw, 0, bytes, st));
  }
  if (w->segst) {
    // stored segments: recompute each segment keeping its stage states, then
    // the fused reverse steps; full segments replay captured graphs
    const bool use_graph = graphs_usable(ctx);
    if (use_graph && w->nsteps >= w->every) {
      if (!w->g_rec)
        MX_TRY(capture_graph(ctx, &w->g_rec, [&](cudaStream_t cs) -> mx_status {
          for (int i = 0; i < w->every; ++i) MX_TRY(stored_recompute_step(ctx, w, i, dt, demag, cs));
          return MX_OK;
        }));
      if (!w->g_rev)
        MX_TRY(capture_graph(ctx, &w->g_rev, [&](cudaStream_t cs) -> mx_status {
          for (int i = w->every - 1; i >= 0; --i) MX_TRY(stored_reverse_step(ctx, w, i, w->every, dt, demag, dmi, cs));
          return MX_OK;
        }));
    }
    for (int kseg = w->nckpt - 1; kseg >= 0; --kseg) {
      const int s0 = kseg * w->every;
      const int len = (s0 + w->every < w->nsteps) ? w->every : w->nsteps - s0;
      // the recorded forward left the last segment stored (first backward only)
      const bool stored = w->last_stored && kseg == w->nckpt - 1;
      if (!stored) {
        MX_CUDA_TRY(cudaMemcpyAsync(w->seg, w->ckpt + (long)kseg * nc, bytes, cudaMemcpyDeviceToDevice, st));
        if (use_graph && len == w->every && w->g_rec)
          MX_CUDA_TRY(cudaGraphLaunch(w->g_rec, st));
        else
          for (int i = 0; i < len; ++i) MX_TRY(stored_recompute_step(ctx, w, i, dt, demag, st));
      }
      if (use_graph && len == w->every && w->g_rev)
        MX_CUDA_TRY(cudaGraphLaunch(w->g_rev, st));
      else
        for (int i = len - 1; i >= 0; --i) MX_TRY(stored_reverse_step(ctx, w, i, len, dt, demag, dmi, st));
    }
    w->last_stored = false;  // the segment buffers now hold the first segment
    adj_end_kernel<<<nb, 256, 0, st>>>(w->raw, w->lam_acc, grad_m0, w->dms, grad_ms, nc);
    return launch_check("adj_end_kernel");
  }
  float4* st1 = w->st;
  float4* st2 = w->st + nc;
  float4* st3 = w->st + 2 * nc;
  for (int kseg = w->nckpt - 1; kseg >= 0; --kseg) {
    const int s0 = kseg * w->every;
    const int s1 = (s0 + w->every < w->nsteps) ? s0 + w->every : w->nsteps;
    // states of the segment
    MX_CUDA_TRY(cudaMemcpyAsync(w->seg, w->ckpt + (long)kseg * nc, bytes, cudaMemcpyDeviceToDevice, st));
    for (int s = s0; s < s1; ++s) {
      float4* nxt = w->seg + (long)(s - s0 + 1) * nc;
      MX_CUDA_TRY(cudaMemcpyAsync(nxt, w->seg + (long)(s - s0) * nc, bytes, cudaMemcpyDeviceToDevice, st));
      MX_TRY(rk4_step_direct(ctx, nxt, dt, st));
    }
    for (int s = s1 - 1; s >= s0; --s) {
      float4* m = w->seg + (long)(s - s0) * nc;
      float4* mnew = m + nc;
      // stage states m1, m2, m3 and the demag field of each stage state
      const float4* states[4] = {m, st1, st2, st3};
      float4* outs[3] = {st1, st2, st3};
      const int modes[3] = {LM_RK4_S0, LM_RK4_S1, LM_RK4_S2};
      for (int q = 0; q < 4; ++q) {
        if (demag) MX_TRY(demag_field(ctx, states[q], w->hd4 + q * nc, st));
        if (q < 3) {
          StageIO io{states[q], demag ? w->hd4 + q * nc : nullptr, m, ctx->acc, outs[q], dt, MX_TERM_ALL};
          MX_TRY(local_stage(ctx, modes[q], io, st));
        }
      }
      adj_begin_kernel<<<nb, 256, 0, st>>>(mnew, w->lam_acc, w->lam_u4, w->lam_k, nc, dt);
      MX_TRY(launch_check("adj_begin_kernel"));
      for (int q = 3; q >= 0; --q) {
        const float4* sm_ = states[q];
        if (dmi)
          adj_prep_kernel<true><<<grid, block, 0, st>>>(sm_, w->hd4 + q * nc, w->lam_k, g, c, w->wbuf, w->gm);
        else
          adj_prep_kernel<false><<<grid, block, 0, st>>>(sm_, w->hd4 + q * nc, w->lam_k, g, c, w->wbuf, w->gm);
        MX_TRY(launch_check("adj_prep_kernel"));
        if (demag) MX_TRY(demag_field(ctx, w->wbuf, w->hdw, st));
        const bool want_ms = grad_ms != nullptr;
        switch (q) {
          case 3: launch_finish<3>(dmi, grid, block, st, w, sm_, g, c, dt, want_ms); break;
          case 2: launch_finish<2>(dmi, grid, block, st, w, sm_, g, c, dt, want_ms); break;
          case 1: launch_finish<1>(dmi, grid, block, st, w, sm_, g, c, dt, want_ms); break;
          default: launch_finish<0>(dmi, grid, block, st, w, sm_, g, c, dt, want_ms); break;
        }
        MX_TRY(launch_check("adj_finish_kernel"));
      }
    }
  }
  adj_end_kernel<<<nb, 256, 0, st>>>(w->raw, w->lam_acc, grad_m0, w->dms, grad_ms, nc);
  return launch_check("adj_end_kernel");
}

}  // namespace mx
