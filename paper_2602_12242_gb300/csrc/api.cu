// C ABI of libmx (declared in include/mx.h): context lifetime, argument
// checks, the stage sequence of one time step, CUDA-graph replay, energies
// and per-kernel timing.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace mx {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

static const char* kNames[KID_COUNT] = {"x_fwd",     "yz_fused", "y_fwd",    "z_mul",    "y_inv",
                                        "x_inv",     "local_stage", "normalize", "copy", "mri_slow",
                                        "mri_fast", "x_inv_local"};
const char* kernel_name(int id) { return (id >= 0 && id < KID_COUNT) ? kNames[id] : ""; }

// ---------------------------------------------------------------------------
// Profiler: an event pair per launch, harvested when the pool runs out.
// ---------------------------------------------------------------------------
struct Profiler {
  std::vector<cudaEvent_t> ev;
  std::vector<int> ids;
  int used = 0;
  double ms[KID_COUNT] = {0};
  int count[KID_COUNT] = {0};
  cudaError_t err = cudaSuccess;
  cudaStream_t last = nullptr;
  void harvest() {
    if (used == 0) return;
    cudaError_t e = cudaEventSynchronize(ev[2 * used - 1]);
    if (e != cudaSuccess) err = e;
    for (int q = 0; q < used; ++q) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]) == cudaSuccess) {
        ms[ids[q]] += t;
        count[ids[q]] += 1;
      }
    }
    used = 0;
  }
};

ProfScope::ProfScope(mx_ctx* c, int i, cudaStream_t s) : ctx(c), id(i), st(s) {
  Profiler* p = ctx->prof;
  if (!p) return;
  if (2 * (p->used + 1) > (int)p->ev.size()) p->harvest();
  p->ids[p->used] = id;
  cudaEventRecord(p->ev[2 * p->used], st);
}
ProfScope::~ProfScope() {
  Profiler* p = ctx->prof;
  if (!p) return;
  cudaEventRecord(p->ev[2 * p->used + 1], st);
  p->used += 1;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int pad_len(int n) {
  if (n <= 1) return 1;
  int p = 1;
  while (p < 2 * n - 1) p <<= 1;
  return p;
}

static mx_status check_vec_ptr(const void* p, const char* what) {
  if (!p) {
    set_error(std::string(what) + " is NULL");
    return MX_ERR_INVALID_ARG;
  }
  if (((uintptr_t)p) & 15) {
    set_error(std::string(what) + " is not 16-byte aligned");
    return MX_ERR_INVALID_ARG;
  }
  return MX_OK;
}

static mx_status check_ctx(const mx_ctx* ctx) {
  if (!ctx) {
    set_error("context is NULL");
    return MX_ERR_INVALID_ARG;
  }
  return MX_OK;
}

static void invalidate_graph(mx_ctx* ctx) {
  adjoint_invalidate_graphs(ctx);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  ctx->graph = nullptr;
  ctx->graph_m = nullptr;
  ctx->graph_method = -1;
}

static std::vector<float2> twiddles32(int L) {
  std::vector<float2> t(L);
  for (int q = 0; q < L; ++q) {
    const double a = -2.0 * kPi * q / L;
    t[q] = make_float2((float)cos(a), (float)sin(a));
  }
  return t;
}

// Whether an RK4 step runs as y/z passes plus one row kernel per stage.
bool row_steps(const mx_ctx* ctx, int method) {
  return method == MX_RK4 && ctx->p.demag && ctx->xrow && !ctx->plane && !ctx->surrogate && !ctx->fno;
}

// The forward x pass of m into w1, which the first row-kernel step of a
// sequence needs (each later step finds it left by the step before).
static mx_status lead_x_pass(mx_ctx* ctx, const float4* m, cudaStream_t st) {
  ProfScope ps(ctx, KID_X_FWD, st);
  return fast_x_pass(ctx, m, nullptr, false, st);
}

// One time step on stream st.  m is the caller's field (step start, updated
// in place).  With row kernels (row_steps), `lead` runs the forward x pass of
// m first (else w1 must already hold it) and `tail` has the last stage leave
// the forward x pass of the new m in w1 for a following step.
static mx_status enqueue_step(mx_ctx* ctx, float4* m, double dt, int method, cudaStream_t st, bool lead = true,
                              bool tail = false) {
  if (method == MX_MRI) return mri_step(ctx, m, dt, st);
  const bool demag = ctx->p.demag != 0;
  float4* hd = demag ? ctx->hd : nullptr;
  const bool xlocal = demag && ctx->xlocal;
  if (method == MX_EULER) {
    StageIO io{m, hd, m, ctx->acc, ctx->sa, (float)dt, MX_TERM_ALL};
    if (xlocal) {
      MX_TRY(plane_stage_xlocal(ctx, LM_EULER, io, st));
    } else {
      if (demag) MX_TRY(demag_field(ctx, m, hd, st));
      MX_TRY(local_stage(ctx, LM_EULER, io, st));
    }
    return copy_field(ctx, m, ctx->sa, st);
  }
  // RK4: m -> sa -> sb -> sa -> m
  const float4* in[4] = {m, ctx->sa, ctx->sb, ctx->sa};
  float4* out[4] = {ctx->sa, ctx->sb, ctx->sa, m};
  const int modes[4] = {LM_RK4_S0, LM_RK4_S1, LM_RK4_S2, LM_RK4_S3};
  if (row_steps(ctx, method)) {
    // few-row grids: per stage the y/z passes and one row kernel (inverse x,
    // local stage, the next stage's forward x)
    if (lead) MX_TRY(lead_x_pass(ctx, m, st));
    for (int s = 0; s < 4; ++s) {
      StageIO io{in[s], nullptr, m, ctx->acc, out[s], (float)dt, MX_TERM_ALL};
      MX_TRY(demag_yz(ctx, st));
      ProfScope ps(ctx, KID_X_INV_LOCAL, st);
      MX_TRY(fast_row_stage(ctx, modes[s], io, s < 3 || tail, nullptr, st));
    }
    return MX_OK;
  }
  for (int s = 0; s < 4; ++s) {
    StageIO io{in[s], hd, m, ctx->acc, out[s], (float)dt, MX_TERM_ALL};
    if (xlocal) {
      MX_TRY(plane_stage_xlocal(ctx, modes[s], io, st));
      continue;
    }
    if (demag) MX_TRY(demag_field(ctx, in[s], hd, st));
    MX_TRY(local_stage(ctx, modes[s], io, st));
  }
  return MX_OK;
}

mx_status rk4_step_direct(mx_ctx* ctx, float4* m, double dt, cudaStream_t st, bool lead, bool tail) {
  return enqueue_step(ctx, m, dt, MX_RK4, st, lead, tail);
}

// sums of |a - b|^2 and |b|^2 over the xyz of float4 records
__global__ void rel_l2_kernel(const float4* __restrict__ a, const float4* __restrict__ b, long n,
                              double* __restrict__ out) {
  double s0 = 0.0, s1 = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float4 x = a[i], y = b[i];
    const double dx = (double)x.x - y.x, dy = (double)x.y - y.y, dz = (double)x.z - y.z;
    s0 += dx * dx + dy * dy + dz * dz;
    s1 += (double)y.x * y.x + (double)y.y * y.y + (double)y.z * y.z;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], s0);
    atomicAdd(&out[1], s1);
  }
}

}  // namespace mx

using namespace mx;

extern "C" {

const char* mx_last_error(void) { return g_err.c_str(); }
const char* mx_version(void) { return "libmx 0.1 (sm_103a)"; }
const char* mx_kernel_slot(int q) { return kernel_name(q); }

const char* mx_kernel_name(const mx_ctx* ctx, int q) {
  if (!ctx || q < 0 || q >= KID_COUNT) return "";
  const bool dft = ctx->p.fft_mode == MX_FFT_SPLIT_BF16;
  switch (q) {
    case KID_X_FWD:
      if (ctx->plane) return dft ? "xfk_dft_kernel" : "xfk_kernel";
      return ctx->fast_x ? "xf_kernel" : "x_fwd_kernel";
    case KID_X_INV:
      if (ctx->plane) return dft ? "xik_dft_kernel" : "xik_kernel";
      return ctx->fast_x ? "xi_kernel" : "x_inv_kernel";
    case KID_YZ:
      if (ctx->plane) return ctx->quad ? "yzq_kernel" : "yzh_kernel";
      return ctx->yz2d ? "yz2d_kernel" : "yz_fused_kernel";
    case KID_Y_FWD: return "y_fwd_kernel";
    case KID_Z_MUL: return "z_mul_kernel";
    case KID_Y_INV: return "y_inv_kernel";
    case KID_LOCAL: return "local_kernel";
    case KID_NORMALIZE: return "normalize_kernel";
    case KID_COPY: return "copy_kernel";
    case KID_MRI_SLOW: return "mri_slow_kernel";
    case KID_MRI_FAST: return "mri_fast_kernel";
    case KID_X_INV_LOCAL: return ctx->xlocal ? "xil_kernel" : (ctx->xrow && !ctx->plane ? "xr_kernel" : "");
    default: return "";
  }
}

mx_status mx_create(mx_ctx** out, const mx_params* p) {
  clear_error();
  if (!out || !p) {
    set_error("mx_create: NULL argument");
    return MX_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 2048 || p->ny > 2048 || p->nz > 2048) {
    set_error("mx_create: grid must be 1..2048 cells per axis");
    return MX_ERR_UNSUPPORTED;
  }
  if (!(p->mri_fast_ratio >= 0.0 && p->mri_fast_ratio <= 1.0)) {
    set_error("mx_create: mri_fast_ratio must be in [0, 1] (0: 0.1)");
    return MX_ERR_INVALID_ARG;
  }
  if (!(p->dx > 0 && p->dy > 0 && p->dz > 0) || !(p->Ms > 0) || !(p->A >= 0) || !(p->alpha >= 0) ||
      !(p->gamma > 0) || !(p->Ku == p->Ku) || !(p->D == p->D)) {
    set_error("mx_create: need dx, dy, dz, Ms, gamma > 0 and A, alpha >= 0");
    return MX_ERR_INVALID_ARG;
  }
  if (p->demag_path < MX_DEMAG_AUTO || p->demag_path > MX_DEMAG_PLANE_XLOCAL) {
    set_error("mx_create: demag_path must be MX_DEMAG_AUTO, MX_DEMAG_GENERIC, MX_DEMAG_PLANE, MX_DEMAG_PLANE_PAIR "
              "or MX_DEMAG_PLANE_XLOCAL");
    return MX_ERR_INVALID_ARG;
  }
  if (p->fft_mode != MX_FFT_FP32 && p->fft_mode != MX_FFT_SPLIT_BF16) {
    set_error("mx_create: fft_mode must be MX_FFT_FP32 or MX_FFT_SPLIT_BF16");
    return MX_ERR_INVALID_ARG;
  }
  if (p->dmi_interfacial && p->D != 0.0 && !(p->A > 0)) {
    set_error("mx_create: DMI boundary condition needs A > 0");
    return MX_ERR_INVALID_ARG;
  }
  mx_ctx* ctx = new mx_ctx();
  ctx->p = *p;
  cudaGetDevice(&ctx->device);
  Grid& g = ctx->g;
  g.nx = p->nx; g.ny = p->ny; g.nz = p->nz;
  g.Px = pad_len(p->nx); g.Py = pad_len(p->ny); g.Pz = pad_len(p->nz);
  if (g.Px > kMaxPad || g.Py > kMaxPad || g.Pz > kMaxPad || !is_pow2(g.Px) || !is_pow2(g.Py) || !is_pow2(g.Pz)) {
    delete ctx;
    set_error("mx_create: padded grid exceeds 4096 per axis");
    return MX_ERR_UNSUPPORTED;
  }
  g.Hx = g.Px > 1 ? g.Px / 2 + 1 : 1;
  g.Oy = g.Py / 2 + 1;
  g.Oz = g.Pz / 2 + 1;
  g.ncell = (long)g.nx * g.ny * g.nz;
  g.oct4 = 0;
  const long nc = g.ncell;
  bool ok = true;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (ok && cudaMalloc(ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  };
  const long no = (long)g.Hx * g.Oy * g.Oz;
  alloc((void**)&ctx->nhat, sizeof(float) * (6 * no > plane_octant_size(g) ? 6 * no : plane_octant_size(g)));
  alloc((void**)&ctx->w1, sizeof(float2) * 3 * (long)g.nz * g.ny * g.Hx);
  alloc((void**)&ctx->tw_x, sizeof(float2) * g.Px);
  alloc((void**)&ctx->tw_m, sizeof(float2) * (g.Px > 1 ? g.Px / 2 : 1));
  alloc((void**)&ctx->tw_y, sizeof(float2) * g.Py);
  alloc((void**)&ctx->tw_yh, sizeof(float2) * (g.Py > 1 ? g.Py / 2 : 1));
  alloc((void**)&ctx->tw_z, sizeof(float2) * g.Pz);
  alloc((void**)&ctx->hd, sizeof(float4) * nc);
  alloc((void**)&ctx->sa, sizeof(float4) * nc);
  alloc((void**)&ctx->sb, sizeof(float4) * nc);
  alloc((void**)&ctx->acc, sizeof(float4) * nc);
  alloc((void**)&ctx->flag, sizeof(int));
  alloc((void**)&ctx->ered, sizeof(double) * 5);
  alloc((void**)&ctx->red2, sizeof(double) * 2);
  mx_status st = MX_OK;
  if (ok) st = demag_setup(ctx);
  if (ok && st == MX_OK) st = fast_setup(ctx);
  if (ok && st == MX_OK) st = plane_setup(ctx);
  if (ok && st == MX_OK && !ctx->fused_yz) alloc((void**)&ctx->w2, sizeof(float2) * 3 * (long)g.nz * g.Py * g.Hx);
  if (!ok) {
    mx_destroy(ctx);
    set_error("mx_create: device allocation failed");
    return MX_ERR_OOM;
  }
  if (st != MX_OK) {
    mx_destroy(ctx);
    return st;
  }
  std::vector<float2> tx = twiddles32(g.Px), ty = twiddles32(g.Py), tz = twiddles32(g.Pz);
  const int Mx = g.Px > 1 ? g.Px / 2 : 1;
  std::vector<float2> tm = twiddles32(Mx);
  const int Hy = g.Py > 1 ? g.Py / 2 : 1;
  std::vector<float2> th = twiddles32(Hy);
  if (cudaMemcpy(ctx->tw_x, tx.data(), sizeof(float2) * g.Px, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->tw_m, tm.data(), sizeof(float2) * Mx, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->tw_yh, th.data(), sizeof(float2) * Hy, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->tw_y, ty.data(), sizeof(float2) * g.Py, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->tw_z, tz.data(), sizeof(float2) * g.Pz, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(ctx->flag, 0, sizeof(int)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error(std::string("mx_create: ") + cudaGetErrorString(cudaGetLastError()));
    mx_destroy(ctx);
    return MX_ERR_CUDA;
  }
  *out = ctx;
  return MX_OK;
}

mx_status mx_destroy(mx_ctx* ctx) {
  if (!ctx) return MX_OK;
  invalidate_graph(ctx);
  adjoint_free(ctx);
  void* ptrs[] = {ctx->ms_map, ctx->ku_map, ctx->axis_map, ctx->nhat, ctx->w1, ctx->w2, ctx->tw_x, ctx->tw_m, ctx->tw_mk, ctx->tw_yh, ctx->tw_y,
                  ctx->tw_z, ctx->t_real, ctx->hd, ctx->sa, ctx->sb, ctx->acc, ctx->flag, ctx->ered, ctx->red2, ctx->dft_a, ctx->mri_f};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
  return MX_OK;
}

mx_status mx_inject_wait_timeout(mx_ctx* ctx, int on) {
  MX_TRY(check_ctx(ctx));
  if (on && !(ctx->plane && !ctx->quad && (ctx->g.ny & 1) == 0 && !ctx->surrogate && !ctx->fno)) {
    set_error("mx_inject_wait_timeout: needs the two-CTA plane kernel with bulk copies (MX_DEMAG_PLANE_PAIR, even ny)");
    return MX_ERR_UNSUPPORTED;
  }
  invalidate_graph(ctx);
  ctx->inject_wait_timeout = on != 0;
  return MX_OK;
}

mx_status mx_padded_dims(const mx_ctx* ctx, int out[3]) {
  MX_TRY(check_ctx(ctx));
  if (!out) {
    set_error("mx_padded_dims: NULL out");
    return MX_ERR_INVALID_ARG;
  }
  out[0] = ctx->g.Px;
  out[1] = ctx->g.Py;
  out[2] = ctx->g.Pz;
  return MX_OK;
}

mx_status mx_set_ms_map(mx_ctx* ctx, const float* ms_dev, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  invalidate_graph(ctx);
  if (!ms_dev) {
    if (ctx->ms_map) cudaFree(ctx->ms_map);
    ctx->ms_map = nullptr;
    return MX_OK;
  }
  if (!ctx->ms_map && cudaMalloc(&ctx->ms_map, sizeof(float) * ctx->g.ncell) != cudaSuccess) {
    cudaGetLastError();
    ctx->ms_map = nullptr;
    set_error("mx_set_ms_map: allocation failed");
    return MX_ERR_OOM;
  }
  MX_CUDA_TRY(cudaMemcpyAsync(ctx->ms_map, ms_dev, sizeof(float) * ctx->g.ncell, cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return MX_OK;
}

mx_status mx_set_anis_map(mx_ctx* ctx, const float* ku_dev, const float* axis_dev, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  invalidate_graph(ctx);
  cudaStream_t st = (cudaStream_t)stream;
  const long nc = ctx->g.ncell;
  if (ku_dev) {
    if (!ctx->ku_map && cudaMalloc(&ctx->ku_map, sizeof(float) * nc) != cudaSuccess) {
      cudaGetLastError();
      ctx->ku_map = nullptr;
      set_error("mx_set_anis_map: allocation failed");
      return MX_ERR_OOM;
    }
    MX_CUDA_TRY(cudaMemcpyAsync(ctx->ku_map, ku_dev, sizeof(float) * nc, cudaMemcpyDeviceToDevice, st));
  } else if (ctx->ku_map) {
    cudaFree(ctx->ku_map);
    ctx->ku_map = nullptr;
  }
  if (axis_dev) {
    MX_TRY(check_vec_ptr(axis_dev, "mx_set_anis_map: axis"));
    if (!ctx->axis_map && cudaMalloc(&ctx->axis_map, sizeof(float4) * nc) != cudaSuccess) {
      cudaGetLastError();
      ctx->axis_map = nullptr;
      set_error("mx_set_anis_map: allocation failed");
      return MX_ERR_OOM;
    }
    MX_CUDA_TRY(cudaMemcpyAsync(ctx->axis_map, axis_dev, sizeof(float4) * nc, cudaMemcpyDeviceToDevice, st));
  } else if (ctx->axis_map) {
    cudaFree(ctx->axis_map);
    ctx->axis_map = nullptr;
  }
  return MX_OK;
}

mx_status mx_set_bias(mx_ctx* ctx, const double h[3]) {
  MX_TRY(check_ctx(ctx));
  if (!h) {
    set_error("mx_set_bias: NULL h");
    return MX_ERR_INVALID_ARG;
  }
  invalidate_graph(ctx);
  for (int q = 0; q < 3; ++q) ctx->p.h_bias[q] = h[q];
  return MX_OK;
}

mx_status mx_build_demag_kernel(mx_ctx* ctx, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  invalidate_graph(ctx);
  return build_demag_kernel(ctx, (cudaStream_t)stream);
}

mx_status mx_heff(mx_ctx* ctx, const float* m, float* h, int terms, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(m, "mx_heff: m"));
  MX_TRY(check_vec_ptr(h, "mx_heff: h"));
  if (m == h || (terms & ~MX_TERM_ALL)) {
    set_error("mx_heff: m and h overlap or bad term mask");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool demag = (terms & MX_TERM_DEMAG) != 0;
  if (demag && !ctx->built && !ctx->surrogate && !ctx->fno) {
    set_error("mx_heff: demag kernel not built");
    return MX_ERR_NOT_BUILT;
  }
  if (demag) MX_TRY(demag_field(ctx, (const float4*)m, ctx->hd, st));
  StageIO io{(const float4*)m, demag ? ctx->hd : nullptr, nullptr, nullptr, (float4*)h, 0.f, terms};
  return local_stage(ctx, LM_HEFF, io, st);
}

mx_status mx_llg_rhs(mx_ctx* ctx, const float* m, float* dmdt, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(m, "mx_llg_rhs: m"));
  MX_TRY(check_vec_ptr(dmdt, "mx_llg_rhs: dmdt"));
  if (m == dmdt) {
    set_error("mx_llg_rhs: m and dmdt overlap");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool demag = ctx->p.demag != 0;
  if (demag && !ctx->built && !ctx->surrogate && !ctx->fno) {
    set_error("mx_llg_rhs: demag kernel not built");
    return MX_ERR_NOT_BUILT;
  }
  if (demag) MX_TRY(demag_field(ctx, (const float4*)m, ctx->hd, st));
  StageIO io{(const float4*)m, demag ? ctx->hd : nullptr, nullptr, nullptr, (float4*)dmdt, 0.f, MX_TERM_ALL};
  return local_stage(ctx, LM_RHS, io, st);
}

static mx_status check_step_args(mx_ctx* ctx, const float* m, int nsteps, double dt, int method) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(m, "mx_rk_step: m"));
  if (nsteps < 0 || !(dt > 0) || !isfinite(dt) || (method != MX_RK4 && method != MX_EULER && method != MX_MRI)) {
    set_error("mx_rk_step: need nsteps >= 0, finite dt > 0, method MX_RK4, MX_EULER or MX_MRI");
    return MX_ERR_INVALID_ARG;
  }
  if (ctx->p.demag && !ctx->built && !ctx->surrogate && !ctx->fno) {
    set_error("mx_rk_step: demag kernel not built");
    return MX_ERR_NOT_BUILT;
  }
  return MX_OK;
}

mx_status mx_rk_step(mx_ctx* ctx, float* m, int nsteps, double dt, int method, mx_stream_t stream) {
  MX_TRY(check_step_args(ctx, m, nsteps, dt, method));
  cudaStream_t st = (cudaStream_t)stream;
  if (nsteps == 0) return MX_OK;
  if (method == MX_MRI) MX_TRY(mri_reserve(ctx));
  MX_TRY(normalize_field(ctx, (float4*)m, st));
  if (!ctx->graph || ctx->graph_m != m || ctx->graph_dt != dt || ctx->graph_method != method) {
    invalidate_graph(ctx);
    cudaGraph_t graph = nullptr;
    MX_CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    // with row kernels the graph step starts from w1 and leaves it for the next
    mx_status s = enqueue_step(ctx, (float4*)m, dt, method, ctx->cap_stream, false, true);
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (s != MX_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) {
      set_error(std::string("mx_rk_step: capture failed: ") + cudaGetErrorString(e));
      return MX_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&ctx->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->graph = nullptr;
      set_error(std::string("mx_rk_step: instantiate failed: ") + cudaGetErrorString(e));
      return MX_ERR_CUDA;
    }
    ctx->graph_m = m;
    ctx->graph_dt = dt;
    ctx->graph_method = method;
  }
  if (row_steps(ctx, method)) MX_TRY(lead_x_pass(ctx, (const float4*)m, st));
  for (int s = 0; s < nsteps; ++s) MX_CUDA_TRY(cudaGraphLaunch(ctx->graph, st));
  return MX_OK;
}

mx_status mx_profile_step(mx_ctx* ctx, float* m, int nsteps, double dt, int method, mx_stream_t stream,
                          double* ms_total, int* launches, int max_kernels, int* n_kernels) {
  MX_TRY(check_step_args(ctx, m, nsteps, dt, method));
  if (!ms_total || !launches || !n_kernels || max_kernels < 1) {
    set_error("mx_profile_step: NULL output");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  Profiler prof;
  const int pool = 4096;
  prof.ev.resize(2 * pool);
  prof.ids.resize(pool);
  for (auto& e : prof.ev) MX_CUDA_TRY(cudaEventCreate(&e));
  ctx->prof = &prof;
  mx_status s = normalize_field(ctx, (float4*)m, st);
  for (int q = 0; q < nsteps && s == MX_OK; ++q) s = enqueue_step(ctx, (float4*)m, dt, method, st, q == 0, true);
  prof.harvest();
  ctx->prof = nullptr;
  for (auto& e : prof.ev) cudaEventDestroy(e);
  if (s != MX_OK) return s;
  if (prof.err != cudaSuccess) {
    set_error(std::string("mx_profile_step: ") + cudaGetErrorString(prof.err));
    return MX_ERR_CUDA;
  }
  const int n = KID_COUNT < max_kernels ? KID_COUNT : max_kernels;
  for (int q = 0; q < n; ++q) {
    ms_total[q] = prof.ms[q];
    launches[q] = prof.count[q];
  }
  *n_kernels = n;
  return MX_OK;
}

mx_status mx_energy(mx_ctx* ctx, const float* m, double e_out[5], mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(m, "mx_energy: m"));
  if (!e_out) {
    set_error("mx_energy: NULL e_out");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool demag = ctx->p.demag != 0;
  if (demag && !ctx->built && !ctx->surrogate && !ctx->fno) {
    set_error("mx_energy: demag kernel not built");
    return MX_ERR_NOT_BUILT;
  }
  if (demag) MX_TRY(demag_field(ctx, (const float4*)m, ctx->hd, st));
  MX_CUDA_TRY(cudaMemsetAsync(ctx->ered, 0, sizeof(double) * 5, st));
  MX_TRY(energy_terms(ctx, (const float4*)m, demag ? ctx->hd : nullptr, ctx->ered, st));
  MX_CUDA_TRY(cudaMemcpyAsync(e_out, ctx->ered, sizeof(double) * 5, cudaMemcpyDeviceToHost, st));
  MX_CUDA_TRY(cudaStreamSynchronize(st));
  return MX_OK;
}

mx_status mx_exchange_energy_central(mx_ctx* ctx, const float* m, double* e_out, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(m, "mx_exchange_energy_central: m"));
  if (!e_out) {
    set_error("mx_exchange_energy_central: NULL e_out");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MX_CUDA_TRY(cudaMemsetAsync(ctx->ered, 0, sizeof(double), st));
  MX_TRY(exchange_energy_central(ctx, (const float4*)m, ctx->ered, st));
  MX_CUDA_TRY(cudaMemcpyAsync(e_out, ctx->ered, sizeof(double), cudaMemcpyDeviceToHost, st));
  MX_CUDA_TRY(cudaStreamSynchronize(st));
  return MX_OK;
}

mx_status mx_sync(mx_ctx* ctx, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  cudaStream_t st = (cudaStream_t)stream;
  int flag = 0;
  MX_CUDA_TRY(cudaMemcpyAsync(&flag, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  MX_CUDA_TRY(cudaStreamSynchronize(st));
  if (ctx->surrogate) {
    int f = 0;
    MX_TRY(cnn_take_flag(ctx->surrogate, st, &f));
    flag |= f;
  }
  if (flag) {
    MX_CUDA_TRY(cudaMemsetAsync(ctx->flag, 0, sizeof(int), st));
    MX_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag & kFlagTimeout) {
      set_error("mx_sync: a bounded wait in a demag or surrogate kernel ran out");
      return MX_ERR_TIMEOUT;
    }
    set_error("mx_sync: a kernel produced a non-finite value");
    return MX_ERR_NONFINITE;
  }
  return MX_OK;
}

mx_status mx_demag_tensor_real(mx_ctx* ctx, double* out, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  if (!out) {
    set_error("mx_demag_tensor_real: NULL out");
    return MX_ERR_INVALID_ARG;
  }
  if (!ctx->built || !ctx->t_real) {
    set_error("mx_demag_tensor_real: demag kernel not built");
    return MX_ERR_NOT_BUILT;
  }
  MX_CUDA_TRY(cudaMemcpyAsync(out, ctx->t_real, sizeof(double) * 6 * ctx->g.ncell, cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return MX_OK;
}

mx_status mx_demag_spectrum(mx_ctx* ctx, float* out, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  if (!out) {
    set_error("mx_demag_spectrum: NULL out");
    return MX_ERR_INVALID_ARG;
  }
  if (!ctx->built) {
    set_error("mx_demag_spectrum: demag kernel not built");
    return MX_ERR_NOT_BUILT;
  }
  if (ctx->plane) return plane_spectrum_out(ctx, out, (cudaStream_t)stream);
  const long no = (long)ctx->g.Hx * ctx->g.Oy * ctx->g.Oz;
  MX_CUDA_TRY(cudaMemcpyAsync(out, ctx->nhat, sizeof(float) * 6 * no, cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return MX_OK;
}

mx_status mx_adjoint_reserve(mx_ctx* ctx, int nsteps, int checkpoint_every) {
  MX_TRY(check_ctx(ctx));
  return adjoint_reserve(ctx, nsteps, checkpoint_every);
}

mx_status mx_rk_forward_record(mx_ctx* ctx, const float* m0_raw, float* m_final, double dt, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(m0_raw, "mx_rk_forward_record: m0_raw"));
  MX_TRY(check_vec_ptr(m_final, "mx_rk_forward_record: m_final"));
  if (!ctx->adj) {
    set_error("mx_rk_forward_record: call mx_adjoint_reserve first");
    return MX_ERR_INVALID_ARG;
  }
  if (!(dt > 0) || !isfinite(dt)) {
    set_error("mx_rk_forward_record: need finite dt > 0");
    return MX_ERR_INVALID_ARG;
  }
  if (ctx->p.demag && !ctx->built) {
    set_error("mx_rk_forward_record: demag kernel not built");
    return MX_ERR_NOT_BUILT;
  }
  if (ctx->p.demag && (ctx->surrogate || ctx->fno)) {
    set_error("mx_rk_forward_record: the adjoint needs the FFT demag (a learned demag backend is set)");
    return MX_ERR_UNSUPPORTED;
  }
  return adjoint_forward(ctx, (const float4*)m0_raw, (float4*)m_final, dt, (cudaStream_t)stream);
}

mx_status mx_rk_backward(mx_ctx* ctx, const float* lam_final, float* grad_m0, float* grad_ms, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(lam_final, "mx_rk_backward: lam_final"));
  MX_TRY(check_vec_ptr(grad_m0, "mx_rk_backward: grad_m0"));
  if (!adjoint_recorded(ctx)) {
    set_error("mx_rk_backward: no recorded forward run (mx_rk_forward_record)");
    return MX_ERR_INVALID_ARG;
  }
  return adjoint_backward(ctx, (const float4*)lam_final, (float4*)grad_m0, grad_ms, (cudaStream_t)stream);
}

mx_status mx_set_demag_surrogate(mx_ctx* ctx, mx_cnn* net) {
  MX_TRY(check_ctx(ctx));
  if (net && !cnn_matches(net, ctx->g)) {
    set_error("mx_set_demag_surrogate: the network's grid differs from the context's");
    return MX_ERR_INVALID_ARG;
  }
  invalidate_graph(ctx);
  ctx->surrogate = net;
  if (net) ctx->fno = nullptr;
  return MX_OK;
}

mx_status mx_set_demag_fno(mx_ctx* ctx, mx_fno* net) {
  MX_TRY(check_ctx(ctx));
  if (net && !fno_matches(net, ctx->g)) {
    set_error("mx_set_demag_fno: the network's grid differs from the context's (or nz != 1)");
    return MX_ERR_INVALID_ARG;
  }
  invalidate_graph(ctx);
  ctx->fno = net;
  if (net) ctx->surrogate = nullptr;
  return MX_OK;
}

mx_status mx_rel_l2(mx_ctx* ctx, const float* a, const float* b, double* out, mx_stream_t stream) {
  MX_TRY(check_ctx(ctx));
  MX_TRY(check_vec_ptr(a, "mx_rel_l2: a"));
  MX_TRY(check_vec_ptr(b, "mx_rel_l2: b"));
  if (!out) {
    set_error("mx_rel_l2: NULL out");
    return MX_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  MX_CUDA_TRY(cudaMemsetAsync(ctx->red2, 0, sizeof(double) * 2, st));
  rel_l2_kernel<<<304, 256, 0, st>>>((const float4*)a, (const float4*)b, ctx->g.ncell, ctx->red2);
  MX_TRY(launch_check("rel_l2_kernel"));
  double h[2];
  MX_CUDA_TRY(cudaMemcpyAsync(h, ctx->red2, sizeof(h), cudaMemcpyDeviceToHost, st));
  MX_CUDA_TRY(cudaStreamSynchronize(st));
  *out = h[1] > 0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
  return MX_OK;
}

}  // extern "C"
