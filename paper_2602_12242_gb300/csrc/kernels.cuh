// Declarations shared by the translation units of libmx.
#pragma once

#include "common.cuh"

namespace mx {

// Kernel identifiers for mx_profile_step.
enum KernelId {
  KID_X_FWD = 0,
  KID_YZ,
  KID_Y_FWD,
  KID_Z_MUL,
  KID_Y_INV,
  KID_X_INV,
  KID_LOCAL,
  KID_NORMALIZE,
  KID_COPY,
  KID_MRI_SLOW,
  KID_MRI_FAST,
  KID_X_INV_LOCAL,
  KID_COUNT
};
const char* kernel_name(int id);

// Records a CUDA event pair around the launches in its scope when the context
// is being profiled; does nothing otherwise.
struct ProfScope {
  mx_ctx* ctx;
  int id;
  cudaStream_t st;
  ProfScope(mx_ctx* c, int i, cudaStream_t s);
  ~ProfScope();
};

// demag.cu
mx_status demag_setup(mx_ctx* ctx);
mx_status demag_field(mx_ctx* ctx, const float4* m, float4* hd, cudaStream_t st);

// demag_fast.cu
mx_status fast_setup(mx_ctx* ctx);
// y transform, tensor multiply and inverse y of a one-z-plane spectrum (Pz == 1), in place on w1.
mx_status yz2d_pass(mx_ctx* ctx, cudaStream_t st);
mx_status fast_x_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st);

// demag_plane.cu
mx_status plane_setup(mx_ctx* ctx);
mx_status plane_field(mx_ctx* ctx, const float4* m, float4* hd, cudaStream_t st);
// One RK4 or Euler stage on the plane path with the inverse x pass fused into
// the local stage (ctx->xlocal): the forward x pass of io.m, the y/z pass,
// then H_demag, the local fields, the LLG right-hand side and the update of
// `mode` in one kernel (io.hd is not used).
struct StageIO;
mx_status plane_stage_xlocal(mx_ctx* ctx, int mode, const StageIO& io, cudaStream_t st);
// The y/z passes of demag_field alone (w1 in place, after the forward x pass).
mx_status demag_yz(mx_ctx* ctx, cudaStream_t st);
// One RK4 stage's row kernel on grids with ctx->xrow (demag_fast.cu): the
// inverse x pass of w1, the local stage of `mode` (with hd_out, the demag
// field of io.m is also written there), and with xf_next the forward x pass
// of io.out into w1 for the next stage.
mx_status fast_row_stage(mx_ctx* ctx, int mode, const StageIO& io, bool xf_next, float4* hd_out, cudaStream_t st);
// Whether RK4 steps of this context run as y/z passes plus row kernels (api.cu).
bool row_steps(const mx_ctx* ctx, int method);
mx_status plane_spectrum_out(mx_ctx* ctx, float* out, cudaStream_t st);

// demag_quad.cu: the four-CTA y/z plane kernel (setup: check the grid fits and
// set its attributes; otherwise launch it on w1 -> w2)
mx_status quad_pass(mx_ctx* ctx, cudaStream_t st, bool setup);

// cnn.cu
mx_status cnn_demag(struct mx_cnn* n, const float4* m, float4* h, cudaStream_t st);
bool cnn_matches(const struct mx_cnn* n, const Grid& g);
// Adam with L2-coupled weight decay (beta 0.9 / 0.999, eps 1e-8), step t >= 1.
mx_status adam_update(float* p, const float* g, float* m, float* v, long n, double lr, double wd, int t,
                      cudaStream_t st);

// fno.cu
mx_status fno_demag(struct ::mx_fno* n, const float4* m, float4* h, cudaStream_t st);
bool fno_matches(const struct ::mx_fno* n, const Grid& g);

// dftgemm.cu
mx_status dft_gemm_setup(mx_ctx* ctx);
mx_status dft_x_pass(mx_ctx* ctx, const float4* m, float4* hd, bool inverse, cudaStream_t st, bool setup);

// newell.cu
mx_status build_demag_kernel(mx_ctx* ctx, cudaStream_t st);

// adjoint.cu
mx_status adjoint_reserve(mx_ctx* ctx, int nsteps, int every);
void adjoint_free(mx_ctx* ctx);
// drop the adjoint's captured graphs (material maps, bias or profiling changed)
void adjoint_invalidate_graphs(mx_ctx* ctx);
mx_status adjoint_forward(mx_ctx* ctx, const float4* m0_raw, float4* m_final, double dt, cudaStream_t st);
mx_status adjoint_backward(mx_ctx* ctx, const float4* lam_final, float4* grad_m0, float* grad_ms, cudaStream_t st);
bool adjoint_recorded(const mx_ctx* ctx);

// api.cu
// With row kernels (row_steps), `lead` runs the forward x pass of m first
// (else w1 must hold it) and `tail` leaves that of the new m in w1.
mx_status rk4_step_direct(mx_ctx* ctx, float4* m, double dt, cudaStream_t st, bool lead = true, bool tail = false);

// local.cu
enum LocalMode { LM_HEFF = 0, LM_RHS, LM_RK4_S0, LM_RK4_S1, LM_RK4_S2, LM_RK4_S3, LM_EULER };
struct StageIO {
  const float4* m;    // field the stencil and LLG act on
  const float4* hd;   // demag field (null: no demag term)
  const float4* m0;   // step start (RK stages 1..3)
  float4* acc;        // RK accumulator
  float4* out;        // H_eff, dm/dt, next stage input or the new m
  float dt;
  int terms;          // MX_TERM_* mask (LM_HEFF only)
};
LocalCoef local_coef(const mx_ctx* ctx);
// the same coefficients from parameters and caller-owned maps (any may be null)
LocalCoef local_coef_from(const mx_params& p, const float* ms_map, const float* ku_map, const float4* axis_map);
mx_status local_stage(mx_ctx* ctx, int mode, const StageIO& io, cudaStream_t st);
mx_status normalize_field(mx_ctx* ctx, float4* m, cudaStream_t st);
mx_status copy_field(mx_ctx* ctx, float4* dst, const float4* src, cudaStream_t st);
// Reads and clears a conv net's device status flag (cnn.cu; synchronises st).
mx_status cnn_take_flag(struct ::mx_cnn* n, cudaStream_t st, int* flag_out);

// One explicit-explicit MRI step (mri.cu); mri_reserve allocates its slow
// right-hand sides (call before a graph capture).
mx_status mri_step(mx_ctx* ctx, float4* m, double dt, cudaStream_t st);
mx_status mri_reserve(mx_ctx* ctx);
mx_status energy_terms(mx_ctx* ctx, const float4* m, const float4* hd, double* e_dev, cudaStream_t st);
mx_status exchange_energy_central(mx_ctx* ctx, const float4* m, double* e_dev, cudaStream_t st);

}  // namespace mx
