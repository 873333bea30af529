/*
 * mx.h -- C ABI of libmx, a GB300 (sm_103a) implementation of the per-stage
 * hot path of the micromagnetics method of MagneX (arXiv 2602.12242):
 * effective field H_eff = H_bias + H_demag + H_ani + H_exch + H_DMI (Eq. 2),
 * the Landau-Lifshitz-Gilbert right-hand side (Eq. 1) and explicit time
 * stepping (classical RK4, forward Euler) with renormalisation |m| = 1
 * after every stage (Sec. II-B).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: nx * ny * nz cells of dx * dy * dz (metres), cell (i, j, k) at flat
 *   index c = i + nx * (j + ny * k).
 * Vector fields (m, H, dm/dt): DEVICE pointers to nx*ny*nz float4 records
 *   (x, y, z, unused), 16-byte aligned, FP32, SI units (H in A/m, dm/dt in
 *   1/s).  m is the unit magnetisation M / Ms.
 * Scalar maps: DEVICE pointers to nx*ny*nz floats.
 * Ownership: the caller owns every pointer it passes; the context owns its
 *   own workspaces (demag spectra, stage buffers) and frees them in
 *   mx_destroy.  No entry point keeps a caller pointer after it returns,
 *   except that a CUDA graph captured by mx_rk_step for a given m pointer is
 *   reused while the same pointer, dt and method come back.
 * Streams: every call that takes a stream enqueues its work on that stream
 *   and returns without waiting, unless its comment says it synchronises.
 *   A NULL stream is the legacy default stream.
 * Errors: every call returns an mx_status; MX_OK is 0.  On failure a message
 *   is kept per host thread and mx_last_error() returns it.  No call aborts,
 *   traps on the device or throws across the ABI.  A context is not
 *   thread-safe: one host thread at a time.
 * Device: a context lives on the CUDA device that is current when
 *   mx_create is called; every later call must run with that device current.
 */
#ifndef MX_H
#define MX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mx_stream_t; /* same type as cudaStream_t */
typedef struct mx_ctx mx_ctx;

typedef enum {
    MX_OK = 0,
    MX_ERR_INVALID_ARG = 1, /* bad size, NULL or misaligned pointer, bad flag   */
    MX_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has details) */
    MX_ERR_OOM = 3,         /* a workspace allocation failed                     */
    MX_ERR_NOT_BUILT = 4,   /* demag needed but mx_build_demag_kernel not run    */
    MX_ERR_NONFINITE = 5,   /* a NaN/Inf was produced (reported by mx_sync)      */
    MX_ERR_TIMEOUT = 6,     /* a bounded device wait gave up                     */
    MX_ERR_UNSUPPORTED = 7  /* size or option outside what this build supports   */
} mx_status;

/* Physical and numerical parameters (SI units).
 *   Ms      saturation magnetisation [A/m] (used where no Ms map is set)
 *   A       exchange stiffness [J/m]                  (Sec. II-A, exchange)
 *   Ku      uniaxial anisotropy constant [J/m^3]      (Sec. II-A, anisotropy)
 *   D       interfacial DMI constant [J/m^2]          (Sec. II-A, DMI)
 *   alpha   Gilbert damping                           (Eq. 1)
 *   gamma   gamma0 = mu0 |gamma| [m/(A s)], e.g. 2.211e5 (Eq. 1 with
 *           gamma = -1.759e11 C/kg)
 *   ku_axis easy axis (normalised internally) where no axis map is set
 *   h_bias  constant applied field [A/m]
 *   dmi_interfacial  1: interfacial DMI field and the chiral boundary
 *           condition dm/dx_k = -(D/2A)(e_z x e_k) x m (Sec. II-A, II-B);
 *           0: no DMI, Neumann boundaries
 *   precession 1: full LLG; 0: damping term only (relaxation)
 *   demag   1: include the demagnetising field
 *   demag_path  schedule of the demag convolution (same result up to FP32
 *           rounding): MX_DEMAG_AUTO picks the fastest that fits the grid;
 *           MX_DEMAG_GENERIC forces the size-generic separate passes;
 *           MX_DEMAG_PLANE forces the per-kx-plane kernels (the y/z kernel
 *           on a cluster of four CTAs per plane where it fits, else the one
 *           on two CTAs; MX_ERR_UNSUPPORTED at mx_create if the grid fits
 *           neither); MX_DEMAG_PLANE_PAIR forces the per-kx-plane path with
 *           the two-CTA y/z kernel; MX_DEMAG_PLANE_XLOCAL forces the
 *           per-kx-plane path and, in the RK4 and Euler steps of
 *           mx_rk_step, fuses the inverse x pass into the local stage
 *           (H_demag stays in shared memory; mx_heff, mx_llg_rhs and
 *           mx_energy still run the separate passes); needs fft_mode
 *           MX_FFT_FP32
 *   fft_mode  MX_FFT_FP32 (default): every FFT stage in FP32 on the CUDA
 *           cores; MX_FFT_SPLIT_BF16: the first radix-32 stage of the x
 *           transforms runs as a DFT-as-GEMM on the tensor cores with operands
 *           split into BF16 hi + lo parts (three products, FP32 accumulation),
 *           relative error near 2^-16 per stage; needs the per-kx-plane path
 *           and Px/2 in {512, 1024} (MX_ERR_UNSUPPORTED otherwise)
 *   mri_fast_ratio  fast step of MX_MRI as a fraction of dt (each slow
 *           stage interval takes ceil(interval / ratio) equal fast steps);
 *           0 selects 0.1 (Sec. III-C); must be in [0, 1]
 */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double Ms, A, Ku, D, alpha, gamma;
    double ku_axis[3];
    double h_bias[3];
    int dmi_interfacial;
    int precession;
    int demag;
    int demag_path;
    int fft_mode;
    double mri_fast_ratio;
} mx_params;

/* Demag convolution schedules for mx_params.demag_path. */
enum { MX_DEMAG_AUTO = 0, MX_DEMAG_GENERIC = 1, MX_DEMAG_PLANE = 2, MX_DEMAG_PLANE_PAIR = 3,
       MX_DEMAG_PLANE_XLOCAL = 4 };

/* Arithmetic of the demag FFT stages for mx_params.fft_mode. */
enum { MX_FFT_FP32 = 0, MX_FFT_SPLIT_BF16 = 1 };

/* Field terms, for mx_heff's term mask. */
enum {
    MX_TERM_DEMAG = 1,
    MX_TERM_EXCH = 2,
    MX_TERM_ANIS = 4,
    MX_TERM_DMI = 8,
    MX_TERM_ZEEMAN = 16,
    MX_TERM_ALL = 31
};

/* Integrators for mx_rk_step.
 *   MX_RK4    classical RK4 (Sec. III-B/C)
 *   MX_EULER  forward Euler (Sec. II-D, III-E)
 *   MX_MRI    explicit-explicit multirate infinitesimal step (Sec. II-C,
 *             III-C): fast part = the exchange-driven LLG right-hand side,
 *             slow part = demag + anisotropy + DMI + Zeeman; Knoth-Wolke
 *             3-stage third-order method on both levels; the slow stage
 *             differences (a_ij - a_{i-1,j}) f_slow(Y_j) / (c_i - c_{i-1})
 *             force the fast problem on each stage interval, integrated with
 *             fast steps of mri_fast_ratio x dt.  Three demag evaluations per
 *             step; every fast stage input and step result renormalised.
 *             Allocates 3 float4 fields at its first use (MX_ERR_OOM). */
enum { MX_RK4 = 0, MX_EULER = 1, MX_MRI = 2 };

/* Message of the last failed call on this host thread ("" if none). */
const char *mx_last_error(void);

/* Version string of this build. */
const char *mx_version(void);

/* Create a context for the grid and parameters in *p on the current device.
 * Allocates every workspace the hot path needs (no allocation happens
 * later).  Sizes: 1 <= nx, ny <= 2048, 1 <= nz <= 2048; the padded grid
 * (smallest power of two >= 2n-1 per axis of n > 1, else 1) must satisfy
 * Px, Py, Pz <= 4096.  Cell sizes, Ms, A must be > 0 (A may be 0 when D is
 * 0), alpha >= 0, gamma > 0.  *out receives the context, NULL on failure.
 * Errors: MX_ERR_INVALID_ARG, MX_ERR_UNSUPPORTED, MX_ERR_OOM, MX_ERR_CUDA. */
mx_status mx_create(mx_ctx **out, const mx_params *p);

/* Free every workspace and the context.  NULL is accepted. */
mx_status mx_destroy(mx_ctx *ctx);

/* Per-cell saturation magnetisation [A/m] (nx*ny*nz floats, all > 0), copied
 * into the context on `stream` (the caller may free its buffer after the
 * stream reaches this point).  NULL reverts to the scalar p->Ms.  The demag
 * field uses M = Ms_i m_i, the exchange/DMI/anisotropy fields divide by Ms_i. */
mx_status mx_set_ms_map(mx_ctx *ctx, const float *ms_dev, mx_stream_t stream);

/* Per-cell anisotropy: ku_dev nx*ny*nz floats [J/m^3] and axis_dev
 * nx*ny*nz float4 unit axes, copied into the context on `stream`.  Either
 * may be NULL to use the scalar value of p. */
mx_status mx_set_anis_map(mx_ctx *ctx, const float *ku_dev, const float *axis_dev,
                          mx_stream_t stream);

/* Replace the constant applied field [A/m] (host array of 3 doubles).
 * Takes effect for work enqueued after this call. */
mx_status mx_set_bias(mx_ctx *ctx, const double h[3]);

/* Build the demag kernel for this grid (Sec. II-B: the tensor of Newell et
 * al. on the zero-padded grid, then its FFT): real-space tensor in FP64
 * (closed form near, Gauss-Legendre quadrature of the defining integral
 * far), FP64 FFT, the real spectrum scaled by -1/(Px Py Pz) and stored in
 * FP32 as one octant per component.  Enqueued on `stream`; synchronises
 * `stream` before returning (it frees its FP64 scratch). */
mx_status mx_build_demag_kernel(mx_ctx *ctx, mx_stream_t stream);

/* Effective field (Eq. 2) of m, restricted to the terms in `terms`
 * (MX_TERM_* bits), written to h.  m and h must not overlap.
 * MX_ERR_NOT_BUILT if the demag term is asked for before the kernel is built. */
mx_status mx_heff(mx_ctx *ctx, const float *m, float *h, int terms, mx_stream_t stream);

/* dm/dt of the LLG equation (Eq. 1 in m-form,
 * dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)]) with the full
 * H_eff of the context.  m and dmdt must not overlap. */
mx_status mx_llg_rhs(mx_ctx *ctx, const float *m, float *dmdt, mx_stream_t stream);

/* Advance m in place by nsteps steps of size dt [s] with MX_RK4 (four
 * right-hand-side evaluations, every stage input and the result
 * renormalised) or MX_EULER.  m is normalised on entry.  The first call for
 * a given (m, dt, method, nsteps > 1) captures one step into a CUDA graph
 * that later calls replay.  Non-finite values set a device flag that
 * mx_sync reports. */
mx_status mx_rk_step(mx_ctx *ctx, float *m, int nsteps, double dt, int method,
                     mx_stream_t stream);

/* Energies [J] of m: e_out[0..4] = demag, exchange, anisotropy, DMI,
 * Zeeman (Sec. II-A energy densities: -mu0/2 Ms m.H_term for demag,
 * exchange and DMI; Ku [1 - (e_K.m)^2]; -mu0 Ms m.H_bias), accumulated in
 * FP64.  e_out is a HOST array.  Synchronises `stream`. */
mx_status mx_energy(mx_ctx *ctx, const float *m, double e_out[5], mx_stream_t stream);

/* Exchange energy [J] of m as the paper tabulates it (Sec. III-B, Table I):
 * V sum_cells A |grad m|^2 (the e_exch density of Sec. II-A) with every
 * derivative the second-order central difference (m_+ - m_-)/(2h) of
 * Sec. II-B, over the same ghost cells as the exchange field (Neumann, or the
 * chiral ghosts with DMI).  mx_energy's exchange term is the variational form
 * -mu0/2 Ms m.H_exch (face differences), whose gradient is the field; the two
 * differ at O(h^2).
 *   m      DEVICE float4 field, nx*ny*nz records (read only)
 *   e_out  HOST pointer to one double
 * Synchronises `stream`.  Errors: MX_ERR_INVALID_ARG for a NULL or misaligned
 * pointer. */
mx_status mx_exchange_energy_central(mx_ctx *ctx, const float *m, double *e_out, mx_stream_t stream);

/* Energies [J] like mx_energy, for callers that cannot allocate device
 * memory -- code that runs inside a device-memory budget owned by another
 * framework, or a latency-critical loop where an allocation's implicit
 * synchronisation would stall other work.  The paper has no counterpart; this
 * is a property of the library, not of the method.
 * No context, no cudaMalloc/cudaFree or allocating library call: the caller
 * passes every input and the output, and the only scratch (five FP64 partial
 * sums per 256-cell block) lives in a fixed-size array inside the library that
 * every GPU which loads the library holds until the process exits (640 KiB).
 *   p        HOST parameters (grid, cell, material; demag fields unused)
 *   m        DEVICE float4 field, nx*ny*nz records
 *   h_demag  DEVICE float4 demag field of m (e.g. from mx_heff with
 *            MX_TERM_DEMAG), or NULL: demag energy 0
 *   ms_map, ku_map  DEVICE nx*ny*nz floats or NULL (scalars of p)
 *   axis_map DEVICE float4 unit axes or NULL (p->ku_axis)
 *   e_out    DEVICE array of 5 doubles: demag, exchange, anisotropy, DMI,
 *            Zeeman, as in mx_energy
 * Limit: 1..2048 cells per axis and nx*ny*nz <= 4,194,304 cells; larger
 * grids return MX_ERR_UNSUPPORTED before any device call.  NULL m or e_out,
 * or a misaligned pointer (m, h_demag, axis_map 16 bytes; ms_map, ku_map 4;
 * e_out 8), returns MX_ERR_INVALID_ARG before any device call.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Enqueued on `stream`, no synchronisation.
 * Every call shares the one array, which keeps the last call's contents (each
 * call overwrites every row it reads), so calls that overlap on the GPU race:
 * order them on one stream or synchronise between them. */
mx_status mx_energy_noalloc(const mx_params *p, const float *m, const float *h_demag,
                            const float *ms_map, const float *ku_map, const float *axis_map,
                            double *e_out, mx_stream_t stream);

/* Synchronise `stream`; return MX_ERR_NONFINITE (and clear the flag) if any
 * kernel of this context produced a NaN or Inf since the last mx_sync, or
 * MX_ERR_TIMEOUT if a bounded wait (bulk copy of the demag kernel, tensor
 * cores of an attached surrogate) ran out (results are then invalid). */
mx_status mx_sync(mx_ctx *ctx, mx_stream_t stream);

/* Failure-detection test hook (no counterpart in the paper).  on != 0: every
 * later demag evaluation of this context arms the two-CTA plane kernel's
 * bulk-copy barrier for the plane's bytes but issues no copy, so the barrier
 * never completes; the kernel's bounded wait gives up after about one
 * second, the kernel runs to its end on stale shared memory (the demag field
 * is then invalid) and the next mx_sync returns MX_ERR_TIMEOUT.  No copy is
 * in flight at any time.  on == 0 restores normal operation; the context
 * stays usable.  MX_ERR_UNSUPPORTED unless the context runs the two-CTA
 * kernel with bulk copies (demag_path MX_DEMAG_PLANE_PAIR, even ny). */
mx_status mx_inject_wait_timeout(mx_ctx *ctx, int on);

/* Padded grid of this context: out[0..2] = Px, Py, Pz. */
mx_status mx_padded_dims(const mx_ctx *ctx, int out[3]);

/* The FP64 real-space tensor on the non-negative offsets (X = i dx,
 * Y = j dy, Z = k dz, 0 <= i < nx, 0 <= j < ny, 0 <= k < nz) as computed by
 * the build, written to the DEVICE array out (6 * nz * ny * nx doubles,
 * layout [c][k][j][i], c = xx, yy, zz, xy, xz, yz).  For checking the build. */
mx_status mx_demag_tensor_real(mx_ctx *ctx, double *out, mx_stream_t stream);

/* The stored FP32 spectrum octant, copied to the DEVICE array out
 * (6 * (Pz/2+1) * (Py/2+1) * (Px/2+1) floats, layout [c][kz][ky][kx]),
 * already scaled by -1/(Px Py Pz).  MX_ERR_NOT_BUILT before the build. */
mx_status mx_demag_spectrum(mx_ctx *ctx, float *out, mx_stream_t stream);

/* Kernel timing for profiling: runs `nsteps` steps exactly like
 * mx_rk_step but launches every kernel directly (no graph) with a CUDA event
 * pair around each launch, then synchronises.  For timing slot q in
 * [0, *n_kernels), ms_total[q] and launches[q] receive the summed duration and
 * the launch count.  Arrays hold max_kernels.
 *   mx_kernel_slot(q)         the slot's role in the step ("x_fwd",
 *                             "yz_fused" for the y/z passes, "x_inv",
 *                             "local_stage", "x_inv_local" for the fused
 *                             inverse x pass and local stage, ...), the same for every context;
 *   mx_kernel_name(ctx, q)    the kernel that this context's schedule
 *                             launches in that slot (e.g. "yzq_kernel");
 *                             "" for an unknown slot or a NULL ctx. */
mx_status mx_profile_step(mx_ctx *ctx, float *m, int nsteps, double dt, int method,
                          mx_stream_t stream, double *ms_total, int *launches,
                          int max_kernels, int *n_kernels);
const char *mx_kernel_slot(int q);
const char *mx_kernel_name(const mx_ctx *ctx, int q);

/* ---------------------------------------------------------------------------
 * Learned demag surrogate (the paper's ML module, Sec. II-D: a network trained
 * offline on (M, H_demag) pairs from the FFT solver replaces the demag term
 * with no change to the integration).  Here: a 3D conv net 3 -> 32 -> 64 ->
 * 32 -> 3 channels, 3x3x3 kernels, zero padding 1, exact GELU after the first
 * three layers; BF16 activations, FP32 master weights, tensor-core implicit
 * GEMM.  Inputs m are normalised per component (mean/std), outputs are the
 * normalised demag field (Gaussian normaliser, Sec. II-D).  Training: SmoothL1
 * loss (beta 1, mean over cells, components and batch) and Adam
 * (beta 0.9/0.999, eps 1e-8) with L2-coupled weight decay.
 * Parameter vector (FP32, DEVICE): W1 (32x3x3x3x3), b1 (32), W2 (64x32x27),
 * b2 (64), W3 (32x64x27), b3 (32), W4 (3x32x27), b4 (3); W[co][ci][dz][dy][dx]
 * multiplies input cell (z+dz-1, y+dy-1, x+dx-1).
 * ------------------------------------------------------------------------- */
typedef struct mx_cnn mx_cnn;

/* Number of parameters (115,907). */
int mx_cnn_num_params(void);

/* Network for fields of nx*ny*nz cells and batches up to max_batch;
 * allocates all of its buffers (about 13 MB per sample of 64x64x4).  The
 * parameters start at zero. */
mx_status mx_cnn_create(mx_cnn **out, int nx, int ny, int nz, int max_batch);
mx_status mx_cnn_destroy(mx_cnn *net);

/* Copy the parameter vector in (resets the Adam moments) / out. */
mx_status mx_cnn_set_params(mx_cnn *net, const float *params, mx_stream_t stream);
mx_status mx_cnn_get_params(const mx_cnn *net, float *params, mx_stream_t stream);

/* Normaliser, host array: input mean[3], input std[3], output mean[3],
 * output std[3] (std > 0). */
mx_status mx_cnn_set_normalizer(mx_cnn *net, const double stats[12]);

/* h = network(m) for `batch` fields stored back to back (DEVICE float4
 * arrays of batch*nx*ny*nz records). */
mx_status mx_cnn_forward(mx_cnn *net, const float *m, float *h, int batch, mx_stream_t stream);

/* Forward + SmoothL1 loss against h_target (DEVICE float4, raw field; the
 * normaliser is applied inside) + backward.  The gradient is kept for
 * mx_cnn_adam_step; loss_out (DEVICE, 1 float) and grad_out (DEVICE,
 * mx_cnn_num_params floats) receive copies when not NULL. */
mx_status mx_cnn_loss_grad(mx_cnn *net, const float *m, const float *h_target, int batch,
                           float *loss_out, float *grad_out, mx_stream_t stream);

/* Synchronise `stream` and report the net's device status: MX_ERR_TIMEOUT
 * (and clear it) if a bounded wait of a convolution kernel for its
 * tensor-core MMAs ran out since the last call (results are then invalid). */
mx_status mx_cnn_sync(mx_cnn *net, mx_stream_t stream);

/* One Adam step with the last gradient: g += weight_decay * theta, then
 * the bias-corrected Adam update with learning rate lr. */
mx_status mx_cnn_adam_step(mx_cnn *net, double lr, double weight_decay, mx_stream_t stream);

/* Use `net` (same grid) for the demag term of every later mx_heff,
 * mx_llg_rhs, mx_rk_step and mx_energy call of ctx; NULL returns to the FFT
 * convolution.  Setting a net replaces a Fourier neural operator set with
 * mx_set_demag_fno.  The caller keeps `net` alive while it is set. */
mx_status mx_set_demag_surrogate(mx_ctx *ctx, mx_cnn *net);

/* ---------------------------------------------------------------------------
 * Fourier-neural-operator demag surrogate of a film (Sec. II-D: the paper's
 * network is a 2D FNO with a lifting layer 3 -> 32 channels, four spectral
 * layers keeping the lowest 12 modes per dimension with complex filters, and
 * a projection to 3 channels).  Fields are one z plane of ny rows (H) by nx
 * columns (W):
 *   v_0 = P x + p;  v_{l+1} = act(K_l v_l + W_l v_l + w_l), act = exact GELU
 *   for l = 0..2 and the identity for l = 3;  y = Q2 gelu(Q1 v_4 + q1) + q2,
 *   K_l v = irfft2(R_l . rfft2(v)) on the kept modes ky in [0, K) and
 *   [H-K, H), kx in [0, K); per mode Y_o = sum_i X_i R_l[mode][i][o].
 * FP32 throughout.  Normaliser, loss and Adam as for the conv net.
 * Parameter vector (FP32, DEVICE): P (32x3), p (32), then per layer
 * R (2K x K x 32 x 32 x 2: mode row with the low corner first, kx, in, out,
 * re/im), W (32x32, [out][in]), w (32); then Q1 (128x32), q1 (128),
 * Q2 (3x128), q2 (3).
 * ------------------------------------------------------------------------- */
typedef struct mx_fno mx_fno;

/* Number of parameters for K = modes (2,368,259 for K = 12); -1 when modes
 * is outside 1..16. */
int mx_fno_num_params(int modes);

/* Network for nx x ny fields (2*modes <= nx, ny <= 1024, 1 <= modes <= 16)
 * and batches up to max_batch (<= 65535); allocates all of its buffers
 * (about 2.6 kB per cell of the largest batch).  The parameters start at
 * zero. */
mx_status mx_fno_create(mx_fno **out, int nx, int ny, int modes, int max_batch);
mx_status mx_fno_destroy(mx_fno *net);

/* Copy the parameter vector in (resets the Adam moments) / out. */
mx_status mx_fno_set_params(mx_fno *net, const float *params, mx_stream_t stream);
mx_status mx_fno_get_params(const mx_fno *net, float *params, mx_stream_t stream);

/* Normaliser, host array: input mean[3], input std[3], output mean[3],
 * output std[3] (std > 0). */
mx_status mx_fno_set_normalizer(mx_fno *net, const double stats[12]);

/* h = network(m) for `batch` fields stored back to back (DEVICE float4
 * arrays of batch*nx*ny records, 16-byte aligned). */
mx_status mx_fno_forward(mx_fno *net, const float *m, float *h, int batch, mx_stream_t stream);

/* Forward + SmoothL1 loss against h_target (DEVICE float4, raw field) +
 * backward; the gradient is kept for mx_fno_adam_step, loss_out (DEVICE, 1
 * float) and grad_out (DEVICE, mx_fno_num_params floats) receive copies
 * when not NULL. */
mx_status mx_fno_loss_grad(mx_fno *net, const float *m, const float *h_target, int batch,
                           float *loss_out, float *grad_out, mx_stream_t stream);

/* One Adam step with the last gradient (as mx_cnn_adam_step). */
mx_status mx_fno_adam_step(mx_fno *net, double lr, double weight_decay, mx_stream_t stream);

/* Use `net` (same nx, ny; the context must have nz = 1) for the demag term
 * of every later mx_heff, mx_llg_rhs, mx_rk_step and mx_energy call of ctx;
 * NULL returns to the FFT convolution.  Replaces a conv net set with
 * mx_set_demag_surrogate.  The caller keeps `net` alive while it is set. */
mx_status mx_set_demag_fno(mx_ctx *ctx, mx_fno *net);

/* Relative L2 difference ||a - b|| / ||b|| of two DEVICE float4 fields of
 * the context's grid (xyz only), in FP64; synchronises `stream`. */
mx_status mx_rel_l2(mx_ctx *ctx, const float *a, const float *b, double *out, mx_stream_t stream);

/* ---------------------------------------------------------------------------
 * Discrete adjoint (gradient of an objective J(m_T) of the final field of an
 * RK4 run with respect to the raw initial field and the per-cell Ms).  The
 * gradient is that of the discrete map this library computes: m_0 =
 * normalize(m0_raw), m_{s+1} = RK4 step of m_s with every stage renormalised.
 * Usage: mx_adjoint_reserve once, mx_rk_forward_record, then mx_rk_backward
 * with dJ/dm_T.  The demag term enters through the self-adjoint tensor
 * convolution; exchange, DMI (with its chiral boundary) and anisotropy through
 * their Ms-weighted symmetric stencils.
 * ------------------------------------------------------------------------- */

/* Allocate the adjoint workspaces for runs of `nsteps` RK4 steps keeping a
 * checkpoint every `checkpoint_every` steps: about
 * (nsteps/checkpoint_every + checkpoint_every + 16) * nx*ny*nz * 16 bytes.
 * Replaces any earlier reservation. */
mx_status mx_adjoint_reserve(mx_ctx *ctx, int nsteps, int checkpoint_every);

/* Forward run for the adjoint: m_final (DEVICE float4) = the field after
 * nsteps RK4 steps of size dt from normalize(m0_raw) (m0_raw DEVICE float4,
 * not modified), keeping the checkpoints the backward run needs.  Direct
 * launches on `stream` (no graph).  MX_ERR_UNSUPPORTED while a learned
 * demag backend is set on a context with demag (the adjoint differentiates
 * the tensor convolution). */
mx_status mx_rk_forward_record(mx_ctx *ctx, const float *m0_raw, float *m_final, double dt,
                               mx_stream_t stream);

/* Reverse run for the last mx_rk_forward_record: lam_final = dJ/dm_T (DEVICE
 * float4; w ignored); grad_m0 (DEVICE float4) receives dJ/dm0_raw; grad_ms
 * (DEVICE, nx*ny*nz floats, may be NULL) receives dJ/dMs per cell.  Each step
 * is recomputed from its segment's checkpoint.  Enqueued on `stream`. */
mx_status mx_rk_backward(mx_ctx *ctx, const float *lam_final, float *grad_m0, float *grad_ms,
                         mx_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MX_H */
