/*
 * acpr.h -- C ABI of the GB300 (sm_103a) Parareal / Allen-Cahn library.
 *
 * The method (Parareal with a learned convolutional coarse propagator for the
 * classic and mass-conservative Allen-Cahn equations) is the one of Sec. 3 of
 * "Operator-learning-enabled Parareal for Allen-Cahn equations" (arXiv 2510.07672).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Fields are row-major [batch][n][n] arrays, contiguous, of float64 when the
 *   precision is AC_F64 and float32 when it is AC_F32.  Grid point (i, j)
 *   is x = (-L/2 + i h, -L/2 + j h), h = L / n, periodic in both directions
 *   (Sec. 3.1: N unknowns per side, U^0 = U^N).  Base pointers must be 16-byte
 *   aligned (what cudaMalloc and torch give).
 * - Pointers documented as "device" must point to memory of the current CUDA
 *   device; "host" pointers are ordinary host memory.  The library never takes
 *   ownership of caller memory.
 * - Every call is asynchronous on `stream` (NULL = the legacy default stream)
 *   unless documented as synchronous.  Calls return AC_OK (0) or a negative
 *   error code; ac_last_error() gives a text message for the calling thread.
 * - There is no CPU fallback: a call that cannot run on the GPU fails.
 */
#ifndef ACPR_H
#define ACPR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* acpr_stream; /* same type as cudaStream_t */

enum {
    AC_OK = 0,
    AC_ERR_ARG = -1,           /* invalid argument (null pointer, bad size, ...) */
    AC_ERR_UNSUPPORTED = -2,   /* size / precision combination not built */
    AC_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    AC_ERR_TIMEOUT = -4,       /* a bounded device-side wait gave up */
    AC_ERR_NONFINITE = -5,     /* a residual came out NaN or Inf */
    AC_ERR_NOT_CONVERGED = -6, /* k reached its limit without meeting tol */
    AC_ERR_NOMEM = -7          /* device allocation failed (create calls only) */
};

enum { AC_CLASSIC = 0, AC_MASS_CONSERVING = 1 };
enum { AC_F64 = 0, AC_F32 = 1 };
enum { AC_ACT_TANH = 0, AC_ACT_GELU = 1 };

/* Problem statement of one Allen-Cahn model on the periodic square (Sec. 2,
 * Sec. 3.1).  The fine step is the stabilised linear semi-implicit scheme
 *   (1 + S dt) u' - dt eps^2 Lap_h u' = (1 + S dt) u + dt (f(u) - beta),
 * f(u) = u - u^3, Lap_h the periodic 5-point Laplacian, beta = 0 for
 * AC_CLASSIC and beta = mean(f(u)) (the Lagrange multiplier of Eq. mass_AC_eq,
 * explicit at u) for AC_MASS_CONSERVING. */
typedef struct {
    int n;          /* grid points per side: power of two, see ac_fine_supported */
    double length;  /* side L of the square (the paper uses [-0.5, 0.5]^2, L = 1) */
    double eps;     /* interface parameter epsilon */
    double S;       /* stabilisation constant (S >= 2 keeps the MBP) */
    double dt;      /* fine time step */
    int variant;    /* AC_CLASSIC or AC_MASS_CONSERVING */
    int precision;  /* AC_F64 (float64 fields) or AC_F32 (float32 fields) */
} ac_params;

/* Coarse propagator G: a stack of `layers` 3x3 convolutions with circular
 * padding 1 (cross-correlation, as torch.nn.Conv2d), widths
 * 1 -> C -> ... -> C -> 1, activation after every layer but the last, and a
 * global residual connection out = u + stack(u) when `residual` is set
 * (Sec. 3.2).  Optional mACNN mass shift (add mean(u) - mean(out)) and bound
 * limiter (clamp to [lo, hi]), applied in that order after the residual add.
 *
 * precision AC_F64: `w`, `b` are device float64 arrays and the conv runs in
 *   float64 on CUDA cores (fields float64).
 * precision AC_F32: `w`, `b` are device float32 master arrays; the conv runs
 *   with bf16 operands (inputs, weights, hidden activations rounded to
 *   nearest-even bf16) and float32 accumulation, fields float32, residual add
 *   in float32.  `packed` must then point to cnn_packed_bytes(desc) bytes of
 *   device memory (caller-owned), filled by cnn_pack_weights() whenever w or b
 *   change.
 * Layout of w: concatenation over layers l of W_l[cout][cin][3][3]; b: the
 * concatenation of b_l[cout]. */
typedef struct {
    int layers;      /* >= 1 */
    int channels;    /* hidden width C (AC_F32: 16, 32 or 64) */
    int act;         /* AC_ACT_TANH or AC_ACT_GELU (exact erf form) */
    int residual;    /* 1: global skip connection */
    int mass_fix;    /* 1: mACNN uniform mass shift */
    int limiter;     /* 1: clamp to [lo, hi] */
    double lo, hi;
    int precision;   /* AC_F64 or AC_F32 */
    const void* w;   /* device */
    const void* b;   /* device */
    void* packed;    /* device, cnn_packed_bytes() bytes (AC_F32), else NULL */
    void* work;      /* device scratch for hidden activations, caller-owned */
    size_t work_bytes; /* size of `work`; see cnn_work_bytes() */
} cnn_desc;

/* Text of the last error raised on the calling thread ("" if none). */
const char* ac_last_error(void);

/* 1 if the fine-step kernels are built for this (n, precision), else 0:
 * n = 8 .. 512 (float32) and 8 .. 256 (float64) on one thread-block cluster
 * per field; n = 1024 float32 through two passes per step over L2/HBM (fine
 * step and slice propagation only, not the adjoint or trajectory modes). */
int ac_fine_supported(int n, int precision);

/* Launch shapes of the fine kernel built for (n, precision) -- cluster size,
 * threads per CTA, occupancy target -- and the one in use.  Every shape
 * computes the same steps; they differ in how the field is split over CTAs
 * and so in which rows share a complex line, which moves results by
 * round-off.  Each shape is a deterministic function of its input; do not
 * change the shape in the middle of a Parareal solve.  ac_fine_autotune runs each shape on the caller's problem
 * (u_in -> u_out, num_fields fields, `steps` steps; twice after a warm-up),
 * writes the mean time per call in ms to ms_out[i] (may be NULL; room for
 * ac_fine_variant_count entries) and keeps the fastest for later calls of this
 * process.  SYNCHRONOUS. */
int ac_fine_variant_count(int n, int precision);
const char* ac_fine_variant_name(int n, int precision, int index);
int ac_fine_get_variant(int n, int precision);
int ac_fine_set_variant(int n, int precision, int index);
int ac_fine_autotune(const ac_params* params, int num_fields, int steps, const void* u_in, void* u_out,
                     float* ms_out, acpr_stream stream);

/* One fine step (Sec. 3.1 fine operator with one step) for each of `batch`
 * fields.  u_in, u_out: device [batch][n][n] in params->precision; they may
 * not overlap.  batch = 0 is a no-op. */
int ac_fine_step(const ac_params* params, int batch, const void* u_in, void* u_out,
                 acpr_stream stream);

/* The paper's own fine scheme (Sec. 3.1, Eq. fully-discrete): for each of
 * `num_fields` fields, `steps` Crank-Nicolson steps
 *   (U' - U)/dt = eps^2 Lap_h (U' + U)/2 + (f(U') + f(U))/2 - g(U, U'),
 * g = 0 (AC_CLASSIC) or the mean of (f(U') + f(U))/2 (AC_MASS_CONSERVING; the
 * first form of the scheme, which conserves mass), each solved by Picard
 * iteration (U^0 = U; every iteration one DFT solve of (I - dt/2 eps^2 Lap_h))
 * until max |U^{m+1} - U^m| <= tol or max_iters iterations.  The mean mode of
 * the mass-conserving variant is held at the field's float64 entry mean.
 * params->S is not used.  u_in, u_out: device [num_fields][n][n] in
 * params->precision, 16-byte aligned, not overlapping.  picard_iters:
 * optional device int[num_fields] receiving each field's total number of
 * Picard iterations.  Built for n = 64, 128, 256 (AC_F32) and n = 64 (AC_F64);
 * other sizes return AC_ERR_UNSUPPORTED.  Asynchronous on `stream`. */
int ac_cn_propagate_slices(const ac_params* params, int num_fields, int steps, const void* u_in, void* u_out,
                           double tol, int max_iters, int* picard_iters, acpr_stream stream);

/* The fine propagator F(t_n, t_{n+1}, U_n) of Eq. (fine_operator): for every
 * one of `num_fields` independent fields, `steps_per_slice` fine steps
 * (Algorithm 2: the parallel fine solves of all slices).  The field stays on
 * chip for all steps (n <= 512; at n = 1024 each step is two passes through
 * L2/HBM); HBM is touched once on entry and once on exit.  In the
 * mass-conserving variant the spectrum's mean mode is held at the field's
 * float64 mean taken on entry, so mass is conserved to rounding.
 * u_starts, u_ends: device [num_fields][n][n]; they may not overlap. */
int ac_fine_propagate_slices(const ac_params* params, int num_fields, int steps_per_slice,
                             const void* u_starts, void* u_ends, acpr_stream stream);

/* Fine propagation of a work list: item i (device int32[count][4], 16-byte
 * aligned) = {in field, out field, steps, unused} advances field `in field`
 * of u_in by `steps` fine steps into field `out field` of u_out (fields of
 * n*n values counted from the base pointers).  Items run in parallel, the
 * first ones first: list long items first.  u_in and u_out may be the same
 * buffer when no item's output is another item's input. */
int ac_fine_propagate_work(const ac_params* params, int count, const void* work, const void* u_in,
                           void* u_out, acpr_stream stream);

/* ac_fine_propagate_slices with a caller-owned workspace: at n = 1024 the
 * two-pass path keeps each field's half spectra between passes in
 * `workspace` (device, 256-byte aligned, at least
 * ac_fine_workspace_bytes(n, num_fields, precision) bytes) and the call
 * allocates nothing.  Without a workspace (ac_fine_propagate_slices) the
 * library keeps its own per-device buffer, allocated on the first n = 1024
 * call and grown when a call needs more (that call then waits for the device
 * and allocates).  Other sizes need no workspace (0 bytes; may be NULL). */
size_t ac_fine_workspace_bytes(int n, int num_fields, int precision);
int ac_fine_propagate_slices_ws(const ac_params* params, int num_fields, int steps_per_slice,
                                const void* u_starts, void* u_ends, void* workspace, size_t workspace_bytes,
                                acpr_stream stream);

/* The fine steps of ac_fine_propagate_slices, also storing every state:
 * traj[s][f] = u^s of field f for s = 0..steps (device [steps+1][num_fields]
 * [n][n]); u0: device [num_fields][n][n]. */
int ac_fine_trajectory(const ac_params* params, int num_fields, int steps, const void* u0, void* traj,
                       acpr_stream stream);

/* Adjoint (transposed Jacobian) of `steps` fine steps, applied backwards:
 * lambda_n = J(u_n)^T lambda_{n+1}.  With A = (1 + S dt) I - dt eps^2 Lap_h
 * symmetric and mu = A^{-1} lambda_{n+1}:
 *   lambda_n = (1 + S dt) mu + dt f'(u_n) * (mu - mean(mu))  (mass-conserving)
 *   lambda_n = (1 + S dt) mu + dt f'(u_n) * mu               (classic),
 * the exact transpose of the step of Sec. 3.1 (with beta = mean f(u_n)).
 * states: device [steps (or more)][num_fields][n][n], states[n][f] = u_n
 * (e.g. from ac_fine_trajectory); lam_end -> lam_start: device
 * [num_fields][n][n]. */
int ac_fine_adjoint(const ac_params* params, int num_fields, int steps, const void* states,
                    const void* lam_end, void* lam_start, acpr_stream stream);

/* Discrete energy E_h(u) = h^2 sum eps^2/2 (|D+x u|^2 + |D+y u|^2) + (u^2-1)^2/4
 * of each field (Sec. 2, Eq. energy), float64, into energy_dev[num_fields]
 * (device).  Deterministic (fixed summation order). */
int ac_energy(const ac_params* params, int num_fields, const void* u, double* energy_dev,
              acpr_stream stream);

/* dE_h/du = h^2 (-eps^2 Lap_h u - f(u)) for each field (device, params precision). */
int ac_energy_grad(const ac_params* params, int num_fields, const void* u, void* grad, acpr_stream stream);

/* Bytes of the workspace ac_energy_gradient_ic needs. */
size_t ac_energy_gradient_workspace(const ac_params* params, int steps, int checkpoint_every);

/* Gradient of E_h(u^steps) with respect to the initial field u0 (one field,
 * device [n][n]) through `steps` fine steps: checkpoints every
 * `checkpoint_every` steps on the way forward, then per segment (last first)
 * the states are recomputed from the checkpoint and the adjoint steps run
 * through them.  workspace: caller-owned device memory. */
int ac_energy_gradient_ic(const ac_params* params, int steps, int checkpoint_every, const void* u0,
                          void* grad, void* workspace, size_t workspace_bytes, acpr_stream stream);

/* Bytes of device workspace cnn_desc.packed needs (0 for AC_F64). */
size_t cnn_packed_bytes(const cnn_desc* desc);

/* Bytes of `work` one cnn_coarse_step call on `batch` n x n fields needs.
 * The workspace starts with a 256-byte header whose first int is the status
 * word of the tensor-core kernels (nonzero after a bounded device wait gave
 * up); the header must be zero when the workspace is first used, and the
 * library clears the word when it reports the error. */
size_t cnn_work_bytes(const cnn_desc* desc, int n, int batch);

/* Convert the float32 master weights into the packed bf16 layout the tensor
 * core kernel reads.  Asynchronous on `stream`. */
int cnn_pack_weights(const cnn_desc* desc, acpr_stream stream);

/* One application of the coarse propagator G (Sec. 3.2) to each of `batch`
 * fields.  u_in, u_out: device [batch][n][n] (float64 for AC_F64, float32 for
 * AC_F32); they may not overlap.  n: power of two, 8 <= n <= 1024.
 * AC_F32 calls synchronise `stream` at the end to read the workspace status
 * word and return AC_ERR_TIMEOUT if a bounded wait of the tensor-core kernels
 * gave up (u_out is then not valid); inside a stream capture the check is
 * skipped and the caller runs ac_conv_status after replaying the graph. */
int cnn_coarse_step(const cnn_desc* desc, int n, int batch, const void* u_in, void* u_out,
                    acpr_stream stream);

/* Shapes of the persistent row-streaming tensor-core conv kernel (n a
 * multiple of 128, channels 16, 32 or 64): depth of the ring of input rows in
 * shared memory (`ring`) and number of TMEM accumulator slots of 3C columns
 * (`slots`).  Every shape computes the same sums in the same order (results
 * are identical); they differ in speed.  cnn_conv_set_variant(n, C, -1) restores the automatic choice.
 * cnn_autotune times every shape on the caller's problem (u_in -> u_out,
 * `batch` fields, three calls after a warm-up; ms per call into ms_out[i],
 * may be NULL), keeps the fastest for (n, C) and synchronises `stream`.
 * Process-wide host state, not thread-safe; a Parareal handle's captured
 * graphs keep the shape they were captured with. */
int cnn_conv_variant_count(int n, int channels);
int cnn_conv_variant_shape(int n, int channels, int index, int* ring, int* slots);
int cnn_conv_set_variant(int n, int channels, int index);
int cnn_conv_get_variant(int n, int channels);
int cnn_autotune(const cnn_desc* desc, int n, int batch, const void* u_in, void* u_out, float* ms_out,
                 acpr_stream stream);

/* Failure detection (no counterpart in the paper): AC_ERR_TIMEOUT if a
 * tensor-core conv kernel that used `workspace` (a cnn_desc.work buffer or a
 * cnn_forward_train workspace) gave up a bounded wait since the last check;
 * the status word is cleared.  Synchronises `stream`. */
int ac_conv_status(void* workspace, acpr_stream stream);

/* Test hook for the failure detection above: with polls > 0, later launches
 * of the persistent tensor-core conv kernel (n >= 128) make their MMA issuer
 * wait, for `polls` polls of about 32 ns, on an mbarrier that nothing arrives
 * on, so that the bounded-wait path runs: the kernel drains its copies, frees
 * its tensor memory and stores the status code.  0 switches it off.  Host
 * state of this process; not thread-safe. */
int ac_test_conv_stall(int polls);

/* Convergence increment of Algorithm 2 between two trajectories
 * U[num_slices + 1][n][n] (slice 0, the fixed initial datum, is skipped):
 *   rel_l2  = sqrt(sum_{j=1..s} |U_new_j - U_old_j|^2) / sqrt(sum_j |U_new_j|^2)
 *   max_abs = max_{j, x} |U_new_j - U_old_j|            (the paper's sup norm)
 * accumulated in float64.  SYNCHRONOUS: returns after the results are in the
 * host doubles *rel_l2_out and *max_abs_out.  Uses a library-owned device
 * scratch buffer, allocated on the first call on each device and kept until
 * process exit; calls are serialised by a lock.  Returns AC_ERR_NONFINITE
 * (with the outputs written) if a NaN or Inf was met. */
int parareal_residual(int num_slices, int n, int precision, const void* U_new,
                      const void* U_old, double* rel_l2_out, double* max_abs_out,
                      acpr_stream stream);

/* The same increment as parareal_residual for callers that cannot allocate
 * memory: code running where cudaMalloc is not allowed or not wanted, such as
 * inside a host callback or a plugin of a framework that owns every device
 * allocation, or a real-time loop that must never wait on the allocator.  It
 * has no counterpart in the paper; it only changes where the scratch lives.
 *   - It allocates nothing (no cudaMalloc, no cudaFree, no pinned host
 *     memory): the block partials live in a fixed 48 KiB device array inside
 *     the library, which every GPU that loads the library keeps until the
 *     process exits.
 *   - Results go to out_dev, a device array of 4 doubles the caller owns:
 *     out_dev[0] = rel_l2, out_dev[1] = max_abs, out_dev[2] = sum of squared
 *     differences, out_dev[3] = sum of squared U_new (slices 1..s, float64).
 *     Asynchronous on `stream`; nothing is read back to the host.
 *   - At most 2048 * 16384 = 33,554,432 elements (num_slices * n * n) per
 *     call; larger sizes return AC_ERR_UNSUPPORTED without launching.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array: calls whose kernels overlap on the GPU (on
 *     different streams without ordering between them) race and give wrong
 *     results.  Order them on one stream, or with events. */
int parareal_residual_noalloc(int num_slices, int n, int precision, const void* U_new,
                              const void* U_old, double* out_dev, acpr_stream stream);

/* ------------------------------------------------------------------------
 * Training of the coarse propagator (AC_F32 path only; residual stack, with
 * or without the mACNN mass shift, no limiter).  G is trained to step the fully discrete fine
 * operator (Sec. 3.2: G(U_n) ~ F(U_n)).  Operands are bf16 as in the forward
 * pass, accumulation float32; the weight gradients are reduced in a fixed
 * order, so results are deterministic.
 * ------------------------------------------------------------------------ */

/* Bytes of the training workspace for `batch` n x n fields (saved layer
 * inputs and pre-activations, gradient buffers, reduction partials).  Like
 * cnn_desc.work it starts with the zero-initialised 256-byte status header;
 * cnn_forward_train and cnn_backward synchronise `stream` at the end to read
 * it (AC_ERR_TIMEOUT after a bounded wait gave up; skipped inside a capture). */
size_t cnn_train_bytes(const cnn_desc* desc, int n, int batch);

/* Forward pass that also saves, into train_ws, what cnn_backward needs.
 * u_in, u_out: device float32 [batch][n][n].  desc->packed must be current
 * (cnn_pack_weights after every weight update). */
int cnn_forward_train(const cnn_desc* desc, int n, int batch, const float* u_in, float* u_out,
                      void* train_ws, acpr_stream stream);

/* Backward pass of the last cnn_forward_train on the same u_in and train_ws:
 * grad_out = dL/du_out (device float32 [batch][n][n]); writes dL/du_in to
 * grad_in (may be NULL) and dL/dW, dL/db (device float32, the layouts of
 * desc->w and desc->b) to grad_w, grad_b, added to their contents when
 * `accumulate` is set, else overwriting them. */
int cnn_backward(const cnn_desc* desc, int n, int batch, const float* u_in, const float* grad_out,
                 float* grad_in, float* grad_w, float* grad_b, int accumulate, void* train_ws,
                 acpr_stream stream);

/* Weight gradients of the hidden C -> C layers of cnn_backward: on the tensor
 * cores (default; C = 64 and n a multiple of 128, bf16 products summed in
 * float32 in TMEM, per-chunk partials reduced in a fixed order) when `on` is
 * nonzero, on the CUDA cores otherwise (both deterministic; they differ by the
 * order of the float32 sums).  Process-wide host state, not thread-safe. */
int cnn_train_set_wgrad_tc(int on);

/* One Adam update of `count` float32 parameters (device arrays w, grad and the
 * moment estimates m, v), step number t >= 1 (bias correction 1 - beta^t). */
int cnn_adam_step(float* w, const float* grad, float* m, float* v, long long count, double lr,
                  double beta1, double beta2, double eps, int t, acpr_stream stream);

/* Mean-squared-error term scale * sum (pred - target)^2 over `count` values:
 * writes grad = 2 * scale * (pred - target), or adds it to grad when
 * grad_accumulate is set (skipped if grad is NULL), and the float64 loss to
 * loss_dev[0] (added when `accumulate` is set).  scratch_dev: device
 * float64[64]. */
int mse_loss_grad(const float* pred, const float* target, long long count, double scale, float* grad,
                  int grad_accumulate, double* loss_dev, double* scratch_dev, int accumulate,
                  acpr_stream stream);

/* ------------------------------------------------------------------------
 * The fine step on the periodic cube (d = 3; the 3D experiments of Sec. 4):
 * the stabilised semi-implicit step of ac_params with the periodic 7-point
 * Laplacian (symbol -(4/h^2)(sin^2(pi a/N) + sin^2(pi b/N) + sin^2(pi c/N))),
 * solved by a 3D FFT in five passes over L2/HBM per step.  Fields are
 * [num_fields][n][n][n] row-major (last index fastest), params->n = n per
 * side.  The mass-conserving variant holds the zero mode at the field's
 * mean taken when the call starts (the scheme conserves it exactly).
 * ------------------------------------------------------------------------ */

/* 1 if the 3D step is built for (n, precision): n = 32, 64 or 128. */
int ac_fine3d_supported(int n, int precision);

/* Device scratch bytes for `num_fields` fields (complex spectra of the field
 * pairs, tables, mean partials). */
size_t ac_fine3d_work_bytes(int n, int num_fields, int precision);

/* `steps` fine steps of every field: u_out = F^steps(u_in).  u_in may equal
 * u_out.  work: ac_fine3d_work_bytes() bytes of device memory.  Asynchronous
 * on `stream`. */
int ac_fine3d_propagate(const ac_params* params, int steps, int num_fields, const void* u_in, void* u_out,
                        void* work, size_t work_bytes, acpr_stream stream);

/* ------------------------------------------------------------------------
 * The paper's ResBlock ACNN / mACNN (Sec. 3.2) and its training with the
 * scheme-residual loss (Eq. loss_ACN, Algorithm 1).
 *
 * Network: an input 3x3 convolution 1 -> C, `blocks` residual blocks that map
 * x to x + tanh(conv2(tanh(conv1(x)))) (C -> C each), an output convolution
 * C -> 1; tanh after every convolution but the output one; circular padding 1,
 * cross-correlation as torch.nn.Conv2d; then the mACNN mass shift (add
 * mean(input) - mean(output)) and the bound limiter (clamp to [lo, hi]).
 * There is no global skip: the output layer produces U_{n+1}.
 * Parameters (device, `precision` floats): w = W_in[C][1][3][3], then per
 * block W_1[C][C][3][3], W_2[C][C][3][3], then W_out[1][C][3][3]; b = b_in[C],
 * per block b_1[C], b_2[C], then b_out[1].  Arithmetic in the field precision
 * on CUDA cores (the float32 tanh is 1 - 2/(1 + e^{2x}) on the fast
 * exponential, absolute error < 1e-6).  C = 4 or 16, blocks 0..4.
 * ------------------------------------------------------------------------ */
typedef struct {
    int channels;    /* C: 4 or 16 */
    int blocks;      /* residual blocks, 0..4 */
    int mass_fix;    /* 1: mACNN mass shift */
    int limiter;     /* 1: clamp to [lo, hi] */
    double lo, hi;
    int precision;   /* AC_F64 or AC_F32 (parameters, fields, arithmetic) */
    void* w;         /* device parameters, layouts above */
    void* b;
} acnn_desc;

/* Number of weights of the network (and of biases in *num_bias if not NULL);
 * -1 if the shape is not built. */
long long acnn_param_count(int channels, int blocks, long long* num_bias);

/* Inference handle: acnn_create copies the parameters once (synchronously)
 * into the handle, which passes them to its kernels by value.  C = 4 with at
 * most 3 blocks runs one fused kernel per 32 x 32 output tile (all layers in
 * shared memory); other shapes run the per-layer kernels. */
typedef struct acnn_net acnn_net;
int acnn_create(const acnn_desc* desc, acnn_net** out);
void acnn_destroy(acnn_net* net);

/* Device scratch bytes acnn_forward needs for `batch` n x n fields. */
size_t acnn_work_bytes(const acnn_net* net, int n, int batch);

/* U_out = G(U_in) for `batch` fields, device [batch][n][n] in the net's
 * precision; n a power of two, 32 <= n <= 1024; u_in and u_out must not
 * overlap.  work: acnn_work_bytes() bytes.  Asynchronous on `stream`. */
int acnn_forward(const acnn_net* net, int n, int batch, const void* u_in, void* u_out, void* work,
                 size_t work_bytes, acpr_stream stream);

/* Training workspace bytes (saved activations, gradient buffers, reduction
 * partials) for `batch` fields. */
size_t acnn_train_bytes(const acnn_desc* desc, int n, int batch);

/* Forward pass with the parameters in desc->w, desc->b (read on the device,
 * so an update between calls needs no host copy) that saves into train_ws
 * what acnn_backward needs. */
int acnn_forward_train(const acnn_desc* desc, int n, int batch, const void* u_in, void* u_out, void* train_ws,
                       acpr_stream stream);

/* Parameter gradients of the last acnn_forward_train on the same u_in and
 * train_ws, for grad_out = dL/d(output): written (not added) to grad_w,
 * grad_b (device, the layouts of desc->w, desc->b), summed over the batch in
 * a fixed order (deterministic).  The limiter passes the gradient where
 * lo < value < hi; the mass shift subtracts its field mean. */
int acnn_backward(const acnn_desc* desc, int n, int batch, const void* u_in, const void* grad_out, void* grad_w,
                  void* grad_b, void* train_ws, acpr_stream stream);

/* Scheme-residual loss (Eq. loss_ACN) of `batch` pairs (U0, U1) with time step
 * params->dt:  r = U1 - U0 - dt/2 (eps^2 Lap_h (U1 + U0) + f(U1) + f(U0)
 * - g(U1) - g(U0)),  g(U) = mean f(U) for AC_MASS_CONSERVING, else 0,
 * L = sum r^2 / (batch n^2), written to loss_dev[0] (float64).  If grad is not
 * NULL it receives dL/dU1 (device, field precision).  work: device,
 * loss_acn_work_bytes(n, batch) bytes.  params->precision gives the field
 * type; S is unused. */
size_t loss_acn_work_bytes(int n, int batch);
int loss_acn(const ac_params* params, int batch, const void* U0, const void* U1, double* loss_dev, void* grad,
             void* work, acpr_stream stream);

/* One Adam step (Kingma & Ba) on `count` parameters of `precision` at step
 * t >= 1: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
int acnn_adam_step(int precision, void* w, const void* grad, void* m, void* v, long long count, double lr,
                   double beta1, double beta2, double eps, int t, acpr_stream stream);

/* Algorithm 1: train desc's parameters in place with the scheme-residual loss.
 * U0s: device [R][n][n] initial conditions; perm: HOST int[epochs][R], the
 * visiting order of each epoch, cut into R/q subsets of q.  For each subset U
 * starts at its q initial conditions; for each of `steps` time steps, b_inner
 * updates each predict U1 = G(U), take the loss of (U, U1), its gradient and
 * one Adam step; U then becomes the U1 of the last update.  adam_m, adam_v:
 * device moments (weights then biases, zeroed by the caller before the first
 * call); *t: Adam step count, carried between calls.  losses_dev: device
 * float64[epochs * (R/q) * steps * b_inner], one loss per update.
 * workspace: caller-owned device memory, 256-byte aligned, of at least
 * acnn_train_alg1_bytes(desc, n, q) bytes (the subset's fields, gradients and
 * the training and loss workspaces); the call allocates nothing.
 * SYNCHRONOUS. */
int acnn_train_alg1(const ac_params* params, const acnn_desc* desc, int R, const void* U0s, const int* perm,
                    int epochs, int q, int steps, int b_inner, double lr, double beta1, double beta2, double eps,
                    void* adam_m, void* adam_v, int* t, double* losses_dev, void* workspace,
                    size_t workspace_bytes, acpr_stream stream);

/* Bytes of the acnn_train_alg1 workspace for n x n fields and subsets of q. */
size_t acnn_train_alg1_bytes(const acnn_desc* desc, int n, int q);

/* ------------------------------------------------------------------------
 * Parareal driver (Algorithm 2) for `problems` independent problems that
 * share one ac_params, one coarse propagator, s slices of c fine steps.
 * ------------------------------------------------------------------------ */
typedef struct ac_parareal ac_parareal;

/* Allocates the device state (trajectory U[problems][s+1][n][n], stored coarse
 * values, fine results, residual scratch) and copies the initial data
 * u0 (device [problems][n][n], precision of params).  *out receives the
 * handle.  The cnn_desc is copied; its device buffers must outlive the handle.
 * coarse may be NULL when G is the ResBlock ACNN, set with
 * ac_parareal_set_coarse_acnn before the first iteration. */
int ac_parareal_create(const ac_params* params, const cnn_desc* coarse, int problems,
                       int num_slices, int steps_per_slice, const void* u0,
                       ac_parareal** out);

/* As ac_parareal_create for problems that share params and coarse net but
 * have their own slice counts num_slices[p] and fine steps per slice
 * steps_per_slice[p] (host arrays of `problems` ints).  The fine solves of all
 * problems run in one launch per iteration (work items longest first); the
 * coarse sweep batches, at each slice, the problems that still have it. */
int ac_parareal_create_uneven(const ac_params* params, const cnn_desc* coarse, int problems,
                              const int* num_slices, const int* steps_per_slice, const void* u0,
                              ac_parareal** out);

/* Capture each iteration's device work into a CUDA graph the first time a
 * (k, active problems) pair is met and replay it afterwards. */
int ac_parareal_enable_graphs(ac_parareal* state, int on);

/* Coarse-time composition (the remark after Algorithm 2): every coarse
 * evaluation of the handle's solves applies G `substeps` times in a row
 * (1 = plain G, the default; at most 64), so one network trained for a
 * shorter step covers the slice.  The first call with substeps > 1 allocates
 * two [problems][n][n] buffers for the intermediate fields.  Drops the
 * handle's captured iteration graphs.  Call between solves. */
int ac_parareal_set_coarse_substeps(ac_parareal* state, int substeps);

/* Use the ResBlock ACNN `net` as the coarse propagator G of the handle's
 * solves instead of the conv stack it was created with (NULL switches back).
 * net must match the handle's precision and outlive its use; allocates the
 * net's scratch for all problems and drops the captured iteration graphs. */
int ac_parareal_set_coarse_acnn(ac_parareal* state, const acnn_net* net);

/* Choose the fine propagator F of the handle's solves: scheme 0 = the
 * stabilised semi-implicit step (the default), 1 = the Crank-Nicolson step of
 * Sec. 3.1 with Picard iteration to max |U^{m+1} - U^m| <= tol (at most
 * max_iters iterations), as in ac_cn_propagate_slices.  Scheme 1 needs a size
 * ac_cn_propagate_slices is built for (else AC_ERR_UNSUPPORTED).  Drops the
 * handle's captured iteration graphs.  Call between solves. */
int ac_parareal_set_fine_scheme(ac_parareal* state, int scheme, double tol, int max_iters);

/* One iteration of Algorithm 2 on every problem not yet converged.
 * *k_inout = 0 runs the initial coarse sweep U^0_{n+1} = G(U^0_n); k >= 1 runs
 * the fine solves F(U^{k-1}_n), n = k-1..s-1, then the sequential correction
 * U^k_{n+1} = G(U^k_n) + F(U^{k-1}_n) - G(U^{k-1}_n) (the new coarse values are
 * stored for the next iteration), then the convergence increment of each
 * problem into rel_l2_out[p], max_abs_out[p] (host arrays of `problems`
 * doubles; untouched for k = 0).  On return *k_inout is k + 1.
 * SYNCHRONOUS (the increments are read back). */
int parareal_iterate(ac_parareal* state, int* k_inout, double* rel_l2_out, double* max_abs_out,
                     acpr_stream stream);

/* Mark problem p converged (it is skipped by later iterations) or active. */
int ac_parareal_set_active(ac_parareal* state, int problem, int active);

/* Device pointer to the trajectory U[problems][s+1][n][n] (owned by state). */
const void* ac_parareal_trajectory(const ac_parareal* state);

/* Copy the trajectory U[problems][s+1][n][n] into the device buffer dst
 * (precision of the params).  Asynchronous on `stream`. */
int ac_parareal_copy_trajectory(const ac_parareal* state, void* dst, acpr_stream stream);

/* Run iterations until every problem has rel_l2 < tol or k = kmax (k <= s).
 * A problem that reaches k = s stops there: its trajectory is then the fine
 * solve itself (Sec. 3.3).  A non-finite increment (a diverging iterate beyond
 * the exact prefix) counts as not converged and the iterations go on.
 * iters_out: host int[problems], the iteration at which each problem stopped;
 * rel_l2_out: host double[problems], its last increment.  SYNCHRONOUS.
 * Returns AC_ERR_NOT_CONVERGED if a problem reached kmax < s above tol. */
int ac_parareal_solve(ac_parareal* state, double tol, int kmax, int* iters_out,
                      double* rel_l2_out, acpr_stream stream);

/* Restart the handle at k = 0 from new initial data u0 (device
 * [problems][n][n]); every problem becomes active.  Asynchronous on `stream`. */
int ac_parareal_reset(ac_parareal* state, const void* u0, acpr_stream stream);

/* Per-phase device time of the iterations run since the last reset of the
 * statistics, measured with CUDA events on the iteration's stream when timing
 * is on (ac_parareal_enable_timing), plus work counters. */
typedef struct {
    double fine_ms;          /* fine-propagator launches */
    double coarse_ms;        /* coarse sweeps (conv stack and corrections) */
    double increment_ms;     /* convergence increments */
    long long fine_launches;
    long long fine_cell_steps;  /* sum over fine launches of fields * steps * n^2 */
    long long coarse_calls;     /* applications of G to a batch of problems */
    long long coarse_cells;     /* sum over G applications of batch * n^2 */
    long long iterations;
} ac_parareal_stats;

int ac_parareal_enable_timing(ac_parareal* state, int on);
int ac_parareal_get_stats(const ac_parareal* state, ac_parareal_stats* out);
int ac_parareal_reset_stats(ac_parareal* state);

/* Number of kernels this library has launched in this process (all entry
 * points, all devices; a replayed CUDA graph adds its kernel nodes).  Lets a
 * caller count the launches of a region. */
long long ac_launch_count(void);

/* ac_parareal_solve on `count` handles (e.g. one per grid size) at once:
 * every iteration is launched on all handles' streams before any is waited
 * for, so their kernels overlap.  iters_out / rel_l2_out: host arrays with the
 * handles' problems one after another.  SYNCHRONOUS. */
int ac_parareal_solve_many(ac_parareal* const* states, int count, const acpr_stream* streams, double tol,
                           int kmax, int* iters_out, double* rel_l2_out);

void ac_parareal_destroy(ac_parareal* state);

#ifdef __cplusplus
}
#endif
#endif /* ACPR_H */
