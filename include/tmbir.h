/*
 * tmbir.h -- C ABI of the Toeplitz-accelerated MBIR gradient path (Kumar & Donatelli,
 * "Fast Large-Scale Model-Based Iterative Tomography ...").
 *
 * The library reconstructs stacks of parallel-beam slices by minimising Eq. 5,
 *     F(f) = 1/2 ||R f - g||^2 + lambda Phi(f),
 * with the fast gradient method of Sec. 2.  Every gradient uses the Toeplitz form of
 * Sec. 2.1 (Eqs. 9-11): R*R f is a zero-padded 2N x 2N FFT convolution with the
 * point-spread kernel K, and R*g is precomputed once.  Phi is the qGGMRF prior over the
 * 26-voxel neighbourhood (Sec. 2, Sec. 2.4).
 *
 * Conventions
 *   - Every call returns an int status: TMBIR_OK (0) or a negative TMBIR_ERR_* code;
 *     tmbir_last_error() gives a message for the calling thread.  No exception crosses
 *     the ABI.
 *   - Work is enqueued asynchronously on the CUDA stream bound at tmbir_create.  Calls
 *     that return host values (stats, objective, lambda_max) synchronise that stream.
 *   - Pointers named d_* are device pointers, h_* host pointers.  The caller owns every
 *     device buffer, including the workspace sized by tmbir_workspace_size; the library
 *     allocates no device memory.  Device buffers must be 16-byte aligned.
 *   - Images are float32 [slice][row][col] (row-major N x N per slice); pixel (r, c) sits at
 *     x = c - N/2, y = r - N/2.  Sinograms are float32 [slice][angle][bin]; bin m sits at
 *     s = m - n_det/2.  An angle theta projects onto s = x cos(theta) + y sin(theta).
 *   - Radial frequencies are k / n_det with |k| <= n_det/2 - 1: the Nyquist bin is dropped,
 *     so R is real and R*R is exactly Toeplitz.
 */
#ifndef TMBIR_H
#define TMBIR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TMBIR_OK = 0,
  TMBIR_ERR_ARG = -1,       /* null pointer, bad value, misaligned buffer */
  TMBIR_ERR_SHAPE = -2,     /* unsupported size (N, n_det, factorisation of 2N) */
  TMBIR_ERR_WORKSPACE = -3, /* no workspace bound, or too small */
  TMBIR_ERR_CUDA = -4,      /* a CUDA runtime call failed */
  TMBIR_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
  TMBIR_ERR_NONFINITE = -6, /* NaN or Inf in a reduction */
  TMBIR_ERR_STATE = -7      /* call order (no geometry, operator not built) */
};

enum { TMBIR_RESTART_GRADIENT = 0, TMBIR_RESTART_NONE = 1, TMBIR_RESTART_FUNCTION = 2 };
enum { TMBIR_SPECTRA_FP32 = 0, TMBIR_SPECTRA_BF16 = 1 };

typedef struct tmbir_ctx tmbir_ctx;

/*
 * One geometry group: n_slices slices of N x N pixels seen under the same n_angles
 * parallel-beam angles by n_det detector bins (Sec. 2, Eq. 1).  Slices of a group are
 * coupled by the 3D prior; different groups are independent.
 *   N        image side: a power of two in [64, 2048], or 1536 or 2560 (mixed-radix FFTs).
 *   n_det    detector bins; must equal N (pixel pitch = bin pitch).
 *   angles   host array of n_angles radians; copied by tmbir_set_geometry.
 *   span     angular range covered by the angles (pi for a full half turn); the FBP
 *            quadrature weight is span / n_angles (Eq. 14).
 */
typedef struct {
  int N;
  int n_det;
  int n_angles;
  const double* angles;
  double span;
  int n_slices;
} tmbir_group;

/*
 * Prior and optimiser parameters (Eq. 5-6, Sec. 2).
 *   p, q, c, sigma  qGGMRF potential rho(D) = |D/sigma|^q / (1 + |D/(c sigma)|^(q-p)),
 *                   1 <= p <= q; q = 2 is the fast path.
 *   lambda          prior weight.
 *   L               step constant; <= 0 selects, per group, 1.01 lambda_max(R*R) of the group +
 *                   lambda*2*(2/sigma^2) (needs q = 2 and a built operator).  Each group runs
 *                   its own momentum sequence and restart test with its own step constant, as
 *                   if reconstructed alone; the stop rule (max_iter, gap_tol on the summed
 *                   objective) and the BF16 -> FP32 switch apply to the whole batch.
 *   max_iter        iterations of the fast gradient method.
 *   gap_tol, F_ref  stop early once (F(y_k) - F_ref) / (F(0) - F_ref) <= gap_tol
 *                   (gap_tol <= 0 disables it).
 *   restart         TMBIR_RESTART_GRADIENT: momentum restarts when <grad F(y_k), x_{k+1}-x_k> > 0;
 *                   TMBIR_RESTART_FUNCTION: when F(y_k) > F(y_{k-1}); TMBIR_RESTART_NONE: never
 *                   (the restart rule is not stated in the paper; Sec. 2 cites the restarted
 *                   fast gradient method).
 *   use_graph       run the iterations as one CUDA graph: a device-driven WHILE loop whose body
 *                   is one iteration; the device stops it at max_iter or the gap tolerance, so
 *                   no launch is spent after the stop.  The executable graph is cached and
 *                   reused while the image and R*g buffers and the prior stay the same.
 *   spectra         storage of the padded intermediate spectrum during the iterations:
 *                   TMBIR_SPECTRA_FP32, or TMBIR_SPECTRA_BF16 (half the bytes; transforms,
 *                   kernel multiply and prior still in FP32).  Not a paper setting: the paper
 *                   computes in FP32 throughout (Sec. 3.1).
 *   refine_gap      with BF16 spectra: switch to FP32 spectra for the remaining iterations
 *                   once the relative gap (as for gap_tol) is <= refine_gap; 0 keeps BF16 to
 *                   the end.
 *   resume          0: start a new run from d_x (x_{-1} = x_0, t = 1).  1: continue the run
 *                   the context holds (the previous tmbir_reconstruct, or a checkpoint loaded
 *                   by tmbir_state_import) for max_iter more iterations; d_x must hold that
 *                   run's x_k.  The result is bitwise the one an uninterrupted run gives.
 *   nonneg          1: project every iterate onto x >= 0 (x_{k+1} = max(y - G/L, 0)), the
 *                   fast gradient method on Eq. 5 restricted to non-negative images (a variant:
 *                   Eq. 5 itself has no constraint); 0: unconstrained.
 */
typedef struct {
  double p, q, c, sigma, lambda;
  double L;
  int max_iter;
  double gap_tol;
  double F_ref;
  int restart;
  int use_graph;
  int spectra;
  double refine_gap;
  int resume;
  int nonneg;
} tmbir_params;

/* Result of tmbir_reconstruct (host struct filled on return). */
typedef struct {
  int iterations;   /* iterations run */
  int restarts;     /* momentum restarts, summed over the groups */
  int status;       /* TMBIR_OK, TMBIR_ERR_NONFINITE */
  double objective; /* F(y_k) of the last iteration (Eq. 10 + lambda Phi) */
  double gap;       /* relative gap of that value when F_ref was given, else 0 */
  double L;         /* step constant of the first group */
  double grad_norm; /* ||grad F(y_k)||_2 of the last iteration */
} tmbir_stats;

/*
 * Create a context bound to a CUDA stream (cudaStream_t passed as void*; NULL = legacy default
 * stream).  On the device current at the call it also commits the fixed scratch arrays of
 * tmbir_normal_apply_static (67 MiB, held until the process exits) and caches their addresses;
 * fails with TMBIR_ERR_CUDA if that device cannot hold them.
 */
int tmbir_create(tmbir_ctx** out, void* stream);
int tmbir_destroy(tmbir_ctx* ctx);
/* Message of the last failing call on this thread ("" if none).  Owned by the library. */
const char* tmbir_last_error(void);

/*
 * Define the slices to reconstruct (Sec. 2: slices are independent in the data term and
 * coupled by the prior).  Copies the groups and angles; invalidates the workspace binding.
 */
int tmbir_set_geometry(tmbir_ctx* ctx, int n_groups, const tmbir_group* groups);

/* Bytes of device workspace the current geometry needs. */
int tmbir_workspace_size(const tmbir_ctx* ctx, size_t* bytes);

/*
 * Bind caller-owned device workspace (16-byte aligned, >= tmbir_workspace_size bytes).  The
 * library keeps the kernel spectrum, twiddle tables, iterate buffers and scratch in it; it
 * must stay valid until the next set_geometry / set_workspace / destroy.  Enqueues the
 * upload of the twiddle tables on the context stream.
 */
int tmbir_set_workspace(tmbir_ctx* ctx, void* d_workspace, size_t bytes);

/*
 * Per-angle weights of the data term (a variant of Eq. 5: F = 1/2 sum_a w_a ||R_a f - g_a||^2 +
 * lambda Phi(f), e.g. to down-weight noisy or partial views).  Weights that depend on the angle
 * alone keep R* W R shift-invariant, so the Toeplitz form holds with the kernel
 * K_w(d) = (1/n_det) sum_{a,k} w_a exp(2 pi i xi_{a,k} . d), and R*g becomes R* W g.
 *   group  index of the geometry group (0 .. n_groups - 1).
 *   h_w    host array of the group's n_angles weights in [0, 1] (copied), or NULL for all 1.
 * The weights enter K, lambda_max, R*g and 1/2 g.g at the next tmbir_build_operator* call (the
 * previous operator is dropped) and the direct gradient (R* W (R x - g)); the FBP start and
 * tmbir_adjoint stay unweighted.  Call after tmbir_set_geometry; a later set_geometry clears them.
 */
int tmbir_set_angle_weights(tmbir_ctx* ctx, int group, const double* h_w);

/*
 * Setup of Sec. 2.1 ("computed once prior to the iterative reconstruction"): per group the
 * point-spread kernel K = NUFFT1(ones) on [-(N-1), N-1]^2 and the real spectrum of its 2N x 2N
 * circulant embedding (kept in the workspace); R*g for every slice into d_atg
 * [slice][row][col]; 1/2 g.g per group; lambda_max(R*R) by 100 power steps (kept in the
 * workspace).  d_sino is [slice][angle][bin] for all groups back to back.  K, its spectrum and
 * the reductions in FP64; R*g (the type-1 NUFFT of Eq. 4 on a 1.25x grid) in double-word FP32
 * arithmetic (hi + lo pairs of FP32, a 48-bit significand: FP64-class accuracy, about 1e-10
 * relative before the FP32 store) on the FP32 pipe, whose rate on GB300 is far above the FP64
 * pipe's.
 */
int tmbir_build_operator(tmbir_ctx* ctx, const float* d_sino, float* d_atg);

/*
 * tmbir_build_operator with R*g computed in FP32: the back-projection of the FBP start without
 * its ramp filter (2N spreading grid, width-10 kernel, FP32 arithmetic: 2e-7 to 4e-7 relative L2
 * against the FP64 sums, where the double-word R*g stays at the FP32 store's 3e-8), at a fraction
 * of that transform's cost.  K, its spectrum, lambda_max and 1/2 g.g are built as in
 * tmbir_build_operator.  Meant for the coarse levels of the hierarchy (Sec. 2.3), whose result
 * only starts the next level; the finest level keeps the double-word R*g.
 */
int tmbir_build_operator_fp32(tmbir_ctx* ctx, const float* d_sino, float* d_atg);

/*
 * Filtered back-projection start of Sec. 2.2 (Eqs. 12-14): every projection row is
 * convolved with the unit-pitch Ram-Lak kernel (zero padded, no wrap-around), back-projected
 * with R* and weighted by span / n_angles.  d_x0 receives [slice][row][col].
 */
int tmbir_fbp(tmbir_ctx* ctx, const float* d_sino, float* d_x0);

/*
 * tmbir_build_operator and tmbir_fbp in one call, the two overlapped: R*g (double-word) runs on the
 * context stream while the FBP start (FP32) runs on a second stream the context owns, joined
 * back into the context stream before any later work.  Same results as the two calls;
 * d_atg and d_x0 must differ.  Needs a non-NULL context stream.
 */
int tmbir_build_operator_fbp(tmbir_ctx* ctx, const float* d_sino, float* d_atg, float* d_x0);

/*
 * Fast gradient method with restart (Sec. 2, Eq. 6 with the '+' sign on the prior term)
 * from the image in d_x, which receives the last iterate.  Each iteration:
 *   y = x_k + beta_k (x_k - x_{k-1});  G = K (*) y - R*g + lambda grad Phi(y)   (Eqs. 9, 11)
 *   x_{k+1} = y - G / L;  restart test; t_{k+1}, beta_{k+1}.
 * d_atg is the R*g from tmbir_build_operator.  h_stats (may be NULL) receives the summary.
 */
int tmbir_reconstruct(tmbir_ctx* ctx, float* d_x, const float* d_atg, const tmbir_params* prm, tmbir_stats* h_stats);

/* Per-iteration log of the last tmbir_reconstruct: h_log[4*k + {0,1,2,3}] = F(y_k),
 * <G, x_{k+1} - x_k>, number of groups whose momentum restarted (0/1 for one group), ||G||^2,
 * the first, second and fourth summed over the groups.  Copies min(max_entries, iterations) rows;
 * *n_out receives that count. */
int tmbir_get_log(tmbir_ctx* ctx, double* h_log, int max_entries, int* n_out);

/* d_z = R*R d_x = Res(F^-1(F K . F Pad x)) for every slice (Eq. 9), FP32. */
int tmbir_normal_apply(tmbir_ctx* ctx, const float* d_x, float* d_z);

/* d_grad = K (*) d_x - d_atg + lambda grad Phi(d_x) (Eq. 11 plus the prior), FP32. */
int tmbir_gradient(tmbir_ctx* ctx, const float* d_x, const float* d_atg, const tmbir_params* prm, float* d_grad);

/*
 * One fused iteration at a given momentum: y = x + beta (x - x_prev), G as in
 * tmbir_gradient at y, x_next = y - G / L.  h_partials (may be NULL) receives, in FP64,
 * { y.(K*y), y.R*g, Phi(y) (without lambda), <G, x_next - x>, ||G||^2 }.
 */
int tmbir_step(tmbir_ctx* ctx, const float* d_x, const float* d_x_prev, double beta, const float* d_atg,
               const tmbir_params* prm, double L, float* d_x_next, double* h_partials);

/* F(x) = 1/2 x.(K*x) - x.R*g + 1/2 g.g + lambda Phi(x) (Eq. 10 plus the prior), FP64 reduction. */
int tmbir_objective(tmbir_ctx* ctx, const float* d_x, const float* d_atg, const tmbir_params* prm, double* h_F);

/*
 * The direct operators of Sec. 2 (Eqs. 3-4), without the Toeplitz structure: R and R* through
 * non-uniform FFTs at the polar samples, FP32 (the paper's gradient before the Toeplitz
 * acceleration of Sec. 2.1, kept for the comparison of Sec. 3.1).
 *   tmbir_forward:  d_sino = R d_x, [slice][angle][bin] for all groups back to back: the image
 *                   divided by the kernel's Fourier transform on the 2N x 2N oversampled grid,
 *                   an FFT, interpolation at the polar samples with the spreading kernel, the
 *                   radial 1D transform (type-2 NUFFT, the adjoint of the back-projection).
 *   tmbir_adjoint:  d_x = R* d_sino (the type-1 NUFFT of tmbir_build_operator, in FP32).
 *   tmbir_gradient_direct: d_grad = R*(R d_x - g) + lambda grad Phi(d_x), the residual formed in
 *                   the sinogram domain and back-projected once; h_F (may be NULL) receives
 *                   F(x) = 1/2 ||R x - g||^2 + lambda Phi(x) (FP64 reductions; synchronises).
 *                   d_sino is the measured sinogram g.  Needs no built operator.
 * All use the setup scratch of the workspace (and the direct gradient its K (*) y buffers and the
 * first iterate buffer), so they must not overlap other calls of the context.
 */
int tmbir_forward(tmbir_ctx* ctx, const float* d_x, float* d_sino);
int tmbir_adjoint(tmbir_ctx* ctx, const float* d_sino, float* d_x);
int tmbir_gradient_direct(tmbir_ctx* ctx, const float* d_x, const float* d_sino, const tmbir_params* prm,
                          float* d_grad, double* h_F);

/* Largest eigenvalue of R*R per group (power iteration of tmbir_build_operator); h_out[n_groups]. */
int tmbir_lambda_max(tmbir_ctx* ctx, double* h_out);

/* FP64 point-spread kernel of one group, K[(dy + N-1) * (2N-1) + (dx + N-1)], into d_K (device). */
int tmbir_kernel(tmbir_ctx* ctx, int group, double* d_K);

/*
 * x2 Lanczos-3 level transfer of Sec. 2.3 (Eqs. 16-17, with the standard windowed sinc
 * L(x) = sinc(x) sinc(x/3)): coarse sample i lands on fine sample 2i; odd fine samples take
 * the six normalised taps at offsets +-0.5, +-1.5, +-2.5; zero outside the grid; separable.
 * d_coarse [n_slices][Nc][Nc] -> d_fine [n_slices][2Nc][2Nc].  No context geometry needed.
 */
int tmbir_upsample_lanczos3(tmbir_ctx* ctx, const float* d_coarse, int n_slices, int Nc, float* d_fine);

/*
 * Coarse projections of Sec. 2.3 ("subsampling the full-resolution projection data"): every
 * factor-th bin aligned on the centre bin, divided by factor (line integrals in coarse-pixel
 * units).  d_sino [n_slices][n_angles][n_det] -> d_out [n_slices][n_angles][n_det/factor].
 */
int tmbir_downsample_sino(tmbir_ctx* ctx, const float* d_sino, int n_slices, int n_angles, int n_det, int factor,
                          float* d_out);

/*
 * Measurement: run `iters` iterations of tmbir_reconstruct's loop eagerly (no graph) from d_x
 * with CUDA events recorded on the context stream around every launch, and return the summed
 * device time per kernel kind in h_ms[5] = { pass 1 (rows), pass 2 (columns), pass 3a (inverse
 * rows), pass 3b (prior + gradient + update), finalize }.  d_x receives the iterate like
 * tmbir_reconstruct.
 */
int tmbir_pass_times(tmbir_ctx* ctx, float* d_x, const float* d_atg, const tmbir_params* prm, int iters, double* h_ms);

/*
 * Autotuner (no counterpart in the paper), per group on d_x / d_atg:
 *  - the slices per spectrum chunk: passes 1, 2 and 3a can run chunk by chunk (a chunk's half
 *    spectra may then stay in L2 between them); chunks of 4, 8 and 16 slices and the whole
 *    group (the default) are timed over the whole group;
 *  - the slices a pass-3b block marches through (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64 up to
 *    the slice count, and the default rule), timing pass 3b of one iteration;
 *  - for sides with transform variants (N = 2048), the rows per block of the row passes 1 and
 *    3a (4 or 8; eight rows move 64-byte segments of the column-major spectrum, four rows leave
 *    room for more blocks per SM), timing each pass.
 * The fastest of each is kept; h_zc and h_sc (either may be NULL) receive the choices per
 * group.  Later contexts of this process with the same image side and slice count start from
 * the choices.  The other transform tile shapes are fixed per image side at compile time.  d_x
 * is not modified.
 */
int tmbir_autotune(tmbir_ctx* ctx, const float* d_x, const float* d_atg, const tmbir_params* prm, int* h_zc,
                   int* h_sc);

/*
 * Checkpoint of a run (no counterpart in the paper): the fast-gradient state after
 * tmbir_reconstruct (per group: momentum t and beta, step constant, restart count and
 * F(y_{k-1}) for the function restart; the iteration count and storage phase) and x_{k-1};
 * x_k is the caller's image.  d_state is a
 * caller-owned device buffer of tmbir_state_size bytes, 16-byte aligned.  Export needs a
 * finished run; import replaces the context's state (same geometry), after which
 * tmbir_reconstruct with resume = 1 continues it.  Both are asynchronous on the context
 * stream except import, which returns after the copy.
 */
int tmbir_state_size(const tmbir_ctx* ctx, size_t* bytes);
int tmbir_state_export(tmbir_ctx* ctx, void* d_state);
int tmbir_state_import(tmbir_ctx* ctx, const void* d_state);

/*
 * Number of library kernels launched so far: the host-side count of every launch by this
 * process plus the kernels this context ran inside device-driven graph loops (counted by the
 * loop's finalize kernel; reading it synchronises the context stream).
 */
int tmbir_launch_count(const tmbir_ctx* ctx, long long* h_count);

/*
 * Learned warm start (not in the paper; an addition that refines the FBP start): a
 * four-layer 3x3 convolutional network, channels 1 -> 32 -> 32 -> 32 -> 1, zero padding, a bias
 * per output channel, ReLU after the first three layers.  FP32 master weights, BF16 activations,
 * FP32 accumulation; the 32 -> 32 layers (forward and data gradient) run as implicit GEMMs on
 * the 5th-generation tensor cores (tcgen05.mma, accumulators in TMEM).  Every wait on the
 * tensor core is bounded: a convolution that gives up sets a flag that the next synchronising
 * call (net_backward, train_step with h_loss, warm_start) reports as TMBIR_ERR_TIMEOUT.
 * Parameter vector (tmbir_cnn_param_count() = 19105 floats), layer by layer: weights
 * [cout][cin][3][3] then biases [cout].  Images are float32 [batch][H][W], all H x W.
 * Applied to a start x it gives x + s * net(x / s), s = RMS of x per image; trained with the
 * mean squared error between net(x / s) and (t - x) / s for targets t, Adam (0.9, 0.999, 1e-8).
 * The network keeps its weights, optimiser state and activations in a caller-owned workspace.
 */
typedef struct tmbir_cnn tmbir_cnn;
int tmbir_cnn_param_count(void);
int tmbir_cnn_workspace_size(int max_batch, int H, int W, size_t* bytes);
/* stream: cudaStream_t as void*; d_workspace 256-byte aligned, >= tmbir_cnn_workspace_size */
int tmbir_cnn_create(tmbir_cnn** out, void* stream, int max_batch, int H, int W, void* d_workspace, size_t bytes);
int tmbir_cnn_destroy(tmbir_cnn* net);
/* He-normal weights (last layer scaled by 0.1 so the refiner starts near the identity), zero biases */
int tmbir_cnn_init(tmbir_cnn* net, unsigned long long seed);
int tmbir_cnn_set_weights(tmbir_cnn* net, const float* h_params);
int tmbir_cnn_get_weights(tmbir_cnn* net, float* h_params);
/* d_y = d_x + s * net(d_x / s) for batch images */
int tmbir_cnn_apply(tmbir_cnn* net, const float* d_x, int batch, float* d_y);
/* one Adam step on a batch of (start, target) pairs; h_loss (may be NULL) receives the loss */
int tmbir_cnn_train_step(tmbir_cnn* net, const float* d_x, const float* d_target, int batch, float lr, double* h_loss);
/* raw network: d_out = net(d_in) (no normalisation, no residual) */
int tmbir_cnn_net_forward(tmbir_cnn* net, const float* d_in, int batch, float* d_out);
/* raw gradients of sum(d_gout * net(d_in)): parameters into h_gparams (host), input into d_gin (may be NULL) */
int tmbir_cnn_net_backward(tmbir_cnn* net, const float* d_in, const float* d_gout, int batch, float* h_gparams,
                           float* d_gin);
/*
 * Warm start with fallback: d_x0 = the refined start if its objective (Eq. 10 plus the prior) is
 * below that of the FBP start d_fbp, else a copy of d_fbp; *h_used_cnn tells which.  Needs one
 * geometry group with N equal to the network's image size.  The network's work is ordered after
 * the context stream's pending work and before the objectives (events, when the two streams
 * differ); the result is ready in stream order on the context's stream.
 */
int tmbir_warm_start(tmbir_ctx* ctx, tmbir_cnn* net, const float* d_fbp, const float* d_atg, const tmbir_params* prm,
                     float* d_x0, int* h_used_cnn);

/*
 * tmbir_normal_apply without device scratch from the workspace: the same d_z = R*R d_x, with the
 * intermediate spectra and reduction partials in a fixed array inside the library.  The paper
 * has no counterpart; this entry point is for callers that cannot allocate device memory at the
 * time of the call (for example code running under a host application that owns the whole
 * device-memory budget, or a latency-critical loop where allocation is not allowed).
 *   - The array holds 8 Mi complex values (64 MiB) of spectra, (N+1) * N per slice, and the
 *     partial sums of 65536 blocks.  The groups run one after another in chunks of as many
 *     slices as fit (at most the context's spectrum chunk); a geometry whose pass 3b needs
 *     more than 65536 blocks is rejected with TMBIR_ERR_SHAPE; nothing is allocated on any
 *     path.
 *   - Every device that loads the library holds the array until the process exits.  The
 *     memory is committed when tmbir_create runs with that device current (it looks up the
 *     array's device address with cudaGetSymbolAddress, which loads the module holding it, and
 *     caches the address), not at this call, so a caller that owns the rest of the memory
 *     budget learns of a shortage at context creation.  On a device where no context was
 *     created, the first call of this entry point does that lookup itself; make that first call
 *     before any stream capture.
 *   - A device reset (cudaDeviceReset) invalidates the cached address along with every context
 *     and workspace on that device: create a new context after a reset, which refreshes it.
 *   - All calls share the one array and it keeps the last call's contents: calls whose work
 *     overlaps on the GPU (different streams or contexts, concurrently) race on it.
 *   - The operator must be built (tmbir_build_operator); its kernel spectrum still lives in the
 *     context workspace.
 */
int tmbir_normal_apply_static(tmbir_ctx* ctx, const float* d_x, float* d_z);

/*
 * Bounded-wait check (failure detection; no counterpart in the paper).  Every wait of the library
 * on a device barrier polls at most a fixed number of times; a wait that gives up records that in
 * a status word and its kernel returns, so the call reports TMBIR_ERR_TIMEOUT instead of hanging
 * the GPU, and the context stays usable.  This call runs that mechanism on its own: one block
 * waits, for at most `polls` polls (1 .. 2^24), on a shared-memory barrier that one of its threads
 * arrives on first (arrive != 0: returns TMBIR_OK) or that nothing arrives on (arrive == 0:
 * returns TMBIR_ERR_TIMEOUT).  The status word is a library-wide device variable: checks that
 * overlap on the GPU race on it.  Synchronises the context stream.
 */
int tmbir_wait_check(tmbir_ctx* ctx, unsigned polls, int arrive);

/*
 * Measurement (no counterpart in the paper): the special-function throughput of the device the
 * context runs on.  Threads run independent chains of log2, exp2 and reciprocal, the three
 * special-function operations per neighbour pair of the prior stencil, `iters` (1 .. 2^20) times
 * eight chains per thread on eight blocks of 256 threads per SM; h_ops_per_s receives those
 * operations per second over the timed launch (CUDA events on the context stream).  Synchronises.
 */
int tmbir_sfu_rate(tmbir_ctx* ctx, int iters, double* h_ops_per_s);

/*
 * Volumes larger than the device's memory (Sec. 2.4: the volume is partitioned along the
 * rotation axis, each partition keeps a halo of boundary slices for the 26-neighbour prior, and
 * a node scheduler overlaps host-device copies with the kernels).  The volume, its sinogram, R*g
 * and the iterates stay in host memory; the context's one geometry group is the slab, its
 * n_slices the slices the GPU holds at a time.  Slabs pass through the GPU in order in three
 * overlapping stages on three streams (copies in, kernels on the context stream, copies out)
 * with two device buffer sets.  Host buffers should be page-locked (cudaHostAlloc or
 * cudaHostRegister); pageable ones work but their copies do not overlap the kernels.  Both calls
 * return after their host outputs are written (they synchronise the three streams).  The context
 * stream must not be the legacy stream.
 *
 * tmbir_stream_workspace_size: bytes of the caller's device buffer d_swork (256-byte aligned)
 *   for a volume of n_slices slices with this context's slab: two buffer sets (x_k, x_{k-1},
 *   R*g and x_{k+1} of a slab with one halo slice each way, and a slab's sinogram), K (*) y of a
 *   slab, and the partial sums of the whole volume's pass-3b blocks (any slices-per-block choice).
 */
int tmbir_stream_workspace_size(const tmbir_ctx* ctx, int n_slices, size_t* bytes);

/*
 * R*g (Eq. 11) and 1/2 g.g of a host volume, and optionally the FBP start (Eq. 12), one slab
 * at a time through tmbir_build_operator (or tmbir_build_operator_fbp).
 *   h_sino  [n_slices][n_angles][n_det] FP32, host.
 *   h_atg   [n_slices][N][N] FP32, host (out).
 *   h_x0    [n_slices][N][N] FP32, host (out), or NULL for no FBP start.
 *   h_gtg   host double (out): 1/2 g.g of the volume, the slabs' sums added in slab order.
 * The setup transforms pair slices 2p and 2p + 1 of each slab, so with an even slab R*g is bit
 * for bit that of the resident volume.
 */
int tmbir_stream_build_operator(tmbir_ctx* ctx, int n_slices, const float* h_sino, float* h_atg, float* h_x0,
                                void* d_swork, size_t swork_bytes, double* h_gtg);

/*
 * tmbir_reconstruct on a host volume: prm->max_iter iterations (fewer when the gap rule stops
 * the run), the step constant from this geometry's lambda_max unless prm->L is given.
 *   h_x       [n_slices][N][N] FP32, host: x_0 in, the final iterate out.
 *   atg       R*g of the volume (tmbir_stream_build_operator) in host memory, or in device memory
 *             (16-byte aligned; read in place, so only the iterates stream); gtg_half its 1/2 g.g.
 *   h_work    2 n_slices N^2 floats of host scratch: with h_x, the three slots x_{k-1}, x_k and
 *             x_{k+1} rotate through.  After a number of iterations that is a multiple of 3 the
 *             final iterate is already in h_x; otherwise it is copied back into h_x through the
 *             device, slab by slab (one more pass of copies in and out).
 * Per iteration each slab copies in x_k and x_{k-1} (with one halo slice on each side) and its
 * R*g (when on the host), runs passes 1-3b on its own slices, and copies out x_{k+1}; the finalize kernel then
 * reduces the partial sums of all slabs in the order of the resident volume's pass-3b blocks, and
 * the host reads the stop flag.  The slices per pass-3b block are the slab's (tuned or default)
 * value lowered to a divisor of the slab; when the resident volume uses the same value, every
 * iterate equals tmbir_reconstruct's bit for bit.  Options as in tmbir_reconstruct, except that
 * use_graph is ignored and resume is refused (TMBIR_ERR_ARG); the iteration log (tmbir_get_log)
 * is kept; the state cannot be exported afterwards.
 */
int tmbir_stream_reconstruct(tmbir_ctx* ctx, int n_slices, float* h_x, const float* atg, double gtg_half,
                             float* h_work, void* d_swork, size_t swork_bytes, const tmbir_params* prm,
                             tmbir_stats* h_stats);

/* Wait for the context stream; reports a pending CUDA error. */
int tmbir_sync(tmbir_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TMBIR_H */
