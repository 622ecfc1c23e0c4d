/*
 * fot.h -- C ABI of the FOT (Fast Optimal Transport) dual-potential iteration on GB300
 * (sm_103a), after Torchylo, Swan, Tellez and Hogan, "A fast, large-scale optimal
 * transport algorithm for holographic beam shaping".
 *
 * The method (Sec. 2-3, Algorithm 1): given an input-beam amplitude g_jk and a target
 * amplitude G_LM on n_r x n_c pixel grids, run entropic Sinkhorn iterations
 *     u <- g^2 / (Lambda V Lambda)      (Eq. 7)
 *     V <- G^2 / (Lambda u Lambda)      (Eq. 8)
 * with the separable Gaussian kernel Lambda_jK = exp(-(j-K)^2 / (2 eps)), then recover the
 * phase from the first moments of the plan Gamma = u exp(-C/eps) V (Eqs. 9-10) and
 * integrate it with the trapezoid rule.  The library works in the log domain,
 * f = eps log u and psi = eps log V ("potentials", px^2 units), which is the same
 * iteration without exponent overflow.
 *
 * Conventions shared by every entry point
 *  - Images are row-major float32, rows x cols, element (j, k) at j*cols + k; row index j
 *    is the x axis, column index k the y axis (Sec. 2).  g and G share one shape.
 *  - Unless stated otherwise, pointers are DEVICE pointers on the context's device,
 *    owned by the caller; the context never keeps a caller pointer after a call returns.
 *  - eps is in px^2 (cost ((j-L)^2 + (k-M)^2)/2).  FOT_EPS_PAPER selects the paper's units,
 *    whose cost carries an extra 1/n^2 (Eq. 3): eps_px = n^2 * eps_paper, n = max(rows, cols).
 *  - All device work is enqueued on the context's stream and is asynchronous.  Argument
 *    errors are returned at once.  Errors found on the device (negative or non-finite
 *    amplitudes: FOT_EINVAL; zero total power: FOT_EMASS; a non-finite potential during
 *    the iteration: FOT_ENONFINITE) are latched in the context and returned by the next
 *    synchronising call (fot_sync, fot_potentials, fot_phase, fot_marginal_error), after
 *    which further enqueued work of that context is skipped until the next fot_solve or
 *    fot_set_problem clears the latch.
 *  - Zero-mass pixels (g = 0 or G = 0) carry potential -INFINITY.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef FOT_H_
#define FOT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fot_ctx fot_ctx;

typedef enum {
  FOT_OK = 0,
  FOT_EINVAL = 1,        /* bad argument, or negative / non-finite amplitude */
  FOT_ENOMEM = 2,        /* device or host allocation failed */
  FOT_ECUDA = 3,         /* a CUDA runtime call failed */
  FOT_ENONFINITE = 4,    /* a potential became NaN / +inf during the iteration */
  FOT_ETIMEOUT = 5,      /* a bounded device wait gave up */
  FOT_EMASS = 6,         /* g or G has zero total power */
  FOT_EUNSUPPORTED = 7,  /* precision or shape not supported by this build */
  FOT_ESTATE = 8         /* call out of order (e.g. fot_phase before fot_solve) */
} fot_status;

typedef enum {
  FOT_FP32 = 0,          /* FP32 on the CUDA cores, banded: every output sums only the terms
                            within 2^-40 of its largest (a provable window per 32-output
                            tile); for large eps the window sum is a tilted FP32 GEMM with
                            per-row max-offsets, for small eps an exact windowed
                            log-sum-exp */
  FOT_MIXED = 1,         /* the banded GEMM on tcgen05 tensor cores (split-BF16 operands,
                            FP32 accumulation in TMEM) with FP32 log-domain potentials */
  FOT_FP32_DENSE = 2,    /* FP32 on the CUDA cores, every output scans every term with its
                            own exact maximum (one exponential per term): the plain form */
  FOT_AUTO = 3,          /* batches only: time FOT_FP32 and FOT_MIXED on the batch when its
                            graph is built and keep the faster */
  FOT_BF16 = 4           /* the tensor-core banded GEMM of FOT_MIXED with single BF16
                            operands: one MMA per term instead of three; each product carries
                            up to 2^-7 relative error (both operands rounded to 8 significant
                            bits), so a half-step moves f or psi by at most 2^-6 eps (against
                            2^-15 eps for FOT_MIXED); single contexts only */
} fot_precision;

typedef enum { FOT_EPS_PX2 = 0, FOT_EPS_PAPER = 1 } fot_eps_units;

/* Create a context for rows x cols problems on `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Allocates all device scratch:
 * about 10 rows*cols float32 buffers plus small reduction scratch.
 * Returns FOT_EINVAL for rows or cols outside [1, 4096], FOT_ENOMEM on allocation failure. */
fot_status fot_create(fot_ctx** out, int rows, int cols, int precision, int device,
                      void* cuda_stream);

/* Release every device buffer of the context (synchronises its stream first). */
void fot_destroy(fot_ctx* ctx);

/* Replace the stream later calls enqueue on. */
fot_status fot_set_stream(fot_ctx* ctx, void* cuda_stream);

/* Load a problem (Sec. 2: marginal constraints g^2 and G^2): a = g^2 / sum g^2 and
 * b = G^2 / sum G^2 (both renormalised to unit mass) and their logs.  g, G: device,
 * rows x cols.  Clears the device error latch. */
fot_status fot_set_problem(fot_ctx* ctx, const float* g, const float* G);

/* Algorithm 1: load the problem (as fot_set_problem), set V = 1/(rows*cols), and run
 * `iters` iterations of Eqs. 7-8.  eps: host array of n_eps values; n_eps == 1 is a fixed
 * eps, n_eps == iters gives iteration t the value eps[t] (an annealing schedule; the
 * potentials keep px^2 units across changes).  dx: input-plane grid spacing used by
 * fot_phase (Sec. 2: x_j = (j - floor(n/2)) dx; dx <= 0 selects 1/sqrt(n), the paper's
 * units).  Stops after a fixed number of iterations (the paper's practice). */
fot_status fot_solve(fot_ctx* ctx, const float* g, const float* G, double dx,
                     const double* eps, int n_eps, int eps_units, int iters);

/* Continue the current problem for `iters` more iterations from the potentials the
 * context holds (checkpoint / resume).  Same eps rules as fot_solve. */
fot_status fot_resume(fot_ctx* ctx, const double* eps, int n_eps, int eps_units, int iters);

/* Algorithm 1 with a convergence stop.  Sec. 3 names the total variation of the
 * marginal-constraint violation as a convergence criterion; this call loads the problem and
 * starts as fot_solve, then runs at most max_iters iterations in blocks of check_every, and
 * after each block (and after the last allowed iteration) measures
 *     tv = sum_jk | (Gamma 1)_jk - a_jk |,   Gamma = exp((f + psi - C) / eps_t),
 * for the current iterate (f_t, psi_t); it stops at the first check with tv <= tol.  Right
 * after a V-half the column sums of Gamma equal b (up to rounding), so this source half is
 * the whole violation there.  The row sums are exp(f/eps + S(psi)) with S from one more
 * u-half on the context's own passes (its precision), reduced in FP64: a check costs one
 * half-step, two small reductions and one device-to-host read (synchronising).
 *   eps: n_eps == 1 (fixed) or n_eps == max_iters (iteration t uses eps[t]); eps_units and dx
 *   as in fot_solve.  max_iters >= 1, check_every >= 1, tol finite and >= 0, iters_out not
 *   NULL: else FOT_EINVAL.  *iters_out receives the iterations done, *tv_out (may be NULL) the
 *   last measured violation.  Afterwards the context holds the state fot_solve reaches after
 *   *iters_out iterations (fot_loop_time then covers the last block). */
fot_status fot_solve_tol(fot_ctx* ctx, const float* g, const float* G, double dx,
                         const double* eps, int n_eps, int eps_units, int max_iters, double tol,
                         int check_every, int* iters_out, double* tv_out);

/* Automatic eps (Sec. 5, the eps hyperparameter: as low as possible while the Sinkhorn
 * iterations stay stable).  Tries the n_cand candidate values cand[] in increasing order; for
 * each it runs, from the standard start, check_every iterations and then the rest of a probe of
 * probe_iters iterations (fot_solve + fot_resume in this context's precision, or cFOT from the
 * start for each part when use_cfot), measuring the marginal violation tv = sum |Gamma 1 - a|
 * (as fot_solve_tol) after the first part (tv1) and at the end (tv2).  A candidate is stable when
 * no potential became non-finite and tv2 <= (1 - min_decrease) tv1; the smallest stable one is
 * chosen.  *index_out receives its index in cand[] (-1 when none is stable), *tv_out (may be
 * NULL) its tv2; afterwards the context holds the last probe's iterate (the chosen candidate's
 * when one was found).  eps_units and dx as in fot_solve.  Errors: FOT_EINVAL (null pointers,
 * n_cand < 1, a candidate not finite and > 0, check_every < 1, probe_iters <= check_every,
 * min_decrease outside [0, 1)); FOT_EUNSUPPORTED (use_cfot on a shape cFOT does not take);
 * other errors of the solves are returned as they occur (a non-finite potential only rejects
 * its candidate). */
fot_status fot_select_eps(fot_ctx* ctx, const float* g, const float* G, double dx, const double* cand,
                          int n_cand, int eps_units, int probe_iters, int check_every,
                          double min_decrease, int use_cfot, int* index_out, double* tv_out);

/* Algorithm 1 between an input grid and an output grid of different sizes (Sec. 2: square,
 * equal arrays are not essential).  Both planes have unit pixel spacing and are centre-aligned,
 * x_j = j - (rows_in - 1)/2 and X_L = L - (rows_out - 1)/2 (columns likewise), so the cost
 * C_jkLM = ((x_j - X_L)^2 + (y_k - Y_M)^2)/2 still separates and each Lambda factor of Eqs. 7-8
 * is a rectangular rows_in x rows_out (cols_in x cols_out) matrix:
 *     f   = eps (log a - log(Lambda_r V Lambda_c^T))    on the input grid,
 *     psi = eps (log b - log(Lambda_r^T u Lambda_c))    on the output grid,
 * a = g^2/sum g^2, b = G^2/sum G^2, start V = 1/(rows_out cols_out).  Every axis pass is dense
 * and exact in FP32 (each output's own maximum, then the sum), as FOT_FP32_DENSE.
 *   g: rows_in x cols_in and G: rows_out x cols_out amplitudes, row-major FP32 device memory;
 *   eps in px^2 (n_eps == 1, or n_eps == iters for one value per iteration); f_out
 *   (rows_in x cols_in) and psi_out (rows_out x cols_out): device buffers of the caller that
 *   receive the potentials (px^2, -inf at zero mass); cuda_stream: the stream (NULL: default).
 * The call allocates and frees its temporaries (3 images and a few words) and synchronises the
 * stream before returning.  Errors: FOT_EINVAL (a null pointer, a size < 1 or > 3072,
 * iters < 1, n_eps other than 1 or iters, eps not finite and > 0), FOT_EMASS (g or G without
 * mass), FOT_ENOMEM, FOT_ENONFINITE (a non-finite potential), FOT_ECUDA. */
fot_status fot_solve_rect(const float* g, int rows_in, int cols_in, const float* G, int rows_out,
                          int cols_out, const double* eps, int n_eps, int iters, float* f_out,
                          float* psi_out, void* cuda_stream);

/* The same solve in FP64 throughout (a GPU reference form, for equal or unequal grids; FP64
 * inputs and outputs, sizes up to 1536 per axis, the arithmetic of the CUDA math library's
 * exp2 / log2 in double precision).  Arguments, ownership and errors as fot_solve_rect. */
fot_status fot_solve_rect_fp64(const double* g, int rows_in, int cols_in, const double* G, int rows_out,
                               int cols_out, const double* eps, int n_eps, int iters, double* f_out,
                               double* psi_out, void* cuda_stream);

/* cFOT (Sec. 3.1): the same problem, start and eps rules as fot_solve, but the iterations run
 * Algorithm 1 in the exponential domain with every Lambda product replaced by a linear
 * convolution with lambda_j = exp(-j^2 / (2 eps)), j = -(n-1) .. n-1, along the columns and
 * the rows, evaluated with FFTs (O(n^2 log n) per iteration instead of O(n^3)):
 *     u = a / (lambda * V * lambda),   V = b / (lambda * u * lambda),   V0 = 1/(rows*cols).
 * FP32 throughout.  Afterwards the context holds f = eps log u, psi = eps log V (px^2, -inf on
 * zero mass) and S_last = log(lambda * V_prev * lambda) of the last u-update, so fot_potentials,
 * fot_phase, fot_marginal_error and fot_intensity_loss apply; fot_backward does not
 * (FOT_ESTATE).  Like any exponential-domain iteration it fails once eps is small against the
 * spread of the potentials (u, V outside the FP32 range, or FFT rounding, a few ulp of a line's
 * largest value, swamping its small entries): a non-positive or non-finite convolution where
 * the marginal has mass latches FOT_ENONFINITE.  rows, cols in [2, 2048] (FFT length up to 4096;
 * else FOT_EUNSUPPORTED); iters >= 1.  Allocates a 32 KB spectrum buffer on its first call. */
fot_status fot_cfot_solve(fot_ctx* ctx, const float* g, const float* G, double dx,
                          const double* eps, int n_eps, int eps_units, int iters);

/* Wait for the context's stream; return the latched device status. */
fot_status fot_sync(fot_ctx* ctx);

/* Copy out f = eps log u and psi = eps log V (px^2; -INFINITY on zero mass).  Either
 * pointer may be NULL.  Synchronising. */
fot_status fot_potentials(fot_ctx* ctx, float* f_out, float* psi_out);

/* Load caller potentials (device, px^2) as the solver state, e.g. to resume from a
 * checkpoint taken with fot_potentials.  f may be NULL (only psi is read by the next
 * iteration). */
fot_status fot_set_potentials(fot_ctx* ctx, const float* f, const float* psi);

/* Phase retrieval (Eqs. 9-10 and the trapezoid "Integrate" step of Algorithm 1):
 *   dphidx_jk = (u/g^2)_jk sum_LM Lambda_jL X_L V_LM Lambda_kM,  dphidy likewise with Y_M,
 * with u from the last u-update and V the final V, X_L = (L - floor(rows/2)) / (rows dx),
 * Y_M = (M - floor(cols/2)) / (cols dx); phi (cycles) integrates them with the trapezoid
 * rule from phi = 0 at the grid centre, first down the centre column (k = floor(cols/2))
 * with dphidx, then along every row with dphidy.  Any output may be NULL.  Synchronising. */
fot_status fot_phase(fot_ctx* ctx, float* phi_out, float* dphidx_out, float* dphidy_out);

/* The same phase step from caller data: psi (target potential, px^2) and logsum_u (the
 * natural-log kernel sum S = log(Lambda V Lambda) of the u-update, so that u/g^2 = e^-S),
 * device rows x cols; eps in px^2; dx as in fot_solve (<= 0: 1/sqrt(n)).  Outputs as in
 * fot_phase (any may be NULL).  Synchronising. */
fot_status fot_moments(fot_ctx* ctx, const float* psi, const float* logsum_u, double eps,
                       double dx, float* phi_out, float* dphidx_out, float* dphidy_out);

/* Marginal violation of the current iterate, ||Gamma 1 - a||_1 + ||Gamma^T 1 - b||_1
 * (the total-variation convergence measure of Sec. 3, times two), from one extra exact
 * FP32 u-half-step evaluated on the stored potentials (never with the mixed-precision
 * kernels); accumulated in double.  Also returns the entropic dual objective
 * <f,a> + <psi,b> - eps sum Gamma + eps when dual_out != NULL.  Synchronising. */
fot_status fot_marginal_error(fot_ctx* ctx, double* l1_out, double* dual_out);

/* L1 intensity loss of a phase solution (Sec. 5, the loss of the eps sweep):
 *   loss = sum_LM | I_LM - b_LM |,   I = |F[g e^{2 pi i phi}]|^2 / sum_LM |F[g e^{2 pi i phi}]|^2,
 * for the loaded problem's input beam g (taken as sqrt(a), a = g^2 / sum g^2: the scale
 * cancels), the phase phi (device, rows x cols, in cycles, e.g. from fot_phase), the target
 * b = G^2 / sum G^2, and F the 2-D DFT between the centred grids of Sec. 2:
 *   F[h]_LM = sum_jk h_jk exp(-2 pi i ((j - r/2)(L - r/2)/rows + (k - c/2)(M - c/2)/cols)),
 * r = rows, c = cols (x_j = (j - rows/2) dx, X_L = (L - rows/2) dX with dx dX = 1/rows).
 * rows and cols must be powers of two in [2, 4096] (else FOT_EUNSUPPORTED); phi and loss_out
 * not NULL (else FOT_EINVAL); a problem loaded by fot_solve / fot_set_problem (else
 * FOT_ESTATE).  intensity_out (device, rows x cols, may be NULL) receives I.  Uses the
 * context's scratch buffers, not its potentials; FP32 transforms, FP64 sums.  Synchronising. */
fot_status fot_intensity_loss(fot_ctx* ctx, const float* phi, double* loss_out, float* intensity_out);

/* One half-step from caller potentials, for verification and custom loops:
 *   fot_u_update: f = eps (log a - S), S = log(Lambda exp(psi/eps) Lambda)   (Eq. 7)
 *   fot_v_update: psi = eps (log b - T), T = log(Lambda exp(f/eps) Lambda)   (Eq. 8)
 * using the problem last loaded.  pot_in, pot_out: device rows x cols px^2; logsum_out
 * (S or T, natural log) may be NULL.  eps in px^2. */
fot_status fot_u_update(fot_ctx* ctx, const float* psi_in, double eps, float* f_out,
                        float* logsum_out);
fot_status fot_v_update(fot_ctx* ctx, const float* f_in, double eps, float* psi_out,
                        float* logsum_out);

/* Allocation-free u-update.  The paper has no counterpart: this entry point exists for
 * callers that must not allocate device memory once they are running, for example a
 * real-time hologram loop that reserves all of its memory at start-up because cudaMalloc
 * can synchronise the device and stall the loop, or a plug-in whose host owns every
 * device allocation through its own allocator.  It gives the same mathematical result as
 * fot_u_update, f = eps (log_a - S) with S = log(Lambda exp(psi/eps) Lambda), but through
 * a different kernel: the dense exact FP32 pass of FOT_FP32_DENSE (every output scans every
 * term, one exponential each: O(rows * cols * (rows + cols)) work, much slower than the
 * banded or tensor-core passes of fot_u_update at large sizes; results agree to FP32
 * rounding).  It needs no fot_ctx: the caller passes every input and output (device,
 * rows x cols float32: psi_in in px^2, log_a = natural log of the normalised source marginal
 * a = g^2/sum g^2, -INFINITY where a = 0; f_out; logsum_out may be NULL), and the
 * intermediate lives in a static device array of FOT_NOALLOC_MAX_PIXELS floats (4 MiB) that
 * every GPU loading this library holds until the process exits.  Nothing is allocated: no
 * cudaMalloc, no cudaFree, no allocating library call.
 *  - rows * cols > FOT_NOALLOC_MAX_PIXELS, or rows / cols outside [1, 4096]: FOT_EINVAL.
 *  - Runs on the current device, enqueued on cuda_stream (NULL = legacy default stream);
 *    asynchronous.  Nothing is read back, so device-side problems are not reported as a
 *    status: a non-finite result shows up as a non-finite value in f_out.
 *  - The first call on a device does a one-time set-up with that device current: it looks
 *    up the static array's device address (cudaGetSymbolAddress) and raises the pass
 *    kernels' shared-memory limit; make that first call before any stream capture begins.
 *    The host-side cache of that set-up is not thread-safe for a device's first call.
 *  - Every call shares the one array and it keeps the last call's contents: calls whose
 *    work overlaps on the GPU (different streams, or different host threads) race on it. */
#define FOT_NOALLOC_MAX_PIXELS (1024 * 1024)
fot_status fot_u_update_noalloc(const float* psi_in, const float* log_a, int rows, int cols,
                                double eps, float* f_out, float* logsum_out, void* cuda_stream);

/* Batched solve: `count` (<= 64) independent problems of their own grid sizes, solved
 * together (Algorithm 1 for each).  Every axis pass of every problem runs in the same
 * multi-problem launches, and the whole solve (setup and all iterations) is captured once
 * into a CUDA graph that each fot_batch_solve replays with one graph launch; the graph is
 * rebuilt when the input pointers, the schedule or the iteration count change.  rows, cols:
 * host arrays of count sizes; precision FOT_FP32, FOT_MIXED or FOT_AUTO.  The batch owns one
 * fot_ctx per problem (fot_batch_context), through which the results are read with
 * fot_potentials / fot_phase / fot_marginal_error. */
typedef struct fot_batch fot_batch;
fot_status fot_batch_create(fot_batch** out, int count, const int* rows, const int* cols,
                            int precision, int device, void* cuda_stream);
void fot_batch_destroy(fot_batch* batch);
fot_ctx* fot_batch_context(fot_batch* batch, int index);

/* g, G: host arrays of `count` device pointers (problem q is rows[q] x cols[q]); eps: host
 * array [count][n_eps] (n_eps == 1 fixed, == iters a per-iteration schedule, per problem);
 * dx as in fot_solve.  Asynchronous; errors per problem through its context. */
fot_status fot_batch_solve(fot_batch* batch, const float* const* g, const float* const* G,
                           double dx, const double* eps, int n_eps, int eps_units, int iters);

/* Kernels per graph launch and whether the tensor-core form was chosen (FOT_AUTO). */
fot_status fot_batch_info(fot_batch* batch, int64_t* kernels_per_solve, int* tensor_path);

/* Reverse-mode gradient of a scalar loss L of the phase and/or the final potentials of the
 * last fot_solve (Algorithm 1 from its standard start, any eps schedule) with respect to the
 * amplitudes g and G, through every unrolled iteration (Eqs. 7-8), the moments (Eqs. 9-10),
 * the trapezoid integration and the normalisation a = g^2/sum g^2, b = G^2/sum G^2.
 * g, G: the device amplitudes of that solve; dL_dphi, dL_df, dL_dpsi: device rows x cols
 * seeds (each may be NULL = 0); dL_dg, dL_dG: device outputs (0 where the amplitude is 0).
 * The forward is recomputed from potentials checkpointed every checkpoint_every iterations,
 * holding one segment (4 images per iteration) at a time; temporary device memory is
 * allocated for the call.  Invalidated by fot_set_potentials.  Synchronising. */
fot_status fot_backward(fot_ctx* ctx, const float* g, const float* G, const float* dL_dphi,
                        const float* dL_df, const float* dL_dpsi, int checkpoint_every,
                        float* dL_dg, float* dL_dG);

/* Exact c-transform, the eps -> 0 limit of a half-step (the log a term vanishes):
 *   out_jk = min_LM [ ((j-L)^2 + (k-M)^2)/2 - pot_LM ],
 * by a lower envelope of parabolas along each row, then along each column.  -INFINITY
 * entries of pot are excluded; rows x cols device buffers, px^2. */
fot_status fot_c_transform(fot_ctx* ctx, const float* pot_in, float* out);

/* End-to-end convenience: HOST float32 g, G in; HOST float32 phi out (rows x cols).
 * Copies in, runs fot_solve and fot_phase, copies out; synchronising. */
fot_status fot_solve_phase_host(fot_ctx* ctx, const float* g_host, const float* G_host,
                                double dx, const double* eps, int n_eps, int eps_units,
                                int iters, float* phi_host);

/* Number of kernels this context has launched since creation (for launch accounting). */
int64_t fot_launch_count(const fot_ctx* ctx);

/* Device time (CUDA events on the context stream) of the Sinkhorn loop of the last
 * fot_solve / fot_resume, and the number of kernels it launched (only axis-pass kernels and
 * their window plans run inside that loop).  Synchronises with the end of the loop. */
fot_status fot_loop_time(fot_ctx* ctx, double* ms_out, int64_t* passes_out);

/* Number of (row, output, summation index) terms the axis passes of this context have
 * evaluated since creation: rows*len*len per dense pass, the window sizes for banded passes
 * (each term is one multiply-add of the exp-domain contraction); tensor_terms_out (may be
 * NULL) receives the part computed on the tensor cores (each term there is three BF16
 * multiply-adds of the split-precision product).  Synchronising. */
fot_status fot_work_count(fot_ctx* ctx, int64_t* terms_out, int64_t* tensor_terms_out);

/* The same count split by where the terms were evaluated: out4[0] banded tilted-GEMM items
 * (CUDA-core FFMA), out4[1] banded exact-window items (one exponential per term), out4[2]
 * tensor cores, out4[3] dense exact passes (including the phase step's moment passes).
 * Synchronising.  The paper has no counterpart: a measurement aid. */
fot_status fot_work_split(fot_ctx* ctx, int64_t* out4);

/* Kernel classes of fot_kernel_times. */
enum {
  FOT_KERNEL_PLAN = 0,     /* window plan of a banded pass (and the B-operand table of the
                              tensor-core pass, written when eps changes) */
  FOT_KERNEL_BAND = 1,     /* banded pass on the CUDA cores (tilted-GEMM and exact-window items) */
  FOT_KERNEL_TENSOR = 2,   /* tensor-core banded pass */
  FOT_KERNEL_DENSE = 3,    /* dense exact pass */
  FOT_KERNEL_CLASSES = 4
};

/* Per-kernel timing of the Sinkhorn loop (a measurement aid; the paper has no counterpart).
 * With on != 0, every kernel the loop of later fot_solve / fot_resume calls launches is
 * bracketed by a pair of CUDA events on the context stream (a few microseconds of host time
 * per launch; the events are created on first use and reused).  on = 0 synchronises the
 * stream and releases the events.  Not for calls captured into a CUDA graph. */
fot_status fot_set_kernel_timing(fot_ctx* ctx, int on);

/* Device time (ms) and launch count per kernel class (arrays of FOT_KERNEL_CLASSES) over
 * every loop since timing was switched on or last read; resets the sums.  FOT_ESTATE when
 * timing is off, FOT_ECUDA when an event could not be created or recorded (the sums are
 * then dropped).  Synchronising. */
fot_status fot_kernel_times(fot_ctx* ctx, double* ms_out, int64_t* launches_out);

const char* fot_status_string(fot_status s);

#ifdef __cplusplus
}
#endif

#endif /* FOT_H_ */
