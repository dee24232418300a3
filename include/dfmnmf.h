/*
 * dfmnmf.h -- C ABI of the GB300 (sm_103a) distributed FastMNMF library.
 *
 * Distributed FastMNMF (arXiv 2605.19388) separates N sources observed by K
 * subarrays of M_k microphones.  The spatial covariance of each source is
 * block diagonal over subarrays and jointly diagonalised inside each block
 * (Sec. III-B); the source PSDs follow an NMF model shared by all subarrays
 * (Eq. 2).  One majorisation-minimisation (MM) iteration is the iterative
 * projection of every diagonaliser block (Eqs. 13-15) followed by the
 * multiplicative updates of the NMF bases, activations and diagonal SCM
 * entries (Eqs. 8-10, with the microphone index taken over all subarrays as
 * stated after Eq. 15).
 *
 * Symbols used in this header (paper symbol in brackets):
 *   f < F frequency bin [i], t < T frame [j], k < K subarray [l],
 *   m < M global microphone, mu < M_k microphone inside subarray k [mu],
 *   o_k = M_0 + ... + M_{k-1} first global microphone of subarray k,
 *   n < N source [n], b < B NMF basis [k],
 *   W[n][f][b] spectral basis [t_ikn], H[n][b][t] activation [v_kjn],
 *   lambda[n][f][t] = sum_b W H source PSD [h_ijn] (Eq. 2),
 *   g[f][n][m] diagonal SCM entry [(Lambda_in)_mm] (Eq. 3, Eq. 10),
 *   Q_f = blkdiag(Q_f0..Q_f,K-1) diagonaliser [W_i^H]; row mu of block k is
 *   w_{i mu}^(l) H, so y_ftk = Q_fk x_ftk (Sec. III-B),
 *   yhat[f][t][m] = max(sum_n lambda g, eps) model variance [eta_ijm],
 *   P[f][t][m] = |y_ftm|^2 projected power [|y_ijm|^2],
 *   V[f][k][mu] = (1/T) sum_t x_ftk x_ftk^H / yhat_ft(o_k+mu)  [Q_{i mu}^(l), Eq. 13].
 *
 * Memory conventions
 *   - All pointers named *_dev are CUDA device pointers (or managed memory)
 *     unless the comment says "host or device": those are copied with
 *     cudaMemcpyAsync(cudaMemcpyDefault), so pinned or pageable host memory
 *     works as well.  The caller owns every pointer it passes; the library
 *     never keeps one after the call returns (x is copied at init).
 *   - complex64 = interleaved float (re, im); complex128 = interleaved double.
 *   - Arrays are C-contiguous in the index order written.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     enqueued on it; only dfmnmf_loglik and dfmnmf_get_params(host) block.
 *
 * Errors
 *   Every entry point returns a dfmnmf_status; nothing throws or traps.  The
 *   message of the last failure on the calling thread is returned by
 *   dfmnmf_last_error().  A non-finite value produced by an update sets a
 *   device flag that the next dfmnmf_loglik reports as DFMNMF_ENUMERIC.
 *
 * Limits of this release
 *   All subarrays must have the same size M_k in 1..4 (the paper's layout is
 *   three 4-microphone subarrays), or K = 1 with M_k = 16 or 32:
 *   conventional all-microphone FastMNMF with a full 16 x 16 or 32 x 32
 *   diagonaliser (Sec. II-A), which the distributed form reduces to at K = 1
 *   and which is its comparator (FP32 form only; no cost gradient at
 *   M_k = 32); other layouts return DFMNMF_EINVAL.
 *   1 <= N <= 16, 1 <= B <= 64, 1 <= K <= 16, F >= 1, T >= 1.
 */
#ifndef DFMNMF_H
#define DFMNMF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DFMNMF_VERSION 100

typedef struct dfmnmf_ctx dfmnmf_ctx; /* opaque, owned by the library */

typedef enum dfmnmf_status {
  DFMNMF_OK = 0,
  DFMNMF_EINVAL = 1,   /* bad argument, size or layout; nothing was enqueued */
  DFMNMF_ENOMEM = 2,   /* device allocation failed */
  DFMNMF_ECUDA = 3,    /* a CUDA runtime call failed (message has the detail) */
  DFMNMF_ENUMERIC = 4, /* a NaN or Inf was produced by an update */
  DFMNMF_ETIMEOUT = 5  /* a bounded device wait gave up (see DFMNMF_OPT_WAIT_CYCLES);
                          destroy the context afterwards                       */
} dfmnmf_status;

/* Arithmetic of the weighted-covariance contraction (Eq. 13). */
typedef enum dfmnmf_precision {
  DFMNMF_FP32 = 0,    /* CUDA cores: x x^H and the weights as exact float pairs
                         (float-float sums), for ill-conditioned covariances     */
  DFMNMF_BF16_TC = 1, /* tensor cores (tcgen05 kind::f16): x x^H and 1/yhat each
                         split in two bfloat16 parts (hi = round to nearest,
                         lo = rest), all four products, FP32 accumulation;
                         M_k = 4 with K in {1, 2, 4, 8}                         */
  DFMNMF_TF32_TC = 2  /* tensor cores (tcgen05 kind::tf32): the same split with
                         TF32 parts (hi = round to nearest TF32, lo = rest), the
                         parts side by side on the contraction axis; same
                         layouts.  Measured about three times less accurate than
                         the bfloat16 form on the 4 x 4-mic workload.  In both
                         tensor-core forms the NMF products run on the CUDA
                         cores unless DFMNMF_OPT_WUPD_TC moves the W update's
                         onto the tensor cores                                  */
} dfmnmf_precision;

/* Arithmetic of the M_k x M_k iterative-projection solves (Eqs. 14-15). */
typedef enum dfmnmf_ip_arith {
  DFMNMF_IP_F64 = 0,   /* native IEEE binary64                            */
  DFMNMF_IP_F32X2 = 1, /* float-float pairs (Dekker/Knuth), ~48-bit mantissa */
  DFMNMF_IP_F32 = 2    /* plain binary32 (for precision studies only)     */
} dfmnmf_ip_arith;

typedef struct dfmnmf_desc {
  int F, T, K;        /* bins, frames, subarrays                               */
  const int* mics;    /* host array of K block sizes M_k; M = sum M_k          */
  int N, B;           /* sources, NMF bases per source                          */
  int precision;      /* dfmnmf_precision                                      */
  int ip_arith;       /* dfmnmf_ip_arith                                       */
  double floor_eps;   /* floor of yhat, MU denominators, IP normaliser (Sec. IV-A: 1e-6); <= 0 means 1e-6;
                         below the smallest normal float (about 1.2e-38) it is raised to that value */
} dfmnmf_desc;

/*
 * Create a context and its state (Sec. III-B model, Eq. 2 and Eq. 3).
 *   x       complex64 [F][T][M], host or device; copied, microphones of one
 *           subarray contiguous (Sec. III-B).
 *   W0      float32 [N][F][B] > 0, H0 float32 [N][B][T] > 0,
 *   g0      float32 [F][N][M] > 0   (host or device; Sec. IV-A: strictly positive).
 *   Q0      complex128 [F][sum_k M_k^2] (block k row-major M_k x M_k, blocks in
 *           subarray order), host or device; NULL means identity blocks.
 * On success *out owns all device state (about 8 F T M + 12 F T M + 16 F T N
 * bytes); free it with dfmnmf_destroy.  EINVAL on a bad descriptor.
 */
int dfmnmf_init(dfmnmf_ctx** out, const dfmnmf_desc* desc, const void* x,
                const float* W0, const float* H0, const float* g0, const void* Q0,
                void* stream);

/* Replace the observation x (same shape), host or device. */
int dfmnmf_set_observation(dfmnmf_ctx* ctx, const void* x, void* stream);

/*
 * Run n_iter MM iterations (Sec. III-B: IP of every block by Eqs. 13-15 with
 * rows mu in ascending order, then Eq. 8, Eq. 9, Eq. 10, the model refreshed
 * after each rule).  Asynchronous; n_iter = 0 is a no-op; n_iter < 0 EINVAL.
 */
int dfmnmf_iterate(dfmnmf_ctx* ctx, int n_iter, void* stream);

/* Stages of one iteration, for step-by-step checking.  Running the five in
 * order equals one dfmnmf_iterate step. */
typedef enum dfmnmf_stage {
  DFMNMF_STAGE_COV = 1, /* yhat from the current model; V (Eq. 13)              */
  DFMNMF_STAGE_IP = 2,  /* Q rows by Eqs. 14-15                                 */
  DFMNMF_STAGE_W = 3,   /* P = |Q x|^2, W by Eq. 8, lambda refreshed           */
  DFMNMF_STAGE_H = 4,   /* H by Eq. 9, lambda refreshed                         */
  DFMNMF_STAGE_G = 5    /* g by Eq. 10                                          */
} dfmnmf_stage;
int dfmnmf_run_stage(dfmnmf_ctx* ctx, int stage, void* stream);

/*
 * Negative log-likelihood of Eq. (12) at the current state:
 *   sum_{f,t,m} (P/yhat + ln yhat) - T sum_f sum_k ln |det Q_fk|^2
 * (no F T M ln(pi) constant).  The data term is accumulated in FP64, the
 * log-determinants by FP64 LU.  Synchronises `stream`.  ENUMERIC when a
 * non-finite value was produced since init or the result is not finite.
 */
int dfmnmf_loglik(dfmnmf_ctx* ctx, double* nll_host, void* stream);

/*
 * Multichannel Wiener filter applied inside each subarray (Sec. III-B, last
 * step): c_nft,(k) = Q_fk^{-1} diag(lambda_nft g_fn(o_k+mu) / yhat_ft(o_k+mu)) Q_fk x_ftk.
 *   c_out   complex64 [N][F][T][M], device, caller-owned (8 N F T M bytes).
 * Q_fk^{-1} is formed in FP64.
 */
int dfmnmf_separate(dfmnmf_ctx* ctx, void* c_out_dev, void* stream);

/*
 * Copy the state out / in (checkpoint and resume).  Any pointer may be NULL
 * to skip that array; host or device.  Layouts as for dfmnmf_init; Q is
 * complex128.  set_params refreshes lambda.  get_params synchronises `stream`
 * when a destination is host memory.
 */
int dfmnmf_get_params(dfmnmf_ctx* ctx, void* Q, float* W, float* H, float* g, void* stream);
int dfmnmf_set_params(dfmnmf_ctx* ctx, const void* Q, const float* W, const float* H,
                      const float* g, void* stream);

/* Intermediate buffers (for step-by-step checks), copied to host or device:
 *   DFMNMF_BUF_V      complex128 [F][K][M_k][M_k][M_k]  (V[f][k][mu][a][b])
 *   DFMNMF_BUF_P      float32   [F][T][M]
 *   DFMNMF_BUF_LAMBDA float32   [N][F][T]
 * Contents are those left by the last stage that wrote them. */
typedef enum dfmnmf_buffer { DFMNMF_BUF_V = 1, DFMNMF_BUF_P = 2, DFMNMF_BUF_LAMBDA = 3 } dfmnmf_buffer;
int dfmnmf_get_buffer(dfmnmf_ctx* ctx, int which, void* dst, size_t dst_bytes, void* stream);

/* Number of kernel launches one dfmnmf_iterate step enqueues. */
int dfmnmf_launches_per_iteration(const dfmnmf_ctx* ctx);

/*
 * Profiling aid: run n_iter >= 1 iterations, each one CUDA graph of the
 * iteration's kernels launched band-wide one after another with a timing
 * event after every kernel (so host launch latency is not counted), and
 * return the mean duration in milliseconds of each kernel of an iteration
 * (avg_ms[i], including the launch gap before it) and its name (names[i],
 * static strings; names may be NULL; a kernel launched twice per iteration
 * appears twice).  *count receives the number of kernels; cap is the
 * capacity of both arrays (EINVAL if smaller).  Advances the state by n_iter
 * iterations.  Synchronises `stream`.
 */
int dfmnmf_kernel_times(dfmnmf_ctx* ctx, int n_iter, double* avg_ms, const char** names, int cap,
                        int* count, void* stream);

/*
 * Profiling aid: each kernel of the iteration alone, `reps` >= 1 band-wide
 * launches back to back in one CUDA graph timed by two events (after one
 * warm-up replay); avg_ms[i] is the mean duration of one launch, including
 * the gap between launches but no timing event.  Names and counts as for
 * dfmnmf_kernel_times.  The repeated launches change the state (an IP or MU
 * kernel applied reps times): restore it with dfmnmf_set_params afterwards.
 * Synchronises `stream`.
 */
int dfmnmf_kernel_times_isolated(dfmnmf_ctx* ctx, int reps, double* avg_ms, const char** names, int cap,
                                 int* count, void* stream);

void dfmnmf_destroy(dfmnmf_ctx* ctx);

/*
 * Gradient of the cost of Eq. (12) at the context's current state (no
 * iteration is taken, nothing of the state changes; the intermediate
 * buffers V, P and lambda are overwritten).  With y = sum_n lambda g and
 * G = 1/y - P/y^2 (zero where the floor of Sec. IV-A holds):
 *   dW[n][f][b] = sum_t H[n][b][t] sum_m g[f][n][m] G[f][t][m]   float32 [N][F][B]
 *   dH[n][b][t] = sum_f W[n][f][b] sum_m g[f][n][m] G[f][t][m]   float32 [N][B][T]
 *   dg[f][n][m] = sum_t lambda[n][f][t] G[f][t][m]                float32 [F][N][M]
 *   dQ          = dL/dRe Q + i dL/dIm Q, block by block,          complex128 like Q:
 *                 dQ[mu][j] = 2 T ((Q V_mu)[mu][j] - conj(Q^{-1})[j][mu])
 * (the first three are the differences denominator - numerator of the
 * multiplicative rules, Eqs. 8-10).  Computed from float-float covariances
 * and compensated projections whatever the precision of the context; the
 * inverse and the Q gradient in FP64.  Any output may be NULL; host or
 * device memory.  *nll_host (may be NULL) receives Eq. (12), and then the
 * call synchronises `stream` and reports DFMNMF_ENUMERIC as dfmnmf_loglik
 * does.  Blocks of 32 microphones return DFMNMF_EINVAL.
 */
int dfmnmf_cost_gradient(dfmnmf_ctx* ctx, void* dQ, float* dW, float* dH, float* dg, double* nll_host,
                         void* stream);

/*
 * Launch shapes picked by measurement (no counterpart in the paper; a GPU
 * concern): in the FP32 form the per-frequency kernels of an iteration run
 * either band-wide on one graph branch or as two halves of the band on two
 * branches (*branches = 1 or 2); in the tensor-core form they stay on one
 * branch (*branches = 1) and the persistent covariance kernel runs with one
 * or two groups of converter warps instead; the split NMF products of
 * Eqs. (8)-(9) aim for 2, 4 or 8 CTAs per SM (*nmf_ctas).  Every combination is timed over
 * iters_per_trial >= 1 replays of the captured iteration (after one warm-up
 * replay); the fastest is kept for this context.  The trials advance a copy
 * of the state only: Q, W, H, g and the device flags are restored, so the
 * call leaves the iterate where it was.  Allocates four temporary device
 * arrays of the state's size.  branches / nmf_ctas may be NULL.
 * Synchronises `stream`.  Results are identical under every choice up to
 * rounding (the split changes the order of the NMF sums).
 */
int dfmnmf_autotune(dfmnmf_ctx* ctx, int iters_per_trial, int* branches, int* nmf_ctas, void* stream);

/*
 * Launch options of a context, set by hand (no counterpart in the paper; a
 * GPU concern).  dfmnmf_autotune sets the first three by measurement.
 *   DFMNMF_OPT_BRANCHES    1 or 2 graph branches for the per-frequency kernels
 *                          (FP32 form; the tensor-core forms use 1)
 *   DFMNMF_OPT_NMF_CTAS    2, 4 or 8: CTAs per SM the split NMF products (the H
 *                          update, and the W update where it is not fused) aim for
 *   DFMNMF_OPT_VX_GROUPS   1 or 2 groups of converter warps in the tensor-core
 *                          covariance kernel
 *   DFMNMF_OPT_WUPD_TC     0: the W update (Eq. 8) on the CUDA cores, fused with
 *                          the refresh of lambda where its shared-memory tile
 *                          fits (otherwise split products and a separate
 *                          refresh); 1: its products on the tensor cores
 *                          (tcgen05 kind::tf32) and a separate refresh, for
 *                          the tensor-core forms only
 *   DFMNMF_OPT_WAIT_CYCLES budget, in SM clock cycles (default 2e9, ~1 s), of
 *                          the pipeline waits of the tensor-core covariance
 *                          kernel; a wait that runs out ends the kernel with
 *                          DFMNMF_ETIMEOUT reported by the next synchronising
 *                          call (the kernel still waits, with the full budget,
 *                          for its copies and tensor-core work in flight before
 *                          it exits).  A small value makes the failure path
 *                          testable; the context is not usable afterwards.
 * Results are identical under every choice up to rounding.  Takes effect at the
 * next captured iteration (the captured graph is rebuilt).  DFMNMF_EINVAL for
 * an unknown option or value; DFMNMF_OPT_WUPD_TC = 1 on the FP32 form is
 * EINVAL.  dfmnmf_get_option returns the value, or -1.
 */
enum { DFMNMF_OPT_BRANCHES = 1, DFMNMF_OPT_NMF_CTAS = 2, DFMNMF_OPT_VX_GROUPS = 3, DFMNMF_OPT_WUPD_TC = 4,
       DFMNMF_OPT_WAIT_CYCLES = 5 };
int dfmnmf_set_option(dfmnmf_ctx* ctx, int option, int value);
int dfmnmf_get_option(const dfmnmf_ctx* ctx, int option);

/*
 * Many mixtures, one CUDA graph launch per iteration (no counterpart in the
 * paper).  dfmnmf_batch_create captures (if not done yet) each context's
 * iteration and places them as independent child graphs of one graph; the
 * contexts may have different sizes and layouts (each keeps its own state,
 * precision and launch shapes).  dfmnmf_batch_iterate advances every
 * mixture by n_iter iterations (asynchronous on `stream`), exactly as
 * dfmnmf_iterate on each context would.  The batch refers to the contexts
 * without owning them: destroy it before any of them, and create it after
 * dfmnmf_autotune (it copies the iteration graphs as they are at creation).
 * All contexts must live on one device.  EINVAL on a NULL or empty list.
 */
typedef struct dfmnmf_batch dfmnmf_batch;
int dfmnmf_batch_create(dfmnmf_batch** out, dfmnmf_ctx* const* ctxs, int count);
int dfmnmf_batch_iterate(dfmnmf_batch* batch, int n_iter, void* stream);
void dfmnmf_batch_destroy(dfmnmf_batch* batch);

/*
 * Initialisation from given source images, Sec. IV-A steps 3, 5 and 6 (the
 * soft masks that produce the images, step 2, and the IS-NMF of step 4 are
 * left to the caller):
 *   c_img  complex64 [N][F][T][M] device memory, the images c_nft (the
 *          layout dfmnmf_separate writes);
 *   h_out  float32 [N][F][T] device memory, or NULL to skip it:
 *          h[n][f][t] = c_nft^H R_fn^{-1} c_nft / M with
 *          R_fn = sum_t c_nft c_nft^H / T (step 3);
 *   the context's Q becomes, block by block, the generalised eigenvectors w
 *   of the pair (R_f,N-2^(k), R_f,N-1^(k)) of the last two sources'
 *   diagonal blocks -- ascending eigenvalues, each w scaled so that
 *   w^H R_f,N-1^(k) w = 1, row mu of Q_fk = w_mu^H (step 5) -- and
 *   g[f][n][o_k + mu] = w_mu^H R_fn^(k) w_mu (step 6).  W and H are kept.
 * Each eigenvector is fixed up to a unit phase factor (any choice is a
 * generalised eigenvector); the cost of Eq. (12) and every update do not
 * depend on it.  R is summed from exact products in float pairs and
 * factorised in FP64 (Cholesky of R_f,N-1^(k), cyclic complex Jacobi
 * rotations); h applies a single-precision L^{-1}.  Needs N >= 2 and
 * M <= 32 (EINVAL otherwise, and for host pointers).  Allocates stream-
 * ordered scratch of N F M^2 * 24 bytes; synchronises `stream`; ENUMERIC if
 * some R_fn (with h) or R_f,N-1^(k) is not positive definite, in which case
 * the affected values are not meaningful.
 */
int dfmnmf_init_from_images(dfmnmf_ctx* ctx, const void* c_img, float* h_out, void* stream);

/*
 * Gradient through unrolled iterations (no counterpart in the paper; it lets
 * a learned model upstream of the separator be trained through it).
 * dfmnmf_adjoint_create prepares, for a context of the FP32 form with
 * subarrays of 1 to 4 microphones, the workspace of a reverse pass through
 * n_iter >= 0 iterations that stores the state every `every` >= 1
 * iterations and recomputes each segment from its checkpoint during the
 * reverse sweep (ceil(n_iter / every) + every + 1 stored states).
 * dfmnmf_adjoint_run then takes the context's current state as the initial
 * state s0 = (Q0, W0, H0, g0), runs n_iter iterations exactly as
 * dfmnmf_iterate does (the context is left at the final state s_T), and
 * returns the loss of s_T and its gradient with respect to s0:
 *   loss DFMNMF_LOSS_NLL          Eq. (12) of s_T (no F T M ln(pi) constant);
 *   loss DFMNMF_LOSS_WIENER_MSE   mean over (n, f, t, m) of |c_n - c_true_n|^2,
 *                                 c_n the Wiener filter output of s_T (as
 *                                 dfmnmf_separate), source n matched to
 *                                 c_true[n]; c_true complex64 [N][F][T][M]
 *                                 device memory.
 * Outputs (each may be NULL; host or device memory): *loss_host,
 *   dQ0 complex128 [F][sum M_k^2] (dL/dRe Q + i dL/dIm Q, Q's layout),
 *   dW0 float64 [N][F][B], dH0 float64 [N][B][T], dg0 float64 [F][N][M].
 * The reverse pass is written out by hand (the transpose of each step's
 * linearisation, FP64, the floors of Sec. IV-A passing no gradient where
 * they hold) around the forward values recomputed in FP64 from the stored
 * FP32-form states.  It needs every IP system to be nonsingular: a system
 * below the singular threshold returns DFMNMF_ENUMERIC (the gradient is not
 * defined there).  Synchronises `stream`.  The workspace refers to the
 * context without owning it: destroy it first.
 */
typedef struct dfmnmf_adj dfmnmf_adj;
enum { DFMNMF_LOSS_NLL = 1, DFMNMF_LOSS_WIENER_MSE = 2 };
int dfmnmf_adjoint_create(dfmnmf_adj** out, dfmnmf_ctx* ctx, int n_iter, int every);
int dfmnmf_adjoint_run(dfmnmf_adj* adj, int loss, const void* c_true, double* loss_host, void* dQ0,
                       double* dW0, double* dH0, double* dg0, void* stream);
void dfmnmf_adjoint_destroy(dfmnmf_adj* adj);

/*
 * Allocation-free negative log-likelihood.  The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory
 * when they need the cost -- for example an audio engine's real-time thread,
 * where cudaMalloc can block and synchronise the whole device and so break
 * the thread's deadline, or a plug-in whose host application owns the GPU
 * memory budget and forbids allocations by guests.  It returns the same value
 * dfmnmf_loglik returns for the same state, computed from arrays the caller
 * already holds in device memory, and needs no context:
 *   desc         F, T, K, mics, N, B and floor_eps as for dfmnmf_init
 *                (precision and ip_arith are ignored; floor_eps <= 0 means
 *                1e-6),
 *   x_dev        complex64 [F][T][M], Q_dev complex128 [F][sum M_k^2],
 *   W_dev        float32 [N][F][B], H_dev float32 [N][B][T],
 *   g_dev        float32 [F][N][M] (all device memory, caller-owned, read
 *                only),
 *   nll_host     receives the cost (the call synchronises `stream`).
 * Limits, each returning DFMNMF_EINVAL before any device work: all subarrays
 * of one size M_k in 1..4, K <= 16, N <= 16, B <= 64, F <= 65535, and
 * F * ceil(T/128) + F * K + 1 <= DFMNMF_NOALLOC_SCRATCH_DOUBLES, because its
 * partial sums live in one static device array of that many doubles
 * (512 KiB) that every GPU which loads this library keeps until the process
 * exits (the 4 x 4-mic, F = 513, T = 626 workload needs 4618).  Null
 * pointers also return DFMNMF_EINVAL.
 * No cudaMalloc, cudaFree or allocating library routine is called.  The
 * first call in each CUDA context (each device's primary context, or any
 * other context the caller makes current) is a set-up step: it looks the
 * array's device address up with cudaGetSymbolAddress, which under lazy
 * module loading (the CUDA default) also loads the module and backs the
 * array.  Make that first call at set-up time, outside any real-time thread
 * and before any stream capture; later calls in the same context take no
 * lock.  All calls share the array, which keeps the last call's partial
 * sums: every entry a call reads it has written first, but calls whose GPU
 * work may overlap (different streams without ordering between them) race on
 * it and must be serialised by the caller.  DFMNMF_ENUMERIC if the cost is
 * not finite.
 */
#define DFMNMF_NOALLOC_SCRATCH_DOUBLES 65536
int dfmnmf_loglik_noalloc(const dfmnmf_desc* desc, const void* x_dev, const void* Q_dev,
                          const float* W_dev, const float* H_dev, const float* g_dev,
                          double* nll_host, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* dfmnmf_last_error(void);

int dfmnmf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DFMNMF_H */
