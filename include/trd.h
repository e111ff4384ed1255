/*
 * trd.h -- C ABI of libtrd: the per-core hot path of auto-weighted robust tensor-ring
 * decomposition (AWRTRD) and its scalable variant with FGMC and RStS (SAWRTRD), from
 * He & Atia, "Scalable and Robust Tensor Ring Decomposition for Large-scale Data",
 * UAI 2023, on one NVIDIA GB300 (sm_103a).
 *
 * Conventions used by every call
 *   - Indices are 0-based.  A tensor of order N with mode sizes I[0..N-1] is stored flat
 *     with i_1 fastest: offset = sum_m i_m * prod_{m'<m} I[m'] (the multi-index
 *     overline{i_1 ... i_N} of Def. 2).
 *   - Ranks: R[k] is r_k, the first rank of core k; core k is r_k x I_k x r_{k+1} with
 *     r_{N+1} = r_1 (Def. 1).
 *   - Host core layout ("mode-2 unfolding, row-major"): core k is I_k rows of
 *     K_k = r_k r_{k+1} doubles; element (alpha, i, beta) of Z_k sits at
 *     i*K_k + beta*r_k + alpha, i.e. row i of Z_{k(2)} with column alpha + beta*r_k.
 *     Gradients d and scaled gradients h use the same layout; Gram matrices are K_k x K_k
 *     row-major with that column order on both sides.
 *   - The observation mask is bit-packed: bit b of 32-bit word w is linear index 32w+b,
 *     1 = observed (the binary tensor P of Eq. TRWOPT).
 *   - Device pointers passed in are BORROWED: the caller owns them, they must stay valid
 *     while the handle uses them, and the library never frees them.  Host pointers are
 *     only read or written during the call.
 *   - Every call is ordered on the handle's CUDA stream.  Calls that return values
 *     through host pointers synchronise that stream before returning.
 *   - No call aborts or throws.  Each returns a trd_status; trd_last_error() gives a
 *     one-line message for the last failure on the handle.  After TRD_ECUDA the handle
 *     should be destroyed.
 *   - The library has no CPU fallback: without a usable CUDA device trd_create fails.
 */
#ifndef TRD_H
#define TRD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRD_MAX_ORDER 8   /* tensor order N is 3..TRD_MAX_ORDER */
#define TRD_MAX_RANK 128  /* every r_k is 1..TRD_MAX_RANK */
#define TRD_MAX_CORE_K 8192  /* every core's r_k r_{k+1} is at most TRD_MAX_CORE_K */

typedef enum {
  TRD_OK = 0,
  TRD_EINVAL = 1,      /* bad argument, unsupported shape, or calls in the wrong order */
  TRD_ENOMEM = 2,      /* a device or host allocation failed */
  TRD_ECUDA = 3,       /* a CUDA runtime call or a kernel launch failed */
  TRD_ESINGULAR = 4,   /* G + lambda I is not numerically positive definite */
  TRD_ENONFINITE = 5,  /* non-finite residuals, gradient or step size */
  TRD_ETIMEOUT = 6,    /* a bounded device-side wait gave up */
  TRD_ENOTIMPL = 7     /* combination not implemented (e.g. precision for this shape) */
} trd_status;

/* Arithmetic of the two data passes (reconstruction, residual and weight, weighted
 * contraction of Eq. hatd, line-search product).  FGMC, the factorisation, the solves and the
 * step size are FP64 in every mode.  K' = r_1 r_{c+1} is the contraction width of the data
 * passes (c = the cut of the ring into two merged halves, chosen per view). */
typedef enum {
  TRD_FP64 = 0,   /* CUDA-core FP64 data passes (small problems, debugging); K' <= 112 */
  TRD_FP32 = 1,   /* CUDA-core FP32 data passes, FP32 accumulation; K' <= 256 */
  TRD_BF16 = 2,   /* tcgen05 tensor cores, mixed BF16: the reconstruction in 3-term split BF16
                     (hi*hi + hi*lo + lo*hi), the gradient and line-search products in one
                     BF16 term, FP32 accumulation; residual and weight in FP32, the weight
                     carried from the residual pass to the line search as 8-bit fixed point
                     (w = q / 255, absolute error <= 1/510); K' <= 256, else TRD_ENOTIMPL */
  TRD_TF32X3 = 3  /* tcgen05 tensor cores, TF32 with the 3-term split of both operands in every
                     product (about 22 significant bits per operand: FP32-level accuracy),
                     FP32 accumulation; K' <= 64 on the tensor cores, wider contractions run
                     the FP32 CUDA-core passes */
} trd_precision;

typedef enum {
  TRD_GRAM_GLOBAL = 0,  /* Eq. hI: G of the full cores, by FGMC (the paper's method) */
  TRD_GRAM_LOCAL = 1,   /* ablation 'local scaled term' (Sec. 5.1): G of the sampled cores */
  TRD_GRAM_NONE = 2     /* ablation 'gradient descent' (Sec. 5.1): h = d */
} trd_gram_kind;

typedef struct trd_handle trd_t;

/* Statistics of one reconstruction/residual/weight pass (Eq. updatew on the sketch). */
typedef struct {
  double sigma;        /* kernel width used (+inf means W = 1) */
  double sum_w;        /* sum of w over observed slots */
  double sum_e2;       /* sum of e^2 over observed slots */
  double sum_we2;      /* sum of w e^2 over observed slots (2x the weighted objective) */
  int64_t n_obs;       /* observed slots */
  int64_t n_nonfinite; /* observed slots whose residual is not finite */
  int64_t n_slots;     /* slots visited (observed or not) */
} trd_resid_stats;

/* Parameters of one outer iteration of Algorithm 1. */
typedef struct {
  int32_t sketch[TRD_MAX_ORDER]; /* RStS size s_j for every non-updated mode j; 0 = full
                                    mode (AWRTRD when all are 0).  s_k = I_k always. */
  double sigma;     /* > 0: fixed kernel width; +inf: W = 1; <= 0: adaptive width */
  double lambda;    /* Eq. sg regulariser; >= 0 absolute, < 0 means |lambda| tr(G)/K */
  uint64_t seed;    /* seed of the RStS index draws (SplitMix64, see trd_draw_indices) */
  int32_t gram;     /* trd_gram_kind */
  int32_t reserved;
} trd_params;

/* Result of one outer iteration. */
typedef struct {
  double e;                    /* Algorithm 1 stopping quantity ||D^t - D^{t-1}|| / ||D^t|| */
  double sigma;                /* kernel width used in this iteration */
  double eta[TRD_MAX_ORDER];   /* step size of every core update */
  double objective[TRD_MAX_ORDER]; /* 0.5 sum w e^2 on the sketch before each update */
  int64_t slots;               /* sketch slots visited by the data passes (all cores) */
  int32_t t;                   /* iteration counter after this step */
  int32_t reserved;
} trd_report;

/* ---------------------------------------------------------------- handle */

/* Create a handle for an order-N tensor (3 <= N <= TRD_MAX_ORDER) with mode sizes I[0..N-1]
 * (each >= 1, product < 2^40) and ring ranks R[0..N-1] (Def. 1, 1 <= r_k <= TRD_MAX_RANK,
 * r_k r_{k+1} <= TRD_MAX_CORE_K).  The data passes further need a cut of the ring whose width
 * r_1 r_c is at most 256 (112 for TRD_FP64); a call that finds none returns TRD_ENOTIMPL.
 * `precision` is a trd_precision.  `cuda_stream` is a cudaStream_t on which every call is
 * ordered; it must outlive the handle.  NULL (the legacy default stream) gives the handle
 * its own blocking stream, which keeps the legacy stream's implicit ordering with the
 * caller's work and can be captured into a CUDA graph (the legacy stream cannot).  Allocates the
 * library's own device state (cores, FGMC factors, work buffers); no data is copied.
 * Errors: TRD_EINVAL (shape), TRD_ENOMEM, TRD_ECUDA (no usable device). */
trd_status trd_create(trd_t** handle, int N, const int64_t* I, const int32_t* R,
                      int precision, void* cuda_stream);

/* Free everything the handle allocated (never the caller's buffers).  NULL is a no-op. */
void trd_destroy(trd_t* handle);

/* Message for the last failing call on `handle` ("" if none); owned by the handle. */
const char* trd_last_error(const trd_t* handle);

/* Static name of a status code. */
const char* trd_status_string(trd_status status);

/* The cut of the ring that the data passes use for a tensor (or a sketch of it) of mode sizes
 * I[0..N-1] and ring ranks R[0..N-1] (Thm. 1's two-block form of the reconstruction): modes
 * [0, c) form one block and [c, N) the other, and the contraction between them is
 * R[0] R[c] = r_1 r_{c+1} wide.  The data passes take widths up to 256 (112 for TRD_FP64);
 * among the cuts that fit, the one whose two blocks are closest in size (by the logarithm
 * of their entry counts; the lowest c on a tie) is used.  Host only: needs no device and no
 * handle, so a caller can check its ranks before allocating anything.
 *   c_out      receives c (1 <= c < N)
 *   width_out  receives R[0] R[c]
 * Errors: TRD_EINVAL (a shape trd_create rejects, or a NULL output), TRD_ENOTIMPL (no cut
 * fits: c_out and width_out then describe the most balanced cut, which the data passes
 * reject). */
trd_status trd_ring_cut(int N, const int64_t* I, const int32_t* R, int precision, int32_t* c_out,
                        int32_t* width_out);

/* ---------------------------------------------------------------- data and cores */

/* Attach the data tensor X (Eq. TRWOPT) and its observation mask P (Eq. TRWOPT; bit-packed,
 * ceil(prod I / 32) words, 1 = observed).  Both are DEVICE pointers, borrowed: X is prod(I)
 * floats in the linear order above, 16-byte aligned.  mask may be NULL, meaning fully
 * observed.  Resets any sketch.  The library caches what it derives from the contents (the
 * mask re-laid for the data passes, the adaptive width's probe values); after changing the
 * contents behind the same pointers, call trd_set_data again, which drops those caches, has
 * the merged subchains formed again from the cores, and ends CUDA-graph replay of trd_step.  Errors: TRD_EINVAL (NULL X, misalignment). */
trd_status trd_set_data(trd_t* handle, const float* X_dev, const uint32_t* mask_dev);

/* Initialise all cores i.i.d. Gaussian (Algorithm 1, 'initialize Z_k'; the law is a
 * reading, the paper does not state it): entry (alpha, i, beta) of core k is
 * stddev * Box-Muller normal number base_k + (i r_{k+1} + beta) r_k + alpha of the
 * SplitMix64 stream of `seed` (u1 from output 2g, u2 from output 2g+1; base_k = entries of
 * the cores before k).  stddev <= 0 means (r_k r_{k+1})^(-1/4).  Refreshes the FGMC
 * factors and D^0 and resets the iteration counter. */
trd_status trd_init_cores(trd_t* handle, uint64_t seed, double stddev);

/* Copy core k (host, I_k * r_k * r_{k+1} doubles, layout above) into / out of the handle.
 * trd_set_core refreshes the FGMC factor of core k and invalidates cached merges; call
 * trd_reset_iteration afterwards to recompute D^0 for the stopping rule. */
trd_status trd_set_core(trd_t* handle, int k, const double* core_host);
trd_status trd_get_core(trd_t* handle, int k, double* core_host);

/* Recompute D^0 from the current cores and set the iteration counter to t. */
trd_status trd_reset_iteration(trd_t* handle, int32_t t);

/* ---------------------------------------------------------------- the hot path */

/* RStS (Sec. 3.2.2, Algorithm 1 'obtain subtensor'): for an update of core k, take the
 * index sets idx[j] (HOST arrays of s[j] int32 each, strictly increasing, in [0, I_j)) for
 * every j != k; idx[k] and s[k] are ignored (mode k is kept whole).  Gathers the sketch
 * X_I and P_I into library-owned device memory and selects the sampled core slices.
 * idx == NULL selects the whole tensor (AWRTRD).  Errors: TRD_EINVAL (unsorted,
 * duplicated or out-of-range indices, no data). */
trd_status trd_sample_subtensor(trd_t* handle, int k, const int32_t* const* idx,
                                const int32_t* s);

/* RStS index draw used by trd_step (host-side, no device work): s distinct indices of
 * [0, I), uniform without replacement, sorted.  Key = SplitMix64 output (t N + k) N + j of
 * `seed`; a partial Fisher-Yates shuffle of 0..I-1 then takes pick m = m + (z_m mod (I-m))
 * with z_m the key's m-th output.  out has room for s ints. */
trd_status trd_draw_indices(uint64_t seed, int32_t t, int k, int j, int N, int64_t I,
                            int32_t s, int32_t* out);

/* Uniform row sampling (the paper's 'uniform row sampling' ablation, Sec. 5): instead of
 * the RStS sketch, the update of core k uses J sampled rows of Z^{!=k}_[2], i.e. the
 * multi-indices rows[j * N + m] (HOST, J x N int32, row-major; column k is ignored; each
 * 0 <= rows[j N + m] < I_m; duplicates allowed), and the matching columns of X_[k] and P_[k]
 * (the J fibres along mode k, gathered here).  The next trd_residual_weights /
 * trd_core_gradient / trd_core_update for core k work on this sample (gradient of Eq. hatd
 * with the sampled rows; FGMC Gram of the full cores; line search on the sample); any other
 * sampling call or trd_step ends it.  TRD_EINVAL for an index out of range;
 * TRD_ENOTIMPL for the local Gram on this sample. */
trd_status trd_sample_rows(trd_t* handle, int k, const int32_t* rows, int64_t J);

/* Steps 'update W' and the first half of 'compute d' for core k on the current sketch:
 * reconstruct X_hat_I[k] = Z_{k(2)} (Z^{!=k}_{I[2]})^T (Thm. 1), residual e = x - x_hat on
 * observed slots, HQ weight w = exp(-e^2/(2 sigma^2)) (Eq. updatew, sign reading) and the
 * weighted contraction of Eq. hatd, all in one pass over the sketch (W is never stored).
 * sigma > 0 fixed, +inf gives w = 1, <= 0 uses the adaptive width of the current
 * iteration (computed by trd_adaptive_sigma, or by trd_step).  `out` (host, nullable)
 * receives the statistics.  Errors: TRD_EINVAL (no data / no sketch for k),
 * TRD_ENONFINITE (some observed residual not finite; stats still written). */
trd_status trd_residual_weights(trd_t* handle, int k, double sigma, trd_resid_stats* out);

/* Step 'compute d_I(Z_{k(2)})' (Eq. hatd): finish the weighted gradient of core k from
 * the last trd_residual_weights pass for k, as an I_k x K_k matrix kept on the device;
 * d_host (nullable) receives a copy (layout above).  d is the NEGATIVE gradient of
 * 0.5 ||sqrt(W) o P o (X_I - X_hat_I)||^2 with W held fixed.
 * Errors: TRD_EINVAL (no residual pass for k). */
trd_status trd_core_gradient(trd_t* handle, int k, double* d_host);

/* Step 'obtain G' (Eq. FGMC, Prop. 2): G = (Z^{!=k}_[2])^T Z^{!=k}_[2] of the FULL cores
 * as a chain product of the per-core factors E_m = sum_i Z_m(i) (x) Z_m(i) (r_m^2 x
 * r_{m+1}^2, FP64) over m = k+1..N, 1..k-1, realigned to K_k x K_k.  Kept on the device;
 * G_host (nullable) receives a copy. */
trd_status trd_fgmc_gram(trd_t* handle, int k, double* G_host);

/* Step 'update Z_k' (Eq. hI, Eq. ftrbcn and the exact line search): h = d (G + lambda I)^-1
 * in FP64 (LDL^T factorisation and substitutions for K_k <= 128, Cholesky above); eta = <d,h> / ||sqrt(W) o P o (h B^T)||^2 on the sketch when eta <= 0
 * (second data pass with the W of the last trd_residual_weights for k: recomputed from the
 * same residuals, or, with TRD_BF16, read back from the one byte per slot that pass stored),
 * else the given eta; a non-finite denominator rejects the step (TRD_ENONFINITE);
 * Z_k <- Z_k + eta fold(h) (update-sign reading); core k's FGMC factor is refreshed
 * before the next Gram that uses it.
 * lambda >= 0 absolute, < 0 means |lambda| tr(G)/K.  `gram` is a trd_gram_kind.
 * eta_out (host, nullable) receives the step used.  Needs trd_core_gradient for k; runs
 * trd_fgmc_gram itself when needed.  Errors: TRD_ESINGULAR, TRD_ENONFINITE. */
trd_status trd_core_update(trd_t* handle, int k, double lambda, double eta, int gram,
                           double* eta_out);

/* Partitioned core update (the exchange step of a multi-GPU update; no counterpart call in
 * the paper, whose d, G and step size are global sums): when the observed columns of X_[k]
 * are split across handles (for example one handle per GPU, each on a slab of one non-updated
 * mode selected with trd_sample_subtensor), d of Eq. hatd and the line-search denominator
 * are sums of per-handle partial sums, while G, h and <d, h> are the same on every handle
 * once d is.  A partitioned update of core k is: trd_residual_weights and trd_core_gradient
 * on every handle (partial d), an all-reduce (sum) of d by the caller, trd_set_gradient with
 * the summed d, trd_line_search_terms (<d, h> and the partial denominator), an all-reduce of
 * the denominators, and trd_core_update with the fixed step eta = <d, h> / sum of
 * denominators.
 *
 * trd_set_gradient: replace the device gradient of core k by d_host (HOST, I_k x K_k, layout
 * above).  Needs trd_residual_weights for k on this handle (the view of the line search).
 * trd_line_search_terms: h = d (G + lambda I)^-1 (as trd_core_update, `gram` a
 * trd_gram_kind), then *num_out = <d, h> and *den_out = sum w (h B^T)^2 over this handle's
 * view (the second data pass, W as in trd_core_update); the core is not changed.  Needs a gradient for
 * k.  Both synchronise.  Errors: TRD_EINVAL (order of calls, NULL), TRD_ESINGULAR. */
trd_status trd_set_gradient(trd_t* handle, int k, const double* d_host);
trd_status trd_line_search_terms(trd_t* handle, int k, double lambda, int gram, double* num_out,
                                 double* den_out);

/* One outer iteration of Algorithm 1: adaptive width (if params->sigma <= 0), then for
 * k = 1..N: index draw + RStS gather (if sketched), residual/weights/gradient pass, FGMC
 * Gram, scaled update with exact line search; then D^t = Z_{N(2)} G^{!=N} Z_{N(2)}^T and
 * e = ||D^t - D^{t-1}||_F / ||D^t||_F.  report (host, nullable) is filled.  Synchronises. */
trd_status trd_step(trd_t* handle, const trd_params* params, trd_report* report);

/* ---------------------------------------------------------------- evaluation helpers */

/* Adaptive kernel width (Sec. 5 cites a rule it does not state; reading):
 * sigma = max(1e-6 rms(x_obs), 2 min(std(e), IQR(e)/1.349), 0.9 sigma_prev) over the
 * observed residuals e of the full tensor (or of a fixed probe of 2^20 entries when the
 * tensor has more than 2^20 entries: probe m is linear index SplitMix64(0x5eed, m) mod
 * numel), population std, type-7 quartiles.  sigma_prev <= 0 or inf disables the
 * limiter.  Becomes the width used by sigma <= 0 calls.  sigma_out (host) receives it. */
trd_status trd_adaptive_sigma(trd_t* handle, double sigma_prev, double* sigma_out);

/* Same rule on a caller-given DEVICE array of n residuals (float), for checking the
 * selection: x_obs_rms is the rms of the observed data used for the floor. */
trd_status trd_sigma_from_residuals(trd_t* handle, const float* resid_dev, int64_t n,
                                    double x_obs_rms, double sigma_prev, double* sigma_out);

/* Allocation-free form of trd_sigma_from_residuals, for callers that cannot allocate device
 * memory: hosts that own all device memory through their own allocator or memory pool and
 * forbid libraries from calling cudaMalloc, processes held to a fixed device-memory budget
 * in which a late allocation could fail, and latency-bound loops that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree may imply.  It needs no handle and
 * allocates nothing: its work space is a fixed device array built into the library (about
 * 16.8 MB: 2^20 x 16 bytes of keys and candidates plus a 72 KB work area), held on every GPU
 * that loads the library until the process exits.  The paper has no counterpart; this is an
 * interface convenience only.
 *   resid_dev      DEVICE array of n float residuals, 1 <= n <= 2^20 (larger n: TRD_EINVAL)
 *   x_obs_rms      rms of the observed data, >= 0 (floor of the width; NaN: TRD_EINVAL)
 *   sigma_prev     previous width (<= 0 or inf disables the 0.9 limiter)
 *   sigma_out_dev  DEVICE pointer receiving the width (one double), written on the stream
 *   cuda_stream    cudaStream_t the work is ordered on (NULL = legacy default stream)
 * The first call on each device looks up the array's device address with that device
 * current; make that first call before any stream capture begins.  All calls share the
 * array and every call clears what must start at zero: calls whose work may overlap on the
 * GPU (different streams, or different host threads on the same device) race and must be
 * serialised by the caller.  The call does not synchronise; it returns TRD_EINVAL for bad
 * arguments and TRD_ECUDA when a launch fails. */
trd_status trd_sigma_from_residuals_noalloc(const float* resid_dev, int64_t n, double x_obs_rms,
                                            double sigma_prev, double* sigma_out_dev,
                                            void* cuda_stream);

/* Full TR reconstruction (Def. 1) of the current cores into the caller's DEVICE buffer
 * out_dev (prod(I) floats, linear order above). */
trd_status trd_reconstruct(trd_t* handle, float* out_dev);

/* Reconstruction (Def. 1) of arbitrary cores given on the HOST (layout above) into out_dev;
 * does not touch the handle's cores.  Used to synthesise exact-rank tensors. */
trd_status trd_reconstruct_from(trd_t* handle, const double* const* cores_host, float* out_dev);

/* ||X_hat - X_ref||_F / ||X_ref||_F over all entries, X_ref a DEVICE tensor (floats). */
trd_status trd_recovery_error(trd_t* handle, const float* Xref_dev, double* err_out);

/* Peak signal-to-noise ratio of the current reconstruction against X_ref (Sec. 5, the quality
 * measure of the image and video completion experiments): 10 log10(peak^2 / MSE), the mean taken
 * over all prod(I_n) entries.  X_ref is a DEVICE tensor of floats in the layout of trd_set_data.
 * peak > 0 is the signal range (1 for data scaled to [0, 1]).  *psnr_out = +inf when the
 * reconstruction equals X_ref.  TRD_EINVAL on NULL or a peak that is not positive and finite. */
trd_status trd_psnr(trd_t* handle, const float* Xref_dev, double peak, double* psnr_out);

/* ---------------------------------------------------------------- tracing */

/* Tracing level `on`: 0 off (default); 1 records CUDA events on the handle's stream around
 * the two fused data-pass kernels only (phases 0 and 1, cheap enough for timed runs); 2 also
 * around every other phase of a core update.  Phases: 0 the fused pass-1 kernel
 * (reconstruction, residual, weight, weighted contraction), 1 the fused pass-2 kernel (line
 * search), 2 operand merges and conversions, 3 reductions of partial results,
 * 4 back-contraction into the gradient, 5 FGMC Gram, 6 LDL^T factorisation, 7 solves and
 * <d,h>, 8 step size, core update and factor refresh, 9 adaptive width, 10 stopping
 * quantity, 11 the RStS gather of the sketch.  TRD_EINVAL for another level. */
trd_status trd_set_profiling(trd_t* handle, int on);

/* Synchronise the handle's stream and write out[2q] = total milliseconds and out[2q+1] = the
 * number of recorded intervals of phase q, for the 12 phases above (host array of 24
 * doubles).  reset != 0 clears the totals afterwards. */
trd_status trd_get_profile(trd_t* handle, int reset, double* out);

/* Number of kernels the library has launched in this process (all handles); a replayed
 * step graph counts its kernel nodes. */
int64_t trd_kernel_launches(void);

/* Execution option (no counterpart in the paper).  With `on` nonzero (the default) an
 * unsketched trd_step that repeats the previous step's arguments, with no other state-changing
 * call in between, is captured once as a CUDA graph and then replayed: the same kernels in the
 * same order on the same buffers, launched as one graph.  Any other call that changes the
 * handle's state (data, cores, sketch, single-core steps, tracing level) ends the replay; the
 * next steps run eagerly and are captured again.  on = 0 always runs eagerly. */
trd_status trd_set_graphs(trd_t* handle, int on);

/* Failure-detection self-test (no counterpart in the paper).  Runs, on the handle's stream,
 * the bounded mbarrier wait that every role of the tensor-core data pass uses, on a fresh
 * barrier whose phase completes only when `arrive` is nonzero, giving up after `limit`
 * polls (1 <= limit <= 2^24).  Returns TRD_OK when the phase completed and TRD_ETIMEOUT when
 * the wait gave up -- the status a stalled pass reports -- and leaves the handle usable in
 * both cases.  TRD_EINVAL for a limit out of range. */
trd_status trd_wait_selftest(trd_t* handle, int arrive, int64_t limit);

/* ---------------------------------------------------------------- sampled correntropy */

/* Forward of the sampled correntropy loss (Eq. corr in Welsch form) for the cores given
 * as DEVICE arrays cores_dev[k] (layout above): for M multi-indices idx_dev (DEVICE,
 * M x N int32, row-major, each i_k in [0, I_k)) and values x_dev (DEVICE, M values):
 * x_hat_m = Tr(prod_k Z_k(i_mk)) (Def. 1), e_m = x_m - x_hat_m,
 * loss = sum_m sigma^2 (1 - exp(-e_m^2 / (2 sigma^2))) (sigma > 0, finite).
 * fp64 = 0: cores, x and resid are float arrays and arithmetic is FP32 (FP64 sums);
 * fp64 = 1: all are double arrays and arithmetic is FP64.  resid_dev (DEVICE, M values,
 * nullable) receives e_m.  loss_out (host) receives the loss.  Entries with an index outside
 * [0, I_k) are skipped and the call returns TRD_EINVAL. */
trd_status trd_sampled_fwd(trd_t* handle, const void* const* cores_dev, const int32_t* idx_dev,
                           const void* x_dev, int64_t M, double sigma, int fp64,
                           void* resid_dev, double* loss_out);

/* Adjoint of trd_sampled_fwd: grad_dev[k] (DEVICE, same layout and type as the cores)
 * receives g_scale * d loss / d Z_k = g_scale * sum_m -w_m e_m (S_m^{!=k})^T, w_m the HQ
 * weight exp(-e_m^2/(2 sigma^2)) and S_m^{!=k} the subchain product of Thm. 1 at entry m,
 * which is recomputed per entry rather than stored.  The arrays are overwritten. */
trd_status trd_sampled_bwd(trd_t* handle, const void* const* cores_dev, const int32_t* idx_dev,
                           const void* x_dev, int64_t M, double sigma, int fp64,
                           double g_scale, void* const* grad_dev);

#ifdef __cplusplus
}
#endif
#endif /* TRD_H */
