// Internal declarations shared by the libtrd translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/trd.h"

namespace trd {
// opt-in dynamic shared memory per block on this GPU (227 KB)
constexpr size_t kSmemOptIn = 232448;

// Programmatic dependent launch along the main stream's chain of small kernels: a kernel so
// launched may become resident while its predecessor in the stream finishes (its launch and
// prologue overlap the predecessor's tail); it calls pdl_wait() before touching anything an
// earlier kernel wrote (the wait returns once the predecessor has completed and its memory is
// visible; it is a no-op for a kernel launched without the attribute), then pdl_trigger() so
// that its own successor may launch.  Only kernels that begin this way are launched with
// pdl_launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Off while the side stream's work is enqueued: kernels launched early there became resident
// next to the data pass's CTAs and slowed it (measured), while the side stream has slack.
inline thread_local bool pdl_on = true;
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_on ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}


constexpr int kMaxN = TRD_MAX_ORDER;
constexpr int kMaxR = TRD_MAX_RANK;
constexpr int64_t kProbeMax = int64_t(1) << 20;   // adaptive-width probe size
constexpr uint64_t kProbeSeed = 0x5eedull;

__host__ __device__ inline int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
// Quotient and remainder of non-negative 64-bit integers through the 32-bit divider when both
// operands fit in 32 bits: the general 64-bit division is a long routine on the FP64 unit,
// which on this GPU issues at a small fraction of the FP32 rate.
__device__ __forceinline__ int64_t qdiv(int64_t n, int64_t d) {
  return ((uint64_t)n | (uint64_t)d) <= 0xffffffffull ? (int64_t)((uint32_t)n / (uint32_t)d) : n / d;
}
__device__ __forceinline__ int64_t qdivmod(int64_t n, int64_t d, int64_t& r) {
  const int64_t q = qdiv(n, d);
  r = n - q * d;
  return q;
}

// BF16 rounding (round to nearest even) through the packed conversion instruction.
__device__ __forceinline__ __nv_bfloat16 bf16_rn(float f) { return __floats2bfloat162_rn(f, 0.f).x; }

// Walks e = e0, e0 + step, ... over a row-major matrix with rows of length n as (row, col),
// with one division at the start instead of one per element (integer division goes through
// the conversion unit, which on this GPU issues near the FP64 rate).
struct RowCol {
  int r, c, dr, dc, n;
  __device__ RowCol(int e0, int step, int n_) : r(e0 / n_), c(e0 % n_), dr(step / n_), dc(step % n_), n(n_) {}
  __device__ void next() {
    r += dr;
    c += dc;
    if (c >= n) {
      c -= n;
      ++r;
    }
  }
};
__host__ __device__ inline int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

// ------------------------------------------------------------------ device-side status
enum DevStatus : int {
  DEV_OK = 0,
  DEV_SINGULAR = 1,   // Cholesky pivot <= 0
  DEV_NONFINITE = 2,  // non-finite step or residual
  DEV_TIMEOUT = 4,    // a bounded wait gave up
  DEV_BOUNDS = 8      // an index check failed (access skipped)
};

// ------------------------------------------------------------------ a subchain of cores
// Chain product Z_{m_0}(i_0) Z_{m_1}(i_1) ... over a multi-index p = overline{i_0 i_1 ..}
// (first digit fastest).  Core slices use the mode-2 row-major layout: slice i of a core
// with ranks (rows, cols) is element (a, b) at i*rows*cols + b*rows + a.
struct Chain {
  int n = 0;                         // number of cores (0 = identity)
  const double* core[kMaxN] = {};
  const float* coref[kMaxN] = {};    // FP32 copy of core[j] (nullptr = convert from core[j])
  const int32_t* idx[kMaxN] = {};    // digit -> core slice (nullptr = identity)
  int64_t dim[kMaxN] = {};           // extent of each digit
  int rows[kMaxN] = {}, cols[kMaxN] = {};
  int64_t count = 1;                 // product of dims
  int out_rows = 0, out_cols = 0;    // product shape
};

// A tensor (full data or RStS sketch) seen by the data passes.
struct View {
  const float* X = nullptr;          // values, linear order (first mode fastest)
  const uint32_t* M = nullptr;       // packed mask (nullptr = all observed)
  int N = 0;
  int64_t dim[kMaxN] = {};           // sizes of the view (s_j)
  const int32_t* idx[kMaxN] = {};    // device map view index -> full index (nullptr = identity)
  int64_t numel = 0;
};

// Split of the modes into an inner block 0..c-1 and an outer block c..N-1.
struct Split {
  int c = 1;
  int64_t P_in = 1, P_out = 1;       // products of the view dims of each block
  int Kp = 1;                        // r_0 * r_c
  bool rows = true;                  // updated core in the inner block (stationary = inner)
  int64_t P_stat = 1, P_strm = 1;
};

// Arguments of the fused data-pass kernels (all precisions).
struct PassArgs {
  const float* X;
  const uint32_t* M;
  int64_t P_in;                      // X(a, b) at a + P_in * b
  int64_t P_stat, P_strm;
  int Kp, ld;                        // row length and stride (elements) of the merged matrices
  const void* Sst;                   // stationary merged matrix [P_stat][ld]
  const void* Sh;                    // stationary merged with h (pass 2)
  const void* Sstr;                  // streaming merged matrix [P_strm][ld]
  const double* sigma;               // device scalar: kernel width (inf -> w = 1)
  void* Tpart;                       // pass 1: partial contractions [splits][P_stat][Kp]
  double* stat_part;                 // per-CTA statistics [ctas][8]
  int64_t tiles_per_split;           // streaming tiles per CTA column split
};

// ------------------------------------------------------------------ work buffers
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace trd

// The opaque handle.
struct trd_handle {
  int N = 0;
  int64_t I[trd::kMaxN] = {};
  int R[trd::kMaxN] = {};
  int K[trd::kMaxN] = {};
  int prec = TRD_FP32;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;

  // data
  const float* X = nullptr;
  const uint32_t* M = nullptr;
  int64_t numel = 0;

  // cores (FP64 master, mode-2 row-major) and FGMC factors E_k (r_k^2 x r_{k+1}^2)
  double* Z[trd::kMaxN] = {};
  float* Zf[trd::kMaxN] = {};          // FP32 copies of the cores, kept in step with Z
  double* E[trd::kMaxN] = {};
  uint64_t ver[trd::kMaxN] = {};     // core versions

  // current view and sketch storage
  trd::View view;
  int view_k = -1;                   // core the current sketch was drawn for (-1: full)
  bool sketched = false;
  int32_t* idx_dev[trd::kMaxN] = {};
  size_t idx_cap[trd::kMaxN] = {};
  trd::DevBuf XI, PI;

  // per-update state
  int pass1_k = -1;                  // core of the last residual pass (-1 none)
  int grad_k = -1;                   // core of the current d
  int gram_k = -1;                   // core of the current G
  uint64_t gram_ver[trd::kMaxN] = {};
  trd::Split split;
  int splits = 1, ctas = 1;
  int64_t slots_last = 0;

  // device scalars: [0] sigma in use, [1] sigma_prev, [2] num <d,h>, [3] den, [4] eta,
  // [5] lambda used, [6] e (stop), [7] status word (as double), [8..] spare
  double* scal = nullptr;
  int* dstatus = nullptr;            // device status word (DevStatus bits)
  double* report_dev = nullptr;      // per-iteration report staging [64]
  double* host_pinned = nullptr;     // pinned staging for read-backs [256]
  int32_t* idx_pinned = nullptr;     // pinned staging for index uploads
  size_t idx_pinned_cap = 0;

  // work buffers
  trd::DevBuf Sst, Sstr, Sh;         // merged matrices (compute type)
  trd::DevBuf Sst_bf, Sstr_bf, Sh_bf, SstrT_bf, SstT_bf; // BF16 operands (hi|lo)
  trd::DevBuf Tpart, Tsum, stat_part, stat_sum;
  trd::DevBuf pre, post, dpart;      // back-contraction
  trd::DevBuf d, h, G, L, T1, T2, D, Dprev;
  trd::DevBuf probe_keys, probe_work;
  bool merged_valid_st = false, merged_valid_str = false;
  uint64_t merged_ver[trd::kMaxN] = {};
  int merged_k = -1;
  int32_t t = 0;
  bool have_D0 = false;
  bool sigma_set = false;
};

namespace trd {

// ------------------------------------------------------------------ launch accounting
// Every kernel launch in the library bumps this counter (read by trd_kernel_launches).
void note_launch();
void note_launches(int64_t n);
int64_t launches_total();

// ------------------------------------------------------------------ host helpers (api)
trd_status set_err(trd_handle* h, trd_status s, const std::string& msg);
trd_status cuda_check(trd_handle* h, cudaError_t e, const char* what);
trd_status ensure(trd_handle* h, DevBuf& b, size_t bytes);

// ------------------------------------------------------------------ launchers
// merge.cu
// out may be null when only the BF16 operand (hi, lo optional, kpad-wide rows) is wanted
cudaError_t launch_chain(const Chain& ch, void* out, bool out_double, bool transposed, int64_t ld, cudaStream_t st,
                         __nv_bfloat16* hi = nullptr, __nv_bfloat16* lo = nullptr, int kpad = 0);
// one core read in place of a merged one-core chain: slice idx[i] (identity when null)
struct BcCore {
  const double* core = nullptr;
  const float* coref = nullptr;      // FP32 copy (read by the FP32 kernel when present)
  const int32_t* idx = nullptr;
};
// partial slots of the tensor-core pass (see k_reduce_slots), read by the back-contraction
struct SlotSrc {
  const float* part = nullptr;
  int64_t RB = 0, NT = 0, bm = 0;
  int G = 0;
  int bm_shift = -1;                 // log2(bm) when bm is a power of two (set at launch)
};
cudaError_t launch_backcontract(const void* Tsum_d, int Kp, bool rows_case, int mr, int mc,
                                const void* pre, int64_t n_pre, const void* post,
                                int64_t n_post, int64_t Ik, int rk, int rk1, double* dpart,
                                int nsplit, double* d, unsigned* ctr, bool fp64, cudaStream_t st,
                                const SlotSrc* slots = nullptr, BcCore preC = BcCore{},
                                BcCore postC = BcCore{});
cudaError_t launch_reduce_T(const void* Tpart, bool is_double, int splits, int64_t n,
                            double* Tsum, cudaStream_t st);
cudaError_t launch_reduce_stats(const double* stat_part, int ctas, double* stat_sum,
                                int* dstatus, cudaStream_t st, double* obj = nullptr);
cudaError_t launch_reconstruct_mats(const void* A, const void* C, bool fp64, int64_t P_in, int64_t P_out,
                                    int Kp, const float* Xref, float* out, double* err_part,
                                    int parts, cudaStream_t st);
cudaError_t launch_gather(const float* X, const uint32_t* M, int N, const int64_t* full_dim,
                          const View& v, float* XI, uint32_t* PI, int64_t* obase, cudaStream_t st);
cudaError_t launch_set_scalar(double* p, double v, cudaStream_t st);
cudaError_t launch_to_bf16_split(const void* src, bool src_double, int64_t rows, int Kp,
                                 int64_t ld_src, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                 __nv_bfloat16* hiT, int64_t ldT, int64_t ld_dst,
                                 cudaStream_t st);

// pass_simt.cu
int simt_blocks_per_sm(bool is_double, bool rows_case, int Kp);   // resident pass-1 CTAs per SM
cudaError_t launch_pass_simt(const PassArgs& a, bool is_double, bool rows_case, bool pass2,
                             int splits, int* ctas_out, int* splits_out, cudaStream_t st);

// pass_tc.cu (tcgen05 BF16 data passes)
// Operands of the tensor-core data passes: device arrays [rows][kpad] of BF16, or of FP32
// holding TF32-rounded values (the TF32 kind).
struct PassOperands {
  const void* S_hi = nullptr;   // stationary operand, hi and lo splits
  const void* S_lo = nullptr;
  const void* S_h = nullptr;    // pass 2: step operand (TF32: its hi split)
  const void* S_h_lo = nullptr; // pass 2, TF32 only: lo split of the step operand
  const void* T_hi = nullptr;   // streaming operand, hi and lo splits
  const void* T_lo = nullptr;
  const void* T_hiT = nullptr;  // TF32 pass 1: the streaming splits transposed, [kpad][ldT]
  const void* T_loT = nullptr;
  int64_t ldT = 0;
};
// padded contraction of the tensor-core passes: BF16 64, 128 or 256, TF32 64; 0 = unsupported
int tc_kpad(int Kp, bool tf32);
int tc_bm();
int tc_bn(int kpad, bool tf32);   // streaming columns per tile of that configuration
cudaError_t launch_wait_selftest(bool arrive, uint32_t limit, int* err, cudaStream_t st);
cudaError_t launch_tc_prep(const float* src, int64_t rows, int Kp, __nv_bfloat16* hi, __nv_bfloat16* lo,
                           cudaStream_t st);
cudaError_t launch_tc_prep_tf32(const float* src, int64_t rows, int Kp, float* hi, float* lo, cudaStream_t st,
                                float* hiT = nullptr, float* loT = nullptr, int64_t ldT = 0);
cudaError_t launch_mask_rows(const uint32_t* M, int64_t P_in, int64_t P_out, int64_t W, uint32_t* out,
                             cudaStream_t st);
cudaError_t launch_mask_transpose(const uint32_t* M, int64_t P_in, int64_t P_out, int64_t WT, uint32_t* out,
                                  cudaStream_t st);
cudaError_t launch_reduce_slots(const float* part, int64_t RB, int64_t NT, int G, int64_t P_stat, int Kp,
                                double* out, cudaStream_t st);
cudaError_t launch_pass_tc(bool tf32, bool rows_case, bool pass2, const PassOperands& o, const float* X,
                           int64_t P_in, int64_t ldx, int64_t P_out, const uint32_t* Mst, int64_t W,
                           int64_t P_stat, int64_t P_strm, int Kp, const double* sigma, float* Tpart,
                           double* stat_part, int* err, int G, bool full_stats, cudaStream_t st,
                           unsigned char* wq = nullptr);
// Bytes of the BF16 pass-1 weight cache for a P_stat x P_strm pass of width Kp (one byte per
// slot of every unit, units padded to whole tiles).
int64_t tc_wq_bytes(int Kp, int64_t P_stat, int64_t P_strm);
// Line-search pass of the BF16 path from the weights cached by pass 1 (same Kp, P_stat,
// P_strm): per-CTA partials of den = sum w (S_h S_str^T)^2 in stat_part[8 c + 6]; nf_in
// (device, nullable): pass 1's count of non-finite observed residuals (non-zero -> den NaN).
cudaError_t launch_pass_wls(const void* S_h, const void* T_hi, const unsigned char* wq, int Kp, int64_t P_stat,
                            int64_t P_strm, double* stat_part, int* err, int G, const double* nf_in,
                            cudaStream_t st);
cudaError_t launch_pad_rows(const float* X, int64_t P_in, int64_t P_out, int64_t ld, float* out, cudaStream_t st);

// fgmc_solve.cu
cudaError_t launch_fgmc_E(const double* Z, const int32_t* idx, int64_t n, int rk, int rk1,
                          double* E, double* work, cudaStream_t st);
cudaError_t launch_dgemm(const double* A, const double* B, double* C, int M, int N, int K,
                         bool transB, cudaStream_t st);
cudaError_t launch_phi(const double* T, int p, int q, double* G, cudaStream_t st);
// one-CTA LDL^T (register-resident triangle) and the warp-per-row solve: K <= kLdlKmax
constexpr int kLdlKmax = 128;
inline bool ldl_fits(int K) { return K >= 1 && K <= kLdlKmax; }
cudaError_t launch_ldl_factor(const double* G, int K, double lambda, double* Lcm, double* Dinv, double* scal,
                              int* dstatus, cudaStream_t st);
// also <d, h> into *num (per-row parts in dot_part[rows]; ctr: a zeroed counter word, left zero)
cudaError_t launch_ldl_solve(const double* Lcm, const double* Dinv, const double* d, double* h, int K, int64_t rows,
                             double* dot_part, unsigned int* ctr, double* num, cudaStream_t st);
// blocked multi-CTA Cholesky for K > kLdlKmax; L holds 2 K^2 + K doubles: the row-major lower
// factor, its reciprocal diagonal, its column-major copy (read by launch_solve_rows)
cudaError_t launch_cholesky(const double* G, int K, double lambda, double* L, double* scal,
                            int* dstatus, cudaStream_t st);
// Identity K x K (FP64); h = d Minv for rows of d with <d, h> fused (as launch_ldl_solve).
cudaError_t launch_identity(double* I, int K, cudaStream_t st);
cudaError_t launch_inv_rows(const double* Minv, const double* d, double* h, int K, int64_t rows, double* dot_part,
                            unsigned int* ctr, double* num, cudaStream_t st);
cudaError_t launch_solve_rows(const double* L, const double* d, double* h, int K, int64_t rows,
                              cudaStream_t st);
cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* out,
                       cudaStream_t st);
// eta (from <d,h> and the line-search partials or a reduced den, or fixed) and Z += eta h
// In-place advance of the merged half that holds the updated core (BF16 path): S += eta S_h
// on [n / Kp][Kp] FP32 rows, with the BF16 hi/lo operand rows [kpad] written again.
struct HalfAdvance {
  float* S = nullptr;
  const float* Sh = nullptr;
  int64_t n = 0;
  int Kp = 0, kpad = 0;
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;
};
cudaError_t launch_step_update(double* Z, float* Zf, const double* h, int64_t n, const double* num, const double* part, int ctas,
                               const double* den, double fixed_eta, int* dstatus, double* eta, double* eta_slot,
                               cudaStream_t st,
                               const HalfAdvance& adv = HalfAdvance{});
constexpr int kStopBlocks = 152;     // most blocks of the stopping-quantity kernel
cudaError_t launch_stop_error(const double* D, double* Dprev, int64_t n, double* part, unsigned int* ctr,
                              double* e_out, cudaStream_t st);

// sigma.cu
size_t sigma_work_doubles();
// probe positions of the adaptive width (host): 0..numel-1, or 2^20 SplitMix64 draws, sorted
void probe_positions(int64_t numel, std::vector<int64_t>& lin);
cudaError_t launch_probe_setup(const float* X, const uint32_t* M, const int64_t* lin_dev, int64_t n, int64_t P_in,
                               int32_t* pa, int32_t* pb, float* px, cudaStream_t st);
// keys and cand: n 64-bit words each (order keys, selection candidates)
cudaError_t launch_probe_sigma_merged(const void* A, const void* C, bool fp64, int Kp, const int32_t* pa,
                                      const int32_t* pb, const float* px, int64_t n, double sigma_prev,
                                      const double* sigma_prev_dev, uint64_t* keys, uint64_t* cand, double* work,
                                      double* sigma_out, cudaStream_t st);
cudaError_t launch_sigma_from_floats(const float* r, int64_t n, double x_obs_rms, double sigma_prev, uint64_t* keys,
                                     uint64_t* cand, double* work, double* sigma_out, cudaStream_t st);

// rows.cu (uniform row sampling of the subchain unfolding)
struct RowsArgs {
  int N = 0, k = 0;
  int64_t Ik = 0, J = 0;
  int64_t stride[kMaxN] = {};        // linear stride of each mode in X
  int R[kMaxN] = {};
  const double* Z[kMaxN] = {};       // FP64 master cores
  const float* Zf[kMaxN] = {};       // their FP32 copies
};
cudaError_t launch_gather_rows(const float* X, const uint32_t* M, const RowsArgs& a, const int32_t* rows, float* XI,
                               uint32_t* PI, cudaStream_t st);
cudaError_t launch_rows_chain(const RowsArgs& a, const int32_t* rows, void* B, bool fp64, cudaStream_t st);

// sampled.cu
// Strides of each mode inside the inner (a) / outer (b) block of a two-block cut (0 if the mode
// belongs to the other block).
struct Split2 {
  int N, c;
  int64_t sin[kMaxN], sout[kMaxN];
  int64_t dim[kMaxN];
  int* err;                          // device status word (DEV_BOUNDS on a bad index)
};
// Work arrays of the sampled loss: per entry its block indices (ka, kb), the entry numbers
// grouped by a and by b, per-block counts and cursors, and the per-entry adjoint factor g.
struct SampledWork {
  int32_t *ka = nullptr, *kb = nullptr, *perm_a = nullptr, *perm_b = nullptr;
  uint32_t *cnt_a = nullptr, *cnt_b = nullptr, *cur_a = nullptr, *cur_b = nullptr;
  void* g = nullptr;
};
cudaError_t launch_sampled_order(const int32_t* idx, const Split2* sp, int64_t M, int64_t P_in, int64_t P_out,
                                 const SampledWork& wk, cudaStream_t st);
cudaError_t launch_sampled_rows(const void* A, const void* C, bool fp64, int Kp, const void* x, int64_t M,
                                int64_t P_in, double sigma, void* resid, double* loss_part, int parts, bool backward,
                                double g_scale, void* gA, void* gC, const SampledWork& wk, cudaStream_t st);
cudaError_t launch_to_double(const float* src, int64_t n, double* dst, cudaStream_t st);
cudaError_t launch_from_double(const double* src, int64_t n, void* dst, bool fp64, cudaStream_t st);

}  // namespace trd
