// C ABI of libtrd: argument checking, device state and the order of the hot-path steps of
// Algorithm 1 (SAWRTRD; AWRTRD when no sketch is drawn).  Every step's arithmetic runs in
// the kernels of the other translation units; this file only launches them.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "trd_internal.cuh"

using namespace trd;

namespace trd {

trd_status set_err(trd_handle* h, trd_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

trd_status cuda_check(trd_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TRD_OK;
  cudaGetLastError();
  return set_err(h, TRD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

trd_status ensure(trd_handle* h, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return TRD_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  bytes = (bytes + 255) / 256 * 256;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(h, TRD_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  b.bytes = bytes;
  return TRD_OK;
}

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// implemented in merge.cu / sampled.cu / pass_tc.cu


}  // namespace trd

#define TRY(x)                         \
  do {                                 \
    trd_status _s = (x);               \
    if (_s != TRD_OK) return _s;       \
  } while (0)
#define CK(x, what) TRY(cuda_check(h, (x), what))

namespace {

// device scalar slots in h->scal
enum : int { S_SIGMA = 0, S_SIGMA_PREV = 1, S_NUM = 2, S_DEN = 3, S_ETA = 4, S_LAMBDA = 5, S_E = 6 };
// report_dev layout: [0..7] eta per core, [8..15] objective per core, [16] e, [17] sigma
enum : int { R_ETA = 0, R_OBJ = 8, R_E = 16, R_SIGMA = 17 };

// Identity of a merged half (inner block 0..c-1 or outer block c..N-1) of the current view:
// which half, which view, and the versions of the cores in it.
struct HalfTag {
  bool valid = false;
  int half = -1;
  uint64_t view_gen = 0;
  int c = 0, Kp = 0;
  uint64_t ver[kMaxN] = {};
  bool operator==(const HalfTag& o) const {
    if (!valid || !o.valid || half != o.half || view_gen != o.view_gen || c != o.c || Kp != o.Kp) return false;
    for (int m = 0; m < kMaxN; ++m)
      if (ver[m] != o.ver[m]) return false;
    return true;
  }
};

// extra per-handle buffers that do not need to be visible to other units
struct Extra {
  DevBuf meta;          // [N] core pointers, [N] dims (int64), [N] ranks (int)
  DevBuf stat_sum2;     // pass-2 statistics
  DevBuf Gloc;          // local Gram (ablation)
  DevBuf Eloc[kMaxN];   // sampled FGMC factors (ablation)
  DevBuf recA, recC;    // reconstruction operands
  DevBuf errp;          // reconstruction error partials
  DevBuf tmpZ[kMaxN];   // cores given to trd_reconstruct_from
  DevBuf probe_a, probe_b, probe_x;   // adaptive-width probe: inner / outer index, data
  DevBuf dotpart, solve_ctr;          // per-row parts of <d, h>, completion counter
  // TF32 x 3 / FP32 with K <= 128: (G + lambda I)^{-1} formed on the side stream, so that the
  // update's h = d (G + lambda I)^{-1} is one row-times-matrix product
  DevBuf Minv, Ident, inv_dot, inv_ctr, inv_num;
  int ident_K = 0;
  int minv_k = -1;            // core whose inverse Minv holds (-1: none)
  DevBuf bc_ctr;                      // per-row completion counters of the back-contraction
  DevBuf stop_part, stop_ctr;         // stopping quantity: per-block sums, completion counter
  DevBuf probe_cand;                  // selection candidates of the adaptive width
  SlotSrc slots;                      // partial slots of the last tensor-core pass 1
  double* obj_slot = nullptr;         // report slot for the objective of the next pass 1
  int adv_k = -1;                     // core whose FP32 step operand S_h is ready for the
                                      // in-place advance of its merged half (BF16 path)
  // uniform row sampling (trd_sample_rows): J multi-indices of the modes other than row_k
  bool row_view = false;
  int row_k = -1;
  int64_t rows_J = 0;
  DevBuf rows_dev;
  uint64_t rows_gen = ~0ull, rows_ver[kMaxN] = {};   // what h->Sst / h->Sstr hold
  // what the merged-half buffers hold (FP32/FP64 h->Sst / h->Sstr, BF16 operands bS* / bT*)
  HalfTag tagSst, tagSstr, tagBst, tagBstr;
  bool graph_tag_cur[4] = {};   // which of the four tags were current at the end of the capture
  bool own_stream = false;      // the handle created h->stream (the caller passed NULL)
  uint64_t view_gen = 0;    // 0 = the full tensor; every drawn sketch gets a new number
  uint64_t sketch_count = 0;
  bool probe_ready = false;
  int64_t probe_Pin = 0;
  DevBuf probe_lin;                   // sorted probe positions (drawn once per tensor size)
  int64_t probe_lin_n = -1;
  DevBuf Ework;         // FGMC factor partial sums
  // FGMC chain prefix Q = E_{k+1} ... E_{k+N-2} for the Gram of core q_k, prepared during the
  // update of core q_k - 1 (which changes only E_{q_k - 1}, the chain's last factor)
  DevBuf Qb[2];
  bool e_stale[kMaxN] = {};   // core updated, FGMC factor not yet refreshed (done by the next
                              // Gram, normally on the side stream)
  const double* q_ptr = nullptr;
  int q_k = -1, q_cols = 0;
  uint64_t q_ver[kMaxN] = {};
  // sampled correntropy loss: cores in FP64, merged halves, their gradients, partials
  DevBuf smpZ[kMaxN], smpA, smpC, smpGA, smpGC, smpGAd, smpGCd, smpPre, smpPost, smpDpart, smpD, smpLoss;
  DevBuf smpKa, smpKb, smpPa, smpPb, smpCa, smpCb, smpUa, smpUb, smpG;   // entry grouping
  // BF16 tensor-core operands and the padded mask rows of the current view
  DevBuf bShi, bSlo, bSh, bThi, bTlo, bTT;
  // observation bits re-laid per stationary index: [0] inner index along the outer one
  // (rows case), [1] outer index along the inner one (cols case); cached per view and split
  DevBuf Mst[2];
  const float* mst_X[2] = {nullptr, nullptr};
  const uint32_t* mst_M[2] = {nullptr, nullptr};
  int64_t mst_Pin[2] = {-1, -1}, mst_Pout[2] = {-1, -1};
  uint64_t mst_gen[2] = {~0ull, ~0ull};   // view (sketch) the relayout was made for
  int64_t mst_W[2] = {0, 0};
  int64_t ldT = 0, W = 0;
  bool tc_pass = false;         // the last pass 1 ran on the tensor cores
  // RStS index staging: a ring of pinned host slots, each reused only after the event recorded
  // behind its previous upload has completed (no host synchronisation per core update)
  static constexpr int kIdxSlots = 4;
  int32_t* idx_ring = nullptr;
  size_t idx_ring_cap = 0;      // int32 entries per slot
  cudaEvent_t idx_ev[kIdxSlots] = {};
  bool idx_ev_live[kIdxSlots] = {};
  int idx_slot = 0;
  DevBuf gbase;                 // RStS gather: offset in X of every fibre of the sketch
  DevBuf bShlo;                 // TF32: lo split of the step operand
  DevBuf bTThi, bTTlo;          // TF32: streaming splits transposed ([kpad][ldTT]), GEMM-2 operand
  HalfTag tagBTT;               // which merged half the transposed splits hold
  int64_t ldTT = 0;
  // the view's data re-laid with a row stride that is a multiple of 4 floats, for the
  // tensor-core passes when the inner block size P_in is not (TMA row strides are multiples
  // of 16 bytes); cached per view like the mask rows
  DevBuf Xpad;
  const float* xpad_src = nullptr;
  uint64_t xpad_gen = ~0ull;
  int64_t xpad_Pin = -1, xpad_Pout = -1;
  const float* Xtc = nullptr;   // data operand of the tensor-core passes (view.X or Xpad)
  int64_t ldx = 0;
  int mst_o = 0;
  int tcG = 0;
  // BF16: the weights of the last tensor-core pass 1 (one byte per slot, unit-major), read by
  // the line-search pass of the same core update instead of the data and the mask
  DevBuf wq;
  int wq_k = -1;                // core whose pass 1 wrote them (-1: none)
  uint64_t wq_gen = 0;
  int64_t wq_Pst = -1, wq_Pstr = -1;
  int wq_Kp = -1;
  bool wq_rows = false;
  // tracing: event pairs around data-pass launches (kind 0 = pass 1, 1 = pass 2)
  int prof = 0;            // 0 off, 1 data passes, 2 every phase
  // CUDA graph of a full (unsketched) trd_step: captured on the second consecutive step with
  // the same arguments and nothing else called in between, then replayed until another call
  // touches the handle
  struct GraphKey {
    double sigma = 0, lambda = 0;
    int gram = -1, prof = -1;
    bool operator==(const GraphKey& o) const {
      return sigma == o.sigma && lambda == o.lambda && gram == o.gram && prof == o.prof;
    }
  } gkey;
  // FGMC Gram + LDL^T of core k on a side stream while the data pass of core k runs (they
  // depend only on the other cores); the first pass then leaves kSideSMs SMs free
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_tail = nullptr;   // after the side stream's last work (chain prefix)
  bool side_tail = false;          // side work after the last join not yet waited for
  int pre_k = -1;            // core whose factor is being prepared on the side stream
  double pre_lambda = 0;
  int reserve_sms = 0;       // SMs the next tensor-core pass leaves to the side stream
  bool graphs_enabled = true;
  bool graph_ok = false;
  int steady = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_kernels = 0, graph_slots = 0;
  struct EvNodes { cudaGraphNode_t a, b; int kind; };
  std::vector<EvNodes> graph_ev;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending { cudaEvent_t a, b; int kind; };
  std::vector<Pending> pending;
  static constexpr int NPROF = 12;
  double prof_ms[NPROF] = {};
  int64_t prof_n[NPROF] = {};
  cudaEvent_t ev_open = nullptr;
};

Extra* X_(trd_handle* h);

bool is_fp64(const trd_handle* h) { return h->prec == TRD_FP64; }
// Whether the scaled step takes h from an explicit inverse formed on the side stream (K <= 128):
// only where the data pass is long enough to hide it.  The side stream has the two SMs the pass
// leaves free; the inverse (K one-warp substitution rows) fits under the TF32 x 3 and FP32
// passes (0.24 and 1 ms at 100^4, measured 2.48 -> 2.43 ms per TF32 x 3 step) but not under
// the BF16 pass 1 (0.12 ms: the step time did not change), and FP64 keeps its substitutions
// for the 1e-10 contract.
bool inverse_path(const trd_handle* h) { return h->prec == TRD_TF32X3 || h->prec == TRD_FP32; }
bool is_tf32(const trd_handle* h) { return h->prec == TRD_TF32X3; }
// the data passes of this contraction width run on the tensor cores (BF16 up to K' = 256,
// TF32 up to K' = 64); FP64, FP32 and wider TF32 contractions run the CUDA-core passes
bool tc_fits(const trd_handle* h, int Kp) {
  return (h->prec == TRD_BF16 || h->prec == TRD_TF32X3) && tc_kpad(Kp, is_tf32(h)) != 0;
}

cudaEvent_t pool_event(Extra* x) {
  if (!x->ev_pool.empty()) {
    cudaEvent_t e = x->ev_pool.back();
    x->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

void prof_begin(trd_handle* h) {
  Extra* x = X_(h);
  if (!x->prof) return;
  x->ev_open = pool_event(x);
  if (x->ev_open) cudaEventRecord(x->ev_open, h->stream);
}

void prof_end(trd_handle* h, int kind) {
  Extra* x = X_(h);
  if (!x->prof || !x->ev_open) return;
  cudaEvent_t b = pool_event(x);
  if (!b) return;
  cudaEventRecord(b, h->stream);
  x->pending.push_back({x->ev_open, b, kind});
  x->ev_open = nullptr;
}

// Phases of a core update timed by the tracing hook (kinds of event pairs).
enum : int { P_PASS1 = 0, P_PASS2 = 1, P_MERGE = 2, P_REDUCE = 3, P_GRAD = 4, P_GRAM = 5, P_CHOL = 6,
             P_SOLVE = 7, P_UPDATE = 8, P_SIGMA = 9, P_STOP = 10, P_GATHER = 11 };

// RAII phase scope: events around a phase, only at tracing level 2 (the data passes are traced
// from level 1); phases never nest.
struct PScope {
  trd_handle* h;
  int kind;
  bool on;
  PScope(trd_handle* hh, int k) : h(hh), kind(k), on(X_(hh)->prof >= 2) {
    if (on) prof_begin(h);
  }
  ~PScope() {
    if (on) prof_end(h, kind);
  }
};

// After a stream synchronisation: fold finished event pairs into the totals.
void prof_harvest(trd_handle* h) {
  Extra* x = X_(h);
  for (auto& p : x->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      x->prof_ms[p.kind] += ms;
      x->prof_n[p.kind] += 1;
    } else {
      cudaGetLastError();
    }
    x->ev_pool.push_back(p.a);
    x->ev_pool.push_back(p.b);
  }
  x->pending.clear();
}
void drop_graph(Extra* x) {
  if (x->graph_exec) cudaGraphExecDestroy(x->graph_exec);
  if (x->graph) cudaGraphDestroy(x->graph);
  x->graph_exec = nullptr;
  x->graph = nullptr;
  x->graph_ok = false;
  x->graph_ev.clear();
}

// Any call other than trd_step (and pure queries) ends graph replay: the captured step
// assumes the device state that the previous step left behind.
void touch(trd_handle* h) {
  Extra* x = X_(h);
  x->steady = 0;
  x->pre_k = -1;
  if (x->graph_ok || x->graph) drop_graph(x);
}

size_t elt(const trd_handle* h) { return is_fp64(h) ? sizeof(double) : sizeof(float); }

// The cut c of the ring (modes [0, c) and [c, N)) for mode sizes dim: the most balanced cut
// (by the logarithm of the two blocks' entry counts) among those whose contraction width
// R[0] R[c] the data passes take (FP64 112, the other precisions 256); when none does, the
// most balanced cut (*fits = false; the pass then reports it).  A ring with two large
// neighbouring ranks (the paper's video rank [80, 80, 3, 20]) is cut through its small edges
// instead of through the balanced but 6400-wide one.
int ring_cut(int N, const int64_t* dim, const int* R, int prec, bool* fits) {
  const int kmax = prec == TRD_FP64 ? 112 : 256;
  double best = 1e300, best_fit = 1e300;
  int bestc = 1, fitc = -1;
  for (int c = 1; c < N; ++c) {
    double a = 0, b = 0;
    for (int m = 0; m < c; ++m) a += log((double)dim[m]);
    for (int m = c; m < N; ++m) b += log((double)dim[m]);
    const double cost = fabs(a - b);
    if (cost < best - 1e-12) { best = cost; bestc = c; }
    if (R[0] * R[c] <= kmax && cost < best_fit - 1e-12) { best_fit = cost; fitc = c; }
  }
  if (fits) *fits = fitc > 0;
  return fitc > 0 ? fitc : bestc;
}

// Split of the view's modes into [0, c) and [c, N) at the cut above.
Split choose_split(const trd_handle* h, const View& v, int k) {
  Split sp;
  const int bestc = ring_cut(h->N, v.dim, h->R, h->prec, nullptr);
  sp.c = bestc;
  sp.P_in = 1;
  sp.P_out = 1;
  for (int m = 0; m < bestc; ++m) sp.P_in *= v.dim[m];
  for (int m = bestc; m < h->N; ++m) sp.P_out *= v.dim[m];
  sp.Kp = h->R[0] * h->R[bestc];
  sp.rows = k < bestc;
  sp.P_stat = sp.rows ? sp.P_in : sp.P_out;
  sp.P_strm = sp.rows ? sp.P_out : sp.P_in;
  return sp;
}

// Chain of cores m0..m1-1 over the view's digits; `subst` replaces core k by another array.
Chain make_chain(const trd_handle* h, const View& v, int m0, int m1, int ksub = -1,
                 const double* subst = nullptr, const double* const* cores = nullptr) {
  Chain ch;
  ch.n = m1 - m0;
  ch.count = 1;
  for (int j = 0; j < ch.n; ++j) {
    const int m = m0 + j;
    ch.core[j] = (m == ksub && subst) ? subst : (cores ? cores[m] : h->Z[m]);
    ch.coref[j] = ((m == ksub && subst) || cores) ? nullptr : h->Zf[m];
    ch.idx[j] = v.idx[m];
    ch.dim[j] = v.dim[m];
    ch.rows[j] = h->R[m];
    ch.cols[j] = h->R[(m + 1) % h->N];
    ch.count *= v.dim[m];
  }
  if (ch.n > 0) {
    ch.out_rows = ch.rows[0];
    ch.out_cols = ch.cols[ch.n - 1];
  }
  return ch;
}

View full_view(const trd_handle* h) {
  View v;
  v.X = h->X;
  v.M = h->M;
  v.N = h->N;
  v.numel = 1;
  for (int m = 0; m < h->N; ++m) {
    v.dim[m] = h->I[m];
    v.idx[m] = nullptr;
    v.numel *= h->I[m];
  }
  return v;
}

trd_status check_handle(trd_handle* h) {
  if (!h) return TRD_EINVAL;
  return TRD_OK;
}

trd_status check_k(trd_handle* h, int k) {
  if (k < 0 || k >= h->N) return set_err(h, TRD_EINVAL, "core index out of range");
  return TRD_OK;
}

trd_status sync_and_status(trd_handle* h) {
  CK(cudaStreamSynchronize(h->stream), "stream synchronize");
  int st = 0;
  CK(cudaMemcpy(&st, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost), "status read");
  if (st) {
    CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->stream), "status reset");
    if (st & DEV_SINGULAR) return set_err(h, TRD_ESINGULAR, "G + lambda I is not positive definite");
    if (st & DEV_NONFINITE) return set_err(h, TRD_ENONFINITE, "non-finite step size");
    if (st & DEV_TIMEOUT) return set_err(h, TRD_ETIMEOUT, "a device wait gave up");
    if (st & DEV_BOUNDS) return set_err(h, TRD_EINVAL, "an index was out of range (entries skipped)");
  }
  return TRD_OK;
}

// ------------------------------------------------------------------ FGMC
trd_status refresh_E(trd_handle* h, int k) {
  const int rk = h->R[k], rk1 = h->R[(k + 1) % h->N];
  TRY(ensure(h, X_(h)->Ework, sizeof(double) * 16 * (size_t)rk * rk * rk1 * rk1));
  CK(launch_fgmc_E(h->Z[k], nullptr, h->I[k], rk, rk1, h->E[k], (double*)X_(h)->Ework.p, h->stream),
     "fgmc factor");
  return TRD_OK;
}

// Refresh the FGMC factors of updated cores on the current stream before any Gram reads them.
trd_status fresh_E(trd_handle* h) {
  Extra* x = X_(h);
  for (int m = 0; m < h->N; ++m)
    if (x->e_stale[m]) {
      TRY(refresh_E(h, m));
      x->e_stale[m] = false;
    }
  return TRD_OK;
}

// G^{!=k} = Phi(E_{k+1} ... E_{k-1}) into `G` from the factors `E` (Prop. 2, E-form).
trd_status gram_chain(trd_handle* h, int k, double* const* E, double* G) {
  const int N = h->N;
  double* cur = nullptr;
  int rows = 0, cols = 0;
  double* bufs[2] = {(double*)h->T1.p, (double*)h->T2.p};
  int which = 0;
  for (int q = 0; q < N - 1; ++q) {
    const int m = (k + 1 + q) % N;
    const int rm = h->R[m], rm1 = h->R[(m + 1) % N];
    if (q == 0) {
      cur = E[m];
      rows = rm * rm;
      cols = rm1 * rm1;
      continue;
    }
    double* out = bufs[which];
    which ^= 1;
    CK(launch_dgemm(cur, E[m], out, rows, rm1 * rm1, cols, false, h->stream), "fgmc chain");
    cur = out;
    cols = rm1 * rm1;
  }
  CK(launch_phi(cur, h->R[(k + 1) % N], h->R[k], G, h->stream), "fgmc realign");
  return TRD_OK;
}

bool gram_valid(const trd_handle* h, int k) {
  if (h->gram_k != k) return false;
  for (int m = 0; m < h->N; ++m)
    if (m != k && h->gram_ver[m] != h->ver[m]) return false;
  return true;
}

bool q_valid(trd_handle* h, int k) {
  const Extra* x = X_(h);
  if (x->q_k != k || !x->q_ptr || h->N < 3) return false;
  for (int q = 1; q <= h->N - 2; ++q)
    if (x->q_ver[(k + q) % h->N] != h->ver[(k + q) % h->N]) return false;
  return true;
}

// Q = E_{k+1} ... E_{k+N-2} into the prefix buffers (N - 3 products; Q = E_{k+1} for N = 3).
trd_status build_q(trd_handle* h, int k) {
  Extra* x = X_(h);
  const int N = h->N;
  if (N < 3) return TRD_OK;
  TRY(fresh_E(h));
  size_t chain = 1;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) chain = std::max(chain, (size_t)h->R[a] * h->R[a] * h->R[b] * h->R[b]);
  TRY(ensure(h, x->Qb[0], sizeof(double) * chain));
  TRY(ensure(h, x->Qb[1], sizeof(double) * chain));
  const int m0 = (k + 1) % N;
  const double* cur = h->E[m0];
  const int rows = h->R[m0] * h->R[m0];
  int cols = h->R[(m0 + 1) % N] * h->R[(m0 + 1) % N];
  int which = 0;
  for (int q = 2; q <= N - 2; ++q) {
    const int m = (k + q) % N;
    const int rm1 = h->R[(m + 1) % N];
    double* out = (double*)x->Qb[which].p;
    which ^= 1;
    CK(launch_dgemm(cur, h->E[m], out, rows, rm1 * rm1, cols, false, h->stream), "fgmc prefix");
    cur = out;
    cols = rm1 * rm1;
  }
  x->q_ptr = cur;
  x->q_k = k;
  x->q_cols = cols;
  for (int q = 1; q <= N - 2; ++q) x->q_ver[(k + q) % N] = h->ver[(k + q) % N];
  return TRD_OK;
}

trd_status ensure_gram(trd_handle* h, int k) {
  if (gram_valid(h, k)) return TRD_OK;
  TRY(fresh_E(h));
  if (q_valid(h, k)) {
    // G = Phi(Q E_{k-1}): the prefix was formed during the previous core's update
    const Extra* x = X_(h);
    const int N = h->N, ml = (k + N - 1) % N;
    const int rows = h->R[(k + 1) % N] * h->R[(k + 1) % N], cols = h->R[k] * h->R[k];
    CK(launch_dgemm(x->q_ptr, h->E[ml], (double*)h->T1.p, rows, cols, x->q_cols, false, h->stream), "fgmc chain");
    CK(launch_phi((const double*)h->T1.p, h->R[(k + 1) % N], h->R[k], (double*)h->G.p, h->stream), "fgmc realign");
  } else {
    double* E[kMaxN];
    for (int m = 0; m < h->N; ++m) E[m] = h->E[m];
    TRY(gram_chain(h, k, E, (double*)h->G.p));
  }
  h->gram_k = k;
  for (int m = 0; m < h->N; ++m) h->gram_ver[m] = h->ver[m];
  return TRD_OK;
}

// Local Gram of the sampled cores (ablation 'local scaled term'): FGMC on sampled factors.
trd_status local_gram(trd_handle* h, int k) {
  Extra* x = X_(h);
  double* E[kMaxN];
  for (int m = 0; m < h->N; ++m) {
    if (m == k) { E[m] = h->E[m]; continue; }
    const int rm = h->R[m], rm1 = h->R[(m + 1) % h->N];
    TRY(ensure(h, x->Eloc[m], sizeof(double) * rm * rm * rm1 * rm1));
    const bool sampled = h->view.idx[m] != nullptr;
    CK(launch_fgmc_E(h->Z[m], h->view.idx[m], sampled ? h->view.dim[m] : h->I[m], rm, rm1,
                     (double*)x->Eloc[m].p, nullptr, h->stream), "local fgmc factor");
    E[m] = (double*)x->Eloc[m].p;
  }
  const int K = h->K[k];
  TRY(ensure(h, x->Gloc, sizeof(double) * K * K));
  return gram_chain(h, k, E, (double*)x->Gloc.p);
}

trd_status compute_D(trd_handle* h, double* D) {
  const int n = h->N - 1;
  TRY(ensure_gram(h, n));
  const int I = (int)h->I[n], K = h->K[n];
  CK(launch_dgemm(h->Z[n], (const double*)h->G.p, (double*)h->h.p, I, K, K, false, h->stream), "D step 1");
  CK(launch_dgemm((const double*)h->h.p, h->Z[n], D, I, I, K, true, h->stream), "D step 2");
  return TRD_OK;
}

trd_status reset_D0(trd_handle* h) {
  TRY(compute_D(h, (double*)h->Dprev.p));
  h->have_D0 = true;
  return TRD_OK;
}

// ------------------------------------------------------------------ data passes
HalfTag half_tag(trd_handle* h, int half, const Split& sp) {
  HalfTag t;
  t.valid = true;
  t.half = half;
  t.view_gen = X_(h)->view_gen;
  t.c = sp.c;
  t.Kp = sp.Kp;
  const int m0 = half == 0 ? 0 : sp.c, m1 = half == 0 ? sp.c : h->N;
  for (int m = m0; m < m1; ++m) t.ver[m] = h->ver[m];
  return t;
}

// Row sampling: the stationary operand is Z_{k(2)} itself (I_k x K), the streaming one the
// sampled rows B (J x K); the contraction index is alpha + beta r_k on both sides.
Split row_split(const trd_handle* h, int k, int64_t J) {
  Split sp;
  sp.c = 1;
  sp.P_in = h->I[k];
  sp.P_out = J;
  sp.Kp = h->K[k];
  sp.rows = true;
  sp.P_stat = sp.P_in;
  sp.P_strm = J;
  return sp;
}

RowsArgs rows_args(const trd_handle* h, int k, int64_t J) {
  RowsArgs a;
  a.N = h->N;
  a.k = k;
  a.Ik = h->I[k];
  a.J = J;
  int64_t st = 1;
  for (int m = 0; m < h->N; ++m) {
    a.stride[m] = st;
    st *= h->I[m];
    a.R[m] = h->R[m];
    a.Z[m] = h->Z[m];
    a.Zf[m] = h->Zf[m];
  }
  return a;
}

trd_status build_rows_operands(trd_handle* h, int k) {
  Extra* x = X_(h);
  bool fresh = x->rows_gen == x->view_gen;
  for (int m = 0; m < h->N && fresh; ++m) fresh = x->rows_ver[m] == h->ver[m];
  if (fresh) return TRD_OK;
  const int64_t J = x->rows_J;
  const size_t e = elt(h);
  TRY(ensure(h, h->Sst, e * h->I[k] * h->K[k]));
  TRY(ensure(h, h->Sstr, e * J * h->K[k]));
  // Z_{k(2)} is the core's own layout (row i, column alpha + beta r_k)
  CK(launch_from_double(h->Z[k], h->I[k] * (int64_t)h->K[k], h->Sst.p, is_fp64(h), h->stream), "Z_k operand");
  CK(launch_rows_chain(rows_args(h, k, J), (const int32_t*)x->rows_dev.p, h->Sstr.p, is_fp64(h), h->stream),
     "sampled rows");
  x->tagSst.valid = x->tagSstr.valid = x->tagBst.valid = x->tagBstr.valid = false;
  x->rows_gen = x->view_gen;
  for (int m = 0; m < h->N; ++m) x->rows_ver[m] = h->ver[m];
  return TRD_OK;
}

// Merged halves of the current view into h->Sst (the stationary role: the half holding
// core k) and h->Sstr.  The two buffers keep what they hold between calls: a half whose cores
// and view are unchanged is not merged again (buffers trade roles when k crosses the cut).
trd_status build_halves(trd_handle* h, int k) {
  Extra* x = X_(h);
  if (x->row_view) return build_rows_operands(h, k);
  const Split& sp = h->split;
  const int hs = k < sp.c ? 0 : 1;
  const HalfTag want_st = half_tag(h, hs, sp), want_str = half_tag(h, 1 - hs, sp);
  // BF16 handles: the tensor-core operands (hi/lo, KP-wide rows) are written by the same
  // merge and trade roles together with the FP32 halves
  const int KP = (h->prec == TRD_BF16 && tc_fits(h, sp.Kp)) ? tc_kpad(sp.Kp, false) : 0;
  if (x->tagSst == want_str || x->tagSstr == want_st) {
    std::swap(h->Sst, h->Sstr);
    std::swap(x->tagSst, x->tagSstr);
    if (KP) {
      std::swap(x->bShi, x->bThi);
      std::swap(x->bSlo, x->bTlo);
      std::swap(x->tagBst, x->tagBstr);
    }
  }
  const size_t e = elt(h);
  const bool dbl = is_fp64(h);
  const void* pst = h->Sst.p;
  const void* pstr = h->Sstr.p;
  TRY(ensure(h, h->Sst, e * sp.P_stat * sp.Kp));
  TRY(ensure(h, h->Sstr, e * sp.P_strm * sp.Kp));
  if (h->Sst.p != pst) x->tagSst.valid = false;
  if (h->Sstr.p != pstr) x->tagSstr.valid = false;
  if (KP) {
    const size_t b2 = sizeof(__nv_bfloat16);
    const void* q[4] = {x->bShi.p, x->bSlo.p, x->bThi.p, x->bTlo.p};
    TRY(ensure(h, x->bShi, b2 * sp.P_stat * KP));
    TRY(ensure(h, x->bSlo, b2 * sp.P_stat * KP));
    TRY(ensure(h, x->bThi, b2 * sp.P_strm * KP));
    TRY(ensure(h, x->bTlo, b2 * sp.P_strm * KP));
    if (x->bShi.p != q[0] || x->bSlo.p != q[1]) x->tagBst.valid = false;
    if (x->bThi.p != q[2] || x->bTlo.p != q[3]) x->tagBstr.valid = false;
  }
  const View& v = h->view;
  const Chain inner = make_chain(h, v, 0, sp.c), outer = make_chain(h, v, sp.c, h->N);
  if (!(x->tagSst == want_st) || (KP && !(x->tagBst == want_st))) {
    CK(launch_chain(hs == 0 ? inner : outer, h->Sst.p, dbl, hs == 1, sp.Kp, h->stream,
                    KP ? (__nv_bfloat16*)x->bShi.p : nullptr, KP ? (__nv_bfloat16*)x->bSlo.p : nullptr, KP),
       "merge stationary half");
    x->tagSst = want_st;
    if (KP) x->tagBst = want_st;
  }
  if (!(x->tagSstr == want_str) || (KP && !(x->tagBstr == want_str))) {
    CK(launch_chain(hs == 0 ? outer : inner, h->Sstr.p, dbl, hs == 0, sp.Kp, h->stream,
                    KP ? (__nv_bfloat16*)x->bThi.p : nullptr, KP ? (__nv_bfloat16*)x->bTlo.p : nullptr, KP),
       "merge streaming half");
    x->tagSstr = want_str;
    if (KP) x->tagBstr = want_str;
  }
  return TRD_OK;
}

trd_status build_merged(trd_handle* h, int k, bool with_h, __nv_bfloat16* bf16_h = nullptr, int kpad = 0,
                        void* fp32_h = nullptr) {
  const View& v = h->view;
  const Split& sp = h->split;
  const int c = sp.c, Kp = sp.Kp;
  const bool dbl = is_fp64(h);
  const size_t e = elt(h);
  if (!with_h) return build_halves(h, k);
  if (X_(h)->row_view) {
    // the step direction h (I_k x K, same layout as Z_{k(2)}) is the stationary operand
    TRY(ensure(h, h->Sh, e * sp.P_stat * Kp));
    CK(launch_from_double((const double*)h->h.p, sp.P_stat * (int64_t)Kp, h->Sh.p, dbl, h->stream), "h operand");
    return TRD_OK;
  }
  const Chain inner = make_chain(h, v, 0, c, k, (const double*)h->h.p);
  const Chain outer = make_chain(h, v, c, h->N, k, (const double*)h->h.p);
  if (bf16_h) {
    // tensor-core path: the BF16 operand of the step direction (and, when asked, its FP32 form
    // for advancing the merged half in place after the step)
    if (sp.rows) CK(launch_chain(inner, fp32_h, dbl, false, Kp, h->stream, bf16_h, nullptr, kpad), "merge A_h");
    else CK(launch_chain(outer, fp32_h, dbl, true, Kp, h->stream, bf16_h, nullptr, kpad), "merge C_h");
    return TRD_OK;
  }
  TRY(ensure(h, h->Sh, e * sp.P_stat * Kp));
  if (sp.rows) CK(launch_chain(inner, h->Sh.p, dbl, false, Kp, h->stream), "merge A_h");
  else CK(launch_chain(outer, h->Sh.p, dbl, true, Kp, h->stream), "merge C_h");
  return TRD_OK;
}

// Column splits of the CUDA-core pass: the grid (row blocks x splits) should fill whole waves
// of resident CTAs; among 1..16 splits take the best filled last wave (the fewest splits on
// ties), since a grid just above a wave doubles the time.
int choose_splits(const trd_handle* h, const Split& sp) {
  const int64_t gx = (sp.P_stat + 63) / 64;
  const int64_t tiles = (sp.P_strm + 63) / 64;
  const int64_t resident = (int64_t)simt_blocks_per_sm(is_fp64(h), sp.rows, sp.Kp) * h->num_sms;
  int64_t best = 1;
  double best_eff = -1.0;
  for (int64_t s = 1; s <= imin(16, tiles); ++s) {
    const int64_t blocks = gx * s;
    const int64_t waves = (blocks + resident - 1) / resident;
    const double eff = (double)blocks / (double)(waves * resident);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = s;
    }
  }
  return (int)best;
}

PassArgs pass_args(trd_handle* h) {
  PassArgs a{};
  const Split& sp = h->split;
  a.X = h->view.X;
  a.M = h->view.M;
  a.P_in = sp.P_in;
  a.P_stat = sp.P_stat;
  a.P_strm = sp.P_strm;
  a.Kp = sp.Kp;
  a.ld = sp.Kp;
  a.Sst = h->Sst.p;
  a.Sh = h->Sh.p;
  a.Sstr = h->Sstr.p;
  a.sigma = h->scal + S_SIGMA;
  a.Tpart = h->Tpart.p;
  a.stat_part = (double*)h->stat_part.p;
  return a;
}

// BF16 hi/lo operands of the two merged halves (rows zero-padded to the tensor-core K),
// cached like the halves themselves.
trd_status tc_operands(trd_handle* h) {
  const Split& sp = h->split;
  Extra* x = X_(h);
  const bool tf = is_tf32(h);
  const int KP = tc_kpad(sp.Kp, tf);
  if (x->tagBst == x->tagSstr || x->tagBstr == x->tagSst) {
    std::swap(x->bShi, x->bThi);
    std::swap(x->bSlo, x->bTlo);
    std::swap(x->tagBst, x->tagBstr);
  }
  const size_t b2 = tf ? sizeof(float) : sizeof(__nv_bfloat16);
  const void* p0 = x->bShi.p;
  const void* p1 = x->bSlo.p;
  const void* p2 = x->bThi.p;
  const void* p3 = x->bTlo.p;
  TRY(ensure(h, x->bShi, b2 * sp.P_stat * KP));
  TRY(ensure(h, x->bSlo, b2 * sp.P_stat * KP));
  TRY(ensure(h, x->bThi, b2 * sp.P_strm * KP));
  TRY(ensure(h, x->bTlo, b2 * sp.P_strm * KP));
  if (x->bShi.p != p0 || x->bSlo.p != p1) x->tagBst.valid = false;
  if (x->bThi.p != p2 || x->bTlo.p != p3) x->tagBstr.valid = false;
  if (!(x->tagBst == x->tagSst)) {
    if (tf)
      CK(launch_tc_prep_tf32((const float*)h->Sst.p, sp.P_stat, sp.Kp, (float*)x->bShi.p, (float*)x->bSlo.p,
                             h->stream), "tf32 stationary operands");
    else
      CK(launch_tc_prep((const float*)h->Sst.p, sp.P_stat, sp.Kp, (__nv_bfloat16*)x->bShi.p,
                        (__nv_bfloat16*)x->bSlo.p, h->stream), "bf16 stationary operands");
    x->tagBst = x->tagSst;
  }
  if (tf) {
    const int64_t ld = (sp.P_strm + 3) / 4 * 4;
    const void* q0 = x->bTThi.p;
    const void* q1 = x->bTTlo.p;
    TRY(ensure(h, x->bTThi, sizeof(float) * (size_t)(KP * ld)));
    TRY(ensure(h, x->bTTlo, sizeof(float) * (size_t)(KP * ld)));
    if (x->bTThi.p != q0 || x->bTTlo.p != q1 || x->ldTT != ld) x->tagBTT.valid = false;
    x->ldTT = ld;
  }
  if (!(x->tagBstr == x->tagSstr) || (tf && !(x->tagBTT == x->tagSstr))) {
    if (tf) {
      CK(launch_tc_prep_tf32((const float*)h->Sstr.p, sp.P_strm, sp.Kp, (float*)x->bThi.p, (float*)x->bTlo.p,
                             h->stream, (float*)x->bTThi.p, (float*)x->bTTlo.p, x->ldTT),
         "tf32 streaming operands");
      x->tagBTT = x->tagSstr;
    }
    else
      CK(launch_tc_prep((const float*)h->Sstr.p, sp.P_strm, sp.Kp, (__nv_bfloat16*)x->bThi.p,
                        (__nv_bfloat16*)x->bTlo.p, h->stream), "bf16 streaming operands");
    x->tagBstr = x->tagSstr;
  }
  return TRD_OK;
}

trd_status run_pass1_tc(trd_handle* h, int k, bool full_stats) {
  const Split& sp = h->split;
  Extra* x = X_(h);
  const int KP = tc_kpad(sp.Kp, is_tf32(h));
  if (!KP) return set_err(h, TRD_ENOTIMPL, "tensor-core path supports r_1 r_c <= 256 (BF16) / 64 (TF32)");
  const View& v = h->view;
  const int64_t RB = (sp.P_stat + tc_bm() - 1) / tc_bm();
  const int64_t NT = (sp.P_strm + tc_bn(KP, is_tf32(h)) - 1) / tc_bn(KP, is_tf32(h));
  const int G = (int)imin(imax(1, h->num_sms - x->reserve_sms), RB * NT);
  const int o = sp.rows ? 0 : 1;
  const int64_t nstat = sp.rows ? sp.P_in : sp.P_out, nstrm = sp.rows ? sp.P_out : sp.P_in;
  const int64_t W = ((nstrm + 31) / 32 + 3) / 4 * 4;
  {
  PScope ps(h, P_MERGE);
  TRY(build_merged(h, k, false));
  // observation bits of every stationary index along the streaming index (cached)
  if (x->mst_X[o] != v.X || x->mst_M[o] != v.M || x->mst_Pin[o] != sp.P_in || x->mst_Pout[o] != sp.P_out ||
      x->mst_gen[o] != x->view_gen) {
    TRY(ensure(h, x->Mst[o], sizeof(uint32_t) * (size_t)(nstat * W)));
    if (sp.rows)
      CK(launch_mask_transpose(v.M, sp.P_in, sp.P_out, W, (uint32_t*)x->Mst[o].p, h->stream), "mask layout");
    else
      CK(launch_mask_rows(v.M, sp.P_in, sp.P_out, W, (uint32_t*)x->Mst[o].p, h->stream), "mask layout");
    x->mst_X[o] = v.X;
    x->mst_M[o] = v.M;
    x->mst_Pin[o] = sp.P_in;
    x->mst_Pout[o] = sp.P_out;
    x->mst_gen[o] = x->view_gen;
  }
  x->W = W;
  x->mst_o = o;
  if (sp.P_in % 4 == 0) {
    x->Xtc = v.X;
    x->ldx = sp.P_in;
  } else {
    const int64_t ld = (sp.P_in + 3) / 4 * 4;
    if (x->xpad_src != v.X || x->xpad_gen != x->view_gen || x->xpad_Pin != sp.P_in || x->xpad_Pout != sp.P_out) {
      TRY(ensure(h, x->Xpad, sizeof(float) * (size_t)(ld * sp.P_out)));
      CK(launch_pad_rows(v.X, sp.P_in, sp.P_out, ld, (float*)x->Xpad.p, h->stream), "padded data rows");
      x->xpad_src = v.X;
      x->xpad_gen = x->view_gen;
      x->xpad_Pin = sp.P_in;
      x->xpad_Pout = sp.P_out;
    }
    x->Xtc = (const float*)x->Xpad.p;
    x->ldx = ld;
  }
  const int64_t ldT = (sp.P_strm + 63) / 64 * 64;
  x->ldT = ldT;
  TRY(tc_operands(h));
  }
  x->tcG = G;
  TRY(ensure(h, h->Tpart, sizeof(float) * (size_t)(G + RB) * tc_bm() * sp.Kp));
  TRY(ensure(h, h->stat_part, sizeof(double) * 8 * (size_t)G));
  TRY(ensure(h, h->Tsum, sizeof(double) * (size_t)sp.P_stat * sp.Kp));
  prof_begin(h);
  PassOperands ops;
  ops.S_hi = x->bShi.p;
  ops.S_lo = x->bSlo.p;
  ops.T_hi = x->bThi.p;
  ops.T_lo = x->bTlo.p;
  if (is_tf32(h)) {
    ops.T_hiT = x->bTThi.p;
    ops.T_loT = x->bTTlo.p;
    ops.ldT = x->ldTT;
  }
  unsigned char* wq = nullptr;
  if (!is_tf32(h)) {
    TRY(ensure(h, x->wq, (size_t)tc_wq_bytes(sp.Kp, sp.P_stat, sp.P_strm)));
    wq = (unsigned char*)x->wq.p;
  }
  x->wq_k = -1;
  CK(launch_pass_tc(is_tf32(h), sp.rows, false, ops, x->Xtc, sp.P_in, x->ldx, sp.P_out, (const uint32_t*)x->Mst[o].p, W, sp.P_stat, sp.P_strm, sp.Kp,
                    h->scal + S_SIGMA, (float*)h->Tpart.p, (double*)h->stat_part.p, h->dstatus, G, full_stats,
                    h->stream, wq),
     "tensor-core data pass 1");
  if (wq) {
    x->wq_k = k;
    x->wq_gen = x->view_gen;
    x->wq_Pst = sp.P_stat;
    x->wq_Pstr = sp.P_strm;
    x->wq_Kp = sp.Kp;
    x->wq_rows = sp.rows;
  }
  prof_end(h, 0);
  PScope ps(h, P_REDUCE);
  // the back-contraction sums the partial slots itself; the row-sampling gradient is the
  // reduced contraction, so it is formed here
  x->slots = SlotSrc{(const float*)h->Tpart.p, RB, NT, (int64_t)tc_bm(), G};
  if (x->row_view)
    CK(launch_reduce_slots((const float*)h->Tpart.p, RB, NT, G, sp.P_stat, sp.Kp, (double*)h->Tsum.p, h->stream),
       "reduce contraction");
  CK(launch_reduce_stats((const double*)h->stat_part.p, G, (double*)h->stat_sum.p, h->dstatus, h->stream,
                         x->obj_slot),
     "reduce statistics");
  h->ctas = G;
  return TRD_OK;
}

trd_status run_pass2_tc(trd_handle* h, int k, double** den) {
  const Split& sp = h->split;
  Extra* x = X_(h);
  const bool tf = is_tf32(h);
  const int KP = tc_kpad(sp.Kp, tf);
  {
    PScope ps(h, P_MERGE);
    TRY(build_halves(h, k));      // normally cached: restores the roles of core k
    TRY(tc_operands(h));
    if (tf) {
      // TF32: the step operand merged in FP32 and split into TF32 hi / lo rows
      TRY(ensure(h, x->bSh, sizeof(float) * sp.P_stat * KP));
      TRY(ensure(h, x->bShlo, sizeof(float) * sp.P_stat * KP));
      TRY(build_merged(h, k, true));
      CK(launch_tc_prep_tf32((const float*)h->Sh.p, sp.P_stat, sp.Kp, (float*)x->bSh.p, (float*)x->bShlo.p,
                             h->stream), "tf32 step operands");
    } else if (x->row_view) {
      TRY(ensure(h, x->bSh, sizeof(__nv_bfloat16) * sp.P_stat * KP));
      TRY(build_merged(h, k, true));
      CK(launch_tc_prep((const float*)h->Sh.p, sp.P_stat, sp.Kp, (__nv_bfloat16*)x->bSh.p, nullptr, h->stream),
         "bf16 step operands");
    } else {
      // the step operand in FP32 too: after the step the stationary half (which holds core k)
      // is advanced in place, S += eta S_h, instead of being merged again
      TRY(ensure(h, x->bSh, sizeof(__nv_bfloat16) * sp.P_stat * KP));
      TRY(ensure(h, h->Sh, sizeof(float) * sp.P_stat * sp.Kp));
      TRY(build_merged(h, k, true, (__nv_bfloat16*)x->bSh.p, KP, h->Sh.p));
      x->adv_k = k;
    }
  }
  // the side stream has joined: the line-search pass takes every SM (its per-CTA partials are
  // summed by the update kernel over the same count)
  {
    const int BN = tc_bn(KP, tf);
    const int64_t units = ((sp.P_stat + tc_bm() - 1) / tc_bm()) * ((sp.P_strm + BN - 1) / BN);
    x->tcG = (int)imin(h->num_sms, units);
    TRY(ensure(h, h->stat_part, sizeof(double) * 8 * (size_t)x->tcG));
  }
  PassOperands ops;
  ops.S_hi = x->bShi.p;
  ops.S_lo = x->bSlo.p;
  ops.S_h = x->bSh.p;
  ops.S_h_lo = tf ? x->bShlo.p : nullptr;
  ops.T_hi = x->bThi.p;
  ops.T_lo = x->bTlo.p;
  // BF16 after this core's pass 1 on the same view: the line search reads pass 1's weights
  const bool cached = !tf && h->pass1_k == k && x->wq_k == k && x->wq_gen == x->view_gen &&
                      x->wq_Pst == sp.P_stat && x->wq_Pstr == sp.P_strm && x->wq_Kp == sp.Kp && x->wq_rows == sp.rows;
  prof_begin(h);
  if (cached)
    CK(launch_pass_wls(x->bSh.p, x->bThi.p, (const unsigned char*)x->wq.p, sp.Kp, sp.P_stat, sp.P_strm,
                       (double*)h->stat_part.p, h->dstatus, x->tcG, (const double*)h->stat_sum.p + 4, h->stream),
       "line-search pass from cached weights");
  else
    CK(launch_pass_tc(tf, sp.rows, true, ops, x->Xtc, sp.P_in, x->ldx, sp.P_out,
                      (const uint32_t*)x->Mst[x->mst_o].p, x->W, sp.P_stat, sp.P_strm, sp.Kp, h->scal + S_SIGMA,
                      (float*)h->Tpart.p, (double*)h->stat_part.p, h->dstatus, x->tcG, false, h->stream),
       "tensor-core data pass 2");
  prof_end(h, 1);
  // the line-search denominator is summed from the per-CTA partials by the update kernel
  *den = nullptr;
  return TRD_OK;
}

trd_status run_pass1(trd_handle* h, int k, bool full_stats = true) {
  if (X_(h)->row_view && X_(h)->row_k != k)
    return set_err(h, TRD_EINVAL, "the current row sample was drawn for another core");
  h->split = X_(h)->row_view ? row_split(h, k, X_(h)->rows_J) : choose_split(h, h->view, k);
  const Split& sp = h->split;
  X_(h)->tc_pass = tc_fits(h, sp.Kp);
  if (h->prec == TRD_BF16 && !X_(h)->tc_pass)
    return set_err(h, TRD_ENOTIMPL, "BF16 path supports r_1 r_c <= 256");
  if (X_(h)->tc_pass) {
    TRY(run_pass1_tc(h, k, full_stats));
  } else {
    if (sp.Kp > 112 && is_fp64(h)) return set_err(h, TRD_ENOTIMPL, "FP64 path supports r_1 r_c <= 112");
    if (sp.Kp > 256) return set_err(h, TRD_ENOTIMPL, "data passes support r_1 r_c <= 256");
    {
      PScope ps(h, P_MERGE);
      TRY(build_merged(h, k, false));
    }
    int splits = choose_splits(h, sp);
    const int64_t gx = (sp.P_stat + 63) / 64;
    TRY(ensure(h, h->Tpart, elt(h) * (size_t)splits * sp.P_stat * sp.Kp));
    TRY(ensure(h, h->stat_part, sizeof(double) * 8 * (size_t)(gx * splits)));
    TRY(ensure(h, h->Tsum, sizeof(double) * (size_t)sp.P_stat * sp.Kp));
    int ctas = 0, used = 0;
    PassArgs a = pass_args(h);
    prof_begin(h);
    CK(launch_pass_simt(a, is_fp64(h), sp.rows, false, splits, &ctas, &used, h->stream), "data pass 1");
    prof_end(h, 0);
    h->splits = used;
    h->ctas = ctas;
    PScope ps(h, P_REDUCE);
    CK(launch_reduce_T(h->Tpart.p, is_fp64(h), used, sp.P_stat * (int64_t)sp.Kp, (double*)h->Tsum.p,
                       h->stream), "reduce contraction");
    CK(launch_reduce_stats((const double*)h->stat_part.p, ctas, (double*)h->stat_sum.p, h->dstatus, h->stream,
                           X_(h)->obj_slot),
       "reduce statistics");
  }
  h->pass1_k = k;
  h->grad_k = -1;
  h->slots_last = h->view.numel;
  return TRD_OK;
}

// a one-core subchain product, read in place by the back-contraction
BcCore bc_core(const Chain& ch) {
  BcCore c;
  if (ch.n == 1) {
    c.core = ch.core[0];
    c.coref = ch.coref[0];
    c.idx = ch.idx[0];
  }
  return c;
}

// split count of the back-contraction: about two (pre, post) pairs per warp of a block, and
// no more blocks than stay resident at once (eight per SM), so that one wave covers the grid
int64_t bc_splits(const trd_handle* h, int64_t npairs, int64_t rows) {
  const int64_t resident = 8 * (int64_t)h->num_sms;
  return imax(1, imin(imin((npairs + 7) / 8, 256), resident / imax(1, rows)));
}

// zeroed completion counters for n rows (each launch's last block resets its row's counter)
trd_status bc_counters(trd_handle* h, int64_t n) {
  Extra* x = X_(h);
  const size_t bytes = sizeof(unsigned) * (size_t)n;
  if (x->bc_ctr.p && x->bc_ctr.bytes >= bytes) return TRD_OK;
  TRY(ensure(h, x->bc_ctr, bytes));
  CK(cudaMemsetAsync(x->bc_ctr.p, 0, x->bc_ctr.bytes, h->stream), "counter");
  return TRD_OK;
}

trd_status run_gradient(trd_handle* h, int k) {
  if (h->pass1_k != k) return set_err(h, TRD_EINVAL, "trd_residual_weights must run for this core first");
  PScope ps(h, P_GRAD);
  if (X_(h)->row_view) {
    // T = Y B is the gradient itself (I_k x K, column alpha + beta r_k)
    TRY(ensure(h, h->d, sizeof(double) * h->I[k] * h->K[k]));
    CK(cudaMemcpyAsync(h->d.p, h->Tsum.p, sizeof(double) * h->I[k] * h->K[k], cudaMemcpyDeviceToDevice, h->stream),
       "gradient");
    h->grad_k = k;
    return TRD_OK;
  }
  const View& v = h->view;
  const Split& sp = h->split;
  const int N = h->N, c = sp.c;
  const int rk = h->R[k], rk1 = h->R[(k + 1) % N];
  int pre0, pre1, post0, post1, mr, mc;
  if (sp.rows) {
    pre0 = 0; pre1 = k; post0 = k + 1; post1 = c;
    mr = h->R[c]; mc = h->R[0];
  } else {
    pre0 = c; pre1 = k; post0 = k + 1; post1 = N;
    mr = h->R[0]; mc = h->R[c];
  }
  const Chain pre = make_chain(h, v, pre0, pre1);
  const Chain post = make_chain(h, v, post0, post1);
  const int64_t n_pre = pre.n > 0 ? pre.count : 1;
  const int64_t n_post = post.n > 0 ? post.count : 1;
  const bool dbl = is_fp64(h);
  const size_t e = elt(h);
  // one-core products are read from the cores by the back-contraction itself
  if (pre.n > 1) {
    TRY(ensure(h, h->pre, e * n_pre * mc * rk));
    CK(launch_chain(pre, h->pre.p, dbl, false, mc * rk, h->stream), "merge prefix");
  }
  if (post.n > 1) {
    TRY(ensure(h, h->post, e * n_post * rk1 * mr));
    CK(launch_chain(post, h->post.p, dbl, false, rk1 * mr, h->stream), "merge suffix");
  }
  const int64_t nsplit = bc_splits(h, n_pre * n_post, h->I[k]);
  const int K = h->K[k];
  TRY(ensure(h, h->d, sizeof(double) * h->I[k] * K));
  if (nsplit > 1) TRY(ensure(h, h->dpart, sizeof(double) * nsplit * h->I[k] * K));
  TRY(bc_counters(h, h->I[k]));
  CK(launch_backcontract(h->Tsum.p, sp.Kp, sp.rows, mr, mc, pre.n > 1 ? h->pre.p : nullptr, n_pre,
                         post.n > 1 ? h->post.p : nullptr, n_post, h->I[k], rk, rk1, (double*)h->dpart.p,
                         (int)nsplit, (double*)h->d.p, (unsigned*)X_(h)->bc_ctr.p, dbl, h->stream,
                         X_(h)->tc_pass ? &X_(h)->slots : nullptr, bc_core(pre), bc_core(post)),
     "back-contraction");
  h->grad_k = k;
  return TRD_OK;
}

// Fork: the FGMC Gram of core k and its LDL^T factorisation on the side stream, ordered after
// everything already on the main stream (the other cores are final for this update).  The
// join is in run_update.  Falls back (returns false) when not applicable.
constexpr int kSideSMs = 2;
bool prefactor(trd_handle* h, int k, double lambda) {
  Extra* x = X_(h);
  const int K = h->K[k];
  if (!ldl_fits(K) || h->N < 3) return false;
  if (!x->side) {
    if (cudaStreamCreateWithFlags(&x->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&x->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x->ev_tail, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  }
  if (!x->solve_ctr.p) {
    if (ensure(h, x->solve_ctr, 256) != TRD_OK) return false;
    if (cudaMemsetAsync(x->solve_ctr.p, 0, 256, h->stream) != cudaSuccess) return false;
  }
  if (cudaEventRecord(x->ev_fork, h->stream) != cudaSuccess ||
      cudaStreamWaitEvent(x->side, x->ev_fork, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaStream_t main_stream = h->stream;
  h->stream = x->side;       // the phase scopes below trace the side stream
  pdl_on = false;            // plain launches on the side stream (restored below)
  trd_status st;
  {
    PScope ps(h, P_GRAM);
    st = ensure_gram(h, k);
  }
  x->minv_k = -1;
  if (st == TRD_OK) {
    PScope ps(h, P_CHOL);
    double* Lcm = (double*)h->L.p;
    if (launch_ldl_factor((const double*)h->G.p, K, lambda, Lcm, Lcm + (size_t)K * K, h->scal, h->dstatus,
                          x->side) != cudaSuccess)
      st = TRD_ECUDA;
    if (st == TRD_OK && inverse_path(h)) {
      // the explicit inverse from the factor (the 1e-5 contract leaves room for the inverse's
      // rounding; the FP64 path keeps the substitutions)
      if (ensure(h, x->Minv, sizeof(double) * (size_t)K * K) != TRD_OK ||
          ensure(h, x->Ident, sizeof(double) * (size_t)K * K) != TRD_OK ||
          ensure(h, x->inv_dot, sizeof(double) * (size_t)K) != TRD_OK || ensure(h, x->inv_num, 64) != TRD_OK) {
        st = TRD_ENOMEM;
      } else {
        if (!x->inv_ctr.p) {
          if (ensure(h, x->inv_ctr, 256) != TRD_OK || cudaMemsetAsync(x->inv_ctr.p, 0, 256, x->side) != cudaSuccess)
            st = TRD_ECUDA;
        }
        if (st == TRD_OK && x->ident_K != K) {
          if (launch_identity((double*)x->Ident.p, K, x->side) != cudaSuccess) st = TRD_ECUDA;
          x->ident_K = K;
        }
        if (st == TRD_OK &&
            launch_ldl_solve(Lcm, Lcm + (size_t)K * K, (const double*)x->Ident.p, (double*)x->Minv.p, K, K,
                             (double*)x->inv_dot.p, (unsigned int*)x->inv_ctr.p, (double*)x->inv_num.p,
                             x->side) != cudaSuccess)
          st = TRD_ECUDA;
        if (st == TRD_OK) x->minv_k = k;
      }
    }
  }
  const bool ok = st == TRD_OK && cudaEventRecord(x->ev_join, x->side) == cudaSuccess;
  // the next core's chain prefix does not involve E_k: form it behind the join, so that it
  // overlaps the rest of this update
  if (ok) {
    if (build_q(h, (k + 1) % h->N) != TRD_OK || cudaEventRecord(x->ev_tail, x->side) != cudaSuccess) {
      cudaGetLastError();
      x->q_k = -1;
      cudaEventRecord(x->ev_tail, x->side);
    }
    x->side_tail = true;
  }
  h->stream = main_stream;
  pdl_on = true;
  if (!ok) {
    // join whatever was forked, then let run_update compute everything on the main stream
    cudaGetLastError();
    cudaEventRecord(x->ev_join, x->side);
    cudaStreamWaitEvent(h->stream, x->ev_join, 0);
    h->gram_k = -1;
    return false;
  }
  x->pre_k = k;
  x->pre_lambda = lambda;
  return true;
}

// terms (host, nullable): instead of updating the core, return <d, h> and this handle's
// line-search denominator sum w (h B^T)^2 over its own view (the exchange step of a
// partitioned update) in terms[0], terms[1].
trd_status run_update(trd_handle* h, int k, double lambda, double eta_fixed, int gram,
                      double* eta_slot, double* terms = nullptr) {
  if (h->grad_k != k) return set_err(h, TRD_EINVAL, "trd_core_gradient must run for this core first");
  if (gram == TRD_GRAM_LOCAL && X_(h)->row_view)
    return set_err(h, TRD_ENOTIMPL, "the local Gram is defined for the RStS sketch, not for sampled rows");
  const int K = h->K[k];
  const int64_t n = h->I[k] * (int64_t)K;
  double* d = (double*)h->d.p;
  double* hh = (double*)h->h.p;
  bool dot_done = false;
  if (gram == TRD_GRAM_NONE) {
    CK(cudaMemcpyAsync(hh, d, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream), "copy d");
  } else if (X_(h)->pre_k == k && X_(h)->pre_lambda == lambda && gram == TRD_GRAM_GLOBAL && ldl_fits(K)) {
    // G and its factor were prepared on the side stream during this core's data pass
    Extra* xs = X_(h);
    xs->pre_k = -1;
    CK(cudaStreamWaitEvent(h->stream, xs->ev_join, 0), "join side stream");
    double* Lcm = (double*)h->L.p;
    double* Dinv = Lcm + (size_t)K * K;
    PScope ps(h, P_SOLVE);
    TRY(ensure(h, xs->dotpart, sizeof(double) * (size_t)h->I[k]));
    if (xs->minv_k == k && inverse_path(h))
      CK(launch_inv_rows((const double*)xs->Minv.p, d, hh, K, h->I[k], (double*)xs->dotpart.p,
                         (unsigned int*)xs->solve_ctr.p, h->scal + S_NUM, h->stream),
         "h from the inverse");
    else
      CK(launch_ldl_solve(Lcm, Dinv, d, hh, K, h->I[k], (double*)xs->dotpart.p, (unsigned int*)xs->solve_ctr.p,
                          h->scal + S_NUM, h->stream),
         "triangular solves");
    xs->minv_k = -1;
    dot_done = true;
  } else {
    const double* G;
    {
      PScope ps(h, P_GRAM);
      if (gram == TRD_GRAM_LOCAL) {
        TRY(local_gram(h, k));
        G = (const double*)X_(h)->Gloc.p;
      } else {
        TRY(ensure_gram(h, k));
        G = (const double*)h->G.p;
      }
    }
    if (ldl_fits(K)) {
      // LDL^T (FP64), then h = d (L D L^T)^{-1} by row-parallel substitutions
      double* Lcm = (double*)h->L.p;
      double* Dinv = Lcm + (size_t)K * K;
      {
        PScope ps(h, P_CHOL);
        CK(launch_ldl_factor(G, K, lambda, Lcm, Dinv, h->scal, h->dstatus, h->stream), "LDL^T factorisation");
      }
      PScope ps(h, P_SOLVE);
      Extra* xs = X_(h);
      TRY(ensure(h, xs->dotpart, sizeof(double) * (size_t)h->I[k]));
      if (!xs->solve_ctr.p) {
        TRY(ensure(h, xs->solve_ctr, 256));
        CK(cudaMemsetAsync(xs->solve_ctr.p, 0, 256, h->stream), "counter");
      }
      CK(launch_ldl_solve(Lcm, Dinv, d, hh, K, h->I[k], (double*)xs->dotpart.p, (unsigned int*)xs->solve_ctr.p,
                          h->scal + S_NUM, h->stream),
         "triangular solves");
      dot_done = true;
    } else {
      {
        PScope ps(h, P_CHOL);
        CK(launch_cholesky(G, K, lambda, (double*)h->L.p, h->scal, h->dstatus, h->stream), "cholesky");
      }
      PScope ps(h, P_SOLVE);
      CK(launch_solve_rows((const double*)h->L.p, d, hh, K, h->I[k], h->stream), "triangular solves");
    }
  }
  if (!dot_done) {
    PScope ps(h, P_SOLVE);
    CK(launch_dot(d, hh, n, h->scal + S_NUM, h->stream), "<d,h>");
  }
  double* den = h->scal + S_DEN;
  if (eta_fixed <= 0 && X_(h)->tc_pass) {
    TRY(run_pass2_tc(h, k, &den));
  } else if (eta_fixed <= 0) {
    {
      PScope ps(h, P_MERGE);
      TRY(build_halves(h, k));    // normally cached: restores the roles of core k
      TRY(build_merged(h, k, true));
    }
    int ctas = 0, used = 0;
    PassArgs a = pass_args(h);
    prof_begin(h);
    CK(launch_pass_simt(a, is_fp64(h), h->split.rows, true, h->splits, &ctas, &used, h->stream),
       "data pass 2");
    prof_end(h, 1);
    double* s2 = (double*)X_(h)->stat_sum2.p;
    CK(launch_reduce_stats((const double*)h->stat_part.p, ctas, s2, h->dstatus, h->stream), "reduce den");
    den = s2 + 6;
  }
  if (terms) {
    double* s2 = (double*)X_(h)->stat_sum2.p;
    if (!den) {
      // tensor-core line search: the per-CTA partials are summed here instead of in the update
      CK(launch_reduce_stats((const double*)h->stat_part.p, X_(h)->tcG, s2, h->dstatus, h->stream), "reduce den");
      den = s2 + 6;
    }
    CK(cudaMemcpyAsync(h->host_pinned, h->scal + S_NUM, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "num");
    CK(cudaMemcpyAsync(h->host_pinned + 1, den, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "den");
    TRY(sync_and_status(h));
    terms[0] = h->host_pinned[0];
    terms[1] = h->host_pinned[1];
    X_(h)->adv_k = -1;
    return TRD_OK;
  }
  PScope psu(h, P_UPDATE);
  const bool from_parts = eta_fixed <= 0 && den == nullptr;   // tensor-core line search
  // BF16 path with the step operand in FP32 at hand: the stationary half (it holds core k)
  // advances in place with the core, and its tags follow the new core version
  Extra* xa = X_(h);
  const Split& spa = h->split;
  const bool advance = from_parts && xa->adv_k == k && h->prec == TRD_BF16 && !xa->row_view &&
                       xa->tagSst.valid && xa->tagBst.valid && xa->tagSst == xa->tagBst &&
                       xa->tagSst.half == (k < spa.c ? 0 : 1);
  HalfAdvance adv;
  if (advance) {
    adv.S = (float*)h->Sst.p;
    adv.Sh = (const float*)h->Sh.p;
    adv.n = spa.P_stat * (int64_t)spa.Kp;
    adv.Kp = spa.Kp;
    adv.kpad = tc_kpad(spa.Kp, false);
    adv.hi = (__nv_bfloat16*)xa->bShi.p;
    adv.lo = (__nv_bfloat16*)xa->bSlo.p;
  }
  xa->adv_k = -1;
  CK(launch_step_update(h->Z[k], h->Zf[k], hh, n, h->scal + S_NUM, from_parts ? (const double*)h->stat_part.p : nullptr,
                        from_parts ? X_(h)->tcG : 0, den, eta_fixed, h->dstatus, h->scal + S_ETA, eta_slot,
                        h->stream, adv),
     "step size and core update");
  h->ver[k]++;
  if (advance) xa->tagSst.ver[k] = xa->tagBst.ver[k] = h->ver[k];
  X_(h)->e_stale[k] = true;   // E_k only feeds the other cores' Grams: refreshed there
  h->grad_k = -1;
  h->pass1_k = -1;
  return TRD_OK;
}

trd_status set_sigma(trd_handle* h, double sigma) {
  if (sigma > 0) {
    CK(launch_set_scalar(h->scal + S_SIGMA, sigma, h->stream), "set sigma");
    h->sigma_set = true;
    return TRD_OK;
  }
  if (!h->sigma_set) return set_err(h, TRD_EINVAL, "adaptive width requested before trd_adaptive_sigma");
  return TRD_OK;
}

trd_status run_adaptive(trd_handle* h, double sigma_prev, const double* sigma_prev_dev = nullptr) {
  if (!h->X) return set_err(h, TRD_EINVAL, "no data attached");
  PScope ps(h, P_SIGMA);
  Extra* x = X_(h);
  const int64_t n = h->numel <= kProbeMax ? h->numel : kProbeMax;
  TRY(ensure(h, h->probe_keys, sizeof(uint64_t) * n));
  TRY(ensure(h, h->probe_work, sizeof(double) * sigma_work_doubles()));
  // merged subchains of the full tensor for the current cores (same split rule as the passes)
  const View fv = full_view(h);
  const Split sp = choose_split(h, fv, 0);
  if (sp.Kp > 256) return set_err(h, TRD_ENOTIMPL, "the adaptive width supports r_1 r_c <= 256");
  if (!x->probe_ready || x->probe_Pin != sp.P_in) {
    // the probe entries, their block indices and data depend only on X, the mask and the cut
    TRY(ensure(h, x->probe_a, sizeof(int32_t) * n));
    TRY(ensure(h, x->probe_b, sizeof(int32_t) * n));
    TRY(ensure(h, x->probe_x, sizeof(float) * n));
    const int64_t* lin_dev = nullptr;
    if (h->numel > kProbeMax) {
      // sorted probe positions: they depend only on the tensor size, so they are drawn and
      // uploaded once and kept for later data sets of that size
      if (x->probe_lin_n != h->numel) {
        std::vector<int64_t> lin;
        probe_positions(h->numel, lin);
        TRY(ensure(h, x->probe_lin, sizeof(int64_t) * lin.size()));
        CK(cudaMemcpyAsync(x->probe_lin.p, lin.data(), sizeof(int64_t) * lin.size(), cudaMemcpyHostToDevice,
                           h->stream), "probe upload");
        CK(cudaStreamSynchronize(h->stream), "probe upload");
        x->probe_lin_n = h->numel;
      }
      lin_dev = (const int64_t*)x->probe_lin.p;
    }
    CK(launch_probe_setup(h->X, h->M, lin_dev, n, sp.P_in, (int32_t*)x->probe_a.p, (int32_t*)x->probe_b.p,
                          (float*)x->probe_x.p, h->stream), "probe set-up");
    x->probe_ready = true;
    x->probe_Pin = sp.P_in;
  }
  const void* A;
  const void* Cm;
  if (!h->sketched) {
    // the full view is current: use (and leave behind) the cached halves, in the roles of
    // the update of core 0; the split of a core update in progress is kept
    const Split saved = h->split;
    h->split = sp;
    const trd_status st = build_halves(h, 0);
    h->split = saved;
    if (st != TRD_OK) return st;
    A = h->Sst.p;
    Cm = h->Sstr.p;
  } else {
    const size_t e = elt(h);
    TRY(ensure(h, x->recA, e * sp.P_in * sp.Kp));
    TRY(ensure(h, x->recC, e * sp.P_out * sp.Kp));
    CK(launch_chain(make_chain(h, fv, 0, sp.c), x->recA.p, is_fp64(h), false, sp.Kp, h->stream), "probe merge inner");
    CK(launch_chain(make_chain(h, fv, sp.c, h->N), x->recC.p, is_fp64(h), true, sp.Kp, h->stream),
       "probe merge outer");
    A = x->recA.p;
    Cm = x->recC.p;
  }
  TRY(ensure(h, x->probe_cand, sizeof(uint64_t) * n));
  CK(launch_probe_sigma_merged(A, Cm, is_fp64(h), sp.Kp, (const int32_t*)x->probe_a.p,
                               (const int32_t*)x->probe_b.p, (const float*)x->probe_x.p, n, sigma_prev,
                               sigma_prev_dev, (uint64_t*)h->probe_keys.p, (uint64_t*)x->probe_cand.p,
                               (double*)h->probe_work.p, h->scal + S_SIGMA, h->stream),
     "adaptive width");
  h->sigma_set = true;
  return TRD_OK;
}

trd_status use_full_view(trd_handle* h) {
  h->view = full_view(h);
  h->view_k = -1;
  h->sketched = false;
  X_(h)->view_gen = 0;
  X_(h)->row_view = false;
  return TRD_OK;
}

trd_status sample(trd_handle* h, int k, const int32_t* const* idx, const int32_t* s) {
  if (!h->X) return set_err(h, TRD_EINVAL, "no data attached");
  if (!idx) return use_full_view(h);
  const int N = h->N;
  View v = full_view(h);
  size_t off = 0;
  const size_t need = [&] { size_t t = 0; for (int m = 0; m < N; ++m) t += (size_t)h->I[m]; return t; }();
  Extra* xr = X_(h);
  if (xr->idx_ring_cap < need) {
    // (re)allocate the staging ring: wait for every upload still reading the old one
    CK(cudaStreamSynchronize(h->stream), "sync");
    if (xr->idx_ring) cudaFreeHost(xr->idx_ring);
    xr->idx_ring = nullptr;
    xr->idx_ring_cap = 0;
    if (cudaMallocHost(&xr->idx_ring, need * Extra::kIdxSlots * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      return set_err(h, TRD_ENOMEM, "pinned allocation failed");
    }
    xr->idx_ring_cap = need;
    for (int q = 0; q < Extra::kIdxSlots; ++q) xr->idx_ev_live[q] = false;
  }
  const int slot = xr->idx_slot;
  xr->idx_slot = (slot + 1) % Extra::kIdxSlots;
  if (!xr->idx_ev[slot] && cudaEventCreateWithFlags(&xr->idx_ev[slot], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return set_err(h, TRD_ECUDA, "event creation failed");
  }
  // this slot's previous upload has been read by the copy engine
  if (xr->idx_ev_live[slot]) CK(cudaEventSynchronize(xr->idx_ev[slot]), "index staging slot");
  int32_t* stage = xr->idx_ring + (size_t)slot * xr->idx_ring_cap;
  bool any = false;
  for (int m = 0; m < N; ++m) {
    if (m == k || !idx[m]) continue;
    const int32_t sm = s[m];
    if (sm < 1 || sm > h->I[m]) return set_err(h, TRD_EINVAL, "sketch size out of range");
    for (int q = 0; q < sm; ++q) {
      const int32_t i = idx[m][q];
      if (i < 0 || i >= h->I[m] || (q > 0 && i <= idx[m][q - 1]))
        return set_err(h, TRD_EINVAL, "sketch indices must be strictly increasing and in range");
    }
    if (sm == h->I[m]) continue;   // whole mode: identity map
    if (h->idx_cap[m] < (size_t)h->I[m]) {
      if (h->idx_dev[m]) cudaFree(h->idx_dev[m]);
      h->idx_dev[m] = nullptr;
      if (cudaMalloc(&h->idx_dev[m], sizeof(int32_t) * h->I[m]) != cudaSuccess) {
        cudaGetLastError();
        return set_err(h, TRD_ENOMEM, "index allocation failed");
      }
      h->idx_cap[m] = (size_t)h->I[m];
    }
    memcpy(stage + off, idx[m], sizeof(int32_t) * sm);
    CK(cudaMemcpyAsync(h->idx_dev[m], stage + off, sizeof(int32_t) * sm, cudaMemcpyHostToDevice,
                       h->stream), "index upload");
    off += sm;
    v.dim[m] = sm;
    v.idx[m] = h->idx_dev[m];
    any = true;
  }
  if (off > 0) {
    CK(cudaEventRecord(xr->idx_ev[slot], h->stream), "index staging event");
    xr->idx_ev_live[slot] = true;
  }
  if (!any) return use_full_view(h);
  v.numel = 1;
  for (int m = 0; m < N; ++m) v.numel *= v.dim[m];
  const int64_t words = ((v.numel + 31) / 32 + 3) / 4 * 4;
  TRY(ensure(h, h->XI, sizeof(float) * (size_t)v.numel));
  TRY(ensure(h, h->PI, sizeof(uint32_t) * (size_t)words));
  {
    PScope ps(h, P_GATHER);
    TRY(ensure(h, X_(h)->gbase, sizeof(int64_t) * (size_t)(v.numel / v.dim[0])));
    CK(launch_gather(h->X, h->M, N, h->I, v, (float*)h->XI.p, (uint32_t*)h->PI.p, (int64_t*)X_(h)->gbase.p,
                     h->stream), "RStS gather");
  }
  v.X = (const float*)h->XI.p;
  v.M = (const uint32_t*)h->PI.p;
  h->view = v;
  h->view_k = k;
  h->sketched = true;
  X_(h)->view_gen = ++X_(h)->sketch_count;
  X_(h)->row_view = false;
  h->pass1_k = -1;
  h->grad_k = -1;
  return TRD_OK;
}

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

void draw(uint64_t seed, int32_t t, int k, int j, int N, int64_t I, int32_t s, int32_t* out) {
  if (s >= I) {
    for (int64_t i = 0; i < I; ++i) out[i] = (int32_t)i;
    return;
  }
  const uint64_t key = mix64(seed + ((uint64_t)(((int64_t)t * N + k) * N + j) + 1) * kGamma);
  std::vector<int32_t> perm((size_t)I);
  for (int64_t i = 0; i < I; ++i) perm[(size_t)i] = (int32_t)i;
  for (int32_t m = 0; m < s; ++m) {
    const uint64_t z = mix64(key + (uint64_t)(m + 1) * kGamma);
    const int64_t pick = m + (int64_t)(z % (uint64_t)(I - m));
    std::swap(perm[(size_t)m], perm[(size_t)pick]);
  }
  std::sort(perm.begin(), perm.begin() + s);
  for (int32_t m = 0; m < s; ++m) out[m] = perm[(size_t)m];
}

trd_status alloc_state(trd_handle* h) {
  const int N = h->N;
  int maxK = 1;
  int64_t maxIK = 1;
  for (int k = 0; k < N; ++k) {
    const int rk = h->R[k], rk1 = h->R[(k + 1) % N];
    h->K[k] = rk * rk1;
    maxK = std::max(maxK, h->K[k]);
    maxIK = std::max(maxIK, h->I[k] * (int64_t)h->K[k]);
    if (cudaMalloc(&h->Z[k], sizeof(double) * h->I[k] * h->K[k]) != cudaSuccess ||
        cudaMalloc(&h->Zf[k], sizeof(float) * h->I[k] * h->K[k]) != cudaSuccess ||
        cudaMalloc(&h->E[k], sizeof(double) * (size_t)rk * rk * rk1 * rk1) != cudaSuccess) {
      cudaGetLastError();
      return set_err(h, TRD_ENOMEM, "core allocation failed");
    }
    cudaMemsetAsync(h->Z[k], 0, sizeof(double) * h->I[k] * h->K[k], h->stream);
    cudaMemsetAsync(h->Zf[k], 0, sizeof(float) * h->I[k] * h->K[k], h->stream);
  }
  // chain buffers hold p^2 x q^2 intermediates: bound by maxR^4
  size_t chain = 1;
  for (int k = 0; k < N; ++k)
    for (int m = 0; m < N; ++m)
      chain = std::max(chain, (size_t)h->R[k] * h->R[k] * h->R[m] * h->R[m]);
  const int64_t IN = h->I[N - 1];
  TRY(ensure(h, h->G, sizeof(double) * maxK * maxK));
  TRY(ensure(h, h->L, sizeof(double) * (2 * maxK * maxK + maxK)));   // factor, D^{-1}, row-major copy
  TRY(ensure(h, h->T1, sizeof(double) * chain));
  TRY(ensure(h, h->T2, sizeof(double) * chain));
  TRY(ensure(h, h->d, sizeof(double) * maxIK));
  TRY(ensure(h, h->h, sizeof(double) * std::max<int64_t>(maxIK, IN * h->K[N - 1])));
  TRY(ensure(h, h->D, sizeof(double) * IN * IN));
  TRY(ensure(h, h->Dprev, sizeof(double) * IN * IN));
  TRY(ensure(h, h->stat_sum, sizeof(double) * 8));
  TRY(ensure(h, X_(h)->stat_sum2, sizeof(double) * 8));
  if (cudaMalloc(&h->scal, sizeof(double) * 64) != cudaSuccess ||
      cudaMalloc(&h->dstatus, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->report_dev, sizeof(double) * 64) != cudaSuccess ||
      cudaMallocHost(&h->host_pinned, sizeof(double) * 256) != cudaSuccess) {
    cudaGetLastError();
    return set_err(h, TRD_ENOMEM, "state allocation failed");
  }
  cudaMemsetAsync(h->scal, 0, sizeof(double) * 64, h->stream);
  cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->stream);
  cudaMemsetAsync(h->report_dev, 0, sizeof(double) * 64, h->stream);
  // meta: core pointers, dims, ranks for kernels that walk all cores
  Extra* x = X_(h);
  TRY(ensure(h, x->meta, 32 * kMaxN));
  char hostmeta[32 * kMaxN];
  memset(hostmeta, 0, sizeof(hostmeta));
  for (int m = 0; m < N; ++m) {
    memcpy(hostmeta + 8 * m, &h->Z[m], 8);
    memcpy(hostmeta + 8 * kMaxN + 8 * m, &h->I[m], 8);
    memcpy(hostmeta + 16 * kMaxN + 4 * m, &h->R[m], 4);
  }
  CK(cudaMemcpy(x->meta.p, hostmeta, sizeof(hostmeta), cudaMemcpyHostToDevice), "meta upload");
  return TRD_OK;
}

void free_buf(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

}  // namespace

// Extra state lives right after the handle in one host allocation.
struct trd_handle_full {
  trd_handle h;
  Extra x;
};
namespace {
Extra* X_(trd_handle* h) { return &reinterpret_cast<trd_handle_full*>(h)->x; }
}  // namespace

// =================================================================== ABI

extern "C" {

const char* trd_status_string(trd_status s) {
  switch (s) {
    case TRD_OK: return "TRD_OK";
    case TRD_EINVAL: return "TRD_EINVAL";
    case TRD_ENOMEM: return "TRD_ENOMEM";
    case TRD_ECUDA: return "TRD_ECUDA";
    case TRD_ESINGULAR: return "TRD_ESINGULAR";
    case TRD_ENONFINITE: return "TRD_ENONFINITE";
    case TRD_ETIMEOUT: return "TRD_ETIMEOUT";
    case TRD_ENOTIMPL: return "TRD_ENOTIMPL";
  }
  return "TRD_UNKNOWN";
}

const char* trd_last_error(const trd_t* h) { return h ? h->err.c_str() : "null handle"; }

// The shape rules of trd_create (order, mode sizes, ranks, r_k r_{k+1}, entry count, precision).
static bool valid_shape(int N, const int64_t* I, const int32_t* R, int precision) {
  if (N < 3 || N > kMaxN || !I || !R) return false;
  if (precision != TRD_FP64 && precision != TRD_FP32 && precision != TRD_BF16 && precision != TRD_TF32X3)
    return false;
  double logtot = 0;
  for (int m = 0; m < N; ++m) {
    if (I[m] < 1 || I[m] > (int64_t(1) << 31) - 1) return false;
    if (R[m] < 1 || R[m] > kMaxR) return false;
    logtot += log2((double)I[m]);
  }
  for (int m = 0; m < N; ++m)
    if (R[m] * R[(m + 1) % N] > TRD_MAX_CORE_K) return false;
  return logtot < 40.0;
}

trd_status trd_ring_cut(int N, const int64_t* I, const int32_t* R, int precision, int32_t* c_out,
                        int32_t* width_out) {
  if (!c_out || !width_out || !valid_shape(N, I, R, precision)) return TRD_EINVAL;
  int Ri[kMaxN];
  for (int m = 0; m < N; ++m) Ri[m] = R[m];
  bool fits = false;
  const int c = ring_cut(N, I, Ri, precision, &fits);
  *c_out = c;
  *width_out = Ri[0] * Ri[c];
  return fits ? TRD_OK : TRD_ENOTIMPL;
}

trd_status trd_create(trd_t** out, int N, const int64_t* I, const int32_t* R, int precision,
                      void* cuda_stream) {
  if (!out) return TRD_EINVAL;
  *out = nullptr;
  if (!valid_shape(N, I, R, precision)) return TRD_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return TRD_ECUDA;
  }
  trd_handle_full* hf = new (std::nothrow) trd_handle_full();
  if (!hf) return TRD_ENOMEM;
  trd_handle* h = &hf->h;
  h->N = N;
  for (int m = 0; m < N; ++m) { h->I[m] = I[m]; h->R[m] = R[m]; }
  h->prec = precision;
  h->stream = (cudaStream_t)cuda_stream;
  if (!h->stream) {
    // a blocking stream of the handle's own: ordered with the legacy stream like the caller
    // expects, and capturable into a graph
    if (cudaStreamCreate(&h->stream) != cudaSuccess) {
      cudaGetLastError();
      delete hf;
      return TRD_ECUDA;
    }
    X_(h)->own_stream = true;
  }
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (h->num_sms < 1) h->num_sms = 1;
  trd_status s = alloc_state(h);
  if (s != TRD_OK) {
    trd_destroy(h);
    return s;
  }
  *out = h;
  return TRD_OK;
}

void trd_destroy(trd_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  {
    Extra* x = X_(h);
    if (x->side) {
      cudaStreamSynchronize(x->side);
      cudaStreamDestroy(x->side);
    }
    if (x->ev_fork) cudaEventDestroy(x->ev_fork);
    if (x->ev_join) cudaEventDestroy(x->ev_join);
    if (x->ev_tail) cudaEventDestroy(x->ev_tail);
  }
  drop_graph(X_(h));
  for (int k = 0; k < kMaxN; ++k) {
    if (h->Z[k]) cudaFree(h->Z[k]);
    if (h->Zf[k]) cudaFree(h->Zf[k]);
    if (h->E[k]) cudaFree(h->E[k]);
    if (h->idx_dev[k]) cudaFree(h->idx_dev[k]);
  }
  DevBuf* bufs[] = {&h->XI, &h->PI, &h->Sst, &h->Sstr, &h->Sh, &h->Sst_bf, &h->Sstr_bf, &h->Sh_bf,
                    &h->SstrT_bf, &h->SstT_bf, &h->Tpart, &h->Tsum, &h->stat_part, &h->stat_sum,
                    &h->pre, &h->post, &h->dpart, &h->d, &h->h, &h->G, &h->L, &h->T1, &h->T2,
                    &h->D, &h->Dprev, &h->probe_keys, &h->probe_work};
  for (DevBuf* b : bufs) free_buf(*b);
  Extra* x = X_(h);
  DevBuf* xb[] = {&x->Ework, &x->meta,    &x->stat_sum2, &x->Gloc,    &x->recA, &x->recC,
                  &x->errp,  &x->probe_a, &x->probe_b,   &x->probe_x, &x->dotpart, &x->solve_ctr, &x->bc_ctr, &x->stop_part, &x->stop_ctr, &x->probe_lin, &x->Qb[0], &x->Qb[1], &x->probe_cand, &x->rows_dev,
                  &x->bShi,  &x->bSlo,    &x->bSh,       &x->bThi,    &x->bTlo,    &x->bTT,
                  &x->Mst[0], &x->Mst[1], &x->bShlo, &x->Xpad, &x->bTThi, &x->bTTlo, &x->gbase, &x->wq,
                  &x->Minv, &x->Ident, &x->inv_dot, &x->inv_ctr, &x->inv_num};
  for (DevBuf* b : xb) free_buf(*b);
  for (int k = 0; k < kMaxN; ++k) { free_buf(x->Eloc[k]); free_buf(x->tmpZ[k]); free_buf(x->smpZ[k]); }
  DevBuf* sb[] = {&x->smpA, &x->smpC, &x->smpGA, &x->smpGC, &x->smpGAd, &x->smpGCd, &x->smpPre, &x->smpPost,
                  &x->smpDpart, &x->smpD, &x->smpLoss, &x->smpKa, &x->smpKb, &x->smpPa, &x->smpPb,
                  &x->smpCa, &x->smpCb, &x->smpUa, &x->smpUb, &x->smpG};
  for (DevBuf* b : sb) free_buf(*b);
  for (auto& p : x->pending) { x->ev_pool.push_back(p.a); x->ev_pool.push_back(p.b); }
  if (x->ev_open) x->ev_pool.push_back(x->ev_open);
  for (cudaEvent_t e : x->ev_pool) cudaEventDestroy(e);
  for (int q = 0; q < Extra::kIdxSlots; ++q)
    if (x->idx_ev[q]) cudaEventDestroy(x->idx_ev[q]);
  if (x->idx_ring) cudaFreeHost(x->idx_ring);
  if (h->scal) cudaFree(h->scal);
  if (h->dstatus) cudaFree(h->dstatus);
  if (h->report_dev) cudaFree(h->report_dev);
  if (h->host_pinned) cudaFreeHost(h->host_pinned);
  if (h->idx_pinned) cudaFreeHost(h->idx_pinned);
  if (x->own_stream && h->stream) cudaStreamDestroy(h->stream);
  cudaGetLastError();
  delete reinterpret_cast<trd_handle_full*>(h);
}

trd_status trd_set_data(trd_t* h, const float* X, const uint32_t* mask) {
  TRY(check_handle(h));
  touch(h);
  if (!X) return set_err(h, TRD_EINVAL, "X must not be NULL");
  if (((uintptr_t)X & 15) || ((uintptr_t)mask & 15))
    return set_err(h, TRD_EINVAL, "X and mask must be 16-byte aligned");
  h->X = X;
  h->M = mask;
  // the contents may have changed behind the same pointers: drop everything derived from them;
  // the merged halves are merged again from the cores as well (a fresh start for the BF16
  // path's in-place advances)
  X_(h)->probe_ready = false;
  X_(h)->mst_X[0] = X_(h)->mst_X[1] = nullptr;
  X_(h)->xpad_src = nullptr;
  X_(h)->tagSst.valid = X_(h)->tagSstr.valid = X_(h)->tagBst.valid = X_(h)->tagBstr.valid = false;
  h->numel = 1;
  for (int m = 0; m < h->N; ++m) h->numel *= h->I[m];
  use_full_view(h);
  h->pass1_k = h->grad_k = -1;
  return TRD_OK;
}

trd_status trd_init_cores(trd_t* h, uint64_t seed, double stddev) {
  TRY(check_handle(h));
  touch(h);
  const int N = h->N;
  uint64_t base = 0;
  for (int k = 0; k < N; ++k) {
    const int rk = h->R[k], rk1 = h->R[(k + 1) % N];
    const double sd = stddev > 0 ? stddev : pow((double)rk * rk1, -0.25);
    const int64_t n = h->I[k] * (int64_t)rk * rk1;
    std::vector<double> v((size_t)n);
    for (int64_t f = 0; f < n; ++f) {
      const uint64_t g = base + (uint64_t)f;
      const uint64_t z1 = mix64(seed + (2 * g + 1) * kGamma);
      const uint64_t z2 = mix64(seed + (2 * g + 2) * kGamma);
      const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;
      const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
      v[(size_t)f] = sd * (sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2));
    }
    CK(cudaMemcpyAsync(h->Z[k], v.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream), "core upload");
    CK(launch_from_double(h->Z[k], n, h->Zf[k], false, h->stream), "FP32 core copy");
    CK(cudaStreamSynchronize(h->stream), "sync");
    h->ver[k]++;
    TRY(refresh_E(h, k));
    X_(h)->e_stale[k] = false;
    base += (uint64_t)n;
  }
  h->t = 0;
  h->pass1_k = h->grad_k = -1;
  TRY(reset_D0(h));
  return sync_and_status(h);
}

trd_status trd_set_core(trd_t* h, int k, const double* core) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  if (!core) return set_err(h, TRD_EINVAL, "NULL core");
  CK(cudaMemcpyAsync(h->Z[k], core, sizeof(double) * h->I[k] * h->K[k], cudaMemcpyHostToDevice, h->stream),
     "core upload");
  CK(launch_from_double(h->Z[k], h->I[k] * (int64_t)h->K[k], h->Zf[k], false, h->stream), "FP32 core copy");
  CK(cudaStreamSynchronize(h->stream), "sync");
  h->ver[k]++;
  h->pass1_k = h->grad_k = -1;
  TRY(refresh_E(h, k));
  X_(h)->e_stale[k] = false;
  return sync_and_status(h);
}

trd_status trd_get_core(trd_t* h, int k, double* core) {
  TRY(check_handle(h));
  TRY(check_k(h, k));
  if (!core) return set_err(h, TRD_EINVAL, "NULL core");
  CK(cudaMemcpyAsync(core, h->Z[k], sizeof(double) * h->I[k] * h->K[k], cudaMemcpyDeviceToHost, h->stream),
     "core download");
  return sync_and_status(h);
}

trd_status trd_reset_iteration(trd_t* h, int32_t t) {
  TRY(check_handle(h));
  touch(h);
  h->t = t;
  TRY(reset_D0(h));
  return sync_and_status(h);
}

trd_status trd_draw_indices(uint64_t seed, int32_t t, int k, int j, int N, int64_t I, int32_t s,
                            int32_t* out) {
  if (!out || N < 1 || I < 1 || s < 1 || s > I || k < 0 || j < 0) return TRD_EINVAL;
  draw(seed, t, k, j, N, I, s, out);
  return TRD_OK;
}

trd_status trd_sample_subtensor(trd_t* h, int k, const int32_t* const* idx, const int32_t* s) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  if (idx && !s) return set_err(h, TRD_EINVAL, "sizes missing");
  return sample(h, k, idx, s);
}

trd_status trd_sample_rows(trd_t* h, int k, const int32_t* rows, int64_t J) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  if (!h->X) return set_err(h, TRD_EINVAL, "no data attached");
  if (!rows || J < 1 || J > ((int64_t)1 << 31) / (h->N > 0 ? h->N : 1))
    return set_err(h, TRD_EINVAL, "rows must be a host array of J >= 1 multi-indices");
  const int N = h->N;
  for (int64_t j = 0; j < J; ++j)
    for (int m = 0; m < N; ++m)
      if (m != k && (rows[j * N + m] < 0 || rows[j * N + m] >= h->I[m]))
        return set_err(h, TRD_EINVAL, "a sampled index is out of range");
  Extra* x = X_(h);
  const int64_t n = h->I[k] * J;
  const int64_t words = ((n + 31) / 32 + 3) / 4 * 4;
  TRY(ensure(h, x->rows_dev, sizeof(int32_t) * (size_t)(J * N)));
  TRY(ensure(h, h->XI, sizeof(float) * (size_t)n));
  TRY(ensure(h, h->PI, sizeof(uint32_t) * (size_t)words));
  CK(cudaMemcpyAsync(x->rows_dev.p, rows, sizeof(int32_t) * (size_t)(J * N), cudaMemcpyHostToDevice, h->stream),
     "rows upload");
  CK(cudaMemsetAsync(h->PI.p, 0, sizeof(uint32_t) * (size_t)words, h->stream), "mask clear");
  CK(launch_gather_rows(h->X, h->M, rows_args(h, k, J), (const int32_t*)x->rows_dev.p, (float*)h->XI.p,
                        (uint32_t*)h->PI.p, h->stream),
     "row gather");
  View v;
  v.X = (const float*)h->XI.p;
  v.M = (const uint32_t*)h->PI.p;
  v.N = N;
  v.numel = n;
  for (int m = 0; m < N; ++m) v.dim[m] = h->I[m];
  h->view = v;
  h->view_k = k;
  h->sketched = true;
  x->view_gen = ++x->sketch_count;
  x->row_view = true;
  x->row_k = k;
  x->rows_J = J;
  h->pass1_k = -1;
  h->grad_k = -1;
  return sync_and_status(h);   // the host rows may be released on return
}

trd_status trd_residual_weights(trd_t* h, int k, double sigma, trd_resid_stats* out) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  if (!h->X) return set_err(h, TRD_EINVAL, "no data attached");
  if (h->sketched && h->view_k != k) return set_err(h, TRD_EINVAL, "the current sketch was drawn for another core");
  TRY(set_sigma(h, sigma));
  TRY(run_pass1(h, k));
  if (!out) return TRD_OK;
  double* hp = h->host_pinned;
  CK(cudaMemcpyAsync(hp, h->stat_sum.p, sizeof(double) * 8, cudaMemcpyDeviceToHost, h->stream), "stats");
  CK(cudaMemcpyAsync(hp + 8, h->scal + S_SIGMA, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "sigma");
  TRY(sync_and_status(h));
  out->sum_w = hp[0];
  out->sum_e2 = hp[1];
  out->sum_we2 = hp[2];
  out->n_obs = (int64_t)hp[3];
  out->n_nonfinite = (int64_t)hp[4];
  out->n_slots = (int64_t)hp[5];
  out->sigma = hp[8];
  if (out->n_nonfinite > 0) return set_err(h, TRD_ENONFINITE, "non-finite residuals");
  return TRD_OK;
}

trd_status trd_core_gradient(trd_t* h, int k, double* d_host) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  TRY(run_gradient(h, k));
  if (!d_host) return TRD_OK;
  CK(cudaMemcpyAsync(d_host, h->d.p, sizeof(double) * h->I[k] * h->K[k], cudaMemcpyDeviceToHost, h->stream),
     "gradient download");
  return sync_and_status(h);
}

trd_status trd_fgmc_gram(trd_t* h, int k, double* G_host) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  TRY(ensure_gram(h, k));
  if (!G_host) return TRD_OK;
  CK(cudaMemcpyAsync(G_host, h->G.p, sizeof(double) * h->K[k] * h->K[k], cudaMemcpyDeviceToHost, h->stream),
     "gram download");
  return sync_and_status(h);
}

trd_status trd_core_update(trd_t* h, int k, double lambda, double eta, int gram, double* eta_out) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  if (gram < TRD_GRAM_GLOBAL || gram > TRD_GRAM_NONE) return set_err(h, TRD_EINVAL, "bad gram kind");
  TRY(run_update(h, k, lambda, eta, gram, nullptr));
  if (!eta_out) return TRD_OK;
  CK(cudaMemcpyAsync(h->host_pinned, h->scal + S_ETA, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
     "eta");
  TRY(sync_and_status(h));
  *eta_out = h->host_pinned[0];
  return TRD_OK;
}

trd_status trd_set_gradient(trd_t* h, int k, const double* d_host) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  if (!d_host) return set_err(h, TRD_EINVAL, "d must not be NULL");
  if (h->pass1_k != k) return set_err(h, TRD_EINVAL, "trd_residual_weights must run for this core first");
  const size_t bytes = sizeof(double) * h->I[k] * h->K[k];
  TRY(ensure(h, h->d, bytes));
  CK(cudaMemcpyAsync(h->d.p, d_host, bytes, cudaMemcpyHostToDevice, h->stream), "gradient upload");
  TRY(sync_and_status(h));
  h->grad_k = k;
  return TRD_OK;
}

trd_status trd_line_search_terms(trd_t* h, int k, double lambda, int gram, double* num_out, double* den_out) {
  TRY(check_handle(h));
  touch(h);
  TRY(check_k(h, k));
  if (gram < TRD_GRAM_GLOBAL || gram > TRD_GRAM_NONE) return set_err(h, TRD_EINVAL, "bad gram kind");
  if (!num_out || !den_out) return set_err(h, TRD_EINVAL, "num_out and den_out must not be NULL");
  double terms[2] = {0.0, 0.0};
  TRY(run_update(h, k, lambda, -1.0, gram, nullptr, terms));
  *num_out = terms[0];
  *den_out = terms[1];
  return TRD_OK;
}

trd_status trd_adaptive_sigma(trd_t* h, double sigma_prev, double* sigma_out) {
  TRY(check_handle(h));
  touch(h);
  TRY(run_adaptive(h, sigma_prev));
  if (!sigma_out) return TRD_OK;
  CK(cudaMemcpyAsync(h->host_pinned, h->scal + S_SIGMA, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
     "sigma");
  TRY(sync_and_status(h));
  *sigma_out = h->host_pinned[0];
  return TRD_OK;
}

trd_status trd_sigma_from_residuals(trd_t* h, const float* r, int64_t n, double rms, double sigma_prev,
                                    double* sigma_out) {
  TRY(check_handle(h));
  if (!r || n < 1 || !(rms >= 0) || !sigma_out) return set_err(h, TRD_EINVAL, "bad arguments");
  TRY(ensure(h, h->probe_keys, sizeof(uint64_t) * n));
  TRY(ensure(h, h->probe_work, sizeof(double) * sigma_work_doubles()));
  TRY(ensure(h, X_(h)->probe_cand, sizeof(uint64_t) * n));
  CK(launch_sigma_from_floats(r, n, rms, sigma_prev, (uint64_t*)h->probe_keys.p, (uint64_t*)X_(h)->probe_cand.p,
                              (double*)h->probe_work.p, h->scal + S_SIGMA + 8, h->stream),
     "sigma from residuals");
  CK(cudaMemcpyAsync(h->host_pinned, h->scal + S_SIGMA + 8, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
     "sigma");
  TRY(sync_and_status(h));
  *sigma_out = h->host_pinned[0];
  return TRD_OK;
}

}  // extern "C"

namespace {

// The device work of one outer iteration (Algorithm 1, every core once), enqueued on the
// handle's stream without any host synchronisation, so that it can be captured as a graph.
trd_status step_device(trd_handle* h, const trd_params* p, int64_t* slots_out) {
  const int N = h->N;
  // the Gram of core 0 depends only on the cores of the previous iteration: fork it before the
  // adaptive width, whose kernels it then overlaps
  X_(h)->pre_k = -1;
  const bool early = p->gram == TRD_GRAM_GLOBAL && prefactor(h, 0, p->lambda);
  if (p->sigma > 0) {
    TRY(set_sigma(h, p->sigma));
  } else {
    // width of this iteration from the residuals of the current cores, limited by the
    // width of the previous iteration (kept on the device, no host round trip)
    if (h->sigma_set && h->t > 0) {
      CK(cudaMemcpyAsync(h->scal + S_SIGMA_PREV, h->scal + S_SIGMA, sizeof(double),
                         cudaMemcpyDeviceToDevice, h->stream), "sigma prev");
      TRY(run_adaptive(h, -1.0, h->scal + S_SIGMA_PREV));
    } else {
      TRY(run_adaptive(h, -1.0));
    }
  }
  int64_t slots = 0;
  for (int k = 0; k < N; ++k) {
    bool sketch = false;
    for (int m = 0; m < N; ++m)
      if (m != k && p->sketch[m] > 0 && p->sketch[m] < h->I[m]) sketch = true;
    if (sketch) {
      std::vector<std::vector<int32_t>> sets(N);
      const int32_t* ptrs[kMaxN] = {};
      int32_t sizes[kMaxN] = {};
      for (int m = 0; m < N; ++m) {
        if (m == k) continue;
        const int32_t s = (p->sketch[m] > 0 && p->sketch[m] < h->I[m]) ? p->sketch[m] : (int32_t)h->I[m];
        sets[m].resize((size_t)s);
        draw(p->seed, h->t, k, m, N, h->I[m], s, sets[m].data());
        ptrs[m] = sets[m].data();
        sizes[m] = s;
      }
      TRY(sample(h, k, ptrs, sizes));
    } else if (h->sketched) {
      use_full_view(h);
    }
    Extra* x = X_(h);
    x->reserve_sms = 0;
    if (!(k == 0 && early)) {
      x->pre_k = -1;
      if (p->gram == TRD_GRAM_GLOBAL && prefactor(h, k, p->lambda)) x->reserve_sms = kSideSMs;
    }
    x->obj_slot = h->report_dev + R_OBJ + k;   // the statistics reduction writes the objective
    const trd_status s1 = run_pass1(h, k, false);
    x->reserve_sms = 0;
    x->obj_slot = nullptr;
    TRY(s1);
    TRY(run_gradient(h, k));
    TRY(run_update(h, k, p->lambda, -1.0, p->gram, h->report_dev + R_ETA + k));
    slots += h->slots_last;
  }
  if (X_(h)->side_tail) {
    // the step ends with everything it forked joined (also required by stream capture)
    CK(cudaStreamWaitEvent(h->stream, X_(h)->ev_tail, 0), "join side stream");
    X_(h)->side_tail = false;
  }
  {
    PScope ps(h, P_STOP);
    TRY(compute_D(h, (double*)h->D.p));
    Extra* xs = X_(h);
    if (!xs->stop_ctr.p) {
      TRY(ensure(h, xs->stop_ctr, 256));
      CK(cudaMemsetAsync(xs->stop_ctr.p, 0, 256, h->stream), "counter");
    }
    TRY(ensure(h, xs->stop_part, sizeof(double) * 2 * kStopBlocks));
    CK(launch_stop_error((const double*)h->D.p, (double*)h->Dprev.p, h->I[N - 1] * h->I[N - 1],
                         (double*)xs->stop_part.p, (unsigned int*)xs->stop_ctr.p, h->report_dev + R_E, h->stream),
       "stopping quantity");
  }
  CK(cudaMemcpyAsync(h->report_dev + R_SIGMA, h->scal + S_SIGMA, sizeof(double), cudaMemcpyDeviceToDevice,
                     h->stream), "sigma");
  *slots_out = slots;
  return TRD_OK;
}

// Whether a merged-half tag describes the current cores (it was merged or advanced in
// place for their versions).
bool tag_current(const trd_handle* h, const HalfTag& t) {
  if (!t.valid) return false;
  const int m0 = t.half == 0 ? 0 : t.c, m1 = t.half == 0 ? t.c : h->N;
  for (int m = m0; m < m1; ++m)
    if (t.ver[m] != h->ver[m]) return false;
  return true;
}

// Host-side state after a step whose device work ran without the host logic (graph replay):
// every core changed once; Gram and pass results are treated as stale. A merged half that
// was current at the end of the captured step is current again after the replay (the replay
// advanced it in place exactly as the captured step did), so its tag follows the versions.
void after_replay(trd_handle* h) {
  Extra* x = X_(h);
  HalfTag* tags[4] = {&x->tagSst, &x->tagSstr, &x->tagBst, &x->tagBstr};
  bool cur[4];
  for (int i = 0; i < 4; ++i) cur[i] = x->graph_tag_cur[i] && tag_current(h, *tags[i]);
  for (int k = 0; k < h->N; ++k) h->ver[k]++;
  for (int i = 0; i < 4; ++i) {
    if (!cur[i]) continue;
    HalfTag& t = *tags[i];
    const int m0 = t.half == 0 ? 0 : t.c, m1 = t.half == 0 ? t.c : h->N;
    for (int m = m0; m < m1; ++m) t.ver[m] = h->ver[m];
  }
  h->pass1_k = -1;
  h->grad_k = -1;
  h->gram_k = -1;
}

// Capture one step into a graph, instantiate it and launch it (this launch is the step).  On
// any failure the capture is abandoned, every cache is invalidated (the host logic ran but
// nothing was executed) and the step runs eagerly instead.
trd_status capture_step(trd_handle* h, const trd_params* p, int64_t* slots) {
  Extra* x = X_(h);
  drop_graph(x);
  const size_t pend0 = x->pending.size();
  bool ok = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  trd_status st = ok ? step_device(h, p, slots) : TRD_ECUDA;
  {
    const HalfTag* tags[4] = {&x->tagSst, &x->tagSstr, &x->tagBst, &x->tagBstr};
    for (int i = 0; i < 4; ++i) x->graph_tag_cur[i] = tag_current(h, *tags[i]);
  }
  cudaGraph_t g = nullptr;
  if (ok) ok = cudaStreamEndCapture(h->stream, &g) == cudaSuccess && st == TRD_OK && g;
  if (ok) ok = cudaGraphInstantiate(&x->graph_exec, g, 0) == cudaSuccess;
  if (ok) {
    x->graph = g;
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    x->graph_kernels = 0;
    std::vector<std::pair<cudaEvent_t, cudaGraphNode_t>> evn;
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType ty;
      if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess) continue;
      if (ty == cudaGraphNodeTypeKernel) ++x->graph_kernels;
      if (ty == cudaGraphNodeTypeEventRecord) {
        cudaEvent_t ev = nullptr;
        if (cudaGraphEventRecordNodeGetEvent(nd, &ev) == cudaSuccess) evn.push_back({ev, nd});
      }
    }
    auto node_of = [&](cudaEvent_t ev) -> cudaGraphNode_t {
      for (auto& q : evn)
        if (q.first == ev) return q.second;
      return nullptr;
    };
    for (size_t i = pend0; i < x->pending.size() && ok; ++i) {
      const cudaGraphNode_t na = node_of(x->pending[i].a), nb = node_of(x->pending[i].b);
      if (!na || !nb) ok = false;
      else x->graph_ev.push_back({na, nb, x->pending[i].kind});
    }
  }
  if (ok) ok = cudaGraphLaunch(x->graph_exec, h->stream) == cudaSuccess;
  if (ok) {
    x->graph_slots = *slots;
    x->graph_ok = true;
    return TRD_OK;
  }
  // abandon: nothing of this step ran
  cudaGetLastError();
  if (!x->graph && g) cudaGraphDestroy(g);
  drop_graph(x);
  for (size_t i = pend0; i < x->pending.size(); ++i) {
    x->ev_pool.push_back(x->pending[i].a);
    x->ev_pool.push_back(x->pending[i].b);
  }
  x->pending.resize(pend0);
  x->tagSst.valid = x->tagSstr.valid = x->tagBst.valid = x->tagBstr.valid = false;
  h->pass1_k = h->grad_k = h->gram_k = -1;
  for (int k = 0; k < h->N; ++k) h->ver[k]++;
  x->graphs_enabled = false;
  h->err.clear();
  return step_device(h, p, slots);
}

// Replay the captured step; with tracing level 1 every replay records its data-pass
// intervals on fresh events.
trd_status replay_step(trd_handle* h) {
  Extra* x = X_(h);
  for (const auto& q : x->graph_ev) {
    cudaEvent_t a = pool_event(x), b = pool_event(x);
    if (!a || !b ||
        cudaGraphExecEventRecordNodeSetEvent(x->graph_exec, q.a, a) != cudaSuccess ||
        cudaGraphExecEventRecordNodeSetEvent(x->graph_exec, q.b, b) != cudaSuccess) {
      cudaGetLastError();
      return set_err(h, TRD_ECUDA, "graph event update failed");
    }
    x->pending.push_back({a, b, q.kind});
  }
  CK(cudaGraphLaunch(x->graph_exec, h->stream), "graph launch");
  note_launches(x->graph_kernels);
  after_replay(h);
  return TRD_OK;
}

}  // namespace

extern "C" {

trd_status trd_step(trd_t* h, const trd_params* p, trd_report* rep) {
  TRY(check_handle(h));
  if (!p) return set_err(h, TRD_EINVAL, "NULL params");
  if (!h->X) return set_err(h, TRD_EINVAL, "no data attached");
  if (p->gram < TRD_GRAM_GLOBAL || p->gram > TRD_GRAM_NONE) return set_err(h, TRD_EINVAL, "bad gram kind");
  const int N = h->N;
  Extra* x = X_(h);
  if (!h->have_D0) {
    touch(h);
    TRY(reset_D0(h));
  }
  bool any_sketch = false;
  for (int m = 0; m < N; ++m)
    if (p->sketch[m] > 0 && p->sketch[m] < h->I[m]) any_sketch = true;
  Extra::GraphKey key;
  key.sigma = p->sigma > 0 ? p->sigma : -1.0;
  key.lambda = p->lambda;
  key.gram = p->gram;
  key.prof = x->prof;
  // graphs: unsketched steps (a sketch is drawn on the host every step), tracing level <= 1
  const bool graphable = x->graphs_enabled && !any_sketch && !h->sketched && x->prof <= 1 && h->t > 0;
  int64_t slots = 0;
  if (graphable && x->graph_ok && x->gkey == key) {
    TRY(replay_step(h));
    slots = x->graph_slots;
  } else {
    if (x->graph_ok || x->graph) drop_graph(x);
    const bool same = x->gkey == key;
    if (graphable && same && x->steady >= 1) {
      TRY(capture_step(h, p, &slots));
    } else {
      TRY(step_device(h, p, &slots));
    }
    x->steady = graphable ? (same ? x->steady + 1 : 1) : 0;
    x->gkey = key;
  }
  CK(cudaMemcpyAsync(h->host_pinned, h->report_dev, sizeof(double) * 32, cudaMemcpyDeviceToHost, h->stream),
     "report");
  trd_status st = sync_and_status(h);
  prof_harvest(h);
  h->t += 1;
  if (rep) {
    memset(rep, 0, sizeof(*rep));
    for (int k = 0; k < N; ++k) {
      rep->eta[k] = h->host_pinned[R_ETA + k];
      rep->objective[k] = 0.5 * h->host_pinned[R_OBJ + k];
    }
    rep->e = h->host_pinned[R_E];
    rep->sigma = h->host_pinned[R_SIGMA];
    rep->slots = slots;
    rep->t = h->t;
  }
  return st;
}

// ------------------------------------------------------------------ reconstruction helpers
/* err_out, when ref is given, receives {sum (x_hat - ref)^2, sum ref^2} over every entry. */
static trd_status reconstruct_impl(trd_t* h, const double* const* cores, float* out, const float* ref,
                                   double* err_out) {
  const View v = full_view(h);
  const Split sp = choose_split(h, v, 0);
  Extra* x = X_(h);
  const bool dbl = is_fp64(h);
  TRY(ensure(h, x->recA, elt(h) * sp.P_in * sp.Kp));
  TRY(ensure(h, x->recC, elt(h) * sp.P_out * sp.Kp));
  const Chain inner = make_chain(h, v, 0, sp.c, -1, nullptr, cores);
  const Chain outer = make_chain(h, v, sp.c, h->N, -1, nullptr, cores);
  CK(launch_chain(inner, x->recA.p, dbl, false, sp.Kp, h->stream), "merge inner");
  CK(launch_chain(outer, x->recC.p, dbl, true, sp.Kp, h->stream), "merge outer");
  const int parts = 4 * h->num_sms;
  TRY(ensure(h, x->errp, sizeof(double) * 2 * parts));
  CK(launch_reconstruct_mats(x->recA.p, x->recC.p, dbl, sp.P_in, sp.P_out, sp.Kp,
                             ref, out, ref ? (double*)x->errp.p : nullptr, parts, h->stream),
     "reconstruct");
  if (!ref) return sync_and_status(h);
  std::vector<double> hp(2 * (size_t)parts);
  CK(cudaMemcpyAsync(hp.data(), x->errp.p, sizeof(double) * 2 * parts, cudaMemcpyDeviceToHost, h->stream),
     "error partials");
  TRY(sync_and_status(h));
  double se = 0, sr = 0;
  for (int i = 0; i < parts; ++i) { se += hp[2 * i]; sr += hp[2 * i + 1]; }
  err_out[0] = se;
  err_out[1] = sr;
  return TRD_OK;
}

trd_status trd_reconstruct(trd_t* h, float* out) {
  TRY(check_handle(h));
  if (!out) return set_err(h, TRD_EINVAL, "NULL output");
  return reconstruct_impl(h, nullptr, out, nullptr, nullptr);
}

trd_status trd_reconstruct_from(trd_t* h, const double* const* cores_host, float* out) {
  TRY(check_handle(h));
  if (!out || !cores_host) return set_err(h, TRD_EINVAL, "NULL argument");
  Extra* x = X_(h);
  const double* ptrs[kMaxN] = {};
  for (int k = 0; k < h->N; ++k) {
    if (!cores_host[k]) return set_err(h, TRD_EINVAL, "NULL core");
    const size_t bytes = sizeof(double) * h->I[k] * h->K[k];
    TRY(ensure(h, x->tmpZ[k], bytes));
    CK(cudaMemcpyAsync(x->tmpZ[k].p, cores_host[k], bytes, cudaMemcpyHostToDevice, h->stream), "core upload");
    ptrs[k] = (const double*)x->tmpZ[k].p;
  }
  return reconstruct_impl(h, ptrs, out, nullptr, nullptr);
}

trd_status trd_recovery_error(trd_t* h, const float* ref, double* err) {
  TRY(check_handle(h));
  if (!ref || !err) return set_err(h, TRD_EINVAL, "NULL argument");
  double s[2];
  TRY(reconstruct_impl(h, nullptr, nullptr, ref, s));
  *err = s[1] > 0 ? sqrt(s[0] / s[1]) : sqrt(s[0]);
  return TRD_OK;
}

trd_status trd_psnr(trd_t* h, const float* ref, double peak, double* psnr_out) {
  TRY(check_handle(h));
  if (!ref || !psnr_out) return set_err(h, TRD_EINVAL, "NULL argument");
  if (!(peak > 0) || !isfinite(peak)) return set_err(h, TRD_EINVAL, "peak must be positive and finite");
  double s[2];
  TRY(reconstruct_impl(h, nullptr, nullptr, ref, s));
  double numel = 1;
  for (int k = 0; k < h->N; ++k) numel *= (double)h->I[k];
  *psnr_out = s[0] > 0 ? 10.0 * log10(peak * peak * numel / s[0]) : INFINITY;
  return TRD_OK;
}

trd_status trd_set_profiling(trd_t* h, int on) {
  TRY(check_handle(h));
  touch(h);
  if (on < 0 || on > 2) return set_err(h, TRD_EINVAL, "profiling level must be 0, 1 or 2");
  X_(h)->prof = on;
  return TRD_OK;
}

trd_status trd_get_profile(trd_t* h, int reset, double* out) {
  TRY(check_handle(h));
  if (!out) return set_err(h, TRD_EINVAL, "NULL output");
  CK(cudaStreamSynchronize(h->stream), "stream synchronize");
  prof_harvest(h);
  Extra* x = X_(h);
  for (int q = 0; q < Extra::NPROF; ++q) {
    out[2 * q] = x->prof_ms[q];
    out[2 * q + 1] = (double)x->prof_n[q];
    if (reset) {
      x->prof_ms[q] = 0;
      x->prof_n[q] = 0;
    }
  }
  return TRD_OK;
}

int64_t trd_kernel_launches(void) { return launches_total(); }

trd_status trd_set_graphs(trd_t* h, int on) {
  TRY(check_handle(h));
  touch(h);
  X_(h)->graphs_enabled = on != 0;
  return TRD_OK;
}

trd_status trd_wait_selftest(trd_t* h, int arrive, int64_t limit) {
  TRY(check_handle(h));
  if (limit < 1 || limit > (int64_t)1 << 24) return set_err(h, TRD_EINVAL, "limit out of range");
  CK(launch_wait_selftest(arrive != 0, (uint32_t)limit, h->dstatus, h->stream), "wait self-test");
  return sync_and_status(h);
}

// ------------------------------------------------------------------ sampled correntropy loss
static trd_status sampled_setup(trd_t* h, const void* const* cores_dev, int fp64, const double** Zc, Split& sp,
                                Split2& s2) {
  Extra* x = X_(h);
  const View fv = full_view(h);
  sp = choose_split(h, fv, 0);
  s2.N = h->N;
  s2.c = sp.c;
  s2.err = h->dstatus;
  for (int m = 0; m < h->N; ++m) s2.dim[m] = h->I[m];
  int64_t st_in = 1, st_out = 1;
  for (int m = 0; m < h->N; ++m) {
    if (m < sp.c) { s2.sin[m] = st_in; s2.sout[m] = 0; st_in *= h->I[m]; }
    else { s2.sin[m] = 0; s2.sout[m] = st_out; st_out *= h->I[m]; }
  }
  for (int k = 0; k < h->N; ++k) {
    if (!cores_dev[k]) return set_err(h, TRD_EINVAL, "NULL core");
    const int64_t n = h->I[k] * (int64_t)h->K[k];
    if (fp64) {
      Zc[k] = (const double*)cores_dev[k];
    } else {
      TRY(ensure(h, x->smpZ[k], sizeof(double) * n));
      CK(launch_to_double((const float*)cores_dev[k], n, (double*)x->smpZ[k].p, h->stream), "core widening");
      Zc[k] = (const double*)x->smpZ[k].p;
    }
  }
  const size_t e = fp64 ? sizeof(double) : sizeof(float);
  TRY(ensure(h, x->smpA, e * sp.P_in * sp.Kp));
  TRY(ensure(h, x->smpC, e * sp.P_out * sp.Kp));
  CK(launch_chain(make_chain(h, fv, 0, sp.c, -1, nullptr, Zc), x->smpA.p, fp64 != 0, false, sp.Kp, h->stream),
     "merge inner block");
  CK(launch_chain(make_chain(h, fv, sp.c, h->N, -1, nullptr, Zc), x->smpC.p, fp64 != 0, true, sp.Kp, h->stream),
     "merge outer block");
  return TRD_OK;
}

// The sampled entries grouped by their inner-block index a and outer-block index b.
static trd_status sampled_order(trd_t* h, const int32_t* idx_dev, int64_t M, const Split& sp, const Split2& s2,
                                bool fp64, SampledWork& wk) {
  Extra* x = X_(h);
  if (M > INT32_MAX || sp.P_in > INT32_MAX || sp.P_out > INT32_MAX)
    return set_err(h, TRD_ENOTIMPL, "sampled loss supports fewer than 2^31 entries and block sizes below 2^31");
  if (sp.Kp > 512) return set_err(h, TRD_ENOTIMPL, "sampled loss supports r_1 r_c <= 512");
  TRY(ensure(h, x->smpKa, sizeof(int32_t) * (size_t)M));
  TRY(ensure(h, x->smpKb, sizeof(int32_t) * (size_t)M));
  TRY(ensure(h, x->smpPa, sizeof(int32_t) * (size_t)M));
  TRY(ensure(h, x->smpPb, sizeof(int32_t) * (size_t)M));
  TRY(ensure(h, x->smpG, (fp64 ? sizeof(double) : sizeof(float)) * (size_t)M));
  TRY(ensure(h, x->smpCa, sizeof(uint32_t) * (size_t)sp.P_in));
  TRY(ensure(h, x->smpCb, sizeof(uint32_t) * (size_t)sp.P_out));
  TRY(ensure(h, x->smpUa, sizeof(uint32_t) * (size_t)sp.P_in));
  TRY(ensure(h, x->smpUb, sizeof(uint32_t) * (size_t)sp.P_out));
  wk.ka = (int32_t*)x->smpKa.p;
  wk.kb = (int32_t*)x->smpKb.p;
  wk.perm_a = (int32_t*)x->smpPa.p;
  wk.perm_b = (int32_t*)x->smpPb.p;
  wk.cnt_a = (uint32_t*)x->smpCa.p;
  wk.cnt_b = (uint32_t*)x->smpCb.p;
  wk.cur_a = (uint32_t*)x->smpUa.p;
  wk.cur_b = (uint32_t*)x->smpUb.p;
  wk.g = x->smpG.p;
  CK(launch_sampled_order(idx_dev, &s2, M, sp.P_in, sp.P_out, wk, h->stream), "sampled entry grouping");
  return TRD_OK;
}

trd_status trd_sampled_fwd(trd_t* h, const void* const* cores_dev, const int32_t* idx_dev, const void* x_dev,
                           int64_t M, double sigma, int fp64, void* resid_dev, double* loss_out) {
  TRY(check_handle(h));
  touch(h);
  if (!cores_dev || !idx_dev || !x_dev || M < 1 || !loss_out || !(sigma > 0) || !isfinite(sigma))
    return set_err(h, TRD_EINVAL, "bad arguments");
  Extra* x = X_(h);
  const double* Zc[kMaxN];
  Split sp;
  Split2 s2;
  TRY(sampled_setup(h, cores_dev, fp64, Zc, sp, s2));
  const int parts = 8 * h->num_sms;
  TRY(ensure(h, x->smpLoss, sizeof(double) * parts));
  SampledWork wk;
  TRY(sampled_order(h, idx_dev, M, sp, s2, fp64 != 0, wk));
  CK(launch_sampled_rows(x->smpA.p, x->smpC.p, fp64 != 0, sp.Kp, x_dev, M, sp.P_in, sigma, resid_dev,
                         (double*)x->smpLoss.p, parts, false, 0.0, nullptr, nullptr, wk, h->stream),
     "sampled forward");
  std::vector<double> lp((size_t)parts);
  CK(cudaMemcpyAsync(lp.data(), x->smpLoss.p, sizeof(double) * parts, cudaMemcpyDeviceToHost, h->stream),
     "loss partials");
  TRY(sync_and_status(h));
  double loss = 0.0;
  for (int i = 0; i < parts; ++i) loss += lp[(size_t)i];
  *loss_out = loss;
  return TRD_OK;
}

trd_status trd_sampled_bwd(trd_t* h, const void* const* cores_dev, const int32_t* idx_dev, const void* x_dev,
                           int64_t M, double sigma, int fp64, double g_scale, void* const* grad_dev) {
  TRY(check_handle(h));
  touch(h);
  if (!cores_dev || !idx_dev || !x_dev || M < 1 || !grad_dev || !(sigma > 0) || !isfinite(sigma))
    return set_err(h, TRD_EINVAL, "bad arguments");
  for (int k = 0; k < h->N; ++k)
    if (!grad_dev[k]) return set_err(h, TRD_EINVAL, "NULL gradient buffer");
  Extra* x = X_(h);
  const double* Zc[kMaxN];
  Split sp;
  Split2 s2;
  TRY(sampled_setup(h, cores_dev, fp64, Zc, sp, s2));
  const bool dbl = fp64 != 0;
  const size_t e = dbl ? sizeof(double) : sizeof(float);
  TRY(ensure(h, x->smpGA, e * sp.P_in * sp.Kp));
  TRY(ensure(h, x->smpGC, e * sp.P_out * sp.Kp));
  CK(cudaMemsetAsync(x->smpGA.p, 0, e * sp.P_in * sp.Kp, h->stream), "clear gA");
  CK(cudaMemsetAsync(x->smpGC.p, 0, e * sp.P_out * sp.Kp, h->stream), "clear gC");
  const int parts = 8 * h->num_sms;
  SampledWork wk;
  TRY(sampled_order(h, idx_dev, M, sp, s2, dbl, wk));
  CK(launch_sampled_rows(x->smpA.p, x->smpC.p, dbl, sp.Kp, x_dev, M, sp.P_in, sigma, nullptr, nullptr, parts, true,
                         g_scale, x->smpGA.p, x->smpGC.p, wk, h->stream),
     "sampled adjoint");
  // the back-contraction reads FP64 halves
  const double* gAd = (const double*)x->smpGA.p;
  const double* gCd = (const double*)x->smpGC.p;
  if (!dbl) {
    TRY(ensure(h, x->smpGAd, sizeof(double) * sp.P_in * sp.Kp));
    TRY(ensure(h, x->smpGCd, sizeof(double) * sp.P_out * sp.Kp));
    CK(launch_to_double((const float*)x->smpGA.p, sp.P_in * sp.Kp, (double*)x->smpGAd.p, h->stream), "widen gA");
    CK(launch_to_double((const float*)x->smpGC.p, sp.P_out * sp.Kp, (double*)x->smpGCd.p, h->stream), "widen gC");
    gAd = (const double*)x->smpGAd.p;
    gCd = (const double*)x->smpGCd.p;
  }
  const View fv = full_view(h);
  const int N = h->N, c = sp.c;
  for (int k = 0; k < N; ++k) {
    const bool rows = k < c;
    const int rk = h->R[k], rk1 = h->R[(k + 1) % N];
    int pre0, pre1, post0, post1, mr, mc;
    if (rows) { pre0 = 0; pre1 = k; post0 = k + 1; post1 = c; mr = h->R[c]; mc = h->R[0]; }
    else { pre0 = c; pre1 = k; post0 = k + 1; post1 = N; mr = h->R[0]; mc = h->R[c]; }
    const Chain pre = make_chain(h, fv, pre0, pre1, -1, nullptr, Zc);
    const Chain post = make_chain(h, fv, post0, post1, -1, nullptr, Zc);
    const int64_t n_pre = pre.n > 0 ? pre.count : 1, n_post = post.n > 0 ? post.count : 1;
    if (pre.n > 1) {
      TRY(ensure(h, x->smpPre, e * n_pre * mc * rk));
      CK(launch_chain(pre, x->smpPre.p, dbl, false, mc * rk, h->stream), "merge prefix");
    }
    if (post.n > 1) {
      TRY(ensure(h, x->smpPost, e * n_post * rk1 * mr));
      CK(launch_chain(post, x->smpPost.p, dbl, false, rk1 * mr, h->stream), "merge suffix");
    }
    const int64_t nsplit = bc_splits(h, n_pre * n_post, h->I[k]);
    const int K = h->K[k];
    TRY(ensure(h, x->smpD, sizeof(double) * h->I[k] * K));
    if (nsplit > 1) TRY(ensure(h, x->smpDpart, sizeof(double) * nsplit * h->I[k] * K));
    TRY(bc_counters(h, h->I[k]));
    CK(launch_backcontract(rows ? (const void*)gAd : (const void*)gCd, sp.Kp, rows, mr, mc,
                           pre.n > 1 ? x->smpPre.p : nullptr, n_pre, post.n > 1 ? x->smpPost.p : nullptr, n_post,
                           h->I[k], rk, rk1, (double*)x->smpDpart.p, (int)nsplit, (double*)x->smpD.p,
                           (unsigned*)x->bc_ctr.p, dbl, h->stream, nullptr, bc_core(pre), bc_core(post)),
       "adjoint back-contraction");
    CK(launch_from_double((const double*)x->smpD.p, h->I[k] * (int64_t)K, grad_dev[k], dbl, h->stream),
       "gradient store");
  }
  return sync_and_status(h);
}

}  // extern "C"
