// Fused data passes on the 5th-generation tensor cores (BF16 operands) and the helpers of the
// tensor-core path: operand preparation, mask re-layout, slot reduction, the bounded-wait
// self-test and the launch dispatch.  The kernel itself is the template in pass_tc.cuh; the
// TF32 instantiations live in pass_tc_tf32.cu.
#include "pass_tc.cuh"

namespace trd {

namespace tc {

// Self-test of the bounded wait the pass uses: one thread waits (at most `limit` polls) for
// phase 0 of a fresh barrier, which completes only if `arrive` is set.  A wait that gives up
// is reported exactly as in the pass (DEV_TIMEOUT in the status word); nothing else is touched.
__global__ void k_wait_selftest(int arrive, uint32_t limit, int* err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_word;
  if (threadIdx.x != 0) return;
  abort_word = 0;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive) mbar_arrive(&bar);
  if (!mbar_wait_n(&bar, 0, reinterpret_cast<volatile int*>(&abort_word), limit)) atomicOr(err, (int)DEV_TIMEOUT);
}

// ------------------------------------------------------------------ operand preparation
// BF16 hi/lo split of a merged matrix [rows][Kp] (float) into [rows][kpad] (zero padded).
__global__ void k_split_rows(const float* __restrict__ src, int64_t rows, int Kp, int kpad,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  pdl_wait();
  pdl_trigger();
  const int64_t n = rows * kpad;
  const int step = gridDim.x * blockDim.x, e0 = blockIdx.x * blockDim.x + threadIdx.x;
  RowCol rc(e0, step, kpad);
  for (int64_t e = e0; e < n; e += step, rc.next()) {
    const int64_t r = rc.r;
    const int k = rc.c;
    const float v = k < Kp ? src[r * Kp + k] : 0.f;
    const __nv_bfloat16 h = bf16_rn(v);
    hi[e] = h;
    if (lo) lo[e] = bf16_rn(v - __bfloat162float(h));
  }
}

// TF32 hi/lo split of a merged matrix [rows][Kp] (float) into [rows][kpad] float arrays whose
// values are TF32-rounded (hi = tf32(v), lo = tf32(v - hi); zero padded), and optionally the
// same splits transposed, [kpad][ldT] (columns >= rows are left as they are: the tensor map
// of the transposed copy ends at `rows`).
__global__ void k_split_rows_tf32(const float* __restrict__ src, int64_t rows, int Kp, int kpad,
                                  float* __restrict__ hi, float* __restrict__ lo, float* __restrict__ hiT,
                                  float* __restrict__ loT, int64_t ldT) {
  const int64_t n = rows * kpad;
  const int step = gridDim.x * blockDim.x, e0 = blockIdx.x * blockDim.x + threadIdx.x;
  RowCol rc(e0, step, kpad);
  for (int64_t e = e0; e < n; e += step, rc.next()) {
    const int64_t r = rc.r;
    const int k = rc.c;
    const float v = k < Kp ? src[r * Kp + k] : 0.f;
    const uint32_t h = tf32_rna(v);
    const float l = __uint_as_float(tf32_rna(v - __uint_as_float(h)));
    hi[e] = __uint_as_float(h);
    if (lo) lo[e] = l;
    if (hiT) {
      hiT[(int64_t)k * ldT + r] = __uint_as_float(h);
      loT[(int64_t)k * ldT + r] = l;
    }
  }
}

// Rows of the data tensor re-laid with a padded stride: out[b][a] = X[b P_in + a] for
// a < P_in, 0 for P_in <= a < ld (TMA needs row strides that are multiples of 16 bytes).
__global__ void k_pad_rows(const float* __restrict__ X, int64_t P_in, int64_t P_out, int64_t ld,
                           float* __restrict__ out) {
  const int64_t n = P_out * ld;
  const int step = gridDim.x * blockDim.x, e0 = blockIdx.x * blockDim.x + threadIdx.x;
  RowCol rc(e0, step, (int)ld);
  for (int64_t e = e0; e < n; e += step, rc.next()) {
    const int64_t b = rc.r, a = rc.c;
    out[e] = a < P_in ? X[b * P_in + a] : 0.f;
  }
}

// Padded mask rows: Mrows[b][w] = bits [P_in b + 32 w, P_in b + 32 w + 32) of the packed mask
// (bits at or beyond P_in are zero).
__global__ void k_mask_rows(const uint32_t* __restrict__ M, int64_t P_in, int64_t P_out, int64_t W,
                            uint32_t* __restrict__ out) {
  const int64_t n = P_out * W;
  const int step = gridDim.x * blockDim.x, e0 = blockIdx.x * blockDim.x + threadIdx.x;
  RowCol rc(e0, step, (int)W);
  for (int64_t e = e0; e < n; e += step, rc.next()) {
    const int64_t b = rc.r, w = rc.c;
    const int64_t a0 = 32 * w;
    uint32_t v = 0;
    if (a0 < P_in) {
      if (!M) {
        const int64_t nb = imin(32, P_in - a0);
        v = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
      } else {
        const int64_t bit = P_in * b + a0;
        const int64_t wd = bit >> 5;
        const int sh = (int)(bit & 31);
        const int64_t nwords = (P_in * P_out + 31) / 32;
        const uint64_t lo = M[wd];
        const uint64_t hi = (sh && wd + 1 < nwords) ? (uint64_t)M[wd + 1] : 0ull;
        v = (uint32_t)(((hi << 32) | lo) >> sh);
        const int64_t nb = imin(32, P_in - a0);
        if (nb < 32) v &= (1u << nb) - 1u;
      }
    }
    out[e] = v;
  }
}

// Transposed padded mask: MT[a][w] bit j = observation bit of (a, b = 32 w + j), i.e. the
// bits of one inner index along the outer index.  One warp per (32 consecutive a, word w):
// lane j fetches the 32-bit window of column b = 32 w + j starting at row a0, then 32 ballots
// transpose the 32 x 32 bit block.
__global__ void k_mask_transpose(const uint32_t* __restrict__ M, int64_t P_in, int64_t P_out, int64_t WT,
                                 uint32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nab = (P_in + 31) / 32;
  const int64_t nwords = (P_in * P_out + 31) / 32;
  const int task0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  RowCol rc(task0, (int)warps, (int)WT);
  for (int64_t task = task0; task < nab * WT; task += warps, rc.next()) {
    const int64_t ab = rc.r, w = rc.c;
    const int64_t a0 = ab * 32;
    const int64_t b = 32 * w + lane;
    uint32_t col = 0;
    if (b < P_out) {
      if (!M) {
        const int64_t nb = imin(32, P_in - a0);
        col = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
      } else {
        const int64_t bit = a0 + P_in * b;
        const int64_t wd = bit >> 5;
        const int sh = (int)(bit & 31);
        const uint64_t lo = M[wd];
        const uint64_t hi = (sh && wd + 1 < nwords) ? (uint64_t)M[wd + 1] : 0ull;
        col = (uint32_t)(((hi << 32) | lo) >> sh);
        const int64_t nb = imin(32, P_in - a0);
        if (nb < 32) col &= (1u << nb) - 1u;
      }
    }
    uint32_t mine = 0;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const uint32_t bits = __ballot_sync(0xffffffffu, (col >> r) & 1u);
      if (lane == r) mine = bits;
    }
    const int64_t a = a0 + lane;
    if (a < P_in) out[a * WT + w] = mine;
  }
}

// T of stationary block rb = sum of the partial slots c + rb of the CTAs c whose unit range
// [c U / G, (c + 1) U / G) meets the block's units [rb NT, (rb + 1) NT), in CTA order.  One
// block per (stationary block, 256 entries of its BM x Kp tile); the CTA range is found once
// per block.
__global__ void k_reduce_slots(const float* __restrict__ part, int64_t RB, int64_t NT, int G, int64_t P_stat,
                               int Kp, double* __restrict__ out) {
  __shared__ int64_t s_c0, s_c1;
  const int64_t rb = blockIdx.x;
  if (threadIdx.x == 0) {
    const int64_t U = RB * NT, ulo = rb * NT, uhi = (rb + 1) * NT;
    int64_t c0 = (ulo * G) / U;
    while (c0 > 0 && (c0 * U) / G > ulo) --c0;
    while (((c0 + 1) * U) / G <= ulo) ++c0;
    int64_t c1 = c0;
    while (c1 < G && (c1 * U) / G < uhi) ++c1;
    s_c0 = c0;
    s_c1 = c1;
  }
  __syncthreads();
  const int64_t c0 = s_c0, c1 = s_c1;
  const int e = blockIdx.y * blockDim.x + threadIdx.x;
  if (e >= BM * Kp) return;
  const int r = e / Kp, k = e % Kp;
  const int64_t srow = rb * BM + r;
  if (srow >= P_stat) return;
  double s = 0.0;
  for (int64_t cc = c0; cc < c1; ++cc) s += (double)part[((cc + rb) * BM + r) * Kp + k];
  out[srow * Kp + k] = s;
}

}  // namespace tc

// ------------------------------------------------------------------ host side
namespace tc {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

bool make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
              uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace tc

int tc_kpad(int Kp, bool tf32) {
  if (Kp <= 64) return 64;
  if (tf32) return 0;
  return Kp <= 128 ? 128 : (Kp <= 256 ? 256 : 0);
}
int tc_bm() { return tc::BM; }
int tc_bn(int kpad, bool tf32) { return (tf32 || kpad > 128) ? 32 : 64; }

cudaError_t launch_wait_selftest(bool arrive, uint32_t limit, int* err, cudaStream_t st) {
  tc::k_wait_selftest<<<1, 32, 0, st>>>(arrive ? 1 : 0, limit, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_prep(const float* src, int64_t rows, int Kp, __nv_bfloat16* hi, __nv_bfloat16* lo,
                           cudaStream_t st) {
  const int kpad = tc_kpad(Kp, false);
  if (!kpad) return cudaErrorInvalidValue;
  const int64_t n = rows * kpad;
  pdl_launch(tc::k_split_rows, dim3((unsigned)imin((n + 255) / 256, 8192)), dim3(256), 0, st, src, rows, Kp, kpad, hi,
             lo);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_pad_rows(const float* X, int64_t P_in, int64_t P_out, int64_t ld, float* out, cudaStream_t st) {
  const int64_t n = P_out * ld;
  tc::k_pad_rows<<<(unsigned)imin((n + 255) / 256, 8192), 256, 0, st>>>(X, P_in, P_out, ld, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mask_rows(const uint32_t* M, int64_t P_in, int64_t P_out, int64_t W, uint32_t* out,
                             cudaStream_t st) {
  const int64_t n = P_out * W;
  tc::k_mask_rows<<<(unsigned)imin((n + 255) / 256, 8192), 256, 0, st>>>(M, P_in, P_out, W, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mask_transpose(const uint32_t* M, int64_t P_in, int64_t P_out, int64_t WT, uint32_t* out,
                                  cudaStream_t st) {
  const int64_t tasks = ((P_in + 31) / 32) * WT;
  const unsigned blocks = (unsigned)imin((tasks * 32 + 255) / 256, 8192);
  tc::k_mask_transpose<<<blocks, 256, 0, st>>>(M, P_in, P_out, WT, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_reduce_slots(const float* part, int64_t RB, int64_t NT, int G, int64_t P_stat, int Kp,
                                double* out, cudaStream_t st) {
  const dim3 grid((unsigned)RB, (unsigned)((tc::BM * Kp + 255) / 256));
  tc::k_reduce_slots<<<grid, 256, 0, st>>>(part, RB, NT, G, P_stat, Kp, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_prep_tf32(const float* src, int64_t rows, int Kp, float* hi, float* lo, cudaStream_t st,
                                float* hiT, float* loT, int64_t ldT) {
  const int kpad = tc_kpad(Kp, true);
  if (!kpad || (hiT && (!loT || ldT < rows))) return cudaErrorInvalidValue;
  const int64_t n = rows * kpad;
  tc::k_split_rows_tf32<<<(unsigned)imin((n + 255) / 256, 8192), 256, 0, st>>>(src, rows, Kp, kpad, hi, lo, hiT,
                                                                                loT, ldT);
  note_launch();
  return cudaGetLastError();
}

// Launch one fused pass.  Operands: [P_stat][KPAD] and [P_strm][KPAD] (BF16, or FP32 arrays of
// TF32-rounded splits); X: P_out rows of P_in floats with row stride ldx; Mst: [P_stat][W]
// mask words.
cudaError_t launch_pass_tc(bool tf32, bool rows_case, bool pass2, const PassOperands& o, const float* X,
                           int64_t P_in, int64_t ldx, int64_t P_out, const uint32_t* Mst, int64_t W,
                           int64_t P_stat, int64_t P_strm, int Kp, const double* sigma, float* Tpart,
                           double* stat_part, int* err, int G, bool full_stats, cudaStream_t st,
                           unsigned char* wq) {
  using namespace tc;
  const int KPAD = tc_kpad(Kp, tf32);
  // BF16 pass 1 always leaves its weights in the cache (the line-search pass reads them)
  if (!tf32 && !pass2 && (!wq || ((uintptr_t)wq & 15))) return cudaErrorInvalidValue;
  // TMA row strides must be multiples of 16 bytes: callers pass X re-laid with ldx % 4 == 0
  if (!KPAD || (ldx % 4) != 0 || ldx < P_in || ((uintptr_t)X & 15)) return cudaErrorInvalidValue;
  Params p{};
  p.P_in = P_in;
  p.P_stat = P_stat;
  p.P_strm = P_strm;
  p.Kp = Kp;
  p.Mst = Mst;
  p.W = W;
  p.sigma = sigma;
  p.Tpart = Tpart;
  p.stat_part = stat_part;
  p.err = err;
  p.wq = wq;
  if (tf32) return launch_pass_tc_tf32(KPAD, rows_case, pass2, full_stats, o, X, P_in, ldx, P_out, p, G, st);
  if (KPAD == 64)
    return launch_pass_tc_kp<64, false>(rows_case, pass2, full_stats, o, X, P_in, ldx, P_out, p, G, st);
  if (KPAD == 128)
    return launch_pass_tc_kp<128, false>(rows_case, pass2, full_stats, o, X, P_in, ldx, P_out, p, G, st);
  return launch_pass_tc_kp<256, false>(rows_case, pass2, full_stats, o, X, P_in, ldx, P_out, p, G, st);
}

int64_t tc_wq_bytes(int Kp, int64_t P_stat, int64_t P_strm) {
  const int kpad = tc_kpad(Kp, false);
  if (!kpad) return 0;
  const int64_t BN = tc_bn(kpad, false);
  return ((P_stat + tc::BM - 1) / tc::BM) * ((P_strm + BN - 1) / BN) * tc::BM * BN;
}

cudaError_t launch_pass_wls(const void* S_h, const void* T_hi, const unsigned char* wq, int Kp, int64_t P_stat,
                            int64_t P_strm, double* stat_part, int* err, int G, const double* nf_in,
                            cudaStream_t st) {
  using namespace tc;
  const int kpad = tc_kpad(Kp, false);
  if (!kpad || !wq || ((uintptr_t)wq & 15)) return cudaErrorInvalidValue;
  if (kpad == 64) return launch_pass_wls_kp<64>(S_h, T_hi, wq, P_stat, P_strm, stat_part, err, G, nf_in, st);
  if (kpad == 128) return launch_pass_wls_kp<128>(S_h, T_hi, wq, P_stat, P_strm, stat_part, err, G, nf_in, st);
  return launch_pass_wls_kp<256>(S_h, T_hi, wq, P_stat, P_strm, stat_part, err, G, nf_in, st);
}

}  // namespace trd
