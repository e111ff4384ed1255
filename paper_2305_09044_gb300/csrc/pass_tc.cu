// Fused data passes on the 5th-generation tensor cores (BF16 path), sm_103a.
//
// Same contraction as the CUDA-core passes (X_hat = S_st S_str^T, row kappa = gamma r_c +
// delta of the merged subchains), mapped onto tcgen05:
//   GEMM 1  D1[m][n]   = sum_k S_st[m][k] S_str[n][k]      (split BF16: hi*hi + hi*lo + lo*hi,
//                                                           FP32 accumulation in TMEM)
//   epilogue (FP32)    e = x - x_hat, w = exp(-e^2 / 2 sigma^2), y = w e on observed slots
//   GEMM 2  T[m][k]   += sum_n Y[m][n] S_str[n][k]          (BF16 Y and S_str, FP32 in TMEM)
// Pass 2 replaces GEMM 2 by D2 = S_h S_str^T (BF16) and reduces den = sum w D2^2.
//
// Work split: the stationary index (128 rows per block, the UMMA M) times the streaming
// tiles (64 columns) form units; CTA c of G (one per SM) takes the contiguous unit range
// [cU/G, (c+1)U/G), which may span several stationary blocks ("segments").  Each segment's
// partial contraction goes to slot c + rb of a partial buffer; a fixed-order reduction adds
// the slots, so results are deterministic.
//
// Warp roles (352 threads): warp 0 operand producer (TMA), warp 1 TMEM allocator +
// single-thread MMA issuer, warps 2..9 epilogue (TMEM lane quarter = warp % 4, two column
// groups), warp 10 data producer (TMA of the X tiles).  The contraction is padded to
// KP = 64 or 128 (r_1 r_c <= 128), stored as 64-wide K sub-tiles.  Tiles move by TMA
// (cp.async.bulk.tensor) into 1024-byte aligned SWIZZLE_128B operand buffers; every mbarrier
// wait is bounded: a wait that runs out sets an error word, all roles drain and the kernel
// returns after freeing its TMEM.
#include <cuda.h>

#include "trd_internal.cuh"

namespace trd {

namespace tc {

constexpr int BM = 128;        // UMMA M: stationary rows per block
constexpr int BN = 64;         // streaming columns per tile
constexpr int NEPI = 8;        // epilogue warps: 4 TMEM lane quarters x NGRP column groups
constexpr int NGRP = NEPI / 4;
constexpr int CPW = BN / NGRP; // columns of a tile handled by one epilogue warp
static_assert(CPW == 32, "the epilogue loads 32 accumulator columns per warp and tile");
constexpr int NTHREADS = 64 + 32 * NEPI + 64;   // operand producer, GEMM-1 issuer, epilogue, data
                                                // producer, GEMM-2 issuer
constexpr int EPI_THREADS = 32 * NEPI;
constexpr int XWARP = 2 + NEPI;                 // warp index of the data producer
constexpr int G2WARP = 3 + NEPI;                // warp index of the GEMM-2 issuer
constexpr uint32_t WAIT_LIMIT = 1u << 24;

// shared-memory carve-up (bytes, every buffer 1024-aligned).  Operands are stored as 64-wide
// K sub-tiles (one 128-byte swizzle atom per row); KP = 64 or 128 is the padded contraction.
constexpr int X_TILE = BN * BM * 4;            // 32 KB: one data tile
constexpr int Y_COLS = BN / 2;                 // TMEM columns of one Y buffer (BF16 pairs)
constexpr int SUB_S = BM * 64 * 2;             // 16 KB: one K sub-tile of a stationary operand
constexpr int SUB_T = BN * 64 * 2;             // 8 KB: one K sub-tile of a streaming operand

constexpr int ND = 4;          // GEMM-1 accumulator buffers in TMEM (the MMA runs ahead of the epilogue)
constexpr int NY = 4;          // weighted-residual (Y) buffers
constexpr uint32_t TMEM_COLS = 512;

template <int KP>
struct Cfg {
  static constexpr int NSUB = KP / 64;
  // data-tile stages (released by the epilogue): as many as shared memory allows
  __host__ __device__ static constexpr int xs(bool pass2) { return KP == 64 ? (pass2 ? 3 : 4) : (pass2 ? 2 : 3); }
  static constexpr int TS = KP == 64 ? 4 : 2;    // streaming-operand stages (released by MMA commits)
  static constexpr int S_TILE = BM * KP * 2;     // one stationary operand
  static constexpr int T_TILE = BN * KP * 2;     // one streaming operand
};

struct Layout {
  int s_hi, s_lo, s_h, x0, t0, y, bars, total;
};

template <int KP>
__host__ __device__ constexpr Layout layout(bool pass2) {
  using C = Cfg<KP>;
  Layout L{};
  int o = 0;
  L.s_hi = o; o += C::S_TILE;
  L.s_lo = o; o += C::S_TILE;
  L.s_h = o; if (pass2) o += C::S_TILE;
  L.x0 = o; o += C::xs(pass2) * X_TILE;
  L.t0 = o; o += C::TS * 2 * C::T_TILE;   // per stage: hi tile then lo tile
  L.y = o;                              // (Y lives in TMEM)
  L.bars = o; o += 1024;
  L.total = o;
  return L;
}
static_assert(layout<64>(false).total + 1024 <= 232448 && layout<64>(true).total + 1024 <= 232448, "smem");
static_assert(layout<128>(false).total + 1024 <= 232448 && layout<128>(true).total + 1024 <= 232448, "smem");

struct Params {
  int64_t P_in, P_stat, P_strm;
  int Kp;                    // valid contraction columns (<= KPAD)
  int64_t RB, NT, U;         // stationary blocks, streaming tiles, units
  int G;                     // CTAs
  const uint32_t* Mst;       // mask bits of each stationary index along the streaming index
  int64_t W;                 // words per mask row
  const double* sigma;
  float* Tpart;              // [G + RB][BM][Kp]
  double* stat_part;         // [G][8]
  int* err;                  // device status word
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false (and the abort flag set) when the limit is reached or another role
// has aborted.
// Non-blocking probe of a phase (for the MMA issuer, which polls two streams of work).
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_n(uint64_t* b, uint32_t parity, volatile int* abort_flag, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  return mbar_wait_n(b, parity, abort_flag, WAIT_LIMIT);
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}
// The same copy with an L2 eviction-priority hint (a policy from createpolicy): the streamed
// data tensor is read once per pass (evict first), the merged operands are re-read by every
// CTA (evict last).
__device__ __forceinline__ void tma_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(su32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// GEMM with the A operand in tensor memory (rows = lanes, K along columns, two BF16 per column).
__device__ __forceinline__ void tc_mma_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// 16 columns of this thread's lane from 16 registers; completed by tmem_wait_st.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// Split form: issue the load, do other work, then wait.  The wait names the destination
// registers as operands so that no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_issue32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait32(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_wait64(uint32_t* r, uint32_t* q) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]),
                 "+r"(q[4]), "+r"(q[5]), "+r"(q[6]), "+r"(q[7]), "+r"(q[8]), "+r"(q[9]), "+r"(q[10]), "+r"(q[11]),
                 "+r"(q[12]), "+r"(q[13]), "+r"(q[14]), "+r"(q[15]), "+r"(q[16]), "+r"(q[17]), "+r"(q[18]),
                 "+r"(q[19]), "+r"(q[20]), "+r"(q[21]), "+r"(q[22]), "+r"(q[23]), "+r"(q[24]), "+r"(q[25]),
                 "+r"(q[26]), "+r"(q[27]), "+r"(q[28]), "+r"(q[29]), "+r"(q[30]), "+r"(q[31])
               :
               : "memory");
}

// columns-per-warp dispatch
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
  if constexpr (N == 32) tmem_ld32(taddr, v);
  else tmem_ld16(taddr, v);
}

// UMMA shared-memory descriptor: K-major, SWIZZLE_128B (8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}
// UMMA shared-memory descriptor: MN-major, SWIZZLE_128B.  64 MN-contiguous elements per
// 128-byte row, one row per K index, 8-row groups 1024 B apart (stride byte offset), and
// 64-wide MN blocks `lbo` bytes apart (leading byte offset).
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::f16: D FP32, A/B BF16, A K-major, B K-major (b_mn = 0) or
// MN-major (b_mn = 1), M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int b_mn = 0) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// 2^x on the special-function unit (ex2.approx, flush-to-zero); the weight needs only
// about 1e-6 relative accuracy in this path.
__device__ __forceinline__ float fast_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// ------------------------------------------------------------------ the kernel
template <bool ROWS, bool PASS2, bool FULL, int KP>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_pass_tc(const __grid_constant__ CUtensorMap mS_hi, const __grid_constant__ CUtensorMap mS_lo,
              const __grid_constant__ CUtensorMap mS_h, const __grid_constant__ CUtensorMap mT_hi,
              const __grid_constant__ CUtensorMap mT_lo, const __grid_constant__ CUtensorMap mX,
              const Params p) {
  constexpr int KPAD = KP, NSUB = Cfg<KP>::NSUB, XS = Cfg<KP>::xs(PASS2), TS = Cfg<KP>::TS;
  constexpr int S_TILE = Cfg<KP>::S_TILE, T_TILE = Cfg<KP>::T_TILE;
  constexpr Layout L = layout<KP>(PASS2);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // align the dynamic window to 1024 bytes (the launcher over-allocates by 1 KB)
  unsigned char* sm = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* x_full = bars;                // [XS]  data tile landed (TMA)
  uint64_t* x_empty = x_full + XS;        // [XS]  data tile read by every epilogue thread
  uint64_t* t_full = x_empty + XS;        // [TS]  streaming operands landed (TMA)
  uint64_t* t_empty = t_full + TS;        // [TS]  streaming operands consumed (MMA commit)
  uint64_t* d_full = t_empty + TS;        // [ND]  GEMM 1 (and the h product) done
  uint64_t* d_empty = d_full + ND;        // [ND]  accumulators read by the epilogue
  uint64_t* y_full = d_empty + ND;        // [NY]  Y written
  uint64_t* y_empty = y_full + NY;        // [NY]  GEMM 2 consumed Y
  uint64_t* s_full = y_empty + NY;        //       stationary operands landed
  uint64_t* s_empty = s_full + 1;         //       segment's GEMM-1 MMAs done with them
  uint64_t* acc_full = s_empty + 1;       //       segment's contraction complete
  uint64_t* acc_empty = acc_full + 1;     //       contraction drained to global
  uint64_t* mma_done = acc_empty + 1;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_done + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 2);
  double* red = reinterpret_cast<double*>(mma_done + 4);   // [NEPI warps][8] statistics

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = blockIdx.x;
  const int64_t u_begin = c * p.U / p.G, u_end = (c + 1) * p.U / p.G;

  if (threadIdx.x == 0) {
    for (int s = 0; s < XS; ++s) {
      mbar_init(&x_full[s], 1);
      mbar_init(&x_empty[s], EPI_THREADS);
    }
    for (int s = 0; s < TS; ++s) {
      mbar_init(&t_full[s], 1);
      mbar_init(&t_empty[s], PASS2 ? 2 : 1);   // pass 2: both issuers read the tile
    }
    for (int b = 0; b < ND; ++b) {
      mbar_init(&d_full[b], PASS2 ? 2 : 1);    // pass 2: X_hat and the step product
      mbar_init(&d_empty[b], EPI_THREADS);
    }
    for (int b = 0; b < NY; ++b) {
      mbar_init(&y_full[b], EPI_THREADS);
      mbar_init(&y_empty[b], 1);
    }
    mbar_init(s_full, 1);
    mbar_init(s_empty, PASS2 ? 2 : 1);       // pass 2: both issuers read the stationary tiles
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, EPI_THREADS);
    mbar_init(mma_done, 2);            // one commit from each issuer
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM columns: D1[b] at b BN (b < ND), then D2[b] (pass 2) at (ND + b) BN or, in pass 1,
  // the T accumulator at ND BN (KPAD columns) followed by the NY weighted-residual buffers Y
  // (BF16 pairs, Y_COLS columns each; the A operand of GEMM 2)
  const uint32_t col_acc = (uint32_t)(ND * BN);
  const uint32_t col_y = col_acc + (uint32_t)KPAD;
  static_assert(ND * BN + KPAD + NY * Y_COLS <= (int)TMEM_COLS, "TMEM columns");

  if (warp == 0) {
    // ---------------------------------------------------------------- operand producer
    if (lane == 0) {
      const uint64_t keep = policy_evict_last();
      int64_t it = 0;
      int g = 0;
      bool ok = true;
      int last_phase[TS];
      for (int s = 0; s < TS; ++s) last_phase[s] = -1;
      int s_phase = -1;
      for (int64_t u = u_begin; u < u_end && ok; ++g) {
        const int64_t rb = u / p.NT;
        const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
        if (g > 0) ok = mbar_wait(s_empty, (uint32_t)((g - 1) & 1), abort_flag);
        if (!ok) break;
        mbar_expect_tx(s_full, (PASS2 ? 3 : 2) * S_TILE);
        s_phase = g & 1;
#pragma unroll
        for (int sb = 0; sb < NSUB; ++sb) {
          tma_2d_hint(sm + L.s_hi + sb * SUB_S, &mS_hi, s_full, sb * 64, (int)(rb * BM), keep);
          tma_2d_hint(sm + L.s_lo + sb * SUB_S, &mS_lo, s_full, sb * 64, (int)(rb * BM), keep);
          if (PASS2) tma_2d_hint(sm + L.s_h + sb * SUB_S, &mS_h, s_full, sb * 64, (int)(rb * BM), keep);
        }
        for (int64_t tc = u - rb * p.NT; u < seg_end; ++u, ++it, ++tc) {
          const int s = (int)(it % TS);
          if (!mbar_wait(&t_empty[s], (uint32_t)(((it / TS) & 1) ^ 1), abort_flag)) { ok = false; break; }
          const int t0 = (int)(tc * BN);
          unsigned char* tb = sm + L.t0 + s * 2 * T_TILE;
          mbar_expect_tx(&t_full[s], 2 * T_TILE);
          last_phase[s] = (int)((it / TS) & 1);
#pragma unroll
          for (int sb = 0; sb < NSUB; ++sb) {
            tma_2d_hint(tb + sb * SUB_T, &mT_hi, &t_full[s], sb * 64, t0, keep);
            tma_2d_hint(tb + T_TILE + sb * SUB_T, &mT_lo, &t_full[s], sb * 64, t0, keep);
          }
        }
      }
      if (!ok) {
        // drain: wait (bounded) for the last copies issued into every buffer
        for (int s = 0; s < TS; ++s)
          if (last_phase[s] >= 0)
            for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
              if (mbar_try(&t_full[s], (uint32_t)last_phase[s])) break;
        if (s_phase >= 0)
          for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
            if (mbar_try(s_full, (uint32_t)s_phase)) break;
      }
    }
  } else if (warp == XWARP) {
    // ---------------------------------------------------------------- data producer
    if (lane == 0) {
      const uint64_t stream_once = policy_evict_first();
      int64_t it = 0;
      bool ok = true;
      int last_phase[XS];
      for (int s = 0; s < XS; ++s) last_phase[s] = -1;
      int64_t rb = u_begin / p.NT, tc = u_begin - rb * p.NT;   // running block / tile counters
      for (int64_t u = u_begin; u < u_end; ++u, ++it) {
        const int s = (int)(it % XS);
        if (!mbar_wait(&x_empty[s], (uint32_t)(((it / XS) & 1) ^ 1), abort_flag)) { ok = false; break; }
        const int t0 = (int)(tc * BN);
        unsigned char* xb = sm + L.x0 + s * X_TILE;
        mbar_expect_tx(&x_full[s], X_TILE);
        last_phase[s] = (int)((it / XS) & 1);
        if (ROWS) {
          tma_2d_hint(xb, &mX, &x_full[s], (int)(rb * BM), t0, stream_once);
        } else {
          tma_2d_hint(xb, &mX, &x_full[s], t0, (int)(rb * BM), stream_once);
          tma_2d_hint(xb + X_TILE / 2, &mX, &x_full[s], t0 + 32, (int)(rb * BM), stream_once);
        }
        if (++tc == p.NT) {
          tc = 0;
          ++rb;
        }
      }
      if (!ok)
        for (int s = 0; s < XS; ++s)
          if (last_phase[s] >= 0)
            for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
              if (mbar_try(&x_full[s], (uint32_t)last_phase[s])) break;
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- GEMM-1 issuer
    // X_hat tiles (and, in pass 2, the step-direction product) into the ND accumulator
    // buffers, as soon as a tile's streaming operands and a free buffer are there
    if (lane == 0) {
      constexpr uint32_t ID1 = idesc_bf16(BM, BN);
      // shared-memory descriptors built once; a K step only adds its byte offset / 16 to the
      // start-address field (addresses stay below 2^18, so the 14-bit field cannot carry)
      const uint64_t dA_hi = sdesc(su32(sm + L.s_hi)), dA_lo = sdesc(su32(sm + L.s_lo));
      int64_t it = 0;
      int g = 0;
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok; ++g) {
        const int64_t rb = u / p.NT;
        const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
        if (!mbar_wait(s_full, (uint32_t)(g & 1), abort_flag)) { ok = false; break; }
        for (; u < seg_end; ++u, ++it) {
          const int s = (int)(it % TS), b = (int)(it & (ND - 1));
          if (!mbar_wait(&t_full[s], (uint32_t)((it / TS) & 1), abort_flag)) { ok = false; break; }
          if (!mbar_wait(&d_empty[b], (uint32_t)(((it / ND) & 1) ^ 1), abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint64_t dB_hi = sdesc(su32(sm + L.t0 + s * 2 * T_TILE));
          const uint64_t dB_lo = dB_hi + (uint64_t)(T_TILE >> 4);
          const uint32_t d1 = tmem + (uint32_t)(b * BN);
#pragma unroll
          for (int kk = 0; kk < KPAD / 16; ++kk) {
            // K step kk: sub-tile kk / 4, 32-byte step kk % 4 inside its swizzle atom
            const uint64_t ka = (uint64_t)(((kk >> 2) * SUB_S + (kk & 3) * 32) >> 4);
            const uint64_t kb = (uint64_t)(((kk >> 2) * SUB_T + (kk & 3) * 32) >> 4);
            tc_mma(d1, dA_hi + ka, dB_hi + kb, ID1, kk > 0);
            tc_mma(d1, dA_hi + ka, dB_lo + kb, ID1, 1);
            tc_mma(d1, dA_lo + ka, dB_hi + kb, ID1, 1);
          }
          tc_commit(&d_full[b]);
          if (PASS2) tc_commit(&t_empty[s]);   // pass 1: released by the GEMM-2 issuer
        }
        if (!ok) break;
        tc_commit(s_empty);                     // the segment's stationary operands may go
      }
      // every issued MMA has finished before TMEM can be released
      tc_commit(mma_done);
      for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try(mma_done, 0)) break;
    }
  } else if (warp == G2WARP) {
    // ---------------------------------------------------------------- GEMM-2 issuer
    // T += Y S_str per tile once the epilogue has written Y (which it does after reading the
    // tile's GEMM-1 result, so GEMM 1 of the tile has completed); releases the tile's
    // streaming operands and Y buffer; a segment's T is complete after its last tile
    if (lane == 0 && PASS2) {
      // pass 2: D2 = S_h S_str^T (plain BF16) into the second accumulator of each buffer slot
      constexpr uint32_t ID1 = idesc_bf16(BM, BN);
      const uint64_t dA_h = sdesc(su32(sm + L.s_h));
      int64_t it = 0;
      int g = 0;
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok; ++g) {
        const int64_t rb = u / p.NT;
        const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
        if (!mbar_wait(s_full, (uint32_t)(g & 1), abort_flag)) { ok = false; break; }
        for (; u < seg_end; ++u, ++it) {
          const int s = (int)(it % TS), b = (int)(it & (ND - 1));
          if (!mbar_wait(&t_full[s], (uint32_t)((it / TS) & 1), abort_flag)) { ok = false; break; }
          if (!mbar_wait(&d_empty[b], (uint32_t)(((it / ND) & 1) ^ 1), abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint64_t dB_hi = sdesc(su32(sm + L.t0 + s * 2 * T_TILE));
          const uint32_t d2 = tmem + (uint32_t)((ND + b) * BN);
#pragma unroll
          for (int kk = 0; kk < KPAD / 16; ++kk) {
            const uint64_t ka = (uint64_t)(((kk >> 2) * SUB_S + (kk & 3) * 32) >> 4);
            const uint64_t kb = (uint64_t)(((kk >> 2) * SUB_T + (kk & 3) * 32) >> 4);
            tc_mma(d2, dA_h + ka, dB_hi + kb, ID1, kk > 0);
          }
          tc_commit(&d_full[b]);
          tc_commit(&t_empty[s]);
        }
        if (!ok) break;
        tc_commit(s_empty);
      }
    }
    if (lane == 0) {
      if (!PASS2) {
        constexpr uint32_t ID2 = idesc_bf16(BM, KPAD, 1);    // B = streaming tile, MN-major
        int64_t it = 0;
        int g = 0;
        bool ok = true;
        for (int64_t u = u_begin; u < u_end && ok; ++g) {
          const int64_t rb = u / p.NT;
          const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
          bool first2 = true;
          for (; u < seg_end; ++u, ++it) {
            const int s = (int)(it % TS), yb = (int)(it & (NY - 1));
            if (first2 && g > 0 && !mbar_wait(acc_empty, (uint32_t)((g - 1) & 1), abort_flag)) { ok = false; break; }
            if (!mbar_wait(&y_full[yb], (uint32_t)((it / NY) & 1), abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint64_t dT = sdesc_mn(su32(sm + L.t0 + s * 2 * T_TILE), BN * 128);
            const uint32_t ay = tmem + col_y + (uint32_t)(yb * Y_COLS);
#pragma unroll
            for (int kk = 0; kk < BN / 16; ++kk)
              tc_mma_ta(tmem + col_acc, ay + (uint32_t)(kk * 8), dT + (uint64_t)(kk * (2048 >> 4)), ID2,
                        (first2 && kk == 0) ? 0u : 1u);
            tc_commit(&y_empty[yb]);
            tc_commit(&t_empty[s]);
            first2 = false;
          }
          if (!ok) break;
          tc_commit(acc_full);
        }
      }
      tc_commit(mma_done);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (NEPI warps)
    // warp w (2..NEPI+1) reads TMEM lane quarter q = w % 4 and column group grp (CPW columns)
    const int q = warp & 3;
    const int grp = (warp - 2) >> 2;
    const int row = q * 32 + lane;          // stationary row within the block
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const double sg = *p.sigma;
    // exp(-e^2 / (2 sigma^2)) = exp2(-e^2 * k), k = log2(e) / (2 sigma^2); sigma = inf -> k = 0
    const float nk = isinf(sg) ? 0.0f : (float)(-1.4426950408889634 / (2.0 * sg * sg));
    // exp(-e^2 / (2 sigma^2)) = exp2(-(e s)^2) with s = sqrt(log2(e) / (2 sigma^2))
    const float sk = isinf(sg) ? 0.0f : (float)sqrt(1.4426950408889634 / (2.0 * sg * sg));
    constexpr uint32_t CMASK = CPW == 32 ? 0xffffffffu : ((1u << CPW) - 1u);
    float sw = 0.f, se2 = 0.f, swe2 = 0.f, sden = 0.f;
    uint32_t nobs = 0, nnf = 0, nslot = 0;
    int64_t it = 0;
    int g = 0;
    bool ok = true;
    for (int64_t u = u_begin; u < u_end && ok; ++g) {
      const int64_t rb = u / p.NT;
      const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
      const int64_t srow = rb * BM + row;
      const bool row_ok = srow < p.P_stat;
      const uint32_t* mrow = p.Mst + (row_ok ? srow : 0) * p.W;
      const int c0 = grp * CPW;                 // first tile column of this warp
      // observation bits: this thread's 32 bits of a tile are one mask word (CPW = 32, tiles
      // 64 columns apart), fetched three tiles ahead (the words of one warp lie in 32
      // different mask rows, so each fetch has the full L2 latency)
      // tiles of this segment are tc0 .. tc_end - 1 of stationary block rb (no divisions in
      // the tile loop)
      const int64_t tc0 = u - rb * p.NT, tc_end = seg_end - rb * p.NT;
      auto mword_of = [&](int64_t tt) -> uint32_t {
        return (row_ok && tt < tc_end) ? __ldg(mrow + ((tt * BN + c0) >> 5)) : 0u;
      };
      uint32_t mq0 = mword_of(tc0), mq1 = mword_of(tc0 + 1), mq2 = mword_of(tc0 + 2);
      for (int64_t tc = tc0; u < seg_end; ++u, ++it, ++tc) {
        const int xs = (int)(it % XS), b = (int)(it & (ND - 1)), yb = (int)(it & (NY - 1));
        const int64_t t0 = tc * BN;
        const uint32_t mword = mq0;
        mq0 = mq1;
        mq1 = mq2;
        mq2 = mword_of(tc + 3);
        const int64_t nc = p.P_strm - t0 - c0;  // valid columns for this warp
        const uint32_t vmask = (!row_ok || nc <= 0) ? 0u : (nc >= CPW ? CMASK : ((1u << nc) - 1u));
        // accumulators first: the TMEM loads are in flight while X is read from shared memory
        if (!mbar_wait(&d_full[b], (uint32_t)((it / ND) & 1), abort_flag)) { ok = false; break; }
        tc_fence_after();
        uint32_t rx[32], rd[32];
        tmem_issue32(tmem + lane_base + (uint32_t)(b * BN + c0), rx);
        if (PASS2) tmem_issue32(tmem + lane_base + (uint32_t)((ND + b) * BN + c0), rd);
        if (!mbar_wait(&x_full[xs], (uint32_t)((it / XS) & 1), abort_flag)) {
          if (PASS2) tmem_wait64(rx, rd);
          else tmem_wait32(rx);
          ok = false;
          break;
        }
        const unsigned char* xt = sm + L.x0 + xs * X_TILE;
        float xh[CPW], dh[CPW], xv[CPW];
        if (ROWS) {
          const float* sx = reinterpret_cast<const float*>(xt) + c0 * BM + row;
#pragma unroll
          for (int j = 0; j < CPW; ++j) xv[j] = sx[j * BM];
        } else {
          // SWIZZLE_128B boxes of 32 columns: 16-byte chunk c of row r sits at chunk c ^ (r & 7)
          const unsigned char* box = xt + (c0 >> 5) * (X_TILE / 2) + row * 128;
          const int cb = (c0 & 31) >> 2;
#pragma unroll
          for (int c4 = 0; c4 < CPW / 4; ++c4) {
            const float4 v = *reinterpret_cast<const float4*>(box + (((cb + c4) ^ (row & 7)) << 4));
            xv[4 * c4 + 0] = v.x; xv[4 * c4 + 1] = v.y; xv[4 * c4 + 2] = v.z; xv[4 * c4 + 3] = v.w;
          }
        }
        mbar_arrive(&x_empty[xs]);
        if (PASS2) tmem_wait64(rx, rd);
        else tmem_wait32(rx);
#pragma unroll
        for (int j = 0; j < CPW; ++j) {
          xh[j] = __uint_as_float(rx[j]);
          if (PASS2) dh[j] = __uint_as_float(rd[j]);
        }
        tc_fence_before();
        mbar_arrive(&d_empty[b]);
        const uint32_t seen = mword & vmask;
        nslot += __popc(vmask);
        nobs += __popc(seen);
        // branch-free slot update (predicated selects keep the slots independent)
        if (FULL) {
          // exact statistics: sum w, sum e^2, sum w e^2 and a count of non-finite residuals
          uint32_t fin = 0;
#pragma unroll
          for (int j = 0; j < CPW; ++j) {
            const float e = xv[j] - xh[j];
            const bool use = ((seen >> j) & 1u) && (fabsf(e) <= 3.402823466e38f);
            fin |= use ? (1u << j) : 0u;
            // selects, not products with 0, so that a NaN stored at an unobserved slot stays out
            const float eu = use ? e : 0.f;
            const float uw = use ? fast_ex2(e * e * nk) : 0.f;
            if (PASS2) {
              sden = fmaf(uw * dh[j], dh[j], sden);
            } else {
              const float y = uw * eu;
              sw += uw;
              se2 = fmaf(eu, eu, se2);
              swe2 = fmaf(y, eu, swe2);
              xv[j] = y;
            }
          }
          nnf += __popc(seen & ~fin);
        } else {
          // lean: only what the update needs (y, or den) and the objective sum w e^2; a
          // non-finite residual on an observed slot propagates as NaN and rejects the step.
          // Pass 1 masks the residual first (e' = 0 off the mask, so w(e') = 1 and y = w e' = 0
          // without further selects); pass 2 masks the weight.
#pragma unroll
          for (int j = 0; j < CPW; ++j) {
            const bool bit = (seen >> j) & 1u;
            if (PASS2) {
              const float t = (xv[j] - xh[j]) * sk;
              const float w = bit ? fast_ex2(-(t * t)) : 0.f;
              sden = fmaf(w * dh[j], dh[j], sden);
            } else {
              const float e = bit ? xv[j] - xh[j] : 0.f;
              const float t = e * sk;
              const float y = fast_ex2(-(t * t)) * e;
              swe2 = fmaf(y, e, swe2);
              xv[j] = y;
            }
          }
        }
        if (!PASS2) {
          uint32_t ypk[CPW / 2];
#pragma unroll
          for (int j = 0; j < CPW; j += 2) ypk[j >> 1] = pack_bf16(xv[j], xv[j + 1]);
          if (!mbar_wait(&y_empty[yb], (uint32_t)(((it / NY) & 1) ^ 1), abort_flag)) { ok = false; break; }
          // this warp's 32 residuals of row `row` -> 16 columns of Y buffer yb in TMEM
          tmem_st16(tmem + lane_base + col_y + (uint32_t)(yb * Y_COLS + (c0 >> 1)), ypk);
          tmem_wait_st();
          tc_fence_before();
          mbar_arrive(&y_full[yb]);
        }
      }
      if (!ok) break;
      if (!PASS2) {
        // drain the segment's contraction: this warp's columns of row `row` of T -> slot c + rb
        if (!mbar_wait(acc_full, (uint32_t)(g & 1), abort_flag)) { ok = false; break; }
        tc_fence_after();
        float* dst = p.Tpart + ((c + rb) * BM + row) * (int64_t)p.Kp;
        constexpr int KPW = KPAD / NGRP;                  // 32 or 64 columns per warp
#pragma unroll
        for (int h0 = 0; h0 < KPW; h0 += 32) {
          float v[32];
          tmem_ld<32>(tmem + lane_base + col_acc + grp * KPW + h0, v);
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (grp * KPW + h0 + j < p.Kp) dst[grp * KPW + h0 + j] = row_ok ? v[j] : 0.f;
        }
        tc_fence_before();
        mbar_arrive(acc_empty);
      }
    }
    if (!FULL) nnf = (isfinite(swe2) && isfinite(sden)) ? 0u : 1u;
    // statistics: warp shuffle, then one row per CTA (fixed order)
    const double fv[7] = {(double)sw, (double)se2, (double)swe2, (double)nobs, (double)nnf, (double)nslot,
                          (double)sden};
#pragma unroll
    for (int f = 0; f < 7; ++f) {
      double x = fv[f];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) red[(warp - 2) * 8 + f] = x;
    }
  }
  // ------------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int f = 0; f < 7; ++f) {
      double x = 0.0;
      for (int w = 0; w < NEPI; ++w) x += red[w * 8 + f];
      p.stat_part[c * 8 + f] = x;
    }
    p.stat_part[c * 8 + 7] = 0.0;
    if (*abort_flag) atomicOr(p.err, (int)DEV_TIMEOUT);
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

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
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
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

bool make_map(CUtensorMap* m, CUtensorMapDataType dt, int esize, const void* base, uint64_t inner, uint64_t outer,
              uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t es[2] = {1, 1};
  (void)esize;
  return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

int tc_kpad(int Kp) { return Kp <= 64 ? 64 : (Kp <= 128 ? 128 : 0); }
int tc_bm() { return tc::BM; }
int tc_bn() { return tc::BN; }

cudaError_t launch_wait_selftest(bool arrive, uint32_t limit, int* err, cudaStream_t st) {
  tc::k_wait_selftest<<<1, 32, 0, st>>>(arrive ? 1 : 0, limit, err);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc_prep(const float* src, int64_t rows, int Kp, __nv_bfloat16* hi, __nv_bfloat16* lo,
                           cudaStream_t st) {
  const int kpad = tc_kpad(Kp);
  if (!kpad) return cudaErrorInvalidValue;
  const int64_t n = rows * kpad;
  tc::k_split_rows<<<(unsigned)imin((n + 255) / 256, 8192), 256, 0, st>>>(src, rows, Kp, kpad, hi, lo);
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

// Launch one fused pass.  S operands: [P_stat][KPAD] bf16 (hi, lo, h); streaming operands:
// [P_strm][KPAD] (hi, lo); X: [P_out][P_in] floats; Mst: [P_stat][W] mask words.
cudaError_t launch_pass_tc(bool rows_case, bool pass2, const __nv_bfloat16* S_hi, const __nv_bfloat16* S_lo,
                           const __nv_bfloat16* S_h, const __nv_bfloat16* T_hi, const __nv_bfloat16* T_lo,
                           const float* X, int64_t P_in, int64_t ldx, int64_t P_out, const uint32_t* Mst, int64_t W,
                           int64_t P_stat, int64_t P_strm, int Kp, const double* sigma, float* Tpart,
                           double* stat_part, int* err, int G, bool full_stats, cudaStream_t st) {
  using namespace tc;
  const int KPAD = tc_kpad(Kp);
  // TMA row strides must be multiples of 16 bytes: callers pass X re-laid with ldx % 4 == 0
  if (!KPAD || (ldx % 4) != 0 || ldx < P_in || ((uintptr_t)X & 15)) return cudaErrorInvalidValue;
  CUtensorMap mS_hi, mS_lo, mS_h, mT_hi, mT_lo, mX;
  const CUtensorMapDataType BF = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapSwizzle SW = CU_TENSOR_MAP_SWIZZLE_128B;
  // operand arrays [rows][KPAD] bf16, fetched as 64-wide sub-tiles (128-byte rows, SW128)
  bool ok = make_map(&mS_hi, BF, 2, S_hi, KPAD, P_stat, KPAD * 2, 64, BM, SW) &&
            make_map(&mS_lo, BF, 2, S_lo, KPAD, P_stat, KPAD * 2, 64, BM, SW) &&
            make_map(&mS_h, BF, 2, pass2 ? S_h : S_hi, KPAD, P_stat, KPAD * 2, 64, BM, SW) &&
            make_map(&mT_hi, BF, 2, T_hi, KPAD, P_strm, KPAD * 2, 64, BN, SW) &&
            make_map(&mT_lo, BF, 2, T_lo, KPAD, P_strm, KPAD * 2, 64, BN, SW);
  if (rows_case)
    ok = ok && make_map(&mX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, X, P_in, P_out, ldx * 4, BM, BN,
                        CU_TENSOR_MAP_SWIZZLE_NONE);
  else
    ok = ok && make_map(&mX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, X, P_in, P_out, ldx * 4, 32, BM, SW);
  if (!ok) return cudaErrorInvalidValue;
  Params p;
  p.P_in = P_in;
  p.P_stat = P_stat;
  p.P_strm = P_strm;
  p.Kp = Kp;
  p.RB = (P_stat + BM - 1) / BM;
  p.NT = (P_strm + BN - 1) / BN;
  p.U = p.RB * p.NT;
  p.G = (int)imin(G, p.U);
  p.Mst = Mst;
  p.W = W;
  p.sigma = sigma;
  p.Tpart = Tpart;
  p.stat_part = stat_part;
  p.err = err;
  const Layout L = KPAD == 64 ? layout<64>(pass2) : layout<128>(pass2);
  const size_t smem = (size_t)L.total + 1024;
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<p.G, NTHREADS, smem, st>>>(mS_hi, mS_lo, mS_h, mT_hi, mT_lo, mX, p);
    note_launch();
    return cudaGetLastError();
  };
  if (KPAD == 64) {
    if (pass2) return rows_case ? go(k_pass_tc<true, true, false, 64>) : go(k_pass_tc<false, true, false, 64>);
    if (full_stats)
      return rows_case ? go(k_pass_tc<true, false, true, 64>) : go(k_pass_tc<false, false, true, 64>);
    return rows_case ? go(k_pass_tc<true, false, false, 64>) : go(k_pass_tc<false, false, false, 64>);
  }
  if (pass2) return rows_case ? go(k_pass_tc<true, true, false, 128>) : go(k_pass_tc<false, true, false, 128>);
  if (full_stats)
    return rows_case ? go(k_pass_tc<true, false, true, 128>) : go(k_pass_tc<false, false, true, 128>);
  return rows_case ? go(k_pass_tc<true, false, false, 128>) : go(k_pass_tc<false, false, false, 128>);
}

}  // namespace trd
