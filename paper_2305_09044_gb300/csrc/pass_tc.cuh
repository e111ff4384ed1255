// The fused data pass on the 5th-generation tensor cores, sm_103a: kernel template shared by
// the BF16 and the TF32 translation units.
//
// Contraction (the ring cut in two, Thm. 1): X_hat = S_st S_str^T, row kappa = gamma r_c +
// delta of the merged subchains.  On tcgen05:
//   GEMM 1  D1[m][n]  = sum_k S_st[m][k] S_str[n][k]   3-term split of both operands:
//                                                       hi*hi + hi*lo + lo*hi, FP32 in TMEM
//   epilogue (FP32)   e = x - x_hat, w = exp(-e^2 / 2 sigma^2), y = w e on observed slots
//   GEMM 2  T[m][k]  += sum_n Y[m][n] S_str[n][k]       BF16 operands: Y and S_str^hi (one
//                                                       term); TF32 operands: 3-term split
// Pass 2 replaces GEMM 2 by D2 = S_h S_str^T (BF16: one term; TF32: 3-term split) and reduces
// den = sum w D2^2 (the exact line search of Sec. 3.2).
//
// Operand kinds: BF16 (kind::f16, K = 16 per MMA) and TF32 (kind::tf32, K = 8 per MMA).  With
// TF32 and three product terms, every contraction keeps about 22 significant bits per operand,
// i.e. FP32-level accuracy on the tensor cores.  Contraction widths KP = 64 / 128 / 256 (BF16)
// and 64 (TF32).  BF16 at KP = 256 and TF32 use 32-column streaming tiles (BN = 32) to fit
// shared memory and keep the step operand S_h of pass 2 in tensor memory (the A operand of D2)
// instead of shared memory.  The tensor cores read TF32 operands K-major only (an MN-major
// TF32 operand gave zero products on this GPU), so the TF32 GEMM 2 reads a transposed copy of
// the streaming operand, while BF16 reads the streaming tile itself MN-major.
//
// Work split: the stationary index (128 rows per block, the UMMA M) times the streaming tiles
// (BN columns) form units; CTA c of G (one per SM) takes the contiguous unit range
// [cU/G, (c+1)U/G), which may span several stationary blocks ("segments").  Each segment's
// partial contraction goes to slot c + rb of a partial buffer; a fixed-order reduction adds
// the slots, so results are deterministic.
//
// Warp roles (352 threads): warp 0 operand producer (TMA), warp 1 TMEM allocator + GEMM-1
// issuer, warps 2..9 epilogue (TMEM lane quarter = warp % 4, two column groups), warp 10 data
// producer (TMA of the X tiles), warp 11 GEMM-2 (pass 1) or D2 (pass 2) issuer.  Operands are
// stored as K sub-tiles one 128-byte swizzle row wide, in 1024-byte aligned SWIZZLE_128B
// buffers; every mbarrier wait is bounded: a wait that runs out sets an error word, all roles
// drain and the kernel returns after freeing its TMEM.
#pragma once

#include <cuda.h>

#include "trd_internal.cuh"

namespace trd {
namespace tc {

constexpr int BM = 128;        // UMMA M: stationary rows per block
constexpr int NEPI = 8;        // epilogue warps: 4 TMEM lane quarters x NGRP column groups
constexpr int NGRP = NEPI / 4;
constexpr int NTHREADS = 64 + 32 * NEPI + 64;   // operand producer, GEMM-1 issuer, epilogue, data
                                                // producer, GEMM-2 issuer
constexpr int EPI_THREADS = 32 * NEPI;
constexpr int XWARP = 2 + NEPI;                 // warp index of the data producer
constexpr int G2WARP = 3 + NEPI;                // warp index of the GEMM-2 issuer
constexpr uint32_t WAIT_LIMIT = 1u << 24;
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_LIMIT = 232448;              // opt-in dynamic shared memory per block

// Static configuration of one pass variant.
template <int KP, bool TF32, bool PASS2>
struct Cfg {
  static constexpr int ESZ = TF32 ? 4 : 2;      // operand element bytes
  static constexpr int SUBW = 128 / ESZ;        // elements in one K sub-tile row (128 bytes)
  static constexpr int NSUB = KP / SUBW;        // K sub-tiles per operand row
  static constexpr int KSTEPS = KP * ESZ / 32;  // MMAs per product term of GEMM 1 (32 bytes of K each)
  static constexpr int KROWS = 32 / ESZ;        // K of one MMA: streaming rows per GEMM-2 step
  static constexpr int BN = (TF32 || KP * ESZ > 256) ? 32 : 64;   // streaming columns per tile
  static constexpr int CPW = BN / NGRP;         // tile columns per epilogue warp
  static constexpr bool SH_TMEM = PASS2 && (TF32 || KP > 128);   // step operand in TMEM
  static constexpr bool SH_SMEM = PASS2 && !SH_TMEM;
  static constexpr int SH_COLS = SH_TMEM ? (TF32 ? 2 * KP : KP / 2) : 0;
  static constexpr int ND = 4;                  // GEMM-1 accumulator buffers in TMEM
  static constexpr int NY = 4;                  // weighted-residual (Y) buffers in TMEM
  static constexpr int Y_COLS = TF32 ? 2 * BN : BN / 2;   // TMEM columns of one Y buffer
  static constexpr int S_TILE = BM * KP * ESZ;  // one stationary operand
  static constexpr int T_TILE = BN * KP * ESZ;  // one streaming operand
  // TF32 pass 1: the streaming operand also as KP rows of BN elements (BN * 4 = 128 bytes), the
  // K-major B operand of GEMM 2 (the tensor cores take TF32 operands K-major only)
  static constexpr bool TT = TF32 && !PASS2;
  static constexpr int TT_TILE = TT ? KP * BN * 4 : 0;
  static constexpr int T_STAGE = 2 * T_TILE + 2 * TT_TILE;   // hi, lo (, hi^T, lo^T)
  static constexpr int SUB_S = BM * 128;        // one K sub-tile of a stationary operand
  static constexpr int SUB_T = BN * 128;        // one K sub-tile of a streaming operand
  static constexpr int X_TILE = BN * BM * 4;    // one data tile
  // data-tile stages (released by the epilogue) and streaming-operand stages (released by
  // MMA commits): as many as shared memory allows
  static constexpr int XS = TF32 ? 4
                            : KP == 64 ? (PASS2 ? 3 : 4)
                            : KP == 128 ? (PASS2 ? 2 : 3) : 2;
  static constexpr int TS = TF32 ? (PASS2 ? 4 : 3) : (KP == 64 ? 4 : 2);
  static constexpr int TMEM_USED = PASS2 ? 2 * ND * BN + SH_COLS : ND * BN + KP + NY * Y_COLS;
  // GEMM-2 tiles per TMEM accumulation chunk.  The tensor cores round the FP32 accumulator
  // toward zero after every MMA, a bias that grows with the number of MMAs summed into it
  // (measured: 2.7e-5 relative after about 2,000); the TF32 path restarts the accumulator every
  // CH tiles and sums the chunks in FP32 registers (round to nearest), BF16 drains once per
  // segment (its tolerance is far above this bias).
  static constexpr int CH = TF32 ? 4 : (1 << 30);
};

struct Layout {
  int s_hi, s_lo, s_h, x0, t0, bars, total;
};

template <class C>
__host__ __device__ constexpr Layout layout() {
  Layout L{};
  int o = 0;
  L.s_hi = o; o += C::S_TILE;
  L.s_lo = o; o += C::S_TILE;
  L.s_h = o; if (C::SH_SMEM) o += C::S_TILE;
  L.x0 = o; o += C::XS * C::X_TILE;
  L.t0 = o; o += C::TS * C::T_STAGE;   // per stage: hi tile, lo tile (, transposed hi, lo)
  L.bars = o; o += 1024;
  L.total = o;
  return L;
}

struct Params {
  int64_t P_in, P_stat, P_strm;
  int Kp;                    // valid contraction columns (<= KP)
  int64_t RB, NT, U;         // stationary blocks, streaming tiles, units
  int G;                     // CTAs
  const uint32_t* Mst;       // mask bits of each stationary index along the streaming index
  int64_t W;                 // words per mask row
  const double* sigma;
  float* Tpart;              // [G + RB][BM][Kp]
  double* stat_part;         // [G][8]
  int* err;                  // device status word
  // step operand rows copied into TMEM (pass 2 with SH_TMEM): column group g reads
  // sh_cols 32-bit words per row from shw[g] + row * sh_ld + sh_off[g]
  const uint32_t* shw[2];
  int sh_off[2];
  int sh_ld;
  // BF16 pass 1: the weight of every slot as 8-bit fixed point (q = round(255 w), 0 off the
  // mask), unit-major: unit u's BM x BN bytes at wq + u BM BN, row r's BN bytes at r BN with
  // its 16-byte chunks permuted by wq_chunk (so that the line-search pass reads them from
  // shared memory without bank conflicts)
  unsigned char* wq;
  // line-search pass from the cache: pass 1's reduced count of non-finite observed residuals
  // (such residuals get weight 0 in the cache; a non-zero count makes den NaN, as a pass that
  // recomputes the weights would)
  const double* nf_in;
};

// Byte offset of 16-byte chunk ch of row r inside one unit's weight block (BN bytes per row):
// the chunk index is XORed with the row's position among the rows that share a 128-byte line,
// so that 16-byte reads of one chunk by 32 consecutive rows fall on distinct banks.
template <int BN>
__host__ __device__ constexpr int wq_chunk(int r, int ch) {
  constexpr int CHR = BN / 16, RPL = 128 / BN;   // chunks per row, rows per 128-byte line
  return r * BN + ((ch ^ ((r / RPL) & (CHR - 1))) << 4);
}

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
  // a phase that has already completed is seen by the non-blocking probe (cheaper than a
  // try_wait, measured)
  if (mbar_test(b, parity)) return true;
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
// One MMA, A and B from shared memory (descriptors), D in TMEM; acc = 0 overwrites D.
template <bool TF32>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// The same with the A operand in tensor memory (rows = lanes, K along columns: two BF16 or one
// TF32 element per 32-bit column).
template <bool TF32>
__device__ __forceinline__ void tc_mma_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// TMEM loads in split form (issue, other work, then wait; the wait names the destination
// registers as operands so that no use of them is scheduled before it) and stores.
__device__ __forceinline__ void tmem_issue16(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_wait16x2(uint32_t* r, uint32_t* q) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), "+r"(q[6]), "+r"(q[7]), "+r"(q[8]), "+r"(q[9]), "+r"(q[10]), "+r"(q[11]), "+r"(q[12]), "+r"(q[13]), "+r"(q[14]), "+r"(q[15])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_issue32(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait32(uint32_t* r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_wait32x2(uint32_t* r, uint32_t* q) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]), "+r"(q[0]), "+r"(q[1]), "+r"(q[2]), "+r"(q[3]), "+r"(q[4]), "+r"(q[5]), "+r"(q[6]), "+r"(q[7]), "+r"(q[8]), "+r"(q[9]), "+r"(q[10]), "+r"(q[11]), "+r"(q[12]), "+r"(q[13]), "+r"(q[14]), "+r"(q[15]), "+r"(q[16]), "+r"(q[17]), "+r"(q[18]), "+r"(q[19]), "+r"(q[20]), "+r"(q[21]), "+r"(q[22]), "+r"(q[23]), "+r"(q[24]), "+r"(q[25]), "+r"(q[26]), "+r"(q[27]), "+r"(q[28]), "+r"(q[29]), "+r"(q[30]), "+r"(q[31])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :
               : "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               :
               : "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
               : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
               :
               : "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
               : "memory");
}
template <int N>
__device__ __forceinline__ void tmem_issue(uint32_t taddr, uint32_t* r) {
  if constexpr (N == 32) tmem_issue32(taddr, r);
  else tmem_issue16(taddr, r);
}
template <int N>
__device__ __forceinline__ void tmem_wait(uint32_t* r) {
  if constexpr (N == 32) tmem_wait32(r);
  else tmem_wait16(r);
}
template <int N>
__device__ __forceinline__ void tmem_wait_x2(uint32_t* r, uint32_t* q) {
  if constexpr (N == 32) tmem_wait32x2(r, q);
  else tmem_wait16x2(r, q);
}
template <int N>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t* r) {
  if constexpr (N == 32) tmem_st32(taddr, r);
  else if constexpr (N == 16) tmem_st16(taddr, r);
  else tmem_st8(taddr, r);
}
// 32 columns of this thread's lane, waited for
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  tmem_issue32(taddr, r);
  tmem_wait32(r);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// UMMA shared-memory descriptor: K-major, SWIZZLE_128B (8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}
// UMMA shared-memory descriptor: MN-major, SWIZZLE_128B.  128 bytes of MN-contiguous elements
// per row, one row per K index, 8-row groups 1024 B apart (stride byte offset), and MN blocks
// of one row's width `lbo` bytes apart (leading byte offset).
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor of kind::f16 (A/B BF16, format 1) or kind::tf32 (A/B TF32, format 2):
// D FP32, A K-major, B K-major (b_mn = 0) or MN-major (b_mn = 1), M x N.
__host__ __device__ constexpr uint32_t idesc_mma(int M, int N, bool tf32, int b_mn = 0) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 2^x on the special-function unit (ex2.approx, flush-to-zero); the weight needs only
// about 1e-6 relative accuracy in this path.
__device__ __forceinline__ float fast_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Weights of two slots -> two bytes round(255 w) in the low half of a word: w * 255 + 1.5 2^23
// (exact for w in [0, 1]; the FMA rounds to the nearest integer) keeps the integer in the low
// mantissa bits.
__device__ __forceinline__ uint32_t quant_pair(float w0, float w1) {
  const float2 q = __ffma2_rn(make_float2(w0, w1), make_float2(255.f, 255.f), make_float2(12582912.f, 12582912.f));
  return __byte_perm(__float_as_uint(q.x), __float_as_uint(q.y), 0x0040);
}

// Contiguous global -> shared copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) completing on an mbarrier, with an L2 policy.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// FP32 -> TF32 bit pattern, round to nearest (ties away from zero); the low 13 mantissa bits
// are zero, so the tensor cores use the value as it is.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// ------------------------------------------------------------------ the kernel
template <bool ROWS, bool PASS2, bool FULL, int KP, bool TF32>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_pass_tc(const __grid_constant__ CUtensorMap mS_hi, const __grid_constant__ CUtensorMap mS_lo,
              const __grid_constant__ CUtensorMap mS_h, const __grid_constant__ CUtensorMap mT_hi,
              const __grid_constant__ CUtensorMap mT_lo, const __grid_constant__ CUtensorMap mX,
              const __grid_constant__ CUtensorMap mTT_hi, const __grid_constant__ CUtensorMap mTT_lo,
              const Params p) {
  using C = Cfg<KP, TF32, PASS2>;
  constexpr int BN = C::BN, CPW = C::CPW, SUBW = C::SUBW, NSUB = C::NSUB, KSTEPS = C::KSTEPS;
  constexpr int XS = C::XS, TS = C::TS, ND = C::ND, NY = C::NY;
  constexpr int S_TILE = C::S_TILE, T_TILE = C::T_TILE, SUB_S = C::SUB_S, SUB_T = C::SUB_T;
  constexpr int X_TILE = C::X_TILE, T_STAGE = C::T_STAGE, TT_TILE = C::TT_TILE;
  constexpr Layout L = layout<C>();
  static_assert(BN % 32 == 0 && (CPW == 16 || CPW == 32), "epilogue column split");
  static_assert(C::TMEM_USED <= (int)TMEM_COLS, "TMEM columns");
  static_assert((ND & (ND - 1)) == 0 && (NY & (NY - 1)) == 0, "buffer counts are powers of two");
  static_assert(L.total + 1024 <= SMEM_LIMIT, "shared memory");
  static_assert(KSTEPS % 4 == 0 || KSTEPS < 4, "K steps within 128-byte rows");
  static_assert(!C::TT || BN * 4 == 128, "transposed TF32 tiles are one swizzle row wide");
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
  uint64_t* sh_full = mma_done + 1;       //       segment's step operand written to TMEM
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sh_full + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sh_full + 2);
  double* red = reinterpret_cast<double*>(sh_full + 4);   // [NEPI warps][8] statistics

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
    mbar_init(sh_full, EPI_THREADS);
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
  // the set-up above touches no global memory: it overlaps the previous kernel's tail
  pdl_wait();
  pdl_trigger();
  // TMEM columns: D1[b] at b BN (b < ND); pass 1: the T accumulator at ND BN (KP columns)
  // followed by the NY weighted-residual buffers Y (the A operand of GEMM 2: BF16 pairs, or
  // TF32 hi then lo); pass 2: D2[b] at (ND + b) BN, then the step operand S_h (SH_TMEM)
  const uint32_t col_acc = (uint32_t)(ND * BN);
  const uint32_t col_y = col_acc + (uint32_t)KP;
  const uint32_t col_sh = (uint32_t)(2 * ND * BN);

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
        mbar_expect_tx(s_full, (C::SH_SMEM ? 3 : 2) * S_TILE);
        s_phase = g & 1;
#pragma unroll
        for (int sb = 0; sb < NSUB; ++sb) {
          tma_2d_hint(sm + L.s_hi + sb * SUB_S, &mS_hi, s_full, sb * SUBW, (int)(rb * BM), keep);
          tma_2d_hint(sm + L.s_lo + sb * SUB_S, &mS_lo, s_full, sb * SUBW, (int)(rb * BM), keep);
          if (C::SH_SMEM) tma_2d_hint(sm + L.s_h + sb * SUB_S, &mS_h, s_full, sb * SUBW, (int)(rb * BM), keep);
        }
        for (int64_t tc = u - rb * p.NT; u < seg_end; ++u, ++it, ++tc) {
          const int s = (int)(it % TS);
          if (!mbar_wait(&t_empty[s], (uint32_t)(((it / TS) & 1) ^ 1), abort_flag)) { ok = false; break; }
          const int t0 = (int)(tc * BN);
          unsigned char* tb = sm + L.t0 + s * T_STAGE;
          mbar_expect_tx(&t_full[s], T_STAGE);
          last_phase[s] = (int)((it / TS) & 1);
#pragma unroll
          for (int sb = 0; sb < NSUB; ++sb) {
            tma_2d_hint(tb + sb * SUB_T, &mT_hi, &t_full[s], sb * SUBW, t0, keep);
            tma_2d_hint(tb + T_TILE + sb * SUB_T, &mT_lo, &t_full[s], sb * SUBW, t0, keep);
          }
          if constexpr (C::TT) {
            // columns t0 .. t0 + BN - 1 of the transposed operand, all KP rows
            tma_2d_hint(tb + 2 * T_TILE, &mTT_hi, &t_full[s], t0, 0, keep);
            tma_2d_hint(tb + 2 * T_TILE + TT_TILE, &mTT_lo, &t_full[s], t0, 0, keep);
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
          // BN / 32 boxes of 32 columns x BM rows (128-byte rows, SWIZZLE_128B)
#pragma unroll
          for (int q = 0; q < BN / 32; ++q)
            tma_2d_hint(xb + q * (BM * 128), &mX, &x_full[s], t0 + 32 * q, (int)(rb * BM), stream_once);
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
    // X_hat tiles into the ND accumulator buffers, as soon as a tile's streaming operands and
    // a free buffer are there
    if (lane == 0) {
      constexpr uint32_t ID1 = idesc_mma(BM, BN, TF32);
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
          const uint64_t dB_hi = sdesc(su32(sm + L.t0 + s * T_STAGE));
          const uint64_t dB_lo = dB_hi + (uint64_t)(T_TILE >> 4);
          const uint32_t d1 = tmem + (uint32_t)(b * BN);
#pragma unroll
          for (int kk = 0; kk < KSTEPS; ++kk) {
            // K step kk: sub-tile kk / 4, 32-byte step kk % 4 inside its swizzle row
            const uint64_t ka = (uint64_t)(((kk >> 2) * SUB_S + (kk & 3) * 32) >> 4);
            const uint64_t kb = (uint64_t)(((kk >> 2) * SUB_T + (kk & 3) * 32) >> 4);
            tc_mma<TF32>(d1, dA_hi + ka, dB_hi + kb, ID1, kk > 0);
            tc_mma<TF32>(d1, dA_hi + ka, dB_lo + kb, ID1, 1);
            tc_mma<TF32>(d1, dA_lo + ka, dB_hi + kb, ID1, 1);
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
    if (lane == 0 && PASS2) {
      // -------------------------------------------------------------- D2 issuer (pass 2)
      // D2 = S_h S_str^T into the second accumulator of each buffer slot; S_h from shared
      // memory (SH_SMEM) or from TMEM, where the epilogue writes it at each segment start
      constexpr uint32_t ID1 = idesc_mma(BM, BN, TF32);
      const uint64_t dA_h = sdesc(su32(sm + L.s_h));
      int64_t it = 0;
      int g = 0;
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok; ++g) {
        const int64_t rb = u / p.NT;
        const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
        if (!mbar_wait(s_full, (uint32_t)(g & 1), abort_flag)) { ok = false; break; }
        if (C::SH_TMEM && !mbar_wait(sh_full, (uint32_t)(g & 1), abort_flag)) { ok = false; break; }
        for (; u < seg_end; ++u, ++it) {
          const int s = (int)(it % TS), b = (int)(it & (ND - 1));
          if (!mbar_wait(&t_full[s], (uint32_t)((it / TS) & 1), abort_flag)) { ok = false; break; }
          if (!mbar_wait(&d_empty[b], (uint32_t)(((it / ND) & 1) ^ 1), abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint64_t dB_hi = sdesc(su32(sm + L.t0 + s * T_STAGE));
          const uint64_t dB_lo = dB_hi + (uint64_t)(T_TILE >> 4);
          const uint32_t d2 = tmem + (uint32_t)((ND + b) * BN);
#pragma unroll
          for (int kk = 0; kk < KSTEPS; ++kk) {
            const uint64_t kb = (uint64_t)(((kk >> 2) * SUB_T + (kk & 3) * 32) >> 4);
            if constexpr (C::SH_TMEM) {
              // K step kk is 8 TMEM columns of S_h (16 BF16 or 8 TF32 elements)
              const uint32_t a_hi = tmem + col_sh + (uint32_t)(kk * 8);
              if constexpr (TF32) {
                const uint32_t a_lo = a_hi + (uint32_t)KP;
                tc_mma_ta<TF32>(d2, a_hi, dB_hi + kb, ID1, kk > 0);
                tc_mma_ta<TF32>(d2, a_hi, dB_lo + kb, ID1, 1);
                tc_mma_ta<TF32>(d2, a_lo, dB_hi + kb, ID1, 1);
              } else {
                tc_mma_ta<TF32>(d2, a_hi, dB_hi + kb, ID1, kk > 0);
              }
            } else {
              const uint64_t ka = (uint64_t)(((kk >> 2) * SUB_S + (kk & 3) * 32) >> 4);
              tc_mma<TF32>(d2, dA_h + ka, dB_hi + kb, ID1, kk > 0);
            }
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
        // ------------------------------------------------------------ GEMM-2 issuer
        // T += Y S_str per tile once the epilogue has written Y (which it does after reading
        // the tile's GEMM-1 result, so GEMM 1 of the tile has completed); releases the tile's
        // streaming operands and Y buffer; a segment's T is complete after its last tile
        // BF16: B = the streaming tile read MN-major; TF32: B = its transposed copy, K-major
        constexpr uint32_t ID2 = idesc_mma(BM, KP, TF32, TF32 ? 0 : 1);
        constexpr int K2 = BN / C::KROWS;                       // MMAs per term over one tile
        constexpr uint32_t KB2 = (uint32_t)(C::KROWS * 128) >> 4;   // BF16 descriptor step per MMA
        int64_t it = 0, ch = 0;   // tiles, accumulation chunks
        int g = 0;
        bool ok = true;
        for (int64_t u = u_begin; u < u_end && ok; ++g) {
          const int64_t rb = u / p.NT;
          const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
          for (int jt = 0; u < seg_end; ++u, ++it, ++jt) {
            const int s = (int)(it % TS), yb = (int)(it & (NY - 1));
            const bool first2 = (jt % C::CH) == 0;                          // chunk's first tile
            const bool last2 = (jt % C::CH) == C::CH - 1 || u + 1 == seg_end;  // chunk's last tile
            if (first2 && ch > 0 && !mbar_wait(acc_empty, (uint32_t)((ch - 1) & 1), abort_flag)) { ok = false; break; }
            if (!mbar_wait(&y_full[yb], (uint32_t)((it / NY) & 1), abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t ay = tmem + col_y + (uint32_t)(yb * C::Y_COLS);
            if constexpr (TF32) {
              // KP rows of one 128-byte swizzle row each: K step kk is 32 bytes into the row
              const uint64_t dT = sdesc(su32(sm + L.t0 + s * T_STAGE + 2 * T_TILE));
              const uint64_t dTlo = dT + (uint64_t)(TT_TILE >> 4);
#pragma unroll
              for (int kk = 0; kk < K2; ++kk) {
                const uint32_t a = ay + (uint32_t)(kk * 8);
                const uint64_t kb = (uint64_t)((kk * 32) >> 4);
                tc_mma_ta<TF32>(tmem + col_acc, a, dT + kb, ID2, (first2 && kk == 0) ? 0u : 1u);
                tc_mma_ta<TF32>(tmem + col_acc, a, dTlo + kb, ID2, 1);
                tc_mma_ta<TF32>(tmem + col_acc, a + (uint32_t)BN, dT + kb, ID2, 1);
              }
            } else {
              const uint64_t dT = sdesc_mn(su32(sm + L.t0 + s * T_STAGE), SUB_T);
#pragma unroll
              for (int kk = 0; kk < K2; ++kk)
                tc_mma_ta<TF32>(tmem + col_acc, ay + (uint32_t)(kk * 8), dT + kk * KB2, ID2,
                                (first2 && kk == 0) ? 0u : 1u);
            }
            tc_commit(&y_empty[yb]);
            tc_commit(&t_empty[s]);
            if (last2) {
              tc_commit(acc_full);
              ++ch;
            }
          }
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
    constexpr uint32_t CMASK = CPW == 32 ? 0xffffffffu : ((1u << CPW) - 1u);
    float sw = 0.f, se2 = 0.f, swe2 = 0.f, sden = 0.f;
    // the lean epilogue works on slot pairs with packed FP32x2 arithmetic and keeps its running
    // sum (w e^2 in pass 1, w D2^2 in pass 2) in two packed accumulators: four independent
    // chains instead of one FMA chain through every slot
    float2 acc2a = make_float2(0.f, 0.f), acc2b = make_float2(0.f, 0.f);
    const float2 nk2 = make_float2(nk, nk), neg1 = make_float2(-1.f, -1.f);
    uint32_t nobs = 0, nnf = 0, nslot = 0;
    constexpr int KPW = KP / NGRP;                  // contraction columns of T per warp
    constexpr bool CHUNKED = TF32 && !PASS2;        // T summed over chunks in registers
    static_assert(!CHUNKED || KPW == 32, "chunk sums held in 32 registers");
    float tacc[CHUNKED ? 32 : 1];
#pragma unroll
    for (int j = 0; j < (CHUNKED ? 32 : 1); ++j) tacc[j] = 0.f;
    int64_t it = 0, ch = 0;
    int g = 0;
    bool ok = true;
    // phases of the next tile's accumulator and data tile already seen complete by an early
    // probe (a probe of a completed phase takes about 110 cycles: issued before the arithmetic,
    // its latency hides behind it; a phase still open is waited for as usual)
    bool pre_d = false, pre_x = false;
    for (int64_t u = u_begin; u < u_end && ok; ++g) {
      const int64_t rb = u / p.NT;
      const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
      const int64_t srow = rb * BM + row;
      const bool row_ok = srow < p.P_stat;
      if constexpr (C::SH_TMEM) {
        // this segment's step-operand rows into TMEM (the A operand of D2).  Every D2 product
        // of the previous segment has completed: this warp has read all of its results.
        constexpr int HALF = C::SH_COLS / 2;
        const uint32_t* src = p.shw[grp] + (row_ok ? srow : 0) * (int64_t)p.sh_ld + p.sh_off[grp];
#pragma unroll
        for (int ch = 0; ch < HALF; ch += 32) {
          uint32_t wv[32];
#pragma unroll
          for (int v4 = 0; v4 < 8; ++v4) {
            const uint4 w4 = row_ok ? __ldg(reinterpret_cast<const uint4*>(src + ch) + v4) : make_uint4(0u, 0u, 0u, 0u);
            wv[4 * v4 + 0] = w4.x; wv[4 * v4 + 1] = w4.y; wv[4 * v4 + 2] = w4.z; wv[4 * v4 + 3] = w4.w;
          }
          tmem_st<32>(tmem + lane_base + col_sh + (uint32_t)(grp * HALF + ch), wv);
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(sh_full);
      }
      const uint32_t* mrow = p.Mst + (row_ok ? srow : 0) * p.W;
      const int c0 = grp * CPW;                 // first tile column of this warp
      // observation bits: this thread's CPW bits of a tile lie in one mask word (BN is a
      // multiple of 32), fetched three tiles ahead (the words of one warp lie in 32 different
      // mask rows, so each fetch has the full L2 latency); tiles of this segment are
      // tc0 .. tc_end - 1 of stationary block rb (no divisions in the tile loop)
      const int64_t tc0 = u - rb * p.NT, tc_end = seg_end - rb * p.NT;
      auto mword_of = [&](int64_t tt) -> uint32_t {
        if (!(row_ok && tt < tc_end)) return 0u;
        const int64_t bit = tt * BN + c0;
        return __ldg(mrow + (bit >> 5)) >> (bit & 31);
      };
      uint32_t mq0 = mword_of(tc0), mq1 = mword_of(tc0 + 1), mq2 = mword_of(tc0 + 2);
      float* dst = p.Tpart + ((c + rb) * BM + row) * (int64_t)p.Kp;
      for (int64_t tc = tc0, jt = 0; u < seg_end; ++u, ++it, ++tc, ++jt) {
        const int xs = (int)(it % XS), b = (int)(it & (ND - 1)), yb = (int)(it & (NY - 1));
        const int64_t t0 = tc * BN;
        const uint32_t mword = mq0;
        mq0 = mq1;
        mq1 = mq2;
        mq2 = mword_of(tc + 3);
        const int64_t nc = p.P_strm - t0 - c0;  // valid columns for this warp
        const uint32_t vmask = (!row_ok || nc <= 0) ? 0u : (nc >= CPW ? CMASK : ((1u << nc) - 1u));
        // accumulators first: the TMEM loads are in flight while X is read from shared memory
        if (!pre_d && !mbar_wait(&d_full[b], (uint32_t)((it / ND) & 1), abort_flag)) { ok = false; break; }
        tc_fence_after();
        uint32_t rx[CPW], rd[CPW];
        tmem_issue<CPW>(tmem + lane_base + (uint32_t)(b * BN + c0), rx);
        if (PASS2) tmem_issue<CPW>(tmem + lane_base + (uint32_t)((ND + b) * BN + c0), rd);
        if (!pre_x && !mbar_wait(&x_full[xs], (uint32_t)((it / XS) & 1), abort_flag)) {
          if (PASS2) tmem_wait_x2<CPW>(rx, rd);
          else tmem_wait<CPW>(rx);
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
          const unsigned char* box = xt + (c0 >> 5) * (BM * 128) + row * 128;
          const int cb = (c0 & 31) >> 2;
#pragma unroll
          for (int c4 = 0; c4 < CPW / 4; ++c4) {
            const float4 v = *reinterpret_cast<const float4*>(box + (((cb + c4) ^ (row & 7)) << 4));
            xv[4 * c4 + 0] = v.x; xv[4 * c4 + 1] = v.y; xv[4 * c4 + 2] = v.z; xv[4 * c4 + 3] = v.w;
          }
        }
        mbar_arrive(&x_empty[xs]);
        // early probes: this tile's Y buffer, the next tile's accumulator and data tile
        const bool pre_y = !PASS2 && mbar_test(&y_empty[yb], (uint32_t)(((it / NY) & 1) ^ 1));
        pre_d = u + 1 < u_end && mbar_test(&d_full[(it + 1) & (ND - 1)], (uint32_t)(((it + 1) / ND) & 1));
        pre_x = u + 1 < u_end && mbar_test(&x_full[(it + 1) % XS], (uint32_t)(((it + 1) / XS) & 1));
        if (PASS2) tmem_wait_x2<CPW>(rx, rd);
        else tmem_wait<CPW>(rx);
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
        // BF16 pass 1: this thread's CPW weights as bytes, four per word (zero off the mask)
        constexpr bool WQ = !PASS2 && !TF32;
        uint32_t qw[WQ ? CPW / 4 : 1];
        // branch-free slot update (predicated selects keep the slots independent)
        if (FULL) {
          // exact statistics: sum w, sum e^2, sum w e^2 and a count of non-finite residuals
          uint32_t fin = 0;
          float wprev = 0.f;   // weight of the even slot of the current pair (WQ)
#pragma unroll
          for (int j = 0; j < CPW; ++j) {
            const float e = xv[j] - xh[j];
            const bool use = ((seen >> j) & 1u) && (fabsf(e) <= 3.402823466e38f);
            fin |= use ? (1u << j) : 0u;
            // selects, not products with 0, so that a NaN stored at an unobserved slot stays out
            const float eu = use ? e : 0.f;
            const float uw = use ? fast_ex2(e * e * nk) : 0.f;
            if constexpr (WQ) {
              if (j & 1) {
                const uint32_t t = quant_pair(wprev, uw);
                qw[j >> 2] = (j & 2) ? __byte_perm(qw[j >> 2], t, 0x5410) : t;
              } else {
                wprev = uw;
              }
            }
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
          // without further selects); pass 2 masks the weight.  w = exp2(e^2 k), as in the
          // full-statistics form.
#pragma unroll
          for (int j = 0; j < CPW; j += 2) {
            const bool b0 = (seen >> j) & 1u, b1 = (seen >> (j + 1)) & 1u;
            float2 e2 = __ffma2_rn(make_float2(xh[j], xh[j + 1]), neg1, make_float2(xv[j], xv[j + 1]));
            if (!PASS2) {
              e2.x = b0 ? e2.x : 0.f;
              e2.y = b1 ? e2.y : 0.f;
            }
            const float2 m2 = __fmul2_rn(__fmul2_rn(e2, e2), nk2);   // -e^2 log2(e) / (2 sigma^2)
            if (PASS2) {
              const float2 w2 = make_float2(b0 ? fast_ex2(m2.x) : 0.f, b1 ? fast_ex2(m2.y) : 0.f);
              const float2 d2 = make_float2(dh[j], dh[j + 1]);
              if ((j >> 1) & 1) acc2b = __ffma2_rn(__fmul2_rn(w2, d2), d2, acc2b);
              else acc2a = __ffma2_rn(__fmul2_rn(w2, d2), d2, acc2a);
            } else {
              const float2 w2 = make_float2(fast_ex2(m2.x), fast_ex2(m2.y));
              const float2 y2 = __fmul2_rn(w2, e2);
              if ((j >> 1) & 1) acc2b = __ffma2_rn(y2, e2, acc2b);
              else acc2a = __ffma2_rn(y2, e2, acc2a);
              xv[j] = y2.x;
              xv[j + 1] = y2.y;
              if constexpr (WQ) {
                const uint32_t t = quant_pair(b0 ? w2.x : 0.f, b1 ? w2.y : 0.f);
                qw[j >> 2] = (j & 2) ? __byte_perm(qw[j >> 2], t, 0x5410) : t;
              }
            }
          }
        }
        if constexpr (WQ) {
          // the unit's weight block: this thread's CPW bytes of row `row`, CPW / 16 chunks
          unsigned char* wb = p.wq + u * (int64_t)(BM * BN);
          if constexpr (CPW == 32) {
            // both chunks lie in one 32-byte sector (the chunk permutation only swaps them when
            // the row's XOR term is odd): one full-sector store; streaming (evict-first), so
            // that the cache written during the pass does not push the pass's own reusable
            // lines (operands, mask rows, tile edges) out of L2
            const int p0 = wq_chunk<BN>(row, c0 >> 4);
            const bool swap = (p0 >> 4) & 1;
            const uint32_t* a = swap ? qw + 4 : qw;
            const uint32_t* b2 = swap ? qw : qw + 4;
            asm volatile("st.global.cs.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(wb + (p0 & ~31)), "r"(a[0]),
                         "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b2[0]), "r"(b2[1]), "r"(b2[2]), "r"(b2[3])
                         : "memory");
          } else {
#pragma unroll
            for (int h = 0; h < CPW / 16; ++h)
              __stcs(reinterpret_cast<uint4*>(wb + wq_chunk<BN>(row, (c0 >> 4) + h)),
                     make_uint4(qw[4 * h], qw[4 * h + 1], qw[4 * h + 2], qw[4 * h + 3]));
          }
        }
        if (!PASS2) {
          if constexpr (TF32) {
            // 3-term split of Y for GEMM 2: hi = tf32(y), lo = tf32(y - hi)
            uint32_t yh[CPW], yl[CPW];
#pragma unroll
            for (int j = 0; j < CPW; ++j) {
              yh[j] = tf32_rna(xv[j]);
              yl[j] = tf32_rna(xv[j] - __uint_as_float(yh[j]));
            }
            if (!pre_y && !mbar_wait(&y_empty[yb], (uint32_t)(((it / NY) & 1) ^ 1), abort_flag)) { ok = false; break; }
            const uint32_t ycol = tmem + lane_base + col_y + (uint32_t)(yb * C::Y_COLS + c0);
            tmem_st<CPW>(ycol, yh);
            tmem_st<CPW>(ycol + (uint32_t)BN, yl);
          } else {
            uint32_t ypk[CPW / 2];
#pragma unroll
            for (int j = 0; j < CPW; j += 2) ypk[j >> 1] = pack_bf16(xv[j], xv[j + 1]);
            if (!pre_y && !mbar_wait(&y_empty[yb], (uint32_t)(((it / NY) & 1) ^ 1), abort_flag)) { ok = false; break; }
            // this warp's CPW residuals of row `row` -> CPW / 2 columns of Y buffer yb in TMEM
            tmem_st<CPW / 2>(tmem + lane_base + col_y + (uint32_t)(yb * C::Y_COLS + (c0 >> 1)), ypk);
          }
          tmem_wait_st();
          tc_fence_before();
          mbar_arrive(&y_full[yb]);
          if ((jt % C::CH) == C::CH - 1 || u + 1 == seg_end) {
            // the chunk's contraction is complete: this warp's columns of row `row` of T
            if (!mbar_wait(acc_full, (uint32_t)(ch & 1), abort_flag)) { ok = false; break; }
            tc_fence_after();
            if constexpr (CHUNKED) {
              float v[32];
              tmem_ld32(tmem + lane_base + col_acc + grp * KPW, v);
#pragma unroll
              for (int j = 0; j < 32; ++j) tacc[j] += v[j];
            } else {
              // one chunk per segment: straight to slot c + rb
#pragma unroll
              for (int h0 = 0; h0 < KPW; h0 += 32) {
                float v[32];
                tmem_ld32(tmem + lane_base + col_acc + grp * KPW + h0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                  if (grp * KPW + h0 + j < p.Kp) dst[grp * KPW + h0 + j] = row_ok ? v[j] : 0.f;
              }
            }
            tc_fence_before();
            mbar_arrive(acc_empty);
            ++ch;
          }
        }
      }
      if (!ok) break;
      if constexpr (CHUNKED) {
        // the segment's contraction, summed over its chunks -> slot c + rb
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (grp * KPW + j < p.Kp) dst[grp * KPW + j] = row_ok ? tacc[j] : 0.f;
          tacc[j] = 0.f;
        }
      }
    }
    if (!FULL) {
      const float lean = (acc2a.x + acc2b.x) + (acc2a.y + acc2b.y);
      if (PASS2) sden += lean;
      else swe2 += lean;
      nnf = (isfinite(swe2) && isfinite(sden)) ? 0u : 1u;
    }
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

// ------------------------------------------------------------------ line search from cached weights
// Pass 2 of the BF16 path after a BF16 pass 1 of the same core update: the exact line search's
// denominator den = sum w D2^2 (Sec. 3.2) with D2 = S_h S_str^T (one BF16 term, FP32 in TMEM)
// and w the weight pass 1 left in its unit-major cache (8-bit fixed point, w = q / 255; zero
// off the mask and outside the tensor).  Pass 1 computed these weights from the same residuals
// (the cores do not change between the passes), so this pass reads one byte per slot instead
// of the data tile and the mask, and runs neither the reconstruction GEMM nor the exponential.
// Units and their partition over the CTAs are those of pass 1 (any partition works: the cache
// is indexed by unit).  Units are handed between the roles in groups of two (one MMA, one
// commit, one weight copy and one accumulator buffer per group): every barrier wait costs about
// a hundred cycles even when its phase has completed, and per unit those waits bounded the pass.
// Roles: warp 0 operand producer (S_h per segment, S_str tiles), warp 1 TMEM allocator + MMA
// issuer, warps 2..9 epilogue (TMEM lane quarter = warp % 4, two column groups), warp 10 weight
// producer (one bulk copy per group).  Every wait is bounded.
template <int KP>
struct WCfg {
  static constexpr int BN = Cfg<KP, false, false>::BN;   // the streaming columns of pass 1's units
  static constexpr int GRP = KP == 64 ? 4 : 2;            // units per handoff (one MMA, one commit)
  static constexpr int GBN = GRP * BN;                    // columns of one group's accumulator
  static constexpr int NSUB = KP / 64;                    // 128-byte K sub-tiles per operand row
  static constexpr int KSTEPS = KP / 16;                  // MMAs of K = 16
  static constexpr int NGRP = 2;                          // column groups of the epilogue
  static constexpr int CPW = BN / NGRP;                   // columns of a unit per epilogue warp (32 or 16)
  static constexpr int EPIW = 4 * NGRP;                   // epilogue warps (4 TMEM lane quarters each)
  static constexpr int WT = BM * BN;                      // bytes of one unit's weights
  static constexpr int S_TILE = BM * KP * 2, T_TILE = BN * KP * 2;
  static constexpr int SUB_S = BM * 128, SUB_T = BN * 128;
  static constexpr int TSTAGE = GRP * T_TILE, WSTAGE = GRP * WT;
  static constexpr int ND = 512 / GBN < 4 ? 512 / GBN : 4;   // accumulator buffers (ND GBN <= 512 columns)
  static constexpr int TS = 3;
  static constexpr int WS = KP == 64 ? 3 : (KP == 128 ? 5 : 6);
  static constexpr int T0 = S_TILE, W0 = T0 + TS * TSTAGE, BARS = W0 + WS * WSTAGE, TOTAL = BARS + 1024;
  static constexpr int WPW = 2 + EPIW;                    // warp index of the weight producer
  static constexpr int NTH = 32 * (3 + EPIW);
};

// Units of a CTA's range are taken in groups of GRP consecutive units of one stationary block
// (the last group of a block may be shorter); every role walks the same group sequence.  The
// epilogue reads a group's accumulators two units at a time (register budget).
// Streaming-operand stage layout: K sub-tile sb of unit h at sb * GRP * SUB_T + h * SUB_T, so
// that the group's GBN rows of each sub-tile are contiguous (one MMA of N = g BN).
template <int KP>
__global__ void __launch_bounds__(WCfg<KP>::NTH, 1)
    k_pass_wls(const __grid_constant__ CUtensorMap mS_h, const __grid_constant__ CUtensorMap mT_hi, const Params p) {
  using C = WCfg<KP>;
  constexpr int BN = C::BN, GRP = C::GRP, GBN = C::GBN, CPW = C::CPW, NSUB = C::NSUB, KSTEPS = C::KSTEPS;
  constexpr int WT = C::WT, ND = C::ND, TS = C::TS, WS = C::WS, EPIW = C::EPIW;
  static_assert(C::TOTAL + 1024 <= SMEM_LIMIT, "shared memory");
  static_assert(CPW == 16 || CPW == 32, "one or two 16-byte weight chunks per epilogue thread");
  static_assert(ND * GBN <= 512, "TMEM columns");
  static_assert(GBN <= 256 && GBN % 16 == 0, "UMMA N");
  static_assert(GRP % 2 == 0, "the epilogue takes units in pairs");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (su32(smem_raw) & 1023)) & 1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::BARS);
  uint64_t* w_full = bars;                // [WS] a group's weight blocks landed
  uint64_t* w_empty = w_full + WS;        // [WS] weight blocks read by every epilogue thread
  uint64_t* t_full = w_empty + WS;        // [TS] a group's streaming operands landed
  uint64_t* t_empty = t_full + TS;        // [TS] streaming operands consumed (MMA commit)
  uint64_t* d_full = t_empty + TS;        // [ND] a group's D2 done
  uint64_t* d_empty = d_full + ND;        // [ND] D2 read by the epilogue
  uint64_t* s_full = d_empty + ND;        //      step operand landed
  uint64_t* s_empty = s_full + 1;         //      segment's MMAs done with it
  uint64_t* mma_done = s_empty + 1;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mma_done + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 2);
  double* red = reinterpret_cast<double*>(mma_done + 4);   // [EPIW epilogue warps]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = blockIdx.x;
  const int64_t u_begin = c * p.U / p.G, u_end = (c + 1) * p.U / p.G;
  if (threadIdx.x == 0) {
    for (int s = 0; s < WS; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&w_empty[s], 32 * EPIW);
    }
    for (int s = 0; s < TS; ++s) {
      mbar_init(&t_full[s], 1);
      mbar_init(&t_empty[s], 1);
    }
    for (int b = 0; b < ND; ++b) {
      mbar_init(&d_full[b], 1);
      mbar_init(&d_empty[b], 32 * EPIW);
    }
    mbar_init(s_full, 1);
    mbar_init(s_empty, 1);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)), "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();
  pdl_trigger();

  if (warp == 0) {
    // ---------------------------------------------------------------- operand producer
    if (lane == 0) {
      const uint64_t keep = policy_evict_last();
      int64_t it = 0;
      int sg = 0;
      bool ok = true;
      int last_phase[TS];
      for (int s = 0; s < TS; ++s) last_phase[s] = -1;
      int s_phase = -1;
      for (int64_t u = u_begin; u < u_end && ok; ++sg) {
        const int64_t rb = u / p.NT;
        const int64_t seg_end = imin(u_end, (rb + 1) * p.NT);
        if (sg > 0) ok = mbar_wait(s_empty, (uint32_t)((sg - 1) & 1), abort_flag);
        if (!ok) break;
        mbar_expect_tx(s_full, C::S_TILE);
        s_phase = sg & 1;
#pragma unroll
        for (int sb = 0; sb < NSUB; ++sb)
          tma_2d_hint(sm + sb * C::SUB_S, &mS_h, s_full, sb * 64, (int)(rb * BM), keep);
        for (; u < seg_end; ++it) {
          const int g = (int)imin(GRP, seg_end - u);
          const int64_t tc = u - rb * p.NT;
          const int s = (int)(it % TS);
          if (!mbar_wait(&t_empty[s], (uint32_t)(((it / TS) & 1) ^ 1), abort_flag)) { ok = false; break; }
          unsigned char* tb = sm + C::T0 + s * C::TSTAGE;
          mbar_expect_tx(&t_full[s], (uint32_t)(g * C::T_TILE));
          last_phase[s] = (int)((it / TS) & 1);
          for (int h = 0; h < g; ++h)
#pragma unroll
            for (int sb = 0; sb < NSUB; ++sb)
              tma_2d_hint(tb + sb * GRP * C::SUB_T + h * C::SUB_T, &mT_hi, &t_full[s], sb * 64, (int)((tc + h) * BN),
                          keep);
          u += g;
        }
      }
      if (!ok) {
        for (int s = 0; s < TS; ++s)
          if (last_phase[s] >= 0)
            for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
              if (mbar_try(&t_full[s], (uint32_t)last_phase[s])) break;
        if (s_phase >= 0)
          for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
            if (mbar_try(s_full, (uint32_t)s_phase)) break;
      }
    }
  } else if (warp == C::WPW) {
    // ---------------------------------------------------------------- weight producer
    if (lane == 0) {
      const uint64_t once = policy_evict_first();
      bool ok = true;
      int last_phase[WS];
      for (int s = 0; s < WS; ++s) last_phase[s] = -1;
      int64_t it = 0;
      for (int64_t u = u_begin; u < u_end && ok;) {
        const int64_t seg_end = imin(u_end, (u / p.NT + 1) * p.NT);
        for (; u < seg_end; ++it) {
          const int g = (int)imin(GRP, seg_end - u);
          const int s = (int)(it % WS);
          if (!mbar_wait(&w_empty[s], (uint32_t)(((it / WS) & 1) ^ 1), abort_flag)) { ok = false; break; }
          mbar_expect_tx(&w_full[s], (uint32_t)(g * WT));
          last_phase[s] = (int)((it / WS) & 1);
          // the group's units are consecutive, so are their weight blocks
          bulk_g2s(sm + C::W0 + s * C::WSTAGE, p.wq + u * (int64_t)WT, (uint32_t)(g * WT), &w_full[s], once);
          u += g;
        }
      }
      if (!ok)
        for (int s = 0; s < WS; ++s)
          if (last_phase[s] >= 0)
            for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
              if (mbar_try(&w_full[s], (uint32_t)last_phase[s])) break;
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint64_t dA = sdesc(su32(sm));
      int64_t it = 0;
      int sg = 0;
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok; ++sg) {
        const int64_t seg_end = imin(u_end, (u / p.NT + 1) * p.NT);
        if (!mbar_wait(s_full, (uint32_t)(sg & 1), abort_flag)) { ok = false; break; }
        for (; u < seg_end; ++it) {
          const int g = (int)imin(GRP, seg_end - u);
          const int s = (int)(it % TS), b = (int)(it & (ND - 1));
          if (!mbar_wait(&t_full[s], (uint32_t)((it / TS) & 1), abort_flag)) { ok = false; break; }
          if (!mbar_wait(&d_empty[b], (uint32_t)(((it / ND) & 1) ^ 1), abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint64_t dB = sdesc(su32(sm + C::T0 + s * C::TSTAGE));
          const uint32_t id = idesc_mma(BM, g * BN, false);   // N = g BN
#pragma unroll
          for (int kk = 0; kk < KSTEPS; ++kk) {
            const uint64_t ka = (uint64_t)(((kk >> 2) * C::SUB_S + (kk & 3) * 32) >> 4);
            const uint64_t kb = (uint64_t)(((kk >> 2) * GRP * C::SUB_T + (kk & 3) * 32) >> 4);
            tc_mma<false>(tmem + (uint32_t)(b * GBN), dA + ka, dB + kb, id, kk > 0);
          }
          tc_commit(&d_full[b]);
          tc_commit(&t_empty[s]);
          u += g;
        }
        if (!ok) break;
        tc_commit(s_empty);
      }
      tc_commit(mma_done);
      for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try(mma_done, 0)) break;
    }
  } else if (warp >= 2 && warp < C::WPW) {
    // ---------------------------------------------------------------- epilogue
    const int q = warp & 3, grp = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int c0 = grp * CPW;
    float2 acc2a = make_float2(0.f, 0.f), acc2b = make_float2(0.f, 0.f);
    const float2 off = make_float2(-8388608.f, -8388608.f);
    int64_t it = 0;
    bool ok = true;
    for (int64_t u = u_begin; u < u_end && ok;) {
      const int64_t seg_end = imin(u_end, (u / p.NT + 1) * p.NT);
      for (; u < seg_end; ++it) {
        const int g = (int)imin(GRP, seg_end - u);
        const int b = (int)(it & (ND - 1)), ws = (int)(it % WS);
        // the warp leaves together when a wait gives up (the TMEM loads are warp-wide)
        if (!__all_sync(0xffffffffu, mbar_wait(&d_full[b], (uint32_t)((it / ND) & 1), abort_flag))) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t rd[2][CPW];
        tmem_issue<CPW>(tmem + lane_base + (uint32_t)(b * GBN + c0), rd[0]);
        if (g > 1) tmem_issue<CPW>(tmem + lane_base + (uint32_t)(b * GBN + BN + c0), rd[1]);
        if (!__all_sync(0xffffffffu, mbar_wait(&w_full[ws], (uint32_t)((it / WS) & 1), abort_flag))) {
          tmem_wait<CPW>(rd[0]);
          if (g > 1) tmem_wait<CPW>(rd[1]);
          ok = false;
          break;
        }
        const unsigned char* wt = sm + C::W0 + ws * C::WSTAGE;
        uint32_t wv[GRP][CPW / 4];
#pragma unroll
        for (int h = 0; h < GRP; ++h) {
          if (h < g) {
#pragma unroll
            for (int m = 0; m < CPW / 16; ++m) {
              const uint4 v = *reinterpret_cast<const uint4*>(wt + h * WT + wq_chunk<BN>(row, (c0 >> 4) + m));
              wv[h][4 * m] = v.x;
              wv[h][4 * m + 1] = v.y;
              wv[h][4 * m + 2] = v.z;
              wv[h][4 * m + 3] = v.w;
            }
          }
        }
        mbar_arrive(&w_empty[ws]);
#pragma unroll
        for (int h0 = 0; h0 < GRP; h0 += 2) {
          if (h0 >= g) break;
          if (h0 > 0) {
            // the next pair of this group's accumulators
            tmem_issue<CPW>(tmem + lane_base + (uint32_t)(b * GBN + h0 * BN + c0), rd[0]);
            if (h0 + 1 < g) tmem_issue<CPW>(tmem + lane_base + (uint32_t)(b * GBN + (h0 + 1) * BN + c0), rd[1]);
          }
          tmem_wait<CPW>(rd[0]);
          if (h0 + 1 < g) tmem_wait<CPW>(rd[1]);
          if (h0 + 2 >= g) {
            // every accumulator of the group is in registers: release the buffer to the MMA
            tc_fence_before();
            mbar_arrive(&d_empty[b]);
          }
          // den += q D2^2 (the factor 1 / 255 is applied once at the end); byte k of a word ->
          // the float 2^23 + q (exponent byte 0x4B above it), minus 2^23, exactly
#pragma unroll
          for (int h1 = 0; h1 < 2; ++h1) {
            if (h0 + h1 < g) {
#pragma unroll
              for (int j = 0; j < CPW; j += 2) {
                const uint32_t wd = wv[h0 + h1][j >> 2];
                const uint32_t sel = (uint32_t)(j & 3);
                const float2 w2 =
                    __fadd2_rn(make_float2(__uint_as_float(__byte_perm(wd, 0x4B000000u, 0x7540u | sel)),
                                           __uint_as_float(__byte_perm(wd, 0x4B000000u, 0x7540u | (sel + 1)))),
                               off);
                const float2 d2 = make_float2(__uint_as_float(rd[h1][j]), __uint_as_float(rd[h1][j + 1]));
                if ((j >> 1) & 1) acc2b = __ffma2_rn(__fmul2_rn(w2, d2), d2, acc2b);
                else acc2a = __ffma2_rn(__fmul2_rn(w2, d2), d2, acc2a);
              }
            }
          }
        }
        u += g;
      }
    }
    double den = (double)((acc2a.x + acc2b.x) + (acc2a.y + acc2b.y)) * (1.0 / 255.0);
    for (int o = 16; o > 0; o >>= 1) den += __shfl_down_sync(0xffffffffu, den, o);
    if (lane == 0) red[warp - 2] = den;
  }
  // ------------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    double den = 0.0;
    for (int w = 0; w < EPIW; ++w) den += red[w];
    if (p.nf_in && !(*p.nf_in == 0.0)) den = __longlong_as_double(0x7ff8000000000000ll);
    for (int f = 0; f < 8; ++f) p.stat_part[c * 8 + f] = 0.0;
    p.stat_part[c * 8 + 4] = isfinite(den) ? 0.0 : 1.0;   // non-finite count (0 or 1)
    p.stat_part[c * 8 + 6] = den;
    if (*abort_flag) atomicOr(p.err, (int)DEV_TIMEOUT);
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// ------------------------------------------------------------------ host side
// Tiled 2-D tensor map (cuTensorMapEncodeTiled through the runtime's driver entry point).
bool make_map(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
              uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw);

// TF32 variants (KP = 64 or 128), instantiated in pass_tc_tf32.cu.
cudaError_t launch_pass_tc_tf32(int kpad, bool rows_case, bool pass2, bool full_stats, const PassOperands& o,
                                const float* X, int64_t P_in, int64_t ldx, int64_t P_out, Params p, int G,
                                cudaStream_t st);

// Launch one fused pass of contraction width KP with operands of kind TF32 (fp32 arrays holding
// TF32-rounded hi/lo splits) or BF16.  S operands: [P_stat][KP]; streaming: [P_strm][KP];
// X: P_out rows of P_in floats, row stride ldx (a multiple of 4); p carries the rest (its
// block and tile counts are filled in here).
template <int KP, bool TF32>
cudaError_t launch_pass_tc_kp(bool rows_case, bool pass2, bool full_stats, const PassOperands& o, const float* X,
                              int64_t P_in, int64_t ldx, int64_t P_out, Params p, int G, cudaStream_t st) {
  using C1 = Cfg<KP, TF32, false>;
  using C2 = Cfg<KP, TF32, true>;
  constexpr int ESZ = C1::ESZ, SUBW = C1::SUBW, BN = C1::BN;
  const CUtensorMapDataType DT = TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const CUtensorMapSwizzle SW = CU_TENSOR_MAP_SWIZZLE_128B;
  CUtensorMap mS_hi, mS_lo, mS_h, mT_hi, mT_lo, mX, mTT_hi, mTT_lo;
  // operand arrays [rows][KP], fetched as K sub-tiles of one 128-byte swizzle row
  bool ok = make_map(&mS_hi, DT, o.S_hi, KP, p.P_stat, (uint64_t)KP * ESZ, SUBW, BM, SW) &&
            make_map(&mS_lo, DT, o.S_lo, KP, p.P_stat, (uint64_t)KP * ESZ, SUBW, BM, SW) &&
            make_map(&mS_h, DT, (pass2 && C2::SH_SMEM) ? o.S_h : o.S_hi, KP, p.P_stat, (uint64_t)KP * ESZ, SUBW,
                     BM, SW) &&
            make_map(&mT_hi, DT, o.T_hi, KP, p.P_strm, (uint64_t)KP * ESZ, SUBW, BN, SW) &&
            make_map(&mT_lo, DT, o.T_lo, KP, p.P_strm, (uint64_t)KP * ESZ, SUBW, BN, SW);
  if (TF32 && !pass2) {
    // transposed streaming operand [KP][ldT] (TF32 pass 1), fetched as KP rows of BN columns
    if (!o.T_hiT || !o.T_loT || o.ldT < p.P_strm || (o.ldT % 4) != 0) return cudaErrorInvalidValue;
    ok = ok && make_map(&mTT_hi, DT, o.T_hiT, p.P_strm, KP, (uint64_t)o.ldT * 4, BN, KP, SW) &&
         make_map(&mTT_lo, DT, o.T_loT, p.P_strm, KP, (uint64_t)o.ldT * 4, BN, KP, SW);
  } else {
    mTT_hi = mT_hi;
    mTT_lo = mT_lo;
  }
  if (rows_case)
    ok = ok && make_map(&mX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, P_in, P_out, ldx * 4, BM, BN,
                        CU_TENSOR_MAP_SWIZZLE_NONE);
  else
    ok = ok && make_map(&mX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, P_in, P_out, ldx * 4, 32, BM, SW);
  if (!ok) return cudaErrorInvalidValue;
  p.RB = (p.P_stat + BM - 1) / BM;
  p.NT = (p.P_strm + BN - 1) / BN;
  p.U = p.RB * p.NT;
  p.G = (int)imin(G, p.U);
  p.shw[0] = p.shw[1] = nullptr;
  p.sh_off[0] = p.sh_off[1] = 0;
  p.sh_ld = 0;
  if (pass2 && C2::SH_TMEM) {
    if (!o.S_h || (TF32 && !o.S_h_lo)) return cudaErrorInvalidValue;
    if (TF32) {
      // group 0 copies the hi split, group 1 the lo split (KP words per row each)
      p.shw[0] = static_cast<const uint32_t*>(o.S_h);
      p.shw[1] = static_cast<const uint32_t*>(o.S_h_lo);
      p.sh_ld = KP;
    } else {
      // BF16 pairs: KP / 2 words per row, each group copies half of them
      p.shw[0] = p.shw[1] = static_cast<const uint32_t*>(o.S_h);
      p.sh_off[1] = KP / 4;
      p.sh_ld = KP / 2;
    }
  }
  auto go = [&](auto kern, int smem_bytes) {
    const size_t smem = (size_t)smem_bytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = pdl_launch(kern, dim3(p.G), dim3(NTHREADS), smem, st, mS_hi, mS_lo, mS_h, mT_hi, mT_lo, mX, mTT_hi, mTT_lo, p);
    if (e != cudaSuccess) return e;
    note_launch();
    return cudaGetLastError();
  };
  constexpr int SM1 = layout<C1>().total, SM2 = layout<C2>().total;
  if (pass2)
    return rows_case ? go(k_pass_tc<true, true, false, KP, TF32>, SM2) : go(k_pass_tc<false, true, false, KP, TF32>, SM2);
  if (full_stats)
    return rows_case ? go(k_pass_tc<true, false, true, KP, TF32>, SM1) : go(k_pass_tc<false, false, true, KP, TF32>, SM1);
  return rows_case ? go(k_pass_tc<true, false, false, KP, TF32>, SM1) : go(k_pass_tc<false, false, false, KP, TF32>, SM1);
}

// Launch the line-search pass from cached weights (BF16 operands [rows][KP]: S_h over the
// stationary rows, the hi split of the streaming operand).
template <int KP>
cudaError_t launch_pass_wls_kp(const void* S_h, const void* T_hi, const unsigned char* wq, int64_t P_stat,
                               int64_t P_strm, double* stat_part, int* err, int G, const double* nf_in,
                               cudaStream_t st) {
  using C = WCfg<KP>;
  CUtensorMap mS_h, mT_hi;
  const CUtensorMapSwizzle SW = CU_TENSOR_MAP_SWIZZLE_128B;
  if (!make_map(&mS_h, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, S_h, KP, P_stat, (uint64_t)KP * 2, 64, BM, SW) ||
      !make_map(&mT_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, T_hi, KP, P_strm, (uint64_t)KP * 2, 64, C::BN, SW))
    return cudaErrorInvalidValue;
  Params p{};
  p.P_stat = P_stat;
  p.P_strm = P_strm;
  p.RB = (P_stat + BM - 1) / BM;
  p.NT = (P_strm + C::BN - 1) / C::BN;
  p.U = p.RB * p.NT;
  p.G = (int)imin(G, p.U);
  p.stat_part = stat_part;
  p.err = err;
  p.wq = const_cast<unsigned char*>(wq);
  p.nf_in = nf_in;
  const size_t smem = (size_t)C::TOTAL + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_pass_wls<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = pdl_launch(k_pass_wls<KP>, dim3(p.G), dim3(C::NTH), smem, st, mS_h, mT_hi, p);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace trd
