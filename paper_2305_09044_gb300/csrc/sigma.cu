// Adaptive kernel width (the paper cites a rule without stating it; reading):
//   sigma = max(1e-6 rms(x_obs), 2 min(std(e), IQR(e) / 1.349), 0.9 sigma_prev)
// over the observed residuals of the full tensor, or of a fixed probe of 2^20 entries.
// Quartiles are type-7 (linear interpolation between order statistics); the order
// statistics come from an exact, deterministic MSB-first radix select on order-preserving
// 64-bit keys (8 passes of 8 bits, integer histograms).
#include <algorithm>
#include <mutex>
#include <vector>

#include <type_traits>

#include "trd_internal.cuh"

namespace trd {

namespace {

__host__ __device__ inline uint64_t sm64(uint64_t seed, uint64_t m) {
  uint64_t z = seed + (m + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ inline uint64_t dkey(double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
// dkey((double)f) for a finite float, from the bits alone (no FP64 instruction): the double
// has the float's sign, the exponent rebiased by 1023 - 127 and the fraction shifted up by 29;
// a subnormal float is normalised first.
__device__ inline uint64_t fkey(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sgn = (uint64_t)(u >> 31) << 63;
  const uint32_t E = (u >> 23) & 0xffu, M = u & 0x7fffffu;
  uint64_t b;
  if (E != 0) {
    b = sgn | ((uint64_t)(E + 896u) << 52) | ((uint64_t)M << 29);
  } else if (M == 0) {
    b = sgn;
  } else {
    const int p = 31 - __clz((int)M);          // leading bit: value = 1.x * 2^(p - 149)
    b = sgn | ((uint64_t)(p + 874) << 52) | (((uint64_t)M << (52 - p)) & 0xfffffffffffffull);
  }
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double dval(uint64_t k) {
  const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

constexpr uint64_t kExcluded = ~0ull;

// ------------------------------------------------------------------ selection chain
// Work area (8-byte words):
//   [0] n (included residuals)  [1] mean  [2] sum x^2  [3] population variance
//   u[8..11]  remaining rank of each of the four target order statistics
//   u[12..15] key prefix selected so far for each target
//   u[16..23] completion counter of each kernel of the chain
//   u[24]     number of candidates appended by the compaction
//   word 64:  uint32 histograms [8 digits][4 targets][256]
//   word 64 + 4096: per-block partial sums [kSelBlocks][4] (count, sum e, sum x^2, sum e^2)
// The chain is: clear (memset) -> first kernel (residual keys, sums, digit-0 histogram) ->
// digit 1 -> digit 2 (the last block of each kernel, found by a completion counter, turns the
// complete histogram into the next digit of each target) -> compaction of the keys still
// matching a target's 24-bit prefix -> one block for digits 3..7 and sigma.
constexpr int kSelBlocks = 1216;
constexpr int kSelThreads = 256;
constexpr int kHistWord = 64;
constexpr int kPartsWord = 64 + 4096;

__device__ __forceinline__ unsigned int* sel_hist(double* work, int digit, int t) {
  return reinterpret_cast<unsigned int*>(work + kHistWord) + (digit * 4 + t) * 256;
}

// Signals completion of this block; true in the block that completes last (which then sees
// every other block's global writes and atomics).
__device__ bool sel_last_block(double* work, int kernel) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(work) + 16 + kernel;
    s_last = atomicAdd(ctr, 1ull) == (unsigned long long)gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Targets whose prefixes coincide share one histogram: alias[t] = first such target.
__device__ __forceinline__ void sel_alias(const uint64_t* pre, int* alias) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    alias[t] = t;
    for (int q = t - 1; q >= 0; --q)
      if (pre[q] == pre[t]) alias[t] = q;
  }
}

// Last block, warps 0..3 (one per target): inclusive scan of the 256 counts of the target's
// histogram (8 bins per lane), find the bin holding the remaining rank, narrow the prefix.
__device__ void sel_pick(double* work, int digit) {
  uint64_t* u = reinterpret_cast<uint64_t*>(work);
  const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t pre[4];
  int alias[4];
  for (int q = 0; q < 4; ++q) pre[q] = __ldcg(u + 12 + q);
  sel_alias(pre, alias);
  __syncthreads();                       // every warp has read the prefixes before any update
  if (t < 4) {
    const unsigned int* h = sel_hist(work, digit, digit == 0 ? 0 : alias[t]);
    const uint64_t rank = __ldcg(u + 8 + t);
    unsigned int c[8];
    unsigned long long loc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      c[i] = __ldcg(h + lane * 8 + i);
      loc += c[i];
    }
    unsigned long long incl = loc;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned long long excl = incl - loc;
    if (rank >= excl && rank < incl) {
      unsigned long long cum = excl;
      int bin = lane * 8 + 7;
      for (int i = 0; i < 8; ++i) {
        if (cum + c[i] > rank) { bin = lane * 8 + i; break; }
        cum += c[i];
      }
      const int shift = 56 - 8 * digit;
      u[8 + t] = rank - cum;
      u[12 + t] = pre[t] | ((uint64_t)bin << shift);
    }
  }
  __syncthreads();
}

// Fixed-order sum of field f of the per-block partials (last block; result in every thread).
__device__ double sel_sum_parts(const double* work, int f, int nb) {
  __shared__ double red[kSelThreads / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(work + kPartsWord + b * 4 + f);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// Per-element step of the first kernel: key, partial sums, digit-0 histogram (warp-aggregated
// shared-memory atomics).  Every lane of the warp calls it (valid = false for lanes without
// an included residual).
__device__ __forceinline__ void sel_consume(bool valid, double e, double x2, uint64_t* keys, int64_t m,
                                            bool write, unsigned int* h0, double& c, double& se, double& sx,
                                            double& s2) {
  const uint64_t key = valid ? dkey(e) : kExcluded;
  if (write) keys[m] = key;
  if (valid) {
    c += 1.0;
    se += e;
    sx += x2;
    s2 = fma(e, e, s2);
  }
  const unsigned dig = (unsigned)(key >> 56);
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  if (valid) {
    const unsigned peers = __match_any_sync(act, dig);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h0[dig], (unsigned)__popc(peers));
  }
}

// sel_consume for FP32 residuals: the same key (fkey) and histogram, the lane's count and sums
// kept in integer / FP32 registers (a lane takes a handful of probes) and widened once at the
// end, so the per-probe work issues no FP64 instruction.
__device__ __forceinline__ void sel_consume_f(bool valid, float e, float x2, uint64_t* keys, int64_t m,
                                              bool write, unsigned int* h0, uint32_t& c, float& se, float& sx,
                                              float& s2) {
  const uint64_t key = valid ? fkey(e) : kExcluded;
  if (write) keys[m] = key;
  if (valid) {
    c += 1u;
    se += e;
    sx += x2;
    s2 = fmaf(e, e, s2);
  }
  const unsigned dig = (unsigned)(key >> 56);
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  if (valid) {
    const unsigned peers = __match_any_sync(act, dig);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h0[dig], (unsigned)__popc(peers));
  }
}

// End of the first kernel: block partials and histogram out; the last block sets n, mean,
// sum x^2, the target ranks, and picks digit 0.
__device__ void sel_first_finish(double* work, unsigned int* h0, double c, double se, double sx, double s2) {
  __shared__ double red[4][kSelThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, o);
    se += __shfl_down_sync(0xffffffffu, se, o);
    sx += __shfl_down_sync(0xffffffffu, sx, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = c;
    red[1][threadIdx.x >> 5] = se;
    red[2][threadIdx.x >> 5] = sx;
    red[3][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, d = 0, q = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; d += red[2][w]; q += red[3][w]; }
    double* part = work + kPartsWord + blockIdx.x * 4;
    part[0] = a;
    part[1] = b;
    part[2] = d;
    part[3] = q;
  }
  unsigned int* g0 = sel_hist(work, 0, 0);
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h0[i]) atomicAdd(&g0[i], h0[i]);
  if (!sel_last_block(work, 0)) return;
  const double n = sel_sum_parts(work, 0, gridDim.x);
  const double sum = sel_sum_parts(work, 1, gridDim.x);
  const double sx2 = sel_sum_parts(work, 2, gridDim.x);
  const double se2 = sel_sum_parts(work, 3, gridDim.x);
  if (threadIdx.x == 0) {
    const double mean = n > 0 ? sum / n : 0.0;
    work[0] = n;
    work[1] = mean;
    work[2] = sx2;
    // population variance in one pass (the residual mean is small against their spread)
    work[3] = n > 0 ? fmax(0.0, se2 / n - mean * mean) : 0.0;
    uint64_t* u = reinterpret_cast<uint64_t*>(work);
    const double ps[2] = {0.25, 0.75};
    for (int q = 0; q < 2; ++q) {
      double hq = (n - 1.0) * ps[q];
      if (hq < 0) hq = 0;
      const double lo = floor(hq);
      const double hi = lo + 1.0 <= n - 1.0 ? lo + 1.0 : lo;
      u[8 + 2 * q] = (uint64_t)lo;
      u[9 + 2 * q] = (uint64_t)hi;
    }
    for (int t = 0; t < 4; ++t) u[12 + t] = 0;
  }
  __syncthreads();
  sel_pick(work, 0);
}

// sigma = max(1e-6 rms, 2 min(std, IQR / 1.349), 0.9 sigma_prev) from the selected keys (type-7
// quartiles with numpy's interpolation form) and the sums.
__device__ void sel_sigma(const double* work, double rms_override, double sigma_prev,
                          const double* __restrict__ sigma_prev_dev, double* __restrict__ sigma_out) {
  if (sigma_prev_dev) sigma_prev = *sigma_prev_dev;
  // L2 reads (ld.global.cg): these words were written earlier in this kernel
  const uint64_t* u = reinterpret_cast<const uint64_t*>(work);
  const double n = __ldcg(work);
  double q[2];
  const double ps[2] = {0.25, 0.75};
  for (int i = 0; i < 2; ++i) {
    const double a = dval(__ldcg(u + 12 + 2 * i)), b = dval(__ldcg(u + 13 + 2 * i));
    double h = (n - 1.0) * ps[i];
    if (h < 0) h = 0;
    const double f = h - floor(h);
    q[i] = f >= 0.5 ? b - (b - a) * (1.0 - f) : a + (b - a) * f;
  }
  const double stdv = sqrt(__ldcg(work + 3));
  const double rms = rms_override >= 0 ? rms_override : (n > 0 ? sqrt(__ldcg(work + 2) / n) : 0.0);
  double s = 2.0 * fmin(stdv, (q[1] - q[0]) / 1.349);
  if (!(n > 0)) s = 0.0;
  s = fmax(s, 1e-6 * rms);
  if (sigma_prev > 0 && isfinite(sigma_prev)) s = fmax(s, 0.9 * sigma_prev);
  *sigma_out = s;
}

// Digit d (1 or 2) of the four targets: histogram of the keys that match each target's
// prefix (digit 1 also accumulates sum (e - mean)^2); the last block picks the digit.  Each
// warp takes chunks of 32 x kSelBatch consecutive keys, all loads issued before use.
constexpr int kSelBatch = 8;

__global__ void __launch_bounds__(kSelThreads) k_sel_digit(const uint64_t* __restrict__ keys, int64_t n,
                                                           double* __restrict__ work, int digit) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned int h[4][256];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&h[0][0])[i] = 0;
  const uint64_t* u = reinterpret_cast<const uint64_t*>(work);
  uint64_t pre[4];
  int alias[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) pre[t] = __ldcg(u + 12 + t);
  sel_alias(pre, alias);
  const int shift = 56 - 8 * digit;
  const uint64_t himask = ~0ull << (shift + 8);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t chunk = 32 * kSelBatch;
  for (int64_t c0 = ((int64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * chunk; c0 < n;
       c0 += (int64_t)gridDim.x * wpb * chunk) {
    uint64_t kb[kSelBatch];
#pragma unroll
    for (int q = 0; q < kSelBatch; ++q) {
      const int64_t m = c0 + q * 32 + lane;
      kb[q] = m < n ? keys[m] : kExcluded;
    }
#pragma unroll
    for (int q = 0; q < kSelBatch; ++q) {
      const uint64_t k = kb[q];
      const bool valid = k != kExcluded;
      const unsigned dig = (unsigned)((k >> shift) & 0xffu);
      // the distinct prefixes of one digit are disjoint, so a key counts for at most one
      // target: one aggregated histogram update per key
      int tk = -1;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (alias[t] == t && valid && (k & himask) == pre[t]) tk = t;
      const unsigned act = __ballot_sync(0xffffffffu, tk >= 0);
      if (tk >= 0) {
        const unsigned peers = __match_any_sync(act, (unsigned)tk << 8 | dig);
        if (lane == __ffs(peers) - 1) atomicAdd(&h[tk][dig], (unsigned)__popc(peers));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (alias[t] != t) continue;
    unsigned int* g = sel_hist(work, digit, t);
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
      if (h[t][i]) atomicAdd(&g[i], h[t][i]);
  }
  if (!sel_last_block(work, digit)) return;
  sel_pick(work, digit);
}

// After three digits: the keys that still match a target's 24-bit prefix (a small fraction)
// are appended to cand[] (warp-aggregated atomic count in u[24]; their order is irrelevant).
__global__ void __launch_bounds__(kSelThreads) k_sel_compact(const uint64_t* __restrict__ keys, int64_t n,
                                                             double* __restrict__ work, uint64_t* __restrict__ cand) {
  pdl_wait();
  pdl_trigger();
  uint64_t* u = reinterpret_cast<uint64_t*>(work);
  uint64_t pre[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) pre[t] = __ldcg(u + 12 + t);
  const uint64_t himask = ~0ull << 40;
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t chunk = 32 * kSelBatch;
  for (int64_t c0 = ((int64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * chunk; c0 < n;
       c0 += (int64_t)gridDim.x * wpb * chunk) {
    uint64_t kb[kSelBatch];
#pragma unroll
    for (int q = 0; q < kSelBatch; ++q) {
      const int64_t m = c0 + q * 32 + lane;
      kb[q] = m < n ? keys[m] : kExcluded;
    }
#pragma unroll
    for (int q = 0; q < kSelBatch; ++q) {
      const uint64_t k = kb[q];
      const uint64_t hk = k & himask;
      const bool hit = k != kExcluded && (hk == pre[0] || hk == pre[1] || hk == pre[2] || hk == pre[3]);
      const unsigned act = __ballot_sync(0xffffffffu, hit);
      if (act) {
        unsigned long long base = 0;
        if (lane == __ffs(act) - 1) base = atomicAdd(reinterpret_cast<unsigned long long*>(u + 24), (unsigned long long)__popc(act));
        base = __shfl_sync(0xffffffffu, base, __ffs(act) - 1);
        if (hit) cand[base + __popc(act & ((1u << lane) - 1u))] = k;
      }
    }
  }
}

// One block: digits 3..7 over the candidates (shared-memory histograms), then sigma.
constexpr int kFinThreads = 1024;
__global__ void __launch_bounds__(kFinThreads) k_sel_finish(const uint64_t* __restrict__ cand, double* __restrict__ work,
                                                            double rms_override, double sigma_prev,
                                                            const double* __restrict__ sigma_prev_dev,
                                                            double* __restrict__ sigma_out) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned int h[4][256];
  __shared__ uint64_t s_pre[4], s_rank[4];
  uint64_t* u = reinterpret_cast<uint64_t*>(work);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 4) {
    s_pre[tid] = __ldcg(u + 12 + tid);
    s_rank[tid] = __ldcg(u + 8 + tid);
  }
  const int64_t cnt = (int64_t)__ldcg(u + 24);
  __syncthreads();
  for (int digit = 3; digit < 8; ++digit) {
    for (int i = tid; i < 1024; i += blockDim.x) (&h[0][0])[i] = 0;
    uint64_t pre[4];
    int alias[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) pre[t] = s_pre[t];
    sel_alias(pre, alias);
    const int shift = 56 - 8 * digit;
    const uint64_t himask = ~0ull << (shift + 8);
    __syncthreads();
    for (int64_t c0 = (int64_t)warp * 32; c0 < cnt; c0 += blockDim.x) {
      const int64_t c = c0 + lane;
      const uint64_t k = c < cnt ? __ldcg(cand + c) : kExcluded;
      const bool valid = k != kExcluded;
      const unsigned dig = (unsigned)((k >> shift) & 0xffu);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (alias[t] != t) continue;
        const bool hit = valid && (k & himask) == pre[t];
        const unsigned act = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const unsigned peers = __match_any_sync(act, dig);
          if (lane == __ffs(peers) - 1) atomicAdd(&h[t][dig], (unsigned)__popc(peers));
        }
      }
    }
    __syncthreads();
    if (warp < 4) {
      const int t = warp;
      const unsigned int* ht = h[alias[t]];
      const uint64_t rank = s_rank[t];
      unsigned int cb[8];
      unsigned long long loc = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        cb[i] = ht[lane * 8 + i];
        loc += cb[i];
      }
      unsigned long long incl = loc;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const unsigned long long excl = incl - loc;
      if (rank >= excl && rank < incl) {
        unsigned long long cum = excl;
        int bin = lane * 8 + 7;
        for (int i = 0; i < 8; ++i) {
          if (cum + cb[i] > rank) { bin = lane * 8 + i; break; }
          cum += cb[i];
        }
        s_rank[t] = rank - cum;
        s_pre[t] = pre[t] | ((uint64_t)bin << shift);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int t = 0; t < 4; ++t) {
      u[8 + t] = s_rank[t];
      u[12 + t] = s_pre[t];
    }
    sel_sigma(work, rms_override, sigma_prev, sigma_prev_dev, sigma_out);
  }
}

// First kernel on given residuals (floats): keys, sums, digit-0 histogram.
__global__ void __launch_bounds__(kSelThreads) k_sel_floats(const float* __restrict__ r, int64_t n,
                                                            uint64_t* __restrict__ keys, double* __restrict__ work) {
  __shared__ unsigned int h0[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h0[i] = 0;
  __syncthreads();
  double c = 0, se = 0, sx = 0, s2 = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); m0 < n; m0 += stride) {
    const int64_t m = m0 + (threadIdx.x & 31);
    const double v = m < n ? (double)r[m] : 0.0;
    const bool valid = m < n && isfinite(v);
    sel_consume(valid, v, 0.0, keys, m, m < n, h0, c, se, sx, s2);
  }
  __syncthreads();
  sel_first_finish(work, h0, c, se, sx, s2);
}

// First kernel of the tensor rule: residuals at the probe entries from the merged subchains
// of the full tensor, x_hat = sum_kappa A[a][kappa] C[b][kappa] (Thm. 1 with the ring cut in two).
// One lane per probe (probe m is described by pa[m] (inner index, -1 when unobserved), pb[m]
// and px[m]); each lane streams its two rows in chunks of 8 values with all loads of a chunk
// issued before its FMAs.  Used when Kp is not a multiple of the 16-byte vector width.
template <typename T>
__global__ void __launch_bounds__(kSelThreads)
    k_sel_probe(const T* __restrict__ A, const T* __restrict__ C, int Kp, const int32_t* __restrict__ pa,
                const int32_t* __restrict__ pb, const float* __restrict__ px, int64_t n,
                uint64_t* __restrict__ keys, double* __restrict__ work) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned int h0[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h0[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  double c = 0, se = 0, sx = 0, s2 = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); m0 < n; m0 += stride) {
    const int64_t m = m0 + lane;
    const bool live = m < n;
    const int32_t a = live ? pa[m] : -1;
    const bool obs = a >= 0;
    const int32_t bi = obs ? pb[m] : 0;
    const float xf = obs ? px[m] : 0.f;
    T p0 = T(0), p1 = T(0);
    if (obs) {
      const T* Ar = A + (int64_t)a * Kp;
      const T* Cr = C + (int64_t)bi * Kp;
      for (int k0 = 0; k0 < Kp; k0 += 8) {
        T xa[8], xc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const bool in = k0 + q < Kp;
          xa[q] = in ? Ar[k0 + q] : T(0);
          xc[q] = in ? Cr[k0 + q] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
          p0 = fma(xa[q], xc[q], p0);
          p1 = fma(xa[q + 1], xc[q + 1], p1);
        }
      }
    }
    double e = 0.0, x2 = 0.0;
    bool valid = false;
    if (obs) {
      const T x = (T)xf;
      const T et = x - (p0 + p1);
      valid = isfinite((double)et);
      e = (double)et;
      x2 = (double)x * (double)x;
    }
    sel_consume(valid, e, x2, keys, m, live, h0, c, se, sx, s2);
  }
  __syncthreads();
  sel_first_finish(work, h0, c, se, sx, s2);
}

// Eight lanes per probe: four probes per step of a warp, each probe's two merged rows read by
// its eight lanes with 16-byte loads (one 128-byte line per probe and load instruction, so the
// loads stay coalesced), a three-level shuffle tree per probe, and one shuffle that hands the
// sum to the lane owning the probe (the warp takes its 32 probes m0 + j in eight steps; lane j
// ends up holding the reconstruction of probe j).  A sixteen-lane form with four probes in
// flight per lane executed 28 warp instructions per probe (measured), most of them index
// shuffles and shuffle trees; this one about a third of that.  Needs Kp a multiple of
// 16 / sizeof(T).
template <typename T>
__global__ void __launch_bounds__(kSelThreads)
    k_sel_probe16(const T* __restrict__ A, const T* __restrict__ C, int Kp, const int32_t* __restrict__ pa,
                  const int32_t* __restrict__ pb, const float* __restrict__ px, int64_t n,
                  uint64_t* __restrict__ keys, double* __restrict__ work) {
  pdl_wait();
  pdl_trigger();
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int VW = 16 / sizeof(T);
  __shared__ unsigned int h0[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h0[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 3, sub = lane & 7;
  const int nv = Kp / VW;
  double c = 0, se = 0, sx = 0, s2 = 0;
  uint32_t cf = 0;
  float sef = 0.f, sxf = 0.f, s2f = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); m0 < n; m0 += stride) {
    const int64_t m = m0 + lane;
    const bool live = m < n;
    const int32_t a = live ? pa[m] : -1;
    const bool obs = a >= 0;
    const int32_t bi = obs ? pb[m] : 0;
    const float xf = obs ? px[m] : 0.f;
    T mine = T(0);
#pragma unroll
    for (int st = 0; st < 8; ++st) {
      // probe st * 4 + g of the warp's 32
      const int32_t ap = __shfl_sync(0xffffffffu, a, st * 4 + g);
      const int32_t bp = __shfl_sync(0xffffffffu, bi, st * 4 + g);
      T acc = T(0);
      if (ap >= 0) {
        const V* ra = reinterpret_cast<const V*>(A + (int64_t)ap * Kp);
        const V* rc = reinterpret_cast<const V*>(C + (int64_t)bp * Kp);
        for (int v = sub; v < nv; v += 8) {
          const V xa = ra[v], xc = rc[v];
          if constexpr (VW == 4) {
            acc = fma(xa.x, xc.x, acc);
            acc = fma(xa.y, xc.y, acc);
            acc = fma(xa.z, xc.z, acc);
            acc = fma(xa.w, xc.w, acc);
          } else {
            acc = fma(xa.x, xc.x, acc);
            acc = fma(xa.y, xc.y, acc);
          }
        }
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      // lane j's probe is computed at step j / 4 by the eight lanes of group j % 4
      const T t = __shfl_sync(0xffffffffu, acc, (lane & 3) * 8);
      if (st == (lane >> 2)) mine = t;
    }
    if constexpr (VW == 4) {
      float e = 0.f, x2 = 0.f;
      bool valid = false;
      if (obs) {
        e = xf - mine;
        valid = isfinite(e);
        x2 = xf * xf;
      }
      sel_consume_f(valid, e, x2, keys, m, live, h0, cf, sef, sxf, s2f);
    } else {
      double e = 0.0, x2 = 0.0;
      bool valid = false;
      if (obs) {
        const T x = (T)xf;
        const T et = x - mine;
        valid = isfinite((double)et);
        e = (double)et;
        x2 = (double)x * (double)x;
      }
      sel_consume(valid, e, x2, keys, m, live, h0, c, se, sx, s2);
    }
  }
  if constexpr (VW == 4) {
    c = (double)cf;
    se = (double)sef;
    sx = (double)sxf;
    s2 = (double)s2f;
  }
  __syncthreads();
  sel_first_finish(work, h0, c, se, sx, s2);
}

// Probe description for the tensor rule: probe m is the entry lin[m] (all entries in order
// when numel <= 2^20, else the SplitMix64(0x5eed, m) mod numel positions sorted ascending, so
// that neighbouring probes share merged rows), split as lin = a + P_in b; pa = -1 when
// unobserved.
__global__ void k_probe_setup(const float* __restrict__ X, const uint32_t* __restrict__ M, const int64_t* __restrict__ lin_in,
                              int64_t n, int64_t P_in, int32_t* __restrict__ pa, int32_t* __restrict__ pb,
                              float* __restrict__ px) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lin = lin_in ? lin_in[m] : m;
    const bool obs = M ? ((M[lin >> 5] >> (lin & 31)) & 1u) : true;
    int64_t a;
    const int64_t b = qdivmod(lin, P_in, a);
    pa[m] = obs ? (int32_t)a : -1;
    pb[m] = (int32_t)b;
    px[m] = X[lin];
  }
}

cudaError_t run_digits(const uint64_t* keys, int64_t n, double* work, uint64_t* cand, double rms_override,
                       double sigma_prev, const double* sigma_prev_dev, double* sigma_out, cudaStream_t st) {
  const int nb = (int)imax(1, imin(kSelBlocks, (n + 32 * kSelBatch * 8 - 1) / (32 * kSelBatch * 8)));
  pdl_launch(k_sel_digit, dim3(nb), dim3(kSelThreads), 0, st, keys, n, work, 1);
  note_launch();
  pdl_launch(k_sel_digit, dim3(nb), dim3(kSelThreads), 0, st, keys, n, work, 2);
  note_launch();
  pdl_launch(k_sel_compact, dim3(nb), dim3(kSelThreads), 0, st, keys, n, work, cand);
  note_launch();
  pdl_launch(k_sel_finish, dim3(1), dim3(kFinThreads), 0, st, cand, work, rms_override, sigma_prev, sigma_prev_dev,
             sigma_out);
  note_launch();
  return cudaGetLastError();
}

int sel_blocks(int64_t n) { return (int)imax(1, imin(kSelBlocks, (n + 4 * kSelThreads - 1) / (4 * kSelThreads))); }

}  // namespace

size_t sigma_work_doubles() { return (size_t)kPartsWord + (size_t)kSelBlocks * 4; }

void probe_positions(int64_t numel, std::vector<int64_t>& lin) {
  const int64_t n = numel <= kProbeMax ? numel : kProbeMax;
  lin.resize((size_t)n);
  if (numel <= kProbeMax) {
    for (int64_t m = 0; m < n; ++m) lin[(size_t)m] = m;
    return;
  }
  for (int64_t m = 0; m < n; ++m) lin[(size_t)m] = (int64_t)(sm64(kProbeSeed, (uint64_t)m) % (uint64_t)numel);
  std::sort(lin.begin(), lin.end());
}

cudaError_t launch_probe_setup(const float* X, const uint32_t* M, const int64_t* lin_dev, int64_t n, int64_t P_in,
                               int32_t* pa, int32_t* pb, float* px, cudaStream_t st) {
  k_probe_setup<<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(X, M, lin_dev, n, P_in, pa, pb, px);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_probe_sigma_merged(const void* A, const void* C, bool fp64, int Kp, const int32_t* pa,
                                      const int32_t* pb, const float* px, int64_t n, double sigma_prev,
                                      const double* sigma_prev_dev, uint64_t* keys, uint64_t* cand, double* work,
                                      double* sigma_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(double) * kPartsWord, st);
  if (e != cudaSuccess) return e;
  // one lane per probe, a few probes per lane
  const int nb = (int)imax(1, imin(kSelBlocks, (n + 2 * kSelThreads - 1) / (2 * kSelThreads)));
  if (fp64 && Kp % 2 == 0)
    pdl_launch(k_sel_probe16<double>, dim3(nb), dim3(kSelThreads), 0, st, (const double*)A, (const double*)C, Kp, pa,
               pb, px, n, keys, work);
  else if (fp64)
    pdl_launch(k_sel_probe<double>, dim3(nb), dim3(kSelThreads), 0, st, (const double*)A, (const double*)C, Kp, pa,
               pb, px, n, keys, work);
  else if (Kp % 4 == 0)
    pdl_launch(k_sel_probe16<float>, dim3(nb), dim3(kSelThreads), 0, st, (const float*)A, (const float*)C, Kp, pa, pb,
               px, n, keys, work);
  else
    pdl_launch(k_sel_probe<float>, dim3(nb), dim3(kSelThreads), 0, st, (const float*)A, (const float*)C, Kp, pa, pb,
               px, n, keys, work);
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return run_digits(keys, n, work, cand, -1.0, sigma_prev, sigma_prev_dev, sigma_out, st);
}

cudaError_t launch_sigma_from_floats(const float* r, int64_t n, double x_obs_rms, double sigma_prev, uint64_t* keys,
                                     uint64_t* cand, double* work, double* sigma_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(double) * kPartsWord, st);
  if (e != cudaSuccess) return e;
  const int nb = sel_blocks(n);
  k_sel_floats<<<nb, kSelThreads, 0, st>>>(r, n, keys, work);
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return run_digits(keys, n, work, cand, x_obs_rms, sigma_prev, nullptr, sigma_out, st);
}

// ------------------------------------------------------------------ allocation-free variant
// Fixed scratch for trd_sigma_from_residuals_noalloc: room for the order keys of NOALLOC_MAX
// residuals and as many selection candidates (8 bytes each) plus the selection work area.
// It is a file-scope device array, so every GPU that loads the library holds it (about
// 16.8 MB) until the process exits; all calls share it.
constexpr int64_t NOALLOC_MAX = int64_t(1) << 20;
constexpr size_t NOALLOC_WORK = kPartsWord + kSelBlocks * 4;   // doubles; equals sigma_work_doubles()
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_MAX * 16 + NOALLOC_WORK * 8];

namespace {
constexpr int NOALLOC_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_DEVICES] = {};   // device address of the scratch, per device ordinal
}  // namespace

}  // namespace trd

extern "C" trd_status trd_sigma_from_residuals_noalloc(const float* resid_dev, int64_t n, double x_obs_rms,
                                                       double sigma_prev, double* sigma_out_dev,
                                                       void* cuda_stream) {
  using namespace trd;
  if (!resid_dev || !sigma_out_dev || n < 1 || n > NOALLOC_MAX || !(x_obs_rms >= 0.0)) return TRD_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TRD_ECUDA;
  }
  if (dev < 0 || dev >= NOALLOC_DEVICES) return TRD_EINVAL;
  void* base = nullptr;
  {
    // one-time set-up per device (with that device current): the host-side name of the array
    // is not a device address, so ask the runtime for the device address of this copy
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return TRD_ECUDA;
      }
      g_noalloc_addr[dev] = ptr;
    }
    base = g_noalloc_addr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  uint64_t* keys = reinterpret_cast<uint64_t*>(b);
  uint64_t* cand = reinterpret_cast<uint64_t*>(b + NOALLOC_MAX * 8);
  double* work = reinterpret_cast<double*>(b + NOALLOC_MAX * 16);
  // every scratch word the selection reads is written first in this call (the counters and
  // histograms are cleared at its start), so stale contents do not leak in
  const cudaError_t e = launch_sigma_from_floats(resid_dev, n, x_obs_rms, sigma_prev, keys, cand, work,
                                                 sigma_out_dev, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TRD_ECUDA;
  }
  return TRD_OK;
}
