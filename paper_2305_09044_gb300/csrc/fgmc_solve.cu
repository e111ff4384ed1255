// FGMC Gram chain (Prop. 2), regularised Cholesky solve of the scaled gradient (Eq. sg /
// Eq. hI), exact line-search step (Sec. 3.2), core update (Eq. updatessd) and the stopping
// quantity of Algorithm 1.  Everything here is FP64 and small (K = r_k r_{k+1} <= 1024).
#include "trd_internal.cuh"

namespace trd {

// ------------------------------------------------------------------ FGMC factor
// E[(a r + a'), (b r1 + b')] = sum_{i in sel} Z(i)[a, b] Z(i)[a', b']  (= sum Z(i) (x) Z(i)),
// Z(i)[a, b] at i*K + b*r + a.  sel = idx[0..n) or 0..n-1 when idx is null.  Slices are
// staged through shared memory in chunks of 32; each thread owns output entries.
__global__ void k_fgmc_E(const double* __restrict__ Z, const int32_t* __restrict__ idx, int64_t n_all,
                         int r, int r1, int CH, double* __restrict__ E) {
  pdl_wait();
  pdl_trigger();
  // slice range of this block row (gridDim.y parts, contiguous)
  const int64_t per = (n_all + gridDim.y - 1) / gridDim.y;
  const int64_t qb = (int64_t)blockIdx.y * per;
  const int64_t n = imax(0, imin(n_all, qb + per) - qb);
  if (idx) idx += qb;
  Z += idx ? 0 : qb * (int64_t)(r * r1);
  extern __shared__ double zs[];
  const int rows = r * r, cols = r1 * r1, K = r * r1;
  const int64_t tot = (int64_t)rows * cols;
  const int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = e0 < tot;
  int o1 = 0, o2 = 0;
  if (active) {
    const int row = (int)(e0 / cols), col = (int)(e0 % cols);
    const int a = row / r, a2 = row % r, b = col / r1, b2 = col % r1;
    o1 = b * r + a;
    o2 = b2 * r + a2;
  }
  double s = 0.0;
  for (int64_t q0 = 0; q0 < n; q0 += CH) {
    const int cnt = (int)imin(CH, n - q0);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * K; e += blockDim.x) {
      const int qq = e / K, kk = e % K;
      const int64_t i = idx ? (int64_t)idx[q0 + qq] : q0 + qq;
      zs[e] = Z[i * K + kk];
    }
    __syncthreads();
    if (active)
      for (int qq = 0; qq < cnt; ++qq) s = fma(zs[qq * K + o1], zs[qq * K + o2], s);
  }
  if (active) E[(int64_t)blockIdx.y * tot + e0] = s;
}

__global__ void k_sum_parts(const double* __restrict__ part, int parts, int64_t n, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < parts; ++q) s += part[(int64_t)q * n + i];
    out[i] = s;
  }
}

// The same factor for large K = r r1 (all slices, no index list), as the realigned Gram of the
// slice matrix: with Z viewed as an I x K row-major matrix (row i = Z(i), column x = b r + a),
// P = Z^T Z is K x K and E[(a r + a'), (b r1 + b')] = P[b r + a, b' r + a'].  P is symmetric, so
// only its 32 x 32 tiles on and below the diagonal are formed (tile pair q -> (tp, tq), tq <= tp),
// each written to both of its places in E.  The slice range is split over gridDim.y parts so
// that the I K^2 / 2 FMAs spread over all SMs; part p writes out[p * tot ...] (summed after, in
// part order: the result does not depend on scheduling).  256 threads, 2 x 2 outputs each.
__global__ void __launch_bounds__(256) k_fgmc_E_gram(const double* __restrict__ Z, int64_t n_all, int r, int r1,
                                                     double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  constexpr int T = 32, CH = 32;
  __shared__ double sa[CH][T + 1], sb[CH][T + 1];
  const int K = r * r1;
  const int64_t tot = (int64_t)K * K;
  const int q = blockIdx.x;
  int tp = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
  while ((tp + 1) * (tp + 2) / 2 <= q) ++tp;
  while (tp * (tp + 1) / 2 > q) --tp;
  const int tq = q - tp * (tp + 1) / 2;
  const int x0 = tp * T, y0 = tq * T;
  const int64_t per = (n_all + gridDim.y - 1) / gridDim.y;
  const int64_t i0 = (int64_t)blockIdx.y * per;
  const int64_t i1 = imin(n_all, i0 + per);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t c0 = i0; c0 < i1; c0 += CH) {
    const int cnt = (int)imin(CH, i1 - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < CH * T; e += 256) {
      const int ii = e >> 5, cc = e & 31;
      const bool ok = ii < cnt;
      sa[ii][cc] = ok && x0 + cc < K ? Z[(c0 + ii) * K + x0 + cc] : 0.0;
      sb[ii][cc] = ok && y0 + cc < K ? Z[(c0 + ii) * K + y0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int ii = 0; ii < CH; ++ii) {
      const double a0 = sa[ii][ty], a1 = sa[ii][ty + 16];
      const double b0 = sb[ii][tx], b1 = sb[ii][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
  }
  double* o = out + (int64_t)blockIdx.y * tot;
  const int cols = r1 * r1;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int x = x0 + ty + 16 * u, y = y0 + tx + 16 * v;
      if (x >= K || y >= K || (tp == tq && y > x)) continue;
      const int a = x % r, b = x / r, a2 = y % r, b2 = y / r;
      o[(int64_t)(a * r + a2) * cols + (b * r1 + b2)] = acc[u][v];
      if (x != y) o[(int64_t)(a2 * r + a) * cols + (b2 * r1 + b)] = acc[u][v];
    }
}

cudaError_t launch_fgmc_E(const double* Z, const int32_t* idx, int64_t n, int rk, int rk1,
                          double* E, double* work, cudaStream_t st) {
  const int64_t tot = (int64_t)rk * rk * rk1 * rk1;
  if (!idx && work && rk * rk1 > kLdlKmax) {
    const int nt = (rk * rk1 + 31) / 32, pairs = nt * (nt + 1) / 2;
    const int parts = (int)imax(1, imin(imin(16, (n + 63) / 64), (2 * 152 + pairs - 1) / pairs));
    pdl_launch(k_fgmc_E_gram, dim3((unsigned)pairs, (unsigned)parts), dim3(256), 0, st, Z, n, rk, rk1,
               parts > 1 ? work : E);
    note_launch();
    if (parts == 1) return cudaGetLastError();
    pdl_launch(k_sum_parts, dim3((unsigned)imin((tot + 255) / 256, 4096)), dim3(256), 0, st, work, parts, tot, E);
    note_launch();
    return cudaGetLastError();
  }
  const unsigned blocks = (unsigned)((tot + 127) / 128);
  // enough slice parts to cover the SMs; partial factors go to `work` ([parts][tot])
  int parts = (int)imax(1, imin(imin(n / 8, 16), (2 * 152 + blocks - 1) / blocks));
  if (!work) parts = 1;
  const int K = rk * rk1;
  const int CH = (int)imax(1, imin(32, (160 * 1024) / (K * 8)));
  const size_t smem = (size_t)CH * K * sizeof(double);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_fgmc_E, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(blocks, (unsigned)parts);
  pdl_launch(k_fgmc_E, dim3(grid), dim3(128), smem, st, Z, idx, n, rk, rk1, CH, parts > 1 ? work : E);
  note_launch();
  if (parts == 1) return cudaGetLastError();
  pdl_launch(k_sum_parts, dim3((unsigned)imin((tot + 255) / 256, 4096)), dim3(256), 0, st, work, parts, tot, E);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 GEMM (small)
// C[M x N] = A[M x K] * B, B is K x N (transB = 0) or N x K (transB = 1); all row-major.
// C = A B (or A B^T), FP64, 8 x 8 output tile per 64-thread block: the products here are
// small (K <= 400), so spreading them over many SMs matters more than operand reuse (GB300's
// FP64 issue rate per SM is low).
__global__ void k_dgemm(const double* __restrict__ A, const double* __restrict__ B,
                        double* __restrict__ C, int M, int N, int K, int transB) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sA[8][9], sB[8][9];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * 8 + ty, col = blockIdx.x * 8 + tx;
  // four independent accumulators keep the dependent FP64 FMA chain short
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < K; k0 += 8) {
    sA[ty][tx] = (row < M && k0 + tx < K) ? A[(int64_t)row * K + k0 + tx] : 0.0;
    const int bk = k0 + ty, bn = blockIdx.x * 8 + tx;
    double bv = 0.0;
    if (bk < K && bn < N) bv = transB ? B[(int64_t)bn * K + bk] : B[(int64_t)bk * N + bn];
    sB[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k & 3] = fma(sA[ty][k], sB[k][tx], acc[k & 3]);
    __syncthreads();
  }
  if (row < M && col < N) C[(int64_t)row * N + col] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

cudaError_t launch_dgemm(const double* A, const double* B, double* C, int M, int N, int K,
                         bool transB, cudaStream_t st) {
  dim3 grid((N + 7) / 8, (M + 7) / 8), block(8, 8);
  pdl_launch(k_dgemm, dim3(grid), dim3(block), 0, st, A, B, C, M, N, K, transB ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ realignment Phi
// G[a + b q, a' + b' q] = T[b p + b', a q + a'] for the subchain with p x q slices
// (p = r_{k+1}, q = r_k); T is p^2 x q^2 row-major.
__global__ void k_phi(const double* __restrict__ T, int p, int q, double* __restrict__ G) {
  pdl_wait();
  pdl_trigger();
  const int K = p * q;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x) {
    const int r = e / K, c = e % K;
    const int a = r % q, b = r / q, a2 = c % q, b2 = c / q;
    G[e] = T[(int64_t)(b * p + b2) * (q * q) + a * q + a2];
  }
}

cudaError_t launch_phi(const double* T, int p, int q, double* G, cudaStream_t st) {
  const int K = p * q;
  pdl_launch(k_phi, dim3((K * K + 255) / 256), dim3(256), 0, st, T, p, q, G);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ LDL^T of G + lambda I
// FP64 throughout.  GB300 issues FP64 FMAs at about 1.6 per clock per SM with a dependent
// latency near 70 clocks, so the factorisation is organised to keep every FP64 instruction
// useful and the per-column critical path short:
//  * one CTA; the lower triangle lives in registers, element e of the order "columns right
//    to left, rows top to bottom" held by thread e % 256 -- the trailing part still active at
//    column j is a prefix of that order, so every step is spread evenly over all threads;
//  * no square roots (LDL^T), one reciprocal per pivot;
//  * per column: update (one FMA per active element, the next pivot column first), publish
//    the next column, one warp forms its reciprocal and scaled column, two barriers.

// 1/p from the hardware's approximate FP64 reciprocal r0 (rcp.approx.ftz.f64) and one step of
// the cubic iteration for the reciprocal (Newton's iteration extended to third order): with
// e = 1 - p r0, 1/p = r0 / (1 - e) = r0 (1 + e + e^2 + O(e^3)).  The seed's relative error is
// far below 2^-18, so e^3 is below FP64 rounding.  Outside [1e-300, 1e300] the exact division
// is used (flush-to-zero seed).
__device__ __forceinline__ double recip_fp64(double p) {
  if (!(p > 1e-300 && p < 1e300)) return 1.0 / p;
  double r0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(p));
  const double e = fma(-p, r0, 1.0);
  return fma(r0, fma(e, e, e), r0);
}

constexpr int LDL_NT = 256;

// Pivot step for column j (one warp): reciprocal of the pivot, scaled column
// l_i = c_i / p (i > j) into s_l and into the column-major factor Lcm[j][i], D^{-1} entry;
// flags a non-positive or non-finite pivot.
__device__ __forceinline__ void ldl_pivot(int j, int K, const double* __restrict__ c, double* __restrict__ l,
                                          double* __restrict__ Lcm, double* __restrict__ Dinv, int* s_bad,
                                          int lane) {
  const double p = c[j];
  const bool bad = !(p > 0.0) || !isfinite(p);
  const double r = bad ? 0.0 : recip_fp64(p);
  for (int i = j + 1 + lane; i < K; i += 32) {
    const double v = c[i] * r;
    l[i] = v;
    Lcm[(int64_t)j * K + i] = v;
  }
  if (lane == 0) {
    Dinv[j] = r;
    if (bad) *s_bad = 1;
  }
}

// S = register slots per thread: K (K + 1) / 2 <= 256 S.
template <int S>
__global__ void __launch_bounds__(LDL_NT, 1)
    k_ldl_factor(const double* __restrict__ G, int K, double lam_in, double* __restrict__ Lcm,
                 double* __restrict__ Dinv, double* __restrict__ scal, int* __restrict__ dstatus) {
  pdl_wait();
  pdl_trigger();
  __shared__ double s_c[2][kLdlKmax];
  __shared__ double s_l[2][kLdlKmax];
  __shared__ double s_red[LDL_NT / 32];
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wbase = tid & ~31;
  double tr = 0.0;
  for (int i = tid; i < K; i += LDL_NT) tr += G[(int64_t)i * K + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
  if (lane == 0) s_red[warp] = tr;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  double trace = 0.0;
#pragma unroll
  for (int w = 0; w < LDL_NT / 32; ++w) trace += s_red[w];
  const double lam = lam_in >= 0 ? lam_in : -lam_in * trace / K;
  if (tid == 0) scal[5] = lam;

  // this thread's elements (i, m), i >= m, packed as i | m << 16; unused slots hold (0, 0),
  // which is never updated or published
  const int nel = K * (K + 1) / 2;
  double w[S];
  uint32_t im[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = tid + s * LDL_NT;
    w[s] = 0.0;
    im[s] = 0u;
    if (e < nel) {
      int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while ((q + 1) * (q + 2) / 2 <= e) ++q;
      while (q * (q + 1) / 2 > e) --q;
      const int m = K - 1 - q, i = m + (e - q * (q + 1) / 2);
      w[s] = G[(int64_t)i * K + m] + (i == m ? lam : 0.0);
      im[s] = (uint32_t)i | ((uint32_t)m << 16);
      if (m == 0) s_c[0][i] = w[s];
    }
  }
  __syncthreads();
  if (warp == 0) ldl_pivot(0, K, s_c[0], s_l[0], Lcm, Dinv, &s_bad, lane);
  __syncthreads();
  for (int j = 0; j + 1 < K; ++j) {
    if (s_bad) break;                       // uniform: read after a barrier
    const double* cj = s_c[j & 1];
    const double* lj = s_l[j & 1];
    double* cn = s_c[(j + 1) & 1];
    // active elements (columns > j) are the first nact of the order; a slot whose whole warp
    // lies beyond them is skipped (warp-uniform), so no FP64 instruction is spent on it.
    // Loads first, then the independent FMAs, then the publication of column j + 1.
    // The warp's active slots are a prefix s < s_end; the loops leave by a (warp-uniform)
    // branch so that no FP64 instruction is even issued for a retired slot.
    const int nact = (K - 1 - j) * (K - j) / 2;
    const int s_end = nact > wbase ? imin(S, (nact - wbase + LDL_NT - 1) / LDL_NT) : 0;
    double li[S], cm[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (s >= s_end) break;
      const int i = (int)(im[s] & 0xFFFFu), m = (int)(im[s] >> 16);
      const bool act = m > j;
      li[s] = act ? lj[i] : 0.0;
      cm[s] = act ? cj[m] : 0.0;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (s >= s_end) break;
      w[s] = fma(-li[s], cm[s], w[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (s >= s_end) break;
      if ((int)(im[s] >> 16) == j + 1) cn[im[s] & 0xFFFFu] = w[s];
    }
    __syncthreads();
    if (warp == 0) ldl_pivot(j + 1, K, cn, s_l[(j + 1) & 1], Lcm, Dinv, &s_bad, lane);
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicOr(dstatus, (int)DEV_SINGULAR);
}

// h = d (L D L^T)^{-1}, one warp per row of d (I_k x K, row-major): v L^T = d (forward),
// u = v D^{-1}, h L = u (backward), both in column-oriented form (the finished unknown is
// broadcast by a shuffle and subtracted from the rest).  The factor is staged in shared
// memory by asynchronous copies (column-major, padded column stride KP + 1 so that columns
// and rows are both read without bank conflicts); only entries below the diagonal are used.
// C = ceil(K / 32) entries per lane.
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}

// One row per warp, LDL_SW warps per block sharing one staged L.  One warp per block (so per
// SM) measured fastest: the substitutions are bound by the SM's FP64 issue rate, and rows
// spread over SMs get the most of it.
constexpr int LDL_SW = 1;
template <int C>
__global__ void __launch_bounds__(32 * LDL_SW) k_ldl_solve(const double* __restrict__ Lcm, const double* __restrict__ Dinv,
                                                  const double* __restrict__ d, double* __restrict__ h, int K,
                                                  int64_t rows, double* __restrict__ dot_part,
                                                  unsigned int* __restrict__ ctr, double* __restrict__ num) {
  constexpr int KP = 32 * C, LD = KP + 1;
  extern __shared__ double sL[];          // [K][LD]: sL[j * LD + i] = L[i][j]
  double* sD = sL + (size_t)K * LD;       // [KP]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < K * KP; e += blockDim.x) {
    const int j = e / KP, i = e - j * KP;
    if (i < K) cp_async8(sL + j * LD + i, Lcm + (int64_t)j * K + i);
  }
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
  for (int i = threadIdx.x; i < KP; i += blockDim.x) sD[i] = i < K ? Dinv[i] : 0.0;
  __syncthreads();
  for (int64_t row = (int64_t)blockIdx.x * LDL_SW + w; row < rows; row += (int64_t)gridDim.x * LDL_SW) {
    const double* dr = d + row * K;
    double s[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int i = c * 32 + lane;
      s[c] = i < K ? dr[i] : 0.0;
    }
    // forward: v_j final at step j; v_i -= L[i][j] v_j for i > j
#pragma unroll
    for (int cc = 0; cc < C; ++cc) {
      const int jend = imin(K, cc * 32 + 32);
      for (int j = cc * 32; j < jend; ++j) {
        const double v = __shfl_sync(0xffffffffu, s[cc], j & 31);
        const double* col = sL + j * LD;
#pragma unroll
        for (int c = cc; c < C; ++c) {
          const int i = c * 32 + lane;
          const double l = (i > j && i < K) ? col[i] : 0.0;
          s[c] = fma(-l, v, s[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) s[c] *= sD[c * 32 + lane];
    // backward: h_j final at step j (descending); h_i -= L[j][i] h_j for i < j
#pragma unroll
    for (int cc = C - 1; cc >= 0; --cc) {
      const int jtop = imin(K, cc * 32 + 32) - 1;
      for (int j = jtop; j >= cc * 32; --j) {
        const double v = __shfl_sync(0xffffffffu, s[cc], j & 31);
#pragma unroll
        for (int c = 0; c <= cc; ++c) {
          const int i = c * 32 + lane;
          const double l = i < j ? sL[i * LD + j] : 0.0;
          s[c] = fma(-l, v, s[c]);
        }
      }
    }
    double* hr = h + row * K;
    double dh = 0.0;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int i = c * 32 + lane;
      if (i < K) {
        hr[i] = s[c];
        dh = fma(dr[i], s[c], dh);
      }
    }
    for (int o = 16; o > 0; o >>= 1) dh += __shfl_xor_sync(0xffffffffu, dh, o);
    if (lane == 0) dot_part[row] = dh;
  }
  // <d, h>: the block that finishes last adds the per-row parts in row order and resets the
  // completion counter for the next call
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last || w != 0) return;
  __threadfence();
  double t = 0.0;
  for (int64_t r = lane; r < rows; r += 32) t += __ldcg(dot_part + r);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (lane == 0) {
    *num = t;
    *ctr = 0u;
  }
}

cudaError_t launch_ldl_factor(const double* G, int K, double lambda, double* Lcm, double* Dinv, double* scal,
                              int* dstatus, cudaStream_t st) {
  if (K < 1 || K > kLdlKmax) return cudaErrorInvalidValue;
  const int nel = K * (K + 1) / 2;
  if (nel <= 9 * LDL_NT)
    pdl_launch(k_ldl_factor<9>, dim3(1), dim3(LDL_NT), 0, st, G, K, lambda, Lcm, Dinv, scal, dstatus);
  else if (nel <= 20 * LDL_NT)
    pdl_launch(k_ldl_factor<20>, dim3(1), dim3(LDL_NT), 0, st, G, K, lambda, Lcm, Dinv, scal, dstatus);
  else
    pdl_launch(k_ldl_factor<33>, dim3(1), dim3(LDL_NT), 0, st, G, K, lambda, Lcm, Dinv, scal, dstatus);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ldl_solve(const double* Lcm, const double* Dinv, const double* d, double* h, int K, int64_t rows,
                             double* dot_part, unsigned int* ctr, double* num, cudaStream_t st) {
  if (K < 1 || K > kLdlKmax || rows < 1) return rows == 0 ? cudaSuccess : cudaErrorInvalidValue;
  const int C = (K + 31) / 32;
  const size_t smem = ((size_t)K * (32 * C + 1) + 32 * C) * sizeof(double);
  // one warp per row of d, LDL_SW rows per block (rows beyond the grid share blocks)
  const unsigned blocks = (unsigned)imin((rows + LDL_SW - 1) / LDL_SW, 65535);
  void (*kern)(const double*, const double*, const double*, double*, int, int64_t, double*, unsigned int*,
               double*) =
      C == 1 ? k_ldl_solve<1> : C == 2 ? k_ldl_solve<2> : C == 3 ? k_ldl_solve<3> : k_ldl_solve<4>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<blocks, 32 * LDL_SW, smem, st>>>(Lcm, Dinv, d, h, K, rows, dot_part, ctr, num);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ explicit inverse, K <= 128
// Minv = (L D L^T)^{-1} from the factor: the row substitutions above applied to the identity
// (Minv is symmetric, so its rows are its columns).  The paths whose per-step contract is 1e-5
// or looser form it on the side stream while the data pass runs; their h = d Minv then costs
// one parallel row-times-matrix product instead of 2 K dependent substitution steps per row.
__global__ void k_identity(double* __restrict__ I, int K) {
  pdl_wait();
  pdl_trigger();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x)
    I[e] = (e / K == e % K) ? 1.0 : 0.0;
}

cudaError_t launch_identity(double* I, int K, cudaStream_t st) {
  pdl_launch(k_identity, dim3((unsigned)((K * K + 255) / 256)), dim3(256), 0, st, I, K);
  note_launch();
  return cudaGetLastError();
}

// h = d Minv for rows of d (I_k x K, row-major), one block per row: thread (j, q) sums the
// terms i of part q (contiguous, ascending) of h_j, the parts are added in q order; <d, h> as
// in k_ldl_solve (per-row parts, the last block adds them in row order and resets the counter).
constexpr int INV_NT = 256;
__global__ void __launch_bounds__(INV_NT) k_inv_rows(const double* __restrict__ Minv, const double* __restrict__ d,
                                                     double* __restrict__ h, int K, int Kpad, int64_t rows,
                                                     double* __restrict__ dot_part, unsigned int* __restrict__ ctr,
                                                     double* __restrict__ num) {
  __shared__ double sd[kLdlKmax];
  __shared__ double part[INV_NT];
  __shared__ double sdot[INV_NT / 32];
  __shared__ int s_last;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int Q = INV_NT / Kpad, j = t % Kpad, q = t / Kpad;
  const int i0 = q * K / Q, i1 = (q + 1) * K / Q;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const double* dr = d + row * K;
    for (int i = t; i < K; i += INV_NT) sd[i] = dr[i];
    __syncthreads();
    double a0 = 0.0, a1 = 0.0;
    if (j < K) {
      int i = i0;
      for (; i + 1 < i1; i += 2) {
        a0 = fma(sd[i], Minv[(int64_t)i * K + j], a0);
        a1 = fma(sd[i + 1], Minv[(int64_t)(i + 1) * K + j], a1);
      }
      if (i < i1) a0 = fma(sd[i], Minv[(int64_t)i * K + j], a0);
    }
    part[t] = a0 + a1;
    __syncthreads();
    double dh = 0.0;
    if (t < K) {
      double hj = 0.0;
      for (int qq = 0; qq < Q; ++qq) hj += part[qq * Kpad + t];
      h[row * K + t] = hj;
      dh = sd[t] * hj;
    }
    for (int o = 16; o > 0; o >>= 1) dh += __shfl_down_sync(0xffffffffu, dh, o);
    if (lane == 0) sdot[w] = dh;
    __syncthreads();
    if (t == 0) {
      double sdh = 0.0;
      for (int ww = 0; ww < INV_NT / 32; ++ww) sdh += sdot[ww];
      dot_part[row] = sdh;
    }
    __syncthreads();
  }
  __threadfence();
  if (t == 0) s_last = atomicAdd(ctr, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last || w != 0) return;
  __threadfence();
  double acc = 0.0;
  for (int64_t r = lane; r < rows; r += 32) acc += __ldcg(dot_part + r);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    *num = acc;
    *ctr = 0u;
  }
}

cudaError_t launch_inv_rows(const double* Minv, const double* d, double* h, int K, int64_t rows, double* dot_part,
                            unsigned int* ctr, double* num, cudaStream_t st) {
  if (K < 1 || K > kLdlKmax || rows < 1) return rows == 0 ? cudaSuccess : cudaErrorInvalidValue;
  int Kpad = 1;
  while (Kpad < K) Kpad <<= 1;
  const unsigned blocks = (unsigned)imin(rows, 65535);
  k_inv_rows<<<blocks, INV_NT, 0, st>>>(Minv, d, h, K, Kpad, rows, dot_part, ctr, num);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Cholesky of G + lambda I (K > 128)
// Blocked right-looking Cholesky (G + lambda I = L L^T, FP64) for the Gram sizes beyond the
// register-resident LDL^T (K > 128), spread over the GPU: per panel of 32 columns, one warp
// factors the diagonal block in registers, one warp per row solves the panel below it against
// that block, and CTAs of 32 x 32 tiles apply the symmetric rank-32 update to the trailing
// lower triangle.  GB300's FP64 rate per SM is low, so the K^3 / 6 update FMAs must not sit on
// one SM.  Output: L row-major lower (diagonal = sqrt of the pivot) in L[0, K^2), the reciprocal
// diagonal in L[K^2, K^2 + K), the column-major copy of L in L[K^2 + K, 2 K^2 + K) (so that both
// substitutions read L with unit stride).  lambda >= 0 absolute, < 0 relative to tr(G) / K.  A
// non-positive or non-finite pivot sets DEV_SINGULAR; the later kernels see it and do nothing.
constexpr int BCH_NB = 32;

__global__ void k_bchol_init(const double* __restrict__ G, int K, double lam_in, double* __restrict__ W,
                             double* __restrict__ scal) {
  pdl_wait();
  pdl_trigger();
  __shared__ double s_red[8];
  __shared__ double s_lam;
  const int tid = threadIdx.x;
  double tr = 0.0;
  for (int i = tid; i < K; i += blockDim.x) tr += G[(int64_t)i * K + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = tr;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    s_lam = lam_in >= 0 ? lam_in : -lam_in * t / K;
    if (blockIdx.x == 0) scal[5] = s_lam;
  }
  __syncthreads();
  const double lam = s_lam;
  const int64_t n = (int64_t)K * K;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + tid; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / K), m = (int)(e - (int64_t)i * K);
    if (m <= i) W[e] = G[e] + (i == m ? lam : 0.0);
  }
}

// 1/sqrt(p) for the pivots of the blocked Cholesky: FP32 seed (rsqrtf, relative error below
// 2^-21) refined by two Newton steps for the inverse square root, y <- y + y (1 - p y^2) / 2,
// each of which squares the relative error, so the result is within a few ulp of FP64.  Kept
// off the exact square root and division, whose long dependent sequences would sit on the
// critical path of every pivot.  Outside [1e-30, 1e30] (beyond the FP32 seed's range) the
// exact expression is used.
__device__ __noinline__ double rsqrt_exact(double p) { return 1.0 / sqrt(p); }

__device__ __forceinline__ double rsqrt_pivot(double p) {
  if (!(p >= 1e-30 && p <= 1e30)) return rsqrt_exact(p);
  double y = (double)rsqrtf((float)p);
  double e = fma(-p * y, y, 1.0);
  y = fma(0.5 * y, e, y);
  e = fma(-p * y, y, 1.0);
  return fma(0.5 * y, e, y);
}

// Cholesky of the 32 x 32 diagonal block at (j0, j0), in shared memory, 128 threads.  The FP64
// unit issues about one warp instruction per 70 clocks per scheduler on this GPU, so the
// trailing update of every pivot is spread over four warps (all four schedulers): thread t
// owns row i = t / 4 of the block and updates its columns j < m <= i with stride 4.  Rows and
// columns beyond the matrix (a ragged last block) are identity.  rdiag receives 1 / L_jj.
constexpr int BCH_DT = 128;
__global__ void __launch_bounds__(BCH_DT) k_bchol_diag(double* __restrict__ W, double* __restrict__ rdiag, int K,
                                                       int j0, int* __restrict__ dstatus) {
  pdl_wait();
  pdl_trigger();
  if (*(volatile int*)dstatus & DEV_SINGULAR) return;
  __shared__ double a[BCH_NB][BCH_NB + 1];
  __shared__ double rr[BCH_NB];
  __shared__ int s_bad;
  const int t = threadIdx.x;
  const int nb = imin(BCH_NB, K - j0);
  for (int e = t; e < BCH_NB * BCH_NB; e += BCH_DT) {
    const int i = e / BCH_NB, m = e % BCH_NB;
    a[i][m] = (i < nb && m < nb) ? (m <= i ? W[(int64_t)(j0 + i) * K + j0 + m] : 0.0) : (i == m ? 1.0 : 0.0);
  }
  if (t == 0) s_bad = 0;
  __syncthreads();
  const int i = t >> 2, sub = t & 3;    // this thread's row and column phase
  for (int j = 0; j < BCH_NB; ++j) {
    if (t == 0) {
      const double piv = a[j][j];
      const bool bad = !(piv > 0.0) || !isfinite(piv);
      if (bad) s_bad = 1;
      const double rj = bad ? 1.0 : rsqrt_pivot(piv);
      rr[j] = rj;
      a[j][j] = bad ? 1.0 : piv * rj;
    }
    __syncthreads();
    // column j below the pivot: L_ij = a_ij / L_jj (row i's four threads read it after the barrier)
    if (sub == 0 && i > j) a[i][j] *= rr[j];
    __syncthreads();
    if (i > j) {
      const double lij = a[i][j];
      for (int m = j + 1 + sub; m <= i; m += 4) a[i][m] = fma(-lij, a[m][j], a[i][m]);
    }
    __syncthreads();
  }
  if (s_bad) {
    if (t == 0) atomicOr(dstatus, (int)DEV_SINGULAR);
    return;
  }
  for (int e = t; e < BCH_NB * BCH_NB; e += BCH_DT) {
    const int r = e / BCH_NB, m = e % BCH_NB;
    if (r < nb && m <= r) W[(int64_t)(j0 + r) * K + j0 + m] = a[r][m];
  }
  if (t < nb) rdiag[j0 + t] = rr[t];
}

// rows i >= j0 + 32: row i of the panel, x, solves x L11^T = a (forward substitution in the
// column-oriented form: x_t is final at step t and is subtracted from the later entries)
__global__ void __launch_bounds__(256) k_bchol_panel(double* __restrict__ W, const double* __restrict__ rdiag,
                                                     int K, int j0, const int* __restrict__ dstatus) {
  pdl_wait();
  pdl_trigger();
  if (*(volatile const int*)dstatus & DEV_SINGULAR) return;
  __shared__ double sL[BCH_NB][BCH_NB + 1];
  __shared__ double sr[BCH_NB];
  for (int e = threadIdx.x; e < BCH_NB * BCH_NB; e += blockDim.x) {
    const int i = e / BCH_NB, m = e % BCH_NB;
    sL[i][m] = m <= i ? W[(int64_t)(j0 + i) * K + j0 + m] : 0.0;
  }
  if (threadIdx.x < BCH_NB) sr[threadIdx.x] = rdiag[j0 + threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  for (int i = j0 + BCH_NB + blockIdx.x * warps + (threadIdx.x >> 5); i < K; i += gridDim.x * warps) {
    double* wr = W + (int64_t)i * K + j0;
    double a = wr[lane];
#pragma unroll
    for (int t = 0; t < BCH_NB; ++t) {
      const double xt = __shfl_sync(0xffffffffu, a, t) * sr[t];
      if (lane == t) a = xt;
      if (lane > t) a = fma(-xt, sL[lane][t], a);
    }
    wr[lane] = a;
  }
}

// trailing update A22 -= L21 L21^T on the lower triangle, one 32 x 32 tile per CTA; tile q of
// the packed lower triangle of tiles -> (bi, bj), bj <= bi
__global__ void __launch_bounds__(256) k_bchol_update(double* __restrict__ W, int K, int j0,
                                                      const int* __restrict__ dstatus) {
  pdl_wait();
  pdl_trigger();
  if (*(volatile const int*)dstatus & DEV_SINGULAR) return;
  __shared__ double sa[BCH_NB][BCH_NB + 1];
  __shared__ double sb[BCH_NB][BCH_NB + 1];
  const int q = blockIdx.x;
  int bi = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
  while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
  while (bi * (bi + 1) / 2 > q) --bi;
  const int bj = q - bi * (bi + 1) / 2;
  const int base = j0 + BCH_NB;
  const int r0 = base + bi * BCH_NB, c0 = base + bj * BCH_NB;
  for (int e = threadIdx.x; e < BCH_NB * BCH_NB; e += blockDim.x) {
    const int i = e / BCH_NB, t = e % BCH_NB;
    sa[i][t] = r0 + i < K ? W[(int64_t)(r0 + i) * K + j0 + t] : 0.0;
    sb[i][t] = c0 + i < K ? W[(int64_t)(c0 + i) * K + j0 + t] : 0.0;
  }
  __syncthreads();
  const int m = threadIdx.x & 31;
  for (int i = threadIdx.x >> 5; i < BCH_NB; i += blockDim.x >> 5) {
    const int gi = r0 + i, gm = c0 + m;
    if (gi >= K || gm >= K || gm > gi) continue;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < BCH_NB; ++t) acc = fma(sa[i][t], sb[m][t], acc);
    W[(int64_t)gi * K + gm] -= acc;
  }
}

// column-major copy of the lower triangle: Lc[j K + i] = L[i][j], i >= j (32 x 32 tiles)
__global__ void __launch_bounds__(256) k_bchol_colcopy(const double* __restrict__ W, double* __restrict__ Lc,
                                                       int K, const int* __restrict__ dstatus) {
  pdl_wait();
  pdl_trigger();
  if (*(volatile const int*)dstatus & DEV_SINGULAR) return;
  __shared__ double t[BCH_NB][BCH_NB + 1];
  const int i0 = blockIdx.y * BCH_NB, j0 = blockIdx.x * BCH_NB;
  if (j0 > i0) return;
  for (int e = threadIdx.x; e < BCH_NB * BCH_NB; e += blockDim.x) {
    const int r = e / BCH_NB, c = e % BCH_NB;
    if (i0 + r < K && j0 + c < K) t[r][c] = W[(int64_t)(i0 + r) * K + j0 + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < BCH_NB * BCH_NB; e += blockDim.x) {
    const int c = e / BCH_NB, r = e % BCH_NB;
    if (i0 + r < K && j0 + c < K && i0 + r >= j0 + c) Lc[(int64_t)(j0 + c) * K + i0 + r] = t[r][c];
  }
}

cudaError_t launch_cholesky(const double* G, int K, double lambda, double* L, double* scal,
                            int* dstatus, cudaStream_t st) {
  double* rdiag = L + (int64_t)K * K;
  double* Lc = rdiag + K;
  const int64_t n = (int64_t)K * K;
  pdl_launch(k_bchol_init, dim3((unsigned)imin((n + 255) / 256, 1024)), dim3(256), 0, st, G, K, lambda, L, scal);
  note_launch();
  for (int j0 = 0; j0 < K; j0 += BCH_NB) {
    pdl_launch(k_bchol_diag, dim3(1), dim3(BCH_DT), 0, st, L, rdiag, K, j0, dstatus);
    note_launch();
    const int rest = K - j0 - BCH_NB;
    if (rest <= 0) break;
    pdl_launch(k_bchol_panel, dim3((unsigned)imin((rest + 7) / 8, 1024)), dim3(256), 0, st, L, rdiag, K, j0, dstatus);
    note_launch();
    const int nt = (rest + BCH_NB - 1) / BCH_NB;
    pdl_launch(k_bchol_update, dim3((unsigned)(nt * (nt + 1) / 2)), dim3(256), 0, st, L, K, j0, dstatus);
    note_launch();
  }
  const unsigned tb = (unsigned)((K + BCH_NB - 1) / BCH_NB);
  pdl_launch(k_bchol_colcopy, dim3(tb, tb), dim3(256), 0, st, L, Lc, K, dstatus);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ h = d (G + lambda I)^{-1}
// b[m] -= v[m] y for m in [m_lo, m_hi), strided over the block's threads, with the factor's
// entries v[] (from L2 or HBM: the factor does not fit in shared memory) loaded SOLVE_U per
// thread at a time and the next group's loads issued before the current group's FMAs (one
// load in flight at a time left each step bound by the load latency: 0.16 TFLOP/s at
// K = 6400).  Per entry the arithmetic is b - v y, as before.
constexpr int SOLVE_U = 16;
constexpr int SOLVE_NT = 128;
__device__ __forceinline__ void axpy_strided(double* __restrict__ b, const double* __restrict__ v, double y,
                                             int m_lo, int m_hi, int tid) {
  int m0 = m_lo + tid;
  double c[SOLVE_U];
#pragma unroll
  for (int u = 0; u < SOLVE_U; ++u) {
    const int m = m0 + SOLVE_NT * u;
    c[u] = m < m_hi ? v[m] : 0.0;
  }
  for (; m0 < m_hi; m0 += SOLVE_NT * SOLVE_U) {
    double n[SOLVE_U];
#pragma unroll
    for (int u = 0; u < SOLVE_U; ++u) {
      const int m = m0 + SOLVE_NT * (SOLVE_U + u);
      n[u] = m < m_hi ? v[m] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < SOLVE_U; ++u) {
      const int m = m0 + SOLVE_NT * u;
      if (m < m_hi) b[m] -= c[u] * y;
    }
#pragma unroll
    for (int u = 0; u < SOLVE_U; ++u) c[u] = n[u];
  }
}

// One block of SOLVE_NT threads per row of d (the row in shared memory, K doubles: at
// K = 6400 four rows fit an SM, so four warps per row keep four warps on each scheduler to
// hide the factor's load latency): forward substitution with L (column j of L read from the
// column-major copy), then back substitution with L^T (row j of L), both with unit stride
// across the threads and a block barrier per step.  For K > 512.
__global__ void __launch_bounds__(SOLVE_NT) k_solve_rows(const double* __restrict__ L, const double* __restrict__ d,
                                                         double* __restrict__ h, int K, int64_t rows) {
  extern __shared__ double b[];
  const int tid = threadIdx.x;
  const double* rdiag = L + (int64_t)K * K;
  const double* Lc = rdiag + K;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    for (int m = tid; m < K; m += SOLVE_NT) b[m] = d[row * K + m];
    __syncthreads();
    for (int j = 0; j < K; ++j) {
      const double yj = b[j] * rdiag[j];
      __syncthreads();
      if (tid == 0) b[j] = yj;
      axpy_strided(b, Lc + (int64_t)j * K, yj, j + 1, K, tid);
      __syncthreads();
    }
    for (int j = K - 1; j >= 0; --j) {
      const double hj = b[j] * rdiag[j];
      __syncthreads();
      if (tid == 0) b[j] = hj;
      axpy_strided(b, L + (int64_t)j * K, hj, 0, j, tid);
      __syncthreads();
    }
    for (int m = tid; m < K; m += SOLVE_NT) h[row * K + m] = b[m];
    __syncthreads();
  }
}

// The same substitutions with the row held in registers: lane l keeps entries l + 32 v (v < NV,
// K <= 32 NV), the solved entry of step j is broadcast by a shuffle from lane j mod 32, and the
// factor's next column (forward) or row (backward) is loaded one step ahead so that its L2
// latency overlaps the current step.  The FP64 pipe (one warp-DFMA per scheduler every few tens
// of cycles on this part) is then the bound instead of shared-memory round trips and barriers.
// Per entry the arithmetic and its order are those of k_solve_rows (fma(-L, y, b), j ascending
// then descending), so both kernels give identical results.
template <int NV>
__global__ void __launch_bounds__(32) k_solve_rows_reg(const double* __restrict__ L, const double* __restrict__ d,
                                                       double* __restrict__ h, int K, int64_t rows) {
  const int lane = threadIdx.x & 31;
  const double* rdiag = L + (int64_t)K * K;
  const double* Lc = rdiag + K;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    double b[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int m = lane + 32 * v;
      b[v] = m < K ? d[row * K + m] : 0.0;
    }
    // forward: y_j = b_j / L_jj, then b_m -= L_mj y_j for m > j; step j = 32 vb + jj
#pragma unroll
    for (int vb = 0; vb < NV; ++vb) {
      const int jend = min(32, K - 32 * vb);
      if (jend <= 0) continue;
      double c[NV], cn[NV];
#pragma unroll
      for (int v = vb; v < NV; ++v) {
        const int m = lane + 32 * v;
        c[v] = m < K ? Lc[(int64_t)(32 * vb) * K + m] : 0.0;
      }
      double rd = rdiag[32 * vb];
      for (int jj = 0; jj < jend; ++jj) {
        const int j = 32 * vb + jj;
        const bool more = jj + 1 < jend;
#pragma unroll
        for (int v = vb; v < NV; ++v) {
          const int m = lane + 32 * v;
          cn[v] = (more && m < K) ? Lc[(int64_t)(j + 1) * K + m] : 0.0;
        }
        const double rdn = more ? rdiag[j + 1] : 0.0;
        const double y = __shfl_sync(0xffffffffu, b[vb], jj) * rd;
        const double t = fma(-c[vb], y, b[vb]);
        b[vb] = lane == jj ? y : (lane > jj ? t : b[vb]);
#pragma unroll
        for (int v = vb + 1; v < NV; ++v) b[v] = fma(-c[v], y, b[v]);
#pragma unroll
        for (int v = vb; v < NV; ++v) c[v] = cn[v];
        rd = rdn;
      }
    }
    // backward: h_j = b_j / L_jj, then b_m -= L_jm h_j for m < j; j descending
#pragma unroll
    for (int vb = NV - 1; vb >= 0; --vb) {
      const int jend = min(32, K - 32 * vb);
      if (jend <= 0) continue;
      double c[NV], cn[NV];
      const int jt = 32 * vb + jend - 1;
#pragma unroll
      for (int v = 0; v <= vb; ++v) {
        const int m = lane + 32 * v;
        c[v] = m < jt ? L[(int64_t)jt * K + m] : 0.0;
      }
      double rd = rdiag[jt];
      for (int jj = jend - 1; jj >= 0; --jj) {
        const int j = 32 * vb + jj;
        const bool more = jj > 0;
#pragma unroll
        for (int v = 0; v <= vb; ++v) {
          const int m = lane + 32 * v;
          cn[v] = (more && m < j - 1) ? L[(int64_t)(j - 1) * K + m] : 0.0;
        }
        const double rdn = more ? rdiag[j - 1] : 0.0;
        const double y = __shfl_sync(0xffffffffu, b[vb], jj) * rd;
        const double t = fma(-c[vb], y, b[vb]);
        b[vb] = lane == jj ? y : (lane < jj ? t : b[vb]);
#pragma unroll
        for (int v = 0; v < vb; ++v) b[v] = fma(-c[v], y, b[v]);
#pragma unroll
        for (int v = 0; v <= vb; ++v) c[v] = cn[v];
        rd = rdn;
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int m = lane + 32 * v;
      if (m < K) h[row * K + m] = b[v];
    }
  }
}

cudaError_t launch_solve_rows(const double* L, const double* d, double* h, int K, int64_t rows,
                              cudaStream_t st) {
  const unsigned blocks = (unsigned)imin(rows, 8192);     // one warp (registers) or block per row
  if (K <= 256) {
    k_solve_rows_reg<8><<<blocks, 32, 0, st>>>(L, d, h, K, rows);
  } else if (K <= 416) {
    k_solve_rows_reg<13><<<blocks, 32, 0, st>>>(L, d, h, K, rows);
  } else if (K <= 512) {
    k_solve_rows_reg<16><<<blocks, 32, 0, st>>>(L, d, h, K, rows);
  } else {
    const size_t smem_row = (size_t)K * sizeof(double);
    if (smem_row > kSmemOptIn) return cudaErrorInvalidValue;
    if (smem_row > 48 * 1024)
      cudaFuncSetAttribute(k_solve_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row);
    k_solve_rows<<<blocks, SOLVE_NT, smem_row, st>>>(L, d, h, K, rows);
  }
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reductions / scalars
__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                      double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

cudaError_t launch_dot(const double* a, const double* b, int64_t n, double* out, cudaStream_t st) {
  k_dot<<<1, 256, 0, st>>>(a, b, n, out);
  note_launch();
  return cudaGetLastError();
}

// Step size and update in one launch: every block forms eta = <d,h> / den (den summed from the
// line-search pass's per-CTA partials in the same fixed order as the statistics reduction,
// field 6, or read from `den`), forced to 0 on a flagged or non-finite step; block 0 records
// it; then Z_k <- Z_k + eta fold(h) (update-sign reading of Eq. updatessd / Eq. ftrbcn), and
// the FP32 copy of the core follows.  With adv.S, the merged half that holds core k moves
// with it: the half is linear in core k, so S += eta S_h equals merging it again (up to FP32
// rounding), and its BF16 hi/lo operand rows are written again.
__global__ void k_step_update(double* __restrict__ Z, float* __restrict__ Zf, HalfAdvance adv,
                              const double* __restrict__ h, int64_t n,
                              const double* __restrict__ num, const double* __restrict__ part, int ctas,
                              const double* __restrict__ den_in, double fixed_eta, int* dstatus,
                              double* __restrict__ eta_out, double* __restrict__ eta_slot) {
  __shared__ double s_eta;
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double dn = 0.0;
    if (part) {
      // the loads are independent: unrolled so that several are in flight (the sum keeps its
      // order)
#pragma unroll 8
      for (int c = lane; c < ctas; c += 32) dn += part[(int64_t)c * 8 + 6];
      for (int o = 16; o > 0; o >>= 1) dn += __shfl_down_sync(0xffffffffu, dn, o);
    } else if (den_in) {
      dn = *den_in;
    }
    if (lane == 0) {
      // a NaN denominator (non-finite weights or direction) rejects the step as non-finite;
      // a zero one (no observed slot) gives no step
      double eta = fixed_eta > 0 ? fixed_eta : (isnan(dn) ? dn : (dn > 0 ? *num / dn : 0.0));
      const bool finite = isfinite(eta);
      if (!finite) eta = 0.0;
      if (*dstatus & (DEV_SINGULAR | DEV_NONFINITE)) eta = 0.0;
      if (blockIdx.x == 0) {
        if (!finite) atomicOr(dstatus, (int)DEV_NONFINITE);
        *eta_out = eta;
        if (eta_slot) *eta_slot = eta;
      }
      s_eta = eta;
    }
  }
  __syncthreads();
  const double e = s_eta;
  if (e == 0.0) return;   // a rejected step leaves the core untouched (h may be non-finite)
#pragma unroll 4
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double z = fma(e, h[i], Z[i]);
    Z[i] = z;
    Zf[i] = (float)z;
  }
  if (!adv.S) return;
  const float ef = (float)e;
  const int step = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
  RowCol rc(i0, step, adv.Kp);
  // four elements per round, all loads first (S and S_h never overlap, but the compiler cannot
  // know it through the struct, so it would not move a load above the previous store)
  int64_t i = i0;
  for (; i + 3 * (int64_t)step < adv.n; i += 4 * (int64_t)step) {
    float sv[4], hv[4];
    int64_t q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t ii = i + u * (int64_t)step;
      sv[u] = adv.S[ii];
      hv[u] = adv.Sh[ii];
      q[u] = (int64_t)rc.r * adv.kpad + rc.c;
      rc.next();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float v = fmaf(ef, hv[u], sv[u]);
      adv.S[i + u * (int64_t)step] = v;
      const __nv_bfloat16 vh = bf16_rn(v);
      adv.hi[q[u]] = vh;
      adv.lo[q[u]] = bf16_rn(v - __bfloat162float(vh));
    }
  }
  for (; i < adv.n; i += step, rc.next()) {
    const float v = fmaf(ef, adv.Sh[i], adv.S[i]);
    adv.S[i] = v;
    const __nv_bfloat16 vh = bf16_rn(v);
    const int64_t q = (int64_t)rc.r * adv.kpad + rc.c;
    adv.hi[q] = vh;
    adv.lo[q] = bf16_rn(v - __bfloat162float(vh));
  }
}

cudaError_t launch_step_update(double* Z, float* Zf, const double* h, int64_t n, const double* num, const double* part,
                               int ctas, const double* den, double fixed_eta, int* dstatus, double* eta,
                               double* eta_slot, cudaStream_t st, const HalfAdvance& adv) {
  // every block forms eta itself (FP64, a few dozen operations in one warp): keep the grid
  // to two blocks per SM so that this stays small next to the element work
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t work = adv.S ? imax(n, adv.n) : n;
  pdl_launch(k_step_update, dim3((unsigned)imax(1, imin((work + 255) / 256, 2 * (int64_t)sms))), dim3(256), 0, st, Z,
             Zf, adv, h, n, num, part, ctas, den, fixed_eta, dstatus, eta, eta_slot);
  note_launch();
  return cudaGetLastError();
}

// e = ||D - Dprev||_F / ||D||_F, then Dprev <- D  (Algorithm 1 stopping quantity).  Spread
// over many blocks (the FP64 work of one SM would take several microseconds): each block
// writes its partial sums to part[2 b], part[2 b + 1] and keeps D for the next iteration; the
// last block to finish adds the partials in block order (counter *ctr is reset by it).
__global__ void __launch_bounds__(256) k_stop_error(const double* __restrict__ D, double* __restrict__ Dprev,
                                                    int64_t n, double* __restrict__ part,
                                                    unsigned int* __restrict__ ctr, double* __restrict__ e_out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double s1[8], s2[8];
  __shared__ int s_last;
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = D[i], dd = x - Dprev[i];
    a = fma(dd, dd, a);
    b = fma(x, x, b);
    Dprev[i] = x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s1[w] = a;
    s2[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      sa += s1[q];
      sb += s2[q];
    }
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
    __threadfence();
    s_last = atomicAdd(ctr, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double sa = 0.0, sb = 0.0;
  for (unsigned q = 0; q < gridDim.x; ++q) {
    sa += __ldcg(part + 2 * q);
    sb += __ldcg(part + 2 * q + 1);
  }
  *e_out = sb > 0 ? sqrt(sa / sb) : 0.0;
  *ctr = 0u;
}

cudaError_t launch_stop_error(const double* D, double* Dprev, int64_t n, double* part, unsigned int* ctr,
                              double* e_out, cudaStream_t st) {
  const unsigned blocks = (unsigned)imax(1, imin((n + 255) / 256, kStopBlocks));
  pdl_launch(k_stop_error, dim3(blocks), dim3(256), 0, st, D, Dprev, n, part, ctr, e_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trd
