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
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < parts; ++q) s += part[(int64_t)q * n + i];
    out[i] = s;
  }
}

cudaError_t launch_fgmc_E(const double* Z, const int32_t* idx, int64_t n, int rk, int rk1,
                          double* E, double* work, cudaStream_t st) {
  const int64_t tot = (int64_t)rk * rk * rk1 * rk1;
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
  k_fgmc_E<<<grid, 128, smem, st>>>(Z, idx, n, rk, rk1, CH, parts > 1 ? work : E);
  note_launch();
  if (parts == 1) return cudaGetLastError();
  k_sum_parts<<<(unsigned)imin((tot + 255) / 256, 4096), 256, 0, st>>>(work, parts, tot, E);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FP64 GEMM (small)
// C[M x N] = A[M x K] * B, B is K x N (transB = 0) or N x K (transB = 1); all row-major.
__global__ void k_dgemm(const double* __restrict__ A, const double* __restrict__ B,
                        double* __restrict__ C, int M, int N, int K, int transB) {
  __shared__ double sA[16][17], sB[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    sA[ty][tx] = (row < M && k0 + tx < K) ? A[(int64_t)row * K + k0 + tx] : 0.0;
    const int bk = k0 + ty, bn = blockIdx.x * 16 + tx;
    double bv = 0.0;
    if (bk < K && bn < N) bv = transB ? B[(int64_t)bn * K + bk] : B[(int64_t)bk * N + bn];
    sB[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(sA[ty][k], sB[k][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) C[(int64_t)row * N + col] = acc;
}

cudaError_t launch_dgemm(const double* A, const double* B, double* C, int M, int N, int K,
                         bool transB, cudaStream_t st) {
  dim3 grid((N + 15) / 16, (M + 15) / 16), block(16, 16);
  k_dgemm<<<grid, block, 0, st>>>(A, B, C, M, N, K, transB ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ realignment Phi
// G[a + b q, a' + b' q] = T[b p + b', a q + a'] for the subchain with p x q slices
// (p = r_{k+1}, q = r_k); T is p^2 x q^2 row-major.
__global__ void k_phi(const double* __restrict__ T, int p, int q, double* __restrict__ G) {
  const int K = p * q;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x) {
    const int r = e / K, c = e % K;
    const int a = r % q, b = r / q, a2 = c % q, b2 = c / q;
    G[e] = T[(int64_t)(b * p + b2) * (q * q) + a * q + a2];
  }
}

cudaError_t launch_phi(const double* T, int p, int q, double* G, cudaStream_t st) {
  const int K = p * q;
  k_phi<<<(K * K + 255) / 256, 256, 0, st>>>(T, p, q, G);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Cholesky of G + lambda I
// One CTA, right-looking, lower triangle in shared memory when it fits (K <= 160), else in
// the output array.  lambda >= 0 absolute, < 0 relative to tr(G)/K.  Per column: every
// thread reads the pivot, the sub-diagonal column is scaled into a buffer, then the
// trailing lower triangle is updated (two barriers per column).  A non-positive or
// non-finite pivot sets DEV_SINGULAR and stops (L is then unusable).
__global__ void k_cholesky(const double* __restrict__ G, int K, double lam_in, double* __restrict__ L,
                           double* __restrict__ scal, int* __restrict__ dstatus, int use_smem) {
  extern __shared__ double smc[];
  __shared__ double s_red[32];
  __shared__ double s_col[1024];
  double* W = use_smem ? smc : L;
  const int tid = threadIdx.x, nt = blockDim.x;
  // lambda (trace reduction in parallel)
  double tr = 0.0;
  for (int i = tid; i < K; i += nt) tr += G[(int64_t)i * K + i];
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = tr;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) t += s_red[w];
    s_red[0] = lam_in >= 0 ? lam_in : -lam_in * t / K;
    scal[5] = s_red[0];
  }
  __syncthreads();
  const double lam = s_red[0];
  for (int e = tid; e < K * K; e += nt) {
    const int i = e / K, j = e % K;
    W[e] = j <= i ? G[e] + (i == j ? lam : 0.0) : 0.0;
  }
  __syncthreads();
  // pivot j's square root and reciprocal are computed once, by thread 0 (which owns the
  // diagonal element of the trailing update), and published through shared memory
  __shared__ double s_dj, s_rj;
  __shared__ int s_bad;
  if (tid == 0) {
    const double piv = W[0];
    s_bad = !(piv > 0.0) || !isfinite(piv);
    s_dj = s_bad ? 1.0 : sqrt(piv);
    s_rj = 1.0 / s_dj;
  }
  __syncthreads();
  bool bad = false;
  for (int j = 0; j < K; ++j) {
    if (s_bad) { bad = true; break; }                  // uniform across threads
    const double dj = s_dj, rj = s_rj;
    for (int i = j + 1 + tid; i < K; i += nt) s_col[i] = W[(int64_t)i * K + j] * rj;
    __syncthreads();
    if (tid == 0) {
      W[(int64_t)j * K + j] = dj;
      L[(int64_t)K * K + j] = rj;       // reciprocal diagonal, used by the solves
    }
    for (int i = j + 1 + tid; i < K; i += nt) W[(int64_t)i * K + j] = s_col[i];
    // trailing lower triangle, 16 x 16 thread tile (blockDim 256): thread (ti, tm) updates
    // rows i = j+1+ti+16a and columns m = j+1+tm+16b with m <= i
    {
      const int ti = tid >> 4, tm = tid & 15;
      for (int i = j + 1 + ti; i < K; i += 16) {
        const double li = s_col[i];
        double* Wi = W + (int64_t)i * K;
        for (int m = j + 1 + tm; m <= i; m += 16) Wi[m] -= li * s_col[m];
      }
    }
    if (tid == 0 && j + 1 < K) {
      // thread 0 updated W[j+1][j+1] above: prepare the next pivot
      const double piv = W[(int64_t)(j + 1) * K + (j + 1)];
      s_bad = !(piv > 0.0) || !isfinite(piv);
      s_dj = s_bad ? 1.0 : sqrt(piv);
      s_rj = 1.0 / s_dj;
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicOr(dstatus, (int)DEV_SINGULAR);
    return;
  }
  if (use_smem)
    for (int e = tid; e < K * K; e += nt) L[e] = W[e];
}

cudaError_t launch_cholesky(const double* G, int K, double lambda, double* L, double* scal,
                            int* dstatus, cudaStream_t st) {
  const size_t bytes = (size_t)K * K * sizeof(double);
  const bool sm = bytes <= 200 * 1024;
  if (sm) cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_cholesky<<<1, 256, sm ? bytes : 0, st>>>(G, K, lambda, L, scal, dstatus, sm ? 1 : 0);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ h = d (G + lambda I)^{-1}
// One warp per row of d: forward substitution with L, then back substitution with L^T.
// L is staged in shared memory when it fits (K <= 160), so each substitution step costs a
// shared-memory load instead of an L2 round trip.
__global__ void k_solve_rows(const double* __restrict__ Lg, const double* __restrict__ d,
                             double* __restrict__ h, int K, int64_t rows, int stage_L) {
  extern __shared__ double sb[];
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* L = Lg;
  const double* rdiag = Lg + (int64_t)K * K;
  double* b = sb + (size_t)w * K;
  if (stage_L) {
    double* Ls = sb + (size_t)warps * K;
    for (int e = threadIdx.x; e < K * K + K; e += blockDim.x) Ls[e] = Lg[e];
    __syncthreads();
    L = Ls;
    rdiag = Ls + (int64_t)K * K;
  }
  for (int64_t row = (int64_t)blockIdx.x * warps + w; row < rows; row += (int64_t)gridDim.x * warps) {
    for (int m = lane; m < K; m += 32) b[m] = d[row * K + m];
    __syncwarp();
    for (int j = 0; j < K; ++j) {
      const double yj = b[j] * rdiag[j];
      __syncwarp();
      if (lane == 0) b[j] = yj;
      for (int m = j + 1 + lane; m < K; m += 32) b[m] -= L[(int64_t)m * K + j] * yj;
      __syncwarp();
    }
    for (int j = K - 1; j >= 0; --j) {
      const double hj = b[j] * rdiag[j];
      __syncwarp();
      if (lane == 0) b[j] = hj;
      for (int m = lane; m < j; m += 32) b[m] -= L[(int64_t)j * K + m] * hj;
      __syncwarp();
    }
    for (int m = lane; m < K; m += 32) h[row * K + m] = b[m];
    __syncwarp();
  }
}

cudaError_t launch_solve_rows(const double* L, const double* d, double* h, int K, int64_t rows,
                              cudaStream_t st) {
  const int warps = 1;
  const bool stage = (size_t)K * K * sizeof(double) <= 160 * 1024;
  const size_t smem = (size_t)warps * K * sizeof(double) + (stage ? (size_t)(K * K + K) * sizeof(double) : 0);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_solve_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned blocks = (unsigned)imin((rows + warps - 1) / warps, 8192);
  k_solve_rows<<<blocks, warps * 32, smem, st>>>(L, d, h, K, rows, stage ? 1 : 0);
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

// eta = <d,h> / den (exact line search of Sec. 3.2) unless a fixed step is given; any
// earlier device error (singular Gram, non-finite values) forces eta = 0 so the core is
// left unchanged.  eta_slot (nullable) receives a copy for the iteration report.
__global__ void k_eta(const double* num, const double* den, double fixed_eta, int* dstatus,
                      double* eta_out, double* eta_slot) {
  double eta;
  if (fixed_eta > 0) {
    eta = fixed_eta;
  } else {
    const double dn = *den;
    eta = dn > 0 ? *num / dn : 0.0;
  }
  if (!isfinite(eta)) {
    atomicOr(dstatus, (int)DEV_NONFINITE);
    eta = 0.0;
  }
  if (*dstatus & (DEV_SINGULAR | DEV_NONFINITE)) eta = 0.0;
  *eta_out = eta;
  if (eta_slot) *eta_slot = eta;
}

cudaError_t launch_eta(const double* num, const double* den, double fixed_eta, int* dstatus,
                       double* eta, double* eta_slot, cudaStream_t st) {
  k_eta<<<1, 1, 0, st>>>(num, den, fixed_eta, dstatus, eta, eta_slot);
  note_launch();
  return cudaGetLastError();
}

// Z_k <- Z_k + eta fold(h)   (update-sign reading of Eq. updatessd / Eq. ftrbcn)
__global__ void k_axpy_core(double* __restrict__ Z, const double* __restrict__ h, int64_t n,
                            const double* __restrict__ eta) {
  const double e = *eta;
  if (e == 0.0) return;   // a rejected step leaves the core untouched (h may be non-finite)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    Z[i] = fma(e, h[i], Z[i]);
}

cudaError_t launch_axpy_core(double* Z, const double* h, int64_t n, const double* eta,
                             cudaStream_t st) {
  k_axpy_core<<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(Z, h, n, eta);
  note_launch();
  return cudaGetLastError();
}

// e = ||D - Dprev||_F / ||D||_F, then Dprev <- D  (Algorithm 1 stopping quantity)
__global__ void k_stop_error(const double* __restrict__ D, double* __restrict__ Dprev, int64_t n,
                             double* __restrict__ e_out) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double dd = D[i] - Dprev[i];
    a = fma(dd, dd, a);
    b = fma(D[i], D[i], b);
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *e_out = s2[0] > 0 ? sqrt(s1[0] / s2[0]) : 0.0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Dprev[i] = D[i];
}

cudaError_t launch_stop_error(const double* D, double* Dprev, int64_t n, double* e_out,
                              cudaStream_t st) {
  k_stop_error<<<1, 256, 0, st>>>(D, Dprev, n, e_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trd
