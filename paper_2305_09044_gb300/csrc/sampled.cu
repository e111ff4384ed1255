// Sampled correntropy loss and its adjoint (differentiation of Def. 1 + Eq. corr at sampled
// entries).
//
// With the ring cut into an inner block (modes 0..c-1, linear index a) and an outer block
// (c..N-1, index b), x_hat_m = Tr(A(a_m) C(b_m)) = <S_A[a_m], S_C[b_m]> (Thm. 1), where S_A / S_C
// are the merged subchains (recomputed on every call; nothing is kept between forward and
// backward).  Backward: g_m = g_scale * (-w_m e_m) is scattered as gA[a_m] += g_m S_C[b_m] and
// gC[b_m] += g_m S_A[a_m]; the gradient of every core then follows from the same
// back-contraction as the data passes (rows case from gA for inner cores, cols case from gC
// for outer cores).
#include <math.h>

#include <algorithm>
#include <vector>

#include "trd_internal.cuh"

namespace trd {

namespace {

// One warp per group of 32 entries: lane m owns entry m (indices, value, outputs); the 32
// dot products <S_A[a], S_C[b]> are computed cooperatively with coalesced row loads.
template <typename T>
__device__ __forceinline__ void group_xhat(const T* __restrict__ A, const T* __restrict__ C, int Kp,
                                           int64_t a, int64_t b, int lane, T& mine) {
  mine = T(0);
  for (int q = 0; q < 32; ++q) {
    const int64_t aq = __shfl_sync(0xffffffffu, a, q), bq = __shfl_sync(0xffffffffu, b, q);
    const T* Ar = A + aq * Kp;
    const T* Cr = C + bq * Kp;
    T part = T(0);
    for (int k = lane; k < Kp; k += 32) part = fma(Ar[k], Cr[k], part);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == q) mine = part;
  }
}

// Linear indices of entry m in the two blocks; false (entry skipped) if an index is out of range.
__device__ __forceinline__ bool entry_ab(const int32_t* __restrict__ idx, const Split2& sp, int64_t m, int64_t& a,
                                         int64_t& b) {
  a = 0;
  b = 0;
  const int32_t* r = idx + m * sp.N;
  bool ok = true;
  for (int j = 0; j < sp.N; ++j) {
    const int64_t i = r[j];
    ok = ok && i >= 0 && i < sp.dim[j];
    a += i * sp.sin[j];
    b += i * sp.sout[j];
  }
  if (!ok) { a = 0; b = 0; }
  return ok;
}

__device__ __forceinline__ float texp(float v) { return expf(v); }
__device__ __forceinline__ double texp(double v) { return exp(v); }

template <typename T>
__global__ void k_sampled(const T* __restrict__ A, const T* __restrict__ C, int Kp, const int32_t* __restrict__ idx,
                          Split2 sp, const T* __restrict__ x, int64_t M, double sigma, T* __restrict__ resid,
                          double* __restrict__ loss_part, int backward, double g_scale, T* __restrict__ gA,
                          T* __restrict__ gC) {
  __shared__ double sred[32];
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  double loss = 0.0;
  for (int64_t g0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; g0 < M; g0 += warps * 32) {
    const int64_t m = g0 + lane;
    bool live = m < M;
    int64_t a = 0, b = 0;
    if (live && !entry_ab(idx, sp, m, a, b)) {
      live = false;
      atomicOr(sp.err, (int)DEV_BOUNDS);
    }
    T xh;
    group_xhat<T>(A, C, Kp, a, b, lane, xh);
    T e = T(0), w = T(0);
    if (live) {
      e = x[m] - xh;
      w = texp(-e * e * (T)inv2s2);
      loss += sigma * sigma * (1.0 - (double)w);
    }
    if (resid && m < M) resid[m] = e;
    if (!backward) continue;
    const T gm = live ? (T)(g_scale * -((double)w * (double)e)) : T(0);   // g_m = g_scale dloss/dx_hat
    for (int q = 0; q < 32; ++q) {
      const int64_t aq = __shfl_sync(0xffffffffu, a, q), bq = __shfl_sync(0xffffffffu, b, q);
      const T gq = __shfl_sync(0xffffffffu, gm, q);
      if (g0 + q >= M) break;
      const T* Ar = A + aq * Kp;
      const T* Cr = C + bq * Kp;
      T* gAr = gA + aq * Kp;
      T* gCr = gC + bq * Kp;
      for (int k = lane; k < Kp; k += 32) {
        atomicAdd(gAr + k, gq * Cr[k]);
        atomicAdd(gCr + k, gq * Ar[k]);
      }
    }
  }
  if (!loss_part) return;
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
  if (lane == 0) sred[threadIdx.x >> 5] = loss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
    loss_part[blockIdx.x] = s;
  }
}

__global__ void k_to_double(const float* __restrict__ src, int64_t n, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

template <typename T>
__global__ void k_from_double(const double* __restrict__ src, int64_t n, T* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

}  // namespace

cudaError_t launch_sampled_kernel(const void* A, const void* C, bool fp64, int Kp, const int32_t* idx,
                                  const Split2* sp, const void* x, int64_t M, double sigma, void* resid,
                                  double* loss_part, int parts, bool backward, double g_scale, void* gA, void* gC,
                                  cudaStream_t st) {
  if (fp64)
    k_sampled<double><<<parts, 256, 0, st>>>((const double*)A, (const double*)C, Kp, idx, *sp, (const double*)x, M,
                                             sigma, (double*)resid, loss_part, backward ? 1 : 0, g_scale,
                                             (double*)gA, (double*)gC);
  else
    k_sampled<float><<<parts, 256, 0, st>>>((const float*)A, (const float*)C, Kp, idx, *sp, (const float*)x, M,
                                            sigma, (float*)resid, loss_part, backward ? 1 : 0, g_scale, (float*)gA,
                                            (float*)gC);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_to_double(const float* src, int64_t n, double* dst, cudaStream_t st) {
  k_to_double<<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(src, n, dst);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_from_double(const double* src, int64_t n, void* dst, bool fp64, cudaStream_t st) {
  if (fp64)
    k_from_double<double><<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(src, n, (double*)dst);
  else
    k_from_double<float><<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(src, n, (float*)dst);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trd
