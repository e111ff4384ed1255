// Sampled correntropy loss and its adjoint (differentiation of Def. 1 + Eq. corr at sampled
// entries).
//
// With the ring cut into an inner block (modes 0..c-1, linear index a) and an outer block
// (c..N-1, index b), x_hat_m = Tr(A(a_m) C(b_m)) = <S_A[a_m], S_C[b_m]> (Thm. 1), where S_A / S_C
// are the merged subchains (recomputed on every call; nothing is kept between forward and
// backward).  Backward: g_m = g_scale * (-w_m e_m), gA[a] = sum_{m: a_m = a} g_m S_C[b_m] and
// gC[b] = sum_{m: b_m = b} g_m S_A[a_m]; the gradient of every core then follows from the same
// back-contraction as the data passes (rows case from gA for inner cores, cols case from gC
// for outer cores).
//
// The entries are first grouped by a and by b (a counting sort: histograms, prefix sums,
// scatter), so that the passes read each merged row once per group of entries and add to gA /
// gC once per row change and work item instead of once per entry (2 K' atomic additions per
// entry before).
#include <math.h>

#include <algorithm>
#include <vector>

#include "trd_internal.cuh"

namespace trd {

namespace {

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

// ---------------------------------------------------------------- entry order (counting sort)
// Keys of every entry (a, b; -1 for an entry with an index out of range) and their histograms.
__global__ void k_smp_keys(const int32_t* __restrict__ idx, Split2 sp, int64_t M, int32_t* __restrict__ ka,
                           int32_t* __restrict__ kb, uint32_t* __restrict__ cnt_a, uint32_t* __restrict__ cnt_b) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    int64_t a, b;
    if (!entry_ab(idx, sp, m, a, b)) {
      atomicOr(sp.err, (int)DEV_BOUNDS);
      ka[m] = kb[m] = -1;
      continue;
    }
    ka[m] = (int32_t)a;
    kb[m] = (int32_t)b;
    atomicAdd(cnt_a + a, 1u);
    atomicAdd(cnt_b + b, 1u);
  }
}

// Exclusive prefix sums of two count arrays in place (one block each: blockIdx.x = 0 / 1);
// each thread sums a contiguous chunk, a block-wide scan of the chunk sums, then the chunk
// prefixes.  cur receives a copy of the result (the scatter cursors).
__global__ void k_smp_scan(uint32_t* __restrict__ c0, int64_t n0, uint32_t* __restrict__ c1, int64_t n1,
                           uint32_t* __restrict__ cur0, uint32_t* __restrict__ cur1) {
  __shared__ uint32_t part[1024];
  uint32_t* c = blockIdx.x == 0 ? c0 : c1;
  uint32_t* cur = blockIdx.x == 0 ? cur0 : cur1;
  const int64_t n = blockIdx.x == 0 ? n0 : n1;
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t per = (n + T - 1) / T, lo = imin(n, t * per), hi = imin(n, lo + per);
  uint32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += c[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < T; off <<= 1) {
    const uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = part[t] - s;
  for (int64_t i = lo; i < hi; ++i) {
    const uint32_t v = c[i];
    c[i] = run;
    cur[i] = run;
    run += v;
  }
}

// Entry numbers grouped by a (perm_a) and by b (perm_b).  The order inside a group follows the
// atomic cursors, so sums over a group are reproducible to rounding, not bitwise.
__global__ void k_smp_scatter(const int32_t* __restrict__ ka, const int32_t* __restrict__ kb, int64_t M,
                              uint32_t* __restrict__ cur_a, uint32_t* __restrict__ cur_b, int32_t* __restrict__ perm_a,
                              int32_t* __restrict__ perm_b) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = ka[m];
    if (a < 0) continue;
    perm_a[atomicAdd(cur_a + a, 1u)] = (int32_t)m;
    perm_b[atomicAdd(cur_b + kb[m], 1u)] = (int32_t)m;
  }
}

// ---------------------------------------------------------------- passes over grouped entries
constexpr int kSmpChunk = 128;   // entries per warp work item
constexpr int kSmpMaxV = 16;     // K' values per lane held in registers (K' <= 512)

// Pass over the entries grouped by a: warp w takes positions [w C, (w + 1) C) of perm_a (C =
// kSmpChunk), keeps its row S_A[a] in registers while a stays the same, and for every entry
// reads S_C[b] once: x_hat = <S_A[a], S_C[b]>, e = x - x_hat, w = exp(-e^2 / 2 sigma^2), the
// loss, optionally e, and (backward) g = g_scale (-w e), stored per entry, with
// sum_entries g S_C[b] accumulated in registers and added to gA[a] once per row change.
template <typename T>
__global__ void k_smp_rows_a(const T* __restrict__ A, const T* __restrict__ C, int Kp,
                             const int32_t* __restrict__ perm_a, const int32_t* __restrict__ ka,
                             const int32_t* __restrict__ kb, const T* __restrict__ x, const uint32_t* __restrict__ n_dev,
                             double sigma, T* __restrict__ resid, double* __restrict__ loss_part, int backward,
                             double g_scale, T* __restrict__ garr, T* __restrict__ gA) {
  __shared__ double sred[32];
  const int64_t n = *n_dev;   // entries with valid indices
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const T nk = (T)(-1.0 / (2.0 * sigma * sigma));
  const T gs = (T)(-g_scale);     // g = g_scale d loss / d x_hat = -g_scale w e
  const int nv = (Kp + 31) >> 5;
  // e, w and g are the same on every lane after the shuffle reduction and are formed in T: the
  // FP64 unit (which also converts between FP32 and FP64) issues at a small fraction of the
  // FP32 rate here, so the FP32 path widens only the per-item loss sum
  double loss = 0.0;
  for (int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w0 * kSmpChunk < n; w0 += warps) {
    const int64_t p0 = w0 * kSmpChunk, p1 = imin(n, p0 + kSmpChunk);
    int32_t cur = -1;
    T lsum = T(0);                // sum of (1 - w) over this work item
    T av[kSmpMaxV], acc[kSmpMaxV];
#pragma unroll
    for (int v = 0; v < kSmpMaxV; ++v) av[v] = acc[v] = T(0);
    // the next entry's number, block indices and value are loaded one step ahead, off the
    // dependent chain perm -> (a, b) -> rows of the current entry
    int32_t mn = perm_a[p0];
    int32_t an = ka[mn], bn = kb[mn];
    T xn = x[mn];
    for (int64_t p = p0; p < p1; ++p) {
      const int32_t m = mn, a = an, b = bn;
      const T xm = xn;
      if (p + 1 < p1) {
        mn = perm_a[p + 1];
        an = ka[mn];
        bn = kb[mn];
        xn = x[mn];
      }
      if (a != cur) {
        if (backward && cur >= 0) {
#pragma unroll
          for (int v = 0; v < kSmpMaxV; ++v) {
            const int k = lane + 32 * v;
            if (v < nv && k < Kp) atomicAdd(gA + (int64_t)cur * Kp + k, acc[v]);
            acc[v] = T(0);
          }
        }
        cur = a;
#pragma unroll
        for (int v = 0; v < kSmpMaxV; ++v) {
          const int k = lane + 32 * v;
          av[v] = (v < nv && k < Kp) ? A[(int64_t)a * Kp + k] : T(0);
        }
      }
      T cv[kSmpMaxV];
      T part = T(0);
#pragma unroll
      for (int v = 0; v < kSmpMaxV; ++v) {
        const int k = lane + 32 * v;
        cv[v] = (v < nv && k < Kp) ? C[(int64_t)b * Kp + k] : T(0);
        part = fma(av[v], cv[v], part);
      }
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      const T e = xm - part;
      const T w = texp(e * e * nk);
      lsum += T(1) - w;
      if (lane == 0 && resid) resid[m] = e;
      if (backward) {
        const T g = gs * (w * e);
        if (lane == 0) garr[m] = g;
#pragma unroll
        for (int v = 0; v < kSmpMaxV; ++v) acc[v] = fma(g, cv[v], acc[v]);
      }
    }
    if (backward && cur >= 0) {
#pragma unroll
      for (int v = 0; v < kSmpMaxV; ++v) {
        const int k = lane + 32 * v;
        if (v < nv && k < Kp) atomicAdd(gA + (int64_t)cur * Kp + k, acc[v]);
      }
    }
    loss += (double)lsum;
  }
  loss *= sigma * sigma;
  if (!loss_part) return;
  if (lane == 0) sred[threadIdx.x >> 5] = loss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sred[w];
    loss_part[blockIdx.x] = s;
  }
}

// Pass over the entries grouped by b (backward): sum_entries g S_A[a] in registers, added to
// gC[b] once per row change.
template <typename T>
__global__ void k_smp_rows_b(const T* __restrict__ A, int Kp, const int32_t* __restrict__ perm_b,
                             const int32_t* __restrict__ ka, const int32_t* __restrict__ kb, const T* __restrict__ garr,
                             const uint32_t* __restrict__ n_dev, T* __restrict__ gC) {
  const int64_t n = *n_dev;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nv = (Kp + 31) >> 5;
  for (int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w0 * kSmpChunk < n; w0 += warps) {
    const int64_t p0 = w0 * kSmpChunk, p1 = imin(n, p0 + kSmpChunk);
    int32_t cur = -1;
    T acc[kSmpMaxV];
#pragma unroll
    for (int v = 0; v < kSmpMaxV; ++v) acc[v] = T(0);
    int32_t mn = perm_b[p0];
    int32_t an = ka[mn], bn = kb[mn];
    T gn = garr[mn];
    for (int64_t p = p0; p < p1; ++p) {
      const int32_t b = bn, a = an;
      const T g = gn;
      if (p + 1 < p1) {
        mn = perm_b[p + 1];
        an = ka[mn];
        bn = kb[mn];
        gn = garr[mn];
      }
      if (b != cur) {
        if (cur >= 0) {
#pragma unroll
          for (int v = 0; v < kSmpMaxV; ++v) {
            const int k = lane + 32 * v;
            if (v < nv && k < Kp) atomicAdd(gC + (int64_t)cur * Kp + k, acc[v]);
            acc[v] = T(0);
          }
        }
        cur = b;
      }
#pragma unroll
      for (int v = 0; v < kSmpMaxV; ++v) {
        const int k = lane + 32 * v;
        if (v < nv && k < Kp) acc[v] = fma(g, A[(int64_t)a * Kp + k], acc[v]);
      }
    }
    if (cur >= 0) {
#pragma unroll
      for (int v = 0; v < kSmpMaxV; ++v) {
        const int k = lane + 32 * v;
        if (v < nv && k < Kp) atomicAdd(gC + (int64_t)cur * Kp + k, acc[v]);
      }
    }
  }
}

__global__ void k_to_double(const float* __restrict__ src, int64_t n, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

template <typename T>
__global__ void k_from_double(const double* __restrict__ src, int64_t n, T* __restrict__ dst) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

}  // namespace

cudaError_t launch_sampled_order(const int32_t* idx, const Split2* sp, int64_t M, int64_t P_in, int64_t P_out,
                                 const SampledWork& wk, cudaStream_t st) {
  // entries with a bad index are left out of the groups; after the scatter the last cursor
  // holds the number of grouped entries, which the passes read
  cudaError_t e = cudaMemsetAsync(wk.cnt_a, 0, sizeof(uint32_t) * (size_t)P_in, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(wk.cnt_b, 0, sizeof(uint32_t) * (size_t)P_out, st);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)imin((M + 255) / 256, 152 * 16);
  k_smp_keys<<<blocks, 256, 0, st>>>(idx, *sp, M, wk.ka, wk.kb, wk.cnt_a, wk.cnt_b);
  note_launch();
  k_smp_scan<<<2, 1024, 0, st>>>(wk.cnt_a, P_in, wk.cnt_b, P_out, wk.cur_a, wk.cur_b);
  note_launch();
  k_smp_scatter<<<blocks, 256, 0, st>>>(wk.ka, wk.kb, M, wk.cur_a, wk.cur_b, wk.perm_a, wk.perm_b);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_sampled_rows(const void* A, const void* C, bool fp64, int Kp, const void* x, int64_t M,
                                int64_t P_in, double sigma, void* resid, double* loss_part, int parts, bool backward,
                                double g_scale, void* gA, void* gC, const SampledWork& wk, cudaStream_t st) {
  if (Kp > 32 * kSmpMaxV) return cudaErrorInvalidValue;
  if (resid) {
    cudaError_t e = cudaMemsetAsync(resid, 0, (fp64 ? sizeof(double) : sizeof(float)) * (size_t)M, st);
    if (e != cudaSuccess) return e;
  }
  const uint32_t* n_valid = wk.cur_a + (P_in - 1);
  if (fp64)
    k_smp_rows_a<double><<<parts, 256, 0, st>>>((const double*)A, (const double*)C, Kp, wk.perm_a, wk.ka, wk.kb,
                                                (const double*)x, n_valid, sigma, (double*)resid, loss_part,
                                                backward ? 1 : 0, g_scale, (double*)wk.g, (double*)gA);
  else
    k_smp_rows_a<float><<<parts, 256, 0, st>>>((const float*)A, (const float*)C, Kp, wk.perm_a, wk.ka, wk.kb,
                                               (const float*)x, n_valid, sigma, (float*)resid, loss_part,
                                               backward ? 1 : 0, g_scale, (float*)wk.g, (float*)gA);
  note_launch();
  if (backward) {
    if (fp64)
      k_smp_rows_b<double><<<parts, 256, 0, st>>>((const double*)A, Kp, wk.perm_b, wk.ka, wk.kb,
                                                  (const double*)wk.g, n_valid, (double*)gC);
    else
      k_smp_rows_b<float><<<parts, 256, 0, st>>>((const float*)A, Kp, wk.perm_b, wk.ka, wk.kb, (const float*)wk.g,
                                                 n_valid, (float*)gC);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_to_double(const float* src, int64_t n, double* dst, cudaStream_t st) {
  k_to_double<<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(src, n, dst);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_from_double(const double* src, int64_t n, void* dst, bool fp64, cudaStream_t st) {
  if (fp64)
    pdl_launch(k_from_double<double>, dim3((unsigned)imin((n + 255) / 256, 4096)), dim3(256), 0, st, src, n,
               (double*)dst);
  else
    pdl_launch(k_from_double<float>, dim3((unsigned)imin((n + 255) / 256, 4096)), dim3(256), 0, st, src, n,
               (float*)dst);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trd
