// Adaptive kernel width (the paper cites a rule without stating it; reading):
//   sigma = max(1e-6 rms(x_obs), 2 min(std(e), IQR(e) / 1.349), 0.9 sigma_prev)
// over the observed residuals of the full tensor, or of a fixed probe of 2^20 entries.
// Quartiles are type-7 (linear interpolation between order statistics); the order
// statistics come from an exact, deterministic MSB-first radix select on order-preserving
// 64-bit keys (8 passes of 8 bits, integer histograms).
#include <mutex>

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
__device__ inline double dval(uint64_t k) {
  const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

constexpr uint64_t kExcluded = ~0ull;

// Residual e = x - Tr(prod Z_j(i_j)) at probe m (or entry m when full), by the row-vector
// chain: for each gamma, v = e_gamma^T Z_1(i_1) ... Z_N(i_N), x_hat += v[gamma].
template <typename T>
__global__ void k_probe_resid(const double* const* __restrict__ Zp, int N, const int64_t* __restrict__ dim,
                              const int* __restrict__ R, const float* __restrict__ X,
                              const uint32_t* __restrict__ M, int64_t numel, int full, int64_t n,
                              double* __restrict__ vals, uint64_t* __restrict__ keys,
                              double* __restrict__ xsq) {
  __shared__ const double* Zs[kMaxN];
  __shared__ int64_t Ds[kMaxN];
  __shared__ int Rs[kMaxN];
  if (threadIdx.x < N) {
    Zs[threadIdx.x] = Zp[threadIdx.x];
    Ds[threadIdx.x] = dim[threadIdx.x];
    Rs[threadIdx.x] = R[threadIdx.x];
  }
  __syncthreads();
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lin = full ? m : (int64_t)(sm64(kProbeSeed, (uint64_t)m) % (uint64_t)numel);
    const bool obs = M ? ((M[lin >> 5] >> (lin & 31)) & 1u) : true;
    double val = 0.0, xs = 0.0;
    uint64_t key = kExcluded;
    if (obs) {
      int64_t ii[kMaxN];
      int64_t rem = lin;
      for (int j = 0; j < N; ++j) { ii[j] = rem % Ds[j]; rem /= Ds[j]; }
      const int r0 = Rs[0];
      T xh = T(0);
      for (int g = 0; g < r0; ++g) {
        T v[kMaxR], u[kMaxR];
        // v = row g of Z_0(i_0): Z_0(i)[g, b] at i*K + b*r0 + g
        {
          const int r1 = Rs[1 % N];
          const double* z = Zs[0] + ii[0] * (int64_t)(r0 * r1);
          for (int b = 0; b < r1; ++b) v[b] = (T)z[b * r0 + g];
        }
        for (int j = 1; j < N; ++j) {
          const int rj = Rs[j], rj1 = Rs[(j + 1) % N];
          const double* z = Zs[j] + ii[j] * (int64_t)(rj * rj1);
          for (int b = 0; b < rj1; ++b) {
            T s = T(0);
            for (int a = 0; a < rj; ++a) s = fma(v[a], (T)z[b * rj + a], s);
            u[b] = s;
          }
          for (int b = 0; b < rj1; ++b) v[b] = u[b];
        }
        xh += v[g];
      }
      const T x = (T)X[lin];
      const T e = x - xh;
      if (isfinite((double)e)) {
        val = (double)e;
        key = dkey(val);
        xs = (double)x * (double)x;
      }
    }
    vals[m] = key == kExcluded ? 0.0 : val;
    keys[m] = key;
    xsq[m] = xs;
  }
}

// Residual at probe m from the merged subchains of the full tensor: with the modes cut into
// an inner block (linear index a) and an outer block (b), x_hat = Tr(A(a) C(b)) =
// sum_kappa A[a][kappa] C[b][kappa] (Thm. 1 with the ring cut in two).
template <typename T>
__global__ void k_probe_merged(const T* __restrict__ A, const T* __restrict__ C, int Kp, int64_t P_in,
                               const float* __restrict__ X, const uint32_t* __restrict__ M, int64_t numel,
                               int full, int64_t n, double* __restrict__ vals, uint64_t* __restrict__ keys,
                               double* __restrict__ xsq) {
  // one warp per group of 32 probes: lane m owns probe m of the group (index, data, output);
  // the 32 dot products are computed cooperatively with coalesced row loads
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; g0 < n; g0 += warps * 32) {
    const int64_t m = g0 + lane;
    const bool live = m < n;
    const int64_t lin = !live ? 0 : (full ? m : (int64_t)(sm64(kProbeSeed, (uint64_t)m) % (uint64_t)numel));
    const bool obs = live && (M ? ((M[lin >> 5] >> (lin & 31)) & 1u) : true);
    const float xf = live ? X[lin] : 0.f;
    const int64_t a = lin % P_in, b = lin / P_in;
    T mine = T(0);
    for (int q = 0; q < 32; ++q) {
      const int64_t aq = __shfl_sync(0xffffffffu, a, q), bq = __shfl_sync(0xffffffffu, b, q);
      const T* Ar = A + aq * Kp;
      const T* Cr = C + bq * Kp;
      T part = T(0);
      for (int k = lane; k < Kp; k += 32) part = fma(Ar[k], Cr[k], part);
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == q) mine = part;
    }
    if (!live) continue;
    double val = 0.0, xs = 0.0;
    uint64_t key = kExcluded;
    if (obs) {
      const T x = (T)xf;
      const T e = x - mine;
      if (isfinite((double)e)) {
        val = (double)e;
        key = dkey(val);
        xs = (double)x * (double)x;
      }
    }
    vals[m] = key == kExcluded ? 0.0 : val;
    keys[m] = key;
    xsq[m] = xs;
  }
}

__global__ void k_float_keys(const float* __restrict__ r, int64_t n, double* __restrict__ vals,
                             uint64_t* __restrict__ keys, double* __restrict__ xsq) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n;
       m += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)r[m];
    const bool ok = isfinite(v);
    vals[m] = ok ? v : 0.0;
    keys[m] = ok ? dkey(v) : kExcluded;
    xsq[m] = 0.0;
  }
}

// Fixed-order sums over the probe: parts[b][4] = (count, sum e, sum x^2, sum (e - mean)^2).
__global__ void k_probe_sums(const double* __restrict__ vals, const uint64_t* __restrict__ keys,
                             const double* __restrict__ xsq, int64_t n, const double* __restrict__ mean,
                             double* __restrict__ parts) {
  __shared__ double sh[3][256];
  double c = 0, s = 0, q = 0;
  const double mu = mean ? *mean : 0.0;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n;
       m += (int64_t)gridDim.x * blockDim.x) {
    if (keys[m] != kExcluded) {
      c += 1.0;
      if (mean) { const double d = vals[m] - mu; s = fma(d, d, s); }
      else { s += vals[m]; q += xsq[m]; }
    }
  }
  sh[0][threadIdx.x] = c; sh[1][threadIdx.x] = s; sh[2][threadIdx.x] = q;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int f = 0; f < 3; ++f) sh[f][threadIdx.x] += sh[f][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int f = 0; f < 3; ++f) parts[blockIdx.x * 3 + f] = sh[f][0];
}

// work layout (doubles): [0] n, [1] mean, [2] sum x^2, [3] var, [8..11] ranks, [12..15] prefixes
// (as uint64 bits), hist at work + 64 as unsigned long long [4][256], parts at work + 64 + 1024.
__global__ void k_finish_sums(const double* __restrict__ parts, int nb, double* __restrict__ work,
                              int second) {
  // one warp: fixed-order strided partial sums, then a fixed shuffle tree
  const int lane = threadIdx.x;
  double c = 0, s = 0, q = 0;
  for (int b = lane; b < nb; b += 32) { c += parts[b * 3]; s += parts[b * 3 + 1]; q += parts[b * 3 + 2]; }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, o);
    s += __shfl_down_sync(0xffffffffu, s, o);
    q += __shfl_down_sync(0xffffffffu, q, o);
  }
  if (lane != 0) return;
  if (!second) {
    work[0] = c;
    work[1] = c > 0 ? s / c : 0.0;
    work[2] = q;
  } else {
    work[3] = c > 0 ? s / c : 0.0;
  }
}

__global__ void k_select_init(double* __restrict__ work) {
  const double n = work[0];
  uint64_t* u = reinterpret_cast<uint64_t*>(work);
  const double ps[2] = {0.25, 0.75};
  for (int q = 0; q < 2; ++q) {
    double h = (n - 1.0) * ps[q];
    if (h < 0) h = 0;
    const double lo = floor(h);
    const double hi = lo + 1.0 <= n - 1.0 ? lo + 1.0 : lo;
    u[8 + 2 * q] = (uint64_t)lo;
    u[9 + 2 * q] = (uint64_t)hi;
  }
  for (int t = 0; t < 4; ++t) u[12 + t] = 0;
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(work + 64);
  for (int i = 0; i < 1024; ++i) hist[i] = 0;
}

__global__ void k_select_hist(const uint64_t* __restrict__ keys, int64_t n, double* __restrict__ work,
                              int shift) {
  __shared__ unsigned int h[4][256];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint64_t* u = reinterpret_cast<const uint64_t*>(work);
  uint64_t pre[4];
  for (int t = 0; t < 4; ++t) pre[t] = u[12 + t];
  const uint64_t himask = shift >= 56 ? 0ull : (~0ull << (shift + 8));
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n;
       m += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[m];
    if (k == kExcluded) continue;
    const unsigned dig = (unsigned)((k >> shift) & 0xffu);
    for (int t = 0; t < 4; ++t)
      if ((k & himask) == pre[t]) atomicAdd(&h[t][dig], 1u);
  }
  __syncthreads();
  unsigned long long* gh = reinterpret_cast<unsigned long long*>(work + 64);
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
    const unsigned v = (&h[0][0])[i];
    if (v) atomicAdd(&gh[i], (unsigned long long)v);
  }
}

// One warp per target: inclusive scan of the 256 bin counts (8 per lane), find the bin
// holding the target rank, narrow the prefix; then clear the histogram.
__global__ void k_select_pick(double* __restrict__ work, int shift) {
  const int t = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* u = reinterpret_cast<uint64_t*>(work);
  unsigned long long* gh = reinterpret_cast<unsigned long long*>(work + 64);
  if (t < 4) {
    const uint64_t rank = u[8 + t];
    unsigned long long c[8], loc = 0;
    for (int i = 0; i < 8; ++i) { c[i] = gh[t * 256 + lane * 8 + i]; loc += c[i]; }
    unsigned long long incl = loc;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned long long excl = incl - loc;
    // the lane whose range [excl, incl) holds the rank finds the bin
    const bool mine = rank >= excl && rank < incl;
    const unsigned who = __ballot_sync(0xffffffffu, mine);
    if (mine) {
      unsigned long long cum = excl;
      int bin = lane * 8 + 7;
      for (int i = 0; i < 8; ++i) {
        if (cum + c[i] > rank) { bin = lane * 8 + i; break; }
        cum += c[i];
      }
      u[8 + t] = rank - cum;
      u[12 + t] |= ((uint64_t)bin) << shift;
    }
    (void)who;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) gh[i] = 0;
}

__global__ void k_sigma_final(double* __restrict__ work, double rms_override, double sigma_prev,
                              const double* __restrict__ sigma_prev_dev, double* __restrict__ sigma_out) {
  if (sigma_prev_dev) sigma_prev = *sigma_prev_dev;
  const uint64_t* u = reinterpret_cast<const uint64_t*>(work);
  const double n = work[0];
  double q[2];
  const double ps[2] = {0.25, 0.75};
  for (int i = 0; i < 2; ++i) {
    const double a = dval(u[12 + 2 * i]), b = dval(u[13 + 2 * i]);
    double h = (n - 1.0) * ps[i];
    if (h < 0) h = 0;
    const double f = h - floor(h);
    q[i] = f >= 0.5 ? b - (b - a) * (1.0 - f) : a + (b - a) * f;
  }
  const double stdv = sqrt(work[3]);
  const double rms = rms_override >= 0 ? rms_override : (n > 0 ? sqrt(work[2] / n) : 0.0);
  double s = 2.0 * fmin(stdv, (q[1] - q[0]) / 1.349);
  if (!(n > 0)) s = 0.0;
  s = fmax(s, 1e-6 * rms);
  if (sigma_prev > 0 && isfinite(sigma_prev)) s = fmax(s, 0.9 * sigma_prev);
  *sigma_out = s;
}

cudaError_t finish_sigma(const double* vals, const uint64_t* keys, const double* xsq, int64_t n,
                         double rms_override, double sigma_prev, const double* sigma_prev_dev,
                         double* work, double* sigma_out, cudaStream_t st) {
  const int nb = 256;
  double* parts = work + 64 + 1024;
  k_probe_sums<<<nb, 256, 0, st>>>(vals, keys, xsq, n, nullptr, parts);
  note_launch();
  k_finish_sums<<<1, 32, 0, st>>>(parts, nb, work, 0);
  note_launch();
  k_probe_sums<<<nb, 256, 0, st>>>(vals, keys, xsq, n, work + 1, parts);
  note_launch();
  k_finish_sums<<<1, 32, 0, st>>>(parts, nb, work, 1);
  note_launch();
  k_select_init<<<1, 1, 0, st>>>(work);
  note_launch();
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    k_select_hist<<<(unsigned)imin((n + 255) / 256, 512), 256, 0, st>>>(keys, n, work, shift);
    note_launch();
    k_select_pick<<<1, 256, 0, st>>>(work, shift);
    note_launch();
  }
  k_sigma_final<<<1, 1, 0, st>>>(work, rms_override, sigma_prev, sigma_prev_dev, sigma_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

size_t sigma_work_doubles() { return 64 + 1024 + 256 * 3 + 64; }

cudaError_t launch_probe_sigma(const double* const* Zdev_ptrs, int N, const int64_t* dim_dev,
                               const int* R_dev, const float* X, const uint32_t* M, int64_t numel,
                               bool fp64, double sigma_prev, const double* sigma_prev_dev,
                               double* vals, uint64_t* keys, double* xsq, double* work,
                               double* sigma_out, cudaStream_t st) {
  const bool full = numel <= kProbeMax;
  const int64_t n = full ? numel : kProbeMax;
  const unsigned blocks = (unsigned)imin((n + 127) / 128, 152 * 16);
  if (fp64)
    k_probe_resid<double><<<blocks, 128, 0, st>>>(Zdev_ptrs, N, dim_dev, R_dev, X, M, numel, full, n, vals, keys, xsq);
  else
    k_probe_resid<float><<<blocks, 128, 0, st>>>(Zdev_ptrs, N, dim_dev, R_dev, X, M, numel, full, n, vals, keys, xsq);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish_sigma(vals, keys, xsq, n, -1.0, sigma_prev, sigma_prev_dev, work, sigma_out, st);
}

cudaError_t launch_probe_sigma_merged(const void* A, const void* C, bool fp64, int Kp, int64_t P_in,
                                      const float* X, const uint32_t* M, int64_t numel, double sigma_prev,
                                      const double* sigma_prev_dev, double* vals, uint64_t* keys, double* xsq,
                                      double* work, double* sigma_out, cudaStream_t st) {
  const bool full = numel <= kProbeMax;
  const int64_t n = full ? numel : kProbeMax;
  const unsigned blocks = (unsigned)imin((n + 255) / 256, 152 * 8);
  if (fp64)
    k_probe_merged<double><<<blocks, 256, 0, st>>>((const double*)A, (const double*)C, Kp, P_in, X, M, numel, full, n,
                                                   vals, keys, xsq);
  else
    k_probe_merged<float><<<blocks, 256, 0, st>>>((const float*)A, (const float*)C, Kp, P_in, X, M, numel, full, n,
                                                  vals, keys, xsq);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish_sigma(vals, keys, xsq, n, -1.0, sigma_prev, sigma_prev_dev, work, sigma_out, st);
}

cudaError_t launch_sigma_from_floats(const float* r, int64_t n, double x_obs_rms, double sigma_prev,
                                     double* vals, uint64_t* keys, double* xsq, double* work,
                                     double* sigma_out, cudaStream_t st) {
  k_float_keys<<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(r, n, vals, keys, xsq);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return finish_sigma(vals, keys, xsq, n, x_obs_rms, sigma_prev, nullptr, work, sigma_out, st);
}

// ------------------------------------------------------------------ allocation-free variant
// Fixed scratch for trd_sigma_from_residuals_noalloc: room for NOALLOC_MAX residuals (values,
// order keys and a zero x^2 column, 8 bytes each) plus the selection work area.  It is a
// file-scope device array, so every GPU that loads the library holds it (about 24 MB) until
// the process exits; all calls share it.
constexpr int64_t NOALLOC_MAX = int64_t(1) << 20;
constexpr size_t NOALLOC_WORK = 64 + 1024 + 256 * 3 + 64;   // doubles; equals sigma_work_doubles()
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_MAX * 24 + NOALLOC_WORK * 8];

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
  double* vals = reinterpret_cast<double*>(b);
  uint64_t* keys = reinterpret_cast<uint64_t*>(b + NOALLOC_MAX * 8);
  double* xsq = reinterpret_cast<double*>(b + NOALLOC_MAX * 16);
  double* work = reinterpret_cast<double*>(b + NOALLOC_MAX * 24);
  // every scratch word the selection reads is written first in this call (the histogram is
  // cleared by the selection's own initialisation), so stale contents do not leak in
  const cudaError_t e = launch_sigma_from_floats(resid_dev, n, x_obs_rms, sigma_prev, vals, keys, xsq, work,
                                                 sigma_out_dev, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TRD_ECUDA;
  }
  return TRD_OK;
}
