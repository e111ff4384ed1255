// Uniform row sampling of the subchain unfolding (the paper's "uniform row sampling"
// ablation, Sec. 5): J sampled multi-indices j over the modes other than k give
//   X_{I[k]}(i, j) = X(j with i_k = i)               (fibres along mode k)
//   B(j)[alpha + beta r_k] = S(j)[beta, alpha],  S(j) = Z_{k+1}(i_{k+1}) ... Z_{k-1}(i_{k-1})
// so that X_hat = Z_{k(2)} B^T (Thm. 1) and the gradient T = Y B is d itself.  These feed the
// same fused data passes as the RStS sketch, with the stationary operand Z_{k(2)}.
#include "trd_internal.cuh"

namespace trd {

namespace {

// Fibre gather: position p = i + I_k j of the I_k x J sample, linear order; one packed
// observation bit per position (ballot over 32 consecutive positions).
__global__ void k_gather_rows(const float* __restrict__ X, const uint32_t* __restrict__ M, RowsArgs a,
                              const int32_t* __restrict__ rows, float* __restrict__ XI, uint32_t* __restrict__ PI) {
  const int64_t n = a.Ik * a.J;
  const int64_t nwarp_pos = (n + 31) / 32 * 32;
  const int lane = threadIdx.x & 31;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nwarp_pos;
       p += (int64_t)gridDim.x * blockDim.x) {
    bool bit = false;
    if (p < n) {
      int64_t i;
      const int64_t j = qdivmod(p, a.Ik, i);
      int64_t lin = i * a.stride[a.k];
      for (int m = 0; m < a.N; ++m)
        if (m != a.k) lin += (int64_t)rows[j * a.N + m] * a.stride[m];
      XI[p] = X[lin];
      bit = M ? ((M[lin >> 5] >> (lin & 31)) & 1u) : true;
    }
    const uint32_t word = __ballot_sync(0xffffffffu, bit);
    if (lane == 0 && p < n) PI[p >> 5] = word;
  }
}

// B(j): one warp per sampled row; the running product (r_{k+1} x r_m, at most CAP = max r^2
// entries, column-major like the core slices), its successor and the next core slice live
// in the warp's shared-memory buffers.  Slices are copied with all lanes and no index
// arithmetic; the FP32 kernel reads the FP32 core copies.
template <typename T>
__device__ __forceinline__ void rows_slice(const RowsArgs& a, int m, int64_t i, int n, T* dst, int lane) {
  const float* zf = sizeof(T) == 4 ? a.Zf[m] : nullptr;
  if (zf) {
    for (int e = lane; e < n; e += 32) dst[e] = (T)zf[i * n + e];
  } else {
    for (int e = lane; e < n; e += 32) dst[e] = (T)a.Z[m][i * n + e];
  }
}

template <typename T>
__global__ void k_rows_chain(RowsArgs a, const int32_t* __restrict__ rows, T* __restrict__ B, int CAP) {
  extern __shared__ __align__(16) unsigned char smem_rows[];
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* cur = reinterpret_cast<T*>(smem_rows) + (size_t)w * 3 * CAP;
  T* nxt = cur + CAP;
  T* zs = nxt + CAP;
  const int N = a.N, k = a.k;
  const int rk = a.R[k], rk1 = a.R[(k + 1) % N];
  for (int64_t j = (int64_t)blockIdx.x * warps + w; j < a.J; j += (int64_t)gridDim.x * warps) {
    // first slice: Z_{k+1}(i), r_{k+1} x r_{k+2}; element (t, c) at c r_{k+1} + t
    int m = (k + 1) % N;
    const int rows_cur = a.R[m];
    int cols_cur = a.R[(m + 1) % N];
    rows_slice(a, m, (int64_t)rows[j * N + m], rows_cur * cols_cur, cur, lane);
    __syncwarp();
    for (int q = 2; q < N; ++q) {
      m = (k + q) % N;
      const int rm = a.R[m], rm1 = a.R[(m + 1) % N];     // rm == cols_cur
      rows_slice(a, m, (int64_t)rows[j * N + m], rm * rm1, zs, lane);
      __syncwarp();
      for (int c = 0; c < rm1; ++c)
        for (int t = lane; t < rows_cur; t += 32) {
          T s = T(0);
          for (int u = 0; u < rm; ++u) s = fma(cur[u * rows_cur + t], zs[c * rm + u], s);
          nxt[c * rows_cur + t] = s;
        }
      __syncwarp();
      T* tmp = cur; cur = nxt; nxt = tmp;
      cols_cur = rm1;
    }
    // S(j) is r_{k+1} x r_k, S[beta][alpha] at alpha r_{k+1} + beta: B[j][alpha + beta r_k]
    T* out = B + j * (int64_t)(rk * rk1);
    for (int beta = 0; beta < rk1; ++beta)
      for (int alpha = lane; alpha < rk; alpha += 32) out[alpha + beta * rk] = cur[alpha * rk1 + beta];
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_gather_rows(const float* X, const uint32_t* M, const RowsArgs& a, const int32_t* rows, float* XI,
                               uint32_t* PI, cudaStream_t st) {
  const int64_t n = a.Ik * a.J;
  k_gather_rows<<<(unsigned)imin((n + 255) / 256, 8192), 256, 0, st>>>(X, M, a, rows, XI, PI);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_rows_chain(const RowsArgs& a, const int32_t* rows, void* B, bool fp64, cudaStream_t st) {
  const int warps = 4;
  const unsigned blocks = (unsigned)imin((a.J + warps - 1) / warps, 65535);
  int rmax = 1;
  for (int m = 0; m < a.N; ++m) rmax = (int)imax(rmax, a.R[m]);
  const int cap = rmax * rmax;
  const size_t per = (size_t)3 * cap;
  if (fp64) {
    const size_t smem = warps * per * sizeof(double);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_rows_chain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_rows_chain<double><<<blocks, warps * 32, smem, st>>>(a, rows, (double*)B, cap);
  } else {
    const size_t smem = warps * per * sizeof(float);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_rows_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_rows_chain<float><<<blocks, warps * 32, smem, st>>>(a, rows, (float*)B, cap);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace trd
