// Subchain merges (Def. 2 / Thm. 1), the back-contraction of the weighted contraction into
// the gradient of one core (Eq. sd / Eq. hatd), RStS gather (Sec. 3.2.2), fixed-order
// reductions and full reconstruction (Def. 1).
#include <algorithm>

#include "trd_internal.cuh"

namespace trd {

// ------------------------------------------------------------------ chain products
// One warp per multi-index p: M = Z_{m0}(i_0) Z_{m1}(i_1) ... (Def. 2 core merging), built
// in shared memory, then written row-major (transposed = false) or column-major
// (transposed = true) into row p of `out` (stride ld; skipped when out is null) and, when
// `hi` is given, as the BF16 tensor-core operand: hi = bf16(v), lo = bf16(v - hi) (lo
// optional), rows of kpad entries with zero padding.
template <typename Tc, typename Tout>
__global__ void k_chain(Chain ch, Tout* __restrict__ out, int transposed, int64_t ld, int cap,
                        __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int kpad) {
  extern __shared__ __align__(16) unsigned char smem_chain[];
  const int warps = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Tc* Mb = reinterpret_cast<Tc*>(smem_chain) + (size_t)w * 3 * cap;
  Tc* Mn = Mb + cap;
  Tc* Zs = Mn + cap;
  for (int64_t p = (int64_t)blockIdx.x * warps + w; p < ch.count; p += (int64_t)gridDim.x * warps) {
    int64_t rem = p;
    int64_t sl[kMaxN];
    for (int j = 0; j < ch.n; ++j) {
      const int64_t i = rem % ch.dim[j];
      rem /= ch.dim[j];
      sl[j] = ch.idx[j] ? (int64_t)ch.idx[j][i] : i;
    }
    int R0 = ch.rows[0], C = ch.cols[0];
    {
      const double* z = ch.core[0] + sl[0] * (int64_t)(R0 * C);
      for (int e = lane; e < R0 * C; e += 32) {
        const int a = e % R0, b = e / R0;     // source is column-major within the slice
        Mb[a * C + b] = (Tc)z[e];
      }
    }
    __syncwarp();
    for (int j = 1; j < ch.n; ++j) {
      const int Rj = ch.rows[j], Cj = ch.cols[j];
      const double* z = ch.core[j] + sl[j] * (int64_t)(Rj * Cj);
      for (int e = lane; e < Rj * Cj; e += 32) {
        const int c = e % Rj, b = e / Rj;
        Zs[c * Cj + b] = (Tc)z[e];
      }
      __syncwarp();
      for (int e = lane; e < R0 * Cj; e += 32) {
        const int a = e / Cj, b = e % Cj;
        Tc acc = Tc(0);
        for (int c = 0; c < C; ++c) acc = fma(Mb[a * C + c], Zs[c * Cj + b], acc);
        Mn[e] = acc;
      }
      __syncwarp();
      Tc* t = Mb; Mb = Mn; Mn = t;
      C = Cj;
      __syncwarp();
    }
    for (int e = lane; e < R0 * C; e += 32) {
      const int a = e / C, b = e % C;
      const int pos = transposed ? b * R0 + a : e;
      const Tout v = (Tout)Mb[e];
      if (out) out[p * ld + pos] = v;
      if (hi) {
        const float f = (float)v;
        const __nv_bfloat16 vh = __float2bfloat16_rn(f);
        hi[p * kpad + pos] = vh;
        if (lo) lo[p * kpad + pos] = __float2bfloat16_rn(f - __bfloat162float(vh));
      }
    }
    if (hi)
      for (int e = R0 * C + lane; e < kpad; e += 32) {
        hi[p * kpad + e] = __float2bfloat16_rn(0.f);
        if (lo) lo[p * kpad + e] = __float2bfloat16_rn(0.f);
      }
    __syncwarp();
  }
}

// out_double: FP64 products and output; otherwise FP32 products and output.
cudaError_t launch_chain(const Chain& ch, void* out, bool out_double, bool transposed,
                         int64_t ld, cudaStream_t st, __nv_bfloat16* hi, __nv_bfloat16* lo, int kpad) {
  if (ch.n <= 0 || ch.count <= 0) return cudaSuccess;
  int cap = 1;
  for (int j = 0; j < ch.n; ++j) {
    cap = max(cap, ch.rows[0] * ch.cols[j]);
    cap = max(cap, ch.rows[j] * ch.cols[j]);
  }
  const int warps = 4;
  int64_t blocks = (ch.count + warps - 1) / warps;
  if (blocks > 65535LL * 8) blocks = 65535LL * 8;
  if (out_double) {
    const size_t smem = (size_t)warps * 3 * cap * sizeof(double);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_chain<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_chain<double, double><<<(unsigned)blocks, warps * 32, smem, st>>>(ch, (double*)out, transposed, ld, cap,
                                                                       hi, lo, kpad);
  } else {
    const size_t smem = (size_t)warps * 3 * cap * sizeof(float);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_chain<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_chain<float, float><<<(unsigned)blocks, warps * 32, smem, st>>>(ch, (float*)out, transposed, ld, cap, hi,
                                                                     lo, kpad);
  }
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ back-contraction
// d(i_k)[alpha, beta] = sum over the other digits of the stationary block of
//   [Post * M(s) * Pre][beta, alpha]
// where M(s) is the r x r matrix held in row s of the reduced weighted contraction
// (ROWS case: Ct[delta, gamma] = T[s][gamma r_c + delta]; COLS case: At[gamma, delta] =
// T[s][gamma r_c + delta]) and s = pre + n_pre (i_k + I_k post).  Pre / Post are the
// products of the cores between the block boundary and core k (identity when empty).
// The reduced contraction row s is read from Tm (FP64, [P_stat][Kp]) or, when sl.part is
// given, summed in CTA order from the tensor-core pass's partial slots (FP32, the sum of slots
// c + rb over the CTAs c whose unit range meets stationary block rb = s / BM).
template <typename T>
__global__ void k_backcontract(const double* __restrict__ Tm, SlotSrc sl, int Kp, int rows_case, int mr, int mc,
                               const T* __restrict__ pre, int64_t n_pre,
                               const T* __restrict__ post, int64_t n_post, int64_t Ik,
                               int rk, int rk1, int64_t pairs_per_split,
                               double* __restrict__ out) {
  // one warp per (pre, post) pair; warp-private shared buffers, no block barriers in the
  // pair loop; per-lane accumulators, summed over warps in a fixed order at the end
  extern __shared__ __align__(16) unsigned char smem_bc[];
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int szM = mr * mc, szPre = mc * rk, szPost = rk1 * mr, szV = mr * rk;
  const int per_warp = szM + szPre + szPost + szV;
  T* sM = reinterpret_cast<T*>(smem_bc) + (size_t)w * per_warp;
  T* sPre = sM + szM;
  T* sPost = sPre + szPre;
  T* sV = sPost + szPost;
  const int64_t ik = blockIdx.x;
  const int K = rk * rk1;
  const int64_t npairs = n_pre * n_post;
  const int64_t q0 = (int64_t)blockIdx.y * pairs_per_split;
  const int64_t q1 = min(npairs, q0 + pairs_per_split);
  T acc[32];
#pragma unroll
  for (int u = 0; u < 32; ++u) acc[u] = T(0);
  for (int64_t q = q0 + w; q < q1; q += warps) {
    const int64_t ip = q % n_pre, iq = q / n_pre;
    const int64_t s = ip + n_pre * (ik + Ik * iq);
    if (sl.part) {
      const int64_t rb = s / sl.bm, r = s % sl.bm;
      const int64_t U = sl.RB * sl.NT, ulo = rb * sl.NT, uhi = (rb + 1) * sl.NT;
      int64_t c0 = (ulo * sl.G) / U;
      while (c0 > 0 && (c0 * U) / sl.G > ulo) --c0;
      while (((c0 + 1) * U) / sl.G <= ulo) ++c0;
      for (int e = lane; e < szM; e += 32) {
        const int i = e / mc, j = e % mc;
        const int q = rows_case ? j * mr + i : i * mc + j;
        double v = 0.0;
        for (int64_t cc = c0; cc < sl.G && (cc * U) / sl.G < uhi; ++cc)
          v += (double)sl.part[((cc + rb) * sl.bm + r) * Kp + q];
        sM[e] = (T)v;
      }
    } else {
      const double* Ts = Tm + s * (int64_t)Kp;
      for (int e = lane; e < szM; e += 32) {
        const int i = e / mc, j = e % mc;
        sM[e] = (T)(rows_case ? Ts[j * mr + i] : Ts[i * mc + j]);
      }
    }
    if (pre)
      for (int e = lane; e < szPre; e += 32) sPre[e] = pre[ip * (int64_t)szPre + e];
    if (post)
      for (int e = lane; e < szPost; e += 32) sPost[e] = post[iq * (int64_t)szPost + e];
    __syncwarp();
    // V = M * Pre  (mr x rk)
    for (int e = lane; e < szV; e += 32) {
      const int i = e / rk, a = e % rk;
      T v;
      if (pre) {
        v = T(0);
        for (int j = 0; j < mc; ++j) v = fma(sM[i * mc + j], sPre[j * rk + a], v);
      } else {
        v = sM[i * mc + a];
      }
      sV[e] = v;
    }
    __syncwarp();
    // U = Post * V  (rk1 x rk); lane owns entries e = lane + 32 u (e = beta*rk + alpha)
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int e = lane + 32 * u;
      if (e < K) {
        const int b = e / rk, a = e % rk;
        T v;
        if (post) {
          v = T(0);
          for (int i = 0; i < mr; ++i) v = fma(sPost[b * mr + i], sV[i * rk + a], v);
        } else {
          v = sV[b * rk + a];
        }
        acc[u] += v;
      }
    }
    __syncwarp();
  }
  // fixed-order sum over the warps of the block (reuses the block's shared memory)
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_bc);
  double* o = out + ((int64_t)blockIdx.y * Ik + ik) * K;
  for (int base = 0; base < K; base += 32 * 32) {
    // stage this chunk of every warp's accumulators
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int e = lane + 32 * u;
      if (e >= base && e < base + 1024 && e < K) red[w * 1024 + (e - base)] = (double)acc[u];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 1024 && base + e < K; e += blockDim.x) {
      double sum = 0.0;
      for (int ww = 0; ww < warps; ++ww) sum += red[ww * 1024 + e];
      o[base + e] = sum;
    }
    __syncthreads();
  }
}

__global__ void k_sum_splits(const double* __restrict__ part, int nsplit, int64_t n,
                             double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nsplit; ++j) s += part[(int64_t)j * n + i];
    out[i] = s;
  }
}

cudaError_t launch_backcontract(const void* Tsum_d, int Kp, bool rows_case, int mr, int mc,
                                const void* pre, int64_t n_pre, const void* post,
                                int64_t n_post, int64_t Ik, int rk, int rk1, double* dpart,
                                int nsplit, double* d, bool fp64, cudaStream_t st, const SlotSrc* slots) {
  const SlotSrc sl = slots ? *slots : SlotSrc{};
  const int64_t npairs = n_pre * n_post;
  const int64_t per = (npairs + nsplit - 1) / nsplit;
  const int threads = 128;
  dim3 grid((unsigned)Ik, (unsigned)nsplit);
  double* target = nsplit == 1 ? d : dpart;
  const int per_warp = mr * mc + mc * rk + rk1 * mr + mr * rk;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  const size_t smem = std::max((size_t)(threads / 32) * per_warp * esz, (size_t)(threads / 32) * 1024 * sizeof(double));
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_backcontract<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_backcontract<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (fp64)
    k_backcontract<double><<<grid, threads, smem, st>>>((const double*)Tsum_d, sl, Kp, rows_case ? 1 : 0, mr, mc,
                                                     (const double*)pre, n_pre, (const double*)post, n_post,
                                                     Ik, rk, rk1, per, target);
  else
    k_backcontract<float><<<grid, threads, smem, st>>>((const double*)Tsum_d, sl, Kp, rows_case ? 1 : 0, mr, mc,
                                                    (const float*)pre, n_pre, (const float*)post, n_post,
                                                    Ik, rk, rk1, per, target);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nsplit == 1) return e;
  const int64_t n = Ik * rk * rk1;
  k_sum_splits<<<(unsigned)imin((n + 255) / 256, 4096), 256, 0, st>>>(dpart, nsplit, n, d);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ fixed-order reductions
template <typename T>
__global__ void k_reduce_T(const T* __restrict__ part, int splits, int64_t n, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < splits; ++j) s += (double)part[(int64_t)j * n + i];
    out[i] = s;
  }
}

cudaError_t launch_reduce_T(const void* Tpart, bool is_double, int splits, int64_t n,
                            double* Tsum, cudaStream_t st) {
  const unsigned blocks = (unsigned)imin((n + 255) / 256, 8192);
  if (is_double) k_reduce_T<double><<<blocks, 256, 0, st>>>((const double*)Tpart, splits, n, Tsum);
  else k_reduce_T<float><<<blocks, 256, 0, st>>>((const float*)Tpart, splits, n, Tsum);
  note_launch();
  return cudaGetLastError();
}

// stat_part[c][8] -> stat_sum[8], fixed order: warp f sums field f (lane-strided partial
// sums, then a fixed shuffle tree).
__global__ void k_reduce_stats(const double* __restrict__ part, int ctas, double* __restrict__ out) {
  const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  for (int c = lane; c < ctas; c += 32) s += part[(int64_t)c * 8 + f];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[f] = s;
}

cudaError_t launch_reduce_stats(const double* stat_part, int ctas, double* stat_sum,
                                int* /*dstatus*/, cudaStream_t st) {
  k_reduce_stats<<<1, 256, 0, st>>>(stat_part, ctas, stat_sum);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reconstruction
// out(a, b) = sum_kappa A[a][kappa] C[b][kappa] = Tr(A(a) C(b)) (Def. 1 via Thm. 1's split);
// optional comparison with a reference tensor accumulates sum (xhat - ref)^2 and sum ref^2.
template <typename T>
__global__ void k_reconstruct(const T* __restrict__ A, const T* __restrict__ C,
                              int64_t P_in, int64_t P_out, int Kp, const float* __restrict__ ref,
                              float* __restrict__ out, double* __restrict__ err_part) {
  __shared__ double sh[2][256];
  double se = 0.0, sr = 0.0;
  const int64_t n = P_in * P_out;
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = l % P_in, b = l / P_in;
    const T* Ar = A + a * Kp;
    const T* Cr = C + b * Kp;
    T v = T(0);
    for (int k = 0; k < Kp; ++k) v = fma(Ar[k], Cr[k], v);
    if (out) out[l] = (float)v;
    if (ref) {
      const double r = (double)ref[l];
      const double dv = (double)v - r;
      se += dv * dv;
      sr += r * r;
    }
  }
  if (!err_part) return;
  sh[0][threadIdx.x] = se;
  sh[1][threadIdx.x] = sr;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    err_part[2 * blockIdx.x] = sh[0][0];
    err_part[2 * blockIdx.x + 1] = sh[1][0];
  }
}

cudaError_t launch_reconstruct_mats(const void* A, const void* C, bool fp64, int64_t P_in, int64_t P_out,
                                    int Kp, const float* Xref, float* out, double* err_part,
                                    int parts, cudaStream_t st) {
  if (fp64)
    k_reconstruct<double><<<parts, 256, 0, st>>>((const double*)A, (const double*)C, P_in, P_out, Kp, Xref, out,
                                                 err_part);
  else
    k_reconstruct<float><<<parts, 256, 0, st>>>((const float*)A, (const float*)C, P_in, P_out, Kp, Xref, out,
                                                err_part);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ RStS gather
// One warp per 32 consecutive sketch entries: each lane maps its sketch multi-index through
// the index sets to the full tensor, copies the value, and the warp packs the mask bits.
struct GatherArgs {
  const float* X;
  const uint32_t* M;
  int N;
  int64_t sdim[kMaxN];
  int64_t fstride[kMaxN];
  const int32_t* idx[kMaxN];
  int64_t numel;
  float* XI;
  uint32_t* PI;
  int64_t words;
};

__global__ void k_gather(GatherArgs g) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t wd = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); wd < g.words;
       wd += (int64_t)gridDim.x * wpb) {
    const int64_t l = wd * 32 + lane;
    bool obs = false;
    if (l < g.numel) {
      int64_t rem = l, full = 0;
      for (int m = 0; m < g.N; ++m) {
        const int64_t i = rem % g.sdim[m];
        rem /= g.sdim[m];
        const int64_t fi = g.idx[m] ? (int64_t)g.idx[m][i] : i;
        full += fi * g.fstride[m];
      }
      g.XI[l] = g.X[full];
      obs = g.M ? ((g.M[full >> 5] >> (full & 31)) & 1u) : true;
    }
    const unsigned bits = __ballot_sync(0xffffffffu, obs);
    if (lane == 0) g.PI[wd] = bits;
  }
}

cudaError_t launch_gather(const float* X, const uint32_t* M, int N, const int64_t* full_dim,
                          const View& v, float* XI, uint32_t* PI, cudaStream_t st) {
  GatherArgs g;
  g.X = X; g.M = M; g.N = N; g.numel = v.numel; g.XI = XI; g.PI = PI;
  int64_t stride = 1;
  for (int m = 0; m < N; ++m) {
    g.sdim[m] = v.dim[m];
    g.fstride[m] = stride;
    stride *= full_dim[m];
    g.idx[m] = v.idx[m];
  }
  g.words = (v.numel + 31) / 32;
  const int64_t words_padded = (g.words + 3) / 4 * 4;
  // zero the padding words
  if (words_padded > g.words) {
    cudaError_t e = cudaMemsetAsync(PI + g.words, 0, (words_padded - g.words) * 4, st);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)imin((g.words + 7) / 8, 152 * 32);
  k_gather<<<blocks, 256, 0, st>>>(g);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ small helpers
__global__ void k_set_scalar(double* p, double v) { *p = v; }

cudaError_t launch_set_scalar(double* p, double v, cudaStream_t st) {
  k_set_scalar<<<1, 1, 0, st>>>(p, v);
  note_launch();
  return cudaGetLastError();
}

// Split a float/double matrix into BF16 hi + lo parts (x ~ hi + lo), optionally with a
// transposed copy of hi ([Kp][rows], stride ldT); columns >= Kp of the destination rows
// are zero-filled up to ld_dst.
template <typename T>
__global__ void k_to_bf16_split(const T* __restrict__ src, int64_t rows, int Kp, int64_t ld_src,
                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                __nv_bfloat16* __restrict__ hiT, int64_t ldT, int64_t ld_dst) {
  const int64_t n = rows * ld_dst;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ld_dst;
    const int c = (int)(e % ld_dst);
    const float v = c < Kp ? (float)src[r * ld_src + c] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    hi[e] = h;
    if (lo) lo[e] = l;
    if (hiT && c < Kp) hiT[(int64_t)c * ldT + r] = h;
  }
}

cudaError_t launch_to_bf16_split(const void* src, bool src_double, int64_t rows, int Kp,
                                 int64_t ld_src, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                 __nv_bfloat16* hiT, int64_t ldT, int64_t ld_dst,
                                 cudaStream_t st) {
  const int64_t n = rows * ld_dst;
  const unsigned blocks = (unsigned)imin((n + 255) / 256, 8192);
  if (src_double)
    k_to_bf16_split<double><<<blocks, 256, 0, st>>>((const double*)src, rows, Kp, ld_src, hi, lo, hiT, ldT, ld_dst);
  else
    k_to_bf16_split<float><<<blocks, 256, 0, st>>>((const float*)src, rows, Kp, ld_src, hi, lo, hiT, ldT, ld_dst);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trd
