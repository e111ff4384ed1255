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
// optional), rows of kpad entries with zero padding.  Products are kept column-major like
// the core slices, so slices are copied with all lanes and no index arithmetic; the FP32
// kernel reads the FP32 core copies when they exist (FP64-to-FP32 conversion, like integer
// division, goes through a unit that issues near the FP64 rate on this GPU).
template <typename Tc>
__device__ __forceinline__ void chain_slice(const Chain& ch, int j, int64_t sl, int n, Tc* dst, int lane) {
  const float* zf = sizeof(Tc) == 4 ? ch.coref[j] : nullptr;
  if (zf) {
    zf += sl * (int64_t)n;
    for (int e = lane; e < n; e += 32) dst[e] = (Tc)zf[e];
  } else {
    const double* z = ch.core[j] + sl * (int64_t)n;
    for (int e = lane; e < n; e += 32) dst[e] = (Tc)z[e];
  }
}

// NC: the chain length as a compile-time constant (1..4; 0 = read from ch.n), so that the
// digit arithmetic stays in registers and the per-core parameters are static operands.
// Per warp: buffer A (capA entries: the first slice, then every other product), buffer B (capP:
// the products of the later slices) and the slice buffer Zs (capZ: the later slices), where
// capP = max_{j>=1} R0 C_j, capZ = max_{j>=1} R_j C_j and capA = max(R0 C_0, capP).
template <typename Tc, typename Tout, int NC>
__global__ void k_chain(Chain ch, Tout* __restrict__ out, int transposed, int64_t ld, int capA, int capP,
                        int capZ, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int kpad) {
  constexpr int JMAX = NC > 0 ? NC : kMaxN;
  const int n = NC > 0 ? NC : ch.n;
  extern __shared__ __align__(16) unsigned char smem_chain[];
  pdl_wait();
  pdl_trigger();
  const int warps = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per_warp = capA + capP + capZ;
  Tc* const bufA = reinterpret_cast<Tc*>(smem_chain) + (size_t)w * per_warp;
  Tc* const bufB = bufA + capA;
  Tc* Zs = bufB + capP;
  // maps shared by every p: output position pos <- column-major entry of the product, and
  // column-major entry e -> (row e mod R0, column e / R0) packed as a | b << 16
  const int R0 = ch.rows[0], CN = ch.cols[n - 1];
  int* tOut = reinterpret_cast<int*>(reinterpret_cast<Tc*>(smem_chain) + (size_t)warps * per_warp);
  int* tAB = tOut + R0 * CN;
  for (int pos = threadIdx.x; pos < R0 * CN; pos += blockDim.x)
    tOut[pos] = transposed ? pos : (pos % CN) * R0 + pos / CN;
  for (int e = threadIdx.x; e < capP; e += blockDim.x) tAB[e] = (e % R0) | (e / R0) << 16;
  __syncthreads();
  // digits of this warp's first p and of the stride between its p's (mixed radix, digit 0
  // fastest), advanced by digit-wise addition with carries
  const int64_t stride = (int64_t)gridDim.x * warps;
  int64_t dig[JMAX], sdig[JMAX];
  {
    int64_t rem = (int64_t)blockIdx.x * warps + w, rs = stride;
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      if (j >= n) break;
      rem = qdivmod(rem, ch.dim[j], dig[j]);
      rs = qdivmod(rs, ch.dim[j], sdig[j]);
    }
  }
  for (int64_t p = (int64_t)blockIdx.x * warps + w; p < ch.count; p += stride) {
    Tc* Mb = bufA;
    Tc* Mn = bufB;
    int C = ch.cols[0];
    // M(a, c) at Mb[c R0 + a]; slice j element (c, b) at Zs[b R_j + c] (the core layout)
    chain_slice(ch, 0, ch.idx[0] ? (int64_t)ch.idx[0][dig[0]] : dig[0], R0 * C, Mb, lane);
    __syncwarp();
#pragma unroll
    for (int j = 1; j < JMAX; ++j) {
      if (j >= n) break;
      const int Rj = ch.rows[j], Cj = ch.cols[j];     // Rj == C
      chain_slice(ch, j, ch.idx[j] ? (int64_t)ch.idx[j][dig[j]] : dig[j], Rj * Cj, Zs, lane);
      __syncwarp();
      for (int e = lane; e < R0 * Cj; e += 32) {
        const int ab = tAB[e], a = ab & 0xffff, b = ab >> 16;
        const Tc* mrow = Mb + a;
        const Tc* zcol = Zs + b * Rj;
        Tc acc = Tc(0);
        for (int c = 0; c < C; ++c) acc = fma(mrow[c * R0], zcol[c], acc);
        Mn[e] = acc;
      }
      __syncwarp();
      Tc* t = Mb; Mb = Mn; Mn = t;
      C = Cj;
    }
    // entry (a, b) goes to position b R0 + a (transposed) or a C + b
    for (int pos = lane; pos < R0 * C; pos += 32) {
      const Tout v = (Tout)Mb[tOut[pos]];
      if (out) out[p * ld + pos] = v;
      if (hi) {
        const float f = (float)v;
        const __nv_bfloat16 vh = bf16_rn(f);
        hi[p * kpad + pos] = vh;
        if (lo) lo[p * kpad + pos] = bf16_rn(f - __bfloat162float(vh));
      }
    }
    if (hi)
      for (int e = R0 * C + lane; e < kpad; e += 32) {
        hi[p * kpad + e] = bf16_rn(0.f);
        if (lo) lo[p * kpad + e] = bf16_rn(0.f);
      }
    __syncwarp();
    int64_t carry = 0;
#pragma unroll
    for (int j = 0; j < JMAX; ++j) {
      if (j >= n) break;
      dig[j] += sdig[j] + carry;
      carry = 0;
      while (dig[j] >= ch.dim[j]) {
        dig[j] -= ch.dim[j];
        ++carry;
      }
    }
  }
}

// out_double: FP64 products and output; otherwise FP32 products and output.
cudaError_t launch_chain(const Chain& ch, void* out, bool out_double, bool transposed,
                         int64_t ld, cudaStream_t st, __nv_bfloat16* hi, __nv_bfloat16* lo, int kpad) {
  if (ch.n <= 0 || ch.count <= 0) return cudaSuccess;
  int capP = 1, capZ = 1;
  for (int j = 1; j < ch.n; ++j) {
    capP = max(capP, ch.rows[0] * ch.cols[j]);
    capZ = max(capZ, ch.rows[j] * ch.cols[j]);
  }
  const int capA = max(capP, ch.rows[0] * ch.cols[0]);
  // a few multi-indices per warp, so that the per-warp set-up is shared; fewer warps per block
  // when the slice products are large (a rank-80 x 80 first slice takes 25.6 KB per warp in
  // FP32)
  const size_t tab = sizeof(int) * ((size_t)ch.rows[0] * ch.cols[ch.n - 1] + capP);
  const size_t esz_max = out_double ? sizeof(double) : sizeof(float);
  const size_t per_warp = (size_t)(capA + capP + capZ) * esz_max;
  const int warps = (int)imax(1, imin(4, (int64_t)((kSmemOptIn - tab) / per_warp)));
  if ((size_t)warps * per_warp + tab > kSmemOptIn) return cudaErrorInvalidValue;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = imax(1, imin((ch.count + warps - 1) / warps, (int64_t)sms * 8));
  auto go = [&](auto kern, size_t esz, auto* o) {
    const size_t smem = (size_t)warps * (capA + capP + capZ) * esz + tab;
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pdl_launch(kern, dim3((unsigned)blocks), dim3(warps * 32), smem, st, ch, o, (int)transposed, ld, capA, capP,
               capZ, hi, lo, kpad);
  };
  if (out_double) {
    double* o = (double*)out;
    switch (ch.n) {
      case 1: go(k_chain<double, double, 1>, sizeof(double), o); break;
      case 2: go(k_chain<double, double, 2>, sizeof(double), o); break;
      case 3: go(k_chain<double, double, 3>, sizeof(double), o); break;
      case 4: go(k_chain<double, double, 4>, sizeof(double), o); break;
      default: go(k_chain<double, double, 0>, sizeof(double), o);
    }
  } else {
    float* o = (float*)out;
    switch (ch.n) {
      case 1: go(k_chain<float, float, 1>, sizeof(float), o); break;
      case 2: go(k_chain<float, float, 2>, sizeof(float), o); break;
      case 3: go(k_chain<float, float, 3>, sizeof(float), o); break;
      case 4: go(k_chain<float, float, 4>, sizeof(float), o); break;
      default: go(k_chain<float, float, 0>, sizeof(float), o);
    }
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
// products of the cores between the block boundary and core k (identity when empty); a
// product of one core is read from the core itself (BcCore) instead of a merged buffer.
// The reduced contraction row s is read from Tm (FP64, [P_stat][Kp]) or, when sl.part is
// given, summed in CTA order from the tensor-core pass's partial slots (FP32, the sum of slots
// c + rb over the CTAs c whose unit range meets stationary block rb = s / BM).  Block (ik, y)
// sums pairs [y P, (y + 1) P); with several splits the last block of ik to finish adds the
// split partials in split order, so the result does not depend on the block schedule.
template <typename T, int UK>
__global__ void k_backcontract(const double* __restrict__ Tm, SlotSrc sl, int Kp, int rows_case, int mr, int mc,
                               const T* __restrict__ pre, int64_t n_pre,
                               const T* __restrict__ post, int64_t n_post, BcCore preC, BcCore postC,
                               int64_t Ik, int rk, int rk1, int64_t pairs_per_split,
                               double* __restrict__ part_out, double* __restrict__ d,
                               unsigned* __restrict__ ctr, int work_bytes, int tab_rb) {
  // one warp per (pre, post) pair; warp-private shared buffers, no block barriers in the
  // pair loop; per-lane accumulators, summed over warps in a fixed order at the end.  The
  // index maps of the small matrix loops (and the CTA range of each stationary block) are
  // tabulated once per block: integer division runs through the conversion unit, whose
  // rate on this GPU is close to the FP64 rate.
  extern __shared__ __align__(16) unsigned char smem_bc[];
  __shared__ int s_last;
  pdl_wait();
  pdl_trigger();
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int szM = mr * mc, szPre = mc * rk, szPost = rk1 * mr, szV = mr * rk;
  const int K = rk * rk1;
  const int per_warp = szM + szPre + szPost + szV;
  T* sM = reinterpret_cast<T*>(smem_bc) + (size_t)w * per_warp;
  T* sPre = sM + szM;
  T* sPost = sPre + szPre;
  T* sV = sPost + szPost;
  int2* tC = reinterpret_cast<int2*>(smem_bc + work_bytes);   // [tab_rb] (first CTA, CTA count)
  int* tM = reinterpret_cast<int*>(tC + tab_rb);              // slot offset of M entry e
  int* tPre = tM + szM;                                       // core offset of Pre entry e
  int* tPost = tPre + szPre;                                  // core offset of Post entry e
  int* tV = tPost + szPost;                                   // (i mc) | a << 16 of V entry e
  int* tU = tV + szV;                                         // (b mr) | a << 16 of U entry e
  for (int e = threadIdx.x; e < szM; e += blockDim.x) {
    const int i = e / mc, j = e % mc;
    tM[e] = rows_case ? j * mr + i : i * mc + j;
  }
  for (int e = threadIdx.x; e < szPre; e += blockDim.x) tPre[e] = (e % rk) * mc + e / rk;
  for (int e = threadIdx.x; e < szPost; e += blockDim.x) tPost[e] = (e % mr) * rk1 + e / mr;
  for (int e = threadIdx.x; e < szV; e += blockDim.x) tV[e] = (e / rk) * mc | (e % rk) << 16;
  for (int e = threadIdx.x; e < K; e += blockDim.x) tU[e] = (e / rk) * mr | (e % rk) << 16;
  const int64_t U = sl.RB * sl.NT, G = sl.G;
  // CTA c covers units [floor(c U / G), floor((c + 1) U / G)); CTAs c0 .. c1 - 1 meet block rb
  auto cta_range = [&](int64_t rb, int& c0o, int& nco) {
    const int64_t ulo = rb * sl.NT, uhi = ulo + sl.NT;
    int64_t c0 = (ulo * G) / U;
    while (c0 > 0 && c0 * U >= (ulo + 1) * G) --c0;
    while ((c0 + 1) * U < (ulo + 1) * G) ++c0;
    int64_t c1 = c0 + 1;
    while (c1 < G && c1 * U < uhi * G) ++c1;
    c0o = (int)c0;
    nco = (int)(c1 - c0);
  };
  for (int rb = threadIdx.x; rb < tab_rb; rb += blockDim.x) {
    int c0, nc;
    cta_range(rb, c0, nc);
    tC[rb] = make_int2(c0, nc);
  }
  __syncthreads();
  const int64_t ik = blockIdx.x;
  const int64_t npairs = n_pre * n_post;
  const int64_t q0 = (int64_t)blockIdx.y * pairs_per_split;
  const int64_t q1 = min(npairs, q0 + pairs_per_split);
  const bool has_pre = pre || preC.core, has_post = post || postC.core;
  const int64_t cs = sl.bm * Kp;
  T acc[UK];                                   // entries lane + 32 u of this warp's sum
#pragma unroll
  for (int u = 0; u < UK; ++u) acc[u] = T(0);
  int64_t ip;
  int64_t iq = qdivmod(q0 + w, n_pre, ip);
  for (int64_t q = q0 + w; q < q1; q += warps) {
    const int64_t s = ip + n_pre * (ik + Ik * iq);
    if (sl.part) {
      int64_t rb, r;
      if (sl.bm_shift >= 0) {
        rb = s >> sl.bm_shift;
        r = s - (rb << sl.bm_shift);
      } else {
        rb = qdivmod(s, sl.bm, r);
      }
      int c0, nc;
      if (rb < tab_rb) {
        const int2 t = tC[rb];
        c0 = t.x;
        nc = t.y;
      } else {
        cta_range(rb, c0, nc);
      }
      const float* src = sl.part + ((c0 + rb) * sl.bm + r) * Kp;
      for (int e = lane; e < szM; e += 32) {
        const float* a = src + tM[e];
        float v = a[0];
        for (int t = 1; t < nc; ++t) v += a[t * cs];
        sM[e] = (T)v;
      }
    } else {
      const double* Ts = Tm + s * (int64_t)Kp;
      for (int e = lane; e < szM; e += 32) sM[e] = (T)Ts[tM[e]];
    }
    if (pre) {
      for (int e = lane; e < szPre; e += 32) sPre[e] = pre[ip * (int64_t)szPre + e];
    } else if (preC.core) {
      // Pre(ip)[j][a] = Z(ip)[j, a], slice stored column-major (mc x rk)
      const int64_t off = (preC.idx ? (int64_t)preC.idx[ip] : ip) * (int64_t)szPre;
      if (sizeof(T) == 4 && preC.coref) {
        for (int e = lane; e < szPre; e += 32) sPre[e] = (T)preC.coref[off + tPre[e]];
      } else {
        for (int e = lane; e < szPre; e += 32) sPre[e] = (T)preC.core[off + tPre[e]];
      }
    }
    if (post) {
      for (int e = lane; e < szPost; e += 32) sPost[e] = post[iq * (int64_t)szPost + e];
    } else if (postC.core) {
      // Post(iq)[b][i] = Z(iq)[b, i], slice stored column-major (rk1 x mr)
      const int64_t off = (postC.idx ? (int64_t)postC.idx[iq] : iq) * (int64_t)szPost;
      if (sizeof(T) == 4 && postC.coref) {
        for (int e = lane; e < szPost; e += 32) sPost[e] = (T)postC.coref[off + tPost[e]];
      } else {
        for (int e = lane; e < szPost; e += 32) sPost[e] = (T)postC.core[off + tPost[e]];
      }
    }
    __syncwarp();
    // V = M * Pre  (mr x rk)
    for (int e = lane; e < szV; e += 32) {
      const int tv = tV[e], imc = tv & 0xffff, a = tv >> 16;
      T v;
      if (has_pre) {
        v = T(0);
        for (int j = 0; j < mc; ++j) v = fma(sM[imc + j], sPre[j * rk + a], v);
      } else {
        v = sM[imc + a];
      }
      sV[e] = v;
    }
    __syncwarp();
    // U = Post * V  (rk1 x rk); lane owns entries e = lane + 32 u (e = beta*rk + alpha)
#pragma unroll
    for (int u = 0; u < UK; ++u) {
      const int e = lane + 32 * u;
      if (e < K) {
        const int tu = tU[e], bmr = tu & 0xffff, a = tu >> 16;
        T v;
        if (has_post) {
          v = T(0);
          for (int i = 0; i < mr; ++i) v = fma(sPost[bmr + i], sV[i * rk + a], v);
        } else {
          v = sV[e];                          // Post = identity: U = V
        }
        acc[u] += v;
      }
    }
    __syncwarp();
    ip += warps;
    while (ip >= n_pre) {
      ip -= n_pre;
      ++iq;
    }
  }
  // fixed-order sum over the warps of the block (reuses the block's work area)
  __syncthreads();
  double* red = reinterpret_cast<double*>(smem_bc);
  const bool split = gridDim.y > 1;
  double* o = split ? part_out + ((int64_t)blockIdx.y * Ik + ik) * K : d + ik * K;
  const int KC = K < 1024 ? K : 1024;          // staged chunk (the work area holds warps x KC)
  for (int base = 0; base < K; base += KC) {
    // stage this chunk of every warp's accumulators
#pragma unroll
    for (int u = 0; u < UK; ++u) {
      const int e = lane + 32 * u;
      if (e >= base && e < base + KC && e < K) red[w * KC + (e - base)] = (double)acc[u];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < KC && base + e < K; e += blockDim.x) {
      double sum = 0.0;
      for (int ww = 0; ww < warps; ++ww) sum += red[ww * KC + e];
      o[base + e] = sum;
    }
    __syncthreads();
  }
  if (!split) return;
  __threadfence();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr + ik, 1u) == gridDim.y - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    double sum = 0.0;
    for (unsigned y = 0; y < gridDim.y; ++y) sum += __ldcg(part_out + ((int64_t)y * Ik + ik) * K + e);
    d[ik * K + e] = sum;
  }
  if (threadIdx.x == 0) ctr[ik] = 0u;
}

// The same back-contraction for K = r_k r_{k+1} > 1024 (two large neighbouring ranks, such as
// the paper's video rank [80, 80, 3, 20]: K = 6400 and 1600): one block of 256 threads per
// (row, split); the K outputs are spread over the block's threads (entry e = t + 256 u, u <
// UW), and the block takes its pairs one after another, staging M(s), Pre and Post in shared
// memory, forming V = M Pre together and then every thread adding its entries of Post V.  The
// index maps (tabulated once per block) and the fixed-order split sum are those of
// k_backcontract.
template <typename T, int UW>
__global__ void __launch_bounds__(256, UW > 8 ? 1 : 4) k_backcontract_wide(
    const double* __restrict__ Tm, SlotSrc sl, int Kp, int rows_case, int mr, int mc, const T* __restrict__ pre,
    int64_t n_pre, const T* __restrict__ post, int64_t n_post, BcCore preC, BcCore postC, int64_t Ik, int rk,
    int rk1, int64_t pairs_per_split, double* __restrict__ part_out, double* __restrict__ d,
    unsigned* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem_bw[];
  __shared__ int s_last;
  pdl_wait();
  pdl_trigger();
  const int t = threadIdx.x, nt = blockDim.x;
  const int szM = mr * mc, szPre = mc * rk, szPost = rk1 * mr, szV = mr * rk;
  const int K = rk * rk1;
  T* sM = reinterpret_cast<T*>(smem_bw);
  T* sPre = sM + szM;
  T* sPost = sPre + szPre;
  T* sV = sPost + szPost;
  int* tM = reinterpret_cast<int*>(sV + szV);
  int* tPre = tM + szM;
  int* tPost = tPre + szPre;
  int* tV = tPost + szPost;
  int* tU = tV + szV;
  for (int e = t; e < szM; e += nt) {
    const int i = e / mc, j = e % mc;
    tM[e] = rows_case ? j * mr + i : i * mc + j;
  }
  for (int e = t; e < szPre; e += nt) tPre[e] = (e % rk) * mc + e / rk;
  for (int e = t; e < szPost; e += nt) tPost[e] = (e % mr) * rk1 + e / mr;
  for (int e = t; e < szV; e += nt) tV[e] = (e / rk) * mc | (e % rk) << 16;
  for (int e = t; e < K; e += nt) tU[e] = (e / rk) * mr | (e % rk) << 16;
  const int64_t U = sl.RB * sl.NT, G = sl.G;
  auto cta_range = [&](int64_t rb, int& c0o, int& nco) {
    const int64_t ulo = rb * sl.NT, uhi = ulo + sl.NT;
    int64_t c0 = (ulo * G) / U;
    while (c0 > 0 && c0 * U >= (ulo + 1) * G) --c0;
    while ((c0 + 1) * U < (ulo + 1) * G) ++c0;
    int64_t c1 = c0 + 1;
    while (c1 < G && c1 * U < uhi * G) ++c1;
    c0o = (int)c0;
    nco = (int)(c1 - c0);
  };
  const int64_t ik = blockIdx.x;
  const int64_t npairs = n_pre * n_post;
  const int64_t q0 = (int64_t)blockIdx.y * pairs_per_split;
  const int64_t q1 = min(npairs, q0 + pairs_per_split);
  const bool has_pre = pre || preC.core, has_post = post || postC.core;
  const int64_t cs = sl.bm * Kp;
  T acc[UW];
#pragma unroll
  for (int u = 0; u < UW; ++u) acc[u] = T(0);
  __syncthreads();
  for (int64_t q = q0; q < q1; ++q) {
    int64_t ip;
    const int64_t iq = qdivmod(q, n_pre, ip);
    const int64_t s = ip + n_pre * (ik + Ik * iq);
    if (sl.part) {
      int64_t r;
      const int64_t rb = qdivmod(s, sl.bm, r);
      int c0, nc;
      cta_range(rb, c0, nc);
      const float* src = sl.part + ((c0 + rb) * sl.bm + r) * Kp;
      for (int e = t; e < szM; e += nt) {
        const float* a = src + tM[e];
        float v = a[0];
        for (int tt = 1; tt < nc; ++tt) v += a[tt * cs];
        sM[e] = (T)v;
      }
    } else {
      const double* Ts = Tm + s * (int64_t)Kp;
      for (int e = t; e < szM; e += nt) sM[e] = (T)Ts[tM[e]];
    }
    if (pre) {
      for (int e = t; e < szPre; e += nt) sPre[e] = pre[ip * (int64_t)szPre + e];
    } else if (preC.core) {
      const int64_t off = (preC.idx ? (int64_t)preC.idx[ip] : ip) * (int64_t)szPre;
      if (sizeof(T) == 4 && preC.coref) {
        for (int e = t; e < szPre; e += nt) sPre[e] = (T)preC.coref[off + tPre[e]];
      } else {
        for (int e = t; e < szPre; e += nt) sPre[e] = (T)preC.core[off + tPre[e]];
      }
    }
    if (post) {
      for (int e = t; e < szPost; e += nt) sPost[e] = post[iq * (int64_t)szPost + e];
    } else if (postC.core) {
      const int64_t off = (postC.idx ? (int64_t)postC.idx[iq] : iq) * (int64_t)szPost;
      if (sizeof(T) == 4 && postC.coref) {
        for (int e = t; e < szPost; e += nt) sPost[e] = (T)postC.coref[off + tPost[e]];
      } else {
        for (int e = t; e < szPost; e += nt) sPost[e] = (T)postC.core[off + tPost[e]];
      }
    }
    __syncthreads();
    // V = M * Pre  (mr x rk)
    for (int e = t; e < szV; e += nt) {
      const int tv = tV[e], imc = tv & 0xffff, a = tv >> 16;
      T v;
      if (has_pre) {
        v = T(0);
        for (int j = 0; j < mc; ++j) v = fma(sM[imc + j], sPre[j * rk + a], v);
      } else {
        v = sM[imc + a];
      }
      sV[e] = v;
    }
    __syncthreads();
    // U = Post * V  (rk1 x rk); thread t owns entries e = t + 256 u (e = beta * rk + alpha)
#pragma unroll
    for (int u = 0; u < UW; ++u) {
      const int e = t + 256 * u;
      if (e < K) {
        const int tu = tU[e], bmr = tu & 0xffff, a = tu >> 16;
        T v;
        if (has_post) {
          v = T(0);
          for (int i = 0; i < mr; ++i) v = fma(sPost[bmr + i], sV[i * rk + a], v);
        } else {
          v = sV[e];
        }
        acc[u] += v;
      }
    }
    __syncthreads();
  }
  const bool split = gridDim.y > 1;
  double* o = split ? part_out + ((int64_t)blockIdx.y * Ik + ik) * K : d + ik * K;
#pragma unroll
  for (int u = 0; u < UW; ++u) {
    const int e = t + 256 * u;
    if (e < K) o[e] = (double)acc[u];
  }
  if (!split) return;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(ctr + ik, 1u) == gridDim.y - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int e = t; e < K; e += nt) {
    double sum = 0.0;
    for (unsigned y = 0; y < gridDim.y; ++y) sum += __ldcg(part_out + ((int64_t)y * Ik + ik) * K + e);
    d[ik * K + e] = sum;
  }
  if (t == 0) ctr[ik] = 0u;
}

cudaError_t launch_backcontract(const void* Tsum_d, int Kp, bool rows_case, int mr, int mc,
                                const void* pre, int64_t n_pre, const void* post,
                                int64_t n_post, int64_t Ik, int rk, int rk1, double* dpart,
                                int nsplit, double* d, unsigned* ctr, bool fp64, cudaStream_t st,
                                const SlotSrc* slots, BcCore preC, BcCore postC) {
  SlotSrc sl = slots ? *slots : SlotSrc{};
  if (sl.part) {
    sl.bm_shift = -1;
    for (int b = 0; b < 31; ++b)
      if (((int64_t)1 << b) == sl.bm) sl.bm_shift = b;
  }
  const int64_t npairs = n_pre * n_post;
  const int64_t per = (npairs + nsplit - 1) / nsplit;
  nsplit = (int)((npairs + per - 1) / per);
  const int threads = 128;
  dim3 grid((unsigned)Ik, (unsigned)nsplit);
  const int per_warp = mr * mc + mc * rk + rk1 * mr + mr * rk;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  const int K = rk * rk1;
  if (K > 1024) {
    // wide form: the K outputs over a block's threads, the staged matrices in shared memory
    if (K > 256 * 32) return cudaErrorInvalidValue;
    const size_t esz_w = fp64 ? sizeof(double) : sizeof(float);
    const int szs = mr * mc + mc * rk + rk1 * mr + mr * rk;
    const size_t smem_w = (size_t)szs * esz_w + sizeof(int) * (size_t)(szs + K) + 16;
    // the packed index maps hold row offsets below 2^16 (M and Post) and columns below 2^15
    if (smem_w > kSmemOptIn || mr * mc > 65535 || rk1 * mr > 65535 || rk > 32767) return cudaErrorInvalidValue;
    auto gow = [&](auto kern, auto tag) -> cudaError_t {
      using E = decltype(tag);
      if (smem_w > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w);
      return pdl_launch(kern, grid, dim3(256), smem_w, st, (const double*)Tsum_d, sl, Kp, rows_case ? 1 : 0, mr, mc,
                        (const E*)pre, n_pre, (const E*)post, n_post, preC, postC, Ik, rk, rk1, per, dpart, d, ctr);
    };
    cudaError_t e;
    if (fp64) e = K <= 256 * 8 ? gow(k_backcontract_wide<double, 8>, 0.0) : gow(k_backcontract_wide<double, 32>, 0.0);
    else e = K <= 256 * 8 ? gow(k_backcontract_wide<float, 8>, 0.0f) : gow(k_backcontract_wide<float, 32>, 0.0f);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  const size_t work = std::max((size_t)(threads / 32) * per_warp * esz,
                               (size_t)(threads / 32) * std::min(K, 1024) * sizeof(double));
  const int tab_rb = (sl.part && sl.RB <= 4096) ? (int)sl.RB : 0;
  const size_t tables = (size_t)tab_rb * 8 + sizeof(int) * (size_t)(mr * mc + mc * rk + rk1 * mr + mr * rk + K);
  const size_t smem = (work + 15) / 16 * 16 + tables;
  const int wb = (int)((work + 15) / 16 * 16);
  auto go = [&](auto kern, auto tag) -> cudaError_t {
    using E = decltype(tag);
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pdl_launch(kern, grid, dim3(threads), smem, st, (const double*)Tsum_d, sl, Kp, rows_case ? 1 : 0, mr, mc,
               (const E*)pre, n_pre, (const E*)post, n_post, preC, postC, Ik, rk, rk1, per, dpart, d, ctr, wb,
               tab_rb);
    return cudaSuccess;
  };
  if (fp64) {
    if (K <= 64) go(k_backcontract<double, 2>, 0.0);
    else if (K <= 256) go(k_backcontract<double, 8>, 0.0);
    else go(k_backcontract<double, 32>, 0.0);
  } else {
    if (K <= 64) go(k_backcontract<float, 2>, 0.0f);
    else if (K <= 256) go(k_backcontract<float, 8>, 0.0f);
    else go(k_backcontract<float, 32>, 0.0f);
  }
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
// Field f of the per-CTA statistics summed by warp f in a fixed order; the objective sum
// (field 2) is also written to `obj` when given (the step report's slot).
__global__ void k_reduce_stats(const double* __restrict__ part, int ctas, double* __restrict__ out,
                               double* __restrict__ obj) {
  pdl_wait();
  pdl_trigger();
  const int f = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0;
  for (int c = lane; c < ctas; c += 32) s += part[(int64_t)c * 8 + f];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    out[f] = s;
    if (f == 2 && obj) *obj = s;
  }
}

cudaError_t launch_reduce_stats(const double* stat_part, int ctas, double* stat_sum,
                                int* /*dstatus*/, cudaStream_t st, double* obj) {
  pdl_launch(k_reduce_stats, dim3(1), dim3(256), 0, st, stat_part, ctas, stat_sum, obj);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reconstruction
// out(a, b) = sum_kappa A[a][kappa] C[b][kappa] = Tr(A(a) C(b)) (Def. 1 via Thm. 1's split);
// optional comparison with a reference tensor accumulates sum (xhat - ref)^2 and sum ref^2.
// X_hat(a, b) = <A[a], C[b]> over 64 x 64 output tiles (rows of A and C staged in shared
// memory, 4 x 4 register micro-tiles, lanes along a so that the output is written
// coalesced), optionally against ref: per-tile partial sums of (x_hat - ref)^2 and ref^2,
// then per-block FP64 partials in err_part[2 block], [2 block + 1].
template <typename T>
__global__ void __launch_bounds__(256) k_reconstruct(const T* __restrict__ A, const T* __restrict__ C,
                                                     int64_t P_in, int64_t P_out, int Kp,
                                                     const float* __restrict__ ref, float* __restrict__ out,
                                                     double* __restrict__ err_part) {
  extern __shared__ __align__(16) unsigned char smem_rec[];
  __shared__ double sh[2][256];
  const int KP1 = Kp | 1;
  T* sA = reinterpret_cast<T*>(smem_rec);   // [64][KP1]
  T* sC = sA + 64 * KP1;                    // [64][KP1]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t na = (P_in + 63) / 64, nb = (P_out + 63) / 64;
  const RowCol stage_rc(tid, 256, Kp);
  double se = 0.0, sr = 0.0;
  for (int64_t t = blockIdx.x; t < na * nb; t += gridDim.x) {
    int64_t ta;
    const int64_t tb = qdivmod(t, na, ta);
    const int64_t a0 = ta * 64, b0 = tb * 64;
    __syncthreads();
    for (RowCol rc = stage_rc; rc.r < 64; rc.next()) {
      const int64_t a = a0 + rc.r, b = b0 + rc.r;
      sA[rc.r * KP1 + rc.c] = a < P_in ? A[a * Kp + rc.c] : T(0);
      sC[rc.r * KP1 + rc.c] = b < P_out ? C[b * Kp + rc.c] : T(0);
    }
    __syncthreads();
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k = 0; k < Kp; ++k) {
      T av[4], cv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sA[(tx + 16 * i) * KP1 + k];
#pragma unroll
      for (int j = 0; j < 4; ++j) cv[j] = sC[(ty + 16 * j) * KP1 + k];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], cv[j], acc[i][j]);
    }
    T tse = T(0), tsr = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t b = b0 + ty + 16 * j;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int64_t a = a0 + tx + 16 * i;
        if (a < P_in && b < P_out) {
          const int64_t l = a + P_in * b;
          const T v = acc[i][j];
          if (out) out[l] = (float)v;
          if (ref) {
            const T r = (T)ref[l];
            const T dv = v - r;
            tse = fma(dv, dv, tse);
            tsr = fma(r, r, tsr);
          }
        }
      }
    }
    se += (double)tse;
    sr += (double)tsr;
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
  const size_t smem = (size_t)2 * 64 * (Kp | 1) * (fp64 ? sizeof(double) : sizeof(float));
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (fp64) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_reconstruct<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_reconstruct<double><<<parts, 256, smem, st>>>((const double*)A, (const double*)C, P_in, P_out, Kp, Xref,
                                                    out, err_part);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_reconstruct<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_reconstruct<float><<<parts, 256, smem, st>>>((const float*)A, (const float*)C, P_in, P_out, Kp, Xref, out,
                                                   err_part);
  }
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
  const int64_t* obase;   // offset in X of fibre o of the sketch (all modes but the first)
  int64_t nouter;         // fibres: numel / sdim[0]
};

// Offset in X of every fibre of the sketch along its first mode: o = overline{i_2 ... i_N}
// (first digit fastest) -> sum_{m >= 1} idx_m(i_m) stride_m.  One thread per fibre.
__global__ void k_gather_base(GatherArgs g, int64_t* __restrict__ obase) {
  pdl_wait();
  pdl_trigger();
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < g.nouter; o += step) {
    int64_t rem = o, full = 0;
    for (int m = 1; m < g.N; ++m) {
      int64_t i;
      rem = qdivmod(rem, g.sdim[m], i);
      full += (g.idx[m] ? (int64_t)g.idx[m][i] : i) * g.fstride[m];
    }
    obase[o] = full;
  }
}

// RStS gather: X_I[l] and the observation bit of sketch entry l (a warp per 32 consecutive
// entries, whose bits one ballot packs; each warp takes GW such words at once so that every
// lane has GW independent loads in flight).  Entry l is position i_1 = l mod s_1 of fibre
// o = l div s_1; the warp divides once per word and steps its lanes across at most a few
// fibres, so consecutive lanes read consecutive positions of X along mode 1 (or its sampled
// indices).
constexpr int GW = 4;
__global__ void k_gather(GatherArgs g) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  const int64_t s1 = g.sdim[0];
  const int32_t* idx1 = g.idx[0];
  for (int64_t wd0 = ((int64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * GW; wd0 < g.words;
       wd0 += (int64_t)gridDim.x * wpb * GW) {
    int64_t full[GW];
    bool live[GW];
#pragma unroll
    for (int q = 0; q < GW; ++q) {
      const int64_t wd = wd0 + q;
      const int64_t l = wd * 32 + lane;
      int64_t r0;
      const int64_t o0 = qdivmod(wd * 32, s1, r0);     // warp-uniform
      int64_t i1 = r0 + lane, o = o0;
      if (s1 >= 32) {
        if (i1 >= s1) { i1 -= s1; ++o; }
      } else {
        int64_t r;
        o += qdivmod(i1, s1, r);
        i1 = r;
      }
      live[q] = wd < g.words && l < g.numel;
      full[q] = live[q] ? g.obase[o] + (idx1 ? (int64_t)idx1[i1] : i1) : 0;
    }
    float xv[GW];
    uint32_t mw[GW];
#pragma unroll
    for (int q = 0; q < GW; ++q) {
      xv[q] = live[q] ? __ldg(g.X + full[q]) : 0.f;
      mw[q] = (live[q] && g.M) ? __ldg(g.M + (full[q] >> 5)) : 0xffffffffu;
    }
#pragma unroll
    for (int q = 0; q < GW; ++q) {
      const int64_t wd = wd0 + q;
      if (live[q]) g.XI[wd * 32 + lane] = xv[q];
      const bool obs = live[q] && ((mw[q] >> (full[q] & 31)) & 1u);
      const unsigned bits = __ballot_sync(0xffffffffu, obs);
      if (lane == 0 && wd < g.words) g.PI[wd] = bits;
    }
  }
}

cudaError_t launch_gather(const float* X, const uint32_t* M, int N, const int64_t* full_dim,
                          const View& v, float* XI, uint32_t* PI, int64_t* obase, cudaStream_t st) {
  GatherArgs g;
  g.X = X; g.M = M; g.N = N; g.numel = v.numel; g.XI = XI; g.PI = PI;
  int64_t stride = 1;
  for (int m = 0; m < N; ++m) {
    g.sdim[m] = v.dim[m];
    g.fstride[m] = stride;
    stride *= full_dim[m];
    g.idx[m] = v.idx[m];
  }
  g.nouter = v.numel / v.dim[0];
  g.obase = obase;
  g.words = (v.numel + 31) / 32;
  const int64_t words_padded = (g.words + 3) / 4 * 4;
  // zero the padding words
  if (words_padded > g.words) {
    cudaError_t e = cudaMemsetAsync(PI + g.words, 0, (words_padded - g.words) * 4, st);
    if (e != cudaSuccess) return e;
  }
  pdl_launch(k_gather_base, dim3((unsigned)imin((g.nouter + 255) / 256, 152 * 8)), dim3(256), 0, st, g, obase);
  note_launch();
  const unsigned blocks = (unsigned)imin((g.words + 8 * GW - 1) / (8 * GW), 152 * 16);
  pdl_launch(k_gather, dim3(blocks), dim3(256), 0, st, g);
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
  const int step = gridDim.x * blockDim.x, e0 = blockIdx.x * blockDim.x + threadIdx.x;
  RowCol rc(e0, step, (int)ld_dst);
  for (int64_t e = e0; e < n; e += step, rc.next()) {
    const int64_t r = rc.r;
    const int c = rc.c;
    const float v = c < Kp ? (float)src[r * ld_src + c] : 0.0f;
    const __nv_bfloat16 h = bf16_rn(v);
    const __nv_bfloat16 l = bf16_rn(v - __bfloat162float(h));
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
