// Fused data passes on CUDA cores (FP32 and FP64 paths).
//
// The (sketched) tensor is viewed as a column-major matrix X(a, b), a over the inner modes
// 0..c-1 and b over the outer modes c..N-1, with X_hat(a, b) = Tr(A(a) C(b)) where A and C
// are the merged subchains of the two blocks (Def. 2; Thm. 1 with the ring cut in two).
// Row kappa of the merged matrices holds A(a)[gamma, delta] / C(b)[delta, gamma] at
// kappa = gamma r_c + delta, so X_hat = S_st S_str^T is a plain dense contraction.
//
// Pass 1 (Eq. updatew + Eq. hatd): per slot e = x - x_hat, w = exp(-e^2 / 2 sigma^2),
//   y = w e on observed slots, and T(s) += sum_t y(s, t) S_str(t) for the stationary
//   index s (the block that contains the updated core).  W is never stored.
// Pass 2 (exact line search of Sec. 3.2): recompute w from the same residuals and
//   accumulate den = sum_obs w (h B^T)^2, with h B^T = S_h S_str^T.
//
// CTA tile: 64 stationary x 64 streaming slots, 256 threads, 4x4 register micro-tiles;
// each CTA keeps its 64 stationary rows resident and streams a contiguous range of
// streaming tiles.  Partial contractions and statistics are written per CTA and reduced
// in a fixed order (no atomics), so results are bitwise reproducible.
#include <type_traits>

#include "trd_internal.cuh"

namespace trd {

namespace {
constexpr int BM = 64, BN = 64, NT = 256;

__device__ __forceinline__ float texp(float x) { return expf(x); }
__device__ __forceinline__ double texp(double x) { return exp(x); }


// cp.async copies into shared memory; src_bytes below the copy size zero-fill the rest (0:
// nothing is read)
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
               "l"(gsrc), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int XLD = 80;   // X tile line stride (floats): 16-byte rows, the two half-warps on disjoint banks

// On the FP32 path with K' <= 128 the X tile, its mask words and the streaming operand are
// double-buffered: the next tile's are prefetched by cp.async during the current one.
// Otherwise (two copies of the wider rows do not fit) one X buffer is filled at the start of
// each tile, behind the reconstruction arithmetic, and the streaming operand is loaded
// directly.
template <typename T>
__host__ __device__ constexpr bool simt_dbt(int Kp) { return sizeof(T) == 4 && Kp <= 128; }

// Row stride of the operand tiles in shared memory: whole 16-byte chunks (vector loads along
// K'), an odd number of them, so that 16 consecutive rows read at one K' offset fall on
// distinct banks; the padding columns hold zeros.
template <typename T>
__host__ __device__ constexpr int simt_kpad(int Kp) {
  const int U = 16 / (int)sizeof(T);
  const int k = (Kp + U - 1) / U * U;
  return ((k / U) % 2 == 0) ? k + U : k;
}
constexpr int SYLD = BN + 4;   // weighted-residual rows: 16-byte aligned, two rows on distinct banks

// Shared-memory bytes of one CTA (the layout of k_pass_simt).
template <typename T>
__host__ __device__ constexpr size_t simt_smem(int Kp, bool rows, bool pass2) {
  const int KPAD = simt_kpad<T>(Kp);
  const int syld = SYLD;
  const int bufs = simt_dbt<T>(Kp) ? 2 : 1;
  return (size_t)((pass2 ? 2 : 1) * BM * KPAD + bufs * BN * KPAD + (pass2 ? 0 : BM * syld)) * sizeof(T) +
         (size_t)bufs * BN * XLD * sizeof(float) + (size_t)bufs * 256 * sizeof(uint32_t);
}

// KM: groups of 16 U-wide column chunks of the contraction per thread (U = 16 / sizeof(T)).
template <typename T, int KM, bool ROWS, bool PASS2>
__global__ void __launch_bounds__(NT) k_pass_simt(const PassArgs p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int U = 16 / sizeof(T);
  const int Kp = p.Kp;
  const bool DBT = simt_dbt<T>(Kp);
  const int KPAD = simt_kpad<T>(Kp);
  // X tiles and mask words of the next streaming tile are prefetched by cp.async while the
  // current one is computed (line L of a tile: streaming index L (ROWS) or stationary index L,
  // 64 consecutive entries of X along it; its mask bits come as 3 words and a bit offset)
  const int nbuf = DBT ? 2 : 1;
  float* sX = reinterpret_cast<float*>(smraw);                      // [nbuf][BN][XLD]
  uint32_t* sMk = reinterpret_cast<uint32_t*>(sX + nbuf * BN * XLD); // [nbuf][64][4]
  T* sS = reinterpret_cast<T*>(sMk + nbuf * 256);                   // [BM][KPAD] stationary rows
  T* sH = sS + BM * KPAD;                                        // [BM][KPAD] with h (pass 2)
  T* sT0 = PASS2 ? sH + BM * KPAD : sS + BM * KPAD;              // [DBT ? 2 : 1][BN][KPAD]
  T* sY = sT0 + (DBT ? 2 : 1) * BN * KPAD;                       // [BM][SYLD] weighted residuals
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t s0 = (int64_t)blockIdx.x * BM;
  const T* Sst = reinterpret_cast<const T*>(p.Sst);
  const T* Sh = reinterpret_cast<const T*>(p.Sh);
  const T* Sstr = reinterpret_cast<const T*>(p.Sstr);
  const int64_t nwords = (p.P_in * (ROWS ? p.P_strm : p.P_stat) + 31) / 32;
  const bool vec = (p.P_in & 3) == 0;   // 16-byte X rows

  for (RowCol rc(tid, NT, KPAD); rc.r < BM; rc.next()) {
    const int r = rc.r, c = rc.c;
    const int64_t s = s0 + r;
    const bool in = s < p.P_stat && c < Kp;
    sS[r * KPAD + c] = in ? Sst[s * p.ld + c] : T(0);
    if (PASS2) sH[r * KPAD + c] = in ? Sh[s * p.ld + c] : T(0);
  }
  const double sig = *p.sigma;
  const T inv2s2 = isinf(sig) ? T(0) : T(1.0 / (2.0 * sig * sig));

  // gradient accumulators: rows ty + 16 i, columns U (tx + 16 m) + u
  T tacc[4][KM * U];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < KM * U; ++j) tacc[i][j] = T(0);
  // statistics: FP32 partial sums per tile (FP64 for the FP64 path), integer counts, widened
  // and added into FP64 once per tile
  double st_w = 0, st_e2 = 0, st_we2 = 0, st_den = 0;
  int64_t st_obs = 0, st_nf = 0, st_slots = 0;
  const RowCol tile_rc(tid, NT, KPAD);
  const int nchunk = KPAD / U;                   // 16-byte chunks per operand row
  const bool vecT = (p.ld % U) == 0;             // streaming rows 16-byte aligned in memory
  const int64_t s_valid = imin(BM, p.P_stat - s0);

  const int64_t ntiles = (p.P_strm + BN - 1) / BN;
  const int64_t tb = (int64_t)blockIdx.y * p.tiles_per_split;
  const int64_t te = imin(ntiles, tb + p.tiles_per_split);

  // streaming rows t0 .. t0 + 63 into dst [BN][KPAD] (zeros beyond P_strm and beyond K')
  auto load_T = [&](int64_t t0, T* dst, bool async) {
    if (async && vecT) {
      for (int q = tid; q < BN * nchunk; q += NT) {
        const int r = q / nchunk, c = (q - r * nchunk) * U;
        const int64_t t = t0 + r;
        const int nv = (t < p.P_strm) ? (int)imax(0, imin(U, Kp - c)) : 0;
        cp_async16(dst + r * KPAD + c, nv > 0 ? Sstr + t * p.ld + c : Sstr, nv * (int)sizeof(T));
      }
      return;
    }
    for (RowCol rc = tile_rc; rc.r < BN; rc.next()) {
      const int64_t t = t0 + rc.r;
      const bool in = t < p.P_strm && rc.c < Kp;
      if (async) {
        const T* src = in ? Sstr + t * p.ld + rc.c : Sstr;
        if (sizeof(T) == 4) cp_async4(dst + rc.r * KPAD + rc.c, src, in ? 4 : 0);
        else cp_async8(dst + rc.r * KPAD + rc.c, src, in ? 8 : 0);
      } else {
        dst[rc.r * KPAD + rc.c] = in ? Sstr[t * p.ld + rc.c] : T(0);
      }
    }
  };
  auto issue = [&](int64_t tile, int buf) {
    const int64_t t0 = tile * BN;
    const int64_t t_valid = imin(BN, p.P_strm - t0);
    const int64_t lines = ROWS ? t_valid : s_valid, along = ROWS ? s_valid : t_valid;
    float* dx = sX + buf * BN * XLD;
    if (vec) {
      for (int q = tid; q < BN * 16; q += NT) {
        const int L = q >> 4, e = (q & 15) * 4;
        if (L < lines) {
          const int64_t base = ROWS ? s0 + p.P_in * (t0 + L) : t0 + p.P_in * (s0 + L);
          const int nv = (int)imax(0, imin(4, along - e));
          cp_async16(dx + L * XLD + e, nv > 0 ? p.X + base + e : p.X, nv * 4);
        }
      }
    } else {
      for (int q = tid; q < BN * 64; q += NT) {
        const int L = q >> 6, e = q & 63;
        if (L < lines && e < along) {
          const int64_t base = ROWS ? s0 + p.P_in * (t0 + L) : t0 + p.P_in * (s0 + L);
          cp_async4(dx + L * XLD + e, p.X + base + e, 4);
        }
      }
    }
    if (p.M) {
      const int L = tid >> 2, k = tid & 3;
      if (L < lines) {
        const int64_t base = ROWS ? s0 + p.P_in * (t0 + L) : t0 + p.P_in * (s0 + L);
        uint32_t* dm = sMk + buf * 256 + tid;
        if (k < 3) {
          const int64_t w = (base >> 5) + k;
          if (w < nwords) cp_async4(dm, p.M + w, 4);
        } else {
          *dm = (uint32_t)(base & 31);
        }
      }
    }
    if (DBT) load_T(t0, sT0 + buf * BN * KPAD, true);
  };

  if (DBT) {
    issue(tb, 0);
    cp_async_commit();
  }
  for (int64_t tile = tb; tile < te; ++tile) {
    const int buf = DBT ? (int)((tile - tb) & 1) : 0;
    const int64_t t0 = tile * BN;
    if (DBT) {
      if (tile + 1 < te) issue(tile + 1, buf ^ 1);
    } else {
      issue(tile, 0);
    }
    cp_async_commit();
    T* sT = sT0 + buf * BN * KPAD;
    if (DBT) cp_async_wait1();
    else load_T(t0, sT, false);
    __syncthreads();
    // micro-tile: the thread index that runs along the memory-contiguous direction of X
    // is tx, so the X tile is read from shared memory without bank conflicts
    T acc[4][4], dacc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { acc[i][j] = T(0); dacc[i][j] = T(0); }
    // 16-byte loads along K' (U values per load; the zero padding adds nothing)
    for (int k = 0; k < KPAD; k += U) {
      V sv[4], hv[4], tv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = ROWS ? tx + 16 * i : ty + 16 * i;
        sv[i] = *reinterpret_cast<const V*>(sS + r * KPAD + k);
        if (PASS2) hv[i] = *reinterpret_cast<const V*>(sH + r * KPAD + k);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = ROWS ? ty + 16 * j : tx + 16 * j;
        tv[j] = *reinterpret_cast<const V*>(sT + c * KPAD + k);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const T* a = reinterpret_cast<const T*>(&sv[i]);
          const T* b = reinterpret_cast<const T*>(&tv[j]);
#pragma unroll
          for (int u = 0; u < U; ++u) acc[i][j] = fma(a[u], b[u], acc[i][j]);
          if (PASS2) {
            const T* hh = reinterpret_cast<const T*>(&hv[i]);
#pragma unroll
            for (int u = 0; u < U; ++u) dacc[i][j] = fma(hh[u], b[u], dacc[i][j]);
          }
        }
    }
    if (!DBT) {
      cp_async_wait0();
      __syncthreads();
    }
    const float* xt = sX + buf * BN * XLD;
    const uint32_t* mk = sMk + buf * 256;
    T tw = T(0), te2 = T(0), twe2 = T(0), tden = T(0);
    int tobs = 0, tnf = 0, tslots = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = ROWS ? tx + 16 * i : ty + 16 * i;
        const int c = ROWS ? ty + 16 * j : tx + 16 * j;
        const int64_t s = s0 + r, t = t0 + c;
        T y = T(0);
        if (s < p.P_stat && t < p.P_strm) {
          const int L = ROWS ? c : r, e = ROWS ? r : c;
          bool obs = true;
          if (p.M) {
            const int q = (int)mk[L * 4 + 3] + e;
            obs = (mk[L * 4 + (q >> 5)] >> (q & 31)) & 1u;
          }
          ++tslots;
          if (obs) {
            ++tobs;
            const T ev = (T)xt[L * XLD + e] - acc[i][j];
            if (isfinite(ev)) {
              const T w = texp(-ev * ev * inv2s2);
              if (PASS2) {
                tden = fma(w * dacc[i][j], dacc[i][j], tden);
              } else {
                y = w * ev;
                tw += w;
                te2 = fma(ev, ev, te2);
                twe2 = fma(y, ev, twe2);
              }
            } else {
              ++tnf;
            }
          }
        }
        if (!PASS2) sY[r * SYLD + c] = y;
      }
    st_slots += tslots;
    st_obs += tobs;
    st_nf += tnf;
    if (PASS2) {
      st_den += (double)tden;
    } else {
      st_w += (double)tw;
      st_e2 += (double)te2;
      st_we2 += (double)twe2;
    }
    if (!PASS2) {
      __syncthreads();
      // T(s, c) += sum_t Y(s, t) S_str(t, c): rows s = ty + 16 i, columns U (tx + 16 m) + u,
      // U streaming indices per step (vector loads of Y rows and of S_str column chunks)
      for (int tt = 0; tt < BN; tt += U) {
        V yv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) yv[i] = *reinterpret_cast<const V*>(sY + (ty + 16 * i) * SYLD + tt);
#pragma unroll
        for (int q = 0; q < U; ++q) {
#pragma unroll
          for (int m = 0; m < KM; ++m) {
            const int c = U * (tx + 16 * m);
            V cv;
            if (c < KPAD) cv = *reinterpret_cast<const V*>(sT + (tt + q) * KPAD + c);
            else cv = V{};
            const T* cc = reinterpret_cast<const T*>(&cv);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const T y = reinterpret_cast<const T*>(&yv[i])[q];
#pragma unroll
              for (int u = 0; u < U; ++u) tacc[i][m * U + u] = fma(y, cc[u], tacc[i][m * U + u]);
            }
          }
        }
      }
    }
    __syncthreads();   // this tile's buffers are refilled by the next iteration
  }
  if (!PASS2) {
    T* Tp = reinterpret_cast<T*>(p.Tpart) + (int64_t)blockIdx.y * p.P_stat * Kp;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t s = s0 + ty + 16 * i;
#pragma unroll
      for (int m = 0; m < KM; ++m)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int c = U * (tx + 16 * m) + u;
          if (s < p.P_stat && c < Kp) Tp[s * Kp + c] = tacc[i][m * U + u];
        }
    }
  }
  // fixed-order block reduction of the statistics
  __shared__ double red[7][NT / 32];
  double v[7] = {st_w, st_e2, st_we2, (double)st_obs, (double)st_nf, (double)st_slots, st_den};
#pragma unroll
  for (int f = 0; f < 7; ++f) {
    double x = v[f];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((tid & 31) == 0) red[f][tid >> 5] = x;
  }
  __syncthreads();
  if (tid < 7) {
    double x = 0.0;
    for (int w = 0; w < NT / 32; ++w) x += red[tid][w];
    p.stat_part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + tid] = x;
  }
  if (tid == 7) p.stat_part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + 7] = 0.0;
}

// Resident CTAs per SM of the pass-1 kernel (registers and shared memory), for the grid size.
template <typename T, int KM>
int blocks_per_sm_kj(int Kp, bool rows) {
  const size_t smem = simt_smem<T>(Kp, rows, false);
  int n = 0;
  auto q = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NT, smem) != cudaSuccess) n = 0;
  };
  if (rows) q(k_pass_simt<T, KM, true, false>);
  else q(k_pass_simt<T, KM, false, false>);
  cudaGetLastError();
  return n > 0 ? n : 1;
}

template <typename T, int KM>
cudaError_t launch_kj(const PassArgs& a, bool rows, bool pass2, dim3 grid, cudaStream_t st) {
  const size_t smem = simt_smem<T>(a.Kp, rows, pass2);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, NT, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
  };
  if (rows) return pass2 ? go(k_pass_simt<T, KM, true, true>) : go(k_pass_simt<T, KM, true, false>);
  return pass2 ? go(k_pass_simt<T, KM, false, true>) : go(k_pass_simt<T, KM, false, false>);
}
}  // namespace

// column groups of the gradient accumulators: 16 threads x U columns per group
inline int simt_km(bool is_double, int Kp) {
  const int per = 16 * (is_double ? 2 : 4);
  return (Kp + per - 1) / per;
}

int simt_blocks_per_sm(bool is_double, bool rows_case, int Kp) {
  const int km = simt_km(is_double, Kp);
  if (is_double) {
    if (km <= 1) return blocks_per_sm_kj<double, 1>(Kp, rows_case);
    if (km <= 2) return blocks_per_sm_kj<double, 2>(Kp, rows_case);
    return blocks_per_sm_kj<double, 4>(Kp, rows_case);
  }
  if (km <= 1) return blocks_per_sm_kj<float, 1>(Kp, rows_case);
  if (km <= 2) return blocks_per_sm_kj<float, 2>(Kp, rows_case);
  return blocks_per_sm_kj<float, 4>(Kp, rows_case);
}

cudaError_t launch_pass_simt(const PassArgs& a_in, bool is_double, bool rows_case, bool pass2,
                             int splits, int* ctas_out, int* splits_out, cudaStream_t st) {
  PassArgs a = a_in;
  const int64_t ntiles = (a.P_strm + BN - 1) / BN;
  if (splits < 1) splits = 1;
  if (splits > ntiles) splits = (int)ntiles;
  a.tiles_per_split = (ntiles + splits - 1) / splits;
  splits = (int)((ntiles + a.tiles_per_split - 1) / a.tiles_per_split);
  dim3 grid((unsigned)((a.P_stat + BM - 1) / BM), (unsigned)splits);
  if (ctas_out) *ctas_out = (int)(grid.x * grid.y);
  if (splits_out) *splits_out = splits;
  const int km = simt_km(is_double, a.Kp);
  if (is_double) {
    if (km <= 1) return launch_kj<double, 1>(a, rows_case, pass2, grid, st);
    if (km <= 2) return launch_kj<double, 2>(a, rows_case, pass2, grid, st);
    if (km <= 4) return launch_kj<double, 4>(a, rows_case, pass2, grid, st);
    return cudaErrorInvalidValue;
  }
  if (km <= 1) return launch_kj<float, 1>(a, rows_case, pass2, grid, st);
  if (km <= 2) return launch_kj<float, 2>(a, rows_case, pass2, grid, st);
  if (km <= 4) return launch_kj<float, 4>(a, rows_case, pass2, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace trd
