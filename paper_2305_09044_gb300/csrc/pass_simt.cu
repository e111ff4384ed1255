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
#include "trd_internal.cuh"

namespace trd {

namespace {
constexpr int BM = 64, BN = 64, NT = 256;

__device__ __forceinline__ float texp(float x) { return expf(x); }
__device__ __forceinline__ double texp(double x) { return exp(x); }


template <typename T, int KJ, bool ROWS, bool PASS2>
__global__ void __launch_bounds__(NT) k_pass_simt(const PassArgs p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int SYLD = ROWS ? BN + 1 : BN + 16;
  const int Kp = p.Kp;
  const int KPAD = Kp | 1;
  T* sS = reinterpret_cast<T*>(smraw);           // [BM][KPAD] stationary rows
  T* sH = sS + BM * KPAD;                        // [BM][KPAD] stationary rows with h (pass 2)
  T* sT = PASS2 ? sH + BM * KPAD : sS + BM * KPAD;  // [BN][KPAD] streaming tile
  T* sY = sT + BN * KPAD;                        // [BM][SYLD] weighted residuals (pass 1)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t s0 = (int64_t)blockIdx.x * BM;
  const T* Sst = reinterpret_cast<const T*>(p.Sst);
  const T* Sh = reinterpret_cast<const T*>(p.Sh);
  const T* Sstr = reinterpret_cast<const T*>(p.Sstr);

  for (RowCol rc(tid, NT, Kp); rc.r < BM; rc.next()) {
    const int r = rc.r, c = rc.c;
    const int64_t s = s0 + r;
    sS[r * KPAD + c] = s < p.P_stat ? Sst[s * p.ld + c] : T(0);
    if (PASS2) sH[r * KPAD + c] = s < p.P_stat ? Sh[s * p.ld + c] : T(0);
  }
  const double sig = *p.sigma;
  const T inv2s2 = isinf(sig) ? T(0) : T(1.0 / (2.0 * sig * sig));

  T tacc[4][KJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < KJ; ++j) tacc[i][j] = T(0);
  // statistics: FP32 partial sums per tile (FP64 for the FP64 path), integer counts, widened
  // and added into FP64 once per tile
  double st_w = 0, st_e2 = 0, st_we2 = 0, st_den = 0;
  int64_t st_obs = 0, st_nf = 0, st_slots = 0;
  const RowCol tile_rc(tid, NT, Kp);

  const int64_t ntiles = (p.P_strm + BN - 1) / BN;
  const int64_t tb = (int64_t)blockIdx.y * p.tiles_per_split;
  const int64_t te = imin(ntiles, tb + p.tiles_per_split);
  for (int64_t tile = tb; tile < te; ++tile) {
    const int64_t t0 = tile * BN;
    __syncthreads();
    for (RowCol rc = tile_rc; rc.r < BN; rc.next()) {
      const int r = rc.r, c = rc.c;
      const int64_t t = t0 + r;
      sT[r * KPAD + c] = t < p.P_strm ? Sstr[t * p.ld + c] : T(0);
    }
    __syncthreads();
    // micro-tile: the thread index that runs along the memory-contiguous direction of X
    // is tx, so global loads of x are coalesced
    T acc[4][4], dacc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { acc[i][j] = T(0); dacc[i][j] = T(0); }
    for (int k = 0; k < Kp; ++k) {
      T sv[4], hv[4], tv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = ROWS ? tx + 16 * i : ty + 16 * i;
        sv[i] = sS[r * KPAD + k];
        if (PASS2) hv[i] = sH[r * KPAD + k];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = ROWS ? ty + 16 * j : tx + 16 * j;
        tv[j] = sT[c * KPAD + k];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j] = fma(sv[i], tv[j], acc[i][j]);
          if (PASS2) dacc[i][j] = fma(hv[i], tv[j], dacc[i][j]);
        }
    }
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
          const int64_t lin = ROWS ? s + p.P_in * t : t + p.P_in * s;
          const bool obs = p.M ? ((p.M[lin >> 5] >> (lin & 31)) & 1u) : true;
          ++tslots;
          if (obs) {
            ++tobs;
            const T e = (T)p.X[lin] - acc[i][j];
            if (isfinite(e)) {
              const T w = texp(-e * e * inv2s2);
              if (PASS2) {
                tden = fma(w * dacc[i][j], dacc[i][j], tden);
              } else {
                y = w * e;
                tw += w;
                te2 = fma(e, e, te2);
                twe2 = fma(y, e, twe2);
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
      for (int tt = 0; tt < BN; ++tt) {
        T yv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) yv[i] = sY[(ty + 16 * i) * SYLD + tt];
#pragma unroll
        for (int j = 0; j < KJ; ++j) {
          const int c = tx + 16 * j;
          const T cv = c < Kp ? sT[tt * KPAD + c] : T(0);
#pragma unroll
          for (int i = 0; i < 4; ++i) tacc[i][j] = fma(yv[i], cv, tacc[i][j]);
        }
      }
    }
  }
  if (!PASS2) {
    T* Tp = reinterpret_cast<T*>(p.Tpart) + (int64_t)blockIdx.y * p.P_stat * Kp;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t s = s0 + ty + 16 * i;
#pragma unroll
      for (int j = 0; j < KJ; ++j) {
        const int c = tx + 16 * j;
        if (s < p.P_stat && c < Kp) Tp[s * Kp + c] = tacc[i][j];
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

template <typename T, int KJ>
cudaError_t launch_kj(const PassArgs& a, bool rows, bool pass2, dim3 grid, cudaStream_t st) {
  const int KPAD = a.Kp | 1;
  const int syld = rows ? BN + 1 : BN + 16;
  const size_t smem = (size_t)((pass2 ? 2 : 1) * BM * KPAD + BN * KPAD + (pass2 ? 0 : BM * syld)) * sizeof(T);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, NT, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
  };
  if (rows) return pass2 ? go(k_pass_simt<T, KJ, true, true>) : go(k_pass_simt<T, KJ, true, false>);
  return pass2 ? go(k_pass_simt<T, KJ, false, true>) : go(k_pass_simt<T, KJ, false, false>);
}
}  // namespace

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
  const int kj = (a.Kp + 15) / 16;
  if (is_double) {
    if (kj <= 1) return launch_kj<double, 1>(a, rows_case, pass2, grid, st);
    if (kj <= 4) return launch_kj<double, 4>(a, rows_case, pass2, grid, st);
    if (kj <= 7) return launch_kj<double, 7>(a, rows_case, pass2, grid, st);
    return cudaErrorInvalidValue;
  }
  if (kj <= 1) return launch_kj<float, 1>(a, rows_case, pass2, grid, st);
  if (kj <= 4) return launch_kj<float, 4>(a, rows_case, pass2, grid, st);
  if (kj <= 7) return launch_kj<float, 7>(a, rows_case, pass2, grid, st);
  if (kj <= 16) return launch_kj<float, 16>(a, rows_case, pass2, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace trd
