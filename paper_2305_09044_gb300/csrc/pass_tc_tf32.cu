// TF32 instantiations of the fused tensor-core data pass (kind::tf32, 3-term split of every
// product): the FP32-accurate tensor-core path.  Kept in a translation unit of its own so that
// the BF16 and TF32 variants compile in parallel.
#include "pass_tc.cuh"

namespace trd {
namespace tc {

cudaError_t launch_pass_tc_tf32(int kpad, bool rows_case, bool pass2, bool full_stats, const PassOperands& o,
                                const float* X, int64_t P_in, int64_t ldx, int64_t P_out, Params p, int G,
                                cudaStream_t st) {
  if (kpad == 64) return launch_pass_tc_kp<64, true>(rows_case, pass2, full_stats, o, X, P_in, ldx, P_out, p, G, st);
  return cudaErrorInvalidValue;
}

}  // namespace tc
}  // namespace trd
