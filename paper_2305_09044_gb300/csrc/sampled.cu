// Sampled correntropy loss and its adjoint (placeholder until the kernels land).
#include "trd_internal.cuh"

extern "C" {

trd_status trd_sampled_fwd(trd_t* h, const void* const*, const int32_t*, const void*, int64_t, double, int,
                           void*, double*) {
  if (!h) return TRD_EINVAL;
  h->err = "sampled loss not built";
  return TRD_ENOTIMPL;
}

trd_status trd_sampled_bwd(trd_t* h, const void* const*, const int32_t*, const void*, int64_t, double, int,
                           double, void* const*) {
  if (!h) return TRD_EINVAL;
  h->err = "sampled loss not built";
  return TRD_ENOTIMPL;
}

}
