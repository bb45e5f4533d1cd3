// Register-resident complex64 SG matvec for fixed (s, r): see the generic
// kernel in k_operator.cu for the operator.  (Specialisations are added per
// chaos size; this translation unit reports "not handled" for the others.)
#include <cuda_runtime.h>

#include "sg_internal.h"

namespace sgi {

cudaError_t matvec_special_f32(const sg_handle* h, const float2* X, float2* Y, cudaStream_t st, const int* skip,
                               bool* handled) {
  (void)h; (void)X; (void)Y; (void)st; (void)skip;
  *handled = false;
  return cudaSuccess;
}

}  // namespace sgi
