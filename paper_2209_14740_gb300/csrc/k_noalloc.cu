// Allocation-free variant of the block preconditioner apply (sg_precond_noalloc).
//
// Who needs it: code that must not allocate device memory while it runs — a
// host callback or real-time loop that may not block on the allocator, a
// process whose device memory is owned by another runtime's pool (so a raw
// cudaMalloc would fragment or exceed its budget), or a caller inside a
// region where allocation is forbidden.  sg_precond itself allocates nothing
// per call either, but it uses scratch that sg_assemble allocated for the
// handle; this entry point instead takes its scratch from a fixed array that
// lives in the library image, so it works with handles whose scratch must
// not be touched (for example while another stream uses it).
//
// The scratch is a file-scope __device__ array: the GPU that loads the
// library holds SG_NOALLOC_MAX_N * 2 complex128 values (16 MiB) until the
// process exits.  All calls share it, so calls that overlap on the GPU (two
// streams, two host threads) race.  Every call fully writes the parts of the
// array it later reads, so nothing has to start at zero.
//
// Host code may not use the array's name as a device address; its address is
// looked up by sg_assemble (sgi::noalloc_scratch_address below), where
// allocation is allowed anyway: that lookup is what loads this file's module
// and commits the array under lazy module loading, so sg_precond_noalloc
// itself never does.
#include <cuda_runtime.h>

#include <string>

#include "sg_internal.h"

namespace {

// Two intermediates of up to SG_NOALLOC_MAX_N complex values each (complex128
// storage; the complex64 path uses the first half of each).
static __device__ __align__(256) double2 g_noalloc_scratch[2 * (size_t)SG_NOALLOC_MAX_N];

}  // namespace

namespace sgi {

// Device address of the scratch array on the current device (called by
// sg_assemble with the handle's device current).
cudaError_t noalloc_scratch_address(void** out) {
  *out = nullptr;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e == cudaSuccess && !p) e = cudaErrorInvalidSymbol;
  if (e == cudaSuccess) *out = p;
  return e;
}

}  // namespace sgi

extern "C" sg_status sg_precond_noalloc(sg_handle* h, sg_prec kind, sg_precision prec, const void* R, void* Z,
                                        void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !R || !Z) return sgi::fail(SG_EINVAL, "NULL handle or vector");
    if (prec != SG_FP64 && prec != SG_FP32) return sgi::fail(SG_EINVAL, "precision must be SG_FP64 or SG_FP32");
    if (kind != SG_PREC_MEAN && kind != SG_PREC_CSL_MEAN)
      return sgi::fail(SG_EINVAL, "sg_precond_noalloc: kind must be SG_PREC_MEAN or SG_PREC_CSL_MEAN");
    if (h->N > (long long)SG_NOALLOC_MAX_N)
      return sgi::fail(SG_EINVAL, "sg_precond_noalloc: N = " + std::to_string(h->N) +
                                      " exceeds the static scratch limit SG_NOALLOC_MAX_N = " +
                                      std::to_string((long long)SG_NOALLOC_MAX_N));
    const int which = kind == SG_PREC_MEAN ? 0 : 1;
    if (!h->blk[which].ready)
      return sgi::fail(SG_EUNSUPPORTED, "no factorisation for this block (2D needs a constant k_0)");
    void* base = h->noalloc_scratch;
    if (!base) return sgi::fail(SG_ECUDA, "sg_precond_noalloc: the static scratch has no device address");
    cudaStream_t st = (cudaStream_t)stream;
    double2* s0 = reinterpret_cast<double2*>(base);
    double2* s1 = s0 + (size_t)SG_NOALLOC_MAX_N;
    cudaError_t e;
    if (prec == SG_FP64)
      e = sgi::launch_precond_scratch<double>(h, which, (const double2*)R, (double2*)Z, st, s0, s1);
    else
      e = sgi::launch_precond_scratch<float>(h, which, (const float2*)R, (float2*)Z, st,
                                             reinterpret_cast<float2*>(s0), reinterpret_cast<float2*>(s1));
    if (e != cudaSuccess) return sgi::fail(SG_ECUDA, std::string("sg_precond_noalloc: ") + cudaGetErrorString(e));
    return SG_OK;
  });
}
