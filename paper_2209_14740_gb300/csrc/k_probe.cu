// Arithmetic peak of the CUDA cores (FP64 and FP32 fused multiply-add),
// measured on the running GPU: the denominator of the ALU roofline of the
// FP64 kernels (complex FP64 transforms, the FP64 operator), for which the
// tensor cores offer nothing on this GPU.  Not part of the paper's method.
//
// Every thread runs 8 independent FMA chains (enough to cover the FMA
// latency at full occupancy); the grid fills every SM several times over.
#include <cuda_runtime.h>

#include <string>

#include "sg_internal.h"

namespace sgi {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T* out, int iters, T a, T b) {
  T x[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += x[i];
  // a store the compiler cannot prove dead (a, b are runtime values)
  if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static sg_status probe(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  SG_CUDA_TRY(cudaGetDevice(&dev));
  SG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8 * 4;          // 8 resident blocks of 256 threads per SM, four waves
  const int iters = sizeof(T) == 8 ? 4096 : 32768;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&out, (size_t)blocks * kProbeThreads * sizeof(T));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    // warm-up launch, then the timed one
    k_fma_probe<T><<<blocks, kProbeThreads, 0, st>>>(out, iters / 8, (T)0.999, (T)1e-4);
    note_launch();
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      k_fma_probe<T><<<blocks, kProbeThreads, 0, st>>>(out, iters, (T)0.999, (T)1e-4);
      note_launch();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return fail(SG_ECUDA, std::string("FMA probe: ") + cudaGetErrorString(e));
  if (!(ms > 0.f)) return fail(SG_ECUDA, "FMA probe: no elapsed time");
  const double flop = 2.0 * kProbeChains * (double)iters * blocks * kProbeThreads;
  *tflops = flop / (ms * 1e-3) / 1e12;
  return SG_OK;
}

}  // namespace sgi

extern "C" sg_status sg_alu_peak(int fp64, double* tflops, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!tflops) return sgi::fail(SG_EINVAL, "NULL tflops");
    cudaStream_t st = (cudaStream_t)stream;
    return fp64 ? sgi::probe<double>(tflops, st) : sgi::probe<float>(tflops, st);
  });
}
