// Post-processing of a stochastic Galerkin solution V = [V_0; ...; V_{P-1}]
// (Sec. 7 of the paper): the expected value E[u~] = V_0, the variances of the
// real and imaginary parts of u~ (sums of squares of the modes i >= 1, by the
// orthonormality of the chaos basis) and the magnitudes
// gamma_j = max { ||V_i||_inf : deg(phi_i) = j }.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "sg_internal.h"

namespace sgi {

constexpr int POST_THREADS = 256;

// One thread per grid unknown: mean and the two variances (accumulated in
// FP64 for both precisions).
template <typename T>
__global__ void __launch_bounds__(POST_THREADS) k_moments(const C2<T>* __restrict__ V, int n, int P,
                                                         C2<T>* __restrict__ mean, T* __restrict__ var_re,
                                                         T* __restrict__ var_im) {
  const int stride = gridDim.x * blockDim.x;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
    if (mean) mean[u] = V[u];
    double sr = 0.0, si = 0.0;
    for (int i = 1; i < P; ++i) {
      const C2<T> v = V[(size_t)i * n + u];
      sr += (double)v.x * v.x;
      si += (double)v.y * v.y;
    }
    if (var_re) var_re[u] = (T)sr;
    if (var_im) var_im[u] = (T)si;
  }
}

// Largest |V_i(x)| of mode i = blockIdx.y over the grid: block maxima folded
// by atomicMax on the bit patterns (non-negative doubles order like their
// bit patterns read as unsigned integers).
template <typename T>
__global__ void __launch_bounds__(POST_THREADS) k_mode_maxabs(const C2<T>* __restrict__ V, int n,
                                                             unsigned long long* __restrict__ out) {
  __shared__ double wmax[POST_THREADS / 32];
  const size_t base = (size_t)blockIdx.y * n;
  double m = 0.0;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const C2<T> v = V[base + u];
    m = fmax(m, hypot((double)v.x, (double)v.y));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < POST_THREADS / 32; ++w) m = fmax(m, wmax[w]);
    atomicMax(out + blockIdx.y, (unsigned long long)__double_as_longlong(m));
  }
}

}  // namespace sgi

extern "C" sg_status sg_statistics(sg_handle* h, sg_precision prec, const void* V, void* mean, void* var_re,
                                   void* var_im, double* gamma, void* stream) {
  using namespace sgi;
  return guarded([&]() -> sg_status {
    if (!h || !V) return fail(SG_EINVAL, "NULL handle or V");
    if (prec != SG_FP64 && prec != SG_FP32) return fail(SG_EINVAL, "sg_statistics precision must be SG_FP64 or SG_FP32");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = h->n, P = h->P;
    const int blocks = std::max(1, std::min(h->num_sms * 8, (n + POST_THREADS - 1) / POST_THREADS));
    if (mean || var_re || var_im) {
      if (prec == SG_FP64)
        k_moments<double><<<blocks, POST_THREADS, 0, st>>>((const double2*)V, n, P, (double2*)mean, (double*)var_re,
                                                           (double*)var_im);
      else
        k_moments<float><<<blocks, POST_THREADS, 0, st>>>((const float2*)V, n, P, (float2*)mean, (float*)var_re,
                                                          (float*)var_im);
      note_launch();
      SG_CUDA_TRY(cudaGetLastError());
    }
    if (gamma) {
      if (!h->d_modemax) SG_CUDA_TRY(cudaMalloc((void**)&h->d_modemax, (size_t)P * sizeof(unsigned long long)));
      SG_CUDA_TRY(cudaMemsetAsync(h->d_modemax, 0, (size_t)P * sizeof(unsigned long long), st));
      const dim3 g((unsigned)std::max(1, std::min(64, (n + POST_THREADS - 1) / POST_THREADS)), (unsigned)P);
      if (prec == SG_FP64)
        k_mode_maxabs<double><<<g, POST_THREADS, 0, st>>>((const double2*)V, n, h->d_modemax);
      else
        k_mode_maxabs<float><<<g, POST_THREADS, 0, st>>>((const float2*)V, n, h->d_modemax);
      note_launch();
      SG_CUDA_TRY(cudaGetLastError());
      std::vector<unsigned long long> bits(P);
      SG_CUDA_TRY(cudaMemcpyAsync(bits.data(), h->d_modemax, (size_t)P * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
      for (int j = 0; j <= h->r; ++j) gamma[j] = 0.0;
      for (int i = 0; i < P; ++i) {
        int deg = 0;
        for (int l = 0; l < h->s; ++l) deg += h->alpha[(size_t)i * h->s + l];
        double v;
        static_assert(sizeof(v) == sizeof(bits[i]), "64-bit patterns");
        std::memcpy(&v, &bits[i], sizeof(v));
        gamma[deg] = std::max(gamma[deg], v);
      }
    }
    return SG_OK;
  });
}
