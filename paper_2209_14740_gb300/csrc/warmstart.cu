// Inference of the learned initial guess (not part of the paper's method: a
// throughput aid whose guess sg_gmres always finishes to the requested
// tolerance).  A model holds the trained network (sg_mlp), a device copy of
// the decoder D = scale * U (rank rows of N complex64 values: the scaled POD
// basis of training solutions) and the box [lo, hi] of the workload
// parameters.  Prediction for `count` parameter rows:
//   1. X = 2 (p - lo) / (hi - lo) - 1 per row (device kernel),
//   2. Y = net(X): count x 2 rank FP32 (the network's forward kernels),
//   3. c = Y viewed as count x rank complex64 (interleaved pairs, no copy),
//   4. x0 = c D: count x N complex128 (the complex expansion kernel).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "sg_internal.h"

struct sg_warmstart {
  sg_mlp* net = nullptr;          // not owned
  int in_dim = 0, rank = 0;
  long long N = 0;
  float2* D = nullptr;            // rank x N complex64, owned
  double* lo = nullptr;           // in_dim, device
  double* hi = nullptr;
  double* p = nullptr;            // cap x in_dim, device (parameters)
  float* X = nullptr;             // cap x in_dim, device (normalised)
  float* Y = nullptr;             // cap x 2 rank, device (network output)
  int cap = 0;
};

namespace sgi {

__global__ void k_normalise(const double* __restrict__ p, const double* __restrict__ lo,
                            const double* __restrict__ hi, int count, int d, float* __restrict__ X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count * d) {
    const int j = i % d;
    X[i] = (float)(2.0 * (p[i] - lo[j]) / (hi[j] - lo[j]) - 1.0);
  }
}

static void free_ws(sg_warmstart* w) {
  cudaFree(w->D); cudaFree(w->lo); cudaFree(w->hi); cudaFree(w->p); cudaFree(w->X); cudaFree(w->Y);
}

}  // namespace sgi

extern "C" {

sg_status sg_warmstart_create(sg_mlp* net, const void* D, int rank, long long N, const double* lo, const double* hi,
                              sg_warmstart** out) {
  using namespace sgi;
  return guarded([&]() -> sg_status {
    if (!net || !D || !lo || !hi || !out || rank <= 0 || N <= 0) return fail(SG_EINVAL, "bad sg_warmstart_create arguments");
    int in_dim = 0, out_dim = 0;
    mlp_dims(net, &in_dim, &out_dim);
    if (out_dim != 2 * rank) return fail(SG_EINVAL, "the network's output width must be 2 * rank");
    for (int j = 0; j < in_dim; ++j)
      if (!(hi[j] > lo[j]) || !std::isfinite(lo[j]) || !std::isfinite(hi[j]))
        return fail(SG_EINVAL, "parameter box needs finite lo < hi");
    auto* w = new sg_warmstart();
    w->net = net;
    w->in_dim = in_dim;
    w->rank = rank;
    w->N = N;
    cudaError_t e = cudaMalloc((void**)&w->D, (size_t)rank * N * sizeof(float2));
    if (!e) e = cudaMemcpy(w->D, D, (size_t)rank * N * sizeof(float2), cudaMemcpyDeviceToDevice);
    if (!e) e = cudaMalloc((void**)&w->lo, in_dim * sizeof(double));
    if (!e) e = cudaMalloc((void**)&w->hi, in_dim * sizeof(double));
    if (!e) e = cudaMemcpy(w->lo, lo, in_dim * sizeof(double), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(w->hi, hi, in_dim * sizeof(double), cudaMemcpyHostToDevice);
    if (e) {
      free_ws(w);
      delete w;
      return fail(SG_ENOMEM, std::string("sg_warmstart_create: ") + cudaGetErrorString(e));
    }
    *out = w;
    return SG_OK;
  });
}

void sg_warmstart_destroy(sg_warmstart* w) {
  if (!w) return;
  cudaDeviceSynchronize();
  sgi::free_ws(w);
  delete w;
}

sg_status sg_warmstart_predict(sg_warmstart* w, const double* params, int count, void* x0, void* stream) {
  using namespace sgi;
  return guarded([&]() -> sg_status {
    if (!w || !params || !x0 || count <= 0) return fail(SG_EINVAL, "bad sg_warmstart_predict arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (count > w->cap) {
      SG_CUDA_TRY(cudaStreamSynchronize(st));
      cudaFree(w->p); cudaFree(w->X); cudaFree(w->Y);
      w->p = nullptr; w->X = nullptr; w->Y = nullptr; w->cap = 0;
      SG_CUDA_TRY(cudaMalloc((void**)&w->p, (size_t)count * w->in_dim * sizeof(double)));
      SG_CUDA_TRY(cudaMalloc((void**)&w->X, (size_t)count * w->in_dim * sizeof(float)));
      SG_CUDA_TRY(cudaMalloc((void**)&w->Y, (size_t)count * 2 * w->rank * sizeof(float)));
      w->cap = count;
    }
    SG_CUDA_TRY(cudaMemcpyAsync(w->p, params, (size_t)count * w->in_dim * sizeof(double), cudaMemcpyHostToDevice, st));
    const int tot = count * w->in_dim;
    k_normalise<<<(tot + 127) / 128, 128, 0, st>>>(w->p, w->lo, w->hi, count, w->in_dim, w->X);
    note_launch();
    SG_CUDA_TRY(cudaGetLastError());
    sg_status s = sg_mlp_forward(w->net, w->X, count, w->Y, stream);
    if (s != SG_OK) return s;
    return sg_cgemm_nn(w->Y, w->D, count, (int)w->N, w->rank, x0, 1, stream);
  });
}

}  // extern "C"
