// Small multilayer perceptron for the learned initial guess of the SG-GMRES
// solve: forward, backward and Adam kernels (no library GEMM).
//
// Network: d_0 = in -> width (tanh) -> ... -> width (tanh) -> out (linear),
// `hidden` tanh layers.  Parameters are kept as FP32 master copies (flat:
// W_0, b_0, W_1, b_1, ..., W_l row-major d_{l+1} x d_l); the products read
// a bf16 copy of the weights and accumulate in FP32.  Loss: mean squared
// error over the batch and the outputs.  Adam (beta1 0.9, beta2 0.999,
// eps 1e-8) with bias correction updates the FP32 masters, then refreshes the
// bf16 copy.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "sg_internal.h"

struct sg_mlp {
  int in = 0, width = 0, hidden = 0, out = 0, layers = 0;
  std::vector<int> dims;          // layers + 1
  std::vector<long long> woff, boff;
  long long nparams = 0;
  float* p = nullptr;             // FP32 master parameters
  float* g = nullptr;             // gradients
  float* m1 = nullptr;            // Adam first moment
  float* m2 = nullptr;            // Adam second moment
  __nv_bfloat16* wb = nullptr;    // bf16 copy of the parameters (same layout)
  long long step = 0;
  int cap_batch = 0;
  std::vector<float*> act;        // activations A_0..A_L, each cap_batch x dims[l]
  float* dz = nullptr;            // cap_batch x max dim
  float* dz2 = nullptr;
  double* loss = nullptr;         // device scalar
};

namespace sgi {

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]) (then tanh), A(m,k) at
// A[m*sam + k*sak], B(k,n) at B[k*sbk + n*sbn], C row-major with ldc.
// 64 x 64 tile, 256 threads, 4 x 4 outputs per thread, FP32 accumulation.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gemm_f32(int M, int N, int K, const TA* __restrict__ A, long long sam,
                                                 long long sak, const TB* __restrict__ B, long long sbk,
                                                 long long sbn, float* __restrict__ C, int ldc,
                                                 const float* __restrict__ bias, int act_tanh, int accumulate) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int mm = e % BM, kk = e / BM;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? (float)A[gm * sam + gk * sak] : 0.0f;
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      const int nn = e % BN, kk = e / BN;
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? (float)B[gk * sbk + gn * sbn] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[gn];
      if (act_tanh) v = tanhf(v);
      float* c = C + (long long)gm * ldc + gn;
      *c = accumulate ? *c + v : v;
    }
  }
}

template <typename TA, typename TB>
static cudaError_t gemm_f32(int M, int N, int K, const TA* A, long long sam, long long sak, const TB* B,
                            long long sbk, long long sbn, float* C, int ldc, const float* bias, int act_tanh,
                            cudaStream_t st) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm_f32<TA, TB><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, act_tanh, 0);
  note_launch();
  return cudaGetLastError();
}

// loss = mean((Y - T)^2) over rows*cols; dY = 2 (Y - T) / (rows*cols).
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, long long count, float* __restrict__ dY,
                      double* loss) {
  __shared__ double sm[32];
  double acc = 0.0;
  const float inv = 2.0f / (float)count;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    acc += (double)d * d;
    dY[i] = inv * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loss, v / (double)count);
  }
}

// dZ = dA * (1 - A^2) (tanh derivative), in place allowed.
__global__ void k_tanh_back(const float* __restrict__ A, const float* dA, float* dZ, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const float a = A[i];
    dZ[i] = dA[i] * (1.0f - a * a);
  }
}

// db[n] = sum_b dZ[b][n]
__global__ void k_colsum(const float* __restrict__ dZ, int rows, int cols, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  float s = 0.0f;
  for (int b = 0; b < rows; ++b) s += dZ[(long long)b * cols + n];
  db[n] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, __nv_bfloat16* __restrict__ wb, long long n, float lr, float c1,
                       float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi;
    const float b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float v = p[i] - lr * (a * c1) / (sqrtf(b * c2) + 1e-8f);
    p[i] = v;
    wb[i] = __float2bfloat16_rn(v);
  }
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(p[i]);
}

static int grid_for(long long n) { return (int)std::max(1LL, std::min((n + 255) / 256, 4096LL)); }

static cudaError_t ensure_batch(sg_mlp* m, int batch) {
  if (batch <= m->cap_batch) return cudaSuccess;
  for (float* a : m->act) cudaFree(a);
  cudaFree(m->dz);
  cudaFree(m->dz2);
  m->act.assign(m->layers + 1, nullptr);
  int maxd = 0;
  for (int d : m->dims) maxd = std::max(maxd, d);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l <= m->layers && e == cudaSuccess; ++l)
    e = cudaMalloc((void**)&m->act[l], (size_t)batch * m->dims[l] * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->dz, (size_t)batch * maxd * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&m->dz2, (size_t)batch * maxd * sizeof(float));
  if (e == cudaSuccess) m->cap_batch = batch;
  return e;
}

// Forward pass; activations kept for the backward pass (act[0] = X copy).
static cudaError_t forward(sg_mlp* m, const float* X, int B, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(m->act[0], X, (size_t)B * m->in * sizeof(float), cudaMemcpyDeviceToDevice, st);
  for (int l = 0; l < m->layers && e == cudaSuccess; ++l) {
    const int di = m->dims[l], dout = m->dims[l + 1];
    // Z = A_l W_l^T + b_l ; A(b, i) = act[b*di + i], B(i, o) = W[o*di + i]
    e = gemm_f32<float, __nv_bfloat16>(B, dout, di, m->act[l], di, 1, m->wb + m->woff[l], 1, di, m->act[l + 1], dout,
                                       m->p + m->boff[l], l < m->layers - 1 ? 1 : 0, st);
  }
  return e;
}

// Backward pass from dY (in m->dz, B x out); gradients into m->g.
static cudaError_t backward(sg_mlp* m, int B, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  float* dcur = m->dz;    // gradient w.r.t. Z of layer l (B x dims[l+1])
  float* dnext = m->dz2;
  for (int l = m->layers - 1; l >= 0 && e == cudaSuccess; --l) {
    const int di = m->dims[l], dout = m->dims[l + 1];
    // dW_l = dZ^T A_l : A(o, b) = dZ[b*dout + o], B(b, i) = act[b*di + i]
    e = gemm_f32<float, float>(dout, di, B, dcur, 1, dout, m->act[l], di, 1, m->g + m->woff[l], di, nullptr, 0, st);
    if (e) break;
    k_colsum<<<(dout + 127) / 128, 128, 0, st>>>(dcur, B, dout, m->g + m->boff[l]);
    note_launch();
    if (l == 0) break;
    // dA_l = dZ W_l : A(b, o) = dZ[b*dout + o], B(o, i) = W[o*di + i]; then tanh'
    e = gemm_f32<float, __nv_bfloat16>(B, di, dout, dcur, dout, 1, m->wb + m->woff[l], di, 1, dnext, di, nullptr, 0,
                                       st);
    if (e) break;
    k_tanh_back<<<grid_for((long long)B * di), 256, 0, st>>>(m->act[l], dnext, dnext, (long long)B * di);
    note_launch();
    std::swap(dcur, dnext);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// The loss is added to *m->loss, which is cleared first when reset_loss.
static cudaError_t loss_and_grad(sg_mlp* m, const float* X, const float* T, int B, cudaStream_t st,
                                 bool reset_loss = true) {
  cudaError_t e = forward(m, X, B, st);
  if (e) return e;
  if (reset_loss && (e = cudaMemsetAsync(m->loss, 0, sizeof(double), st))) return e;
  const long long cnt = (long long)B * m->out;
  k_mse<<<grid_for(cnt), 256, 0, st>>>(m->act[m->layers], T, cnt, m->dz, m->loss);
  note_launch();
  if ((e = cudaGetLastError())) return e;
  return backward(m, B, st);
}

}  // namespace sgi

using namespace sgi;

extern "C" {

sg_status sg_mlp_create(int in_dim, int width, int hidden, int out_dim, sg_mlp** out) {
  return sgi::guarded([&]() -> sg_status {
    if (!out || in_dim <= 0 || width <= 0 || hidden < 0 || out_dim <= 0 || width > 1 << 14)
      return fail(SG_EINVAL, "bad MLP shape");
    auto* m = new sg_mlp();
    m->in = in_dim;
    m->width = width;
    m->hidden = hidden;
    m->out = out_dim;
    m->layers = hidden + 1;
    m->dims.push_back(in_dim);
    for (int l = 0; l < hidden; ++l) m->dims.push_back(width);
    m->dims.push_back(out_dim);
    long long off = 0;
    for (int l = 0; l < m->layers; ++l) {
      m->woff.push_back(off);
      off += (long long)m->dims[l + 1] * m->dims[l];
      m->boff.push_back(off);
      off += m->dims[l + 1];
    }
    m->nparams = off;
    cudaError_t e = cudaSuccess;
    if (!e) e = cudaMalloc((void**)&m->p, off * sizeof(float));
    if (!e) e = cudaMalloc((void**)&m->g, off * sizeof(float));
    if (!e) e = cudaMalloc((void**)&m->m1, off * sizeof(float));
    if (!e) e = cudaMalloc((void**)&m->m2, off * sizeof(float));
    if (!e) e = cudaMalloc((void**)&m->wb, off * sizeof(__nv_bfloat16));
    if (!e) e = cudaMalloc((void**)&m->loss, sizeof(double));
    if (!e) e = cudaMemset(m->p, 0, off * sizeof(float));
    if (!e) e = cudaMemset(m->m1, 0, off * sizeof(float));
    if (!e) e = cudaMemset(m->m2, 0, off * sizeof(float));
    if (!e) e = cudaMemset(m->wb, 0, off * sizeof(__nv_bfloat16));
    if (e) {
      sg_mlp_destroy(m);
      return fail(SG_ENOMEM, std::string("MLP allocation: ") + cudaGetErrorString(e));
    }
    *out = m;
    return SG_OK;
  });
}

void sg_mlp_destroy(sg_mlp* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  cudaFree(m->p); cudaFree(m->g); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->wb); cudaFree(m->loss);
  for (float* a : m->act) cudaFree(a);
  cudaFree(m->dz); cudaFree(m->dz2);
  delete m;
}

long long sg_mlp_num_params(const sg_mlp* m) { return m ? m->nparams : -1; }

sg_status sg_mlp_set_params(sg_mlp* m, const float* src, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!m || !src) return fail(SG_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    SG_CUDA_TRY(cudaMemcpyAsync(m->p, src, m->nparams * sizeof(float), cudaMemcpyDeviceToDevice, st));
    SG_CUDA_TRY(cudaMemsetAsync(m->m1, 0, m->nparams * sizeof(float), st));
    SG_CUDA_TRY(cudaMemsetAsync(m->m2, 0, m->nparams * sizeof(float), st));
    k_to_bf16<<<grid_for(m->nparams), 256, 0, st>>>(m->p, m->wb, m->nparams);
    note_launch();
    SG_CUDA_TRY(cudaGetLastError());
    m->step = 0;
    return SG_OK;
  });
}

sg_status sg_mlp_get_params(const sg_mlp* m, float* dst, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!m || !dst) return fail(SG_EINVAL, "NULL argument");
    SG_CUDA_TRY(cudaMemcpyAsync(dst, m->p, m->nparams * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SG_OK;
  });
}

sg_status sg_mlp_forward(sg_mlp* m, const float* X, int batch, float* Y, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!m || !X || !Y || batch <= 0) return fail(SG_EINVAL, "bad sg_mlp_forward arguments");
    cudaStream_t st = (cudaStream_t)stream;
    SG_CUDA_TRY(ensure_batch(m, batch));
    SG_CUDA_TRY(forward(m, X, batch, st));
    SG_CUDA_TRY(cudaMemcpyAsync(Y, m->act[m->layers], (size_t)batch * m->out * sizeof(float), cudaMemcpyDeviceToDevice,
                                st));
    return SG_OK;
  });
}

sg_status sg_mlp_loss_grad(sg_mlp* m, const float* X, const float* T, int batch, double* loss, float* grad,
                           void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!m || !X || !T || batch <= 0) return fail(SG_EINVAL, "bad sg_mlp_loss_grad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    SG_CUDA_TRY(ensure_batch(m, batch));
    SG_CUDA_TRY(loss_and_grad(m, X, T, batch, st));
    if (grad) SG_CUDA_TRY(cudaMemcpyAsync(grad, m->g, m->nparams * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (loss) {
      SG_CUDA_TRY(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return SG_OK;
  });
}

sg_status sg_mlp_train(sg_mlp* m, const float* X, const float* T, int nsamples, int batch, int epochs, float lr,
                       double* loss_history, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!m || !X || !T || nsamples <= 0 || batch <= 0 || epochs < 0 || !(lr > 0))
      return fail(SG_EINVAL, "bad sg_mlp_train arguments");
    cudaStream_t st = (cudaStream_t)stream;
    batch = std::min(batch, nsamples);
    SG_CUDA_TRY(ensure_batch(m, batch));
    for (int ep = 0; ep < epochs; ++ep) {
      // the epoch's mini-batch losses accumulate on the device: one read per epoch
      SG_CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(double), st));
      int nb = 0;
      for (int s0 = 0; s0 + batch <= nsamples; s0 += batch, ++nb) {
        SG_CUDA_TRY(loss_and_grad(m, X + (size_t)s0 * m->in, T + (size_t)s0 * m->out, batch, st, false));
        ++m->step;
        const float c1 = 1.0f / (1.0f - powf(0.9f, (float)m->step));
        const float c2 = 1.0f / (1.0f - powf(0.999f, (float)m->step));
        k_adam<<<grid_for(m->nparams), 256, 0, st>>>(m->p, m->g, m->m1, m->m2, m->wb, m->nparams, lr, c1, c2);
        note_launch();
        SG_CUDA_TRY(cudaGetLastError());
      }
      if (loss_history) {
        double l = 0;
        SG_CUDA_TRY(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        loss_history[ep] = nb ? l / nb : 0.0;
      }
    }
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    return SG_OK;
  });
}

}  // extern "C"

namespace sgi {
// Input and output widths of a network (for the warm-start model's checks).
void mlp_dims(const sg_mlp* m, int* in_dim, int* out_dim) {
  *in_dim = m->in;
  *out_dim = m->out;
}
}  // namespace sgi
