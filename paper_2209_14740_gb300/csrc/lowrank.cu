// Complex products for the low-rank (POD) decoder of the learned initial
// guess: Gram matrices and projections onto a basis (conjugated rows), and
// the expansion x = c U.  Complex64 operands, FP32 accumulation in tiles
// with FP64 accumulation across tiles of the long dimension.
#include <cuda_runtime.h>

#include <algorithm>

#include "sg_internal.h"

namespace sgi {

// C[i][j] = sum_t conj(A[i][t]) B[j][t]; A: m rows, B: n rows, length k each
// (row stride lda / ldb), C row-major complex64 (ldc).  32 x 32 tile of C per
// CTA, 256 threads (2 x 2 outputs each); the k loop is split over gridDim.z
// slices whose FP32 partials are added in FP64 to Cacc (m x n complex128).
__global__ void __launch_bounds__(256) k_cgemm_hn(int m, int n, long long k, const float2* __restrict__ A,
                                                 long long lda, const float2* __restrict__ B, long long ldb,
                                                 double2* __restrict__ Cacc) {
  constexpr int BT = 32, BK = 16;
  __shared__ float2 As[BK][BT + 1];
  __shared__ float2 Bs[BK][BT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * BT, j0 = blockIdx.x * BT;
  const long long per = (k + gridDim.z - 1) / gridDim.z;
  const long long k0 = blockIdx.z * per, k1 = min(k, k0 + per);
  float ar[2][2] = {}, ai[2][2] = {};
  for (long long kb = k0; kb < k1; kb += BK) {
    for (int e = threadIdx.x; e < BT * BK; e += 256) {
      const int r = e / BK, kk = e % BK;
      const long long gk = kb + kk;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (gk < k1) {
        if (i0 + r < m) va = A[(long long)(i0 + r) * lda + gk];
        if (j0 + r < n) vb = B[(long long)(j0 + r) * ldb + gk];
      }
      As[kk][r] = va;
      Bs[kk][r] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[2], b[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          // conj(a) * b
          ar[p][q] += a[p].x * b[q].x + a[p].y * b[q].y;
          ai[p][q] += a[p].x * b[q].y - a[p].y * b[q].x;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + ty + 16 * p, j = j0 + tx + 16 * q;
      if (i < m && j < n) {
        double2* c = Cacc + (long long)i * n + j;
        atomicAdd(&c->x, (double)ar[p][q]);
        atomicAdd(&c->y, (double)ai[p][q]);
      }
    }
}

__global__ void k_c128_to_c64(const double2* __restrict__ a, float2* __restrict__ b, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// C = A B, row-major complex64 A (m x k) and B (k x n); C complex64 or
// complex128 (row-major, n columns).  32 x 64 tile per CTA.
template <typename TC>
__global__ void __launch_bounds__(256) k_cgemm_nn(int m, int n, int k, const float2* __restrict__ A,
                                                 const float2* __restrict__ B, TC* __restrict__ C) {
  constexpr int BM = 32, BN = 64, BK = 16;
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float cr[2][4] = {}, ci[2][4] = {};
  for (int kb = 0; kb < k; kb += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int r = e / BK, kk = e % BK;
      As[kk][r] = (m0 + r < m && kb + kk < k) ? A[(long long)(m0 + r) * k + kb + kk] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      const int kk = e / BN, c = e % BN;
      Bs[kk][c] = (kb + kk < k && n0 + c < n) ? B[(long long)(kb + kk) * n + n0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[2], b[4];
#pragma unroll
      for (int p = 0; p < 2; ++p) a[p] = As[kk][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          cr[p][q] += a[p].x * b[q].x - a[p].y * b[q].y;
          ci[p][q] += a[p].x * b[q].y + a[p].y * b[q].x;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + ty + 16 * p, j = n0 + tx + 16 * q;
      if (i < m && j < n) {
        TC v;
        v.x = cr[p][q];
        v.y = ci[p][q];
        C[(long long)i * n + j] = v;
      }
    }
}

}  // namespace sgi

using namespace sgi;

extern "C" {

sg_status sg_cgemm_hn(const void* A, long long lda, const void* B, long long ldb, int m, int n, long long k, void* C,
                      void* workspace, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!A || !B || !C || !workspace || m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < k)
      return fail(SG_EINVAL, "bad sg_cgemm_hn arguments");
    cudaStream_t st = (cudaStream_t)stream;
    double2* acc = reinterpret_cast<double2*>(workspace);
    SG_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)m * n * sizeof(double2), st));
    const long long tiles = (long long)((m + 31) / 32) * ((n + 31) / 32);
    // slices of at most 1024 terms keep the FP32 partial sums short; more
    // slices than that only when the tiles alone would leave SMs idle
    const long long by_len = (k + 1023) / 1024;
    const long long by_occ = std::min((k + 15) / 16, (4LL * 152 + tiles - 1) / tiles);
    const int slices = (int)std::min(65535LL, std::max(by_len, by_occ));
    dim3 grid((n + 31) / 32, (m + 31) / 32, slices);
    k_cgemm_hn<<<grid, 256, 0, st>>>(m, n, k, (const float2*)A, lda, (const float2*)B, ldb, acc);
    note_launch();
    SG_CUDA_TRY(cudaGetLastError());
    const long long cnt = (long long)m * n;
    k_c128_to_c64<<<(int)std::min((cnt + 255) / 256, 4096LL), 256, 0, st>>>(acc, (float2*)C, cnt);
    note_launch();
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
  });
}

sg_status sg_cgemm_nn(const void* A, const void* B, int m, int n, int k, void* C, int out_c128, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!A || !B || !C || m <= 0 || n <= 0 || k <= 0) return fail(SG_EINVAL, "bad sg_cgemm_nn arguments");
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid((n + 63) / 64, (m + 31) / 32);
    if (out_c128)
      k_cgemm_nn<double2><<<grid, 256, 0, st>>>(m, n, k, (const float2*)A, (const float2*)B, (double2*)C);
    else
      k_cgemm_nn<float2><<<grid, 256, 0, st>>>(m, n, k, (const float2*)A, (const float2*)B, (float2*)C);
    note_launch();
    SG_CUDA_TRY(cudaGetLastError());
    return SG_OK;
  });
}

}  // extern "C"
