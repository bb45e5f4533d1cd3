// Banded LU with FP64 partial pivoting on the device, and its solves for
// many right-hand sides (band_core.h holds the per-thread phases).
//
// Uses: the mean-value and CSL mean-value blocks S(xi_bar) of 2D problems
// whose k_0 varies in space (the paper's wedge, Sec. 7), which have no
// separable inverse: the n x n block, unknowns x fastest, has kl = ku = mx
// (UMFPACK's LU in the paper, Sec. 6.3; one factorisation for all P modes);
// and the coupled CSL matrix M(beta) = A - i beta K of Sec. 4 in 1D, banded
// with kl = ku = P when the unknowns are numbered point by point.
//
//  * k_band_factor: one CTA walks the n columns (the elimination is
//    sequential in j); in each step the CTA finds the pivot, swaps, forms the
//    multipliers and applies the rank-one update of the (kl) x (kl + ku)
//    window, phases separated by barriers.  FP64 throughout.
//  * k_band_solve: one CTA per group of right-hand sides; a window of the
//    last rows of its right-hand sides lives in shared memory (forward sweep
//    kl + 1 rows, backward sweep kl + ku + 1 rows), the factor columns are
//    copied ahead in chunks by cp.async (double buffered), so each step
//    costs three barriers and a few shared-memory updates.  FP64 or FP32
//    (an FP32 copy of the factor, pivots from the FP64 factorisation).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <string>

#include "band_core.h"
#include "sg_internal.h"

namespace sgi {

constexpr int BF_THREADS = 1024;
constexpr int BS_THREADS = 512;

__global__ void __launch_bounds__(BF_THREADS) k_band_factor(int n, int kl, int ku, int ldab, double2* ab, int* piv,
                                                            int* bad) {
  extern __shared__ double2 bf_sm[];           // multipliers (kl) and U row (kl + ku)
  __shared__ double rv[BF_THREADS / 32];
  __shared__ int ri[BF_THREADS / 32];
  __shared__ int s_p;
  __shared__ double2 s_rinv;
  const int kv = kl + ku, t = threadIdx.x, nt = blockDim.x, lane = t & 31, warp = t >> 5;
  double2* lcol = bf_sm;
  double2* urow = bf_sm + kl;
  for (int j = 0; j < n; ++j) {
    const int last = min(n - 1, j + kl), clast = min(n - 1, j + kv);
    double best;
    int row;
    band::pivot_candidates(ab, kv, ldab, j, last, t, nt, &best, &row);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, row, o);
      if (ob > best || (ob == best && oi < row)) {
        best = ob;
        row = oi;
      }
    }
    if (lane == 0) {
      rv[warp] = best;
      ri[warp] = row;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < nt / 32 ? rv[lane] : -1.0;
      row = lane < nt / 32 ? ri[lane] : INT_MAX;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, row, o);
        if (ob > best || (ob == best && oi < row)) {
          best = ob;
          row = oi;
        }
      }
      if (lane == 0) {
        s_p = row;
        piv[j] = row;
        if (!(best > 0.0)) *bad = 1;
      }
    }
    __syncthreads();
    band::swap_rows(ab, kv, ldab, j, s_p, clast, t, nt);
    __syncthreads();
    if (t == 0) {
      const double2 d = ab[band::at(kv, ldab, j, j)];
      double den = d.x * d.x + d.y * d.y;
      if (!(den > 0.0)) {
        *bad = 1;
        den = 1e-300;
      }
      s_rinv = make_double2(d.x / den, -d.y / den);
    }
    __syncthreads();
    band::multipliers(ab, kv, ldab, j, last, clast, s_rinv, lcol, urow, t, nt);
    __syncthreads();
    band::rank1_update(ab, kv, ldab, j, last, clast, lcol, urow, t, nt);
    __syncthreads();
  }
}

__global__ void k_band_to32(const double2* __restrict__ a, float2* __restrict__ b, long long count) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

template <typename T>
__device__ __forceinline__ void cp_elem(C2<T>* dst, const C2<T>* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

// Z = U^-1 L^-1 P (s R) for nrhs right-hand sides (column q at q * ld; s =
// *in_scale or 1), Y the intermediate L^-1 P s R (may alias R and Z).
// CTA b owns right-hand sides [b pc, b pc + pc).  Shared memory: the window
// ((kv + 1) x pc), two buffers of nch factor columns ((kv + 1) each) and
// their pivots.
template <typename T>
__global__ void __launch_bounds__(BS_THREADS) k_band_solve(int n, int kl, int ku, int ldab,
                                                           const C2<T>* __restrict__ ab, const int* __restrict__ piv,
                                                           int nrhs, int pc, int nch, const C2<T>* R, C2<T>* Y,
                                                           C2<T>* Z, long long ld, const int* skip,
                                                           const double* in_scale) {
  using C = C2<T>;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char bs_raw[];
  const int kv = kl + ku, W = kv + 1, t = threadIdx.x, nt = blockDim.x;
  const int q0 = blockIdx.x * pc, pcb = min(pc, nrhs - q0);
  C* win = reinterpret_cast<C*>(bs_raw);
  C* fb = win + (size_t)W * pc;                                   // [2][nch][W]
  int* pb = reinterpret_cast<int*>(fb + (size_t)2 * nch * W);     // [2][nch]
  const T sc = in_scale ? (T)*in_scale : (T)1;

  // ---------------------------------------------------------------- forward sweep
  const int W1 = kl + 1;
  auto issue_fwd = [&](int c) {
    const int j0 = c * nch;
    if (j0 >= n) return;
    C* dst = fb + (size_t)(c & 1) * nch * W;
    for (int idx = t; idx < nch * kl; idx += nt) {
      const int jj = idx / kl, ii = idx - jj * kl, j = j0 + jj;
      if (j < n && j + 1 + ii < n) cp_elem<T>(dst + (size_t)jj * W + ii, ab + band::at(kv, ldab, j + 1 + ii, j));
    }
    for (int jj = t; jj < nch; jj += nt)
      if (j0 + jj < n) pb[(c & 1) * nch + jj] = piv[j0 + jj];
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  {
    const int rows = min(kl, n - 1) + 1;
    for (int idx = t; idx < rows * pcb; idx += nt) {
      const int r = idx / pcb, q = idx - r * pcb;
      C v = R[(long long)(q0 + q) * ld + r];
      v.x *= sc;
      v.y *= sc;
      win[(size_t)(r % W1) * pcb + q] = v;
    }
  }
  issue_fwd(0);
  for (int j = 0; j < n; ++j) {
    const int c = j / nch, jj = j - c * nch;
    if (jj == 0) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
      issue_fwd(c + 1);
    }
    band::fwd_swap(win, W1, pcb, j, pb[(c & 1) * nch + jj], t);
    __syncthreads();
    band::fwd_update(win, W1, pcb, fb + ((size_t)(c & 1) * nch + jj) * W, j, n, kl, t, nt, Y, ld, q0);
    __syncthreads();
    if (j + kl + 1 < n && t < pcb) {
      C v = R[(long long)(q0 + t) * ld + j + kl + 1];
      v.x *= sc;
      v.y *= sc;
      win[(size_t)(j % W1) * pcb + t] = v;
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();

  // ---------------------------------------------------------------- backward sweep
  auto issue_bwd = [&](int c) {
    const int jtop = n - 1 - c * nch;
    if (jtop < 0) return;
    C* dst = fb + (size_t)(c & 1) * nch * W;
    for (int idx = t; idx < nch * W; idx += nt) {
      const int jj = idx / W, e = idx - jj * W, j = jtop - jj;
      if (j >= 0 && e >= kv - j) cp_elem<T>(dst + (size_t)jj * W + e, ab + (long long)j * ldab + e);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  {
    const int lo = max(0, n - 1 - kv);
    for (int idx = t; idx < (n - lo) * pcb; idx += nt) {
      const int r = lo + idx / pcb, q = idx % pcb;
      win[(size_t)(r % W) * pcb + q] = Y[(long long)(q0 + q) * ld + r];
    }
  }
  issue_bwd(0);
  for (int j = n - 1; j >= 0; --j) {
    const int k = n - 1 - j, c = k / nch, jj = k - c * nch;
    if (jj == 0) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
      issue_bwd(c + 1);
    }
    const C* col = fb + ((size_t)(c & 1) * nch + jj) * W;
    const C d = col[kv];
    const T den = d.x * d.x + d.y * d.y;
    C dinv;
    dinv.x = d.x / den;
    dinv.y = -d.y / den;
    band::bwd_update(win, W, pcb, col, dinv, j, kv, t, nt, Z, ld, q0);
    __syncthreads();
    if (j - kv - 1 >= 0 && t < pcb) win[(size_t)(j % W) * pcb + t] = Y[(long long)(q0 + t) * ld + j - kv - 1];
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Shared memory budget of the solve kernel, and its split: right-hand sides
// per CTA (pc) and factor columns per prefetched chunk (nch).
constexpr size_t kBandSmem = 200 * 1024;

static bool band_plan(int kl, int ku, int nrhs, size_t esize, int* pc, int* nch, size_t* smem) {
  const size_t W = (size_t)kl + ku + 1;
  for (int ch = 8; ch >= 1; ch /= 2) {
    const size_t fixed = 2 * (size_t)ch * W * esize + 2 * (size_t)ch * sizeof(int);
    if (fixed + W * esize > kBandSmem) continue;
    int p = (int)std::min<size_t>((kBandSmem - fixed) / (W * esize), 64);
    p = std::min(p, nrhs);
    if (p < 1) continue;
    *pc = p;
    *nch = ch;
    *smem = fixed + W * esize * (size_t)p;
    return true;
  }
  return false;
}

cudaError_t band_factor(BandFactor& f, int* d_bad, cudaStream_t st) {
  const size_t smem = (size_t)(2 * f.kl + f.ku) * sizeof(double2);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_band_factor<<<1, BF_THREADS, smem, st>>>(f.n, f.kl, f.ku, f.ldab, f.ab, f.piv, d_bad);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long cnt = (long long)f.ldab * f.n;
  k_band_to32<<<(unsigned)std::min<long long>((cnt + 255) / 256, 4096), 256, 0, st>>>(f.ab, f.ab32, cnt);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t band_solve(const BandFactor& f, int nrhs, const C2<T>* R, C2<T>* Y, C2<T>* Z, long long ld,
                       cudaStream_t st, const int* skip, const double* in_scale) {
  int pc = 0, nch = 0;
  size_t smem = 0;
  if (!band_plan(f.kl, f.ku, nrhs, sizeof(C2<T>), &pc, &nch, &smem)) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_band_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmem);
  if (e != cudaSuccess) return e;
  const C2<T>* fab;
  if constexpr (sizeof(T) == 8) fab = f.ab; else fab = f.ab32;
  k_band_solve<T><<<(nrhs + pc - 1) / pc, BS_THREADS, smem, st>>>(f.n, f.kl, f.ku, f.ldab, fab, f.piv, nrhs, pc, nch,
                                                                 R, Y, Z, ld, skip, in_scale);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t band_solve<double>(const BandFactor&, int, const double2*, double2*, double2*, long long,
                                        cudaStream_t, const int*, const double*);
template cudaError_t band_solve<float>(const BandFactor&, int, const float2*, float2*, float2*, long long, cudaStream_t,
                                       const int*, const double*);

// Whether a band of this shape fits the solve kernel's shared memory.
bool band_fits(int kl, int ku) {
  int pc, nch;
  size_t smem;
  return band_plan(kl, ku, 1, sizeof(double2), &pc, &nch, &smem);
}

}  // namespace sgi
