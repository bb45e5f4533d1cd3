// Block preconditioners of Sec. 5 and Sec. 6.3 applied to all P chaos modes
// with one factorisation:  Z = (I_P (x) S_blk)^-1 R.
//
// 1D: S_blk is tridiagonal (Theorems A.1/A.2); LU with partial pivoting in
//     FP64 (LAPACK gttrf scheme) and a forward/back substitution per mode.
// 2D with constant k_0 (Theorems A.5/A.6): S_blk = D_y (x) H_x + H_y (x) D_x
//     with H = T - i (k_0/h) E - (k_0^2/2) D per direction.  With
//     G = D^-1/2 H D^-1/2 = Q Lambda Q^T (complex symmetric, Q^T Q = I) the
//     Sylvester form G_x W + W G_y = D_x^-1/2 R D_y^-1/2 is solved by
//       (1) Z' = R Qhat            (Qhat = D_x^-1/2 Q; one complex GEMM over
//                                   all P*my lines of length mx),
//       (2) per eigen-index i: ((lambda_i + shift) I + G_y) z_i = d_y^-1/2 z'_i
//           (tridiagonal along y, LU with partial pivoting in FP64),
//       (3) Z = (d_y^-1/2 z) Qhat^T (second GEMM).
//     The CSL block adds -i beta k_0^2 D_2, i.e. shift = -i beta k_0^2.
//     FP32 applies on grids with lines of at most 320 unknowns diagonalise
//     the y direction too (G_y = Q_y Lambda_y Q_y^T; the fast diagonalisation
//     of Lynch, Rice and Thomas, 1964): four GEMMs and an elementwise
//     division by lambda_y,j + lambda_x,i + shift, which keeps every step
//     parallel instead of mx * P sequential sweeps of length my.
#include <cuda_runtime.h>

#include <cmath>

#include <mutex>

#include "sg_internal.h"

namespace sgi {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double zabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / den, (a.y - a.x * r) / den);
  } else {
    double r = b.x / b.y, den = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / den, (a.y * r - a.x) / den);
  }
}

// One thread per system: LU with partial pivoting of the tridiagonal matrix
// with diagonal diag[j] + lam_shift[sys] and symmetric off-diagonal off[j]
// (real).  Writes FP64 factors and FP32 copies; sets *bad on a zero pivot.
__global__ void k_tri_factor(int nsys, int len, const double2* __restrict__ diag,
                             const double2* __restrict__ lam_shift, const double* __restrict__ off,
                             TriFactors<double> F, TriFactors<float> G, int* bad) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= nsys) return;
  const double2 sh = lam_shift ? lam_shift[sys] : make_double2(0, 0);
  auto at = [&](int j) { return (size_t)j * nsys + sys; };
  // d_j, du_j, dl_j of the current (partially eliminated) rows
  double2 dcur = make_double2(diag[0].x + sh.x, diag[0].y + sh.y);
  double2 ducur = make_double2(len > 1 ? off[0] : 0.0, 0.0);
  double2 du2prev = make_double2(0, 0);
  bool zero = false;
  for (int j = 0; j < len; ++j) {
    if (j == len - 1) {
      if (dcur.x == 0.0 && dcur.y == 0.0) zero = true;
      const double2 di = zero ? make_double2(0, 0) : zdiv(make_double2(1, 0), dcur);
      F.dinv[at(j)] = di;
      F.du[at(j)] = make_double2(0, 0);
      F.du2[at(j)] = make_double2(0, 0);
      F.dl[at(j)] = make_double2(0, 0);
      F.piv[at(j)] = 0;
      break;
    }
    const double2 dl = make_double2(off[j], 0.0);             // sub-diagonal entry (row j+1, col j)
    const double2 dnext = make_double2(diag[j + 1].x + sh.x, diag[j + 1].y + sh.y);
    const double2 dunext = make_double2(j + 2 < len ? off[j + 1] : 0.0, 0.0);
    double2 fact, d_j, du_j, du2_j, d_n, du_n;
    uint8_t p;
    if (zabs1(dcur) >= zabs1(dl)) {
      if (dcur.x == 0.0 && dcur.y == 0.0) { zero = true; fact = make_double2(0, 0); }
      else fact = zdiv(dl, dcur);
      d_j = dcur; du_j = ducur; du2_j = make_double2(0, 0);
      d_n = zsub(dnext, zmul(fact, ducur));
      du_n = dunext;
      p = 0;
    } else {
      fact = zdiv(dcur, dl);
      d_j = dl;
      du_j = dnext;
      d_n = zsub(ducur, zmul(fact, dnext));
      du2_j = dunext;
      du_n = make_double2(-(fact.x * dunext.x - fact.y * dunext.y), -(fact.x * dunext.y + fact.y * dunext.x));
      p = 1;
    }
    (void)du2prev;
    F.dl[at(j)] = fact;
    F.dinv[at(j)] = zdiv(make_double2(1, 0), d_j);
    F.du[at(j)] = du_j;
    F.du2[at(j)] = du2_j;
    F.piv[at(j)] = p;
    dcur = d_n;
    ducur = du_n;
  }
  for (int j = 0; j < len; ++j) {
    const size_t k = at(j);
    G.dl[k] = make_float2((float)F.dl[k].x, (float)F.dl[k].y);
    G.dinv[k] = make_float2((float)F.dinv[k].x, (float)F.dinv[k].y);
    G.du[k] = make_float2((float)F.du[k].x, (float)F.du[k].y);
    G.du2[k] = make_float2((float)F.du2[k].x, (float)F.du2[k].y);
  }
  if (zero) atomicExch(bad, 1);
}

cudaError_t launch_tri_factor(int nsys, int len, const double2* diag, const double2* lam_shift, const double* off,
                              TriFactors<double> f64, TriFactors<float> f32, int* d_bad, cudaStream_t st) {
  const int blk = 128;
  k_tri_factor<<<(nsys + blk - 1) / blk, blk, 0, st>>>(nsys, len, diag, lam_shift, off, f64, f32, d_bad); note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- complex helpers
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  C2<T> r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) {
  C2<T> r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}
template <typename T>
__device__ __forceinline__ C2<T> cscale(C2<T> a, T s) {
  C2<T> r;
  r.x = a.x * s;
  r.y = a.y * s;
  return r;
}

// Multi-RHS tridiagonal solve with gttrf factors.  Thread (sys, rhs) walks
// j = 0..len-1; element address rhs*sR + j*sJ + sys*sS; factors at
// j*nsys + sys.  Optional row scaling s_j applied to the input and the output
// (2D: d_y^-1/2) and an optional scalar on the input (the solve is linear).
// R and Z must not overlap: the sweeps load CH rows ahead of the dependent
// recurrence so the loads of a chunk overlap each other.
template <typename T>
__global__ void k_tri_solve(int nsys, int nrhs, int len, long long sR, long long sJ, long long sS,
                            TriFactors<T> F, const T* __restrict__ rowscale, const C2<T>* __restrict__ R,
                            C2<T>* __restrict__ Z, const int* skip, const double* in_scale) {
  if (skip && *skip) return;
  constexpr int CH = 8;
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y * blockDim.y + threadIdx.y;
  if (sys >= nsys || rhs >= nrhs) return;
  const C2<T>* r = R + rhs * sR + sys * sS;
  C2<T>* z = Z + rhs * sR + sys * sS;
  auto f = [&](int j) { return (size_t)j * nsys + sys; };
  const T s0 = in_scale ? (T)*in_scale : T(1);
  // forward: row interchanges and L
  C2<T> cur = cscale<T>(r[0], rowscale ? rowscale[0] * s0 : s0);
  for (int j0 = 0; j0 + 1 < len; j0 += CH) {
    C2<T> rv[CH], lv[CH];
    uint8_t pv[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int j = j0 + q;
      if (j + 1 < len) {
        rv[q] = cscale<T>(r[(j + 1) * sJ], rowscale ? rowscale[j + 1] * s0 : s0);
        lv[q] = F.dl[f(j)];
        pv[q] = F.piv[f(j)];
      }
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int j = j0 + q;
      if (j + 1 < len) {
        if (!pv[q]) {
          z[j * sJ] = cur;
          cur = csub<T>(rv[q], cmul<T>(lv[q], cur));
        } else {
          z[j * sJ] = rv[q];
          cur = csub<T>(cur, cmul<T>(lv[q], rv[q]));
        }
      }
    }
  }
  // back substitution with U (diagonal, du, du2)
  C2<T> x1 = cmul<T>(cur, F.dinv[f(len - 1)]);  // x_{j+1}
  C2<T> x2;                                        // x_{j+2}
  x2.x = T(0);
  x2.y = T(0);
  z[(len - 1) * sJ] = rowscale ? cscale<T>(x1, rowscale[len - 1]) : x1;
  for (int j0 = len - 2; j0 >= 0; j0 -= CH) {
    C2<T> bv[CH], uv[CH], u2v[CH], dv[CH];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int j = j0 - q;
      if (j >= 0) {
        bv[q] = z[j * sJ];
        uv[q] = F.du[f(j)];
        u2v[q] = F.du2[f(j)];
        dv[q] = F.dinv[f(j)];
      }
    }
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int j = j0 - q;
      if (j >= 0) {
        C2<T> b = csub<T>(bv[q], cmul<T>(uv[q], x1));
        b = csub<T>(b, cmul<T>(u2v[q], x2));
        const C2<T> xj = cmul<T>(b, dv[q]);
        z[j * sJ] = rowscale ? cscale<T>(xj, rowscale[j]) : xj;
        x2 = x1;
        x1 = xj;
      }
    }
  }
}

// 1D block solve for a few right-hand sides: the factors and this CTA's
// right-hand sides are staged in shared memory (coalesced), one thread per
// right-hand side sweeps forward and back in shared memory (a dependent step
// costs a shared-memory latency instead of a global one), then the CTA writes
// the solutions back.  Same gttrs steps as k_tri_solve; in place in shared
// memory (step j writes row j after reading row j+1).  R and Z may coincide.
template <typename T>
__global__ void __launch_bounds__(256) k_tri_solve_1d(int n, int P, int rhs_per_cta, TriFactors<T> F,
                                                      const C2<T>* R, C2<T>* Z,
                                                      const int* skip, const double* in_scale) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  C2<T>* sdl = reinterpret_cast<C2<T>*>(smraw);
  C2<T>* sdu = sdl + n;
  C2<T>* sdu2 = sdu + n;
  C2<T>* sdinv = sdu2 + n;
  C2<T>* sx = sdinv + n;                                   // [rhs][n + 1]
  uint8_t* spiv = reinterpret_cast<uint8_t*>(sx + (size_t)rhs_per_cta * (n + 1));
  const int p0 = blockIdx.x * rhs_per_cta, np = min(rhs_per_cta, P - p0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sdl[i] = F.dl[i];
    sdu[i] = F.du[i];
    sdu2[i] = F.du2[i];
    sdinv[i] = F.dinv[i];
    spiv[i] = F.piv[i];
  }
  const T s0 = in_scale ? (T)*in_scale : T(1);
  for (int i = threadIdx.x; i < np * n; i += blockDim.x) {
    const int q = i / n, j = i - q * n;
    sx[q * (n + 1) + j] = cscale<T>(R[(size_t)p0 * n + i], s0);
  }
  __syncthreads();
  if (threadIdx.x < np) {
    C2<T>* x = sx + threadIdx.x * (n + 1);
    C2<T> cur = x[0];
    for (int j = 0; j + 1 < n; ++j) {
      const C2<T> rn = x[j + 1], l = sdl[j];
      if (!spiv[j]) {
        x[j] = cur;
        cur = csub<T>(rn, cmul<T>(l, cur));
      } else {
        x[j] = rn;
        cur = csub<T>(cur, cmul<T>(l, rn));
      }
    }
    C2<T> x1 = cmul<T>(cur, sdinv[n - 1]), x2;
    x2.x = T(0);
    x2.y = T(0);
    x[n - 1] = x1;
    for (int j = n - 2; j >= 0; --j) {
      C2<T> b = csub<T>(x[j], cmul<T>(sdu[j], x1));
      b = csub<T>(b, cmul<T>(sdu2[j], x2));
      const C2<T> xj = cmul<T>(b, sdinv[j]);
      x[j] = xj;
      x2 = x1;
      x1 = xj;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < np * n; i += blockDim.x) {
    const int q = i / n, j = i - q * n;
    Z[(size_t)p0 * n + i] = sx[q * (n + 1) + j];
  }
}

// Shared memory of k_tri_solve_1d for rhs right-hand sides of length n.
template <typename T>
static size_t tri1d_smem(int n, int rhs) {
  return (size_t)n * (4 * sizeof(C2<T>) + 1) + (size_t)rhs * (n + 1) * sizeof(C2<T>) + 16;
}
constexpr size_t kTri1dSmemMax = 200 * 1024;

// ---------------------------------------------------------------- batched complex GEMM
// C_b = A_b B_b for b = blockIdx.z, complex, row-major with row strides lda,
// ldb, ldc and batch strides sA, sB, sC (0: operand shared by the batch).
// Optional epilogue: C *= E[m * N + n] * (*escale).  CUDA cores, FP32 or FP64
// accumulation in the element type.  (16*TM) x (16*TN) output tile per CTA,
// 256 threads with TM x TN outputs each; K in chunks of KC staged in shared
// memory by cp.async, two chunks in flight.
__device__ __forceinline__ void cp_async_zfill(void* smem, const void* gmem, int bytes_valid, int size) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
  if (size == 16)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem), "r"(bytes_valid));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gmem), "r"(bytes_valid));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND)); }

__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

template <typename T, int TM, int TN, bool EPI>
__global__ void __launch_bounds__(256) k_cgemm(int M, int Nn, int K, const C2<T>* __restrict__ A, long long lda,
                                              long long sA, const C2<T>* __restrict__ B, long long ldb, long long sB,
                                              C2<T>* __restrict__ C, long long ldc, long long sC,
                                              const C2<T>* __restrict__ E, const double* __restrict__ escale,
                                              const int* skip) {
  if (skip && *skip) return;
  constexpr int BM = 16 * TM, BN = 16 * TN, KC = sizeof(T) == 4 ? 16 : 8;   // 33 KB of shared memory at 4 x 4
  constexpr int ES = (int)sizeof(C2<T>);
  __shared__ C2<T> As[2][KC][BM + 1];
  __shared__ C2<T> Bs[2][KC][BN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
  C += blockIdx.z * sC;
  auto load = [&](int buf, int k0) {
    for (int e = threadIdx.x; e < BM * KC; e += 256) {
      const int mm = e / KC, kk = e % KC;
      const int gm = m0 + mm, gk = k0 + kk;
      const bool ok = gm < M && gk < K;
      cp_async_zfill(&As[buf][kk][mm], ok ? (const void*)(A + (size_t)gm * lda + gk) : (const void*)A, ok ? ES : 0,
                     ES);
    }
    for (int e = threadIdx.x; e < KC * BN; e += 256) {
      const int kk = e / BN, nn = e % BN;
      const int gk = k0 + kk, gn = n0 + nn;
      const bool ok = gk < K && gn < Nn;
      cp_async_zfill(&Bs[buf][kk][nn], ok ? (const void*)(B + (size_t)gk * ldb + gn) : (const void*)B, ok ? ES : 0,
                     ES);
    }
    cp_async_commit();
  };
  T accr[TM][TN], acci[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) accr[i][j] = acci[i][j] = T(0);
  const int nch = (K + KC - 1) / KC;
  load(0, 0);
  for (int c = 0; c < nch; ++c) {
    const int buf = c & 1;
    if (c + 1 < nch) {
      load(buf ^ 1, (c + 1) * KC);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      C2<T> a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          // four fused multiply-adds per complex product
          accr[i][j] = fmat(a[i].x, b[j].x, fmat(-a[i].y, b[j].y, accr[i][j]));
          acci[i][j] = fmat(a[i].x, b[j].y, fmat(a[i].y, b[j].x, acci[i][j]));
        }
    }
    __syncthreads();
  }
  T es = T(1);
  if (EPI && escale) es = (T)*escale;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < Nn) {
        C2<T> v;
        v.x = accr[i][j];
        v.y = acci[i][j];
        if (EPI) {
          const C2<T> w = E[(size_t)gm * Nn + gn];
          C2<T> u;
          u.x = (v.x * w.x - v.y * w.y) * es;
          u.y = (v.x * w.y + v.y * w.x) * es;
          v = u;
        }
        C[(size_t)gm * ldc + gn] = v;
      }
    }
  }
}

// C_b = A_b B_b (+ epilogue E, escale) over `batch` problems; picks the
// larger tile when it still gives two CTAs per SM.
template <typename T>
static cudaError_t cgemm(const sg_handle* h, int M, int Nn, int K, const C2<T>* A, long long lda, long long sA,
                         const C2<T>* B, long long ldb, long long sB, C2<T>* C, long long ldc, long long sC,
                         int batch, cudaStream_t st, const int* skip, const C2<T>* E = nullptr,
                         const double* escale = nullptr) {
  const long long tiles64 = (long long)((Nn + 63) / 64) * ((M + 63) / 64) * batch;
  const bool big = tiles64 >= 2LL * h->num_sms;
  const int bm = big ? 64 : 32, bn = big ? 64 : 32;
  dim3 grid((Nn + bn - 1) / bn, (M + bm - 1) / bm, batch);
  if (big) {
    if (E) k_cgemm<T, 4, 4, true><<<grid, 256, 0, st>>>(M, Nn, K, A, lda, sA, B, ldb, sB, C, ldc, sC, E, escale, skip);
    else k_cgemm<T, 4, 4, false><<<grid, 256, 0, st>>>(M, Nn, K, A, lda, sA, B, ldb, sB, C, ldc, sC, E, escale, skip);
  } else {
    if (E) k_cgemm<T, 2, 2, true><<<grid, 256, 0, st>>>(M, Nn, K, A, lda, sA, B, ldb, sB, C, ldc, sC, E, escale, skip);
    else k_cgemm<T, 2, 2, false><<<grid, 256, 0, st>>>(M, Nn, K, A, lda, sA, B, ldb, sB, C, ldc, sC, E, escale, skip);
  }
  note_launch();
  return cudaGetLastError();
}

// FP32 2D apply by fast diagonalisation: tensor-core transforms, each a GEMM
// with a constant right factor; the per-batch transposes in (1) and (3) move
// the direction being transformed into the rows' contiguous index:
//   (1) T1'_p = (R_p Qhat_x)^T          [p][i][y]
//   (2) T2'_p = L^-1 o (T1'_p Qhat_y)   [p][i][j], L^-1 indexed (j, i)
//   (3) T3_p  = (T2'_p Qhat_y^T)^T      [p][y][i]
//   (4) Z_p   = T3_p Qhat_x^T           [p][y][x]
// The intermediates keep rows of even length (my or mx rounded up to even),
// so the next transform reads them with 16-byte copies; their P mx myp or
// P my mxp complex values fit in the scratch of N complex128 (= 2N
// complex64).  split: FP32 accuracy (3xTF32), else plain TF32.
static cudaError_t fd_apply(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                            const int* skip, const double* in_scale, float2* tmp, float2* tmp2, bool split) {
  const int mx = h->mx, my = h->my, P = h->P;
  const int mxp = mx + (mx & 1), myp = my + (my & 1);
  // plain TF32 on the handle's own intermediates: transforms 2-4 read them by
  // tensor copies (maps encoded at set-up)
  const bool maps = !split && h->tc_xmap_ok && tmp == reinterpret_cast<const float2*>(h->d_tmp) &&
                    tmp2 == reinterpret_cast<const float2*>(h->d_tmp2);
  cudaError_t e =
      tc_cgemm(h->tcB[0], R, mx, P * my, tmp, myp, 1, my, nullptr, 0, 1, nullptr, skip, h->d_err, st, split);
  if (e == cudaSuccess)
    e = tc_cgemm(h->tcB[1], tmp, myp, P * mx, tmp2, myp, 0, 0, h->d_Linv32[which], mx, mx, in_scale, skip,
                 h->d_err, st, split, maps ? &h->tc_xmap[0] : nullptr);
  if (e == cudaSuccess)
    e = tc_cgemm(h->tcB[2], tmp2, myp, P * mx, tmp, mxp, 1, mx, nullptr, 0, 1, nullptr, skip, h->d_err, st, split,
                 maps ? &h->tc_xmap[1] : nullptr);
  if (e == cudaSuccess)
    e = tc_cgemm(h->tcB[3], tmp, mxp, P * my, Z, mx, 0, 0, nullptr, 0, 1, nullptr, skip, h->d_err, st, split,
                 maps ? &h->tc_xmap[2] : nullptr);
  return e;
}

// Binary16 transform t: the paired 256-column form where the handle is tuned
// to it, else the persistent 64/128-column form.
static cudaError_t hgemm(const sg_handle* h, int t, const void* X, int M, void* C, long long ldc, int mode, int MB,
                         const float2* E, int e_ld, int e_mod, const double* escale, float oscale, bool out_half,
                         const int* skip, int* err, cudaStream_t st, const CUtensorMap* xmap) {
  if (h->tc_wide && h->tcW[t].h16)
    return tc_hgemm_w(h->tcW[t], X, M, C, ldc, mode, MB, E, e_ld, e_mod, escale, oscale, out_half, skip, err, st,
                      xmap);
  return tc_hgemm(h->tcB[t], X, M, C, ldc, mode, MB, E, e_ld, e_mod, escale, oscale, out_half, skip, err, st, xmap);
}

// One plain-TF32 transform t of fd_apply (0 .. 3) on caller buffers, in the
// layouts listed there; X by tensor copies where its row pitch allows (a map
// encoded for X on each call), as the apply does on the handle's own buffers.
cudaError_t fd_transform(const sg_handle* h, int which, int t, const float2* X, float2* Y, cudaStream_t st,
                         bool f16) {
  if (h->dim != 2 || !h->fd || !h->blk[which].ready || t < 0 || t > 3) return cudaErrorNotSupported;
  if (f16) {
    // the binary16 route's transform t with the apply's fixed scales (the
    // input taken as unit norm): complex64 in for t = 0, out for t = 3,
    // binary16 pairs with rows padded to a multiple of 4 in between
    if (!h->fd16) return cudaErrorNotSupported;
    const int mx = h->mx, my = h->my, P = h->P;
    const int mx4 = (mx + 3) & ~3, my4 = (my + 3) & ~3;
    const float c1 = (float)std::sqrt((double)h->N), c2 = h->fd16_scale[which];
    if (t == 0)
      return tc_cgemm(h->tcB[0], X, mx, P * my, Y, my4, 1, my, nullptr, 0, 1, nullptr, nullptr, h->d_err, st, false,
                      nullptr, true, c1);
    const long long ldx[4] = {0, my4, my4, mx4}, ldc[4] = {0, my4, mx4, mx};
    const int rows[4] = {0, P * mx, P * mx, P * my}, kdim[4] = {0, my, my, mx};
    CUtensorMap map;
    if (!tc_make_xmap16(&map, X, ldx[t], rows[t], kdim[t])) return cudaErrorInvalidValue;
    if (t == 1)
      return hgemm(h, 1, X, rows[1], Y, ldc[1], 0, 0, h->d_Linv32[which], mx, mx, nullptr, c2, true, nullptr,
                      h->d_err, st, &map);
    if (t == 2)
      return hgemm(h, 2, X, rows[2], Y, ldc[2], 1, mx, nullptr, 0, 1, nullptr, 1.0f, true, nullptr, h->d_err,
                      st, &map);
    return hgemm(h, 3, X, rows[3], Y, ldc[3], 0, 0, nullptr, 0, 1, nullptr, 1.0f / (c1 * c2), false, nullptr,
                    h->d_err, st, &map);
  }
  const int mx = h->mx, my = h->my, P = h->P;
  const int mxp = mx + (mx & 1), myp = my + (my & 1);
  // (input pitch, rows, K, output pitch, mode, batch rows) of the four transforms
  const long long ldx[4] = {mx, myp, myp, mxp}, ldc[4] = {myp, myp, mxp, mx};
  const int rows[4] = {P * my, P * mx, P * mx, P * my}, kdim[4] = {mx, my, my, mx};
  const int mode[4] = {1, 0, 1, 0}, mb[4] = {my, 0, mx, 0};
  CUtensorMap map;
  const bool okm = tc_make_xmap(&map, X, ldx[t], rows[t], kdim[t]);
  return tc_cgemm(h->tcB[t], X, ldx[t], rows[t], Y, ldc[t], mode[t], mb[t], t == 1 ? h->d_Linv32[which] : nullptr,
                  t == 1 ? mx : 0, t == 1 ? mx : 1, nullptr, nullptr, h->d_err, st, false, okm ? &map : nullptr);
}

// ||R||^2 of N complex64 values in a fixed order: kFd16Blocks block sums,
// then one block adds them in order and stores 1 / ||R|| and ||R||.
__global__ void __launch_bounds__(256) k_fd16_norm_part(const float2* __restrict__ R, long long N,
                                                        double* __restrict__ part) {
  __shared__ double sm[256];
  // a thread's sum in FP32 (a scale factor needs no more), four loads in
  // flight; block and final sums in FP64
  float acc = 0.0f;
  const long long stride = (long long)gridDim.x * 256;
  long long e = blockIdx.x * 256LL + threadIdx.x;
  for (; e + 3 * stride < N; e += 4 * stride) {
    const float2 v0 = R[e], v1 = R[e + stride], v2 = R[e + 2 * stride], v3 = R[e + 3 * stride];
    acc += v0.x * v0.x + v0.y * v0.y + v1.x * v1.x + v1.y * v1.y + v2.x * v2.x + v2.y * v2.y + v3.x * v3.x +
           v3.y * v3.y;
  }
  for (; e < N; e += stride) {
    const float2 v = R[e];
    acc += v.x * v.x + v.y * v.y;
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void __launch_bounds__(256) k_fd16_norm_final(const double* __restrict__ part, int nb,
                                                         double* __restrict__ out) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += 256) acc += part[b];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nrm = sqrt(sm[0]);
    out[0] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    out[1] = nrm;
  }
}

// fd_apply with transforms 2-4 in binary16 (kind::f16): transform 1 (the
// odd-pitch complex64 input) stays TF32 and writes binary16 pairs.  Scaling
// keeps the binary16 values near 1: the input normalised (in_scale, else 1 /
// ||R|| computed here) times sqrt(N) (unit-norm vectors have entries near
// 1 / sqrt(N)); transform 2's L^-1 times 1 / max |L^-1|; transform 4 undoes
// both (and the norm when it was computed here).
static cudaError_t fd16_tail(const sg_handle* h, int which, float2* Z, cudaStream_t st, const int* skip,
                             const double* s_out);
static cudaError_t fd_apply_h(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                              const int* skip, const double* in_scale) {
  const int mx = h->mx, my = h->my, P = h->P;
  const int my4 = (my + 3) & ~3;
  const float c1 = (float)std::sqrt((double)h->N);
  const double* s_in = in_scale;
  const double* s_out = nullptr;
  cudaError_t e = cudaSuccess;
  if (!s_in) {
    k_fd16_norm_part<<<kFd16Blocks, 256, 0, st>>>(R, h->N, h->d_fd16part); note_launch();
    k_fd16_norm_final<<<1, 256, 0, st>>>(h->d_fd16part, kFd16Blocks, h->d_fd16s); note_launch();
    if ((e = cudaGetLastError())) return e;
    s_in = h->d_fd16s;
    s_out = h->d_fd16s + 1;
  }
  e = tc_cgemm(h->tcB[0], R, mx, P * my, reinterpret_cast<float2*>(h->d_tmp), my4, 1, my, nullptr, 0, 1, s_in,
               skip, h->d_err, st, false, nullptr, true, c1);
  return e ? e : fd16_tail(h, which, Z, st, skip, s_out);
}

// Transforms 2-4 of the binary16 apply: d_tmp (transform 1's output, scaled
// to sqrt(N) times a unit vector) -> Z, times *s_out if given.
static cudaError_t fd16_tail(const sg_handle* h, int which, float2* Z, cudaStream_t st, const int* skip,
                             const double* s_out) {
  const int mx = h->mx, my = h->my, P = h->P;
  const int mx4 = (mx + 3) & ~3, my4 = (my + 3) & ~3;
  const float c1 = (float)std::sqrt((double)h->N), c2 = h->fd16_scale[which];
  void* t1 = h->d_tmp;
  void* t2 = h->d_tmp2;
  cudaError_t e = hgemm(h, 1, t1, P * mx, t2, my4, 0, 0, h->d_Linv32[which], mx, mx, nullptr, c2, true,
                           skip, h->d_err, st, &h->tc_xmap16[0]);
  if (!e)
    e = hgemm(h, 2, t2, P * mx, t1, mx4, 1, mx, nullptr, 0, 1, nullptr, 1.0f, true, skip, h->d_err, st,
                 &h->tc_xmap16[1]);
  if (!e)
    e = hgemm(h, 3, t1, P * my, Z, mx, 0, 0, nullptr, 0, 1, s_out, 1.0f / (c1 * c2), false, skip,
                 h->d_err, st, &h->tc_xmap16[2]);
  return e;
}

cudaError_t launch_precond_f16_copy(const sg_handle* h, int which, const void* X16, const CUtensorMap* xmap,
                                    float2* Z, cudaStream_t st, const int* skip, const double* in_scale,
                                    float oscale) {
  if (h->dim != 2 || !h->fd || !h->fd16 || !h->blk[which].ready || !h->tcB[0].h16 || !X16 || !xmap || !in_scale)
    return cudaErrorNotSupported;
  // transform 1 as a binary16 GEMM: the copy's rows (K = mx) against Qhat_x,
  // per-batch transposed into d_tmp as fd_apply_h's transform 1 writes it
  const cudaError_t e = hgemm(h, 0, X16, h->P * h->my, h->d_tmp, (h->my + 3) & ~3, 1, h->my, nullptr, 0, 1,
                                 in_scale, oscale, true, skip, h->d_err, st, xmap);
  return e ? e : fd16_tail(h, which, Z, st, skip, nullptr);
}

cudaError_t launch_precond_f16(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                               const int* skip, const double* in_scale) {
  if (h->dim != 2 || !h->fd || !h->fd16 || !h->blk[which].ready) return cudaErrorNotSupported;
  if (!in_scale && (!h->d_fd16s || !h->d_fd16part)) return cudaErrorNotSupported;
  return fd_apply_h(h, which, R, Z, st, skip, in_scale);
}

cudaError_t launch_precond_fast(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                                const int* skip, const double* in_scale) {
  if (h->fd16 && !h->tune_tf32 && in_scale) return fd_apply_h(h, which, R, Z, st, skip, in_scale);
  return launch_precond_tf32(h, which, R, Z, st, skip, in_scale);
}

cudaError_t launch_precond_tf32(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                                const int* skip, const double* in_scale) {
  if (h->dim != 2 || !h->fd || !h->blk[which].ready) return cudaErrorNotSupported;
  return fd_apply(h, which, R, Z, st, skip, in_scale, reinterpret_cast<float2*>(h->d_tmp),
                  reinterpret_cast<float2*>(h->d_tmp2), false);
}

// Z = M^-1 R for block `which`; tmp and tmp2 hold N complex128 values each
// (tmp2 only for 2D; the FP32 2D transforms use up to 2N complex64 of each
// for their even-length rows).  R and Z may be the same vector.
// Mode-major (V_a over the grid, the ABI's layout) <-> point-by-point order
// (row u P + a, the coupled CSL band's numbering), with the input scale.
template <typename T>
__global__ void k_to_points(const C2<T>* __restrict__ R, int n, int P, C2<T>* __restrict__ out,
                            const double* __restrict__ in_scale, const int* skip) {
  if (skip && *skip) return;
  const T s = in_scale ? (T)*in_scale : (T)1;
  const long long N = (long long)n * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const long long u = e / P, a = e - u * P;
    C2<T> v = R[a * n + u];
    v.x *= s;
    v.y *= s;
    out[e] = v;
  }
}

template <typename T>
__global__ void k_from_points(const C2<T>* __restrict__ in, int n, int P, C2<T>* __restrict__ Z, const int* skip) {
  if (skip && *skip) return;
  const long long N = (long long)n * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const long long a = e / n, u = e - a * n;
    Z[e] = in[u * P + a];
  }
}

template <typename T>
static cudaError_t precond_apply(const sg_handle* h, int which, const C2<T>* R, C2<T>* Z, cudaStream_t st,
                                 const int* skip, const double* in_scale, C2<T>* tmp, C2<T>* tmp2) {
  if (which == 2) {
    // the coupled CSL matrix: its band is numbered point by point, one right-hand side
    if (!h->csl_full.ab) return cudaErrorNotReady;
    const long long N = h->N;
    const int grid = (int)std::min<long long>((N + 255) / 256, 4096);
    k_to_points<T><<<grid, 256, 0, st>>>(R, h->n, h->P, tmp, in_scale, skip);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = band_solve<T>(h->csl_full, 1, tmp, tmp, tmp, N, st, skip, nullptr);
    if (e != cudaSuccess) return e;
    k_from_points<T><<<grid, 256, 0, st>>>(tmp, h->n, h->P, Z, skip);
    note_launch();
    return cudaGetLastError();
  }
  const PrecBlock& blk = h->blk[which];
  TriFactors<T> F;
  if constexpr (sizeof(T) == 8) F = blk.f64; else F = blk.f32;
  if (h->dim == 1) {
    // one system of length n, P right-hand sides (the modes)
    const int n = h->n, P = h->P;
    if (tri1d_smem<T>(n, 1) <= kTri1dSmemMax) {
      static std::once_flag once;
      std::call_once(once, [] {
        cudaFuncSetAttribute(k_tri_solve_1d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTri1dSmemMax);
      });
      int rhs = 1;
      while (rhs < P && rhs < 256 && tri1d_smem<T>(n, rhs + 1) <= kTri1dSmemMax) ++rhs;
      const int grid = (P + rhs - 1) / rhs;
      k_tri_solve_1d<T><<<grid, 256, tri1d_smem<T>(n, rhs), st>>>(n, P, rhs, F, R, Z, skip, in_scale);
      note_launch();
      return cudaGetLastError();
    }
    // longer lines: sweeps from global memory, out of place
    dim3 b(1, 64), g(1, (h->P + 63) / 64);
    C2<T>* out = (R == Z) ? tmp : Z;
    k_tri_solve<T><<<g, b, 0, st>>>(1, h->P, h->n, h->n, 1, 0, F, nullptr, R, out, skip, in_scale);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && out != Z)
      e = cudaMemcpyAsync(Z, out, (size_t)h->N * sizeof(C2<T>), cudaMemcpyDeviceToDevice, st);
    return e;
  }
  const int mx = h->mx, my = h->my, P = h->P;
  const long long plane = (long long)mx * my;
  if (blk.band.ab)   // k_0 varies in space: banded LU of the n x n block, the P modes as right-hand sides
    return band_solve<T>(blk.band, P, R, tmp, Z, h->n, st, skip, in_scale);
  if constexpr (sizeof(T) == 4) {
    if (h->fd && h->fd_fp32) return fd_apply(h, which, R, Z, st, skip, in_scale, tmp, tmp2, true);
  }
  const C2<T>* Q;
  const C2<T>* Qt;
  const T* dyinv;
  if constexpr (sizeof(T) == 8) { Q = h->d_Q; Qt = h->d_Qt; dyinv = h->d_dyinv; }
  else { Q = h->d_Q32; Qt = h->d_Qt32; dyinv = h->d_dyinv32; }
  // FP32: the x transforms on the tensor cores (factors built at set-up for
  // lines longer than the fast-diagonalisation limit); FP64: CUDA cores
  bool tcx = false;
  if constexpr (sizeof(T) == 4) tcx = h->tcB[0].hi != nullptr && h->tcB[3].hi != nullptr;
  cudaError_t e = cudaSuccess;
  if (tcx) {
    if constexpr (sizeof(T) == 4)
      e = tc_cgemm(h->tcB[0], R, mx, P * my, tmp, mx, 0, 0, nullptr, 0, 1, nullptr, skip, h->d_err, st);   // (1)
  } else {
    e = cgemm<T>(h, P * my, mx, mx, R, mx, 0, Q, mx, 0, tmp, mx, 0, 1, st, skip);   // (1)
  }
  if (e != cudaSuccess) return e;
  dim3 b(32, 8), g((mx + 31) / 32, (P + 7) / 8);                     // (2) sys = i, rhs = mode, j = y line
  k_tri_solve<T><<<g, b, 0, st>>>(mx, P, my, plane, mx, 1, F, dyinv, tmp, tmp2, skip, in_scale);
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (tcx) {
    if constexpr (sizeof(T) == 4)
      return tc_cgemm(h->tcB[3], tmp2, mx, P * my, Z, mx, 0, 0, nullptr, 0, 1, nullptr, skip, h->d_err, st);   // (3)
  }
  return cgemm<T>(h, P * my, mx, mx, tmp2, mx, 0, Qt, mx, 0, Z, mx, 0, 1, st, skip);        // (3)
}

template <typename T>
cudaError_t launch_precond(const sg_handle* h, int which, const C2<T>* R, C2<T>* Z, cudaStream_t st,
                           const int* skip, const double* in_scale) {
  return precond_apply<T>(h, which, R, Z, st, skip, in_scale, reinterpret_cast<C2<T>*>(h->d_tmp),
                          reinterpret_cast<C2<T>*>(h->d_tmp2));
}

// Same preconditioner apply with caller-provided scratch: tmp and tmp2 each
// hold at least N complex128 values (2N complex64 when T is float; tmp2 is
// used by 2D problems only).
// Used by the allocation-free entry point.
template <typename T>
cudaError_t launch_precond_scratch(const sg_handle* h, int which, const C2<T>* R, C2<T>* Z, cudaStream_t st,
                                   C2<T>* tmp, C2<T>* tmp2) {
  return precond_apply<T>(h, which, R, Z, st, nullptr, nullptr, tmp, tmp2);
}

template cudaError_t launch_precond_scratch<double>(const sg_handle*, int, const double2*, double2*, cudaStream_t,
                                                    double2*, double2*);
template cudaError_t launch_precond_scratch<float>(const sg_handle*, int, const float2*, float2*, cudaStream_t,
                                                   float2*, float2*);

template cudaError_t launch_precond<double>(const sg_handle*, int, const double2*, double2*, cudaStream_t,
                                           const int*, const double*);
template cudaError_t launch_precond<float>(const sg_handle*, int, const float2*, float2*, cudaStream_t, const int*,
                                          const double*);

}  // namespace sgi
