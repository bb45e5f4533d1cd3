// Restarted, right-preconditioned GMRES for the SG system (Sec. 6.3: GMRES
// with A M^-1 y = b, x = M^-1 y and relres = ||b - A x|| / ||b||), kept on
// the device:
//
//  * Arnoldi step j:  z = M^-1 v_j,  w = A z,  classical Gram-Schmidt applied
//    twice (d1 = V^H w; w -= V c1; d2 = V^H w; w -= V c2), ||w||.
//  * Lazy normalisation: the basis is stored raw, v_i = vscale_i * V_i; the
//    factor is applied where a vector is read (inside the preconditioner's
//    tridiagonal solve, in the CGS coefficients, in the final combination),
//    so no separate scaling pass is needed.
//  * Complex Givens rotations, the Hessenberg matrix, the residual estimate
//    |g_{j+1}| and the least-squares solve stay in FP64 on the device; one
//    thread updates them.
//  * Every step kernel returns at once when the device flag `done` is set, so
//    the host reads that flag only every `check_every` steps.
//  * SG_MIXED: FP64 iterative refinement around a complex64 GMRES cycle:
//    r = b - A x (FP64 matvec), inner solve A d = r in complex64, x += d.
//
// Reductions: per thread in the vector precision, across warps and blocks in
// FP64, blocks combined by the last block to finish (fixed order, so results
// are bitwise reproducible).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "sg_internal.h"

namespace sgi {

constexpr int RED_THREADS = 256;
constexpr int MAXV = 512;   // maximum basis vectors handled by the coefficient kernels (restart + 1)

// ------------------------------------------------------------------ device scalar layout
struct DevLayout {
  int m;                    // restart capacity
  size_t H, cs, sn, g, vscale, d1, c1, d2, c2, yc, sc;   // offsets in doubles
  size_t R;                 // flexible cycles' basis factor, (m+1) x (m+1) complex, column-major
  size_t total;
  // Every array starts on a 16-byte boundary (an even double offset) because
  // the complex ones are accessed as double2.
  explicit DevLayout(int m_ = 0) : m(m_) {
    size_t o = 0;
    auto take = [&o](size_t count) {
      const size_t at = o;
      o += (count + 1) & ~(size_t)1;
      return at;
    };
    H = take(2 * (size_t)(m + 1) * m);
    cs = take(m);
    sn = take(2 * (size_t)m);
    g = take(2 * (size_t)(m + 1));
    vscale = take(m + 1);
    d1 = take(2 * (size_t)(m + 1));
    c1 = take(2 * (size_t)(m + 1));
    d2 = take(2 * (size_t)(m + 1));
    c2 = take(2 * (size_t)(m + 1));
    yc = take(2 * (size_t)(m + 1));
    sc = take(16);
    R = take(2 * (size_t)(m + 1) * (m + 1));
    total = o;
  }
};
// sc[] slots
enum {
  SC_NORMSQ = 0, SC_BNORM = 1, SC_RNORM2 = 2, SC_EST = 3, SC_TOL = 4, SC_REF = 5, SC_WORK = 6, SC_ZETA = 8,
  SC_H16 = 10,     // scale of the binary16 copy of the newest basis vector (flexible pass 1)
  SC_H16IN = 11    // its input scale for the next binary16 transform 1 (flexible pass 2)
};
// ctl[] slots
enum { CTL_DONE = 0, CTL_ITERS = 1, CTL_K = 2, CTL_FLAGS = 3, CTL_MAXIT = 4 };
enum { FL_CONV = 1, FL_BREAK = 2, FL_NAN = 4, FL_MAXIT = 8 };

template <typename T>
__device__ __forceinline__ C2<T> mkc(T a, T b) {
  C2<T> r;
  r.x = a;
  r.y = b;
  return r;
}

// ------------------------------------------------------------------ block reduction
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm /* NV * 32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sm[k * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nw ? sm[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;  // valid in thread 0
    }
  }
  __syncthreads();
}

// Sum over all blocks of the partials part[b * pstride + k], k < nvals, done
// by the warps of one block in parallel: lanes stride over the blocks, then a
// shuffle tree (fixed order, so the result is reproducible).  emit(k, sum) is
// called by lane 0 of the warp that owns k.
template <typename F>
__device__ __forceinline__ void sum_block_partials(const double* part, int pstride, int nvals, F&& emit) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int k = warp; k < nvals; k += nw) {
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < nb; b += 64) {
      s0 += __ldcg(part + (size_t)b * pstride + k);
      s1 += __ldcg(part + (size_t)(b + 32) * pstride + k);
    }
    if (b < nb) s0 += __ldcg(part + (size_t)b * pstride + k);
    double s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) emit(k, s);
  }
}

// Called by every thread after it stored its block partials; returns true in
// the last block (all partials visible).  The counter is reset by that block.
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// ------------------------------------------------------------------ kernels
// ------------------------------------------------------------------ CGS2 passes
// The Arnoldi step orthogonalises w against the raw basis V_0..V_{nv-1} in
// three passes over V:
//   k_cgs_dots             d1 = V^H w                      (c1 = vscale^2 d1)
//   k_cgs_update<DOTS>     w -= V c1, then d2 = V^H w      (c2 = vscale^2 d2)
//   k_cgs_update<GIVENS>   w -= V c2, ||w||^2, then the Givens update of
//                          column j in the last block to finish.
// Flexible complex64 cycles take two passes instead (k_cgs_dots, then
// k_cgs2_second) over slots that are never finalised in place: the second
// projection of each new vector is kept as a column of a small triangular
// factor R that both passes apply to their coefficients (see tri_forward_h).
// Each block walks chunks of RED_THREADS * CG_EPT consecutive elements (grid
// stride), a thread keeps its CG_EPT elements of w in registers, and every
// pass reads each V_i element once (the DOTS re-read of the chunk it just
// updated comes from L1 or L2).  Complex64 passes read the basis four
// vectors at a time, all loads of a group issued (predicated, not behind a
// branch per vector) before any is used, so that a thread keeps 16 in
// flight; they are limited to 85 registers so that three blocks fit an SM
// and the grid runs in one wave.  Per-warp sums go to a [warp][value] table in
// shared memory, block sums to part[value * gridDim.x + block], and the last
// block adds the blocks in a fixed order (bitwise reproducible).
#ifndef SG_CG_EPT
#define SG_CG_EPT 4
#endif
constexpr int CG_EPT = SG_CG_EPT;
constexpr int CG_WARPS = RED_THREADS / 32;
constexpr int CG_QB = 4;   // complex64: basis vectors per group of loads in flight
// Resident blocks per SM the complex64 passes are compiled for (at most 85
// registers a thread); their complex128 forms keep the compiler's choice.
constexpr int CG_MIN_BLOCKS_C64 = 3;

// v[q][k] = V_{i0+q}[base + k RED_THREADS] for i0 + q < nv and elements below
// N, else zero; every load is issued before the caller uses any.
template <typename T>
__device__ __forceinline__ void load_group(const C2<T>* __restrict__ V, long long N, int nv, int i0,
                                           long long base, C2<T> (&v)[CG_QB][CG_EPT]) {
  // the whole group in range (all but the last chunk, all but the last group
  // of vectors; a block-uniform test): plain loads at constant offsets
  if (i0 + CG_QB <= nv && base - (long long)threadIdx.x + (long long)RED_THREADS * CG_EPT <= N) {
    const C2<T>* __restrict__ p = V + (size_t)i0 * N + base;
#pragma unroll
    for (int q = 0; q < CG_QB; ++q)
#pragma unroll
      for (int k = 0; k < CG_EPT; ++k) v[q][k] = __ldg(p + (size_t)q * N + k * RED_THREADS);
    return;
  }
#pragma unroll
  for (int q = 0; q < CG_QB; ++q) {
    const bool live = i0 + q < nv;
    const C2<T>* Vi = V + (size_t)(live ? i0 + q : 0) * N;
#pragma unroll
    for (int k = 0; k < CG_EPT; ++k) {
      const long long e = base + k * RED_THREADS;
      v[q][k] = live && e < N ? __ldg(Vi + e) : mkc<T>(T(0), T(0));
    }
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of 16 values per lane with 16 shuffles (instead of 16 trees of
// 5): each step halves the values a lane keeps and exchanges the other half
// with the partner lane.  Afterwards lanes 2q and 2q+1 hold the warp sum of
// value cg_value_of_lane(2q).
template <typename T>
__device__ __forceinline__ T warp_sum16(T (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16, c = 16; o >= 2; o >>= 1, c >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < c / 2; ++k) {
      const T send = up ? v[k] : v[k + c / 2];
      const T keep = up ? v[k + c / 2] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
__device__ __forceinline__ int cg_value_of_lane(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// red[warp * ld + i] += warp sum of conj(V_i[e]) w_e over the thread's
// elements of the chunk starting at `base`, eight vectors at a time (i < nv).
template <typename T>
__device__ __forceinline__ void chunk_dots(const C2<T>* __restrict__ V, long long N, int nv, long long base,
                                           const C2<T> (&wk)[CG_EPT], double2* red, int ld) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    T acc[16];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int qb = 0; qb < 8; qb += CG_QB) {
        if (i0 + qb >= nv) {   // warp-uniform: a group with no vector left
#pragma unroll
          for (int q = 0; q < 2 * CG_QB; ++q) acc[2 * qb + q] = T(0);
          continue;
        }
        C2<T> v[CG_QB][CG_EPT];
        load_group<T>(V, N, nv, i0 + qb, base, v);
#pragma unroll
        for (int q = 0; q < CG_QB; ++q) {
          T ax = T(0), ay = T(0);
#pragma unroll
          for (int k = 0; k < CG_EPT; ++k) {
            ax += v[q][k].x * wk[k].x + v[q][k].y * wk[k].y;
            ay += v[q][k].x * wk[k].y - v[q][k].y * wk[k].x;
          }
          acc[2 * (qb + q)] = ax;
          acc[2 * (qb + q) + 1] = ay;
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        T ax = T(0), ay = T(0);
        if (i0 + q < nv) {
          const C2<T>* Vi = V + (size_t)(i0 + q) * N;
#pragma unroll
          for (int k = 0; k < CG_EPT; ++k) {
            const long long e = base + k * RED_THREADS;
            if (e < N) {
              const C2<T> v = __ldg(Vi + e);
              ax += v.x * wk[k].x + v.y * wk[k].y;
              ay += v.x * wk[k].y - v.y * wk[k].x;
            }
          }
        }
        acc[2 * q] = ax;
        acc[2 * q + 1] = ay;
      }
    }
    const T sum = warp_sum16(acc);
    if ((lane & 1) == 0) {
      const int val = cg_value_of_lane(lane), i = i0 + (val >> 1);
      if (i < nv) {
        double2& r = red[warp * ld + i];
        if (val & 1) r.y += (double)sum; else r.x += (double)sum;
      }
    }
  }
}

// Block sums of the per-warp table into part, then (last block only) the
// sums over blocks: d_out[k] and c_out[k] = vscale_i^2 d_out[k], k < 2 nv.
// Returns true in the last block.
__device__ __forceinline__ bool finish_dots(int nv, const double2* red, double* part, unsigned* counter,
                                            const double* vscale, double* d_out, double* c_out) {
  const int G = gridDim.x;
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int w = 0; w < CG_WARPS; ++w) {
      sx += red[w * nv + i].x;
      sy += red[w * nv + i].y;
    }
    part[(size_t)(2 * i) * G + blockIdx.x] = sx;
    part[(size_t)(2 * i + 1) * G + blockIdx.x] = sy;
  }
  if (!last_block(counter)) return false;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < 2 * nv; k += CG_WARPS) {
    const double* pk = part + (size_t)k * G;
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < G; b += 64) {
      s0 += __ldcg(pk + b);
      s1 += __ldcg(pk + b + 32);
    }
    if (b < G) s0 += __ldcg(pk + b);
    double s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      d_out[k] = s;
      const double vs = vscale[k >> 1];
      c_out[k] = vs * vs * s;
    }
  }
  if (threadIdx.x == 0) *counter = 0;
  return true;
}

// The flexible cycles never finalise a basis slot in place: slot k keeps
// u_k, the step's w after one projection, and the orthogonal directions are
// V_k = u_k - sum_{i<k} V_i R_ik, i.e. U = V R with R unit upper triangular,
// column k holding the second-pass coefficients of slot k (written by step
// k-1's pass 2).  Dots with V come from dots with U by forward substitution,
// V^H x = R^-H U^H x, and an update by V is one by U with back-substituted
// coefficients, V c = U (R^-1 c).  (R's off-diagonal entries are of the size
// of the first pass's rounding, so neither solve loses anything.)  One warp,
// t[0 .. nv) in shared memory.  R is read through `at` (R_kl, k < l): the
// device array (column-major, leading dimension ldr) or, for nv <=
// TRI_SMEM_MAX, a copy of its strict upper triangle that the whole block
// stages in shared memory first (the solves' steps are sequential, so each
// one waiting on a global load would cost a load latency per step).
constexpr int TRI_SMEM_MAX = 64;
struct RGlobal {
  const double* R;
  int ldr;
  __device__ double2 operator()(int k, int l) const {
    return *reinterpret_cast<const double2*>(R + 2 * ((size_t)l * ldr + k));
  }
};
struct RShared {
  const double2* rt;   // column l at rt[l (l - 1) / 2 + k], k < l
  __device__ double2 operator()(int k, int l) const { return rt[l * (l - 1) / 2 + k]; }
};
// All threads of the block: rt <- the strict upper triangle of R (nv columns),
// entry idx = l (l - 1) / 2 + k with l = floor((1 + sqrt(1 + 8 idx)) / 2)
// (corrected by one where the square root rounds): every load independent,
// so the block waits for one load latency, not one per column.
__device__ __forceinline__ void tri_stage(double2* rt, const double* __restrict__ R, int ldr, int nv) {
  const int ntri = nv * (nv - 1) / 2;
  for (int idx = threadIdx.x; idx < ntri; idx += blockDim.x) {
    int l = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)idx)) * 0.5f);
    if (l * (l - 1) / 2 > idx) --l;
    else if ((l + 1) * l / 2 <= idx) ++l;
    const int k = idx - l * (l - 1) / 2;
    rt[idx] = *reinterpret_cast<const double2*>(R + 2 * ((size_t)l * ldr + k));
  }
}
template <typename At>
__device__ __forceinline__ void tri_forward_h(double2* t, const At& at, int nv) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k + 1 < nv; ++k) {
    const double2 dk = t[k];
    for (int l = k + 1 + lane; l < nv; l += 32) {   // t_l -= conj(R_kl) t_k
      const double2 r = at(k, l);
      t[l].x -= r.x * dk.x + r.y * dk.y;
      t[l].y -= r.x * dk.y - r.y * dk.x;
    }
    __syncwarp();
  }
}
template <typename At>
__device__ __forceinline__ void tri_back(double2* t, const At& at, int nv) {
  const int lane = threadIdx.x & 31;
  for (int l = nv - 1; l > 0; --l) {
    const double2 cl = t[l];
    for (int k = lane; k < l; k += 32) {            // t_k -= R_kl t_l
      const double2 r = at(k, l);
      t[k].x -= r.x * cl.x - r.y * cl.y;
      t[k].y -= r.x * cl.y + r.y * cl.x;
    }
    __syncwarp();
  }
}
// double2 entries of dynamic shared memory a flexible CGS2 pass needs: the per-warp
// table, or the solves' vector and R's staged triangle if larger.
__host__ __device__ constexpr size_t cgs_flex_smem_entries(int nv, int warps) {
  return nv <= TRI_SMEM_MAX && (size_t)nv + (size_t)nv * (nv - 1) / 2 > (size_t)warps * nv
             ? (size_t)nv + (size_t)nv * (nv - 1) / 2
             : (size_t)warps * nv;
}

// Pass 1: d = V^H w, c = vscale^2 d.  Dynamic shared memory: CG_WARPS * nv double2.
// Two-pass form (R != null): V holds the unfinalised slots u_0 .. u_j; the
// last block turns the sums U^H w into d = V^H w (forward substitution), c =
// vscale^2 d, and stores the U-basis coefficients R^-1 c that pass 2 applies.
// With sc (the binary16 route) it also sums ||w||^2 and stores in
// sc[SC_H16] the scale of pass 2's binary16 copy of w - sum_i c_i V_i:
// sqrt(N) / 4 over that vector's norm, which Pythagoras gives from the dots
// (||w||^2 - sum_i vscale_i^2 |d_i|^2; taken as at least 1e-8 ||w||^2, as the
// difference cancels when w is nearly in the span).  The copy's entries then
// have a root mean square near 1/4, far inside the binary16 range.
// The end of pass 1 for every block (its ||w||^2 when sc is set, the dots'
// block sums) and, in the last block, the sums over blocks, the two-pass
// form's triangular solves (R set) and the binary16 scale (sc set).
__device__ __forceinline__ void pass1_finish(double nacc, int nv, double2* red, double* sm, double* part,
                                             unsigned* counter, const double* vscale, double* d_out,
                                             double* c_out, const double* R, int ldr, double* sc, long long N) {
  const int G = gridDim.x;
  if (sc) {
    // this block's ||w||^2 in the row after the dots' 2 nv rows
    double dv[1] = {nacc};
    block_sum<1>(dv, sm);
    if (threadIdx.x == 0) part[(size_t)(2 * nv) * G + blockIdx.x] = dv[0];
  }
  if (!finish_dots(nv, red, part, counter, vscale, d_out, c_out)) return;
  if (R) {
    // (the per-warp table is no longer needed: its first nv entries hold
    // the solves' vector, the rest R's staged triangle)
    __syncthreads();
    const bool staged = nv <= TRI_SMEM_MAX;
    if (staged) {
      tri_stage(red + nv, R, ldr, nv);
      __syncthreads();
    }
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int l = lane; l < nv; l += 32) red[l] = make_double2(d_out[2 * l], d_out[2 * l + 1]);
      __syncwarp();
      if (staged) tri_forward_h(red, RShared{red + nv}, nv);
      else tri_forward_h(red, RGlobal{R, ldr}, nv);
      for (int l = lane; l < nv; l += 32) {
        const double2 d = red[l];
        d_out[2 * l] = d.x;
        d_out[2 * l + 1] = d.y;
        const double vs2 = vscale[l] * vscale[l];
        red[l] = make_double2(vs2 * d.x, vs2 * d.y);
      }
      __syncwarp();
      if (staged) tri_back(red, RShared{red + nv}, nv);
      else tri_back(red, RGlobal{R, ldr}, nv);
      for (int l = lane; l < nv; l += 32) {
        c_out[2 * l] = red[l].x;
        c_out[2 * l + 1] = red[l].y;
      }
    }
  }
  if (sc) {
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const double* pk = part + (size_t)(2 * nv) * G;
      double s0 = 0.0;
      for (int b = lane; b < G; b += 32) s0 += __ldcg(pk + b);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s0 += __shfl_down_sync(0xffffffffu, s0, o);
      if (lane == 0) {
        double corr = 0.0;
        for (int i = 0; i < nv; ++i) {
          const double vs = vscale[i];
          corr += vs * vs * (d_out[2 * i] * d_out[2 * i] + d_out[2 * i + 1] * d_out[2 * i + 1]);
        }
        const double est2 = fmax(s0 - corr, 1e-8 * s0);
        const double q = 0.25 * sqrt((double)N);
        sc[SC_H16] = est2 > 0.0 && est2 < 1e300 ? q / sqrt(est2) : 1.0;
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void cgs_dots_body(
    const C2<T>* __restrict__ V, long long N, int nv, const C2<T>* __restrict__ w, double* part,
    unsigned* counter, const double* vscale, double* d_out, double* c_out, const int* ctl, const double* R,
    int ldr, double* sc) {
  if (ctl[CTL_DONE]) return;
  extern __shared__ double2 red[];
  __shared__ double sm[32];
  for (int i = threadIdx.x; i < CG_WARPS * nv; i += blockDim.x) red[i] = make_double2(0.0, 0.0);
  __syncthreads();
  const long long chunk = (long long)RED_THREADS * CG_EPT;
  T nacc = T(0);
  for (long long base = blockIdx.x * chunk + threadIdx.x; base - threadIdx.x < N; base += gridDim.x * chunk) {
    C2<T> wk[CG_EPT];
#pragma unroll
    for (int k = 0; k < CG_EPT; ++k) {
      const long long e = base + k * RED_THREADS;
      wk[k] = e < N ? w[e] : mkc<T>(T(0), T(0));
    }
    if (sc) {
#pragma unroll
      for (int k = 0; k < CG_EPT; ++k) nacc += wk[k].x * wk[k].x + wk[k].y * wk[k].y;
    }
    chunk_dots<T>(V, N, nv, base, wk, red, nv);
  }
  pass1_finish((double)nacc, nv, red, sm, part, counter, vscale, d_out, c_out, R, ldr, sc, N);
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cgs_dots(
    const C2<T>* __restrict__ V, long long N, int nv, const C2<T>* __restrict__ w, double* part,
    unsigned* counter, const double* vscale, double* d_out, double* c_out, const int* ctl, const double* R,
    int ldr, double* sc) {
  cgs_dots_body<T>(V, N, nv, w, part, counter, vscale, d_out, c_out, ctl, R, ldr, sc);
}
template <>
__global__ void __launch_bounds__(RED_THREADS, CG_MIN_BLOCKS_C64) k_cgs_dots<float>(
    const C2<float>* __restrict__ V, long long N, int nv, const C2<float>* __restrict__ w, double* part,
    unsigned* counter, const double* vscale, double* d_out, double* c_out, const int* ctl, const double* R,
    int ldr, double* sc) {
  cgs_dots_body<float>(V, N, nv, w, part, counter, vscale, d_out, c_out, ctl, R, ldr, sc);
}

__device__ void givens_column(double* D, int* ctl, const DevLayout& L, int j);

// Passes 2 and 3: w -= sum_i c_i V_i, then either d2 = V^H w (DOTS) or
// ||w||^2 and the Givens update of column j (GIVENS).
// Dynamic shared memory (DOTS): CG_WARPS * nv double2.
template <typename T, bool DOTS>
__device__ __forceinline__ void cgs_update_body(
    const C2<T>* __restrict__ V, long long N, int nv, C2<T>* __restrict__ w,
    const double* __restrict__ c, double* part, unsigned* counter, const double* vscale, double* d_out,
    double* c_out, double* D, int* ctl, DevLayout L, int j) {
  if (ctl[CTL_DONE]) return;
  extern __shared__ double2 red[];
  __shared__ C2<T> cs[MAXV];
  __shared__ double sm[32];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = mkc<T>((T)c[2 * i], (T)c[2 * i + 1]);
  if (DOTS)
    for (int i = threadIdx.x; i < CG_WARPS * nv; i += blockDim.x) red[i] = make_double2(0.0, 0.0);
  __syncthreads();
  const long long chunk = (long long)RED_THREADS * CG_EPT;
  T nacc = T(0);
  for (long long base = blockIdx.x * chunk + threadIdx.x; base - threadIdx.x < N; base += gridDim.x * chunk) {
    C2<T> wk[CG_EPT];
#pragma unroll
    for (int k = 0; k < CG_EPT; ++k) {
      const long long e = base + k * RED_THREADS;
      wk[k] = e < N ? w[e] : mkc<T>(T(0), T(0));
    }
    if constexpr (sizeof(T) == 4) {
      for (int i0 = 0; i0 < nv; i0 += CG_QB) {
        C2<T> v[CG_QB][CG_EPT];
        load_group<T>(V, N, nv, i0, base, v);
#pragma unroll
        for (int q = 0; q < CG_QB; ++q) {
          if (i0 + q >= nv) break;
          const C2<T> ci = cs[i0 + q];
#pragma unroll
          for (int k = 0; k < CG_EPT; ++k) {
            wk[k].x -= ci.x * v[q][k].x - ci.y * v[q][k].y;
            wk[k].y -= ci.x * v[q][k].y + ci.y * v[q][k].x;
          }
        }
      }
    } else {
#pragma unroll 4
      for (int i = 0; i < nv; ++i) {
        const C2<T>* Vi = V + (size_t)i * N;
        const C2<T> ci = cs[i];
#pragma unroll
        for (int k = 0; k < CG_EPT; ++k) {
          const long long e = base + k * RED_THREADS;
          if (e < N) {
            const C2<T> v = __ldg(Vi + e);
            wk[k].x -= ci.x * v.x - ci.y * v.y;
            wk[k].y -= ci.x * v.y + ci.y * v.x;
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CG_EPT; ++k) {
      const long long e = base + k * RED_THREADS;
      if (e < N) {
        w[e] = wk[k];
        nacc += wk[k].x * wk[k].x + wk[k].y * wk[k].y;
      }
    }
    if (DOTS) chunk_dots<T>(V, N, nv, base, wk, red, nv);
  }
  if (DOTS) {
    finish_dots(nv, red, part, counter, vscale, d_out, c_out);
    return;
  }
  double dv[1] = {(double)nacc};
  block_sum<1>(dv, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = dv[0];
  if (!last_block(counter)) return;
  sum_block_partials(part, 1, 1, [&](int, double s) { D[L.sc + SC_NORMSQ] = s; });
  if (threadIdx.x == 0) *counter = 0;
  __syncthreads();
  if (threadIdx.x < 32) givens_column(D, ctl, L, j);
}
template <typename T, bool DOTS>
__global__ void __launch_bounds__(RED_THREADS) k_cgs_update(
    const C2<T>* __restrict__ V, long long N, int nv, C2<T>* __restrict__ w,
    const double* __restrict__ c, double* part, unsigned* counter, const double* vscale, double* d_out,
    double* c_out, double* D, int* ctl, DevLayout L, int j) {
  cgs_update_body<T, DOTS>(V, N, nv, w, c, part, counter, vscale, d_out, c_out, D, ctl, L, j);
}
template <>
__global__ void __launch_bounds__(RED_THREADS, CG_MIN_BLOCKS_C64) k_cgs_update<float, true>(
    const C2<float>* __restrict__ V, long long N, int nv, C2<float>* __restrict__ w,
    const double* __restrict__ c, double* part, unsigned* counter, const double* vscale, double* d_out,
    double* c_out, double* D, int* ctl, DevLayout L, int j) {
  cgs_update_body<float, true>(V, N, nv, w, c, part, counter, vscale, d_out, c_out, D, ctl, L, j);
}
template <>
__global__ void __launch_bounds__(RED_THREADS, CG_MIN_BLOCKS_C64) k_cgs_update<float, false>(
    const C2<float>* __restrict__ V, long long N, int nv, C2<float>* __restrict__ w,
    const double* __restrict__ c, double* part, unsigned* counter, const double* vscale, double* d_out,
    double* c_out, double* D, int* ctl, DevLayout L, int j) {
  cgs_update_body<float, false>(V, N, nv, w, c, part, counter, vscale, d_out, c_out, D, ctl, L, j);
}

// Two-pass form, pass 2 (flexible cycles): with j = nv - 1 and c1 the U-basis
// coefficients from pass 1,
//   w -= sum_{i<=j} c1_i u_i                      (slot j+1, once projected)
// then the sums U^H w over slots 0..j and ||w||^2; the last block turns the
// sums into d2 = V^H w (forward substitution), stores c2 = vscale^2 d2 as
// column j+1 of R (w = V_{j+1} + sum_i V_i c2_i: the second projection is
// never applied to the stored vector), ||V_{j+1}||^2 = ||w||^2 -
// sum_i vscale_i^2 |d2_i|^2 (the directions are orthogonal) and runs the
// Givens update of column j.
// With a half copy (hc.p), w is also written, times pass 1's scale
// D[sc + SC_H16], as binary16 pairs in rows of mx4 pairs (the input of the
// next step's binary16 transform 1): element e = row mx + col goes to row
// mx4 + col, row = e / mx by a multiply-shift (hc.mul = ceil(2^(32+s) / mx),
// hc.shift = 32 + s, s = ceil(log2 mx): exact for e < 2^31); the last block
// stores in D[sc + SC_H16IN] the factor that turns the copy into
// sqrt(N) v_{j+1} (vscale_{j+1} sqrt(N) / scale), transform 1's input scale.
// Dynamic shared memory: CG_WARPS * nv double2.
struct HalfCopy {
  __half2* p;
  unsigned long long mul;
  int shift;
  int mx, mx4;
};
template <typename T>
__device__ __forceinline__ void cgs2_second_body(
    C2<T>* __restrict__ V, long long N, int nv, const double* __restrict__ c1, const double* __restrict__ R,
    int ldr, double* part, unsigned* counter, const double* vscale, double* d_out, double* D, int* ctl,
    DevLayout L, HalfCopy hc) {
  if (ctl[CTL_DONE]) return;
  extern __shared__ double2 red[];
  __shared__ C2<T> cs1[MAXV];
  __shared__ double sm[32];
  const int j = nv - 1;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs1[i] = mkc<T>((T)c1[2 * i], (T)c1[2 * i + 1]);
  for (int i = threadIdx.x; i < CG_WARPS * nv; i += blockDim.x) red[i] = make_double2(0.0, 0.0);
  __syncthreads();
  C2<T>* w = V + (size_t)(j + 1) * N;
  const float hs = hc.p ? (float)D[L.sc + SC_H16] : 0.0f;
  const long long chunk = (long long)RED_THREADS * CG_EPT;
  T nacc = T(0);
  for (long long base = blockIdx.x * chunk + threadIdx.x; base - threadIdx.x < N; base += gridDim.x * chunk) {
    C2<T> wk[CG_EPT];
#pragma unroll
    for (int k = 0; k < CG_EPT; ++k) {
      const long long e = base + k * RED_THREADS;
      wk[k] = e < N ? w[e] : mkc<T>(T(0), T(0));
    }
    if constexpr (sizeof(T) == 4) {
      for (int i0 = 0; i0 < nv; i0 += CG_QB) {
        C2<T> v[CG_QB][CG_EPT];
        load_group<T>(V, N, nv, i0, base, v);
#pragma unroll
        for (int q = 0; q < CG_QB; ++q) {
          if (i0 + q >= nv) break;
          const C2<T> a = cs1[i0 + q];
#pragma unroll
          for (int k = 0; k < CG_EPT; ++k) {
            wk[k].x -= a.x * v[q][k].x - a.y * v[q][k].y;
            wk[k].y -= a.x * v[q][k].y + a.y * v[q][k].x;
          }
        }
      }
    } else {
#pragma unroll 4
      for (int i = 0; i < nv; ++i) {
        const C2<T>* Vi = V + (size_t)i * N;
        const C2<T> a = cs1[i];
#pragma unroll
        for (int k = 0; k < CG_EPT; ++k) {
          const long long e = base + k * RED_THREADS;
          if (e < N) {
            const C2<T> v = __ldg(Vi + e);
            wk[k].x -= a.x * v.x - a.y * v.y;
            wk[k].y -= a.x * v.y + a.y * v.x;
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CG_EPT; ++k) {
      const long long e = base + k * RED_THREADS;
      if (e < N) {
        w[e] = wk[k];
        nacc += wk[k].x * wk[k].x + wk[k].y * wk[k].y;
        if (hc.p) {
          const unsigned long long row = ((unsigned long long)e * hc.mul) >> hc.shift;
          const long long col = e - (long long)row * hc.mx;
          hc.p[(size_t)row * hc.mx4 + col] = __floats2half2_rn(hs * (float)wk[k].x, hs * (float)wk[k].y);
        }
      }
    }
    // dots with slots 0..j (read-only path: the chunk was just read above)
    chunk_dots<T>(V, N, nv, base, wk, red, nv);
  }
  // block sums of the dots (as finish_dots) and of ||w||^2 in one table
  const int G = gridDim.x;
  double dv[1] = {(double)nacc};
  block_sum<1>(dv, sm);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int ww = 0; ww < CG_WARPS; ++ww) {
      sx += red[ww * nv + i].x;
      sy += red[ww * nv + i].y;
    }
    part[(size_t)(2 * i) * G + blockIdx.x] = sx;
    part[(size_t)(2 * i + 1) * G + blockIdx.x] = sy;
  }
  if (threadIdx.x == 0) part[(size_t)(2 * nv) * G + blockIdx.x] = dv[0];
  if (!last_block(counter)) return;
  __shared__ double wn2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // (the per-warp table is free now: its first nv entries take the sums)
  for (int k = warp; k <= 2 * nv; k += CG_WARPS) {
    const double* pk = part + (size_t)k * G;
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < G; b += 64) {
      s0 += __ldcg(pk + b);
      s1 += __ldcg(pk + b + 32);
    }
    if (b < G) s0 += __ldcg(pk + b);
    double ssum = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ssum += __shfl_down_sync(0xffffffffu, ssum, o);
    if (lane == 0) {
      if (k < 2 * nv) {
        if (k & 1) red[k >> 1].y = ssum;
        else red[k >> 1].x = ssum;
      } else {
        wn2 = ssum;
      }
    }
  }
  __syncthreads();
  const bool staged = nv <= TRI_SMEM_MAX;
  if (staged) {
    tri_stage(red + nv, R, ldr, nv);
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    if (staged) tri_forward_h(red, RShared{red + nv}, nv);
    else tri_forward_h(red, RGlobal{R, ldr}, nv);
    double2* rcol = reinterpret_cast<double2*>(D + L.R) + (size_t)(j + 1) * ldr;
    double corr = 0.0;
    for (int l = lane; l < nv; l += 32) {
      const double2 d = red[l];
      d_out[2 * l] = d.x;
      d_out[2 * l + 1] = d.y;
      const double vs2 = vscale[l] * vscale[l];
      rcol[l] = make_double2(vs2 * d.x, vs2 * d.y);
      corr += vs2 * (d.x * d.x + d.y * d.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) corr += __shfl_down_sync(0xffffffffu, corr, o);
    if (lane == 0) {
      const double r = wn2 - corr;
      D[L.sc + SC_NORMSQ] = r > 0.0 ? r : 0.0;
      *counter = 0;
    }
    __syncwarp();
    givens_column(D, ctl, L, j);
    if (hc.p && lane == 0) D[L.sc + SC_H16IN] = D[L.vscale + j + 1] * sqrt((double)N) / (double)hs;
  }
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_cgs2_second(
    C2<T>* __restrict__ V, long long N, int nv, const double* __restrict__ c1, const double* __restrict__ R,
    int ldr, double* part, unsigned* counter, const double* vscale, double* d_out, double* D, int* ctl,
    DevLayout L, HalfCopy hc) {
  cgs2_second_body<T>(V, N, nv, c1, R, ldr, part, counter, vscale, d_out, D, ctl, L, hc);
}
template <>
__global__ void __launch_bounds__(RED_THREADS, CG_MIN_BLOCKS_C64) k_cgs2_second<float>(
    C2<float>* __restrict__ V, long long N, int nv, const double* __restrict__ c1, const double* __restrict__ R,
    int ldr, double* part, unsigned* counter, const double* vscale, double* d_out, double* D, int* ctl,
    DevLayout L, HalfCopy hc) {
  cgs2_second_body<float>(V, N, nv, c1, R, ldr, part, counter, vscale, d_out, D, ctl, L, hc);
}

// ------------------------------------------------------------------ binary16 basis
// The mixed solver's flexible cycles on the binary16 route keep their basis
// slots as binary16 pairs (the storage idea of compressed-basis GMRES,
// Aliaga et al.: the orthogonalisation is bound by reading the basis, and
// the FP64 refinement around the cycles absorbs the coarser storage).  A slot
// has the layout the binary16 transform 1 reads by tensor copies: P my rows
// of mx values padded with zeros to mx4 pairs, so the preconditioner of the
// next step reads the slot itself.  The passes walk a slot in quads of 4
// positions (16 bytes, never across a row since mx4 is a multiple of 4), two
// per thread, so that a thread keeps as many bytes in flight as the
// complex64 passes; w (the operator's output, complex64, unpadded) is read
// at the quad's unknowns and is zero at the pads.  Arithmetic stays FP32
// with FP64 sums.  A slot's scale (pass 1's, for the new vector) is never
// needed by the basis arithmetic, because the directions' inverse norms
// vscale are taken from the stored values; only the Hessenberg column
// converts the stored units back to w's (see k_hb_second).
constexpr int HB_QPT = 2;   // quads per thread and chunk
constexpr int HB_EPT = 4 * HB_QPT;
struct HalfBasis {
  __half2* V;              // slot i at V + i np
  long long np;            // pairs per slot: P my mx4 (a multiple of 4, below 2^31)
  unsigned long long mulq; // row = quad / (mx4 / 4) by multiply-shift: ceil(2^(32+s) / (mx4/4))
  int shiftq, mx, mx4;
};
__device__ __forceinline__ float2 hb_f2(unsigned u) {
  __half2 h;
  memcpy(&h, &u, sizeof(h));
  return __half22float2(h);
}
__device__ __forceinline__ unsigned hb_h2(float x, float y) {
  const __half2 h = __floats2half2_rn(x, y);
  unsigned u;
  memcpy(&u, &h, sizeof(u));
  return u;
}
// First column of quad qd within its row, and the row.
__device__ __forceinline__ int hb_quad_col(const HalfBasis& hb, long long qd, long long* row) {
  const long long r = (long long)(((unsigned long long)qd * hb.mulq) >> hb.shiftq);
  *row = r;
  return (int)(4 * (qd - r * (hb.mx4 >> 2)));
}
// The thread's elements of w at its quads qbase + k RED_THREADS (zero at pads
// and past the end).
__device__ __forceinline__ void hb_load_w(const HalfBasis& hb, const float2* __restrict__ w, long long qbase,
                                          long long nq, float2 (&wk)[HB_EPT]) {
#pragma unroll
  for (int k = 0; k < HB_QPT; ++k) {
    const long long qd = qbase + k * RED_THREADS;
    long long row = 0;
    const int c0 = qd < nq ? hb_quad_col(hb, qd, &row) : hb.mx;
    const long long e0 = row * hb.mx + c0;
#pragma unroll
    for (int t = 0; t < 4; ++t) wk[4 * k + t] = c0 + t < hb.mx ? w[e0 + t] : make_float2(0.f, 0.f);
  }
}
// v[q][k] = quad qbase + k RED_THREADS of slot i0 + q (zero for slots >= nv
// or quads past the end); every load is issued before any is used.
__device__ __forceinline__ void hb_load_group(const HalfBasis& hb, int nv, int i0, long long qbase, long long nq,
                                              uint4 (&v)[CG_QB][HB_QPT]) {
#pragma unroll
  for (int q = 0; q < CG_QB; ++q) {
    const bool live = i0 + q < nv;
    const uint4* Vi = reinterpret_cast<const uint4*>(hb.V + (size_t)(live ? i0 + q : 0) * hb.np);
#pragma unroll
    for (int k = 0; k < HB_QPT; ++k) {
      const long long qd = qbase + k * RED_THREADS;
      v[q][k] = live && qd < nq ? __ldg(Vi + qd) : make_uint4(0u, 0u, 0u, 0u);
    }
  }
}
__device__ __forceinline__ float2 hb_elem(const uint4 (&v)[HB_QPT], int m) {
  const uint4 u = v[m >> 2];
  const int t = m & 3;
  return hb_f2(t == 0 ? u.x : t == 1 ? u.y : t == 2 ? u.z : u.w);
}

// Slot 0 of a cycle: the starting residual r (complex64, in the workspace's
// complex64 slot 0) stored as binary16 times sqrt(N) / 4 / ||r|| (||r||^2 in
// sc[SC_RNORM2]); the last block sets vscale_0 = 1 / ||stored slot 0||.
__global__ void __launch_bounds__(RED_THREADS) k_hb_slot0(const float2* __restrict__ r, HalfBasis hb, double* D,
                                                         const int* ctl, DevLayout L, double* part, int pstride,
                                                         unsigned* counter, long long N) {
  if (ctl[CTL_DONE]) return;
  __shared__ double sm[32];
  const double rn2 = D[L.sc + SC_RNORM2];
  const float s0 = rn2 > 0.0 && rn2 < 1e300 ? (float)(0.25 * sqrt((double)N) / sqrt(rn2)) : 1.0f;
  const long long nq = hb.np / 4;
  float acc = 0.f;
  uint4* out = reinterpret_cast<uint4*>(hb.V);
  for (long long qd = blockIdx.x * (long long)blockDim.x + threadIdx.x; qd < nq; qd += (long long)gridDim.x * blockDim.x) {
    long long row = 0;
    const int c0 = hb_quad_col(hb, qd, &row);
    const long long e0 = row * hb.mx + c0;
    unsigned u[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 v = c0 + t < hb.mx ? r[e0 + t] : make_float2(0.f, 0.f);
      u[t] = hb_h2(s0 * v.x, s0 * v.y);
      const float2 f = hb_f2(u[t]);
      acc += f.x * f.x + f.y * f.y;
    }
    out[qd] = make_uint4(u[0], u[1], u[2], u[3]);
  }
  double dv[1] = {(double)acc};
  block_sum<1>(dv, sm);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * pstride] = dv[0];
  if (last_block(counter)) {
    sum_block_partials(part, pstride, 1, [&](int, double t) { D[L.vscale] = t > 0.0 ? 1.0 / sqrt(t) : 0.0; });
    if (threadIdx.x == 0) *counter = 0;
  }
}

// red[warp * ld + i] += warp sums of conj(U_i) w and, at red[warp * ld + nv
// + i], of conj(U_i) u (u = the newest slot's values) over the thread's
// elements, for slots i < ns, four slots at a time.
__device__ __forceinline__ void hb_chunk_dots2(const HalfBasis& hb, int ns, int nv, long long qbase, long long nq,
                                               const float2 (&wk)[HB_EPT], const float2 (&uk)[HB_EPT],
                                               double2* red, int ld) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2 ws[HB_EPT], us[HB_EPT];
#pragma unroll
  for (int m = 0; m < HB_EPT; ++m) {
    ws[m] = make_float2(wk[m].y, -wk[m].x);
    us[m] = make_float2(uk[m].y, -uk[m].x);
  }
  for (int i0 = 0; i0 < ns; i0 += CG_QB) {
    uint4 v[CG_QB][HB_QPT];
    hb_load_group(hb, ns, i0, qbase, nq, v);
    float acc[16];
#pragma unroll
    for (int q = 0; q < CG_QB; ++q) {
      // packed FP32 FMAs: (x.x, x.y) * (w.x, w.y) sums to Re conj(x) w and
      // (x.x, x.y) * (w.y, -w.x) to Im conj(x) w (ws, us: the swapped pairs)
      float2 pa = make_float2(0.f, 0.f), pb = pa, pc = pa, pd = pa;
#pragma unroll
      for (int m = 0; m < HB_EPT; ++m) {
        const float2 x = hb_elem(v[q], m);
        pa = __ffma2_rn(x, wk[m], pa);
        pb = __ffma2_rn(x, ws[m], pb);
        pc = __ffma2_rn(x, uk[m], pc);
        pd = __ffma2_rn(x, us[m], pd);
      }
      acc[4 * q] = pa.x + pa.y;
      acc[4 * q + 1] = pb.x + pb.y;
      acc[4 * q + 2] = pc.x + pc.y;
      acc[4 * q + 3] = pd.x + pd.y;
    }
    const float sum = warp_sum16(acc);
    if ((lane & 1) == 0) {
      const int val = cg_value_of_lane(lane), i = i0 + (val >> 2);
      if (i < ns) {
        double2& r = red[warp * ld + ((val >> 1) & 1) * nv + i];
        if (val & 1) r.y += (double)sum; else r.x += (double)sum;
      }
    }
  }
}

// Pass 1 on the binary16 basis, step j = nv - 1.  Slot j holds u_j, the
// previous step's vector after one projection, stored as pass 2 left it:
// its second projection is computed here, from the same reads, instead of in
// pass 2 (delayed reorthogonalisation).  Sums: U_i^H w for i <= j, U_i^H u_j
// for i < j, ||w||^2.  The last block
//   1. turns U_{<j}^H u_j into d2 = V_{<j}^H u_j (forward substitution over
//      R's first j columns), stores c2 = vscale^2 d2 as column j of R and
//      vscale_j = 1 / sqrt(||u_j||^2 - sum_i vscale_i^2 |d2_i|^2), with
//      ||u_j||^2 = 1 / vscale_j^2 as pass 2 stored it;
//   2. turns U^H w into d1 = V^H w with all of R, c1 = vscale^2 d1, and
//      stores the U-basis coefficients R^-1 c1 that pass 2 applies;
//   3. stores the scale of the new slot, sqrt(N) / 4 over the projected norm
//      of w (Pythagoras from d1, as in the complex64 form).
// Dynamic shared memory: hb_dots_smem_entries(nv) double2.
__host__ __device__ constexpr size_t hb_dots_smem_entries(int nv, int warps) {
  return nv <= TRI_SMEM_MAX && (size_t)2 * nv + (size_t)nv * (nv - 1) / 2 > (size_t)warps * 2 * nv
             ? (size_t)2 * nv + (size_t)nv * (nv - 1) / 2
             : (size_t)warps * 2 * nv;
}
__global__ void __launch_bounds__(RED_THREADS, CG_MIN_BLOCKS_C64) k_hb_dots(
    HalfBasis hb, long long N, int nv, const float2* __restrict__ w, double* part, unsigned* counter,
    double* vscale, double* d_out, double* c_out, const int* ctl, double* R, int ldr, double* sc) {
  if (ctl[CTL_DONE]) return;
  extern __shared__ double2 red[];
  __shared__ double sm[32];
  const int j = nv - 1, ld = 2 * nv;
  for (int i = threadIdx.x; i < CG_WARPS * ld; i += blockDim.x) red[i] = make_double2(0.0, 0.0);
  __syncthreads();
  const long long nq = hb.np / 4, chunk = (long long)RED_THREADS * HB_QPT;
  const uint4* uj = reinterpret_cast<const uint4*>(hb.V + (size_t)j * hb.np);
  float nacc = 0.f, ex = 0.f, ey = 0.f;
  for (long long qbase = blockIdx.x * chunk + threadIdx.x; qbase - threadIdx.x < nq; qbase += gridDim.x * chunk) {
    float2 wk[HB_EPT], uk[HB_EPT];
    hb_load_w(hb, w, qbase, nq, wk);
#pragma unroll
    for (int k = 0; k < HB_QPT; ++k) {
      const long long qd = qbase + k * RED_THREADS;
      const uint4 u = qd < nq ? __ldg(uj + qd) : make_uint4(0u, 0u, 0u, 0u);
      uk[4 * k] = hb_f2(u.x);
      uk[4 * k + 1] = hb_f2(u.y);
      uk[4 * k + 2] = hb_f2(u.z);
      uk[4 * k + 3] = hb_f2(u.w);
    }
#pragma unroll
    for (int m = 0; m < HB_EPT; ++m) {
      nacc += wk[m].x * wk[m].x + wk[m].y * wk[m].y;
      ex += uk[m].x * wk[m].x + uk[m].y * wk[m].y;   // u_j^H w from registers
      ey += uk[m].x * wk[m].y - uk[m].y * wk[m].x;
    }
    hb_chunk_dots2(hb, j, nv, qbase, nq, wk, uk, red, ld);
  }
  ex = warp_sum(ex);
  ey = warp_sum(ey);
  if ((threadIdx.x & 31) == 0) {
    double2& r = red[(threadIdx.x >> 5) * ld + j];
    r.x += (double)ex;
    r.y += (double)ey;
  }
  // block sums: rows 0 .. 2 nv - 1 of the table (U^H w, then U_{<j}^H u_j),
  // row 2 nv ||w||^2
  const int G = gridDim.x;
  double dv[1] = {(double)nacc};
  block_sum<1>(dv, sm);   // (synchronises the block: the table is complete)
  for (int i = threadIdx.x; i < ld; i += blockDim.x) {
    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int ww = 0; ww < CG_WARPS; ++ww) {
      sx += red[ww * ld + i].x;
      sy += red[ww * ld + i].y;
    }
    part[(size_t)(2 * i) * G + blockIdx.x] = sx;
    part[(size_t)(2 * i + 1) * G + blockIdx.x] = sy;
  }
  if (threadIdx.x == 0) part[(size_t)(2 * ld) * G + blockIdx.x] = dv[0];
  if (!last_block(counter)) return;
  __shared__ double wn2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // sums over blocks: e = U^H w into red[0 .. nv), f = U_{<j}^H u_j into
  // red[nv .. nv + j); R's staged triangle from red[2 nv]
  for (int k = warp; k <= 2 * ld; k += CG_WARPS) {
    const double* pk = part + (size_t)k * G;
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < G; b += 64) {
      s0 += __ldcg(pk + b);
      s1 += __ldcg(pk + b + 32);
    }
    if (b < G) s0 += __ldcg(pk + b);
    double ssum = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ssum += __shfl_down_sync(0xffffffffu, ssum, o);
    if (lane == 0) {
      if (k < 2 * ld) {
        if (k & 1) red[k >> 1].y = ssum;
        else red[k >> 1].x = ssum;
      } else {
        wn2 = ssum;
      }
    }
  }
  __syncthreads();
  double2* rt = red + 2 * nv;
  const bool staged = nv <= TRI_SMEM_MAX;
  if (staged) {
    tri_stage(rt, R, ldr, j);   // columns 1 .. j-1; column j follows from step 1
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    double2* t = red;          // e
    double2* f = red + nv;     // f
    if (j > 0) {
      if (staged) tri_forward_h(f, RShared{rt}, j);
      else tri_forward_h(f, RGlobal{R, ldr}, j);
      double2* rcol = reinterpret_cast<double2*>(R) + (size_t)j * ldr;
      double corr = 0.0;
      for (int l = lane; l < j; l += 32) {
        const double2 d = f[l];
        const double vs2 = vscale[l] * vscale[l];
        const double2 c = make_double2(vs2 * d.x, vs2 * d.y);
        rcol[l] = c;
        if (staged) rt[j * (j - 1) / 2 + l] = c;
        corr += vs2 * (d.x * d.x + d.y * d.y);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) corr += __shfl_xor_sync(0xffffffffu, corr, o);
      const double vj = vscale[j];
      const double un2 = vj > 0.0 ? 1.0 / (vj * vj) : 0.0;
      const double nsq = un2 - corr;
      __syncwarp();
      if (lane == 0) vscale[j] = nsq > 0.0 ? 1.0 / sqrt(nsq) : vj;
      __syncwarp();
    }
    if (staged) tri_forward_h(t, RShared{rt}, nv);
    else tri_forward_h(t, RGlobal{R, ldr}, nv);
    double corr1 = 0.0;
    for (int l = lane; l < nv; l += 32) {
      const double2 d = t[l];
      d_out[2 * l] = d.x;
      d_out[2 * l + 1] = d.y;
      const double vs2 = vscale[l] * vscale[l];
      t[l] = make_double2(vs2 * d.x, vs2 * d.y);
      corr1 += vs2 * (d.x * d.x + d.y * d.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) corr1 += __shfl_xor_sync(0xffffffffu, corr1, o);
    __syncwarp();
    if (staged) tri_back(t, RShared{rt}, nv);
    else tri_back(t, RGlobal{R, ldr}, nv);
    for (int l = lane; l < nv; l += 32) {
      c_out[2 * l] = t[l].x;
      c_out[2 * l + 1] = t[l].y;
    }
    if (lane == 0) {
      const double est2 = fmax(wn2 - corr1, 1e-8 * wn2);
      const double q = 0.25 * sqrt((double)N);
      sc[SC_H16] = est2 > 0.0 && est2 < 1e300 ? q / sqrt(est2) : 1.0;
      *counter = 0;
    }
  }
}

// Pass 2 on the binary16 basis, step j = nv - 1: w' = w - sum_{i<=j} c1_i U_i
// (c1 the U-basis coefficients from pass 1), stored as slot j+1 = s w'
// rounded to binary16 (s = pass 1's scale, D[sc + SC_H16]), and the squared
// norm of the stored slot, ||u_{j+1}||^2.  No dots: the second projection of
// slot j+1 comes from the next step's pass 1.  The Hessenberg column takes
// the first projection only, h_ij = vscale_i d1_i and h_{j+1,j} =
// ||u_{j+1}|| / s: the second projection's part, vscale_i d2_i / s, is of the
// size of the FP32 first pass's rounding, far below the binary16 storage's
// (about 5e-4 of the slot), which bounds the cycle's Arnoldi relation
// anyway.  vscale_{j+1} = 1 / ||u_{j+1}|| until the next pass 1 refines it.
__global__ void __launch_bounds__(RED_THREADS, CG_MIN_BLOCKS_C64) k_hb_second(
    HalfBasis hb, long long N, int nv, const float2* __restrict__ w, const double* __restrict__ c1,
    double* part, unsigned* counter, double* d_out, double* D, int* ctl, DevLayout L) {
  if (ctl[CTL_DONE]) return;
  __shared__ float2 cs1[MAXV];
  __shared__ double sm[32];
  const int j = nv - 1;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs1[i] = make_float2((float)c1[2 * i], (float)c1[2 * i + 1]);
  __syncthreads();
  const double sd = D[L.sc + SC_H16];
  const float hs = (float)sd;
  uint4* wout = reinterpret_cast<uint4*>(hb.V + (size_t)(j + 1) * hb.np);
  const long long nq = hb.np / 4, chunk = (long long)RED_THREADS * HB_QPT;
  float nacc = 0.f;
  for (long long qbase = blockIdx.x * chunk + threadIdx.x; qbase - threadIdx.x < nq; qbase += gridDim.x * chunk) {
    float2 wk[HB_EPT];
    hb_load_w(hb, w, qbase, nq, wk);
    for (int i0 = 0; i0 < nv; i0 += CG_QB) {
      uint4 v[CG_QB][HB_QPT];
      hb_load_group(hb, nv, i0, qbase, nq, v);
#pragma unroll
      for (int q = 0; q < CG_QB; ++q) {
        if (i0 + q >= nv) break;
        const float2 a = cs1[i0 + q];
#pragma unroll
        for (int m = 0; m < HB_EPT; ++m) {
          const float2 x = hb_elem(v[q], m);
          wk[m].x -= a.x * x.x - a.y * x.y;
          wk[m].y -= a.x * x.y + a.y * x.x;
        }
      }
    }
    // the new slot (pads stay zero: w and every slot are zero there)
#pragma unroll
    for (int k = 0; k < HB_QPT; ++k) {
      const long long qd = qbase + k * RED_THREADS;
      unsigned u[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        u[t] = hb_h2(hs * wk[4 * k + t].x, hs * wk[4 * k + t].y);
        const float2 f = hb_f2(u[t]);
        nacc += f.x * f.x + f.y * f.y;
      }
      if (qd < nq) wout[qd] = make_uint4(u[0], u[1], u[2], u[3]);
    }
  }
  double dv[1] = {(double)nacc};
  block_sum<1>(dv, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = dv[0];
  if (!last_block(counter)) return;
  __shared__ double un2;
  sum_block_partials(part, 1, 1, [&](int, double t) { un2 = t; });
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int l = lane; l < nv; l += 32) {
      d_out[2 * l] = 0.0;
      d_out[2 * l + 1] = 0.0;
    }
    const double is = sd > 0.0 ? 1.0 / sd : 0.0;
    if (lane == 0) {
      D[L.sc + SC_NORMSQ] = un2 * is * is;
      *counter = 0;
    }
    __syncwarp();
    givens_column(D, ctl, L, j);
    if (lane == 0) D[L.vscale + j + 1] = un2 > 0.0 ? 1.0 / sqrt(un2) : 0.0;
  }
}

// r = b - Ax (or r = b when Ax == nullptr) written in the inner precision;
// ||r||^2 accumulated in the outer precision, last block writes *norm_out.
template <typename TO, typename TI>
__global__ void __launch_bounds__(RED_THREADS) k_residual(const C2<TO>* __restrict__ b, const C2<TO>* __restrict__ Ax,
                                                         C2<TI>* __restrict__ r, long long N, double* part,
                                                         int pstride, unsigned* counter, double* norm_out) {
  __shared__ double sm[32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  TO nacc = TO(0);
  // four elements a thread per round, all loads issued first (the grid is a
  // few blocks per SM: one load in flight per thread left HBM half idle)
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < N; e += 4 * stride) {
    C2<TO> v[4], a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = b[e + k * stride];
      a[k] = Ax ? Ax[e + k * stride] : mkc<TO>(TO(0), TO(0));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k].x -= a[k].x;
      v[k].y -= a[k].y;
      if (r) r[e + k * stride] = mkc<TI>((TI)v[k].x, (TI)v[k].y);
      nacc += v[k].x * v[k].x + v[k].y * v[k].y;
    }
  }
  for (; e < N; e += stride) {
    C2<TO> v = b[e];
    if (Ax) {
      const C2<TO> a = Ax[e];
      v.x -= a.x;
      v.y -= a.y;
    }
    if (r) r[e] = mkc<TI>((TI)v.x, (TI)v.y);
    nacc += v.x * v.x + v.y * v.y;
  }
  double dv[1] = {(double)nacc};
  block_sum<1>(dv, sm);
  if (threadIdx.x == 0) part[(size_t)blockIdx.x * pstride] = dv[0];
  if (last_block(counter)) {
    sum_block_partials(part, pstride, 1, [&](int, double s) { *norm_out = s; });
    if (threadIdx.x == 0) *counter = 0;
  }
}

// Start of a cycle: vscale_0 = 1/||r||, g = (||r||, 0, ...), k = 0.
// Sets done if ||r|| / ref <= tol already (or r is zero / not finite).
__global__ void k_cycle_init(double* D, int* ctl, DevLayout L, double tol_est, double ref) {
  const double rn = sqrt(D[L.sc + SC_RNORM2]);
  for (int i = 0; i < 2 * (L.m + 1); ++i) D[L.g + i] = 0.0;
  D[L.g] = rn;
  D[L.vscale] = rn > 0 ? 1.0 / rn : 0.0;
  D[L.sc + SC_TOL] = tol_est;
  D[L.sc + SC_REF] = ref;
  D[L.sc + SC_EST] = rn / ref;
  ctl[CTL_K] = 0;
  ctl[CTL_DONE] = 0;
  ctl[CTL_FLAGS] = 0;
  if (!(rn == rn) || rn > 1e300) {
    ctl[CTL_DONE] = 1;
    ctl[CTL_FLAGS] |= FL_NAN;
  } else if (rn / ref <= tol_est || rn == 0.0) {
    ctl[CTL_DONE] = 1;
    ctl[CTL_FLAGS] |= FL_CONV;
  }
}

// Givens update for column j, by one warp (lanes 0-31 of the calling block;
// the memory it reads was written before a block-wide fence).  w = A M^-1 v_j was formed from the
// normalised v_j, so H[i][j] = v_i^H w = vscale_i (d1_i + d2_i) and
// H[j+1][j] = ||w||.  The column and the previous rotations are read and
// written by all lanes in parallel through shared memory; lane 0 applies the
// rotations (a sequential recurrence) and forms the new one.
__device__ void givens_column(double* D, int* ctl, const DevLayout& L, int j) {
  __shared__ double2 col[MAXV + 1];
  __shared__ double2 snr[MAXV];
  __shared__ double csr[MAXV];
  const int lane = threadIdx.x;
  const int m = L.m;
  double2* H = reinterpret_cast<double2*>(D + L.H);     // column-major, ld m+1
  double* cs = D + L.cs;
  double2* sn = reinterpret_cast<double2*>(D + L.sn);
  double2* g = reinterpret_cast<double2*>(D + L.g);
  double* vs = D + L.vscale;
  const double2* d1 = reinterpret_cast<const double2*>(D + L.d1);
  const double2* d2 = reinterpret_cast<const double2*>(D + L.d2);
  for (int i = lane; i <= j; i += 32) {
    const double f = vs[i];
    const double2 a = d1[i], b = d2[i];
    col[i] = make_double2(f * (a.x + b.x), f * (a.y + b.y));
    if (i < j) {
      csr[i] = cs[i];
      snr[i] = sn[i];
    }
  }
  __syncwarp();
  double aa = 0, ab = 0, hn = 0, wn = 0;
  if (lane == 0) {
    wn = sqrt(D[L.sc + SC_NORMSQ]);
    hn = wn;
    col[j + 1] = make_double2(hn, 0.0);
    double2 a = col[0];
    for (int i = 0; i < j; ++i) {
      const double2 b = col[i + 1];
      const double c = csr[i];
      const double2 s = snr[i];
      // t = c a + s b ; b' = -conj(s) a + c b
      col[i] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
      a = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    }
    // new rotation zeroing the subdiagonal entry
    const double2 b = col[j + 1];
    aa = hypot(a.x, a.y);
    ab = hypot(b.x, b.y);
    double c;
    double2 s;
    if (ab == 0.0) {
      c = 1.0;
      s = make_double2(0, 0);
    } else if (aa == 0.0) {
      c = 0.0;
      s = make_double2(b.x / ab, -b.y / ab);
    } else {
      const double rr = hypot(aa, ab);
      c = aa / rr;
      // s = (a/|a|) conj(b) / rr
      const double2 u = make_double2(a.x / aa, a.y / aa);
      s = make_double2((u.x * b.x + u.y * b.y) / rr, (u.y * b.x - u.x * b.y) / rr);
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = make_double2(c * a.x + (s.x * b.x - s.y * b.y), c * a.y + (s.x * b.y + s.y * b.x));
    col[j + 1] = make_double2(0, 0);
    const double2 gj = g[j];
    const double2 g1 = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j + 1] = g1;
    g[j] = make_double2(c * gj.x, c * gj.y);
    const double est = hypot(g1.x, g1.y) / D[L.sc + SC_REF];
    D[L.sc + SC_EST] = est;
    vs[j + 1] = wn > 0 ? 1.0 / wn : 0.0;
    ctl[CTL_ITERS] += 1;
    ctl[CTL_K] = j + 1;
    const bool bad = !(est == est) || !(hn == hn) || !(col[j].x == col[j].x);
    if (bad) {
      ctl[CTL_FLAGS] |= FL_NAN;
      ctl[CTL_DONE] = 1;
    } else if (est <= D[L.sc + SC_TOL]) {
      ctl[CTL_FLAGS] |= FL_CONV;
      ctl[CTL_DONE] = 1;
    } else if (hn <= 1e-300 * (aa + ab + 1e-300) || wn == 0.0) {
      ctl[CTL_FLAGS] |= FL_BREAK;   // (lucky) breakdown: Krylov space invariant
      ctl[CTL_DONE] = 1;
    } else if (ctl[CTL_ITERS] >= ctl[CTL_MAXIT] || j + 1 >= m) {
      if (ctl[CTL_ITERS] >= ctl[CTL_MAXIT]) ctl[CTL_FLAGS] |= FL_MAXIT;
      ctl[CTL_DONE] = 1;
    }
  }
  __syncwarp();
  double2* hcol = H + (size_t)j * (m + 1);
  for (int i = lane; i <= j + 1; i += 32) hcol[i] = col[i];
}

// y = R^-1 g (k x k upper triangle of the rotated Hessenberg matrix);
// yc_i = y_i * vscale_i for the raw-basis linear combination (raw != 0), or
// y_i itself for the combination of the stored z_j (flexible GMRES).
constexpr int LSQ_SMEM_K = 64;      // triangles up to this size are solved from shared memory
constexpr int LSQ_THREADS = 128;

__global__ void __launch_bounds__(LSQ_THREADS) k_lsq(double* D, const int* ctl, DevLayout L, int raw) {
  extern __shared__ double2 Hs[];   // k x k upper triangle, column-major (k <= LSQ_SMEM_K)
  __shared__ double2 y[LSQ_SMEM_K];
  const int k = ctl[CTL_K];
  const int m = L.m;
  const int tid = threadIdx.x;
  const double2* H = reinterpret_cast<const double2*>(D + L.H);
  const double2* g = reinterpret_cast<const double2*>(D + L.g);
  double2* yc = reinterpret_cast<double2*>(D + L.yc);
  const double* vs = D + L.vscale;
  auto cdiv = [](double2 s, double2 d) {
    const double den = d.x * d.x + d.y * d.y;
    return den > 0 ? make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den)
                   : make_double2(0, 0);
  };
  if (k <= LSQ_SMEM_K) {
    // the triangle and g into shared memory by all threads, then column by
    // column: y_i = y_i / R_ii, y_l -= R_li y_i for l < i (in parallel)
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
      const int i = idx / k, l = idx - i * k;
      if (l <= i) Hs[idx] = H[(size_t)i * (m + 1) + l];
    }
    for (int i = tid; i < k; i += blockDim.x) y[i] = g[i];
    __syncthreads();
    for (int i = k - 1; i >= 0; --i) {
      if (tid == 0) y[i] = cdiv(y[i], Hs[i * k + i]);
      __syncthreads();
      const double2 yi = y[i];
      for (int l = tid; l < i; l += blockDim.x) {
        const double2 h = Hs[i * k + l];
        y[l].x -= h.x * yi.x - h.y * yi.y;
        y[l].y -= h.x * yi.y + h.y * yi.x;
      }
      __syncthreads();
    }
    for (int i = tid; i < k; i += blockDim.x)
      yc[i] = raw ? make_double2(y[i].x * vs[i], y[i].y * vs[i]) : y[i];
  } else if (tid == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double2 sum = g[i];
      for (int l = i + 1; l < k; ++l) {
        const double2 h = H[(size_t)l * (m + 1) + i];
        const double2 yl = yc[l];   // still unscaled y_l here
        sum.x -= h.x * yl.x - h.y * yl.y;
        sum.y -= h.x * yl.y + h.y * yl.x;
      }
      yc[i] = cdiv(sum, H[(size_t)i * (m + 1) + i]);
    }
    if (raw)
      for (int i = 0; i < k; ++i) yc[i] = make_double2(yc[i].x * vs[i], yc[i].y * vs[i]);
  }
  for (int i = k + tid; i <= m; i += blockDim.x) yc[i] = make_double2(0, 0);
}

// u = sum_{i<k} yc_i V_i  (k read on the device).  Chunks of RED_THREADS *
// CG_EPT elements per block as in the CGS2 passes: a thread keeps CG_EPT
// accumulators and issues the loads of CG_QB basis vectors (CG_QB * CG_EPT
// values) before using any; each element adds the terms in the order
// i = 0 .. k-1.
template <typename T>
__device__ __forceinline__ void lincomb_body(const C2<T>* __restrict__ V, long long N,
                                             const double* __restrict__ yc, const int* ctl, C2<T>* __restrict__ u) {
  __shared__ C2<T> cs[MAXV];
  const int k = ctl[CTL_K];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = mkc<T>((T)yc[2 * i], (T)yc[2 * i + 1]);
  __syncthreads();
  const long long chunk = (long long)RED_THREADS * CG_EPT;
  for (long long base = blockIdx.x * chunk + threadIdx.x; base - threadIdx.x < N; base += gridDim.x * chunk) {
    C2<T> acc[CG_EPT];
#pragma unroll
    for (int kk = 0; kk < CG_EPT; ++kk) acc[kk] = mkc<T>(T(0), T(0));
    for (int i0 = 0; i0 < k; i0 += CG_QB) {
      C2<T> v[CG_QB][CG_EPT];
      load_group<T>(V, N, k, i0, base, v);
#pragma unroll
      for (int q = 0; q < CG_QB; ++q) {
        if (i0 + q >= k) break;
        const C2<T> c = cs[i0 + q];
#pragma unroll
        for (int kk = 0; kk < CG_EPT; ++kk) {
          acc[kk].x += c.x * v[q][kk].x - c.y * v[q][kk].y;
          acc[kk].y += c.x * v[q][kk].y + c.y * v[q][kk].x;
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < CG_EPT; ++kk) {
      const long long e = base + kk * RED_THREADS;
      if (e < N) u[e] = acc[kk];
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_lincomb(const C2<T>* __restrict__ V, long long N,
                                                        const double* __restrict__ yc, const int* ctl,
                                                        C2<T>* __restrict__ u) {
  lincomb_body<T>(V, N, yc, ctl, u);
}
template <>
__global__ void __launch_bounds__(RED_THREADS, CG_MIN_BLOCKS_C64) k_lincomb<float>(
    const C2<float>* __restrict__ V, long long N, const double* __restrict__ yc, const int* ctl,
    C2<float>* __restrict__ u) {
  lincomb_body<float>(V, N, yc, ctl, u);
}

// x += z (z may be lower precision); skipped if k == 0.
template <typename TX, typename TZ>
__global__ void k_axpy(C2<TX>* __restrict__ x, const C2<TZ>* __restrict__ z, long long N, const int* ctl) {
  if (ctl && ctl[CTL_K] == 0) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < N; e += 4 * stride) {   // four elements a round, loads first
    C2<TZ> v[4];
    C2<TX> a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = z[e + k * stride];
      a[k] = x[e + k * stride];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k].x += (TX)v[k].x;
      a[k].y += (TX)v[k].y;
      x[e + k * stride] = a[k];
    }
  }
  for (; e < N; e += stride) {
    const C2<TZ> v = z[e];
    C2<TX> a = x[e];
    a.x += (TX)v.x;
    a.y += (TX)v.y;
    x[e] = a;
  }
}

// z = s * v, s read on the device.
template <typename T>
__global__ void k_scale_copy(const C2<T>* __restrict__ v, C2<T>* __restrict__ z, long long N,
                             const double* __restrict__ s, const int* skip) {
  if (skip && *skip) return;
  const T f = (T)*s;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride)
    z[e] = mkc<T>(v[e].x * f, v[e].y * f);
}

// zeta = (Ax)^H b / ||Ax||^2 (zero when Ax = 0): the multiple of the initial
// guess with the smallest residual.  Partial sums in FP64, last block writes
// zeta (complex, two doubles).
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_x0_zeta(const C2<T>* __restrict__ b, const C2<T>* __restrict__ Ax,
                                                        long long N, double* part, int pstride, unsigned* counter,
                                                        double* zeta) {
  __shared__ double sm[3 * 32];
  __shared__ double tot[3];
  const long long stride = (long long)gridDim.x * blockDim.x;
  double acc[3] = {0.0, 0.0, 0.0};
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    const C2<T> a = Ax[e], v = b[e];
    acc[0] += (double)a.x * v.x + (double)a.y * v.y;
    acc[1] += (double)a.x * v.y - (double)a.y * v.x;
    acc[2] += (double)a.x * a.x + (double)a.y * a.y;
  }
  block_sum<3>(acc, sm);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) part[(size_t)blockIdx.x * pstride + k] = acc[k];
  if (last_block(counter)) {
    sum_block_partials(part, pstride, 3, [&](int k, double v) { tot[k] = v; });
    __syncthreads();
    if (threadIdx.x == 0) {
      const bool ok = tot[2] > 0.0;
      zeta[0] = ok ? tot[0] / tot[2] : 0.0;
      zeta[1] = ok ? tot[1] / tot[2] : 0.0;
      *counter = 0;
    }
  }
}

// x *= zeta and Ax *= zeta (complex zeta read on the device).
template <typename T>
__global__ void k_cscale2(C2<T>* __restrict__ x, C2<T>* __restrict__ Ax, long long N,
                          const double* __restrict__ zeta) {
  const double zr = zeta[0], zi = zeta[1];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride) {
    const C2<T> v = x[e], a = Ax[e];
    x[e] = mkc<T>((T)(zr * v.x - zi * v.y), (T)(zr * v.y + zi * v.x));
    Ax[e] = mkc<T>((T)(zr * a.x - zi * a.y), (T)(zr * a.y + zi * a.x));
  }
}

template <typename TA, typename TB>
__global__ void k_convert(const C2<TA>* __restrict__ a, C2<TB>* __restrict__ b, long long N) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += stride)
    b[e] = mkc<TB>((TB)a[e].x, (TB)a[e].y);
}

}  // namespace sgi

using namespace sgi;

void sgi_forget_batched_graphs(unsigned long long uid);   // below

void sgi_free_gmres_work(sg_handle* h) {
  GmresWork& w = h->gw;
  if (w.uid) sgi_forget_batched_graphs(w.uid);
  for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second.exec);
  if (w.stream) cudaStreamDestroy(w.stream);
  if (w.ev) cudaEventDestroy(w.ev);
  cudaFree(w.V); cudaFree(w.Z); cudaFree(w.Zb); cudaFree(w.V16); cudaFree(w.Vh); cudaFree(w.R64); cudaFree(w.X64); cudaFree(w.B64);
  cudaFree(w.dscal); cudaFree(w.dctl); cudaFree(w.part); cudaFree(w.counter);
  w = GmresWork{};
}

// The CGS2 passes keep CG_WARPS * nv double2 per-warp sums in dynamic shared
// memory: up to 64 KB at nv = MAXV, above the default 48 KB limit.
static void cgs_attributes() {
  static std::once_flag once;
  std::call_once(once, [] {
    const int bytes = CG_WARPS * MAXV * (int)sizeof(double2);
    cudaFuncSetAttribute(k_cgs_dots<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_hb_dots, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * bytes);   // (two dot sets)
    cudaFuncSetAttribute(k_cgs_dots<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_cgs_update<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_cgs_update<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_cgs2_second<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_lsq, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         LSQ_SMEM_K * LSQ_SMEM_K * (int)sizeof(double2));
  });
}

// Grid of the CGS2 passes: blocks per SM (the tuner's choice, else 4), at
// most one block per chunk of RED_THREADS * CG_EPT elements.
constexpr int CG_DEFAULT_BPSM = 4;
constexpr int CG_MAX_BPSM = 8;
static int cgs_blocks(const sg_handle* h, int bpsm) {
  const long long chunks = ((long long)h->N + RED_THREADS * CG_EPT - 1) / (RED_THREADS * CG_EPT);
  return (int)std::max<long long>(1, std::min<long long>((long long)bpsm * h->num_sms, chunks));
}

static sg_status ensure_work(sg_handle* h, int m, int elem_bytes) {
  GmresWork& w = h->gw;
  if (w.V && w.restart >= m && w.prec_bytes == elem_bytes) return SG_OK;
  sgi_free_gmres_work(h);
  const size_t N = (size_t)h->N;
  DevLayout L(m);
  w.nblk = std::max(1, std::min(h->num_sms * 2, (int)((N + 2 * RED_THREADS - 1) / (2 * RED_THREADS))));
  w.cg_nblk = cgs_blocks(h, h->tune_cgs_bpsm > 0 ? h->tune_cgs_bpsm : CG_DEFAULT_BPSM);
  cgs_attributes();
  cudaError_t e = cudaSuccess;
  if (!e) e = cudaMalloc(&w.V, (size_t)(m + 1) * N * elem_bytes);
  if (!e) e = cudaMalloc(&w.Z, N * elem_bytes);
  // complex64 inner cycles on 2D problems with the fast-diagonalisation route
  // run flexible GMRES with the TF32 preconditioner: keep every z_j
  if (!e && elem_bytes == (int)sizeof(float2) && h->dim == 2 && h->fd) e = cudaMalloc(&w.Zb, (size_t)m * N * elem_bytes);
  // and with the binary16 transforms, the newest basis vector's binary16 copy
  // (its padding columns stay zero); the copy's row index is formed by a
  // multiply-shift that is exact for indices below 2^31
  const bool v16 = elem_bytes == (int)sizeof(float2) && h->dim == 2 && h->fd && h->fd16 && h->tcB[0].h16 &&
                   N < (1ULL << 31);
  if (!e && v16) {
    const size_t rows = (size_t)h->P * h->my, mx4 = (size_t)((h->mx + 3) & ~3);
    e = cudaMalloc(&w.V16, rows * mx4 * sizeof(__half2));
    if (!e) e = cudaMemset(w.V16, 0, rows * mx4 * sizeof(__half2));
    if (!e && !tc_make_xmap16(&w.v16map, w.V16, (long long)mx4, (int)rows, h->mx)) {
      cudaFree(w.V16);   // no tensor map: the step keeps the complex64 transform 1
      w.V16 = nullptr;
    }
    // the binary16 basis of the mixed solver's cycles (positions within a
    // slot are ints)
    const long long np = (long long)rows * (long long)mx4;
    if (!e && w.V16 && np < (1LL << 31)) {
      e = cudaMalloc(&w.Vh, (size_t)(m + 1) * np * sizeof(__half2));
      if (!e) e = cudaMemset(w.Vh, 0, (size_t)(m + 1) * np * sizeof(__half2));
      if (!e) {
        w.vh_np = np;
        w.vhmaps.resize(m + 1);
        for (int i = 0; i <= m; ++i)
          if (!tc_make_xmap16(&w.vhmaps[i], reinterpret_cast<__half2*>(w.Vh) + (size_t)i * np, (long long)mx4,
                              (int)rows, h->mx)) {
            cudaFree(w.Vh);   // no tensor maps: the cycles keep the complex64 basis
            w.Vh = nullptr;
            w.vhmaps.clear();
            break;
          }
      }
    }
  }
  if (!e) e = cudaMalloc(&w.R64, N * sizeof(double2));
  if (!e) e = cudaMalloc(&w.X64, N * sizeof(double2));
  if (!e) e = cudaMalloc(&w.B64, N * sizeof(double2));
  if (!e) e = cudaMalloc((void**)&w.dscal, L.total * sizeof(double));
  if (!e) e = cudaMalloc((void**)&w.dctl, 16 * sizeof(int));
  // block partials: the reduction kernels use nblk * 2 (MAXV + 2) doubles, the
  // CGS2 passes up to (2 MAXV + 1) * cg_nblk
  // (sized for the largest grid the tuner may choose, so that a new choice
  // needs no new allocation)
  const size_t part_doubles =
      std::max((size_t)w.nblk * 2 * (MAXV + 2), (size_t)(2 * MAXV + 2) * cgs_blocks(h, CG_MAX_BPSM));
  if (!e) e = cudaMalloc((void**)&w.part, part_doubles * sizeof(double));
  if (!e) e = cudaMalloc((void**)&w.counter, sizeof(unsigned));
  if (!e) e = cudaMemset(w.counter, 0, sizeof(unsigned));
  if (!e) e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming);
  if (e) {
    sgi_free_gmres_work(h);
    return fail(SG_ENOMEM, std::string("GMRES workspace: ") + cudaGetErrorString(e));
  }
  static std::atomic<unsigned long long> next_uid{1};
  w.restart = m;
  w.prec_bytes = elem_bytes;
  w.uid = next_uid.fetch_add(1);
  return SG_OK;
}

namespace {

struct Ctx {
  sg_handle* h;
  cudaStream_t st;
  DevLayout L;
  int grid;
  int pstride;
  int cg_grid;   // blocks of the CGS2 passes
  bool left = false;   // left preconditioning: Arnoldi on M^-1 A
  bool hb = false;     // flexible cycles on the binary16 basis (SG_MIXED, basis16 = 0)
};

// The workspace holds the binary16 basis and the binary16 route is in use.
bool hb_available(const sg_handle* h) {
  const GmresWork& w = h->gw;
  return h->fd16 && !h->tune_tf32 && w.Vh && (int)w.vhmaps.size() == w.restart + 1 && w.prec_bytes == 8;
}
HalfBasis half_basis(const sg_handle* h) {
  HalfBasis hb{};
  const int mx = h->mx, mq = ((mx + 3) & ~3) / 4;   // quads per row
  int sft = 0;
  while ((1 << sft) < mq) ++sft;
  hb.V = reinterpret_cast<__half2*>(h->gw.Vh);
  hb.np = h->gw.vh_np;
  hb.mulq = ((1ULL << (32 + sft)) + (unsigned long long)mq - 1) / (unsigned long long)mq;
  hb.shiftq = 32 + sft;
  hb.mx = mx;
  hb.mx4 = 4 * mq;
  return hb;
}

// Z = M^-1 (s R) with s = *in_scale (1 if null).
template <typename T>
cudaError_t precond_apply(Ctx& c, sg_prec prec, const C2<T>* R, C2<T>* Z, const int* skip,
                          const double* in_scale = nullptr) {
  if (prec == SG_PREC_NONE) {
    if (in_scale) {
      k_scale_copy<T><<<c.grid, RED_THREADS, 0, c.st>>>(R, Z, c.h->N, in_scale, skip);
      note_launch();
      return cudaGetLastError();
    }
    if (R != Z) return cudaMemcpyAsync(Z, R, (size_t)c.h->N * sizeof(C2<T>), cudaMemcpyDeviceToDevice, c.st);
    return cudaSuccess;
  }
  return launch_precond<T>(c.h, prec == SG_PREC_MEAN ? 0 : prec == SG_PREC_CSL_MEAN ? 1 : 2, R, Z, c.st, skip,
                           in_scale);
}

// Flexible GMRES (complex64 inner cycles with a preconditioner that has a
// plain-TF32 route): z_j = M^-1 v_j is kept for every step and the cycle's
// correction is sum_j y_j z_j, so A Z = V H holds for the z_j actually
// computed and the inexact (relative error ~1e-3) preconditioner changes
// only the iteration count, not the attainable residual.
template <typename T>
static bool flexible(const Ctx& c, sg_prec prec) {
  return sizeof(T) == sizeof(float) && !c.left && (prec == SG_PREC_MEAN || prec == SG_PREC_CSL_MEAN) &&
         c.h->gw.Zb != nullptr;
}

// The binary16 route's half copy of the newest basis vector (pass 2 writes
// it, the next step's transform 1 reads it): on 2D problems with that route
// and a complex64 workspace that holds the copy.
bool use_half_copy(const Ctx& c) {
  return c.h->fd16 && !c.h->tune_tf32 && c.h->gw.V16 && !c.left;
}
HalfCopy half_copy(const sg_handle* h) {
  HalfCopy hc{};
  const int mx = h->mx;
  int sft = 0;
  while ((1 << sft) < mx) ++sft;
  hc.p = reinterpret_cast<__half2*>(h->gw.V16);
  hc.mul = ((1ULL << (32 + sft)) + (unsigned long long)mx - 1) / (unsigned long long)mx;
  hc.shift = 32 + sft;
  hc.mx = mx;
  hc.mx4 = (mx + 3) & ~3;
  return hc;
}

template <typename T>
cudaError_t cgs_passes(Ctx& c, sg_prec prec, int j, int only = 0);

// One Arnoldi step j with CGS2 on the inner-precision basis.
template <typename T>
cudaError_t arnoldi_step(Ctx& c, sg_prec prec, int j) {
  GmresWork& w = c.h->gw;
  const long long N = c.h->N;
  C2<T>* V = reinterpret_cast<C2<T>*>(w.V);
  C2<T>* vj = V + (size_t)j * N;
  C2<T>* wv = V + (size_t)(j + 1) * N;
  double* D = w.dscal;
  cudaError_t e = cudaSuccess;
  // z = M^-1 v_j with v_j = vscale_j V_j (normalised on the fly, so the raw
  // basis norms stay of the size of h_{j+1,j})
  C2<T>* Z;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (c.hb && flexible<T>(c, prec)) {
      // the binary16 basis: slot 0 converted from the cycle's residual at
      // the first step, the preconditioner reading slot j itself
      // (sqrt(N) v_j = sqrt(N) vscale_j u_j), w = A z_j into its own buffer
      const HalfBasis hb = half_basis(c.h);
      if (j == 0) {
        k_hb_slot0<<<c.grid, RED_THREADS, 0, c.st>>>(reinterpret_cast<const float2*>(w.V), hb, D, w.dctl, c.L,
                                                     w.part, c.pstride, w.counter, N);
        note_launch();
        if ((e = cudaGetLastError())) return e;
      }
      Z = reinterpret_cast<C2<T>*>(w.Zb) + (size_t)j * N;
      const int which = prec == SG_PREC_MEAN ? 0 : 1;
      if ((e = launch_precond_f16_copy(c.h, which, reinterpret_cast<const __half2*>(w.Vh) + (size_t)j * hb.np,
                                       &w.vhmaps[j], Z, c.st, w.dctl, D + c.L.vscale + j,
                                       (float)std::sqrt((double)N))))
        return e;
      if ((e = launch_matvec<T>(c.h, Z, reinterpret_cast<C2<T>*>(w.Z), c.st, w.dctl))) return e;
      return cgs_passes<T>(c, prec, j);
    }
  }
  if (flexible<T>(c, prec)) {
    Z = reinterpret_cast<C2<T>*>(w.Zb) + (size_t)j * N;
    if constexpr (sizeof(T) == sizeof(float)) {
      const int which = prec == SG_PREC_MEAN ? 0 : 1;
      if (j >= 1 && use_half_copy(c))   // V_j's binary16 copy, written by step j-1's pass 2
        e = launch_precond_f16_copy(c.h, which, w.V16, &w.v16map, Z, c.st, w.dctl, D + c.L.sc + SC_H16IN);
      else
        e = launch_precond_fast(c.h, which, vj, Z, c.st, w.dctl, D + c.L.vscale + j);
    }
    if (e) return e;
  } else if (c.left) {
    // left: w = M^-1 (vscale_j A V_j) = M^-1 A v_j
    Z = reinterpret_cast<C2<T>*>(w.Z);
    if ((e = launch_matvec<T>(c.h, vj, Z, c.st, w.dctl))) return e;
    if ((e = precond_apply<T>(c, prec, Z, wv, w.dctl, D + c.L.vscale + j))) return e;
  } else {
    Z = reinterpret_cast<C2<T>*>(w.Z);
    if ((e = precond_apply<T>(c, prec, vj, Z, w.dctl, D + c.L.vscale + j))) return e;
  }
  if (!c.left && (e = launch_matvec<T>(c.h, Z, wv, c.st, w.dctl))) return e;
  return cgs_passes<T>(c, prec, j);
}

// The CGS2 passes of Arnoldi step j (w = V_{j+1} against V_0 .. V_j); only =
// 1 or 2 launches just that pass of the flexible two-pass form (timing).
template <typename T>
cudaError_t cgs_passes(Ctx& c, sg_prec prec, int j, int only) {
  GmresWork& w = c.h->gw;
  const long long N = c.h->N;
  C2<T>* V = reinterpret_cast<C2<T>*>(w.V);
  C2<T>* wv = V + (size_t)(j + 1) * N;
  double* D = w.dscal;
  const int nv = j + 1;
  size_t red_bytes = (size_t)CG_WARPS * nv * sizeof(double2);
  const int G = c.cg_grid;
  if (flexible<T>(c, prec)) {
    red_bytes = cgs_flex_smem_entries(nv, CG_WARPS) * sizeof(double2);
    if (sizeof(T) == sizeof(float) && c.hb) {
      const HalfBasis hb = half_basis(c.h);
      const float2* wz = reinterpret_cast<const float2*>(w.Z);
      if (only != 2) {
        k_hb_dots<<<G, RED_THREADS, hb_dots_smem_entries(nv, CG_WARPS) * sizeof(double2), c.st>>>(
            hb, N, nv, wz, w.part, w.counter, D + c.L.vscale, D + c.L.d1, D + c.L.c1, w.dctl, D + c.L.R,
            c.L.m + 1, D + c.L.sc);
        note_launch();
      }
      if (only != 1) {
        k_hb_second<<<G, RED_THREADS, 0, c.st>>>(hb, N, nv, wz, D + c.L.c1, w.part, w.counter, D + c.L.d2, D,
                                                 w.dctl, c.L);
        note_launch();
      }
      return cudaGetLastError();
    }
    // two passes over unfinalised slots (the second projection kept in R;
    // flexible GMRES lets the preconditioner take the once-projected vector)
    // the binary16 route: pass 2 also writes w as the next step's binary16
    // input, at a scale pass 1 derives from ||w||
    HalfCopy hc{};
    if (sizeof(T) == sizeof(float) && use_half_copy(c)) hc = half_copy(c.h);
    if (only != 2) {
      k_cgs_dots<T><<<G, RED_THREADS, red_bytes, c.st>>>(V, N, nv, wv, w.part, w.counter, D + c.L.vscale,
                                                        D + c.L.d1, D + c.L.c1, w.dctl, D + c.L.R, c.L.m + 1,
                                                        hc.p ? D + c.L.sc : nullptr); note_launch();
    }
    if (only != 1) {
      k_cgs2_second<T><<<G, RED_THREADS, red_bytes, c.st>>>(V, N, nv, D + c.L.c1, D + c.L.R, c.L.m + 1, w.part,
                                                           w.counter, D + c.L.vscale, D + c.L.d2, D, w.dctl,
                                                           c.L, hc);
      note_launch();
    }
    return cudaGetLastError();
  }
  if (only) return cudaErrorNotSupported;
  k_cgs_dots<T><<<G, RED_THREADS, red_bytes, c.st>>>(V, N, nv, wv, w.part, w.counter, D + c.L.vscale,
                                                    D + c.L.d1, D + c.L.c1, w.dctl, nullptr, 0, nullptr);
  note_launch();
  k_cgs_update<T, true><<<G, RED_THREADS, red_bytes, c.st>>>(V, N, nv, wv, D + c.L.c1, w.part, w.counter,
                                                            D + c.L.vscale, D + c.L.d2, D + c.L.c2, D, w.dctl,
                                                            c.L, j); note_launch();
  k_cgs_update<T, false><<<G, RED_THREADS, 0, c.st>>>(V, N, nv, wv, D + c.L.c2, w.part, w.counter,
                                                     D + c.L.vscale, nullptr, nullptr, D, w.dctl, c.L, j);
  note_launch();
  return cudaGetLastError();
}

// Arnoldi steps j0 .. j0+len-1: launched directly on the first use of the
// chunk, captured into a CUDA graph on the second, replayed afterwards.  The
// kernels read the done flag and skip their work once the cycle has ended, so
// a replayed chunk is correct whichever step converges.
template <typename T>
cudaError_t arnoldi_steps(Ctx& c, sg_prec prec, int j0, int len) {
  GmresWork& w = c.h->gw;
  const unsigned long long key = ((unsigned long long)(sizeof(T) == 4) << 60) |
                                 ((unsigned long long)(c.left ? 1 : 0) << 59) |
                                 ((unsigned long long)(c.hb ? 1 : 0) << 58) | ((unsigned long long)prec << 55) |
                                 ((unsigned long long)j0 << 28) | (unsigned long long)len;
  auto it = w.graphs.find(key);
  if (it == w.graphs.end()) {
    if (++w.graph_uses[key] < 2) {
      for (int j = j0; j < j0 + len; ++j) {
        cudaError_t e = arnoldi_step<T>(c, prec, j);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    const long long t0 = thread_launches();
    cudaError_t e = cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int j = j0; j < j0 + len && e == cudaSuccess; ++j) e = arnoldi_step<T>(c, prec, j);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c.st, &g);
    const long long nk = thread_launches() - t0;
    note_launches(-nk);   // recorded, not launched
    if (e == cudaSuccess) e = e2;
    GmresWork::Graph gr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gr.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    gr.kernels = nk;
    it = w.graphs.emplace(key, gr).first;
  }
  note_launches(it->second.kernels);
  return cudaGraphLaunch(it->second.exec, c.st);
}

// Runs one restart cycle whose starting residual is already in V[0] with its
// squared norm in sc[RNORM2].  Leaves the correction u = M^-1 (V y) (or, for
// flexible GMRES, sum_j y_j z_j) in Z.
template <typename T>
sg_status run_cycle(Ctx& c, sg_prec prec, int m, double tol_est, double ref, int check_every, bool* any_step) {
  GmresWork& w = c.h->gw;
  k_cycle_init<<<1, 1, 0, c.st>>>(w.dscal, w.dctl, c.L, tol_est, ref); note_launch();
  int done = 0;
  SG_CUDA_TRY(cudaMemcpyAsync(&done, w.dctl + CTL_DONE, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  SG_CUDA_TRY(cudaStreamSynchronize(c.st));
  *any_step = false;
  if (done) return SG_OK;
  for (int j0 = 0; j0 < m; j0 += check_every) {
    const int len = std::min(check_every, m - j0);
    SG_CUDA_TRY(arnoldi_steps<T>(c, prec, j0, len));
    SG_CUDA_TRY(cudaMemcpyAsync(&done, w.dctl + CTL_DONE, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    SG_CUDA_TRY(cudaStreamSynchronize(c.st));
    if (done) break;
  }
  *any_step = true;
  C2<T>* V = reinterpret_cast<C2<T>*>(w.V);
  C2<T>* Z = reinterpret_cast<C2<T>*>(w.Z);
  const bool flex = flexible<T>(c, prec);
  {
    const int kmax = std::min(m, LSQ_SMEM_K);
    k_lsq<<<1, LSQ_THREADS, (size_t)kmax * kmax * sizeof(double2), c.st>>>(w.dscal, w.dctl, c.L, flex ? 0 : 1);
    note_launch();
  }
  const C2<T>* basis = flex ? reinterpret_cast<const C2<T>*>(w.Zb) : V;
  k_lincomb<T><<<c.cg_grid, RED_THREADS, 0, c.st>>>(basis, c.h->N, w.dscal + c.L.yc, w.dctl, Z); note_launch();
  SG_CUDA_TRY(cudaGetLastError());
  if (!flex && !c.left) SG_CUDA_TRY(precond_apply<T>(c, prec, Z, Z, nullptr));
  return SG_OK;
}

// x <- zeta x with zeta the minimal-residual multiple of x (SG_X0_SCALED);
// Ax (N outer-precision values) is left holding A (zeta x) for the first
// residual.
template <typename TX>
sg_status scale_guess(Ctx& c, const C2<TX>* b, C2<TX>* x, C2<TX>* Ax) {
  GmresWork& w = c.h->gw;
  SG_CUDA_TRY(launch_matvec<TX>(c.h, x, Ax, c.st));
  double* zeta = w.dscal + c.L.sc + SC_ZETA;
  k_x0_zeta<TX><<<c.grid, RED_THREADS, 0, c.st>>>(b, Ax, c.h->N, w.part, c.pstride, w.counter, zeta);
  note_launch();
  SG_CUDA_TRY(cudaGetLastError());
  k_cscale2<TX><<<c.grid, RED_THREADS, 0, c.st>>>(x, Ax, c.h->N, zeta);
  note_launch();
  SG_CUDA_TRY(cudaGetLastError());
  return SG_OK;
}

template <typename TX>
sg_status residual_norm(Ctx& c, const C2<TX>* b, const C2<TX>* x, bool x_zero, C2<TX>* Ax, void* rout_inner,
                        bool inner_f32, double* rnorm2_host, bool ax_ready = false) {
  GmresWork& w = c.h->gw;
  const C2<TX>* axp = nullptr;
  if (!x_zero) {
    if (!ax_ready) SG_CUDA_TRY(launch_matvec<TX>(c.h, x, Ax, c.st));
    axp = Ax;
  }
  double* out = w.dscal + c.L.sc + SC_RNORM2;
  if (inner_f32)
    k_residual<TX, float><<<c.grid, RED_THREADS, 0, c.st>>>(b, axp, (float2*)rout_inner, c.h->N, w.part, c.pstride,
                                                           w.counter, out);
  else
    k_residual<TX, double><<<c.grid, RED_THREADS, 0, c.st>>>(b, axp, (double2*)rout_inner, c.h->N, w.part,
                                                            c.pstride, w.counter, out);
  note_launch();
  SG_CUDA_TRY(cudaGetLastError());
  SG_CUDA_TRY(cudaMemcpyAsync(rnorm2_host, out, sizeof(double), cudaMemcpyDeviceToHost, c.st));
  SG_CUDA_TRY(cudaStreamSynchronize(c.st));
  return SG_OK;
}

}  // namespace

// Allocates the GMRES workspace sg_gmres will need for these options (used by
// the batched solver so that no allocation happens while solves run).
sg_status sgi_prepare_workspace(sg_handle* h, const sg_gmres_opts* opts) {
  if (!h || !opts) return fail(SG_EINVAL, "NULL argument");
  int m = opts->restart <= 0 ? (int)std::min<long long>(h->N, MAXV - 1) : opts->restart;
  if (m > MAXV - 1) return fail(SG_EINVAL, "restart must be <= 511");
  m = (int)std::min<long long>(m, h->N);
  const bool inner32 = opts->mode == SG_MIXED || opts->mode == SG_FP32;
  return ensure_work(h, m, inner32 ? 8 : 16);
}

extern "C" sg_status sg_gmres(sg_handle* h, const sg_gmres_opts* opts, const void* b, void* x,
                              sg_gmres_info* info, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !opts || !b || !x) return fail(SG_EINVAL, "NULL argument to sg_gmres");
    if (opts->mode != SG_FP64 && opts->mode != SG_FP32 && opts->mode != SG_MIXED)
      return fail(SG_EINVAL, "bad mode");
    if (opts->prec != SG_PREC_NONE && opts->prec != SG_PREC_MEAN && opts->prec != SG_PREC_CSL_MEAN &&
        opts->prec != SG_PREC_CSL)
      return fail(SG_EINVAL, "bad preconditioner");
    if (!(opts->tol > 0) || !std::isfinite(opts->tol)) return fail(SG_EINVAL, "tol must be positive");
    if (opts->x0_policy < SG_X0_AS_GIVEN || opts->x0_policy > SG_X0_SCALED) return fail(SG_EINVAL, "bad x0_policy");
    if (opts->side != 0 && opts->side != 1) return fail(SG_EINVAL, "side must be 0 (right) or 1 (left)");
    const bool left = opts->side == 1 && opts->prec != SG_PREC_NONE;
    if (left && opts->mode == SG_MIXED)
      return fail(SG_EUNSUPPORTED, "left preconditioning is available for SG_FP64 and SG_FP32, not SG_MIXED");
    if (opts->prec == SG_PREC_CSL) {
      sg_status s = ensure_csl_full(h, (cudaStream_t)stream);
      if (s != SG_OK) return s;
    } else if (opts->prec != SG_PREC_NONE && !prec_available(h, opts->prec)) {
      return fail(SG_EUNSUPPORTED, "preconditioner not available for this problem (its band is too wide)");
    }
    const long long N = h->N;
    int m = opts->restart <= 0 ? (int)std::min<long long>(N, MAXV - 1) : opts->restart;
    if (m > MAXV - 1) return fail(SG_EINVAL, "restart must be <= 511");
    m = (int)std::min<long long>(m, N);
    const int maxit = opts->maxit <= 0 ? (int)std::min<long long>(N, 1 << 30) : opts->maxit;
    const int check_every = opts->check_every <= 0 ? 8 : opts->check_every;
    const bool mixed = opts->mode == SG_MIXED;
    const bool f32 = opts->mode == SG_FP32;
    const bool inner32 = mixed || f32;
    sg_status st0 = ensure_work(h, m, inner32 ? 8 : 16);
    if (st0 != SG_OK) return st0;
    GmresWork& w = h->gw;
    // All work runs on the handle's private stream (stream capture needs a
    // non-legacy stream), ordered after the caller's stream and joined back
    // into it on every return.
    cudaStream_t caller = (cudaStream_t)stream;
    cudaStream_t st = w.stream;
    SG_CUDA_TRY(cudaEventRecord(w.ev, caller));
    SG_CUDA_TRY(cudaStreamWaitEvent(st, w.ev, 0));
    struct Rejoin {
      cudaEvent_t ev;
      cudaStream_t from, to;
      ~Rejoin() {
        if (cudaEventRecord(ev, from) == cudaSuccess) cudaStreamWaitEvent(to, ev, 0);
      }
    } rejoin{w.ev, st, caller};
    Ctx c{h, st, DevLayout(w.restart), w.nblk, 2 * (MAXV + 2), w.cg_nblk};
    c.L = DevLayout(w.restart);
    c.left = left;
    if (opts->basis16 != 0 && opts->basis16 != -1) return fail(SG_EINVAL, "basis16 must be 0 or -1");
    c.hb = mixed && !left && opts->basis16 == 0 && flexible<float>(c, opts->prec) && hb_available(h);
    // the Hessenberg layout uses the allocated capacity; cycles use m <= capacity
    const size_t obytes = (size_t)N * (f32 ? sizeof(float2) : sizeof(double2));

    // outer vectors (x, b) in the outer precision
    void* xd = x;
    const void* bd = b;
    if (opts->host_io) {
      SG_CUDA_TRY(cudaMemcpyAsync(w.B64, b, obytes, cudaMemcpyHostToDevice, st));
      bd = w.B64;
      xd = w.X64;
    }
    bool x_zero = opts->x0 == nullptr;
    if (opts->x0 && opts->x0 != xd) {
      SG_CUDA_TRY(cudaMemcpyAsync(xd, opts->x0, obytes, opts->host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    } else if (!opts->x0) {
      SG_CUDA_TRY(cudaMemsetAsync(xd, 0, obytes, st));
    }
    int ctl0[16] = {0};
    ctl0[CTL_MAXIT] = maxit;
    SG_CUDA_TRY(cudaMemcpyAsync(w.dctl, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, st));

    // ||b||
    double bn2 = 0;
    {
      double* out = w.dscal + c.L.sc + SC_BNORM;
      if (f32)
        k_residual<float, float><<<c.grid, RED_THREADS, 0, st>>>((const float2*)bd, nullptr, nullptr, N, w.part,
                                                                 c.pstride, w.counter, out);
      else
        k_residual<double, double><<<c.grid, RED_THREADS, 0, st>>>((const double2*)bd, nullptr, nullptr, N, w.part,
                                                                   c.pstride, w.counter, out);
      note_launch();
      SG_CUDA_TRY(cudaGetLastError());
      SG_CUDA_TRY(cudaMemcpyAsync(&bn2, out, sizeof(double), cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
    }
    const double bnorm = std::sqrt(bn2);
    sg_gmres_info inf{};
    sg_status status = SG_ENOTCONV;
    if (!std::isfinite(bnorm)) {
      status = fail(SG_EINVAL, "right-hand side is not finite");
      if (info) { inf.status = status; *info = inf; }
      return status;
    }
    if (bnorm == 0.0) {
      SG_CUDA_TRY(cudaMemsetAsync(xd, 0, obytes, st));
      if (opts->host_io) SG_CUDA_TRY(cudaMemcpyAsync(x, xd, obytes, cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
      inf.status = SG_OK;
      if (info) *info = inf;
      return SG_OK;
    }
    // left preconditioning measures residuals after M^-1: ||M^-1 b|| is the reference
    // (M^-1 (b - A x) against it is the stopping test, MATLAB's convention)
    auto prec_norm2 = [&](const void* v, double* out_host) -> sg_status {
      double* out = w.dscal + c.L.sc + SC_WORK;
      if (f32)
        k_residual<float, float><<<c.grid, RED_THREADS, 0, st>>>((const float2*)v, nullptr, nullptr, N, w.part,
                                                                 c.pstride, w.counter, out);
      else
        k_residual<double, double><<<c.grid, RED_THREADS, 0, st>>>((const double2*)v, nullptr, nullptr, N, w.part,
                                                                   c.pstride, w.counter, out);
      note_launch();
      SG_CUDA_TRY(cudaGetLastError());
      SG_CUDA_TRY(cudaMemcpyAsync(out_host, out, sizeof(double), cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
      return SG_OK;
    };
    double bnorm_ref = bnorm;
    if (left) {
      double bl2 = 0;
      if (f32) SG_CUDA_TRY(precond_apply<float>(c, opts->prec, (const float2*)bd, (float2*)w.Z, nullptr));
      else SG_CUDA_TRY(precond_apply<double>(c, opts->prec, (const double2*)bd, (double2*)w.R64, nullptr));
      sg_status s = prec_norm2(f32 ? (const void*)w.Z : (const void*)w.R64, &bl2);
      if (s != SG_OK) return s;
      bnorm_ref = std::sqrt(bl2);
      if (!(bnorm_ref > 0.0) || !std::isfinite(bnorm_ref)) return fail(SG_EBREAKDOWN, "||M^-1 b|| is zero or not finite");
    }
    const int max_outer = mixed ? (opts->max_outer <= 0 ? 20 : opts->max_outer) : 1 << 30;
    // (the binary16 basis limits a cycle's reduction to about 1e-3)
    const double inner_tol = opts->inner_tol > 0 ? opts->inner_tol : c.hb ? 1e-3 : 1e-5;
    int iters = 0, cycles = 0, outer = 0;
    double relres = 1.0, relres_p = 1.0;
    int ctl[16];
    bool ax_ready = false;   // A x already in the residual scratch (scaled guess)
    if (!x_zero && opts->x0_policy == SG_X0_SCALED) {
      sg_status s = f32 ? scale_guess<float>(c, (const float2*)bd, (float2*)xd, (float2*)w.Z)
                        : scale_guess<double>(c, (const double2*)bd, (double2*)xd, (double2*)w.R64);
      if (s != SG_OK) return s;
      ax_ready = true;
    }
    for (;;) {
      double rn2 = 0;
      sg_status s;
      if (f32)
        s = residual_norm<float>(c, (const float2*)bd, (const float2*)xd, x_zero, (float2*)w.Z, w.V, true, &rn2,
                                 ax_ready);
      else
        s = residual_norm<double>(c, (const double2*)bd, (const double2*)xd, x_zero, (double2*)w.R64, w.V, inner32,
                                  &rn2, ax_ready);
      ax_ready = false;
      if (s != SG_OK) return s;
      relres = std::sqrt(rn2) / bnorm;
      relres_p = relres;
      if (cycles == 0 && !x_zero && opts->x0_policy != SG_X0_AS_GIVEN && !(relres <= 1.0)) {
        // the supplied guess is worse than zero: start from zero instead
        SG_CUDA_TRY(cudaMemsetAsync(xd, 0, obytes, st));
        x_zero = true;
        continue;
      }
      if (left) {
        // the cycle starts from M^-1 r (in place in V_0) and its norm
        double rp2 = 0;
        if (f32) SG_CUDA_TRY(precond_apply<float>(c, opts->prec, (const float2*)w.V, (float2*)w.V, nullptr));
        else SG_CUDA_TRY(precond_apply<double>(c, opts->prec, (const double2*)w.V, (double2*)w.V, nullptr));
        s = prec_norm2(w.V, &rp2);
        if (s != SG_OK) return s;
        SG_CUDA_TRY(cudaMemcpyAsync(w.dscal + c.L.sc + SC_RNORM2, w.dscal + c.L.sc + SC_WORK, sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
        relres_p = std::sqrt(rp2) / bnorm_ref;
      }
      if (!std::isfinite(relres) || !std::isfinite(relres_p)) { status = SG_EBREAKDOWN; break; }
      if (relres_p <= opts->tol) { status = SG_OK; break; }
      if (iters >= maxit) { status = SG_ENOTCONV; break; }
      if (mixed && outer >= max_outer) { status = SG_ENOTCONV; break; }
      // inner tolerance on |g| relative to ref
      double tol_est, ref;
      if (mixed) {
        // reduce by inner_tol per refinement step, but finish in this step when
        // the remaining reduction is within 20x of it (saves a refinement step
        // that would only cover the last factor)
        ref = std::sqrt(rn2);
        const double need = 0.5 * opts->tol * bnorm / ref;
        tol_est = need >= 0.05 * inner_tol ? need : inner_tol;
        tol_est = std::min(tol_est, 0.5);
      } else {
        ref = bnorm_ref;
        tol_est = opts->tol;
      }
      bool any = false;
      s = inner32 ? run_cycle<float>(c, opts->prec, m, tol_est, ref, check_every, &any)
                  : run_cycle<double>(c, opts->prec, m, tol_est, ref, check_every, &any);
      if (s != SG_OK) return s;
      SG_CUDA_TRY(cudaMemcpyAsync(ctl, w.dctl, sizeof(ctl), cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
      if (ctl[CTL_FLAGS] & FL_NAN) { status = SG_EBREAKDOWN; break; }
      if (any) {
        if (f32)
          k_axpy<float, float><<<c.grid, RED_THREADS, 0, st>>>((float2*)xd, (const float2*)w.Z, N, w.dctl);
        else if (mixed)
          k_axpy<double, float><<<c.grid, RED_THREADS, 0, st>>>((double2*)xd, (const float2*)w.Z, N, w.dctl);
        else
          k_axpy<double, double><<<c.grid, RED_THREADS, 0, st>>>((double2*)xd, (const double2*)w.Z, N, w.dctl);
        note_launch();
        SG_CUDA_TRY(cudaGetLastError());
        x_zero = false;
      }
      iters = ctl[CTL_ITERS];
      ++cycles;
      if (mixed) ++outer;
      if (!any && !(ctl[CTL_FLAGS] & FL_CONV)) { status = SG_ENOTCONV; break; }
      if (!any && (ctl[CTL_FLAGS] & FL_CONV)) {
        // estimate says converged at zero steps but the true residual disagrees
        status = SG_ENOTCONV;
        break;
      }
      if ((ctl[CTL_FLAGS] & FL_BREAK) && !(ctl[CTL_FLAGS] & FL_CONV)) {
        // invariant subspace: the update solved the system up to rounding; one more residual check
        ctl[CTL_FLAGS] &= ~FL_BREAK;
      }
    }
    if (opts->host_io) SG_CUDA_TRY(cudaMemcpyAsync(x, xd, obytes, cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    int werr = 0;   // a bounded wait inside a kernel ran out (tensor-core transforms)
    SG_CUDA_TRY(cudaMemcpyAsync(&werr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    if (werr) {
      SG_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
      status = SG_ETIMEOUT;
    }
    inf.iters = iters;
    inf.cycles = cycles;
    inf.outer = outer;
    inf.relres = relres;
    inf.relres_prec = relres_p;
    inf.status = status;
    if (info) *info = inf;
    if (status == SG_ENOTCONV) set_error("GMRES did not reach tol within maxit");
    if (status == SG_EBREAKDOWN) set_error("GMRES breakdown: non-finite values");
    if (status == SG_ETIMEOUT) set_error("a device-side wait timed out in a preconditioner transform");
    return status;
  });
}

// ------------------------------------------------------------------ launch-shape tuning support
namespace sgi {

// Drops the graphs captured from this handle's launches (the Arnoldi-step
// chunks and the batched solves that name its workspace): they hold the
// launch shapes and the operand addresses of the time of capture.
void drop_graphs(sg_handle* h) {
  GmresWork& w = h->gw;
  cudaDeviceSynchronize();   // no replay of the old graphs still running
  for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second.exec);
  w.graphs.clear();
  w.graph_uses.clear();
  if (w.uid) sgi_forget_batched_graphs(w.uid);
}

// A new CGS2 grid for the handle: the existing workspace takes it at once
// (its partial-sum buffer is sized for the largest grid); captured graphs
// hold the old grid and are dropped.
void set_cgs_blocks(sg_handle* h, int bpsm) {
  h->tune_cgs_bpsm = bpsm;
  GmresWork& w = h->gw;
  if (!w.V) return;
  const int nb = cgs_blocks(h, bpsm > 0 ? bpsm : CG_DEFAULT_BPSM);
  if (nb == w.cg_nblk) return;
  drop_graphs(h);
  w.cg_nblk = nb;
}

sg_status time_cgs_passes(sg_handle* h, sg_prec prec, int j, int reps, cudaStream_t st, double* us) {
  GmresWork& w = h->gw;
  if (!w.V || w.prec_bytes != (int)sizeof(float2) || j < 0 || j + 1 > w.restart || reps < 1)
    return fail(SG_EINVAL, "CGS2 timing needs a complex64 workspace with room for step j");
  Ctx c{h, st, DevLayout(w.restart), w.nblk, 2 * (MAXV + 2), w.cg_nblk};
  c.hb = flexible<float>(c, prec) && hb_available(h);   // as the mixed solver's cycles run them
  // zero basis and scalars: the passes read and write the same amount
  // whatever the values; the done flag is cleared before every step so that
  // no pass skips its work
  SG_CUDA_TRY(cudaMemsetAsync(w.V, 0, (size_t)(j + 2) * h->N * sizeof(float2), st));
  SG_CUDA_TRY(cudaMemsetAsync(w.dscal, 0, (size_t)c.L.total * sizeof(double), st));
  auto step = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(w.dctl, 0, 16 * sizeof(int), st);
    return e ? e : cgs_passes<float>(c, prec, j);
  };
  for (int r = 0; r < 2; ++r) SG_CUDA_TRY(step());
  cudaEvent_t e0, e1;
  SG_CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e) {
    cudaEventDestroy(e0);
    return fail(SG_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
  }
  e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && !e; ++r) e = step();
  if (!e) e = cudaEventRecord(e1, st);
  if (!e) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e) return fail(SG_ECUDA, std::string("CGS2 timing: ") + cudaGetErrorString(e));
  *us = 1000.0 * ms / reps;
  return SG_OK;
}

}  // namespace sgi

extern "C" sg_status sg_cgs2_pass(sg_handle* h, int restart, int j, int pass, void* stream) {
  using namespace sgi;
  return guarded([&]() -> sg_status {
    if (!h) return fail(SG_EINVAL, "NULL handle");
    if (pass < 0 || pass > 2) return fail(SG_EINVAL, "pass must be 0, 1 or 2");
    cudaStream_t st = (cudaStream_t)stream;
    const sg_prec pk = SG_PREC_MEAN;
    if (pass == 0) {
      sg_gmres_opts o{};
      o.restart = restart <= 0 ? 30 : restart;
      o.mode = SG_MIXED;
      o.prec = pk;
      sg_status s = sgi_prepare_workspace(h, &o);
      if (s != SG_OK) return s;
    }
    GmresWork& w = h->gw;
    if (!w.V || w.prec_bytes != (int)sizeof(float2) || j < 0 || j + 1 > w.restart)
      return fail(SG_EINVAL, "needs a complex64 workspace (pass 0) with room for step j");
    Ctx c{h, st, DevLayout(w.restart), w.nblk, 2 * (MAXV + 2), w.cg_nblk};
    c.hb = flexible<float>(c, pk) && hb_available(h);   // the mixed solver's default form
    if (!flexible<float>(c, pk) || !prec_available(h, pk))
      return fail(SG_EUNSUPPORTED, "the two-pass CGS2 form runs in the flexible cycles of 2D separable problems");
    if (pass == 0) {
      // zero basis and scalars: the passes read and write the same amount
      // whatever the values
      SG_CUDA_TRY(cudaMemsetAsync(w.V, 0, (size_t)(j + 2) * h->N * sizeof(float2), st));
      SG_CUDA_TRY(cudaMemsetAsync(w.dscal, 0, (size_t)c.L.total * sizeof(double), st));
      return SG_OK;
    }
    // the done flag (set by a zero basis's breakdown) is cleared first, so
    // that the pass does its work
    SG_CUDA_TRY(cudaMemsetAsync(w.dctl, 0, 16 * sizeof(int), st));
    SG_CUDA_TRY(cgs_passes<float>(c, pk, j, pass));
    return SG_OK;
  });
}

// ------------------------------------------------------------------ stationary iteration
// The stationary iteration of Sec. 5 with the mean-value (or CSL mean-value)
// block as the splitting matrix B: B x^(i+1) = b - (A - B) x^(i), i.e.
// x^(i+1) = x^(i) + B^-1 (b - A x^(i)).  Each step is one operator
// application with the residual and its norm (FP64 reduction), one block
// solve for all P modes and one update, on the handle's private stream.
extern "C" sg_status sg_stationary(sg_handle* h, const sg_stationary_opts* opts, const void* b, void* x,
                                   sg_stationary_info* info, double* history, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !opts || !b || !x) return fail(SG_EINVAL, "NULL argument to sg_stationary");
    if (opts->mode != SG_FP64 && opts->mode != SG_FP32) return fail(SG_EINVAL, "mode must be SG_FP64 or SG_FP32");
    if (opts->prec != SG_PREC_MEAN && opts->prec != SG_PREC_CSL_MEAN)
      return fail(SG_EINVAL, "the splitting matrix must be SG_PREC_MEAN or SG_PREC_CSL_MEAN");
    if (opts->maxit < 0) return fail(SG_EINVAL, "maxit must be >= 0");
    if (!(opts->tol >= 0) || !std::isfinite(opts->tol)) return fail(SG_EINVAL, "tol must be finite and >= 0");
    if (!h->blk[opts->prec == SG_PREC_MEAN ? 0 : 1].ready)
      return fail(SG_EUNSUPPORTED, "preconditioner not available for this problem (2D needs a constant k_0)");
    const bool f32 = opts->mode == SG_FP32;
    sg_status st0 = ensure_work(h, 1, f32 ? 8 : 16);
    if (st0 != SG_OK) return st0;
    GmresWork& w = h->gw;
    cudaStream_t caller = (cudaStream_t)stream;
    cudaStream_t st = w.stream;
    SG_CUDA_TRY(cudaEventRecord(w.ev, caller));
    SG_CUDA_TRY(cudaStreamWaitEvent(st, w.ev, 0));
    struct Rejoin {
      cudaEvent_t ev;
      cudaStream_t from, to;
      ~Rejoin() {
        if (cudaEventRecord(ev, from) == cudaSuccess) cudaStreamWaitEvent(to, ev, 0);
      }
    } rejoin{w.ev, st, caller};
    Ctx c{h, st, DevLayout(w.restart), w.nblk, 2 * (MAXV + 2), w.cg_nblk};
    const long long N = h->N;
    const size_t bytes = (size_t)N * (f32 ? sizeof(float2) : sizeof(double2));
    bool x_zero = !opts->x0_given;
    if (x_zero) SG_CUDA_TRY(cudaMemsetAsync(x, 0, bytes, st));
    // ||b||
    double bn2 = 0;
    {
      double* out = w.dscal + c.L.sc + SC_BNORM;
      if (f32)
        k_residual<float, float><<<c.grid, RED_THREADS, 0, st>>>((const float2*)b, nullptr, nullptr, N, w.part,
                                                                 c.pstride, w.counter, out);
      else
        k_residual<double, double><<<c.grid, RED_THREADS, 0, st>>>((const double2*)b, nullptr, nullptr, N, w.part,
                                                                   c.pstride, w.counter, out);
      note_launch();
      SG_CUDA_TRY(cudaGetLastError());
      SG_CUDA_TRY(cudaMemcpyAsync(&bn2, out, sizeof(double), cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
    }
    const double bnorm = std::sqrt(bn2);
    if (!std::isfinite(bnorm)) return fail(SG_EINVAL, "right-hand side is not finite");
    sg_stationary_info inf{};
    inf.status = SG_ENOTCONV;
    double relres0 = -1.0;
    for (int it = 0;; ++it) {
      // r = b - A x (into the basis slot V_0), ||r||^2
      double rn2 = 0;
      sg_status s = f32 ? residual_norm<float>(c, (const float2*)b, (const float2*)x, x_zero, (float2*)w.Z, w.V, true,
                                               &rn2)
                        : residual_norm<double>(c, (const double2*)b, (const double2*)x, x_zero, (double2*)w.R64, w.V,
                                                false, &rn2);
      if (s != SG_OK) return s;
      const double relres = bnorm > 0 ? std::sqrt(rn2) / bnorm : 0.0;
      if (history) history[it] = relres;
      inf.iters = it;
      inf.relres = relres;
      if (relres0 < 0) relres0 = relres;
      if (!std::isfinite(relres)) {
        inf.status = SG_EBREAKDOWN;
        inf.diverged = 1;
        break;
      }
      if (relres <= opts->tol) {
        inf.status = SG_OK;
        break;
      }
      if (it >= opts->maxit) {
        // a residual that grew by 1e6 over the first one: the splitting does not converge
        inf.diverged = relres > 1e6 * relres0 ? 1 : 0;
        break;
      }
      // x += B^-1 r
      if (f32) {
        SG_CUDA_TRY(precond_apply<float>(c, opts->prec, (const float2*)w.V, (float2*)w.Z, nullptr));
        k_axpy<float, float><<<c.grid, RED_THREADS, 0, st>>>((float2*)x, (const float2*)w.Z, N, nullptr);
      } else {
        SG_CUDA_TRY(precond_apply<double>(c, opts->prec, (const double2*)w.V, (double2*)w.R64, nullptr));
        k_axpy<double, double><<<c.grid, RED_THREADS, 0, st>>>((double2*)x, (const double2*)w.R64, N, nullptr);
      }
      note_launch();
      SG_CUDA_TRY(cudaGetLastError());
      x_zero = false;
    }
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    int werr = 0;
    SG_CUDA_TRY(cudaMemcpyAsync(&werr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    if (werr) {
      SG_CUDA_TRY(cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
      inf.status = SG_ETIMEOUT;
    }
    if (info) *info = inf;
    if (inf.status == SG_ENOTCONV) set_error("stationary iteration did not reach tol within maxit");
    if (inf.status == SG_EBREAKDOWN) set_error("stationary iteration: non-finite residual (diverged)");
    return inf.status;
  });
}

// ------------------------------------------------------------------ batched solve as one graph
// Independent SG systems solved by ONE cudaGraphLaunch: the graph holds one
// chain per system, and the device decides the control flow the host takes
// in sg_gmres.  Per system (mixed precision):
//   init: x = 0 or the system's guess (scaled by its minimal-residual
//         multiple under SG_X0_SCALED), ||b||^2, r = b - A x (complex64, V_0);
//   R times: [decide: relres = ||r|| / ||b||; at tol, maxit or a non-finite
//            value the system stops, else a cycle starts (same inner
//            tolerance rule as sg_gmres)] -> IF(cycle) {
//              C times: [decide: not done] -> IF { Arnoldi steps 8c .. 8c+7 }
//              least squares, correction, x += correction (FP64),
//              r = b - A x (FP64 operator, FP64 norm) }
//   finish: the system's record (steps, refinements, relres, status).
// The plain kernel sequences are captured with the same launch code as
// sg_gmres (so a system's arithmetic is the one-at-a-time solve's, bit for
// bit); the IF nodes are conditional graph nodes whose values the decide
// kernels set (cudaGraphSetConditional).  Systems still above tol after R
// refinement steps are finished by the caller from where the graph left them;
// a system whose guess is worse than zero (sg_gmres would restart it from
// zero) or whose b is zero is solved again by the caller with sg_gmres.
namespace {

constexpr int BG_CHUNK = 8;        // Arnoldi steps per conditional chunk
constexpr int BG_MAX_OUTER = 4;    // refinement steps unrolled in the graph

struct BgRecord {                  // per system, device
  int status;                      // 0 running, 1 converged, 2 breakdown, 3 step or refinement cap,
                                   // 4 right-hand side not finite, 5 start over on the per-system
                                   // route (a guess worse than zero, or b = 0 with a guess)
  int outer;                       // refinement steps started
  int taken;                       // chunk bodies taken but the last of a cycle (for the launch count)
  int taken_last;                  // last-chunk bodies taken
  int iters;
  double relres;
};

__global__ void k_bg_init(int* ctl, int maxit, BgRecord* rec) {
  for (int i = 0; i < 16; ++i) ctl[i] = 0;
  ctl[CTL_MAXIT] = maxit;
  rec->status = 0;
  rec->outer = 0;
  rec->taken = 0;
  rec->taken_last = 0;
  rec->iters = 0;
  rec->relres = 1.0;
}

// Start of refinement step: stop or start a cycle (k_cycle_init's work with
// sg_gmres's mixed inner tolerance: reduce by inner_tol, or aim at tol
// directly when that is within 20x of it).
__global__ void k_bg_decide_outer(double* D, int* ctl, DevLayout L, double tol, double inner_tol, int max_outer,
                                  int guess, cudaGraphConditionalHandle hdl, BgRecord* rec) {
  const double bnorm = sqrt(D[L.sc + SC_BNORM]);
  const double rn = sqrt(D[L.sc + SC_RNORM2]);
  const double relres = bnorm == 0.0 ? 0.0 : rn / bnorm;   // b = 0: x = 0 is the solution
  rec->relres = relres;
  rec->iters = ctl[CTL_ITERS];
  unsigned go = 0;
  if (rec->status == 0) {
    if (!(bnorm <= 1.7976931348623157e308)) {
      rec->status = 4;
    } else if (rec->outer == 0 && (((guess & 1) && bnorm == 0.0) || ((guess & 2) && !(rn / bnorm <= 1.0)))) {
      // an initial guess that is worse than zero (sg_gmres restarts from
      // zero), or b = 0 with a guess (sg_gmres returns x = 0)
      rec->status = 5;
    } else if (!(relres == relres) || relres > 1e300 || (ctl[CTL_FLAGS] & FL_NAN)) {
      rec->status = 2;
    } else if (relres <= tol) {
      rec->status = 1;
    } else if (ctl[CTL_ITERS] >= ctl[CTL_MAXIT] || rec->outer >= max_outer) {
      rec->status = 3;
    } else {
      const double need = 0.5 * tol * bnorm / rn;
      double tol_est = need >= 0.05 * inner_tol ? need : inner_tol;
      tol_est = fmin(tol_est, 0.5);
      for (int i = 0; i < 2 * (L.m + 1); ++i) D[L.g + i] = 0.0;
      D[L.g] = rn;
      D[L.vscale] = rn > 0 ? 1.0 / rn : 0.0;
      D[L.sc + SC_TOL] = tol_est;
      D[L.sc + SC_REF] = rn;
      D[L.sc + SC_EST] = 1.0;
      ctl[CTL_K] = 0;
      ctl[CTL_DONE] = 0;
      ctl[CTL_FLAGS] = 0;
      rec->outer += 1;
      go = 1;
    }
  }
  cudaGraphSetConditional(hdl, go);
}

__global__ void k_bg_decide_chunk(const int* ctl, int last, cudaGraphConditionalHandle hdl, BgRecord* rec) {
  const unsigned go = ctl[CTL_DONE] ? 0u : 1u;
  if (last) rec->taken_last += (int)go;
  else rec->taken += (int)go;
  cudaGraphSetConditional(hdl, go);
}

// After the unrolled steps: the last residual decides (as the next
// refinement step's test would).
__global__ void k_bg_finish(const double* D, const int* ctl, DevLayout L, double tol, BgRecord* rec) {
  const double bnorm = sqrt(D[L.sc + SC_BNORM]);
  const double relres = bnorm == 0.0 ? 0.0 : sqrt(D[L.sc + SC_RNORM2]) / bnorm;
  rec->iters = ctl[CTL_ITERS];
  if (rec->status == 0) {
    rec->relres = relres;
    if (!(relres == relres) || relres > 1e300 || (ctl[CTL_FLAGS] & FL_NAN)) rec->status = 2;
    else if (relres <= tol) rec->status = 1;
  }
}

struct BgGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  BgRecord* rec = nullptr;           // count records, device
  long long k_fixed = 0;             // kernels that run on every launch
  std::vector<long long> k_outer;    // per system: kernels of one taken refinement step (without its chunks)
  std::vector<long long> k_chunk;    // per system: kernels of a taken chunk (all but the last of a cycle)
  std::vector<long long> k_last;     // per system: kernels of a taken last chunk
  int count = 0;
};

// Graphs keyed by (restart, maxit, max_outer, preconditioner, tol, inner_tol,
// guess policy, then per system: workspace id, b, x, x0).  Workspace ids are never reused, so a
// graph can never name a freed or reallocated workspace; freeing a workspace
// also drops the graphs that name it.
constexpr int BG_KEY_HEAD = 7;
constexpr int BG_KEY_PER_SYSTEM = 4;
std::mutex g_bg_mu;
std::map<std::vector<uintptr_t>, BgGraph> g_bg_cache;

void bg_free(BgGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  cudaFree(g.rec);
  g = BgGraph{};
}

// Captures fn()'s launches on stream st into a new graph; the kernels it
// records are counted in *nk and removed from the launch counter (they run
// when the graph does).
template <typename F>
cudaError_t bg_capture(cudaStream_t st, F&& fn, cudaGraph_t* out, long long* nk) {
  const long long t0 = thread_launches();
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = fn();
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &g);
  *nk = thread_launches() - t0;
  note_launches(-*nk);
  if (e1 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e1;
  }
  if (e2 != cudaSuccess) return e2;
  *out = g;
  return cudaSuccess;
}

cudaError_t bg_add_child(cudaGraph_t parent, cudaGraphNode_t* prev, cudaGraph_t child) {
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, *prev ? prev : nullptr, *prev ? 1 : 0, child);
  cudaGraphDestroy(child);
  if (e == cudaSuccess) *prev = node;
  return e;
}

cudaError_t bg_add_if(cudaGraph_t parent, cudaGraphNode_t* prev, cudaGraphConditionalHandle hdl, cudaGraph_t* body) {
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hdl;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphAddNode(&node, parent, *prev ? prev : nullptr, nullptr, *prev ? 1 : 0, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  *prev = node;
  return cudaSuccess;
}

cudaError_t bg_build(sg_handle* const* h, int count, const sg_gmres_opts* opts, const void* const* b, void* const* x,
                     const void* const* x0, int m, int maxit, int max_outer, BgGraph* out) {
  BgGraph G;
  G.count = count;
  G.k_outer.assign(count, 0);
  G.k_chunk.assign(count, 0);
  G.k_last.assign(count, 0);
  cudaError_t e = cudaGraphCreate(&G.graph, 0);
  if (!e) e = cudaMalloc((void**)&G.rec, (size_t)count * sizeof(BgRecord));
  const double tol = opts->tol;
  const int nch = (m + BG_CHUNK - 1) / BG_CHUNK;
  for (int s = 0; s < count && !e; ++s) {
    sg_handle* hs = h[s];
    GmresWork& w = hs->gw;
    Ctx c{hs, w.stream, DevLayout(w.restart), w.nblk, 2 * (MAXV + 2), w.cg_nblk};
    c.hb = opts->basis16 == 0 && flexible<float>(c, opts->prec) && hb_available(hs);
    const double inner_tol = opts->inner_tol > 0 ? opts->inner_tol : c.hb ? 1e-3 : 1e-5;
    const long long N = hs->N;
    const sg_prec prec = opts->prec;
    BgRecord* rec = G.rec + s;
    const double2* bs = static_cast<const double2*>(b[s]);
    double2* xs = static_cast<double2*>(x[s]);
    double* D = w.dscal;
    // sg_gmres's step cap: opts->maxit, else min(N, 2^30)
    const int maxit_s = maxit > 0 ? maxit : (int)std::min<long long>(N, 1 << 30);
    cudaGraphNode_t prev = nullptr;
    cudaGraph_t g = nullptr;
    long long nk = 0;
    // init (sg_gmres's sequence: x0 or zero, ||b||, the scaled guess, r)
    const double2* x0s = x0 ? static_cast<const double2*>(x0[s]) : nullptr;
    const int policy = opts->x0_policy;
    // bit 0: a guess is given; bit 1: it must not be worse than zero
    const int guess = x0s ? (policy != SG_X0_AS_GIVEN ? 3 : 1) : 0;
    e = bg_capture(c.st, [&]() -> cudaError_t {
      cudaError_t e3 = cudaSuccess;
      if (!x0s) e3 = cudaMemsetAsync(xs, 0, (size_t)N * sizeof(double2), c.st);
      else if (x0s != xs) e3 = cudaMemcpyAsync(xs, x0s, (size_t)N * sizeof(double2), cudaMemcpyDeviceToDevice, c.st);
      if (e3) return e3;
      k_bg_init<<<1, 1, 0, c.st>>>(w.dctl, maxit_s, rec); note_launch();
      k_residual<double, double><<<c.grid, RED_THREADS, 0, c.st>>>(bs, nullptr, nullptr, N, w.part, c.pstride,
                                                                   w.counter, D + c.L.sc + SC_BNORM); note_launch();
      if (!x0s) {
        k_residual<double, float><<<c.grid, RED_THREADS, 0, c.st>>>(bs, nullptr, (float2*)w.V, N, w.part, c.pstride,
                                                                    w.counter, D + c.L.sc + SC_RNORM2); note_launch();
        return cudaGetLastError();
      }
      double2* ax = (double2*)w.R64;
      if ((e3 = launch_matvec<double>(hs, xs, ax, c.st))) return e3;
      if (policy == SG_X0_SCALED) {
        double* zeta = D + c.L.sc + SC_ZETA;
        k_x0_zeta<double><<<c.grid, RED_THREADS, 0, c.st>>>(bs, ax, N, w.part, c.pstride, w.counter, zeta);
        note_launch();
        k_cscale2<double><<<c.grid, RED_THREADS, 0, c.st>>>(xs, ax, N, zeta); note_launch();
      }
      k_residual<double, float><<<c.grid, RED_THREADS, 0, c.st>>>(bs, ax, (float2*)w.V, N, w.part, c.pstride,
                                                                  w.counter, D + c.L.sc + SC_RNORM2); note_launch();
      return cudaGetLastError();
    }, &g, &nk);
    if (!e) e = bg_add_child(G.graph, &prev, g);
    G.k_fixed += nk;
    for (int o = 0; o < BG_MAX_OUTER && !e; ++o) {
      cudaGraphConditionalHandle ho;
      e = cudaGraphConditionalHandleCreate(&ho, G.graph, 0, cudaGraphCondAssignDefault);
      if (!e) e = bg_capture(c.st, [&]() -> cudaError_t {
        k_bg_decide_outer<<<1, 1, 0, c.st>>>(D, w.dctl, c.L, tol, inner_tol, max_outer, guess, ho, rec);
        note_launch();
        return cudaGetLastError();
      }, &g, &nk);
      if (!e) e = bg_add_child(G.graph, &prev, g);
      G.k_fixed += nk;
      cudaGraph_t body = nullptr;
      if (!e) e = bg_add_if(G.graph, &prev, ho, &body);
      cudaGraphNode_t bprev = nullptr;
      for (int ch = 0; ch < nch && !e; ++ch) {
        cudaGraphConditionalHandle hc;
        e = cudaGraphConditionalHandleCreate(&hc, G.graph, 0, cudaGraphCondAssignDefault);
        if (!e) e = bg_capture(c.st, [&]() -> cudaError_t {
          k_bg_decide_chunk<<<1, 1, 0, c.st>>>(w.dctl, ch == nch - 1 ? 1 : 0, hc, rec); note_launch();
          return cudaGetLastError();
        }, &g, &nk);
        if (!e) e = bg_add_child(body, &bprev, g);
        if (o == 0) G.k_outer[s] += nk;
        cudaGraph_t cbody = nullptr;
        if (!e) e = bg_add_if(body, &bprev, hc, &cbody);
        const int j0 = ch * BG_CHUNK, j1 = std::min(m, j0 + BG_CHUNK);
        if (!e) e = bg_capture(c.st, [&]() -> cudaError_t {
          for (int j = j0; j < j1; ++j) {
            cudaError_t e3 = arnoldi_step<float>(c, prec, j);
            if (e3) return e3;
          }
          return cudaSuccess;
        }, &g, &nk);
        cudaGraphNode_t cprev = nullptr;
        if (!e) e = bg_add_child(cbody, &cprev, g);
        if (o == 0) {
          long long& slot = ch == nch - 1 ? G.k_last[s] : G.k_chunk[s];
          slot = std::max(slot, nk);
        }
      }
      // end of the cycle: correction, x += correction, new FP64 residual
      if (!e) e = bg_capture(c.st, [&]() -> cudaError_t {
        const bool flex = flexible<float>(c, prec);
        const int kmax = std::min(m, LSQ_SMEM_K);
        k_lsq<<<1, LSQ_THREADS, (size_t)kmax * kmax * sizeof(double2), c.st>>>(D, w.dctl, c.L, flex ? 0 : 1);
        note_launch();
        const float2* basis = flex ? reinterpret_cast<const float2*>(w.Zb) : reinterpret_cast<const float2*>(w.V);
        float2* Z = reinterpret_cast<float2*>(w.Z);
        k_lincomb<float><<<c.cg_grid, RED_THREADS, 0, c.st>>>(basis, N, D + c.L.yc, w.dctl, Z); note_launch();
        cudaError_t e3 = cudaGetLastError();
        if (!e3 && !flex) e3 = precond_apply<float>(c, prec, Z, Z, nullptr);
        if (e3) return e3;
        k_axpy<double, float><<<c.grid, RED_THREADS, 0, c.st>>>(xs, Z, N, w.dctl); note_launch();
        e3 = launch_matvec<double>(hs, xs, (double2*)w.R64, c.st);
        if (e3) return e3;
        k_residual<double, float><<<c.grid, RED_THREADS, 0, c.st>>>(bs, (const double2*)w.R64, (float2*)w.V, N,
                                                                    w.part, c.pstride, w.counter,
                                                                    D + c.L.sc + SC_RNORM2); note_launch();
        return cudaGetLastError();
      }, &g, &nk);
      if (!e) e = bg_add_child(body, &bprev, g);
      if (o == 0) G.k_outer[s] += nk;
    }
    if (!e) e = bg_capture(c.st, [&]() -> cudaError_t {
      k_bg_finish<<<1, 1, 0, c.st>>>(D, w.dctl, c.L, tol, rec); note_launch();
      return cudaGetLastError();
    }, &g, &nk);
    if (!e) e = bg_add_child(G.graph, &prev, g);
    G.k_fixed += nk;
  }
  if (!e) e = cudaGraphInstantiate(&G.exec, G.graph, 0);
  if (e) {
    bg_free(G);
    return e;
  }
  *out = G;
  return cudaSuccess;
}

}  // namespace

// Whether sg_gmres_batched can take the one-graph route for these options.
bool sgi_batched_graph_eligible(const sg_gmres_opts* opts, const void* const* x0, int count) {
  (void)x0;
  (void)count;
  if (opts->mode != SG_MIXED || opts->host_io || opts->x0 || opts->side != 0) return false;
  if (opts->basis16 != 0 && opts->basis16 != -1) return false;   // (the per-system route reports it)
  if (opts->x0_policy != SG_X0_AS_GIVEN && opts->x0_policy != SG_X0_FALLBACK && opts->x0_policy != SG_X0_SCALED)
    return false;
  return opts->prec == SG_PREC_NONE || opts->prec == SG_PREC_MEAN || opts->prec == SG_PREC_CSL_MEAN;
}

// Drops the cached batch graphs that name workspace `uid` (it is being freed).
void sgi_forget_batched_graphs(unsigned long long uid) {
  std::lock_guard<std::mutex> lock(g_bg_mu);
  for (auto it = g_bg_cache.begin(); it != g_bg_cache.end();) {
    bool hit = false;
    for (size_t i = BG_KEY_HEAD; i < it->first.size(); i += BG_KEY_PER_SYSTEM) hit = hit || it->first[i] == (uintptr_t)uid;
    if (hit) {
      bg_free(it->second);
      it = g_bg_cache.erase(it);
    } else {
      ++it;
    }
  }
}

// One-graph batched solve (see above).  infos[k] gets the graph's share of
// system k's solve; *pending lists the systems still running after the
// unrolled refinement steps (the caller continues them from x[k]; their
// infos then hold the steps taken so far and status SG_ENOTCONV).
sg_status sgi_batched_graph(sg_handle* const* h, int count, const sg_gmres_opts* opts, const void* const* b,
                            void* const* x, const void* const* x0, sg_gmres_info* infos, void* stream,
                            std::vector<int>* pending, std::vector<int>* redo) {
  pending->clear();
  redo->clear();
  int m = 0;
  for (int k = 0; k < count; ++k) {
    int mk = opts->restart <= 0 ? (int)std::min<long long>(h[k]->N, MAXV - 1) : opts->restart;
    mk = (int)std::min<long long>(mk, h[k]->N);
    if (k == 0) m = mk;
    if (mk != m || h[k]->gw.restart < m || h[k]->gw.prec_bytes != (int)sizeof(float2) || !h[k]->gw.uid)
      return fail(SG_EUNSUPPORTED, "batch graph: the systems need the same restart length and complex64 workspaces");
  }
  // sg_gmres's defaults: maxit min(N, 2^30) per system (bg_build), max_outer 20
  const int maxit = opts->maxit <= 0 ? 0 : opts->maxit;
  const int max_outer = opts->max_outer <= 0 ? 20 : opts->max_outer;
  std::vector<uintptr_t> key;
  key.push_back((uintptr_t)m);
  key.push_back((uintptr_t)maxit);
  key.push_back((uintptr_t)max_outer);
  key.push_back((uintptr_t)opts->prec);
  uint64_t tb, ib;
  std::memcpy(&tb, &opts->tol, 8);
  const double itol = opts->inner_tol;
  std::memcpy(&ib, &itol, 8);
  key.push_back((uintptr_t)tb);
  key.push_back((uintptr_t)ib);
  key.push_back((uintptr_t)opts->x0_policy | ((uintptr_t)(opts->basis16 != 0) << 8));
  for (int k = 0; k < count; ++k) {
    key.push_back((uintptr_t)h[k]->gw.uid);
    key.push_back((uintptr_t)b[k]);
    key.push_back((uintptr_t)x[k]);
    key.push_back((uintptr_t)(x0 ? x0[k] : nullptr));
  }
  std::lock_guard<std::mutex> lock(g_bg_mu);
  auto it = g_bg_cache.find(key);
  if (it == g_bg_cache.end()) {
    if (g_bg_cache.size() >= 4) {
      for (auto& kv : g_bg_cache) bg_free(kv.second);
      g_bg_cache.clear();
    }
    BgGraph G;
    SG_CUDA_TRY(bg_build(h, count, opts, b, x, x0, m, maxit, max_outer, &G));
    it = g_bg_cache.emplace(key, G).first;
  }
  BgGraph& G = it->second;
  cudaStream_t st = (cudaStream_t)stream;
  SG_CUDA_TRY(cudaGraphLaunch(G.exec, st));
  std::vector<BgRecord> rec(count);
  SG_CUDA_TRY(cudaMemcpyAsync(rec.data(), G.rec, (size_t)count * sizeof(BgRecord), cudaMemcpyDeviceToHost, st));
  std::vector<int> werr(count, 0);   // bounded waits that ran out (tensor-core transforms)
  for (int k = 0; k < count; ++k)
    SG_CUDA_TRY(cudaMemcpyAsync(&werr[k], h[k]->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA_TRY(cudaStreamSynchronize(st));
  long long kernels = G.k_fixed;
  for (int k = 0; k < count; ++k) {
    kernels += (long long)rec[k].outer * G.k_outer[k] + (long long)rec[k].taken * G.k_chunk[k] +
               (long long)rec[k].taken_last * G.k_last[k];
    sg_gmres_info inf{};
    inf.iters = rec[k].iters;
    inf.outer = rec[k].outer;
    inf.cycles = rec[k].outer;
    inf.graph_outer = rec[k].outer;
    inf.relres = rec[k].relres;
    inf.relres_prec = rec[k].relres;
    const int r = rec[k].status;
    inf.status = r == 1 ? SG_OK : r == 2 ? SG_EBREAKDOWN : r == 4 ? SG_EINVAL : SG_ENOTCONV;
    if (werr[k]) {
      SG_CUDA_TRY(cudaMemsetAsync(h[k]->d_err, 0, sizeof(int), st));
      inf.status = SG_ETIMEOUT;
    } else if (r == 0) {
      pending->push_back(k);
    } else if (r == 5) {
      redo->push_back(k);
    }
    if (infos) infos[k] = inf;
  }
  note_launches(kernels);
  return SG_OK;
}
