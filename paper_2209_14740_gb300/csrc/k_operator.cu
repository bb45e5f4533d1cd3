// Matrix-free SG operator Y = A X (Theorem 3.4 with Theorems A.1/A.2/A.5/A.6):
//
//   (A X)_a(x) = (L X_a)(x) + sum_b M_ab(x) X_b(x),
//   M(x) = -i w1(x) <k phi phi> - w2(x) <k^2 phi phi>,
//
// where L is the FD Laplacian on the unknown grid, w1 the boundary weight of
// D_1 (1/h on absorbing boundary nodes) and w2 the D_2 weight (1/2 on an
// absorbing edge per direction).  With k = k_0 + sum_l xi_l k_l (Sec. 2.2):
//   <k phi_a phi_b>   = k_0 delta_ab + sum_l k_l G_l[a,b]
//   <k^2 phi_a phi_b> = k_0^2 delta_ab + 2 k_0 sum_l k_l G_l[a,b]
//                       + sum_{l,l'} k_l k_l' G_{l,l'}[a,b]
// Every off-diagonal pair (a, b) couples through exactly one term t (the
// multi-indices differ by e_l, 2 e_l or e_l +- e_l'), so the host stores per
// row a list (b, t, g_ab) and the kernel forms c_t(x) * g_ab on the fly.
//
// Layout: X, Y are mode-major (X[a * n + u]), u = iu + mx * ju, complex
// interleaved.  One thread owns one grid unknown; all P modes of the CTA's
// unknowns are staged in shared memory so the x-neighbours of the stencil
// and the coupling read shared memory; y-neighbours come through L1/L2.
#include <cuda_runtime.h>

#include <mutex>

#include "sg_internal.h"
#include "k_operator_geom.cuh"

namespace sgi {

// Generic table-driven kernel: any (s, r).  Shared memory per CTA of
// MV_BLK = blockDim.x threads: xs[P][MV_BLK] complex, cf[T][MV_BLK] complex
// term coefficients, kl2[s][MV_BLK] real (-w2 k_l^2 for the diagonal moments).
template <typename T>
__global__ void __launch_bounds__(128) k_matvec_generic(OpParams<T> p, const C2<T>* __restrict__ X,
                                                       C2<T>* __restrict__ Y) {
  if (p.skip && *p.skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int MV_BLK = blockDim.x;
  C2<T>* xs = reinterpret_cast<C2<T>*>(smem_raw);
  C2<T>* cf = xs + (size_t)p.P * MV_BLK;
  T* kl2 = reinterpret_cast<T*>(cf + (size_t)max(p.T_terms, 1) * MV_BLK);
  const int tid = threadIdx.x;
  const int u = blockIdx.x * MV_BLK + tid;
  const bool valid = u < p.n;
  const int uu = valid ? u : p.n - 1;
  for (int a = 0; a < p.P; ++a) xs[a * MV_BLK + tid] = X[(size_t)a * p.n + uu];

  const int iu = uu % p.mx, ju = uu / p.mx;
  const NodeGeom<T> g = node_geom<T>(p, iu, ju);
  const T k0 = p.fields[uu];
  // term coefficients c_t(x)
  for (int l = 0; l < p.s; ++l) {
    const T kl = p.fields[(size_t)(l + 1) * p.n + uu];
    cf[l * MV_BLK + tid] = mk<T>(-T(2) * g.w2 * k0 * kl, -g.w1 * kl);
    cf[(p.s + l) * MV_BLK + tid] = mk<T>(-g.w2 * kl * kl, T(0));
    kl2[l * MV_BLK + tid] = -g.w2 * kl * kl;
  }
  {
    int t = 2 * p.s;
    for (int l = 0; l < p.s; ++l) {
      const T kl = p.fields[(size_t)(l + 1) * p.n + uu];
      for (int lp = l + 1; lp < p.s; ++lp, ++t) {
        const T klp = p.fields[(size_t)(lp + 1) * p.n + uu];
        cf[t * MV_BLK + tid] = mk<T>(-T(2) * g.w2 * kl * klp, T(0));
      }
    }
  }
  const T dre0 = g.ldiag - g.w2 * k0 * k0;
  const T dim0 = -g.w1 * k0;
  __syncthreads();
  if (!valid) return;

  const bool xm_s = g.hxm && tid > 0;
  const bool xp_s = g.hxp && tid < MV_BLK - 1 && u + 1 < p.n;
  for (int a = 0; a < p.P; ++a) {
    const C2<T> xa = xs[a * MV_BLK + tid];
    T dre = dre0;
    for (int l = 0; l < p.s; ++l) dre += kl2[l * MV_BLK + tid] * p.gdiag[l * p.P + a];
    T accr = dre * xa.x - dim0 * xa.y;
    T acci = dre * xa.y + dim0 * xa.x;
    const C2<T>* Xa = X + (size_t)a * p.n;
    if (g.hxm) {
      const C2<T> v = xm_s ? xs[a * MV_BLK + tid - 1] : Xa[u - 1];
      accr -= g.wxm * v.x;
      acci -= g.wxm * v.y;
    }
    if (g.hxp) {
      const C2<T> v = xp_s ? xs[a * MV_BLK + tid + 1] : Xa[u + 1];
      accr -= g.wxp * v.x;
      acci -= g.wxp * v.y;
    }
    if (g.hym) {
      const C2<T> v = Xa[u - p.mx];
      accr -= g.wym * v.x;
      acci -= g.wym * v.y;
    }
    if (g.hyp) {
      const C2<T> v = Xa[u + p.mx];
      accr -= g.wyp * v.x;
      acci -= g.wyp * v.y;
    }
    const int k1 = p.rowptr[a + 1];
    for (int k = p.rowptr[a]; k < k1; ++k) {
      const int b = p.col[k];
      const int t = p.term[k];
      const T gv = p.gval[k];
      const C2<T> c = cf[t * MV_BLK + tid];
      const C2<T> xb = xs[b * MV_BLK + tid];
      const T cr = c.x * gv, ci = c.y * gv;
      accr += cr * xb.x - ci * xb.y;
      acci += cr * xb.y + ci * xb.x;
    }
    Y[(size_t)a * p.n + u] = mk<T>(accr, acci);
  }
}

template <typename T>
static size_t generic_smem_per_thread(const sg_handle* h) {
  return sizeof(C2<T>) * (h->P + std::max(h->T_terms, 1)) + sizeof(T) * std::max(h->s, 1);
}

cudaError_t matvec_special_f32(const sg_handle* h, const float2* X, float2* Y, cudaStream_t st, const int* skip,
                               bool* handled);
cudaError_t matvec_special_f64(const sg_handle* h, const double2* X, double2* Y, cudaStream_t st, const int* skip,
                               bool* handled);

template <typename T>
cudaError_t launch_matvec(const sg_handle* h, const C2<T>* X, C2<T>* Y, cudaStream_t st, const int* skip) {
  {
    bool handled = false;
    cudaError_t e;
    if constexpr (sizeof(T) == 4) e = matvec_special_f32(h, X, Y, st, skip, &handled);
    else e = matvec_special_f64(h, X, Y, st, skip, &handled);
    if (handled || e != cudaSuccess) return e;
  }
  const size_t per = generic_smem_per_thread<T>(h);
  int blk = 128;
  while (blk > 32 && per * blk > 200 * 1024) blk /= 2;
  if (per * blk > 220 * 1024) return cudaErrorInvalidConfiguration;
  const size_t smem = per * blk;
  if (smem > 48 * 1024) {
    // one process-wide limit, set once: a per-call value would race between
    // host threads (batched solves) and between capture and graph replay
    static std::once_flag once;
    static cudaError_t set_err = cudaSuccess;
    std::call_once(once, [] {
      set_err = cudaFuncSetAttribute(k_matvec_generic<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    });
    if (set_err != cudaSuccess) return set_err;
  }
  OpParams<T> p;
  if constexpr (sizeof(T) == 8) p = h->op64(); else p = h->op32();
  p.skip = skip;
  const int grid = (h->n + blk - 1) / blk;
  k_matvec_generic<T><<<grid, blk, smem, st>>>(p, X, Y); note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_matvec<double>(const sg_handle*, const double2*, double2*, cudaStream_t, const int*);
template cudaError_t launch_matvec<float>(const sg_handle*, const float2*, float2*, cudaStream_t, const int*);

// b = e_0 (x) b_0 (Sec. 3.1): mode 0 holds the FD-weighted source, other
// modes are zero.
template <typename T>
__global__ void k_rhs(long long N, int n, const double* __restrict__ b0, C2<T>* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    b[i] = mk<T>(i < n ? T(b0[i]) : T(0), T(0));
}

template <typename T>
cudaError_t launch_rhs(const sg_handle* h, C2<T>* b, cudaStream_t st) {
  const int grid = std::max(1, std::min((int)((h->N + 255) / 256), h->num_sms * 8));
  k_rhs<T><<<grid, 256, 0, st>>>(h->N, h->n, h->d_b0, b); note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_rhs<double>(const sg_handle*, double2*, cudaStream_t);
template cudaError_t launch_rhs<float>(const sg_handle*, float2*, cudaStream_t);

}  // namespace sgi
