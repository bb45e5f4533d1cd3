// Host side of the SG Helmholtz library: problem validation, chaos tables,
// node fields, preconditioner set-up and the operator entry points of the
// C ABI (include/sg.h).
//
// Paper sections implemented here:
//  * Sec. 2.2/2.3: multi-indices of total degree <= r, orthonormal Legendre
//    chaos; Galerkin products of the wavenumber model k = k_0 + sum xi_l k_l.
//  * Lemma 3.2 / Lemma A.3: the coupling of modes a, b is a sum of
//    coefficient fields times <xi_l phi_a phi_b> or <xi_l xi_l' phi_a phi_b>;
//    only pairs whose multi-indices differ by e_l, 2 e_l or e_l +- e_l' couple.
//  * Appendix A: FD weights; the right-hand side b_0 = D_2-weights * f.
//  * Sec. 5 / Sec. 6.3: mean-value and CSL-mean blocks and their one-time
//    factorisation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>

#include "csym_eig.h"
#include "sg_internal.h"

namespace sgi {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_device{-1};   // the one CUDA device this process's handles use

static thread_local long long t_launches = 0;
void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long thread_launches() { return t_launches; }

void set_error(const std::string& msg) { g_err = msg; }
sg_status fail(sg_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

// ------------------------------------------------------------------ chaos tables
// Recurrence coefficient of the orthonormal Legendre polynomials under the
// uniform density on [-1, 1]: xi p_n = b_{n+1} p_{n+1} + b_n p_{n-1}.
static double leg_b(int n) { return n <= 0 ? 0.0 : n / std::sqrt(4.0 * n * n - 1.0); }

// Multi-indices of total degree <= r: graded, descending lexicographic inside
// a degree (the ordering the ABI documents).
static void enumerate_level(int s, int left, std::vector<int>& cur, std::vector<int>& out) {
  int pos = (int)cur.size();
  if (pos == s - 1) {
    cur.push_back(left);
    out.insert(out.end(), cur.begin(), cur.end());
    cur.pop_back();
    return;
  }
  for (int a = left; a >= 0; --a) {
    cur.push_back(a);
    enumerate_level(s, left - a, cur, out);
    cur.pop_back();
  }
}

static std::vector<int> multi_indices(int s, int r) {
  std::vector<int> out;
  if (s == 0) return out;
  std::vector<int> cur;
  for (int d = 0; d <= r; ++d) enumerate_level(s, d, cur, out);
  return out;
}

static int pair_index(int s, int l, int lp) {  // l < lp
  int idx = 0;
  for (int a = 0; a < l; ++a) idx += s - 1 - a;
  return idx + (lp - l - 1);
}

// Coupling of mode a with mode b != a.  Returns false if they do not couple.
// Term ids: [0, s) <xi_l phi phi> (coefficient -2 w2 k0 k_l - i w1 k_l);
// [s, 2s) <xi_l^2 phi phi> off the diagonal (coefficient -w2 k_l^2);
// [2s, 2s + s(s-1)/2) <xi_l xi_l' phi phi>, l < l' (coefficient -2 w2 k_l k_l').
static bool coupling(int s, const int* aa, const int* bb, int* term, double* g) {
  int nd = 0, l1 = -1, l2 = -1, dmax = 0;
  for (int t = 0; t < s; ++t) {
    int d = std::abs(aa[t] - bb[t]);
    if (d) {
      ++nd;
      if (l1 < 0) l1 = t; else l2 = t;
      dmax = std::max(dmax, d);
    }
  }
  if (nd == 1 && dmax == 1) {
    *term = l1;
    *g = leg_b(std::max(aa[l1], bb[l1]));
    return true;
  }
  if (nd == 1 && dmax == 2) {
    int m = std::min(aa[l1], bb[l1]);
    *term = s + l1;
    *g = leg_b(m + 1) * leg_b(m + 2);
    return true;
  }
  if (nd == 2 && dmax == 1) {
    *term = 2 * s + pair_index(s, l1, l2);
    *g = leg_b(std::max(aa[l1], bb[l1])) * leg_b(std::max(aa[l2], bb[l2]));
    return true;
  }
  return false;
}

static int binom(int n, int k) {
  long long v = 1;
  for (int i = 1; i <= k; ++i) v = v * (n - k + i) / i;
  return (int)v;
}

// ------------------------------------------------------------------ eigenpairs
// Accepted eigenvector factors of the 1D pencils: the preconditioner applies
// Q^T as Q^-1, so Q^T Q = I must hold far below the 1e-10 parity of the FP64
// apply, and the FP32/TF32 transforms amplify rounding by up to cond(Q).
constexpr double kEigOrthMax = 1e-10;
constexpr double kEigKappaMax = 100.0;

static bool pencil_eig(int n, const std::vector<cd>& diag, const std::vector<cd>& off, std::vector<cd>& lam,
                       std::vector<cd>& Q, double* orth_err, double* kappa) {
  if (!csym::tridiag_eig(n, diag, off, lam, Q, orth_err, kappa)) return false;
  return *orth_err <= kEigOrthMax && *kappa <= kEigKappaMax;
}

}  // namespace sgi

using namespace sgi;

// ------------------------------------------------------------------ handle helpers
OpParams<double> sg_handle::op64() const {
  OpParams<double> p{};
  p.dim = dim; p.mx = mx; p.my = my; p.n = n; p.P = P; p.s = s; p.T_terms = T_terms;
  p.absL = bc[0] == SG_BC_ABSORBING; p.absR = bc[1] == SG_BC_ABSORBING;
  p.absB = dim == 2 && bc[2] == SG_BC_ABSORBING; p.absT = dim == 2 && bc[3] == SG_BC_ABSORBING;
  p.h = h; p.inv_h = 1.0 / h; p.inv_h2 = 1.0 / (h * h);
  p.rowptr = d_rowptr; p.col = d_col; p.term = d_term; p.gval = d_gval; p.gdiag = d_gdiag;
  p.fields = d_fields;
  p.skip = nullptr;
  return p;
}

OpParams<float> sg_handle::op32() const {
  OpParams<float> p{};
  p.dim = dim; p.mx = mx; p.my = my; p.n = n; p.P = P; p.s = s; p.T_terms = T_terms;
  p.absL = bc[0] == SG_BC_ABSORBING; p.absR = bc[1] == SG_BC_ABSORBING;
  p.absB = dim == 2 && bc[2] == SG_BC_ABSORBING; p.absT = dim == 2 && bc[3] == SG_BC_ABSORBING;
  p.h = (float)h; p.inv_h = (float)(1.0 / h); p.inv_h2 = (float)(1.0 / (h * h));
  p.rowptr = d_rowptr; p.col = d_col; p.term = d_term; p.gval = d_gval32; p.gdiag = d_gdiag32;
  p.fields = d_fields32;
  p.skip = nullptr;
  return p;
}

template <typename T>
static cudaError_t upload(T** dst, const T* src, size_t count) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (count) e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

static void free_factors(PrecBlock& b) {
  cudaFree(b.f64.dl); cudaFree(b.f64.dinv); cudaFree(b.f64.du); cudaFree(b.f64.du2); cudaFree(b.f64.piv);
  cudaFree(b.f32.dl); cudaFree(b.f32.dinv); cudaFree(b.f32.du); cudaFree(b.f32.du2);
  cudaFree(b.band.ab); cudaFree(b.band.ab32); cudaFree(b.band.piv);
  b = PrecBlock{};
}

static cudaError_t alloc_factors(PrecBlock& b, size_t cnt) {
  cudaError_t e;
  if ((e = cudaMalloc((void**)&b.f64.dl, cnt * sizeof(double2)))) return e;
  if ((e = cudaMalloc((void**)&b.f64.dinv, cnt * sizeof(double2)))) return e;
  if ((e = cudaMalloc((void**)&b.f64.du, cnt * sizeof(double2)))) return e;
  if ((e = cudaMalloc((void**)&b.f64.du2, cnt * sizeof(double2)))) return e;
  if ((e = cudaMalloc((void**)&b.f64.piv, cnt))) return e;
  if ((e = cudaMalloc((void**)&b.f32.dl, cnt * sizeof(float2)))) return e;
  if ((e = cudaMalloc((void**)&b.f32.dinv, cnt * sizeof(float2)))) return e;
  if ((e = cudaMalloc((void**)&b.f32.du, cnt * sizeof(float2)))) return e;
  if ((e = cudaMalloc((void**)&b.f32.du2, cnt * sizeof(float2)))) return e;
  b.f32.piv = b.f64.piv;
  return cudaSuccess;
}

void sgi_free_gmres_work(sg_handle* h);  // solver.cu

namespace sgi {
// Device operands of the four tensor-core transforms from the host factors
// (hi / lo TF32 parts in the MMA's core-matrix order, tile width bn or the
// rule).  The old operands are freed only once the new ones are in place.
sg_status tc_build_operands(sg_handle* h, int bn) {
  if (bn != 0 && bn != 64 && bn != 128 && bn != 256)
    return fail(SG_EINVAL, "transform tile width must be 64, 128 or 256");
  const bool wide = bn == 256;
  if (wide && !tc_wide_available())
    return fail(SG_EUNSUPPORTED, "the 256-column transforms need clusters of two CTAs, which this GPU cannot hold");
  TcDevOperand fresh[4], freshW[4];
  auto free_fresh = [&]() {
    for (int u = 0; u < 4; ++u) {
      cudaFree(fresh[u].hi); cudaFree(fresh[u].lo); cudaFree(fresh[u].h16);
      cudaFree(freshW[u].h16);
    }
  };
  for (int t = 0; t < 4; ++t) {
    if (h->tc_fac[t].empty()) {
      free_fresh();
      return fail(SG_EUNSUPPORTED, "this problem has no tensor-core transforms");
    }
    if (wide) {
      TcOperand ow = tc_make_operand16(h->tc_fac[t], h->tc_dim[t], h->tc_dim[t], 256);
      TcDevOperand& d = freshW[t];
      d.kdim = ow.kdim; d.ndim = ow.ndim; d.nks = ow.nks; d.ntiles = ow.ntiles; d.bn = ow.bn;
      d.nks16 = ow.nks16;
      if (upload(&d.h16, ow.h16.data(), ow.h16.size())) {
        free_fresh();
        return fail(SG_ENOMEM, "transform operand upload");
      }
    }
    const int w = wide ? 128 : bn ? bn : tc_tile_width(h->tc_rows[t], h->tc_dim[t], h->num_sms);
    TcOperand op = tc_make_operand(h->tc_fac[t], h->tc_dim[t], h->tc_dim[t], w);
    TcDevOperand& d = fresh[t];
    d.kdim = op.kdim; d.ndim = op.ndim; d.nks = op.nks; d.ntiles = op.ntiles; d.bn = op.bn;
    d.nks16 = op.nks16;
    if (upload(&d.hi, op.hi.data(), op.hi.size()) || upload(&d.lo, op.lo.data(), op.lo.size()) ||
        upload(&d.h16, op.h16.data(), op.h16.size())) {
      free_fresh();
      return fail(SG_ENOMEM, "transform operand upload");
    }
  }
  // no transform of the old operands still running, and no captured graph
  // left that names them
  drop_graphs(h);
  for (int t = 0; t < 4; ++t) {
    cudaFree(h->tcB[t].hi);
    cudaFree(h->tcB[t].lo);
    cudaFree(h->tcB[t].h16);
    cudaFree(h->tcW[t].h16);
    h->tcB[t] = fresh[t];
    h->tcW[t] = freshW[t];
  }
  h->tc_wide = wide;
  return SG_OK;
}
}  // namespace sgi

static void destroy_impl(sg_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->d_rowptr); cudaFree(h->d_col); cudaFree(h->d_term);
  cudaFree(h->d_gval); cudaFree(h->d_gdiag); cudaFree(h->d_fields); cudaFree(h->d_b0);
  cudaFree(h->d_gval32); cudaFree(h->d_gdiag32); cudaFree(h->d_fields32);
  for (auto& b : h->blk) if (b.f64.dl || b.band.ab) free_factors(b);
  cudaFree(h->csl_full.ab); cudaFree(h->csl_full.ab32); cudaFree(h->csl_full.piv);
  cudaFree(h->d_Q); cudaFree(h->d_Qt); cudaFree(h->d_Q32); cudaFree(h->d_Qt32);
  cudaFree(h->d_dyinv); cudaFree(h->d_dyinv32); cudaFree(h->d_tmp); cudaFree(h->d_tmp2);
  cudaFree(h->d_Qy32); cudaFree(h->d_Qyt32); cudaFree(h->d_Linv32[0]); cudaFree(h->d_Linv32[1]);
  for (auto& t : h->tcB) { cudaFree(t.hi); cudaFree(t.lo); cudaFree(t.h16); }
  for (auto& t : h->tcW) cudaFree(t.h16);
  cudaFree(h->d_fd16s); cudaFree(h->d_fd16part);
  cudaFree(h->d_err);
  cudaFree(h->d_modemax);
  sgi_free_gmres_work(h);
  delete h;
}

// 1D pencil of one grid direction on its unknowns: T (Theorems A.1/A.2),
// end weights d (1/2 at an absorbing end) and absorbing-end indicator e.
struct Pencil1D {
  std::vector<double> tdiag, toff, d, e;
};

static Pencil1D pencil(int m, double h, int left_abs, int right_abs) {
  Pencil1D p;
  p.tdiag.assign(m, 2.0 / (h * h));
  p.toff.assign(m > 1 ? m - 1 : 0, -1.0 / (h * h));
  p.d.assign(m, 1.0);
  p.e.assign(m, 0.0);
  if (left_abs) { p.tdiag[0] = 1.0 / (h * h); p.d[0] = 0.5; p.e[0] = 1.0; }
  if (right_abs) { p.tdiag[m - 1] = 1.0 / (h * h); p.d[m - 1] = 0.5; p.e[m - 1] = 1.0; }
  return p;
}

// Longest grid line for which the FP32 2D preconditioner uses the fast
// diagonalisation instead of the tridiagonal solves along y.
constexpr int kFdMaxLine = 320;

static sg_status setup_preconditioners(sg_handle* h, cudaStream_t st) {
  const int n = h->n;
  SG_CUDA_TRY(cudaMalloc((void**)&h->d_err, sizeof(int)));
  SG_CUDA_TRY(cudaMemset(h->d_err, 0, sizeof(int)));
  int* d_bad = nullptr;
  SG_CUDA_TRY(cudaMalloc((void**)&d_bad, sizeof(int)));
  SG_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  sg_status status = SG_OK;
  if (h->dim == 1) {
    // S_blk = T - i D_1(k_0) - (1 + i beta_c) D_2(k_0^2), one tridiagonal system.
    Pencil1D px = pencil(h->mx, h->h, h->bc[0] == SG_BC_ABSORBING, h->bc[1] == SG_BC_ABSORBING);
    std::vector<double> off(px.toff);
    off.resize(std::max(n, 1), 0.0);
    double* d_off = nullptr;
    double2* d_diag = nullptr;
    if (upload(&d_off, off.data(), off.size())) return fail(SG_ENOMEM, "precond upload");
    for (int which = 0; which < 2; ++which) {
      double bc_ = which == 0 ? 0.0 : h->beta;
      std::vector<double2> diag(n);
      for (int i = 0; i < n; ++i) {
        double w1 = px.e[i] / h->h, w2 = px.d[i], k = h->k0u[i];
        diag[i] = make_double2(px.tdiag[i] - w2 * k * k, -w1 * k - bc_ * w2 * k * k);
      }
      if (upload(&d_diag, diag.data(), diag.size())) return fail(SG_ENOMEM, "precond upload");
      if (alloc_factors(h->blk[which], (size_t)n)) return fail(SG_ENOMEM, "factor alloc");
      SG_CUDA_TRY(launch_tri_factor(1, n, d_diag, nullptr, d_off, h->blk[which].f64, h->blk[which].f32,
                                    d_bad, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
      cudaFree(d_diag);
      d_diag = nullptr;
      h->blk[which].ready = true;
    }
    cudaFree(d_off);
  } else if (h->separable) {
    const double kb = h->kbar, hh = h->h;
    Pencil1D px = pencil(h->mx, hh, h->bc[0] == SG_BC_ABSORBING, h->bc[1] == SG_BC_ABSORBING);
    Pencil1D py = pencil(h->my, hh, h->bc[2] == SG_BC_ABSORBING, h->bc[3] == SG_BC_ABSORBING);
    // G = D^-1/2 (T - i (kbar/h) E - (kbar^2/2) D) D^-1/2, per direction.
    auto gmat = [&](const Pencil1D& p, std::vector<cd>& gd, std::vector<cd>& go) {
      int m = (int)p.d.size();
      gd.resize(m);
      go.resize(m > 1 ? m - 1 : 0);
      for (int i = 0; i < m; ++i)
        gd[i] = cd(p.tdiag[i] - 0.5 * kb * kb * p.d[i], -(kb / hh) * p.e[i]) / p.d[i];
      for (int i = 0; i + 1 < m; ++i) go[i] = p.toff[i] / std::sqrt(p.d[i] * p.d[i + 1]);
    };
    std::vector<cd> gxd, gxo, gyd, gyo, lam, Q;
    gmat(px, gxd, gxo);
    gmat(py, gyd, gyo);
    double oerr = 0, kap = 0;
    if (!pencil_eig(h->mx, gxd, gxo, lam, Q, &oerr, &kap))
      return fail(SG_ESINGULAR, "eigen-decomposition of the x pencil failed (|Q^T Q - I| = " + std::to_string(oerr) +
                                    ", cond(Q) = " + std::to_string(kap) + ")");
    h->eig_orth_err = oerr;
    h->eig_kappa = kap;
    const int mx = h->mx, my = h->my;
    std::vector<double2> Qh((size_t)mx * mx), Qt((size_t)mx * mx);
    std::vector<float2> Qh32((size_t)mx * mx), Qt32((size_t)mx * mx);
    for (int i = 0; i < mx; ++i)
      for (int k = 0; k < mx; ++k) {
        cd v = Q[(size_t)i * mx + k] / std::sqrt(px.d[i]);
        Qh[(size_t)i * mx + k] = make_double2(v.real(), v.imag());
        Qt[(size_t)k * mx + i] = make_double2(v.real(), v.imag());
        Qh32[(size_t)i * mx + k] = make_float2((float)v.real(), (float)v.imag());
        Qt32[(size_t)k * mx + i] = make_float2((float)v.real(), (float)v.imag());
      }
    std::vector<double> dyinv(my);
    std::vector<float> dyinv32(my);
    for (int j = 0; j < my; ++j) { dyinv[j] = 1.0 / std::sqrt(py.d[j]); dyinv32[j] = (float)dyinv[j]; }
    if (upload(&h->d_Q, Qh.data(), Qh.size()) || upload(&h->d_Qt, Qt.data(), Qt.size()) ||
        upload(&h->d_Q32, Qh32.data(), Qh32.size()) || upload(&h->d_Qt32, Qt32.data(), Qt32.size()) ||
        upload(&h->d_dyinv, dyinv.data(), dyinv.size()) || upload(&h->d_dyinv32, dyinv32.data(), dyinv32.size()))
      return fail(SG_ENOMEM, "precond upload");
    // y-direction systems: (lam_i + shift) I + G_y, shift 0 (mean) or -i beta kbar^2 (CSL).
    std::vector<double2> gdiag(my), lsh(mx);
    std::vector<double> goff(std::max(my, 1), 0.0);
    for (int j = 0; j < my; ++j) gdiag[j] = make_double2(gyd[j].real(), gyd[j].imag());
    for (int j = 0; j + 1 < my; ++j) goff[j] = gyo[j].real();
    double2* d_gd = nullptr;
    double2* d_ls = nullptr;
    double* d_go = nullptr;
    if (upload(&d_gd, gdiag.data(), gdiag.size()) || upload(&d_go, goff.data(), goff.size()))
      return fail(SG_ENOMEM, "precond upload");
    SG_CUDA_TRY(cudaMalloc((void**)&d_ls, sizeof(double2) * mx));
    for (int which = 0; which < 2; ++which) {
      cd shift = which == 0 ? cd(0, 0) : cd(0, -h->beta * kb * kb);
      for (int i = 0; i < mx; ++i) {
        cd v = lam[i] + shift;
        lsh[i] = make_double2(v.real(), v.imag());
      }
      SG_CUDA_TRY(cudaMemcpy(d_ls, lsh.data(), sizeof(double2) * mx, cudaMemcpyHostToDevice));
      if (alloc_factors(h->blk[which], (size_t)mx * my)) return fail(SG_ENOMEM, "factor alloc");
      SG_CUDA_TRY(launch_tri_factor(mx, my, d_gd, d_ls, d_go, h->blk[which].f64, h->blk[which].f32, d_bad, st));
      SG_CUDA_TRY(cudaStreamSynchronize(st));
      h->blk[which].ready = true;
    }
    cudaFree(d_gd); cudaFree(d_ls); cudaFree(d_go);
    SG_CUDA_TRY(cudaMalloc(&h->d_tmp2, (size_t)h->N * sizeof(double2)));
    // Fast diagonalisation: also diagonalise the y pencil (the same matrix as
    // x on a square grid), so the block inverse is four dense transforms on
    // the tensor cores.  The plain-TF32 form (SG_TF32, the preconditioner of
    // the complex64 GMRES cycles) always takes it.  The FP32-accurate form
    // (3xTF32, three MMAs per product) takes it only while the lines are
    // short: four such GEMMs replace two GEMMs and mx * P sequential
    // tridiagonal solves, and the GEMM work grows with mx^2; longer lines
    // keep the y sweeps and use the x factors (slots 0 and 3) alone.
    h->fd_fp32 = mx <= kFdMaxLine && my <= kFdMaxLine;
    {
      std::vector<cd> lamy, Qy;
      bool ok = true;
      if (my == mx) {
        lamy = lam;
        Qy = Q;
      } else {
        double oerr_y = 0, kap_y = 0;
        ok = pencil_eig(my, gyd, gyo, lamy, Qy, &oerr_y, &kap_y);
        h->eig_orth_err = std::max(h->eig_orth_err, oerr_y);
        h->eig_kappa = std::max(h->eig_kappa, kap_y);
      }
      if (ok) {
        std::vector<float2> Qy32((size_t)my * my), Qyt32((size_t)my * my), Linv((size_t)my * mx);
        for (int j = 0; j < my; ++j)
          for (int k = 0; k < my; ++k) {
            const cd v = Qy[(size_t)j * my + k] / std::sqrt(py.d[j]);
            Qy32[(size_t)j * my + k] = make_float2((float)v.real(), (float)v.imag());
            Qyt32[(size_t)k * my + j] = make_float2((float)v.real(), (float)v.imag());
          }
        if (upload(&h->d_Qy32, Qy32.data(), Qy32.size()) || upload(&h->d_Qyt32, Qyt32.data(), Qyt32.size()))
          return fail(SG_ENOMEM, "precond upload");
        // tensor-core factors of the four transforms (complex FP64 on the host)
        std::vector<cd> qx((size_t)mx * mx), qxt((size_t)mx * mx), qy((size_t)my * my), qyt((size_t)my * my);
        for (int a = 0; a < mx; ++a)
          for (int b = 0; b < mx; ++b) {
            const cd v = Q[(size_t)a * mx + b] / std::sqrt(px.d[a]);
            qx[(size_t)a * mx + b] = v;
            qxt[(size_t)b * mx + a] = v;
          }
        for (int a = 0; a < my; ++a)
          for (int b = 0; b < my; ++b) {
            const cd v = Qy[(size_t)a * my + b] / std::sqrt(py.d[a]);
            qy[(size_t)a * my + b] = v;
            qyt[(size_t)b * my + a] = v;
          }
        std::vector<cd>* facs[4] = {&qx, &qy, &qyt, &qxt};
        const int dims[4] = {mx, my, my, mx};
        // rows of the four GEMMs: P my, P mx, P mx, P my
        const long long rows[4] = {(long long)h->P * my, (long long)h->P * mx, (long long)h->P * mx,
                                   (long long)h->P * my};
        for (int t = 0; t < 4; ++t) {
          h->tc_fac[t] = std::move(*facs[t]);
          h->tc_dim[t] = dims[t];
          h->tc_rows[t] = rows[t];
        }
        sg_status bst = tc_build_operands(h, 0);
        if (bst != SG_OK) return bst;
        for (int which = 0; which < 2; ++which) {
          const cd shift = which == 0 ? cd(0, 0) : cd(0, -h->beta * kb * kb);
          double lmax = 0.0;
          for (int j = 0; j < my; ++j)
            for (int i = 0; i < mx; ++i) {
              const cd v = 1.0 / (lamy[j] + lam[i] + shift);
              Linv[(size_t)j * mx + i] = make_float2((float)v.real(), (float)v.imag());
              lmax = std::max(lmax, std::abs(v));
            }
          h->fd16_scale[which] = lmax > 0.0 && std::isfinite(lmax) ? (float)(1.0 / lmax) : 1.0f;
          if (upload(&h->d_Linv32[which], Linv.data(), Linv.size())) return fail(SG_ENOMEM, "precond upload");
        }
        h->fd = true;
      }
    }
  } else {
    // 2D with k_0 varying in space (the paper's wedge): S_blk has no
    // separable inverse.  Band LU of the n x n block, unknowns x fastest, so
    // kl = ku = mx; pivots in FP64 (Sec. 6.3 factors the block once for all
    // P modes).  Entries from Theorem A.5 / A.6: L = D_y (x) T_x + T_y (x) D_x
    // (D = I for Dirichlet sides), D_1 = k/h on every absorbing boundary node
    // (corners once), D_2 = d_x d_y k^2.
    const int mx = h->mx, my = h->my, kl = mx, ku = mx, kv = kl + ku, ldab = 2 * kl + ku + 1;
    const double bytes = 2.0 * (double)ldab * n * (sizeof(double2) + sizeof(float2));
    if (band_fits(kl, ku) && bytes <= 16e9) {
      Pencil1D px = pencil(mx, h->h, h->bc[0] == SG_BC_ABSORBING, h->bc[1] == SG_BC_ABSORBING);
      Pencil1D py = pencil(my, h->h, h->bc[2] == SG_BC_ABSORBING, h->bc[3] == SG_BC_ABSORBING);
      for (int which = 0; which < 2; ++which) {
        const double bc_ = which == 0 ? 0.0 : h->beta;
        std::vector<double2> ab((size_t)ldab * n, make_double2(0.0, 0.0));
        auto set = [&](int i, int c, double re, double im) {
          ab[(size_t)kv + i - c + (size_t)c * ldab] = make_double2(re, im);
        };
        for (int jy = 0; jy < my; ++jy)
          for (int ix = 0; ix < mx; ++ix) {
            const int u = ix + mx * jy;
            const double w2 = px.d[ix] * py.d[jy];
            const double w1 = (px.e[ix] > 0.0 || py.e[jy] > 0.0) ? 1.0 / h->h : 0.0;
            const double k = h->k0u[u];
            set(u, u, py.d[jy] * px.tdiag[ix] + py.tdiag[jy] * px.d[ix] - w2 * k * k, -w1 * k - bc_ * w2 * k * k);
            if (ix > 0) set(u, u - 1, py.d[jy] * px.toff[ix - 1], 0.0);
            if (ix + 1 < mx) set(u, u + 1, py.d[jy] * px.toff[ix], 0.0);
            if (jy > 0) set(u, u - mx, py.toff[jy - 1] * px.d[ix], 0.0);
            if (jy + 1 < my) set(u, u + mx, py.toff[jy] * px.d[ix], 0.0);
          }
        BandFactor& f = h->blk[which].band;
        f.n = n; f.kl = kl; f.ku = ku; f.ldab = ldab;
        if (upload(&f.ab, ab.data(), ab.size())) return fail(SG_ENOMEM, "band factor upload");
        SG_CUDA_TRY(cudaMalloc((void**)&f.ab32, ab.size() * sizeof(float2)));
        SG_CUDA_TRY(cudaMalloc((void**)&f.piv, (size_t)n * sizeof(int)));
        SG_CUDA_TRY(band_factor(f, d_bad, st));
        SG_CUDA_TRY(cudaStreamSynchronize(st));
        h->blk[which].ready = true;
      }
    }
  }
  SG_CUDA_TRY(cudaMalloc(&h->d_tmp, (size_t)h->N * sizeof(double2)));
  if (h->dim == 2 && h->fd) {
    // inputs of transforms 2-4 of the plain-TF32 apply (rows of even length)
    const int mx = h->mx, my = h->my, P = h->P;
    const int mxp = mx + (mx & 1), myp = my + (my & 1);
    const float2* t1 = reinterpret_cast<const float2*>(h->d_tmp);
    const float2* t2 = reinterpret_cast<const float2*>(h->d_tmp2);
    h->tc_xmap_ok = tc_make_xmap(&h->tc_xmap[0], t1, myp, P * mx, my) &&
                    tc_make_xmap(&h->tc_xmap[1], t2, myp, P * mx, my) &&
                    tc_make_xmap(&h->tc_xmap[2], t1, mxp, P * my, mx);
    // the binary16 route: rows of mx or my pairs padded to a multiple of 4
    const int mx4 = (mx + 3) & ~3, my4 = (my + 3) & ~3;
    // (boxes of 64 values x 128 rows inside the tensors: lines of at least 32
    // unknowns, at least 128 rows)
    h->fd16 = h->tcB[1].h16 && mx >= 32 && my >= 32 && (long long)P * mx >= 128 && (long long)P * my >= 128 &&
              tc_make_xmap16(&h->tc_xmap16[0], h->d_tmp, my4, P * mx, my) &&
              tc_make_xmap16(&h->tc_xmap16[1], h->d_tmp2, my4, P * mx, my) &&
              tc_make_xmap16(&h->tc_xmap16[2], h->d_tmp, mx4, P * my, mx);
    if (h->fd16) {
      SG_CUDA_TRY(cudaMalloc((void**)&h->d_fd16s, 2 * sizeof(double)));
      SG_CUDA_TRY(cudaMalloc((void**)&h->d_fd16part, (size_t)kFd16Blocks * sizeof(double)));
    }
  }
  int bad = 0;
  SG_CUDA_TRY(cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost));
  cudaFree(d_bad);
  if (bad) {
    for (auto& b : h->blk) b.ready = false;
    status = fail(SG_ESINGULAR, "zero pivot in a preconditioner factorisation");
  }
  return status;
}

namespace sgi {

// The coupled CSL matrix M(beta) = L - iB - (1 + i beta) C = A - i beta K of
// Sec. 4 (K = [C_ij], the k^2 part of A; Theorem 3.4), numbered point by
// point: row u P + a for grid unknown u and chaos mode a.  Within a grid
// unknown the P x P coupling of Sec. 3.2 (<k phi_a phi_b> with D_1, <k^2
// phi_a phi_b> with D_2); between neighbouring unknowns the FD stencil of
// L on each mode.  So the band has kl = ku = P in 1D and mx P in 2D.
// Assembled on the host from the chaos tables and factored (FP64 pivots) on
// first use; too wide a band returns SG_EUNSUPPORTED.
sg_status ensure_csl_full(sg_handle* h, cudaStream_t st) {
  if (h->csl_full.ab) return SG_OK;
  const int n = h->n, P = h->P, s = h->s, mx = h->mx, my = h->my;
  const long long N = h->N;
  const int kl = (h->dim == 1 ? 1 : mx) * P, ku = kl, kv = kl + ku, ldab = 2 * kl + ku + 1;
  if (!band_fits(kl, ku) || (double)N * kl * (double)(kl + ku) > 2e9)
    return fail(SG_EUNSUPPORTED, "the coupled CSL matrix's band (" + std::to_string(kl) +
                                     " sub-diagonals) is too wide for the banded factorisation");
  // term t -> (l, l') of its coefficient field(s)
  std::vector<int> tl(h->T_terms, 0), tl2(h->T_terms, 0);
  for (int l = 0; l < s; ++l) {
    tl[l] = l;
    tl[s + l] = l;
    for (int lp = l + 1; lp < s; ++lp) {
      const int t = 2 * s + pair_index(s, l, lp);
      tl[t] = l;
      tl2[t] = lp;
    }
  }
  Pencil1D px = pencil(mx, h->h, h->bc[0] == SG_BC_ABSORBING, h->bc[1] == SG_BC_ABSORBING);
  Pencil1D py = h->dim == 2 ? pencil(my, h->h, h->bc[2] == SG_BC_ABSORBING, h->bc[3] == SG_BC_ABSORBING) : Pencil1D{};
  const double beta = h->beta;
  std::vector<double2> ab((size_t)ldab * N, make_double2(0.0, 0.0));
  auto set = [&](long long i, long long c, double re, double im) {
    ab[(size_t)(kv + i - c) + (size_t)c * ldab] = make_double2(re, im);
  };
  const double* F = h->fields_host.data();
  for (int jy = 0; jy < my; ++jy)
    for (int ix = 0; ix < mx; ++ix) {
      const int u = ix + mx * jy;
      double lu, w1, w2;
      if (h->dim == 1) {
        lu = px.tdiag[ix];
        w1 = px.e[ix] / h->h;
        w2 = px.d[ix];
      } else {
        lu = py.d[jy] * px.tdiag[ix] + py.tdiag[jy] * px.d[ix];
        w1 = (px.e[ix] > 0.0 || py.e[jy] > 0.0) ? 1.0 / h->h : 0.0;
        w2 = px.d[ix] * py.d[jy];
      }
      const double k0 = F[u];
      for (int a = 0; a < P; ++a) {
        const long long row = (long long)u * P + a;
        // <k^2 phi_a phi_a> and <k phi_a phi_a> = k_0
        double d2 = k0 * k0;
        for (int l = 0; l < s; ++l) {
          const double kl_ = F[(size_t)(l + 1) * n + u];
          d2 += kl_ * kl_ * h->gdiag[(size_t)l * P + a];
        }
        set(row, row, lu - w2 * d2, -w1 * k0 - beta * w2 * d2);
        for (int e = h->rowptr[a]; e < h->rowptr[a + 1]; ++e) {
          const int b = h->col[e], t = h->term[e];
          const double g = h->gval[e];
          const double kA = F[(size_t)(tl[t] + 1) * n + u];
          double c1 = 0.0, c2;
          if (t < s) {
            c1 = kA;
            c2 = 2.0 * k0 * kA;
          } else if (t < 2 * s) {
            c2 = kA * kA;
          } else {
            c2 = 2.0 * kA * F[(size_t)(tl2[t] + 1) * n + u];
          }
          set(row, (long long)u * P + b, -w2 * c2 * g, -w1 * c1 * g - beta * w2 * c2 * g);
        }
        // the FD stencil between neighbouring unknowns, mode by mode
        if (h->dim == 1) {
          if (ix > 0) set(row, row - P, px.toff[ix - 1], 0.0);
          if (ix + 1 < mx) set(row, row + P, px.toff[ix], 0.0);
        } else {
          if (ix > 0) set(row, row - P, py.d[jy] * px.toff[ix - 1], 0.0);
          if (ix + 1 < mx) set(row, row + P, py.d[jy] * px.toff[ix], 0.0);
          if (jy > 0) set(row, row - (long long)mx * P, py.toff[jy - 1] * px.d[ix], 0.0);
          if (jy + 1 < my) set(row, row + (long long)mx * P, py.toff[jy] * px.d[ix], 0.0);
        }
      }
    }
  BandFactor f;
  f.n = (int)N; f.kl = kl; f.ku = ku; f.ldab = ldab;
  int* d_bad = nullptr;
  cudaError_t e = cudaSuccess;
  if (upload(&f.ab, ab.data(), ab.size())) e = cudaErrorMemoryAllocation;
  if (!e) e = cudaMalloc((void**)&f.ab32, ab.size() * sizeof(float2));
  if (!e) e = cudaMalloc((void**)&f.piv, (size_t)N * sizeof(int));
  if (!e) e = cudaMalloc((void**)&d_bad, sizeof(int));
  if (!e) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (!e) e = band_factor(f, d_bad, st);
  int bad = 0;
  if (!e) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  cudaFree(d_bad);
  if (e || bad) {
    cudaFree(f.ab); cudaFree(f.ab32); cudaFree(f.piv);
    if (e) return fail(SG_ECUDA, std::string("coupled CSL factorisation: ") + cudaGetErrorString(e));
    return fail(SG_ESINGULAR, "zero pivot in the coupled CSL factorisation");
  }
  h->csl_full = f;
  return SG_OK;
}

// Block index of a preconditioner kind (0 mean value, 1 CSL mean value, 2
// coupled CSL) and whether it is available for the handle.
bool prec_available(const sg_handle* h, sg_prec kind) {
  if (kind == SG_PREC_MEAN) return h->blk[0].ready;
  if (kind == SG_PREC_CSL_MEAN) return h->blk[1].ready;
  return kind == SG_PREC_CSL;
}

}  // namespace sgi

extern "C" {

const char* sg_last_error(void) { return sgi::g_err.c_str(); }
int sg_version(void) { return 100; }
long long sg_kernel_launches(void) { return sgi::g_launches.load(); }

sg_status sg_assemble(const sg_desc* desc, void* stream, sg_handle** out) {
  return sgi::guarded([&]() -> sg_status {
    g_err.clear();
    if (!desc || !out) return fail(SG_EINVAL, "NULL desc or out");
    const sg_desc& D = *desc;
    if (D.dim != 1 && D.dim != 2) return fail(SG_EINVAL, "dim must be 1 or 2");
    if (D.nx < 3 || (D.dim == 2 && D.ny < 3) || (D.dim == 1 && D.ny != 1))
      return fail(SG_EINVAL, "grid too small (nx, ny >= 3; ny = 1 in 1D)");
    if (!(D.h > 0) || !std::isfinite(D.h)) return fail(SG_EINVAL, "h must be positive");
    if (D.s < 0 || D.s > 16 || D.r < 0 || D.r > 12) return fail(SG_EINVAL, "s in [0,16], r in [0,12]");
    for (int i = 0; i < (D.dim == 2 ? 4 : 2); ++i)
      if (D.bc[i] != SG_BC_DIRICHLET && D.bc[i] != SG_BC_ABSORBING) return fail(SG_EINVAL, "bad bc");
    if (D.dim == 2 && !(D.bc[0] == D.bc[1] && D.bc[1] == D.bc[2] && D.bc[2] == D.bc[3]))
      return fail(SG_EINVAL, "2D needs all-Dirichlet or all-absorbing boundaries (Theorems A.5/A.6)");
    // unknowns are indexed with 32-bit integers on the device (2 n + 1 < 2^31)
    if ((long long)D.nx * (D.dim == 2 ? D.ny : 1) > (1LL << 30))
      return fail(SG_EINVAL, "grid too large (at most 2^30 nodes)");
    if (!D.k0 || (D.s > 0 && !D.kl)) return fail(SG_EINVAL, "NULL wavenumber field");
    if (!std::isfinite(D.beta)) return fail(SG_EINVAL, "beta not finite");
    if (D.point_source && (!(D.point_x >= 0.0 && D.point_x <= 1.0) ||
                           (D.dim == 2 && !(D.point_y >= 0.0 && D.point_y <= 1.0))))
      return fail(SG_EINVAL, "point source outside the unit interval / square");

    auto* h = new sg_handle();
    h->dim = D.dim; h->nx = D.nx; h->ny = D.dim == 2 ? D.ny : 1; h->h = D.h; h->beta = D.beta;
    for (int i = 0; i < 4; ++i) h->bc[i] = (D.dim == 1 && i >= 2) ? SG_BC_DIRICHLET : D.bc[i];
    h->s = D.s; h->r = D.r;
    h->offx = h->bc[0] == SG_BC_DIRICHLET ? 1 : 0;
    h->mx = D.nx - h->offx - (h->bc[1] == SG_BC_DIRICHLET ? 1 : 0);
    if (D.dim == 2) {
      h->offy = h->bc[2] == SG_BC_DIRICHLET ? 1 : 0;
      h->my = D.ny - h->offy - (h->bc[3] == SG_BC_DIRICHLET ? 1 : 0);
    }
    h->n = h->mx * h->my;
    h->P = D.s == 0 ? 1 : binom(D.s + D.r, D.s);
    h->N = (long long)h->n * h->P;
    h->T_terms = 2 * D.s + D.s * (D.s - 1) / 2;
    if (h->P > 4096) { delete h; return fail(SG_EINVAL, "too many chaos modes"); }

    // node fields restricted to the unknowns, validation k > 0 (Sec. 3.2)
    const int n = h->n, s = h->s, P = h->P;
    const size_t nodes = (size_t)D.nx * h->ny;
    std::vector<double> fields((size_t)(s + 1) * n);
    h->b0.assign(n, 0.0);
    double kmin = 1e300, kmax = -1e300, k0min = 1e300, k0max = -1e300;
    for (int ju = 0; ju < h->my; ++ju)
      for (int iu = 0; iu < h->mx; ++iu) {
        size_t node = (size_t)(iu + h->offx) + (size_t)D.nx * (ju + h->offy);
        int u = iu + h->mx * ju;
        double k0 = D.k0[node], spread = 0;
        fields[u] = k0;
        for (int l = 0; l < s; ++l) {
          double kl = D.kl[(size_t)l * nodes + node];
          fields[(size_t)(l + 1) * n + u] = kl;
          spread += std::fabs(kl);
          if (!std::isfinite(kl)) { delete h; return fail(SG_EINVAL, "non-finite k_l"); }
        }
        if (!std::isfinite(k0)) { delete h; return fail(SG_EINVAL, "non-finite k_0"); }
        kmin = std::min(kmin, k0 - spread);
        kmax = std::max(kmax, k0 + spread);
        k0min = std::min(k0min, k0);
        k0max = std::max(k0max, k0);
        double f = D.f ? D.f[node] : 0.0;
        if (!std::isfinite(f)) { delete h; return fail(SG_EINVAL, "non-finite f"); }
        bool xabs = (iu == 0 && h->bc[0] == SG_BC_ABSORBING) || (iu == h->mx - 1 && h->bc[1] == SG_BC_ABSORBING);
        bool yabs = D.dim == 2 && ((ju == 0 && h->bc[2] == SG_BC_ABSORBING) ||
                                   (ju == h->my - 1 && h->bc[3] == SG_BC_ABSORBING));
        h->b0[u] = (xabs ? 0.5 : 1.0) * (yabs ? 0.5 : 1.0) * f;
      }
    if (!(kmin > 0)) { delete h; return fail(SG_EINVAL, "k(x, xi) must be positive for all xi (k_0 - sum|k_l| <= 0)"); }
    if (D.point_source) {
      // App. A.3: delta(x - a) becomes 1/h^dim at the node closest to a (the
      // smaller index on a tie; the small guard keeps an exact tie from being
      // split by the rounding of a / h), weighted like f by the D_2 weights
      auto nearest = [&](double a, int nodes_dir) {
        const int j = (int)std::ceil(a / D.h - 0.5 - 1e-9);
        return std::min(std::max(j, 0), nodes_dir - 1);
      };
      const int iu = nearest(D.point_x, D.nx) - h->offx;
      const int ju = D.dim == 2 ? nearest(D.point_y, h->ny) - h->offy : 0;
      if (iu >= 0 && iu < h->mx && ju >= 0 && ju < h->my) {
        const bool xabs = (iu == 0 && h->bc[0] == SG_BC_ABSORBING) || (iu == h->mx - 1 && h->bc[1] == SG_BC_ABSORBING);
        const bool yabs = D.dim == 2 && ((ju == 0 && h->bc[2] == SG_BC_ABSORBING) ||
                                         (ju == h->my - 1 && h->bc[3] == SG_BC_ABSORBING));
        const double val = D.dim == 2 ? 1.0 / (D.h * D.h) : 1.0 / D.h;
        h->b0[(size_t)iu + (size_t)h->mx * ju] += (xabs ? 0.5 : 1.0) * (yabs ? 0.5 : 1.0) * val;
      }
    }
    h->kbar = 0.5 * (k0min + k0max);
    h->specialised = matvec_is_specialised(h->s, h->r) ? 1 : 0;
    h->separable = (k0max - k0min) <= 1e-13 * k0max;
    h->k0u.assign(fields.begin(), fields.begin() + n);
    h->fields_host = fields;

    // chaos tables
    h->alpha = multi_indices(s, h->r);
    if (s == 0) h->alpha.clear();
    h->rowptr.assign(P + 1, 0);
    for (int a = 0; a < P; ++a) {
      for (int b = 0; b < P; ++b) {
        if (a == b) continue;
        int t;
        double g;
        if (coupling(s, &h->alpha[(size_t)a * s], &h->alpha[(size_t)b * s], &t, &g)) {
          h->col.push_back(b);
          h->term.push_back(t);
          h->gval.push_back(g);
        }
      }
      h->rowptr[a + 1] = (int)h->col.size();
    }
    h->gdiag.assign((size_t)std::max(s, 1) * P, 0.0);
    for (int l = 0; l < s; ++l)
      for (int a = 0; a < P; ++a) {
        int al = h->alpha[(size_t)a * s + l];
        h->gdiag[(size_t)l * P + a] = leg_b(al) * leg_b(al) + leg_b(al + 1) * leg_b(al + 1);
      }

    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) { delete h; return fail(SG_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e)); }
    // one device per process: kernel attributes (dynamic shared memory
    // limits) and SM counts are set up once, on the first device used
    {
      int expected = -1;
      if (!g_device.compare_exchange_strong(expected, h->device) && expected != h->device) {
        const int first = expected;
        delete h;
        return fail(SG_EUNSUPPORTED, "the library serves one CUDA device per process (first used: device " +
                                         std::to_string(first) + "); run one process per GPU");
      }
    }
    // the allocation-free entry point's static scratch: its address is looked
    // up here, where allocation is allowed (the lookup loads its module)
    if ((e = noalloc_scratch_address(&h->noalloc_scratch)) != cudaSuccess) {
      delete h;
      return fail(SG_ECUDA, std::string("static scratch address: ") + cudaGetErrorString(e));
    }

    std::vector<float> gval32(h->gval.begin(), h->gval.end()), gdiag32(h->gdiag.begin(), h->gdiag.end()),
        fields32(fields.begin(), fields.end());
    if (upload(&h->d_rowptr, h->rowptr.data(), h->rowptr.size()) ||
        upload(&h->d_col, h->col.data(), h->col.size()) || upload(&h->d_term, h->term.data(), h->term.size()) ||
        upload(&h->d_gval, h->gval.data(), h->gval.size()) || upload(&h->d_gdiag, h->gdiag.data(), h->gdiag.size()) ||
        upload(&h->d_fields, fields.data(), fields.size()) || upload(&h->d_b0, h->b0.data(), h->b0.size()) ||
        upload(&h->d_gval32, gval32.data(), gval32.size()) ||
        upload(&h->d_gdiag32, gdiag32.data(), gdiag32.size()) ||
        upload(&h->d_fields32, fields32.data(), fields32.size())) {
      destroy_impl(h);
      return fail(SG_ENOMEM, "device allocation for fields/tables failed");
    }
    sg_status ps = setup_preconditioners(h, st);
    if (ps != SG_OK && ps != SG_ESINGULAR) {
      destroy_impl(h);
      return ps;
    }
    if (ps == SG_ESINGULAR) {
      destroy_impl(h);
      return ps;
    }
    *out = h;
    return SG_OK;
  });
}

void sg_destroy(sg_handle* h) { destroy_impl(h); }

sg_status sg_get_info(const sg_handle* h, sg_info* info) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !info) return fail(SG_EINVAL, "NULL handle or info");
    info->dim = h->dim; info->mx = h->mx; info->my = h->my; info->n = h->n; info->P = h->P;
    info->N = h->N; info->s = h->s; info->r = h->r; info->terms = h->T_terms;
    info->coupling_nnz = (int)h->col.size() + h->P;
    info->separable = h->separable ? 1 : 0;
    info->specialised = h->specialised;
    info->fast_diag = h->fd && h->fd_fp32 ? 1 : 0;
    info->tf32_route = h->fd ? 1 : 0;
    info->fp16_route = h->fd16 ? 1 : 0;
    info->eig_orth_err = h->eig_orth_err;
    info->eig_kappa = h->eig_kappa;
    return SG_OK;
  });
}

sg_status sg_rhs(sg_handle* h, sg_precision prec, void* b, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !b) return fail(SG_EINVAL, "NULL handle or b");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == SG_FP64) SG_CUDA_TRY(launch_rhs<double>(h, (double2*)b, st));
    else if (prec == SG_FP32) SG_CUDA_TRY(launch_rhs<float>(h, (float2*)b, st));
    else return fail(SG_EINVAL, "sg_rhs precision must be SG_FP64 or SG_FP32");
    return SG_OK;
  });
}

sg_status sg_matvec(sg_handle* h, sg_precision prec, const void* X, void* Y, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !X || !Y) return fail(SG_EINVAL, "NULL handle or vector");
    if (X == Y) return fail(SG_EINVAL, "sg_matvec: X and Y must not overlap");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == SG_FP64) SG_CUDA_TRY(launch_matvec<double>(h, (const double2*)X, (double2*)Y, st));
    else if (prec == SG_FP32) SG_CUDA_TRY(launch_matvec<float>(h, (const float2*)X, (float2*)Y, st));
    else return fail(SG_EINVAL, "sg_matvec precision must be SG_FP64 or SG_FP32");
    return SG_OK;
  });
}

sg_status sg_precond(sg_handle* h, sg_prec kind, sg_precision prec, const void* R, void* Z, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !R || !Z) return fail(SG_EINVAL, "NULL handle or vector");
    if (prec != SG_FP64 && prec != SG_FP32 && prec != SG_TF32 && prec != SG_FP16)
      return fail(SG_EINVAL, "sg_precond precision must be SG_FP64, SG_FP32, SG_TF32 or SG_FP16");
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = (size_t)h->N * (prec == SG_FP64 ? sizeof(double2) : sizeof(float2));
    if (kind == SG_PREC_NONE) {
      if (R != Z) SG_CUDA_TRY(cudaMemcpyAsync(Z, R, bytes, cudaMemcpyDeviceToDevice, st));
      return SG_OK;
    }
    if (kind != SG_PREC_MEAN && kind != SG_PREC_CSL_MEAN && kind != SG_PREC_CSL)
      return fail(SG_EINVAL, "unknown preconditioner");
    const int which = kind == SG_PREC_MEAN ? 0 : kind == SG_PREC_CSL_MEAN ? 1 : 2;
    if (which == 2) {
      if (prec == SG_TF32 || prec == SG_FP16) return fail(SG_EUNSUPPORTED, "SG_TF32 / SG_FP16 have no coupled CSL route");
      sg_status s = ensure_csl_full(h, st);
      if (s != SG_OK) return s;
    } else if (!h->blk[which].ready) {
      return fail(SG_EUNSUPPORTED, "no factorisation for this block (its band is too wide for the device solve)");
    }
    if (prec == SG_TF32) {
      if (h->dim != 2 || !h->fd)
        return fail(SG_EUNSUPPORTED, "SG_TF32 needs a 2D problem with constant k_0 (the fast-diagonalisation route)");
      SG_CUDA_TRY(launch_precond_tf32(h, which, (const float2*)R, (float2*)Z, st, nullptr, nullptr));
    } else if (prec == SG_FP16) {
      if (!h->fd16) return fail(SG_EUNSUPPORTED, "no SG_FP16 route for this problem");
      SG_CUDA_TRY(launch_precond_f16(h, which, (const float2*)R, (float2*)Z, st, nullptr, nullptr));
    } else if (prec == SG_FP64) {
      SG_CUDA_TRY(launch_precond<double>(h, which, (const double2*)R, (double2*)Z, st));
    } else {
      SG_CUDA_TRY(launch_precond<float>(h, which, (const float2*)R, (float2*)Z, st));
    }
    return SG_OK;
  });
}

sg_status sg_fd_transform(sg_handle* h, sg_prec kind, sg_precision prec, int t, const void* X, void* Y,
                          void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (!h || !X || !Y) return fail(SG_EINVAL, "NULL handle or vector");
    if (prec != SG_TF32 && prec != SG_FP16) return fail(SG_EINVAL, "precision must be SG_TF32 or SG_FP16");
    if (prec == SG_FP16 && !h->fd16) return fail(SG_EUNSUPPORTED, "no SG_FP16 route for this problem");
    if (t < 0 || t > 3) return fail(SG_EINVAL, "transform index must be 0 .. 3");
    if (kind != SG_PREC_MEAN && kind != SG_PREC_CSL_MEAN) return fail(SG_EINVAL, "kind must be SG_PREC_MEAN or SG_PREC_CSL_MEAN");
    const int which = kind == SG_PREC_MEAN ? 0 : 1;
    if (h->dim != 2 || !h->fd || !h->blk[which].ready)
      return fail(SG_EUNSUPPORTED, "the fast-diagonalisation transforms need a 2D problem with constant k_0");
    SG_CUDA_TRY(fd_transform(h, which, t, (const float2*)X, (float2*)Y, (cudaStream_t)stream, prec == SG_FP16));
    return SG_OK;
  });
}

sg_status sg_selftest_wait_timeout(void* stream, int* timed_out, double* seconds) {
  return sgi::guarded([&]() -> sg_status {
    g_err.clear();
    if (!timed_out) return fail(SG_EINVAL, "NULL timed_out");
    *timed_out = 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int* d = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int hflags[2] = {0, 0};
    float ms = 0.f;
    cudaError_t e = cudaMalloc((void**)&d, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = tc_wait_selftest(d, d + 1, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, d, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return fail(SG_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
    if (!hflags[1]) return fail(SG_ECUDA, "wait self-test: the kernel did not reach its end");
    *timed_out = hflags[0];
    if (seconds) *seconds = ms * 1e-3;
    if (hflags[0]) return fail(SG_ETIMEOUT, "a device-side wait timed out (self-test: the expected outcome)");
    return SG_OK;
  });
}

}  // extern "C"
