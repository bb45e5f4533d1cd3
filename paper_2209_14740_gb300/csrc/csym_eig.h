// Eigen-decomposition of a complex symmetric tridiagonal matrix on the host
// (FP64).  Used once per problem by the 2D preconditioner set-up: the 1D
// pencils of the mean-value block S(xi_bar) = D (x) T + T (x) D - ... of
// Theorem A.6 are complex symmetric (the absorbing ends put -i k/h on two
// diagonal entries), and their eigenvectors give the separable inverse.
//
// Plain C++ (no CUDA), so that a CPU test can compile it on its own.
//
//  * Eigenvalues: the implicit symmetric QR algorithm (Golub & Van Loan,
//    "Matrix Computations", Sec. 8.3: Wilkinson shift from the trailing 2 x 2
//    block, bulge chased down the band by plane rotations, deflation of
//    negligible off-diagonal entries).  For a complex symmetric matrix the
//    rotations are complex orthogonal (c^2 + s^2 = 1, not unitary), which
//    keeps the tridiagonal matrix complex symmetric (the variant Cullum &
//    Willoughby describe for complex symmetric Lanczos matrices).  The
//    update formulas below are derived from T' = R^T T R with
//    R = [c s; -s c] acting on two neighbouring coordinates.
//  * Eigenvectors: inverse iteration with the shifted tridiagonal matrix,
//    factored with partial pivoting; each vector is scaled so that
//    v^T v = 1 (the bilinear form, not the Hermitian one), so Q^T Q = I for
//    distinct eigenvalues and Q^-1 = Q^T.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace sgi {
namespace csym {

using cd = std::complex<double>;

inline bool finite(cd z) { return std::isfinite(z.real()) && std::isfinite(z.imag()); }

// Eigenvalues of the complex symmetric tridiagonal matrix with diagonal a (n)
// and off-diagonal b (n-1); a is overwritten with them (unsorted).  False if
// the iteration does not converge or a rotation is undefined (x^2 + z^2 = 0
// with x, z nonzero: an isotropic vector, where no complex orthogonal
// rotation exists).
inline bool qr_eigvals(int n, std::vector<cd>& a, std::vector<cd> b) {
  const double eps = 2.220446049250313e-16;
  if (n <= 0) return true;
  b.resize(std::max(n - 1, 1), cd(0.0));
  auto negligible = [&](int k) { return std::abs(b[k]) <= eps * (std::abs(a[k]) + std::abs(a[k + 1])); };
  int q = n - 1;             // the unreduced block being iterated ends at row q
  int sweeps = 0, since = 0;
  while (q > 0) {
    if (negligible(q - 1)) {
      b[q - 1] = 0.0;
      --q;
      since = 0;
      continue;
    }
    int p = q - 1;           // ... and starts at row p
    while (p > 0 && !negligible(p - 1)) --p;
    if (p > 0) b[p - 1] = 0.0;
    if (++sweeps > 60 * n + 60) return false;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer a[q]
    const cd d = 0.5 * (a[q - 1] - a[q]);
    const cd bb = b[q - 1] * b[q - 1];
    const cd root = std::sqrt(d * d + bb);
    const cd den = std::abs(d + root) >= std::abs(d - root) ? d + root : d - root;
    cd mu = std::abs(den) > 0.0 ? a[q] - bb / den : a[q];
    if (++since % 16 == 0) mu = a[q] + cd(0.75, 0.25) * std::abs(b[q - 1]);   // exceptional shift
    // bulge chase: the first rotation comes from the shifted first column,
    // each later one returns the band to tridiagonal form
    cd x = a[p] - mu, z = b[p];
    for (int k = p; k < q; ++k) {
      const cd r = std::sqrt(x * x + z * z);
      if (!(std::abs(r) > 1e-300 * (std::abs(x) + std::abs(z))) && (std::abs(x) + std::abs(z)) > 0.0) return false;
      cd c = 1.0, s = 0.0;
      if (std::abs(x) + std::abs(z) > 0.0) {
        c = x / r;
        s = -z / r;
      }
      if (k > p) b[k - 1] = r;          // the rotated sub-diagonal entry; the bulge below it is now zero
      const cd ak = a[k], ak1 = a[k + 1], e = b[k];
      const cd cc = c * c, ss = s * s, cs = c * s;
      a[k] = cc * ak - 2.0 * cs * e + ss * ak1;
      a[k + 1] = ss * ak + 2.0 * cs * e + cc * ak1;
      b[k] = cs * ak + (cc - ss) * e - cs * ak1;
      if (k + 1 < q) {
        const cd f = b[k + 1];
        x = b[k];
        z = -s * f;                       // new bulge at (k+2, k)
        b[k + 1] = c * f;
      }
    }
  }
  for (int i = 0; i < n; ++i)
    if (!finite(a[i])) return false;
  return true;
}

// Solves (T - mu I) x = v in place for the tridiagonal T (diag, off), with
// partial pivoting between neighbouring rows (the elimination keeps a second
// super-diagonal for the fill a row swap creates).
inline void shifted_solve(int n, const std::vector<cd>& diag, const std::vector<cd>& off, cd mu, std::vector<cd>& v) {
  std::vector<cd> d(n), l(std::max(n - 1, 1)), u1(std::max(n - 1, 1)), u2(std::max(n - 2, 1), cd(0.0));
  std::vector<char> swapped(n, 0);
  for (int i = 0; i < n; ++i) d[i] = diag[i] - mu;
  for (int i = 0; i + 1 < n; ++i) l[i] = u1[i] = off[i];
  for (int i = 0; i + 1 < n; ++i) {
    if (std::abs(d[i]) >= std::abs(l[i])) {
      if (std::abs(d[i]) < 1e-300) d[i] = 1e-300;
      const cd m = l[i] / d[i];
      l[i] = m;
      d[i + 1] -= m * u1[i];
    } else {
      // row i+1 becomes the pivot row
      const cd m = d[i] / l[i];
      const cd piv_row_diag = l[i], piv_row_u1 = d[i + 1];
      const cd old_u1 = u1[i];
      d[i] = piv_row_diag;
      u1[i] = piv_row_u1;
      d[i + 1] = old_u1 - m * piv_row_u1;
      if (i + 2 < n) {
        u2[i] = u1[i + 1];
        u1[i + 1] = -m * u1[i + 1];
      }
      l[i] = m;
      swapped[i] = 1;
    }
  }
  if (std::abs(d[n - 1]) < 1e-250) d[n - 1] = 1e-250;
  for (int i = 0; i + 1 < n; ++i) {
    if (swapped[i]) std::swap(v[i], v[i + 1]);
    v[i + 1] -= l[i] * v[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    cd t = v[i];
    if (i + 1 < n) t -= u1[i] * v[i + 1];
    if (i + 2 < n) t -= u2[i] * v[i + 2];
    v[i] = t / d[i];
  }
}

// Eigenpairs of the complex symmetric tridiagonal matrix (diag, off):
// lam in the order of the real parts of the QR estimates, each refined by
// its eigenvector's Rayleigh quotient; Q row-major n x n with column k the
// eigenvector of lam[k], normalised to v^T v = 1.
//   orth_err  max |(Q^T Q - I)_ab|   (the inverse the preconditioner uses is Q^T)
//   kappa     condition number ||Q||_2 ||Q^-1||_2 = ||Q||_2^2 (Q^-1 = Q^T),
//             estimated from below by 200 power iterations on Q^H Q (within
//             a few per cent when the two largest singular values are close)
// Returns false if an eigenvalue or eigenvector cannot be formed.
inline bool tridiag_eig(int n, const std::vector<cd>& diag, const std::vector<cd>& off, std::vector<cd>& lam,
                        std::vector<cd>& Q, double* orth_err, double* kappa) {
  lam = diag;
  if (!qr_eigvals(n, lam, off)) return false;
  std::sort(lam.begin(), lam.end(), [](cd a, cd b) { return a.real() < b.real(); });
  Q.assign((size_t)n * n, cd(0.0));
  double scale = 0;
  for (int i = 0; i < n; ++i) scale = std::max(scale, std::abs(diag[i]) + 2 * (i < n - 1 ? std::abs(off[i]) : 0));
  std::vector<cd> v(n);
  for (int k = 0; k < n; ++k) {
    const cd mu = lam[k] + cd(1e-13 * scale, 1e-13 * scale);
    for (int i = 0; i < n; ++i) v[i] = cd(1.0 + 0.37 * std::sin(1.7 * i + 0.3 * k), 0.11 * std::cos(0.9 * i));
    for (int it = 0; it < 3; ++it) {
      shifted_solve(n, diag, off, mu, v);
      double m = 0;
      for (int i = 0; i < n; ++i) m = std::max(m, std::abs(v[i]));
      if (!(m > 0) || !std::isfinite(m)) return false;
      for (int i = 0; i < n; ++i) v[i] /= m;
    }
    cd vtv = 0;
    for (int i = 0; i < n; ++i) vtv += v[i] * v[i];
    const cd nrm = std::sqrt(vtv);
    if (std::abs(nrm) < 1e-200) return false;
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + k] = v[i] / nrm;
    // refine the eigenvalue by the bilinear Rayleigh quotient q^T T q
    // (q^T q = 1): the QR sweeps' complex orthogonal rotations are not
    // norm-preserving and leave eigenvalues ~1e-11 off at n ~ 500, while
    // the inverse-iteration vector is accurate to rounding
    cd rq = 0;
    for (int i = 0; i < n; ++i) {
      cd tq = diag[i] * Q[(size_t)i * n + k];
      if (i > 0) tq += off[i - 1] * Q[(size_t)(i - 1) * n + k];
      if (i + 1 < n) tq += off[i] * Q[(size_t)(i + 1) * n + k];
      rq += Q[(size_t)i * n + k] * tq;
    }
    if (finite(rq)) lam[k] = rq;
  }
  double err = 0;
  for (int a = 0; a < n; ++a)
    for (int b = a; b < n; ++b) {
      cd acc = 0;
      for (int i = 0; i < n; ++i) acc += Q[(size_t)i * n + a] * Q[(size_t)i * n + b];
      err = std::max(err, std::abs(acc - (a == b ? 1.0 : 0.0)));
    }
  if (orth_err) *orth_err = err;
  if (kappa) {
    // ||Q||_2^2 = largest eigenvalue of Q^H Q, by power iteration
    std::vector<cd> x(n), y(n), w(n);
    for (int k = 0; k < n; ++k) x[k] = cd(1.0 + 0.5 * std::sin(2.3 * k + 0.7), 0.5 * std::cos(1.3 * k));
    double lamax = 0;
    for (int it = 0; it < 200; ++it) {
      for (int i = 0; i < n; ++i) {
        cd s = 0;
        for (int k = 0; k < n; ++k) s += Q[(size_t)i * n + k] * x[k];
        y[i] = s;
      }
      double nn = 0;
      for (int k = 0; k < n; ++k) {
        cd s = 0;
        for (int i = 0; i < n; ++i) s += std::conj(Q[(size_t)i * n + k]) * y[i];
        w[k] = s;
        nn += std::norm(s);
      }
      double xx = 0;
      for (int k = 0; k < n; ++k) xx += std::norm(x[k]);
      nn = std::sqrt(nn);
      if (!(nn > 0)) break;
      lamax = nn / std::sqrt(xx);
      for (int k = 0; k < n; ++k) x[k] = w[k] / nn;
    }
    *kappa = lamax;
  }
  return true;
}

}  // namespace csym
}  // namespace sgi
