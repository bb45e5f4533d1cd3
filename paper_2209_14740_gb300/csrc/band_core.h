// Banded LU with partial row pivoting and its multi-right-hand-side solves:
// the phases each thread of a CTA runs between barriers.  Used by the CUDA
// kernels of k_band.cu (one CTA, phases separated by __syncthreads) and, for
// the index arithmetic, by a CPU test that runs the same phases thread by
// thread on the host.  Within one phase the threads touch disjoint entries.
//
// Storage: the LAPACK band layout (gbtrf): an n x n matrix with kl sub- and
// ku super-diagonals, column-major with leading dimension ldab = 2 kl + ku +
// 1; entry (i, c) at ab[kv + i - c + c * ldab], kv = kl + ku.  The top kl
// rows hold the fill of U that row swaps create (U has kl + ku
// super-diagonals); they start at zero.  After the factorisation, column j
// holds U(j - kv .. j, j) and the multipliers L(j + 1 .. j + kl, j), and
// piv[j] is the row swapped with row j at step j (j <= piv[j] <= j + kl).
//
// Pivots are chosen by the largest |re| + |im| (ties: smallest row).
#pragma once

#if defined(__CUDACC__)
#define BAND_HD __host__ __device__ __forceinline__
#else
#define BAND_HD inline
#endif

namespace sgi {
namespace band {

template <typename C>
BAND_HD C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

BAND_HD long long at(int kv, int ldab, int i, int c) { return (long long)kv + i - c + (long long)c * ldab; }

// ---------------------------------------------------------------- factorisation, step j
// Phase 1 (pivot search), per thread: the best candidate among rows
// j + t, j + t + nt, ... <= last; the CTA then reduces (best, row).
template <typename C>
BAND_HD void pivot_candidates(const C* ab, int kv, int ldab, int j, int last, int t, int nt, double* best, int* row) {
  double bv = -1.0;
  int bi = j;
  for (int i = j + t; i <= last; i += nt) {
    const C a = ab[at(kv, ldab, i, j)];
    const double m = (a.x < 0 ? -a.x : a.x) + (a.y < 0 ? -a.y : a.y);
    if (m > bv) {
      bv = m;
      bi = i;
    }
  }
  *best = bv;
  *row = bi;
}

// Phase 2: swap rows j and p in columns j .. clast.
template <typename C>
BAND_HD void swap_rows(C* ab, int kv, int ldab, int j, int p, int clast, int t, int nt) {
  if (p == j) return;
  for (int c = j + t; c <= clast; c += nt) {
    const long long a = at(kv, ldab, j, c), b = at(kv, ldab, p, c);
    const C v = ab[a];
    ab[a] = ab[b];
    ab[b] = v;
  }
}

// Phase 3: multipliers L(i, j) = A(i, j) / A(j, j) (stored in place and in
// lcol[i - j - 1]) and the row of U (urow[c - j - 1] = A(j, c)).  rinv is
// 1 / A(j, j).
template <typename C>
BAND_HD void multipliers(C* ab, int kv, int ldab, int j, int last, int clast, C rinv, C* lcol, C* urow, int t,
                         int nt) {
  for (int i = j + 1 + t; i <= last; i += nt) {
    const long long a = at(kv, ldab, i, j);
    const C l = cmul(ab[a], rinv);
    ab[a] = l;
    lcol[i - j - 1] = l;
  }
  for (int c = j + 1 + t; c <= clast; c += nt) urow[c - j - 1] = ab[at(kv, ldab, j, c)];
}

// Phase 4: A(i, c) -= L(i, j) U(j, c), i in (j, last], c in (j, clast];
// consecutive threads on consecutive rows of one column (contiguous in the
// band layout).
template <typename C>
BAND_HD void rank1_update(C* ab, int kv, int ldab, int j, int last, int clast, const C* lcol, const C* urow, int t,
                          int nt) {
  const int ni = last - j, nc = clast - j;
  const long long tot = (long long)ni * nc;
  for (long long idx = t; idx < tot; idx += nt) {
    const int ci = (int)(idx / ni), ii = (int)(idx - (long long)ci * ni);
    const long long a = at(kv, ldab, j + 1 + ii, j + 1 + ci);
    const C p = cmul(lcol[ii], urow[ci]);
    ab[a].x -= p.x;
    ab[a].y -= p.y;
  }
}

// ---------------------------------------------------------------- solves
// The right-hand sides are columns of an n x nrhs matrix (column q at
// offset q * ld).  A window of W consecutive rows of the pc right-hand sides
// a CTA owns lives in shared memory, row r in slot r % W, win[slot * pc + q].
// Thread t owns right-hand side q = t % pc and the rows g = t / pc, g + ng,
// ... of an update (ng = nt / pc).

// Forward sweep y = L^-1 P r, step j (window W = kl + 1):
//   (a) swap rows j and piv[j]             [threads t < pc]
//   (b) y_j to Y, rows j+1..j+kl -= L(., j) y_j
//   (c) row j + kl + 1 of R into slot j    [threads t < pc]
template <typename C>
BAND_HD void fwd_swap(C* win, int W, int pc, int j, int p, int t) {
  if (t < pc && p != j) {
    C* a = win + (size_t)(j % W) * pc + t;
    C* b = win + (size_t)(p % W) * pc + t;
    const C v = *a;
    *a = *b;
    *b = v;
  }
}

template <typename C, typename F>
BAND_HD void fwd_update(C* win, int W, int pc, const F* lcol /* L(j+1.., j) */, int j, int n, int kl, int t, int nt,
                        C* Y, long long ld, int q0) {
  const int q = t % pc, g = t / pc, ng = nt / pc;
  if (g >= ng) return;
  const C yj = win[(size_t)(j % W) * pc + q];
  if (g == 0 && Y) Y[(long long)(q0 + q) * ld + j] = yj;
  const int ni = (j + kl < n ? kl : n - 1 - j);
  for (int ii = g; ii < ni; ii += ng) {
    C f;
    f.x = lcol[ii].x;
    f.y = lcol[ii].y;
    C* w = win + (size_t)((j + 1 + ii) % W) * pc + q;
    const C pr = cmul(f, yj);
    w->x -= pr.x;
    w->y -= pr.y;
  }
}

// Backward sweep x = U^-1 y, step j from n - 1 down (window W = kv + 1):
//   x_j = win(j) / U(j, j) to Z, rows j-1..j-kv -= U(., j) x_j; then row
//   j - kv - 1 of Y into slot j.
// col: band column j as stored (col[kv - c] = U(j - c, j), col[kv] =
// U(j, j)); dinv = 1 / U(j, j).
template <typename C, typename F>
BAND_HD void bwd_update(C* win, int W, int pc, const F* col, F dinv, int j, int kv, int t, int nt, C* Z, long long ld,
                        int q0) {
  const int q = t % pc, g = t / pc, ng = nt / pc;
  if (g >= ng) return;
  C di;
  di.x = dinv.x;
  di.y = dinv.y;
  const C xj = cmul(win[(size_t)(j % W) * pc + q], di);
  if (g == 0) Z[(long long)(q0 + q) * ld + j] = xj;
  const int nc = j < kv ? j : kv;
  for (int c = 1 + g; c <= nc; c += ng) {
    C f;
    f.x = col[kv - c].x;
    f.y = col[kv - c].y;
    C* w = win + (size_t)((j - c) % W) * pc + q;
    const C pr = cmul(f, xj);
    w->x -= pr.x;
    w->y -= pr.y;
  }
}

}  // namespace band
}  // namespace sgi
