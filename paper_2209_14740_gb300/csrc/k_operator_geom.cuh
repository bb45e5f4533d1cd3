// Per-node FD geometry shared by the SG operator kernels (Appendix A).
#pragma once
#include "sg_internal.h"

namespace sgi {

template <typename T>
__device__ __forceinline__ C2<T> mk(T a, T b) {
  C2<T> r;
  r.x = a;
  r.y = b;
  return r;
}

template <typename T>
struct NodeGeom {
  T w1, w2, wxm, wxp, wym, wyp, ldiag;
  bool hxm, hxp, hym, hyp;  // neighbour present in the unknown grid
};

// FD weights of one unknown (iu, ju): D_2 weight w2 = d_x d_y, D_1 weight
// w1 = 1/h on absorbing boundary nodes, link weights of L (x-links carry d_y,
// y-links carry d_x, Theorem A.6; a Dirichlet side keeps its link to the
// eliminated zero node, Theorems A.1/A.5).
template <typename T>
__device__ __forceinline__ NodeGeom<T> node_geom(const OpParams<T>& p, int iu, int ju) {
  NodeGeom<T> g;
  const bool xlo = iu == 0, xhi = iu == p.mx - 1;
  const bool ylo = ju == 0, yhi = ju == p.my - 1;
  const bool xabs = (xlo && p.absL) || (xhi && p.absR);
  const bool yabs = p.dim == 2 && ((ylo && p.absB) || (yhi && p.absT));
  const T dx = xabs ? T(0.5) : T(1);
  const T dy = yabs ? T(0.5) : T(1);
  g.w2 = dx * dy;
  g.w1 = (xabs || yabs) ? p.inv_h : T(0);
  g.hxm = !xlo;
  g.hxp = !xhi;
  g.wxm = (!xlo || !p.absL) ? dy * p.inv_h2 : T(0);
  g.wxp = (!xhi || !p.absR) ? dy * p.inv_h2 : T(0);
  if (p.dim == 2) {
    g.hym = !ylo;
    g.hyp = !yhi;
    g.wym = (!ylo || !p.absB) ? dx * p.inv_h2 : T(0);
    g.wyp = (!yhi || !p.absT) ? dx * p.inv_h2 : T(0);
  } else {
    g.hym = g.hyp = false;
    g.wym = g.wyp = T(0);
  }
  g.ldiag = g.wxm + g.wxp + g.wym + g.wyp;
  return g;
}

}  // namespace sgi
