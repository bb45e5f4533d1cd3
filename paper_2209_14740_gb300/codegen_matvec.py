"""Generates register-resident complex64 SG matvec kernels for fixed (s, r).

The generated kernel computes the same operator as the table-driven kernel
in csrc/k_operator.cu (Theorem 3.4 with Theorems A.1/A.2/A.5/A.6):

    (A X)_a(x) = (L X_a)(x) + sum_b M_ab(x) X_b(x),
    M(x) = -i w1 <k phi phi> - w2 <k^2 phi phi>,  k = k_0 + sum_l xi_l k_l,

but with the chaos structure unrolled at compile time.  The default kernels
(gen_kernel_tk) factor the coupling through degree r + 1,
<k phi phi> = T_k and <k^2 phi phi> = T_k^T T_k, which cuts the arithmetic
of the per-term form (gen_kernel_tile, kept for comparison).  Common to
both:

* one thread per (grid unknown, real/imaginary component): it keeps its
  component of all P modes in registers, so X is read from HBM once and in
  fully coalesced 128-byte warp transactions (adjacent threads read the
  re/im words of adjacent unknowns);
* the real part of M couples only equal components; each row a is the
  diagonal moment plus, per coupling term t, c_t(x) times a short
  compile-time-weighted sum of the neighbours of alpha_a (alpha +- e_l,
  alpha +- 2 e_l, alpha +- e_l +- e_l');
* the imaginary part of M, -w1 (k_0 I + sum_l k_l G_l), lives on absorbing
  boundary nodes only: each thread forms that row for its own component and
  swaps it with its partner lane (shfl.xor 1), only in warps that hold a
  boundary node.

Galerkin constants: orthonormal Legendre recurrence b_n = n/sqrt(4n^2-1),
<xi p_a p_b> = b_max(a,b) for |a-b| = 1, <xi^2 p_a p_a> = b_a^2 + b_{a+1}^2,
<xi^2 p_a p_{a+2}> = b_{a+1} b_{a+2} (Sec. 2.3 basis, Lemma 3.2 products).
Multi-index order: graded, descending lexicographic within a degree (the
order the C ABI documents).
"""
from __future__ import annotations

import math
import os

# (s, r) chaos sizes that get a specialised kernel
SPECIALISED = [(1, 5), (2, 2), (2, 3), (3, 2), (3, 3), (4, 2), (4, 3), (6, 3)]
BLOCK = 128          # threads per CTA (64 unknowns)
OPAQUE = False       # per-row opaque zero in the products (blocks cross-row merging)
MINBLOCKS = 0        # __launch_bounds__ min blocks per SM (0 = none)
STENCIL = "tile"     # "tile": 2D tile staged in shared memory; "split": coupling then stencil loop; "inline"
SERIAL = True        # rows evaluated one after another (bounded register pressure)
ROWS_PER_FENCE = 4   # tile mode: rows between register fences
COUPLING = "tk"      # tile mode: "tk" = factorised through degree r + 1, "direct" = one product per term
PERSISTENT = True    # complex64 "tk" kernels: persistent CTAs, next tile copied during the coupling
# persistent kernels with at least this many modes emit the rows of degree
# <= r twice (with and without the boundary exchange) so interior warps run
# them without branches, and issue the next tile's copies right after the
# last row that reads shared memory; smaller P keeps one copy of the rows and
# issues the copies at the first row of degree r + 1 (fewer registers, more
# CTAs; measured faster at P = 20)
BND_SPLIT_MIN_P = 56
# persistent kernels with at least BND_SPLIT_MIN_P modes copy whole unknowns
# (8 bytes) and keep the wavenumber fields, and up to DBUF_MAX_K of the modes
# read last (the highest, in graded order), in two shared buffers, so that
# those copies of the next tile go out at the start of this one; the other
# modes are copied once the rows that read them are done.  Measured at
# P = 84: 56 double-buffered modes made the kernel slower (0.150 against
# 0.129 ms; the 231 KB carve-out leaves ~28 KB of L1 to the cp.async.ca
# copies), so none are.
DBUF = True
DBUF_MAX_K = 0
SMEM_LIMIT = 227 * 1024   # dynamic shared memory per CTA (opt-in maximum)
# FP64 kernels are generated for P up to this (two registers per value: the
# mode values and accumulators of larger P do not fit)
F64_MAX_P = 35
# larger P: mode values in shared memory, accumulators in two parts; 16 x 4
# unknowns per CTA keep P (tile + halo) FP64 values under the shared limit
F64_HALVES_TILE = (16, 4)

# Unknowns per CTA in x and y for 2D grids (two threads each).  Swept on GB300
# over 16x4, 16x8, 32x4, 8x16, 32x8, 16x16, 64x4 and 32x16 for P = 10 ... 84:
# 16x8 was fastest for every P (its halo is 37.5 % of the tile, 16x4's 62.5 %).
TILE_2D = (16, 8)


# Persistent complex64 kernels: swept on GB300 over 16x4, 32x4, 16x8 and 8x8
# at P = 84 and P = 20; 32x4 was fastest or level (P = 84: 134 us against
# 138 us for 16x8).
PTILE_2D = (32, 4)


def tile_2d(P):
    return TILE_2D


def _multi_indices(s, r):
    out = []

    def rec(prefix, left, slots):
        if slots == 1:
            out.append(tuple(prefix + [left]))
            return
        for a in range(left, -1, -1):
            rec(prefix + [a], left - a, slots - 1)

    for d in range(r + 1):
        rec([], d, s)
    return out


def _b(n):
    return 0.0 if n <= 0 else n / math.sqrt(4.0 * n * n - 1.0)


def _f(v):
    return "%.9ef" % v


def gen_kernel(s, r):
    al = _multi_indices(s, r)
    P = len(al)
    idx = {a: i for i, a in enumerate(al)}
    name = "k_mv_s%dr%d" % (s, r)
    L = []
    w = L.append
    lb = "%d, %d" % (BLOCK, MINBLOCKS) if MINBLOCKS else "%d" % BLOCK
    w("__global__ void __launch_bounds__(%s) %s(OpParams<float> p, const float* __restrict__ X, "
      "float* __restrict__ Y) {" % (lb, name))
    w("  if (p.skip && *p.skip) return;")
    w("  const int c = threadIdx.x & 1;")
    w("  const int u0 = blockIdx.x * %d + (threadIdx.x >> 1);" % (BLOCK // 2))
    w("  const bool valid = u0 < p.n;")
    w("  const int u = valid ? u0 : p.n - 1;")
    w("  const long long n2 = 2ll * p.n;")
    w("  const float* __restrict__ xp = X + 2ll * u + c;")
    w("  float* __restrict__ yp = Y + 2ll * u + c;")
    w("  const int iu = u % p.mx, ju = u / p.mx;")
    w("  const NodeGeom<float> g = node_geom<float>(p, iu, ju);")
    if STENCIL == "smem_first":
        # Phase 0: Laplacian neighbours of every mode into shared memory (a
        # streaming loop with many loads in flight, few registers).
        w("  __shared__ float lap[%d * %d];" % (P, BLOCK))
        w("  {")
        w("    const float wxm0 = g.hxm ? g.wxm : 0.0f, wxp0 = g.hxp ? g.wxp : 0.0f;")
        w("    const float wym0 = g.hym ? g.wym : 0.0f, wyp0 = g.hyp ? g.wyp : 0.0f;")
        w("    const long long oy0 = 2ll * p.mx;")
        w("#pragma unroll 6")
        w("    for (int a = 0; a < %d; ++a) {" % P)
        w("      const float* q = xp + a * n2;")
        w("      float t = 0.0f;")
        w("      if (g.hxm) t = fmaf(-wxm0, q[-2], t);")
        w("      if (g.hxp) t = fmaf(-wxp0, q[2], t);")
        w("      if (g.hym) t = fmaf(-wym0, q[-oy0], t);")
        w("      if (g.hyp) t = fmaf(-wyp0, q[oy0], t);")
        w("      lap[a * %d + threadIdx.x] = t;" % BLOCK)
        w("    }")
        w("  }")
    for a in range(P):
        w("  const float x%d = __ldg(xp + %d * n2);" % (a, a))
    w("  const float k0 = __ldg(p.fields + u);")
    for l in range(s):
        w("  const float k%d = __ldg(p.fields + (long long)%d * p.n + u);" % (l + 1, l + 1))
    # coefficient registers (real parts)
    w("  const float w2 = g.w2;")
    for l in range(s):
        w("  const float cl%d = -2.0f * w2 * k0 * k%d;" % (l + 1, l + 1))
        w("  const float cq%d = -w2 * k%d * k%d;" % (l + 1, l + 1, l + 1))
    for l in range(s):
        for lp in range(l + 1, s):
            w("  const float cp%d_%d = -2.0f * w2 * k%d * k%d;" % (l + 1, lp + 1, l + 1, lp + 1))
    # diagonal base: ldiag - w2 k0^2 + sum_l cq_l * gd(0)
    gd0 = _b(1) ** 2
    base = "g.ldiag - w2 * k0 * k0"
    for l in range(s):
        base += " + cq%d * %s" % (l + 1, _f(gd0))
    w("  const float dbase = %s;" % base)
    w("  const bool bnd = __any_sync(0xffffffffu, g.w1 != 0.0f);")
    w("  const float sw1 = c ? -g.w1 : g.w1;")
    w("  const float wxm = g.hxm ? g.wxm : 0.0f, wxp = g.hxp ? g.wxp : 0.0f;")
    w("  const float wym = g.hym ? g.wym : 0.0f, wyp = g.hyp ? g.wyp : 0.0f;")
    w("  const long long ox = 2, oy = 2ll * p.mx;")
    w("  const float* xq = X + 2ll * u + c;   // plain loads: ordered by the per-row barrier")
    for a, alpha in enumerate(al):
        if STENCIL == "inline":
            # compiler barrier: keeps each row's neighbour loads inside the row
            # (otherwise they are hoisted to the top and the kernel spills)
            w("  asm volatile(\"\" ::: \"memory\");")
        w("  {  // row %d, alpha = %s" % (a, alpha))
        # diagonal
        w("    const float z = %s;" % ("opaque_zero()" if (OPAQUE or SERIAL) else "0.0f"))
        if SERIAL:
            w("    float y = fmaf(dbase, x%d, z);" % a)
        else:
            w("    float y = dbase * x%d;" % a)
        if STENCIL == "smem_first":
            # the address depends on the row's opaque zero, so the load stays in its row
            w("    y += lap[%d * %d + threadIdx.x + __float_as_int(z)];" % (a, BLOCK))
        for l in range(s):
            if alpha[l] > 0:
                gd = _b(alpha[l]) ** 2 + _b(alpha[l] + 1) ** 2
                w("    y = fmaf(cq%d, fmaf(%s, x%d, z), y);" % (l + 1, _f(gd - gd0), a))
        # G_l terms: alpha +- e_l
        k1terms = []   # for the boundary K1 row: (gval, b)
        for l in range(s):
            parts = []
            for sg in (+1, -1):
                beta = list(alpha)
                beta[l] += sg
                beta = tuple(beta)
                if beta in idx:
                    gv = _b(max(alpha[l], beta[l]))
                    parts.append((gv, idx[beta]))
            k1terms.append((l, parts))
            if len(parts) == 1:
                w("    y = fmaf(cl%d, fmaf(%s, x%d, z), y);" % (l + 1, _f(parts[0][0]), parts[0][1]))
            elif len(parts) == 2:
                w("    y = fmaf(cl%d, fmaf(%s, x%d, fmaf(%s, x%d, z)), y);" % (l + 1, _f(parts[0][0]), parts[0][1],
                                                                      _f(parts[1][0]), parts[1][1]))
        # G_ll off-diagonal: alpha +- 2 e_l
        for l in range(s):
            parts = []
            for sg in (+2, -2):
                beta = list(alpha)
                beta[l] += sg
                beta = tuple(beta)
                if beta in idx:
                    m = min(alpha[l], beta[l])
                    parts.append((_b(m + 1) * _b(m + 2), idx[beta]))
            if len(parts) == 1:
                w("    y = fmaf(cq%d, fmaf(%s, x%d, z), y);" % (l + 1, _f(parts[0][0]), parts[0][1]))
            elif len(parts) == 2:
                w("    y = fmaf(cq%d, fmaf(%s, x%d, fmaf(%s, x%d, z)), y);" % (l + 1, _f(parts[0][0]), parts[0][1],
                                                                      _f(parts[1][0]), parts[1][1]))
        # G_ll' (l < l'): alpha +- e_l +- e_l'
        for l in range(s):
            for lp in range(l + 1, s):
                parts = []
                for s1 in (+1, -1):
                    for s2 in (+1, -1):
                        beta = list(alpha)
                        beta[l] += s1
                        beta[lp] += s2
                        beta = tuple(beta)
                        if beta in idx:
                            gv = _b(max(alpha[l], beta[l])) * _b(max(alpha[lp], beta[lp]))
                            parts.append((gv, idx[beta]))
                if not parts:
                    continue
                if len(parts) == 1:
                    w("    y = fmaf(cp%d_%d, fmaf(%s, x%d, z), y);" % (l + 1, lp + 1, _f(parts[0][0]), parts[0][1]))
                else:
                    t = "fmaf(%s, x%d, z)" % (_f(parts[0][0]), parts[0][1])
                    for gv, bb in parts[1:]:
                        t = "fmaf(%s, x%d, %s)" % (_f(gv), bb, t)
                    w("    y = fmaf(cp%d_%d, %s, y);" % (l + 1, lp + 1, t))
        if STENCIL == "inline":
            # Laplacian neighbours (same component of mode a)
            w("    {")
            w("      const float* q = xq + %d * n2;" % a)
            w("      if (g.hxm) y = fmaf(-wxm, q[-ox], y);")
            w("      if (g.hxp) y = fmaf(-wxp, q[ox], y);")
            w("      if (g.hym) y = fmaf(-wym, q[-oy], y);")
            w("      if (g.hyp) y = fmaf(-wyp, q[oy], y);")
            w("    }")
        # boundary: imaginary part of M (-w1 K1), exchanged with the partner component
        t = "k0 * x%d" % a
        for l, parts in k1terms:
            for gv, bb in parts:
                t = "fmaf(k%d, fmaf(%s, x%d, z), %s)" % (l + 1, _f(gv), bb, t)
        w("    if (bnd) {")
        w("      const float tk = %s;" % t)
        w("      y = fmaf(sw1, __shfl_xor_sync(0xffffffffu, tk, 1), y);")
        w("    }")
        if SERIAL:
            # row end marker: the row is complete before the next row's opaque
            # start value is produced, so rows are evaluated one after another
            w("    asm volatile(\"\" : \"+f\"(y));")
        w("    if (valid) yp[%d * n2] = y;" % a)
        w("  }")
    if STENCIL == "split":
        # Second phase: the Laplacian neighbours of every mode, after the
        # registers holding X are dead.  A runtime loop keeps several rows'
        # loads in flight; the row results of the first phase are re-read from
        # L1/L2 (written by this thread just before).
        w("  if (!valid) return;")
        w("  const float* q = X + 2ll * u + c;")
        w("#pragma unroll 4")
        w("  for (int a = 0; a < %d; ++a) {" % P)
        w("    const long long o = a * n2;")
        w("    float y = yp[o];")
        w("    if (g.hxm) y = fmaf(-wxm, q[o - ox], y);")
        w("    if (g.hxp) y = fmaf(-wxp, q[o + ox], y);")
        w("    if (g.hym) y = fmaf(-wym, q[o - oy], y);")
        w("    if (g.hyp) y = fmaf(-wyp, q[o + oy], y);")
        w("    yp[o] = y;")
        w("  }")
    w("}")
    return name, P, "\n".join(L)


def gen_kernel_tile(s, r):
    """Tiled variant: the CTA owns TX x TY grid unknowns (two threads each,
    one per component).  Each thread loads its component of all P modes once
    (all loads in flight together), publishes them to shared memory, the CTA
    loads the one-node halo of the tile, and after one barrier every row takes
    its four stencil neighbours from shared memory.  Rows are evaluated one
    after another (row-start opaque zero, row-end register fence), which
    bounds the live registers to the P mode values plus the coefficients."""
    al = _multi_indices(s, r)
    P = len(al)
    idx = {a: i for i, a in enumerate(al)}
    name = "k_mvt_s%dr%d" % (s, r)
    L = []
    w = L.append
    w("template <int TX, int TY>")
    w("__global__ void __launch_bounds__(2 * TX * TY) %s(OpParams<float> p, const float* __restrict__ X, "
      "float* __restrict__ Y) {" % name)
    w("  constexpr int NT = 2 * TX * TY;            // threads = (unknown, component) pairs")
    w("  constexpr int NH = 2 * (2 * TX + 2 * TY);  // halo entries per mode")
    w("  constexpr int ST = NT + NH;                // shared-memory row stride per mode")
    w("  extern __shared__ float xs[];              // [P][ST]: tile values, then halo values")
    w("  if (p.skip && *p.skip) return;")
    w("  const int t = threadIdx.x, c = t & 1, nid = t >> 1;")
    w("  const int lx = nid % TX, ly = nid / TX;")
    w("  const int iu0 = blockIdx.x * TX + lx, ju0 = blockIdx.y * TY + ly;")
    w("  const bool valid = iu0 < p.mx && ju0 < p.my;")
    w("  const int iu = min(iu0, p.mx - 1), ju = min(ju0, p.my - 1);")
    w("  const int u = iu + p.mx * ju;")
    w("  const long long n2 = 2ll * p.n;")
    w("  const float* __restrict__ xp = X + 2ll * u + c;")
    for a in range(P):
        w("  float x%d = __ldg(xp + %d * n2);" % (a, a))
    # halo: top row (ly=-1), bottom row (ly=TY), left col (lx=-1), right col (lx=TX)
    # the whole halo is loaded in one batch (all loads in flight together),
    # then written to shared memory
    w("  {")
    w("    constexpr int HALO_PER_THREAD = (%d * NH + NT - 1) / NT;" % P)
    w("    const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;")
    w("    float hv[HALO_PER_THREAD];")
    w("#pragma unroll")
    w("    for (int i = 0; i < HALO_PER_THREAD; ++i) {")
    w("      const int k = t + i * NT;")
    w("      const int a = k / NH, e = k - a * NH, hc = e & 1, h = e >> 1;")
    w("      int hx, hy;")
    w("      if (h < TX) { hx = bx0 + h; hy = by0 - 1; }")
    w("      else if (h < 2 * TX) { hx = bx0 + h - TX; hy = by0 + TY; }")
    w("      else if (h < 2 * TX + TY) { hx = bx0 - 1; hy = by0 + h - 2 * TX; }")
    w("      else { hx = bx0 + TX; hy = by0 + h - 2 * TX - TY; }")
    w("      hv[i] = 0.0f;")
    w("      if (k < %d * NH && hx >= 0 && hx < p.mx && hy >= 0 && hy < p.my)" % P)
    w("        hv[i] = __ldg(X + (long long)a * n2 + 2ll * (hx + (long long)p.mx * hy) + hc);")
    w("    }")
    w("#pragma unroll")
    w("    for (int i = 0; i < HALO_PER_THREAD; ++i) {")
    w("      const int k = t + i * NT;")
    w("      if (k < %d * NH) {" % P)
    w("        const int a = k / NH, e = k - a * NH;")
    w("        xs[a * ST + NT + e] = hv[i];")
    w("      }")
    w("    }")
    w("  }")
    for a in range(P):
        w("  xs[%d * ST + t] = x%d;" % (a, a))
    w("  const NodeGeom<float> g = node_geom<float>(p, iu, ju);")
    # neighbour offsets inside a mode row of xs
    w("  const int oxm = lx > 0 ? t - 2 : NT + 2 * (2 * TX + ly) + c;")
    w("  const int oxp = lx < TX - 1 ? t + 2 : NT + 2 * (2 * TX + TY + ly) + c;")
    w("  const int oym = ly > 0 ? t - 2 * TX : NT + 2 * lx + c;")
    w("  const int oyp = ly < TY - 1 ? t + 2 * TX : NT + 2 * (TX + lx) + c;")
    w("  const float wxm = g.hxm ? g.wxm : 0.0f, wxp = g.hxp ? g.wxp : 0.0f;")
    w("  const float wym = g.hym ? g.wym : 0.0f, wyp = g.hyp ? g.wyp : 0.0f;")
    w("  const float k0 = __ldg(p.fields + u);")
    for l in range(s):
        w("  const float k%d = __ldg(p.fields + (long long)%d * p.n + u);" % (l + 1, l + 1))
    w("  const float w2 = g.w2;")
    for l in range(s):
        w("  const float cl%d = -2.0f * w2 * k0 * k%d;" % (l + 1, l + 1))
        w("  const float cq%d = -w2 * k%d * k%d;" % (l + 1, l + 1, l + 1))
    for l in range(s):
        for lp in range(l + 1, s):
            w("  const float cp%d_%d = -2.0f * w2 * k%d * k%d;" % (l + 1, lp + 1, l + 1, lp + 1))
    gd0 = _b(1) ** 2
    base = "g.ldiag - w2 * k0 * k0"
    for l in range(s):
        base += " + cq%d * %s" % (l + 1, _f(gd0))
    w("  const float dbase = %s;" % base)
    w("  const bool bnd = __any_sync(0xffffffffu, g.w1 != 0.0f);")
    w("  const float sw1 = c ? -g.w1 : g.w1;")
    w("  float* __restrict__ yp = Y + 2ll * u + c;")
    w("  __syncthreads();")

    def fence():
        # Empty asm that "redefines" every mode register and clobbers memory:
        # nothing computed from X or shared memory moves across it, so at most
        # ROWS_PER_FENCE rows are in flight and the live registers stay the
        # P mode values plus the coefficients.  It emits no instruction.
        for i0 in range(0, P, 28):
            ops = ", ".join('"+f"(x%d)' % i for i in range(i0, min(P, i0 + 28)))
            w('  asm volatile("" : %s :: "memory");' % ops)

    for a, alpha in enumerate(al):
        if a % ROWS_PER_FENCE == 0:
            fence()
        w("  {  // row %d, alpha = %s" % (a, alpha))
        w("    float y = dbase * x%d;" % a)
        w("    {")
        w("      const float* q = xs + %d * ST;" % a)
        w("      y = fmaf(-wxm, q[oxm], y);")
        w("      y = fmaf(-wxp, q[oxp], y);")
        w("      y = fmaf(-wym, q[oym], y);")
        w("      y = fmaf(-wyp, q[oyp], y);")
        w("    }")
        for l in range(s):
            if alpha[l] > 0:
                gd = _b(alpha[l]) ** 2 + _b(alpha[l] + 1) ** 2
                w("    y = fmaf(cq%d, %s * x%d, y);" % (l + 1, _f(gd - gd0), a))
        k1terms = []

        def group(coef, parts):
            if not parts:
                return
            t = "%s * x%d" % (_f(parts[0][0]), parts[0][1])
            for gv, bb in parts[1:]:
                t = "fmaf(%s, x%d, %s)" % (_f(gv), bb, t)
            w("    y = fmaf(%s, %s, y);" % (coef, t))

        for l in range(s):
            parts = []
            for sg in (+1, -1):
                beta = list(alpha)
                beta[l] += sg
                beta = tuple(beta)
                if beta in idx:
                    parts.append((_b(max(alpha[l], beta[l])), idx[beta]))
            k1terms.append((l, parts))
            group("cl%d" % (l + 1), parts)
        for l in range(s):
            parts = []
            for sg in (+2, -2):
                beta = list(alpha)
                beta[l] += sg
                beta = tuple(beta)
                if beta in idx:
                    m = min(alpha[l], beta[l])
                    parts.append((_b(m + 1) * _b(m + 2), idx[beta]))
            group("cq%d" % (l + 1), parts)
        for l in range(s):
            for lp in range(l + 1, s):
                parts = []
                for s1 in (+1, -1):
                    for s2 in (+1, -1):
                        beta = list(alpha)
                        beta[l] += s1
                        beta[lp] += s2
                        beta = tuple(beta)
                        if beta in idx:
                            parts.append((_b(max(alpha[l], beta[l])) * _b(max(alpha[lp], beta[lp])), idx[beta]))
                group("cp%d_%d" % (l + 1, lp + 1), parts)
        t = "k0 * x%d" % a
        for l, parts in k1terms:
            for gv, bb in parts:
                t = "fmaf(k%d, %s * x%d, %s)" % (l + 1, _f(gv), bb, t)
        w("    if (bnd) {")
        w("      const float tk = %s;" % t)
        w("      y = fmaf(sw1, __shfl_xor_sync(0xffffffffu, tk, 1), y);")
        w("    }")
        w("    if (valid) yp[%d * n2] = y;" % a)
        w("  }")
    w("}")
    return name, P, "\n".join(L)


def _tk_rows(s, r):
    """Rows of the factorised coupling in graded order: for every g of degree
    <= r + 1 the entries T_k[g][b] (coefficient name, b) with b = g, g - e_l,
    g + e_l in degree <= r.  The scatter of T_k^T touches the same entries:
    Z_a += T_k[g][a] W_g."""
    al = _multi_indices(s, r)
    ext = _multi_indices(s, r + 1)
    idx = {a: i for i, a in enumerate(al)}
    rows = []
    for gm in ext:
        terms = []
        if gm in idx:
            terms.append(("k0", idx[gm]))
        for l in range(s):
            if gm[l] >= 1:
                lo = list(gm)
                lo[l] -= 1
                terms.append(("kb%d_%d" % (l + 1, gm[l]), idx[tuple(lo)]))
            hi = list(gm)
            hi[l] += 1
            if tuple(hi) in idx:
                terms.append(("kb%d_%d" % (l + 1, gm[l] + 1), idx[tuple(hi)]))
        if terms:
            rows.append((gm, terms))
    return idx, rows


def _emit_tk_coupling(w, s, r, finish, hook=None, first_x=None, first_z=None):
    """Z += -w2 T_k^T T_k X (and -i w1 (T_k X) on absorbing boundary nodes,
    exchanged with the partner lane) in registers, one W_g at a time.  In
    graded order X_b is dead after the last W_g that reads it and Z_a is
    complete after the last W_g scattered into it; finish(a) is emitted right
    then, so only the values of about two degrees are live at a time.
    hook(), if given, is emitted before the first row of degree r + 1 (where
    the fewest values are live); first_x(b) and first_z(a), if given, before
    the first row that reads X_b or updates Z_a (all of degree <= r, so
    before the hook).""" 
    idx, rows = _tk_rows(s, r)
    P = len(idx)
    last_x = {}
    last_z = {}
    for ri, (gm, terms) in enumerate(rows):
        for _, b in terms:
            last_x[b] = ri
            last_z[b] = ri
    done_at = {}
    for a in range(P):
        done_at.setdefault(last_z[a], []).append(a)

    seen = set()

    def fence(ri):
        # values declared so far (all of them when first_x is not used) that
        # are still to be read
        live = [b for b in range(P) if last_x.get(b, -1) >= ri and (first_x is None or b in seen)]
        for i0 in range(0, len(live), 28):
            ops = ", ".join('"+f"(x%d)' % i for i in live[i0:i0 + 28])
            w('  asm volatile("" : %s :: "memory");' % ops)

    first_top = min(ri for ri, (gm, _) in enumerate(rows) if sum(gm) == r + 1)
    for ri, (gm, terms) in enumerate(rows):
        if ri == first_top and hook:
            fence(ri)
            hook()
        for _, b in terms:
            if b not in seen:
                assert ri < first_top
                seen.add(b)
                if first_x:
                    first_x(b)
                if first_z:
                    first_z(b)
        if ri % (2 * ROWS_PER_FENCE) == 0:
            fence(ri)
        e = "%s * x%d" % (terms[0][0], terms[0][1])
        for cf, b in terms[1:]:
            e = "fmaf(%s, x%d, %s)" % (cf, b, e)
        w("  {  // g = %s" % (gm,))
        w("    float wv = %s;" % e)
        if gm in idx:
            w("    if (bnd) z%d = fmaf(sw1, __shfl_xor_sync(0xffffffffu, wv, 1), z%d);" % (idx[gm], idx[gm]))
        w("    wv *= nw2;")
        for cf, a in terms:
            w("    z%d = fmaf(%s, wv, z%d);" % (a, cf, a))
        w("  }")
        for a in done_at.get(ri, []):
            finish(a)


def gen_kernel_tk(s, r, prec="f32"):
    """Tiled variant with the coupling factorised through degree r + 1.

    With K = sum_l k_l xi_l and k = k_0 + K, the Galerkin moments are
    <k phi_a phi_b> = (T_k)_{ab} and <k^2 phi_a phi_b> = (T_k^T T_k)_{ab},
    where T_k maps the degree <= r coefficients to degree <= r + 1:
        (T_k X)_g = k_0 X_g + sum_l k_l (b_{g_l} X_{g - e_l} + b_{g_l + 1} X_{g + e_l})
    (the three-term recurrence of the orthonormal Legendre polynomials; terms
    outside degree <= r are absent).  This is exact: k phi_b lies in degree
    <= r + 1, so the inner product over that space is the full expectation.
    Each thread (one component of one unknown) forms W_g = (T_k X)_g for every
    g of degree <= r + 1 and scatters -w2 T_k^T W into its P accumulators
    straight away, so only X, the accumulators and one W value are live.  The
    imaginary part, -i w1 (T_k X)_a, exists on absorbing boundary nodes only
    and is exchanged with the partner lane there.  Then
        Y_a = ldiag X_a - sum_nb w_nb X_a(nb) + Z_a.
    The arithmetic per unknown is about 2 |T_k| + 6 P instead of one product
    per coupling nonzero and term."""
    al = _multi_indices(s, r)
    ext = _multi_indices(s, r + 1)
    P = len(al)
    idx = {a: i for i, a in enumerate(al)}
    name = ("k_mvk_s%dr%d" if prec == "f32" else "k_mvk64_s%dr%d") % (s, r)
    lit = _f if prec == "f32" else (lambda v: "%.17e" % v)
    L = []
    w = L.append

    def xv(a):
        return "x%d" % a

    w("template <int TX, int TY>")
    w("__global__ void __launch_bounds__(2 * TX * TY) %s(OpParams<float> p, const float* __restrict__ X, "
      "float* __restrict__ Y) {" % name)
    w("  constexpr int NT = 2 * TX * TY;            // threads = (unknown, component) pairs")
    w("  constexpr int NH = 2 * (2 * TX + 2 * TY);  // halo entries per mode")
    w("  constexpr int ST = NT + NH;                // shared-memory row stride per mode")
    w("  extern __shared__ float xs[];              // [P][ST]: tile values, then halo values")
    w("  if (p.skip && *p.skip) return;")
    w("  const int t = threadIdx.x, c = t & 1, nid = t >> 1;")
    w("  const int lx = nid % TX, ly = nid / TX;")
    w("  const int iu0 = blockIdx.x * TX + lx, ju0 = blockIdx.y * TY + ly;")
    w("  const bool valid = iu0 < p.mx && ju0 < p.my;")
    w("  const int iu = min(iu0, p.mx - 1), ju = min(ju0, p.my - 1);")
    w("  const int u = iu + p.mx * ju;")
    w("  const long long n2 = 2ll * p.n;")
    w("  const float* __restrict__ xp = X + 2ll * u + c;")
    for a in range(P):
        w("  float x%d = __ldg(xp + %d * n2);" % (a, a))
    w("  {")
    w("    constexpr int HALO_PER_THREAD = (%d * NH + NT - 1) / NT;" % P)
    w("    const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;")
    w("    float hv[HALO_PER_THREAD];")
    w("#pragma unroll")
    w("    for (int i = 0; i < HALO_PER_THREAD; ++i) {")
    w("      const int k = t + i * NT;")
    w("      const int a = k / NH, e = k - a * NH, hc = e & 1, h = e >> 1;")
    w("      int hx, hy;")
    w("      if (h < TX) { hx = bx0 + h; hy = by0 - 1; }")
    w("      else if (h < 2 * TX) { hx = bx0 + h - TX; hy = by0 + TY; }")
    w("      else if (h < 2 * TX + TY) { hx = bx0 - 1; hy = by0 + h - 2 * TX; }")
    w("      else { hx = bx0 + TX; hy = by0 + h - 2 * TX - TY; }")
    w("      hv[i] = 0.0f;")
    w("      if (k < %d * NH && hx >= 0 && hx < p.mx && hy >= 0 && hy < p.my)" % P)
    w("        hv[i] = __ldg(X + (long long)a * n2 + 2ll * (hx + (long long)p.mx * hy) + hc);")
    w("    }")
    w("#pragma unroll")
    w("    for (int i = 0; i < HALO_PER_THREAD; ++i) {")
    w("      const int k = t + i * NT;")
    w("      if (k < %d * NH) {" % P)
    w("        const int a = k / NH, e = k - a * NH;")
    w("        xs[a * ST + NT + e] = hv[i];")
    w("      }")
    w("    }")
    w("  }")
    for a in range(P):
        w("  xs[%d * ST + t] = x%d;" % (a, a))
    w("  const NodeGeom<float> g = node_geom<float>(p, iu, ju);")
    w("  const int oxm = lx > 0 ? t - 2 : NT + 2 * (2 * TX + ly) + c;")
    w("  const int oxp = lx < TX - 1 ? t + 2 : NT + 2 * (2 * TX + TY + ly) + c;")
    w("  const int oym = ly > 0 ? t - 2 * TX : NT + 2 * lx + c;")
    w("  const int oyp = ly < TY - 1 ? t + 2 * TX : NT + 2 * (TX + lx) + c;")
    w("  const float wxm = g.hxm ? g.wxm : 0.0f, wxp = g.hxp ? g.wxp : 0.0f;")
    w("  const float wym = g.hym ? g.wym : 0.0f, wyp = g.hyp ? g.wyp : 0.0f;")
    w("  const float k0 = __ldg(p.fields + u);")
    for l in range(s):
        w("  const float k%d = __ldg(p.fields + (long long)%d * p.n + u);" % (l + 1, l + 1))
    w("  const float nw2 = -g.w2;")
    # kb[l][n] = k_l * b_n, n = 1 .. r + 1
    for l in range(s):
        for n in range(1, r + 2):
            w("  const float kb%d_%d = k%d * %s;" % (l + 1, n, l + 1, lit(_b(n))))
    w("  const bool bnd = __any_sync(0xffffffffu, g.w1 != 0.0f);")
    w("  const float sw1 = c ? -g.w1 : g.w1;   // -i w1 W: re gets +w1 Im W, im gets -w1 Re W")
    for a in range(P):
        w("  float z%d = 0.0f;" % a)
    w("  float* __restrict__ yp = Y + 2ll * u + c;")
    w("  __syncthreads();")

    def finish(a):
        w("  {")
        w("    const float* q = xs + %d * ST;" % a)
        w("    float y = fmaf(g.ldiag, q[t], z%d);" % a)
        w("    y = fmaf(-wxm, q[oxm], y);")
        w("    y = fmaf(-wxp, q[oxp], y);")
        w("    y = fmaf(-wym, q[oym], y);")
        w("    y = fmaf(-wyp, q[oyp], y);")
        w("    if (valid) yp[%d * n2] = y;" % a)
        w("  }")

    _emit_tk_coupling(w, s, r, finish)
    w("}")
    src = "\n".join(L)
    if prec == "f64":
        # the same kernel on complex128 data: FP64 registers, shared memory
        # and arithmetic (the Legendre constants are printed to 17 digits)
        for a_, b_ in (("float", "double"), ("fmaf(", "fma("), ("0.0f", "0.0"), ('"+f"', '"+d"')):
            src = src.replace(a_, b_)
        # one extern shared array per element type in a translation unit
        src = src.replace("  extern __shared__ double xs[];",
                          "  extern __shared__ __align__(16) unsigned char xs64_raw[];\n"
                          "  double* xs = reinterpret_cast<double*>(xs64_raw);")
    return name, P, src


def _emit_tk_rows(w, s, r, rows, lo, hi, finish, bnd, first_x=None, first_z=None, declared=()):
    """Rows lo .. hi - 1 of the factorised coupling for the persistent kernel,
    on mode values already scaled by -w2 (so W'_g = -w2 W_g and the scatter
    needs no extra product).  bnd: emit the -i w1 W exchange with the partner
    lane (warps holding an absorbing boundary node) unconditionally (True),
    behind the warp-uniform flag ("branch") or not at all (False).  first_x(b) and
    first_z(a) are emitted before the first row that reads X_b or updates
    Z_a; `declared` lists the values that exist before row lo."""
    idx, _ = _tk_rows(s, r)
    P = len(idx)
    last_x = {}
    last_z = {}
    for ri, (gm, terms) in enumerate(rows):
        for _, b in terms:
            last_x[b] = ri
            last_z[b] = ri
    seen = set(declared)

    def fence(ri):
        live = [b for b in range(P) if last_x.get(b, -1) >= ri and b in seen]
        for i0 in range(0, len(live), 28):
            ops = ", ".join('"+f"(x%d)' % i for i in live[i0:i0 + 28])
            w('    asm volatile("" : %s :: "memory");' % ops)

    for ri in range(lo, hi):
        gm, terms = rows[ri]
        if (ri - lo) % (2 * ROWS_PER_FENCE) == 0:
            fence(ri)
        for _, b in terms:
            if b not in seen:
                seen.add(b)
                first_x(b)
                first_z(b)
        e = "%s * x%d" % (terms[0][0], terms[0][1])
        for cf, b in terms[1:]:
            e = "fmaf(%s, x%d, %s)" % (cf, b, e)
        w("    {  // g = %s" % (gm,))
        w("      const float wv = %s;" % e)
        if bnd == "branch" and gm in idx:
            w("      if (bnd) z%d = fmaf(sw1, __shfl_xor_sync(0xffffffffu, wv, 1), z%d);" % (idx[gm], idx[gm]))
        elif bnd and gm in idx:
            w("      z%d = fmaf(sw1, __shfl_xor_sync(0xffffffffu, wv, 1), z%d);" % (idx[gm], idx[gm]))
        for cf, a in terms:
            w("      z%d = fmaf(%s, wv, z%d);" % (a, cf, a))
        w("    }")
        for a in range(P):
            if last_z[a] == ri:
                finish(a)
    return seen


def dbuf_modes(s, r):
    """Number of double-buffered modes of the persistent kernel for (s, r):
    None for the single-buffer form (gen_kernel_tkp), else K >= 0 for
    _gen_kernel_tkp_dbuf, at most DBUF_MAX_K and as many as the shared-memory
    limit allows for both tile shapes (with two buffers of the s+1
    wavenumber fields)."""
    P = len(_multi_indices(s, r))
    if not (PERSISTENT and DBUF) or P < BND_SPLIT_MIN_P:
        return None
    k = min(P, DBUF_MAX_K)
    for tx, ty in (PTILE_2D, (64, 1)):
        nt = 2 * tx * ty
        st = nt + 2 * (2 * tx + 2 * ty)
        k = min(k, (SMEM_LIMIT // 4 - 2 * (s + 1) * (nt // 2)) // st - P)
    return max(k, 0)


def gen_kernel_tkp(s, r):
    """Persistent form of the factorised complex64 kernel (gen_kernel_tk):
    each CTA walks tiles of TX x TY unknowns with a stride of the grid size,
    and the copies of the next tile overlap the coupling of this one:

      wait for this tile's copies -> Z_a = ldiag X_a - sum_nb w_nb X_a(nb)
      straight from shared memory (X_a into registers, each just before its
      first use) -> coupling rows up to the last one that reads shared memory
      -> barrier -> issue the cp.async copies of the next tile's values and
      halo into the same shared rows -> the remaining rows -> Y_a = Z_a as
      each completes.

    The stencil reads every shared value before the barrier, so one buffer
    serves both tiles, and the CTA's single set of P accumulators (the
    register file holds one CTA of 256 threads at P = 84) is no longer idle
    while its next tile is in flight."""
    idx, _ = _tk_rows(s, r)
    P = len(idx)
    K = dbuf_modes(s, r)
    if K is not None:
        return _gen_kernel_tkp_dbuf(s, r, K)
    name = "k_mvkp_s%dr%d" % (s, r)
    L = []
    w = L.append
    w("template <int TX, int TY>")
    w("__global__ void __launch_bounds__(2 * TX * TY) %s(OpParams<float> p, const float* __restrict__ X, "
      "float* __restrict__ Y) {" % name)
    w("  constexpr int NT = 2 * TX * TY;            // threads = (unknown, component) pairs")
    w("  constexpr int NH = 2 * (2 * TX + 2 * TY);  // halo entries per mode")
    w("  constexpr int ST = NT + NH;                // shared-memory row stride per mode")
    w("  constexpr int FS = %d * ST;                // then the %d wavenumber fields of the tile's unknowns" % (P, s + 1))
    w("  extern __shared__ float xs[];              // [P][ST]: tile values, then halo values; [s+1][NT/2] fields")
    w("  if (p.skip && *p.skip) return;")
    w("  const int t = threadIdx.x, c = t & 1, nid = t >> 1;")
    w("  const int lx = nid % TX, ly = nid / TX;")
    w("  const int tiles_x = (p.mx + TX - 1) / TX;")
    w("  const int tiles = tiles_x * ((p.my + TY - 1) / TY);")
    w("  const long long n2 = 2ll * p.n;")
    w("  const uint32_t xs0 = (uint32_t)__cvta_generic_to_shared(xs);")
    w("  const int oxm = lx > 0 ? t - 2 : NT + 2 * (2 * TX + ly) + c;")
    w("  const int oxp = lx < TX - 1 ? t + 2 : NT + 2 * (2 * TX + TY + ly) + c;")
    w("  const int oym = ly > 0 ? t - 2 * TX : NT + 2 * lx + c;")
    w("  const int oyp = ly < TY - 1 ? t + 2 * TX : NT + 2 * (TX + lx) + c;")
    w("  // copies of one tile's values (this thread's unknown, every mode) and of")
    w("  // its halo (with NT >= NH thread t < HG * NH owns halo slot t % NH of")
    w("  // every HG-th mode); halo entries outside the grid are zero-filled")
    w("  constexpr int HG = NT >= NH ? NT / NH : 1;")
    w("  auto issue = [&](int tile) {")
    w("    const int bx0 = (tile % tiles_x) * TX, by0 = (tile / tiles_x) * TY;")
    w("    {")
    w("      const int iu = min(bx0 + lx, p.mx - 1), ju = min(by0 + ly, p.my - 1);")
    w("      const float* src = X + 2ll * (iu + (long long)p.mx * ju) + c;")
    w("      uint32_t dst = xs0 + 4u * t;")
    w("#pragma unroll 4")
    w("      for (int a = 0; a < %d; ++a, src += n2, dst += 4u * ST) mv_cp_async4(dst, src, 4);" % P)
    w("      // the (s+1) wavenumber fields k_0 .. k_s of the unknown (one thread of the pair)")
    w("      if (c == 0) {")
    w("        const float* fsrc = p.fields + iu + (long long)p.mx * ju;")
    w("        uint32_t fdst = xs0 + 4u * (FS + nid);")
    w("#pragma unroll")
    w("        for (int l = 0; l <= %d; ++l, fsrc += p.n, fdst += 4u * (NT / 2)) mv_cp_async4(fdst, fsrc, 4);" % s)
    w("      }")
    w("    }")
    w("    // halo slot e of modes a0, a0 + hg, ...")
    w("    auto halo = [&](int e, int a0, int hg) {")
    w("      const int hc = e & 1, h = e >> 1;")
    w("      int hx, hy;")
    w("      if (h < TX) { hx = bx0 + h; hy = by0 - 1; }")
    w("      else if (h < 2 * TX) { hx = bx0 + h - TX; hy = by0 + TY; }")
    w("      else if (h < 2 * TX + TY) { hx = bx0 - 1; hy = by0 + h - 2 * TX; }")
    w("      else { hx = bx0 + TX; hy = by0 + h - 2 * TX - TY; }")
    w("      const bool ok = hx >= 0 && hx < p.mx && hy >= 0 && hy < p.my;")
    w("      const float* src = ok ? X + (long long)a0 * n2 + 2ll * (hx + (long long)p.mx * hy) + hc : X;")
    w("      const long long step = ok ? hg * n2 : 0;")
    w("      uint32_t dst = xs0 + 4u * (a0 * ST + NT + e);")
    w("#pragma unroll 4")
    w("      for (int a = a0; a < %d; a += hg, src += step, dst += 4u * hg * ST) mv_cp_async4(dst, src, ok ? 4 : 0);" % P)
    w("    };")
    w("    if (NT >= NH) {")
    w("      if (t < HG * NH) halo(t % NH, t / NH, HG);")
    w("    } else {")
    w("      for (int e = t; e < NH; e += NT) halo(e, 0, 1);")
    w("    }")
    w('    asm volatile("cp.async.commit_group;" ::: "memory");')
    w("  };")
    w("  int tile = blockIdx.x;")
    w("  if (tile < tiles) issue(tile);")
    w("  for (; tile < tiles; tile += gridDim.x) {")
    w("    const int iu0 = (tile % tiles_x) * TX + lx, ju0 = (tile / tiles_x) * TY + ly;")
    w("    const bool valid = iu0 < p.mx && ju0 < p.my;")
    w("    const int iu = min(iu0, p.mx - 1), ju = min(ju0, p.my - 1);")
    w("    const int u = iu + p.mx * ju;")
    w("    const NodeGeom<float> g = node_geom<float>(p, iu, ju);")
    w("    const float wxm = g.hxm ? g.wxm : 0.0f, wxp = g.hxp ? g.wxp : 0.0f;")
    w("    const float wym = g.hym ? g.wym : 0.0f, wyp = g.hyp ? g.wyp : 0.0f;")
    w("    // mode values in registers are scaled by -w2 (a power of two: exact),")
    w("    // so the diagonal and boundary weights applied to them take the")
    w("    // inverse factor; the neighbours come unscaled from shared memory")
    w("    const float nw2 = -g.w2, inw2 = -1.0f / g.w2;")
    w("    const float ldg2 = g.ldiag * inw2;")
    w("    const bool bnd = __any_sync(0xffffffffu, g.w1 != 0.0f);")
    w("    const float sw1 = (c ? -g.w1 : g.w1) * inw2;   // -i w1 W: re gets +w1 Im W, im gets -w1 Re W")
    w("    float* __restrict__ yp = Y + 2ll * u + c;")
    w('    asm volatile("cp.async.wait_all;" ::: "memory");')
    w("    __syncthreads();")
    w("    const float k0 = xs[FS + nid];")
    for l in range(s):
        w("    const float k%d = xs[FS + %d * (NT / 2) + nid];" % (l + 1, l + 1))
    for l in range(s):
        for n in range(1, r + 2):
            w("    const float kb%d_%d = k%d * %s;" % (l + 1, n, l + 1, _f(_b(n))))
    w("    float %s;" % ", ".join("x%d" % a for a in range(P)))
    w("    float %s;" % ", ".join("z%d" % a for a in range(P)))

    # mode values into registers (scaled), and the stencil part of each output
    # straight from shared memory, just before their first use
    def first_x(b):
        w("    x%d = nw2 * xs[%d * ST + t];" % (b, b))

    def first_z(a):
        w("    z%d = fmaf(ldg2, x%d, fmaf(-wxm, xs[%d * ST + oxm], fmaf(-wxp, xs[%d * ST + oxp], "
          "fmaf(-wym, xs[%d * ST + oym], -wyp * xs[%d * ST + oyp]))));" % (a, a, a, a, a, a))

    def finish(a):
        w("    if (valid) yp[%d * n2] = z%d;" % (a, a))

    idx_, rows = _tk_rows(s, r)
    top = min(ri for ri, (gm, _) in enumerate(rows) if sum(gm) == r + 1)
    # the next tile's copies go out right after the last row that reads
    # shared memory (the first use of a mode value or of an output's stencil)
    seen = set()
    hook = 0
    for ri, (gm, terms) in enumerate(rows):
        for _, b in terms:
            if b not in seen:
                seen.add(b)
                hook = ri + 1
    assert hook <= top
    if P < BND_SPLIT_MIN_P:
        # measured: small P is faster with the copies issued at the first row
        # of degree r + 1 (fewer registers while they are issued)
        hook = top
    # rows of degree <= r: warps holding an absorbing boundary node exchange
    # -i w1 W with the partner lane; the others run the same rows without
    # (two regions, so the barrier before the copies stays outside branches)
    def region(lo, hi, declared=()):
        if hi <= lo:
            return set(declared)
        if P >= BND_SPLIT_MIN_P:
            w("    if (bnd) {")
            d = _emit_tk_rows(w, s, r, rows, lo, hi, finish, True, first_x, first_z, declared)
            w("    } else {")
            _emit_tk_rows(w, s, r, rows, lo, hi, finish, False, first_x, first_z, declared)
            w("    }")
            return d
        return _emit_tk_rows(w, s, r, rows, lo, hi, finish, "branch", first_x, first_z, declared)
    declared = region(0, hook)
    w("    __syncthreads();   // every shared value of this tile has been read")
    w("    if (tile + (int)gridDim.x < tiles) issue(tile + gridDim.x);")
    declared = region(hook, top, declared)
    # rows of degree r + 1 (no output of their own: no exchange)
    _emit_tk_rows(w, s, r, rows, top, len(rows), finish, False, declared=declared)
    w("  }")
    w("}")
    return name, P, "\n".join(L)


def _gen_kernel_tkp_dbuf(s, r, K):
    """gen_kernel_tkp with the modes P0 = P - K .. P - 1 and the wavenumber
    fields in two shared buffers (tile parity q):

      wait for this tile's copies -> copy the next tile's modes P0.. and
      fields into the other buffer -> rows up to the last one that reads a
      mode < P0 from shared memory -> barrier -> copy the next tile's modes
      < P0 -> the remaining rows.

    In graded order the modes < P0 are the low degrees, which the first rows
    already read in full, so the single-buffered copies go out after a few
    rows and the double-buffered ones a whole tile ahead.  Same arithmetic,
    in the same order, as the single-buffer form."""
    idx, rows = _tk_rows(s, r)
    P = len(idx)
    P0 = P - K
    name = "k_mvkp_s%dr%d" % (s, r)
    L = []
    w = L.append
    w("template <int TX, int TY>")
    w("__global__ void __launch_bounds__(2 * TX * TY) %s(OpParams<float> p, const float* __restrict__ X, "
      "float* __restrict__ Y) {" % name)
    w("  constexpr int NT = 2 * TX * TY;            // threads = (unknown, component) pairs")
    w("  constexpr int NN = NT / 2;                 // unknowns of a tile")
    w("  constexpr int NH = 2 * (2 * TX + 2 * TY);  // halo entries per mode")
    w("  constexpr int NHN = NH / 2;                // halo unknowns")
    w("  constexpr int ST = NT + NH;                // shared-memory row stride per mode")
    w("  constexpr int P0 = %d;                     // modes 0 .. P0-1: one buffer" % P0)
    if K:
        w("  constexpr int K = %d;                      // modes P0 .. %d: two buffers of K rows" % (K, P - 1))
    else:
        w("  constexpr int K = 0;                       // (no double-buffered modes)")
    w("  constexpr int NF = %d;                     // wavenumber fields k_0 .. k_s" % (s + 1))
    if K:
        w("  constexpr int FS = (P0 + 2 * K) * ST;      // then two buffers of [NF][NN] fields")
        w("  // [P0][ST] | [2][K][ST] | [2][NF][NN]; a mode row holds the tile's values")
    else:
        w("  constexpr int FS = P0 * ST;                // then the [NF][NN] fields")
        w("  // [P][ST] | [NF][NN]; a mode row holds the tile's values")
    w("  // (unknown-major, re/im adjacent), then the halo's")
    w("  extern __shared__ __align__(16) float xs[];")
    w("  if (p.skip && *p.skip) return;")
    w("  const int t = threadIdx.x, c = t & 1, nid = t >> 1;")
    w("  const int lx = nid % TX, ly = nid / TX;")
    w("  const int tiles_x = (p.mx + TX - 1) / TX;")
    w("  const int tiles = tiles_x * ((p.my + TY - 1) / TY);")
    w("  const long long n2 = 2ll * p.n;")
    w("  const uint32_t xs0 = (uint32_t)__cvta_generic_to_shared(xs);")
    w("  const int oxm = lx > 0 ? t - 2 : NT + 2 * (2 * TX + ly) + c;")
    w("  const int oxp = lx < TX - 1 ? t + 2 : NT + 2 * (2 * TX + TY + ly) + c;")
    w("  const int oym = ly > 0 ? t - 2 * TX : NT + 2 * lx + c;")
    w("  const int oyp = ly < TY - 1 ? t + 2 * TX : NT + 2 * (TX + lx) + c;")
    w("  // 8-byte copies of modes a_lo .. a_hi - 1 of one tile into the rows")
    w("  // starting at shared byte address base (row a_lo first): thread t copies")
    w("  // unknown t % NN of every other mode, and (NT >= NHN) halo unknown")
    w("  // t % NHN of every HG-th mode; halo unknowns outside the grid are")
    w("  // zero-filled, tile unknowns outside it repeat the last row or column")
    w("  auto copy_modes = [&](int tile, int a_lo, int a_hi, uint32_t base) {")
    w("    const int bx0 = (tile % tiles_x) * TX, by0 = (tile / tiles_x) * TY;")
    w("    {")
    w("      const int nd = t % NN, a0 = t / NN;")
    w("      const int iu = min(bx0 + nd % TX, p.mx - 1), ju = min(by0 + nd / TX, p.my - 1);")
    w("      const float* src = X + (long long)(a_lo + a0) * n2 + 2ll * (iu + (long long)p.mx * ju);")
    w("      uint32_t dst = base + 4u * (a0 * ST + 2 * nd);")
    w("#pragma unroll 4")
    w("      for (int a = a_lo + a0; a < a_hi; a += 2, src += 2 * n2, dst += 8u * ST) mv_cp_async8(dst, src, 8);")
    w("    }")
    w("    auto halo = [&](int hn, int a0, int hg) {")
    w("      int hx, hy;")
    w("      if (hn < TX) { hx = bx0 + hn; hy = by0 - 1; }")
    w("      else if (hn < 2 * TX) { hx = bx0 + hn - TX; hy = by0 + TY; }")
    w("      else if (hn < 2 * TX + TY) { hx = bx0 - 1; hy = by0 + hn - 2 * TX; }")
    w("      else { hx = bx0 + TX; hy = by0 + hn - 2 * TX - TY; }")
    w("      const bool ok = hx >= 0 && hx < p.mx && hy >= 0 && hy < p.my;")
    w("      const float* src = ok ? X + (long long)a0 * n2 + 2ll * (hx + (long long)p.mx * hy) : X;")
    w("      const long long step = ok ? hg * n2 : 0;")
    w("      uint32_t dst = base + 4u * ((a0 - a_lo) * ST + NT + 2 * hn);")
    w("#pragma unroll 4")
    w("      for (int a = a0; a < a_hi; a += hg, src += step, dst += 4u * hg * ST) mv_cp_async8(dst, src, ok ? 8 : 0);")
    w("    };")
    w("    constexpr int HG = NT >= NHN ? NT / NHN : 0;")
    w("    if (HG > 0) {")
    w("      if (t < HG * NHN) halo(t % NHN, a_lo + t / NHN, HG);")
    w("    } else {")
    w("      for (int hn = t; hn < NHN; hn += NT) halo(hn, a_lo, 1);")
    w("    }")
    w("  };")
    # the s+1 wavenumber fields of the tile's unknowns (one thread of each pair)
    def emit_fields(dst_expr):
        w("    if (c == 0) {")
        w("      const int bx0 = (tile % tiles_x) * TX, by0 = (tile / tiles_x) * TY;")
        w("      const int iu = min(bx0 + lx, p.mx - 1), ju = min(by0 + ly, p.my - 1);")
        w("      const float* fsrc = p.fields + iu + (long long)p.mx * ju;")
        w("      uint32_t fdst = xs0 + 4u * (%s + nid);" % dst_expr)
        w("#pragma unroll")
        w("      for (int l = 0; l < NF; ++l, fsrc += p.n, fdst += 4u * NN) mv_cp_async4(fdst, fsrc, 4);")
        w("    }")
    if K:
        w("  // modes P0.. and the fields of a tile into buffer q")
        w("  auto issue_early = [&](int tile, int q) {")
        w("    copy_modes(tile, P0, P0 + K, xs0 + 4u * ((P0 + q * K) * ST));")
        emit_fields("FS + q * NF * NN")
        w('    asm volatile("cp.async.commit_group;" ::: "memory");')
        w("  };")
        w("  // modes 0 .. P0-1 of a tile (single buffer)")
    else:
        w("  // all modes and the fields of a tile")
    w("  auto issue_late = [&](int tile) {")
    w("    copy_modes(tile, 0, P0, xs0);")
    if not K:
        emit_fields("FS")
    w('    asm volatile("cp.async.commit_group;" ::: "memory");')
    w("  };")
    if K:
        w("  int tile = blockIdx.x, q = 0;")
        w("  if (tile < tiles) {")
        w("    issue_early(tile, 0);")
        w("    issue_late(tile);")
        w("  }")
        w("  for (; tile < tiles; tile += gridDim.x, q ^= 1) {")
    else:
        w("  int tile = blockIdx.x;")
        w("  if (tile < tiles) issue_late(tile);")
        w("  for (; tile < tiles; tile += gridDim.x) {")
    w("    const int iu0 = (tile % tiles_x) * TX + lx, ju0 = (tile / tiles_x) * TY + ly;")
    w("    const bool valid = iu0 < p.mx && ju0 < p.my;")
    w("    const int iu = min(iu0, p.mx - 1), ju = min(ju0, p.my - 1);")
    w("    const int u = iu + p.mx * ju;")
    w("    const NodeGeom<float> g = node_geom<float>(p, iu, ju);")
    w("    const float wxm = g.hxm ? g.wxm : 0.0f, wxp = g.hxp ? g.wxp : 0.0f;")
    w("    const float wym = g.hym ? g.wym : 0.0f, wyp = g.hyp ? g.wyp : 0.0f;")
    w("    // mode values in registers are scaled by -w2 (a power of two: exact),")
    w("    // so the diagonal and boundary weights applied to them take the")
    w("    // inverse factor; the neighbours come unscaled from shared memory")
    w("    const float nw2 = -g.w2, inw2 = -1.0f / g.w2;")
    w("    const float ldg2 = g.ldiag * inw2;")
    w("    const bool bnd = __any_sync(0xffffffffu, g.w1 != 0.0f);")
    w("    const float sw1 = (c ? -g.w1 : g.w1) * inw2;   // -i w1 W: re gets +w1 Im W, im gets -w1 Re W")
    w("    float* __restrict__ yp = Y + 2ll * u + c;")
    w('    asm volatile("cp.async.wait_all;" ::: "memory");')
    w("    __syncthreads();")
    if K:
        w("    // every read of the other buffer (the previous tile's) is done")
        w("    if (tile + (int)gridDim.x < tiles) issue_early(tile + gridDim.x, q ^ 1);")
        w("    const float* __restrict__ xq = xs + q * (K * ST);   // xq[a * ST + ..]: mode a >= P0")
        w("    const float* __restrict__ fq = xs + FS + q * (NF * NN);")
    else:
        w("    const float* __restrict__ fq = xs + FS;")
    w("    const float k0 = fq[nid];")
    for l in range(s):
        w("    const float k%d = fq[%d * NN + nid];" % (l + 1, l + 1))
    for l in range(s):
        for n in range(1, r + 2):
            w("    const float kb%d_%d = k%d * %s;" % (l + 1, n, l + 1, _f(_b(n))))
    w("    float %s;" % ", ".join("x%d" % a for a in range(P)))
    w("    float %s;" % ", ".join("z%d" % a for a in range(P)))

    def arr(b):
        return "xs" if b < P0 else "xq"

    def first_x(b):
        w("    x%d = nw2 * %s[%d * ST + t];" % (b, arr(b), b))

    def first_z(a):
        m = arr(a)
        w("    z%d = fmaf(ldg2, x%d, fmaf(-wxm, %s[%d * ST + oxm], fmaf(-wxp, %s[%d * ST + oxp], "
          "fmaf(-wym, %s[%d * ST + oym], -wyp * %s[%d * ST + oyp]))));" % (a, a, m, a, m, a, m, a, m, a))

    def finish(a):
        w("    if (valid) yp[%d * n2] = z%d;" % (a, a))

    top = min(ri for ri, (gm, _) in enumerate(rows) if sum(gm) == r + 1)
    # the single-buffered copies go out right after the last row that reads a
    # mode < P0 from shared memory (its first use or its output's stencil)
    seen = set()
    hook = 0
    for ri, (gm, terms) in enumerate(rows):
        for _, b in terms:
            if b not in seen:
                seen.add(b)
                if b < P0:
                    hook = ri + 1
    assert hook <= top

    def region(lo, hi, declared=()):
        if hi <= lo:
            return set(declared)
        w("    if (bnd) {")
        d = _emit_tk_rows(w, s, r, rows, lo, hi, finish, True, first_x, first_z, declared)
        w("    } else {")
        _emit_tk_rows(w, s, r, rows, lo, hi, finish, False, first_x, first_z, declared)
        w("    }")
        return d
    declared = region(0, hook)
    w("    __syncthreads();   // every shared value of modes < P0 has been read")
    w("    if (tile + (int)gridDim.x < tiles) issue_late(tile + gridDim.x);")
    declared = region(hook, top, declared)
    _emit_tk_rows(w, s, r, rows, top, len(rows), finish, False, declared=declared)
    w("  }")
    w("}")
    return name, P, "\n".join(L)


def gen_kernel_tk64_halves(s, r, halves=3):
    """FP64 factorised kernel for chaos sizes whose FP64 mode values and
    accumulators do not fit in registers together.  The tile and its halo are
    copied to shared memory by cp.async (no registers held in flight); the
    accumulators are built for one part of the modes at a time, each part
    recomputing the W_g it needs from shared memory.  Same arithmetic as
    gen_kernel_tk otherwise (see there)."""
    al = _multi_indices(s, r)
    ext = _multi_indices(s, r + 1)
    P = len(al)
    idx = {a: i for i, a in enumerate(al)}
    name = "k_mvk64h_s%dr%d" % (s, r)
    lit = lambda v: "%.17e" % v
    L = []
    w = L.append
    w("template <int TX, int TY>")
    w("__global__ void __launch_bounds__(2 * TX * TY) %s(OpParams<double> p, const double* __restrict__ X, "
      "double* __restrict__ Y) {" % name)
    w("  constexpr int NT = 2 * TX * TY;")
    w("  constexpr int NH = 2 * (2 * TX + 2 * TY);")
    w("  constexpr int ST = NT + NH;")
    w("  extern __shared__ __align__(16) unsigned char xs64h_raw[];")
    w("  double* xs = reinterpret_cast<double*>(xs64h_raw);   // [P][ST]")
    w("  if (p.skip && *p.skip) return;")
    w("  const int t = threadIdx.x, c = t & 1, nid = t >> 1;")
    w("  const int lx = nid % TX, ly = nid / TX;")
    w("  const int iu0 = blockIdx.x * TX + lx, ju0 = blockIdx.y * TY + ly;")
    w("  const bool valid = iu0 < p.mx && ju0 < p.my;")
    w("  const int iu = min(iu0, p.mx - 1), ju = min(ju0, p.my - 1);")
    w("  const int u = iu + p.mx * ju;")
    w("  const long long n2 = 2ll * p.n;")
    w("  const double* __restrict__ xp = X + 2ll * u + c;")
    w("  {")
    w("    const unsigned xs0 = (unsigned)__cvta_generic_to_shared(xs);")
    w("    for (int a = 0; a < %d; ++a)" % P)
    w('      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(xs0 + 8u * (a * ST + t)), '
      '"l"(xp + a * n2) : "memory");')
    w("    const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;")
    w("    for (int k = t; k < %d * NH; k += NT) {" % P)
    w("      const int a = k / NH, e = k - a * NH, hc = e & 1, h = e >> 1;")
    w("      int hx, hy;")
    w("      if (h < TX) { hx = bx0 + h; hy = by0 - 1; }")
    w("      else if (h < 2 * TX) { hx = bx0 + h - TX; hy = by0 + TY; }")
    w("      else if (h < 2 * TX + TY) { hx = bx0 - 1; hy = by0 + h - 2 * TX; }")
    w("      else { hx = bx0 + TX; hy = by0 + h - 2 * TX - TY; }")
    w("      const bool in = hx >= 0 && hx < p.mx && hy >= 0 && hy < p.my;")
    w("      const double* src = in ? X + (long long)a * n2 + 2ll * (hx + (long long)p.mx * hy) + hc : X;")
    w('      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(xs0 + 8u * (a * ST + NT + e)), '
      '"l"(src), "r"(in ? 8 : 0) : "memory");')
    w("    }")
    w('    asm volatile("cp.async.wait_all;" ::: "memory");')
    w("  }")
    w("  const NodeGeom<double> g = node_geom<double>(p, iu, ju);")
    w("  const int oxm = lx > 0 ? t - 2 : NT + 2 * (2 * TX + ly) + c;")
    w("  const int oxp = lx < TX - 1 ? t + 2 : NT + 2 * (2 * TX + TY + ly) + c;")
    w("  const int oym = ly > 0 ? t - 2 * TX : NT + 2 * lx + c;")
    w("  const int oyp = ly < TY - 1 ? t + 2 * TX : NT + 2 * (TX + lx) + c;")
    w("  const double wxm = g.hxm ? g.wxm : 0.0, wxp = g.hxp ? g.wxp : 0.0;")
    w("  const double wym = g.hym ? g.wym : 0.0, wyp = g.hyp ? g.wyp : 0.0;")
    w("  const double k0 = __ldg(p.fields + u);")
    for l in range(s):
        w("  const double k%d = __ldg(p.fields + (long long)%d * p.n + u);" % (l + 1, l + 1))
    w("  const double nw2 = -g.w2;")
    for l in range(s):
        for n in range(1, r + 2):
            w("  const double kb%d_%d = k%d * %s;" % (l + 1, n, l + 1, lit(_b(n))))
    w("  const bool bnd = __any_sync(0xffffffffu, g.w1 != 0.0);")
    w("  const double sw1 = c ? -g.w1 : g.w1;")
    w("  double* __restrict__ yp = Y + 2ll * u + c;")
    w("  __syncthreads();")

    def xv(a):
        return "xs[%d * ST + t]" % a

    bounds = [round(P * h / halves) for h in range(halves + 1)]
    for hp in range(halves):
        lo_a, hi_a = bounds[hp], bounds[hp + 1]
        part = set(range(lo_a, hi_a))
        w("  {  // modes %d .. %d" % (lo_a, hi_a - 1))
        for a in range(lo_a, hi_a):
            w("    double z%d = 0.0;" % a)
        for gm in ext:
            terms = []
            if gm in idx:
                terms.append(("k0", idx[gm]))
            for l in range(s):
                if gm[l] >= 1:
                    lo = list(gm)
                    lo[l] -= 1
                    terms.append(("kb%d_%d" % (l + 1, gm[l]), idx[tuple(lo)]))
                hi = list(gm)
                hi[l] += 1
                if tuple(hi) in idx:
                    terms.append(("kb%d_%d" % (l + 1, gm[l] + 1), idx[tuple(hi)]))
            # targets of the scatter inside this part
            scat = []
            if gm in idx and idx[gm] in part:
                scat.append(("k0", idx[gm]))
            for l in range(s):
                if gm[l] >= 1:
                    lo = list(gm)
                    lo[l] -= 1
                    if idx[tuple(lo)] in part:
                        scat.append(("kb%d_%d" % (l + 1, gm[l]), idx[tuple(lo)]))
                hi = list(gm)
                hi[l] += 1
                if tuple(hi) in idx and idx[tuple(hi)] in part:
                    scat.append(("kb%d_%d" % (l + 1, gm[l] + 1), idx[tuple(hi)]))
            own = gm in idx and idx[gm] in part
            if not terms or (not scat and not own):
                continue
            e = "%s * %s" % (terms[0][0], xv(terms[0][1]))
            for cf, b in terms[1:]:
                e = "fma(%s, %s, %s)" % (cf, xv(b), e)
            w('    asm volatile("" ::: "memory");')
            w("    {")
            w("      double wv = %s;" % e)
            if own:
                w("      if (bnd) z%d = fma(sw1, __shfl_xor_sync(0xffffffffu, wv, 1), z%d);" % (idx[gm], idx[gm]))
            w("      wv *= nw2;")
            for cf, a in scat:
                w("      z%d = fma(%s, wv, z%d);" % (a, cf, a))
            w("    }")
        w('    asm volatile("" ::: "memory");')
        # running store pointer, opaque to the compiler: the P store addresses
        # are formed one at a time instead of all up front
        w("    double* yq = yp + %d * n2;" % lo_a)
        for a in range(lo_a, hi_a):
            w("    {")
            w("      const double* q = xs + %d * ST;" % a)
            w("      double y = fma(g.ldiag, %s, z%d);" % (xv(a), a))
            w("      y = fma(-wxm, q[oxm], y);")
            w("      y = fma(-wxp, q[oxp], y);")
            w("      y = fma(-wym, q[oym], y);")
            w("      y = fma(-wyp, q[oyp], y);")
            w("      if (valid) *yq = y;")
            w("      yq += n2;")
            w('      asm volatile("" : "+l"(yq));')
            w("    }")
        w("  }")
    w("}")
    return name, P, "\n".join(L)


def gen_kernel_packed(s, r):
    """One thread per grid unknown holding both components (float2) of all P
    modes; the coupling uses packed FP32x2 FMAs (__ffma2_rn: the real
    coefficient acts on re and im at once).  CTAs are 2D tiles (TX x TY
    unknowns), so the stencil's neighbours inside the tile are L1 hits."""
    al = _multi_indices(s, r)
    P = len(al)
    idx = {a: i for i, a in enumerate(al)}
    name = "k_mv2_s%dr%d" % (s, r)
    L = []
    w = L.append

    def f2(v):
        return "make_float2(%s, %s)" % (_f(v), _f(v))

    w("template <int TX, int TY>")
    w("__global__ void __launch_bounds__(TX * TY) %s(OpParams<float> p, const float2* __restrict__ X, "
      "float2* __restrict__ Y) {" % name)
    w("  if (p.skip && *p.skip) return;")
    w("  const int iu0 = blockIdx.x * TX + (int)(threadIdx.x % TX);")
    w("  const int ju0 = blockIdx.y * TY + (int)(threadIdx.x / TX);")
    w("  const bool valid = iu0 < p.mx && ju0 < p.my;")
    w("  const int iu = min(iu0, p.mx - 1), ju = min(ju0, p.my - 1);")
    w("  const int u = iu + p.mx * ju;")
    w("  const long long n = p.n;")
    w("  const float2* __restrict__ xp = X + u;")
    w("  float2* __restrict__ yp = Y + u;")
    for a in range(P):
        w("  const float2 x%d = __ldg(xp + %d * n);" % (a, a))
    w("  const NodeGeom<float> g = node_geom<float>(p, iu, ju);")
    w("  const float k0 = __ldg(p.fields + u);")
    for l in range(s):
        w("  const float k%d = __ldg(p.fields + (long long)%d * p.n + u);" % (l + 1, l + 1))
    w("  const float w2 = g.w2;")
    for l in range(s):
        w("  const float cl%d_ = -2.0f * w2 * k0 * k%d;" % (l + 1, l + 1))
        w("  const float2 cl%d = make_float2(cl%d_, cl%d_);" % (l + 1, l + 1, l + 1))
        w("  const float cq%d_ = -w2 * k%d * k%d;" % (l + 1, l + 1, l + 1))
        w("  const float2 cq%d = make_float2(cq%d_, cq%d_);" % (l + 1, l + 1, l + 1))
    for l in range(s):
        for lp in range(l + 1, s):
            w("  const float cp%d_%d_ = -2.0f * w2 * k%d * k%d;" % (l + 1, lp + 1, l + 1, lp + 1))
            w("  const float2 cp%d_%d = make_float2(cp%d_%d_, cp%d_%d_);" % ((l + 1, lp + 1) * 3))
    gd0 = _b(1) ** 2
    base = "g.ldiag - w2 * k0 * k0"
    for l in range(s):
        base += " + cq%d_ * %s" % (l + 1, _f(gd0))
    w("  const float dbase_ = %s;" % base)
    w("  const float2 dbase = make_float2(dbase_, dbase_);")
    w("  const bool bnd = g.w1 != 0.0f;")
    w("  const float2 mwxm = make_float2(-g.wxm, -g.wxm), mwxp = make_float2(-g.wxp, -g.wxp);")
    w("  const float2 mwym = make_float2(-g.wym, -g.wym), mwyp = make_float2(-g.wyp, -g.wyp);")
    w("  const float2* xq = X + u;   // plain loads, kept inside their row by the barrier")
    for a, alpha in enumerate(al):
        w("  asm volatile(\"\" ::: \"memory\");")
        w("  {  // row %d, alpha = %s" % (a, alpha))
        w("    float2 y = __fmul2_rn(dbase, x%d);" % a)
        for l in range(s):
            if alpha[l] > 0:
                gd = _b(alpha[l]) ** 2 + _b(alpha[l] + 1) ** 2
                w("    y = __ffma2_rn(cq%d, __fmul2_rn(%s, x%d), y);" % (l + 1, f2(gd - gd0), a))
        k1terms = []

        def group(coef, parts):
            if not parts:
                return
            t = "__fmul2_rn(%s, x%d)" % (f2(parts[0][0]), parts[0][1])
            for gv, bb in parts[1:]:
                t = "__ffma2_rn(%s, x%d, %s)" % (f2(gv), bb, t)
            w("    y = __ffma2_rn(%s, %s, y);" % (coef, t))

        for l in range(s):
            parts = []
            for sg in (+1, -1):
                beta = list(alpha)
                beta[l] += sg
                beta = tuple(beta)
                if beta in idx:
                    parts.append((_b(max(alpha[l], beta[l])), idx[beta]))
            k1terms.append((l, parts))
            group("cl%d" % (l + 1), parts)
        for l in range(s):
            parts = []
            for sg in (+2, -2):
                beta = list(alpha)
                beta[l] += sg
                beta = tuple(beta)
                if beta in idx:
                    m = min(alpha[l], beta[l])
                    parts.append((_b(m + 1) * _b(m + 2), idx[beta]))
            group("cq%d" % (l + 1), parts)
        for l in range(s):
            for lp in range(l + 1, s):
                parts = []
                for s1 in (+1, -1):
                    for s2 in (+1, -1):
                        beta = list(alpha)
                        beta[l] += s1
                        beta[lp] += s2
                        beta = tuple(beta)
                        if beta in idx:
                            parts.append((_b(max(alpha[l], beta[l])) * _b(max(alpha[lp], beta[lp])), idx[beta]))
                group("cp%d_%d" % (l + 1, lp + 1), parts)
        w("    {")
        w("      const float2* q = xq + %d * n;" % a)
        w("      if (g.hxm) y = __ffma2_rn(mwxm, q[-1], y);")
        w("      if (g.hxp) y = __ffma2_rn(mwxp, q[1], y);")
        w("      if (g.hym) y = __ffma2_rn(mwym, q[-p.mx], y);")
        w("      if (g.hyp) y = __ffma2_rn(mwyp, q[p.mx], y);")
        w("    }")
        t = "k0 * x%d.x" % a
        ti = "k0 * x%d.y" % a
        for l, parts in k1terms:
            for gv, bb in parts:
                t = "fmaf(k%d * %s, x%d.x, %s)" % (l + 1, _f(gv), bb, t)
                ti = "fmaf(k%d * %s, x%d.y, %s)" % (l + 1, _f(gv), bb, ti)
        w("    if (bnd) {   // -i w1 <k phi phi>: y += w1 * (i^-1 times K1 x) componentwise")
        w("      const float tr = %s;" % t)
        w("      const float ti = %s;" % ti)
        w("      y.x = fmaf(g.w1, ti, y.x);")
        w("      y.y = fmaf(-g.w1, tr, y.y);")
        w("    }")
        w("    if (valid) yp[%d * n] = y;" % a)
        w("  }")
    w("}")
    return name, P, "\n".join(L)


def generate(path: str) -> str:
    parts = ["// GENERATED by paper_2209_14740_gb300/codegen_matvec.py -- do not edit.",
             "#include <cuda_runtime.h>",
             "#include <algorithm>",
             '#include "sg_internal.h"',
             '#include "k_operator_geom.cuh"',
             "namespace sgi {",
             "// A zero the optimiser cannot see through: products fmaf(g, x, z) stay",
             "// local to their row instead of being merged across rows and kept live.",
             "__device__ __forceinline__ float opaque_zero() {",
             "  float z;",
             "  asm volatile(\"mov.b32 %0, 0;\" : \"=f\"(z));",
             "  return z;",
             "}",
             "// 4-byte asynchronous global -> shared copy; bytes = 0 writes a zero",
             "__device__ __forceinline__ void mv_cp_async4(uint32_t dst, const float* src, int bytes) {",
             "  asm volatile(\"cp.async.ca.shared.global [%0], [%1], 4, %2;\" :: \"r\"(dst), \"l\"(src), \"r\"(bytes) : \"memory\");",
             "}",
             "__device__ __forceinline__ void mv_cp_async8(uint32_t dst, const float* src, int bytes) {",
             "  asm volatile(\"cp.async.ca.shared.global [%0], [%1], 8, %2;\" :: \"r\"(dst), \"l\"(src), \"r\"(bytes) : \"memory\");",
             "}"]
    table = []
    table64 = []
    for s, r in SPECIALISED:
        if STENCIL == "tile":
            if COUPLING == "tk":
                name, P, src = gen_kernel_tkp(s, r) if PERSISTENT else gen_kernel_tk(s, r)
            else:
                name, P, src = gen_kernel_tile(s, r)
        else:
            name, P, src = gen_kernel(s, r)
        parts.append(src)
        table.append((s, r, name, P))
        if STENCIL == "tile" and COUPLING == "tk":
            if P <= F64_MAX_P:
                name64, _, src64 = gen_kernel_tk(s, r, "f64")
                table64.append((s, r, name64, P, tile_2d(P)))
            else:
                name64, _, src64 = gen_kernel_tk64_halves(s, r)
                table64.append((s, r, name64, P, F64_HALVES_TILE))
            parts.append(src64)
    if STENCIL == "tile":
        parts += [
            "// Launch of a tiled kernel: 2D problems use 16 x 4 unknowns per CTA,",
            "// 1D problems 64 x 1; dynamic shared memory holds P rows of",
            "// (tile + halo) values.",
            "template <int TX, int TY, typename T>",
            "static cudaError_t launch_tile(void (*kern)(OpParams<T>, const T*, T*), int P,",
            "                               const sg_handle* h, const OpParams<T>& p, const C2<T>* X, C2<T>* Y,",
            "                               cudaStream_t st) {",
            "  const int nt = 2 * TX * TY, nh = 2 * (2 * TX + 2 * TY);",
            "  const size_t smem = (size_t)P * (nt + nh) * sizeof(T);",
            "  if (smem > 48 * 1024) {",
            "    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);",
            "    if (e != cudaSuccess) return e;",
            "  }",
            "  dim3 grid((h->mx + TX - 1) / TX, (h->my + TY - 1) / TY);",
            "  kern<<<grid, nt, smem, st>>>(p, (const T*)X, (T*)Y);",
            "  note_launch();",
            "  return cudaGetLastError();",
            "}",
            "// Shared memory of a persistent kernel's CTA: P rows of (tile + halo)",
            "// values and the tile's wavenumber fields; K > 0: the last K rows and",
            "// the fields twice (double-buffered).",
            "template <int TX, int TY>",
            "static size_t persist_smem(int P, int nfields, int K) {",
            "  const int nt = 2 * TX * TY, nh = 2 * (2 * TX + 2 * TY);",
            "  const int rows = K > 0 ? P + K : P, fbufs = K > 0 ? 2 : 1;",
            "  return ((size_t)rows * (nt + nh) + (size_t)fbufs * nfields * (nt / 2)) * sizeof(float);",
            "}",
            "// CTAs per SM of a persistent kernel (its shared-memory limit raised first);",
            "// each call site keeps the value in a static initialised once (thread-safe).",
            "template <int TX, int TY>",
            "static int persist_occupancy(void (*kern)(OpParams<float>, const float*, float*), int P, int nfields,",
            "                             int K) {",
            "  const size_t smem = persist_smem<TX, TY>(P, nfields, K);",
            "  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);",
            "  int o = 0;",
            "  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, 2 * TX * TY, smem) != cudaSuccess) o = 0;",
            "  return o > 0 ? o : 1;",
            "}",
            "// Launch of a persistent kernel: as many CTAs as fit on the GPU at once",
            "// (at most one per tile); occ = CTAs per SM of this kernel.",
            "template <int TX, int TY>",
            "static cudaError_t launch_persist(void (*kern)(OpParams<float>, const float*, float*), int P, int nfields,",
            "                                  int K, int occ,",
            "                                  const sg_handle* h, const OpParams<float>& p, const float2* X,",
            "                                  float2* Y, cudaStream_t st) {",
            "  const int nt = 2 * TX * TY;",
            "  const size_t smem = persist_smem<TX, TY>(P, nfields, K);",
            "  if (smem > 48 * 1024) {",
            "    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);",
            "    if (e != cudaSuccess) return e;",
            "  }",
            "  const long long tiles = (long long)((h->mx + TX - 1) / TX) * ((h->my + TY - 1) / TY);",
            "  const int grid = (int)std::min<long long>(tiles, (long long)h->num_sms * occ);",
            "  kern<<<grid, nt, smem, st>>>(p, reinterpret_cast<const float*>(X), reinterpret_cast<float*>(Y));",
            "  note_launch();",
            "  return cudaGetLastError();",
            "}",
        ]
    if STENCIL == "tile" and COUPLING == "tk" and PERSISTENT:
        # CTAs per SM of the persistent kernels: the tuner's choice (at most
        # the occupancy), else the occupancy
        parts.append("static int tuned_occ(const sg_handle* h, int occ) {")
        parts.append("  return h->tune_op_occ > 0 ? std::min(h->tune_op_occ, occ) : occ;")
        parts.append("}")
        parts.append("int matvec_special_occupancy(const sg_handle* h) {")
        for s, r, name, P in table:
            tx, ty = PTILE_2D
            K = dbuf_modes(s, r)
            K = -1 if K is None else K
            parts.append("  if (h->s == %d && h->r == %d)" % (s, r))
            parts.append("    return h->dim == 2 ? persist_occupancy<%d, %d>(%s<%d, %d>, %d, %d, %d)"
                         % (tx, ty, name, tx, ty, P, s + 1, K))
            parts.append("                       : persist_occupancy<64, 1>(%s<64, 1>, %d, %d, %d);"
                         % (name, P, s + 1, K))
        parts.append("  return 0;")
        parts.append("}")
    else:
        parts.append("int matvec_special_occupancy(const sg_handle*) { return 0; }")
    parts.append("cudaError_t matvec_special_f32(const sg_handle* h, const float2* X, float2* Y, cudaStream_t st,")
    parts.append("                               const int* skip, bool* handled) {")
    parts.append("  *handled = false;")
    parts.append("  OpParams<float> p = h->op32();")
    parts.append("  p.skip = skip;")
    parts.append("  const int grid = (h->n + %d - 1) / %d;" % (BLOCK // 2, BLOCK // 2))
    parts.append("  (void)grid;")
    for s, r, name, P in table:
        parts.append("  if (h->s == %d && h->r == %d) {" % (s, r))
        parts.append("    *handled = true;")
        if STENCIL == "tile" and COUPLING == "tk" and PERSISTENT:
            tx, ty = PTILE_2D
            K = dbuf_modes(s, r)
            K = -1 if K is None else K
            parts.append("    if (h->dim == 2) {")
            parts.append("      static const int occ2 = persist_occupancy<%d, %d>(%s<%d, %d>, %d, %d, %d);"
                         % (tx, ty, name, tx, ty, P, s + 1, K))
            parts.append("      return launch_persist<%d, %d>(%s<%d, %d>, %d, %d, %d, tuned_occ(h, occ2), h, p, X, Y, st);"
                         % (tx, ty, name, tx, ty, P, s + 1, K))
            parts.append("    }")
            parts.append("    static const int occ1 = persist_occupancy<64, 1>(%s<64, 1>, %d, %d, %d);"
                         % (name, P, s + 1, K))
            parts.append("    return launch_persist<64, 1>(%s<64, 1>, %d, %d, %d, tuned_occ(h, occ1), h, p, X, Y, st);"
                         % (name, P, s + 1, K))
        elif STENCIL == "tile":
            tx, ty = tile_2d(P)
            parts.append("    if (h->dim == 2) return launch_tile<%d, %d>(%s<%d, %d>, %d, h, p, X, Y, st);"
                         % (tx, ty, name, tx, ty, P))
            parts.append("    return launch_tile<64, 1>(%s<64, 1>, %d, h, p, X, Y, st);" % (name, P))
        else:
            parts.append("    %s<<<grid, %d, 0, st>>>(p, (const float*)X, (float*)Y); note_launch();" % (name, BLOCK))
            parts.append("    return cudaGetLastError();")
        parts.append("  }")
    parts.append("  return cudaSuccess;")
    parts.append("}")
    parts.append("cudaError_t matvec_special_f64(const sg_handle* h, const double2* X, double2* Y, cudaStream_t st,")
    parts.append("                               const int* skip, bool* handled) {")
    parts.append("  *handled = false;")
    parts.append("  OpParams<double> p = h->op64();")
    parts.append("  p.skip = skip;")
    for s, r, name, P, (tx, ty) in table64:
        parts.append("  if (h->s == %d && h->r == %d) {" % (s, r))
        parts.append("    *handled = true;")
        parts.append("    if (h->dim == 2) return launch_tile<%d, %d>(%s<%d, %d>, %d, h, p, X, Y, st);"
                     % (tx, ty, name, tx, ty, P))
        parts.append("    return launch_tile<64, 1>(%s<64, 1>, %d, h, p, X, Y, st);" % (name, P))
        parts.append("  }")
    parts.append("  return cudaSuccess;")
    parts.append("}")
    parts.append("bool matvec_is_specialised(int s, int r) {")
    for s, r, _, _ in table:
        parts.append("  if (s == %d && r == %d) return true;" % (s, r))
    parts.append("  return false;")
    parts.append("}")
    parts.append("}  // namespace sgi")
    src = "\n".join(parts) + "\n"
    os.makedirs(os.path.dirname(path), exist_ok=True)
    old = open(path).read() if os.path.exists(path) else None
    if old != src:
        with open(path, "w") as fh:
            fh.write(src)
    return path
