"""CPU check of the copy index arithmetic of the persistent complex64 operator
kernels, on the generator's own output (no GPU).

The kernel preamble (tile geometry, stencil offsets and the lambdas that issue
the cp.async copies of a tile's values, halo and wavenumber fields) is cut out
of the generated CUDA source and compiled as host C++ with the copy
instructions replaced by a recorder.  For every tile of several grids
(ragged edges, grids smaller than one tile, 1D) and every thread it checks:

* every copy lands inside the CTA's dynamic shared memory (the size the host
  launches with), aligned to its width, and every shared slot of the P mode
  rows (tile and halo) and of the field rows is written exactly once;
* every copy with a non-zero size reads inside X (P * n complex) or the
  fields (s+1 real rows of n);
* the data lands where the arithmetic reads it: a thread's own slot holds its
  unknown's value of that mode, and each stencil neighbour slot (oxm, oxp,
  oym, oyp) holds the neighbouring unknown's value, or zero / any in-grid
  value where the neighbour is outside the grid (its weight is zero there);
  the field slots hold the unknown's k_0 .. k_s.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2209_14740_gb300 import codegen_matvec

HARNESS = r'''
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>
using std::min;

struct Params { int mx, my; long long n; const float* fields; };
struct Rec { uint32_t dst; const float* src; int bytes; int size; };
static std::vector<Rec> g_recs;
static inline void mv_cp_async4(uint32_t dst, const float* src, int bytes) { g_recs.push_back({dst, src, bytes, 4}); }
static inline void mv_cp_async8(uint32_t dst, const float* src, int bytes) { g_recs.push_back({dst, src, bytes, 8}); }
static inline void commit_group_() {}
static constexpr uint32_t XS0 = 4096;   // shared-memory base address of the CTA

static int fails = 0;
#define CHECK(cond, ...) do { if (!(cond)) { if (fails < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } ++fails; } } while (0)

template <int TX, int TY>
void run(int mx, int my, int P, int NFI) {
  constexpr int NT_ = 2 * TX * TY, NN_ = NT_ / 2, NH_ = 2 * (2 * TX + 2 * TY), ST_ = NT_ + NH_;
  const long long n = (long long)mx * my;
  const float* X = reinterpret_cast<const float*>(uintptr_t(1) << 40);
  const float* F = reinterpret_cast<const float*>(uintptr_t(1) << 42);
  Params p{mx, my, n, F};
  const int FS_ = P * ST_;
  const size_t smem_floats = (size_t)P * ST_ + (size_t)NFI * NN_;   // size the host launches with
  const int tiles_x_ = (mx + TX - 1) / TX, tiles_ = tiles_x_ * ((my + TY - 1) / TY);
  for (int tile = 0; tile < tiles_; ++tile) {
    g_recs.clear();
    std::vector<int> ox(NT_ * 4);
    for (int tid_ = 0; tid_ < NT_; ++tid_) {
PREAMBLE
      ISSUE(tile);
      ox[4 * tid_ + 0] = oxm; ox[4 * tid_ + 1] = oxp; ox[4 * tid_ + 2] = oym; ox[4 * tid_ + 3] = oyp;
    }
    // slot contents: -2 unwritten, -1 zero fill, >= 0 X element, <= -10 field element (-10 - index)
    std::vector<long long> slot(smem_floats, -2);
    for (const Rec& r : g_recs) {
      const long long off = (long long)r.dst - XS0;
      CHECK(off >= 0 && off % r.size == 0 && (size_t)(off + r.size) <= smem_floats * 4,
            "tile %d: dst %lld outside or misaligned (size %d)", tile, off, r.size);
      if (!(off >= 0 && (size_t)(off + r.size) <= smem_floats * 4)) continue;
      const long long xi = r.src - X, fi = r.src - F;
      for (int k = 0; k < r.size / 4; ++k) {
        long long& s = slot[off / 4 + k];
        CHECK(s == -2, "tile %d: slot %lld written twice", tile, off / 4 + k);
        if (r.bytes == 0) { s = -1; continue; }
        CHECK(r.bytes == r.size, "tile %d: partial copy", tile);
        if (xi >= 0 && xi < 2 * n * P) {
          CHECK(xi + r.size / 4 <= 2 * n * P, "tile %d: X read past the end", tile);
          CHECK(r.size != 8 || xi % 2 == 0, "tile %d: 8-byte copy of a split unknown", tile);
          s = xi + k;
        } else {
          CHECK(fi >= 0 && fi + r.size / 4 <= (long long)NFI * n, "tile %d: source outside X and fields", tile);
          s = -10 - (fi + k);
        }
      }
    }
    for (int a = 0; a < P; ++a)
      for (int e = 0; e < ST_; ++e) CHECK(slot[(size_t)a * ST_ + e] != -2, "tile %d: mode %d slot %d unwritten", tile, a, e);
    for (int e = 0; e < NFI * NN_; ++e) CHECK(slot[FS_ + e] != -2, "tile %d: field slot %d unwritten", tile, e);
    // what the arithmetic reads
    const int bx0 = (tile % tiles_x_) * TX, by0 = (tile / tiles_x_) * TY;
    for (int t = 0; t < NT_; ++t) {
      const int c = t & 1, nid = t >> 1, lx = nid % TX, ly = nid / TX;
      const int iu0 = bx0 + lx, ju0 = by0 + ly;
      const bool valid = iu0 < mx && ju0 < my;
      const int iu = min(iu0, mx - 1), ju = min(ju0, my - 1);
      for (int a = 0; a < P; ++a) {
        const long long base = (long long)a * 2 * n;
        CHECK(slot[(size_t)a * ST_ + t] == base + 2 * (iu + (long long)mx * ju) + c, "tile %d t %d mode %d: own value", tile, t, a);
        if (!valid) continue;
        const int nb[4][3] = {{iu > 0, iu - 1, ju}, {iu < mx - 1, iu + 1, ju}, {ju > 0, iu, ju - 1}, {ju < my - 1, iu, ju + 1}};
        for (int d = 0; d < 4; ++d) {
          const long long v = slot[(size_t)a * ST_ + ox[4 * t + d]];
          if (nb[d][0])
            CHECK(v == base + 2 * (nb[d][1] + (long long)mx * nb[d][2]) + c, "tile %d t %d mode %d dir %d: neighbour", tile, t, a, d);
          else
            CHECK(v == -1 || (v >= base && v < base + 2 * n), "tile %d t %d mode %d dir %d: outside value", tile, t, a, d);
        }
      }
      if (c == 0)
        for (int l = 0; l < NFI; ++l)
          CHECK(slot[FS_ + l * NN_ + nid] == -10 - (l * n + iu + (long long)mx * ju), "tile %d t %d: field %d", tile, t, l);
    }
  }
}

int main() {
  const int P = PMODES, NFI = NFIELDS;
  const int g2[][2] = {{37, 29}, {5, 3}, {64, 8}, {65, 9}, {33, 5}, {127, 127}, {32, 4}};
  for (auto& g : g2) run<32, 4>(g[0], g[1], P, NFI);
  for (int mx : {129, 64, 7, 200, 1}) run<64, 1>(mx, 1, P, NFI);
  std::printf("fails %d\n", fails);
  return fails ? 1 : 0;
}
'''


def preamble(src):
    """The generated kernel body up to its tile loop, made host C++."""
    lines = src.splitlines()
    start = next(i for i, l in enumerate(lines) if l.startswith("__global__")) + 1
    stop = next(i for i, l in enumerate(lines) if l.strip().startswith("int tile = blockIdx.x"))
    out = []
    for l in lines[start:stop]:
        if "extern __shared__" in l or "p.skip" in l:
            continue
        l = l.replace("threadIdx.x", "tid_")
        l = l.replace("(uint32_t)__cvta_generic_to_shared(xs)", "XS0")
        l = l.replace('asm volatile("cp.async.commit_group;" ::: "memory");', "commit_group_();")
        assert "asm" not in l and "__" not in l.replace("__restrict__", ""), l
        out.append(l)
    return "\n".join(out)


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
@pytest.mark.parametrize("s,r", [(6, 3), (3, 3), (4, 3)])
def test_generated_copy_indices(s, r):
    name, P, src = codegen_matvec.gen_kernel_tkp(s, r)
    body = preamble(src)
    issue = "issue_late" if "auto issue_late" in body else "issue"
    code = (HARNESS.replace("PREAMBLE", body).replace("ISSUE(tile)", "%s(tile)" % issue)
            .replace("PMODES", str(P)).replace("NFIELDS", str(s + 1)))
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "h.cpp")
        exe = os.path.join(d, "h")
        open(cpp, "w").write(code)
        cc = subprocess.run(["g++", "-std=c++17", "-O1", "-w", cpp, "-o", exe], capture_output=True, text=True)
        assert cc.returncode == 0, cc.stderr[-3000:]
        run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.strip().endswith("fails 0"), run.stdout[-3000:]
