"""CPU parity of the generated complex64 operator kernels: their emitted
arithmetic, run on the host, against the oracle's explicit SG matrix.

The persistent kernel's preamble and its tile body (the stencil, the
factorised coupling rows, the stores) are cut out of the generated CUDA
source and compiled as host C++ together with the library's own per-node
geometry (k_operator_geom.cuh):

* the kernel's copy code fills a host copy of the CTA's shared memory
  (values, halo, wavenumber fields) for each tile;
* every thread's tile body then runs one after another; the two threads of
  an unknown exchange W through a warp shuffle on boundary warps, emulated
  in two passes (the W rows never depend on the exchange: pass 1 records
  each thread's shuffled values, pass 2 replays the partner's);
* barriers, the copy waits and the register fences are dropped (between
  them a thread only reads shared memory the copies already filled).

Every product is written out as fmaf or a single multiply in the emitted
code, so the host runs the same FP32 operations in the same order.  The
result must match the oracle's A x (complex128) within the FP32 bound of the
GPU parity tests (3e-6 of the row's absolute scale).  The FP64 kernels (one
CTA per tile, register-resident for P <= 35, mode values in shared memory
for P = 84) run the same way, whole, against the FP64 bound (1e-13).  This
lets the generator be checked without a GPU.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import sg
from paper_2209_14740_gb300 import codegen_matvec, inputs

HERE = os.path.dirname(os.path.abspath(__file__))
GEOM = os.path.join(os.path.dirname(HERE), "paper_2209_14740_gb300", "csrc", "k_operator_geom.cuh")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r'''
#include "GEOM_HEADER"
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
using namespace sgi;
using std::min;

static float* g_xs = nullptr;
static constexpr uint32_t XS0 = 4096;
static inline void copy_(uint32_t dst, const float* src, int bytes, int size) {
  float* d = g_xs + (dst - XS0) / 4;
  if (bytes) std::memcpy(d, src, size); else std::memset(d, 0, size);
}
static inline void mv_cp_async4(uint32_t dst, const float* src, int bytes) { copy_(dst, src, bytes, 4); }
static inline void mv_cp_async8(uint32_t dst, const float* src, int bytes) { copy_(dst, src, bytes, 8); }
static inline void commit_group_() {}

static int g_pass = 0, g_lane = 0;
static size_t g_pos = 0;
static std::vector<std::vector<float>> g_rec;
static inline float shfl_partner_(float v) {
  if (g_pass == 0) { g_rec[g_lane].push_back(v); return 0.0f; }
  return g_rec[g_lane ^ 1][g_pos++];
}

template <int TX, int TY>
void run(const OpParams<float>& p, const float* X, float* Y, int P, int NFI) {
  constexpr int NT_ = 2 * TX * TY, NH_ = 2 * (2 * TX + 2 * TY), ST_ = NT_ + NH_;
  std::vector<float> xs_buf((size_t)P * ST_ + (size_t)NFI * (NT_ / 2));
  float* xs = xs_buf.data();   // the kernel's shared array
  g_xs = xs;
  g_rec.assign(NT_, {});
  const int tiles_x_ = (p.mx + TX - 1) / TX, tiles_ = tiles_x_ * ((p.my + TY - 1) / TY);
  std::vector<char> any_w1(NT_ / 32 + 1);
  for (int tile = 0; tile < tiles_; ++tile) {
    std::fill(xs_buf.begin(), xs_buf.end(), std::nanf(""));
    for (int tid_ = 0; tid_ < NT_; ++tid_) {
PREAMBLE
      ISSUE(tile);
    }
    // the warp-uniform boundary flag (__any_sync over the warp)
    std::fill(any_w1.begin(), any_w1.end(), 0);
    for (int t = 0; t < NT_; ++t) {
      const int lx = (t >> 1) % TX, ly = (t >> 1) / TX;
      const int iu = min((tile % tiles_x_) * TX + lx, p.mx - 1), ju = min((tile / tiles_x_) * TY + ly, p.my - 1);
      if (node_geom<float>(p, iu, ju).w1 != 0.0f) any_w1[t >> 5] = 1;
    }
    for (g_pass = 0; g_pass < 2; ++g_pass) {
      for (int tid_ = 0; tid_ < NT_; ++tid_) {
        g_lane = tid_;
        g_pos = 0;
        if (g_pass == 0) g_rec[tid_].clear();
PREAMBLE
        {
BODY
        }
      }
    }
  }
}

int main(int argc, char** argv) {
  // input file: dim mx my P s absL absR absB absT h, then fields (s+1)*n, then X 2*n*P floats
  FILE* f = std::fopen(argv[1], "rb");
  int hdr[9];
  double h;
  if (std::fread(hdr, sizeof(int), 9, f) != 9 || std::fread(&h, sizeof(double), 1, f) != 1) return 2;
  OpParams<float> p{};
  p.dim = hdr[0]; p.mx = hdr[1]; p.my = hdr[2]; p.P = hdr[3]; p.s = hdr[4];
  p.absL = hdr[5]; p.absR = hdr[6]; p.absB = hdr[7]; p.absT = hdr[8];
  p.n = p.mx * p.my;
  p.h = (float)h; p.inv_h = (float)(1.0 / h); p.inv_h2 = (float)(1.0 / (h * h));
  const int NFI = p.s + 1;
  std::vector<float> fields((size_t)NFI * p.n), X(2 * (size_t)p.n * p.P), Y(2 * (size_t)p.n * p.P, 0.0f);
  if (std::fread(fields.data(), sizeof(float), fields.size(), f) != fields.size()) return 2;
  if (std::fread(X.data(), sizeof(float), X.size(), f) != X.size()) return 2;
  std::fclose(f);
  p.fields = fields.data();
  if (p.dim == 2) run<TX2, TY2>(p, X.data(), Y.data(), p.P, NFI);
  else run<64, 1>(p, X.data(), Y.data(), p.P, NFI);
  FILE* o = std::fopen(argv[2], "wb");
  std::fwrite(Y.data(), sizeof(float), Y.size(), o);
  std::fclose(o);
  return 0;
}
'''


def _split(src):
    """(preamble, body) of the generated persistent kernel, made host C++."""
    lines = src.splitlines()
    start = next(i for i, l in enumerate(lines) if l.startswith("__global__")) + 1
    loop = next(i for i, l in enumerate(lines) if l.strip().startswith("for (; tile < tiles"))
    pre_end = next(i for i, l in enumerate(lines) if l.strip().startswith("int tile = blockIdx.x"))
    # the tile loop's body: up to its closing brace (the line before the kernel's)
    assert lines[-1] == "}" and lines[-2] == "  }"
    body = lines[loop + 1:-2]

    def host(l):
        l = l.replace("threadIdx.x", "tid_")
        l = l.replace("(uint32_t)__cvta_generic_to_shared(xs)", "XS0")
        l = l.replace('asm volatile("cp.async.commit_group;" ::: "memory");', "commit_group_();")
        l = l.replace("__any_sync(0xffffffffu, g.w1 != 0.0f)", "(any_w1[tid_ >> 5] != 0)")
        l = l.replace("__shfl_xor_sync(0xffffffffu, wv, 1)", "shfl_partner_(wv)")
        return l

    pre = []
    for l in lines[start:pre_end]:
        if "extern __shared__" in l or "p.skip" in l:
            continue
        pre.append(host(l))
    out = []
    for l in body:
        s = l.strip()
        if (s.startswith('asm volatile("cp.async.wait_all') or s == "__syncthreads();"
                or s.startswith("__syncthreads();") or "issue" in s or s.startswith('asm volatile("" :')):
            continue
        out.append(host(l))
    text = "\n".join(pre + out)
    assert "asm" not in text and "__shfl" not in text and "__any" not in text and "__sync" not in text, \
        [l for l in (pre + out) if "asm" in l or "__" in l.replace("__restrict__", "")][:3]
    return "\n".join(pre), "\n".join(out)


CASES = [
    # (s, r, dim, g, bc)
    (2, 3, 2, 37, "abs"),
    (3, 3, 2, 29, "abs"),
    (3, 3, 2, 13, "dir"),
    (6, 3, 2, 9, "abs"),
    (1, 5, 1, 150, "mixed"),
    (4, 3, 1, 70, "abs"),
]


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and CUDA headers")
@pytest.mark.parametrize("s,r,dim,g,bc", CASES)
def test_generated_operator_on_host(s, r, dim, g, bc):
    A_, D_ = inputs.ABSORBING, inputs.DIRICHLET
    bcs = {"abs": (A_,) * 4 if dim == 2 else (A_, A_, D_, D_), "dir": (D_,) * 4,
           "mixed": (D_, A_, D_, D_)}[bc]
    pr = inputs.random_problem(100 * s + r + g, dim=dim, g=g, s=s, r=r, bc=bcs)
    ref = sg.assemble_problem(pr)
    grid = ref.grid
    mx = len(np.unique(grid.unknowns % pr.nx))
    my = grid.unknowns.size // mx
    n = grid.unknowns.size
    name, P, src = codegen_matvec.gen_kernel_tkp(s, r)
    assert P == ref.P
    pre, body = _split(src)
    issue = "issue_late" if "auto issue_late" in pre else "issue"
    tx, ty = codegen_matvec.PTILE_2D
    code = (HARNESS.replace("GEOM_HEADER", GEOM).replace("PREAMBLE", pre).replace("BODY", body)
            .replace("ISSUE(tile)", "%s(tile)" % issue).replace("TX2", str(tx)).replace("TY2", str(ty)))
    # device layout: fields on the unknowns, X mode-major (x fastest), complex interleaved
    k0 = np.asarray(pr.k0, float).reshape(-1)[grid.unknowns]
    kl = np.asarray(pr.kl, float).reshape(s, -1)[:, grid.unknowns]
    fields = np.concatenate([k0[None, :], kl], 0).astype(np.float32)
    rng = np.random.default_rng(s * 1000 + g)
    x = (rng.standard_normal(n * P) + 1j * rng.standard_normal(n * P)).astype(np.complex64)
    bnd = [1 if pr.bc[i] == A_ else 0 for i in range(4)]
    hdr = np.array([dim, mx, my, P, s] + bnd, dtype=np.int32)
    with tempfile.TemporaryDirectory() as d:
        cpp, exe = os.path.join(d, "h.cpp"), os.path.join(d, "h")
        fin, fout = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
        open(cpp, "w").write(code)
        cc = subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-w", "-I", CUDA_INC, cpp, "-o", exe],
                            capture_output=True, text=True, timeout=600)
        assert cc.returncode == 0, cc.stderr[-3000:]
        with open(fin, "wb") as fh:
            fh.write(hdr.tobytes())
            fh.write(np.array([pr.h], dtype=np.float64).tobytes())
            fh.write(fields.tobytes())
            fh.write(x.view(np.float32).tobytes())
        run = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=300)
        assert run.returncode == 0, run.stderr
        y = np.fromfile(fout, dtype=np.float32).view(np.complex64).astype(np.complex128)
    x64 = x.astype(np.complex128)
    yr = ref.A @ x64
    scale = abs(ref.A) @ np.abs(x64) + abs(ref.Lbig) @ np.abs(x64)
    err = np.abs(y - yr) / scale
    assert np.all(err <= 3e-6), (err.max(), int(err.argmax()))


# ---------------------------------------------------------------- FP64 kernels
# One CTA per tile (launch_tile): every thread loads its unknown's values, the
# CTA fills shared memory (tile and halo), a barrier, then the coupling.  On
# the host each CTA runs its threads three times: pass 0 fills the shared
# copy (its arithmetic is discarded), pass 1 records the shuffled W values,
# pass 2 replays the partner's and stores.
HARNESS64 = r'''
#include "GEOM_HEADER"
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
using namespace sgi;
using std::min;

static double* g_xs64 = nullptr;
static constexpr uint32_t XS0 = 4096;
template <class T> static inline T ldg_(const T* q) { return *q; }
static inline void cpa64_(uint32_t dst, const double* src, int bytes) { g_xs64[(dst - XS0) / 8] = bytes ? *src : 0.0; }

static int g_pass = 0, g_lane = 0;
static size_t g_pos = 0;
static std::vector<std::vector<double>> g_rec;
static inline double shfl_partner_(double v) {
  if (g_pass == 0) { g_rec[g_lane].push_back(v); return 0.0; }
  return g_rec[g_lane ^ 1][g_pos++];
}

template <int TX, int TY>
void run(const OpParams<double>& p, const double* X, double* Y, int P) {
  constexpr int NT_ = 2 * TX * TY, NH_ = 2 * (2 * TX + 2 * TY), ST_ = NT_ + NH_;
  std::vector<double> xs_buf((size_t)P * ST_);
  g_xs64 = xs_buf.data();
  g_rec.assign(NT_, {});
  std::vector<char> any_w1(NT_ / 32 + 1);
  for (int by_ = 0; by_ < (p.my + TY - 1) / TY; ++by_)
    for (int bx_ = 0; bx_ < (p.mx + TX - 1) / TX; ++bx_) {
      std::fill(xs_buf.begin(), xs_buf.end(), std::nan(""));
      std::fill(any_w1.begin(), any_w1.end(), 0);
      for (int t = 0; t < NT_; ++t) {
        const int lx = (t >> 1) % TX, ly = (t >> 1) / TX;
        if (node_geom<double>(p, min(bx_ * TX + lx, p.mx - 1), min(by_ * TY + ly, p.my - 1)).w1 != 0.0) any_w1[t >> 5] = 1;
      }
      for (int pass = 0; pass < 3; ++pass) {
        g_pass = pass == 2 ? 1 : 0;
        for (int tid_ = 0; tid_ < NT_; ++tid_) {
          g_lane = tid_;
          g_pos = 0;
          if (pass < 2) g_rec[tid_].clear();
BODY
        }
      }
    }
}

int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "rb");
  int hdr[9];
  double h;
  if (std::fread(hdr, sizeof(int), 9, f) != 9 || std::fread(&h, sizeof(double), 1, f) != 1) return 2;
  OpParams<double> p{};
  p.dim = hdr[0]; p.mx = hdr[1]; p.my = hdr[2]; p.P = hdr[3]; p.s = hdr[4];
  p.absL = hdr[5]; p.absR = hdr[6]; p.absB = hdr[7]; p.absT = hdr[8];
  p.n = p.mx * p.my;
  p.h = h; p.inv_h = 1.0 / h; p.inv_h2 = 1.0 / (h * h);
  std::vector<double> fields((size_t)(p.s + 1) * p.n), X(2 * (size_t)p.n * p.P), Y(2 * (size_t)p.n * p.P, 0.0);
  if (std::fread(fields.data(), sizeof(double), fields.size(), f) != fields.size()) return 2;
  if (std::fread(X.data(), sizeof(double), X.size(), f) != X.size()) return 2;
  std::fclose(f);
  p.fields = fields.data();
  if (p.dim == 2) run<TX2, TY2>(p, X.data(), Y.data(), p.P);
  else run<64, 1>(p, X.data(), Y.data(), p.P);
  FILE* o = std::fopen(argv[2], "wb");
  std::fwrite(Y.data(), sizeof(double), Y.size(), o);
  std::fclose(o);
  return 0;
}
'''


def _balanced(s, i):
    """s[i] == '(' -> index of the matching ')'."""
    depth = 0
    for j in range(i, len(s)):
        depth += s[j] == "("
        depth -= s[j] == ")"
        if depth == 0:
            return j
    raise ValueError(s)


def _host64(src):
    """The whole generated FP64 kernel body, made host C++."""
    lines = src.splitlines()
    assert lines[1].startswith("__global__") and lines[-1] == "}"
    out = []
    for l in lines[2:-1]:
        s = l.strip()
        if ("extern __shared__" in l or "p.skip" in l or s == "__syncthreads();" or s.startswith('asm volatile("" ')
                or s.startswith('asm volatile("cp.async.wait_all')):
            continue
        if "cp.async.ca.shared.global" in l:
            # asm volatile("cp.async... [%0], [%1], 8[, %2];" :: "r"(DST), "l"(SRC)[, "r"(SZ)] : "memory");
            i = l.index('"r"(') + 3
            j = _balanced(l, i)
            dst = l[i + 1:j]
            k = l.index('"l"(', j) + 3
            m = _balanced(l, k)
            srcx = l[k + 1:m]
            sz = "8"
            if '"r"(' in l[m:]:
                q = l.index('"r"(', m) + 3
                sz = l[q + 1:_balanced(l, q)]
            l = l[:len(l) - len(l.lstrip())] + "cpa64_(%s, %s, %s);" % (dst, srcx, sz)
        l = l.replace("reinterpret_cast<double*>(xs64_raw)", "g_xs64").replace("reinterpret_cast<double*>(xs64h_raw)", "g_xs64")
        l = l.replace("(unsigned)__cvta_generic_to_shared(xs)", "XS0")
        l = l.replace("threadIdx.x", "tid_").replace("blockIdx.x", "bx_").replace("blockIdx.y", "by_")
        l = l.replace("__ldg(", "ldg_(")
        l = l.replace("__any_sync(0xffffffffu, g.w1 != 0.0)", "(any_w1[tid_ >> 5] != 0)")
        l = l.replace("__shfl_xor_sync(0xffffffffu, wv, 1)", "shfl_partner_(wv)")
        out.append(l)
    text = "\n".join(out)
    bad = [l for l in out if "asm" in l or "__" in l.replace("__restrict__", "").replace("__align__", "")]
    assert not bad, bad[:3]
    return "{\n" + text + "\n}"


CASES64 = [
    # (s, r, dim, g, bc)
    (2, 3, 2, 37, "abs"),
    (3, 3, 2, 21, "dir"),
    (4, 3, 2, 18, "abs"),
    (1, 5, 1, 150, "mixed"),
    (6, 3, 2, 20, "abs"),
    (6, 3, 1, 70, "abs"),
]


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INC), reason="needs g++ and CUDA headers")
@pytest.mark.parametrize("s,r,dim,g,bc", CASES64)
def test_generated_fp64_operator_on_host(s, r, dim, g, bc):
    A_, D_ = inputs.ABSORBING, inputs.DIRICHLET
    bcs = {"abs": (A_,) * 4 if dim == 2 else (A_, A_, D_, D_), "dir": (D_,) * 4,
           "mixed": (D_, A_, D_, D_)}[bc]
    pr = inputs.random_problem(7 * s + r + g, dim=dim, g=g, s=s, r=r, bc=bcs)
    ref = sg.assemble_problem(pr)
    grid = ref.grid
    mx = len(np.unique(grid.unknowns % pr.nx))
    my = grid.unknowns.size // mx
    n = grid.unknowns.size
    P = ref.P
    if P <= codegen_matvec.F64_MAX_P:
        name, _, src = codegen_matvec.gen_kernel_tk(s, r, "f64")
        tx, ty = codegen_matvec.tile_2d(P)
    else:
        name, _, src = codegen_matvec.gen_kernel_tk64_halves(s, r)
        tx, ty = codegen_matvec.F64_HALVES_TILE
    code = (HARNESS64.replace("GEOM_HEADER", GEOM).replace("BODY", _host64(src))
            .replace("TX2", str(tx)).replace("TY2", str(ty)))
    k0 = np.asarray(pr.k0, float).reshape(-1)[grid.unknowns]
    kl = np.asarray(pr.kl, float).reshape(s, -1)[:, grid.unknowns]
    fields = np.concatenate([k0[None, :], kl], 0)
    rng = np.random.default_rng(s * 77 + g)
    x = rng.standard_normal(n * P) + 1j * rng.standard_normal(n * P)
    bnd = [1 if pr.bc[i] == A_ else 0 for i in range(4)]
    hdr = np.array([dim, mx, my, P, s] + bnd, dtype=np.int32)
    with tempfile.TemporaryDirectory() as d:
        cpp, exe = os.path.join(d, "h.cpp"), os.path.join(d, "h")
        fin, fout = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
        open(cpp, "w").write(code)
        cc = subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-w", "-I", CUDA_INC, cpp, "-o", exe],
                            capture_output=True, text=True, timeout=900)
        assert cc.returncode == 0, cc.stderr[-3000:]
        with open(fin, "wb") as fh:
            fh.write(hdr.tobytes())
            fh.write(np.array([pr.h], dtype=np.float64).tobytes())
            fh.write(fields.astype(np.float64).tobytes())
            fh.write(x.view(np.float64).tobytes())
        run = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=300)
        assert run.returncode == 0, run.stderr
        y = np.fromfile(fout, dtype=np.float64).view(np.complex128)
    yr = ref.A @ x
    scale = abs(ref.A) @ np.abs(x) + abs(ref.Lbig) @ np.abs(x)
    err = np.abs(y - yr) / scale
    assert np.all(err <= 1e-13), (err.max(), int(err.argmax()))
