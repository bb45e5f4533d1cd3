// Internal declarations of the GB300 SG Helmholtz library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <exception>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/sg.h"

namespace sgi {

using cd = std::complex<double>;

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
sg_status fail(sg_status st, const std::string& msg);
// Runs the body of an ABI entry point: no C++ exception (a failed host
// allocation, a container error) may cross the C ABI, so each becomes a
// status and a message.
template <typename F>
sg_status guarded(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(SG_ENOMEM, "host memory allocation failed");
  } catch (const std::exception& e) {
    return fail(SG_EINVAL, std::string("host exception: ") + e.what());
  } catch (...) {
    return fail(SG_EINVAL, "unknown host exception");
  }
}
#define SG_CUDA_TRY(expr)                                                       \
  do {                                                                          \
    cudaError_t e_ = (expr);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return ::sgi::fail(SG_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------- device complex helpers
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using C2 = typename Vec2<T>::type;

// ---------------------------------------------------------------- operator description
// Parameters every operator kernel needs: unknown-grid geometry and the
// chaos coupling tables (device pointers).
template <typename T>
struct OpParams {
  int dim, mx, my, n, P, s, T_terms;
  int absL, absR, absB, absT;      // 1 if that side is absorbing
  T h, inv_h, inv_h2;
  const int* rowptr;               // P+1, off-diagonal coupling rows
  const int* col;                  // nnz_off
  const int* term;                 // nnz_off, term id in [0, T_terms)
  const T* gval;                   // nnz_off, Galerkin product value
  const T* gdiag;                  // s*P, <xi_l^2 phi_a phi_a>, layout [l][a]
  const T* fields;                 // (s+1)*n: k_0, k_1..k_s on the unknowns
  const int* skip;                 // optional device flag: kernel returns at once if *skip != 0
};

// Tridiagonal LU factors with partial pivoting (LAPACK gttrf layout) for
// `nsys` systems of length `len`; element (j, sys) at j*nsys + sys.
template <typename T>
struct TriFactors {
  C2<T>* dl = nullptr;    // multipliers
  C2<T>* dinv = nullptr;  // 1 / U diagonal
  C2<T>* du = nullptr;    // U first superdiagonal
  C2<T>* du2 = nullptr;   // U second superdiagonal (fill from pivoting)
  uint8_t* piv = nullptr; // 1 if rows j, j+1 were swapped
};

// Banded LU with partial pivoting (k_band.cu; LAPACK gbtrf layout: column j
// at ab + j * ldab, entry (i, j) at row kl + ku + i - j, ldab = 2 kl + ku + 1),
// factored in FP64 with an FP32 copy for complex64 solves.
struct BandFactor {
  int n = 0, kl = 0, ku = 0, ldab = 0;
  double2* ab = nullptr;
  float2* ab32 = nullptr;
  int* piv = nullptr;
};
// Factors f.ab in place (FP64 pivots), fills f.piv and f.ab32; *d_bad = 1 on
// a zero pivot.
cudaError_t band_factor(BandFactor& f, int* d_bad, cudaStream_t st);
// Z = A^-1 (s R) for nrhs right-hand sides (column q at q * ld, s = *in_scale
// or 1), through the intermediate Y; R, Y, Z may be the same vector.
template <typename T>
cudaError_t band_solve(const BandFactor& f, int nrhs, const C2<T>* R, C2<T>* Y, C2<T>* Z, long long ld,
                       cudaStream_t st, const int* skip, const double* in_scale);
// Whether the solve kernel's shared memory holds a window of this band.
bool band_fits(int kl, int ku);

struct PrecBlock {
  bool ready = false;
  TriFactors<double> f64;
  TriFactors<float> f32;
  BandFactor band;          // 2D blocks without a separable inverse (k_0 varies in space)
};

// Constant right factor of a tensor-core complex GEMM (k_tc_gemm.cu): the
// real embedding of a kdim x ndim complex matrix, split hi / lo in TF32,
// in [column tile][K stage][bn x 32 core-matrix block] order, bn = 64 or 128
// real output columns per CTA.
// The same factor in binary16 (h16): K stages of 64 values in 128-byte rows,
// core matrices of 8 rows x 8 values, for the FP16 transforms.
struct TcOperand {
  int kdim = 0, ndim = 0, nks = 0, ntiles = 0, bn = 64, nks16 = 0;
  std::vector<float> hi, lo;
  std::vector<uint16_t> h16;
};
struct TcDevOperand {
  int kdim = 0, ndim = 0, nks = 0, ntiles = 0, bn = 64, nks16 = 0;
  float* hi = nullptr;
  float* lo = nullptr;
  uint16_t* h16 = nullptr;
};
TcOperand tc_make_operand(const std::vector<std::complex<double>>& Q, int kdim, int ndim, int bn);
// Binary16 tiles only (op.h16, op.nks16) for tile width bn (64, 128 or 256).
TcOperand tc_make_operand16(const std::vector<std::complex<double>>& Q, int kdim, int ndim, int bn);
void tc_fill_h16(TcOperand& op, const std::vector<std::complex<double>>& Q, int bn);
// Tile width (64 or 128 real columns) for a GEMM of `rows` rows and ndim
// complex output columns on a GPU with num_sms SMs.
int tc_tile_width(long long rows, int ndim, int num_sms);
// C = X Q for M complex64 rows X (row stride ldx complex), placement mode 0
// (row-major, ldc) or 1 (per-batch transpose, batches of MB rows, transposed
// rows ldc >= MB apart); 16-byte loads of X when ldx is even; split: FP32
// accuracy (3xTF32), else plain TF32 (one MMA per K step); optional
// elementwise factor E[n * e_ld + m % e_mod] * (*escale).
// out_half: C gets binary16 pairs; every output value is scaled by oscale
// (and by *escale if given).
cudaError_t tc_cgemm(const TcDevOperand& B, const float2* X, long long ldx, int M, float2* C, long long ldc,
                     int mode, int MB, const float2* E, int e_ld, int e_mod, const double* escale, const int* skip,
                     int* err, cudaStream_t st, bool split = true, const CUtensorMap* xmap = nullptr,
                     bool out_half = false, float oscale = 1.0f);
// The FP16 form (persistent, kind::f16 MMAs): X binary16 pairs by tensor
// copies through xmap (tc_make_xmap16), B's binary16 tiles, output binary16
// pairs (out_half) or complex64, scaled by (*escale) * oscale.
cudaError_t tc_hgemm(const TcDevOperand& B, const void* X, int M, void* C, long long ldc, int mode, int MB,
                     const float2* E, int e_ld, int e_mod, const double* escale, float oscale, bool out_half,
                     const int* skip, int* err, cudaStream_t st, const CUtensorMap* xmap);
// The same product by the paired 256-column kernel (clusters of two CTAs on
// adjacent row tiles sharing each B stage through multicast copies): B is a
// 256-wide binary16 operand (tc_make_operand16 with bn = 256).  Not supported
// when the GPU cannot hold a cluster of two such CTAs.
cudaError_t tc_hgemm_w(const TcDevOperand& B, const void* X, int M, void* C, long long ldc, int mode, int MB,
                       const float2* E, int e_ld, int e_mod, const double* escale, float oscale, bool out_half,
                       const int* skip, int* err, cudaStream_t st, const CUtensorMap* xmap);
bool tc_wide_available();
// Tensor map of M rows of kdim binary16 pairs, row pitch ldx pairs (ldx a
// multiple of 4, X 16-byte aligned): boxes of 64 values x 128 rows in the
// 128-byte swizzle.
bool tc_make_xmap16(CUtensorMap* map, const void* X, long long ldx, int M, int kdim);
// One warp waits on an mbarrier nothing arrives on, with the transform
// kernel's bounded wait; sets *err = 1 when the wait gives up, *done = 1 at
// the end (device ints).
cudaError_t tc_wait_selftest(int* err, int* done, cudaStream_t st);
// Tensor map of X (M complex64 rows of kdim values, row pitch ldx complex, 16-byte
// aligned, ldx even) for the plain-TF32 transform: a 2D view (2 kdim real values,
// M rows) whose 32 x 128 box is one K stage of one row tile, landing in the
// 128-byte swizzle layout of the MMA's A operand.  False if the driver entry
// point or the encoding is unavailable (the kernel then copies X itself).
bool tc_make_xmap(CUtensorMap* map, const float2* X, long long ldx, int M, int kdim);

struct GmresWork {
  int restart = 0;         // basis capacity (columns restart+1)
  int prec_bytes = 0;      // 8 (c64) or 16 (c128) per element of V
  void* V = nullptr;       // (restart+1) * N inner precision
  void* Z = nullptr;       // N inner precision
  void* Zb = nullptr;      // flexible GMRES (complex64 inner cycles with the TF32 preconditioner):
                           // z_j = M^-1 v_j for every step j, restart * N complex64
  void* V16 = nullptr;     // the binary16 route of those cycles: the newest basis vector as binary16
                           // pairs, P my rows of mx4 (mx rounded up to a multiple of 4) pairs, written
                           // by the second CGS2 pass, read by the next step's transform 1 through v16map
  CUtensorMap v16map;
  void* Vh = nullptr;      // SG_MIXED flexible cycles on the binary16 route: the Krylov basis as binary16
                           // pairs, (restart+1) slots of vh_np pairs (P my rows of mx4), slot i read by
                           // the preconditioner's transform 1 through vhmaps[i]
  long long vh_np = 0;
  std::vector<CUtensorMap> vhmaps;
  void* R64 = nullptr;     // N complex128 (mixed: outer residual; fp64: A x)
  void* X64 = nullptr;     // N complex128 staging for host_io / x0
  void* B64 = nullptr;     // N complex128 staging for host_io
  double* dscal = nullptr; // device scalars (see solver.cu)
  int* dctl = nullptr;     // device control words
  double* part = nullptr;  // partial sums [nblk][2*(restart+2)]
  unsigned* counter = nullptr;
  int nblk = 0;            // blocks of the reduction kernels
  int cg_nblk = 0;         // blocks of the CGS2 passes
  // Arnoldi step chunks captured as CUDA graphs, keyed by (inner precision,
  // preconditioner, first step, steps): a key is captured on its second use
  // and replayed from then on (one-shot solves never pay for instantiation).
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;   // kernel launches recorded in the graph
  };
  std::map<unsigned long long, Graph> graphs;
  std::map<unsigned long long, int> graph_uses;
  cudaStream_t stream = nullptr;   // private stream: capture needs a non-legacy stream
  cudaEvent_t ev = nullptr;
  unsigned long long uid = 0;      // unique per allocation: keys the batched-solve graphs
};

}  // namespace sgi

struct sg_handle {
  int dim = 1, nx = 0, ny = 1, mx = 0, my = 1, offx = 0, offy = 0, n = 0, P = 0, s = 0, r = 0;
  int T_terms = 0;
  // tensor maps of the plain-TF32 transforms' inputs (fast diagonalisation,
  // transforms 2-4: d_tmp, d_tmp2, d_tmp with their even row pitches)
  CUtensorMap tc_xmap[3];
  bool tc_xmap_ok = false;
  // binary16 route of the same transforms (the solver's flexible cycles):
  // inputs of transforms 2-4 as binary16 pairs in d_tmp / d_tmp2 with rows
  // padded to a multiple of 4 pairs, and transform 2's output scale per block
  // (1 / max |L^-1|, so that the scaled values stay near 1)
  CUtensorMap tc_xmap16[3];
  bool fd16 = false;
  float fd16_scale[2] = {1.0f, 1.0f};
  double* d_fd16s = nullptr;          // sg_precond(SG_FP16): 1 / ||R|| and ||R|| (device)
  double* d_fd16part = nullptr;       // its block partial sums
  long long N = 0;
  double h = 0, beta = 0.5, kbar = 0;
  int bc[4] = {0, 0, 0, 0};
  bool separable = false;
  int specialised = 0;
  int num_sms = 0;
  int device = 0;

  // host tables
  std::vector<int> alpha;            // P*s multi-indices
  std::vector<int> rowptr, col, term;
  std::vector<double> gval, gdiag;   // off-diagonal values, diagonal moments [l][a]
  std::vector<double> b0;            // n, FD-weighted source on the unknowns
  std::vector<double> k0u;           // n, k_0 on the unknowns
  std::vector<double> fields_host;   // (s+1) n: k_0, k_1..k_s on the unknowns

  // device tables
  int *d_rowptr = nullptr, *d_col = nullptr, *d_term = nullptr;
  double *d_gval = nullptr, *d_gdiag = nullptr, *d_fields = nullptr, *d_b0 = nullptr;
  float *d_gval32 = nullptr, *d_gdiag32 = nullptr, *d_fields32 = nullptr;

  // preconditioner data
  sgi::PrecBlock blk[2];             // [0] mean value S(xi_bar), [1] CSL M_0 block
  // the coupled CSL matrix M(beta) = A - i beta K (Sec. 4), numbered point by
  // point (row u P + a), banded; factored on first use
  sgi::BandFactor csl_full;
  double2* d_Q = nullptr;            // 2D: Qhat = D_x^-1/2 Q, row-major mx x mx
  double2* d_Qt = nullptr;           // 2D: Qhat^T
  float2* d_Q32 = nullptr;
  float2* d_Qt32 = nullptr;
  double* d_dyinv = nullptr;         // 2D: d_y^-1/2 per y line
  float* d_dyinv32 = nullptr;
  void* d_tmp = nullptr;             // N complex128 scratch (preconditioner intermediate)
  void* d_tmp2 = nullptr;            // N complex128 scratch (2D: second intermediate)
  double eig_orth_err = 0.0;         // max |Q^T Q - I| of the host eigenvectors (<= 1e-10 accepted)
  double eig_kappa = 0.0;            // cond(Q) of the eigenvector factors (<= 100 accepted)
  // 2D fast diagonalisation (FP32 applies): both directions transformed,
  // S^-1 = (Qhat_y (x) Qhat_x) diag(1 / (lambda_y,j + lambda_x,i + shift)) (Qhat_y (x) Qhat_x)^T
  bool fd = false;                   // fast-diagonalisation factors built (SG_TF32 route)
  bool fd_fp32 = false;              // FP32 (3xTF32) applies use them too (lines <= 320)
  float2* d_Qy32 = nullptr;          // Qhat_y = D_y^-1/2 Q_y, row-major my x my
  float2* d_Qyt32 = nullptr;         // Qhat_y^T
  float2* d_Linv32[2] = {nullptr, nullptr};   // [block] my x mx: 1 / (lambda_y,j + lambda_x,i + shift)
  sgi::TcDevOperand tcB[4];          // tensor-core factors: Qhat_x, Qhat_y, Qhat_y^T, Qhat_x^T
  int* d_err = nullptr;              // device flag: a bounded wait in a kernel timed out
  void* noalloc_scratch = nullptr;   // device address of the static scratch of sg_precond_noalloc
  unsigned long long* d_modemax = nullptr;   // P per-mode maxima of sg_statistics (allocated on first use)
  // launch shapes chosen by sg_autotune / sg_tune_set (0: built-in rule)
  int tune_cgs_bpsm = 0;             // CGS2 passes: grid of this many blocks per SM
  int tune_op_occ = 0;               // persistent complex64 operator: CTAs per SM (at most its occupancy)
  int tune_tc_bn = 0;                // transforms: output tile width (64 or 128; 256: the binary16
                                     // transforms in the paired 256-column form, the TF32 ones at 128)
  sgi::TcDevOperand tcW[4];          // binary16 factors for the 256-column form (h16 only)
  bool tc_wide = false;              // the binary16 transforms run the 256-column form
  int tune_tf32 = 0;                 // 1: the solver's transforms in TF32 even where the binary16 route exists
  double tune_us[3] = {0.0, 0.0, 0.0};   // measured: CGS2 step, operator, TF32 apply (microseconds)
  // host factors of the four tensor-core transforms (kept to rebuild them
  // for another tile width), their sizes and GEMM row counts
  std::vector<sgi::cd> tc_fac[4];
  int tc_dim[4] = {0, 0, 0, 0};
  long long tc_rows[4] = {0, 0, 0, 0};

  sgi::GmresWork gw;

  sgi::OpParams<double> op64() const;
  sgi::OpParams<float> op32() const;
};

namespace sgi {
// kernels / launchers (defined in the .cu files)
template <typename T>
cudaError_t launch_matvec(const sg_handle* h, const C2<T>* X, C2<T>* Y, cudaStream_t st,
                          const int* skip = nullptr);
template <typename T>
cudaError_t launch_rhs(const sg_handle* h, C2<T>* b, cudaStream_t st);

cudaError_t launch_tri_factor(int nsys, int len, const double2* diag, const double2* lam_shift,
                              const double* off, TriFactors<double> f64, TriFactors<float> f32,
                              int* d_bad, cudaStream_t st);
template <typename T>
cudaError_t launch_precond(const sg_handle* h, int which, const C2<T>* R, C2<T>* Z, cudaStream_t st,
                           const int* skip = nullptr, const double* in_scale = nullptr);

// FP32 apply of a 2D preconditioner with the fast-diagonalisation transforms
// in plain TF32 (relative error ~1e-3: a fixed but inexact preconditioner,
// used by flexible GMRES); cudaErrorNotSupported without that route.
cudaError_t launch_precond_tf32(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                                const int* skip, const double* in_scale);
// The same apply with transforms 2-4 on binary16 operands (kind::f16 MMAs)
// and binary16 intermediates: the same 11-bit significands as TF32, twice
// the K per copied stage.  The input is taken as normalised by in_scale (the
// solver's v_j = vscale_j V_j); without in_scale its norm is computed first.
cudaError_t launch_precond_f16(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                               const int* skip, const double* in_scale);
// Block partial sums of the input norm of the binary16 apply without in_scale.
constexpr int kFd16Blocks = 1024;
// The solver's fast apply: binary16 where available (and not switched off by
// the tuner), else TF32.
// The binary16 apply from a binary16 copy X16 (P my rows of mx4 pairs,
// read through xmap): Z = M^-1 (s X16) with s = *in_scale * oscale, which
// must turn the copy into sqrt(N) times the unit vector to precondition (the
// scale the binary16 transforms expect).
cudaError_t launch_precond_f16_copy(const sg_handle* h, int which, const void* X16, const CUtensorMap* xmap,
                                    float2* Z, cudaStream_t st, const int* skip, const double* in_scale,
                                    float oscale = 1.0f);
cudaError_t launch_precond_fast(const sg_handle* h, int which, const float2* R, float2* Z, cudaStream_t st,
                                const int* skip, const double* in_scale);

// One of the four plain-TF32 transforms of that apply on caller buffers.
cudaError_t fd_transform(const sg_handle* h, int which, int t, const float2* X, float2* Y, cudaStream_t st,
                         bool f16 = false);

template <typename T>
cudaError_t launch_precond_scratch(const sg_handle* h, int which, const C2<T>* R, C2<T>* Z, cudaStream_t st,
                                   C2<T>* tmp, C2<T>* tmp2);

// The coupled CSL matrix of Sec. 4 as a band, factored on first use
// (sg_host.cpp); SG_EUNSUPPORTED when its band is too wide.
sg_status ensure_csl_full(sg_handle* h, cudaStream_t st);
// Whether a preconditioner kind can be applied for this handle (the coupled
// CSL one is decided by ensure_csl_full).
bool prec_available(const sg_handle* h, sg_prec kind);

// Input and output widths of a warm-start network (mlp.cu).
void mlp_dims(const sg_mlp* m, int* in_dim, int* out_dim);

// Device address of the allocation-free entry point's static scratch on the
// current device (loads its module; called once per handle by sg_assemble).
cudaError_t noalloc_scratch_address(void** out);

// launch bookkeeping (sg_kernel_launches)
void note_launch();
void note_launches(long long n);      // graph replays (n kernels) and capture corrections (-n)
long long thread_launches();          // kernels noted by this host thread so far

// true if a register-resident complex64 matvec kernel exists for (s, r)
bool matvec_is_specialised(int s, int r);
// CTAs per SM that fit of the persistent complex64 operator kernel of this
// handle (0: it has none)
int matvec_special_occupancy(const sg_handle* h);

// (Re)builds the device operands of the four tensor-core transforms from
// the host factors, with tile width bn (0: the built-in rule per transform).
sg_status tc_build_operands(sg_handle* h, int bn);
// Times the CGS2 passes of Arnoldi step j (complex64) on the handle's
// workspace, whose contents it overwrites: mean microseconds over reps.
sg_status time_cgs_passes(sg_handle* h, sg_prec prec, int j, int reps, cudaStream_t st, double* us);
// Applies a CGS2 grid choice (blocks per SM, 0 = rule) to the handle and
// its workspace, dropping graphs captured with the old grid.
void set_cgs_blocks(sg_handle* h, int bpsm);
// Drops every graph captured from the handle's launches (after any change of
// its launch shapes, operands or preconditioner route).
void drop_graphs(sg_handle* h);

}  // namespace sgi
