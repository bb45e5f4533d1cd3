// Launch-shape tuning (sg_autotune, sg_tune_get, sg_tune_set): the CGS2
// grid, the persistent operator's CTAs per SM and the transform tile width
// (64, 128, or the paired 256-column form of the binary16 transforms) are timed on the handle's own problem with CUDA events and the fastest of
// each is kept in the handle.  The candidates change no arithmetic of the
// operator or the transforms (every output element is formed by one thread
// or one MMA tile whatever the shape); the CGS2 grid changes only the order
// in which block sums of the inner products are added.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sg_internal.h"

sg_status sgi_prepare_workspace(sg_handle* h, const sg_gmres_opts* opts);   // solver.cu

namespace {

using namespace sgi;

constexpr int TUNE_REPS = 10;

// Mean time of fn() over reps launches after two warm-up calls (microseconds).
template <typename F>
sg_status time_us(cudaStream_t st, int reps, F&& fn, double* us) {
  for (int r = 0; r < 2; ++r) SG_CUDA_TRY(fn());
  cudaEvent_t e0, e1;
  SG_CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e) {
    cudaEventDestroy(e0);
    return fail(SG_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
  }
  e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && !e; ++r) e = fn();
  if (!e) e = cudaEventRecord(e1, st);
  if (!e) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e) return fail(SG_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
  *us = 1000.0 * ms / reps;
  return SG_OK;
}

void fill(const sg_handle* h, sg_tune* t) {
  t->cgs_blocks_per_sm = h->tune_cgs_bpsm;
  t->op_ctas_per_sm = h->tune_op_occ;
  t->tc_tile_n = h->tune_tc_bn;
  t->tf32_transforms = h->tune_tf32;
  t->cgs_us = h->tune_us[0];
  t->op_us = h->tune_us[1];
  t->apply_us = h->tune_us[2];
}

}  // namespace

extern "C" sg_status sg_tune_get(const sg_handle* h, sg_tune* out) {
  return guarded([&]() -> sg_status {
    if (!h || !out) return fail(SG_EINVAL, "NULL argument");
    fill(h, out);
    return SG_OK;
  });
}

extern "C" sg_status sg_tune_set(sg_handle* h, const sg_tune* t) {
  return guarded([&]() -> sg_status {
    if (!h || !t) return fail(SG_EINVAL, "NULL argument");
    if (t->cgs_blocks_per_sm < 0 || t->cgs_blocks_per_sm > 8) return fail(SG_EINVAL, "cgs_blocks_per_sm must be 0 .. 8");
    if (t->op_ctas_per_sm < 0 || t->op_ctas_per_sm > 16) return fail(SG_EINVAL, "op_ctas_per_sm must be 0 .. 16");
    if (t->tc_tile_n != 0 && t->tc_tile_n != 64 && t->tc_tile_n != 128 && t->tc_tile_n != 256)
      return fail(SG_EINVAL, "tc_tile_n must be 0, 64, 128 or 256");
    if (t->tc_tile_n == 256 && !h->fd16)
      return fail(SG_EUNSUPPORTED, "tc_tile_n 256 is the binary16 transforms' form; this problem has none");
    if (t->tf32_transforms != 0 && t->tf32_transforms != 1) return fail(SG_EINVAL, "tf32_transforms must be 0 or 1");
    if (t->tc_tile_n != h->tune_tc_bn && h->fd) {
      sg_status s = tc_build_operands(h, t->tc_tile_n);
      if (s != SG_OK) return s;
    }
    const int tf32 = h->fd16 ? t->tf32_transforms : 0;
    if (tf32 != h->tune_tf32 || t->op_ctas_per_sm != h->tune_op_occ) drop_graphs(h);   // captured shapes
    h->tune_tc_bn = h->fd ? t->tc_tile_n : 0;
    h->tune_tf32 = tf32;
    h->tune_op_occ = t->op_ctas_per_sm;
    set_cgs_blocks(h, t->cgs_blocks_per_sm);
    return SG_OK;
  });
}

extern "C" sg_status sg_autotune(sg_handle* h, int restart, sg_tune* out, void* stream) {
  return guarded([&]() -> sg_status {
    if (!h) return fail(SG_EINVAL, "NULL handle");
    cudaStream_t st = (cudaStream_t)stream;
    sg_gmres_opts o{};
    o.restart = restart <= 0 ? 30 : restart;
    o.mode = SG_MIXED;
    o.prec = SG_PREC_MEAN;
    sg_status s = sgi_prepare_workspace(h, &o);
    if (s != SG_OK) return s;
    drop_graphs(h);   // the shapes change while they are timed
    GmresWork& w = h->gw;
    const long long N = h->N;
    float2* V0 = reinterpret_cast<float2*>(w.V);
    float2* V1 = V0 + N;
    // 1. CGS2 grid, timed at the middle step of a cycle
    {
      const int j = std::max(0, std::min(w.restart - 1, o.restart / 2));
      const sg_prec pk = prec_available(h, SG_PREC_MEAN) ? SG_PREC_MEAN : SG_PREC_NONE;
      double best = 0.0;
      int choice = 0;
      for (int bpsm : {2, 3, 4, 6, 8}) {
        set_cgs_blocks(h, bpsm);
        double us = 0.0;
        s = time_cgs_passes(h, pk, j, TUNE_REPS, st, &us);
        if (s != SG_OK) return s;
        if (choice == 0 || us < best) {
          best = us;
          choice = bpsm;
        }
      }
      set_cgs_blocks(h, choice);
      h->tune_us[0] = best;
    }
    // 2. CTAs per SM of the persistent complex64 operator
    h->tune_us[1] = 0.0;
    {
      SG_CUDA_TRY(cudaMemsetAsync(V0, 0, (size_t)N * sizeof(float2), st));
      const int occ = matvec_special_occupancy(h);
      double best = 0.0;
      int choice = 0;
      for (int c = 1; c <= std::max(occ, 1); ++c) {
        if (occ > 0) h->tune_op_occ = c;
        double us = 0.0;
        s = time_us(st, TUNE_REPS, [&]() { return launch_matvec<float>(h, V0, V1, st); }, &us);
        if (s != SG_OK) return s;
        if (c == 1 || us < best) {
          best = us;
          choice = occ > 0 ? c : 0;
        }
      }
      h->tune_op_occ = choice;
      h->tune_us[1] = best;
    }
    // 3. tile width and precision (binary16 where it exists, TF32) of the
    // transforms of the cycles' preconditioner (2D separable problems); the
    // input is scaled to unit norm as in the cycles.  (A back-to-back loop of
    // the complex64-input apply times its TF32 transform 1 as the dependent
    // launch of the previous apply's transform 4, a sequence the cycles never
    // run; measured that way the 256-column form came out no faster than the
    // 128-column one, although it saves ~40 us per transform in the cycles.)
    h->tune_us[2] = 0.0;
    if (h->fd) {
      double* unit = nullptr;   // a unit input scale on the device
      const double one = 1.0;
      SG_CUDA_TRY(cudaMalloc((void**)&unit, sizeof(double)));
      struct Free {
        double* p;
        ~Free() { cudaFree(p); }
      } free_unit{unit};
      SG_CUDA_TRY(cudaMemcpy(unit, &one, sizeof(double), cudaMemcpyHostToDevice));
      // the apply as an Arnoldi step j >= 1 of the flexible cycles runs it: in
      // binary16 from the workspace's binary16 copy of the basis vector where
      // the workspace has one, else from the complex64 vector
      auto cycle_apply = [&]() -> cudaError_t {
        if (h->fd16 && !h->tune_tf32 && w.V16)
          return launch_precond_f16_copy(h, 0, w.V16, &w.v16map, V1, st, nullptr, unit);
        return launch_precond_fast(h, 0, V0, V1, st, nullptr, unit);
      };
      double best = 0.0;
      int choice = 0, tf32 = 0, last = 0;
      for (int bn : {64, 128, 256}) {
        // 256: the paired binary16 form (TF32 transforms stay at 128)
        if (bn == 256 && !(h->fd16 && tc_wide_available())) continue;
        s = tc_build_operands(h, bn);
        if (s != SG_OK) return s;
        last = bn;
        for (int use_tf32 : {0, 1}) {
          if (!use_tf32 && !h->fd16) continue;
          if (use_tf32 && bn == 256) continue;
          h->tune_tf32 = use_tf32;
          double us = 0.0;
          s = time_us(st, TUNE_REPS, [&]() { return cycle_apply(); }, &us);
          if (s != SG_OK) return s;
          if (choice == 0 || us < best) {
            best = us;
            choice = bn;
            tf32 = use_tf32;
          }
        }
      }
      if (choice != last) {
        s = tc_build_operands(h, choice);
        if (s != SG_OK) return s;
      }
      h->tune_tc_bn = choice;
      h->tune_tf32 = tf32;
      h->tune_us[2] = best;
    }
    SG_CUDA_TRY(cudaStreamSynchronize(st));
    if (out) fill(h, out);
    return SG_OK;
  });
}
