// Batched solve of independent SG systems (sg_gmres_batched).
//
// Every system keeps its own device-resident GMRES state (the handle's
// workspace).  Two routes:
//  * one graph (mixed precision, device buffers, right or no
//    preconditioning, zero or per-system initial guesses): the whole batch is
//    one cudaGraphLaunch whose conditional nodes let the device take the
//    restart, refinement and convergence decisions (solver.cu,
//    sgi_batched_graph); the few systems still above tol after the graph's
//    unrolled refinement steps continue on the per-system route from their
//    current iterate, and a system whose guess is worse than zero (or whose
//    b is zero) is solved again there from the start;
//  * per system: each system runs sg_gmres on its own non-blocking CUDA
//    stream, driven by a small pool of host threads (each thread owns one
//    stream and takes the next unsolved system from a shared counter).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "sg_internal.h"

sg_status sgi_prepare_workspace(sg_handle* h, const sg_gmres_opts* opts);   // solver.cu
bool sgi_batched_graph_eligible(const sg_gmres_opts* opts, const void* const* x0, int count);
sg_status sgi_batched_graph(sg_handle* const* h, int count, const sg_gmres_opts* opts, const void* const* b,
                            void* const* x, const void* const* x0, sg_gmres_info* infos, void* stream,
                            std::vector<int>* pending, std::vector<int>* redo);

namespace {

// The per-system route over the entries `idx`; from_x: start each system
// from its current x (graph leftovers) instead of opts->x0 / x0[k].
sg_status run_pool(sg_handle* const* h, const std::vector<int>& idx, const sg_gmres_opts* opts, const void* const* b,
                   void* const* x, const void* const* x0, std::vector<sg_gmres_info>& inf,
                   std::vector<sg_status>& status, std::vector<std::string>& errs, int concurrency, void* stream,
                   bool from_x) {
  const int count = (int)idx.size();
  if (count == 0) return SG_OK;
  int dev = 0;
  SG_CUDA_TRY(cudaGetDevice(&dev));
  const int nthreads = std::max(1, std::min(count, concurrency <= 0 ? 16 : concurrency));
  cudaEvent_t ready;
  SG_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  {
    const cudaError_t e = cudaEventRecord(ready, (cudaStream_t)stream);
    if (e != cudaSuccess) {
      cudaEventDestroy(ready);
      return sgi::fail(SG_ECUDA, std::string("cudaEventRecord: ") + cudaGetErrorString(e));
    }
  }
  std::vector<cudaStream_t> streams(nthreads, nullptr);
  for (int t = 0; t < nthreads; ++t) {
    cudaError_t e = cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(streams[t], ready, 0);
    if (e != cudaSuccess) {
      for (int u = 0; u <= t; ++u)
        if (streams[u]) cudaStreamDestroy(streams[u]);
      cudaEventDestroy(ready);
      return sgi::fail(SG_ECUDA, std::string("stream set-up: ") + cudaGetErrorString(e));
    }
  }
  std::atomic<int> next{0};
  auto worker = [&](int t) {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      const int k = idx[i];
      sg_gmres_opts ok = *opts;
      if (from_x) {
        // continue where the graph left the system: what remains of the step
        // and refinement caps, from the current iterate as given
        const long long cap = opts->maxit > 0 ? opts->maxit : std::min<long long>(h[k]->N, 1 << 30);
        const int outer_cap = opts->max_outer > 0 ? opts->max_outer : 20;
        if (inf[k].iters >= cap || inf[k].outer >= outer_cap) {
          status[k] = SG_ENOTCONV;
          continue;
        }
        ok.maxit = (int)(cap - inf[k].iters);
        ok.max_outer = outer_cap - inf[k].outer;
        ok.x0 = x[k];
        ok.x0_policy = SG_X0_AS_GIVEN;
      } else if (x0) {
        ok.x0 = x0[k];
      }
      sg_gmres_info add{};
      status[k] = sg_gmres(h[k], &ok, b[k], x[k], &add, streams[t]);
      if (status[k] != SG_OK) errs[k] = sg_last_error();
      if (from_x) {
        inf[k].iters += add.iters;
        inf[k].outer += add.outer;
        inf[k].cycles += add.cycles;
        inf[k].relres = add.relres;
        inf[k].relres_prec = add.relres_prec;
        inf[k].status = add.status;
      } else {
        inf[k] = add;
      }
    }
  };
  // the systems are taken from a shared counter, so if a host thread cannot
  // be started the ones running (at least this one) solve the rest
  std::vector<std::thread> pool;
  for (int t = 1; t < nthreads; ++t) {
    try {
      pool.emplace_back(worker, t);
    } catch (...) {
      break;
    }
  }
  worker(0);
  for (auto& th : pool) th.join();
  for (auto s : streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  cudaEventDestroy(ready);
  return SG_OK;
}

}  // namespace

extern "C" sg_status sg_gmres_batched(sg_handle* const* h, int count, const sg_gmres_opts* opts,
                                      const void* const* b, void* const* x, const void* const* x0,
                                      sg_gmres_info* infos, int concurrency, void* stream) {
  return sgi::guarded([&]() -> sg_status {
    if (count < 0 || (count > 0 && (!h || !b || !x)) || !opts) return sgi::fail(SG_EINVAL, "bad batch arguments");
    if (count == 0) return SG_OK;
    for (int k = 0; k < count; ++k) {
      if (!h[k] || !b[k] || !x[k]) return sgi::fail(SG_EINVAL, "NULL handle or vector in batch entry " + std::to_string(k));
      for (int l = 0; l < k; ++l)
        if (h[l] == h[k]) return sgi::fail(SG_EINVAL, "the same handle appears twice in the batch");
    }
    // workspaces first: allocation would serialise the concurrent solves
    for (int k = 0; k < count; ++k) {
      sg_status s = sgi_prepare_workspace(h[k], opts);
      if (s != SG_OK) return s;
    }
    std::vector<sg_status> status(count, SG_OK);
    std::vector<sg_gmres_info> inf(count);
    std::vector<std::string> errs(count);
    std::vector<int> all(count);
    for (int k = 0; k < count; ++k) all[k] = k;
    bool done = false;
    if (concurrency >= 0 && sgi_batched_graph_eligible(opts, x0, count)) {
      std::vector<int> pending, redo;
      if (sgi_batched_graph(h, count, opts, b, x, x0, inf.data(), stream, &pending, &redo) == SG_OK) {
        for (int k = 0; k < count; ++k) status[k] = inf[k].status;
        for (int k : pending) status[k] = SG_OK;
        for (int k : redo) status[k] = SG_OK;
        sg_status s = run_pool(h, pending, opts, b, x, x0, inf, status, errs, concurrency, stream, true);
        if (s == SG_OK) s = run_pool(h, redo, opts, b, x, x0, inf, status, errs, concurrency, stream, false);
        if (s != SG_OK) return s;
        done = true;
      }
      // any failure to build or launch the graph leaves the systems untouched:
      // the per-system route below solves them all
    }
    if (!done) {
      sg_status s = run_pool(h, all, opts, b, x, x0, inf, status, errs, concurrency < 0 ? 0 : concurrency, stream,
                             false);
      if (s != SG_OK) return s;
    }
    if (infos)
      for (int k = 0; k < count; ++k) infos[k] = inf[k];
    sg_status result = SG_OK;
    for (int k = 0; k < count; ++k) {
      if (status[k] == SG_OK) continue;
      if (status[k] == SG_ENOTCONV) {
        if (result == SG_OK) {
          result = SG_ENOTCONV;
          sgi::set_error("batch entry " + std::to_string(k) + ": " + (errs[k].empty() ? "not converged" : errs[k]));
        }
      } else {
        sgi::set_error("batch entry " + std::to_string(k) + ": " + errs[k]);
        return status[k];
      }
    }
    return result;
  });
}
