// Batched solve of independent SG systems (sg_gmres_batched).
//
// Every system keeps its own device-resident GMRES state (the handle's
// workspace) and runs on its own non-blocking CUDA stream, so the kernels of
// different systems overlap on the GPU.  A small pool of host threads drives
// the streams (each thread owns one stream and takes the next unsolved
// system from a shared counter), which keeps the per-system host decisions
// (restart, refinement, convergence) off the critical path of the others.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "sg_internal.h"

sg_status sgi_prepare_workspace(sg_handle* h, const sg_gmres_opts* opts);   // solver.cu

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
    int dev = 0;
    SG_CUDA_TRY(cudaGetDevice(&dev));
    // workspaces first: allocation would serialise the concurrent solves
    for (int k = 0; k < count; ++k) {
      sg_status s = sgi_prepare_workspace(h[k], opts);
      if (s != SG_OK) return s;
    }
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
    std::vector<sg_status> status(count, SG_OK);
    std::vector<sg_gmres_info> inf(count);
    std::vector<std::string> errs(count);
    std::atomic<int> next{0};
    auto worker = [&](int t) {
      cudaSetDevice(dev);
      for (;;) {
        const int k = next.fetch_add(1);
        if (k >= count) break;
        sg_gmres_opts ok = *opts;
        if (x0) ok.x0 = x0[k];
        status[k] = sg_gmres(h[k], &ok, b[k], x[k], &inf[k], streams[t]);
        if (status[k] != SG_OK) errs[k] = sg_last_error();
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
    if (infos)
      for (int k = 0; k < count; ++k) infos[k] = inf[k];
    sg_status result = SG_OK;
    for (int k = 0; k < count; ++k) {
      if (status[k] == SG_OK) continue;
      if (status[k] == SG_ENOTCONV) {
        if (result == SG_OK) {
          result = SG_ENOTCONV;
          sgi::set_error("batch entry " + std::to_string(k) + ": " + errs[k]);
        }
      } else {
        sgi::set_error("batch entry " + std::to_string(k) + ": " + errs[k]);
        return status[k];
      }
    }
    return result;
  });
}
