// Uneven batches: dbar_solve_batches.
//
// Many CGO problems on grids of different sizes (or with different potentials)
// need one plan per grid, and one plan's solves run one after the other.  The
// scheduler here runs the batches of different plans at the same time: one host
// thread per plan, each on a CUDA stream of its own, so that the small launches
// of a coarse grid overlap the long ones of a fine grid on the GPU instead of
// waiting for them.  Batches of the same plan keep their order.
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <thread>
#include <vector>

#include "plan_internal.h"

extern "C" dbar_status dbar_solve_batches(dbar_batch* b, int nbatch, void* stream) {
  if (nbatch < 0 || (nbatch > 0 && !b)) return dbar_internal_fail(DBAR_EINVAL, "dbar_solve_batches: bad batch list");
  for (int i = 0; i < nbatch; ++i)
    if (!b[i].plan) return dbar_internal_fail(DBAR_EINVAL, "dbar_solve_batches: batch without a plan");
  // work already queued on the caller's stream (inputs written there) comes first
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return dbar_internal_fail(DBAR_ECUDA, std::string("dbar_solve_batches: ") + cudaGetErrorString(cudaGetLastError()));
  std::map<dbar_plan_t, std::vector<int>> by_plan;  // batch indices per plan, in order
  for (int i = 0; i < nbatch; ++i) by_plan[b[i].plan].push_back(i);
  std::vector<std::string> msg(nbatch);
  int device = 0;
  cudaGetDevice(&device);
  std::vector<std::thread> workers;
  workers.reserve(by_plan.size());
  for (auto& kv : by_plan) {
    const std::vector<int>* idx = &kv.second;
    workers.emplace_back([b, idx, &msg, device] {
      cudaSetDevice(device);
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        for (int i : *idx) {
          b[i].status = DBAR_ECUDA;
          msg[i] = "dbar_solve_batches: stream creation failed";
        }
        return;
      }
      for (int i : *idx) {
        dbar_batch& q = b[i];
        q.status = dbar_solve_cgo(q.plan, q.Q, q.nk, q.k, q.x0, q.S_out, q.m_out, q.iters, q.resid, q.io_on_device,
                                  st);
        if (q.status != DBAR_OK) msg[i] = dbar_last_error();
      }
      cudaStreamDestroy(st);
    });
  }
  for (std::thread& t : workers) t.join();
  // the first failure (in batch order) decides; DBAR_ENOCONV only when nothing failed
  int noconv = -1;
  for (int i = 0; i < nbatch; ++i) {
    if (b[i].status == DBAR_OK) continue;
    if (b[i].status == DBAR_ENOCONV) {
      if (noconv < 0) noconv = i;
      continue;
    }
    return dbar_internal_fail(b[i].status, "batch " + std::to_string(i) + ": " + msg[i]);
  }
  if (noconv >= 0) return dbar_internal_fail(DBAR_ENOCONV, "batch " + std::to_string(noconv) + ": " + msg[noconv]);
  return DBAR_OK;
}
