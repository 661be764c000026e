// Batched scan (pq_batch_*): several plans, e.g. one per schema of a
// heterogeneous set of files, run as one unit.  Each plan gets its own
// stream (forked from the launch stream and joined back), so the plans'
// kernels overlap on the device; with PQ_SCAN_GRAPH the whole batch is
// captured once into one CUDA graph and every launch is a single graph
// launch.
#include <algorithm>
#include <cstring>

#include "engine.h"

using namespace pqe;

struct pq_batch {
  pq_ctx* ctx = nullptr;
  uint32_t flags = 0;
  std::vector<pq_plan*> plans;
  std::vector<std::vector<pq_column>> outs;
  std::vector<cudaStream_t> streams;  // one per plan
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t graph = nullptr;
};

namespace {

constexpr int kMaxBatchStreams = 16;

pq_status enqueue_batch(pq_batch* b, cudaStream_t s) {
  pq_ctx* ctx = b->ctx;
  cudaError_t e = cudaEventRecord(b->fork, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch fork");
  for (size_t i = 0; i < b->plans.size(); ++i) {
    cudaStream_t ps = b->streams[i % b->streams.size()];
    cudaStreamWaitEvent(ps, b->fork, 0);
    const pq_status st = scan_enqueue(b->plans[i], b->outs[i].data(), ps, &ps, 1, false);
    if (st != PQ_OK) return st;
    cudaEventRecord(b->join[i], ps);
  }
  for (size_t i = 0; i < b->plans.size(); ++i) cudaStreamWaitEvent(s, b->join[i], 0);
  return PQ_OK;
}

}  // namespace

extern "C" {

pq_status pq_batch_create(pq_ctx* ctx, int n_plans, pq_plan* const* plans, const pq_column* const* outs,
                          uint32_t flags, pq_batch** out) {
  if (!ctx || n_plans <= 0 || !plans || !outs || !out) return fail(ctx, PQ_ERR_INVALID_ARG, "pq_batch_create");
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "cudaSetDevice");
  auto b = std::make_unique<pq_batch>();
  b->ctx = ctx;
  b->flags = flags;
  for (int i = 0; i < n_plans; ++i) {
    if (!plans[i] || plans[i]->ctx != ctx || (!outs[i] && !plans[i]->outcols.empty()))
      return fail(ctx, PQ_ERR_INVALID_ARG, "pq_batch_create: bad plan or outputs");
    if (plans[i]->flags & (PQ_SCAN_TIMING | PQ_SCAN_GRAPH))
      return fail(ctx, PQ_ERR_INVALID_ARG, "pq_batch_create: plans must not carry TIMING or GRAPH");
    b->plans.push_back(plans[i]);
    b->outs.emplace_back(outs[i], outs[i] + plans[i]->outcols.size());
  }
  const int ns = std::min(n_plans, kMaxBatchStreams);
  b->streams.assign(ns, nullptr);
  b->join.assign(n_plans, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
  for (auto& st : b->streams) ok = ok && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (auto& ev : b->join) ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pq_batch_free(b.release());
    return fail(ctx, PQ_ERR_CUDA, "batch streams and events");
  }
  *out = b.release();
  return PQ_OK;
}

pq_status pq_batch_launch(pq_batch* b, void* stream) {
  if (!b) return PQ_ERR_INVALID_ARG;
  pq_ctx* ctx = b->ctx;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->flags & PQ_SCAN_GRAPH) {
    if (!b->graph) {
      // the plans' uploads are done before the capture (see scan_enqueue)
      for (pq_plan* p : b->plans)
        if (p->ready) {
          const cudaError_t e = cudaEventSynchronize(p->ready);
          if (e != cudaSuccess) return cuda_fail(ctx, e, "plan ready");
        }
      cudaStream_t cs = nullptr;
      cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "capture stream");
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(ctx, e, "batch capture");
      }
      const pq_status st = enqueue_batch(b, cs);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      if (st != PQ_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "batch capture");
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "batch graph instantiate");
    }
    cudaError_t e = cudaGraphLaunch(b->graph, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch graph launch");
    // the plans' completion events were recorded inside the capture; record
    // them again on the launch stream so that pq_scan_wait can use them
    for (pq_plan* p : b->plans) {
      e = cudaEventRecord(p->done, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "plan done event");
    }
  } else {
    const pq_status st = enqueue_batch(b, s);
    if (st != PQ_OK) return st;
  }
  const cudaError_t e = cudaEventRecord(b->done, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch done event");
  return PQ_OK;
}

pq_status pq_batch_wait(pq_batch* b) {
  if (!b) return PQ_ERR_INVALID_ARG;
  pq_ctx* ctx = b->ctx;
  const cudaError_t e = cudaEventSynchronize(b->done);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batch wait");
  for (pq_plan* p : b->plans) {
    pqi::DevStatus st;
    memcpy(&st, p->h_out.p, sizeof st);
    if (st.flags) return status_from_device(ctx, st);
  }
  return PQ_OK;
}

void pq_batch_free(pq_batch* b) {
  if (!b) return;
  cudaSetDevice(b->ctx->device);
  if (b->done) cudaEventSynchronize(b->done);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (auto ev : b->join)
    if (ev) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  delete b;
}

}  // extern "C"
