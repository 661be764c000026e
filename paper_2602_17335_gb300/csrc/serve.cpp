// Continuous-batching scan server (pq_serve_*).
//
// Requests name columns and a row range of one index; the range wraps
// cyclically over the indexed rows.  At submit the host half of the plan is
// built, which gives the request's device bytes (outputs + plan scratch);
// a request that alone exceeds the budget is refused.  A scheduler thread
// admits queued requests first come, first served, whenever a slot (a CUDA
// stream with its own column branches) is free and the budget has room, so
// requests that arrive while others run start as soon as memory and a slot
// free up, and their kernels overlap on the device.  Completion is observed
// through each plan's event.  Dictionaries of every chunk are decoded once
// at creation and stay resident; the page index is the caller's index.
// Outputs stay allocated (and counted against the budget) until the caller
// releases the ticket.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "engine.h"

using namespace pqe;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kSlotBranches = 4;

struct Req {
  uint64_t ticket = 0;
  std::unique_ptr<pq_plan> plan;
  std::vector<pq_out_size> sizes;
  std::vector<pq_column> outs;
  std::vector<void*> bufs;
  uint64_t out_bytes = 0, plan_bytes = 0;
  Clock::time_point t_submit, t_admit, t_done;
  pq_status status = PQ_OK;
  int state = 0;  // 0 queued, 1 on the device, 2 finished
  bool launched = false;
  uint64_t decoded = 0;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaStream_t br[kSlotBranches] = {};
  Req* req = nullptr;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct pq_server {
  pq_ctx* ctx = nullptr;
  Clock::time_point t_create = Clock::now();  // origin of the results' admit / done times
  pq_index* idx = nullptr;
  pq_serve_config cfg{};
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  uint64_t used = 0;  // budget bytes held by admitted and unreleased requests
  std::vector<Slot> slots;
  std::thread th;
};

namespace {

void free_outputs(pq_ctx* ctx, Req* r) {
  for (void* p : r->bufs) ctx->pool.free(p);
  r->bufs.clear();
}

// Device half of a request: plan upload, outputs from the pool, scan
// enqueue on the slot.  Runs on the scheduler thread.
pq_status launch(pq_server* srv, Req* r, Slot& slot) {
  pq_ctx* ctx = srv->ctx;
  std::lock_guard<std::mutex> lk(ctx->mu);
  pq_status st = plan_upload(r->plan.get());
  if (st != PQ_OK) return st;
  r->outs.assign(r->sizes.size(), pq_column{});
  for (size_t i = 0; i < r->sizes.size(); ++i) {
    const auto& z = r->sizes[i];
    auto take = [&](uint64_t n) -> void* {
      void* p = ctx->pool.alloc(std::max<uint64_t>(n, 16));
      if (p) r->bufs.push_back(p);
      return p;
    };
    r->outs[i].values = take(z.values_bytes);
    if (!r->outs[i].values) return fail(ctx, PQ_ERR_OOM, "serving output");
    if (z.optional) {
      r->outs[i].validity = static_cast<uint32_t*>(take(z.validity_bytes));
      if (!r->outs[i].validity) return fail(ctx, PQ_ERR_OOM, "serving output");
    }
    if (z.type == PQ_TYPE_BYTE_ARRAY) {
      r->outs[i].chars = static_cast<uint8_t*>(take(z.chars_bytes));
      r->outs[i].chars_capacity = z.chars_bytes;
      if (!r->outs[i].chars) return fail(ctx, PQ_ERR_OOM, "serving output");
    }
  }
  return scan_enqueue(r->plan.get(), r->outs.data(), slot.s, slot.br, kSlotBranches, false);
}

// Status and string sizes of a finished request; frees its plan.
void finish(pq_server* srv, Req* r) {
  pq_plan* plan = r->plan.get();
  pqi::DevStatus st;
  memcpy(&st, plan->h_out.p, sizeof st);
  uint64_t decoded = 0;
  size_t j = 0;
  for (size_t i = 0; i < r->sizes.size(); ++i) {
    auto& z = r->sizes[i];
    if (z.type == PQ_TYPE_BYTE_ARRAY) {
      int64_t v;
      memcpy(&v, plan->h_out.p + sizeof(pqi::DevStatus) + 8 * j, 8);
      z.chars_bytes = static_cast<uint64_t>(v);
      ++j;
    }
    decoded += z.values_bytes + z.validity_bytes + z.chars_bytes;
  }
  r->decoded = decoded;
  {
    std::lock_guard<std::mutex> lk(srv->ctx->mu);
    r->status = status_from_device(srv->ctx, st);
  }
  pq_free_plan(r->plan.release());
}

void scheduler(pq_server* srv) {
  cudaSetDevice(srv->ctx->device);
  for (;;) {
    std::vector<std::pair<Req*, int>> admit;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      if (srv->stop) break;
      const auto now = Clock::now();
      if (srv->cfg.timeout_ms > 0) {
        for (auto it = srv->queue.begin(); it != srv->queue.end();) {
          Req* r = *it;
          if (ms_between(r->t_submit, now) > srv->cfg.timeout_ms) {
            r->status = PQ_ERR_TIMEOUT;
            r->state = 2;
            r->t_admit = r->t_done = now;
            r->plan.reset();
            it = srv->queue.erase(it);
            srv->cv.notify_all();
          } else {
            ++it;
          }
        }
      }
      while (!srv->queue.empty()) {
        Req* r = srv->queue.front();
        int free_slot = -1;
        for (size_t k = 0; k < srv->slots.size(); ++k)
          if (!srv->slots[k].req) {
            free_slot = static_cast<int>(k);
            break;
          }
        if (free_slot < 0 || srv->used + r->out_bytes + r->plan_bytes > srv->cfg.budget_bytes) break;
        srv->queue.pop_front();
        srv->used += r->out_bytes + r->plan_bytes;
        r->state = 1;
        r->t_admit = now;
        srv->slots[free_slot].req = r;
        admit.emplace_back(r, free_slot);
      }
    }
    for (auto& [r, k] : admit) {
      const pq_status st = launch(srv, r, srv->slots[k]);
      if (st != PQ_OK) {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (r->plan) {
          cudaStreamSynchronize(srv->slots[k].s);
          pq_free_plan(r->plan.release());
        }
        free_outputs(srv->ctx, r);
        srv->used -= r->out_bytes + r->plan_bytes;
        r->status = st;
        r->state = 2;
        r->t_done = Clock::now();
        srv->slots[k].req = nullptr;
        srv->cv.notify_all();
      } else {
        r->launched = true;
      }
    }
    bool busy = false;
    for (auto& slot : srv->slots) {
      Req* r = slot.req;
      if (!r || !r->launched) continue;
      const cudaError_t q = cudaEventQuery(r->plan->done);
      if (q == cudaErrorNotReady) {
        busy = true;
        continue;
      }
      if (q != cudaSuccess) cudaGetLastError();
      finish(srv, r);
      std::lock_guard<std::mutex> lk(srv->mu);
      srv->used -= r->plan_bytes;  // outputs stay held until release
      r->t_done = Clock::now();
      r->state = 2;
      slot.req = nullptr;
      srv->cv.notify_all();
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->stop) break;
    if (busy || !admit.empty())
      srv->cv.wait_for(lk, std::chrono::microseconds(20));
    else
      srv->cv.wait_for(lk, std::chrono::milliseconds(srv->queue.empty() ? 5 : 1));
  }
}

// Decodes every chunk's dictionary once (a one-row scan of every row group
// with resident dictionaries), so requests never decode dictionaries.
pq_status warm_dictionaries(pq_server* srv) {
  pq_ctx* ctx = srv->ctx;
  pq_index* idx = srv->idx;
  std::vector<int64_t> firsts(idx->chunk_first_row.begin(), idx->chunk_first_row.end());
  std::sort(firsts.begin(), firsts.end());
  firsts.erase(std::unique(firsts.begin(), firsts.end()), firsts.end());
  std::vector<RowSeg> segs;
  for (int64_t f : firsts)
    if (f < idx->num_rows) segs.push_back(RowSeg{f, f + 1, static_cast<int64_t>(segs.size())});
  if (segs.empty()) return PQ_OK;
  std::vector<int32_t> cols(idx->n_columns);
  for (int i = 0; i < idx->n_columns; ++i) cols[i] = i;
  Req r;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    pq_status st = plan_build(ctx, idx, cols, segs, static_cast<int64_t>(segs.size()), PQ_SCAN_RESIDENT_DICT, &r.plan);
    if (st != PQ_OK) return st;
  }
  r.sizes = r.plan->sizes;
  pq_status st = launch(srv, &r, srv->slots[0]);
  if (st == PQ_OK) {
    cudaStreamSynchronize(srv->slots[0].s);
    finish(srv, &r);
    st = r.status;
  } else if (r.plan) {
    cudaStreamSynchronize(srv->slots[0].s);
    pq_free_plan(r.plan.release());
  }
  free_outputs(ctx, &r);
  return st;
}

void destroy_slots(pq_server* srv) {
  for (auto& s : srv->slots) {
    if (s.s) {
      cudaStreamSynchronize(s.s);
      cudaStreamDestroy(s.s);
    }
    for (auto& b : s.br)
      if (b) {
        cudaStreamSynchronize(b);
        cudaStreamDestroy(b);
      }
  }
  srv->slots.clear();
}

}  // namespace

extern "C" {

pq_status pq_serve_create(pq_ctx* ctx, pq_index* idx, const pq_serve_config* cfg, pq_server** out) {
  if (!ctx || !idx || !cfg || !out || cfg->slots <= 0 || cfg->budget_bytes == 0)
    return fail(ctx, PQ_ERR_INVALID_ARG, "pq_serve_create: bad arguments");
  *out = nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "cudaSetDevice");
  auto srv = std::make_unique<pq_server>();
  srv->ctx = ctx;
  srv->idx = idx;
  srv->cfg = *cfg;
  srv->slots.resize(cfg->slots);
  for (auto& s : srv->slots) {
    bool ok = cudaStreamCreateWithFlags(&s.s, cudaStreamNonBlocking) == cudaSuccess;
    for (auto& b : s.br) ok = ok && cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      destroy_slots(srv.get());
      return fail(ctx, PQ_ERR_CUDA, "serving streams");
    }
  }
  const pq_status st = warm_dictionaries(srv.get());
  if (st != PQ_OK) {
    destroy_slots(srv.get());
    return st;
  }
  pq_server* p = srv.release();
  p->th = std::thread(scheduler, p);
  *out = p;
  return PQ_OK;
}

pq_status pq_serve_submit(pq_server* srv, const pq_serve_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return PQ_ERR_INVALID_ARG;
  pq_ctx* ctx = srv->ctx;
  pq_index* idx = srv->idx;
  if (!req->columns || req->n_columns <= 0 || req->row_begin < 0 || req->row_count <= 0 || idx->num_rows <= 0)
    return fail(ctx, PQ_ERR_INVALID_ARG, "pq_serve_submit: empty or negative request");
  std::vector<int32_t> cols(req->columns, req->columns + req->n_columns);
  for (int32_t c : cols)
    if (c < 0 || c >= idx->n_columns) return fail(ctx, PQ_ERR_INVALID_ARG, "pq_serve_submit: column id out of range");
  // the row range wraps cyclically over the indexed rows
  std::vector<RowSeg> segs;
  int64_t rb = req->row_begin % idx->num_rows, left = req->row_count, out0 = 0;
  while (left > 0) {
    const int64_t take = std::min(idx->num_rows - rb, left);
    segs.push_back(RowSeg{rb, rb + take, out0});
    out0 += take;
    left -= take;
    rb = 0;
  }
  auto r = std::make_unique<Req>();
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    const pq_status st = plan_build(ctx, idx, cols, segs, req->row_count, PQ_SCAN_RESIDENT_DICT, &r->plan);
    if (st != PQ_OK) return st;
  }
  r->sizes = r->plan->sizes;
  for (const auto& z : r->sizes) r->out_bytes += std::max<uint64_t>(z.values_bytes, 16) +
                                                  (z.optional ? std::max<uint64_t>(z.validity_bytes, 16) : 0) +
                                                  (z.type == PQ_TYPE_BYTE_ARRAY ? std::max<uint64_t>(z.chars_bytes, 16) : 0);
  r->plan_bytes = r->plan->device_bytes;
  if (r->out_bytes + r->plan_bytes > srv->cfg.budget_bytes)
    return fail(ctx, PQ_ERR_BUDGET, "request needs more device memory than the serving budget");
  std::lock_guard<std::mutex> lk(srv->mu);
  r->ticket = srv->next_ticket++;
  *ticket = r->ticket;
  srv->queue.push_back(r.get());
  srv->reqs.emplace(r->ticket, std::move(r));
  srv->cv.notify_all();
  return PQ_OK;
}

pq_status pq_serve_poll(pq_server* srv, uint64_t ticket, pq_serve_result* out, int* done) {
  if (!srv || !out || !done) return PQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return PQ_ERR_INVALID_ARG;
  Req* r = it->second.get();
  *done = r->state == 2 ? 1 : 0;
  memset(out, 0, sizeof *out);
  if (!*done) return PQ_OK;
  out->status = r->status;
  out->n_columns = static_cast<int32_t>(r->sizes.size());
  out->columns = r->status == PQ_OK ? r->outs.data() : nullptr;
  out->sizes = r->sizes.data();
  out->queue_ms = ms_between(r->t_submit, r->t_admit);
  out->latency_ms = ms_between(r->t_submit, r->t_done);
  out->decoded_bytes = r->decoded;
  out->admit_ms = ms_between(srv->t_create, r->t_admit);
  out->done_ms = ms_between(srv->t_create, r->t_done);
  return PQ_OK;
}

pq_status pq_serve_release(pq_server* srv, uint64_t ticket) {
  if (!srv) return PQ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end() || it->second->state != 2) return PQ_ERR_INVALID_ARG;
  Req* r = it->second.get();
  if (!r->bufs.empty()) {
    free_outputs(srv->ctx, r);
    srv->used -= r->out_bytes;
  }
  srv->reqs.erase(it);
  srv->cv.notify_all();
  return PQ_OK;
}

void pq_serve_destroy(pq_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    srv->cv.notify_all();
  }
  if (srv->th.joinable()) srv->th.join();
  cudaSetDevice(srv->ctx->device);
  for (auto& s : srv->slots) {
    if (s.s) cudaStreamSynchronize(s.s);
    if (s.req && s.req->plan) pq_free_plan(s.req->plan.release());
  }
  for (auto& kv : srv->reqs) free_outputs(srv->ctx, kv.second.get());
  destroy_slots(srv);
  delete srv;
}

}  // extern "C"
