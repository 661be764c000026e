// pq_scan_host: the end-to-end call from host memory — files copied to the
// device, indexed, planned and scanned, columns copied back.
#include <string.h>

#include <algorithm>
#include <vector>

#include "engine.h"

using namespace pqe;

namespace {

struct HostScanGuard {
  pq_ctx* ctx;
  cudaStream_t s = nullptr;
  std::vector<void*> blocks;
  pq_index* idx = nullptr;
  pq_plan* plan = nullptr;
  ~HostScanGuard() {
    if (plan) pq_free_plan(plan);
    if (idx) pq_free_index(idx);
    if (s) cudaStreamSynchronize(s);
    for (void* b : blocks) ctx->pool.free(b);
    if (s) cudaStreamDestroy(s);
  }
  void* alloc(size_t n) {
    void* p = ctx->pool.alloc(n);
    if (p) blocks.push_back(p);
    return p;
  }
};

}  // namespace

extern "C" pq_status pq_scan_host(pq_ctx* ctx, const pq_file* host_files, int n_files, const pq_request* req,
                                  const pq_column* host_outs, pq_out_size* sizes) {
  if (!ctx || !host_files || n_files <= 0 || !req) return fail(ctx, PQ_ERR_INVALID_ARG, "pq_scan_host");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "cudaSetDevice");
  HostScanGuard g{ctx};
  if (cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(ctx, PQ_ERR_CUDA, "stream");
  std::vector<pq_file> dev(n_files);
  for (int f = 0; f < n_files; ++f) {
    if (!host_files[f].data && host_files[f].size) return fail(ctx, PQ_ERR_INVALID_ARG, "null host file");
    void* d = g.alloc(host_files[f].size + 64);
    if (!d) return fail(ctx, PQ_ERR_OOM, "device file buffer");
    if (cudaMemcpyAsync(d, host_files[f].data, host_files[f].size, cudaMemcpyHostToDevice, g.s) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "host-to-device copy");
    dev[f].data = d;
    dev[f].size = host_files[f].size;
  }
  pq_status st = pq_index_chunks(ctx, dev.data(), n_files, g.s, &g.idx);
  if (st != PQ_OK) return st;
  const int ncols = req->columns ? req->n_columns : g.idx->n_columns;
  std::vector<pq_out_size> szs(static_cast<size_t>(std::max(ncols, 1)));
  st = pq_plan_scan(ctx, g.idx, req, &g.plan, szs.data());
  if (st != PQ_OK) return st;
  if (sizes) memcpy(sizes, szs.data(), sizeof(pq_out_size) * ncols);
  if (!host_outs) return PQ_OK;
  std::vector<pq_column> douts(ncols);
  for (int c = 0; c < ncols; ++c) {
    const pq_out_size& z = szs[c];
    douts[c].values = z.values_bytes ? g.alloc(z.values_bytes) : nullptr;
    douts[c].validity = z.validity_bytes ? static_cast<uint32_t*>(g.alloc(z.validity_bytes)) : nullptr;
    douts[c].chars = z.chars_bytes ? g.alloc(z.chars_bytes) : nullptr;
    douts[c].chars_capacity = z.chars_bytes;
    if ((z.values_bytes && !douts[c].values) || (z.validity_bytes && !douts[c].validity) ||
        (z.chars_bytes && !douts[c].chars))
      return fail(ctx, PQ_ERR_OOM, "device output buffers");
    if (host_outs[c].chars_capacity < z.chars_bytes && z.type == PQ_TYPE_BYTE_ARRAY)
      return fail(ctx, PQ_ERR_CAPACITY, "host chars buffer smaller than chars_bytes");
  }
  st = pq_scan_columns(ctx, g.plan, douts.data(), g.s);
  if (st != PQ_OK) return st;
  std::vector<uint64_t> chars(ncols);
  st = pq_scan_wait(ctx, g.plan, g.s, chars.data());
  if (st != PQ_OK) return st;
  for (int c = 0; c < ncols; ++c) {
    const pq_out_size& z = szs[c];
    if (z.values_bytes && cudaMemcpyAsync(host_outs[c].values, douts[c].values, z.values_bytes,
                                          cudaMemcpyDeviceToHost, g.s) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "device-to-host copy");
    if (z.validity_bytes && cudaMemcpyAsync(host_outs[c].validity, douts[c].validity, z.validity_bytes,
                                            cudaMemcpyDeviceToHost, g.s) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "device-to-host copy");
    if (chars[c] && cudaMemcpyAsync(host_outs[c].chars, douts[c].chars, chars[c], cudaMemcpyDeviceToHost, g.s) !=
                        cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "device-to-host copy");
  }
  if (cudaStreamSynchronize(g.s) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "synchronize");
  return PQ_OK;
}
