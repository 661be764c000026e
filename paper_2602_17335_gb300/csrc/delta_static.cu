// pq_delta_decode_static: one DELTA_BINARY_PACKED stream decoded without any
// device allocation.  All scratch (status, the one-page plan, region tables,
// block positions and bases) lives in a fixed device array of this file;
// its address is looked up once per device and handed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "decode_job.h"
#include "engine.h"

namespace {

constexpr int kMaxDevices = 64;

// Fixed scratch of pq_delta_decode_static (pqi::DS_SCRATCH_BYTES, about
// 1.3 MB).  Shared by every call on a device, so calls must not overlap.
static __device__ __align__(256) uint8_t g_delta_scratch[pqi::DS_SCRATCH_BYTES];

std::mutex g_mu;
uint8_t* g_scratch_addr[kMaxDevices] = {};

// Set-up, once per device, with that device current.
pq_status scratch_for(pq_ctx* ctx, uint8_t** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[ctx->device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_delta_scratch);
    if (e != cudaSuccess) return pqe::cuda_fail(ctx, e, "cudaGetSymbolAddress of the DELTA scratch");
    g_scratch_addr[ctx->device] = static_cast<uint8_t*>(p);
  }
  *out = g_scratch_addr[ctx->device];
  return PQ_OK;
}

}  // namespace

extern "C" pq_status pq_delta_decode_static(pq_ctx* ctx, const void* d_stream, uint64_t stream_len, pq_type type,
                                            int64_t n_values, void* d_values, void* stream_ptr) {
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  if (!ctx) return PQ_ERR_INVALID_ARG;
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return pqe::fail(ctx, PQ_ERR_INVALID_ARG, "device id out of range for the fixed DELTA scratch");
  if (type != PQ_TYPE_INT32 && type != PQ_TYPE_INT64)
    return pqe::fail(ctx, PQ_ERR_INVALID_ARG, "DELTA_BINARY_PACKED decodes INT32 or INT64 only");
  if (!d_stream || stream_len == 0 || n_values < 0 || (n_values > 0 && !d_values))
    return pqe::fail(ctx, PQ_ERR_INVALID_ARG, "null stream or output, empty stream, or negative count");
  if (stream_len > pqi::DS_MAX_STREAM || n_values > pqi::DS_MAX_VALUES)
    return pqe::fail(ctx, PQ_ERR_CAPACITY,
                     "stream exceeds the fixed scratch of pq_delta_decode_static (at most 1 MiB of stream "
                     "and 4194305 values)");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return pqe::cuda_fail(ctx, e, "cudaSetDevice");
  uint8_t* scratch = nullptr;
  const pq_status s = scratch_for(ctx, &scratch);
  if (s != PQ_OK) return s;
  pqi::launch_delta_static(scratch, static_cast<const uint8_t*>(d_stream), static_cast<uint32_t>(stream_len),
                           type == PQ_TYPE_INT32 ? pqi::T_INT32 : pqi::T_INT64, static_cast<int32_t>(n_values),
                           d_values, stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) return pqe::cuda_fail(ctx, e, "DELTA decode launch");
  pqi::DevStatus st{};
  e = cudaMemcpyAsync(&st, scratch + pqi::DS_OFF_STATUS, sizeof st, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return pqe::cuda_fail(ctx, e, "DELTA decode");
  if (!st.flags) return PQ_OK;
  if (st.flags & pqi::DERR_TIMEOUT) return pqe::fail(ctx, PQ_ERR_TIMEOUT, "DELTA decode: a bounded wait ran out");
  if (st.flags & pqi::DERR_UNSUPPORTED)
    return pqe::fail(ctx, PQ_ERR_UNSUPPORTED, "DELTA decode: stream header outside the supported subset");
  return pqe::fail(ctx, PQ_ERR_CORRUPT, "DELTA decode: corrupt stream or value count mismatch");
}
