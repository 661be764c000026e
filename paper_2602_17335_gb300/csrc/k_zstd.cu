// Zstandard page decompression (the codec the paper's Section 2 lists beside
// Snappy): one thread block per page, whose first thread runs the decoding
// core of zstd_dec.cuh with its tables in shared memory.  The page jobs
// have the Snappy jobs' layout (verbatim V2 level prefix, then the frame).
// Jobs of another codec are skipped (the Snappy kernel runs over the same
// job list).
#include "dev_util.cuh"
#include "snappy_job.h"
#include "zstd_dec.cuh"

namespace pqi {
namespace {

__global__ void __launch_bounds__(32) k_zstd(const SnappyJob* __restrict__ jobs, int n_jobs, DevStatus* st) {
  __shared__ ZState z;
  for (int j = blockIdx.x; j < n_jobs; j += gridDim.x) {
    const SnappyJob jb = jobs[j];
    if (jb.codec != CODEC_ZSTD) continue;
    if (threadIdx.x == 0) {
      int rc = 0;
      if (jb.prefix > jb.src_len || jb.prefix > jb.dst_len) {
        rc = ZE_TRUNC;
      } else {
        for (uint32_t i = 0; i < jb.prefix; ++i) jb.dst[i] = jb.src[i];
        if (jb.raw) {
          if (jb.src_len != jb.dst_len) rc = ZE_SIZE;
          else
            for (uint32_t i = jb.prefix; i < jb.src_len; ++i) jb.dst[i] = jb.src[i];
        } else {
          rc = zstd_decode(jb.src + jb.prefix, jb.src_len - jb.prefix, jb.dst + jb.prefix, jb.dst_len - jb.prefix, &z);
        }
      }
      if (rc) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 100 + rc);
    }
    __syncthreads();
  }
}

}  // namespace

void launch_zstd(const SnappyJob* jobs, int n_jobs, int n_sms, DevStatus* st, cudaStream_t s) {
  if (n_jobs <= 0) return;
  const int grid = n_jobs < 8 * n_sms ? n_jobs : 8 * n_sms;
  k_zstd<<<grid, 32, 0, s>>>(jobs, n_jobs, st);
}

}  // namespace pqi
