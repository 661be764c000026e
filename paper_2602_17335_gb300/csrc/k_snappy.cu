// K1 — Snappy page decompression, one warp per page.
//
// Parquet compresses every page body separately with its chunk's codec
// (paper Section 2; Section 3 "No Unnecessary Compression" weighs its cost).
// A raw Snappy block is a ULEB128 length followed by elements chosen by the
// low two tag bits: a literal (length in the tag, or in 1-4 following
// bytes) or a copy of `length` bytes from `offset` bytes back in the output
// (1-, 2- or 4-byte offsets).  Copies are defined byte by byte, so an offset
// smaller than the length repeats a pattern; output byte i of such a copy is
// out[start - offset + (i mod offset)], which every lane computes on its own.
//
// Lane 0 parses a batch of up to 32 element headers (the tag stream is
// serial) into a per-warp shared-memory slot; then the warp executes the
// batch in order, all 32 lanes copying the bytes of one element at a time.
// Long literals and non-overlapping copies move 16-byte vectors (aligned
// loads funnel-shifted to the destination's alignment); copies out of the
// output use coherent loads, since other lanes wrote those bytes.
#include "dev_util.cuh"
#include "snappy_job.h"

namespace pqi {

constexpr int kSnappyWarps = 4;  // warps per block
constexpr uint32_t kRing = 8192;  // recent output kept in shared memory per warp (power of two)

__global__ void __launch_bounds__(32 * kSnappyWarps) k_snappy(const SnappyJob* __restrict__ jobs, int n_jobs,
                                                              DevStatus* st) {
  __shared__ uint32_t s_kind_len[kSnappyWarps][32];
  __shared__ uint32_t s_arg[kSnappyWarps][32];
  __shared__ uint8_t s_ring[kSnappyWarps][kRing];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = wid; j < n_jobs; j += nwarps) {
    const SnappyJob jb = jobs[j];
    if (jb.prefix > jb.src_len || jb.prefix > jb.dst_len) {
      if (lane == 0) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 1);
      continue;
    }
    warp_copy<true>(jb.dst, jb.src, jb.prefix, lane);  // V2 level bytes, never compressed
    if (jb.raw) {
      if (jb.src_len != jb.dst_len) {
        if (lane == 0) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 2);
        continue;
      }
      warp_copy<true>(jb.dst + jb.prefix, jb.src + jb.prefix, jb.src_len - jb.prefix, lane);
      __syncwarp();
      continue;
    }
    const uint8_t* in = jb.src + jb.prefix;
    const uint32_t in_len = jb.src_len - jb.prefix;
    uint8_t* out = jb.dst + jb.prefix;
    const uint32_t out_len = jb.dst_len - jb.prefix;
    uint64_t declared = 0;
    int pl = uleb([&](uint32_t k) { return static_cast<uint32_t>(__ldg(in + k)); }, 0, in_len, &declared);
    if (pl == 0 || declared != out_len) {
      if (lane == 0) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 3);
      continue;
    }
    uint32_t ip = static_cast<uint32_t>(pl);
    uint32_t op = 0;
    int bad = 0;
    // each element consumes >= 2 input bytes, so in_len bounds the batches
    for (uint32_t guard = 0; guard <= in_len && ip < in_len && !bad; ++guard) {
      int n_el = 0;
      if (lane == 0) {
        uint32_t p = ip, o = op;
        for (int e = 0; e < 32 && p < in_len; ++e) {
          uint32_t tag = __ldg(in + p++);
          uint32_t kind = tag & 3, len, arg;
          if (kind == 0) {
            uint32_t l = tag >> 2;
            if (l < 60) {
              len = l + 1;
            } else {
              uint32_t nb = l - 59;
              if (nb > in_len - p) { bad = 1; break; }
              uint32_t v = 0;
              for (uint32_t b = 0; b < nb; ++b) v |= static_cast<uint32_t>(__ldg(in + p + b)) << (8 * b);
              p += nb;
              if (v == 0xffffffffu) { bad = 1; break; }
              len = v + 1;
            }
            if (len > in_len - p) { bad = 1; break; }
            arg = p;
            p += len;
          } else if (kind == 1) {
            if (p >= in_len) { bad = 1; break; }
            len = 4 + ((tag >> 2) & 7);
            arg = ((tag >> 5) << 8) | __ldg(in + p);
            p += 1;
          } else if (kind == 2) {
            if (2 > in_len - p) { bad = 1; break; }
            len = (tag >> 2) + 1;
            arg = __ldg(in + p) | (static_cast<uint32_t>(__ldg(in + p + 1)) << 8);
            p += 2;
          } else {
            if (4 > in_len - p) { bad = 1; break; }
            len = (tag >> 2) + 1;
            arg = ld_le32_g(in + p);
            p += 4;
          }
          if (len > out_len - o || (kind != 0 && (arg == 0 || arg > o))) { bad = 1; break; }
          o += len;
          s_kind_len[w][e] = kind | (len << 2);
          s_arg[w][e] = arg;
          n_el = e + 1;
        }
        ip = p;
      }
      __syncwarp();
      n_el = __shfl_sync(0xffffffffu, n_el, 0);
      bad = __shfl_sync(0xffffffffu, bad, 0);
      ip = __shfl_sync(0xffffffffu, ip, 0);
      // Execute the batch.  Every output byte also goes to the warp's ring
      // of recent output in shared memory, so that back-references into the
      // last kRing bytes read shared memory instead of waiting on L2 for
      // bytes the warp has just stored.  Pass 1, in parallel: literals and
      // copies whose source lies wholly before the batch's first output
      // byte; short ones one lane each, long literals by the whole warp.
      // Pass 2, in order: copies that read output of this batch (or overlap
      // themselves).
      uint8_t* ring = s_ring[w];
      constexpr uint32_t RM = kRing - 1;
      uint32_t kl = 0, arg = 0;
      if (lane < n_el) {
        kl = s_kind_len[w][lane];
        arg = s_arg[w][lane];
      }
      const uint32_t kind = kl & 3, len = kl >> 2;
      uint32_t incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t o0 = op + incl - len;  // this lane's element output offset
      const uint32_t bend = op + __shfl_sync(0xffffffffu, incl, 31);
      // ring slots hold positions [ring_lo, bend) after this batch; writes of
      // positions below ring_lo are skipped (each slot has one writer) and
      // reads below it go to global memory
      const uint32_t ring_lo = bend > kRing ? bend - kRing : 0u;
      auto src_byte = [&](uint32_t pos, uint32_t first) -> uint8_t {
        return first >= ring_lo ? ring[pos & RM] : ld_src<false>(out + pos);
      };
      const bool valid = lane < n_el;
      const bool indep = valid && (kind == 0 || (arg >= len && o0 - arg + len <= op));
      const bool small = kind != 0 || len <= 32;
      if (indep && small) {
        if (kind == 0) {
          for (uint32_t i = 0; i < len; ++i) {
            const uint8_t b = __ldg(in + arg + i);
            out[o0 + i] = b;
            if (o0 + i >= ring_lo) ring[(o0 + i) & RM] = b;
          }
        } else {
          const uint32_t first = o0 - arg;
          for (uint32_t i = 0; i < len; ++i) {
            const uint8_t b = src_byte(first + i, first);
            out[o0 + i] = b;
            if (o0 + i >= ring_lo) ring[(o0 + i) & RM] = b;
          }
        }
      }
      for (uint32_t m = __ballot_sync(0xffffffffu, indep && !small); m; m &= m - 1) {
        const int e = __ffs(m) - 1;
        const uint32_t el = __shfl_sync(0xffffffffu, len, e);
        const uint32_t ea = __shfl_sync(0xffffffffu, arg, e), eo = __shfl_sync(0xffffffffu, o0, e);
        if (el > 512) {
          warp_copy<true>(out + eo, in + ea, el, lane);
          for (uint32_t i = (eo >= ring_lo ? 0u : ring_lo - eo) + lane; i < el; i += 32)
            ring[(eo + i) & RM] = __ldg(in + ea + i);
        } else {
          for (uint32_t i = lane; i < el; i += 32) {
            const uint8_t b = __ldg(in + ea + i);
            out[eo + i] = b;
            if (eo + i >= ring_lo) ring[(eo + i) & RM] = b;
          }
        }
      }
      __syncwarp();
      for (uint32_t m = __ballot_sync(0xffffffffu, valid && !indep); m; m &= m - 1) {
        const int e = __ffs(m) - 1;
        const uint32_t el = __shfl_sync(0xffffffffu, len, e);
        const uint32_t ea = __shfl_sync(0xffffffffu, arg, e), eo = __shfl_sync(0xffffffffu, o0, e);
        const uint32_t first = eo - ea;
        for (uint32_t i = lane; i < el; i += 32) {
          const uint32_t pos = ea >= el ? first + i : first + (i % ea);
          const uint8_t b = src_byte(pos, first);
          out[eo + i] = b;
          if (eo + i >= ring_lo) ring[(eo + i) & RM] = b;
        }
        __syncwarp();
      }
      op += __shfl_sync(0xffffffffu, incl, 31);
      __syncwarp();
    }
    if (lane == 0 && (bad || op != out_len || ip != in_len)) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 4);
    __syncwarp();
  }
}

void launch_snappy(const SnappyJob* jobs, int n_jobs, int n_sms, DevStatus* st, cudaStream_t s) {
  if (n_jobs <= 0) return;
  int warps = n_jobs < n_sms * 48 ? n_jobs : n_sms * 48;
  int blocks = (warps + kSnappyWarps - 1) / kSnappyWarps;
  k_snappy<<<blocks, 32 * kSnappyWarps, 0, s>>>(jobs, n_jobs, st);
}

}  // namespace pqi
