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
// The compressed page streams through two shared-memory windows filled by
// the bulk-copy engine (the next window is in flight while the current one
// is parsed).  Lane 0 parses up to 32 element headers from the window (the
// tag stream is serial); the warp then executes the batch into a ring of
// recent output in shared memory -- literals and copies whose source lies
// before the batch in parallel, one element per lane (long ones by the whole
// warp), copies that read output of the same batch in order -- and writes
// the batch's output bytes to global memory with 16-byte stores.  Literals
// longer than the ring go straight from the input to the output as
// 16-byte vector copies.  Copy sources older than the ring are read back
// from the output with coherent loads (this warp wrote them).
#include "dev_util.cuh"
#include "snappy_job.h"

namespace pqi {

constexpr int kSnappyWarps = 4;     // warps per block
constexpr uint32_t kRing = 8192;    // recent output kept in shared memory per warp (power of two)
constexpr uint32_t kWin = 4096;     // input window (two per warp)
constexpr uint32_t kBatchOut = kRing / 2;  // output bytes of one batch assembled in the ring

struct SnWarp {
  uint64_t bar[2];
  uint32_t kl[32];   // kind | len << 2
  uint32_t arg[32];  // literal: input offset; copy: back offset
  uint8_t win[2][kWin + 16];
  uint8_t ring[kRing];
};

// Input windows: window b holds input bytes [w[b], w[b] + n[b]).
struct SnIn {
  const uint8_t* in;
  uint32_t in_len;
  uint32_t w[2], n[2];
  uint32_t par[2];
  int cur;        // window being parsed
  int pending;    // the other window has a copy in flight
};

// Lane 0: start the copy of input [from, from + kWin) (16-byte aligned
// start, at most 16 bytes past the input) into window b.
__device__ __forceinline__ void sn_issue(SnIn& s, SnWarp& sw, int b, uint32_t from) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(s.in);
  const uintptr_t a = (base + from) & ~uintptr_t(15);
  const uintptr_t lim = (base + s.in_len + 16) & ~uintptr_t(15);
  uint32_t bytes = static_cast<uint32_t>(lim > a ? lim - a : 16);
  if (bytes > kWin) bytes = kWin;
  if (bytes < 16) bytes = 16;
  s.w[b] = static_cast<uint32_t>(a - base);  // may wrap below 0 by up to 15: unsigned arithmetic below
  s.n[b] = bytes;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&sw.bar[b], bytes);
  bulk_g2s(sw.win[b], reinterpret_cast<const void*>(a), bytes, &sw.bar[b]);
}

// Lane 0: make input bytes [p, p + 5) readable in the current window (or up
// to the end of the input).  False if a copy never arrived.
__device__ __forceinline__ bool sn_ensure(SnIn& s, SnWarp& sw, uint32_t p) {
  const uint32_t need = p + 5 < s.in_len ? 5u : s.in_len - p;
  if (p - s.w[s.cur] + need <= s.n[s.cur] && p - s.w[s.cur] < s.n[s.cur]) return true;
  const int o = s.cur ^ 1;
  if (s.pending) {
    const bool ok = mbar_wait(&sw.bar[o], s.par[o]);
    s.par[o] ^= 1u;
    s.pending = 0;
    if (!ok) return false;
    if (p - s.w[o] < s.n[o] && p - s.w[o] + need <= s.n[o]) {
      s.cur = o;
      // prefetch the window after it (16 bytes of overlap for headers)
      const uint32_t nx = s.w[o] + s.n[o] - 16;
      if (s.w[o] + s.n[o] < s.in_len + 16 && nx < s.in_len) {
        sn_issue(s, sw, o ^ 1, nx);
        s.pending = 1;
      }
      return true;
    }
  }
  // a jump past the prefetched window (a long literal): load at p
  sn_issue(s, sw, o, p);
  const bool ok = mbar_wait(&sw.bar[o], s.par[o]);
  s.par[o] ^= 1u;
  if (!ok) return false;
  s.cur = o;
  const uint32_t nx = s.w[o] + s.n[o] - 16;
  if (s.w[o] + s.n[o] < s.in_len + 16 && nx < s.in_len) {
    sn_issue(s, sw, o ^ 1, nx);
    s.pending = 1;
  }
  return true;
}

__device__ __forceinline__ uint32_t sn_byte(const SnIn& s, const SnWarp& sw, uint32_t p) {
  return sw.win[s.cur][p - s.w[s.cur]];
}

// `n` bytes from ring positions [from, from + n) (positions are output
// offsets; the ring holds position x at x mod kRing) to global dst, 16-byte
// stores where the destination allows.
__device__ __forceinline__ void ring_out(uint8_t* dst, const uint8_t* ring, uint32_t from, uint32_t n, int lane) {
  constexpr uint32_t RM = kRing - 1;
  const uint32_t head0 = static_cast<uint32_t>((16 - (reinterpret_cast<uintptr_t>(dst) & 15)) & 15);
  const uint32_t head = head0 < n ? head0 : n;
  if (static_cast<uint32_t>(lane) < head) dst[lane] = ring[(from + lane) & RM];
  const uint32_t nv = (n - head) >> 4;
  for (uint32_t v = lane; v < nv; v += 32) {
    const uint32_t q = from + head + 16 * v;
    uint32_t w4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t b = q + 4 * k;
      w4[k] = static_cast<uint32_t>(ring[b & RM]) | (static_cast<uint32_t>(ring[(b + 1) & RM]) << 8) |
              (static_cast<uint32_t>(ring[(b + 2) & RM]) << 16) | (static_cast<uint32_t>(ring[(b + 3) & RM]) << 24);
    }
    *reinterpret_cast<uint4*>(dst + head + 16 * v) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
  }
  for (uint32_t i = head + (nv << 4) + lane; i < n; i += 32) dst[i] = ring[(from + i) & RM];
}

__global__ void __launch_bounds__(32 * kSnappyWarps) k_snappy(const SnappyJob* __restrict__ jobs, int n_jobs,
                                                              DevStatus* st) {
  extern __shared__ __align__(16) uint8_t sn_smem[];
  const int lane = threadIdx.x & 31;
  SnWarp& sw = reinterpret_cast<SnWarp*>(sn_smem)[threadIdx.x >> 5];
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  if (lane == 0) {
    mbar_init(&sw.bar[0], 1);
    mbar_init(&sw.bar[1], 1);
  }
  fence_mbar_init();
  __syncwarp();
  uint32_t par[2] = {0, 0};
  uint8_t* ring = sw.ring;
  constexpr uint32_t RM = kRing - 1;
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
    // lane 0's window state
    SnIn sin{in, in_len, {0, 0}, {0, 0}, {par[0], par[1]}, 0, 0};
    int bad = 0;
    if (lane == 0) {
      sn_issue(sin, sw, 0, 0);
      if (!mbar_wait(&sw.bar[0], sin.par[0])) bad = 2;
      sin.par[0] ^= 1u;
      const uint32_t nx = sin.w[0] + sin.n[0] - 16;
      if (!bad && sin.w[0] + sin.n[0] < in_len + 16 && nx < in_len) {
        sn_issue(sin, sw, 1, nx);
        sin.pending = 1;
      }
    }
    uint32_t ip = static_cast<uint32_t>(pl);
    uint32_t op = 0;
    bad = __shfl_sync(0xffffffffu, bad, 0);
    // each element consumes >= 2 input bytes, so in_len bounds the batches
    for (uint32_t guard = 0; guard <= in_len && ip < in_len && !bad; ++guard) {
      int n_el = 0;
      if (lane == 0) {
        uint32_t p = ip, o = op, bo = 0;
        for (int e = 0; e < 32 && p < in_len; ++e) {
          if (!sn_ensure(sin, sw, p)) { bad = 2; break; }
          const uint32_t tag = sn_byte(sin, sw, p++);
          uint32_t kind = tag & 3, len, arg;
          if (kind == 0) {
            uint32_t l = tag >> 2;
            if (l < 60) {
              len = l + 1;
            } else {
              uint32_t nb = l - 59;
              if (nb > in_len - p) { bad = 1; break; }
              uint32_t v = 0;
              for (uint32_t b = 0; b < nb; ++b) v |= sn_byte(sin, sw, p + b) << (8 * b);
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
            arg = ((tag >> 5) << 8) | sn_byte(sin, sw, p);
            p += 1;
          } else if (kind == 2) {
            if (2 > in_len - p) { bad = 1; break; }
            len = (tag >> 2) + 1;
            arg = sn_byte(sin, sw, p) | (sn_byte(sin, sw, p + 1) << 8);
            p += 2;
          } else {
            if (4 > in_len - p) { bad = 1; break; }
            len = (tag >> 2) + 1;
            arg = sn_byte(sin, sw, p) | (sn_byte(sin, sw, p + 1) << 8) | (sn_byte(sin, sw, p + 2) << 16) |
                  (sn_byte(sin, sw, p + 3) << 24);
            p += 4;
          }
          if (len > out_len - o || (kind != 0 && (arg == 0 || arg > o))) { bad = 1; break; }
          sw.kl[e] = kind | (len << 2);
          sw.arg[e] = arg;
          n_el = e + 1;
          o += len;
          bo += len;
          // a batch's short output is assembled in the ring; a long literal
          // ends its batch (it is copied to global memory directly)
          if (bo >= kBatchOut - 64 || (kind == 0 && len > 256)) break;
        }
        ip = p;
      }
      __syncwarp();
      n_el = __shfl_sync(0xffffffffu, n_el, 0);
      bad = __shfl_sync(0xffffffffu, bad, 0);
      ip = __shfl_sync(0xffffffffu, ip, 0);
      uint32_t kl = 0, arg = 0;
      if (lane < n_el) {
        kl = sw.kl[lane];
        arg = sw.arg[lane];
      }
      const uint32_t kind = kl & 3, len = kl >> 2;
      uint32_t incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t o0 = op + incl - len;  // this lane's element output offset
      const uint32_t btot = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t bend = op + btot;
      // the ring holds positions [max(0, op - (kRing - btot)), op) before the
      // batch and gets [op, bend); sources below `rlo` come from global memory
      const uint32_t keep = btot <= kRing ? kRing - btot : 0u;
      const uint32_t rlo = op > keep ? op - keep : 0u;
      const bool valid = lane < n_el;
      // long literals (the batch's last element): global to global, the
      // tail into the ring
      const bool longlit = valid && kind == 0 && len > 256;
      const bool indep = valid && !longlit && (kind == 0 || (arg >= len && o0 - arg + len <= op));
      auto src_byte = [&](uint32_t pos) -> uint8_t {
        return pos >= rlo ? ring[pos & RM] : ld_src<false>(out + pos);
      };
      if (indep) {
        if (kind == 0) {
          // literal bytes from the input (global; it sits in L2)
          for (uint32_t i = 0; i < len; ++i) ring[(o0 + i) & RM] = __ldg(in + arg + i);
        } else {
          const uint32_t first = o0 - arg;
          for (uint32_t i = 0; i < len; ++i) ring[(o0 + i) & RM] = src_byte(first + i);
        }
      }
      __syncwarp();
      for (uint32_t m = __ballot_sync(0xffffffffu, valid && !indep && !longlit); m; m &= m - 1) {
        const int e = __ffs(m) - 1;
        const uint32_t el = __shfl_sync(0xffffffffu, len, e);
        const uint32_t ea = __shfl_sync(0xffffffffu, arg, e), eo = __shfl_sync(0xffffffffu, o0, e);
        const uint32_t first = eo - ea;
        for (uint32_t i0 = 0; i0 < el; i0 += 32) {
          const uint32_t i = i0 + lane;
          uint8_t b = 0;
          if (i < el) b = src_byte(ea >= el ? first + i : first + (i % ea));
          __syncwarp();
          if (i < el) ring[(eo + i) & RM] = b;
          __syncwarp();
        }
      }
      const uint32_t lm = __ballot_sync(0xffffffffu, longlit);
      // the batch's short output, ring -> global
      const uint32_t short_end = lm ? __shfl_sync(0xffffffffu, o0, __ffs(lm) - 1) : bend;
      if (short_end > op) ring_out(out + op, ring, op, short_end - op, lane);
      __syncwarp();  // the ring's short bytes are out before a long literal's tail overwrites slots
      if (lm) {
        const int e = __ffs(lm) - 1;
        const uint32_t el = __shfl_sync(0xffffffffu, len, e);
        const uint32_t ea = __shfl_sync(0xffffffffu, arg, e), eo = __shfl_sync(0xffffffffu, o0, e);
        warp_copy<true>(out + eo, in + ea, el, lane);
        const uint32_t t0 = el > kRing ? el - kRing : 0u;
        for (uint32_t i = t0 + lane; i < el; i += 32) ring[(eo + i) & RM] = __ldg(in + ea + i);
      }
      __syncwarp();
      op = bend;
    }
    if (lane == 0) {
      // settle the window copy still in flight before the buffers are reused
      if (sin.pending) {
        mbar_wait(&sw.bar[sin.cur ^ 1], sin.par[sin.cur ^ 1]);
        sin.par[sin.cur ^ 1] ^= 1u;
      }
      if (bad == 2) report(st, DERR_TIMEOUT, jb.page, WHERE_SNAPPY, 5);
      else if (bad || op != out_len || ip != in_len) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 4);
    }
    par[0] = __shfl_sync(0xffffffffu, sin.par[0], 0);
    par[1] = __shfl_sync(0xffffffffu, sin.par[1], 0);
    __syncwarp();
  }
}

void launch_snappy(const SnappyJob* jobs, int n_jobs, int n_sms, DevStatus* st, cudaStream_t s) {
  if (n_jobs <= 0) return;
  constexpr uint32_t smem = kSnappyWarps * sizeof(SnWarp);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_snappy, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_snappy, 32 * kSnappyWarps, smem);
  if (bps < 1) bps = 1;
  int blocks = (n_jobs + kSnappyWarps - 1) / kSnappyWarps;
  if (blocks > n_sms * bps) blocks = n_sms * bps;
  k_snappy<<<blocks, 32 * kSnappyWarps, smem, s>>>(jobs, n_jobs, st);
}

}  // namespace pqi
