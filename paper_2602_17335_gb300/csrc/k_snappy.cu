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
constexpr uint32_t kMidLit = 2048;  // literals up to this long go from the input window through the ring

struct SnWarp {
  uint64_t bar[2];
  uint32_t pos[32];      // input offsets of a batch's headers
  uint8_t win[2][kWin + 16];
  uint8_t ring[kRing];
};

// Lane 0's input windows, all scalars (they stay in registers): the current
// window (*0) and the other one (*1), swapped when the parse moves on.
// Window offsets are input offsets modulo 2^32 (a window may start up to 15
// bytes before the input).
struct SnIn {
  const uint8_t* in;
  uint32_t in_len;
  uint8_t* b0;
  uint8_t* b1;
  uint64_t* m0;
  uint64_t* m1;
  uint32_t w0, w1, n0, n1, p0, p1;
  uint32_t e1;  // a copy into window 1 is in flight
  uint32_t cap; // window bytes
};

__device__ __forceinline__ void sn_swap(SnIn& s) {
  uint8_t* tb = s.b0; s.b0 = s.b1; s.b1 = tb;
  uint64_t* tm = s.m0; s.m0 = s.m1; s.m1 = tm;
  uint32_t t = s.w0; s.w0 = s.w1; s.w1 = t;
  t = s.n0; s.n0 = s.n1; s.n1 = t;
  t = s.p0; s.p0 = s.p1; s.p1 = t;
}

// Copy of input [from, from + s.cap) (16-byte aligned start, at most 16
// bytes past the input) into buffer `buf`.
__device__ __forceinline__ void sn_issue(const SnIn& s, uint8_t* buf, uint64_t* bar, uint32_t from, uint32_t* w,
                                         uint32_t* n) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(s.in);
  const uintptr_t a = (base + from) & ~uintptr_t(15);
  const uintptr_t lim = (base + s.in_len + 16) & ~uintptr_t(15);
  uint32_t bytes = static_cast<uint32_t>(lim > a ? lim - a : 16);
  if (bytes > s.cap) bytes = s.cap;
  if (bytes < 16) bytes = 16;
  *w = static_cast<uint32_t>(a - base);
  *n = bytes;
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, bytes);
  bulk_g2s(buf, reinterpret_cast<const void*>(a), bytes, bar);
}

__device__ __forceinline__ void sn_prefetch(SnIn& s) {
  const uint32_t end = s.w0 + s.n0;  // input offset just past window 0
  if (end < s.in_len) {  // input left beyond window 0
    sn_issue(s, s.b1, s.m1, end - 16, &s.w1, &s.n1);
    s.e1 = 1;
  } else {
    s.n1 = 0;
  }
}

// 32-bit load from a shared-memory address (the windows are read this way
// on the serial header chains: fewer and cheaper loads than bytes through
// generic pointers).
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

// Makes input bytes [p, p + 5) readable in window 0 (bytes past the input
// end are slack).  False if a copy never arrived.
__device__ __forceinline__ bool sn_ensure(SnIn& s, uint32_t p) {
  if (p - s.w0 < s.n0 && (p - s.w0 + 5 <= s.n0 || s.w0 + s.n0 >= s.in_len)) return true;
  if (s.e1) {
    const bool ok = mbar_wait(s.m1, s.p1);
    s.p1 ^= 1u;
    s.e1 = 0;
    if (!ok) return false;
    if (p - s.w1 < s.n1 && (p - s.w1 + 5 <= s.n1 || s.w1 + s.n1 >= s.in_len)) {
      sn_swap(s);
      sn_prefetch(s);
      return true;
    }
  }
  // a jump past the prefetched window (a long literal): load at p
  sn_issue(s, s.b1, s.m1, p, &s.w1, &s.n1);
  const bool ok = mbar_wait(s.m1, s.p1);
  s.p1 ^= 1u;
  if (!ok) return false;
  sn_swap(s);
  sn_prefetch(s);
  return true;
}

// The element whose header sits at input offset pa, from its bytes h[0..4]
// (bytes past the input are never used): kind, length, argument (literal:
// input offset of its bytes; copy: back offset) and the next header's input
// offset.  False when the header or the literal runs past the input.
__device__ __forceinline__ bool sn_hdr(uint32_t tag, uint32_t x, uint32_t pa, uint32_t in_len, uint32_t* kind,
                                       uint32_t* len, uint32_t* arg, uint32_t* next) {
  const uint32_t k = tag & 3, t6 = tag >> 2, left = in_len - pa - 1;  // bytes after the tag
  uint32_t l, a, hl;
  if (k == 0) {
    const uint32_t nb = t6 < 60 ? 0u : t6 - 59;
    const uint32_t vm = nb == 0 ? t6 : (nb == 4 ? x : (x & ((1u << (8 * nb)) - 1u)));
    if (nb > left || vm == 0xffffffffu) return false;
    l = vm + 1;
    hl = 1 + nb;
    if (l > left - nb) return false;
    a = pa + hl;
  } else {
    hl = k == 1 ? 2u : (k == 2 ? 3u : 5u);
    if (hl - 1 > left) return false;
    l = k == 1 ? 4 + (t6 & 7) : t6 + 1;
    a = k == 1 ? (((tag >> 5) << 8) | (x & 0xffu)) : (k == 2 ? (x & 0xffffu) : x);
  }
  *kind = k;
  *len = l;
  *arg = a;
  *next = pa + hl + (k == 0 ? l : 0u);
  return true;
}

// Bytes [q, q + 5) of a window as (tag, the 4 bytes after it), from two
// 32-bit shared loads (the window buffer is readable for 16 bytes past its
// end).
__device__ __forceinline__ void sn_bytes5(uint32_t sa, uint32_t* tag, uint32_t* x) {
  const uint32_t a = sa & ~3u, sh = (sa & 3u) * 8;
  const uint32_t lo = lds32(a), hi = lds32(a + 4);
  *tag = __funnelshift_r(lo, hi, sh) & 0xffu;
  *x = __funnelshift_rc(lo, hi, sh + 8);  // (a shift of 32 gives hi)
}

// The element whose header sits at input offset p, from its tag and the 4
// bytes after it, without any check (the element's own decode, or the
// caller, checks it): the offset of the next header, the output length and
// the copy offset.  Straight-line code: the header chain is serial, so each
// step is kept short.
struct SnStep {
  uint32_t next, len, arg, kind;
};
__device__ __forceinline__ SnStep sn_step(uint32_t tag, uint32_t x, uint32_t p) {
  const uint32_t kind = tag & 3, t6 = tag >> 2;
  const uint32_t nb = t6 > 59 ? t6 - 59 : 0u;  // literal length bytes after the tag
  // (a shift by 32 - 8 nb, nb in 1..4: the low nb bytes of x)
  const uint32_t lv = nb == 0 ? t6 : (x & (0xffffffffu >> ((32 - 8 * nb) & 31)));
  const uint32_t hl = (0x5320u >> (4 * kind)) & 15u;  // copy header bytes (kind 1, 2, 3: 2, 3, 5)
  SnStep r;
  r.kind = kind;
  r.next = p + (kind == 0 ? 2 + nb + lv : hl);
  r.len = kind == 0 ? lv + 1 : (kind == 1 ? 4 + (t6 & 7) : t6 + 1);
  r.arg = kind == 1 ? (((tag >> 5) << 8) | (x & 0xffu)) : (kind == 2 ? (x & 0xffffu) : x);
  return r;
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
  const uint32_t q0 = from + head;
  if ((q0 & 15) == 0) {
    // ring slots congruent with the destination: whole 16-byte ring words
    for (uint32_t v = lane; v < nv; v += 32)
      *reinterpret_cast<uint4*>(dst + head + 16 * v) = *reinterpret_cast<const uint4*>(ring + ((q0 + 16 * v) & RM));
  } else {
    for (uint32_t v = lane; v < nv; v += 32) {
      const uint32_t q = q0 + 16 * v;
      uint32_t w4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t b = q + 4 * k;
        w4[k] = static_cast<uint32_t>(ring[b & RM]) | (static_cast<uint32_t>(ring[(b + 1) & RM]) << 8) |
                (static_cast<uint32_t>(ring[(b + 2) & RM]) << 16) | (static_cast<uint32_t>(ring[(b + 3) & RM]) << 24);
      }
      *reinterpret_cast<uint4*>(dst + head + 16 * v) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
  }
  for (uint32_t i = head + (nv << 4) + lane; i < n; i += 32) dst[i] = ring[(from + i) & RM];
}

// A short literal (len <= 64) from global input to the ring: its aligned
// 16-byte words are loaded together, then placed byte by byte.
__device__ __forceinline__ void lit_to_ring(uint8_t* ring, uint32_t o0, const uint8_t* src, uint32_t len) {
  constexpr uint32_t RM = kRing - 1;
  const uint32_t sh = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 15);
  const uint4* sv = reinterpret_cast<const uint4*>(src - sh);
  const uint32_t nv = (sh + len + 15) >> 4;  // <= 5
  uint4 v[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) v[k] = static_cast<uint32_t>(k) < nv ? __ldg(sv + k) : make_uint4(0, 0, 0, 0);
  // every byte position of the five words is a constant: registers only
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const uint32_t wk[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      const uint32_t q = 16u * k + b;
      if (q >= sh && q < sh + len) ring[(o0 + q - sh) & RM] = static_cast<uint8_t>(wk[b >> 2] >> (8 * (b & 3)));
    }
  }
}

// Input bytes src[0, n) to ring positions [pos0, pos0 + n): whole 16-byte
// ring words built from two aligned source words, the partial words at the
// two ends byte by byte.
__device__ __forceinline__ void ring_fill(uint8_t* ring, uint32_t pos0, const uint8_t* src, uint32_t n, int lane) {
  constexpr uint32_t RM = kRing - 1;
  const uint32_t head0 = (16 - (pos0 & 15)) & 15;
  const uint32_t head = head0 < n ? head0 : n;
  if (static_cast<uint32_t>(lane) < head) ring[(pos0 + lane) & RM] = __ldg(src + lane);
  const uint32_t nv = (n - head) >> 4;
  const uint8_t* s1 = src + head;
  const uint32_t sh = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(s1) & 15);
  const uint4* sa = reinterpret_cast<const uint4*>(s1 - sh);
  for (uint32_t v = lane; v < nv; v += 32) {
    const uint4 A = __ldg(sa + v);
    const uint4 B = sh ? __ldg(sa + v + 1) : A;
    *reinterpret_cast<uint4*>(ring + ((pos0 + head + 16 * v) & RM)) = sh ? shift_pair(A, B, sh) : A;
  }
  for (uint32_t i = head + (nv << 4) + lane; i < n; i += 32) ring[(pos0 + i) & RM] = __ldg(src + i);
}

// A cooperative copy request from warp 0 to the other warps of its block.
struct SnCoop {
  uint8_t* dst;
  const uint8_t* src;
  uint32_t len;  // 0: the page is done
  uint32_t pad;
};

__device__ __forceinline__ void coop_bar() { asm volatile("bar.sync 1, %0;" ::"r"(32 * 8) : "memory"); }

// Slice w of 8 of a copy (16-byte aligned destination boundaries).
__device__ __forceinline__ void coop_slice(const SnCoop& c, int w, int lane) {
  const uint64_t per = ((static_cast<uint64_t>(c.len) + 8 * 16 - 1) / (8 * 16)) * 16;
  const uint64_t b = per * w, e = b + per < c.len ? b + per : c.len;
  if (b < e) warp_copy<true>(c.dst + b, c.src + b, e - b, lane);
}

// kCoop: one block of 8 warps per page; warp 0 parses and executes, and the
// literals of at least kCoopLit bytes are copied by all 8 warps.  Otherwise
// one warp per page.
constexpr uint32_t kCoopLit = 4096;

template <bool kCoop>
__global__ void __launch_bounds__(kCoop ? 256 : 32 * kSnappyWarps) k_snappy(const SnappyJob* __restrict__ jobs,
                                                                            int n_jobs, DevStatus* st) {
  extern __shared__ __align__(16) uint8_t sn_smem[];
  const int lane = threadIdx.x & 31;
  SnWarp& sw = reinterpret_cast<SnWarp*>(sn_smem)[kCoop ? 0 : threadIdx.x >> 5];
  SnCoop& cq = *reinterpret_cast<SnCoop*>(sn_smem + sizeof(SnWarp) * (kCoop ? 1 : kSnappyWarps));
  const int wid = kCoop ? blockIdx.x : (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = kCoop ? gridDim.x : (gridDim.x * blockDim.x) >> 5;
  if (kCoop && threadIdx.x >= 32) {
    // helper warps: slices of warp 0's long literals until it says the page is done
    for (int j = wid; j < n_jobs; j += nwarps) {
      for (;;) {
        coop_bar();
        const SnCoop c = cq;
        if (c.len == 0) break;
        coop_slice(c, threadIdx.x >> 5, lane);
        coop_bar();
      }
    }
    return;
  }
  if (lane == 0) {
    mbar_init(&sw.bar[0], 1);
    mbar_init(&sw.bar[1], 1);
  }
  fence_mbar_init();
  __syncwarp();
  uint32_t par[2] = {0, 0};
  uint8_t* ring = sw.ring;
  constexpr uint32_t RM = kRing - 1;
  auto page_done = [&]() {
    if (kCoop) {
      if (lane == 0) cq.len = 0;
      __syncwarp();
      coop_bar();
    }
  };
  for (int j = wid; j < n_jobs; j += nwarps) {
    const SnappyJob jb = jobs[j];
    if (jb.codec != CODEC_SNAPPY || jb.nsub > 1) {  // another codec's kernel, or the page's blocks, take it
      page_done();
      continue;
    }
    if (jb.prefix > jb.src_len || jb.prefix > jb.dst_len) {
      if (lane == 0) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 1);
      page_done();
      continue;
    }
    warp_copy<true>(jb.dst, jb.src, jb.prefix, lane);  // V2 level bytes, never compressed
    if (jb.raw) {
      if (jb.src_len != jb.dst_len) {
        if (lane == 0) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 2);
        page_done();
        continue;
      }
      warp_copy<true>(jb.dst + jb.prefix, jb.src + jb.prefix, jb.src_len - jb.prefix, lane);
      __syncwarp();
      page_done();
      continue;
    }
    const uint8_t* in = jb.src + jb.prefix;
    const uint32_t in_len = jb.src_len - jb.prefix;
    uint8_t* out = jb.dst + jb.prefix;
    const uint32_t out_len = jb.dst_len - jb.prefix;
    uint64_t declared = out_len;
    int pl = 0;  // a block of a split page has no length preamble
    if (!(jb.flags & SJ_BLOCK)) {
      pl = uleb([&](uint32_t k) { return static_cast<uint32_t>(__ldg(in + k)); }, 0, in_len, &declared);
      if (pl == 0 || declared != out_len) {
        if (lane == 0) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 3);
        page_done();
        continue;
      }
    }
    // lane 0's window state
    SnIn sin{in, in_len, sw.win[0], sw.win[1], &sw.bar[0], &sw.bar[1], 0, 0, 0, 0, par[0], par[1], 0, kWin};
    int bad = 0;
    if (lane == 0) {
      sn_issue(sin, sin.b0, sin.m0, 0, &sin.w0, &sin.n0);
      if (!mbar_wait(sin.m0, sin.p0)) bad = 2;
      sin.p0 ^= 1u;
      if (!bad) sn_prefetch(sin);
    }
    uint32_t ip = static_cast<uint32_t>(pl);
    uint32_t op = 0;
    bad = __shfl_sync(0xffffffffu, bad, 0);
    // each element consumes >= 2 input bytes, so in_len bounds the batches
    for (uint32_t guard = 0; guard <= in_len && ip < in_len && !bad; ++guard) {
      // the batch's window: switched now when ip has left window 0 (a batch's
      // headers and window literals all sit in one window)
      if (lane == 0) {
        const bool here = ip - sin.w0 < sin.n0 && (ip - sin.w0 + 5 <= sin.n0 || sin.w0 + sin.n0 >= in_len);
        if (!here && !sn_ensure(sin, ip)) bad = 2;
      }
      bad = __shfl_sync(0xffffffffu, bad, 0);
      if (bad) break;
      const uint8_t* wbuf = sw.win[__shfl_sync(0xffffffffu, lane == 0 && sin.b0 == sw.win[1] ? 1 : 0, 0)];
      const uint32_t w0 = __shfl_sync(0xffffffffu, sin.w0, 0), n0 = __shfl_sync(0xffffffffu, sin.n0, 0);
      // lane 0 follows the header chain to up to 32 headers inside the window;
      // it stops after an element that ends the batch anyway (a literal that
      // is long or runs past the window, the output budget) or does not parse
      // (its own lane reports it)
      int n_pos = 0;
      if (lane == 0) {
        uint32_t p = ip, ob = 0;
        const uint32_t lim = w0 + n0 >= in_len ? n0 : n0 - 4;  // offsets whose header bytes are all here
        const uint32_t sb = smem_u32(wbuf) - w0;  // shared address of input offset x: sb + x
        while (n_pos < 32 && p < in_len) {
          if (p - w0 >= lim) break;
          sw.pos[n_pos++] = p;
          uint32_t tag, x;
          sn_bytes5(sb + p, &tag, &x);
          const SnStep e = sn_step(tag, x, p);
          ob += e.len;
          if (e.next <= p || e.next > in_len || ob >= kBatchOut - 64 ||
              (e.kind == 0 && (e.len > kMidLit || e.next - w0 > n0)))
            break;
          p = e.next;
        }
      }
      __syncwarp();
      n_pos = __shfl_sync(0xffffffffu, n_pos, 0);
      // every lane decodes its header from the window
      uint32_t kind = 0, len = 0, arg = 0, nextp = 0;
      bool hok = true;
      if (lane < n_pos) {
        const uint32_t mypos = sw.pos[lane];
        uint32_t tag, x;
        sn_bytes5(smem_u32(wbuf) + (mypos - w0), &tag, &x);
        hok = sn_hdr(tag, x, mypos, in_len, &kind, &len, &arg, &nextp);
      }
      // output offsets; the batch ends after its first element that fills the
      // ring's budget or is a literal outside the window (copied directly)
      const uint32_t plen = lane < n_pos ? len : 0u;
      uint32_t pinc = plen;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, pinc, o);
        if (lane >= o) pinc += y;
      }
      const bool inwin = kind == 0 && len <= kMidLit && arg - w0 + len <= n0;
      const bool trig = lane < n_pos && (!hok || pinc >= kBatchOut - 64 || (kind == 0 && !inwin));
      const uint32_t tm = __ballot_sync(0xffffffffu, trig);
      const int n_el = tm ? __ffs(tm) : n_pos;
      const uint32_t o_e = op + pinc - plen;
      const bool evalid = hok && len <= out_len - o_e && (kind == 0 || (arg != 0 && arg <= o_e));
      if (n_el == 0 || __any_sync(0xffffffffu, lane < n_el && !evalid)) {
        bad = 1;
        break;
      }
      ip = __shfl_sync(0xffffffffu, nextp, n_el - 1);
      int32_t woff = -1;
      if (lane < n_el && inwin) woff = static_cast<int32_t>(arg - w0);
      if (lane >= n_el) kind = len = arg = 0;
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
      const bool longlit = valid && kind == 0 && woff < 0;
      const bool indep = valid && !longlit && (kind == 0 || (arg >= len && o0 - arg + len <= op));
      auto src_byte = [&](uint32_t pos) -> uint8_t {
        return pos >= rlo ? ring[pos & RM] : ld_src<false>(out + pos);
      };
      if (indep) {
        if (kind == 0 && len <= 32) {
          for (uint32_t i = 0; i < len; ++i) ring[(o0 + i) & RM] = wbuf[woff + i];
        } else if (kind == 0) {
          // longer literals from the window: by the whole warp, below
        } else {
          const uint32_t first = o0 - arg;
          uint32_t i = 0;
          for (; i + 4 <= len; i += 4) {  // four independent reads in flight
            const uint8_t c0 = src_byte(first + i), c1 = src_byte(first + i + 1), c2 = src_byte(first + i + 2),
                          c3 = src_byte(first + i + 3);
            ring[(o0 + i) & RM] = c0;
            ring[(o0 + i + 1) & RM] = c1;
            ring[(o0 + i + 2) & RM] = c2;
            ring[(o0 + i + 3) & RM] = c3;
          }
          for (; i < len; ++i) ring[(o0 + i) & RM] = src_byte(first + i);
        }
      }
      __syncwarp();
      for (uint32_t m = __ballot_sync(0xffffffffu, indep && kind == 0 && len > 32); m; m &= m - 1) {
        const int e = __ffs(m) - 1;
        const uint32_t el = __shfl_sync(0xffffffffu, len, e), eo = __shfl_sync(0xffffffffu, o0, e);
        const int32_t ew = __shfl_sync(0xffffffffu, woff, e);
        for (uint32_t i = lane; i < el; i += 32) ring[(eo + i) & RM] = wbuf[ew + i];
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
        if (kCoop && el >= kCoopLit) {
          if (lane == 0) cq = SnCoop{out + eo, in + ea, el, 0};
          __syncwarp();
          coop_bar();
          coop_slice(SnCoop{out + eo, in + ea, el, 0}, 0, lane);
          coop_bar();
        } else {
          warp_copy<true>(out + eo, in + ea, el, lane);
        }
        const uint32_t t0 = el > kRing ? el - kRing : 0u;
        ring_fill(ring, eo + t0, in + ea + t0, el - t0, lane);
      }
      __syncwarp();
      op = bend;
    }
    if (lane == 0) {
      // settle the window copy still in flight before the buffers are reused
      if (sin.e1) {
        mbar_wait(sin.m1, sin.p1);
        sin.p1 ^= 1u;
        sin.e1 = 0;
      }
      if (bad == 2) report(st, DERR_TIMEOUT, jb.page, WHERE_SNAPPY, 5);
      else if (bad || op != out_len || ip != in_len) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 4);
    }
    // carry the physical buffers' parities to the next page
    const bool sw0 = sin.b0 == sw.win[0];
    par[0] = __shfl_sync(0xffffffffu, sw0 ? sin.p0 : sin.p1, 0);
    par[1] = __shfl_sync(0xffffffffu, sw0 ? sin.p1 : sin.p0, 0);
    __syncwarp();
    page_done();
  }
}

// Fragment scan of the split pages: lane 0 of a warp follows a page's
// element headers through two shared-memory windows (as the decoder does,
// wider) and cuts a block wherever the output reaches a multiple of
// SNAPPY_FRAGMENT at an element boundary.  A copy whose source lies before
// its block's start, or anything the decoder would reject, makes the page
// one job again (decompressed whole, where the decoder reports what is
// wrong).  The blocks go to the plan's block list at the page's slots; slots
// the page does not use become no-op jobs.
constexpr uint32_t kSplitWin = 8192;
constexpr int kSplitWarps = 4;
struct SnSplitWarp {
  uint64_t bar[2];
  uint8_t win[2][kSplitWin + 16];
};

__global__ void __launch_bounds__(32 * kSplitWarps) k_snappy_split(const SnappyJob* __restrict__ jobs, int n_jobs,
                                                                   SnappyJob* blocks, DevStatus* st) {
  extern __shared__ __align__(16) uint8_t sp_smem[];
  const int lane = threadIdx.x & 31;
  SnSplitWarp& sw = reinterpret_cast<SnSplitWarp*>(sp_smem)[threadIdx.x >> 5];
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  if (lane == 0) {
    mbar_init(&sw.bar[0], 1);
    mbar_init(&sw.bar[1], 1);
  }
  fence_mbar_init();
  __syncwarp();
  uint32_t par[2] = {0, 0};
  for (int j = wid; j < n_jobs; j += nwarps) {
    const SnappyJob jb = jobs[j];
    if (jb.codec != CODEC_SNAPPY || jb.nsub <= 1) continue;
    const bool shape = !jb.raw && jb.prefix <= jb.src_len && jb.prefix <= jb.dst_len;
    if (shape) warp_copy<true>(jb.dst, jb.src, jb.prefix, lane);  // V2 level bytes, never compressed
    if (lane == 0) {
      const uint8_t* in = jb.src + jb.prefix;
      uint8_t* out = jb.dst + jb.prefix;
      const uint32_t in_len = shape ? jb.src_len - jb.prefix : 0u;
      const uint32_t out_len = shape ? jb.dst_len - jb.prefix : 0u;
      SnappyJob* bl = blocks + jb.sub;
      auto emit = [&](uint32_t q, uint32_t i0, uint32_t i1, uint32_t o0, uint32_t o1) {
        SnappyJob b{};
        b.src = in + i0;
        b.dst = out + o0;
        b.src_len = i1 - i0;
        b.dst_len = o1 - o0;
        b.page = jb.page;
        b.codec = CODEC_SNAPPY;
        b.flags = SJ_BLOCK;
        bl[q] = b;
      };
      auto empty = [&](uint32_t q) {
        SnappyJob b{};
        b.page = jb.page;
        bl[q] = b;  // codec 0: no kernel takes it
      };
      uint64_t declared = 0;
      int pl = 0;
      bool ok = shape;
      if (ok) {
        pl = uleb([&](uint32_t k) { return static_cast<uint32_t>(__ldg(in + k)); }, 0, in_len, &declared);
        ok = pl != 0 && declared == out_len;
      }
      SnIn sin{in, in_len, sw.win[0], sw.win[1], &sw.bar[0], &sw.bar[1], 0, 0, 0, 0, par[0], par[1], 0, kSplitWin};
      bool loaded = false, timeout = false;
      if (ok) {
        sn_issue(sin, sin.b0, sin.m0, 0, &sin.w0, &sin.n0);
        loaded = true;
        if (!mbar_wait(sin.m0, sin.p0)) timeout = true;
        sin.p0 ^= 1u;
        if (!timeout) sn_prefetch(sin);
        ok = !timeout;
      }
      uint32_t p = static_cast<uint32_t>(pl), o = 0, k = 0, bi = p, bo = 0;
      uint32_t next_cut = SNAPPY_FRAGMENT;
      uint32_t sb = smem_u32(sin.b0) - sin.w0;  // shared address of input offset x: sb + x
      // offsets below plim have all their header bytes in window 0 (the
      // window test is one compare per element)
      auto window_end = [&]() {
        const uint32_t e = sin.w0 + sin.n0;
        return sin.w0 + sin.n0 >= in_len ? in_len : e - 4;
      };
      uint32_t plim = ok ? window_end() : 0u;
      // each element consumes >= 2 input bytes
      for (uint32_t guard = 0; ok && p < in_len && guard <= in_len; ++guard) {
        if (p - sin.w0 >= plim - sin.w0) {
          if (!sn_ensure(sin, p)) {
            timeout = true;
            ok = false;
            break;
          }
          sb = smem_u32(sin.b0) - sin.w0;
          plim = window_end();
        }
        uint32_t tag, x;
        sn_bytes5(sb + p, &tag, &x);
        const SnStep e = sn_step(tag, x, p);
        // the element's bytes are in the input (no wrap, a literal's length
        // below 2^32); a copy's source lies in its block; the output stays
        // inside the page
        if ((e.next - p - 1) >= in_len - p || e.len - 1 >= out_len - o || (e.kind != 0 && e.arg - 1 >= o - bo)) {
          ok = false;
          break;
        }
        o += e.len;
        p = e.next;
        if (o >= next_cut && o < out_len) {
          const uint32_t nk = o / SNAPPY_FRAGMENT;
          if (nk >= jb.nsub) {
            ok = false;
            break;
          }
          emit(k, bi, p, bo, o);
          for (uint32_t e2 = k + 1; e2 < nk; ++e2) empty(e2);
          k = nk;
          bi = p;
          bo = o;
          next_cut = (k + 1) * SNAPPY_FRAGMENT;
        }
      }
      if (ok && p == in_len && o == out_len) {
        emit(k, bi, p, bo, o);
        for (uint32_t e = k + 1; e < jb.nsub; ++e) empty(e);
      } else {
        // one job for the whole page (its prefix is copied again there)
        SnappyJob w = jb;
        w.nsub = 0;
        w.sub = 0;
        bl[0] = w;
        for (uint32_t e = 1; e < jb.nsub; ++e) empty(e);
        if (timeout) report(st, DERR_TIMEOUT, jb.page, WHERE_SNAPPY, 6);
      }
      if (loaded && sin.e1) {  // settle the window copy still in flight before the buffers are reused
        mbar_wait(sin.m1, sin.p1);
        sin.p1 ^= 1u;
        sin.e1 = 0;
      }
      const bool sw0 = sin.b0 == sw.win[0];
      par[0] = sw0 ? sin.p0 : sin.p1;
      par[1] = sw0 ? sin.p1 : sin.p0;
    }
    __syncwarp();
  }
}

void launch_snappy_split(const SnappyJob* jobs, int n_jobs, SnappyJob* blocks, int n_sms, DevStatus* st,
                         cudaStream_t s) {
  if (n_jobs <= 0) return;
  static bool attr = false;
  constexpr uint32_t smem = kSplitWarps * sizeof(SnSplitWarp);
  if (!attr) {
    cudaFuncSetAttribute(k_snappy_split, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  int blocks_n = (n_jobs + kSplitWarps - 1) / kSplitWarps;
  if (blocks_n > n_sms * 3) blocks_n = n_sms * 3;
  k_snappy_split<<<blocks_n, 32 * kSplitWarps, smem, s>>>(jobs, n_jobs, blocks, st);
}

void launch_snappy(const SnappyJob* jobs, int n_jobs, int n_sms, DevStatus* st, cudaStream_t s, bool coop) {
  if (n_jobs <= 0) return;
  static bool attr = false;
  constexpr uint32_t smem_w = kSnappyWarps * sizeof(SnWarp) + sizeof(SnCoop);
  constexpr uint32_t smem_c = sizeof(SnWarp) + sizeof(SnCoop);
  if (!attr) {
    cudaFuncSetAttribute(k_snappy<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_w);
    cudaFuncSetAttribute(k_snappy<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c);
    attr = true;
  }
  int bps = 0;
  if (coop) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_snappy<true>, 256, smem_c);
    if (bps < 1) bps = 1;
    const int blocks = n_jobs < n_sms * bps ? n_jobs : n_sms * bps;
    k_snappy<true><<<blocks, 256, smem_c, s>>>(jobs, n_jobs, st);
    return;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_snappy<false>, 32 * kSnappyWarps, smem_w);
  if (bps < 1) bps = 1;
  int blocks = (n_jobs + kSnappyWarps - 1) / kSnappyWarps;
  if (blocks > n_sms * bps) blocks = n_sms * bps;
  k_snappy<false><<<blocks, 32 * kSnappyWarps, smem_w, s>>>(jobs, n_jobs, st);
}

}  // namespace pqi
