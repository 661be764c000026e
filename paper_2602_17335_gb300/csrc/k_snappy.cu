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
// is parsed).  When the parse enters a window, the warp's 32 lanes follow
// header chains from 32 evenly spaced offsets of it into a next-header
// table (chains that start inside literal bytes fall onto the true chain
// within a few elements); lane 0 then walks the table to up to 32 headers
// and every lane decodes one of them.  The warp executes the batch into a
// ring of recent output in shared memory -- literals and copies whose
// source lies before the batch in parallel, one element per lane, literals
// from the staged window by 16-byte vectors, copies that read output of the
// same batch in order -- and writes the batch's output to global memory
// with 16-byte stores.  Literals longer than kMidLit, or outside the
// window, go straight from the input to the output as 16-byte vector copies
// (by the whole block in the block-per-page mode for large pages).  Copy
// sources older than the ring are read back from the output with coherent
// loads (this warp wrote them).
#include "dev_util.cuh"
#include "snappy_job.h"

namespace pqi {

constexpr int kSnappyWarps = 4;     // warps per block
constexpr uint32_t kRing = 8192;    // recent output kept in shared memory per warp (power of two)
constexpr uint32_t kWin = 4096;     // input window (two per warp)
constexpr uint32_t kBatchOut = kRing / 2;  // output bytes of one batch assembled in the ring
constexpr uint32_t kMidLit = 2048;  // literals up to this long go from the input window through the ring
constexpr uint16_t kNxUnk = 0xffffu;   // no chain reached this offset
constexpr uint16_t kNxOut = 0xfffeu;   // the next header lies past the window

struct SnWarp {
  uint16_t nxt[kWin];  // window offset -> the next header's window offset (kNxUnk / kNxOut)
  uint32_t pos[32];    // input offsets of a batch's headers
  uint64_t bar[2];
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
};

__device__ __forceinline__ void sn_swap(SnIn& s) {
  uint8_t* tb = s.b0; s.b0 = s.b1; s.b1 = tb;
  uint64_t* tm = s.m0; s.m0 = s.m1; s.m1 = tm;
  uint32_t t = s.w0; s.w0 = s.w1; s.w1 = t;
  t = s.n0; s.n0 = s.n1; s.n1 = t;
  t = s.p0; s.p0 = s.p1; s.p1 = t;
}

// Copy of input [from, from + kWin) (16-byte aligned start, at most 16 bytes
// past the input) into buffer `buf`.
__device__ __forceinline__ void sn_issue(const SnIn& s, uint8_t* buf, uint64_t* bar, uint32_t from, uint32_t* w,
                                         uint32_t* n) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(s.in);
  const uintptr_t a = (base + from) & ~uintptr_t(15);
  const uintptr_t lim = (base + s.in_len + 16) & ~uintptr_t(15);
  uint32_t bytes = static_cast<uint32_t>(lim > a ? lim - a : 16);
  if (bytes > kWin) bytes = kWin;
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
__device__ __forceinline__ bool sn_hdr(const uint8_t* h, uint32_t pa, uint32_t in_len, uint32_t* kind, uint32_t* len,
                                       uint32_t* arg, uint32_t* next) {
  const uint32_t tag = h[0], x1 = h[1], x2 = h[2], x3 = h[3], x4 = h[4];
  const uint32_t k = tag & 3, left = in_len - pa - 1;  // bytes after the tag
  uint32_t l, a, hl;
  if (k == 0) {
    const uint32_t t = tag >> 2;
    if (t < 60) {
      l = t + 1;
      hl = 1;
    } else {
      const uint32_t nb = t - 59;
      if (nb > left) return false;
      const uint32_t v = x1 | (x2 << 8) | (x3 << 16) | (x4 << 24);
      const uint32_t vm = nb == 4 ? v : (v & ((1u << (8 * nb)) - 1u));
      if (vm == 0xffffffffu) return false;
      l = vm + 1;
      hl = 1 + nb;
    }
    if (l > in_len - pa - hl) return false;
    a = pa + hl;
  } else if (k == 1) {
    if (left < 1) return false;
    l = 4 + ((tag >> 2) & 7);
    a = ((tag >> 5) << 8) | x1;
    hl = 2;
  } else if (k == 2) {
    if (left < 2) return false;
    l = (tag >> 2) + 1;
    a = x1 | (x2 << 8);
    hl = 3;
  } else {
    if (left < 4) return false;
    l = (tag >> 2) + 1;
    a = x1 | (x2 << 8) | (x3 << 16) | (x4 << 24);
    hl = 5;
  }
  *kind = k;
  *len = l;
  *arg = a;
  *next = pa + hl + (k == 0 ? l : 0u);
  return true;
}

// The whole warp: chains of headers from 32 evenly spaced offsets of the
// window (each a guess at a header) into the next-header table.  The
// element after a header depends only on the header's position, so an entry
// is right however its chain got there; chains that start inside literal
// bytes usually land on the true chain after a few elements, and from there
// the table covers it.
__device__ __forceinline__ void sn_spec(uint16_t* nxt, const uint8_t* win, uint32_t w0, uint32_t n0, uint32_t in_len,
                                        int lane) {
  for (uint32_t q = lane; q < n0; q += 32) nxt[q] = kNxUnk;
  __syncwarp();
  const uint32_t per = (n0 + 31) / 32;
  const uint32_t start = lane * per;
  const uint32_t end = start + per + 32 < n0 ? start + per + 32 : n0;
  const bool tail = w0 + n0 >= in_len;  // the window reaches the input's end
  uint32_t q = start;
  for (int steps = 0; q < end && steps < 48; ++steps) {
    if (nxt[q] != kNxUnk) break;  // parsed already: the chain goes on from there
    if ((q + 5 > n0 && !tail) || w0 + q >= in_len) break;
    uint32_t kind, len, arg, next;
    if (!sn_hdr(win + q, w0 + q, in_len, &kind, &len, &arg, &next)) break;
    const uint32_t nr = next - w0;
    nxt[q] = nr < n0 ? static_cast<uint16_t>(nr) : kNxOut;
    if (nr >= n0) break;
    q = nr;
  }
  __syncwarp();
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

// `n` bytes from shared memory `src` (any alignment, readable for 16 bytes
// past the end) to ring positions [pos0, pos0 + n): whole 16-byte ring words
// from two aligned shared words, the partial words at the two ends byte by
// byte.
__device__ __forceinline__ void win_to_ring(uint8_t* ring, uint32_t pos0, const uint8_t* src, uint32_t n, int lane) {
  constexpr uint32_t RM = kRing - 1;
  const uint32_t head0 = (16 - (pos0 & 15)) & 15;
  const uint32_t head = head0 < n ? head0 : n;
  if (static_cast<uint32_t>(lane) < head) ring[(pos0 + lane) & RM] = src[lane];
  const uint32_t nv = (n - head) >> 4;
  const uint8_t* s1 = src + head;
  const uint32_t sh = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(s1) & 15);
  const uint4* sa = reinterpret_cast<const uint4*>(s1 - sh);
  for (uint32_t v = lane; v < nv; v += 32) {
    const uint4 A = sa[v];
    const uint4 B = sh ? sa[v + 1] : A;
    *reinterpret_cast<uint4*>(ring + ((pos0 + head + 16 * v) & RM)) = sh ? shift_pair(A, B, sh) : A;
  }
  for (uint32_t i = head + (nv << 4) + lane; i < n; i += 32) ring[(pos0 + i) & RM] = src[i];
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
    if (jb.codec != CODEC_SNAPPY) {  // another codec's kernel takes it
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
    uint64_t declared = 0;
    int pl = uleb([&](uint32_t k) { return static_cast<uint32_t>(__ldg(in + k)); }, 0, in_len, &declared);
    if (pl == 0 || declared != out_len) {
      if (lane == 0) report(st, DERR_CORRUPT, jb.page, WHERE_SNAPPY, 3);
      page_done();
      continue;
    }
    // lane 0's window state
    SnIn sin{in, in_len, sw.win[0], sw.win[1], &sw.bar[0], &sw.bar[1], 0, 0, 0, 0, par[0], par[1], 0};
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
    uint32_t tab_w0 = 0, tab_n0 = 0;   // window the next-header table describes (lane 0)
    const uint8_t* tab_b = nullptr;
    for (uint32_t guard = 0; guard <= in_len && ip < in_len && !bad; ++guard) {
      // the batch's window: switched now when ip has left window 0; a new
      // window's next-header table is filled by the whole warp
      int need = 0;
      if (lane == 0) {
        const bool here = ip - sin.w0 < sin.n0 && (ip - sin.w0 + 5 <= sin.n0 || sin.w0 + sin.n0 >= in_len);
        if (!here && !sn_ensure(sin, ip)) bad = 2;
        need = !bad && (sin.w0 != tab_w0 || sin.n0 != tab_n0 || sin.b0 != tab_b);
        if (need) {
          tab_w0 = sin.w0;
          tab_n0 = sin.n0;
          tab_b = sin.b0;
        }
      }
      bad = __shfl_sync(0xffffffffu, bad, 0);
      if (bad) break;
      const int wsel = __shfl_sync(0xffffffffu, lane == 0 && sin.b0 == sw.win[1] ? 1 : 0, 0);
      const uint8_t* wbuf = sw.win[wsel];
      const uint32_t w0 = __shfl_sync(0xffffffffu, sin.w0, 0), n0 = __shfl_sync(0xffffffffu, sin.n0, 0);
      if (__shfl_sync(0xffffffffu, need, 0)) sn_spec(sw.nxt, wbuf, w0, n0, in_len, lane);
      // lane 0 follows the table (parsing itself where no chain went) to up
      // to 32 headers inside the window
      int n_pos = 0;
      if (lane == 0) {
        uint32_t p = ip;
        while (n_pos < 32 && p < in_len) {
          const uint32_t q = p - w0;
          if (!(q < n0 && (q + 5 <= n0 || w0 + n0 >= in_len))) break;
          uint32_t nx;
          const uint16_t t = sw.nxt[q];
          if (t < kNxOut) {
            nx = w0 + t;
          } else {
            uint32_t k, l, a2;
            if (!sn_hdr(wbuf + q, p, in_len, &k, &l, &a2, &nx)) {
              sw.pos[n_pos++] = p;  // the lane that parses it reports it
              break;
            }
          }
          sw.pos[n_pos++] = p;
          p = nx;
        }
      }
      __syncwarp();
      n_pos = __shfl_sync(0xffffffffu, n_pos, 0);
      // every lane parses its header from the window
      uint32_t kind = 0, len = 0, arg = 0, nextp = 0;
      bool hok = true;
      const uint32_t mypos = lane < n_pos ? sw.pos[lane] : 0u;
      if (lane < n_pos) hok = sn_hdr(wbuf + (mypos - w0), mypos, in_len, &kind, &len, &arg, &nextp);
      // output offsets; the batch ends after its first element that fills the
      // ring's budget or is a literal outside the window (copied directly)
      const uint32_t plen = lane < n_pos ? len : 0u;
      uint32_t pinc = plen;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, pinc, o);
        if (lane >= o) pinc += y;
      }
      const bool inwin0 = kind == 0 && len <= kMidLit && arg - w0 + len <= n0;
      const bool trig = lane < n_pos && (pinc >= kBatchOut - 64 || (kind == 0 && !inwin0));
      const uint32_t tm = __ballot_sync(0xffffffffu, trig);
      const int n_el = tm ? __ffs(tm) : n_pos;
      const uint32_t o_e = op + pinc - plen;
      const bool evalid = !hok ? false : (len <= out_len - o_e && (kind == 0 || (arg != 0 && arg <= o_e)));
      if (__any_sync(0xffffffffu, lane < n_el && !evalid)) {
        bad = 1;
        break;
      }
      if (n_el == 0) {
        bad = 1;
        break;
      }
      ip = __shfl_sync(0xffffffffu, nextp, n_el - 1);
      int32_t woff = -1;
      if (lane < n_el && inwin0) woff = static_cast<int32_t>(arg - w0);
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
        win_to_ring(ring, eo, wbuf + ew, el, lane);
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
