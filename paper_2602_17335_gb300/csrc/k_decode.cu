// K2-K8 — dictionary decode, page walk, warp-granular expansion, string
// passes and the plain one-page-per-block baseline.
//
// What a page holds (paper Section 2; byte layouts from the Parquet format):
//   V1 data page: [4-byte LE length + RLE/bit-packed def levels]? values
//   V2 data page: [rep levels][def levels] values (level lengths in header)
//   values: PLAIN (fixed width LE, or 4-byte length + bytes), dictionary
//   indices (1-byte bit width + RLE/bit-packed hybrid), or
//   DELTA_BINARY_PACKED (header, then blocks of miniblocks).
//
// Run and block headers make every stream a chain: the next header's
// position is only known after the current one is read.  The scan keeps
// that chain as short as the format allows and moves everything else off it
// (paper Section 3, Insight 1: a page must not be the unit of parallelism):
//
//  walk   one thread block per page that needs it; thread 0 follows the
//         header chain through two shared-memory windows it fills with the
//         bulk-copy engine (the next window streams in while the current one
//         is read), a handful of dependent instructions per run; the block's
//         other threads turn each batch of runs into the validity bitmap and
//         into checkpoints (stream position at the first value) for the
//         work items.  DELTA pages record every block's position.
//  bases  DELTA only: one warp per block sums its deltas, a block-wide scan
//         gives every block the value that precedes it.
//  expand one warp per work item (ITEM_ROWS rows), no block-wide barriers:
//         from the checkpoint the warp decodes its runs 32 values per lane
//         step, gathers issued back to back, and writes every output row
//         once (nulls as zero).
//  strings expand records per row the dictionary index (or PLAIN value
//         offset) and per-item chars totals; a scan makes item bases; the
//         copy pass writes int64 offsets and the chars.
#include <algorithm>
#include <type_traits>

#include "decode_job.h"
#include "dev_util.cuh"

namespace pqi {

constexpr int WALK_THREADS = 256;
constexpr int EXP_THREADS = 256;
constexpr int EXP_WARPS = EXP_THREADS / 32;
constexpr int EXP_COUNTER0 = 4;  // item_counter[4 + c]: next item of output column c
constexpr uint32_t CWIN = 16384;      // chain window (two per walking block)
constexpr uint32_t CWIN_MAX = 65536;  // window of walks over few pages
constexpr uint32_t COVL = 64;     // overlap of consecutive chain windows
constexpr int RB = 1024;          // runs per walk batch

// ------------------------------------------------------------------ global bit readers

// Bits [b, b + w) (w <= 32) of the little-endian bit stream at `base`,
// through aligned 32-bit loads (reads at most 8 bytes past the value).
__device__ __forceinline__ uint32_t gbits32(const uint8_t* base, uint64_t b, int w) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(base) + (b >> 3);
  const uint32_t* q = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const uint32_t sh = static_cast<uint32_t>((a & 3) * 8 + (b & 7));
  const uint64_t v = ((static_cast<uint64_t>(__ldg(q + 1)) << 32) | __ldg(q)) >> sh;
  return w >= 32 ? static_cast<uint32_t>(v) : static_cast<uint32_t>(v) & ((1u << w) - 1u);
}

__device__ __forceinline__ uint64_t gbits64(const uint8_t* base, uint64_t b, int w) {
  if (w <= 32) return gbits32(base, b, w);
  const uintptr_t a = reinterpret_cast<uintptr_t>(base) + (b >> 3);
  const uint32_t* q = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const uint32_t sh = static_cast<uint32_t>((a & 3) * 8 + (b & 7));
  const uint64_t lo = (static_cast<uint64_t>(__ldg(q + 1)) << 32) | __ldg(q);
  const uint64_t hi = __ldg(q + 2);
  const uint64_t v = sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
  return w >= 64 ? v : (v & ((1ull << w) - 1));
}

// Bits [b, b + 64) of the little-endian bit stream at `base` (three
// aligned 32-bit loads; reads at most 12 bytes past bit b + 64).
__device__ __forceinline__ uint64_t gwin64(const uint8_t* base, uint64_t b) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(base) + (b >> 3);
  const uint32_t* q = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const uint32_t sh = static_cast<uint32_t>((a & 3) * 8 + (b & 7));  // 0..31
  const uint32_t r0 = __ldg(q), r1 = __ldg(q + 1), r2 = __ldg(q + 2);
  return (static_cast<uint64_t>(__funnelshift_r(r1, r2, sh)) << 32) | __funnelshift_r(r0, r1, sh);
}

// DELTA_BINARY_PACKED block header with 4 miniblocks: min delta (zigzag
// ULEB128, 1-10 bytes) then 4 bit-width bytes, parsed from the 16 bytes at
// p held in registers (5 aligned 32-bit loads; reads at most 19 bytes past
// p).  Returns the varint length (0 when longer than 10 bytes); *z the
// varint, *w4 the widths (byte m = miniblock m).
template <bool kShared>
__device__ __forceinline__ int delta_header16(const uint8_t* p, uint64_t* z, uint32_t* w4) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t* q = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const uint32_t sh = static_cast<uint32_t>(a & 3) * 8;
  uint32_t r[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if constexpr (kShared)
      r[k] = q[k];
    else
      r[k] = __ldg(q + k);
  }
  const uint64_t lo = (static_cast<uint64_t>(__funnelshift_r(r[1], r[2], sh)) << 32) | __funnelshift_r(r[0], r[1], sh);
  const uint64_t hi = (static_cast<uint64_t>(__funnelshift_r(r[3], r[4], sh)) << 32) | __funnelshift_r(r[2], r[3], sh);
  // first byte with its high bit clear ends the varint
  const uint64_t mlo = ~lo & 0x8080808080808080ull;
  const uint64_t mhi = ~hi & 0x8080ull;
  const int vl = mlo ? (__ffsll(static_cast<long long>(mlo)) >> 3) : (mhi ? 8 + (__ffsll(static_cast<long long>(mhi)) >> 3) : 0);
  if (!vl) return 0;
  uint64_t v = 0;
  for (int i = 0; i < vl; ++i) {
    const uint64_t byte = i < 8 ? (lo >> (8 * i)) & 0x7f : (hi >> (8 * (i - 8))) & 0x7f;
    v |= byte << (7 * i);
  }
  *z = v;
  *w4 = vl < 8 ? static_cast<uint32_t>((lo >> (8 * vl)) | (vl ? hi << (64 - 8 * vl) : 0ull))
               : static_cast<uint32_t>(hi >> (8 * (vl - 8)));
  return vl;
}

// ------------------------------------------------------------------ K6 dictionaries

// Fixed-width dictionary: an aligned copy of the PLAIN page body.
__global__ void k_dict_fixed(const DictJob* __restrict__ jobs, DictDev* dicts, DevStatus* st) {
  const DictJob j = jobs[blockIdx.y];
  if (j.ptype == T_BYTE_ARRAY) return;
  const uint64_t bytes = static_cast<uint64_t>(j.n) * j.width;
  if (bytes > static_cast<uint64_t>(j.body_len) || j.n < 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) report(st, DERR_CORRUPT, j.page, WHERE_DICT, 1);
    return;
  }
  const uint64_t words = (bytes + 3) / 4;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(reinterpret_cast<uintptr_t>(j.body) & ~uintptr_t(3));
  const uint32_t sh = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(j.body) & 3) * 8;
  uint32_t* dst = reinterpret_cast<uint32_t*>(j.values);
  for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < words;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t lo = __ldg(src + i);
    dst[i] = sh ? __funnelshift_r(lo, __ldg(src + i + 1), sh) : lo;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DictDev d{};
    d.values = j.values;
    d.n = j.n;
    d.width = j.width;
    d.valid = 1;
    dicts[j.chunk] = d;
  }
}

// ------------------------------------------------------------------ the header chain

// Two shared-memory windows owned by one thread: the current one (fields
// *0) and the other one (*1), swapped when the chain moves on.  A window
// holds stream bytes [w, w + n); consecutive windows overlap by COVL bytes
// so that any read of up to COVL bytes fits in one of them.  Only the owning
// thread issues copies into them and reads them.  All state is scalar so
// that it stays in registers.
struct Chain {
  uint8_t* b0;
  uint8_t* b1;
  uint64_t* m0;
  uint64_t* m1;
  uint32_t p0, p1;   // mbarrier phase parities
  int64_t w0, w1;    // stream offset of the window's first byte
  uint32_t n0, n1;   // bytes held
  uint32_t e0, e1;   // a copy is in flight
  uint32_t swapped;  // 1 when b0 is the second physical buffer
  const uint8_t* sb;
  uint32_t slen;
  uint32_t cap;      // bytes per window
};

__device__ __forceinline__ void ch_swap(Chain& c) {
  uint8_t* tb = c.b0; c.b0 = c.b1; c.b1 = tb;
  uint64_t* tm = c.m0; c.m0 = c.m1; c.m1 = tm;
  uint32_t t = c.p0; c.p0 = c.p1; c.p1 = t;
  int64_t tw = c.w0; c.w0 = c.w1; c.w1 = tw;
  t = c.n0; c.n0 = c.n1; c.n1 = t;
  t = c.e0; c.e0 = c.e1; c.e1 = t;
  c.swapped ^= 1u;
}

// Copies stream bytes from `from` (rounded down to 16) into a window: up to
// the window capacity, at most 16 bytes past the stream end (readable padding).
__device__ __forceinline__ void ch_issue(const Chain& c, uint8_t* buf, uint64_t* bar, int64_t from, int64_t* w,
                                         uint32_t* n, uint32_t* e) {
  const uint8_t* a = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(c.sb + from) & ~uintptr_t(15));
  int64_t want = (static_cast<int64_t>((c.sb + c.slen) - a) + 16) & ~int64_t(15);
  if (want < 16) want = 16;
  const uint32_t bytes = static_cast<uint32_t>(want < c.cap ? want : c.cap);
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, bytes);
  bulk_g2s(buf, a, bytes, bar);
  *w = a - c.sb;
  *n = bytes;
  *e = 1;
}

__device__ __forceinline__ bool ch_wait0(Chain& c) {
  if (!c.e0) return true;
  const bool ok = mbar_wait(c.m0, c.p0);
  c.p0 ^= 1u;
  c.e0 = 0;
  return ok;
}

__device__ __forceinline__ bool ch_wait1(Chain& c) {
  if (!c.e1) return true;
  const bool ok = mbar_wait(c.m1, c.p1);
  c.p1 ^= 1u;
  c.e1 = 0;
  return ok;
}

// Starts the copy of the window that follows the current one.  None when
// the current window already reaches the stream's end: for a stream shorter
// than the overlap, the next window's start (window end - COVL) would lie
// before the stream, and, for the first page of a file, before the buffer.
__device__ __forceinline__ void ch_prefetch(Chain& c) {
  const int64_t end = c.w0 + c.n0;  // stream offset just past the window
  const int64_t nxt = end - COVL;
  if (end <= static_cast<int64_t>(c.slen) && nxt > c.w0)
    ch_issue(c, c.b1, c.m1, nxt, &c.w1, &c.n1, &c.e1);
  else
    c.n1 = 0;
}

__device__ __forceinline__ void ch_init(Chain& c, uint8_t* buf0, uint8_t* buf1, uint64_t* bar0, uint64_t* bar1,
                                        uint32_t par0, uint32_t par1, uint32_t cap = CWIN) {
  c.cap = cap;
  c.b0 = buf0;
  c.b1 = buf1;
  c.m0 = bar0;
  c.m1 = bar1;
  c.p0 = par0;
  c.p1 = par1;
  c.w0 = c.w1 = 0;
  c.n0 = c.n1 = 0;
  c.e0 = c.e1 = 0;
  c.swapped = 0;
  c.sb = nullptr;
  c.slen = 0;
}

// Physical-buffer parities (to carry them across uses of the windows).
__device__ __forceinline__ uint32_t ch_par(const Chain& c, int phys) {
  return (phys == 0) == (c.swapped == 0) ? c.p0 : c.p1;
}

__device__ __forceinline__ bool ch_start(Chain& c, const uint8_t* sb, uint32_t slen) {
  c.sb = sb;
  c.slen = slen;
  c.n1 = 0;
  ch_issue(c, c.b0, c.m0, 0, &c.w0, &c.n0, &c.e0);
  if (!ch_wait0(c)) return false;
  ch_prefetch(c);
  return true;
}

// Makes stream bytes [pos, pos + need) readable in the current window.
__device__ __forceinline__ bool ch_ensure(Chain& c, int64_t pos, uint32_t need) {
  int64_t o = pos - c.w0;
  if (o >= 0 && o + need <= c.n0) return true;
  if (!ch_wait1(c)) return false;
  o = pos - c.w1;
  if (c.n1 && o >= 0 && o + need <= c.n1) {
    ch_swap(c);
    ch_prefetch(c);
    return true;
  }
  // a jump past the prefetched window: load at pos, then prefetch after it
  ch_issue(c, c.b0, c.m0, pos, &c.w0, &c.n0, &c.e0);
  if (!ch_wait0(c)) return false;
  ch_prefetch(c);
  return true;
}

__device__ __forceinline__ bool ch_drain(Chain& c) {
  const bool a = ch_wait0(c);
  const bool b = ch_wait1(c);
  return a && b;
}

__device__ __forceinline__ const uint8_t* ch_ptr(const Chain& c, int64_t pos) { return c.b0 + (pos - c.w0); }

// 8 bytes at stream position pos as two little-endian words (aligned loads).
__device__ __forceinline__ void ch_read8(const Chain& c, int64_t pos, uint32_t* lo, uint32_t* hi) {
  const uint32_t o = static_cast<uint32_t>(pos - c.w0);
  const uint32_t* w = reinterpret_cast<const uint32_t*>(c.b0) + (o >> 2);
  const uint32_t sh = (o & 3) * 8;
  const uint32_t a = w[0], b = w[1], d = w[2];
  *lo = sh ? __funnelshift_r(a, b, sh) : a;
  *hi = sh ? __funnelshift_r(b, d, sh) : b;
}

// ULEB128 from a window pointer with 16 readable bytes.
__device__ __forceinline__ int uleb_p(const uint8_t* q, uint64_t* v) {
  uint64_t r = 0;
#pragma unroll 1
  for (int i = 0; i < 10; ++i) {
    const uint32_t b = q[i];
    r |= static_cast<uint64_t>(b & 0x7f) << (7 * i);
    if (!(b & 0x80)) {
      *v = r;
      return i + 1;
    }
  }
  return 0;
}

// ------------------------------------------------------------------ string dictionaries

// BYTE_ARRAY dictionary pages: entries are (4-byte little-endian length,
// bytes) back to back, so the entry starts form a chain.  The chain is found
// per STR_REGION bytes in parallel: region i > 0 searches a lead-in before
// its first byte for an offset where four consecutive entries are plausible
// (a length that fits in the page), a look-alike start usually rejoins the
// true chain within an entry or two, and k_sfix stitches the regions,
// walking serially only where a region's start was wrong.
constexpr int SREG_LEAD = 1024;
constexpr int SREG_SMEM = SREG_LEAD + STR_REGION + 64;

__device__ __forceinline__ uint32_t sle32(const uint8_t* b, uint32_t o) {
  return static_cast<uint32_t>(b[o]) | (static_cast<uint32_t>(b[o + 1]) << 8) |
         (static_cast<uint32_t>(b[o + 2]) << 16) | (static_cast<uint32_t>(b[o + 3]) << 24);
}

__global__ void __launch_bounds__(32) k_sreg(const DictJob* __restrict__ jobs, DictScratch ds, DevStatus* st) {
  extern __shared__ __align__(16) uint8_t smraw[];
  __shared__ uint64_t bar;
  const int lane = threadIdx.x;
  const DictJob j = jobs[blockIdx.y];
  if (j.ptype != T_BYTE_ARRAY || static_cast<int>(blockIdx.x) >= j.sreg_cap) return;
  const int i = blockIdx.x;
  const uint32_t blen = static_cast<uint32_t>(j.body_len);
  DeltaRegion* R = ds.regs + j.sreg + i;
  uint64_t* list = ds.lists + static_cast<uint64_t>(j.sreg + i) * STR_REGION_LIST;
  const uint64_t start64 = static_cast<uint64_t>(i) * STR_REGION;
  if (start64 >= blen) {
    if (lane == 0) *R = DeltaRegion{-1, -1, 0, 0};
    return;
  }
  const uint32_t start = static_cast<uint32_t>(start64);
  const uint32_t end = blen - start < static_cast<uint32_t>(STR_REGION) ? blen : start + STR_REGION;
  const uint32_t sstart = i == 0 ? 0u : start - SREG_LEAD;
  // stage [sstart, end + 8), 16-byte aligned; at most 16 bytes past the body
  const uint8_t* g = j.body + sstart;
  const uint8_t* ga = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(g) & ~uintptr_t(15));
  const uint32_t shift = static_cast<uint32_t>(g - ga);
  const uint64_t lim_end = end + 8 < blen ? end + 8 : blen;
  uint32_t bytes = static_cast<uint32_t>(((j.body + lim_end) - ga + 16) & ~int64_t(15));
  if (bytes > static_cast<uint32_t>(SREG_SMEM)) bytes = SREG_SMEM;
  if (lane == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar, bytes);
    bulk_g2s(smraw, ga, bytes, &bar);
  }
  __syncwarp();
  const bool ok = mbar_wait(&bar, 0);
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) {
      report(st, DERR_TIMEOUT, j.page, WHERE_DICT, 30);
      mbar_wait(&bar, 0);
      *R = DeltaRegion{-1, -1, 0, 0};
    }
    return;
  }
  const uint32_t known_end = sstart - shift + bytes > blen ? blen : sstart - shift + bytes;
  auto at = [&](uint32_t s) -> uint32_t { return s - sstart + shift; };
  // next entry start after the entry at p: 0 when implausible, 0xffffffff when not decidable
  auto next = [&](uint32_t p) -> uint32_t {
    if (p + 4 > known_end) return 0xffffffffu;
    const uint32_t L = sle32(smraw, at(p));
    if (L > blen - p - 4) return 0u;
    return p + 4 + L;
  };
  uint32_t q = 0xffffffffu;
  if (i == 0) {
    q = 0;
  } else {
    for (uint32_t c0 = sstart; c0 < end && q == 0xffffffffu; c0 += 32) {
      const uint32_t cand = c0 + lane;
      bool good = cand < end;
      uint32_t p = cand;
      // four entries in a row, each decided from the staged bytes (a
      // look-alike length can jump past them: undecided is not plausible)
      for (int k = 0; good && k < 4 && p < blen; ++k) {
        const uint32_t nx = next(p);
        if (nx == 0u || nx == 0xffffffffu) good = false;
        else p = nx;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, good);
      if (m) q = c0 + __ffs(m) - 1;
    }
  }
  if (lane == 0) {
    int32_t first = -1, cnt = 0, x = -1;
    if (q != 0xffffffffu) {
      uint32_t p = q;
      while (true) {
        if (p >= end) {
          x = static_cast<int32_t>(p);
          break;
        }
        const uint32_t nx = next(p);
        if (p >= start) {
          if (cnt == STR_REGION_LIST) break;
          if (first < 0) first = static_cast<int32_t>(p);
          // the entry as the dictionary holds it, when its length is known
          list[cnt++] = nx == 0u || nx == 0xffffffffu ? (static_cast<uint64_t>(p + 4) << 32) | 0xffffffffu
                                                      : (static_cast<uint64_t>(p + 4) << 32) | (nx - p - 4);
        }
        if (nx == 0u || nx == 0xffffffffu) break;  // a look-alike chain
        p = nx;
      }
    }
    *R = DeltaRegion{first, first >= 0 ? x : -1, cnt, 0};
  }
}

// Per BYTE_ARRAY dictionary page: stitch the regions (as k_dfix does for
// DELTA blocks), then write every entry as (chars offset << 32) | length.
// A region whose found start is not the true entry is walked again from the
// true entry, in shared memory (the region is staged by one bulk copy), its
// entries written directly.
__global__ void __launch_bounds__(256) k_sfix(const DictJob* __restrict__ jobs, DictScratch ds, DictDev* dicts,
                                              DevStatus* st) {
  constexpr int MAXR = 2048;
  __shared__ int32_t s_q[MAXR], s_x[MAXR], s_c[MAXR];
  __shared__ int32_t s_skip[MAXR], s_base[MAXR];
  __shared__ int32_t s_nreg, s_ok;
  __shared__ uint64_t s_bar;
  __shared__ __align__(16) uint8_t s_stage[STR_REGION + 64];
  const DictJob j = jobs[blockIdx.x];
  if (j.ptype != T_BYTE_ARRAY) return;
  const uint32_t blen = static_cast<uint32_t>(j.body_len);
  const int32_t n = j.n;
  const int nreg = static_cast<int>((static_cast<uint64_t>(blen) + STR_REGION - 1) / STR_REGION);
  const bool regions = nreg <= j.sreg_cap && nreg <= MAXR;
  if (regions)
    for (int i = threadIdx.x; i < nreg; i += blockDim.x) {
      const DeltaRegion r = ds.regs[j.sreg + i];
      s_q[i] = r.q;
      s_x[i] = r.x;
      s_c[i] = r.cnt;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    uint32_t parity = 0;
    bool bad = false;
    uint32_t e = 0;
    int32_t b = 0;
    if (!regions) {
      // pages too large for the region tables: one serial walk in global memory
      while (e < blen && b < n) {
        if (e + 4 > blen) { bad = true; break; }
        const uint32_t L = ld_le32_g(j.body + e);
        if (L > blen - e - 4) { bad = true; break; }
        j.str_ent[b++] = (static_cast<uint64_t>(e + 4) << 32) | L;
        e += 4 + L;
      }
      s_nreg = 0;
    } else {
      for (int i = 0; i < nreg; ++i) {
        const uint32_t start = static_cast<uint32_t>(i) * STR_REGION;
        const uint32_t end = blen - start < static_cast<uint32_t>(STR_REGION) ? blen : start + STR_REGION;
        s_skip[i] = -1;
        if (b >= n || e >= end || bad) continue;
        if (s_q[i] >= 0 && s_c[i] > 0 && s_x[i] >= 0 && static_cast<uint32_t>(s_q[i]) == e) {
          const int32_t c = s_c[i] < n - b ? s_c[i] : n - b;
          s_skip[i] = c;  // entries taken from the list
          s_base[i] = b;
          b += c;
          e = static_cast<uint32_t>(s_x[i]);
          continue;
        }
        // stage [e, end + 8) (at most STR_REGION + 24 bytes: e >= start)
        const uint8_t* g = j.body + e;
        const uint8_t* ga = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(g) & ~uintptr_t(15));
        const uint32_t shift = static_cast<uint32_t>(g - ga);
        const uint64_t lim = end + 8 < blen ? end + 8 : blen;
        uint32_t bytes = static_cast<uint32_t>(((j.body + lim) - ga + 16) & ~int64_t(15));
        if (bytes > sizeof(s_stage)) bytes = sizeof(s_stage);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar, bytes);
        bulk_g2s(s_stage, ga, bytes, &s_bar);
        if (!mbar_wait(&s_bar, parity)) {
          report(st, DERR_TIMEOUT, j.page, WHERE_DICT, 31);
          mbar_wait(&s_bar, parity);
          bad = true;
          continue;
        }
        parity ^= 1u;
        const uint32_t e0 = e;
        const uint32_t known = e0 - shift + bytes > blen ? blen : e0 - shift + bytes;
        while (e < end && b < n) {
          if (e + 4 > known) { bad = true; break; }
          const uint32_t L = sle32(s_stage, e - e0 + shift);
          if (L > blen - e - 4) { bad = true; break; }
          j.str_ent[b++] = (static_cast<uint64_t>(e + 4) << 32) | L;
          e += 4 + L;
        }
      }
      s_nreg = nreg;
    }
    s_ok = !bad && b == n && (n == 0 || e == blen);
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) report(st, DERR_CORRUPT, j.page, WHERE_DICT, 2);
    return;
  }
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = threadIdx.x >> 5; i < s_nreg; i += nw) {
    if (s_skip[i] <= 0) continue;
    const uint64_t* list = ds.lists + static_cast<uint64_t>(j.sreg + i) * STR_REGION_LIST;
    for (int k = lane; k < s_skip[i]; k += 32) j.str_ent[s_base[i] + k] = list[k];
  }
  __syncthreads();
  // longest entry: picks the padded layout (copied by k_dict_pad)
  __shared__ int32_t s_max;
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  int32_t mx = 0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int32_t L = static_cast<int32_t>(static_cast<uint32_t>(j.str_ent[i]));
    mx = L > mx ? L : mx;
  }
  atomicMax(&s_max, mx);
  __syncthreads();
  if (threadIdx.x == 0) {
    DictDev d{};
    d.str_ent = j.str_ent;
    d.n = n;
    d.max_len = s_max;
    d.chars = j.pad && n > 0 && s_max <= PAD_STRIDE_MAX ? j.pad : j.body;
    d.valid = 1;
    dicts[j.chunk] = d;
  }
}

// Padded copy of the string dictionaries k_sfix marked for it: thread i
// copies entry i (aligned words, the last one masked) to pad + i * stride
// and points the entry there.  The bytes after an entry up to the next
// stride are left as they are (never read as data).
__global__ void __launch_bounds__(256) k_dict_pad(const DictJob* __restrict__ jobs, const DictDev* dicts) {
  const DictJob j = jobs[blockIdx.y];
  if (j.ptype != T_BYTE_ARRAY || !j.pad) return;
  const DictDev d = dicts[j.chunk];
  if (!d.valid || d.chars != j.pad) return;
  const uint32_t stride = (static_cast<uint32_t>(d.max_len) + 15u) & ~15u;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < j.n; i += gridDim.x * blockDim.x) {
    const uint64_t e = j.str_ent[i];
    const uint32_t len = static_cast<uint32_t>(e);
    const uint8_t* src = j.body + (e >> 32);
    uint32_t* dst = reinterpret_cast<uint32_t*>(j.pad + static_cast<uint64_t>(i) * stride);
    const uint32_t* q = reinterpret_cast<const uint32_t*>(reinterpret_cast<uintptr_t>(src) & ~uintptr_t(3));
    const uint32_t sh = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 3) * 8;
    const uint32_t nw = (len + 3) >> 2;
    uint32_t cur = nw ? q[0] : 0u;
    for (uint32_t k = 0; k < nw; ++k) {
      const uint32_t nx = q[k + 1];
      dst[k] = __funnelshift_r(cur, nx, sh);
      cur = nx;
    }
    j.str_ent[i] = (static_cast<uint64_t>(static_cast<uint64_t>(i) * stride) << 32) | len;
  }
}

void launch_dict(const DictJob* jobs, int n_jobs, int max_fixed_bytes, int max_str_regions, DictScratch ds,
                 DictDev* dicts, int n_sms, DevStatus* st, cudaStream_t s) {
  if (n_jobs <= 0) return;
  int gx = (max_fixed_bytes / 4 + 256 * 16 - 1) / (256 * 16);
  if (gx < 1) gx = 1;
  if (gx > 4 * n_sms) gx = 4 * n_sms;
  k_dict_fixed<<<dim3(gx, n_jobs), 256, 0, s>>>(jobs, dicts, st);
  if (max_str_regions > 0) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_sreg, cudaFuncAttributeMaxDynamicSharedMemorySize, SREG_SMEM);
      attr = true;
    }
    k_sreg<<<dim3(max_str_regions, n_jobs), 32, SREG_SMEM, s>>>(jobs, ds, st);
    k_sfix<<<n_jobs, 256, 0, s>>>(jobs, ds, dicts, st);
    k_dict_pad<<<dim3(32, n_jobs), 256, 0, s>>>(jobs, dicts);
  }
}

// ------------------------------------------------------------------ walk

struct WalkSmem {
  uint64_t bar[2];
  int32_t ctl[24];
  int64_t c64[8];
  uint32_t rpos[RB];   // hybrid: run header offset; levels: run data offset
  int32_t rk[RB];      // hybrid: dense index at run start; levels: row at run start
  int32_t rcnt[RB];    // levels: rows of the run inside the page
  uint32_t rmeta[RB];  // levels: 0x80000000 bit-packed, else the repeated value
  int32_t rpre[RB];    // levels: valid rows before the run (page-relative)
  int32_t tmp32[32];
  uint32_t hop[RB / 32];  // levels: table offsets of chain positions 32 runs apart
  // two chain windows of ctl[13] + 16 bytes each follow the struct, then
  // (level walks) three jump tables of ctl[16] 16-bit entries
};
constexpr uint32_t JW = 2048;  // level-stream bytes covered by one set of jump tables
constexpr uint16_t JSENT = 0xffffu;
__host__ __device__ constexpr uint32_t walk_smem_bytes(uint32_t cap, uint32_t jw = 0) {
  return ((static_cast<uint32_t>(sizeof(WalkSmem)) + 15u) & ~15u) + 2u * (cap + 16u) + 3u * 2u * jw;
}

// Page layout.
struct PageCtx {
  const uint8_t* body;
  uint32_t blen;
  uint32_t lv0, lv1;  // definition levels
  uint32_t v0;        // value stream start
  int32_t nrows;
  int32_t pgid;
  int32_t enc;
  int32_t ptype;
  int32_t width;
  int32_t max_def;
};

__device__ bool page_ctx(const DecodeArgs& a, const PlanPage& pp, PageCtx* pc) {
  const PageDev pg = a.pages[pp.page];
  const ChunkDev ch = a.chunks[pp.chunk];
  pc->body = pp.body;
  pc->blen = static_cast<uint32_t>(pp.body_len);
  pc->nrows = pg.num_values;
  pc->pgid = static_cast<int32_t>(pp.page);
  pc->enc = pp.enc;
  pc->ptype = ch.ptype;
  pc->width = ch.width;
  pc->max_def = ch.max_def;
  pc->lv0 = pc->lv1 = 0;
  if (pg.page_type == PAGE_DATA) {
    if (ch.max_def) {
      if (pc->blen < 4) return false;
      const uint32_t L = ld_le32_g(pc->body);
      if (L > pc->blen - 4) return false;
      pc->lv0 = 4;
      pc->lv1 = 4 + L;
    }
    pc->v0 = pc->lv1;
  } else {
    if (pg.rep_len != 0) return false;
    if (static_cast<uint32_t>(pg.def_len) > pc->blen) return false;
    if (!ch.max_def && pg.def_len != 0) return false;
    pc->lv1 = static_cast<uint32_t>(pg.def_len);
    pc->v0 = pc->lv1;
  }
  return true;
}

__device__ __forceinline__ Chain make_chain(WalkSmem& sm) {
  Chain c;
  const uint32_t cap = static_cast<uint32_t>(sm.ctl[13]);
  uint8_t* w0 = reinterpret_cast<uint8_t*>(&sm) + ((sizeof(WalkSmem) + 15) & ~size_t(15));
  ch_init(c, w0, w0 + cap + 16, &sm.bar[0], &sm.bar[1], static_cast<uint32_t>(sm.ctl[14]),
          static_cast<uint32_t>(sm.ctl[15]), cap);
  return c;
}

__device__ __forceinline__ void keep_parity(WalkSmem& sm, const Chain& c) {
  sm.ctl[14] = static_cast<int32_t>(ch_par(c, 0));
  sm.ctl[15] = static_cast<int32_t>(ch_par(c, 1));
}

// Valid rows among the first `n` rows of level run j (bits from global memory).
// Bits [b, b + w) (w <= 32) at `base`, shared or global memory (plain loads).
__device__ __forceinline__ uint32_t lbits32(const uint8_t* base, uint64_t b, int w) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(base) + (b >> 3);
  const uint32_t* q = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  const uint32_t sh = static_cast<uint32_t>((a & 3) * 8 + (b & 7));
  const uint64_t v = ((static_cast<uint64_t>(q[1]) << 32) | q[0]) >> sh;
  return w >= 32 ? static_cast<uint32_t>(v) : static_cast<uint32_t>(v) & ((1u << w) - 1u);
}

// Valid rows among the first `n` rows of level run j.  Stream byte p is at
// lb[p - lp0] (the staged window, or the page in global memory).
__device__ __forceinline__ int32_t run_valid(const WalkSmem& sm, const uint8_t* lb, uint32_t lp0, int j, int32_t n) {
  const uint32_t meta = sm.rmeta[j];
  if (!(meta & 0x80000000u)) return static_cast<int32_t>(meta) * n;
  int32_t c = 0;
  const uint64_t b0 = static_cast<uint64_t>(sm.rpos[j] - lp0) * 8;
  for (int32_t x = 0; x < n; x += 32) {
    const int m = n - x < 32 ? n - x : 32;
    c += __popc(lbits32(lb, b0 + x, m));
  }
  return c;
}

__device__ __forceinline__ int find_run(const int32_t* key, int nb, int32_t v) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Definition levels of one page: validity bits of rows [row_lo, row_hi) and
// the dense start (k0) / count (nn) of every item.  Returns the page's
// non-null count, -1 on error.
__device__ int32_t walk_levels(WalkSmem& sm, const PageCtx& pc, const PlanPage& pp, Item* items, const OutCol& col,
                               DevStatus* st) {
  const int tid = threadIdx.x;
  const uint8_t* lsb = pc.body + pc.lv0;
  const uint32_t slen = pc.lv1 - pc.lv0;
  Chain c = make_chain(sm);
  if (tid == 0) {
    sm.ctl[0] = 0;   // chain position
    sm.ctl[1] = 0;   // rows consumed
    sm.c64[0] = 0;   // valid rows before the batch
    sm.c64[1] = -1;  // k at row_hi
    sm.ctl[6] = 0;   // a malformed header in a batch
    sm.ctl[5] = pc.nrows > 0 && !ch_start(c, lsb, slen) ? 3 : 0;
  }
  __syncthreads();
  const uint32_t jw = static_cast<uint32_t>(sm.ctl[16]);
  for (uint32_t guard = 0; guard <= slen + 2 && !sm.ctl[5] && sm.ctl[1] < pc.nrows; ++guard) {
    // With jump tables: for every byte of the next jw stream bytes, the
    // block computes where a run starting there would end (were that byte a
    // one-byte header), then doubles the map five times; thread 0 steps 32
    // runs at a time through it and the block fills in the runs between the
    // steps.  Such a batch ends where the tables end; when it would hold no
    // run (a longer header, the stream's or the window's end) the batch is
    // gathered by the serial walk instead.
    bool jumped = false;
    const uint8_t* lb = lsb;  // where the batch's level bytes are read: stream byte p at lb[p - lp0]
    uint32_t lp0 = 0;
    if (jw) {
      uint16_t* j1 = reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(&sm) +
                                                 walk_smem_bytes(static_cast<uint32_t>(sm.ctl[13])));
      uint16_t* ja = j1 + jw;
      uint16_t* jb = ja + jw;
      if (tid == 0) {
        const uint32_t pos = static_cast<uint32_t>(sm.ctl[0]);
        int err = 0;
        // the window must hold the tables' bytes and 16 more
        const uint32_t need = (slen - pos < jw ? slen - pos : jw) + 16;
        if (pos >= slen)
          err = 1;
        else if (!ch_ensure(c, pos, need))
          err = 3;
        sm.ctl[5] = err;
        if (!err) {
          const uint32_t o0 = static_cast<uint32_t>(pos - c.w0);
          const uint32_t room = c.n0 - 16 > o0 ? c.n0 - 16 - o0 : 0u;
          uint32_t L = room < jw ? room : jw;
          L = L < slen - pos ? L : slen - pos;
          sm.ctl[17] = static_cast<int32_t>(c.b0 - reinterpret_cast<uint8_t*>(&sm)) + static_cast<int32_t>(o0);
          sm.ctl[18] = static_cast<int32_t>(L);
        }
      }
      __syncthreads();
      if (sm.ctl[5]) break;
      const uint8_t* wb = reinterpret_cast<const uint8_t*>(&sm) + sm.ctl[17];
      const uint32_t L = static_cast<uint32_t>(sm.ctl[18]);
      const uint32_t pos0 = static_cast<uint32_t>(sm.ctl[0]);
      // bit width 1: a bit-packed run spans its header and a byte per group,
      // a repeated run its header and one value byte (headers of 1-5 bytes;
      // the window holds 16 bytes past the tables)
      for (uint32_t q = tid; q < L; q += blockDim.x) {
        uint32_t h = wb[q], hl = 1;
        if (h & 0x80u) {
          h &= 0x7fu;
          for (uint32_t k = 1; k < 5; ++k) {
            const uint32_t bk = wb[q + k];
            h |= (bk & 0x7fu) << (7 * k);
            ++hl;
            if (!(bk & 0x80u)) break;
            if (k == 4) hl = 0;  // longer than five bytes: left to the serial walk
          }
        }
        const uint64_t nx = static_cast<uint64_t>(q) + hl + ((h & 1u) ? (h >> 1) : 1u);
        const uint16_t v = !hl || nx >= L ? JSENT : static_cast<uint16_t>(nx);
        j1[q] = v;
        ja[q] = v;
      }
      __syncthreads();
      uint16_t* src = ja;
      uint16_t* dst = jb;
#pragma unroll 1
      for (int r = 0; r < 5; ++r) {  // 2, 4, 8, 16, 32 runs
        for (uint32_t q = tid; q < L; q += blockDim.x) {
          const uint16_t m = src[q];
          dst[q] = m == JSENT ? JSENT : src[m];
        }
        __syncthreads();
        uint16_t* t = src;
        src = dst;
        dst = t;
      }
      if (tid == 0) {
        int nb = 0, nh = 0;
        uint32_t q = 0;
        while (L > 0 && nb + 32 <= RB && src[q] != JSENT) {
          sm.hop[nh++] = q;
          nb += 32;
          q = src[q];
        }
        while (L > 0 && nb < RB && j1[q] != JSENT) {
          sm.rpos[nb++] = pos0 + q;
          q = j1[q];
        }
        sm.ctl[19] = nh;
        sm.ctl[2] = nb;
        if (nb) sm.ctl[0] = static_cast<int32_t>(pos0 + q);
      }
      __syncthreads();
      const int nh = sm.ctl[19];
      for (int h = tid; h < nh; h += blockDim.x) {
        uint32_t q = sm.hop[h];
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
          sm.rpos[32 * h + k] = pos0 + q;
          q = j1[q];
        }
      }
      jumped = sm.ctl[2] > 0;
      if (jumped) {
        lb = wb;
        lp0 = pos0;
      }
      __syncthreads();
    }
    // thread 0 follows the chain and records only each run's header
    // offset; the block decodes the headers of the batch afterwards
    if (!jumped && tid == 0) {
      uint32_t pos = static_cast<uint32_t>(sm.ctl[0]);
      int32_t row = sm.ctl[1];
      int nb = 0, err = 0;
      while (nb < RB && row < pc.nrows) {
        if (pos >= slen) { err = 1; break; }
        if (!ch_ensure(c, pos, 16)) { err = 3; break; }
        {
          // fast steps: one-byte run headers inside the current window
          uint32_t o = static_cast<uint32_t>(pos - c.w0);
          const uint32_t lim = c.n0 - 16;
          const uint32_t wb = static_cast<uint32_t>(c.w0);
          const uint8_t* b = c.b0;
          uint32_t h = o <= lim ? b[o] : 0x80u;
          while (nb < RB && row < pc.nrows && !(h & 0x80u)) {
            const uint32_t g = h >> 1;
            const uint32_t on = o + ((h & 1u) ? 1 + g : 2);
            const uint32_t hn = on <= lim ? b[on] : 0x80u;
            sm.rpos[nb++] = o + wb;
            row += static_cast<int32_t>((h & 1u) ? g << 3 : g);
            o = on;
            h = hn;
          }
          pos = o + wb;
          if (nb >= RB || row >= pc.nrows) break;
          if (pos >= slen) { err = 1; break; }
          if (!ch_ensure(c, pos, 16)) { err = 3; break; }
        }
        const uint8_t* q = ch_ptr(c, pos);
        uint64_t h;
        const int hl = uleb_p(q, &h);
        if (!hl) { err = 1; break; }
        const uint64_t cnt = (h & 1) ? (h >> 1) * 8 : h >> 1;
        const uint64_t adv = hl + ((h & 1) ? (h >> 1) : 1);
        if (static_cast<uint64_t>(pos) + adv > slen) { err = 1; break; }
        sm.rpos[nb++] = pos;
        row = cnt >= static_cast<uint64_t>(pc.nrows - row) ? pc.nrows : row + static_cast<int32_t>(cnt);
        pos += static_cast<uint32_t>(adv);
      }
      if (!err && pos > slen) err = 1;
      sm.ctl[0] = static_cast<int32_t>(pos);
      sm.ctl[2] = nb;
      sm.ctl[5] = err;
    }
    __syncthreads();
    if (sm.ctl[5]) break;
    const int nb = sm.ctl[2];
    const int32_t b0 = sm.ctl[1];
    // decode the batch's headers: data offset, rows (clipped to the page),
    // kind / repeated value; rows before each run by a block scan
    {
      int32_t cntv[4];
      uint32_t dpos[4], meta[4];
      int32_t mine = 0;
      int bad = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = tid * 4 + q;
        cntv[q] = 0;
        dpos[q] = 0;
        meta[q] = 0;
        if (j < nb) {
          const uint32_t hp = sm.rpos[j];
          uint64_t h = 0;
          const int hl = uleb([&](uint32_t x) { return static_cast<uint32_t>(lb[x - lp0]); }, hp, slen, &h);
          if (!hl) bad = 1;
          const bool packed = h & 1;
          const uint64_t cnt = packed ? (h >> 1) * 8 : h >> 1;
          dpos[q] = hp + hl;
          if (!packed) {
            meta[q] = hp + hl < slen ? static_cast<uint32_t>(lb[hp + hl - lp0]) : 2u;
            if (meta[q] > 1) bad = 1;
          } else {
            meta[q] = 0x80000000u;
          }
          cntv[q] = cnt > static_cast<uint64_t>(pc.nrows) ? pc.nrows : static_cast<int32_t>(cnt);
          mine += cntv[q];
        }
      }
      if (bad) sm.ctl[6] = 1;
      int32_t total;
      int32_t run = b0 + block_exclusive_sum(mine, sm.tmp32, &total);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = tid * 4 + q;
        if (j < nb) {
          const int32_t take = cntv[q] < pc.nrows - run ? cntv[q] : (pc.nrows - run > 0 ? pc.nrows - run : 0);
          sm.rpos[j] = dpos[q];
          sm.rk[j] = run;
          sm.rcnt[j] = take;
          sm.rmeta[j] = meta[q];
          run += cntv[q];
        }
      }
      __syncthreads();
      if (tid == 0) {
        int32_t e = b0 + total;
        sm.ctl[4] = e < pc.nrows ? e : pc.nrows;
        if (sm.ctl[6]) sm.ctl[5] = 1;
      }
      __syncthreads();
      if (sm.ctl[5]) break;
    }
    const int32_t b1 = sm.ctl[4];
    // valid counts per run, prefix over the batch (4 consecutive runs per thread)
    int32_t loc[4];
    int32_t mine = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = tid * 4 + q;
      loc[q] = j < nb ? run_valid(sm, lb, lp0, j, sm.rcnt[j]) : 0;
      mine += loc[q];
    }
    int32_t total;
    const int32_t pre = block_exclusive_sum(mine, sm.tmp32, &total);
    const int32_t vb = static_cast<int32_t>(sm.c64[0]);
    {
      int32_t run = vb + pre;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = tid * 4 + q;
        if (j < nb) sm.rpre[j] = run;
        run += loc[q];
      }
    }
    __syncthreads();
    // validity bits of rows [max(b0,row_lo), min(b1,row_hi))
    if (nb > 0 && col.validity) {
      const int32_t r_lo = b0 > pp.row_lo ? b0 : pp.row_lo;
      const int32_t r_hi = b1 < pp.row_hi ? b1 : pp.row_hi;
      if (r_lo < r_hi) {
        const int64_t o0 = pp.out_row + r_lo, o1 = pp.out_row + r_hi;
        const int64_t w0 = o0 >> 5, w1 = (o1 - 1) >> 5;
        for (int64_t w = w0 + tid; w <= w1; w += blockDim.x) {
          const int64_t a0 = w * 32 > o0 ? w * 32 : o0;
          const int64_t e0 = w * 32 + 32 < o1 ? w * 32 + 32 : o1;
          uint32_t word = 0;
          int32_t r = static_cast<int32_t>(a0 - pp.out_row);
          const int32_t rend = static_cast<int32_t>(e0 - pp.out_row);
          for (int j = find_run(sm.rk, nb, r); j < nb && r < rend; ++j) {
            int32_t s1 = sm.rk[j] + sm.rcnt[j];
            if (s1 > rend) s1 = rend;
            if (s1 <= r) continue;
            const int n = s1 - r;
            const uint32_t meta = sm.rmeta[j];
            uint32_t bitsv;
            if (meta & 0x80000000u)
              bitsv = lbits32(lb, static_cast<uint64_t>(sm.rpos[j] - lp0) * 8 + (r - sm.rk[j]), n);
            else
              bitsv = meta ? (n == 32 ? 0xffffffffu : ((1u << n) - 1u)) : 0u;
            word |= bitsv << static_cast<uint32_t>((pp.out_row + r) - w * 32);
            r = s1;
          }
          if (a0 == w * 32 && e0 == w * 32 + 32)
            col.validity[w] = word;
          else if (word)
            atomicOr(col.validity + w, word);
        }
      }
    }
    // dense index at each item start (and at row_hi) inside the batch
    for (uint32_t i = tid; i <= pp.item_count; i += blockDim.x) {
      const int32_t R = i < pp.item_count ? items[pp.item_begin + i].row0 : pp.row_hi;
      if (nb > 0 && R >= b0 && R < b1) {
        const int j = find_run(sm.rk, nb, R);
        const int32_t kR = sm.rpre[j] + run_valid(sm, lb, lp0, j, R - sm.rk[j]);
        if (i < pp.item_count)
          items[pp.item_begin + i].k0 = kR;
        else
          sm.c64[1] = kR;
      }
    }
    __syncthreads();
    if (tid == 0) {
      sm.c64[0] = vb + total;
      sm.ctl[1] = b1;
      if (nb == 0 && b1 < pc.nrows) sm.ctl[5] = 1;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (!ch_drain(c) && !sm.ctl[5]) sm.ctl[5] = 3;
    if (!sm.ctl[5] && sm.ctl[1] < pc.nrows) sm.ctl[5] = 1;
    keep_parity(sm, c);
  }
  __syncthreads();
  if (sm.ctl[5]) {
    if (tid == 0) report(st, sm.ctl[5] == 3 ? DERR_TIMEOUT : DERR_CORRUPT, pc.pgid, WHERE_WALK_LEVELS, sm.ctl[5]);
    return -1;
  }
  const int32_t nonnull = static_cast<int32_t>(sm.c64[0]);
  const int32_t k_hi = sm.c64[1] >= 0 ? static_cast<int32_t>(sm.c64[1]) : nonnull;
  for (uint32_t i = tid; i < pp.item_count; i += blockDim.x) {
    const int32_t ka = items[pp.item_begin + i].k0;
    const int32_t kb = i + 1 < pp.item_count ? items[pp.item_begin + i + 1].k0 : k_hi;
    items[pp.item_begin + i].nn = kb - ka;
  }
  __syncthreads();
  return nonnull;
}

// Dictionary indices: checkpoints (run header offset, dense index at run
// start) for every item with values.
__device__ bool walk_hybrid(WalkSmem& sm, const uint8_t* sb, uint32_t slen, int bw, int32_t total,
                            const PlanPage& pp, Item* items, int pgid, DevStatus* st) {
  const int tid = threadIdx.x;
  const uint32_t vbytes = (bw + 7) / 8;
  Chain c = make_chain(sm);
  // a bit-packed run of the most groups a one-byte header holds (63, header
  // byte 127) spans `stride` bytes; streams of random indices are made of
  // little else, so such stretches are checked by the whole block at once
  constexpr uint32_t kMaxRun = 127;
  constexpr int kSerialMax = 32;
  const uint64_t stride = 1 + 63ull * static_cast<uint64_t>(bw);
  if (tid == 0) {
    sm.ctl[0] = 0;  // position
    sm.ctl[1] = 0;  // dense index
    sm.ctl[5] = ch_start(c, sb, slen) ? 0 : 3;
    sm.ctl[7] = !sm.ctl[5] && slen > 0 && c.b0[0] == kMaxRun;  // next batch starts with a parallel check
  }
  __syncthreads();
  for (uint32_t guard = 0; guard <= slen + 2 && !sm.ctl[5] && sm.ctl[1] < total; ++guard) {
    if (tid == 0) {
      sm.ctl[9] = 0;             // runs recorded in the batch
      sm.ctl[10] = sm.ctl[1];    // dense index reached
    }
    __syncthreads();
    // a batch is gathered in segments: a parallel check of a stretch of
    // maximal runs (when the next header says one starts there), then thread
    // 0 stepping along the chain until kSerialMax maximal runs in a row
    for (;;) {
      if (sm.ctl[7]) {
        // consecutive maximal runs at pos0 + i * stride, confirmed by reading
        // their header bytes in parallel (the run at pos0 is known to be one)
        const uint32_t pos0 = static_cast<uint32_t>(sm.ctl[0]);
        const int32_t kb = sm.ctl[10];
        const int nb0 = sm.ctl[9];
        const int64_t need = (static_cast<int64_t>(total) - kb + 503) / 504;
        const int imax = static_cast<int>(need < RB - nb0 ? need : RB - nb0);
        __syncthreads();
        if (tid == 0) sm.ctl[8] = imax;
        __syncthreads();
        for (int i = tid; i < imax; i += blockDim.x) {
          const uint64_t p = pos0 + static_cast<uint64_t>(i) * stride;
          if (p + stride > slen || __ldg(sb + p) != kMaxRun) {
            atomicMin(&sm.ctl[8], i);
            break;
          }
        }
        __syncthreads();
        const int m = sm.ctl[8];
        for (int i = tid; i < m; i += blockDim.x) sm.rpos[nb0 + i] = pos0 + static_cast<uint32_t>(i * stride);
        if (tid == 0) {
          sm.ctl[9] = nb0 + m;
          sm.ctl[0] = static_cast<int32_t>(pos0 + m * stride);
          const int64_t ke = static_cast<int64_t>(kb) + 504ll * m;
          sm.ctl[10] = static_cast<int32_t>(ke < total ? ke : total);
        }
      }
      if (tid == 0) {
        uint32_t pos = static_cast<uint32_t>(sm.ctl[0]);
        int64_t k = sm.ctl[10];
        int nb = sm.ctl[9], err = 0;
        int maxrun = 0;  // consecutive maximal runs stepped through
        while (nb < RB && k < total && maxrun < kSerialMax) {
          if (pos >= slen) { err = 1; break; }
          if (!ch_ensure(c, pos, 16)) { err = 3; break; }
          {
            // fast steps: one-byte run headers inside the current window
            uint32_t o = static_cast<uint32_t>(pos - c.w0);
            const uint32_t lim = c.n0 - 16;
            const uint32_t wb = static_cast<uint32_t>(c.w0);
            const uint8_t* b = c.b0;
            int32_t kk = static_cast<int32_t>(k);
            uint32_t h = o <= lim ? b[o] : 0x80u;
            while (nb < RB && kk < total && !(h & 0x80u) && maxrun < kSerialMax) {
              const uint32_t g = h >> 1;
              const uint32_t packed = h & 1u;
              const uint32_t on = o + 1 + (packed ? g * static_cast<uint32_t>(bw) : vbytes);
              const uint32_t hn = on <= lim ? b[on] : 0x80u;
              const uint32_t cnt = packed ? g << 3 : g;
              sm.rpos[nb++] = o + wb;
              kk = static_cast<int32_t>(cnt) < total - kk ? kk + static_cast<int32_t>(cnt) : total;
              maxrun = h == kMaxRun ? maxrun + 1 : 0;
              o = on;
              h = hn;
            }
            pos = o + wb;
            k = kk;
            if (nb >= RB || k >= total || maxrun >= kSerialMax) {
              if (pos > slen) err = 1;
              break;
            }
            if (pos >= slen) { err = 1; break; }
            if (!ch_ensure(c, pos, 16)) { err = 3; break; }
          }
          const uint8_t* q = ch_ptr(c, pos);
          uint64_t h;
          int hl;
          if (q[0] < 0x80) {
            h = q[0];
            hl = 1;
          } else {
            hl = uleb_p(q, &h);
            if (!hl) { err = 1; break; }
          }
          uint64_t cnt, adv;
          if (h & 1) {
            cnt = (h >> 1) << 3;
            adv = hl + (h >> 1) * static_cast<uint64_t>(bw);
          } else {
            cnt = h >> 1;
            adv = hl + vbytes;
          }
          if (static_cast<uint64_t>(pos) + adv > slen) { err = 1; break; }
          sm.rpos[nb++] = pos;
          pos += static_cast<uint32_t>(adv);
          k = k + static_cast<int64_t>(cnt) > total ? total : k + static_cast<int64_t>(cnt);
          maxrun = 0;
        }
        sm.ctl[0] = static_cast<int32_t>(pos);
        sm.ctl[2] = nb;
        sm.ctl[3] = static_cast<int32_t>(k);
        sm.ctl[5] = err;
        sm.ctl[7] = !err && k < total && pos < slen && __ldg(sb + pos) == kMaxRun;
        sm.ctl[9] = nb;
        sm.ctl[10] = static_cast<int32_t>(k);
        sm.ctl[11] = sm.ctl[7] && nb < RB;  // the batch goes on with a parallel check
      }
      __syncthreads();
      if (!sm.ctl[11]) break;
    }
    if (sm.ctl[5]) break;
    {
      // dense index at each run start: headers decoded by the block, a scan
      const int nbb = sm.ctl[2];
      int32_t cntv[4];
      int32_t mine = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = tid * 4 + q;
        cntv[q] = 0;
        if (j < nbb) {
          uint64_t h = 0;
          uleb([&](uint32_t x) { return static_cast<uint32_t>(__ldg(sb + x)); }, sm.rpos[j], slen, &h);
          const uint64_t cnt = (h & 1) ? (h >> 1) << 3 : h >> 1;
          cntv[q] = cnt > static_cast<uint64_t>(total) ? total : static_cast<int32_t>(cnt);
          mine += cntv[q];
        }
      }
      int32_t tot;
      int32_t run = sm.ctl[1] + block_exclusive_sum(mine, sm.tmp32, &tot);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = tid * 4 + q;
        if (j < nbb) sm.rk[j] = run < total ? run : total;
        run += cntv[q];
      }
      __syncthreads();
    }
    const int nb = sm.ctl[2];
    const int32_t kb0 = sm.ctl[1], kb1 = sm.ctl[3];
    for (uint32_t i = tid; i < pp.item_count; i += blockDim.x) {
      Item& it = items[pp.item_begin + i];
      const int32_t ik = it.k0;
      if (nb > 0 && it.nn > 0 && ik >= kb0 && ik < kb1) {
        const int j = find_run(sm.rk, nb, ik);
        it.pos = static_cast<int32_t>(sm.rpos[j]);
        it.run_k0 = sm.rk[j];
        it.base = 0;
      }
    }
    __syncthreads();
    if (tid == 0) {
      sm.ctl[1] = kb1;
      if (nb == 0 && kb1 < total) sm.ctl[5] = 1;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (!ch_drain(c) && !sm.ctl[5]) sm.ctl[5] = 3;
    if (!sm.ctl[5] && sm.ctl[1] < total) sm.ctl[5] = 1;
    keep_parity(sm, c);
  }
  __syncthreads();
  if (sm.ctl[5]) {
    if (tid == 0) report(st, sm.ctl[5] == 3 ? DERR_TIMEOUT : DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 1);
    return false;
  }
  return true;
}

struct DeltaHdr {
  int32_t block, mbc, vpm, total, hlen;
  int64_t first;
};

// DELTA_BINARY_PACKED header: block size (multiple of 128, <= 4096),
// miniblocks per block (<= 32, values per miniblock a multiple of 32),
// total values, first value.
__device__ bool delta_header(const uint8_t* sb, uint32_t slen, DeltaHdr* d) {
  auto get = [&](uint32_t q) { return static_cast<uint32_t>(__ldg(sb + q)); };
  uint64_t a, b, c, f;
  uint32_t p = 0;
  int n;
  if (!(n = uleb(get, p, slen, &a))) return false;
  p += n;
  if (!(n = uleb(get, p, slen, &b))) return false;
  p += n;
  if (!(n = uleb(get, p, slen, &c))) return false;
  p += n;
  if (!(n = uleb(get, p, slen, &f))) return false;
  p += n;
  if (a == 0 || a % 128 || a > 4096 || b == 0 || b > 32 || a % b || (a / b) % 32 || c > 0x7fffffff) return false;
  d->block = static_cast<int32_t>(a);
  d->mbc = static_cast<int32_t>(b);
  d->vpm = static_cast<int32_t>(a / b);
  d->total = static_cast<int32_t>(c);
  d->first = unzigzag(f);
  d->hlen = static_cast<int32_t>(p);
  return true;
}

// DELTA: thread 0 follows the block chain and records every block's stream
// offset.  The common layout (4 miniblocks of 32 values, one-byte min delta,
// a full block) takes the fast step: size = 5 + 4 * (sum of the 4 widths).
__device__ bool walk_delta(WalkSmem& sm, const uint8_t* sb, uint32_t slen, int type_bits, int32_t total,
                           PlanPage* ppw, uint32_t* dpos, uint32_t dcap, bool serial, int pgid, DevStatus* st) {
  if (threadIdx.x == 0) {
    int err = 0;
    DeltaHdr d{};
    if (!delta_header(sb, slen, &d)) err = 2;
    else if (d.total != total) err = 1;
    int32_t nblocks = 0;
    Chain c = make_chain(sm);
    if (!err && !serial) {
      // batched scan: the block chain is found by the parallel region walk
      ppw->dfirst = d.first;
      ppw->dbs = d.block;
      ppw->dvpm = d.vpm;
      ppw->dmbc = d.mbc;
      ppw->dhlen = d.hlen;
      ppw->dblocks = total > 1 ? -2 : 0;
      sm.ctl[5] = 0;
      goto done;
    }
    if (!err && total > 1) {
      if (!ch_start(c, sb, slen)) err = 3;
      int64_t pos = d.hlen;
      int64_t k = 1;
      const bool fast_layout = d.mbc == 4 && d.vpm == 32;
      const int64_t full_end = 1 + static_cast<int64_t>((total - 1) / d.block) * d.block;  // k after the full blocks
      while (!err && k < total) {
        if (pos >= slen || static_cast<uint32_t>(nblocks) >= dcap) { err = 1; break; }
        if (!ch_ensure(c, pos, 48)) { err = 3; break; }
        if (fast_layout && k < full_end) {
          // fast steps: size = 5 + 4 * (sum of the 4 width bytes), all in registers
          uint32_t o = static_cast<uint32_t>(pos - c.w0);
          // near the stream's end the window may hold fewer than 48 bytes:
          // then no fast step (lim would wrap around)
          const bool roomy = c.n0 >= 48u;
          const uint32_t lim = roomy ? c.n0 - 48 : 0u;
          const uint32_t wb = static_cast<uint32_t>(c.w0);
          const uint32_t* w32 = reinterpret_cast<const uint32_t*>(c.b0);
          uint32_t left = static_cast<uint32_t>((full_end - k) / d.block);
          const uint32_t room = dcap - static_cast<uint32_t>(nblocks);
          if (left > room) left = room;
          uint32_t* out = dpos + nblocks;
          uint32_t done = 0;
          // software-pipelined: the next block's header words are loaded
          // before this block's position is stored
          uint32_t x0 = 0, x1 = 0, x2 = 0;
          if (roomy && o <= lim) {
            const uint32_t i = o >> 2;
            x0 = w32[i];
            x1 = w32[i + 1];
            x2 = w32[i + 2];
          }
          while (done < left && roomy && o <= lim) {
            const uint32_t sh = (o & 3u) << 3;
            const uint32_t lo = __funnelshift_r(x0, x1, sh);
            const uint32_t hi = __funnelshift_r(x1, x2, sh);
            const uint32_t wid = __funnelshift_r(lo, hi, 8);
            if ((lo | wid) & 0x80u || wid & 0x80808080u) break;
            const uint32_t on = o + 5u + 4u * __dp4a(wid, 0x01010101u, 0u);
            if (on <= lim) {
              const uint32_t i = on >> 2;
              x0 = w32[i];
              x1 = w32[i + 1];
              x2 = w32[i + 2];
            }
            out[done++] = o + wb;
            o = on;
          }
          nblocks += static_cast<int32_t>(done);
          k += static_cast<int64_t>(done) * d.block;
          pos = o + wb;
          if (k >= total) break;
          if (pos >= slen || static_cast<uint32_t>(nblocks) >= dcap) { err = 1; break; }
          if (!ch_ensure(c, pos, 48)) { err = 3; break; }
        }
        const int32_t nv = total - k < d.block ? static_cast<int32_t>(total - k) : d.block;
        uint32_t size;
        uint32_t lo, hi;
        ch_read8(c, pos, &lo, &hi);
        const uint32_t widths = (lo >> 8) | (hi << 24);
        if (fast_layout && nv == d.block && !(lo & 0x80u) && !(widths & 0x80808080u)) {
          size = 5u + 4u * __dp4a(widths, 0x01010101u, 0u);
        } else {
          if (!ch_ensure(c, pos, 48)) { err = 3; break; }
          const uint8_t* q = ch_ptr(c, pos);
          uint64_t z;
          const int vl = uleb_p(q, &z);
          if (!vl) { err = 1; break; }
          const int used = (nv + d.vpm - 1) / d.vpm;
          uint64_t bits = 0;
          for (int m = 0; m < used; ++m) {
            const uint32_t w = q[vl + m];
            if (static_cast<int>(w) > type_bits) { err = 1; break; }
            bits += static_cast<uint64_t>(w) * d.vpm;
          }
          if (err) break;
          size = static_cast<uint32_t>(vl + d.mbc + bits / 8);
        }
        if (pos + size > slen) { err = 1; break; }
        dpos[nblocks++] = static_cast<uint32_t>(pos);
        pos += size;
        k += nv;
      }
      if (!err && pos > slen) err = 1;
      if (!ch_drain(c) && !err) err = 3;
    }
    keep_parity(sm, c);
    if (err) {
      report(st, err == 3 ? DERR_TIMEOUT : (err == 2 ? DERR_UNSUPPORTED : DERR_CORRUPT), pgid, WHERE_WALK_VALUES, 3);
      ppw->dblocks = -1;
    } else {
      ppw->dblocks = nblocks;
      ppw->dfirst = d.first;
      ppw->dbs = d.block;
      ppw->dvpm = d.vpm;
      ppw->dmbc = d.mbc;
      ppw->dhlen = d.hlen;
    }
    sm.ctl[5] = err;
  }
done:
  __syncthreads();
  return sm.ctl[5] == 0;
}

// PLAIN BYTE_ARRAY: thread 0 follows the (length, bytes) chain and records
// for every item the offset of its first value and the chars before it.
__device__ bool walk_plain_ba(WalkSmem& sm, const uint8_t* sb, uint32_t slen, int32_t total, const PlanPage& pp,
                              Item* items, int pgid, DevStatus* st, const uint32_t* vp) {
  if (vp) {
    // a transcoded page: the transcoder recorded where every value starts
    // (vp[k], and vp[total] = the end of the stream it wrote), so each
    // item's checkpoint is a lookup; the chars before value k are vp[k] - 4 k
    int bad = 0;
    // the table covers exactly `total` values of at least 4 bytes each
    if (threadIdx.x == 0 && (total < 0 || static_cast<uint64_t>(total) * 4 > slen || vp[total] != slen)) bad = 1;
    for (uint32_t i = threadIdx.x; i < pp.item_count; i += blockDim.x) {
      Item& it = items[pp.item_begin + i];
      if (it.nn <= 0) continue;
      const int32_t k = it.k0;
      const uint32_t pos = (k >= 0 && k <= total) ? vp[k] : 0xffffffffu;
      if (pos > slen || pos < 4u * static_cast<uint32_t>(k)) {
        bad = 1;
        continue;
      }
      it.pos = static_cast<int32_t>(pos);
      it.run_k0 = k;
      it.base = static_cast<int64_t>(pos) - 4 * static_cast<int64_t>(k);
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
      if (bad) report(st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 8);
      sm.ctl[5] = bad;
    }
    __syncthreads();
    return !bad;
  }
  if (threadIdx.x == 0) {
    int err = 0;
    Chain c = make_chain(sm);
    uint32_t pos = 0;
    int64_t chars = 0;
    int32_t nk0 = 0;
    auto next_item = [&](uint32_t from) -> uint32_t {
      for (; from < pp.item_count; ++from) {
        const Item& it = items[pp.item_begin + from];
        if (it.nn > 0) {
          nk0 = it.k0;
          return from;
        }
      }
      return from;
    };
    uint32_t ni = next_item(0);
    if (total > 0 && !ch_start(c, sb, slen)) err = 3;
    for (int32_t k = 0; !err && k <= total; ++k) {
      while (ni < pp.item_count && nk0 == k) {
        Item& it = items[pp.item_begin + ni];
        it.pos = static_cast<int32_t>(pos);
        it.run_k0 = k;
        it.base = chars;
        ni = next_item(ni + 1);
      }
      if (k == total) break;
      if (pos + 4 > slen) { err = 1; break; }
      if (!ch_ensure(c, pos, 16)) { err = 3; break; }
      uint32_t len, hi;
      ch_read8(c, pos, &len, &hi);
      if (len > slen - pos - 4) { err = 1; break; }
      pos += 4 + len;
      chars += len;
    }
    if (total > 0 && !ch_drain(c) && !err) err = 3;
    keep_parity(sm, c);
    if (err) report(st, err == 3 ? DERR_TIMEOUT : DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 7);
    sm.ctl[5] = err;
  }
  __syncthreads();
  return sm.ctl[5] == 0;
}

// Walk of one page (block-collective).
__device__ void walk_page(const DecodeArgs& a, int p, WalkSmem& sm, bool serial_delta) {
  const int tid = threadIdx.x;
  const PlanPage pp = a.pps[p];
  const PageDev pg = a.pages[pp.page];
  const OutCol col = a.cols[pp.col];
  PageCtx pc;
  const int pgid = static_cast<int>(pp.page);
  if (!page_ctx(a, pp, &pc)) {
    if (tid == 0) report(a.st, pg.rep_len ? DERR_UNSUPPORTED : DERR_CORRUPT, pgid, WHERE_WALK_LEVELS, 10);
    return;
  }
  if (pg.pad) {  // deprecated BIT_PACKED definition levels
    if (tid == 0) report(a.st, DERR_UNSUPPORTED, pgid, WHERE_WALK_LEVELS, 11);
    return;
  }
  int32_t nonnull;
  if (pc.max_def) {
    nonnull = walk_levels(sm, pc, pp, a.items, col, a.st);
    if (nonnull < 0) return;
    if (pg.page_type == PAGE_DATA_V2 && pg.num_nulls != pc.nrows - nonnull) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_LEVELS, 12);
      return;
    }
  } else {
    nonnull = pc.nrows;  // items carry k0 = row0, nn = nrows from the planner
  }
  const uint8_t* sb = pc.body + pc.v0;
  const uint32_t slen = pc.blen - pc.v0;
  bool ok = true;
  if (pc.enc == ENC_PLAIN) {
    if (pc.ptype == T_BYTE_ARRAY) {
      ok = walk_plain_ba(sm, sb, slen, nonnull, pp, a.items, pgid, a.st,
                         pp.vtab && a.vpos ? a.vpos + (pp.vtab - 1) : nullptr);
    } else if (static_cast<uint64_t>(nonnull) * pc.width > slen) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 9);
      ok = false;
    }
  } else if (pc.enc == ENC_RLE_DICT || pc.enc == ENC_PLAIN_DICT) {
    if (pp.dict < 0) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 10);
      ok = false;
    } else if (nonnull > 0) {
      const int bw = slen >= 1 ? __ldg(sb) : 255;
      if (bw > 32) {
        if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 12);
        ok = false;
      } else {
        ok = walk_hybrid(sm, sb + 1, slen - 1, bw, nonnull, pp, a.items, pgid, a.st);
      }
    }
  } else if (pc.enc == ENC_DELTA_BP) {
    if (pc.ptype != T_INT32 && pc.ptype != T_INT64) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 13);
      ok = false;
    } else {
      const uint32_t cap = static_cast<uint32_t>(nonnull > 1 ? (nonnull - 2) / 128 + 1 : 0);
      ok = walk_delta(sm, sb, slen, pc.ptype == T_INT32 ? 32 : 64, nonnull, a.pps + p, a.dpos + pp.dtab, cap,
                      serial_delta, pgid, a.st);
    }
  } else {
    if (tid == 0) report(a.st, DERR_UNSUPPORTED, pgid, WHERE_WALK_VALUES, 14);
    ok = false;
  }
  if (tid == 0 && ok) {
    a.pps[p].values_off = static_cast<int32_t>(pc.v0);
    a.pps[p].nonnull = nonnull;
  }
  __syncthreads();
}

__device__ __forceinline__ void walk_init(WalkSmem& sm, uint32_t cap, uint32_t jw = 0) {
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    fence_mbar_init();
    sm.ctl[13] = static_cast<int32_t>(cap);
    sm.ctl[14] = sm.ctl[15] = 0;
    sm.ctl[16] = static_cast<int32_t>(jw);
  }
  __syncthreads();
}

// One thread block per page of walk list entries [wbegin, wbegin + gridDim.x).
__global__ void __launch_bounds__(WALK_THREADS, 4) k_walk(DecodeArgs a, int wbegin, uint32_t cap, uint32_t jw) {
  extern __shared__ __align__(16) uint8_t smraw[];
  WalkSmem& sm = *reinterpret_cast<WalkSmem*>(smraw);
  walk_init(sm, cap, jw);
  walk_page(a, static_cast<int>(a.walk_pps[wbegin + blockIdx.x]), sm, false);
}

// ------------------------------------------------------------------ DELTA: parallel block chain

constexpr int DREG_TAIL = 256;       // bytes staged past a region (the header of its last block)
constexpr int DREG_LEAD = 1024;      // lead-in searched before a region for a block start
constexpr int DREG_SMEM = DREG_LEAD + DELTA_REGION + DREG_TAIL + 32;
constexpr uint32_t DB_UNKNOWN = 0xffffffffu;

// Size of the full block whose header starts at smem offset o (avail bytes
// staged from there): 0 when implausible (varint too long, a width above the
// type's bits), DB_UNKNOWN when the staged bytes do not decide.
__device__ __forceinline__ uint32_t dblock_size_s(const uint8_t* sm, uint32_t o, uint32_t avail, int mbc, int vpm,
                                                  int type_bits) {
  if (mbc == 4 && avail >= 20u) {  // the common layout: the header from registers
    uint64_t z;
    uint32_t w4;
    const int vl = delta_header16<true>(sm + o, &z, &w4);
    if (!vl || (type_bits == 32 && vl > 5)) return 0;
    const uint32_t w0 = w4 & 0xffu, w1 = (w4 >> 8) & 0xffu, w2 = (w4 >> 16) & 0xffu, w3 = w4 >> 24;
    const uint32_t tb = static_cast<uint32_t>(type_bits);
    if (w0 > tb || w1 > tb || w2 > tb || w3 > tb) return 0;
    return static_cast<uint32_t>(vl + 4) + (w0 + w1 + w2 + w3) * static_cast<uint32_t>(vpm) / 8;
  }
  if (avail < 10u + static_cast<uint32_t>(mbc)) return DB_UNKNOWN;
  int vl = 0;
  for (int i = 0; i < 10; ++i)
    if (!(sm[o + i] & 0x80u)) {
      vl = i + 1;
      break;
    }
  if (!vl || (type_bits == 32 && vl > 5)) return 0;
  uint32_t bits = 0;
  for (int m = 0; m < mbc; ++m) {
    const uint32_t w = sm[o + vl + m];
    if (static_cast<int>(w) > type_bits) return 0;
    bits += w * static_cast<uint32_t>(vpm);
  }
  return static_cast<uint32_t>(vl + mbc) + bits / 8;
}

// Same from global memory (slow path).
__device__ uint32_t dblock_size_g(const uint8_t* sb, uint32_t pos, uint32_t slen, int mbc, int vpm, int type_bits) {
  if (pos >= slen) return 0;
  int vl = 0;
  for (int i = 0; i < 10 && pos + i < slen; ++i)
    if (!(__ldg(sb + pos + i) & 0x80u)) {
      vl = i + 1;
      break;
    }
  if (!vl || (type_bits == 32 && vl > 5) || pos + vl + mbc > slen) return 0;
  uint32_t bits = 0;
  for (int m = 0; m < mbc; ++m) {
    const uint32_t w = __ldg(sb + pos + vl + m);
    if (static_cast<int>(w) > type_bits) return 0;
    bits += w * static_cast<uint32_t>(vpm);
  }
  return static_cast<uint32_t>(vl + mbc) + bits / 8;
}

// One warp per region of one DELTA page.  Region i covers stream bytes
// [h + i*R, h + (i+1)*R) (h: stream header bytes).  Region 0 starts on the
// first block; region i > 0 searches its lead-in, DREG_LEAD bytes before the
// region, for the first offset where four consecutive block headers are
// plausible, and follows the chain from there.  A chain that starts on a
// look-alike usually joins the true chain within a block or two, so by the
// region's first byte it is on the true chain; k_dfix checks that and
// repairs the rare region where it is not.  Block starts inside the region
// go to the region's list; the first start at or after its end is its exit.
__global__ void __launch_bounds__(32) k_dreg(DecodeArgs a, int dbegin) {
  extern __shared__ __align__(16) uint8_t smraw[];
  __shared__ uint64_t bar;
  const int lane = threadIdx.x;
  const int p = static_cast<int>(a.delta_pps[dbegin + blockIdx.y]);
  const PlanPage pp = a.pps[p];
  if (pp.dblocks != -2 || pp.nonnull < 0 || static_cast<int>(blockIdx.x) >= pp.dreg_cap) return;
  const int i = blockIdx.x;
  const uint8_t* sb = pp.body + pp.values_off;
  const uint32_t slen = static_cast<uint32_t>(pp.body_len - pp.values_off);
  const int type_bits = a.chunks[pp.chunk].ptype == T_INT32 ? 32 : 64;
  DeltaRegion* R = a.dregs + pp.dreg + i;
  uint32_t* list = a.dreg_lists + static_cast<uint64_t>(pp.dreg + i) * DELTA_REGION_LIST;
  const uint64_t start64 = static_cast<uint64_t>(pp.dhlen) + static_cast<uint64_t>(i) * DELTA_REGION;
  if (start64 >= slen) {
    if (lane == 0) *R = DeltaRegion{-1, -1, 0, 0};
    return;
  }
  const uint32_t start = static_cast<uint32_t>(start64);
  const uint32_t end = slen - start < static_cast<uint32_t>(DELTA_REGION) ? slen : start + DELTA_REGION;
  const uint32_t sstart = i == 0 ? start : start - DREG_LEAD;  // region i > 0: start >= h + R > DREG_LEAD
  // stage [sstart, end + tail), 16-byte aligned, at most 16 bytes past the stream
  const uint8_t* g = sb + sstart;
  const uint8_t* ga = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(g) & ~uintptr_t(15));
  const uint32_t shift = static_cast<uint32_t>(g - ga);
  const uint64_t lim_end = (end + DREG_TAIL < slen ? end + DREG_TAIL : slen);
  uint32_t bytes = static_cast<uint32_t>(((sb + lim_end) - ga + 16) & ~int64_t(15));
  if (bytes > static_cast<uint32_t>(DREG_SMEM)) bytes = DREG_SMEM;
  if (lane == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar, bytes);
    bulk_g2s(smraw, ga, bytes, &bar);
  }
  __syncwarp();
  const bool ok = mbar_wait(&bar, 0);
  if (!__all_sync(0xffffffffu, ok)) {
    if (lane == 0) {
      report(a.st, DERR_TIMEOUT, static_cast<int>(pp.page), WHERE_WALK_VALUES, 30);
      mbar_wait(&bar, 0);
      *R = DeltaRegion{-1, -1, 0, 0};
    }
    return;
  }
  // stream offset s is at smem offset s - sstart + shift; staged bytes end at known_end
  const uint32_t known_end = sstart - shift + bytes > slen + 16 ? slen + 16 : sstart - shift + bytes;
  auto avail = [&](uint32_t s) -> uint32_t { return s < known_end ? known_end - s : 0u; };
  auto at = [&](uint32_t s) -> uint32_t { return s - sstart + shift; };
  uint32_t q = 0xffffffffu;
  if (i == 0) {
    q = start;
  } else {
    for (uint32_t c0 = sstart; c0 < end && q == 0xffffffffu; c0 += 32) {
      const uint32_t cand = c0 + lane;
      bool good = cand < end;
      uint32_t pos = cand;
      for (int k = 0; good && k < 4 && pos < slen; ++k) {
        const uint32_t sz = dblock_size_s(smraw, at(pos), avail(pos), pp.dmbc, pp.dvpm, type_bits);
        if (sz == 0) good = false;
        else if (sz == DB_UNKNOWN) break;
        else pos += sz;
      }
      const uint32_t m = __ballot_sync(0xffffffffu, good);
      if (m) q = c0 + __ffs(m) - 1;
    }
  }
  if (lane == 0) {
    int32_t first = -1, cnt = 0, x = -1;
    if (q != 0xffffffffu) {
      uint32_t pos = q;
      while (true) {
        if (pos >= end) {
          x = static_cast<int32_t>(pos);
          break;
        }
        if (pos >= start) {
          if (cnt == DELTA_REGION_LIST) break;  // list full: k_dfix walks the rest
          if (first < 0) first = static_cast<int32_t>(pos);
          list[cnt++] = pos;
        }
        const uint32_t sz = dblock_size_s(smraw, at(pos), avail(pos), pp.dmbc, pp.dvpm, type_bits);
        if (sz == 0 || sz == DB_UNKNOWN) break;  // the page's last block, or a false chain
        pos += sz;
      }
    }
    *R = DeltaRegion{first, first >= 0 ? x : -1, cnt, 0};
  }
}

// Serial chain of one region from its true entry `pos`: block starts go
// straight to `out` until the chain reaches `end`, `want` blocks, or one of
// the region's recorded starts (list[j..cnt), from which the list is right).
// Returns the blocks written; *pe gets the offset reached, *jm the list
// index joined (-1 if none), *bad is set when a block other than the page's
// last looks malformed.
__device__ int32_t dwalk_join(const uint8_t* sb, uint32_t slen, uint32_t pos, uint32_t end, int32_t want,
                              const uint32_t* list, int32_t cnt, bool list_exits, int mbc, int vpm,
                              int type_bits, uint32_t* out, uint32_t* pe, int32_t* jm, bool* bad) {
  int32_t j = 0;
  if (cnt > 0) {  // first recorded start >= pos
    int lo = 0, hi = cnt;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (list[mid] < pos) lo = mid + 1; else hi = mid;
    }
    j = lo;
  }
  int32_t c = 0;
  *jm = -1;
  while (pos < end && c < want) {
    while (j < cnt && list[j] < pos) ++j;
    if (j < cnt && list[j] == pos && (list_exits || cnt - j >= want - c)) {
      *jm = j;
      break;
    }
    out[c++] = pos;
    const uint32_t sz = dblock_size_g(sb, pos, slen, mbc, vpm, type_bits);
    if (sz == 0) {
      if (c < want) *bad = true;
      break;
    }
    pos += sz;
  }
  *pe = pos;
  return c;
}

// Per DELTA page: stitch the regions.  The true chain enters region i at the
// exit of region i-1; when that is the region's first recorded start the
// list is taken whole, otherwise the region is walked serially from the
// entry until it joins the list.  The lists are then copied to the page's
// block table in parallel and the last block is checked against the
// stream's end.
__global__ void __launch_bounds__(256) k_dfix(DecodeArgs a, int dbegin) {
  constexpr int MAXR = 1024;
  __shared__ int32_t s_q[MAXR], s_x[MAXR], s_c[MAXR];
  __shared__ int32_t s_skip[MAXR], s_cnt[MAXR], s_base[MAXR];
  __shared__ int32_t s_nreg, s_ok;
  const int p = static_cast<int>(a.delta_pps[dbegin + blockIdx.x]);
  const PlanPage pp = a.pps[p];
  if (pp.dblocks != -2 || pp.nonnull < 0) return;
  const uint8_t* sb = pp.body + pp.values_off;
  const uint32_t slen = static_cast<uint32_t>(pp.body_len - pp.values_off);
  const int type_bits = a.chunks[pp.chunk].ptype == T_INT32 ? 32 : 64;
  const int32_t B = (pp.nonnull - 1 + pp.dbs - 1) / pp.dbs;  // blocks of the page
  uint32_t* dpos = a.dpos + pp.dtab;
  const uint32_t h = static_cast<uint32_t>(pp.dhlen);
  const int nreg = slen > h ? static_cast<int>((slen - h + DELTA_REGION - 1) / DELTA_REGION) : 0;
  const bool regions = nreg <= pp.dreg_cap && nreg <= MAXR;
  if (regions)
    for (int i = threadIdx.x; i < nreg; i += blockDim.x) {
      const DeltaRegion r = a.dregs[pp.dreg + i];
      s_q[i] = r.q;
      s_x[i] = r.x;
      s_c[i] = r.cnt;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool bad = false;
    uint32_t e = h;
    int32_t b = 0, jm;
    if (!regions) {
      b = dwalk_join(sb, slen, e, slen, B, nullptr, 0, false, pp.dmbc, pp.dvpm, type_bits, dpos, &e, &jm, &bad);
      s_nreg = 0;
    } else {
      for (int i = 0; i < nreg; ++i) {
        const uint32_t start = h + static_cast<uint32_t>(i) * DELTA_REGION;
        const uint32_t end = slen - start < static_cast<uint32_t>(DELTA_REGION) ? slen : start + DELTA_REGION;
        s_skip[i] = -1;
        s_cnt[i] = 0;
        if (b >= B || e >= end || bad) continue;
        const int32_t cnt = s_q[i] >= 0 ? s_c[i] : 0;
        const bool exits = s_x[i] >= 0;
        int32_t j = -1;
        if (cnt > 0 && static_cast<uint32_t>(s_q[i]) == e && (exits || cnt >= B - b)) {
          j = 0;
        } else {
          const uint32_t* list = a.dreg_lists + static_cast<uint64_t>(pp.dreg + i) * DELTA_REGION_LIST;
          b += dwalk_join(sb, slen, e, end, B - b, list, cnt, exits, pp.dmbc, pp.dvpm, type_bits, dpos + b, &e,
                          &j, &bad);
        }
        if (j >= 0) {
          const int32_t c = cnt - j < B - b ? cnt - j : B - b;
          s_skip[i] = j;
          s_cnt[i] = c;
          s_base[i] = b;
          b += c;
          e = exits ? static_cast<uint32_t>(s_x[i]) : end;
        }
      }
      s_nreg = nreg;
    }
    s_ok = !bad && b == B;
  }
  __syncthreads();
  if (s_ok) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x >> 5; i < s_nreg; i += nw) {
      if (s_skip[i] < 0) continue;
      const uint32_t* list = a.dreg_lists + static_cast<uint64_t>(pp.dreg + i) * DELTA_REGION_LIST + s_skip[i];
      for (int j = lane; j < s_cnt[i]; j += 32) dpos[s_base[i] + j] = list[j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = s_ok;
    if (ok && B > 0) {
      // the last block, partial or not: its used miniblocks lie inside the stream
      const uint32_t pos = dpos[B - 1];
      const int32_t nv = pp.nonnull - 1 - (B - 1) * pp.dbs;
      const int used = (nv + pp.dvpm - 1) / pp.dvpm;
      int vl = 0;
      for (int k = 0; k < 10 && pos + k < slen; ++k)
        if (!(__ldg(sb + pos + k) & 0x80u)) {
          vl = k + 1;
          break;
        }
      uint64_t bits = 0;
      if (!vl || pos + vl + pp.dmbc > slen) ok = false;
      for (int m = 0; ok && m < used; ++m) {
        const uint32_t w = __ldg(sb + pos + vl + m);
        if (static_cast<int>(w) > type_bits) ok = false;
        bits += static_cast<uint64_t>(w) * pp.dvpm;
      }
      if (ok && pos + vl + pp.dmbc + bits / 8 > slen) ok = false;
    }
    if (!ok) {
      report(a.st, DERR_CORRUPT, static_cast<int>(pp.page), WHERE_WALK_VALUES, 31);
      a.pps[p].dblocks = -1;
    } else {
      a.pps[p].dblocks = B;
    }
  }
}

// ------------------------------------------------------------------ DELTA block bases

// Per-lane miniblock layout of the block at `pos`: width of miniblock `lane`
// and its exclusive bit offset.  Returns the header length (0: malformed).
__device__ __forceinline__ int delta_block_layout(const uint8_t* sb, uint32_t pos, const PlanPage& pp, int32_t nv,
                                                  int type_bits, int lane, int64_t* mn, uint32_t* wbyte,
                                                  uint32_t* excl, bool* bad) {
  uint64_t z = 0;
  const int vl = uleb([&](uint32_t q) { return static_cast<uint32_t>(__ldg(sb + pos + q)); }, 0, 10, &z);
  *mn = unzigzag(z);
  const uint32_t wb = lane < pp.dmbc ? __ldg(sb + pos + vl + lane) : 0u;
  const int used = (nv + pp.dvpm - 1) / pp.dvpm;
  *bad = __any_sync(0xffffffffu, lane < used && static_cast<int>(wb) > type_bits) || !vl;
  const uint32_t mbits = lane < used ? wb * static_cast<uint32_t>(pp.dvpm) : 0u;
  uint32_t incl = mbits;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  *wbyte = wb;
  *excl = incl - mbits;
  return vl;
}

// Delta sum of block b of a DELTA page (one warp): sum over its values of
// (min delta + packed delta), wrapping mod 2^64.  Returns false when the
// block is malformed.
__device__ bool delta_block_sum(const uint8_t* sb, const PlanPage& pp, const uint32_t* dpos, int type_bits, int b,
                                int lane, uint64_t* sum) {
  const uint32_t pos = dpos[b];
  const int64_t bk = 1 + static_cast<int64_t>(b) * pp.dbs;
  const int32_t nv = static_cast<int32_t>(pp.nonnull - bk < pp.dbs ? pp.nonnull - bk : pp.dbs);
  int64_t mn;
  uint32_t wb, excl;
  bool bad;
  const int vl = delta_block_layout(sb, pos, pp, nv, type_bits, lane, &mn, &wb, &excl, &bad);
  if (bad) return false;
  const uint64_t dbit = static_cast<uint64_t>(pos + vl + pp.dmbc) * 8;
  uint64_t x[4] = {0, 0, 0, 0};
#pragma unroll
  for (int u = 0; u < 4; ++u) {  // up to 128 values per block with all loads issued together
    const int v = u * 32 + lane;
    const int m = (v < nv ? v : nv - 1) / pp.dvpm;
    const int w = __shfl_sync(0xffffffffu, static_cast<int>(wb), m);
    const uint32_t off = __shfl_sync(0xffffffffu, excl, m);
    if (v < nv) x[u] = gbits64(sb, dbit + off + static_cast<uint64_t>(v - m * pp.dvpm) * w, w);
  }
  uint64_t s = 0;
  for (int v = lane; v < nv; v += 32) s += static_cast<uint64_t>(mn);
#pragma unroll
  for (int u = 0; u < 4; ++u) s += x[u];
  for (int v = 128 + lane; v < nv; v += 32) {  // blocks larger than 128 values
    const int m = v / pp.dvpm;
    const int w = __shfl_sync(__activemask(), static_cast<int>(wb), m);
    const uint32_t off = __shfl_sync(__activemask(), excl, m);
    s += gbits64(sb, dbit + off + static_cast<uint64_t>(v - m * pp.dvpm) * w, w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  *sum = s;
  return true;
}

// Block sums of every DELTA page, spread over the whole GPU: blockIdx.y is
// the page.  Blocks of the common layout (4 miniblocks) go four to a warp,
// eight lanes per block and each lane 1/8 of the values, so that the loads
// of four blocks are in flight together; other layouts take a warp per
// block.  Every block is summed as a full block: only the page's last
// block can be partial and the bases never use its sum.  The sums land in
// dbase.
__global__ void __launch_bounds__(256) k_delta_sums(DecodeArgs a, int dbegin) {
  const int lane = threadIdx.x & 31;
  const int p = static_cast<int>(a.delta_pps[dbegin + blockIdx.y]);
  const PlanPage pp = a.pps[p];
  if (pp.dblocks <= 0 || pp.nonnull < 0) return;
  const uint8_t* sb = pp.body + pp.values_off;
  const uint32_t* dpos = a.dpos + pp.dtab;
  int64_t* dsum = a.dbase + pp.dtab;
  const int type_bits = a.chunks[pp.chunk].ptype == T_INT32 ? 32 : 64;
  const int w0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  if (pp.dmbc != 4 || pp.dbs % 8) {
    for (int b = w0; b < pp.dblocks; b += nw) {
      uint64_t sum = 0;
      if (!delta_block_sum(sb, pp, dpos, type_bits, b, lane, &sum)) {
        if (lane == 0) report(a.st, DERR_CORRUPT, static_cast<int>(pp.page), WHERE_WALK_VALUES, 20);
        sum = 0;
      }
      if (lane == 0) dsum[b] = static_cast<int64_t>(sum);
    }
    return;
  }
  const int sub = lane >> 3, sl = lane & 7;
  const int nv = pp.dbs, vpm = pp.dvpm;
  for (int b0 = w0 * 4; b0 < pp.dblocks; b0 += nw * 4) {
    const int b = b0 + sub;
    const bool have = b < pp.dblocks;
    uint64_t acc = 0;
    bool bad = false;
    // the last block's sum is never used (and its unused miniblock widths may be anything)
    if (have && b + 1 < pp.dblocks) {
      const uint32_t pos = dpos[b];
      uint64_t z = 0;
      uint32_t w4 = 0;
      const int vl = delta_header16<false>(sb + pos, &z, &w4);
      const uint32_t wv[4] = {w4 & 0xffu, (w4 >> 8) & 0xffu, (w4 >> 16) & 0xffu, w4 >> 24};
      bad = !vl || static_cast<int>(wv[0]) > type_bits || static_cast<int>(wv[1]) > type_bits ||
            static_cast<int>(wv[2]) > type_bits || static_cast<int>(wv[3]) > type_bits;
      if (!bad && vpm == 32) {
        // lane sl sums values [16 sl, 16 sl + 16): half of miniblock sl / 2,
        // four values per 64-bit window when the width is at most 16 bits
        const int m = sl >> 1;
        const uint32_t w = wv[m];
        const uint32_t offm = 32u * (m == 0 ? 0u : m == 1 ? wv[0] : m == 2 ? wv[0] + wv[1] : wv[0] + wv[1] + wv[2]);
        const uint64_t b0 = static_cast<uint64_t>(pos + vl + 4) * 8 + offm + static_cast<uint64_t>(sl & 1) * 16 * w;
        if (w <= 16) {
          const uint64_t mask = (1ull << w) - 1;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t win = gwin64(sb, b0 + static_cast<uint64_t>(k) * 4 * w);
            acc += (win & mask) + ((win >> w) & mask) + ((win >> (2 * w)) & mask) + ((win >> (3 * w)) & mask);
          }
        } else {
          for (int i = 0; i < 16; ++i) acc += gbits64(sb, b0 + static_cast<uint64_t>(i) * w, static_cast<int>(w));
        }
        if (sl == 0) acc += static_cast<uint64_t>(unzigzag(z)) * static_cast<uint64_t>(nv);
      } else if (!bad) {
        const uint64_t dbit = static_cast<uint64_t>(pos + vl + 4) * 8;
        const uint32_t o1 = wv[0] * vpm, o2 = o1 + wv[1] * vpm, o3 = o2 + wv[2] * vpm;
        for (int v = sl; v < nv; v += 8) {
          const int m = v / vpm;
          const uint32_t w = m == 0 ? wv[0] : m == 1 ? wv[1] : m == 2 ? wv[2] : wv[3];
          const uint32_t off = (m == 0 ? 0u : m == 1 ? o1 : m == 2 ? o2 : o3) + static_cast<uint32_t>(v - m * vpm) * w;
          acc += gbits64(sb, dbit + off, static_cast<int>(w));
        }
        if (sl == 0) acc += static_cast<uint64_t>(unzigzag(z)) * static_cast<uint64_t>(nv);
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (have && sl == 0) {
      if (bad) report(a.st, DERR_CORRUPT, static_cast<int>(pp.page), WHERE_WALK_VALUES, 20);
      dsum[b] = static_cast<int64_t>(bad ? 0 : acc);
    }
  }
}

// In-place exclusive scan of one page's block sums, from its first value.
__device__ void delta_scan_page(const DecodeArgs& a, int p, uint64_t* tmp) {
  const PlanPage pp = a.pps[p];
  if (pp.dblocks <= 0 || pp.nonnull < 0) return;
  int64_t* d = a.dbase + pp.dtab;
  uint64_t carry = static_cast<uint64_t>(pp.dfirst);
  for (int b0 = 0; b0 < pp.dblocks; b0 += blockDim.x * 4) {
    uint64_t loc[4];
    uint64_t mine = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = b0 + threadIdx.x * 4 + q;
      loc[q] = j < pp.dblocks ? static_cast<uint64_t>(d[j]) : 0;
      mine += loc[q];
    }
    uint64_t tot;
    uint64_t run = carry + block_exclusive_sum(mine, tmp, &tot);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = b0 + threadIdx.x * 4 + q;
      if (j < pp.dblocks) d[j] = static_cast<int64_t>(run);
      run += loc[q];
    }
    carry += tot;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) k_delta_scan(DecodeArgs a, int dbegin) {
  __shared__ uint64_t tmp[32];
  delta_scan_page(a, static_cast<int>(a.delta_pps[dbegin + blockIdx.x]), tmp);
}

// One DELTA page inside one thread block (plain baseline).
__device__ void delta_bases_page(const DecodeArgs& a, int p, uint64_t* tmp) {
  const PlanPage pp = a.pps[p];
  if (pp.dblocks <= 0 || pp.nonnull < 0) return;
  const int lane = threadIdx.x & 31;
  const uint8_t* sb = pp.body + pp.values_off;
  const int type_bits = a.chunks[pp.chunk].ptype == T_INT32 ? 32 : 64;
  for (int b = threadIdx.x >> 5; b < pp.dblocks; b += blockDim.x >> 5) {
    uint64_t sum = 0;
    if (!delta_block_sum(sb, pp, a.dpos + pp.dtab, type_bits, b, lane, &sum)) {
      if (lane == 0) report(a.st, DERR_CORRUPT, static_cast<int>(pp.page), WHERE_WALK_VALUES, 20);
      sum = 0;
    }
    if (lane == 0) a.dbase[pp.dtab + b] = static_cast<int64_t>(sum);
  }
  __syncthreads();
  delta_scan_page(a, p, tmp);
}

// ------------------------------------------------------------------ expand (one warp per item)

struct WarpSmem {
  uint64_t vbuf[ITEM_ROWS_OPT];  // dense values of an OPTIONAL item (non-PLAIN)
};

__device__ __forceinline__ void store_val(uint8_t* base, int64_t row, int width, uint64_t v) {
  if (width == 4)
    reinterpret_cast<uint32_t*>(base)[row] = static_cast<uint32_t>(v);
  else
    reinterpret_cast<uint64_t*>(base)[row] = v;
}

// Where dense values go: straight to the output rows (REQUIRED), to the
// string scratch (REQUIRED BYTE_ARRAY), or to the warp's staging buffer
// (OPTIONAL, scattered to rows afterwards).
struct Sink {
  uint8_t* out;
  uint64_t* sidx;
  uint64_t* vbuf;
  int64_t orow0;
  int width;
  __device__ __forceinline__ void put(int32_t j, uint64_t v) const {
    if (vbuf)
      vbuf[j] = v;
    else if (sidx)
      sidx[orow0 + j] = v;
    else
      store_val(out, orow0 + j, width, v);
  }
};

// Dictionary indices of dense values [k0, k1), from the checkpoint run;
// up to 4 gathers per lane are issued before any result is used.
__device__ bool warp_hybrid(const uint8_t* sb, uint32_t slen, int bw, int32_t total, uint32_t pos, int32_t rk,
                            int32_t k0, int32_t k1, const DictDev& dd, bool idx_only, const Sink& sink,
                            uint64_t* chars, int lane) {
  const uint32_t vbytes = (bw + 7) / 8;
  {
    // the runs of [rk, k1) as if all were bit-packed: an upper bound of the
    // item's bytes unless headers are long; lines fetched into L2 up front
    const uint64_t span = 16 + (static_cast<uint64_t>(k1 - rk) * bw + 7) / 8;
    const uint64_t end = pos + span < slen ? pos + span : slen;
    if (pos < end) prefetch_l2(sb + pos, sb + end, lane);
  }
  // lane 0 keeps the next run's first 8 bytes in flight: one-byte headers
  // (and their repeated value) are decoded from them without a new load
  uint64_t win = 0;
  if (lane == 0 && pos < slen) win = ld_unaligned_g(sb + pos, 8);
  for (uint32_t guard = 0; rk < k1 && guard <= slen; ++guard) {
    uint64_t h = 0;
    int hl = 0;
    uint32_t rle = 0;
    if (lane == 0 && pos < slen) {
      const uint32_t b0 = static_cast<uint32_t>(win & 0xffu);
      if (!(b0 & 0x80u) && (b0 & 1u || 1 + vbytes <= 8)) {
        h = b0;
        hl = 1;
        if (!(h & 1)) {
          if (pos + 1 + vbytes > slen)
            hl = 0;
          else
            rle = vbytes ? static_cast<uint32_t>((win >> 8) & (vbytes >= 4 ? 0xffffffffull : ((1ull << (8 * vbytes)) - 1)))
                         : 0u;
        }
      } else {
        hl = uleb([&](uint32_t q) { return static_cast<uint32_t>(__ldg(sb + q)); }, pos, slen, &h);
        if (hl && !(h & 1)) {
          if (pos + hl + vbytes > slen)
            hl = 0;
          else
            for (uint32_t q = 0; q < vbytes; ++q) rle |= static_cast<uint32_t>(__ldg(sb + pos + hl + q)) << (8 * q);
        }
      }
      if (hl) {
        const uint64_t adv = hl + ((h & 1) ? (h >> 1) * static_cast<uint64_t>(bw) : vbytes);
        if (pos + adv < slen) win = ld_unaligned_g(sb + pos + adv, 8);  // next run, loaded ahead
      }
    }
    hl = __shfl_sync(0xffffffffu, hl, 0);
    if (!hl) return false;
    h = __shfl_sync(0xffffffffu, h, 0);
    rle = __shfl_sync(0xffffffffu, rle, 0);
    const bool packed = h & 1;
    const uint64_t cnt = packed ? (h >> 1) << 3 : h >> 1;
    const uint64_t adv = hl + (packed ? (h >> 1) * static_cast<uint64_t>(bw) : vbytes);
    if (pos + adv > slen) return false;
    const int64_t rend64 = static_cast<int64_t>(rk) + static_cast<int64_t>(cnt);
    const int32_t s = rk > k0 ? rk : k0;
    int64_t e64 = rend64 < k1 ? rend64 : k1;
    if (e64 > total) e64 = total;
    const int32_t e = static_cast<int32_t>(e64);
    const uint64_t dbit = static_cast<uint64_t>(pos + hl) * 8;
    bool bad = false;
    if (dd.n == 0 && s < e) return false;
    constexpr int U = 8;  // values per lane in flight
    if (!idx_only && sink.out && !sink.vbuf && !sink.sidx && packed) {
      // REQUIRED fixed-width output from a bit-packed run: word-aligned
      // loads, a funnel shift, a gather, a store per value
      const uintptr_t ab = reinterpret_cast<uintptr_t>(sb);
      const uint32_t* wq = reinterpret_cast<const uint32_t*>(ab & ~uintptr_t(3));
      const uint64_t b0 = (ab & 3) * 8 + dbit + static_cast<uint64_t>(s - rk) * bw;
      const uint32_t mask = bw >= 32 ? 0xffffffffu : ((1u << bw) - 1u);
      const uint32_t n = static_cast<uint32_t>(dd.n);
      uint8_t* out = sink.out;
      const int64_t orow = sink.orow0 + (s - k0);
      for (int32_t j0 = 0; j0 < e - s; j0 += 32 * U) {
        uint32_t x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t j = j0 + u * 32 + lane;
          const uint64_t b = b0 + static_cast<uint64_t>(j) * bw;
          const uint32_t* q = wq + (b >> 5);
          x[u] = j < e - s ? __funnelshift_r(__ldg(q), __ldg(q + 1), static_cast<uint32_t>(b & 31)) & mask : 0u;
          bad |= x[u] >= n;
          x[u] = x[u] < n ? x[u] : 0u;
        }
        if (dd.width == 4) {
          const uint32_t* dv = reinterpret_cast<const uint32_t*>(dd.values);
          uint32_t v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) v[u] = __ldg(dv + x[u]);
          uint32_t* o32 = reinterpret_cast<uint32_t*>(out) + orow;
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (j0 + u * 32 + lane < e - s) o32[j0 + u * 32 + lane] = v[u];
        } else {
          const uint64_t* dv = reinterpret_cast<const uint64_t*>(dd.values);
          uint64_t v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) v[u] = __ldg(dv + x[u]);
          uint64_t* o64 = reinterpret_cast<uint64_t*>(out) + orow;
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (j0 + u * 32 + lane < e - s) o64[j0 + u * 32 + lane] = v[u];
        }
      }
    } else if (!idx_only && sink.out && !sink.vbuf && !sink.sidx && s < e) {
      // REQUIRED fixed-width output from a repeated run: one gather, a fill
      if (rle >= static_cast<uint32_t>(dd.n)) return false;
      const int64_t orow = sink.orow0 + (s - k0);
      const int32_t m = e - s;
      if (dd.width == 4) {
        const uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(dd.values) + rle);
        uint32_t* o32 = reinterpret_cast<uint32_t*>(sink.out) + orow;
        for (int32_t j = lane; j < m; j += 32) o32[j] = v;
      } else {
        const uint64_t v = __ldg(reinterpret_cast<const uint64_t*>(dd.values) + rle);
        uint64_t* o64 = reinterpret_cast<uint64_t*>(sink.out) + orow;
        for (int32_t j = lane; j < m; j += 32) o64[j] = v;
      }
    } else
    for (int32_t j0 = s; j0 < e; j0 += 32 * U) {
      uint32_t idx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t j = j0 + u * 32 + lane;
        uint32_t x = 0;
        if (j < e) {
          x = packed ? gbits32(sb, dbit + static_cast<uint64_t>(j - rk) * bw, bw) : rle;
          if (x >= static_cast<uint32_t>(dd.n)) {
            bad = true;
            x = 0;
          }
        }
        idx[u] = x;
      }
      if (idx_only) {
        uint64_t ent[U];
#pragma unroll
        for (int u = 0; u < U; ++u) ent[u] = j0 + u * 32 + lane < e ? __ldg(dd.str_ent + idx[u]) : 0ull;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t j = j0 + u * 32 + lane;
          if (j < e) {
            sink.put(j - k0, ent[u]);
            *chars += static_cast<uint32_t>(ent[u]);
          }
        }
      } else if (dd.width == 4) {
        uint32_t v[U];
        const uint32_t* dv = reinterpret_cast<const uint32_t*>(dd.values);
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(dv + idx[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t j = j0 + u * 32 + lane;
          if (j < e) sink.put(j - k0, v[u]);
        }
      } else {
        uint64_t v[U];
        const uint64_t* dv = reinterpret_cast<const uint64_t*>(dd.values);
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(dv + idx[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t j = j0 + u * 32 + lane;
          if (j < e) sink.put(j - k0, v[u]);
        }
      }
    }
    if (__any_sync(0xffffffffu, bad)) return false;
    pos += static_cast<uint32_t>(adv);
    rk = rend64 > total ? total : static_cast<int32_t>(rend64);
  }
  return rk >= k1;
}

// DELTA values [k0, k1) from the block tables.
__device__ bool warp_delta(const uint8_t* sb, const PlanPage& pp, const uint32_t* dpos, const int64_t* dbase,
                           int type_bits, int32_t k0, int32_t k1, const Sink& sink, int lane) {
  const int32_t total = pp.nonnull;
  if (k0 == 0 && k1 > 0 && lane == 0) sink.put(0, static_cast<uint64_t>(pp.dfirst));
  const int32_t ka = k0 > 1 ? k0 : 1;
  if (ka >= k1) return true;
  const int bfirst = (ka - 1) / pp.dbs, blast = (k1 - 2) / pp.dbs;
  if (blast >= pp.dblocks) return false;
  {
    const uint32_t slen = static_cast<uint32_t>(pp.body_len - pp.values_off);
    const uint32_t p0 = dpos[bfirst];
    const uint32_t p1 = blast + 1 < pp.dblocks ? dpos[blast + 1] : slen;
    if (p0 < p1 && p1 <= slen) prefetch_l2(sb + p0, sb + p1, lane);
  }
  if (pp.dbs == 128 && pp.dmbc == 4 && pp.dvpm == 32) {
    // the common layout: lane j parses the header of block jb + j, then the
    // blocks are decoded two at a time from the parsed headers (each block
    // starts from its base, so blocks do not wait on one another)
    for (int jb = bfirst; jb <= blast; jb += 32) {
      const int b = jb + lane;
      const bool have = b <= blast;
      uint32_t hpos = 0, hw = 0;
      int hvl = 0;
      int64_t hmn = 0, hbase = 0;
      bool badl = false;
      if (have) {
        hpos = dpos[b];
        hbase = dbase[b];
        uint64_t z = 0;
        hvl = delta_header16<false>(sb + hpos, &z, &hw);
        hmn = unzigzag(z);
        const int64_t bk = 1 + static_cast<int64_t>(b) * 128;
        const int nvb = static_cast<int>(total - bk < 128 ? total - bk : 128);
        const int used = (nvb + 31) >> 5;
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (m < used && static_cast<int>((hw >> (8 * m)) & 0xffu) > type_bits) badl = true;
        badl |= !hvl;
      }
      if (__any_sync(0xffffffffu, badl)) return false;
      const int nb = blast - jb + 1 < 32 ? blast - jb + 1 : 32;
      for (int t = 0; t < nb; ++t) {
        // lane l takes values [4l, 4l + 4) of the block (miniblock l / 8):
        // one 64-bit window when the width is at most 16 bits, a local
        // prefix, then one warp scan of the lane totals
        const uint32_t pos = __shfl_sync(0xffffffffu, hpos, t);
        const int vl = __shfl_sync(0xffffffffu, hvl, t);
        const uint32_t w4 = __shfl_sync(0xffffffffu, hw, t);
        const uint64_t mn = static_cast<uint64_t>(__shfl_sync(0xffffffffu, hmn, t));
        const uint64_t base = static_cast<uint64_t>(__shfl_sync(0xffffffffu, hbase, t));
        const int64_t bk = 1 + static_cast<int64_t>(jb + t) * 128;
        const int32_t nv = static_cast<int32_t>(total - bk < 128 ? total - bk : 128);
        const int m = lane >> 3;
        const uint32_t w0 = w4 & 0xffu, w1 = (w4 >> 8) & 0xffu, w2 = (w4 >> 16) & 0xffu;
        const uint32_t w = (w4 >> (8 * m)) & 0xffu;
        const uint32_t offm = 32u * (m == 0 ? 0u : m == 1 ? w0 : m == 2 ? w0 + w1 : w0 + w1 + w2);
        const uint64_t b0 = static_cast<uint64_t>(pos + vl + 4) * 8 + offm + static_cast<uint64_t>(lane & 7) * 4 * w;
        const int v0 = 4 * lane;
        uint64_t x[4];
        if (v0 < nv) {
          if (w <= 16) {
            const uint64_t win = gwin64(sb, b0);
            const uint64_t mask = (1ull << w) - 1;
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = (win >> (i * w)) & mask;
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = v0 + i < nv ? gbits64(sb, b0 + static_cast<uint64_t>(i) * w, w) : 0;
          }
        } else {
          x[0] = x[1] = x[2] = x[3] = 0;
        }
        uint64_t loc[4];
        uint64_t run = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          run += v0 + i < nv ? mn + x[i] : 0;
          loc[i] = run;
        }
        uint64_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const uint64_t before = base + (incl - run);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t dense = bk + v0 + i;
          if (v0 + i < nv && dense >= k0 && dense < k1) sink.put(static_cast<int32_t>(dense - k0), before + loc[i]);
        }
      }
    }
    return true;
  }
  for (int b = bfirst; b <= blast; ++b) {
    const uint32_t pos = dpos[b];
    const int64_t bk = 1 + static_cast<int64_t>(b) * pp.dbs;
    const int32_t nv = static_cast<int32_t>(total - bk < pp.dbs ? total - bk : pp.dbs);
    int64_t mn;
    uint32_t wb, excl;
    bool bad;
    const int vl = delta_block_layout(sb, pos, pp, nv, type_bits, lane, &mn, &wb, &excl, &bad);
    if (bad) return false;
    const uint64_t dbit = static_cast<uint64_t>(pos + vl + pp.dmbc) * 8;
    uint64_t carry = static_cast<uint64_t>(dbase[b]);
    for (int r0 = 0; r0 < nv; r0 += 128) {
      // 4 rounds of 32 values: all packed deltas loaded before the scans
      uint64_t x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int v = r0 + u * 32 + lane;
        const int m = (v < nv ? v : nv - 1) / pp.dvpm;
        const int w = __shfl_sync(0xffffffffu, static_cast<int>(wb), m);
        const uint32_t off = __shfl_sync(0xffffffffu, excl, m);
        x[u] = v < nv ? static_cast<uint64_t>(mn) +
                            gbits64(sb, dbit + off + static_cast<uint64_t>(v - m * pp.dvpm) * w, w)
                      : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        uint64_t y = x[u];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint64_t t = __shfl_up_sync(0xffffffffu, y, o);
          if (lane >= o) y += t;
        }
        const int v = r0 + u * 32 + lane;
        const int64_t dense = bk + v;
        if (v < nv && dense >= k0 && dense < k1) sink.put(static_cast<int32_t>(dense - k0), carry + y);
        carry += __shfl_sync(0xffffffffu, y, 31);
      }
    }
  }
  return true;
}

// PLAIN BYTE_ARRAY: lane 0 follows the values from the checkpoint.
__device__ bool warp_plain_ba(const uint8_t* sb, uint32_t slen, uint32_t pos, int32_t k0, int32_t k1,
                              const Sink& sink, uint64_t* chars, int lane) {
  int ok = 1;
  if (lane == 0) {
    for (int32_t k = k0; k < k1; ++k) {
      if (pos + 4 > slen) { ok = 0; break; }
      const uint32_t len = ld_le32_g(sb + pos);
      if (len > slen - pos - 4) { ok = 0; break; }
      sink.put(k - k0, (static_cast<uint64_t>(pos + 4) << 32) | len);
      *chars += len;
      pos += 4 + len;
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Bits of the validity bitmap for output rows [r, r + n), n <= 32.
__device__ __forceinline__ uint32_t bitmap_bits(const uint32_t* v, int64_t r, int n) {
  const int64_t wi = r >> 5;
  const uint32_t sh = static_cast<uint32_t>(r & 31);
  const uint32_t lo = v[wi];
  const uint32_t hi = (sh && sh + n > 32) ? v[wi + 1] : 0u;
  const uint32_t b = sh ? __funnelshift_r(lo, hi, sh) : lo;
  return n < 32 ? b & ((1u << n) - 1u) : b;
}

// Columns whose pages are all REQUIRED PLAIN fixed-width: every item is a
// straight copy of nrows * width bytes, handed out through the column's
// counter.
__global__ void __launch_bounds__(256) k_copy_items(DecodeArgs a, int ibegin, int icount, int cidx) {
  const int lane = threadIdx.x & 31;
  uint32_t* ctr = a.item_counter + 4 + cidx;
  for (;;) {
    int u = 0;
    if (lane == 0) u = static_cast<int>(atomicAdd(ctr, 1u));
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= icount) break;
    const Item it = a.items[ibegin + u];
    if (it.nrows <= 0) continue;
    const PlanPage pp = a.pps[it.pp];
    const OutCol col = a.cols[pp.col];
    const int width = col.width;
    if (static_cast<uint64_t>(it.k0 + it.nrows) * width > static_cast<uint64_t>(pp.body_len - pp.values_off)) {
      if (lane == 0) report(a.st, DERR_CORRUPT, static_cast<int>(pp.page), WHERE_EXPAND, 10);
      continue;
    }
    warp_copy(col.values + (pp.out_row + it.row0) * width, pp.body + pp.values_off + static_cast<int64_t>(it.k0) * width,
              static_cast<uint64_t>(it.nrows) * width, lane);
  }
}

__device__ void expand_item(const DecodeArgs& a, int it_id, WarpSmem& ws, int lane) {
  const Item it = a.items[it_id];
  if (it.nrows <= 0) return;
  const PlanPage pp = a.pps[it.pp];
  if (pp.nonnull < 0) return;  // the walk of this page failed (error recorded)
  const OutCol col = a.cols[pp.col];
  const int pgid = static_cast<int>(pp.page);
  const uint8_t* sb = pp.body + pp.values_off;
  const uint32_t slen = static_cast<uint32_t>(pp.body_len - pp.values_off);
  const int enc = pp.enc;
  const bool isdict = enc == ENC_RLE_DICT || enc == ENC_PLAIN_DICT;
  const bool isdelta = enc == ENC_DELTA_BP;
  const bool isba = col.ptype == T_BYTE_ARRAY;
  const int width = col.width;
  const int64_t orow0 = pp.out_row + it.row0;
  const int32_t k0 = it.k0, nn = it.nn;
  // an item that fails leaves empty string entries behind (the string copy
  // then reads nothing for its rows; the error is recorded)
  auto clear_strings = [&]() {
    if (isba)
      for (int32_t r = lane; r < it.nrows; r += 32) col.str_scratch[orow0 + r] = 0ull;
  };
  if (k0 < 0 || nn < 0 || static_cast<int64_t>(k0) + nn > pp.nonnull ||
      (col.optional && !isba && enc != ENC_PLAIN && nn > ITEM_ROWS_OPT) ||
      (col.optional && isba && nn > ITEM_ROWS_OPT)) {
    if (lane == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_EXPAND, 9);
    clear_strings();
    return;
  }
  uint64_t chars = 0;
  bool ok = true;
  if (enc == ENC_PLAIN && !isba) {
    if (static_cast<uint64_t>(k0 + nn) * width > slen) {
      if (lane == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_EXPAND, 10);
      return;
    }
    const uint8_t* src = sb + static_cast<int64_t>(k0) * width;
    if (!col.optional) {
      for (int32_t r0 = 0; r0 < it.nrows; r0 += 256) {
        uint64_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int32_t r = r0 + u * 32 + lane;
          v[u] = r < it.nrows ? ld_unaligned_g(src + static_cast<int64_t>(r) * width, width) : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int32_t r = r0 + u * 32 + lane;
          if (r < it.nrows) store_val(col.values, orow0 + r, width, v[u]);
        }
      }
    } else {
      if (nn > 0) prefetch_l2(src, src + static_cast<int64_t>(nn) * width, lane);
      int32_t rank = 0;
      const uint32_t sh = static_cast<uint32_t>(orow0 & 31);
      for (int32_t r0 = 0; r0 < it.nrows; r0 += 256) {
        // the bitmap words of these 256 rows (9 at most), one per lane,
        // loaded together; each 32-row group's bits by two shuffles
        const int64_t wbase = (orow0 + r0) >> 5;
        const int64_t wend = (orow0 + it.nrows - 1) >> 5;
        const uint32_t myw = lane < 9 && wbase + lane <= wend ? col.validity[wbase + lane] : 0u;
        uint32_t bits[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int32_t c0 = r0 + u * 32;
          const int n = it.nrows - c0 < 32 ? it.nrows - c0 : 32;
          const uint32_t lo = __shfl_sync(0xffffffffu, myw, u);
          const uint32_t hi = __shfl_sync(0xffffffffu, myw, u + 1);
          const uint32_t b = sh ? __funnelshift_r(lo, hi, sh) : lo;
          bits[u] = n <= 0 ? 0u : (n < 32 ? b & ((1u << n) - 1u) : b);
        }
        uint64_t v[8];
        int32_t rr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          rr[u] = rank + __popc(bits[u] & ((1u << lane) - 1u));
          rank += __popc(bits[u]);
          v[u] = (bits[u] >> lane) & 1u ? ld_unaligned_g(src + static_cast<int64_t>(rr[u]) * width, width) : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int32_t r = r0 + u * 32 + lane;
          if (r < it.nrows) store_val(col.values, orow0 + r, width, v[u]);
        }
      }
    }
    return;
  }
  const int type_bits = col.ptype == T_INT32 ? 32 : 64;
  Sink sink{nullptr, nullptr, nullptr, orow0, width};
  if (col.optional)
    sink.vbuf = ws.vbuf;
  else if (isba)
    sink.sidx = col.str_scratch;
  else
    sink.out = col.values;
  if (nn > 0) {
    if (isdict) {
      const DictDev dd = a.dicts[pp.dict];
      const int bw = __ldg(sb);
      ok = bw <= 32 && warp_hybrid(sb + 1, slen - 1, bw, pp.nonnull, static_cast<uint32_t>(it.pos), it.run_k0, k0,
                                   k0 + nn, dd, isba, sink, &chars, lane);
    } else if (isdelta) {
      ok = warp_delta(sb, pp, a.dpos + pp.dtab, a.dbase + pp.dtab, type_bits, k0, k0 + nn, sink, lane);
    } else if (isba) {
      ok = warp_plain_ba(sb, slen, static_cast<uint32_t>(it.pos), k0, k0 + nn, sink, &chars, lane);
    } else {
      ok = false;
    }
  }
  if (!ok) {
    if (lane == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_EXPAND, 1);
    __syncwarp();
    clear_strings();
    return;
  }
  __syncwarp();
  if (col.optional) {
    // scatter the staged dense values to rows, nulls as zero
    int32_t rank = 0;
    for (int32_t r0 = 0; r0 < it.nrows; r0 += 32) {
      const int n = it.nrows - r0 < 32 ? it.nrows - r0 : 32;
      const uint32_t bits = bitmap_bits(col.validity, orow0 + r0, n);
      const bool valid = (bits >> lane) & 1u;
      const int32_t rr = rank + __popc(bits & ((1u << lane) - 1u));
      if (lane < n) {
        if (isba)
          col.str_scratch[orow0 + r0 + lane] = valid ? ws.vbuf[rr] : 0ull;
        else
          store_val(col.values, orow0 + r0 + lane, width, valid ? ws.vbuf[rr] : 0);
      }
      rank += __popc(bits);
    }
    __syncwarp();
  }
  if (isba) {
    uint64_t t = chars;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) col.str_item_bytes[it_id] = t;
  }
}

// Items [ibegin, ibegin + icount), handed out one at a time to warps through
// the column's counter (items differ in cost), over a grid sized to the
// resident capacity.
__global__ void __launch_bounds__(EXP_THREADS, 4) k_expand(DecodeArgs a, int ibegin, int icount, int cidx) {
  __shared__ WarpSmem ws[EXP_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* ctr = a.item_counter + EXP_COUNTER0 + cidx;
  // each warp holds one claimed item in reserve: the next claim is issued
  // before the current item is decoded, so its latency is hidden
  int u = 0;
  if (lane == 0) u = static_cast<int>(atomicAdd(ctr, 1u));
  u = __shfl_sync(0xffffffffu, u, 0);
  while (u < icount) {
    int un = 0;
    if (lane == 0) un = static_cast<int>(atomicAdd(ctr, 1u));
    expand_item(a, ibegin + u, ws[warp], lane);
    u = __shfl_sync(0xffffffffu, un, 0);
  }
}

// ------------------------------------------------------------------ staged dictionary expand

// REQUIRED fixed-width columns with dictionary pages.  A thread block claims
// spans of SX_SPAN consecutive work items; its SX_WARPS warps take every
// SX_WARPS-th item of the span.  Each warp stages an item's index bytes
// (from the checkpoint run header on) into shared memory with one bulk copy,
// issued one item ahead into the warp's other buffer, so that the next
// item's bytes stream in while the current one is decoded; the item and
// page fields it needs are loaded two items ahead.  Lane 0 lists the item's
// runs from the staged bytes; every lane then decodes 16 output bytes (4
// INT32 / 2 INT64 values) per step from one 64-bit window of the staged bits
// and writes them with one 16-byte store.  Dictionaries of at most
// SX_DICT_MAX bytes are gathered from a copy in shared memory, loaded once per
// span when the span's chunk changes; larger ones from global memory (L2).
// Items whose runs do not fit the staged bytes or the run table, and items
// of pages that are not dictionary encoded, take the general warp decode.
constexpr int SX_WARPS = 8;
constexpr int SX_THREADS = 32 * SX_WARPS;
constexpr int SX_SPAN = 32;
constexpr int SX_MAXRUNS = 96;
constexpr uint32_t SX_DICT_MAX = 48 * 1024;

struct SxWarp {
  uint64_t full[2];
  int32_t rk[SX_MAXRUNS + 1];  // dense index (page) at each run start; rk[nr] = end
  int32_t rb[SX_MAXRUNS];      // bit-packed: bit offset of the run's data in the buffer; -1: repeated
  uint32_t rv[SX_MAXRUNS];     // repeated: the value
};
struct SxBlock {
  uint64_t dbar;
  int32_t span;    // the span claimed for the next round
  int32_t dchunk;  // chunk whose dictionary is in shared memory (-1 none)
  SxWarp w[SX_WARPS];
};
__host__ __device__ constexpr uint32_t sx_smem_bytes(uint32_t stage, uint32_t dict_cap) {
  return ((static_cast<uint32_t>(sizeof(SxBlock)) + 15u) & ~15u) + SX_WARPS * 2u * (stage + 16u) + dict_cap;
}

// What a warp knows about one of its items (lane-uniform).
struct SxItem {
  int32_t item;     // absolute id, -1 none
  int32_t nrows, nn, k0, pos, run_k0, row0, pp;
};
struct SxPage {
  int32_t pp;       // plan page these fields belong to (-1 none)
  const uint8_t* sb;  // value stream (bit-width byte first)
  uint32_t slen;
  int32_t staged;   // dictionary indices the staged decode can take
  int32_t dict, nonnull, page, bw, dn;
  int64_t out_row;
  const uint8_t* dvals;
};

__device__ __forceinline__ SxItem sx_item(const DecodeArgs& a, int item, int iend) {
  SxItem r{-1, 0, 0, 0, 0, 0, 0, 0};
  if (item >= 0 && item < iend) {
    const Item& it = a.items[item];
    r = SxItem{item, it.nrows, it.nn, it.k0, it.pos, it.run_k0, it.row0, static_cast<int32_t>(it.pp)};
  }
  return r;
}

__device__ __forceinline__ void sx_page(const DecodeArgs& a, int32_t ppi, SxPage* g) {
  if (ppi == g->pp) return;
  const PlanPage& pp = a.pps[ppi];
  g->pp = ppi;
  g->sb = pp.body + pp.values_off;
  g->slen = static_cast<uint32_t>(pp.body_len - pp.values_off);
  g->dict = pp.dict;
  g->nonnull = pp.nonnull;
  g->page = static_cast<int32_t>(pp.page);
  g->out_row = pp.out_row;
  g->staged = (pp.enc == ENC_RLE_DICT || pp.enc == ENC_PLAIN_DICT) && pp.dict >= 0 && g->slen >= 1 &&
              pp.nonnull >= 0;
  g->dvals = nullptr;
  g->dn = 0;
  g->bw = 0;
  if (g->staged) {
    const DictDev& dd = a.dicts[pp.dict];
    g->dvals = dd.values;
    g->dn = dd.n;
    g->bw = __ldg(g->sb);
  }
}

// Lane 0 issues the bulk copy of an item's index bytes; returns (in every
// lane) the staged bytes, 0 when the item does not take the staged decode.
__device__ __forceinline__ uint32_t sx_issue(const SxItem& t, const SxPage& g, uint8_t* buf, uint32_t stage,
                                             uint64_t* bar, int32_t* s0, int lane) {
  if (t.item < 0 || !g.staged || t.nrows <= 0 || t.nn <= 0 || static_cast<uint32_t>(t.pos) >= g.slen - 1) return 0;
  const uint8_t* from = g.sb + 1 + t.pos;
  const uint8_t* al = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(from) & ~uintptr_t(15));
  // readable: the stream and the 16 bytes after it (chunk slack / scratch padding)
  const uint64_t lim = static_cast<uint64_t>((g.sb + g.slen + 16) - al) & ~uint64_t(15);
  const uint32_t tx = static_cast<uint32_t>(lim < stage ? lim : stage);
  *s0 = static_cast<int32_t>(al - (g.sb + 1));
  if (lane == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, tx);
    bulk_g2s(buf, al, tx, bar);
  }
  return tx;
}

// Decodes a staged item; false: the general decode must take it (runs past
// the staged bytes or the run table) -- nothing has been written then.
template <int kWidth>
__device__ bool sx_decode(const DecodeArgs& a, const SxItem& t, const SxPage& g, int32_t s0, uint32_t bytes,
                          const uint8_t* buf, SxWarp& w, const uint8_t* sdict, int32_t sdict_chunk,
                          uint8_t* col_values, int lane) {
  const int bw = g.bw;
  const int32_t k0 = t.k0, nn = t.nn, k1 = t.k0 + t.nn;
  int nr = 0, status = 0;  // 0 ok, 1 fall back, 2 corrupt
  if (lane == 0) {
    if (bw > 32 || g.dn <= 0 || t.run_k0 > k0) {
      status = 2;
    } else {
      const uint32_t vbytes = (static_cast<uint32_t>(bw) + 7) / 8;
      int64_t o = static_cast<int64_t>(t.pos) - s0;  // buffer offset of the run header
      int32_t rk = t.run_k0;
      while (rk < k1) {
        // (the buffer holds 16 bytes past `bytes`: a header read may look there)
        if (nr == SX_MAXRUNS || o < 0 || o >= bytes) { status = 1; break; }
        uint64_t h = 0;
        const int hl = uleb_p(buf + o, &h);
        if (!hl) { status = 2; break; }
        if (o + hl + ((h & 1) ? 0u : vbytes) > bytes) { status = 1; break; }
        const uint64_t cnt = (h & 1) ? (h >> 1) << 3 : h >> 1;
        if (cnt == 0) { status = 2; break; }
        w.rk[nr] = rk;
        if (h & 1) {
          const int64_t data = o + hl;
          // bits of the values this item needs, plus 16 bytes of read-ahead
          const int64_t upto = (rk + static_cast<int64_t>(cnt) < k1 ? static_cast<int64_t>(cnt) : k1 - rk);
          if (data + (upto * bw + 7) / 8 + 16 > bytes) { status = 1; break; }
          w.rb[nr] = static_cast<int32_t>(data * 8);
          o = data + static_cast<int64_t>(h >> 1) * bw;
        } else {
          uint32_t v = 0;
          for (uint32_t b = 0; b < vbytes; ++b) v |= static_cast<uint32_t>(buf[o + hl + b]) << (8 * b);
          w.rb[nr] = -1;
          w.rv[nr] = v;
          o += hl + vbytes;
        }
        ++nr;
        const int64_t re = static_cast<int64_t>(rk) + static_cast<int64_t>(cnt);
        rk = re > g.nonnull ? g.nonnull : static_cast<int32_t>(re);
      }
      if (status == 0 && nr == 0) status = 2;
      w.rk[nr] = k1 > rk ? k1 : rk;
    }
  }
  status = __shfl_sync(0xffffffffu, status, 0);
  if (status == 2) {
    if (lane == 0) report(a.st, DERR_CORRUPT, g.page, WHERE_EXPAND, 40);
    return true;
  }
  if (status == 1) return false;
  nr = __shfl_sync(0xffffffffu, nr, 0);
  __syncwarp();
  using T = typename std::conditional<kWidth == 4, uint32_t, unsigned long long>::type;
  constexpr int VPL = 16 / kWidth;  // values per lane per 16-byte store
  const uint32_t* bw32 = reinterpret_cast<const uint32_t*>(buf);
  const uint32_t nmax = static_cast<uint32_t>(g.dn) - 1u;
  const uint32_t mask = bw >= 32 ? 0xffffffffu : ((1u << bw) - 1u);
  const T* dsrc = reinterpret_cast<const T*>(sdict != nullptr && sdict_chunk == g.dict ? sdict : g.dvals);
  const bool use_s = sdict != nullptr && sdict_chunk == g.dict;
  uint8_t* out = col_values + (g.out_row + t.row0) * kWidth;
  const int32_t head = static_cast<int32_t>((reinterpret_cast<uintptr_t>(out) & 15) / kWidth);
  T* outa = reinterpret_cast<T*>(out) - head;  // 16-byte aligned
  const int32_t npos = head + nn;
  // the lane's current run (positions only grow)
  int r = 0;
  int32_t rend = w.rk[1], bbase = 0;  // bbase: bit of value k0 as if the run started there
  uint32_t rval = 0;
  bool rep = false;
  auto set_run = [&](int rr) {
    r = rr;
    rend = w.rk[rr + 1];
    const int32_t b = w.rb[rr];
    rep = b < 0;
    rval = w.rv[rr];
    bbase = b - (w.rk[rr] - k0) * bw;
  };
  set_run(0);
  uint32_t over = 0;  // largest index seen (checked against the dictionary once)
  auto one = [&](int32_t j) -> uint32_t {  // the index of value j, any run
    const int32_t k = k0 + j;
    if (k >= rend) {
      int rr = r + 1;
      while (rr + 1 < nr && w.rk[rr + 1] <= k) ++rr;
      set_run(rr);
    }
    uint32_t v = rval;
    if (!rep) {
      const uint32_t bp = static_cast<uint32_t>(bbase + j * bw);
      v = __funnelshift_r(bw32[bp >> 5], bw32[(bp >> 5) + 1], bp & 31u) & mask;
    }
    return v;
  };
  for (int32_t p0 = lane * VPL; p0 < npos; p0 += 32 * VPL) {
    const int32_t j0 = p0 - head;  // first value of the lane's 16 bytes
    uint32_t x[VPL];
    if (j0 >= 0 && j0 + VPL <= nn && k0 + j0 >= w.rk[r] && k0 + j0 + VPL <= rend) {
      // all values in the current run
      if (rep) {
#pragma unroll
        for (int u = 0; u < VPL; ++u) x[u] = rval;
      } else {
        const uint32_t bp = static_cast<uint32_t>(bbase + j0 * bw);
        const uint32_t* wp = bw32 + (bp >> 5);
        const uint32_t sh = bp & 31u;
        if (bw <= 8) {  // every value of the lane in one 32-bit window
          const uint32_t win = __funnelshift_r(wp[0], wp[1], sh);
#pragma unroll
          for (int u = 0; u < VPL; ++u) x[u] = (win >> (u * bw)) & mask;
        } else {
          // 64-bit windows of VPL / 2 values each (2 * bw <= 64)
#pragma unroll
          for (int h = 0; h < VPL; h += 2) {
            const uint32_t bq = sh + static_cast<uint32_t>(h * bw);
            const uint32_t* wq = wp + (bq >> 5);
            const uint32_t s2 = bq & 31u;
            const uint32_t lo = __funnelshift_r(wq[0], wq[1], s2), hi = __funnelshift_r(wq[1], wq[2], s2);
            x[h] = lo & mask;
            x[h + 1] = __funnelshift_rc(lo, hi, static_cast<uint32_t>(bw)) & mask;  // (clamped: bw may be 32)
          }
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < VPL; ++u) {
        const int32_t j = j0 + u;
        x[u] = (j >= 0 && j < nn) ? one(j) : 0u;
      }
    }
    T v[VPL];
#pragma unroll
    for (int u = 0; u < VPL; ++u) {
      over = max(over, x[u]);
      const uint32_t xi = min(x[u], nmax);
      v[u] = use_s ? dsrc[xi] : __ldg(dsrc + xi);
    }
    if (j0 >= 0 && j0 + VPL <= nn) {
      if constexpr (kWidth == 4)
        *reinterpret_cast<uint4*>(outa + p0) = make_uint4(v[0], v[1], v[2], v[3]);
      else
        *reinterpret_cast<uint4*>(outa + p0) = make_uint4(static_cast<uint32_t>(v[0]), static_cast<uint32_t>(v[0] >> 32),
                                                          static_cast<uint32_t>(v[1]), static_cast<uint32_t>(v[1] >> 32));
    } else {
#pragma unroll
      for (int u = 0; u < VPL; ++u)
        if (j0 + u >= 0 && j0 + u < nn) outa[p0 + u] = v[u];
    }
  }
  if (__any_sync(0xffffffffu, over > nmax) && lane == 0) report(a.st, DERR_CORRUPT, g.page, WHERE_EXPAND, 41);
  return true;
}

template <int kWidth>
__global__ void __launch_bounds__(SX_THREADS) k_dict_expand(DecodeArgs a, int ibegin, int icount, int cidx,
                                                            uint32_t stage, uint32_t dict_cap) {
  extern __shared__ __align__(16) uint8_t sxraw[];
  SxBlock& sm = *reinterpret_cast<SxBlock*>(sxraw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  SxWarp& w = sm.w[wid];
  uint8_t* bufs = sxraw + ((sizeof(SxBlock) + 15) & ~size_t(15));
  uint8_t* const buf0 = bufs + (2 * wid) * (stage + 16);
  uint8_t* const buf1 = buf0 + (stage + 16);
  uint8_t* sdict = dict_cap ? bufs + SX_WARPS * 2u * (stage + 16) : nullptr;
  uint32_t* ctr = a.item_counter + EXP_COUNTER0 + cidx;
  uint8_t* const col_values = a.cols[cidx].values;
  const int nspans = (icount + SX_SPAN - 1) / SX_SPAN;
  const int iend = ibegin + icount;
  if (threadIdx.x == 0) {
    mbar_init(&sm.dbar, 1);
    sm.span = static_cast<int>(atomicAdd(ctr, 1u));
    sm.dchunk = -1;
  }
  if (lane == 0) {
    mbar_init(&w.full[0], 1);
    mbar_init(&w.full[1], 1);
  }
  fence_mbar_init();
  __syncthreads();
  uint32_t par0 = 0, par1 = 0, dpar = 0;
  SxPage pg;
  pg.pp = -1;
  for (;;) {
    const int span = sm.span;
    if (span >= nspans) break;
    __syncthreads();  // every thread has read sm.span
    const int first = ibegin + span * SX_SPAN;
    const int last = first + SX_SPAN < iend ? first + SX_SPAN : iend;
    if (threadIdx.x == 0) sm.span = static_cast<int>(atomicAdd(ctr, 1u));
    if (sdict) {
      // the span's dictionary: that of its first item
      if (threadIdx.x == 0) {
        const Item& it = a.items[first];
        const PlanPage& pp = a.pps[it.pp];
        const bool dict = (pp.enc == ENC_RLE_DICT || pp.enc == ENC_PLAIN_DICT) && pp.dict >= 0;
        int want = dict ? pp.dict : -1;
        if (want >= 0 && want != sm.dchunk) {
          const DictDev& dd = a.dicts[want];
          const uint64_t db = ((static_cast<uint64_t>(dd.n) * dd.width) + 15) & ~uint64_t(15);
          if (db > 0 && db <= dict_cap && dd.values) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&sm.dbar, static_cast<uint32_t>(db));
            bulk_g2s(sdict, dd.values, static_cast<uint32_t>(db), &sm.dbar);
          } else {
            want = -1;
          }
          sm.dchunk = want >= 0 ? -2 - want : -1;  // -2 - chunk: loading
        }
      }
      __syncthreads();
      if (sm.dchunk <= -2) {
        const bool ok = mbar_wait(&sm.dbar, dpar);
        dpar ^= 1u;
        if (!ok) {
          if (threadIdx.x == 0) report(a.st, DERR_TIMEOUT, -1, WHERE_EXPAND, 42);
          mbar_wait(&sm.dbar, dpar ^ 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) sm.dchunk = ok ? -2 - sm.dchunk : -1;
        __syncthreads();
      }
    }
    const int32_t dchunk = sm.dchunk;
    // this warp's items of the span: first + wid, first + wid + SX_WARPS, ...
    int it_c = first + wid;
    SxItem tc = sx_item(a, it_c, last);
    SxItem tn = sx_item(a, it_c + SX_WARPS, last);
    int32_t s0c = 0;
    sx_page(a, tc.item >= 0 ? tc.pp : pg.pp, &pg);
    uint32_t bc = sx_issue(tc, pg, buf0, stage, &w.full[0], &s0c, lane);
    bool cur1 = false;  // the current item sits in buf1
    while (tc.item >= 0) {
      // the next item's copy, and the item after it, while this one is decoded
      SxItem tnn = sx_item(a, it_c + 2 * SX_WARPS, last);
      SxPage pn = pg;
      if (tn.item >= 0) sx_page(a, tn.pp, &pn);
      int32_t s0n = 0;
      const uint32_t bn = sx_issue(tn, pn, cur1 ? buf0 : buf1, stage, cur1 ? &w.full[0] : &w.full[1], &s0n, lane);
      bool done = false;
      if (bc) {
        uint32_t& par = cur1 ? par1 : par0;
        const bool ok = mbar_wait(cur1 ? &w.full[1] : &w.full[0], par);
        par ^= 1u;
        if (!ok) {
          if (lane == 0) report(a.st, DERR_TIMEOUT, pg.page, WHERE_EXPAND, 43);
          mbar_wait(cur1 ? &w.full[1] : &w.full[0], par ^ 1u);
          done = true;
        } else {
          done = sx_decode<kWidth>(a, tc, pg, s0c, bc, cur1 ? buf1 : buf0, w, sdict, dchunk, col_values, lane);
        }
      }
      // (the general decode gets the buffer as its staging area, which only
      // OPTIONAL columns use: this kernel serves REQUIRED ones)
      if (!done) expand_item(a, tc.item, *reinterpret_cast<WarpSmem*>(cur1 ? buf1 : buf0), lane);
      __syncwarp();
      tc = tn;
      tn = tnn;
      pg = pn;
      s0c = s0n;
      bc = bn;
      cur1 = !cur1;
      it_c += SX_WARPS;
    }
    __syncthreads();  // the span is done: the dictionary may be replaced
  }
}

// ------------------------------------------------------------------ strings

// Per string column: exclusive prefix of item chars; writes the final offset.
__global__ void __launch_bounds__(1024) k_str_scan(DecodeArgs a, int c) {
  const OutCol col = a.cols[c];
  __shared__ uint64_t tmp[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b = 0; b < col.item_count; b += blockDim.x * 4) {
    uint64_t loc[4];
    uint64_t mine = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = b + threadIdx.x * 4 + q;
      loc[q] = i < col.item_count ? col.str_item_bytes[col.item_begin + i] : 0;
      mine += loc[q];
    }
    uint64_t tot;
    uint64_t run = carry + block_exclusive_sum(mine, tmp, &tot);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t i = b + threadIdx.x * 4 + q;
      if (i < col.item_count) col.str_item_bytes[col.item_begin + i] = run;
      run += loc[q];
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    reinterpret_cast<int64_t*>(col.values)[col.n_rows] = static_cast<int64_t>(carry);
    if (carry > col.chars_cap) report(a.st, DERR_CAPACITY, -1, WHERE_STRINGS, 1);
  }
}

// Copies `len` bytes from global `src` (any alignment) to shared `d` (any
// alignment) whose words start at zero.  The source is read as aligned
// 16-byte words (about (len + 15) / 16 + 1 sectors per string, instead of
// one per 4 bytes), the destination is OR-ed in as 4-byte words
// funnel-shifted from them, the partial words at the string's two ends
// masked (neighbouring strings OR their own bytes into them).  The aligned
// words may reach up to 16 bytes past `src + len`; callers guarantee those
// bytes are readable.
__device__ __forceinline__ void stage_string(uint8_t* d, const uint8_t* src, uint32_t len) {
  const int p = static_cast<int>(reinterpret_cast<uintptr_t>(src) & 15);
  const uint4* sv = reinterpret_cast<const uint4*>(reinterpret_cast<uintptr_t>(src) - p);
  const int dd = static_cast<int>(reinterpret_cast<uintptr_t>(d) & 3);
  uint32_t* dw = reinterpret_cast<uint32_t*>(d - dd);
  const int nw = (dd + static_cast<int>(len) + 3) >> 2;  // destination words touched
  const int q0 = p - dd;                                  // span byte of destination word 0 (>= -3)
  const uint32_t sh = static_cast<uint32_t>(q0 & 3) * 8;
  int wi = q0 >> 2;                                       // span word (-1 when q0 < 0)
  auto pick = [](const uint4& x, int k) -> uint32_t {
    return (k & 2) ? ((k & 1) ? x.w : x.z) : ((k & 1) ? x.y : x.x);
  };
  uint4 v = __ldg(sv + (wi < 0 ? 0 : (wi >> 2)));
  uint32_t cur = wi < 0 ? 0u : pick(v, wi & 3);
  const int end = dd + static_cast<int>(len);             // destination bytes [dd, end) relative to dw
  const uint32_t mfirst = 0xffffffffu << (8 * dd);
  const uint32_t mlast = (end & 3) ? (0xffffffffu >> (8 * (4 - (end & 3)))) : 0xffffffffu;
  for (int k = 0; k < nw; ++k) {
    ++wi;
    if ((wi & 3) == 0) v = __ldg(sv + (wi >> 2));
    const uint32_t nxt = pick(v, wi & 3);
    uint32_t val = __funnelshift_r(cur, nxt, sh);
    cur = nxt;
    if (k == 0) val &= mfirst;
    if (k == nw - 1) val &= mlast;
    atomicOr(dw + k, val);
  }
}

// Same copy from a shared-memory copy of the aligned source span (`raw`,
// 16-byte aligned, holding span bytes [0, p + len) and readable for 16
// bytes more).
__device__ __forceinline__ void stage_from_raw(uint8_t* d, const uint8_t* raw, int p, uint32_t len) {
  const uint32_t* rw = reinterpret_cast<const uint32_t*>(raw);
  const int dd = static_cast<int>(reinterpret_cast<uintptr_t>(d) & 3);
  uint32_t* dw = reinterpret_cast<uint32_t*>(d - dd);
  const int nw = (dd + static_cast<int>(len) + 3) >> 2;
  const int q0 = p - dd;
  const uint32_t sh = static_cast<uint32_t>(q0 & 3) * 8;
  int wi = q0 >> 2;
  uint32_t cur = wi < 0 ? 0u : rw[wi];
  const int end = dd + static_cast<int>(len);
  // the destination words start at zero and may be shared with neighbouring
  // strings at the two ends: every word is OR-ed in, the end words masked
  const uint32_t mfirst = 0xffffffffu << (8 * dd);
  const uint32_t mlast = (end & 3) ? (0xffffffffu >> (8 * (4 - (end & 3)))) : 0xffffffffu;
  for (int k = 0; k < nw; ++k) {
    ++wi;
    const uint32_t nxt = rw[wi];
    uint32_t val = __funnelshift_r(cur, nxt, sh);
    cur = nxt;
    if (k == 0) val &= mfirst;
    if (k == nw - 1) val &= mlast;
    atomicOr(dw + k, val);
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Per item of a string column, one warp: offsets by a warp scan of the
// lengths; strings are processed 64 at a time: each lane's source spans
// (up to STR_RAW_BLK aligned 16-byte blocks) are fetched together with
// asynchronous global-to-shared copies, then each 32-string chunk is
// assembled in shared memory (lanes place their own string) and written out
// with aligned 16-byte stores, bytes only at the chunk's two ends.  Longer
// strings are read straight from global memory.
constexpr int STR_STAGE = 2016;
constexpr int STR_RAW_BLK = 4;  // strings up to 49 bytes go through the async copies
constexpr int STR_SLOT = STR_RAW_BLK + 1;  // slot stride in 16-byte blocks (spreads lanes over banks)
struct StrWarpSmem {
  uint8_t stage[STR_STAGE + 16];
  uint4 raw[64 * STR_SLOT + 1];  // +1: the last slot's read-ahead word
};
constexpr int STR_SMEM = 8 * sizeof(StrWarpSmem);

__global__ void __launch_bounds__(256, 4) k_str_copy(DecodeArgs a, int c) {
  extern __shared__ __align__(16) uint8_t str_smem[];
  StrWarpSmem& ws = reinterpret_cast<StrWarpSmem*>(str_smem)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  uint8_t* sbuf = ws.stage;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int ib = static_cast<int>(a.cols[c].item_begin);
  const int ie = ib + static_cast<int>(a.cols[c].item_count);
  {
    uint4* zv = reinterpret_cast<uint4*>(sbuf);
    for (int q = lane; q < (STR_STAGE + 16) / 16; q += 32) zv[q] = make_uint4(0, 0, 0, 0);
    __syncwarp();
  }
  for (int itx = ib + gw; itx < ie; itx += nw) {
    const Item it = a.items[itx];
    if (it.nrows <= 0) continue;
    const PlanPage pp = a.pps[it.pp];
    const OutCol col = a.cols[pp.col];
    if (col.ptype != T_BYTE_ARRAY || pp.nonnull < 0) continue;
    // (a transcoded page is never a dictionary page: its own encoding decides)
    const PageDev pg = a.pages[pp.page];
    const bool isdict = pg.encoding == ENC_RLE_DICT || pg.encoding == ENC_PLAIN_DICT;
    DictDev dd{};
    if (isdict && pp.dict >= 0) dd = a.dicts[pp.dict];
    const uint8_t* sb = pp.body + pp.values_off;
    uint64_t base = col.str_item_bytes[itx];
    const int64_t orow0 = pp.out_row + it.row0;
    int64_t* offs = reinterpret_cast<int64_t*>(col.values);
    const uint8_t* cbase = isdict ? dd.chars : sb;
    // PLAIN pages: every string lies inside the page's value bytes (an entry
    // that does not is dropped and reported; the expand writes none such)
    const uint64_t clen = isdict ? ~0ull : static_cast<uint64_t>(pp.body_len > pp.values_off
                                                                     ? pp.body_len - pp.values_off : 0);
    for (int g0 = 0; g0 < it.nrows; g0 += 256) {
      // metadata of 4 chunks of 64 strings, loads issued together; lane l
      // takes rows 2l and 2l+1 of each chunk (adjacent in the output)
      uint64_t ent[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int r = g0 + (u >> 1) * 64 + 2 * lane + (u & 1);
        ent[u] = r < it.nrows ? col.str_scratch[orow0 + r] : 0ull;
      }
      bool outside = false;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if ((ent[u] >> 32) + static_cast<uint32_t>(ent[u]) > clen) {
          ent[u] = 0;
          outside = true;
        }
      }
      if (__any_sync(0xffffffffu, outside) && lane == 0) report(a.st, DERR_CORRUPT, static_cast<int>(pp.page), WHERE_EXPAND, 60);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int r0 = g0 + cc * 64;
        if (r0 >= it.nrows) break;
        // source spans of the lane's two strings, fetched together
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const uint32_t len = static_cast<uint32_t>(ent[2 * cc + t]);
          const uint8_t* src = cbase + (ent[2 * cc + t] >> 32);
          const uint32_t p = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 15);
          const uint32_t nb = (p + len + 15) >> 4;
          if (len && nb <= STR_RAW_BLK) {
            const uint8_t* sa = src - p;
            uint4* slot = ws.raw + (t * 32 + lane) * STR_SLOT;
            for (uint32_t b = 0; b < nb; ++b) cp_async16(slot + b, sa + 16 * b);
          }
        }
        const uint32_t lena = static_cast<uint32_t>(ent[2 * cc]), lenb = static_cast<uint32_t>(ent[2 * cc + 1]);
        const uint32_t mine = lena + lenb;
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t rel = incl - mine;  // chunk-relative offset of the lane's first string
        const int ra = r0 + 2 * lane;
        if (ra < it.nrows) offs[orow0 + ra] = static_cast<int64_t>(base + rel);
        if (ra + 1 < it.nrows) offs[orow0 + ra + 1] = static_cast<int64_t>(base + rel + lena);
        cp_async_wait_all();
        __syncwarp();
        if (base + tot <= col.chars_cap) {
          const uint32_t a0 = static_cast<uint32_t>(base & 15);
          if (a0 + tot <= STR_STAGE) {
            // the chunk is assembled in shared memory congruent to the output
            // mod 16.  Fast path: every lane with rows holds at least 4 bytes
            // and both its strings sit in its source slots; each staging
            // word is then written once, by the lane whose span holds the
            // word's first byte, and the few bytes of a word that belong to
            // the next lane's span come from that lane by a shuffle.
            const int pa = static_cast<int>(reinterpret_cast<uintptr_t>(cbase + (ent[2 * cc] >> 32)) & 15);
            const int pb = static_cast<int>(reinterpret_cast<uintptr_t>(cbase + (ent[2 * cc + 1] >> 32)) & 15);
            const bool has = ra < it.nrows;
            const bool good = !has || (lena + lenb >= 4 && ((pa + lena + 15) >> 4) <= STR_RAW_BLK &&
                                       ((pb + lenb + 15) >> 4) <= STR_RAW_BLK);
            if (__all_sync(0xffffffffu, good)) {
              const uint32_t* rwa = reinterpret_cast<const uint32_t*>(ws.raw + lane * STR_SLOT);
              const uint32_t* rwb = reinterpret_cast<const uint32_t*>(ws.raw + (32 + lane) * STR_SLOT);
              const int sa = static_cast<int>(a0 + rel), ea = sa + static_cast<int>(lena),
                        eb = ea + static_cast<int>(lenb);
              // 4 bytes at byte `off` (>= -3) of a source slot
              auto srcw = [](const uint32_t* rw, int off) -> uint32_t {
                const int q = off >> 2;
                return __funnelshift_r(rw[q], rw[q + 1], static_cast<uint32_t>(off & 3) * 8);
              };
              auto bmask = [](int n) -> uint32_t {
                return n <= 0 ? 0u : (n >= 4 ? 0xffffffffu : ((1u << (8 * n)) - 1u));
              };
              // staging word w from the lane's two strings and `nxt` (bytes at
              // and past eb, placed in the word)
              auto mix = [&](int w, uint32_t nxt) -> uint32_t {
                const int x = 4 * w;
                const uint32_t ma = bmask(ea - x), mab = bmask(eb - x);
                const uint32_t va = x < ea ? srcw(rwa, pa + x - sa) : 0u;
                const uint32_t vb = (x + 4 > ea && x < eb) ? srcw(rwb, pb + x - ea) : 0u;
                return (va & ma) | (vb & mab & ~ma) | (nxt & ~mab);
              };
              const uint32_t head = (has && (sa & 3)) ? (mix(sa >> 2, 0u) & ~bmask(sa & 3)) : 0u;
              uint32_t nxt = __shfl_down_sync(0xffffffffu, head, 1);
              if (lane == 31) nxt = 0;
              if (has) {
                uint32_t* sw = reinterpret_cast<uint32_t*>(sbuf);
                int w = (lane == 0) ? (sa >> 2) : ((sa + 3) >> 2);
                const int wa = ea >> 2, wb = eb >> 2;
                if (w < wa) {  // words wholly inside the first string
                  const int off = pa + 4 * w - sa;
                  int q = off >> 2;
                  const uint32_t sh = static_cast<uint32_t>(off & 3) * 8;
                  uint32_t cur = rwa[q];
                  for (; w < wa; ++w) {
                    const uint32_t n2 = rwa[++q];
                    sw[w] = __funnelshift_r(cur, n2, sh);
                    cur = n2;
                  }
                }
                if ((ea & 3) && w == wa) sw[w++] = mix(wa, nxt);  // end of the first string
                if (w < wb) {  // words wholly inside the second string
                  const int off = pb + 4 * w - ea;
                  int q = off >> 2;
                  const uint32_t sh = static_cast<uint32_t>(off & 3) * 8;
                  uint32_t cur = rwb[q];
                  for (; w < wb; ++w) {
                    const uint32_t n2 = rwb[++q];
                    sw[w] = __funnelshift_r(cur, n2, sh);
                    cur = n2;
                  }
                }
                if ((eb & 3) && w == wb) sw[w] = mix(wb, nxt);  // end of the span
              }
            } else {
              // general path: the staging area starts at zero and lanes OR
              // their strings in (end words are shared)
              uint4* zv = reinterpret_cast<uint4*>(sbuf);
              for (uint32_t q = lane; q < (a0 + tot + 15) / 16; q += 32) zv[q] = make_uint4(0, 0, 0, 0);
              __syncwarp();
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const uint32_t len = t ? lenb : lena;
                if (!len) continue;
                const uint8_t* src = cbase + (ent[2 * cc + t] >> 32);
                const int p = static_cast<int>(reinterpret_cast<uintptr_t>(src) & 15);
                uint8_t* d = sbuf + a0 + rel + (t ? lena : 0u);
                if (((p + len + 15) >> 4) <= STR_RAW_BLK)
                  stage_from_raw(d, reinterpret_cast<const uint8_t*>(ws.raw + (t * 32 + lane) * STR_SLOT), p, len);
                else
                  stage_string(d, src, len);
              }
            }
            __syncwarp();
            uint8_t* g = col.chars + base;
            const uint32_t head = a0 ? 16 - a0 : 0;
            const uint32_t hh = head < tot ? head : tot;
            if (static_cast<uint32_t>(lane) < hh) g[lane] = sbuf[a0 + lane];
            const uint32_t nv = (tot - hh) >> 4;
            const uint4* sv = reinterpret_cast<const uint4*>(sbuf + a0 + hh);
            uint4* gv = reinterpret_cast<uint4*>(g + hh);
            for (uint32_t q = lane; q < nv; q += 32) gv[q] = sv[q];
            for (uint32_t q = hh + (nv << 4) + lane; q < tot; q += 32) g[q] = sbuf[a0 + q];
            __syncwarp();
          } else {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
              const uint32_t len = t ? lenb : lena;
              const uint8_t* src = cbase + (ent[2 * cc + t] >> 32);
              uint8_t* d = col.chars + base + rel + (t ? lena : 0u);
              for (uint32_t q = 0; q < len; ++q) d[q] = __ldg(src + q);
            }
          }
        }
        base += tot;
        __syncwarp();
      }
    }
  }
}

// ------------------------------------------------------------------ plain baseline

// One page per thread block: the walk, DELTA bases, then the block's warps
// decode the page's items.
__global__ void __launch_bounds__(WALK_THREADS) k_plain_page(DecodeArgs a, int pp_begin) {
  extern __shared__ __align__(16) uint8_t smraw[];
  WalkSmem& sm = *reinterpret_cast<WalkSmem*>(smraw);
  const int p = pp_begin + blockIdx.x;
  walk_init(sm, CWIN);
  const PlanPage pp0 = a.pps[p];
  const ChunkDev ch = a.chunks[pp0.chunk];
  const bool needs_walk = ch.max_def || pp0.enc != ENC_PLAIN || ch.ptype == T_BYTE_ARRAY;
  if (needs_walk) walk_page(a, p, sm, true);
  __syncthreads();
  // the chain windows, free again: scan scratch, then the warps' staging
  uint8_t* wins = smraw + ((sizeof(WalkSmem) + 15) & ~size_t(15));
  if (pp0.enc == ENC_DELTA_BP) {
    delta_bases_page(a, p, reinterpret_cast<uint64_t*>(wins + CWIN + 16));
    __syncthreads();
  }
  const PlanPage pp = a.pps[p];
  static_assert(sizeof(WarpSmem) * (WALK_THREADS / 32) <= 2 * (CWIN + 16), "warp staging must fit the windows");
  WarpSmem* ws = reinterpret_cast<WarpSmem*>(wins);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t i = warp; i < pp.item_count; i += nw) expand_item(a, static_cast<int>(pp.item_begin + i), ws[warp], lane);
}

// ------------------------------------------------------------------ per-scan reset

// Zeroes the validity bitmaps (bits are OR-ed in by the walk), the string
// item totals, the work counters and the error word.
__global__ void k_prepare(DecodeArgs a, int n_cols) {
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint64_t nthr = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  if (tid < static_cast<uint64_t>(EXP_COUNTER0 + n_cols)) a.item_counter[tid] = 0;
  if (tid == 0) {
    a.st->flags = 0;
    a.st->first_page = -1;
    a.st->where = 0;
    a.st->detail = 0;
  }
  for (int c = 0; c < n_cols; ++c) {
    const OutCol col = a.cols[c];
    if (col.validity) {
      const uint64_t words = (static_cast<uint64_t>(col.n_rows) + 31) / 32;
      for (uint64_t i = tid; i < words; i += nthr) col.validity[i] = 0;
    }
    if (col.str_item_bytes)
      for (uint64_t i = tid; i < col.item_count; i += nthr) col.str_item_bytes[col.item_begin + i] = 0;
  }
}

__global__ void k_add_offsets(int64_t* offs, int64_t n, int64_t base) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    offs[i] += base;
}

// Exactly `bytes` bytes (no read past them), 4-byte words when both ends
// allow: small control transfers into pinned host memory.
__global__ void k_copy_small(uint8_t* dst, const uint8_t* src, uint32_t bytes) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 3) == 0) {
    const uint32_t nw = bytes >> 2;
    for (uint32_t i = t; i < nw; i += nt)
      reinterpret_cast<uint32_t*>(dst)[i] = reinterpret_cast<const uint32_t*>(src)[i];
    for (uint32_t i = (nw << 2) + t; i < bytes; i += nt) dst[i] = src[i];
  } else {
    for (uint32_t i = t; i < bytes; i += nt) dst[i] = src[i];
  }
}

void launch_copy_small(void* dst, const void* src, uint32_t bytes, cudaStream_t s) {
  if (!bytes) return;
  const uint32_t blocks = std::min<uint32_t>((bytes / 4 + 255) / 256 + 1, 32);
  k_copy_small<<<blocks, 256, 0, s>>>(static_cast<uint8_t*>(dst), static_cast<const uint8_t*>(src), bytes);
}

void launch_add_offsets(int64_t* offs, int64_t n, int64_t base, cudaStream_t s) {
  if (n <= 0 || base == 0) return;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  k_add_offsets<<<static_cast<unsigned>(blocks), 256, 0, s>>>(offs, n, base);
}

void launch_prepare(const DecodeArgs& a, int n_cols, int grid, cudaStream_t s) {
  k_prepare<<<grid, 256, 0, s>>>(a, n_cols);
}

// ------------------------------------------------------------------ work items

// One warp per plan page: item j covers page rows [row_lo + j*R, ...) with R
// the page's item rows; the dense range starts equal to the row range (the
// walk rewrites it for pages with levels).
__global__ void __launch_bounds__(256) k_make_items(DecodeArgs a, int n_pp) {
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= n_pp) return;
  const PlanPage pp = a.pps[p];
  for (uint32_t j = lane; j < pp.item_count; j += 32) {
    Item it{};
    it.pp = static_cast<uint32_t>(p);
    it.row0 = pp.row_lo + static_cast<int32_t>(j) * pp.item_rows;
    const int32_t left = pp.row_hi - it.row0;
    it.nrows = left < pp.item_rows ? left : pp.item_rows;
    it.k0 = it.row0;
    it.nn = it.nrows;
    a.items[pp.item_begin + j] = it;
  }
}

// ------------------------------------------------------------------ one DELTA stream, fixed scratch

// Fills the one-page plan of a bare DELTA stream: status cleared, header
// parsed and checked against the expected value count.
__global__ void k_dstatic_init(DecodeArgs a, ChunkDev* chunk, uint32_t* delta_pps, const uint8_t* stream,
                               uint32_t len, int ptype, int32_t n) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  *a.st = DevStatus{0u, -1, 0, 0};
  ChunkDev ch{};
  ch.ptype = ptype;
  ch.width = ptype == T_INT32 ? 4 : 8;
  *chunk = ch;
  *delta_pps = 0;
  PlanPage pp{};
  pp.body = stream;
  pp.body_len = static_cast<int32_t>(len);
  pp.values_off = 0;
  pp.nonnull = -1;
  pp.dtab = 0;
  pp.dreg = 0;
  pp.dreg_cap = static_cast<int32_t>(len / DELTA_REGION + 2);
  pp.dblocks = -1;
  DeltaHdr d{};
  if (!delta_header(stream, len, &d)) {
    report(a.st, DERR_UNSUPPORTED, 0, WHERE_WALK_VALUES, 40);
  } else if (d.total != n || (n > 1 && (n - 2) / d.block + 1 > DS_MAX_BLOCKS)) {
    report(a.st, DERR_CORRUPT, 0, WHERE_WALK_VALUES, 41);
  } else {
    pp.nonnull = n;
    pp.dfirst = d.first;
    pp.dbs = d.block;
    pp.dvpm = d.vpm;
    pp.dmbc = d.mbc;
    pp.dhlen = d.hlen;
    pp.dblocks = n > 1 ? -2 : 0;
  }
  a.pps[0] = pp;
}

// One warp per DS_WARP_VALUES values, from the block tables.
constexpr int DS_WARP_VALUES = 4096;
__global__ void __launch_bounds__(256) k_dstatic_expand(DecodeArgs a, uint8_t* out, int32_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t w = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t k0 = w * DS_WARP_VALUES;
  if (k0 >= n) return;
  const int32_t k1 = static_cast<int32_t>(k0 + DS_WARP_VALUES < n ? k0 + DS_WARP_VALUES : n);
  const PlanPage pp = a.pps[0];
  if (pp.nonnull < 0 || (n > 1 && pp.dblocks <= 0)) return;  // error already reported
  const int ptype = a.chunks[0].ptype;
  Sink sink{out, nullptr, nullptr, k0, ptype == T_INT32 ? 4 : 8};
  if (!warp_delta(pp.body, pp, a.dpos, a.dbase, ptype == T_INT32 ? 32 : 64, static_cast<int32_t>(k0), k1, sink,
                  lane) &&
      lane == 0)
    report(a.st, DERR_CORRUPT, 0, WHERE_EXPAND, 42);
}

void launch_make_items(const DecodeArgs& a, int n_pp, cudaStream_t s) {
  if (n_pp > 0) k_make_items<<<(n_pp + 7) / 8, 256, 0, s>>>(a, n_pp);
}

void launch_delta_static(uint8_t* scratch, const uint8_t* stream, uint32_t len, int ptype, int32_t n, void* out,
                         cudaStream_t s) {
  DecodeArgs a{};
  a.st = reinterpret_cast<DevStatus*>(scratch + DS_OFF_STATUS);
  a.chunks = reinterpret_cast<ChunkDev*>(scratch + DS_OFF_CHUNK);
  a.pps = reinterpret_cast<PlanPage*>(scratch + DS_OFF_PAGE);
  a.delta_pps = reinterpret_cast<uint32_t*>(scratch + DS_OFF_PPS);
  a.dregs = reinterpret_cast<DeltaRegion*>(scratch + DS_OFF_REGIONS);
  a.dreg_lists = reinterpret_cast<uint32_t*>(scratch + DS_OFF_LISTS);
  a.dpos = reinterpret_cast<uint32_t*>(scratch + DS_OFF_DPOS);
  a.dbase = reinterpret_cast<int64_t*>(scratch + DS_OFF_DBASE);
  a.n_pp = 1;
  a.n_delta = 1;
  k_dstatic_init<<<1, 32, 0, s>>>(a, reinterpret_cast<ChunkDev*>(scratch + DS_OFF_CHUNK),
                                  reinterpret_cast<uint32_t*>(scratch + DS_OFF_PPS), stream, len, ptype, n);
  launch_delta_bases(a, 0, 1, static_cast<int>(len / DELTA_REGION + 2), s);
  if (n > 0) {
    const int64_t warps = (static_cast<int64_t>(n) + DS_WARP_VALUES - 1) / DS_WARP_VALUES;
    k_dstatic_expand<<<static_cast<unsigned>((warps + 7) / 8), 256, 0, s>>>(a, static_cast<uint8_t*>(out), n);
  }
}

// ------------------------------------------------------------------ launchers

static int g_walk_bps = 0, g_exp_bps = 0;

int walk_blocks_per_sm() {
  if (!g_walk_bps) {
    cudaFuncSetAttribute(k_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, walk_smem_bytes(CWIN_MAX, JW));
    cudaFuncSetAttribute(k_plain_page, cudaFuncAttributeMaxDynamicSharedMemorySize, walk_smem_bytes(CWIN));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_walk_bps, k_walk, WALK_THREADS, walk_smem_bytes(CWIN));
    if (g_walk_bps < 1) g_walk_bps = 1;
  }
  return g_walk_bps;
}

int expand_blocks_per_sm() {
  if (!g_exp_bps) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_exp_bps, k_expand, EXP_THREADS, 0);
    if (g_exp_bps < 1) g_exp_bps = 1;
  }
  return g_exp_bps;
}

void launch_walk(const DecodeArgs& a, int wbegin, int n, int n_sms, bool levels, uint32_t window, cudaStream_t s) {
  if (n <= 0) return;
  walk_blocks_per_sm();  // sets the shared-memory attributes
  // few pages (long chains each): larger windows, fewer refills on the
  // chain's path; many pages: more resident walkers
  const uint32_t cap = window ? (window < CWIN_MAX ? window : CWIN_MAX)
                              : (n <= n_sms ? CWIN_MAX : (n <= 2 * n_sms ? CWIN_MAX / 2 : CWIN));
  // level walks: smaller chain windows, so that the jump tables leave room
  // for as many resident walkers
  const uint32_t jw = levels ? JW : 0u;
  const uint32_t wcap = levels && cap > CWIN / 2 ? CWIN / 2 : cap;
  k_walk<<<n, WALK_THREADS, walk_smem_bytes(wcap, jw), s>>>(a, wbegin, wcap, jw);
}

void launch_delta_bases(const DecodeArgs& a, int dbegin, int n, int max_regions, cudaStream_t s) {
  if (n <= 0) return;
  static bool attr = false;
  constexpr int dreg_smem = DREG_SMEM;
  if (!attr) {
    cudaFuncSetAttribute(k_dreg, cudaFuncAttributeMaxDynamicSharedMemorySize, dreg_smem);
    attr = true;
  }
  if (max_regions > 0) {
    k_dreg<<<dim3(max_regions, n), 32, dreg_smem, s>>>(a, dbegin);
    k_dfix<<<n, 256, 0, s>>>(a, dbegin);
  }
  k_delta_sums<<<dim3(64, n), 256, 0, s>>>(a, dbegin);
  k_delta_scan<<<n, 1024, 0, s>>>(a, dbegin);
}

void launch_copy_items(const DecodeArgs& a, int ibegin, int n, int cidx, int n_sms, int ctas_per_sm,
                       cudaStream_t s) {
  if (n <= 0) return;
  static int bps = 0;
  if (!bps) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_copy_items, 256, 0);
    if (bps < 1) bps = 1;
  }
  const int per_sm = ctas_per_sm > 0 && ctas_per_sm < bps ? ctas_per_sm : bps;
  int blocks = (n + 7) / 8;
  if (blocks > n_sms * per_sm) blocks = n_sms * per_sm;
  k_copy_items<<<blocks, 256, 0, s>>>(a, ibegin, n, cidx);
}

uint32_t dict_expand_stage_bytes(int item_rows, int bw_est) {
  // the checkpoint run may start up to 504 values before the item
  const uint64_t bits = static_cast<uint64_t>(item_rows + 512) * static_cast<uint64_t>(bw_est < 1 ? 1 : bw_est);
  const uint64_t b = bits / 8 + bits / 128 + 160;
  return static_cast<uint32_t>((b + 15) & ~uint64_t(15));
}

bool dict_expand_fits(uint32_t stage, uint32_t dict_cap) {
  return sx_smem_bytes(stage, dict_cap) <= 227u * 1024u && dict_cap <= SX_DICT_MAX;
}

void launch_dict_expand(const DecodeArgs& a, int ibegin, int n, int cidx, int n_sms, int width, uint32_t stage,
                        uint32_t dict_cap, cudaStream_t s) {
  if (n <= 0) return;
  const uint32_t smem = sx_smem_bytes(stage, dict_cap);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_dict_expand<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_dict_expand<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr = true;
  }
  int bps = 0;
  if (width == 4)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_dict_expand<4>, SX_THREADS, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_dict_expand<8>, SX_THREADS, smem);
  if (bps < 1) bps = 1;
  const int spans = (n + SX_SPAN - 1) / SX_SPAN;
  int blocks = n_sms * bps;
  if (blocks > spans) blocks = spans;
  if (width == 4)
    k_dict_expand<4><<<blocks, SX_THREADS, smem, s>>>(a, ibegin, n, cidx, stage, dict_cap);
  else
    k_dict_expand<8><<<blocks, SX_THREADS, smem, s>>>(a, ibegin, n, cidx, stage, dict_cap);
}

void launch_expand(const DecodeArgs& a, int ibegin, int n, int cidx, int n_sms, int ctas_per_sm, cudaStream_t s) {
  if (n <= 0) return;
  int blocks = (n + EXP_WARPS - 1) / EXP_WARPS;
  const int bps = expand_blocks_per_sm();
  const int cap = n_sms * (ctas_per_sm > 0 && ctas_per_sm < bps ? ctas_per_sm : bps);
  if (blocks > cap) blocks = cap;
  k_expand<<<blocks, EXP_THREADS, 0, s>>>(a, ibegin, n, cidx);
}

void launch_strings(const DecodeArgs& a, int col, int n_items, int n_sms, bool copy_chars, cudaStream_t s) {
  if (n_items <= 0) return;
  k_str_scan<<<1, 1024, 0, s>>>(a, col);
  if (!copy_chars) return;
  int blocks = (n_items + 7) / 8;
  if (blocks > n_sms * 8) blocks = n_sms * 8;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_str_copy, cudaFuncAttributeMaxDynamicSharedMemorySize, STR_SMEM);
    attr = true;
  }
  k_str_copy<<<blocks, 256, STR_SMEM, s>>>(a, col);
}

void launch_plain_pages(const DecodeArgs& a, int pp_begin, int n, cudaStream_t s) {
  if (n <= 0) return;
  k_plain_page<<<n, WALK_THREADS, walk_smem_bytes(CWIN), s>>>(a, pp_begin);
}

}  // namespace pqi
