// V2 page encodings turned into PLAIN page bodies before the walk.
//
// The paper's Section 3 ("Encoding Flexibility", Insight 3) counts the V2
// encodings among the GPU-friendly ones.  Three of them are read here by
// rewriting each page into the PLAIN layout that the walk and expand kernels
// already decode at full speed:
//
//   BYTE_STREAM_SPLIT        K streams of N bytes (stream b = byte b of every
//                            value)  ->  N little-endian K-byte values
//   DELTA_LENGTH_BYTE_ARRAY  DELTA_BINARY_PACKED INT32 lengths, then the bytes
//                            ->  (4-byte length, bytes) per value
//   DELTA_BYTE_ARRAY         DELTA_BINARY_PACKED INT32 prefix lengths, then the
//                            suffixes as DELTA_LENGTH_BYTE_ARRAY; value i is
//                            the first prefix[i] bytes of value i-1 followed by
//                            suffix i  ->  (4-byte length, bytes) per value
//
// One thread block per page.  The page's level bytes (V1: 4-byte length +
// levels; V2: def_len bytes) are copied unchanged in front of the new values,
// so the walk parses the new body exactly like a PLAIN page.  The kernel sets
// the plan page's body and body_len; on an error it points the page at its
// level bytes only, so that later stages read nothing past them.
//
// DELTA_BYTE_ARRAY resolves prefixes 256 values at a time: a value's own
// suffix gives its bytes from prefix[i] on; its bytes below that come, by
// walking back through the batch, from the suffix of the nearest earlier
// value whose prefix is shorter, and the bytes that no value in the batch
// supplies come from the previous batch's last value, already written out.
#include "decode_job.h"
#include "dev_util.cuh"

namespace pqi {
namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_PER_THREAD = 8;
constexpr uint32_t TC_MAX_BLOCK = TC_THREADS * TC_PER_THREAD;  // DELTA block values a cursor holds
constexpr uint32_t TC_MAX_MB = TC_MAX_BLOCK / 32;

// Block-shared state of one DELTA_BINARY_PACKED INT32 stream.
struct DCursor {
  uint32_t hdr_end;   // first block header
  uint32_t pos;       // next block header
  uint32_t end;       // end of the readable bytes
  uint32_t left;      // values still to decode after the buffered ones
  uint32_t nbuf;      // values in buf
  uint32_t cnt;       // values in the block being decoded
  uint32_t bs, mbc, vpm, total;
  int32_t first;
  int32_t last;       // last decoded value
  int32_t started;
  int32_t pad;
  int64_t minv[TC_MAX_MB];  // min delta of each buffered miniblock's block
  uint32_t mboff[TC_MAX_MB];
  uint8_t width[TC_MAX_MB];
  int32_t buf[TC_MAX_BLOCK];
};

struct TcSmem {
  DCursor c[2];
  int64_t tmp[32];
  int64_t lb[TC_THREADS];   // DELTA_BYTE_ARRAY: value lengths of the batch
  int64_t db[TC_THREADS];   // chars start of each value (offset into dst)
  int64_t sb[TC_THREADS];   // suffix start of each value (offset into src)
  int32_t pb[TC_THREADS];   // prefix lengths of the batch
  int32_t err;
  int32_t flag;             // DERR_* of the first error
  int32_t detail;
  uint32_t v0;
  uint64_t dst_off;
};

__device__ __forceinline__ void tc_fail(TcSmem& sm, uint32_t flag, int detail) {
  if (atomicCAS(&sm.err, 0, 1) == 0) {
    sm.flag = static_cast<int32_t>(flag);
    sm.detail = detail;
  }
}

__device__ __forceinline__ uint32_t get_bits(const uint8_t* b, uint32_t byte0, uint32_t bit, int w) {
  if (w == 0) return 0;
  const uint32_t p = byte0 + (bit >> 3), sh = bit & 7;
  const int nb = static_cast<int>((sh + w + 7) >> 3);
  uint64_t v = 0;
  for (int i = 0; i < nb; ++i) v |= static_cast<uint64_t>(ld_u8(b + p + i)) << (8 * i);
  return static_cast<uint32_t>((v >> sh) & ((1ull << w) - 1));
}

// Thread 0: parses the stream header at `p` and walks the block headers to
// the stream end (after the last miniblock that holds values).  Records the
// result in `c`; errors go to sm.
__device__ void dstream_open(const uint8_t* b, uint32_t p, uint32_t end, DCursor& c, TcSmem& sm) {
  auto get = [b](uint32_t i) { return ld_u8(b + i); };
  uint64_t v[4];
  uint32_t q = p;
  for (int k = 0; k < 4; ++k) {
    const int n = uleb(get, q, end, &v[k]);
    if (!n) {
      tc_fail(sm, DERR_CORRUPT, 1);
      return;
    }
    q += static_cast<uint32_t>(n);
  }
  if (v[0] == 0 || v[0] % 128 || v[1] == 0 || v[0] % v[1] || (v[0] / v[1]) % 32) {
    tc_fail(sm, DERR_CORRUPT, 2);
    return;
  }
  if (v[0] > TC_MAX_BLOCK || v[2] > 0x7fffffffull) {
    tc_fail(sm, DERR_UNSUPPORTED, 3);
    return;
  }
  c.bs = static_cast<uint32_t>(v[0]);
  c.mbc = static_cast<uint32_t>(v[1]);
  c.vpm = c.bs / c.mbc;
  c.total = static_cast<uint32_t>(v[2]);
  c.first = static_cast<int32_t>(static_cast<uint32_t>(static_cast<uint64_t>(unzigzag(v[3]))));
  c.hdr_end = q;
  c.end = end;
  uint32_t left = c.total ? c.total - 1 : 0;
  while (left) {
    uint64_t mn;
    const int n = uleb(get, q, end, &mn);
    if (!n || end - (q + n) < c.mbc) {
      tc_fail(sm, DERR_CORRUPT, 4);
      return;
    }
    q += static_cast<uint32_t>(n);
    const uint32_t wpos = q;
    q += c.mbc;
    for (uint32_t m = 0; m < c.mbc && left; ++m) {
      const uint32_t w = ld_u8(b + wpos + m);
      if (w > 32) {
        tc_fail(sm, DERR_CORRUPT, 5);
        return;
      }
      const uint32_t nbytes = c.vpm * w / 8;
      if (end - q < nbytes) {
        tc_fail(sm, DERR_CORRUPT, 6);
        return;
      }
      q += nbytes;
      left -= left < c.vpm ? left : c.vpm;
    }
  }
  c.pos = q;  // stream end, until dstream_rewind
}

__device__ __forceinline__ void dstream_rewind(DCursor& c) {
  c.pos = c.hdr_end;
  c.started = 0;
  c.nbuf = 0;
}

// All threads: decodes the next buffer of values (the header's first value,
// then as many whole blocks as the buffer holds: thread 0 lists their
// miniblocks, every thread decodes TC_PER_THREAD values).  Returns false on
// an error.
__device__ bool dstream_refill(const uint8_t* b, DCursor& c, TcSmem& sm) {
  if (threadIdx.x == 0) {
    c.cnt = 0;
    if (!c.started) {
      c.started = 1;
      c.left = c.total ? c.total - 1 : 0;
      c.nbuf = c.total ? 1 : 0;
      c.buf[0] = c.first;
      c.last = c.first;
    } else if (c.left) {
      auto get = [b](uint32_t i) { return ld_u8(b + i); };
      uint32_t q = c.pos, cnt = 0, nm = 0, left = c.left;
      // whole blocks while they fit (one block always does: bs <= TC_MAX_BLOCK)
      while (left) {
        const uint32_t bc = left < c.bs ? left : c.bs;
        const uint32_t need = (bc + c.vpm - 1) / c.vpm;
        if (cnt + bc > TC_MAX_BLOCK || nm + need > TC_MAX_MB) break;
        uint64_t mn;
        const int n = uleb(get, q, c.end, &mn);
        if (!n || c.end - (q + n) < c.mbc) {
          tc_fail(sm, DERR_CORRUPT, 7);
          break;
        }
        q += static_cast<uint32_t>(n);
        const int64_t minv = unzigzag(mn);
        const uint32_t wpos = q;
        q += c.mbc;
        bool bad = false;
        for (uint32_t m = 0; m < need; ++m) {
          const uint32_t w = ld_u8(b + wpos + m);
          const uint32_t nbytes = c.vpm * w / 8;
          if (w > 32 || c.end - q < nbytes) {
            bad = true;
            break;
          }
          c.width[nm + m] = static_cast<uint8_t>(w);
          c.mboff[nm + m] = q;
          c.minv[nm + m] = minv;
          q += nbytes;
        }
        if (bad) {
          tc_fail(sm, DERR_CORRUPT, 8);
          break;
        }
        nm += need;
        cnt += bc;
        left -= bc;
      }
      c.pos = q;
      c.cnt = cnt;
    } else {
      tc_fail(sm, DERR_CORRUPT, 9);  // more values asked for than the stream holds
    }
  }
  __syncthreads();
  if (sm.err) return false;
  const uint32_t cnt = c.cnt;
  if (cnt) {
    const uint32_t k0 = threadIdx.x * TC_PER_THREAD;
    int64_t d[TC_PER_THREAD];
    int64_t s = 0;
#pragma unroll
    for (int u = 0; u < TC_PER_THREAD; ++u) {
      const uint32_t k = k0 + u;
      if (k < cnt) {
        const uint32_t m = k / c.vpm, i = k % c.vpm;
        const int w = c.width[m];
        s += c.minv[m] + static_cast<int64_t>(get_bits(b, c.mboff[m], i * static_cast<uint32_t>(w), w));
      }
      d[u] = s;
    }
    int64_t tot;
    const int64_t ex = block_exclusive_sum<int64_t>(s, sm.tmp, &tot);
    const int64_t base = static_cast<int64_t>(c.last) + ex;
#pragma unroll
    for (int u = 0; u < TC_PER_THREAD; ++u) {
      const uint32_t k = k0 + u;
      if (k < cnt) c.buf[k] = static_cast<int32_t>(static_cast<uint32_t>(static_cast<uint64_t>(base + d[u])));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      c.last = c.buf[cnt - 1];
      c.nbuf = cnt;
      c.left -= cnt;
    }
    __syncthreads();
  }
  return true;
}

__device__ __forceinline__ void put_le32(uint8_t* p, uint32_t v) {
  p[0] = static_cast<uint8_t>(v);
  p[1] = static_cast<uint8_t>(v >> 8);
  p[2] = static_cast<uint8_t>(v >> 16);
  p[3] = static_cast<uint8_t>(v >> 24);
}

__device__ __forceinline__ void copy_bytes(uint8_t* d, const uint8_t* s, int64_t n) {
  for (int64_t i = 0; i < n; ++i) d[i] = ld_u8(s + i);
}

// DELTA_LENGTH_BYTE_ARRAY values at src[vp, src_len) -> PLAIN at dst + v0.
// Returns the PLAIN bytes written after v0, or -1 on an error.
__device__ int64_t tc_dlba(const TranscodeJob& j, TcSmem& sm, uint32_t v0, uint8_t* dst, uint32_t* vp) {
  DCursor& c = sm.c[0];
  if (threadIdx.x == 0) dstream_open(j.src, v0, j.src_len, c, sm);
  __syncthreads();
  if (sm.err) return -1;
  const uint32_t M = c.total;
  const uint32_t cstart = c.pos;
  if (M > static_cast<uint32_t>(j.num_values) || (j.required && M != static_cast<uint32_t>(j.num_values))) {
    if (threadIdx.x == 0) tc_fail(sm, DERR_CORRUPT, 20);
    return -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) dstream_rewind(c);
  __syncthreads();
  const int64_t room = static_cast<int64_t>(j.src_len) - cstart;
  const int t = threadIdx.x;
  int64_t K = 0, C = 0;
  uint32_t used = 0, nbuf = 0;
  while (K < M) {
    if (used == nbuf) {
      if (!dstream_refill(j.src, c, sm)) return -1;
      nbuf = c.nbuf;
      used = 0;
    }
    const uint32_t n = min(nbuf - used, static_cast<uint32_t>(TC_THREADS));
    const bool on = t < static_cast<int>(n);
    const int64_t len = on ? c.buf[used + t] : 0;
    if (len < 0) tc_fail(sm, DERR_CORRUPT, 21);
    int64_t tot;
    const int64_t ex = block_exclusive_sum<int64_t>(len, sm.tmp, &tot);
    if (sm.err) return -1;
    if (C + tot > room) {
      if (t == 0) tc_fail(sm, DERR_CORRUPT, 22);
      return -1;
    }
    if (on) {
      uint8_t* out = dst + v0 + 4 * (K + t) + C + ex;
      put_le32(out, static_cast<uint32_t>(len));
      copy_bytes(out + 4, j.src + cstart + C + ex, len);
      if (vp) vp[K + t] = static_cast<uint32_t>(4 * (K + t) + C + ex);
    }
    K += n;
    C += tot;
    used += n;
    __syncthreads();
  }
  if (vp && threadIdx.x == 0) vp[M] = static_cast<uint32_t>(4 * static_cast<int64_t>(M) + C);
  return 4 * static_cast<int64_t>(M) + C;
}

// One lockstep pass over the prefix and suffix-length streams of a
// DELTA_BYTE_ARRAY page.  emit false: checks and totals only (*T = value
// bytes, *S = suffix bytes); emit true: writes the PLAIN values at dst + v0.
__device__ bool dba_pass(const TranscodeJob& j, TcSmem& sm, uint32_t v0, uint32_t cstart, bool emit, uint8_t* dst,
                         uint32_t* vp, int64_t* T_out, int64_t* S_out) {
  DCursor& cp = sm.c[0];
  DCursor& cs = sm.c[1];
  if (threadIdx.x == 0) {
    dstream_rewind(cp);
    dstream_rewind(cs);
  }
  __syncthreads();
  const uint32_t M = cp.total;
  const int64_t room = static_cast<int64_t>(j.src_len) - cstart;
  const int t = threadIdx.x;
  int64_t K = 0, T = 0, S = 0, prevL = 0, prevD = 0;
  uint32_t up = 0, np = 0, us = 0, ns = 0;
  while (K < M) {
    if (up == np) {
      if (!dstream_refill(j.src, cp, sm)) return false;
      np = cp.nbuf;
      up = 0;
    }
    if (us == ns) {
      if (!dstream_refill(j.src, cs, sm)) return false;
      ns = cs.nbuf;
      us = 0;
    }
    const uint32_t n = min(min(np - up, ns - us), static_cast<uint32_t>(TC_THREADS));
    const bool on = t < static_cast<int>(n);
    const int64_t p = on ? cp.buf[up + t] : 0;
    const int64_t s = on ? cs.buf[us + t] : 0;
    const int64_t L = p + s;
    if (p < 0 || s < 0) tc_fail(sm, DERR_CORRUPT, 30);
    if (on) {
      sm.lb[t] = L;
      sm.pb[t] = static_cast<int32_t>(p);
    }
    __syncthreads();
    // a prefix may not be longer than the value before it (none before value 0)
    if (on && p > (t ? sm.lb[t - 1] : prevL)) tc_fail(sm, DERR_CORRUPT, 31);
    int64_t totL, totS;
    const int64_t exL = block_exclusive_sum<int64_t>(L, sm.tmp, &totL);
    const int64_t exS = block_exclusive_sum<int64_t>(s, sm.tmp, &totS);
    if (sm.err) return false;
    if (S + totS > room) {
      if (t == 0) tc_fail(sm, DERR_CORRUPT, 32);
      return false;
    }
    if (emit) {
      const int64_t dch = static_cast<int64_t>(v0) + 4 * (K + t + 1) + T + exL;  // chars of value t
      const int64_t soff = static_cast<int64_t>(cstart) + S + exS;            // its suffix in src
      if (on) {
        put_le32(dst + dch - 4, static_cast<uint32_t>(L));
        copy_bytes(dst + dch + p, j.src + soff, s);
        sm.db[t] = dch;
        sm.sb[t] = soff;
        if (vp) vp[K + t] = static_cast<uint32_t>(dch - 4 - v0);
      }
      __syncthreads();
      if (on) {
        // bytes below p: from the suffix of the nearest earlier value whose
        // prefix is shorter, then from the previous batch's last value
        int64_t cur = p;
        for (int i = t - 1; i >= 0 && cur > 0; --i) {
          const int64_t pi = sm.pb[i];
          if (pi < cur) {
            copy_bytes(dst + dch + pi, j.src + sm.sb[i], cur - pi);
            cur = pi;
          }
        }
        for (int64_t y = 0; y < cur; ++y) dst[dch + y] = dst[prevD + y];
      }
      prevD = sm.db[n - 1];
    }
    prevL = sm.lb[n - 1];
    K += n;
    T += totL;
    S += totS;
    up += n;
    us += n;
    __syncthreads();
  }
  if (emit && vp && threadIdx.x == 0) vp[M] = static_cast<uint32_t>(4 * static_cast<int64_t>(M) + T);
  *T_out = T;
  *S_out = S;
  return true;
}

// DELTA_BYTE_ARRAY values at src[v0, src_len) -> PLAIN in a piece of the
// pool sized by a first pass.  Returns the PLAIN bytes after v0 (sm.dst_off
// holds the piece), or -1 on an error.
__device__ int64_t tc_dba(const TranscodeJob& j, TcSmem& sm, uint32_t v0, uint8_t* pool, uint64_t pool_cap,
                          unsigned long long* pool_used, uint32_t* vp) {
  if (threadIdx.x == 0) {
    dstream_open(j.src, v0, j.src_len, sm.c[0], sm);
    if (!sm.err) dstream_open(j.src, sm.c[0].pos, j.src_len, sm.c[1], sm);
  }
  __syncthreads();
  if (sm.err) return -1;
  const uint32_t M = sm.c[0].total;
  const uint32_t cstart = sm.c[1].pos;
  if (sm.c[1].total != M || M > static_cast<uint32_t>(j.num_values) ||
      (j.required && M != static_cast<uint32_t>(j.num_values))) {
    if (threadIdx.x == 0) tc_fail(sm, DERR_CORRUPT, 33);
    return -1;
  }
  __syncthreads();
  int64_t T, S;
  if (!dba_pass(j, sm, v0, cstart, false, nullptr, nullptr, &T, &S)) return -1;
  const int64_t vlen = 4 * static_cast<int64_t>(M) + T;
  if (threadIdx.x == 0) {
    const uint64_t need = (static_cast<uint64_t>(v0) + static_cast<uint64_t>(vlen) + 32 + 15) & ~uint64_t(15);
    if (static_cast<uint64_t>(v0) + static_cast<uint64_t>(vlen) > 0x7fffffffull) {
      tc_fail(sm, DERR_UNSUPPORTED, 34);
    } else if (need > pool_cap) {
      tc_fail(sm, DERR_CAPACITY, 35);
    } else {
      const unsigned long long off = atomicAdd(pool_used, static_cast<unsigned long long>(need));
      if (off + need > pool_cap) tc_fail(sm, DERR_CAPACITY, 36);
      else sm.dst_off = off;
    }
  }
  __syncthreads();
  if (sm.err) return -1;
  uint8_t* dst = pool + sm.dst_off;
  if (!dba_pass(j, sm, v0, cstart, true, dst, vp, &T, &S)) return -1;
  return vlen;
}

// BYTE_STREAM_SPLIT values at src[v0, src_len) -> PLAIN at dst + v0 (a byte
// transpose; every whole value of the streams is written).
__device__ int64_t tc_bss(const TranscodeJob& j, TcSmem& sm, uint32_t v0, uint8_t* dst) {
  const uint32_t R = j.src_len - v0, w = static_cast<uint32_t>(j.width);
  if (w == 0 || R % w) {
    if (threadIdx.x == 0) tc_fail(sm, DERR_CORRUPT, 40);
    return -1;
  }
  const uint32_t N = R / w;
  const uint8_t* s = j.src + v0;
  uint8_t* d = dst + v0;
  for (uint32_t k = threadIdx.x; k < N; k += blockDim.x) {
    uint64_t v = 0;
    for (uint32_t b = 0; b < w; ++b) v |= static_cast<uint64_t>(ld_u8(s + static_cast<uint64_t>(b) * N + k)) << (8 * b);
    uint8_t* o = d + static_cast<uint64_t>(k) * w;
    for (uint32_t b = 0; b < w; ++b) o[b] = static_cast<uint8_t>(v >> (8 * b));
  }
  return R;
}

__global__ void __launch_bounds__(TC_THREADS) k_transcode(const TranscodeJob* jobs, PlanPage* pps, uint8_t* pool,
                                                         uint64_t pool_cap, unsigned long long* pool_used,
                                                         uint32_t* vpos, DevStatus* st) {
  __shared__ TcSmem sm;
  const TranscodeJob j = jobs[blockIdx.x];
  // string pages: the value-position table the walk reads instead of
  // following the (length, bytes) chain
  const uint32_t vtab = pps[j.pp].vtab;
  uint32_t* vp = vtab && vpos ? vpos + (vtab - 1) : nullptr;
  {
    // the page's bytes into L2 first (a hint): the stream headers are then
    // followed by one thread at L2 rather than DRAM latency
    const uintptr_t e = reinterpret_cast<uintptr_t>(j.src) + j.src_len;
    for (uintptr_t q = (reinterpret_cast<uintptr_t>(j.src) & ~uintptr_t(127)) + 128u * threadIdx.x; q < e;
         q += 128u * blockDim.x)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
  }
  if (threadIdx.x == 0) {
    sm.err = 0;
    sm.flag = 0;
    sm.detail = 0;
    sm.dst_off = 0;
    sm.c[0].started = sm.c[1].started = 0;
    uint32_t v0 = 0;
    if (j.levels < 0) {
      const uint32_t L = j.src_len >= 4 ? ld_le32_g(j.src) : 0xffffffffu;
      if (j.src_len < 4 || L > j.src_len - 4) tc_fail(sm, DERR_CORRUPT, 10);
      else v0 = 4 + L;
    } else if (static_cast<uint32_t>(j.levels) > j.src_len) {
      tc_fail(sm, DERR_CORRUPT, 11);
    } else {
      v0 = static_cast<uint32_t>(j.levels);
    }
    sm.v0 = v0;
  }
  __syncthreads();
  const uint32_t v0 = sm.v0;
  int64_t vlen = -1;
  uint8_t* dst = j.dst;
  if (!sm.err) {
    if (j.enc == ENC_BSS) {
      vlen = tc_bss(j, sm, v0, dst);
    } else if (j.enc == ENC_DELTA_LBA) {
      vlen = tc_dlba(j, sm, v0, dst, vp);
    } else if (j.enc == ENC_DELTA_BA) {
      vlen = tc_dba(j, sm, v0, pool, pool_cap, pool_used, vp);
      dst = pool + sm.dst_off;
    } else if (threadIdx.x == 0) {
      tc_fail(sm, DERR_UNSUPPORTED, 12);
    }
  }
  __syncthreads();
  if (vlen >= 0 && !sm.err)
    for (uint32_t i = threadIdx.x; i < v0; i += blockDim.x) dst[i] = ld_u8(j.src + i);
  if (threadIdx.x == 0) {
    PlanPage* pp = pps + j.pp;
    if (vlen >= 0 && !sm.err) {
      pp->body = dst;
      pp->body_len = static_cast<int32_t>(v0 + vlen);
    } else {
      // the page keeps its level bytes only: later stages find no values
      // (and the walk does not read the value-position table, which this
      // page never filled)
      pp->body = j.src;
      pp->body_len = static_cast<int32_t>(v0);
      pp->vtab = 0;
      report(st, static_cast<uint32_t>(sm.flag), j.page, WHERE_TRANSCODE, sm.detail);
    }
  }
}

}  // namespace

void launch_transcode(const TranscodeJob* jobs, int n, PlanPage* pps, uint8_t* pool, uint64_t pool_cap,
                      uint32_t* counters, uint32_t* vpos, DevStatus* st, cudaStream_t s) {
  if (n <= 0) return;
  k_transcode<<<n, TC_THREADS, 0, s>>>(jobs, pps, pool, pool_cap,
                                       reinterpret_cast<unsigned long long*>(counters + TC_POOL_COUNTER), vpos, st);
}

}  // namespace pqi
