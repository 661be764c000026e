// K2-K8 — dictionary decode, page walk, tiled expansion, string passes and
// the plain one-page-per-block baseline.
//
// What a page holds (paper Section 2; byte layouts from the Parquet format):
//   V1 data page: [4-byte LE length + RLE/bit-packed def levels]? values
//   V2 data page: [rep levels][def levels] values (level lengths in header)
//   values: PLAIN (fixed width LE, or 4-byte length + bytes), dictionary
//   indices (1-byte bit width + RLE/bit-packed hybrid), or
//   DELTA_BINARY_PACKED (header, then blocks of miniblocks).
//
// The scan runs in two phases so that pages larger than a thread block's
// share of the GPU still use the whole GPU (paper Section 3, Insight 1):
//
//  walk   (one block per page): reads each stream's run / block headers —
//         serial by construction — through a shared-memory window filled by
//         the bulk-copy engine, writes the validity bitmap, and records for
//         every ITEM_ROWS-row work item the stream position it starts from
//         (a checkpoint).  DELTA blocks are summed in parallel so that each
//         checkpoint carries the value preceding its block.
//  expand (persistent blocks, one work item at a time): starts from the
//         checkpoint, decodes TILE_ROWS rows at a time into shared memory
//         (dictionary gather, delta prefix sums via warp shuffles, PLAIN
//         loads) and writes each output row once, nulls as zero.
//
// Strings add a pass: expand records per row the dictionary index (or the
// PLAIN value offset) plus per-item chars totals; a scan turns those into
// item bases, and the copy pass writes int64 offsets and the chars.
#include "decode_job.h"
#include "dev_util.cuh"

namespace pqi {

constexpr int WALK_THREADS = 128;
constexpr int EXP_THREADS = 256;
constexpr uint32_t WIN_BYTES = 16384;
constexpr int LV_BATCH = 128;
constexpr int BLK_BATCH = 128;
constexpr int SEG_MAX = 256;
constexpr int DB_MAX = 24;
constexpr uint32_t NULL_IDX = 0xffffffffu;

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
    uint32_t lo = __ldg(src + i);
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

struct DictStrSmem {
  uint64_t bar;
  uint32_t ctl[4];
  alignas(16) uint8_t win[WIN_BYTES + 16];
};

// BYTE_ARRAY dictionary: the entries are (4-byte length, bytes) back to back;
// the walk over them is serial, done by thread 0 in a staged window.
__global__ void __launch_bounds__(128) k_dict_str(const DictJob* __restrict__ jobs, DictDev* dicts,
                                                  DevStatus* st) {
  __shared__ DictStrSmem sm;
  const DictJob j = jobs[blockIdx.x];
  if (j.ptype != T_BYTE_ARRAY) return;
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  Win win{sm.win, nullptr, WIN_BYTES, 0, &sm.bar, 0};
  const uint8_t* body = j.body;
  const uint32_t blen = static_cast<uint32_t>(j.body_len);
  uint32_t pos = 0, k = 0, maxlen = 0;
  bool bad = false;
  if (!win_load(win, body, body + blen, st, j.page, WHERE_DICT)) return;
  for (uint32_t guard = 0; guard <= blen + 1; ++guard) {
    if (threadIdx.x == 0) {
      uint32_t reload = 0;
      while (k < static_cast<uint32_t>(j.n)) {
        uint32_t wrel = static_cast<uint32_t>((body + pos) - win.g0);
        if (pos + 4 > blen) { bad = true; break; }
        if (wrel + 4 > win.n) { reload = 1; break; }
        const uint8_t* q = win.s + wrel;
        uint32_t len = q[0] | (q[1] << 8) | (q[2] << 16) | (static_cast<uint32_t>(q[3]) << 24);
        if (len > blen - pos - 4) { bad = true; break; }
        j.str_pos[k] = pos + 4;
        j.str_len[k] = len;
        maxlen = len > maxlen ? len : maxlen;
        pos += 4 + len;
        ++k;
      }
      sm.ctl[0] = reload;
      sm.ctl[1] = bad ? 1u : 0u;
      sm.ctl[2] = pos;
    }
    __syncthreads();
    uint32_t reload = sm.ctl[0];
    if (sm.ctl[1]) break;
    if (!reload) break;
    if (!win_load(win, body + sm.ctl[2], body + blen, st, j.page, WHERE_DICT)) return;
  }
  if (threadIdx.x == 0) {
    if (bad || k != static_cast<uint32_t>(j.n)) {
      report(st, DERR_CORRUPT, j.page, WHERE_DICT, 2);
      return;
    }
    DictDev d{};
    d.str_pos = j.str_pos;
    d.str_len = j.str_len;
    d.chars = body;
    d.n = j.n;
    d.max_len = static_cast<int32_t>(maxlen);
    d.valid = 1;
    dicts[j.chunk] = d;
  }
}

void launch_dict(const DictJob* jobs, int n_jobs, int max_fixed_bytes, DictDev* dicts, int n_sms, DevStatus* st,
                 cudaStream_t s) {
  if (n_jobs <= 0) return;
  int gx = (max_fixed_bytes / 4 + 256 * 16 - 1) / (256 * 16);
  if (gx < 1) gx = 1;
  if (gx > 4 * n_sms) gx = 4 * n_sms;
  k_dict_fixed<<<dim3(gx, n_jobs), 256, 0, s>>>(jobs, dicts, st);
  k_dict_str<<<n_jobs, 128, 0, s>>>(jobs, dicts, st);
}

// ------------------------------------------------------------------ shared layouts

struct WalkSmem {
  uint64_t bar;
  int32_t ctl[16];
  int64_t c64[8];
  // level runs of one batch
  int32_t lrow[LV_BATCH];
  int32_t lcnt[LV_BATCH];
  uint32_t lmeta[LV_BATCH];  // bit 31 set: bit-packed, low bits = window bit position; else value
  int32_t lpre[LV_BATCH];
  // delta blocks of one batch
  uint32_t bstart[BLK_BATCH];  // stream offset of the block
  uint32_t bdata[BLK_BATCH];   // window offset of the first miniblock
  uint32_t bwid[BLK_BATCH];    // window offset of the width bytes
  int32_t bcnt[BLK_BATCH];     // values in the block
  int32_t bk[BLK_BATCH];       // dense index of the block's first value
  int64_t bmin[BLK_BATCH];
  uint64_t bsum[BLK_BATCH];
  int32_t tmp32[32];
  alignas(16) uint8_t win[WIN_BYTES + 16];
};

struct ExpSmem {
  uint64_t bar;
  int32_t ctl[16];
  int64_t c64[8];
  uint32_t wbits[TILE_ROWS / 32];
  uint32_t wpre[TILE_ROWS / 32];
  int32_t sdst[SEG_MAX];
  int32_t scnt[SEG_MAX];
  uint32_t smeta[SEG_MAX];
  uint32_t sval[SEG_MAX];
  uint32_t dstart[DB_MAX];
  uint32_t ddata[DB_MAX];
  uint32_t dwid[DB_MAX];
  int32_t dk[DB_MAX];
  int32_t dcnt[DB_MAX];
  int32_t dnext[DB_MAX];
  int64_t dmin[DB_MAX];
  uint64_t dsum[DB_MAX];
  uint64_t dbase[DB_MAX];
  uint32_t tmp32[32];
  uint64_t tmp64[32];
  alignas(16) uint64_t vbuf[TILE_ROWS];
  alignas(16) uint8_t win[WIN_BYTES + 16];
};

// Page layout resolved by the walk and reused by the expansion.
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

// ------------------------------------------------------------------ walk: levels

// k at row R of this batch: valid rows before R (R inside run j).
__device__ __forceinline__ int32_t level_k_at(const WalkSmem& sm, const uint32_t* w32, int nb, int32_t R) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sm.lrow[mid] <= R) lo = mid; else hi = mid - 1;
  }
  int32_t off = R - sm.lrow[lo];
  int32_t part;
  uint32_t meta = sm.lmeta[lo];
  if (meta & 0x80000000u) {
    uint32_t bp = meta & 0x7fffffffu;
    part = 0;
    for (int32_t x = 0; x < off; x += 32) {
      int n = off - x < 32 ? off - x : 32;
      part += __popc(bits32(w32, bp + x, n));
    }
  } else {
    part = static_cast<int32_t>(meta) * off;
  }
  return sm.lpre[lo] + part;
}

// Walks the definition levels [lv0, lv1) of a page: writes the validity
// bits of rows [row_lo, row_hi) and the dense start (k0) / count (nn) of
// every item.  Returns the page's non-null count (-1 on error).
__device__ int32_t walk_levels(WalkSmem& sm, Win& win, const PageCtx& pc, const PlanPage& pp, Item* items,
                               const OutCol& col, DevStatus* st) {
  const int tid = threadIdx.x;
  const uint8_t* sb = pc.body + pc.lv0;
  const uint32_t slen = pc.lv1 - pc.lv0;
  if (!win_load(win, sb, sb + slen, st, pc.pgid, WHERE_WALK_LEVELS)) return -1;
  if (tid == 0) {
    sm.ctl[0] = 0;  // stream position
    sm.ctl[1] = 0;  // rows consumed
    sm.ctl[5] = 0;  // error
    sm.c64[0] = 0;  // valid rows before the batch
    sm.c64[1] = -1; // k at row_hi when found inside the walk
  }
  __syncthreads();
  const uint32_t* w32 = reinterpret_cast<const uint32_t*>(win.s);
  for (uint32_t guard = 0; guard <= slen + 2; ++guard) {
    if (tid == 0) {
      uint32_t hp = static_cast<uint32_t>(sm.ctl[0]);
      int32_t row = sm.ctl[1];
      int nb = 0, reload = 0, err = 0;
      while (nb < LV_BATCH && row < pc.nrows) {
        if (hp >= slen) { err = 1; break; }
        uint32_t wrel = static_cast<uint32_t>((sb + hp) - win.g0);
        uint32_t lim_w = win.n, lim_s = wrel + (slen - hp);
        uint32_t lim = lim_w < lim_s ? lim_w : lim_s;
        uint64_t h = 0;
        int hl = uleb([&](uint32_t q) { return static_cast<uint32_t>(win.s[q]); }, wrel, lim, &h);
        if (hl == 0) {
          if (lim == lim_s) err = 1; else reload = 1;
          break;
        }
        int32_t take;
        if (h & 1) {
          uint64_t g = h >> 1;
          if (g > slen) { err = 1; break; }
          uint32_t nbody = static_cast<uint32_t>(g);  // bit width 1: one byte per group
          if (hp + hl + nbody > slen) { err = 1; break; }
          if (wrel + hl + nbody > win.n) {
            if (wrel == 0) err = 2; else reload = 1;
            break;
          }
          uint64_t c = g * 8;
          take = static_cast<int32_t>(c < static_cast<uint64_t>(pc.nrows - row) ? c : (pc.nrows - row));
          sm.lrow[nb] = row;
          sm.lcnt[nb] = take;
          sm.lmeta[nb] = 0x80000000u | ((wrel + hl) * 8);
          hp += hl + nbody;
        } else {
          if (wrel + hl + 1 > win.n) {
            if (hp + hl + 1 > slen) err = 1; else reload = 1;
            break;
          }
          if (hp + hl + 1 > slen) { err = 1; break; }
          uint32_t v = win.s[wrel + hl];
          if (v > 1) { err = 1; break; }
          uint64_t c = h >> 1;
          take = static_cast<int32_t>(c < static_cast<uint64_t>(pc.nrows - row) ? c : (pc.nrows - row));
          sm.lrow[nb] = row;
          sm.lcnt[nb] = take;
          sm.lmeta[nb] = v;
          hp += hl + 1;
        }
        if (take > 0) {
          row += take;
          ++nb;
        }
      }
      sm.ctl[0] = static_cast<int32_t>(hp);
      sm.ctl[2] = nb;
      sm.ctl[3] = reload;
      sm.ctl[4] = row;
      sm.ctl[5] = err;
    }
    __syncthreads();
    const int nb = sm.ctl[2];
    const int err = sm.ctl[5];
    if (err) {
      if (tid == 0) report(st, err == 2 ? DERR_UNSUPPORTED : DERR_CORRUPT, pc.pgid, WHERE_WALK_LEVELS, err);
      return -1;
    }
    const int32_t b0 = sm.ctl[1];
    const int32_t b1 = sm.ctl[4];
    // (1) valid count per run, prefix over the batch
    int32_t cnt = 0;
    if (tid < nb) {
      uint32_t meta = sm.lmeta[tid];
      if (meta & 0x80000000u) {
        uint32_t bp = meta & 0x7fffffffu;
        for (int32_t x = 0; x < sm.lcnt[tid]; x += 32) {
          int n = sm.lcnt[tid] - x < 32 ? sm.lcnt[tid] - x : 32;
          cnt += __popc(bits32(w32, bp + x, n));
        }
      } else {
        cnt = static_cast<int32_t>(meta) * sm.lcnt[tid];
      }
    }
    int32_t total;
    int32_t pre = block_exclusive_sum(cnt, sm.tmp32, &total);
    const int64_t vb = sm.c64[0];
    if (tid < nb) sm.lpre[tid] = static_cast<int32_t>(vb) + pre;
    __syncthreads();
    // (2) bitmap words of rows [max(b0,row_lo), min(b1,row_hi))
    if (nb > 0 && col.validity) {
      int32_t r_lo = b0 > pp.row_lo ? b0 : pp.row_lo;
      int32_t r_hi = b1 < pp.row_hi ? b1 : pp.row_hi;
      if (r_lo < r_hi) {
        int64_t o0 = pp.out_row + r_lo, o1 = pp.out_row + r_hi;
        int64_t w0 = o0 >> 5, w1 = (o1 - 1) >> 5;
        for (int64_t w = w0 + tid; w <= w1; w += blockDim.x) {
          int64_t a = w * 32 > o0 ? w * 32 : o0;
          int64_t e = w * 32 + 32 < o1 ? w * 32 + 32 : o1;
          uint32_t word = 0;
          int32_t r = static_cast<int32_t>(a - pp.out_row);
          const int32_t rend = static_cast<int32_t>(e - pp.out_row);
          // run containing r
          int lo = 0, hi = nb - 1;
          while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sm.lrow[mid] <= r) lo = mid; else hi = mid - 1;
          }
          for (int j = lo; j < nb && r < rend; ++j) {
            int32_t s0 = r, s1 = sm.lrow[j] + sm.lcnt[j];
            if (s1 > rend) s1 = rend;
            if (s1 <= s0) continue;
            int n = s1 - s0;
            uint32_t meta = sm.lmeta[j];
            uint32_t bitsv;
            if (meta & 0x80000000u)
              bitsv = bits32(w32, (meta & 0x7fffffffu) + (s0 - sm.lrow[j]), n);
            else
              bitsv = meta ? (n == 32 ? 0xffffffffu : ((1u << n) - 1)) : 0u;
            word |= bitsv << static_cast<uint32_t>((pp.out_row + s0) - w * 32);
            r = s1;
          }
          if (a == w * 32 && e == w * 32 + 32)
            col.validity[w] = word;
          else if (word)
            atomicOr(col.validity + w, word);
        }
      }
    }
    // (3) item starts inside this batch
    for (uint32_t i = tid; i <= pp.item_count; i += blockDim.x) {
      int32_t R = i < pp.item_count ? pp.row_lo + static_cast<int32_t>(i) * ITEM_ROWS : pp.row_hi;
      if (nb > 0 && R >= b0 && R < b1) {
        int32_t kR = level_k_at(sm, w32, nb, R);
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
    }
    const int reload = sm.ctl[3];
    const bool done = b1 >= pc.nrows;
    __syncthreads();
    if (done) break;
    if (reload) {
      if (!win_load(win, sb + sm.ctl[0], sb + slen, st, pc.pgid, WHERE_WALK_LEVELS)) return -1;
    } else if (nb == 0) {
      if (tid == 0) report(st, DERR_CORRUPT, pc.pgid, WHERE_WALK_LEVELS, 9);
      return -1;
    }
  }
  __syncthreads();
  const int32_t nonnull = static_cast<int32_t>(sm.c64[0]);
  const int64_t k_hi = sm.c64[1] >= 0 ? sm.c64[1] : nonnull;
  __syncthreads();
  // item counts: nn_i = k_{i+1} - k_i
  for (uint32_t i = tid; i < pp.item_count; i += blockDim.x) {
    int32_t ka = items[pp.item_begin + i].k0;
    int32_t kb = i + 1 < pp.item_count ? items[pp.item_begin + i + 1].k0 : static_cast<int32_t>(k_hi);
    items[pp.item_begin + i].nn = kb - ka;
  }
  __syncthreads();
  return nonnull;
}

// ------------------------------------------------------------------ walk: value streams

// Dictionary indices: records (run header offset, dense index at run start)
// for each item start.
__device__ bool walk_hybrid(WalkSmem& sm, Win& win, const uint8_t* sb, uint32_t slen, int bw, int32_t total,
                            const PlanPage& pp, Item* items, int pgid, DevStatus* st) {
  const int tid = threadIdx.x;
  if (!win_load(win, sb, sb + slen, st, pgid, WHERE_WALK_VALUES)) return false;
  if (tid == 0) {
    sm.ctl[0] = 0;  // header position
    sm.ctl[1] = 0;  // dense index at that header
    sm.ctl[2] = 0;  // next item
  }
  __syncthreads();
  const uint32_t vbytes = (bw + 7) / 8;
  for (uint32_t guard = 0; guard <= slen + 2; ++guard) {
    if (tid == 0) {
      uint32_t hp = static_cast<uint32_t>(sm.ctl[0]);
      int32_t kk = sm.ctl[1];
      uint32_t ni = static_cast<uint32_t>(sm.ctl[2]);
      int reload = 0, err = 0, done = 0;
      for (;;) {
        while (ni < pp.item_count && items[pp.item_begin + ni].nn == 0) ++ni;
        if (ni >= pp.item_count) { done = 1; break; }
        if (kk >= total || hp >= slen) { err = 1; break; }
        uint32_t wrel = static_cast<uint32_t>((sb + hp) - win.g0);
        uint32_t lim_w = win.n, lim_s = wrel + (slen - hp);
        uint32_t lim = lim_w < lim_s ? lim_w : lim_s;
        uint64_t h = 0;
        int hl = uleb([&](uint32_t q) { return static_cast<uint32_t>(win.s[q]); }, wrel, lim, &h);
        if (hl == 0) {
          if (lim == lim_s) err = 1; else reload = 1;
          break;
        }
        uint64_t c, body;
        if (h & 1) {
          c = (h >> 1) * 8;
          body = (h >> 1) * static_cast<uint64_t>(bw);
        } else {
          c = h >> 1;
          body = vbytes;
        }
        if (hp + hl + body > slen) { err = 1; break; }
        int64_t end = static_cast<int64_t>(kk) + static_cast<int64_t>(c);
        while (ni < pp.item_count) {
          Item& it = items[pp.item_begin + ni];
          if (it.nn == 0) { ++ni; continue; }
          if (it.k0 < end) {
            it.pos = static_cast<int32_t>(hp);
            it.run_k0 = kk;
            it.base = 0;
            ++ni;
          } else {
            break;
          }
        }
        hp += hl + static_cast<uint32_t>(body);
        kk = end > total ? total : static_cast<int32_t>(end);
      }
      sm.ctl[0] = static_cast<int32_t>(hp);
      sm.ctl[1] = kk;
      sm.ctl[2] = static_cast<int32_t>(ni);
      sm.ctl[3] = reload;
      sm.ctl[4] = err;
      sm.ctl[5] = done;
    }
    __syncthreads();
    if (sm.ctl[4]) {
      if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 1);
      return false;
    }
    if (sm.ctl[5]) return true;
    if (!win_load(win, sb + sm.ctl[0], sb + slen, st, pgid, WHERE_WALK_VALUES)) return false;
  }
  if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 2);
  return false;
}

struct DeltaHdr {
  int32_t block, mbc, vpm, total, hlen;
  int64_t first;
};

// Parses the DELTA_BINARY_PACKED header from global memory.
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
  if (a == 0 || a % 128 || a > 4096 || b == 0 || b > 64 || a % b || (a / b) % 32 || c > 0x7fffffff) return false;
  d->block = static_cast<int32_t>(a);
  d->mbc = static_cast<int32_t>(b);
  d->vpm = static_cast<int32_t>(a / b);
  d->total = static_cast<int32_t>(c);
  d->first = unzigzag(f);
  d->hlen = static_cast<int32_t>(p);
  return true;
}

// Parses one block header at window offset `wrel`: fills min delta, width
// offset and data offset; returns the block's byte size (header included)
// or 0 when it does not fit in [wrel, lim) (*need_more set) or is malformed.
__device__ __forceinline__ uint32_t delta_block(const Win& win, uint32_t wrel, uint32_t lim, const DeltaHdr& d,
                                                int32_t nvals, int type_bits, int64_t* mn, uint32_t* wpos,
                                                uint32_t* dpos, int* need_more, int* bad) {
  uint64_t z = 0;
  int hl = uleb([&](uint32_t q) { return static_cast<uint32_t>(win.s[q]); }, wrel, lim, &z);
  if (hl == 0) {
    *need_more = 1;
    return 0;
  }
  if (wrel + hl + d.mbc > lim) {
    *need_more = 1;
    return 0;
  }
  *mn = unzigzag(z);
  *wpos = wrel + hl;
  uint64_t bits = 0;
  const int used = (nvals + d.vpm - 1) / d.vpm;  // miniblocks holding values
  for (int m = 0; m < used; ++m) {
    uint32_t w = win.s[wrel + hl + m];
    if (static_cast<int>(w) > type_bits) {
      *bad = 1;
      return 0;
    }
    bits += static_cast<uint64_t>(w) * d.vpm;
  }
  uint32_t size = static_cast<uint32_t>(hl + d.mbc + bits / 8);
  *dpos = wrel + hl + d.mbc;
  if (wrel + size > lim) {
    *need_more = 1;
    return 0;
  }
  return size;
}

// Value v of a DELTA block (packed delta, min not added).
__device__ __forceinline__ uint64_t delta_packed(const Win& win, uint32_t wpos, uint32_t dpos, int vpm, int v) {
  const uint32_t* w32 = reinterpret_cast<const uint32_t*>(win.s);
  int m = v / vpm;
  uint64_t bit = static_cast<uint64_t>(dpos) * 8;
  for (int q = 0; q < m; ++q) bit += static_cast<uint64_t>(win.s[wpos + q]) * vpm;
  int w = win.s[wpos + m];
  return bits64(w32, bit + static_cast<uint64_t>(v - m * vpm) * w, w);
}

// DELTA: walks blocks, sums them in parallel, and records for each item the
// block containing its first value plus the value preceding that block.
__device__ bool walk_delta(WalkSmem& sm, Win& win, const uint8_t* sb, uint32_t slen, int type_bits,
                           int32_t total, const PlanPage& pp, Item* items, int pgid, DevStatus* st) {
  const int tid = threadIdx.x;
  DeltaHdr d;
  bool ok = delta_header(sb, slen, &d);
  if (!ok || d.total != total) {
    if (tid == 0) report(st, ok ? DERR_CORRUPT : DERR_UNSUPPORTED, pgid, WHERE_WALK_VALUES, 3);
    return false;
  }
  if (total == 0) return true;
  if (!win_load(win, sb + d.hlen, sb + slen, st, pgid, WHERE_WALK_VALUES)) return false;
  if (tid == 0) {
    sm.ctl[0] = d.hlen;  // block position
    sm.ctl[1] = 1;       // dense index of the block's first value
    sm.ctl[2] = 0;       // next item
    sm.c64[0] = d.first; // value preceding the block
    // items starting at the first value
    uint32_t ni = 0;
    while (ni < pp.item_count) {
      Item& it = items[pp.item_begin + ni];
      if (it.nn != 0 && it.k0 > 0) break;
      if (it.nn != 0) {
        it.pos = d.hlen;
        it.run_k0 = 1;
        it.base = d.first;
      }
      ++ni;
    }
    sm.ctl[2] = static_cast<int32_t>(ni);
  }
  __syncthreads();
  for (uint32_t guard = 0; guard <= slen + 2; ++guard) {
    if (tid == 0) {
      uint32_t bp = static_cast<uint32_t>(sm.ctl[0]);
      int32_t kk = sm.ctl[1];
      int nb = 0, reload = 0, bad = 0;
      while (nb < BLK_BATCH && kk < total) {
        if (bp >= slen) { bad = 1; break; }
        uint32_t wrel = static_cast<uint32_t>((sb + bp) - win.g0);
        uint32_t lim_w = win.n, lim_s = wrel + (slen - bp);
        uint32_t lim = lim_w < lim_s ? lim_w : lim_s;
        int32_t nvals = total - kk < d.block ? total - kk : d.block;
        int64_t mn;
        uint32_t wpos, dpos;
        int more = 0;
        uint32_t size = delta_block(win, wrel, lim, d, nvals, type_bits, &mn, &wpos, &dpos, &more, &bad);
        if (bad) break;
        if (size == 0) {
          if (lim == lim_s) bad = 1; else if (wrel == 0) bad = 2; else reload = 1;
          break;
        }
        sm.bstart[nb] = bp;
        sm.bdata[nb] = dpos;
        sm.bwid[nb] = wpos;
        sm.bcnt[nb] = nvals;
        sm.bk[nb] = kk;
        sm.bmin[nb] = mn;
        ++nb;
        bp += size;
        kk += nvals;
      }
      sm.ctl[3] = nb;
      sm.ctl[4] = reload;
      sm.ctl[5] = bad;
      sm.ctl[6] = static_cast<int32_t>(bp);
      sm.ctl[7] = kk;
    }
    __syncthreads();
    const int nb = sm.ctl[3];
    if (sm.ctl[5]) {
      if (tid == 0) report(st, sm.ctl[5] == 2 ? DERR_UNSUPPORTED : DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 4);
      return false;
    }
    for (int b = tid; b < nb; b += blockDim.x) {
      uint64_t s = 0;
      for (int v = 0; v < sm.bcnt[b]; ++v) s += delta_packed(win, sm.bwid[b], sm.bdata[b], d.vpm, v);
      sm.bsum[b] = s + static_cast<uint64_t>(sm.bmin[b]) * static_cast<uint64_t>(sm.bcnt[b]);
    }
    __syncthreads();
    if (tid == 0) {
      uint64_t prev = static_cast<uint64_t>(sm.c64[0]);
      uint32_t ni = static_cast<uint32_t>(sm.ctl[2]);
      for (int b = 0; b < nb; ++b) {
        const int32_t end = sm.bk[b] + sm.bcnt[b];
        while (ni < pp.item_count) {
          Item& it = items[pp.item_begin + ni];
          if (it.nn == 0) { ++ni; continue; }
          if (it.k0 < end) {
            it.pos = static_cast<int32_t>(sm.bstart[b]);
            it.run_k0 = sm.bk[b];
            it.base = static_cast<int64_t>(prev);
            ++ni;
          } else {
            break;
          }
        }
        prev += sm.bsum[b];
      }
      sm.c64[0] = static_cast<int64_t>(prev);
      sm.ctl[2] = static_cast<int32_t>(ni);
      sm.ctl[0] = sm.ctl[6];
      sm.ctl[1] = sm.ctl[7];
    }
    __syncthreads();
    if (sm.ctl[1] >= total) return true;
    if (sm.ctl[4]) {
      if (!win_load(win, sb + sm.ctl[0], sb + slen, st, pgid, WHERE_WALK_VALUES)) return false;
    } else if (nb == 0) {
      if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 5);
      return false;
    }
  }
  if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 6);
  return false;
}

// PLAIN BYTE_ARRAY: serial walk over (length, bytes) values; records the
// offset of each item's first value and the chars before it.
__device__ bool walk_plain_ba(const uint8_t* sb, uint32_t slen, int32_t total, const PlanPage& pp, Item* items,
                              int pgid, DevStatus* st) {
  if (threadIdx.x == 0) {
    uint32_t pos = 0;
    int64_t chars = 0;
    uint32_t ni = 0;
    for (int32_t k = 0; k <= total; ++k) {
      while (ni < pp.item_count) {
        Item& it = items[pp.item_begin + ni];
        if (it.nn == 0) { ++ni; continue; }
        if (it.k0 == k) {
          it.pos = static_cast<int32_t>(pos);
          it.run_k0 = k;
          it.base = chars;
          ++ni;
        } else {
          break;
        }
      }
      if (k == total) break;
      if (pos + 4 > slen) {
        report(st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 7);
        return false;
      }
      uint32_t len = ld_le32_g(sb + pos);
      if (len > slen - pos - 4) {
        report(st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 8);
        return false;
      }
      pos += 4 + len;
      chars += len;
    }
  }
  __syncthreads();
  return true;
}

// Resolves the page layout; returns false (error recorded) when the page is
// outside the supported subset or malformed.
__device__ bool page_ctx(const DecodeArgs& a, const PlanPage& pp, PageCtx* pc) {
  const PageDev pg = a.pages[pp.page];
  const ChunkDev ch = a.chunks[pp.chunk];
  pc->body = pp.body;
  pc->blen = static_cast<uint32_t>(pp.body_len);
  pc->nrows = pg.num_values;
  pc->pgid = static_cast<int32_t>(pp.page);
  pc->enc = pg.encoding;
  pc->ptype = ch.ptype;
  pc->width = ch.width;
  pc->max_def = ch.max_def;
  pc->lv0 = pc->lv1 = 0;
  if (pg.page_type == PAGE_DATA) {
    if (ch.max_def) {
      if (pc->blen < 4) return false;
      uint32_t L = ld_le32_g(pc->body);
      if (L > pc->blen - 4) return false;
      pc->lv0 = 4;
      pc->lv1 = 4 + L;
    }
    pc->v0 = pc->lv1;
  } else {
    if (pg.rep_len != 0) return false;
    if (static_cast<uint32_t>(pg.def_len) > pc->blen) return false;
    if (!ch.max_def && pg.def_len != 0) return false;
    pc->lv0 = 0;
    pc->lv1 = static_cast<uint32_t>(pg.def_len);
    pc->v0 = pc->lv1;
  }
  return true;
}

// Walk of one page (block-collective).
__device__ void walk_page(const DecodeArgs& a, int p, WalkSmem& sm, Win& win) {
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
    nonnull = walk_levels(sm, win, pc, pp, a.items, col, a.st);
    if (nonnull < 0) return;
    if (pg.page_type == PAGE_DATA_V2 && pg.num_nulls != pc.nrows - nonnull) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_LEVELS, 12);
      return;
    }
  } else {
    nonnull = pc.nrows;
    for (uint32_t i = tid; i < pp.item_count; i += blockDim.x) {
      Item& it = a.items[pp.item_begin + i];
      it.k0 = it.row0;
      it.nn = it.nrows;
    }
    __syncthreads();
  }
  const uint8_t* sb = pc.body + pc.v0;
  const uint32_t slen = pc.blen - pc.v0;
  bool ok = true;
  if (pc.enc == ENC_PLAIN) {
    if (pc.ptype == T_BYTE_ARRAY) {
      ok = walk_plain_ba(sb, slen, nonnull, pp, a.items, pgid, a.st);
    } else if (static_cast<uint64_t>(nonnull) * pc.width > slen) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 9);
      ok = false;
    }
  } else if (pc.enc == ENC_RLE_DICT || pc.enc == ENC_PLAIN_DICT) {
    const DictDev dd = a.dicts[pp.dict >= 0 ? pp.dict : 0];
    if (pp.dict < 0) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 10);
      ok = false;
    } else if (nonnull > 0) {
      if (slen < 1) {
        if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 11);
        ok = false;
      } else {
        int bw = __ldg(sb);
        if (bw > 32) {
          if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 12);
          ok = false;
        } else {
          ok = walk_hybrid(sm, win, sb + 1, slen - 1, bw, nonnull, pp, a.items, pgid, a.st);
        }
      }
    }
    (void)dd;
  } else if (pc.enc == ENC_DELTA_BP) {
    if (pc.ptype != T_INT32 && pc.ptype != T_INT64) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_WALK_VALUES, 13);
      ok = false;
    } else {
      ok = walk_delta(sm, win, sb, slen, pc.ptype == T_INT32 ? 32 : 64, nonnull, pp, a.items, pgid, a.st);
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

__global__ void __launch_bounds__(WALK_THREADS) k_walk(DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smraw[];
  WalkSmem& sm = *reinterpret_cast<WalkSmem*>(smraw);
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  Win win{sm.win, nullptr, WIN_BYTES, 0, &sm.bar, 0};
  for (int p = blockIdx.x; p < a.n_pp; p += gridDim.x) walk_page(a, p, sm, win);
}

// ------------------------------------------------------------------ expand

// Validity of tile rows [orow, orow + nt): word bits and ranks in shared
// memory; returns the number of valid rows.
__device__ int32_t tile_validity(ExpSmem& sm, const OutCol& col, int64_t orow, int nt) {
  const int nw = (nt + 31) >> 5;
  uint32_t bits = 0;
  if (threadIdx.x < nw) {
    int64_t b = orow + threadIdx.x * 32;
    int n = nt - static_cast<int>(threadIdx.x) * 32;
    if (n > 32) n = 32;
    int64_t wi = b >> 5;
    uint32_t sh = static_cast<uint32_t>(b & 31);
    uint32_t lo = col.validity[wi];
    uint32_t hi = (sh && (b & 31) + n > 32) ? col.validity[wi + 1] : 0u;
    bits = sh ? __funnelshift_r(lo, hi, sh) : lo;
    if (n < 32) bits &= (1u << n) - 1;
  }
  uint32_t total;
  uint32_t pre = block_exclusive_sum(static_cast<uint32_t>(__popc(bits)), sm.tmp32, &total);
  if (threadIdx.x < nw) {
    sm.wbits[threadIdx.x] = bits;
    sm.wpre[threadIdx.x] = pre;
  }
  __syncthreads();
  return static_cast<int32_t>(total);
}

__device__ __forceinline__ int32_t row_rank(const ExpSmem& sm, int r, bool* valid) {
  uint32_t w = sm.wbits[r >> 5];
  uint32_t b = static_cast<uint32_t>(r & 31);
  *valid = (w >> b) & 1u;
  return static_cast<int32_t>(sm.wpre[r >> 5] + __popc(w & ((1u << b) - 1u)));
}

// Hybrid (dictionary index) stream state, kept in ctl/c64 between tiles.
//  ctl[0] hp      next run header (stream offset)
//  ctl[1] kk      dense index of the next value
//  ctl[2] left    values left in the current run
//  ctl[3] rle     current run is repeated
//  c64[0] cur     repeated value, or stream bit position of the next packed value
__device__ bool hyb_tile(ExpSmem& sm, Win& win, const uint8_t* sb, uint32_t slen, int bw, int32_t total,
                         int32_t kneed, int nvals, const DictDev& dd, int ptype, int pgid, DevStatus* st) {
  const int tid = threadIdx.x;
  const uint32_t* w32 = reinterpret_cast<const uint32_t*>(win.s);
  const uint32_t vbytes = (bw + 7) / 8;
  int produced = 0;
  for (uint32_t guard = 0; guard < 4u * (slen + 64) && produced < nvals; ++guard) {
    if (tid == 0) {
      uint32_t hp = static_cast<uint32_t>(sm.ctl[0]);
      int32_t kk = sm.ctl[1];
      int32_t left = sm.ctl[2];
      int rle = sm.ctl[3];
      uint64_t cur = static_cast<uint64_t>(sm.c64[0]);
      int nseg = 0, reload = 0, err = 0;
      int prod = produced;
      const int64_t wbit0 = (sb - win.g0) * 8;  // window bit of stream bit 0
      while (prod < nvals && nseg < SEG_MAX) {
        if (left == 0) {
          if (kk >= total || hp >= slen) { err = 1; break; }
          int64_t wrel_s = (sb + hp) - win.g0;
          if (wrel_s < 0 || wrel_s >= win.n) { reload = 1; break; }
          uint32_t wrel = static_cast<uint32_t>(wrel_s);
          uint32_t lim_w = win.n, lim_s = wrel + (slen - hp);
          uint32_t lim = lim_w < lim_s ? lim_w : lim_s;
          uint64_t h = 0;
          int hl = uleb([&](uint32_t q) { return static_cast<uint32_t>(win.s[q]); }, wrel, lim, &h);
          if (hl == 0) {
            if (lim == lim_s) err = 1; else reload = 1;
            break;
          }
          uint64_t c;
          if (h & 1) {
            c = (h >> 1) * 8;
            uint64_t body = (h >> 1) * static_cast<uint64_t>(bw);
            if (hp + hl + body > slen) { err = 1; break; }
            cur = static_cast<uint64_t>(hp + hl) * 8;
            rle = 0;
            hp += hl + static_cast<uint32_t>(body);
          } else {
            c = h >> 1;
            if (hp + hl + vbytes > slen) { err = 1; break; }
            if (wrel + hl + vbytes > win.n) { reload = 1; break; }
            uint32_t v = 0;
            for (uint32_t q = 0; q < vbytes; ++q) v |= static_cast<uint32_t>(win.s[wrel + hl + q]) << (8 * q);
            cur = v;
            rle = 1;
            hp += hl + vbytes;
          }
          int64_t room = static_cast<int64_t>(total) - kk;
          left = static_cast<int32_t>(static_cast<int64_t>(c) < room ? static_cast<int64_t>(c) : room);
          continue;
        }
        if (kk < kneed) {  // skip values before the item's first
          int32_t s = kneed - kk < left ? kneed - kk : left;
          left -= s;
          kk += s;
          if (!rle) cur += static_cast<uint64_t>(s) * bw;
          continue;
        }
        int32_t take = nvals - prod < left ? nvals - prod : left;
        uint32_t meta = 0x80000000u;
        if (!rle) {
          int64_t wb = wbit0 + static_cast<int64_t>(cur);
          if (wb < 0) { reload = 1; break; }
          int64_t room = bw ? (static_cast<int64_t>(win.n) * 8 - wb) / bw : take;
          if (room < take) {
            take = static_cast<int32_t>(room > 0 ? room : 0);
            reload = 1;
          }
          if (take == 0) break;
          meta = static_cast<uint32_t>(wb);
        }
        sm.sdst[nseg] = prod;
        sm.scnt[nseg] = take;
        sm.smeta[nseg] = meta;
        sm.sval[nseg] = rle ? static_cast<uint32_t>(cur) : 0u;
        ++nseg;
        prod += take;
        left -= take;
        kk += take;
        if (!rle) cur += static_cast<uint64_t>(take) * bw;
        if (reload) break;
      }
      sm.ctl[0] = static_cast<int32_t>(hp);
      sm.ctl[1] = kk;
      sm.ctl[2] = left;
      sm.ctl[3] = rle;
      sm.c64[0] = static_cast<int64_t>(cur);
      sm.ctl[4] = nseg;
      sm.ctl[5] = reload;
      sm.ctl[6] = err;
      sm.ctl[7] = prod;
    }
    __syncthreads();
    if (sm.ctl[6]) {
      if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_EXPAND, 1);
      return false;
    }
    const int nseg = sm.ctl[4];
    const int prod = sm.ctl[7];
    // expand the segments into vbuf
    for (int j = produced + tid; j < prod; j += blockDim.x) {
      int lo = 0, hi = nseg - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sm.sdst[mid] <= j) lo = mid; else hi = mid - 1;
      }
      uint32_t meta = sm.smeta[lo];
      uint32_t idx;
      if (meta == 0x80000000u)
        idx = sm.sval[lo];
      else
        idx = bits32(w32, static_cast<uint64_t>(meta) + static_cast<uint64_t>(j - sm.sdst[lo]) * bw, bw);
      if (idx >= static_cast<uint32_t>(dd.n)) {
        report(st, DERR_CORRUPT, pgid, WHERE_EXPAND, 2);
        idx = 0;
        if (dd.n == 0) {
          sm.vbuf[j] = 0;
          continue;
        }
      }
      if (ptype == T_BYTE_ARRAY) {
        sm.vbuf[j] = idx;
      } else if (dd.width == 4) {
        sm.vbuf[j] = reinterpret_cast<const uint32_t*>(dd.values)[idx];
      } else {
        sm.vbuf[j] = reinterpret_cast<const uint64_t*>(dd.values)[idx];
      }
    }
    const int reload = sm.ctl[5];
    produced = prod;
    if (reload) {
      int64_t from;
      if (sm.ctl[2] > 0 && !sm.ctl[3])
        from = static_cast<int64_t>(static_cast<uint64_t>(sm.c64[0]) >> 3);
      else
        from = sm.ctl[0];
      if (!win_load(win, sb + from, sb + slen, st, pgid, WHERE_EXPAND)) return false;
    } else {
      __syncthreads();
      if (nseg == 0 && produced < nvals) {
        if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_EXPAND, 3);
        return false;
      }
    }
  }
  if (produced < nvals) {
    if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_EXPAND, 4);
    return false;
  }
  return true;
}

// DELTA stream state, kept between tiles:
//  ctl[8]  block position (stream offset) of the current block
//  ctl[9]  dense index of its first value
//  c64[1]  value preceding it
__device__ bool delta_tile(ExpSmem& sm, Win& win, const uint8_t* sb, uint32_t slen, const DeltaHdr& d,
                           int type_bits, int32_t kneed, int nvals, int pgid, DevStatus* st) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int32_t kend = kneed + nvals;
  // the first value of the page comes from the header
  if (kneed == 0 && nvals > 0 && tid == 0) sm.vbuf[0] = static_cast<uint64_t>(d.first);
  for (uint32_t guard = 0; guard < 4u * (slen + 64); ++guard) {
    if (tid == 0) {
      uint32_t bp = static_cast<uint32_t>(sm.ctl[8]);
      int32_t kk = sm.ctl[9];
      int nb = 0, reload = 0, bad = 0;
      while (nb < DB_MAX && kk < kend && kk < d.total) {
        if (bp >= slen) { bad = 1; break; }
        int64_t wrel_s = (sb + bp) - win.g0;
        if (wrel_s < 0 || wrel_s >= win.n) { reload = 1; break; }
        uint32_t wrel = static_cast<uint32_t>(wrel_s);
        uint32_t lim_w = win.n, lim_s = wrel + (slen - bp);
        uint32_t lim = lim_w < lim_s ? lim_w : lim_s;
        int32_t nv = d.total - kk < d.block ? d.total - kk : d.block;
        int64_t mn;
        uint32_t wpos, dpos;
        int more = 0;
        uint32_t size = delta_block(win, wrel, lim, d, nv, type_bits, &mn, &wpos, &dpos, &more, &bad);
        if (bad) break;
        if (size == 0) {
          if (lim == lim_s) bad = 1; else if (wrel == 0) bad = 2; else reload = 1;
          break;
        }
        sm.dstart[nb] = bp;
        sm.ddata[nb] = dpos;
        sm.dwid[nb] = wpos;
        sm.dk[nb] = kk;
        sm.dcnt[nb] = nv;
        sm.dmin[nb] = mn;
        sm.dnext[nb] = static_cast<int32_t>(bp + size);
        ++nb;
        bp += size;
        kk += nv;
      }
      sm.ctl[10] = nb;
      sm.ctl[11] = reload;
      sm.ctl[12] = bad;
    }
    __syncthreads();
    const int nb = sm.ctl[10];
    if (sm.ctl[12]) {
      if (tid == 0) report(st, sm.ctl[12] == 2 ? DERR_UNSUPPORTED : DERR_CORRUPT, pgid, WHERE_EXPAND, 5);
      return false;
    }
    // each warp decodes whole blocks: local inclusive prefix of (min + packed)
    for (int b = warp; b < nb; b += nwarps) {
      const int32_t cnt = sm.dcnt[b];
      const uint64_t mn = static_cast<uint64_t>(sm.dmin[b]);
      uint64_t carry = 0;
      for (int r0 = 0; r0 < cnt; r0 += 32) {
        int v = r0 + lane;
        uint64_t x = v < cnt ? mn + delta_packed(win, sm.dwid[b], sm.ddata[b], d.vpm, v) : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        x += carry;
        int32_t dense = sm.dk[b] + v;
        if (v < cnt && dense >= kneed && dense < kend) sm.vbuf[dense - kneed] = x;
        carry = __shfl_sync(0xffffffffu, x, 31);
      }
      if (lane == 0) sm.dsum[b] = carry;
    }
    __syncthreads();
    if (tid == 0) {
      uint64_t prev = static_cast<uint64_t>(sm.c64[1]);
      int adv = 1;
      for (int b = 0; b < nb; ++b) {
        sm.dbase[b] = prev;
        prev += sm.dsum[b];
        if (adv && sm.dk[b] + sm.dcnt[b] <= kend) {
          sm.ctl[8] = sm.dnext[b];
          sm.ctl[9] = sm.dk[b] + sm.dcnt[b];
          sm.c64[1] = static_cast<int64_t>(prev);
        } else {
          adv = 0;
        }
      }
    }
    __syncthreads();
    for (int b = warp; b < nb; b += nwarps) {
      for (int v = lane; v < sm.dcnt[b]; v += 32) {
        int32_t dense = sm.dk[b] + v;
        if (dense >= kneed && dense < kend) sm.vbuf[dense - kneed] += sm.dbase[b];
      }
    }
    __syncthreads();
    const int reload = sm.ctl[11];
    const bool finished = nb > 0 ? (sm.dk[nb - 1] + sm.dcnt[nb - 1] >= kend || sm.dk[nb - 1] + sm.dcnt[nb - 1] >= d.total)
                                 : (kend <= 1);
    __syncthreads();
    if (finished) return true;
    if (reload) {
      if (!win_load(win, sb + sm.ctl[8], sb + slen, st, pgid, WHERE_EXPAND)) return false;
    } else if (nb == 0) {
      if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_EXPAND, 6);
      return false;
    }
  }
  if (tid == 0) report(st, DERR_CORRUPT, pgid, WHERE_EXPAND, 7);
  return false;
}

// PLAIN BYTE_ARRAY: thread 0 walks the values of the tile (serial).
//  ctl[13] position of the next value's length prefix
__device__ bool plain_ba_tile(ExpSmem& sm, const uint8_t* sb, uint32_t slen, int nvals, int pgid, DevStatus* st) {
  if (threadIdx.x == 0) {
    uint32_t pos = static_cast<uint32_t>(sm.ctl[13]);
    int err = 0;
    for (int j = 0; j < nvals; ++j) {
      if (pos + 4 > slen) { err = 1; break; }
      uint32_t len = ld_le32_g(sb + pos);
      if (len > slen - pos - 4) { err = 1; break; }
      sm.vbuf[j] = pos;
      pos += 4 + len;
    }
    sm.ctl[13] = static_cast<int32_t>(pos);
    sm.ctl[14] = err;
  }
  __syncthreads();
  if (sm.ctl[14]) {
    if (threadIdx.x == 0) report(st, DERR_CORRUPT, pgid, WHERE_EXPAND, 8);
    return false;
  }
  return true;
}

__device__ __forceinline__ void store_val(uint8_t* base, int64_t row, int width, uint64_t v) {
  if (width == 4)
    reinterpret_cast<uint32_t*>(base)[row] = static_cast<uint32_t>(v);
  else
    reinterpret_cast<uint64_t*>(base)[row] = v;
}

// Decodes one work item (block-collective).
__device__ void expand_item(const DecodeArgs& a, int it_id, ExpSmem& sm, Win& win) {
  const int tid = threadIdx.x;
  const Item it = a.items[it_id];
  if (it.nrows <= 0) return;
  const PlanPage pp = a.pps[it.pp];
  const PageDev pg = a.pages[pp.page];
  const OutCol col = a.cols[pp.col];
  const int pgid = static_cast<int>(pp.page);
  if (pp.nonnull < 0) return;  // the walk of this page failed (error already recorded)
  const uint8_t* body = pp.body;
  const uint32_t v0 = static_cast<uint32_t>(pp.values_off);
  const uint8_t* sb = body + v0;
  uint32_t slen = static_cast<uint32_t>(pp.body_len) - v0;
  const int32_t nonnull = pp.nonnull;
  const int enc = pg.encoding;
  const bool isdict = enc == ENC_RLE_DICT || enc == ENC_PLAIN_DICT;
  const bool isdelta = enc == ENC_DELTA_BP;
  const bool isba = col.ptype == T_BYTE_ARRAY;
  const int width = col.width;
  DictDev dd{};
  int bw = 0;
  DeltaHdr dh{};
  const int type_bits = col.ptype == T_INT32 ? 32 : 64;
  if (isdict && it.nn > 0) {
    dd = a.dicts[pp.dict];
    bw = __ldg(sb);
    sb += 1;
    slen -= 1;
    if (tid == 0) {
      sm.ctl[0] = it.pos;
      sm.ctl[1] = it.run_k0;
      sm.ctl[2] = 0;
      sm.ctl[3] = 0;
      sm.c64[0] = 0;
    }
    if (!win_load(win, sb + it.pos, sb + slen, a.st, pgid, WHERE_EXPAND)) return;
  } else if (isdelta && it.nn > 0) {
    if (!delta_header(sb, slen, &dh)) return;
    if (tid == 0) {
      sm.ctl[8] = it.pos;
      sm.ctl[9] = it.run_k0;
      sm.c64[1] = it.base;
    }
    if (!win_load(win, sb + it.pos, sb + slen, a.st, pgid, WHERE_EXPAND)) return;
  } else if (isba && enc == ENC_PLAIN && it.nn > 0) {
    if (tid == 0) sm.ctl[13] = it.pos;
  }
  __syncthreads();
  int32_t k = it.k0;
  uint64_t chars_sum = 0;
  const int64_t orow0 = pp.out_row + it.row0;
  for (int t0 = 0; t0 < it.nrows; t0 += TILE_ROWS) {
    const int nt = it.nrows - t0 < TILE_ROWS ? it.nrows - t0 : TILE_ROWS;
    const int64_t orow = orow0 + t0;
    int32_t nv = col.optional ? tile_validity(sm, col, orow, nt) : nt;
    if (k + nv > nonnull) {
      if (tid == 0) report(a.st, DERR_CORRUPT, pgid, WHERE_EXPAND, 9);
      return;
    }
    bool ok = true;
    if (nv > 0) {
      if (isdict)
        ok = hyb_tile(sm, win, sb, slen, bw, nonnull, k, nv, dd, col.ptype, pgid, a.st);
      else if (isdelta)
        ok = delta_tile(sm, win, sb, slen, dh, type_bits, k, nv, pgid, a.st);
      else if (isba)
        ok = plain_ba_tile(sm, sb, slen, nv, pgid, a.st);
    }
    __syncthreads();
    if (!ok) return;
    // emit rows
    if (isba) {
      for (int r = tid; r < nt; r += blockDim.x) {
        bool valid = true;
        int32_t rank = r;
        if (col.optional) rank = row_rank(sm, r, &valid);
        uint32_t s = valid ? static_cast<uint32_t>(sm.vbuf[rank]) : NULL_IDX;
        col.str_scratch[orow + r] = s;
        if (valid) chars_sum += isdict ? dd.str_len[s] : ld_le32_g(sb + s);
      }
    } else if (!isdict && !isdelta) {
      // PLAIN fixed width: straight from the page
      const uint8_t* src = sb + static_cast<int64_t>(k) * width;
      for (int r = tid; r < nt; r += blockDim.x) {
        bool valid = true;
        int32_t rank = r;
        if (col.optional) rank = row_rank(sm, r, &valid);
        uint64_t v = valid ? ld_unaligned_g(src + static_cast<int64_t>(rank) * width, width) : 0;
        store_val(col.values, orow + r, width, v);
      }
    } else {
      for (int r = tid; r < nt; r += blockDim.x) {
        bool valid = true;
        int32_t rank = r;
        if (col.optional) rank = row_rank(sm, r, &valid);
        store_val(col.values, orow + r, width, valid ? sm.vbuf[rank] : 0);
      }
    }
    k += nv;
    __syncthreads();
  }
  if (isba) {
    uint64_t tot;
    (void)block_exclusive_sum(chars_sum, sm.tmp64, &tot);
    if (tid == 0) col.str_item_bytes[it_id] = tot;
  }
}

__global__ void __launch_bounds__(EXP_THREADS) k_expand(DecodeArgs a) {
  extern __shared__ __align__(16) uint8_t smraw[];
  ExpSmem& sm = *reinterpret_cast<ExpSmem*>(smraw);
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  Win win{sm.win, nullptr, WIN_BYTES, 0, &sm.bar, 0};
  for (uint32_t guard = 0; guard <= static_cast<uint32_t>(a.n_items); ++guard) {
    if (threadIdx.x == 0) sm.ctl[15] = static_cast<int32_t>(atomicAdd(a.item_counter, 1u));
    __syncthreads();
    const int it = sm.ctl[15];
    __syncthreads();
    if (it >= a.n_items) break;
    expand_item(a, it, sm, win);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ strings

// Per string column: exclusive prefix of item chars; writes the final offset.
__global__ void k_str_scan(DecodeArgs a, const int* __restrict__ str_cols) {
  const OutCol col = a.cols[str_cols[blockIdx.x]];
  __shared__ uint64_t tmp[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b = 0; b < col.item_count; b += blockDim.x) {
    uint32_t i = b + threadIdx.x;
    uint64_t v = i < col.item_count ? col.str_item_bytes[col.item_begin + i] : 0;
    uint64_t tot;
    uint64_t pre = block_exclusive_sum(v, tmp, &tot);
    if (i < col.item_count) col.str_item_bytes[col.item_begin + i] = carry + pre;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    reinterpret_cast<int64_t*>(col.values)[col.n_rows] = static_cast<int64_t>(carry);
    if (carry > col.chars_cap) report(a.st, DERR_CAPACITY, -1, WHERE_STRINGS, 1);
  }
}

// Per item of a string column: int64 offsets and the chars copy.
__global__ void __launch_bounds__(256) k_str_copy(DecodeArgs a) {
  __shared__ uint64_t tmp[32];
  for (int itx = blockIdx.x; itx < a.n_items; itx += gridDim.x) {
    const Item it = a.items[itx];
    if (it.nrows <= 0) continue;
    const PlanPage pp = a.pps[it.pp];
    const OutCol col = a.cols[pp.col];
    if (col.ptype != T_BYTE_ARRAY) continue;
    const PageDev pg = a.pages[pp.page];
    const bool isdict = pg.encoding == ENC_RLE_DICT || pg.encoding == ENC_PLAIN_DICT;
    DictDev dd{};
    if (isdict && pp.dict >= 0) dd = a.dicts[pp.dict];
    const uint8_t* sb = pp.body + pp.values_off;
    uint64_t base = col.str_item_bytes[itx];
    const int64_t orow0 = pp.out_row + it.row0;
    int64_t* offs = reinterpret_cast<int64_t*>(col.values);
    for (int r0 = 0; r0 < it.nrows; r0 += blockDim.x) {
      int r = r0 + threadIdx.x;
      uint32_t len = 0;
      const uint8_t* src = nullptr;
      if (r < it.nrows) {
        uint32_t s = col.str_scratch[orow0 + r];
        if (s != NULL_IDX) {
          if (isdict) {
            len = dd.str_len[s];
            src = dd.chars + dd.str_pos[s];
          } else {
            len = ld_le32_g(sb + s);
            src = sb + s + 4;
          }
        }
      }
      uint64_t tot;
      uint64_t pre = block_exclusive_sum(static_cast<uint64_t>(len), tmp, &tot);
      if (r < it.nrows) {
        uint64_t off = base + pre;
        offs[orow0 + r] = static_cast<int64_t>(off);
        if (off + len <= col.chars_cap)
          for (uint32_t q = 0; q < len; ++q) col.chars[off + q] = __ldg(src + q);
      }
      base += tot;
    }
  }
}

// ------------------------------------------------------------------ plain baseline

union PlainSmem {
  WalkSmem w;
  ExpSmem e;
};

// One page per thread block: walk then expand the page's single item.
__global__ void __launch_bounds__(EXP_THREADS) k_plain_page(DecodeArgs a, int pp_begin) {
  extern __shared__ __align__(16) uint8_t smraw[];
  PlainSmem& sm = *reinterpret_cast<PlainSmem*>(smraw);
  const int p = pp_begin + blockIdx.x;
  if (threadIdx.x == 0) {
    mbar_init(&sm.w.bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // both layouts start with the same barrier word; the expansion continues
  // with the phase parity the walk left
  Win ww{sm.w.win, nullptr, WIN_BYTES, 0, &sm.w.bar, 0};
  walk_page(a, p, sm.w, ww);
  __syncthreads();
  Win we{sm.e.win, nullptr, WIN_BYTES, 0, &sm.e.bar, ww.parity};
  const PlanPage pp = a.pps[p];
  for (uint32_t i = 0; i < pp.item_count; ++i) {
    expand_item(a, static_cast<int>(pp.item_begin + i), sm.e, we);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ per-scan reset

// Zeroes the validity bitmaps (bits are OR-ed in by the walk), the string
// item totals, the item counter and the error word.
__global__ void k_prepare(DecodeArgs a, int n_cols) {
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint64_t nthr = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  if (tid == 0) {
    *a.item_counter = 0;
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

void launch_prepare(const DecodeArgs& a, int n_cols, int grid, cudaStream_t s) {
  k_prepare<<<grid, 256, 0, s>>>(a, n_cols);
}

// ------------------------------------------------------------------ launchers

static int g_walk_bps = 0, g_exp_bps = 0;

int walk_blocks_per_sm() {
  if (!g_walk_bps) {
    cudaFuncSetAttribute(k_walk, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(WalkSmem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_walk_bps, k_walk, WALK_THREADS, sizeof(WalkSmem));
    if (g_walk_bps < 1) g_walk_bps = 1;
  }
  return g_walk_bps;
}

int expand_blocks_per_sm() {
  if (!g_exp_bps) {
    cudaFuncSetAttribute(k_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(ExpSmem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_exp_bps, k_expand, EXP_THREADS, sizeof(ExpSmem));
    if (g_exp_bps < 1) g_exp_bps = 1;
  }
  return g_exp_bps;
}

void launch_walk(const DecodeArgs& a, int grid, cudaStream_t s) {
  if (a.n_pp <= 0) return;
  walk_blocks_per_sm();
  k_walk<<<grid, WALK_THREADS, sizeof(WalkSmem), s>>>(a);
}

void launch_expand(const DecodeArgs& a, int grid, cudaStream_t s) {
  if (a.n_items <= 0) return;
  expand_blocks_per_sm();
  k_expand<<<grid, EXP_THREADS, sizeof(ExpSmem), s>>>(a);
}

void launch_strings(const DecodeArgs& a, const int* str_cols, int n_str_cols, int n_cols_total, int grid,
                    cudaStream_t s) {
  (void)n_cols_total;
  if (n_str_cols <= 0) return;
  k_str_scan<<<n_str_cols, 256, 0, s>>>(a, str_cols);
  k_str_copy<<<grid, 256, 0, s>>>(a);
}

void launch_plain_pages(const DecodeArgs& a, int pp_begin, int n, cudaStream_t s) {
  if (n <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_plain_page, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(PlainSmem));
    attr = true;
  }
  k_plain_page<<<n, EXP_THREADS, sizeof(PlainSmem), s>>>(a, pp_begin);
}

}  // namespace pqi
