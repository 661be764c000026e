// K0 — page-header indexing.
//
// A column chunk is a sequence of pages, each a Thrift PageHeader followed
// by compressed_page_size body bytes; the next header starts right after the
// body (paper Section 2: chunk -> pages).  The walk inside one chunk is
// serial by nature, so each thread walks one chunk and the grid covers all
// chunks; a first launch counts pages, the host sizes the page table, and a
// second launch fills it.  When the file carries an OffsetIndex, the page
// locations are read from it instead and every page header is parsed by its
// own thread.
#include "dev_util.cuh"
#include "thrift_dev.cuh"

namespace pqi {

// mode 0: count pages into counts[c]; mode 1: fill pages[] (page_begin set).
__global__ void k_index_walk(const ChunkDev* __restrict__ chunks, int n_chunks, PageDev* pages,
                             uint32_t* counts, int mode, DevStatus* st) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  const ChunkDev ch = chunks[c];
  uint64_t pos = 0;
  int64_t seen = 0;
  int64_t row = 0;
  uint32_t np = 0;
  const uint8_t* end = ch.base + ch.size;
  // every page consumes >= 2 header bytes, so the walk is bounded by size / 2
  const uint64_t max_pages = ch.size / 2 + 1;
  while (seen < ch.num_values) {
    if (np >= max_pages || pos >= ch.size) {
      report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 1);
      return;
    }
    PageDev pg;
    pg.pad = 0;
    int hl = parse_page_header(ch.base + pos, end, &pg);
    if (hl < 0) {
      report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 2);
      return;
    }
    uint64_t body_end = pos + static_cast<uint64_t>(hl) + static_cast<uint64_t>(pg.compressed);
    if (body_end > ch.size) {
      report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 3);
      return;
    }
    if (pg.page_type == PAGE_INDEX) {  // never written in practice; skipped
      pos = body_end;
      continue;
    }
    if (pg.page_type != PAGE_DATA && pg.page_type != PAGE_DICT && pg.page_type != PAGE_DATA_V2) {
      report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 4);
      return;
    }
    if (pg.page_type == PAGE_DICT && np != 0) {
      report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 5);  // a dictionary page must come first
      return;
    }
    pg.offset = pos;
    pg.header_len = hl;
    pg.chunk = static_cast<uint32_t>(c);
    pg.first_row = pg.page_type == PAGE_DICT ? 0 : row;
    if (pg.page_type != PAGE_DICT) {
      if (pg.num_values < 0 || seen + pg.num_values > ch.num_values) {
        report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 6);
        return;
      }
      row += pg.num_values;
      seen += pg.num_values;
    }
    if (mode == 1) {
      if (np >= ch.page_count) {
        report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 7);
        return;
      }
      pages[ch.page_begin + np] = pg;
    }
    ++np;
    pos = body_end;
  }
  if (mode == 0) counts[c] = np;
}

// OffsetIndex path, step 1 (one warp per chunk): read the page locations
// list {1: offset i64, 2: compressed_page_size i32, 3: first_row_index i64}
// into the page table's offset field (file offset, rebased to the chunk).
// Slot 0 of a dictionary chunk is reserved for its dictionary page, which
// starts at the chunk start.  The usual serialization is parsed by the whole
// warp from shared memory (oi_locations_tokens); any other form by lane 0
// with the general Thrift reader.
constexpr int OI_WARPS = 4;
constexpr uint32_t OI_SMEM = 8192;  // bytes staged per warp

template <bool kGlobal>
__device__ void oi_locations(TRdT<kGlobal> r, int c, const ChunkDev& ch, int64_t file_off, PageDev* pages,
                             DevStatus* st) {
  int last = 0, fid = 0, type = 0;
  const uint32_t slot = ch.dict_page >= 0 ? 1u : 0u;
  bool got = false;
  for (int g = 0; g < 16 && r.field(&last, &fid, &type); ++g) {
    if (fid == 1 && type == 9) {
      uint32_t h = r.byte();
      uint64_t n = h >> 4;
      if ((h & 15) != 12) r.err = true;
      if (n == 15) n = r.varint();
      if (r.err || n != ch.oi_pages) {
        report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 10);
        return;
      }
      for (uint64_t i = 0; i < n; ++i) {
        int l2 = 0, f2 = 0, t2 = 0;
        int64_t off = -1;
        for (int g2 = 0; g2 < 16 && r.field(&l2, &f2, &t2); ++g2) {
          if (f2 == 1)
            off = r.zz();
          else
            r.skip(t2, 1);
        }
        const int64_t rel = off - file_off;
        if (r.err || rel < 0 || static_cast<uint64_t>(rel) >= ch.size) {
          report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 11);
          return;
        }
        PageDev d{};
        d.offset = static_cast<uint64_t>(rel);
        d.chunk = static_cast<uint32_t>(c);
        pages[ch.page_begin + slot + i] = d;
      }
      got = true;
    } else {
      r.skip(type, 0);
    }
    if (r.err) break;
  }
  if (r.err || !got) report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 12);
}

// The usual serialization of the OffsetIndex: field 1, a list of n structs,
// each {1: i64 offset, 2: i32 compressed_page_size, 3: i64 first_row_index}
// with one-byte field headers (0x16, 0x15, 0x16) and a stop byte.  Each of
// those single bytes has its high bit clear, as has the last byte of a
// varint and no other varint byte: in this form a struct is exactly seven
// tokens, each ending at a high-bit-clear byte, and struct k starts right
// after token 7k - 1.  The warp streams the list through shared memory in
// windows that start at a struct (16-byte loads; the OffsetIndex lies inside
// the file, before its footer, so the aligned words around it are readable);
// it finds a window's struct starts by counting token ends (4 bytes per lane,
// a warp scan per 128 bytes), then every lane parses whole structs from its
// starts, checking each byte against the form.  False (nothing assumed
// written) when the bytes take any other form; the general parser then
// reads the list.
constexpr uint32_t OI_STARTS = OI_SMEM / 7 + 2;  // a struct takes at least 7 bytes

__device__ bool oi_locations_tokens(uint8_t* raw, uint16_t* starts, const uint8_t* oi, uint32_t oi_len, int c,
                                    const ChunkDev& ch, int64_t file_off, PageDev* pages, int lane) {
  const uint32_t slot = ch.dict_page >= 0 ? 1u : 0u;
  // list header (every lane reads the same bytes): 0x19, then (n << 4) | 12
  // with n < 15, or 0xfc and n as a varint
  if (oi_len < 2 || __ldg(oi) != 0x19 || (__ldg(oi + 1) & 15) != 12) return false;
  uint64_t n = __ldg(oi + 1) >> 4;
  uint32_t pos = 2;
  if (n == 15) {
    uint64_t v = 0;
    int b = 0;
    for (; b < 10 && pos < oi_len; ++b) {
      const uint32_t y = __ldg(oi + pos++);
      v |= static_cast<uint64_t>(y & 0x7f) << (7 * b);
      if (!(y & 0x80)) break;
    }
    if (b == 10 || (__ldg(oi + pos - 1) & 0x80)) return false;
    n = v;
  }
  if (n != ch.oi_pages) return false;
  uint64_t i = 0;  // structs written
  for (uint32_t guard = 0; i < n && guard <= oi_len; ++guard) {
    if (pos >= oi_len) return false;
    const uint32_t wlen = oi_len - pos < OI_SMEM ? oi_len - pos : OI_SMEM;
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(oi + pos);
    const uint32_t sh = static_cast<uint32_t>(a0 & 15);
    const uint4* src = reinterpret_cast<const uint4*>(a0 - sh);
    const uint32_t nv = (sh + wlen + 15) >> 4;
    for (uint32_t v = lane; v < nv; v += 32) reinterpret_cast<uint4*>(raw)[v] = __ldg(src + v);
    if (lane == 0) starts[0] = 0;
    __syncwarp();
    const uint8_t* w = raw + sh;
    uint32_t tb = 0;  // token ends before this step
    for (uint32_t q0 = 0; q0 < wlen; q0 += 128) {
      const uint32_t q = q0 + 4 * static_cast<uint32_t>(lane);
      uint32_t em = 0;  // bit j: byte q + j ends a token
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (q + j < wlen && !(w[q + j] & 0x80)) em |= 1u << j;
      const uint32_t cnt = __popc(em);
      uint32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint32_t t = tb + incl - cnt;  // index of the lane's first token end
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if ((em >> j) & 1u) {
          if ((t + 1) % 7 == 0) {
            const uint32_t sidx = (t + 1) / 7;
            if (sidx < OI_STARTS) starts[sidx] = static_cast<uint16_t>(q + j + 1);
          }
          ++t;
        }
      }
      tb += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    // structs whose seven tokens all end in the window
    const uint64_t whole = tb / 7;
    const uint32_t take = static_cast<uint32_t>(whole < n - i ? whole : n - i);
    if (take == 0) return false;  // no whole struct in a window of OI_SMEM bytes: not this form
    bool ok = true;
    for (uint32_t k = lane; k < take; k += 32) {
      const uint8_t* p = w + starts[k];
      const uint8_t* e = w + starts[k + 1];
      auto varint = [&](uint64_t* v) -> bool {
        uint64_t x = 0;
        for (int b = 0; b < 10 && p < e; ++b) {
          const uint32_t y = *p++;
          x |= static_cast<uint64_t>(y & 0x7f) << (7 * b);
          if (!(y & 0x80)) {
            *v = x;
            return true;
          }
        }
        return false;
      };
      uint64_t off = 0, skip = 0;
      bool sok = p < e && *p++ == 0x16 && varint(&off);
      sok = sok && p < e && *p++ == 0x15 && varint(&skip);
      sok = sok && p < e && *p++ == 0x16 && varint(&skip);
      sok = sok && p < e && *p++ == 0x00 && p == e;
      const int64_t rel = static_cast<int64_t>(off >> 1) ^ -static_cast<int64_t>(off & 1);
      const int64_t r = rel - file_off;
      sok = sok && r >= 0 && static_cast<uint64_t>(r) < ch.size;
      if (sok) {
        PageDev d{};
        d.offset = static_cast<uint64_t>(r);
        d.chunk = static_cast<uint32_t>(c);
        pages[ch.page_begin + slot + i + k] = d;
      }
      ok = ok && sok;
    }
    if (!__all_sync(0xffffffffu, ok)) return false;
    i += take;
    pos += starts[take];
    __syncwarp();  // the window and its starts are reused
  }
  return i == n;
}

// Chunks whose OffsetIndex exceeds OI_SMEM take a block: the page-location
// list is cut into OI_SEG-byte segments, one per warp per round; each warp
// counts the token ends of its segment, a block scan gives every segment the
// number of tokens before it, and each warp then finds the structs that
// start in its segment (struct k starts after token 7k - 1; a segment
// starts one when the tokens before it are a multiple of seven) and parses
// them, one per lane, from a staged copy that runs 64 bytes into the next
// segment (a struct takes at most 34 bytes).  Smaller ones take the warp
// path above, one chunk per warp of the block.
constexpr int OI_BWARPS = 8;
constexpr uint32_t OI_SEG = 4096;
constexpr uint32_t OI_SEG_STARTS = OI_SEG / 7 + 2;
static_assert(OI_BWARPS == 2 * OI_WARPS, "a block holds OI_WARPS warp-path chunks or one segmented chunk");

__device__ bool oi_locations_segments(uint8_t (*raw)[OI_SEG + 96], uint16_t (*starts)[OI_SEG_STARTS], uint32_t* wcnt,
                                      int* flags, const uint8_t* oi, uint32_t oi_len, int c, const ChunkDev& ch,
                                      int64_t file_off, PageDev* pages) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t slot = ch.dict_page >= 0 ? 1u : 0u;
  // list header (every thread reads the same bytes)
  if (oi_len < 2 || __ldg(oi) != 0x19 || (__ldg(oi + 1) & 15) != 12) return false;
  uint64_t n = __ldg(oi + 1) >> 4;
  uint32_t pos0 = 2;
  if (n == 15) {
    uint64_t v = 0;
    int b = 0;
    for (; b < 10 && pos0 < oi_len; ++b) {
      const uint32_t y = __ldg(oi + pos0++);
      v |= static_cast<uint64_t>(y & 0x7f) << (7 * b);
      if (!(y & 0x80)) break;
    }
    if (b == 10 || (__ldg(oi + pos0 - 1) & 0x80)) return false;
    n = v;
  }
  if (n != ch.oi_pages) return false;
  const uint32_t L = oi_len - pos0;  // bytes from struct 0 on
  if (threadIdx.x == 0) {
    flags[0] = 0;  // a struct that does not parse
    flags[1] = 0;  // structs written
  }
  __syncthreads();
  uint64_t carry = 0;  // token ends before this round
  for (uint32_t r0 = 0; r0 < L; r0 += OI_BWARPS * OI_SEG) {
    const uint32_t g0 = r0 + static_cast<uint32_t>(w) * OI_SEG;
    const uint32_t glen = g0 < L ? min(OI_SEG, L - g0) : 0u;
    const uint32_t slen = g0 < L ? min(glen + 64, L - g0) : 0u;  // staged bytes
    uint32_t sh = 0;
    if (slen) {
      const uintptr_t a0 = reinterpret_cast<uintptr_t>(oi + pos0 + g0);
      sh = static_cast<uint32_t>(a0 & 15);
      const uint4* src = reinterpret_cast<const uint4*>(a0 - sh);
      const uint32_t nv = (sh + slen + 15) >> 4;
      for (uint32_t v = lane; v < nv; v += 32) reinterpret_cast<uint4*>(raw[w])[v] = __ldg(src + v);
    }
    __syncwarp();
    const uint8_t* sb = raw[w] + sh;
    // token ends of the segment
    uint32_t cnt = 0;
    for (uint32_t q = 4 * static_cast<uint32_t>(lane); q < glen; q += 128)
#pragma unroll
      for (int j = 0; j < 4; ++j) cnt += (q + j < glen && !(sb[q + j] & 0x80)) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) wcnt[w] = cnt;
    __syncthreads();
    uint64_t base = carry;
    uint64_t total = 0;
    for (int k = 0; k < OI_BWARPS; ++k) {
      if (k < w) base += wcnt[k];
      total += wcnt[k];
    }
    // struct starts in [0, glen): byte 0 when the tokens before it are a
    // multiple of seven, and the byte after every 7th token end
    const uint64_t first = (base + 6) / 7;  // index of the first struct starting here
    if (glen && lane == 0 && base % 7 == 0) starts[w][0] = 0;
    uint64_t tb = base;
    for (uint32_t q0 = 0; q0 < glen; q0 += 128) {
      const uint32_t q = q0 + 4 * static_cast<uint32_t>(lane);
      uint32_t em = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (q + j < glen && !(sb[q + j] & 0x80)) em |= 1u << j;
      const uint32_t ec = __popc(em);
      uint32_t incl = ec;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      uint64_t t = tb + incl - ec;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if ((em >> j) & 1u) {
          if ((t + 1) % 7 == 0 && q + j + 1 < glen) {
            const uint64_t k = (t + 1) / 7 - first;
            if (k < OI_SEG_STARTS) starts[w][k] = static_cast<uint16_t>(q + j + 1);
          }
          ++t;
        }
      }
      tb += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    // the structs starting here are those whose preceding token count, a
    // multiple of seven, is reached before the segment's last byte (a token
    // ending at the last byte starts the next segment's first struct)
    const uint64_t tex = tb - ((glen && !(sb[glen - 1] & 0x80)) ? 1u : 0u);
    const uint64_t last = tex / 7 + 1;  // first struct index not starting here
    const uint64_t nhere = (glen && last > first) ? last - first : 0;
    // (structs whose index reaches n are past the list)
    const uint64_t left = first < n ? n - first : 0;
    const uint64_t lim = nhere < left ? nhere : left;
    int wrote = 0;
    for (uint64_t k = lane; k < lim; k += 32) {
      const uint8_t* p = sb + starts[w][k];
      const uint8_t* e = sb + slen;
      auto varint = [&](uint64_t* v) -> bool {
        uint64_t x = 0;
        for (int b = 0; b < 10 && p < e; ++b) {
          const uint32_t y = *p++;
          x |= static_cast<uint64_t>(y & 0x7f) << (7 * b);
          if (!(y & 0x80)) {
            *v = x;
            return true;
          }
        }
        return false;
      };
      uint64_t off = 0, skip = 0;
      bool sok = p < e && *p++ == 0x16 && varint(&off);
      sok = sok && p < e && *p++ == 0x15 && varint(&skip);
      sok = sok && p < e && *p++ == 0x16 && varint(&skip);
      sok = sok && p < e && *p++ == 0x00;
      const int64_t rel = static_cast<int64_t>(off >> 1) ^ -static_cast<int64_t>(off & 1);
      const int64_t r = rel - file_off;
      sok = sok && r >= 0 && static_cast<uint64_t>(r) < ch.size;
      if (sok) {
        PageDev d{};
        d.offset = static_cast<uint64_t>(r);
        d.chunk = static_cast<uint32_t>(c);
        pages[ch.page_begin + slot + first + k] = d;
        ++wrote;
      } else {
        flags[0] = 1;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wrote += __shfl_xor_sync(0xffffffffu, wrote, o);
    if (lane == 0 && wrote) atomicAdd(&flags[1], wrote);
    __syncthreads();
    const bool stop = flags[0] != 0 || (carry + total) / 7 >= n;
    carry += total;
    __syncthreads();  // the staged bytes, starts and counts are rewritten next round
    if (stop) break;
  }
  return flags[0] == 0 && static_cast<uint64_t>(flags[1]) == n;
}

__global__ void __launch_bounds__(32 * OI_BWARPS) k_index_oi_locations(const ChunkDev* __restrict__ chunks,
                                                                       int n_chunks,
                                                                       const int64_t* __restrict__ chunk_file_off,
                                                                       PageDev* pages, DevStatus* st) {
  __shared__ __align__(16) uint8_t raw[OI_BWARPS][OI_SEG + 96];
  __shared__ uint16_t starts[OI_BWARPS][OI_SEG_STARTS];
  __shared__ uint32_t wcnt[OI_BWARPS];
  __shared__ int flags[2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // block b: either chunk b when its OffsetIndex is large (segments), or
  // chunks of the warp path: the small chunks among [OI_WARPS b, OI_WARPS (b + 1))
  const int big = blockIdx.x;
  if (big < n_chunks && chunks[big].oi_len > OI_SMEM) {
    const ChunkDev ch = chunks[big];
    if (threadIdx.x == 0 && ch.dict_page >= 0) {
      PageDev d{};
      d.offset = 0;
      d.chunk = static_cast<uint32_t>(big);
      pages[ch.page_begin] = d;
    }
    if (!oi_locations_segments(raw, starts, wcnt, flags, ch.oi_base, ch.oi_len, big, ch, chunk_file_off[big], pages)) {
      if (threadIdx.x == 0)
        oi_locations(TRd{ch.oi_base, ch.oi_base + ch.oi_len, false}, big, ch, chunk_file_off[big], pages, st);
    }
  }
  __syncthreads();  // the shared buffers are reused by the warp path
  if (w >= OI_WARPS) return;
  const int c = blockIdx.x * OI_WARPS + w;
  if (c >= n_chunks) return;
  const ChunkDev ch = chunks[c];
  if (ch.oi_len > OI_SMEM) return;  // (its own block takes it)
  if (lane == 0 && ch.dict_page >= 0) {
    PageDev d{};
    d.offset = 0;
    d.chunk = static_cast<uint32_t>(c);
    pages[ch.page_begin] = d;
  }
  uint8_t* wraw = raw[2 * w];  // OI_SMEM + 32 bytes: two segment buffers
  uint16_t* wst = starts[2 * w];
  if (!oi_locations_tokens(wraw, wst, ch.oi_base, ch.oi_len, c, ch, chunk_file_off[c], pages, lane)) {
    if (lane == 0) oi_locations(TRd{ch.oi_base, ch.oi_base + ch.oi_len, false}, c, ch, chunk_file_off[c], pages, st);
  }
}

// OffsetIndex path, step 2: one thread per page parses its header.
__global__ void k_index_oi_headers(const ChunkDev* __restrict__ chunks, PageDev* pages, int n_pages,
                                   DevStatus* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pages) return;
  PageDev pg = pages[i];
  const ChunkDev ch = chunks[pg.chunk];
  uint64_t off = pg.offset;
  PageDev h;
  h.pad = 0;
  int hl = parse_page_header(ch.base + off, ch.base + ch.size, &h);
  if (hl < 0 || off + hl + static_cast<uint64_t>(h.compressed) > ch.size ||
      (h.page_type != PAGE_DATA && h.page_type != PAGE_DATA_V2 && h.page_type != PAGE_DICT)) {
    report(st, DERR_CORRUPT, i, WHERE_INDEX, 13);
    return;
  }
  bool is_dict_slot = ch.dict_page >= 0 && static_cast<uint32_t>(i) == ch.page_begin;
  if ((h.page_type == PAGE_DICT) != is_dict_slot) {
    report(st, DERR_CORRUPT, i, WHERE_INDEX, 14);
    return;
  }
  h.offset = off;
  h.header_len = hl;
  h.chunk = pg.chunk;
  h.first_row = 0;
  pages[i] = h;
}

// OffsetIndex path, step 3 (one block per chunk): first_row of every data
// page (an exclusive scan of num_values over the chunk's pages, OI_ROWS
// pages a step), a check that each page starts where the previous one ends,
// and that the pages cover the chunk's values.
constexpr int OI_ROWS = 256;

__global__ void __launch_bounds__(OI_ROWS) k_index_oi_rows(const ChunkDev* __restrict__ chunks, int n_chunks,
                                                           PageDev* pages, DevStatus* st) {
  constexpr int kWarps = OI_ROWS / 32;
  __shared__ int64_t wsum[kWarps];
  __shared__ uint64_t wend[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x;
  if (c >= n_chunks) return;
  const ChunkDev ch = chunks[c];
  int64_t row = 0;
  uint64_t prev_end = 0;  // end of the page before this step's pages
  bool bad = false;
  for (uint32_t k0 = 0; k0 < ch.page_count; k0 += OI_ROWS) {
    const uint32_t k = k0 + threadIdx.x;
    const bool have = k < ch.page_count;
    PageDev* pg = pages + ch.page_begin + k;
    uint64_t off = 0, end = 0;
    int64_t nv = 0;
    int32_t type = PAGE_DICT;
    if (have) {
      off = pg->offset;
      end = off + static_cast<uint64_t>(pg->header_len) + static_cast<uint64_t>(pg->compressed);
      type = pg->page_type;
      nv = type != PAGE_DICT ? pg->num_values : 0;
    }
    int64_t incl = nv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint64_t before = __shfl_up_sync(0xffffffffu, end, 1);
    if (lane == 31) {
      wsum[w] = incl;
      wend[w] = end;
    }
    __syncthreads();
    if (lane == 0) before = w == 0 ? prev_end : wend[w - 1];
    int64_t base = row;
    for (int q = 0; q < w; ++q) base += wsum[q];
    bad |= have && off != before;
    if (have && type != PAGE_DICT) pg->first_row = base + incl - nv;
    for (int q = 0; q < kWarps; ++q) row += wsum[q];
    prev_end = wend[kWarps - 1];  // (unused after a partial last step)
    __syncthreads();  // wsum and wend are rewritten by the next step
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 15);
  } else if (threadIdx.x == 0 && row != ch.num_values) {
    report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 16);
  }
}

// The first min(len[i], 16) bytes at ptr[i] into out[16 i ..] (the rest
// zero), one thread per pointer: many small reads in one launch.
__global__ void k_gather16(const uint8_t* const* __restrict__ ptr, const int32_t* __restrict__ len, int n,
                           uint8_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint8_t* p = ptr[i];
  const int m = len[i] < 16 ? len[i] : 16;
  for (int k = 0; k < 16; ++k) out[16 * i + k] = k < m ? __ldg(p + k) : 0;
}

}  // namespace pqi

// Host-side launchers (C++ linkage, used by the engine).
namespace pqi {
void launch_index_walk(const ChunkDev* chunks, int n_chunks, PageDev* pages, uint32_t* counts, int mode,
                       DevStatus* st, cudaStream_t s) {
  if (n_chunks <= 0) return;
  int bs = 64;
  k_index_walk<<<(n_chunks + bs - 1) / bs, bs, 0, s>>>(chunks, n_chunks, pages, counts, mode, st);
}
void launch_index_oi(const ChunkDev* chunks, int n_chunks, const int64_t* chunk_file_off, PageDev* pages,
                     int n_pages, DevStatus* st, cudaStream_t s) {
  if (n_chunks <= 0) return;
  // enough blocks for every chunk's own block and for the warp path
  k_index_oi_locations<<<n_chunks, 32 * OI_BWARPS, 0, s>>>(chunks, n_chunks, chunk_file_off, pages, st);
  if (n_pages > 0) k_index_oi_headers<<<(n_pages + 127) / 128, 128, 0, s>>>(chunks, pages, n_pages, st);
  k_index_oi_rows<<<n_chunks, OI_ROWS, 0, s>>>(chunks, n_chunks, pages, st);
}
void launch_gather16(const uint8_t* const* ptr, const int32_t* len, int n, uint8_t* out, cudaStream_t s) {
  if (n <= 0) return;
  k_gather16<<<(n + 127) / 128, 128, 0, s>>>(ptr, len, n, out);
}
}  // namespace pqi
