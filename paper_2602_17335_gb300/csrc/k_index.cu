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

__global__ void __launch_bounds__(32 * OI_WARPS) k_index_oi_locations(const ChunkDev* __restrict__ chunks,
                                                                      int n_chunks,
                                                                      const int64_t* __restrict__ chunk_file_off,
                                                                      PageDev* pages, DevStatus* st) {
  __shared__ __align__(16) uint8_t raw[OI_WARPS][OI_SMEM + 32];
  __shared__ uint16_t starts[OI_WARPS][OI_STARTS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = blockIdx.x * OI_WARPS + w;
  if (c >= n_chunks) return;
  const ChunkDev ch = chunks[c];
  if (lane == 0 && ch.dict_page >= 0) {
    PageDev d{};
    d.offset = 0;
    d.chunk = static_cast<uint32_t>(c);
    pages[ch.page_begin] = d;
  }
  if (!oi_locations_tokens(raw[w], starts[w], ch.oi_base, ch.oi_len, c, ch, chunk_file_off[c], pages, lane)) {
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
  const int blocks = (n_chunks + OI_WARPS - 1) / OI_WARPS;
  k_index_oi_locations<<<blocks, 32 * OI_WARPS, 0, s>>>(chunks, n_chunks, chunk_file_off, pages, st);
  if (n_pages > 0) k_index_oi_headers<<<(n_pages + 127) / 128, 128, 0, s>>>(chunks, pages, n_pages, st);
  k_index_oi_rows<<<n_chunks, OI_ROWS, 0, s>>>(chunks, n_chunks, pages, st);
}
void launch_gather16(const uint8_t* const* ptr, const int32_t* len, int n, uint8_t* out, cudaStream_t s) {
  if (n <= 0) return;
  k_gather16<<<(n + 127) / 128, 128, 0, s>>>(ptr, len, n, out);
}
}  // namespace pqi
