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

// OffsetIndex path, step 1 (one thread per chunk): read the page locations
// list {1: offset i64, 2: compressed_page_size i32, 3: first_row_index i64}
// into the page table's offset field (file offset, rebased to the chunk).
// Slot 0 of a dictionary chunk is reserved for its dictionary page, which
// starts at the chunk start.
__global__ void k_index_oi_locations(const ChunkDev* __restrict__ chunks, int n_chunks,
                                     const int64_t* __restrict__ chunk_file_off, PageDev* pages,
                                     DevStatus* st) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  const ChunkDev ch = chunks[c];
  TRd r{ch.oi_base, ch.oi_base + ch.oi_len, false};
  int last = 0, fid = 0, type = 0;
  uint32_t slot = ch.dict_page >= 0 ? 1u : 0u;
  if (slot) {
    PageDev d{};
    d.offset = 0;
    d.chunk = static_cast<uint32_t>(c);
    pages[ch.page_begin] = d;
  }
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
        int64_t rel = off - chunk_file_off[c];
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

// OffsetIndex path, step 3: one thread per chunk sets first_row (prefix of
// num_values) and checks that the pages are contiguous and cover the chunk's
// values.
__global__ void k_index_oi_rows(const ChunkDev* __restrict__ chunks, int n_chunks, PageDev* pages,
                                DevStatus* st) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  const ChunkDev ch = chunks[c];
  int64_t row = 0;
  uint64_t expect = 0;
  for (uint32_t k = 0; k < ch.page_count; ++k) {
    PageDev& pg = pages[ch.page_begin + k];
    if (pg.offset != expect) {
      report(st, DERR_CORRUPT, static_cast<int>(ch.page_begin + k), WHERE_INDEX, 15);
      return;
    }
    expect = pg.offset + pg.header_len + static_cast<uint64_t>(pg.compressed);
    if (pg.page_type != PAGE_DICT) {
      pg.first_row = row;
      row += pg.num_values;
    }
  }
  if (row != ch.num_values) report(st, DERR_CORRUPT, -1 - c, WHERE_INDEX, 16);
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
  int bs = 64;
  k_index_oi_locations<<<(n_chunks + bs - 1) / bs, bs, 0, s>>>(chunks, n_chunks, chunk_file_off, pages, st);
  if (n_pages > 0) k_index_oi_headers<<<(n_pages + 127) / 128, 128, 0, s>>>(chunks, pages, n_pages, st);
  k_index_oi_rows<<<(n_chunks + bs - 1) / bs, bs, 0, s>>>(chunks, n_chunks, pages, st);
}
}  // namespace pqi
