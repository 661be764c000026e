// The index's header walk (Section 2: a chunk is a sequence of pages, each a
// Thrift PageHeader followed by its body) over a chunk in host memory.  The
// row-group pipeline of pq_scan_host holds the file in host memory, so it
// builds each row group's page table here: no index kernels compete with
// the scans of earlier row groups, and no page table is read back over the
// host link, whose device-to-host direction the bulk copy-out keeps busy.
#include <stdint.h>

#include <string>
#include <vector>

// The device index's Thrift reader (thrift_dev.cuh), with its device
// qualifiers and read-only loads taking their host meaning in this file.
#define __device__
#define __forceinline__ inline
template <typename T>
static inline T __ldg(const T* p) {
  return *p;
}
#include "thrift_dev.cuh"
#undef __forceinline__
#undef __device__

#include "host_pages.h"

namespace pqe {

bool host_page_walk(const uint8_t* base, uint64_t size, int64_t num_values, uint32_t chunk,
                    std::vector<pqi::PageDev>* pages, std::string* err) {
  uint64_t pos = 0;
  int64_t seen = 0, row = 0;
  uint64_t np = 0;
  const uint64_t max_pages = size / 2 + 1;  // a header takes at least 2 bytes
  const uint8_t* end = base + size;
  while (seen < num_values) {
    if (np >= max_pages || pos >= size) {
      *err = "chunk pages end before its values";
      return false;
    }
    pqi::PageDev pg{};
    const int hl = pqi::parse_page_header(base + pos, end, &pg);
    if (hl < 0) {
      *err = "malformed page header";
      return false;
    }
    const uint64_t body_end = pos + static_cast<uint64_t>(hl) + static_cast<uint64_t>(pg.compressed);
    if (pg.compressed < 0 || body_end > size) {
      *err = "page body outside its chunk";
      return false;
    }
    if (pg.page_type == pqi::PAGE_INDEX) {  // never written in practice; skipped
      pos = body_end;
      continue;
    }
    if (pg.page_type != pqi::PAGE_DATA && pg.page_type != pqi::PAGE_DICT && pg.page_type != pqi::PAGE_DATA_V2) {
      *err = "unknown page type";
      return false;
    }
    if (pg.page_type == pqi::PAGE_DICT && np != 0) {
      *err = "dictionary page after a data page";
      return false;
    }
    pg.offset = pos;
    pg.header_len = hl;
    pg.chunk = chunk;
    pg.first_row = pg.page_type == pqi::PAGE_DICT ? 0 : row;
    if (pg.page_type != pqi::PAGE_DICT) {
      if (pg.num_values < 0 || seen + pg.num_values > num_values) {
        *err = "page values beyond the chunk's";
        return false;
      }
      row += pg.num_values;
      seen += pg.num_values;
    }
    pages->push_back(pg);
    ++np;
    pos = body_end;
  }
  return true;
}

}  // namespace pqe
