// Test harness: the pipeline's host page walk (csrc/host_pages.cpp) behind a
// C entry point that writes each page's fields as ten int64 values.
#include <stdint.h>

#include <string>
#include <vector>

#include "host_pages.h"

extern "C" int64_t host_walk(const uint8_t* base, uint64_t size, int64_t num_values, int64_t* out, int64_t cap) {
  std::vector<pqi::PageDev> pages;
  std::string err;
  if (!pqe::host_page_walk(base, size, num_values, 7, &pages, &err)) return -1;
  const int64_t n = static_cast<int64_t>(pages.size());
  for (int64_t i = 0; i < n && i < cap; ++i) {
    const pqi::PageDev& p = pages[i];
    int64_t* o = out + 10 * i;
    o[0] = static_cast<int64_t>(p.offset);
    o[1] = p.first_row;
    o[2] = p.page_type;
    o[3] = p.encoding;
    o[4] = p.num_values;
    o[5] = p.num_nulls;
    o[6] = p.def_len;
    o[7] = p.header_len;
    o[8] = p.uncompressed;
    o[9] = p.compressed + (p.chunk == 7 ? 0 : (int64_t(1) << 40));  // chunk row passed through
  }
  return n;
}
