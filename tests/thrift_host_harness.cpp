// Test harness: the index kernel's page-header parser (thrift_dev.cuh)
// compiled for the CPU.  The device qualifiers and the read-only load are
// mapped to their host meaning here; the parser's source is unchanged.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define __device__
#define __forceinline__ inline
template <typename T>
static inline T __ldg(const T* p) { return *p; }

#include "thrift_dev.cuh"

extern "C" int page_header_host(const uint8_t* p, uint64_t len, int32_t* out /* 9 ints */) {
  pqi::PageDev pg{};
  const int n = pqi::parse_page_header(p, p + len, &pg);
  out[0] = pg.page_type;
  out[1] = pg.uncompressed;
  out[2] = pg.compressed;
  out[3] = pg.num_values;
  out[4] = pg.encoding;
  out[5] = pg.num_nulls;
  out[6] = pg.def_len;
  out[7] = pg.rep_len;
  out[8] = static_cast<int32_t>(pg.v2_compressed);
  return n;
}

// The same with the bytes in a heap block of exactly their size.
extern "C" int page_header_host_exact(const uint8_t* p, uint64_t len, int32_t* out) {
  uint8_t* b = static_cast<uint8_t*>(malloc(len ? len : 1));
  memcpy(b, p, len);
  const int n = page_header_host(b, len, out);
  free(b);
  return n;
}
