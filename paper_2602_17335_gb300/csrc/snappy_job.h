// One page to decompress (K1): built by the planner, read by the Snappy or
// the Zstandard kernel.
#pragma once
#include <stdint.h>

namespace pqi {

struct SnappyJob {
  const uint8_t* src;  // stored page body
  uint8_t* dst;        // decompressed page body (capacity dst_len + 16)
  uint32_t src_len;
  uint32_t dst_len;    // expected output bytes, including the verbatim prefix
  uint32_t prefix;     // bytes copied verbatim first (V2 level bytes)
  uint32_t raw;        // 1: no decompression (V2 page with is_compressed = false)
  int32_t page;        // page-table row, for error reports
  int32_t codec;       // CODEC_SNAPPY or CODEC_ZSTD: the kernel of the other codec skips the job
};

}  // namespace pqi
