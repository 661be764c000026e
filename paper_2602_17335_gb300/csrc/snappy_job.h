// One page to decompress (K1): built by the planner, read by the Snappy or
// the Zstandard kernel.
#pragma once
#include <stdint.h>

namespace pqi {

// The reference Snappy compressor works on 64 KiB fragments of its input,
// each on its own: no copy reaches into an earlier fragment and no element
// spans two.  A Snappy page whose decompressed stream is longer than
// SNAPPY_SPLIT_MIN is first scanned header by header for those fragment
// starts; where the page has that structure, its fragments are then
// decompressed as separate jobs ("blocks").
constexpr uint32_t SNAPPY_FRAGMENT = 65536;
constexpr uint32_t SNAPPY_SPLIT_MIN = 2 * SNAPPY_FRAGMENT;
constexpr uint32_t SJ_BLOCK = 1;  // flags: a block of a split page (no length preamble)

struct SnappyJob {
  const uint8_t* src;  // stored page body
  uint8_t* dst;        // decompressed page body (capacity dst_len + 16)
  uint32_t src_len;
  uint32_t dst_len;    // expected output bytes, including the verbatim prefix
  uint32_t prefix;     // bytes copied verbatim first (V2 level bytes)
  uint32_t raw;        // 1: no decompression (V2 page with is_compressed = false)
  int32_t page;        // page-table row, for error reports
  int32_t codec;       // CODEC_SNAPPY or CODEC_ZSTD: the kernel of the other codec skips the job
  uint32_t nsub;       // > 1: a split page, whose blocks are jobs [sub, sub + nsub) of the plan's block list
  uint32_t sub;
  uint32_t flags;      // SJ_BLOCK
  uint32_t pad;
};

}  // namespace pqi
