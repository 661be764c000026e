// Internal definitions shared by the host engine and the device kernels.
//
// Data layout in device memory (per index / plan):
//   ChunkDev[n_chunks]   one row per column chunk (file-major, row group, column)
//   PageDev[n_pages]     page table built by the header walk (chunk order)
//   DictDev[n_chunks]    decoded dictionary of each dictionary chunk
//   PlanPage[n_pp]       the data pages a plan touches, with their output placement
//   Item[n_items]        decode work items: a row range of one page plus the
//                        stream checkpoint the walk kernel found for it
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define PQ_HD __host__ __device__
#else
#define PQ_HD
#endif

namespace pqi {

// Parquet enum values (format's Encoding / PageType / Type / CompressionCodec).
enum : int32_t {
  ENC_PLAIN = 0, ENC_PLAIN_DICT = 2, ENC_RLE = 3, ENC_BIT_PACKED = 4, ENC_DELTA_BP = 5,
  ENC_DELTA_LBA = 6, ENC_DELTA_BA = 7, ENC_RLE_DICT = 8, ENC_BSS = 9
};
enum : int32_t { PAGE_DATA = 0, PAGE_INDEX = 1, PAGE_DICT = 2, PAGE_DATA_V2 = 3 };
enum : int32_t {
  T_BOOLEAN = 0, T_INT32 = 1, T_INT64 = 2, T_INT96 = 3, T_FLOAT = 4, T_DOUBLE = 5,
  T_BYTE_ARRAY = 6, T_FLBA = 7
};
enum : int32_t { CODEC_NONE = 0, CODEC_SNAPPY = 1, CODEC_ZSTD = 6 };

// Device error word flags.
enum : uint32_t {
  DERR_CORRUPT = 1u, DERR_UNSUPPORTED = 2u, DERR_TIMEOUT = 4u, DERR_CAPACITY = 8u
};

// Where in the engine an error was raised (stored with the first error).
enum : int32_t {
  WHERE_INDEX = 1, WHERE_SNAPPY = 2, WHERE_DICT = 3, WHERE_WALK_LEVELS = 4, WHERE_WALK_VALUES = 5,
  WHERE_EXPAND = 6, WHERE_STRINGS = 7, WHERE_PLAIN = 8, WHERE_TRANSCODE = 9
};

struct DevStatus {
  unsigned int flags;   // OR of DERR_*
  int first_page;       // page-table row of the first error (-1 none)
  int where;            // WHERE_* of the first error
  int detail;           // small code of the first error
};

struct ChunkDev {
  const uint8_t* base;  // device address of the chunk's first byte
  uint64_t size;        // stored chunk bytes
  int64_t num_values;   // rows of the chunk (flat schema)
  int32_t ptype;
  int32_t codec;
  int32_t max_def;      // 0 REQUIRED, 1 OPTIONAL
  int32_t width;        // fixed-width bytes, 0 for BYTE_ARRAY
  uint32_t page_begin;  // first page-table row
  uint32_t page_count;
  int32_t dict_page;    // page-table row of the dictionary page, -1 if none
  int32_t file;
  // OffsetIndex (device address of the serialized struct), or null
  const uint8_t* oi_base;
  uint32_t oi_len;
  uint32_t oi_pages;    // data pages listed in the OffsetIndex
};

struct PageDev {
  uint64_t offset;      // header offset within the chunk
  int64_t first_row;    // within the chunk (data pages); 0 for dictionary pages
  uint32_t chunk;
  int32_t page_type;
  int32_t encoding;
  int32_t num_values;   // rows (flat) / dictionary entries
  int32_t num_nulls;    // V2 header, -1 otherwise
  int32_t def_len;      // V2 only
  int32_t rep_len;      // V2 only
  int32_t uncompressed;
  int32_t compressed;
  int32_t header_len;
  uint32_t v2_compressed; // V2 is_compressed flag (1 default)
  uint32_t pad;           // 1: definition levels use the deprecated BIT_PACKED encoding
};

// Decoded dictionary of one chunk.
struct DictDev {
  const uint8_t* values;   // fixed width: n * width bytes, 16-byte aligned copy
  const uint64_t* str_ent; // BYTE_ARRAY: n entries; entry i = (offset of its chars in
                           // `chars` << 32) | its length
  const uint8_t* chars;    // BYTE_ARRAY: the (decompressed) dictionary page body
  int32_t n;
  int32_t width;
  int32_t max_len;         // longest entry (BYTE_ARRAY)
  int32_t valid;           // 1 once decoded
};

// A data page as a plan uses it.
struct PlanPage {
  const uint8_t* body;     // page body (decompressed when the chunk is compressed)
  int64_t out_row;         // output row of the page's row 0 (may be < 0 when the
                           // request starts inside the page)
  int64_t dfirst;          // DELTA: first value (from the stream header)   [walk]
  uint32_t page;           // page-table row
  uint32_t chunk;
  int32_t col;             // output column (request order)
  int32_t row_lo;          // first page row the request covers
  int32_t row_hi;          // one past the last
  uint32_t item_begin;     // first work item of this page
  uint32_t item_count;
  int32_t dict;            // chunk id of its dictionary (DictDev row), -1 none
  int32_t body_len;        // bytes of `body` (levels + values, uncompressed)
  int32_t values_off;      // start of the value stream within `body`   [host or walk]
  int32_t nonnull;         // non-null values on the page; -1 until known [host or walk]
  uint32_t dtab;           // DELTA: first row of the page's block tables
  int32_t dblocks;         // DELTA: blocks found by the walk                [walk]
  int32_t dbs;             // DELTA: values per block                        [walk]
  int32_t dvpm;            // DELTA: values per miniblock                    [walk]
  int32_t dmbc;            // DELTA: miniblocks per block                    [walk]
  int32_t dhlen;           // DELTA: stream header bytes (first block offset) [walk]
  uint32_t dreg;           // DELTA: first row of the page's region tables
  int32_t dreg_cap;        // DELTA: region rows reserved for the page
  int32_t pad;             // host: 1 while `body` is a scratch offset
  int32_t item_rows;       // rows per work item of this page
  int32_t enc;             // encoding the kernels decode: the page's own, or PLAIN once a
                           // BYTE_STREAM_SPLIT / DELTA_(LENGTH_)BYTE_ARRAY page is transcoded
  uint32_t vtab;           // transcoded string pages: 1 + first row of the page's value-position
                           // table (DecodeArgs::vpos, written by the transcoder); 0 none
};

// DELTA block-chain region (speculative parallel walk): regions of
// DELTA_REGION stream bytes, each walked from its first plausible block start.
constexpr int DELTA_REGION = 8192;
constexpr int DELTA_REGION_LIST = DELTA_REGION / 5 + 2;  // blocks are >= 5 bytes
struct DeltaRegion {
  int32_t q;      // first block start found in the region (-1: none)
  int32_t x;      // first chain position at or past the region end
  int32_t cnt;    // block starts recorded in [q, region end)
  int32_t pad;
};

// Decode work item: rows [row0, row0 + nrows) of one plan page.
struct Item {
  uint32_t pp;        // PlanPage row
  int32_t row0;       // page-relative first row
  int32_t nrows;
  int32_t k0;         // dense (non-null) index of the first value     [walk]
  int32_t pos;        // value-stream byte offset of the run / block / value
                      // that contains dense index k0                   [walk]
  int32_t run_k0;     // dense index at that run / block start          [walk]
  int64_t base;       // DELTA: value preceding that block; PLAIN BYTE_ARRAY:
                      // chars bytes before k0 within the page           [walk]
  int32_t run_left;   // hybrid: values left in a run split across items (unused: 0)
  int32_t nn;         // non-null values in the item                     [walk]
};

// Output column as the kernels see it.
struct OutCol {
  uint8_t* values;       // fixed width values, or int64 offsets for BYTE_ARRAY
  uint32_t* validity;    // null for REQUIRED
  uint8_t* chars;        // BYTE_ARRAY
  uint64_t chars_cap;
  int64_t n_rows;
  int32_t ptype;
  int32_t width;
  int32_t optional;
  int32_t pad;
  uint64_t* str_scratch; // BYTE_ARRAY: per row (offset of its chars << 32) | its length, the
                         // offset into the dictionary page (dictionary pages) or the page's
                         // values (PLAIN pages); 0 for a null
  uint64_t* str_item_bytes; // BYTE_ARRAY: chars bytes per item, then exclusive prefix
  uint32_t item_begin;   // items of this column are contiguous in item order
  uint32_t item_count;
};

PQ_HD inline int type_width(int32_t t) {
  return t == T_INT32 || t == T_FLOAT ? 4 : (t == T_INT64 || t == T_DOUBLE) ? 8 : 0;
}

// Rows per decode work item (one warp decodes one item): ITEM_ROWS for pages
// without definition levels, ITEM_ROWS_OPT for pages with them (OPTIONAL
// columns other than PLAIN fixed-width stage an item's dense values in
// shared memory; OPTIONAL PLAIN fixed-width write straight to the output).
constexpr int ITEM_ROWS = 2048;
constexpr int ITEM_ROWS_OPT = 512;

}  // namespace pqi
