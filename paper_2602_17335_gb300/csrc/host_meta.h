// Host-side Parquet footer (FileMetaData) parsing — the metadata of the
// file -> row group -> column chunk hierarchy of the paper's Section 2.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace pqh {

struct ColumnMeta {
  std::string name;
  int32_t type = -1;
  int32_t repetition = 0;  // 0 REQUIRED, 1 OPTIONAL, 2 REPEATED
  int32_t type_length = 0;
};

struct ChunkMeta {
  int32_t type = -1;
  int32_t codec = 0;
  int64_t num_values = 0;
  int64_t total_uncompressed = 0;
  int64_t total_compressed = 0;
  int64_t data_page_offset = -1;
  int64_t dict_page_offset = -1;   // -1 when absent
  int64_t oi_offset = -1;          // OffsetIndex location, -1 when absent
  int32_t oi_length = 0;
  int64_t byte_array_bytes = -1;   // SizeStatistics.unencoded_byte_array_data_bytes
  bool has_meta = false;
  int64_t start() const {
    return (dict_page_offset > 0 && dict_page_offset < data_page_offset) ? dict_page_offset : data_page_offset;
  }
  bool has_dict() const { return dict_page_offset > 0 && dict_page_offset < data_page_offset; }
};

struct RowGroupMeta {
  int64_t num_rows = 0;
  std::vector<ChunkMeta> chunks;
};

struct FileMeta {
  int64_t num_rows = 0;
  std::vector<ColumnMeta> columns;  // leaf columns
  std::vector<RowGroupMeta> rgs;
  uint32_t footer_len = 0;
};

enum { META_OK = 0, META_CORRUPT = 2, META_UNSUPPORTED = 3 };

// Parses FileMetaData from `p[0..n)`; returns META_* and sets *err.
int parse_file_metadata(const uint8_t* p, size_t n, FileMeta* out, std::string* err);

// Reads the page count of a serialized OffsetIndex (its list header).
int offset_index_pages(const uint8_t* p, size_t n, int64_t* pages);

}  // namespace pqh
