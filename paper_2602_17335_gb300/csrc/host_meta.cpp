// Host Thrift compact-protocol reader for the Parquet footer.
//
// Compact protocol: field header byte = (id delta << 4) | type (delta 0:
// zigzag varint id follows); integers are zigzag ULEB128; bools live in the
// type nibble; binary = varint length + bytes; list header =
// (size << 4) | element type (size 15: varint size follows); structs end
// with a 0 byte.  Field ids follow the public parquet.thrift:
//   FileMetaData{1 version, 2 schema, 3 num_rows, 4 row_groups, ...}
//   SchemaElement{1 type, 2 type_length, 3 repetition_type, 4 name, 5 num_children}
//   RowGroup{1 columns, 2 total_byte_size, 3 num_rows, ...}
//   ColumnChunk{1 file_path, 2 file_offset, 3 meta_data, 4 offset_index_offset,
//               5 offset_index_length, ...}
//   ColumnMetaData{1 type, 2 encodings, 3 path_in_schema, 4 codec, 5 num_values,
//                  6 total_uncompressed_size, 7 total_compressed_size, 9 data_page_offset,
//                  11 dictionary_page_offset, 16 size_statistics{1 unencoded bytes}}
#include "host_meta.h"

#include <string.h>

namespace pqh {
namespace {

struct Rd {
  const uint8_t* p;
  const uint8_t* end;
  bool err = false;
  int depth = 0;

  uint32_t byte() {
    if (p >= end) {
      err = true;
      return 0;
    }
    return *p++;
  }
  uint64_t varint() {
    uint64_t v = 0;
    for (int i = 0; i < 10; ++i) {
      uint32_t b = byte();
      if (err) return 0;
      v |= static_cast<uint64_t>(b & 0x7f) << (7 * i);
      if (!(b & 0x80)) return v;
    }
    err = true;
    return 0;
  }
  int64_t zz() {
    uint64_t u = varint();
    return static_cast<int64_t>(u >> 1) ^ -static_cast<int64_t>(u & 1);
  }
  std::string binary() {
    uint64_t n = varint();
    if (err || n > static_cast<uint64_t>(end - p)) {
      err = true;
      return std::string();
    }
    std::string s(reinterpret_cast<const char*>(p), static_cast<size_t>(n));
    p += n;
    return s;
  }
  bool field(int* last, int* fid, int* type) {
    uint32_t h = byte();
    if (err || h == 0) return false;
    *type = h & 15;
    int d = h >> 4;
    *fid = d ? *last + d : static_cast<int>(zz());
    *last = *fid;
    return !err;
  }
  // list header: returns element count and type
  uint64_t list(int* et) {
    uint32_t h = byte();
    uint64_t n = h >> 4;
    *et = h & 15;
    if (n == 15) n = varint();
    if (n > static_cast<uint64_t>(end - p)) err = true;
    return err ? 0 : n;
  }
  void skip(int t) {
    if (err) return;
    if (++depth > 32) {
      err = true;
      return;
    }
    switch (t) {
      case 1:
      case 2:
        break;
      case 3:
        byte();
        break;
      case 4:
      case 5:
      case 6:
        varint();
        break;
      case 7:
        if (end - p < 8) err = true; else p += 8;
        break;
      case 8:
        binary();
        break;
      case 9:
      case 10: {
        int et;
        uint64_t n = list(&et);
        for (uint64_t i = 0; i < n && !err; ++i) {
          if (et == 1 || et == 2) byte(); else skip(et);
        }
        break;
      }
      case 11: {
        uint64_t n = varint();
        if (n) {
          uint32_t kv = byte();
          if (n > static_cast<uint64_t>(end - p)) err = true;
          for (uint64_t i = 0; i < n && !err; ++i) {
            int kt = kv >> 4, vt = kv & 15;
            if (kt == 1 || kt == 2) byte(); else skip(kt);
            if (vt == 1 || vt == 2) byte(); else skip(vt);
          }
        }
        break;
      }
      case 12: {
        int last = 0, fid, ty;
        while (field(&last, &fid, &ty)) skip(ty);
        break;
      }
      default:
        err = true;
    }
    --depth;
  }
  int32_t i32(int t) {
    if (t != 4 && t != 5 && t != 6) {
      err = true;
      return 0;
    }
    int64_t v = zz();
    if (v < INT32_MIN || v > INT32_MAX) err = true;
    return static_cast<int32_t>(v);
  }
  int64_t i64(int t) {
    if (t != 4 && t != 5 && t != 6) {
      err = true;
      return 0;
    }
    return zz();
  }
};

void parse_schema_element(Rd& r, ColumnMeta* c, int* num_children) {
  int last = 0, fid, t;
  *num_children = 0;
  while (r.field(&last, &fid, &t)) {
    switch (fid) {
      case 1: c->type = r.i32(t); break;
      case 2: c->type_length = r.i32(t); break;
      case 3: c->repetition = r.i32(t); break;
      case 4: c->name = r.binary(); break;
      case 5: *num_children = r.i32(t); break;
      default: r.skip(t);
    }
    if (r.err) return;
  }
}

void parse_size_statistics(Rd& r, ChunkMeta* m) {
  int last = 0, fid, t;
  while (r.field(&last, &fid, &t)) {
    if (fid == 1) m->byte_array_bytes = r.i64(t); else r.skip(t);
    if (r.err) return;
  }
}

void parse_column_metadata(Rd& r, ChunkMeta* m) {
  int last = 0, fid, t;
  m->has_meta = true;
  while (r.field(&last, &fid, &t)) {
    switch (fid) {
      case 1: m->type = r.i32(t); break;
      case 4: m->codec = r.i32(t); break;
      case 5: m->num_values = r.i64(t); break;
      case 6: m->total_uncompressed = r.i64(t); break;
      case 7: m->total_compressed = r.i64(t); break;
      case 9: m->data_page_offset = r.i64(t); break;
      case 11: m->dict_page_offset = r.i64(t); break;
      case 16:
        if (t == 12) parse_size_statistics(r, m); else r.skip(t);
        break;
      default: r.skip(t);
    }
    if (r.err) return;
  }
}

void parse_column_chunk(Rd& r, ChunkMeta* m) {
  int last = 0, fid, t;
  while (r.field(&last, &fid, &t)) {
    switch (fid) {
      case 3:
        if (t == 12) parse_column_metadata(r, m); else r.skip(t);
        break;
      case 4: m->oi_offset = r.i64(t); break;
      case 5: m->oi_length = r.i32(t); break;
      default: r.skip(t);
    }
    if (r.err) return;
  }
}

void parse_row_group(Rd& r, RowGroupMeta* g) {
  int last = 0, fid, t;
  while (r.field(&last, &fid, &t)) {
    if (fid == 1 && t == 9) {
      int et;
      uint64_t n = r.list(&et);
      if (et != 12) { r.err = true; return; }
      g->chunks.resize(n);
      for (uint64_t i = 0; i < n && !r.err; ++i) parse_column_chunk(r, &g->chunks[i]);
    } else if (fid == 3) {
      g->num_rows = r.i64(t);
    } else {
      r.skip(t);
    }
    if (r.err) return;
  }
}

}  // namespace

int parse_file_metadata(const uint8_t* p, size_t n, FileMeta* out, std::string* err) {
  Rd r{p, p + n};
  int last = 0, fid, t;
  bool have_schema = false, have_rgs = false, have_rows = false;
  std::vector<ColumnMeta> schema;
  std::vector<int> children;
  while (r.field(&last, &fid, &t)) {
    if (fid == 2 && t == 9) {
      int et;
      uint64_t cnt = r.list(&et);
      if (et != 12) { r.err = true; break; }
      schema.resize(cnt);
      children.resize(cnt);
      for (uint64_t i = 0; i < cnt && !r.err; ++i) parse_schema_element(r, &schema[i], &children[i]);
      have_schema = true;
    } else if (fid == 3) {
      out->num_rows = r.i64(t);
      have_rows = true;
    } else if (fid == 4 && t == 9) {
      int et;
      uint64_t cnt = r.list(&et);
      if (et != 12) { r.err = true; break; }
      out->rgs.resize(cnt);
      for (uint64_t i = 0; i < cnt && !r.err; ++i) parse_row_group(r, &out->rgs[i]);
      have_rgs = true;
    } else {
      r.skip(t);
    }
    if (r.err) break;
  }
  if (r.err || !have_schema || !have_rgs || !have_rows) {
    *err = "malformed FileMetaData";
    return META_CORRUPT;
  }
  if (schema.empty()) {
    *err = "empty schema";
    return META_CORRUPT;
  }
  const int ncols = children[0];
  if (static_cast<size_t>(ncols) + 1 != schema.size()) {
    *err = "nested schemas are not supported";
    return META_UNSUPPORTED;
  }
  for (size_t i = 1; i < schema.size(); ++i) {
    if (children[i] != 0) {
      *err = "nested schemas are not supported";
      return META_UNSUPPORTED;
    }
    if (schema[i].repetition == 2) {
      *err = "repeated columns are not supported";
      return META_UNSUPPORTED;
    }
    out->columns.push_back(schema[i]);
  }
  int64_t rows = 0;
  for (auto& g : out->rgs) {
    if (g.chunks.size() != static_cast<size_t>(ncols)) {
      *err = "row group column count differs from the schema";
      return META_CORRUPT;
    }
    for (auto& c : g.chunks) {
      if (!c.has_meta) {
        *err = "column metadata outside the footer is not supported";
        return META_UNSUPPORTED;
      }
    }
    rows += g.num_rows;
  }
  if (rows != out->num_rows) {
    *err = "row group rows do not add up to num_rows";
    return META_CORRUPT;
  }
  return META_OK;
}

int offset_index_pages(const uint8_t* p, size_t n, int64_t* pages) {
  // only a prefix of the struct is given: read field 1's list header without
  // checking the element count against the bytes at hand
  Rd r{p, p + n};
  int last = 0, fid, t;
  if (!r.field(&last, &fid, &t) || fid != 1 || t != 9) return META_CORRUPT;
  uint32_t h = r.byte();
  uint64_t cnt = h >> 4;
  if ((h & 15) != 12) return META_CORRUPT;
  if (cnt == 15) cnt = r.varint();
  if (r.err || cnt > (1u << 30)) return META_CORRUPT;
  *pages = static_cast<int64_t>(cnt);
  return META_OK;
}

}  // namespace pqh
