// Device-side Thrift compact-protocol reader for Parquet PageHeader structs
// (the page headers of the paper's Section 2 hierarchy).
//
// Compact protocol: a field header byte holds (field-id delta << 4) | type,
// or the type followed by a zigzag varint id when the delta is 0; integers
// are zigzag ULEB128; a bool field keeps its value in the type nibble
// (1 true, 2 false); binary = varint length + bytes; list/set header =
// (size << 4) | element type, size 15 meaning a varint size follows;
// map = varint size then a key/value type byte; a struct ends with 0.
#pragma once
#include <stdint.h>

#include "pq_internal.h"

namespace pqi {

// kGlobal: the bytes are in global memory (read-only loads); otherwise in
// shared memory.
template <bool kGlobal>
struct TRdT {
  const uint8_t* p;
  const uint8_t* end;
  bool err;

  __device__ __forceinline__ uint32_t byte() {
    if (p >= end) {
      err = true;
      return 0;
    }
    if constexpr (kGlobal)
      return __ldg(p++);
    else
      return *p++;
  }
  __device__ __forceinline__ uint64_t varint() {
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
  __device__ __forceinline__ int64_t zz() {
    uint64_t u = varint();
    return static_cast<int64_t>(u >> 1) ^ -static_cast<int64_t>(u & 1);
  }
  // Skips one value of compact type `t`.  Nested containers are walked with
  // an explicit bound on depth.
  __device__ void skip(int t, int depth) {
    if (err) return;
    if (depth > 8) {
      err = true;
      return;
    }
    switch (t) {
      case 1:
      case 2:
        return;  // bool field: value in the type nibble
      case 3:
        byte();
        return;
      case 4:
      case 5:
      case 6:
        varint();
        return;
      case 7:
        for (int i = 0; i < 8; ++i) byte();
        return;
      case 8: {
        uint64_t n = varint();
        if (err || n > static_cast<uint64_t>(end - p)) {
          err = true;
          return;
        }
        p += n;
        return;
      }
      case 9:
      case 10: {
        uint32_t h = byte();
        uint64_t n = h >> 4;
        int et = h & 15;
        if (n == 15) n = varint();
        if (n > static_cast<uint64_t>(end - p)) {
          err = true;
          return;
        }
        for (uint64_t i = 0; i < n && !err; ++i) {
          if (et == 1 || et == 2)
            byte();  // bools inside containers take one byte
          else
            skip(et, depth + 1);
        }
        return;
      }
      case 11: {
        uint64_t n = varint();
        if (n == 0) return;
        uint32_t kv = byte();
        if (n > static_cast<uint64_t>(end - p)) {
          err = true;
          return;
        }
        for (uint64_t i = 0; i < n && !err; ++i) {
          int kt = kv >> 4, vt = kv & 15;
          if (kt == 1 || kt == 2) byte(); else skip(kt, depth + 1);
          if (vt == 1 || vt == 2) byte(); else skip(vt, depth + 1);
        }
        return;
      }
      case 12: {
        int last = 0;
        for (int guard = 0; guard < 65536 && !err; ++guard) {
          uint32_t h = byte();
          if (err || h == 0) return;
          int ft = h & 15;
          int d = h >> 4;
          int fid = d ? last + d : static_cast<int>(zz());
          last = fid;
          skip(ft, depth + 1);
        }
        err = true;
        return;
      }
      default:
        err = true;
        return;
    }
  }
  // Reads the next field header of a struct: returns false at STOP.
  __device__ __forceinline__ bool field(int* last, int* fid, int* type) {
    uint32_t h = byte();
    if (err || h == 0) return false;
    *type = h & 15;
    int d = h >> 4;
    *fid = d ? *last + d : static_cast<int>(zz());
    *last = *fid;
    return !err;
  }
  __device__ __forceinline__ int32_t i32(int type) {
    if (type != 5 && type != 4 && type != 6) {
      err = true;
      return 0;
    }
    int64_t v = zz();
    if (v < INT32_MIN || v > INT32_MAX) err = true;
    return static_cast<int32_t>(v);
  }
};
using TRd = TRdT<true>;

// Parses one PageHeader at [p, end).  On success fills `pg` (except offset,
// first_row and chunk) and returns the header length; returns -1 on a
// malformed header.
__device__ inline int parse_page_header(const uint8_t* p, const uint8_t* end, PageDev* pg) {
  TRd r{p, end, false};
  pg->page_type = -1;
  pg->uncompressed = -1;
  pg->compressed = -1;
  pg->num_values = -1;
  pg->num_nulls = -1;
  pg->def_len = 0;
  pg->rep_len = 0;
  pg->encoding = -1;
  pg->v2_compressed = 1;
  int last = 0, fid = 0, type = 0;
  bool have_sub = false;
  for (int guard = 0; guard < 64; ++guard) {
    if (!r.field(&last, &fid, &type)) break;
    if (fid == 1) {
      pg->page_type = r.i32(type);
    } else if (fid == 2) {
      pg->uncompressed = r.i32(type);
    } else if (fid == 3) {
      pg->compressed = r.i32(type);
    } else if ((fid == 5 || fid == 7 || fid == 8) && type == 12) {
      have_sub = true;
      int l2 = 0, f2 = 0, t2 = 0;
      for (int g2 = 0; g2 < 64; ++g2) {
        if (!r.field(&l2, &f2, &t2)) break;
        if (f2 == 1 && t2 != 12) {
          pg->num_values = r.i32(t2);
        } else if (fid == 5 && f2 == 2) {
          pg->encoding = r.i32(t2);
        } else if (fid == 5 && (f2 == 3 || f2 == 4)) {
          int32_t e = r.i32(t2);  // level encodings: RLE (3) or BIT_PACKED (4)
          if (f2 == 3 && e != ENC_RLE && e != ENC_BIT_PACKED) r.err = true;
          if (f2 == 3 && e == ENC_BIT_PACKED) pg->pad = 1;  // deprecated level encoding
        } else if (fid == 7 && f2 == 2) {
          pg->encoding = r.i32(t2);
        } else if (fid == 8 && f2 == 2) {
          pg->num_nulls = r.i32(t2);
        } else if (fid == 8 && f2 == 3) {
          (void)r.i32(t2);  // num_rows: equal to num_values for flat columns
        } else if (fid == 8 && f2 == 4) {
          pg->encoding = r.i32(t2);
        } else if (fid == 8 && f2 == 5) {
          pg->def_len = r.i32(t2);
        } else if (fid == 8 && f2 == 6) {
          pg->rep_len = r.i32(t2);
        } else if (fid == 8 && f2 == 7 && (t2 == 1 || t2 == 2)) {
          pg->v2_compressed = t2 == 1 ? 1u : 0u;
        } else {
          r.skip(t2, 1);
        }
        if (r.err) return -1;
      }
    } else {
      r.skip(type, 0);
    }
    if (r.err) return -1;
  }
  if (r.err || pg->page_type < 0 || pg->uncompressed < 0 || pg->compressed < 0) return -1;
  if (pg->page_type != PAGE_INDEX && (!have_sub || pg->num_values < 0 || pg->encoding < 0)) return -1;
  if (pg->def_len < 0 || pg->rep_len < 0) return -1;
  return static_cast<int>(r.p - p);
}

}  // namespace pqi
