// Parquet writer — the offline rewriter of the paper's Sections 3 and 5:
// a flat table is written with a chosen row-group size, page size,
// encoding per column chunk (V1 PLAIN / dictionary, the V2 set
// DELTA_BINARY_PACKED, DELTA_LENGTH_BYTE_ARRAY, DELTA_BYTE_ARRAY and
// BYTE_STREAM_SPLIT), page version, and per-chunk compression (Snappy or
// Zstandard) kept only when it shrinks the chunk by more than a threshold
// (Section 3, "No Unnecessary Compression").  With encoding -1 every chunk tries each valid encoding of
// its type and keeps the one with the smallest encoded (uncompressed) chunk
// (Section 3, "Encoding Flexibility").
//
// Layout rules (identical to the ones the engine documents for pq_write_table):
//  * row group k holds rows [k*rg_rows, (k+1)*rg_rows);
//  * rows per data page: max(8, floor(page_bytes*8 / b) rounded down to a
//    multiple of 8), b = 8*width (PLAIN) or max(index bit width, 1)
//    (dictionary), +1 when OPTIONAL (BYTE_STREAM_SPLIT as PLAIN); REQUIRED
//    DELTA pages hold 1 + 128k values (the most whole blocks that fit
//    page_bytes, a shorter tail taken whole when it fits); BYTE_ARRAY pages
//    that are not dictionary encoded take rows while the page has fewer than
//    8 rows or the PLAIN-encoded bytes still fit;
//  * dictionary entries in order of first appearance, index bit width =
//    bit length of (entries - 1);
//  * hybrid runs: a repeated run for >= 8 equal values when the pending
//    literal values fill whole groups, otherwise bit-packed runs of at most
//    63 groups;
//  * V1 pages compress levels + values, V2 pages values only; the dictionary
//    page body is compressed with the chunk codec;
//  * an OffsetIndex per chunk after the last row group when requested.
// Chunks are encoded in parallel on `n_threads` host threads.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pq.h"
#include "huf_lengths.h"
#include "zstd_dec.cuh"

namespace {

using Bytes = std::vector<uint8_t>;

// ------------------------------------------------------------------ Thrift compact writer

struct TW {
  Bytes& o;
  std::vector<int> last{0};
  explicit TW(Bytes& out) : o(out) {}
  void varint(uint64_t v) {
    while (v >= 0x80) {
      o.push_back(static_cast<uint8_t>(v | 0x80));
      v >>= 7;
    }
    o.push_back(static_cast<uint8_t>(v));
  }
  static uint64_t zz(int64_t v) { return (static_cast<uint64_t>(v) << 1) ^ static_cast<uint64_t>(v >> 63); }
  void head(int fid, int type) {
    int d = fid - last.back();
    if (d > 0 && d <= 15) {
      o.push_back(static_cast<uint8_t>((d << 4) | type));
    } else {
      o.push_back(static_cast<uint8_t>(type));
      varint(zz(fid));
    }
    last.back() = fid;
  }
  void i32(int fid, int64_t v) { head(fid, 5); varint(zz(v)); }
  void i64(int fid, int64_t v) { head(fid, 6); varint(zz(v)); }
  void i16(int fid, int64_t v) { head(fid, 4); varint(zz(v)); }
  void boolean(int fid, bool v) { head(fid, v ? 1 : 2); }
  void binary(int fid, const std::string& s) {
    head(fid, 8);
    varint(s.size());
    o.insert(o.end(), s.begin(), s.end());
  }
  void list_begin(int fid, int elem_type, size_t n) {
    head(fid, 9);
    if (n < 15) {
      o.push_back(static_cast<uint8_t>((n << 4) | elem_type));
    } else {
      o.push_back(static_cast<uint8_t>(0xF0 | elem_type));
      varint(n);
    }
  }
  void struct_begin(int fid) {
    head(fid, 12);
    last.push_back(0);
  }
  void elem_struct_begin() { last.push_back(0); }
  void struct_end() {
    o.push_back(0);
    last.pop_back();
  }
  void stop() { o.push_back(0); }
};

void uleb(Bytes& o, uint64_t v) {
  while (v >= 0x80) {
    o.push_back(static_cast<uint8_t>(v | 0x80));
    v >>= 7;
  }
  o.push_back(static_cast<uint8_t>(v));
}

int bit_length(uint64_t v) { return v ? 64 - __builtin_clzll(v) : 0; }

// LSB-first packing of `n` values of `w` bits.
void pack_bits(Bytes& o, const uint64_t* v, size_t n, int w) {
  if (w == 0) return;
  size_t nbytes = (n * static_cast<size_t>(w) + 7) / 8;
  size_t base = o.size();
  o.resize(base + nbytes, 0);
  uint8_t* d = o.data() + base;
  uint64_t bit = 0;
  for (size_t i = 0; i < n; ++i) {
    uint64_t x = w == 64 ? v[i] : (v[i] & ((1ull << w) - 1));
    for (int b = 0; b < w;) {
      size_t byte = (bit + b) >> 3;
      int off = static_cast<int>((bit + b) & 7);
      int take = std::min(8 - off, w - b);
      d[byte] |= static_cast<uint8_t>(((x >> b) & ((1u << take) - 1)) << off);
      b += take;
    }
    bit += w;
  }
}

// ------------------------------------------------------------------ hybrid encoder

void packed_run(Bytes& o, const uint64_t* v, size_t n, int w) {
  size_t groups = (n + 7) / 8;
  uleb(o, (groups << 1) | 1);
  std::vector<uint64_t> pad(groups * 8, 0);
  std::copy(v, v + n, pad.begin());
  pack_bits(o, pad.data(), pad.size(), w);
}

void rle_run(Bytes& o, uint64_t value, size_t count, int w) {
  uleb(o, static_cast<uint64_t>(count) << 1);
  for (int b = 0; b < (w + 7) / 8; ++b) o.push_back(static_cast<uint8_t>(value >> (8 * b)));
}

void hybrid_encode(Bytes& o, const uint64_t* v, size_t n, int w) {
  // run[i] = equal values starting at i
  std::vector<uint32_t> run(n);
  for (size_t i = n; i-- > 0;) run[i] = (i + 1 < n && v[i] == v[i + 1]) ? run[i + 1] + 1 : 1;
  std::vector<uint64_t> pending;
  auto flush = [&]() {
    for (size_t a = 0; a < pending.size(); a += 504)
      packed_run(o, pending.data() + a, std::min<size_t>(504, pending.size() - a), w);
    pending.clear();
  };
  size_t i = 0;
  while (i < n) {
    if (run[i] >= 8 && pending.size() % 8 == 0) {
      flush();
      rle_run(o, v[i], run[i], w);
      i += run[i];
    } else {
      pending.push_back(v[i]);
      ++i;
    }
  }
  flush();
}

// ------------------------------------------------------------------ DELTA encoder

struct DeltaEnc {
  int bits;
  uint64_t wrap(uint64_t v) const { return bits == 32 ? static_cast<uint32_t>(v) : v; }
  int64_t sgn(uint64_t v) const {
    return bits == 32 ? static_cast<int64_t>(static_cast<int32_t>(static_cast<uint32_t>(v))) : static_cast<int64_t>(v);
  }
  void header(Bytes& o, size_t count, int64_t first) const {
    uleb(o, 128);
    uleb(o, 4);
    uleb(o, count);
    uleb(o, TW::zz(count ? first : 0));
  }
  // deltas: signed (sign-extended) values
  void block(Bytes& o, const int64_t* d, size_t n) const {
    int64_t mn = *std::min_element(d, d + n);
    uleb(o, TW::zz(mn));
    uint64_t packed[128];
    int widths[4] = {0, 0, 0, 0};
    for (size_t i = 0; i < n; ++i) packed[i] = wrap(static_cast<uint64_t>(d[i]) - static_cast<uint64_t>(mn));
    for (int m = 0; m < 4; ++m) {
      uint64_t mx = 0;
      bool any = false;
      for (size_t i = m * 32; i < std::min<size_t>(n, (m + 1) * 32); ++i) {
        mx = std::max(mx, packed[i]);
        any = true;
      }
      widths[m] = any ? bit_length(mx) : 0;
    }
    for (int m = 0; m < 4; ++m) o.push_back(static_cast<uint8_t>(widths[m]));
    for (int m = 0; m < 4; ++m) {
      if (static_cast<size_t>(m) * 32 >= n) break;
      uint64_t mb[32] = {0};
      for (size_t i = m * 32; i < std::min<size_t>(n, (m + 1) * 32); ++i) mb[i - m * 32] = packed[i];
      pack_bits(o, mb, 32, widths[m]);
    }
  }
  static size_t block_size(int64_t mn, const int* widths, size_t n) {
    Bytes t;
    uleb(t, TW::zz(mn));
    size_t s = t.size() + 4;
    for (int m = 0; m < 4; ++m)
      if (static_cast<size_t>(m) * 32 < n) s += 4 * widths[m];
    return s;
  }
};

// One DELTA_BINARY_PACKED INT32 stream (the length streams of the delta
// string encodings).
void delta_stream32(Bytes& o, const std::vector<int64_t>& v) {
  const DeltaEnc de{32};
  const size_t n = v.size();
  de.header(o, n, n ? v[0] : 0);
  int64_t dd[128];
  for (size_t b = 1; b < n; b += 128) {
    const size_t m = std::min<size_t>(128, n - b);
    for (size_t q = 0; q < m; ++q)
      dd[q] = de.sgn(static_cast<uint64_t>(v[b + q]) - static_cast<uint64_t>(v[b + q - 1]));
    de.block(o, dd, m);
  }
}

// ------------------------------------------------------------------ Snappy compressor

// Greedy LZ77 over 4-byte sequences with a hash table of recent positions,
// in 64 KiB fragments of the input, each on its own (the table starts empty,
// and matches and literals stay inside the fragment), which is how the
// reference Snappy compressor frames its output.
void snappy_compress(const uint8_t* in, size_t n, Bytes& o) {
  o.clear();
  uleb(o, n);
  auto literal = [&](size_t a, size_t b) {
    while (a < b) {
      size_t len = std::min<size_t>(b - a, 65536);
      if (len <= 60) {
        o.push_back(static_cast<uint8_t>((len - 1) << 2));
      } else {
        size_t v = len - 1;
        int nb = v < 256 ? 1 : v < 65536 ? 2 : v < (1u << 24) ? 3 : 4;
        o.push_back(static_cast<uint8_t>((59 + nb) << 2));
        for (int k = 0; k < nb; ++k) o.push_back(static_cast<uint8_t>(v >> (8 * k)));
      }
      o.insert(o.end(), in + a, in + a + len);
      a += len;
    }
  };
  auto copy = [&](size_t off, size_t len) {
    while (len > 0) {
      if (len >= 4 && len <= 11 && off < 2048) {
        o.push_back(static_cast<uint8_t>(((off >> 8) << 5) | ((len - 4) << 2) | 1));
        o.push_back(static_cast<uint8_t>(off));
        return;
      }
      size_t c = std::min<size_t>(len, 64);
      if (off < 65536) {
        o.push_back(static_cast<uint8_t>(((c - 1) << 2) | 2));
        o.push_back(static_cast<uint8_t>(off));
        o.push_back(static_cast<uint8_t>(off >> 8));
      } else {
        o.push_back(static_cast<uint8_t>(((c - 1) << 2) | 3));
        for (int k = 0; k < 4; ++k) o.push_back(static_cast<uint8_t>(off >> (8 * k)));
      }
      len -= c;
    }
  };
  const int kBits = 14;
  std::vector<int64_t> table(size_t(1) << kBits);
  auto h4 = [&](size_t i) {
    uint32_t x;
    memcpy(&x, in + i, 4);
    return (x * 0x1e35a7bdu) >> (32 - kBits);
  };
  constexpr size_t kFragment = 65536;
  for (size_t f0 = 0; f0 < n; f0 += kFragment) {
    const size_t f1 = std::min(n, f0 + kFragment);
    if (f1 - f0 < 16) {
      literal(f0, f1);
      continue;
    }
    std::fill(table.begin(), table.end(), int64_t(-1));
    size_t i = f0, lit = f0;
    const size_t limit = f1 - 4;
    while (i <= limit) {
      uint32_t h = h4(i);
      int64_t cand = table[h];
      table[h] = static_cast<int64_t>(i);
      if (cand >= 0 && memcmp(in + cand, in + i, 4) == 0) {
        size_t len = 4;
        while (i + len < f1 && in[cand + len] == in[i + len]) ++len;
        literal(lit, i);
        copy(i - cand, len);
        size_t end = i + len;
        for (size_t k = i + 1; k < end && k <= limit; k += 2) table[h4(k)] = static_cast<int64_t>(k);
        i = end;
        lit = i;
      } else {
        ++i;
      }
    }
    literal(lit, f1);
  }
}

// ------------------------------------------------------------------ Zstandard compressor

// One Zstandard frame per page (single segment, content size in the
// header, no checksum).  Each block of up to 128 KB of input is coded as
// sequences from greedy LZ77 matches: the previous match's offset is tried
// first, then a 4-byte hash over the whole frame so far; offsets are coded
// as repeat offsets where the history allows.  The sequence codes use FSE
// tables fitted to the block (an RLE table for a single code, or the
// predefined tables, whichever is smaller).  Literals are Huffman-coded (1
// or 4 streams) when that pays, else stored raw.  A block without matches,
// or one that would not shrink, is stored as a raw (or RLE) block.  Every
// Zstandard decoder reads the result.

struct ZBitW {  // little-endian bit writer
  Bytes& o;
  uint64_t acc = 0;
  int n = 0;
  explicit ZBitW(Bytes& out) : o(out) {}
  void put(uint64_t v, int nb) {  // nb <= 32
    if (nb == 0) return;
    acc |= (v & ((1ull << nb) - 1)) << n;
    n += nb;
    while (n >= 8) {
      o.push_back(static_cast<uint8_t>(acc));
      acc >>= 8;
      n -= 8;
    }
  }
  void finish() {  // end marker, then the last partial byte
    put(1, 1);
    if (n) o.push_back(static_cast<uint8_t>(acc));
    acc = 0;
    n = 0;
  }
};

// FSE encoding of one predefined distribution: the decoder's table (symbols
// spread over the states, each state's bit count and next-state base), and
// for every symbol and every next state the state that leads there.
struct ZFseEnc {
  int al = 0, size = 0;
  std::vector<uint8_t> sym, nb;
  std::vector<uint16_t> base;
  std::vector<std::vector<uint16_t>> from;  // [symbol][next state] -> state
  ZFseEnc(const int16_t* norm, int nsym, int a) : al(a), size(1 << a), sym(size), nb(size), base(size), from(nsym) {
    int high = size - 1;
    std::vector<uint32_t> next(nsym);
    for (int s = 0; s < nsym; ++s) {
      if (norm[s] == -1) {
        sym[high--] = static_cast<uint8_t>(s);
        next[s] = 1;
      } else {
        next[s] = static_cast<uint32_t>(norm[s]);
      }
    }
    const int step = (size >> 1) + (size >> 3) + 3, mask = size - 1;
    int pos = 0;
    for (int s = 0; s < nsym; ++s)
      for (int i = 0; i < norm[s]; ++i) {
        sym[pos] = static_cast<uint8_t>(s);
        do pos = (pos + step) & mask; while (pos > high);
      }
    for (int s = 0; s < nsym; ++s) from[s].assign(size, 0);
    for (int st = 0; st < size; ++st) {
      const uint32_t x = next[sym[st]]++;
      nb[st] = static_cast<uint8_t>(al - (bit_length(x) - 1));
      base[st] = static_cast<uint16_t>((x << nb[st]) - size);
      for (int y = base[st]; y < base[st] + (1 << nb[st]); ++y) from[sym[st]][y] = static_cast<uint16_t>(st);
    }
  }
  int any_state(int s) const {
    for (int st = 0; st < size; ++st)
      if (sym[st] == s) return st;
    return 0;
  }
};

const ZFseEnc& zenc_table(int which) {  // 0 literal lengths, 1 offsets, 2 match lengths
  static const int16_t LL[36] = {4, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 3, 2, 1,
                                1, 1, 1, 1, -1, -1, -1, -1};
  static const int16_t OF[29] = {1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1,
                                -1, -1};
  static const int16_t ML[53] = {1, 4, 3, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1, -1};
  static const ZFseEnc t_ll(LL, 36, 6), t_of(OF, 29, 5), t_ml(ML, 53, 6);
  return which == 0 ? t_ll : which == 1 ? t_of : t_ml;
}

// (code, extra-bit count, extra bits) of a literal length / match length
void zll_code(uint32_t ll, int* code, int* nb, uint32_t* extra) {
  static const uint32_t B[20] = {16, 18, 20, 22, 24, 28, 32, 40, 48, 64, 128, 256, 512, 1024, 2048, 4096, 8192,
                                 16384, 32768, 65536};
  static const int N[20] = {1, 1, 1, 1, 2, 2, 3, 3, 4, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16};
  if (ll < 16) {
    *code = static_cast<int>(ll);
    *nb = 0;
    *extra = 0;
    return;
  }
  int k = 19;
  while (ll < B[k]) --k;
  *code = 16 + k;
  *nb = N[k];
  *extra = ll - B[k];
}

void zml_code(uint32_t ml, int* code, int* nb, uint32_t* extra) {
  static const uint32_t B[21] = {35, 37, 39, 41, 43, 47, 51, 59, 67, 83, 99, 131, 259, 515, 1027, 2051, 4099, 8195,
                                 16387, 32771, 65539};
  static const int N[21] = {1, 1, 1, 1, 2, 2, 3, 3, 4, 4, 5, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16};
  if (ml - 3 < 32) {
    *code = static_cast<int>(ml - 3);
    *nb = 0;
    *extra = 0;
    return;
  }
  int k = 20;
  while (ml < B[k]) --k;
  *code = 32 + k;
  *nb = N[k];
  *extra = ml - B[k];
}

struct ZSeq {
  uint32_t ll, off, ml;
};

// Normalized counts of cnt[0, nsym) to 2^al: every present symbol at least
// 1, the rounding remainder on the most frequent one.  False if impossible.
bool fse_normalize(const uint32_t* cnt, int nsym, int al, int16_t* norm) {
  uint64_t total = 0;
  for (int s = 0; s < nsym; ++s) total += cnt[s];
  if (total == 0) return false;
  const int64_t L = int64_t(1) << al;
  int64_t sum = 0;
  int big = -1;
  for (int s = 0; s < nsym; ++s) {
    norm[s] = 0;
    if (!cnt[s]) continue;
    norm[s] = static_cast<int16_t>(std::max<int64_t>(1, static_cast<int64_t>(cnt[s]) * L / static_cast<int64_t>(total)));
    sum += norm[s];
    if (big < 0 || norm[s] > norm[big]) big = s;
  }
  const int64_t fixed = norm[big] + (L - sum);
  if (fixed < 1) return false;
  norm[big] = static_cast<int16_t>(fixed);
  return true;
}

// FSE table description of norm[0, nsym): accuracy log, then probability
// + 1 per symbol (the small values one bit shorter), 2-bit repeat flags
// after a zero probability, up to the last symbol.  Appends whole bytes.
bool fse_describe(const int16_t* norm, int nsym, int al, Bytes& out) {
  ZBitW bw(out);
  bw.put(al - 5, 4);
  int remaining = 1 << al;
  for (int s = 0; s < nsym && remaining > 0; ++s) {
    const uint32_t v = static_cast<uint32_t>(norm[s]) + 1;
    const uint32_t nv = static_cast<uint32_t>(remaining) + 2;
    const int nbits = bit_length(nv - 1);
    const uint32_t spare = (1u << nbits) - nv;
    if (v < spare)
      bw.put(v, nbits - 1);
    else if (v < (1u << (nbits - 1)))
      bw.put(v, nbits);
    else
      bw.put(v + spare, nbits);
    remaining -= norm[s];
    if (norm[s] == 0) {
      int run = 0;
      while (s + 1 + run < nsym && norm[s + 1 + run] == 0) ++run;
      s += run;
      for (;;) {
        const int r = std::min(run, 3);
        bw.put(r, 2);
        run -= r;
        if (r < 3) break;
      }
    }
  }
  if (bw.n) out.push_back(static_cast<uint8_t>(bw.acc));
  return remaining == 0;
}

// FSE-compressed Huffman weights (the tree description form for literal
// bytes of 128 and above): normalized counts at accuracy log 6, the table
// description, then the weights in two interleaved states.  The result is
// checked by decoding it with the engine's own decoding core; any case the
// simple scheme cannot express returns false (the literals then go raw).
bool fse_weights(const int* w, int nw, int mb, Bytes& out) {
  if (nw < 2) return false;
  const int al = 6, L = 1 << al;
  int cnt[16] = {0}, top = 0;
  for (int i = 0; i < nw; ++i) {
    ++cnt[w[i]];
    top = std::max(top, w[i]);
  }
  int distinct = 0;
  for (int s = 0; s <= top; ++s) distinct += cnt[s] > 0;
  if (distinct < 2) return false;
  uint32_t ucnt[16];
  for (int s = 0; s <= top; ++s) ucnt[s] = static_cast<uint32_t>(cnt[s]);
  int16_t norm[16] = {0};
  if (!fse_normalize(ucnt, top + 1, al, norm)) return false;
  Bytes desc;
  if (!fse_describe(norm, top + 1, al, desc)) return false;
  const ZFseEnc t(norm, top + 1, al);
  // decoder: states A (even weights) and B (odd) start from the last two
  // fields written; after each weight but the last two its state reads its
  // update; the update after weight nw-2 runs past the stream's start
  std::vector<int> st(nw);
  st[nw - 1] = t.any_state(w[nw - 1]);
  st[nw - 2] = -1;
  for (int k = 0; k < L; ++k)
    if (t.sym[k] == w[nw - 2] && t.nb[k] > 0) {
      st[nw - 2] = k;
      break;
    }
  if (st[nw - 2] < 0) return false;
  for (int i = nw - 3; i >= 0; --i) st[i] = t.from[w[i]][st[i + 2]];
  Bytes bits;
  {
    ZBitW bw(bits);
    for (int i = nw - 3; i >= 0; --i) bw.put(st[i + 2] - t.base[st[i]], t.nb[st[i]]);
    bw.put(st[1], al);
    bw.put(st[0], al);
    bw.finish();
  }
  const size_t size = desc.size() + bits.size();
  if (size >= 128) return false;
  out.clear();
  out.push_back(static_cast<uint8_t>(size));
  out.insert(out.end(), desc.begin(), desc.end());
  out.insert(out.end(), bits.begin(), bits.end());
  // check with the decoding core
  static thread_local pqi::ZState z;
  uint32_t used = 0;
  if (pqi::z_read_huf(out.data(), static_cast<uint32_t>(out.size()), &z, &used) || used != out.size() ||
      z.huf_bits != mb)
    return false;
  for (int i = 0; i < nw; ++i)
    if (z.weights[i] != w[i]) return false;
  return true;
}

// Huffman-coded literals section (tree description with direct 4-bit
// weights for literal bytes below 128, else FSE-compressed weights; 1
// stream up to 1023 literals, else 4 streams).  False when it does not
// apply or would not shrink.
bool huf_literals(const Bytes& lits, Bytes& out) {
  const size_t n = lits.size();
  if (n < 64 || n > 262143) return false;
  uint32_t cnt[256] = {0};
  for (uint8_t c : lits) ++cnt[c];
  int top = 255;
  while (top > 0 && cnt[top] == 0) --top;
  int len[256];
  if (!pqw::huf_lengths(cnt, top + 1, len)) return false;
  int mb = 0;
  for (int s = 0; s <= top; ++s) mb = std::max(mb, len[s]);
  // weights: nbits = mb + 1 - weight; the Kraft sum must be exactly full
  int64_t kraft = 0;
  for (int s = 0; s <= top; ++s)
    if (len[s]) kraft += int64_t(1) << (mb - len[s]);
  if (kraft != (int64_t(1) << mb)) return false;
  int w[256];
  for (int s = 0; s <= top; ++s) w[s] = len[s] ? mb + 1 - len[s] : 0;
  // canonical codes in the format's order: weight 1 first, symbols ascending
  uint32_t code[256] = {0};
  uint32_t start = 0;
  for (int wt = 1; wt <= mb; ++wt)
    for (int s = 0; s <= top; ++s)
      if (w[s] == wt) {
        code[s] = start >> (wt - 1);
        start += 1u << (wt - 1);
      }
  // tree description: the last symbol's weight is implied
  Bytes tree;
  const int nw = top;  // weights of symbols 0 .. top-1 are written
  if (nw <= 128) {
    tree.push_back(static_cast<uint8_t>(127 + nw));
    for (int i = 0; i < nw; i += 2)
      tree.push_back(static_cast<uint8_t>((w[i] << 4) | (i + 1 < nw ? w[i + 1] : 0)));
  } else if (!fse_weights(w, nw, mb, tree)) {
    return false;
  }
  auto stream = [&](size_t a, size_t b, Bytes& o) {
    ZBitW bw(o);
    for (size_t k = b; k-- > a;) bw.put(code[lits[k]], len[lits[k]]);
    bw.finish();
  };
  Bytes body = tree;
  int sf;
  if (n <= 1023) {
    sf = 0;
    Bytes s1;
    stream(0, n, s1);
    body.insert(body.end(), s1.begin(), s1.end());
  } else {
    const size_t per = (n + 3) / 4;
    Bytes s[4];
    for (int k = 0; k < 4; ++k) stream(std::min(n, k * per), std::min(n, (k + 1) * per), s[k]);
    for (int k = 0; k < 3; ++k) {
      if (s[k].size() > 65535) return false;
      body.push_back(static_cast<uint8_t>(s[k].size()));
      body.push_back(static_cast<uint8_t>(s[k].size() >> 8));
    }
    for (int k = 0; k < 4; ++k) body.insert(body.end(), s[k].begin(), s[k].end());
    sf = n <= 1023 ? 1 : n <= 16383 ? 2 : 3;
  }
  const size_t csize = body.size();
  const int bits = sf < 2 ? 10 : sf == 2 ? 14 : 18;
  if (csize >= (size_t(1) << bits) || csize >= n) return false;
  const int hlen = sf < 2 ? 3 : sf == 2 ? 4 : 5;
  const uint64_t h = 2u | (static_cast<uint64_t>(sf) << 2) | (static_cast<uint64_t>(n) << 4) |
                     (static_cast<uint64_t>(csize) << (4 + bits));
  out.clear();
  for (int k = 0; k < hlen; ++k) out.push_back(static_cast<uint8_t>(h >> (8 * k)));
  out.insert(out.end(), body.begin(), body.end());
  return true;
}

// Offset value of a match under the format's three repeat offsets (the
// decoder's history, updated the way the decoder updates it).
uint32_t zoffset_value(uint32_t ll, uint32_t off, uint32_t* r) {
  uint32_t ov;
  if (ll > 0 && off == r[0]) return 1;
  if (off == r[1]) {
    ov = ll > 0 ? 2 : 1;
    std::swap(r[0], r[1]);
    return ov;
  }
  if (off == r[2]) {
    ov = ll > 0 ? 3 : 2;
    const uint32_t t = r[2];
    r[2] = r[1];
    r[1] = r[0];
    r[0] = t;
    return ov;
  }
  if (ll == 0 && r[0] > 1 && off == r[0] - 1) {
    r[2] = r[1];
    r[1] = r[0];
    r[0] = off;
    return 3;
  }
  r[2] = r[1];
  r[1] = r[0];
  r[0] = off;
  return off + 3;
}

// Compressed-block body for `seqs` and `lits`; false when it would not be
// smaller than `raw` bytes.  `rep` is the frame's repeat-offset history,
// advanced only when the block is kept.
bool zstd_block_body(const std::vector<ZSeq>& seqs, const Bytes& lits, size_t raw, Bytes& body, uint32_t* rep) {
  body.clear();
  const size_t n = lits.size();
  Bytes hl;
  if (huf_literals(lits, hl)) {
    body = hl;
  } else if (n <= 31) {
    body.push_back(static_cast<uint8_t>(n << 3));
  } else if (n <= 4095) {
    body.push_back(static_cast<uint8_t>(((n & 15) << 4) | (1 << 2)));
    body.push_back(static_cast<uint8_t>(n >> 4));
  } else {
    body.push_back(static_cast<uint8_t>(((n & 15) << 4) | (3 << 2)));
    body.push_back(static_cast<uint8_t>(n >> 4));
    body.push_back(static_cast<uint8_t>(n >> 12));
  }
  if (hl.empty()) body.insert(body.end(), lits.begin(), lits.end());
  // sequences: with the predefined tables, and with tables fitted to this
  // block (an RLE table for a single code); the smaller section is kept
  const size_t ns = seqs.size();
  std::vector<int> code[3], nbx[3];
  std::vector<uint32_t> extra[3];
  for (int k = 0; k < 3; ++k) {
    code[k].resize(ns);
    nbx[k].resize(ns);
    extra[k].resize(ns);
  }
  uint32_t r[3] = {rep[0], rep[1], rep[2]};
  for (size_t i = 0; i < ns; ++i) {
    zll_code(seqs[i].ll, &code[0][i], &nbx[0][i], &extra[0][i]);
    const uint32_t ov = zoffset_value(seqs[i].ll, seqs[i].off, r);
    code[1][i] = bit_length(ov) - 1;
    nbx[1][i] = code[1][i];
    extra[1][i] = ov - (1u << code[1][i]);
    zml_code(seqs[i].ml, &code[2][i], &nbx[2][i], &extra[2][i]);
  }
  Bytes best, trial;
  bool have = false;
  for (int variant = 0; variant < 2; ++variant) {
    const ZFseEnc* t[3];
    std::unique_ptr<ZFseEnc> own[3];
    int mode[3];
    Bytes desc[3];
    bool ok = true;
    for (int k = 0; k < 3 && ok; ++k) {
      const int nsym = k == 0 ? 36 : k == 1 ? 32 : 53;
      if (variant == 0) {
        t[k] = &zenc_table(k);
        mode[k] = 0;
        if (k == 1)
          for (size_t i = 0; i < ns && ok; ++i) ok = code[1][i] <= 28;  // the predefined offset codes
        continue;
      }
      uint32_t cnt[53] = {0};
      int distinct = 0, last = 0;
      for (size_t i = 0; i < ns; ++i) distinct += cnt[code[k][i]]++ == 0;
      for (int s2 = 0; s2 < nsym; ++s2)
        if (cnt[s2]) last = s2;
      int16_t norm[53] = {0};
      if (distinct == 1) {
        norm[last] = 1;
        own[k].reset(new ZFseEnc(norm, last + 1, 0));
        mode[k] = 1;
        desc[k].push_back(static_cast<uint8_t>(last));
      } else {
        const int max_al = k == 1 ? 8 : 9;
        const int al = std::min(max_al, std::max(6, bit_length(ns)));
        ok = fse_normalize(cnt, last + 1, al, norm) && fse_describe(norm, last + 1, al, desc[k]);
        if (ok) own[k].reset(new ZFseEnc(norm, last + 1, al));
        mode[k] = 2;
      }
      t[k] = own[k].get();
    }
    if (!ok) continue;
    trial.clear();
    if (ns < 128) {
      trial.push_back(static_cast<uint8_t>(ns));
    } else if (ns < 0x7F00) {
      trial.push_back(static_cast<uint8_t>((ns >> 8) + 128));
      trial.push_back(static_cast<uint8_t>(ns));
    } else {
      trial.push_back(255);
      trial.push_back(static_cast<uint8_t>(ns - 0x7F00));
      trial.push_back(static_cast<uint8_t>((ns - 0x7F00) >> 8));
    }
    trial.push_back(static_cast<uint8_t>((mode[0] << 6) | (mode[1] << 4) | (mode[2] << 2)));
    for (int k = 0; k < 3; ++k) trial.insert(trial.end(), desc[k].begin(), desc[k].end());
    // the decoder reads, per sequence: offset, match-length and
    // literal-length extra bits, then (but after the last) the
    // literal-length, match-length and offset state bits; and first of all
    // the three initial states.  The stream is read from its end, so it is
    // written in exactly the reverse order, last sequence first.
    const ZFseEnc& tl = *t[0];
    const ZFseEnc& to = *t[1];
    const ZFseEnc& tm = *t[2];
    ZBitW w(trial);
    int sl = 0, so = 0, sm = 0;
    for (size_t i = ns; i-- > 0;) {
      const int lc = code[0][i], oc = code[1][i], mc = code[2][i];
      if (i + 1 == ns) {
        sl = tl.any_state(lc);
        sm = tm.any_state(mc);
        so = to.any_state(oc);
      } else {
        const int pl = tl.from[lc][sl], pm = tm.from[mc][sm], po = to.from[oc][so];
        w.put(so - to.base[po], to.nb[po]);
        w.put(sm - tm.base[pm], tm.nb[pm]);
        w.put(sl - tl.base[pl], tl.nb[pl]);
        sl = pl;
        sm = pm;
        so = po;
      }
      w.put(extra[0][i], nbx[0][i]);
      w.put(extra[2][i], nbx[2][i]);
      w.put(extra[1][i], nbx[1][i]);
    }
    w.put(sm, tm.al);
    w.put(so, to.al);
    w.put(sl, tl.al);
    w.finish();
    if (!have || trial.size() < best.size()) {
      best.swap(trial);
      have = true;
    }
  }
  if (!have) return false;
  body.insert(body.end(), best.begin(), best.end());
  if (body.size() >= raw) return false;
  rep[0] = r[0];
  rep[1] = r[1];
  rep[2] = r[2];
  return true;
}

void zstd_compress(const uint8_t* in, size_t n, Bytes& o) {
  o.clear();
  const uint32_t magic = 0xFD2FB528u;
  o.insert(o.end(), reinterpret_cast<const uint8_t*>(&magic), reinterpret_cast<const uint8_t*>(&magic) + 4);
  if (n < 256) {
    o.push_back(0x20);
    o.push_back(static_cast<uint8_t>(n));
  } else if (n < 65536 + 256) {
    o.push_back(0x60);
    o.push_back(static_cast<uint8_t>(n - 256));
    o.push_back(static_cast<uint8_t>((n - 256) >> 8));
  } else {
    o.push_back(0xA0);
    for (int k = 0; k < 4; ++k) o.push_back(static_cast<uint8_t>(n >> (8 * k)));
  }
  auto block_header = [&](size_t size, int type, bool last) {
    const uint32_t h = static_cast<uint32_t>((size << 3) | (type << 1) | (last ? 1 : 0));
    o.push_back(static_cast<uint8_t>(h));
    o.push_back(static_cast<uint8_t>(h >> 8));
    o.push_back(static_cast<uint8_t>(h >> 16));
  };
  if (n == 0) {
    block_header(0, 0, true);
    return;
  }
  const int kBits = 16;
  std::vector<int64_t> table(size_t(1) << kBits, -1);
  auto h4 = [&](size_t i) {
    uint32_t x;
    memcpy(&x, in + i, 4);
    return (x * 0x9E3779B1u) >> (32 - kBits);
  };
  std::vector<ZSeq> seqs;
  Bytes lits, body;
  uint32_t rep[3] = {1, 4, 8};
  size_t last_off = 0;
  const size_t kBlock = 128 * 1024;
  for (size_t b0 = 0; b0 < n; b0 += kBlock) {
    const size_t b1 = std::min(n, b0 + kBlock);
    const bool last = b1 == n;
    seqs.clear();
    lits.clear();
    size_t i = b0, lit = b0;
    while (i + 4 <= b1) {
      const uint32_t h = h4(i);
      int64_t cand = table[h];
      table[h] = static_cast<int64_t>(i);
      // the previous match's offset first: repeat offsets code cheaply
      if (last_off && i >= last_off && memcmp(in + i - last_off, in + i, 4) == 0)
        cand = static_cast<int64_t>(i - last_off);
      if (cand >= 0 && memcmp(in + cand, in + i, 4) == 0) {
        last_off = i - static_cast<size_t>(cand);
        size_t len = 4;
        while (i + len < b1 && in[cand + len] == in[i + len]) ++len;
        seqs.push_back({static_cast<uint32_t>(i - lit), static_cast<uint32_t>(i - cand), static_cast<uint32_t>(len)});
        lits.insert(lits.end(), in + lit, in + i);
        for (size_t k = i + 1; k < i + len && k + 4 <= b1; k += 3) table[h4(k)] = static_cast<int64_t>(k);
        i += len;
        lit = i;
      } else {
        ++i;
      }
    }
    lits.insert(lits.end(), in + lit, in + b1);
    const size_t raw = b1 - b0;
    bool same = true;
    for (size_t k = b0 + 1; k < b1 && same; ++k) same = in[k] == in[b0];
    if (same && raw > 1) {
      block_header(raw, 1, last);
      o.push_back(in[b0]);
    } else if (!seqs.empty() && zstd_block_body(seqs, lits, raw, body, rep)) {
      block_header(body.size(), 2, last);
      o.insert(o.end(), body.begin(), body.end());
    } else {
      block_header(raw, 0, last);
      o.insert(o.end(), in + b0, in + b1);
    }
  }
}

// ------------------------------------------------------------------ chunk encoder

struct ChunkOut {
  Bytes data;
  int64_t dict_off = -1;    // relative to the chunk start
  int64_t data_off = 0;
  int64_t total_unc = 0;
  int64_t total_cmp = 0;
  int codec = 0;
  std::vector<int> encodings;
  std::vector<std::array<int64_t, 3>> locations;  // (relative offset, size incl. header, first row)
  int64_t ba_bytes = -1;
  bool ok = true;
};

struct ColIn {
  const pq_write_column* c;
  int64_t r0, r1;
};

int type_width(int t) { return t == PQ_TYPE_INT32 || t == PQ_TYPE_FLOAT ? 4 : (t == PQ_TYPE_INT64 || t == PQ_TYPE_DOUBLE) ? 8 : 0; }

void page_header(Bytes& o, int type, int64_t unc, int64_t cmp, int sub, const std::vector<std::pair<int, int64_t>>& f,
                 int v2_bool = -1) {
  TW t(o);
  t.i32(1, type);
  t.i32(2, unc);
  t.i32(3, cmp);
  t.struct_begin(sub);
  for (auto& kv : f) t.i32(kv.first, kv.second);
  if (v2_bool >= 0) t.boolean(7, v2_bool != 0);
  t.struct_end();
  t.stop();
}

std::array<int64_t, 3> A3(int64_t a, int64_t b, int64_t c) { return {a, b, c}; }

void encode_chunk(const ColIn& in, int64_t page_bytes, int codec, ChunkOut* out) {
  const pq_write_column& c = *in.c;
  const int64_t n = in.r1 - in.r0;
  const int width = type_width(c.type);
  const bool optional = c.valid != nullptr;
  const bool is_ba = c.type == PQ_TYPE_BYTE_ARRAY;
  const uint8_t* valid = optional ? c.valid + in.r0 : nullptr;
  // non-null value indices (row ids) in order
  std::vector<int64_t> rows_nn;
  rows_nn.reserve(n);
  for (int64_t r = 0; r < n; ++r)
    if (!optional || valid[r]) rows_nn.push_back(r);
  auto fixed_bits = [&](int64_t r) -> uint64_t {
    const uint8_t* p = static_cast<const uint8_t*>(c.values) + (in.r0 + r) * width;
    uint64_t v = 0;
    memcpy(&v, p, width);
    return v;
  };
  const int64_t* offs = is_ba ? static_cast<const int64_t*>(c.values) + in.r0 : nullptr;
  auto str = [&](int64_t r, const uint8_t** p) -> int64_t {
    *p = c.chars + offs[r];
    return offs[r + 1] - offs[r];
  };
  if (is_ba) {
    int64_t s = 0;
    for (int64_t r : rows_nn) s += offs[r + 1] - offs[r];
    out->ba_bytes = s;
  }
  // dictionary
  const bool dict = c.encoding == 8 || c.encoding == 2;
  const bool delta = c.encoding == 5;
  std::vector<uint64_t> idx;  // per non-null value
  Bytes dict_body;
  int64_t dict_n = 0;
  int bw = 0;
  if (dict) {
    idx.resize(rows_nn.size());
    if (is_ba) {
      std::unordered_map<std::string, uint32_t> pos;
      pos.reserve(1024);
      for (size_t k = 0; k < rows_nn.size(); ++k) {
        const uint8_t* p;
        int64_t len = str(rows_nn[k], &p);
        std::string key(reinterpret_cast<const char*>(p), static_cast<size_t>(len));
        auto it = pos.find(key);
        if (it == pos.end()) {
          uint32_t id = static_cast<uint32_t>(pos.size());
          pos.emplace(key, id);
          uint32_t l = static_cast<uint32_t>(len);
          dict_body.insert(dict_body.end(), reinterpret_cast<uint8_t*>(&l), reinterpret_cast<uint8_t*>(&l) + 4);
          dict_body.insert(dict_body.end(), p, p + len);
          idx[k] = id;
        } else {
          idx[k] = it->second;
        }
      }
      dict_n = static_cast<int64_t>(pos.size());
    } else {
      std::unordered_map<uint64_t, uint32_t> pos;
      pos.reserve(1024);
      for (size_t k = 0; k < rows_nn.size(); ++k) {
        uint64_t v = fixed_bits(rows_nn[k]);
        auto it = pos.find(v);
        if (it == pos.end()) {
          uint32_t id = static_cast<uint32_t>(pos.size());
          pos.emplace(v, id);
          dict_body.insert(dict_body.end(), reinterpret_cast<uint8_t*>(&v), reinterpret_cast<uint8_t*>(&v) + width);
          idx[k] = id;
        } else {
          idx[k] = it->second;
        }
      }
      dict_n = static_cast<int64_t>(pos.size());
    }
    bw = bit_length(dict_n > 0 ? static_cast<uint64_t>(dict_n - 1) : 0);
  }
  DeltaEnc de{c.type == PQ_TYPE_INT32 ? 32 : 64};
  auto sval = [&](int64_t r) -> int64_t { return de.sgn(fixed_bits(r)); };
  // ---- page row counts
  std::vector<int64_t> counts;
  if (is_ba && !dict) {
    int64_t r = 0;
    while (r < n) {
      int64_t used = 0, rows = 0;
      while (r + rows < n) {
        int64_t rr = r + rows;
        int64_t cost = (!optional || valid[rr]) ? 4 + (offs[rr + 1] - offs[rr]) : 0;
        if (rows >= 8 && used + cost > page_bytes) break;
        used += cost;
        ++rows;
      }
      counts.push_back(rows);
      r += rows;
    }
  } else if (delta && !optional) {
    int64_t a = 0;
    std::vector<int64_t> d;
    while (a < n) {
      int64_t rem = n - a;
      if (rem <= 129) {
        counts.push_back(rem);
        break;
      }
      // size with k whole blocks: header(1 + 128k) + sum of block sizes
      auto hdr = [&](int64_t cnt) {
        Bytes t;
        de.header(t, static_cast<size_t>(cnt), sval(a));
        return static_cast<int64_t>(t.size());
      };
      auto blk = [&](int64_t j0, int64_t nd) {  // deltas j0.. (value index a+1+j0 ..)
        int64_t dd[128];
        for (int64_t q = 0; q < nd; ++q)
          dd[q] = de.sgn(static_cast<uint64_t>(sval(a + 1 + j0 + q)) - static_cast<uint64_t>(sval(a + j0 + q)));
        int64_t mn = *std::min_element(dd, dd + nd);
        int w[4] = {0, 0, 0, 0};
        for (int m = 0; m < 4; ++m) {
          uint64_t mx = 0;
          for (int64_t q = m * 32; q < std::min<int64_t>(nd, (m + 1) * 32); ++q)
            mx = std::max(mx, de.wrap(static_cast<uint64_t>(dd[q]) - static_cast<uint64_t>(mn)));
          w[m] = bit_length(mx);
        }
        return static_cast<int64_t>(DeltaEnc::block_size(mn, w, static_cast<size_t>(nd)));
      };
      int64_t k = 1;
      int64_t body = blk(0, 128);
      int64_t result = -1;
      while (1 + 128 * (k + 1) <= rem) {
        int64_t nxt = body + blk(128 * k, 128);
        if (hdr(1 + 128 * (k + 1)) + nxt > page_bytes) {
          result = 1 + 128 * k;
          break;
        }
        body = nxt;
        ++k;
      }
      if (result < 0) {
        // whole tail: remaining deltas after k blocks form one more (partial) block
        int64_t tail_deltas = rem - 1 - 128 * k;
        int64_t full = hdr(rem) + body + (tail_deltas > 0 ? blk(128 * k, tail_deltas) : 0);
        result = full <= page_bytes ? rem : 1 + 128 * k;
      }
      counts.push_back(result);
      a += result;
    }
  } else {
    int64_t bits = dict ? std::max(bw, 1) : 8 * width;
    if (optional) bits += 1;
    int64_t per = std::max<int64_t>(8, (page_bytes * 8 / bits) / 8 * 8);
    for (int64_t r = 0; r < n; r += per) counts.push_back(std::min(per, n - r));
  }
  // ---- build pages
  auto build = [&](int use_codec, ChunkOut* co) {
    co->data.clear();
    co->locations.clear();
    co->total_unc = co->total_cmp = 0;
    co->dict_off = -1;
    Bytes body, cbody, hdr;
    auto compress = [&](const Bytes& src, Bytes& dst) {
      if (use_codec == 1)
        snappy_compress(src.data(), src.size(), dst);
      else if (use_codec == 6)
        zstd_compress(src.data(), src.size(), dst);
      else
        dst = src;
    };
    if (dict) {
      compress(dict_body, cbody);
      hdr.clear();
      page_header(hdr, 2, static_cast<int64_t>(dict_body.size()), static_cast<int64_t>(cbody.size()), 7,
                  {{1, dict_n}, {2, 0}});
      co->dict_off = static_cast<int64_t>(co->data.size());
      co->data.insert(co->data.end(), hdr.begin(), hdr.end());
      co->data.insert(co->data.end(), cbody.begin(), cbody.end());
      co->total_unc += static_cast<int64_t>(hdr.size() + dict_body.size());
      co->total_cmp += static_cast<int64_t>(hdr.size() + cbody.size());
    }
    co->data_off = static_cast<int64_t>(co->data.size());
    int64_t row = 0;
    size_t vpos = 0;
    Bytes levels, vals;
    std::vector<uint64_t> tmp;
    for (int64_t cnt : counts) {
      // levels
      size_t nn = 0;
      levels.clear();
      if (optional) {
        tmp.resize(cnt);
        for (int64_t r = 0; r < cnt; ++r) {
          tmp[r] = valid[row + r] ? 1 : 0;
          nn += tmp[r];
        }
        hybrid_encode(levels, tmp.data(), tmp.size(), 1);
      } else {
        nn = static_cast<size_t>(cnt);
      }
      // values
      vals.clear();
      if (dict) {
        vals.push_back(static_cast<uint8_t>(bw));
        hybrid_encode(vals, idx.data() + vpos, nn, bw);
      } else if (delta) {
        de.header(vals, nn, nn ? sval(rows_nn[vpos]) : 0);
        int64_t dd[128];
        for (size_t b = 1; b < nn; b += 128) {
          size_t m = std::min<size_t>(128, nn - b);
          for (size_t q = 0; q < m; ++q)
            dd[q] = de.sgn(static_cast<uint64_t>(sval(rows_nn[vpos + b + q])) -
                           static_cast<uint64_t>(sval(rows_nn[vpos + b + q - 1])));
          de.block(vals, dd, m);
        }
      } else if (c.encoding == 9) {
        // BYTE_STREAM_SPLIT: stream b holds byte b of every value
        size_t base = vals.size();
        vals.resize(base + nn * width);
        for (size_t k = 0; k < nn; ++k) {
          const uint64_t v = fixed_bits(rows_nn[vpos + k]);
          for (int b = 0; b < width; ++b) vals[base + b * nn + k] = static_cast<uint8_t>(v >> (8 * b));
        }
      } else if (c.encoding == 6 || c.encoding == 7) {
        // DELTA_LENGTH_BYTE_ARRAY: lengths, then bytes; DELTA_BYTE_ARRAY:
        // prefix lengths against the previous value of the page, then the
        // suffixes as DELTA_LENGTH_BYTE_ARRAY
        std::vector<int64_t> pre(nn, 0), suf(nn);
        const uint8_t* prev = nullptr;
        int64_t prev_len = 0;
        for (size_t k = 0; k < nn; ++k) {
          const uint8_t* p;
          const int64_t len = str(rows_nn[vpos + k], &p);
          int64_t cp = 0;
          if (c.encoding == 7)
            while (cp < len && cp < prev_len && p[cp] == prev[cp]) ++cp;
          pre[k] = cp;
          suf[k] = len - cp;
          prev = p;
          prev_len = len;
        }
        if (c.encoding == 7) delta_stream32(vals, pre);
        delta_stream32(vals, suf);
        for (size_t k = 0; k < nn; ++k) {
          const uint8_t* p;
          str(rows_nn[vpos + k], &p);
          vals.insert(vals.end(), p + pre[k], p + pre[k] + suf[k]);
        }
      } else if (is_ba) {
        for (size_t k = 0; k < nn; ++k) {
          const uint8_t* p;
          int64_t len = str(rows_nn[vpos + k], &p);
          uint32_t l = static_cast<uint32_t>(len);
          vals.insert(vals.end(), reinterpret_cast<uint8_t*>(&l), reinterpret_cast<uint8_t*>(&l) + 4);
          vals.insert(vals.end(), p, p + len);
        }
      } else {
        size_t base = vals.size();
        vals.resize(base + nn * width);
        for (size_t k = 0; k < nn; ++k) {
          uint64_t v = fixed_bits(rows_nn[vpos + k]);
          memcpy(vals.data() + base + k * width, &v, width);
        }
      }
      const int enc = c.encoding == 2 ? 8 : c.encoding;
      hdr.clear();
      size_t page_start = co->data.size();
      if (c.page_version == 2) {
        compress(vals, cbody);
        const int64_t unc = static_cast<int64_t>(levels.size() + vals.size());
        const int64_t cmp = static_cast<int64_t>(levels.size() + cbody.size());
        page_header(hdr, 3, unc, cmp, 8,
                    {{1, cnt}, {2, cnt - static_cast<int64_t>(nn)}, {3, cnt}, {4, enc},
                     {5, static_cast<int64_t>(levels.size())}, {6, 0}},
                    use_codec != 0);
        co->data.insert(co->data.end(), hdr.begin(), hdr.end());
        co->data.insert(co->data.end(), levels.begin(), levels.end());
        co->data.insert(co->data.end(), cbody.begin(), cbody.end());
        co->total_unc += static_cast<int64_t>(hdr.size()) + unc;
        co->total_cmp += static_cast<int64_t>(hdr.size()) + cmp;
      } else {
        body.clear();
        if (optional) {
          uint32_t L = static_cast<uint32_t>(levels.size());
          body.insert(body.end(), reinterpret_cast<uint8_t*>(&L), reinterpret_cast<uint8_t*>(&L) + 4);
          body.insert(body.end(), levels.begin(), levels.end());
        }
        body.insert(body.end(), vals.begin(), vals.end());
        compress(body, cbody);
        page_header(hdr, 0, static_cast<int64_t>(body.size()), static_cast<int64_t>(cbody.size()), 5,
                    {{1, cnt}, {2, enc}, {3, 3}, {4, 3}});
        co->data.insert(co->data.end(), hdr.begin(), hdr.end());
        co->data.insert(co->data.end(), cbody.begin(), cbody.end());
        co->total_unc += static_cast<int64_t>(hdr.size() + body.size());
        co->total_cmp += static_cast<int64_t>(hdr.size() + cbody.size());
      }
      co->locations.push_back(A3(static_cast<int64_t>(page_start), static_cast<int64_t>(co->data.size() - page_start), row));
      row += cnt;
      vpos += nn;
    }
    co->codec = use_codec;
  };
  build(codec, out);
  if (codec != 0 && c.compress_threshold >= 0) {
    ChunkOut plain;
    build(0, &plain);
    if (static_cast<double>(out->total_cmp) > static_cast<double>(plain.total_cmp) * (1.0 - c.compress_threshold)) {
      plain.ba_bytes = out->ba_bytes;
      *out = std::move(plain);
    }
  }
  std::vector<int> encs = {c.encoding == 2 ? 8 : c.encoding};
  if (dict) encs.push_back(0);
  if (optional) encs.push_back(3);
  std::sort(encs.begin(), encs.end());
  encs.erase(std::unique(encs.begin(), encs.end()), encs.end());
  out->encodings = encs;
}

}  // namespace

extern "C" {

pq_status pq_write_table(const pq_write_column* cols, int n_cols, int64_t n_rows, int64_t rg_rows,
                         int64_t page_bytes, int offset_index, int n_threads, uint8_t** out, uint64_t* out_size) {
  if (!cols || n_cols <= 0 || n_rows < 0 || rg_rows <= 0 || page_bytes <= 0 || !out || !out_size)
    return PQ_ERR_INVALID_ARG;
  for (int c = 0; c < n_cols; ++c) {
    const auto& col = cols[c];
    const bool fixed = col.type == PQ_TYPE_INT32 || col.type == PQ_TYPE_INT64 || col.type == PQ_TYPE_DOUBLE ||
                       col.type == PQ_TYPE_FLOAT;
    if (!fixed && col.type != PQ_TYPE_BYTE_ARRAY) return PQ_ERR_UNSUPPORTED;
    const int e = col.encoding;
    if (e != -1 && e != 0 && e != 2 && e != 8 && e != 5 && e != 6 && e != 7 && e != 9) return PQ_ERR_UNSUPPORTED;
    if (e == 5 && col.type != PQ_TYPE_INT32 && col.type != PQ_TYPE_INT64) return PQ_ERR_INVALID_ARG;
    if ((e == 6 || e == 7) && col.type != PQ_TYPE_BYTE_ARRAY) return PQ_ERR_INVALID_ARG;
    if (e == 9 && !fixed) return PQ_ERR_INVALID_ARG;
    if (col.codec != 0 && col.codec != 1 && col.codec != 6) return PQ_ERR_UNSUPPORTED;
    if (col.page_version != 1 && col.page_version != 2) return PQ_ERR_INVALID_ARG;
    if (!col.values && n_rows > 0) return PQ_ERR_INVALID_ARG;
    if (col.type == PQ_TYPE_BYTE_ARRAY && !col.chars && n_rows > 0) return PQ_ERR_INVALID_ARG;
  }
  const int64_t n_rg = n_rows == 0 ? 0 : (n_rows + rg_rows - 1) / rg_rows;
  std::vector<ColIn> jobs;
  for (int64_t g = 0; g < n_rg; ++g)
    for (int c = 0; c < n_cols; ++c) jobs.push_back({&cols[c], g * rg_rows, std::min(n_rows, (g + 1) * rg_rows)});
  std::vector<ChunkOut> chunks(jobs.size());
  int nt = n_threads > 0 ? n_threads : static_cast<int>(std::thread::hardware_concurrency());
  nt = std::max(1, std::min<int>(nt, static_cast<int>(jobs.size())));
  std::atomic<size_t> next{0};
  // encoding -1: the chunk keeps the valid encoding of its type with the
  // smallest encoded (uncompressed) size; ties go to the earlier candidate
  std::vector<pq_write_column> chosen(jobs.size());
  auto worker = [&]() {
    for (size_t j; (j = next.fetch_add(1)) < jobs.size();) {
      if (jobs[j].c->encoding != -1) {
        encode_chunk(jobs[j], page_bytes, jobs[j].c->codec, &chunks[j]);
        continue;
      }
      static const int kInt[] = {0, 8, 5, 9}, kFloat[] = {0, 8, 9}, kStr[] = {0, 8, 6, 7};
      const int t = jobs[j].c->type;
      const int* cand = t == PQ_TYPE_BYTE_ARRAY ? kStr : (t == PQ_TYPE_INT32 || t == PQ_TYPE_INT64) ? kInt : kFloat;
      const int n_cand = t == PQ_TYPE_DOUBLE || t == PQ_TYPE_FLOAT ? 3 : 4;
      int best = -1;
      int64_t best_size = 0;
      for (int k = 0; k < n_cand; ++k) {
        pq_write_column trial = *jobs[j].c;
        trial.encoding = cand[k];
        ChunkOut co;
        encode_chunk(ColIn{&trial, jobs[j].r0, jobs[j].r1}, page_bytes, 0, &co);
        if (best < 0 || co.total_unc < best_size) {
          best = cand[k];
          best_size = co.total_unc;
        }
      }
      chosen[j] = *jobs[j].c;
      chosen[j].encoding = best;
      encode_chunk(ColIn{&chosen[j], jobs[j].r0, jobs[j].r1}, page_bytes, chosen[j].codec, &chunks[j]);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(worker);
  worker();
  for (auto& t : th) t.join();
  // assemble
  Bytes file = {'P', 'A', 'R', '1'};
  std::vector<int64_t> start(jobs.size());
  size_t total = 4;
  for (auto& ch : chunks) total += ch.data.size();
  file.reserve(total + 1024 + jobs.size() * 64);
  for (size_t j = 0; j < jobs.size(); ++j) {
    start[j] = static_cast<int64_t>(file.size());
    file.insert(file.end(), chunks[j].data.begin(), chunks[j].data.end());
    Bytes().swap(chunks[j].data);
  }
  std::vector<std::pair<int64_t, int64_t>> oi(jobs.size(), {-1, 0});
  if (offset_index) {
    for (size_t j = 0; j < jobs.size(); ++j) {
      Bytes b;
      TW t(b);
      t.list_begin(1, 12, chunks[j].locations.size());
      for (auto& l : chunks[j].locations) {
        t.elem_struct_begin();
        t.i64(1, start[j] + l[0]);
        t.i32(2, l[1]);
        t.i64(3, l[2]);
        t.struct_end();
      }
      t.stop();
      oi[j] = {static_cast<int64_t>(file.size()), static_cast<int64_t>(b.size())};
      file.insert(file.end(), b.begin(), b.end());
    }
  }
  Bytes f;
  TW t(f);
  t.i32(1, 2);
  t.list_begin(2, 12, static_cast<size_t>(n_cols) + 1);
  t.elem_struct_begin();
  t.binary(4, "schema");
  t.i32(5, n_cols);
  t.struct_end();
  for (int c = 0; c < n_cols; ++c) {
    t.elem_struct_begin();
    t.i32(1, cols[c].type);
    t.i32(3, cols[c].valid ? 1 : 0);
    t.binary(4, cols[c].name ? cols[c].name : "");
    t.struct_end();
  }
  t.i64(3, n_rows);
  t.list_begin(4, 12, static_cast<size_t>(n_rg));
  for (int64_t g = 0; g < n_rg; ++g) {
    int64_t unc = 0, cmp = 0;
    for (int c = 0; c < n_cols; ++c) {
      unc += chunks[g * n_cols + c].total_unc;
      cmp += chunks[g * n_cols + c].total_cmp;
    }
    t.elem_struct_begin();
    t.list_begin(1, 12, n_cols);
    for (int c = 0; c < n_cols; ++c) {
      const size_t j = static_cast<size_t>(g * n_cols + c);
      const ChunkOut& ch = chunks[j];
      t.elem_struct_begin();
      t.i64(2, start[j]);
      t.struct_begin(3);
      t.i32(1, cols[c].type);
      t.list_begin(2, 5, ch.encodings.size());
      for (int e : ch.encodings) t.varint(TW::zz(e));
      t.list_begin(3, 8, 1);
      std::string name = cols[c].name ? cols[c].name : "";
      t.varint(name.size());
      f.insert(f.end(), name.begin(), name.end());
      t.i32(4, ch.codec);
      t.i64(5, jobs[j].r1 - jobs[j].r0);
      t.i64(6, ch.total_unc);
      t.i64(7, ch.total_cmp);
      t.i64(9, start[j] + ch.data_off);
      if (ch.dict_off >= 0) t.i64(11, start[j] + ch.dict_off);
      if (cols[c].type == PQ_TYPE_BYTE_ARRAY) {
        t.struct_begin(16);
        t.i64(1, ch.ba_bytes);
        t.struct_end();
      }
      t.struct_end();
      if (offset_index) {
        t.i64(4, oi[j].first);
        t.i32(5, oi[j].second);
      }
      t.struct_end();
    }
    t.i64(2, unc);
    t.i64(3, jobs[g * n_cols].r1 - jobs[g * n_cols].r0);
    t.i64(5, start[g * n_cols]);
    t.i64(6, cmp);
    t.i16(7, g);
    t.struct_end();
  }
  t.binary(6, "pqscan-gb300");
  t.stop();
  file.insert(file.end(), f.begin(), f.end());
  uint32_t fl = static_cast<uint32_t>(f.size());
  file.insert(file.end(), reinterpret_cast<uint8_t*>(&fl), reinterpret_cast<uint8_t*>(&fl) + 4);
  file.insert(file.end(), {'P', 'A', 'R', '1'});
  uint8_t* buf = static_cast<uint8_t*>(malloc(file.size()));
  if (!buf) return PQ_ERR_OOM;
  memcpy(buf, file.data(), file.size());
  *out = buf;
  *out_size = file.size();
  return PQ_OK;
}

void pq_write_free(uint8_t* buf) { free(buf); }

}  // extern "C"
