// Zstandard frame decoding core (the codec the paper's Section 2 lists
// beside Snappy for Parquet column chunks), written as host/device
// functions over plain pointers so that the same code runs in a kernel and
// in a host test harness.
//
// Format steps, in order: frame header (magic 0xFD2FB528; descriptor with
// content-size, single-segment, checksum and dictionary flags; window
// descriptor; content size) -> blocks (3-byte header: last bit, type, size;
// raw, RLE or compressed) -> a compressed block is a literals section (raw,
// RLE, or Huffman-coded in 1 or 4 backward bitstreams, with a new or the
// previous table) and a sequences section (literal-length, offset and
// match-length codes from FSE tables that are predefined, RLE, transmitted
// or repeated; extra bits; three repeat offsets) -> the sequences are
// executed against the output.  Skippable frames are skipped, checksums are
// not verified, dictionaries are rejected.
//
// Memory: the output buffer also holds each block's literals, decoded into
// its tail; the sequences then read them from there while the output grows
// towards them (the output never passes the unread literals unless the
// block would overflow the page, which is reported).
#pragma once
#include <stdint.h>

#include "pq_internal.h"

namespace pqi {

struct ZFse {
  uint8_t sym;
  uint8_t nbits;
  uint16_t base;
};

// Decoder state of one frame (tables persist across its blocks).
struct ZState {
  uint16_t huf[1 << 11];  // (code bits << 8) | symbol, indexed by the next max_bits bits
  ZFse ll[1 << 9];
  ZFse of[1 << 8];
  ZFse ml[1 << 9];
  ZFse hw[1 << 6];        // table of the Huffman weights being read
  int32_t huf_bits;       // max code bits of the current Huffman table, 0: none yet
  int32_t ll_al, of_al, ml_al;  // accuracy logs, -1: no table yet
  uint32_t rep[3];
  int16_t norm[64];
  uint16_t next[64];
  uint8_t weights[256];
};

enum : int {
  ZE_OK = 0, ZE_MAGIC = 1, ZE_HEADER = 2, ZE_DICT = 3, ZE_TRUNC = 4, ZE_BLOCK = 5, ZE_LIT = 6, ZE_HUF = 7,
  ZE_FSE = 8, ZE_SEQ = 9, ZE_OFFSET = 10, ZE_SIZE = 11, ZE_STREAM = 12
};

PQ_HD inline int z_hb(uint32_t x) {  // index of the highest set bit, x > 0
#if defined(__CUDA_ARCH__)
  return 31 - __clz(x);
#else
  return 31 - __builtin_clz(x);
#endif
}

// Bits written backwards: the last byte carries a 1 marker above the data;
// reading starts just below it.  `pos` counts the unread bits; reading past
// the first byte yields zeros and drives pos below 0.
struct ZBack {
  const uint8_t* p;
  int64_t pos;
};

PQ_HD inline bool zb_init(ZBack& b, const uint8_t* p, uint32_t len) {
  if (len == 0 || p[len - 1] == 0) return false;
  b.p = p;
  b.pos = static_cast<int64_t>(len - 1) * 8 + z_hb(p[len - 1]);
  return true;
}

PQ_HD inline uint32_t zb_peek(const ZBack& b, int n) {  // n <= 32
  if (n == 0 || b.pos <= 0) return 0;
  int64_t lo = b.pos - n;
  int sh = 0;
  int take = n;
  if (lo < 0) {
    sh = static_cast<int>(-lo);
    take = static_cast<int>(b.pos);
    lo = 0;
  }
  const int64_t b0 = lo >> 3, b1 = (lo + take - 1) >> 3;
  uint64_t v = 0;
  for (int64_t i = b1; i >= b0; --i) v = (v << 8) | b.p[i];
  v >>= (lo & 7);
  v &= (take >= 64 ? ~0ull : ((1ull << take) - 1));
  return static_cast<uint32_t>(v << sh);
}

PQ_HD inline uint32_t zb_read(ZBack& b, int n) {
  const uint32_t v = zb_peek(b, n);
  b.pos -= n;
  return v;
}

// ------------------------------------------------------------------ FSE

// Normalized counts of a table description at p[0, len).  Returns 0 or an
// error; *used = bytes consumed.
PQ_HD inline int z_read_norm(const uint8_t* p, uint32_t len, int max_al, int max_sym, int16_t* norm, int* nsym,
                             int* al, uint32_t* used) {
  uint32_t bit = 0;
  auto peek = [&](int n) -> uint32_t {
    uint64_t v = 0;
    const uint32_t b0 = bit >> 3;
    for (int i = 0; i < 5; ++i)
      if (b0 + i < len) v |= static_cast<uint64_t>(p[b0 + i]) << (8 * i);
    return static_cast<uint32_t>((v >> (bit & 7)) & ((1ull << n) - 1));
  };
  auto skip = [&](int n) -> bool {
    bit += n;
    return (bit + 7) / 8 <= len;
  };
  if (len == 0) return ZE_FSE;
  const int a = static_cast<int>(peek(4)) + 5;
  if (!skip(4) || a > max_al) return ZE_FSE;
  int32_t remaining = 1 << a;
  int s = 0;
  while (remaining > 0) {
    if (s >= max_sym) return ZE_FSE;
    const uint32_t nv = static_cast<uint32_t>(remaining) + 2;  // values 0 .. remaining + 1
    int nbits = z_hb(nv - 1) + 1;                              // 2^nbits >= nv
    const uint32_t spare = (1u << nbits) - nv;
    uint32_t value;
    const uint32_t low = peek(nbits - 1);
    if (low < spare) {
      value = low;
      if (!skip(nbits - 1)) return ZE_FSE;
    } else {
      value = peek(nbits);
      if (value >= (1u << (nbits - 1))) value -= spare;
      if (!skip(nbits)) return ZE_FSE;
    }
    const int prob = static_cast<int>(value) - 1;
    norm[s++] = static_cast<int16_t>(prob);
    remaining -= prob == -1 ? 1 : prob;
    if (prob == 0) {
      for (;;) {
        const uint32_t rep = peek(2);
        if (!skip(2)) return ZE_FSE;
        for (uint32_t r = 0; r < rep; ++r) {
          if (s >= max_sym) return ZE_FSE;
          norm[s++] = 0;
        }
        if (rep != 3) break;
      }
    }
  }
  if (remaining < 0) return ZE_FSE;
  *nsym = s;
  *al = a;
  *used = (bit + 7) / 8;
  return ZE_OK;
}

PQ_HD inline int z_build_fse(const int16_t* norm, int nsym, int al, uint16_t* next, ZFse* t) {
  const int size = 1 << al;
  int high = size - 1;
  for (int s = 0; s < nsym; ++s) {
    if (norm[s] == -1) {
      if (high < 0) return ZE_FSE;
      t[high--].sym = static_cast<uint8_t>(s);
      next[s] = 1;
    } else {
      next[s] = static_cast<uint16_t>(norm[s]);
    }
  }
  const int step = (size >> 1) + (size >> 3) + 3, mask = size - 1;
  int pos = 0;
  for (int s = 0; s < nsym; ++s) {
    for (int i = 0; i < norm[s]; ++i) {
      t[pos].sym = static_cast<uint8_t>(s);
      int guard = 0;
      do {
        pos = (pos + step) & mask;
      } while (pos > high && ++guard <= size);
      if (guard > size) return ZE_FSE;
    }
  }
  if (pos != 0) return ZE_FSE;
  for (int st = 0; st < size; ++st) {
    const uint32_t x = next[t[st].sym]++;
    const int nb = al - z_hb(x);
    t[st].nbits = static_cast<uint8_t>(nb);
    t[st].base = static_cast<uint16_t>((x << nb) - size);
  }
  return ZE_OK;
}

// Predefined distributions of the format.
PQ_HD inline void z_default_norm(int which, int16_t* norm, int* nsym, int* al) {
  // 0 literal lengths, 1 offsets, 2 match lengths
  const int8_t LL[36] = {4, 3, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 3, 2, 1, 1, 1, 1, 1,
                         -1, -1, -1, -1};
  const int8_t OF[29] = {1, 1, 1, 1, 1, 1, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1};
  const int8_t ML[53] = {1, 4, 3, 2, 2, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                         1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1, -1};
  const int8_t* src = which == 0 ? LL : which == 1 ? OF : ML;
  *nsym = which == 0 ? 36 : which == 1 ? 29 : 53;
  *al = which == 1 ? 5 : 6;
  for (int i = 0; i < *nsym; ++i) norm[i] = src[i];
}

// ------------------------------------------------------------------ Huffman

// Table from `n` transmitted weights (the last symbol's weight is implied).
PQ_HD inline int z_build_huf(uint8_t* w, int n, ZState* z) {
  uint32_t total = 0;
  for (int s = 0; s < n; ++s) {
    if (w[s] > 11) return ZE_HUF;
    if (w[s]) total += 1u << (w[s] - 1);
  }
  if (total == 0) return ZE_HUF;
  const int mb = z_hb(total) + 1;
  const uint32_t rest = (1u << mb) - total;
  if (mb > 11 || (rest & (rest - 1)) || n >= 256) return ZE_HUF;
  w[n] = static_cast<uint8_t>(z_hb(rest) + 1);
  const int ns = n + 1;
  uint32_t idx = 0;
  for (int wt = 1; wt <= mb; ++wt)
    for (int s = 0; s < ns; ++s)
      if (w[s] == wt) {
        const uint16_t e = static_cast<uint16_t>(((mb + 1 - wt) << 8) | s);
        const uint32_t span = 1u << (wt - 1);
        if (idx + span > (1u << mb)) return ZE_HUF;
        for (uint32_t k = 0; k < span; ++k) z->huf[idx++] = e;
      }
  if (idx != (1u << mb)) return ZE_HUF;
  z->huf_bits = mb;
  return ZE_OK;
}

// Huffman tree description at p[0, len): returns 0 or an error; *used bytes.
PQ_HD inline int z_read_huf(const uint8_t* p, uint32_t len, ZState* z, uint32_t* used) {
  if (len == 0) return ZE_HUF;
  const uint32_t head = p[0];
  int n = 0;
  if (head >= 128) {
    n = static_cast<int>(head) - 127;
    const uint32_t nbytes = (n + 1) / 2;
    if (1 + nbytes > len) return ZE_HUF;
    for (int i = 0; i < n; ++i) {
      const uint8_t b = p[1 + i / 2];
      z->weights[i] = (i & 1) ? (b & 15) : (b >> 4);
    }
    *used = 1 + nbytes;
  } else {
    const uint32_t size = head;
    if (size == 0 || 1 + size > len) return ZE_HUF;
    int nsym, al;
    uint32_t u;
    if (z_read_norm(p + 1, size, 6, 16, z->norm, &nsym, &al, &u)) return ZE_HUF;
    ZFse* t = z->hw;
    if (z_build_fse(z->norm, nsym, al, z->next, t)) return ZE_HUF;
    ZBack b;
    if (!zb_init(b, p + 1 + u, size - u)) return ZE_HUF;
    uint32_t s1 = zb_read(b, al), s2 = zb_read(b, al);
    for (;;) {
      if (n > 253) return ZE_HUF;
      z->weights[n++] = t[s1].sym;
      s1 = t[s1].base + zb_read(b, t[s1].nbits);
      if (b.pos < 0) {
        z->weights[n++] = t[s2].sym;
        break;
      }
      z->weights[n++] = t[s2].sym;
      s2 = t[s2].base + zb_read(b, t[s2].nbits);
      if (b.pos < 0) {
        z->weights[n++] = t[s1].sym;
        break;
      }
    }
    *used = 1 + size;
  }
  return z_build_huf(z->weights, n, z);
}

PQ_HD inline int z_huf_stream(const uint8_t* p, uint32_t len, uint32_t count, const ZState* z, uint8_t* out) {
  ZBack b;
  if (!zb_init(b, p, len)) return ZE_STREAM;
  const int mb = z->huf_bits;
  for (uint32_t i = 0; i < count; ++i) {
    const uint16_t e = z->huf[zb_peek(b, mb)];
    b.pos -= e >> 8;
    out[i] = static_cast<uint8_t>(e & 0xff);
  }
  return b.pos == 0 ? ZE_OK : ZE_STREAM;
}

// ------------------------------------------------------------------ blocks

PQ_HD inline uint32_t z_le(const uint8_t* p, int n) {
  uint32_t v = 0;
  for (int i = n - 1; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}

// The Huffman streams of a literals section: 1 stream, or 4 after a jump
// table of three 2-byte sizes, each stream decoding (n + 3) / 4 literals
// (the last one the rest).  Independent of one another: one decoder each.
struct ZHufStreams {
  const uint8_t* p[4];
  uint32_t len[4];
  uint32_t cnt[4];
  uint32_t out[4];  // offset of the stream's literals within the section's
  int n;
};

PQ_HD inline int z_huf_split(const uint8_t* q, uint32_t qlen, uint32_t regen, int streams, ZHufStreams* hs) {
  if (streams == 1) {
    hs->n = 1;
    hs->p[0] = q;
    hs->len[0] = qlen;
    hs->cnt[0] = regen;
    hs->out[0] = 0;
    return ZE_OK;
  }
  if (qlen < 6) return ZE_LIT;
  const uint32_t s1 = z_le(q, 2), s2 = z_le(q + 2, 2), s3 = z_le(q + 4, 2);
  if (6ull + s1 + s2 + s3 > qlen) return ZE_LIT;
  const uint32_t per = (regen + 3) / 4;
  if (3 * per > regen) return ZE_LIT;
  const uint32_t lens[4] = {s1, s2, s3, qlen - 6 - s1 - s2 - s3};
  const uint8_t* sp = q + 6;
  hs->n = 4;
  for (int k = 0; k < 4; ++k) {
    hs->p[k] = sp;
    hs->len[k] = lens[k];
    hs->cnt[k] = k < 3 ? per : regen - 3 * per;
    hs->out[k] = static_cast<uint32_t>(k) * per;
    sp += lens[k];
  }
  return ZE_OK;
}

// Literals of a compressed block at p[0, len), decoded to dst[lit0, lit0 +
// *nlit) (lit0 chosen here: the tail of the output).  Returns 0 or an error;
// *used = section bytes.
PQ_HD inline int z_literals(const uint8_t* p, uint32_t len, ZState* z, uint8_t* dst, uint64_t out_pos,
                            uint64_t dst_len, uint64_t* lit0, uint32_t* nlit, uint32_t* used) {
  if (len == 0) return ZE_LIT;
  const uint32_t b0 = p[0], type = b0 & 3, sf = (b0 >> 2) & 3;
  uint32_t regen, hlen;
  if (type < 2) {
    if (sf == 0 || sf == 2) {
      regen = b0 >> 3;
      hlen = 1;
    } else if (sf == 1) {
      if (len < 2) return ZE_LIT;
      regen = (b0 >> 4) + (static_cast<uint32_t>(p[1]) << 4);
      hlen = 2;
    } else {
      if (len < 3) return ZE_LIT;
      regen = (b0 >> 4) + (static_cast<uint32_t>(p[1]) << 4) + (static_cast<uint32_t>(p[2]) << 12);
      hlen = 3;
    }
    if (regen > dst_len - out_pos) return ZE_SIZE;
    *lit0 = dst_len - regen;
    *nlit = regen;
    if (type == 0) {
      if (hlen + regen > len) return ZE_LIT;
      uint32_t i = 0;
      for (; i + 16 <= regen; i += 16) {  // 16 loads in flight, then the stores
        uint8_t t[16];
        for (int k = 0; k < 16; ++k) t[k] = p[hlen + i + k];
        for (int k = 0; k < 16; ++k) dst[*lit0 + i + k] = t[k];
      }
      for (; i < regen; ++i) dst[*lit0 + i] = p[hlen + i];
      *used = hlen + regen;
    } else {
      if (hlen + 1 > len) return ZE_LIT;
      for (uint32_t i = 0; i < regen; ++i) dst[*lit0 + i] = p[hlen];
      *used = hlen + 1;
    }
    return ZE_OK;
  }
  const uint32_t bits = sf < 2 ? 10 : sf == 2 ? 14 : 18;
  hlen = sf < 2 ? 3 : sf == 2 ? 4 : 5;
  const int streams = sf == 0 ? 1 : 4;
  if (len < hlen) return ZE_LIT;
  uint64_t h = 0;
  for (int i = static_cast<int>(hlen) - 1; i >= 0; --i) h = (h << 8) | p[i];
  regen = static_cast<uint32_t>((h >> 4) & ((1u << bits) - 1));
  const uint32_t csize = static_cast<uint32_t>((h >> (4 + bits)) & ((1u << bits) - 1));
  if (hlen + csize > len) return ZE_LIT;
  if (regen > dst_len - out_pos) return ZE_SIZE;
  const uint8_t* q = p + hlen;
  uint32_t qlen = csize;
  if (type == 2) {
    uint32_t u;
    const int e = z_read_huf(q, qlen, z, &u);
    if (e) return e;
    q += u;
    qlen -= u;
  } else if (z->huf_bits == 0) {
    return ZE_HUF;
  }
  *lit0 = dst_len - regen;
  *nlit = regen;
  ZHufStreams hs;
  const int e = z_huf_split(q, qlen, regen, streams, &hs);
  if (e) return e;
  for (int k = 0; k < hs.n; ++k) {
    const int e2 = z_huf_stream(hs.p[k], hs.len[k], hs.cnt[k], z, dst + *lit0 + hs.out[k]);
    if (e2) return e2;
  }
  *used = hlen + csize;
  return ZE_OK;
}

PQ_HD inline int z_table(const uint8_t* p, uint32_t len, int mode, int which, ZState* z, uint32_t* used) {
  ZFse* t = which == 0 ? z->ll : which == 1 ? z->of : z->ml;
  int32_t* al = which == 0 ? &z->ll_al : which == 1 ? &z->of_al : &z->ml_al;
  const int max_al = which == 1 ? 8 : 9;
  const int max_sym = which == 0 ? 36 : which == 1 ? 32 : 53;
  *used = 0;
  if (mode == 0) {
    int nsym, a;
    z_default_norm(which, z->norm, &nsym, &a);
    if (z_build_fse(z->norm, nsym, a, z->next, t)) return ZE_FSE;
    *al = a;
  } else if (mode == 1) {
    if (len < 1 || p[0] >= max_sym) return ZE_SEQ;
    t[0].sym = p[0];
    t[0].nbits = 0;
    t[0].base = 0;
    *al = 0;
    *used = 1;
  } else if (mode == 2) {
    int nsym, a;
    if (z_read_norm(p, len, max_al, max_sym, z->norm, &nsym, &a, used)) return ZE_FSE;
    if (z_build_fse(z->norm, nsym, a, z->next, t)) return ZE_FSE;
    *al = a;
  } else if (*al < 0) {
    return ZE_SEQ;
  }
  return ZE_OK;
}

PQ_HD inline void z_ll(uint32_t code, uint32_t* base, int* bits) {
  if (code < 16) {
    *base = code;
    *bits = 0;
    return;
  }
  const uint16_t B[20] = {16, 18, 20, 22, 24, 28, 32, 40, 48, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384,
                          32768, 0};
  const uint8_t N[20] = {1, 1, 1, 1, 2, 2, 3, 3, 4, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16};
  *base = code == 35 ? 65536u : B[code - 16];
  *bits = N[code - 16];
}

PQ_HD inline void z_ml(uint32_t code, uint32_t* base, int* bits) {
  if (code < 32) {
    *base = code + 3;
    *bits = 0;
    return;
  }
  const uint32_t B[21] = {35, 37, 39, 41, 43, 47, 51, 59, 67, 83, 99, 131, 259, 515, 1027, 2051, 4099, 8195,
                          16387, 32771, 65539};
  const uint8_t N[21] = {1, 1, 1, 1, 2, 2, 3, 3, 4, 4, 5, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16};
  *base = B[code - 32];
  *bits = N[code - 32];
}

// Sequence decoding in steps, so that a caller can decode a batch of
// sequences and execute them separately: z_seq_begin parses the section
// header and tables and reads the initial states; z_seq_next decodes one
// sequence (its literal length, offset and match length, the offset resolved
// through the repeat-offset history); z_exec copies one sequence's literals
// and match into the output.
struct ZSeqState {
  ZBack b;
  uint32_t sl, so, sm;
  uint32_t nseq, done;
};

PQ_HD inline int z_seq_begin(const uint8_t* p, uint32_t len, ZState* z, ZSeqState* s) {
  if (len == 0) return ZE_SEQ;
  uint32_t q;
  const uint32_t b0 = p[0];
  s->done = 0;
  if (b0 == 0) {
    if (len != 1) return ZE_SEQ;
    s->nseq = 0;
    return ZE_OK;
  } else if (b0 < 128) {
    s->nseq = b0;
    q = 1;
  } else if (b0 < 255) {
    if (len < 2) return ZE_SEQ;
    s->nseq = ((b0 - 128) << 8) + p[1];
    q = 2;
  } else {
    if (len < 3) return ZE_SEQ;
    s->nseq = p[1] + (static_cast<uint32_t>(p[2]) << 8) + 0x7F00;
    q = 3;
  }
  if (q >= len) return ZE_SEQ;
  const uint32_t modes = p[q++];
  if (modes & 3) return ZE_SEQ;
  const int ms[3] = {static_cast<int>(modes >> 6), static_cast<int>((modes >> 4) & 3),
                     static_cast<int>((modes >> 2) & 3)};
  for (int which = 0; which < 3; ++which) {
    uint32_t u;
    const int e = z_table(p + q, len - q, ms[which], which, z, &u);
    if (e) return e;
    q += u;
  }
  if (!zb_init(s->b, p + q, len - q)) return ZE_SEQ;
  s->sl = zb_read(s->b, z->ll_al);
  s->so = zb_read(s->b, z->of_al);
  s->sm = zb_read(s->b, z->ml_al);
  return ZE_OK;
}

PQ_HD inline int z_seq_next(ZState* z, ZSeqState* s, uint32_t* ll_out, uint32_t* off_out, uint32_t* ml_out) {
  const uint32_t of_code = z->of[s->so].sym, ml_code = z->ml[s->sm].sym, ll_code = z->ll[s->sl].sym;
  if (of_code > 31 || ll_code > 35 || ml_code > 52) return ZE_SEQ;
  const uint32_t ov = (1u << of_code) + zb_read(s->b, static_cast<int>(of_code));
  uint32_t mbase, lbase;
  int mbits, lbits;
  z_ml(ml_code, &mbase, &mbits);
  z_ll(ll_code, &lbase, &lbits);
  const uint32_t ml = mbase + zb_read(s->b, mbits);
  const uint32_t ll = lbase + zb_read(s->b, lbits);
  if (++s->done < s->nseq) {
    s->sl = z->ll[s->sl].base + zb_read(s->b, z->ll[s->sl].nbits);
    s->sm = z->ml[s->sm].base + zb_read(s->b, z->ml[s->sm].nbits);
    s->so = z->of[s->so].base + zb_read(s->b, z->of[s->so].nbits);
  }
  uint32_t off;
  if (ov > 3) {
    off = ov - 3;
    z->rep[2] = z->rep[1];
    z->rep[1] = z->rep[0];
    z->rep[0] = off;
  } else {
    const uint32_t idx = ll > 0 ? ov - 1 : ov;  // with no literals the repeat index shifts by one
    if (idx == 0) {
      off = z->rep[0];
    } else if (idx == 1) {
      off = z->rep[1];
      z->rep[1] = z->rep[0];
      z->rep[0] = off;
    } else if (idx == 2) {
      off = z->rep[2];
      z->rep[2] = z->rep[1];
      z->rep[1] = z->rep[0];
      z->rep[0] = off;
    } else {
      off = z->rep[0] - 1;
      z->rep[2] = z->rep[1];
      z->rep[1] = z->rep[0];
      z->rep[0] = off;
    }
  }
  *ll_out = ll;
  *off_out = off;
  *ml_out = ml;
  return ZE_OK;
}

// dst[d, d + n) = dst[s, s + n), with the result of a byte-by-byte forward
// copy.  When the source lies ahead of the destination, or at least 16
// bytes behind it, no byte of a 16-byte step is written before it is read,
// so each step loads its 16 bytes before storing them: one thread keeps 16
// loads in flight instead of one (the output was just written and is read
// back from L2).  A nearer source (an overlapping match) goes byte by byte.
PQ_HD inline void z_copy(uint8_t* dst, uint64_t d, uint64_t s, uint32_t n) {
  uint32_t k = 0;
  if (s > d || d - s >= 16) {
    for (; k + 16 <= n; k += 16) {
      uint8_t t[16];
      for (int i = 0; i < 16; ++i) t[i] = dst[s + k + i];
      for (int i = 0; i < 16; ++i) dst[d + k + i] = t[i];
    }
  }
  for (; k < n; ++k) dst[d + k] = dst[s + k];
}

// One sequence into dst: ll literals from the block's literals at *r (which
// end at lit_end, ahead of the output), then ml bytes from `off` back (a
// match may overlap its own output).  The frame's output starts at out0.
PQ_HD inline int z_exec(uint8_t* dst, uint64_t* w, uint64_t* r, uint64_t lit_end, uint64_t out0, uint32_t ll,
                        uint32_t off, uint32_t ml) {
  if (*r + ll > lit_end) return ZE_SEQ;
  z_copy(dst, *w, *r, ll);
  *w += ll;
  *r += ll;
  if (off == 0 || off > *w - out0) return ZE_OFFSET;
  if (*w + ml > *r) return ZE_SIZE;  // the output would run into unread literals: the page is too small
  z_copy(dst, *w, *w - off, ml);
  *w += ml;
  return ZE_OK;
}

// Sequences section at p[0, len), executed into dst (output so far ends at
// *out_pos; the block's literals at dst[lit0, lit0 + nlit)).
PQ_HD inline int z_sequences(const uint8_t* p, uint32_t len, ZState* z, uint8_t* dst, uint64_t* out_pos,
                             uint64_t out0, uint64_t lit0, uint32_t nlit) {
  ZSeqState s;
  int e = z_seq_begin(p, len, z, &s);
  if (e) return e;
  uint64_t w = *out_pos, r = lit0;
  const uint64_t lit_end = lit0 + nlit;
  for (uint32_t i = 0; i < s.nseq; ++i) {
    uint32_t ll, off, ml;
    e = z_seq_next(z, &s, &ll, &off, &ml);
    if (e) return e;
    e = z_exec(dst, &w, &r, lit_end, out0, ll, off, ml);
    if (e) return e;
  }
  if (s.nseq && s.b.pos != 0) return ZE_STREAM;
  z_copy(dst, w, r, static_cast<uint32_t>(lit_end - r));
  w += lit_end - r;
  *out_pos = w;
  return ZE_OK;
}

// Decodes every frame of src[0, src_len) into dst; the output must be
// exactly dst_len bytes.  Returns 0 or an error code.
PQ_HD inline int zstd_decode(const uint8_t* src, uint32_t src_len, uint8_t* dst, uint64_t dst_len, ZState* z) {
  uint32_t pos = 0;
  uint64_t out = 0;
  while (pos < src_len) {
    if (src_len - pos < 4) return ZE_TRUNC;
    const uint32_t magic = z_le(src + pos, 4);
    if ((magic & 0xFFFFFFF0u) == 0x184D2A50u) {
      if (src_len - pos < 8) return ZE_TRUNC;
      const uint32_t sz = z_le(src + pos + 4, 4);
      if (static_cast<uint64_t>(pos) + 8 + sz > src_len) return ZE_TRUNC;
      pos += 8 + sz;
      continue;
    }
    if (magic != 0xFD2FB528u) return ZE_MAGIC;
    pos += 4;
    if (pos >= src_len) return ZE_TRUNC;
    const uint32_t fhd = src[pos++];
    if (fhd & 8) return ZE_HEADER;
    const uint32_t fcs_flag = fhd >> 6, single = (fhd >> 5) & 1, checksum = (fhd >> 2) & 1, dflag = fhd & 3;
    if (!single) ++pos;  // window descriptor
    const uint32_t dlen = dflag == 3 ? 4 : dflag;
    const uint32_t flen = fcs_flag == 0 ? single : fcs_flag == 1 ? 2 : fcs_flag == 2 ? 4 : 8;
    if (static_cast<uint64_t>(pos) + dlen + flen > src_len) return ZE_TRUNC;
    if (dlen && z_le(src + pos, static_cast<int>(dlen)) != 0) return ZE_DICT;
    pos += dlen;
    int64_t fcs = -1;
    if (flen) {
      uint64_t v = 0;
      for (int i = static_cast<int>(flen) - 1; i >= 0; --i) v = (v << 8) | src[pos + i];
      fcs = static_cast<int64_t>(v + (flen == 2 ? 256 : 0));
      pos += flen;
    }
    z->huf_bits = 0;
    z->ll_al = z->of_al = z->ml_al = -1;
    z->rep[0] = 1;
    z->rep[1] = 4;
    z->rep[2] = 8;
    const uint64_t out0 = out;
    for (;;) {
      if (src_len - pos < 3) return ZE_TRUNC;
      const uint32_t h = z_le(src + pos, 3);
      pos += 3;
      const uint32_t last = h & 1, type = (h >> 1) & 3, bsize = h >> 3;
      if (type == 0) {
        if (bsize > src_len - pos) return ZE_TRUNC;
        if (bsize > dst_len - out) return ZE_SIZE;
        for (uint32_t i = 0; i < bsize; ++i) dst[out + i] = src[pos + i];
        out += bsize;
        pos += bsize;
      } else if (type == 1) {
        if (pos >= src_len) return ZE_TRUNC;
        if (bsize > dst_len - out) return ZE_SIZE;
        for (uint32_t i = 0; i < bsize; ++i) dst[out + i] = src[pos];
        out += bsize;
        pos += 1;
      } else if (type == 2) {
        if (bsize > (128u << 10) || bsize > src_len - pos) return ZE_BLOCK;
        uint64_t lit0 = 0;
        uint32_t nlit = 0, used = 0;
        int e = z_literals(src + pos, bsize, z, dst, out, dst_len, &lit0, &nlit, &used);
        if (e) return e;
        e = z_sequences(src + pos + used, bsize - used, z, dst, &out, out0, lit0, nlit);
        if (e) return e;
        pos += bsize;
      } else {
        return ZE_BLOCK;
      }
      if (last) break;
    }
    if (checksum) {
      if (src_len - pos < 4) return ZE_TRUNC;
      pos += 4;
    }
    if (fcs >= 0 && static_cast<uint64_t>(fcs) != out - out0) return ZE_SIZE;
  }
  return out == dst_len ? ZE_OK : ZE_SIZE;
}

}  // namespace pqi
