// Test harness: runs the engine's Zstandard decoding core (the same
// host/device functions the kernel calls) on the CPU.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "zstd_dec.cuh"

extern "C" int zstd_host_decode(const uint8_t* src, uint32_t src_len, uint8_t* dst, uint64_t dst_len) {
  static thread_local pqi::ZState z;
  return pqi::zstd_decode(src, src_len, dst, dst_len, &z);
}

// The same decode with the input and output in heap blocks of exactly
// their sizes, so that a memory checker sees any access outside them.
extern "C" int zstd_host_decode_exact(const uint8_t* src, uint32_t src_len, uint8_t* dst, uint64_t dst_len) {
  uint8_t* s = static_cast<uint8_t*>(malloc(src_len ? src_len : 1));
  uint8_t* d = static_cast<uint8_t*>(malloc(dst_len ? dst_len : 1));
  memcpy(s, src, src_len);
  const int rc = zstd_host_decode(s, src_len, d, dst_len);
  memcpy(dst, d, dst_len);
  free(s);
  free(d);
  return rc;
}
