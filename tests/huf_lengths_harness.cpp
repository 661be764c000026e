// Test harness: the writer's length-limited Huffman code lengths on the CPU.
#include "huf_lengths.h"

extern "C" int huf_lengths_host(const uint32_t* cnt, int nsym, int* len) {
  return pqw::huf_lengths(cnt, nsym, len) ? 1 : 0;
}
