// Length-limited Huffman code lengths (host code of the writer's
// Zstandard encoder; the format caps literal codes at 11 bits).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

namespace pqw {

// Huffman code lengths for byte counts, limited to kHufMaxBits: plain
// Huffman merging, then, if the longest code is too long, lengths above the
// limit are cut to it and the Kraft sum is repaid by lengthening the longest
// codes still below the limit (least frequent first).
constexpr int kHufMaxBits = 11;

inline bool huf_lengths(const uint32_t* cnt, int nsym, int* len) {
  struct Node {
    uint64_t w;
    int l, r;
  };
  std::vector<Node> nodes;
  std::vector<std::pair<uint64_t, int>> heap;  // (weight, node) min-heap
  for (int s = 0; s < nsym; ++s) {
    len[s] = 0;
    if (cnt[s]) {
      nodes.push_back({cnt[s], -1 - s, -1});
      heap.push_back({cnt[s], static_cast<int>(nodes.size()) - 1});
    }
  }
  if (heap.size() < 2) return false;  // one symbol: RLE literals instead
  auto cmp = [](const std::pair<uint64_t, int>& a, const std::pair<uint64_t, int>& b) { return a > b; };
  std::make_heap(heap.begin(), heap.end(), cmp);
  while (heap.size() > 1) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    const auto a = heap.back();
    heap.pop_back();
    std::pop_heap(heap.begin(), heap.end(), cmp);
    const auto b = heap.back();
    heap.pop_back();
    nodes.push_back({a.first + b.first, a.second, b.second});
    heap.push_back({a.first + b.first, static_cast<int>(nodes.size()) - 1});
    std::push_heap(heap.begin(), heap.end(), cmp);
  }
  // depths by an explicit stack walk from the root
  std::vector<std::pair<int, int>> st = {{heap[0].second, 0}};
  while (!st.empty()) {
    const auto [n, d] = st.back();
    st.pop_back();
    if (nodes[n].l < 0) {
      len[-1 - nodes[n].l] = std::max(d, 1);
    } else {
      st.push_back({nodes[n].l, d + 1});
      st.push_back({nodes[n].r, d + 1});
    }
  }
  // limit: Kraft sum in units of 2^-kHufMaxBits must stay <= 2^kHufMaxBits
  int64_t kraft = 0;
  for (int s = 0; s < nsym; ++s)
    if (len[s]) {
      if (len[s] > kHufMaxBits) len[s] = kHufMaxBits;
      kraft += int64_t(1) << (kHufMaxBits - len[s]);
    }
  const int64_t cap = int64_t(1) << kHufMaxBits;
  if (kraft > cap) {
    std::vector<int> order;
    for (int s = 0; s < nsym; ++s)
      if (len[s]) order.push_back(s);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] < cnt[b] || (cnt[a] == cnt[b] && a < b); });
    while (kraft > cap) {
      bool moved = false;
      for (int s : order)
        if (len[s] < kHufMaxBits) {
          kraft -= int64_t(1) << (kHufMaxBits - len[s] - 1);
          ++len[s];
          moved = true;
          if (kraft <= cap) break;
        }
      if (!moved) return false;
    }
    // then spend what is left of the Kraft sum on the most frequent codes,
    // so that the code stays complete
    for (auto it = order.rbegin(); it != order.rend(); ++it)
      while (len[*it] > 1 && kraft + (int64_t(1) << (kHufMaxBits - len[*it])) <= cap) {
        kraft += int64_t(1) << (kHufMaxBits - len[*it]);
        --len[*it];
      }
  }
  return true;
}

}  // namespace pqw
