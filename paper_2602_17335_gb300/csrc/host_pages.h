// Page table of column chunks that are in host memory (the serial header
// walk of the index, run on the host).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "pq_internal.h"

namespace pqe {

// Appends the pages of the chunk at `base` (`size` bytes, `num_values`
// values) to *pages, with the same fields, checks and order as the index's
// device walk (k_index_walk); `chunk` is their chunk row.  False, with
// *err set, when the chunk is malformed.
bool host_page_walk(const uint8_t* base, uint64_t size, int64_t num_values, uint32_t chunk,
                    std::vector<pqi::PageDev>* pages, std::string* err);

}  // namespace pqe
