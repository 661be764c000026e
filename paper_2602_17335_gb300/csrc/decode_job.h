// Host <-> device job descriptors of the decode kernels.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

#include "pq_internal.h"
#include "snappy_job.h"

namespace pqi {

// K6: one dictionary page to decode.
struct DictJob {
  const uint8_t* body;  // dictionary page body (decompressed)
  int32_t body_len;
  int32_t n;            // entries (page header num_values)
  int32_t ptype;
  int32_t width;
  int32_t page;         // page-table row
  int32_t chunk;        // DictDev row
  uint8_t* values;      // fixed width: n * width bytes (16-byte aligned)
  uint64_t* str_ent;    // BYTE_ARRAY: n entries, (chars offset << 32) | length
  uint8_t* pad;         // BYTE_ARRAY: PAD_STRIDE_MAX * n + 64 bytes for the padded copy
  uint32_t sreg;        // BYTE_ARRAY: first row of the job's chain-region tables
  int32_t sreg_cap;     // BYTE_ARRAY: region rows reserved (body_len / STR_REGION + 2)
};

// Chain regions of PLAIN BYTE_ARRAY dictionary pages: (4-byte length, bytes)
// entries are found per STR_REGION bytes in parallel, then stitched.
constexpr int STR_REGION = 4096;
// A string dictionary whose longest entry has at most PAD_STRIDE_MAX bytes is
// also laid out with entry i at i * stride (stride: the longest entry rounded
// up to 16 bytes), every entry 16-byte aligned; the entries then point there.
constexpr int PAD_STRIDE_MAX = 48;
constexpr int STR_REGION_LIST = STR_REGION / 4 + 2;  // entries are >= 4 bytes
struct DictScratch {
  DeltaRegion* regs;    // one summary per region
  uint64_t* lists;      // STR_REGION_LIST entries per region, (chars offset << 32) | length
};

// A BYTE_STREAM_SPLIT, DELTA_LENGTH_BYTE_ARRAY or DELTA_BYTE_ARRAY data page
// rewritten into a PLAIN body (level bytes kept in front) before the walk.
struct TranscodeJob {
  const uint8_t* src;   // page body (decompressed): level bytes + encoded values
  uint8_t* dst;         // BYTE_STREAM_SPLIT, DELTA_LENGTH_BYTE_ARRAY: dst_cap bytes for the PLAIN
                        // body; DELTA_BYTE_ARRAY: null (a piece of the plan's pool)
  uint32_t src_len;
  uint32_t dst_cap;     // src_len (BYTE_STREAM_SPLIT), src_len + 4 * num_values (DELTA_LENGTH_BYTE_ARRAY)
  uint32_t pp;          // plan page whose body and body_len the kernel sets
  int32_t page;         // page-table row (errors)
  int32_t enc;          // ENC_BSS, ENC_DELTA_LBA or ENC_DELTA_BA
  int32_t width;        // BYTE_STREAM_SPLIT value bytes
  int32_t levels;       // level bytes in front of the values: V2 def_len + rep_len;
                        // -1: V1 with levels (4-byte length + levels); 0: none
  int32_t num_values;   // page rows
  int32_t required;     // 1: REQUIRED column (value count = rows)
  int32_t pad;
};
// item_counter[TC_POOL_COUNTER .. +1]: bytes of the DELTA_BYTE_ARRAY pool
// handed out in this scan (a 64-bit counter, zeroed by the per-scan reset).
constexpr int TC_POOL_COUNTER = 2;

struct DecodeArgs {
  const ChunkDev* chunks;
  const PageDev* pages;
  const DictDev* dicts;
  PlanPage* pps;
  Item* items;
  const OutCol* cols;
  DevStatus* st;
  uint32_t* item_counter;   // [2..3] transcode pool bytes, [4 + c] next work item of output column c
  const uint32_t* walk_pps; // plan pages that need the walk, longest chains first
  const uint32_t* delta_pps;// DELTA plan pages (block bases)
  uint32_t* dpos;           // DELTA block positions (stream offsets)
  int64_t* dbase;           // DELTA value preceding each block
  DeltaRegion* dregs;       // DELTA region summaries
  uint32_t* dreg_lists;     // DELTA region block lists (DELTA_REGION_LIST per region)
  uint32_t* vpos;           // transcoded string pages: value-stream offset of each value (and of the end)
  int n_pp;
  int n_items;
  int n_walk;
  int n_delta;
};

// One block per job; `counters` is the plan's item_counter array (its pool
// word); `pool` holds `pool_cap` bytes for DELTA_BYTE_ARRAY bodies; string
// pages with a value-position table (PlanPage::vtab) get it filled in `vpos`.
void launch_transcode(const TranscodeJob* jobs, int n, PlanPage* pps, uint8_t* pool, uint64_t pool_cap,
                      uint32_t* counters, uint32_t* vpos, DevStatus* st, cudaStream_t s);
void launch_dict(const DictJob* jobs, int n_jobs, int max_fixed_bytes, int max_str_regions, DictScratch ds,
                 DictDev* dicts, int n_sms, DevStatus* st, cudaStream_t s);
// Launches over sub-ranges (one output column's share of the plan).
// levels: the pages have definition levels (their walks use jump tables)
// window: bytes per chain window (0: chosen by page count)
void launch_walk(const DecodeArgs& a, int wbegin, int n, int n_sms, bool levels, uint32_t window, cudaStream_t s);
void launch_delta_bases(const DecodeArgs& a, int dbegin, int n, int max_regions, cudaStream_t s);
void launch_expand(const DecodeArgs& a, int ibegin, int n, int cidx, int n_sms, int ctas_per_sm, cudaStream_t s);
// REQUIRED fixed-width columns with dictionary pages: items staged in shared
// memory (`stage` bytes per buffer, dict_expand_stage_bytes), dictionaries of
// up to `dict_cap` bytes gathered from shared memory (0: from global memory).
uint32_t dict_expand_stage_bytes(int item_rows, int bw_est);
bool dict_expand_fits(uint32_t stage, uint32_t dict_cap);
void launch_dict_expand(const DecodeArgs& a, int ibegin, int n, int cidx, int n_sms, int width, uint32_t stage,
                        uint32_t dict_cap, cudaStream_t s);
// Items of a column whose pages are all REQUIRED PLAIN fixed-width: copies.
void launch_copy_items(const DecodeArgs& a, int ibegin, int n, int cidx, int n_sms, int ctas_per_sm,
                       cudaStream_t s);
// copy_chars false: only the offsets pass (chars totals), no chars written
void launch_strings(const DecodeArgs& a, int col, int n_items, int n_sms, bool copy_chars, cudaStream_t s);
// Plain baseline: pages [pp_begin, pp_begin + n) decoded one page per block.
void launch_plain_pages(const DecodeArgs& a, int pp_begin, int n, cudaStream_t s);
void launch_prepare(const DecodeArgs& a, int n_cols, int grid, cudaStream_t s);
// offs[0..n) += base (string offsets of a slice placed after earlier slices).
void launch_add_offsets(int64_t* offs, int64_t n, int64_t base, cudaStream_t s);
// device memory -> pinned host memory for small control transfers (by
// stores rather than the copy engine), reading exactly `bytes` bytes
void launch_copy_small(void* dst, const void* src, uint32_t bytes, cudaStream_t s);
// Fills the work items of plan pages [0, n_pp) from their item ranges.
void launch_make_items(const DecodeArgs& a, int n_pp, cudaStream_t s);
int expand_blocks_per_sm();
int walk_blocks_per_sm();
// coop: one block of 8 warps per page (large pages), else one warp per page;
// pages with nsub > 1 are skipped (their blocks are separate jobs)
void launch_snappy(const SnappyJob* jobs, int n_jobs, int n_sms, DevStatus* st, cudaStream_t s, bool coop);
// The blocks of the pages of jobs [0, n_jobs) that have nsub > 1, written to
// blocks[sub .. sub + nsub) (SNAPPY_FRAGMENT)
void launch_snappy_split(const SnappyJob* jobs, int n_jobs, SnappyJob* blocks, int n_sms, DevStatus* st,
                         cudaStream_t s);
// Zstandard pages of jobs [0, n_jobs) (the others are skipped)
void launch_zstd(const SnappyJob* jobs, int n_jobs, int n_sms, DevStatus* st, cudaStream_t s);
void launch_index_walk(const ChunkDev* chunks, int n_chunks, PageDev* pages, uint32_t* counts, int mode,
                       DevStatus* st, cudaStream_t s);
void launch_gather16(const uint8_t* const* ptr, const int32_t* len, int n, uint8_t* out, cudaStream_t s);
void launch_index_oi(const ChunkDev* chunks, int n_chunks, const int64_t* chunk_file_off, PageDev* pages,
                     int n_pages, DevStatus* st, cudaStream_t s);

// One DELTA_BINARY_PACKED stream decoded with every piece of scratch inside
// one caller-provided block laid out as below (the allocation-free entry
// point keeps it in a fixed device array).  Limits: a stream of at most
// DS_MAX_STREAM bytes and at most DS_MAX_VALUES values.
constexpr uint64_t ds_align(uint64_t x) { return (x + 255) & ~uint64_t(255); }
constexpr uint64_t DS_MAX_STREAM = 1u << 20;
constexpr int32_t DS_MAX_BLOCKS = 32768;                      // blocks hold >= 128 values
constexpr int64_t DS_MAX_VALUES = int64_t(DS_MAX_BLOCKS) * 128 + 1;
constexpr int32_t DS_MAX_REGIONS = int32_t(DS_MAX_STREAM / DELTA_REGION) + 2;
constexpr uint64_t DS_OFF_STATUS = 0;
constexpr uint64_t DS_OFF_CHUNK = ds_align(DS_OFF_STATUS + sizeof(DevStatus));
constexpr uint64_t DS_OFF_PAGE = ds_align(DS_OFF_CHUNK + sizeof(ChunkDev));
constexpr uint64_t DS_OFF_PPS = ds_align(DS_OFF_PAGE + sizeof(PlanPage));
constexpr uint64_t DS_OFF_REGIONS = ds_align(DS_OFF_PPS + sizeof(uint32_t));
constexpr uint64_t DS_OFF_LISTS = ds_align(DS_OFF_REGIONS + sizeof(DeltaRegion) * DS_MAX_REGIONS);
constexpr uint64_t DS_OFF_DPOS = ds_align(DS_OFF_LISTS + 4ull * DELTA_REGION_LIST * DS_MAX_REGIONS);
constexpr uint64_t DS_OFF_DBASE = ds_align(DS_OFF_DPOS + 4ull * DS_MAX_BLOCKS);
constexpr uint64_t DS_SCRATCH_BYTES = ds_align(DS_OFF_DBASE + 8ull * DS_MAX_BLOCKS);
// Enqueues the decode of `n` values from `stream` (len bytes, 32 readable
// bytes after them) into `out` (4- or 8-byte values per ptype); the status
// lands at scratch + DS_OFF_STATUS.  Caller checks the limits first.
void launch_delta_static(uint8_t* scratch, const uint8_t* stream, uint32_t len, int ptype, int32_t n, void* out,
                         cudaStream_t s);

}  // namespace pqi
