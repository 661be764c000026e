// Internal host-side objects behind the C ABI handles.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/pq.h"
#include "decode_job.h"
#include "host_meta.h"
#include "pq_internal.h"
#include "snappy_job.h"

namespace pqe {

// Caching device allocator: freed blocks go to a free list keyed by size and
// are reused by later requests of up to the same size (within 2x), so that a
// repeated index/plan/scan cycle makes no cudaMalloc calls after warm-up.
class DevPool {
 public:
  void* alloc(size_t n);
  void free(void* p);
  void trim();
  ~DevPool();

 private:
  std::mutex mu_;
  std::multimap<size_t, void*> free_;
  std::unordered_map<void*, size_t> used_;
};

// Growable pinned host buffer.
struct Pinned {
  uint8_t* p = nullptr;
  size_t cap = 0;
  bool reserve(size_t n);
  ~Pinned();
};

// Cache of pinned host blocks for the plans' and indexes' staging (uploads,
// output descriptors, status words), so that a repeated index/plan cycle
// makes no cudaMallocHost/cudaFreeHost calls after warm-up and no upload
// is a pageable copy (which the driver may queue behind bulk copies).
class PinnedPool {
 public:
  bool take(size_t n, Pinned* out);  // a block of at least n bytes into the empty *out
  void give(Pinned* in);             // back to the cache (the caller's copies from it are done)
  ~PinnedPool();

 private:
  std::mutex mu_;
  std::multimap<size_t, uint8_t*> free_;
};

// Cache of the plans' synchronisation events (created without timing), so
// that a repeated plan cycle creates and destroys none after warm-up.
class EventPool {
 public:
  cudaError_t take(cudaEvent_t* e);
  void give(cudaEvent_t e);  // the event's last record has completed
  ~EventPool();

 private:
  std::mutex mu_;
  std::vector<cudaEvent_t> free_;
};

}  // namespace pqe

struct pq_ctx {
  int device = 0;
  int n_sms = 0;
  static constexpr int kBranches = 8;
  cudaStream_t branch[kBranches] = {};  // per-column branches of a scan
  std::string last_error;
  pq_tuning tuning{pqi::ITEM_ROWS, pqi::ITEM_ROWS_OPT, 0, kBranches, 0, 256, 1, 0};
  pqe::DevPool pool;
  pqe::PinnedPool pinned;
  pqe::EventPool events;
  pqe::Pinned tail;     // footer staging
  std::mutex mu;        // serialises use from the serving thread and the API
};

struct pq_index {
  pq_ctx* ctx = nullptr;
  std::vector<pq_file> files;
  std::vector<pqh::FileMeta> metas;
  std::vector<pqh::ColumnMeta> schema;
  int n_columns = 0;
  int n_row_groups = 0;
  int64_t num_rows = 0;
  // chunks: file-major, row group, column
  std::vector<pqi::ChunkDev> chunks;
  std::vector<int32_t> chunk_col;
  std::vector<int64_t> chunk_first_row;   // global row of the chunk's first row
  std::vector<int64_t> chunk_file_off;    // file offset of the chunk's first byte
  std::vector<int64_t> chunk_ba_bytes;    // SizeStatistics chars total, -1 unknown
  std::vector<pqi::PageDev> pages;
  pqi::ChunkDev* d_chunks = nullptr;
  pqi::PageDev* d_pages = nullptr;
  pqi::DictDev* d_dicts = nullptr;
  int64_t* d_chunk_file_off = nullptr;
  pqi::DevStatus* d_status = nullptr;
  // dictionary buffers (index-owned), per chunk
  std::vector<uint8_t*> dict_values;
  std::vector<uint64_t*> dict_str_ent;
  std::vector<uint8_t*> dict_body;        // decompressed dictionary page (compressed chunks)
  std::vector<uint8_t*> dict_pad;         // BYTE_ARRAY: the dictionary's 16-byte aligned copy
  std::vector<uint8_t> dict_resident;     // 1 once decoded and kept
  uint64_t stored_bytes = 0;
  uint64_t uncompressed_bytes = 0;
  int64_t n_data_pages = 0;
  bool used_oi = false;
};

struct pq_plan {
  pq_ctx* ctx = nullptr;
  pq_index* idx = nullptr;
  uint32_t flags = 0;
  std::vector<int32_t> cols;
  int64_t row_begin = 0, n_rows = 0;
  std::vector<pq_out_size> sizes;
  std::vector<pqi::PlanPage> pps;
  uint64_t n_items = 0;                      // work items (built on the device)
  std::vector<pqi::OutCol> outcols;
  std::vector<pqi::SnappyJob> snappy_data;   // data pages
  std::vector<pqi::SnappyJob> snappy_dict;   // dictionary pages (into index buffers)
  uint32_t snap_data_max = 0;                 // largest compressed data page of the plan
  int zstd_jobs = 0;                          // Zstandard pages among the decompression jobs
  uint32_t snap_blocks = 0;                   // blocks of the split Snappy pages (SNAPPY_FRAGMENT)
  bool needs_sizing = false;                  // string chars counted by a sizing scan at upload
  bool sizing = false;                        // that scan is being enqueued (no chars copy)
  std::vector<pqi::DictJob> dict_jobs;
  std::vector<int32_t> dict_chunks;          // chunk of each dict job
  std::vector<int32_t> str_cols;             // output columns of type BYTE_ARRAY
  std::vector<uint32_t> walk_pps;            // plan pages that need the walk, longest first
  std::vector<uint32_t> delta_pps;           // DELTA plan pages
  // V2 pages rewritten into PLAIN bodies (plan page order); host side: where
  // each job's source and destination lie (scratch offset, or -1: `src` is
  // the stored page / the destination is the pool)
  std::vector<pqi::TranscodeJob> tc_jobs;
  std::vector<int64_t> tc_src_off, tc_dst_off;
  uint64_t tc_pool_off = 0, tc_pool_bytes = 0;  // DELTA_BYTE_ARRAY pool within the scratch
  uint64_t delta_blocks = 0;                 // capacity of the DELTA block tables
  uint64_t delta_regions = 0;                // capacity of the DELTA region tables
  uint64_t dict_regions = 0;                 // capacity of the string-dictionary region tables
  uint64_t vpos_rows = 0;                    // value-position table rows of the transcoded string pages
  // per chunk: range of plan pages (plain baseline launches per chunk)
  std::vector<std::pair<int32_t, int32_t>> chunk_pp;  // (first pp, count)
  std::vector<int32_t> chunk_pp_chunk;
  int max_fixed_dict_bytes = 0;
  uint64_t read_bytes = 0;
  uint64_t decoded_bytes = 0;
  uint64_t scratch_bytes = 0;
  uint64_t host_scratch = 0;                 // decompression scratch bytes (plan_build)
  uint64_t device_bytes = 0;                 // device bytes plan_upload will take
  pq_tuning tuning{};                        // the context's knobs when the plan was built
  // device
  pqi::PlanPage* d_pps = nullptr;
  pqi::Item* d_items = nullptr;
  pqi::OutCol* d_cols = nullptr;
  pqi::SnappyJob* d_snappy = nullptr;        // data jobs then dict jobs
  pqi::SnappyJob* d_snap_blocks = nullptr;   // blocks of the split Snappy pages
  uint32_t* d_vpos = nullptr;                // value positions of the transcoded string pages
  pqi::DictJob* d_dict_jobs = nullptr;
  pqi::TranscodeJob* d_tc_jobs = nullptr;
  int32_t* d_str_cols = nullptr;
  uint8_t* d_scratch = nullptr;
  uint64_t* d_str_scratch = nullptr;
  uint64_t* d_str_items = nullptr;
  uint32_t* d_counter = nullptr;
  uint32_t* d_walk_pps = nullptr;
  uint32_t* d_delta_pps = nullptr;
  uint32_t* d_dpos = nullptr;
  int64_t* d_dbase = nullptr;
  pqi::DeltaRegion* d_dregs = nullptr;
  uint32_t* d_dreg_lists = nullptr;
  pqi::DeltaRegion* d_sregs = nullptr;
  uint64_t* d_slists = nullptr;
  pqi::DevStatus* d_status = nullptr;
  std::vector<void*> owned;                  // pool blocks to release
  // host staging (pinned, from the context's cache): output descriptors in,
  // status + string totals out, the plan's uploads
  pqe::Pinned h_cols;
  pqe::Pinned h_out;
  pqe::Pinned h_up;
  cudaEvent_t done = nullptr;
  cudaEvent_t ready = nullptr;  // the plan's uploads and item table are in place
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  bool dicts_in_graph = true;
  bool staged_expand = true;  // the staged dictionary expand (PQ_NO_STAGED_EXPAND=1: the warp decode)
  int walk_grid = 0, expand_grid = 0;
  int launches = 0;
  // per output column: ranges into the job lists
  struct ColWork {
    int snap_data_begin = 0, snap_data_n = 0;  // into snappy_data
    uint32_t snap_data_max = 0;                // largest compressed data page (bytes)
    int snap_dict_begin = 0, snap_dict_n = 0;  // into snappy_dict
    uint32_t blk_data_begin = 0, blk_data_n = 0;  // blocks of its split data pages
    uint32_t blk_dict_begin = 0, blk_dict_n = 0;  // blocks of its split dictionary pages
    int dict_begin = 0, dict_n = 0;            // into dict_jobs
    int max_fixed_dict = 0;
    int walk_begin = 0, walk_n = 0;            // into walk_pps
    int delta_begin = 0, delta_n = 0;          // into delta_pps
    int tc_begin = 0, tc_n = 0;                // into tc_jobs
    int max_regions = 0;                       // most DELTA regions of one page
    int max_str_regions = 0;                   // most chain regions of one string dictionary
    bool copy_only = false;                    // every page REQUIRED PLAIN fixed-width
    int dict_pages = 0;                        // data pages with dictionary indices
    int64_t max_dict_n = 0;                    // most entries of one of its dictionaries
    int64_t max_dict_bytes = 0;                // largest fixed-width dictionary (bytes)
    bool unsized = false;                      // BYTE_ARRAY chunks without SizeStatistics
  };
  std::vector<ColWork> colwork;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaEvent_t stage_ev[PQ_N_STAGES + 1] = {};
};

namespace pqe {
// Rows [rb, re) of the index, written to output rows starting at out0.
struct RowSeg {
  int64_t rb, re, out0;
};
// Shared helpers (engine.cpp)
pq_status fail(pq_ctx* ctx, pq_status s, const std::string& msg);
pq_status plan_build(pq_ctx* ctx, pq_index* idx, const std::vector<int32_t>& cols, const std::vector<RowSeg>& segs,
                     int64_t n_rows, uint32_t flags, std::unique_ptr<pq_plan>* out);
pq_status plan_upload(pq_plan* plan, cudaStream_t s = nullptr);
// pq_plan_scan with the plan's uploads on `stream` (nullptr: the legacy
// default stream).  The row-group pipeline plans on a slot's own stream, so
// that these small copies do not queue behind the bulk copies of other row
// groups.
pq_status plan_scan_on(pq_ctx* ctx, pq_index* idx, const pq_request* req, cudaStream_t stream, pq_plan** out,
                       pq_out_size* sizes);
uint64_t plan_device_bytes(const pq_plan* plan, uint64_t scratch);
// Enqueues one scan of `plan` into `outs` on `s`, columns forked onto
// `branches` (n_branches >= 1); no host synchronisation.
pq_status scan_enqueue(pq_plan* plan, const pq_column* outs, cudaStream_t s, const cudaStream_t* branches,
                       int n_branches, bool allow_graph);
pq_status status_from_device(pq_ctx* ctx, const pqi::DevStatus& st);
// host_pages: a page table the caller built on the host (chunk order), used
// instead of the device walk and its readback
pq_status index_build(pq_ctx* ctx, std::unique_ptr<pq_index> idx, bool allow_oi, cudaStream_t s, pq_index** out,
                      const std::vector<pqi::PageDev>* host_pages = nullptr);
void index_release(pq_index* idx);
pq_status cuda_fail(pq_ctx* ctx, cudaError_t e, const char* what);
pqi::DecodeArgs decode_args(pq_plan* plan);
}  // namespace pqe
