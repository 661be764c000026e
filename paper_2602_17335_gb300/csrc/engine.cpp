// Host engine behind the C ABI: context, page index, planner and scan.
//
// Index (paper Section 2 hierarchy): footers are read with one small
// device-to-host copy per file and parsed on the host; the page headers are
// walked on the device (K0) and the page table comes back to the host,
// which plans with it.  Plan: the pages overlapping the request become
// ITEM_ROWS-row work items (paper Section 3, Insight 1: parallelism finer
// than a page), compressed pages get decompression buffers.  Scan: prepare
// -> Snappy -> dictionaries -> page walk -> expansion -> strings, all on one
// stream, optionally captured once into a CUDA graph and replayed.
#include "engine.h"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <memory>

namespace pqe {

static size_t round_size(size_t n) {
  if (n <= 4096) return 4096;
  return (n + 65535) & ~size_t(65535);
}

void* DevPool::alloc(size_t n) {
  n = round_size(n);
  std::lock_guard<std::mutex> g(mu_);
  auto it = free_.lower_bound(n);
  if (it != free_.end() && it->first <= 2 * n) {
    void* p = it->second;
    size_t sz = it->first;
    free_.erase(it);
    used_[p] = sz;
    return p;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (auto& kv : free_) cudaFree(kv.second);
    free_.clear();
    e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  used_[p] = n;
  return p;
}

void DevPool::free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(mu_);
  auto it = used_.find(p);
  if (it == used_.end()) return;
  free_.emplace(it->second, p);
  used_.erase(it);
}

void DevPool::trim() {
  std::lock_guard<std::mutex> g(mu_);
  for (auto& kv : free_) cudaFree(kv.second);
  free_.clear();
}

DevPool::~DevPool() {
  for (auto& kv : free_) cudaFree(kv.second);
  for (auto& kv : used_) cudaFree(kv.first);
}

bool Pinned::reserve(size_t n) {
  if (n <= cap) return true;
  if (p) cudaFreeHost(p);
  p = nullptr;
  cap = 0;
  size_t c = std::max<size_t>(n, 4096);
  if (cudaMallocHost(&p, c) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return false;
  }
  cap = c;
  return true;
}

Pinned::~Pinned() {
  if (p) cudaFreeHost(p);
}

bool PinnedPool::take(size_t n, Pinned* out) {
  n = std::max<size_t>((n + 4095) & ~size_t(4095), 4096);
  {
    std::lock_guard<std::mutex> g(mu_);
    auto it = free_.lower_bound(n);
    if (it != free_.end() && it->first <= 4 * n) {
      out->p = it->second;
      out->cap = it->first;
      free_.erase(it);
      return true;
    }
  }
  return out->reserve(n);
}

void PinnedPool::give(Pinned* in) {
  if (!in->p) return;
  {
    std::lock_guard<std::mutex> g(mu_);
    if (free_.size() < 64 && in->cap <= (size_t(64) << 20)) {
      free_.emplace(in->cap, in->p);
      in->p = nullptr;
      in->cap = 0;
      return;
    }
  }
  cudaFreeHost(in->p);
  in->p = nullptr;
  in->cap = 0;
}

PinnedPool::~PinnedPool() {
  for (auto& kv : free_) cudaFreeHost(kv.second);
}

cudaError_t EventPool::take(cudaEvent_t* e) {
  {
    std::lock_guard<std::mutex> g(mu_);
    if (!free_.empty()) {
      *e = free_.back();
      free_.pop_back();
      return cudaSuccess;
    }
  }
  return cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}

void EventPool::give(cudaEvent_t e) {
  if (!e) return;
  {
    std::lock_guard<std::mutex> g(mu_);
    if (free_.size() < 1024) {
      free_.push_back(e);
      return;
    }
  }
  cudaEventDestroy(e);
}

EventPool::~EventPool() {
  for (cudaEvent_t e : free_) cudaEventDestroy(e);
}

pq_status fail(pq_ctx* ctx, pq_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

pq_status cuda_fail(pq_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, PQ_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

pqi::DecodeArgs decode_args(pq_plan* plan) {
  pqi::DecodeArgs a{};
  a.chunks = plan->idx->d_chunks;
  a.pages = plan->idx->d_pages;
  a.dicts = plan->idx->d_dicts;
  a.pps = plan->d_pps;
  a.items = plan->d_items;
  a.cols = plan->d_cols;
  a.st = plan->d_status;
  a.item_counter = plan->d_counter;
  a.walk_pps = plan->d_walk_pps;
  a.delta_pps = plan->d_delta_pps;
  a.dpos = plan->d_dpos;
  a.dbase = plan->d_dbase;
  a.dregs = plan->d_dregs;
  a.dreg_lists = plan->d_dreg_lists;
  a.vpos = plan->d_vpos;
  a.n_pp = static_cast<int>(plan->pps.size());
  a.n_items = static_cast<int>(plan->n_items);
  a.n_walk = static_cast<int>(plan->walk_pps.size());
  a.n_delta = static_cast<int>(plan->delta_pps.size());
  return a;
}

static const char* where_name(int w) {
  switch (w) {
    case pqi::WHERE_INDEX: return "page-header index";
    case pqi::WHERE_SNAPPY: return "snappy";
    case pqi::WHERE_DICT: return "dictionary";
    case pqi::WHERE_WALK_LEVELS: return "definition levels";
    case pqi::WHERE_WALK_VALUES: return "value stream walk";
    case pqi::WHERE_EXPAND: return "value expansion";
    case pqi::WHERE_STRINGS: return "strings";
    default: return "device";
  }
}

pq_status status_from_device(pq_ctx* ctx, const pqi::DevStatus& st) {
  if (!st.flags) return PQ_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s at page %d (code %d)", where_name(st.where),
           (st.flags & pqi::DERR_TIMEOUT) ? "bounded wait ran out"
           : (st.flags & pqi::DERR_CAPACITY) ? "output buffer too small"
           : (st.flags & pqi::DERR_UNSUPPORTED) ? "unsupported feature"
                                                : "corrupt data",
           st.first_page, st.detail);
  pq_status s = (st.flags & pqi::DERR_TIMEOUT) ? PQ_ERR_TIMEOUT
                : (st.flags & pqi::DERR_CORRUPT) ? PQ_ERR_CORRUPT
                : (st.flags & pqi::DERR_UNSUPPORTED) ? PQ_ERR_UNSUPPORTED
                                                     : PQ_ERR_CAPACITY;
  return fail(ctx, s, buf);
}

}  // namespace pqe

using namespace pqe;

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

extern "C" {

const char* pq_version(void) { return "pqscan-gb300 0.1 (sm_103a)"; }

const char* pq_status_string(pq_status s) {
  switch (s) {
    case PQ_OK: return "ok";
    case PQ_ERR_INVALID_ARG: return "invalid argument";
    case PQ_ERR_CORRUPT: return "corrupt data";
    case PQ_ERR_UNSUPPORTED: return "unsupported";
    case PQ_ERR_OOM: return "out of memory";
    case PQ_ERR_BUDGET: return "over budget";
    case PQ_ERR_TIMEOUT: return "timeout";
    case PQ_ERR_CUDA: return "cuda error";
    case PQ_ERR_CAPACITY: return "capacity";
  }
  return "unknown";
}

pq_status pq_ctx_create(int device, pq_ctx** out) {
  if (!out) return PQ_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PQ_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return PQ_ERR_CUDA;
  pq_ctx* ctx = new pq_ctx();
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->n_sms, cudaDevAttrMultiProcessorCount, device);
  if (ctx->n_sms <= 0) ctx->n_sms = 1;
  for (auto& b : ctx->branch) {
    if (cudaStreamCreateWithFlags(&b, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      pq_ctx_destroy(ctx);
      return PQ_ERR_CUDA;
    }
  }
  *out = ctx;
  return PQ_OK;
}

void pq_ctx_destroy(pq_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& b : ctx->branch)
    if (b) cudaStreamDestroy(b);
  delete ctx;
}

const char* pq_last_error(const pq_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

pq_status pq_ctx_set_tuning(pq_ctx* ctx, const pq_tuning* t) {
  if (!ctx || !t) return PQ_ERR_INVALID_ARG;
  if (t->item_rows < 256 || t->item_rows > 65536 || t->item_rows % 32 || t->item_rows_opt < 32 ||
      t->item_rows_opt > pqi::ITEM_ROWS_OPT || t->item_rows_opt % 32 || t->expand_ctas_per_sm < 0 ||
      t->branches < 1 || t->branches > pq_ctx::kBranches ||
      (t->walk_window != 0 && (t->walk_window < 4096 || t->walk_window > 65536 ||
                               (t->walk_window & (t->walk_window - 1)))) ||
      t->snappy_block_kib < 1 || t->snappy_block_kib > (1 << 20) || (t->staged_expand != 0 && t->staged_expand != 1))
    return fail(ctx, PQ_ERR_INVALID_ARG, "pq_ctx_set_tuning: knob out of range");
  ctx->tuning = *t;
  return PQ_OK;
}

pq_status pq_ctx_get_tuning(const pq_ctx* ctx, pq_tuning* t) {
  if (!ctx || !t) return PQ_ERR_INVALID_ARG;
  *t = ctx->tuning;
  return PQ_OK;
}

// ------------------------------------------------------------------ index

// Small device-to-host reads (status words, page counts, the page table)
// go by a copy kernel into pinned host memory rather than by the copy
// engine, where they would wait behind bulk transfers of other streams.
static cudaError_t d2h_small(void* pinned_dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!bytes) return cudaSuccess;
  void* dv = nullptr;
  if (bytes >= (1u << 31) || cudaHostGetDevicePointer(&dv, pinned_dst, 0) != cudaSuccess || !dv) {
    cudaGetLastError();
    return cudaMemcpyAsync(pinned_dst, src, bytes, cudaMemcpyDeviceToHost, s);
  }
  pqi::launch_copy_small(dv, src, static_cast<uint32_t>(bytes), s);
  return cudaGetLastError();
}

static void free_index_device(pq_index* idx) {
  DevPool& pool = idx->ctx->pool;
  pool.free(idx->d_chunks);
  pool.free(idx->d_pages);
  pool.free(idx->d_dicts);
  pool.free(idx->d_chunk_file_off);
  pool.free(idx->d_status);
  for (auto p : idx->dict_values) pool.free(p);
  for (auto p : idx->dict_str_ent) pool.free(p);
  for (auto p : idx->dict_body) pool.free(p);
  for (auto p : idx->dict_pad) pool.free(p);
}

void pq_free_index(pq_index* idx) {
  if (!idx) return;
  cudaSetDevice(idx->ctx->device);
  cudaDeviceSynchronize();
  free_index_device(idx);
  delete idx;
}

}  // extern "C"

namespace pqe {
// Frees an index whose device work has already completed (no device-wide sync).
void index_release(pq_index* idx) {
  if (!idx) return;
  free_index_device(idx);
  delete idx;
}
}  // namespace pqe

extern "C" {

static bool env_flag(const char* name) {
  const char* v = getenv(name);
  return v && *v && strcmp(v, "0") != 0;
}

pq_status pq_index_chunks(pq_ctx* ctx, const pq_file* files, int n_files, void* stream, pq_index** out) {
  if (!ctx || !out || (!files && n_files > 0) || n_files <= 0)
    return fail(ctx, PQ_ERR_INVALID_ARG, "pq_index_chunks: bad arguments");
  *out = nullptr;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(ctx->mu);
  // 1. footers: one copy of each file's head magic + tail
  const size_t kTail = 64 * 1024;
  std::vector<size_t> toff(n_files), tlen(n_files);
  size_t total = 0;
  for (int f = 0; f < n_files; ++f) {
    if (!files[f].data || files[f].size < 12)
      return fail(ctx, PQ_ERR_CORRUPT, "file " + std::to_string(f) + " is too small for Parquet");
    tlen[f] = static_cast<size_t>(std::min<uint64_t>(files[f].size, kTail));
    toff[f] = total;
    total += tlen[f] + 16;
  }
  if (!ctx->tail.reserve(total)) return fail(ctx, PQ_ERR_OOM, "pinned staging");
  for (int f = 0; f < n_files; ++f) {
    const uint8_t* base = static_cast<const uint8_t*>(files[f].data);
    CK(cudaMemcpyAsync(ctx->tail.p + toff[f], base, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctx->tail.p + toff[f] + 16, base + files[f].size - tlen[f], tlen[f],
                       cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  auto idx = std::make_unique<pq_index>();
  idx->ctx = ctx;
  idx->files.assign(files, files + n_files);
  idx->metas.resize(n_files);
  std::vector<uint8_t> big;
  for (int f = 0; f < n_files; ++f) {
    const uint8_t* head = ctx->tail.p + toff[f];
    const uint8_t* tail = ctx->tail.p + toff[f] + 16;
    const size_t tl = tlen[f];
    if (memcmp(head, "PAR1", 4) || memcmp(tail + tl - 4, "PAR1", 4))
      return fail(ctx, PQ_ERR_CORRUPT, "file " + std::to_string(f) + ": missing PAR1 magic");
    uint32_t flen;
    memcpy(&flen, tail + tl - 8, 4);
    if (static_cast<uint64_t>(flen) + 12 > files[f].size || flen < 8)
      return fail(ctx, PQ_ERR_CORRUPT, "file " + std::to_string(f) + ": bad footer length");
    const uint8_t* fp;
    if (flen + 8 <= tl) {
      fp = tail + tl - 8 - flen;
    } else {
      big.resize(flen);
      const uint8_t* base = static_cast<const uint8_t*>(files[f].data);
      CK(cudaMemcpy(big.data(), base + files[f].size - 8 - flen, flen, cudaMemcpyDeviceToHost));
      fp = big.data();
    }
    std::string err;
    int rc = pqh::parse_file_metadata(fp, flen, &idx->metas[f], &err);
    if (rc != pqh::META_OK)
      return fail(ctx, rc == pqh::META_UNSUPPORTED ? PQ_ERR_UNSUPPORTED : PQ_ERR_CORRUPT,
                  "file " + std::to_string(f) + ": " + err);
    idx->metas[f].footer_len = flen;
  }
  return index_build(ctx, std::move(idx), !env_flag("PQ_NO_OFFSET_INDEX"), s, out);
}

}  // extern "C"

namespace pqe {

// Index from parsed footers: `idx` holds files (device base, size) and
// metas; chunks at base + chunk offset.  allow_oi: page locations may be
// read from OffsetIndex structures on the device.
pq_status index_build(pq_ctx* ctx, std::unique_ptr<pq_index> idx, bool allow_oi, cudaStream_t s, pq_index** out,
                      const std::vector<pqi::PageDev>* host_pages) {
  const int n_files = static_cast<int>(idx->files.size());
  const pq_file* files = idx->files.data();
  // 2. schema
  idx->schema = idx->metas[0].columns;
  idx->n_columns = static_cast<int>(idx->schema.size());
  for (int f = 1; f < n_files; ++f) {
    const auto& c = idx->metas[f].columns;
    bool same = c.size() == idx->schema.size();
    for (size_t i = 0; same && i < c.size(); ++i)
      same = c[i].name == idx->schema[i].name && c[i].type == idx->schema[i].type &&
             c[i].repetition == idx->schema[i].repetition;
    if (!same) return fail(ctx, PQ_ERR_INVALID_ARG, "files do not share one schema");
  }
  for (auto& c : idx->schema) {
    if (c.type != pqi::T_INT32 && c.type != pqi::T_INT64 && c.type != pqi::T_DOUBLE && c.type != pqi::T_FLOAT &&
        c.type != pqi::T_BYTE_ARRAY)
      return fail(ctx, PQ_ERR_UNSUPPORTED, "column " + c.name + ": physical type not supported");
  }
  // 3. chunks
  int64_t row = 0;
  bool all_oi = allow_oi;
  for (int f = 0; f < n_files; ++f) {
    const auto& m = idx->metas[f];
    const uint64_t fsize = files[f].size;
    for (const auto& g : m.rgs) {
      for (int c = 0; c < idx->n_columns; ++c) {
        const auto& cm = g.chunks[c];
        const int64_t start = cm.start();
        if (cm.type != idx->schema[c].type)
          return fail(ctx, PQ_ERR_CORRUPT, "chunk type differs from the schema");
        if (cm.num_values != g.num_rows)
          return fail(ctx, PQ_ERR_CORRUPT, "chunk value count differs from its row group (nested data?)");
        if (cm.codec != pqi::CODEC_NONE && cm.codec != pqi::CODEC_SNAPPY && cm.codec != pqi::CODEC_ZSTD)
          return fail(ctx, PQ_ERR_UNSUPPORTED, "codec " + std::to_string(cm.codec) + " not supported");
        if (start < 4 || cm.total_compressed < 0 ||
            static_cast<uint64_t>(start) + static_cast<uint64_t>(cm.total_compressed) + 8 + m.footer_len > fsize ||
            static_cast<uint64_t>(start) + static_cast<uint64_t>(cm.total_compressed) + 32 > fsize)
          return fail(ctx, PQ_ERR_CORRUPT, "chunk byte range outside the file");
        pqi::ChunkDev cd{};
        cd.base = static_cast<const uint8_t*>(files[f].data) + start;
        cd.size = static_cast<uint64_t>(cm.total_compressed);
        cd.num_values = cm.num_values;
        cd.ptype = cm.type;
        cd.codec = cm.codec;
        cd.max_def = idx->schema[c].repetition == 1 ? 1 : 0;
        cd.width = pqi::type_width(cm.type);
        cd.dict_page = -1;
        cd.file = f;
        idx->chunks.push_back(cd);
        idx->chunk_col.push_back(c);
        idx->chunk_first_row.push_back(row);
        idx->chunk_file_off.push_back(start);
        idx->chunk_ba_bytes.push_back(cm.byte_array_bytes);
        idx->stored_bytes += cd.size;
        if (cm.oi_offset < 0 || cm.oi_length <= 0 ||
            static_cast<uint64_t>(cm.oi_offset) + static_cast<uint64_t>(cm.oi_length) > fsize)
          all_oi = false;
      }
      row += g.num_rows;
      idx->n_row_groups++;
    }
  }
  idx->num_rows = row;
  const int nch = static_cast<int>(idx->chunks.size());
  DevPool& pool = ctx->pool;
  idx->d_chunks = static_cast<pqi::ChunkDev*>(pool.alloc(sizeof(pqi::ChunkDev) * std::max(nch, 1)));
  idx->d_status = static_cast<pqi::DevStatus*>(pool.alloc(sizeof(pqi::DevStatus)));
  idx->d_dicts = static_cast<pqi::DictDev*>(pool.alloc(sizeof(pqi::DictDev) * std::max(nch, 1)));
  idx->d_chunk_file_off = static_cast<int64_t*>(pool.alloc(sizeof(int64_t) * std::max(nch, 1)));
  if (!idx->d_chunks || !idx->d_status || !idx->d_dicts || !idx->d_chunk_file_off) {
    free_index_device(idx.get());
    return fail(ctx, PQ_ERR_OOM, "index allocation");
  }
  // uploads go through a pinned block from the context's cache (returned
  // once the stream has drained: every path below ends in a stream sync)
  struct Stage {
    pq_ctx* ctx;
    cudaStream_t s;
    Pinned b;
    size_t off = 0;
    ~Stage() {
      if (b.p) {
        cudaStreamSynchronize(s);
        ctx->pinned.give(&b);
      }
    }
    const void* put(const void* src, size_t n) {
      uint8_t* d = b.p + off;
      memcpy(d, src, n);
      off += (n + 15) & ~size_t(15);
      return d;
    }
  } up{ctx, s, {}};
  const size_t chunk_bytes = sizeof(pqi::ChunkDev) * static_cast<size_t>(std::max(nch, 0));
  if (!ctx->pinned.take(64 + 8 * static_cast<size_t>(nch) + 3 * (chunk_bytes + 16), &up.b)) {
    free_index_device(idx.get());
    return fail(ctx, PQ_ERR_OOM, "pinned staging");
  }
  auto upload_chunks = [&]() -> cudaError_t {
    return cudaMemcpyAsync(idx->d_chunks, up.put(idx->chunks.data(), chunk_bytes), chunk_bytes,
                           cudaMemcpyHostToDevice, s);
  };
  pqi::DevStatus st0{0, -1, 0, 0};
  CK(cudaMemcpyAsync(idx->d_status, up.put(&st0, sizeof st0), sizeof st0, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(idx->d_dicts, 0, sizeof(pqi::DictDev) * std::max(nch, 1), s));
  CK(cudaMemcpyAsync(idx->d_chunk_file_off, up.put(idx->chunk_file_off.data(), sizeof(int64_t) * nch),
                     sizeof(int64_t) * nch, cudaMemcpyHostToDevice, s));
  int64_t n_pages = 0;
  Stage up_pages{ctx, s, {}};
  if (host_pages) {
    // 4. the caller's page table (chunk order), walked on the host
    std::vector<uint32_t> count(static_cast<size_t>(std::max(nch, 0)), 0);
    uint32_t prev = 0;
    for (const auto& pg : *host_pages) {
      if (static_cast<int64_t>(pg.chunk) >= nch || pg.chunk < prev) {
        free_index_device(idx.get());
        return fail(ctx, PQ_ERR_INVALID_ARG, "host page table out of chunk order");
      }
      prev = pg.chunk;
      ++count[pg.chunk];
    }
    for (int c = 0; c < nch; ++c) {
      idx->chunks[c].page_begin = static_cast<uint32_t>(n_pages);
      idx->chunks[c].page_count = count[c];
      n_pages += count[c];
    }
    const size_t bytes = sizeof(pqi::PageDev) * static_cast<size_t>(n_pages);
    idx->d_pages = static_cast<pqi::PageDev*>(pool.alloc(std::max<size_t>(bytes, sizeof(pqi::PageDev))));
    if (!idx->d_pages || !ctx->pinned.take(bytes + 16, &up_pages.b)) {
      free_index_device(idx.get());
      return fail(ctx, PQ_ERR_OOM, "page table");
    }
    if (bytes)
      CK(cudaMemcpyAsync(idx->d_pages, up_pages.put(host_pages->data(), bytes), bytes, cudaMemcpyHostToDevice, s));
    idx->pages = *host_pages;
  } else if (all_oi && nch > 0) {
    // 4a. OffsetIndex: page counts from the list headers (the first 16 bytes
    // of every chunk's OffsetIndex, fetched in one round trip into the
    // footer staging, which is free again), then one thread per page
    // staging: [0, 16 n) the list headers, [16 n, 24 n) their addresses,
    // [24 n, 28 n) the OffsetIndex lengths; one gather launch between one
    // upload and one download
    const size_t n16 = 16 * static_cast<size_t>(nch);
    if (!ctx->tail.reserve(28 * static_cast<size_t>(nch))) {
      free_index_device(idx.get());
      return fail(ctx, PQ_ERR_OOM, "pinned staging");
    }
    {
      const uint8_t** hp = reinterpret_cast<const uint8_t**>(ctx->tail.p + n16);
      int32_t* hl = reinterpret_cast<int32_t*>(ctx->tail.p + 24 * static_cast<size_t>(nch));
      int ci = 0;
      for (int f = 0; f < n_files; ++f) {
        const uint8_t* base = static_cast<const uint8_t*>(files[f].data);
        for (const auto& g : idx->metas[f].rgs)
          for (int c = 0; c < idx->n_columns; ++c, ++ci) {
            hp[ci] = base + g.chunks[c].oi_offset;
            hl[ci] = g.chunks[c].oi_length;
          }
      }
      uint8_t* d_g = static_cast<uint8_t*>(pool.alloc(28 * static_cast<size_t>(nch)));
      if (!d_g) {
        free_index_device(idx.get());
        return fail(ctx, PQ_ERR_OOM, "index staging");
      }
      CK(cudaMemcpyAsync(d_g + n16, ctx->tail.p + n16, 12 * static_cast<size_t>(nch), cudaMemcpyHostToDevice, s));
      pqi::launch_gather16(reinterpret_cast<const uint8_t* const*>(d_g + n16),
                           reinterpret_cast<const int32_t*>(d_g + 24 * static_cast<size_t>(nch)), nch, d_g, s);
      CK(cudaMemcpyAsync(ctx->tail.p, d_g, n16, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      pool.free(d_g);
    }
    int ci = 0;
    for (int f = 0; f < n_files; ++f) {
      for (const auto& g : idx->metas[f].rgs) {
        for (int c = 0; c < idx->n_columns; ++c, ++ci) {
          const auto& cm = g.chunks[c];
          const uint8_t* base = static_cast<const uint8_t*>(files[f].data);
          int64_t np = 0;
          if (pqh::offset_index_pages(ctx->tail.p + 16 * ci, std::min<int32_t>(cm.oi_length, 16), &np) !=
                  pqh::META_OK ||
              np < 0) {
            free_index_device(idx.get());
            return fail(ctx, PQ_ERR_CORRUPT, "malformed OffsetIndex");
          }
          auto& cd = idx->chunks[ci];
          cd.oi_base = base + cm.oi_offset;
          cd.oi_len = static_cast<uint32_t>(cm.oi_length);
          cd.oi_pages = static_cast<uint32_t>(np);
          cd.page_begin = static_cast<uint32_t>(n_pages);
          cd.page_count = static_cast<uint32_t>(np + (cm.has_dict() ? 1 : 0));
          cd.dict_page = cm.has_dict() ? static_cast<int32_t>(n_pages) : -1;
          n_pages += cd.page_count;
        }
      }
    }
    idx->d_pages = static_cast<pqi::PageDev*>(pool.alloc(sizeof(pqi::PageDev) * std::max<int64_t>(n_pages, 1)));
    if (!idx->d_pages) {
      free_index_device(idx.get());
      return fail(ctx, PQ_ERR_OOM, "page table");
    }
    CK(upload_chunks());
    pqi::launch_index_oi(idx->d_chunks, nch, idx->d_chunk_file_off, idx->d_pages, static_cast<int>(n_pages),
                         idx->d_status, s);
    idx->used_oi = true;
  } else if (nch > 0) {
    // 4b. serial header walk: count, size, fill
    CK(upload_chunks());
    uint32_t* d_counts = static_cast<uint32_t*>(pool.alloc(sizeof(uint32_t) * nch));
    if (!d_counts) {
      free_index_device(idx.get());
      return fail(ctx, PQ_ERR_OOM, "page counts");
    }
    pqi::launch_index_walk(idx->d_chunks, nch, nullptr, d_counts, 0, idx->d_status, s);
    std::vector<uint32_t> counts(nch);
    pqi::DevStatus st{};
    if (!ctx->tail.reserve(sizeof st + sizeof(uint32_t) * nch)) {
      free_index_device(idx.get());
      return fail(ctx, PQ_ERR_OOM, "pinned staging");
    }
    CK(d2h_small(ctx->tail.p, idx->d_status, sizeof st, s));
    CK(d2h_small(ctx->tail.p + sizeof st, d_counts, sizeof(uint32_t) * nch, s));
    CK(cudaStreamSynchronize(s));
    memcpy(&st, ctx->tail.p, sizeof st);
    memcpy(counts.data(), ctx->tail.p + sizeof st, sizeof(uint32_t) * nch);
    pool.free(d_counts);
    if (st.flags) {
      pq_status r = status_from_device(ctx, st);
      free_index_device(idx.get());
      return r;
    }
    for (int c = 0; c < nch; ++c) {
      idx->chunks[c].page_begin = static_cast<uint32_t>(n_pages);
      idx->chunks[c].page_count = counts[c];
      n_pages += counts[c];
    }
    idx->d_pages = static_cast<pqi::PageDev*>(pool.alloc(sizeof(pqi::PageDev) * std::max<int64_t>(n_pages, 1)));
    if (!idx->d_pages) {
      free_index_device(idx.get());
      return fail(ctx, PQ_ERR_OOM, "page table");
    }
    CK(upload_chunks());
    pqi::launch_index_walk(idx->d_chunks, nch, idx->d_pages, nullptr, 1, idx->d_status, s);
  }
  // 5. page table back to the host (built on the device)
  if (!host_pages) {
    idx->pages.resize(n_pages);
    pqi::DevStatus st{};
    if (!ctx->tail.reserve(sizeof st + sizeof(pqi::PageDev) * n_pages)) {
      free_index_device(idx.get());
      return fail(ctx, PQ_ERR_OOM, "pinned staging");
    }
    CK(d2h_small(ctx->tail.p, idx->d_status, sizeof st, s));
    CK(d2h_small(ctx->tail.p + sizeof st, idx->d_pages, sizeof(pqi::PageDev) * n_pages, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    memcpy(&st, ctx->tail.p, sizeof st);
    if (n_pages) memcpy(idx->pages.data(), ctx->tail.p + sizeof st, sizeof(pqi::PageDev) * n_pages);
    if (st.flags) {
      pq_status r = status_from_device(ctx, st);
      free_index_device(idx.get());
      return r;
    }
  }
  // 6. host checks, dictionary buffers
  idx->dict_values.assign(nch, nullptr);
  idx->dict_str_ent.assign(nch, nullptr);
  idx->dict_body.assign(nch, nullptr);
  idx->dict_pad.assign(nch, nullptr);
  idx->dict_resident.assign(nch, 0);
  for (int c = 0; c < nch; ++c) {
    auto& cd = idx->chunks[c];
    cd.dict_page = -1;
    for (uint32_t k = 0; k < cd.page_count; ++k) {
      const auto& pg = idx->pages[cd.page_begin + k];
      if (pg.page_type == pqi::PAGE_DICT) {
        cd.dict_page = static_cast<int32_t>(cd.page_begin + k);
      } else {
        idx->n_data_pages++;
      }
      if (cd.codec == pqi::CODEC_NONE && pg.compressed != pg.uncompressed) {
        free_index_device(idx.get());
        return fail(ctx, PQ_ERR_CORRUPT, "uncompressed page with differing sizes");
      }
      idx->uncompressed_bytes += static_cast<uint64_t>(pg.header_len) + static_cast<uint64_t>(pg.uncompressed);
    }
    if (cd.dict_page >= 0) {
      const auto& dp = idx->pages[cd.dict_page];
      if (dp.num_values < 0 || (dp.encoding != pqi::ENC_PLAIN && dp.encoding != pqi::ENC_PLAIN_DICT)) {
        free_index_device(idx.get());
        return fail(ctx, PQ_ERR_UNSUPPORTED, "dictionary page encoding");
      }
      const size_t n = static_cast<size_t>(dp.num_values);
      if (cd.ptype == pqi::T_BYTE_ARRAY) {
        idx->dict_str_ent[c] = static_cast<uint64_t*>(pool.alloc(8 * n + 16));
        idx->dict_pad[c] = static_cast<uint8_t*>(pool.alloc(static_cast<size_t>(pqi::PAD_STRIDE_MAX) * n + 64));
        if (!idx->dict_str_ent[c] || !idx->dict_pad[c]) {
          free_index_device(idx.get());
          return fail(ctx, PQ_ERR_OOM, "dictionary");
        }
      } else {
        idx->dict_values[c] = static_cast<uint8_t*>(pool.alloc(n * cd.width + 16));
        if (!idx->dict_values[c]) {
          free_index_device(idx.get());
          return fail(ctx, PQ_ERR_OOM, "dictionary");
        }
      }
      if (cd.codec != pqi::CODEC_NONE) {
        idx->dict_body[c] = static_cast<uint8_t*>(pool.alloc(static_cast<size_t>(dp.uncompressed) + 32));
        if (!idx->dict_body[c]) {
          free_index_device(idx.get());
          return fail(ctx, PQ_ERR_OOM, "dictionary page buffer");
        }
      }
    }
  }
  CK(upload_chunks());
  CK(cudaStreamSynchronize(s));
  *out = idx.release();
  return PQ_OK;
}

}  // namespace pqe

extern "C" {

pq_status pq_index_get_info(const pq_index* idx, pq_index_info* out) {
  if (!idx || !out) return PQ_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  out->n_files = static_cast<int32_t>(idx->files.size());
  out->n_columns = idx->n_columns;
  out->n_row_groups = idx->n_row_groups;
  out->n_chunks = static_cast<int32_t>(idx->chunks.size());
  out->n_pages = static_cast<int64_t>(idx->pages.size());
  out->n_data_pages = idx->n_data_pages;
  out->num_rows = idx->num_rows;
  out->stored_bytes = idx->stored_bytes;
  out->uncompressed_bytes = idx->uncompressed_bytes;
  out->used_offset_index = idx->used_oi ? 1 : 0;
  return PQ_OK;
}

pq_status pq_index_get_column(const pq_index* idx, int column, pq_column_info* out) {
  if (!idx || !out || column < 0 || column >= idx->n_columns) return PQ_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  const auto& c = idx->schema[column];
  strncpy(out->name, c.name.c_str(), sizeof(out->name) - 1);
  out->type = c.type;
  out->optional = c.repetition == 1;
  out->type_length = pqi::type_width(c.type);
  return PQ_OK;
}

pq_status pq_index_copy_pages(const pq_index* idx, pq_page_info* out, int64_t cap, int64_t* n_out) {
  if (!idx || (!out && cap > 0)) return PQ_ERR_INVALID_ARG;
  const int64_t n = static_cast<int64_t>(idx->pages.size());
  if (n_out) *n_out = n;
  for (int64_t i = 0; i < n && i < cap; ++i) {
    const auto& pg = idx->pages[i];
    const auto& cd = idx->chunks[pg.chunk];
    pq_page_info& o = out[i];
    o.header_offset = idx->chunk_file_off[pg.chunk] + static_cast<int64_t>(pg.offset);
    o.file = cd.file;
    o.chunk = static_cast<int32_t>(pg.chunk);
    o.page_type = pg.page_type;
    o.encoding = pg.encoding;
    o.header_len = pg.header_len;
    o.uncompressed_size = pg.uncompressed;
    o.compressed_size = pg.compressed;
    o.num_values = pg.num_values;
    o.num_nulls = pg.num_nulls;
    o.def_len = pg.def_len;
    o.first_row = pg.first_row;
  }
  return PQ_OK;
}

// ------------------------------------------------------------------ plan

static void free_plan_device(pq_plan* plan) {
  for (void* p : plan->owned) plan->ctx->pool.free(p);
  plan->owned.clear();
}

void pq_free_plan(pq_plan* plan) {
  if (!plan) return;
  cudaSetDevice(plan->ctx->device);
  // once `done` (recorded after the scan's last work) and `ready` have
  // completed, so have the fork and join records: all go back to the cache
  if (plan->done) cudaEventSynchronize(plan->done);
  if (plan->ready) cudaEventSynchronize(plan->ready);
  if (plan->graph) cudaGraphExecDestroy(plan->graph);
  for (auto& e : plan->stage_ev)
    if (e) cudaEventDestroy(e);
  pqe::EventPool& ev = plan->ctx->events;
  ev.give(plan->done);
  ev.give(plan->ready);
  ev.give(plan->fork);
  for (auto& e : plan->join) ev.give(e);
  free_plan_device(plan);
  for (pqe::Pinned* b : {&plan->h_cols, &plan->h_out, &plan->h_up}) plan->ctx->pinned.give(b);
  delete plan;
}

static void* plan_alloc_bytes(pq_plan* plan, size_t bytes) {
  void* p = plan->ctx->pool.alloc(std::max<size_t>(bytes, 1));
  plan->owned.push_back(p);
  return p;
}
#define plan_alloc(T, plan, count) static_cast<T*>(plan_alloc_bytes(plan, std::max<size_t>(count, 1) * sizeof(T)))

}  // extern "C"

namespace pqe {

// Host half of planning: plan pages, work item counts, job lists and the
// scratch layout for the rows of `segs` (each segment's rows go to output
// rows starting at its out0), nothing on the device yet.
// A Snappy page decompressed by fragments (SNAPPY_FRAGMENT): nsub block slots
// numbered from *counter.  Dictionary and data pages count separately (their
// blocks sit in two ranges of the block list, like their jobs).
static void plan_split(pqi::SnappyJob& sj, bool plain, uint32_t* counter) {
  if (plain || sj.codec != pqi::CODEC_SNAPPY || sj.raw || sj.prefix > sj.dst_len) return;
  const uint32_t out = sj.dst_len - sj.prefix;
  if (out <= pqi::SNAPPY_SPLIT_MIN) return;
  sj.nsub = (out + pqi::SNAPPY_FRAGMENT - 1) / pqi::SNAPPY_FRAGMENT;
  sj.sub = *counter;
  *counter += sj.nsub;
}

pq_status plan_build(pq_ctx* ctx, pq_index* idx, const std::vector<int32_t>& cols, const std::vector<RowSeg>& segs,
                     int64_t n_rows, uint32_t flags, std::unique_ptr<pq_plan>* out) {
  if ((flags & PQ_SCAN_TIMING) && (flags & PQ_SCAN_GRAPH))
    return fail(ctx, PQ_ERR_INVALID_ARG, "PQ_SCAN_TIMING cannot be combined with PQ_SCAN_GRAPH");
  auto plan = std::make_unique<pq_plan>();
  plan->ctx = ctx;
  plan->idx = idx;
  plan->flags = flags;
  plan->cols = cols;
  plan->row_begin = segs.empty() ? 0 : segs[0].rb;
  plan->n_rows = n_rows;
  const bool plain = (flags & PQ_SCAN_PLAIN) != 0;
  plan->tuning = ctx->tuning;
  plan->staged_expand = plan->tuning.staged_expand && !env_flag("PQ_NO_STAGED_EXPAND");
  const int64_t item_rows_max = plan->tuning.item_rows;
  uint64_t scratch = 0;
  uint64_t tc_pool = 0;               // DELTA_BYTE_ARRAY pool bytes
  std::vector<int64_t> data_job_off;  // scratch offset per data snappy job
  std::vector<int64_t> walk_cost;     // estimated chain steps per walked page
  std::vector<int32_t> dict_job_of_chunk(idx->chunks.size(), -1);
  uint32_t blk_data = 0, blk_dict = 0;  // block slots of split data / dictionary pages
  {
    // at most every indexed page of the requested columns, once per row segment
    size_t np = 0;
    for (size_t ch = 0; ch < idx->chunks.size(); ++ch)
      for (int32_t c : cols)
        if (idx->chunk_col[ch] == c) np += idx->chunks[ch].page_count;
    np *= segs.size();
    plan->pps.reserve(np);
    plan->walk_pps.reserve(np);
    walk_cost.reserve(np);
    if (idx->chunks.size() && idx->chunks[0].codec != pqi::CODEC_NONE) {
      plan->snappy_data.reserve(np);
      data_job_off.reserve(np);
    }
  }
  for (size_t oc = 0; oc < plan->cols.size(); ++oc) {
    const int c = plan->cols[oc];
    const auto& cm = idx->schema[c];
    pq_plan::ColWork cw;
    cw.snap_data_begin = static_cast<int>(plan->snappy_data.size());
    cw.snap_dict_begin = static_cast<int>(plan->snappy_dict.size());
    cw.dict_begin = static_cast<int>(plan->dict_jobs.size());
    cw.walk_begin = static_cast<int>(plan->walk_pps.size());
    cw.delta_begin = static_cast<int>(plan->delta_pps.size());
    cw.tc_begin = static_cast<int>(plan->tc_jobs.size());
    cw.blk_data_begin = blk_data;
    cw.blk_dict_begin = blk_dict;
    cw.copy_only = cm.repetition != 1 && cm.type != pqi::T_BYTE_ARRAY;
    const int max_fixed_before = plan->max_fixed_dict_bytes;
    plan->max_fixed_dict_bytes = 0;
    pqi::OutCol col{};
    col.n_rows = plan->n_rows;
    col.ptype = cm.type;
    col.width = pqi::type_width(cm.type);
    col.optional = cm.repetition == 1;
    col.item_begin = static_cast<uint32_t>(plan->n_items);
    pq_out_size sz{};
    sz.n_rows = plan->n_rows;
    sz.type = cm.type;
    sz.optional = col.optional;
    sz.values_bytes = cm.type == pqi::T_BYTE_ARRAY ? static_cast<uint64_t>(plan->n_rows + 1) * 8
                                                   : static_cast<uint64_t>(plan->n_rows) * col.width;
    sz.validity_bytes = col.optional ? static_cast<uint64_t>((plan->n_rows + 31) / 32) * 4 : 0;
    uint64_t chars = 0;
    for (const RowSeg& seg : segs)
    for (size_t ch = 0; ch < idx->chunks.size(); ++ch) {
      const int64_t rb = seg.rb, re = seg.re;
      if (idx->chunk_col[ch] != c) continue;
      const auto& cd = idx->chunks[ch];
      const int64_t c0 = idx->chunk_first_row[ch];
      const int64_t c1 = c0 + cd.num_values;
      if (c1 <= rb || c0 >= re) continue;
      if (cm.type == pqi::T_BYTE_ARRAY) {
        if (idx->chunk_ba_bytes[ch] < 0)
          cw.unsized = true;  // no SizeStatistics: a sizing scan at upload counts the chars
        else
          chars += static_cast<uint64_t>(idx->chunk_ba_bytes[ch]);
      }
      const int32_t pp_first = static_cast<int32_t>(plan->pps.size());
      bool tc_chunk_counted = false;  // this visit's chars are in the pool size
      // dictionary of this chunk
      int32_t dict = -1;
      if (cd.dict_page >= 0) {
        dict = static_cast<int32_t>(ch);
        if (dict_job_of_chunk[ch] < 0) {
          const auto& dp = idx->pages[cd.dict_page];
          pqi::DictJob dj{};
          const uint8_t* stored = cd.base + dp.offset + dp.header_len;
          if (cd.codec != pqi::CODEC_NONE) {
            pqi::SnappyJob sj{};
            sj.src = stored;
            sj.dst = idx->dict_body[ch];
            sj.src_len = static_cast<uint32_t>(dp.compressed);
            sj.dst_len = static_cast<uint32_t>(dp.uncompressed);
            sj.page = cd.dict_page;
            sj.codec = cd.codec;
            plan_split(sj, plain, &blk_dict);
            if (cd.codec == pqi::CODEC_ZSTD) plan->zstd_jobs++;
            plan->snappy_dict.push_back(sj);
            dj.body = idx->dict_body[ch];
          } else {
            dj.body = stored;
          }
          dj.body_len = dp.uncompressed;
          dj.n = dp.num_values;
          dj.ptype = cd.ptype;
          dj.width = cd.width;
          dj.page = cd.dict_page;
          dj.chunk = static_cast<int32_t>(ch);
          dj.values = idx->dict_values[ch];
          dj.str_ent = idx->dict_str_ent[ch];
          dj.pad = idx->dict_pad[ch];
          if (cd.ptype == pqi::T_BYTE_ARRAY) {
            dj.sreg = static_cast<uint32_t>(plan->dict_regions);
            dj.sreg_cap = static_cast<int32_t>(dp.uncompressed / pqi::STR_REGION + 2);
            plan->dict_regions += static_cast<uint64_t>(dj.sreg_cap);
            cw.max_str_regions = std::max(cw.max_str_regions, dj.sreg_cap);
          }
          if (cd.ptype != pqi::T_BYTE_ARRAY)
            plan->max_fixed_dict_bytes =
                std::max<int>(plan->max_fixed_dict_bytes, dp.num_values * cd.width);
          dict_job_of_chunk[ch] = static_cast<int32_t>(plan->dict_jobs.size());
          plan->dict_jobs.push_back(dj);
          plan->dict_chunks.push_back(static_cast<int32_t>(ch));
          plan->read_bytes += static_cast<uint64_t>(dp.header_len) + static_cast<uint64_t>(dp.compressed);
        }
      }
      if (dict >= 0) {
        const int64_t dn = idx->pages[cd.dict_page].num_values;
        cw.max_dict_n = std::max(cw.max_dict_n, dn);
        if (cd.ptype != pqi::T_BYTE_ARRAY) cw.max_dict_bytes = std::max<int64_t>(cw.max_dict_bytes, dn * cd.width);
      }
      for (uint32_t k = 0; k < cd.page_count; ++k) {
        const uint32_t pid = cd.page_begin + k;
        const auto& pg = idx->pages[pid];
        if (pg.page_type == pqi::PAGE_DICT) continue;
        const int64_t p0 = c0 + pg.first_row;
        const int64_t p1 = p0 + pg.num_values;
        if (p1 <= rb || p0 >= re || pg.num_values == 0) continue;
        // BYTE_STREAM_SPLIT and the delta string encodings are rewritten into
        // PLAIN bodies first; the decode kernels then read them as PLAIN
        const int32_t enc = pg.encoding;
        const bool tc = enc == pqi::ENC_BSS || enc == pqi::ENC_DELTA_LBA || enc == pqi::ENC_DELTA_BA;
        if (tc && (enc == pqi::ENC_BSS) == (cd.ptype == pqi::T_BYTE_ARRAY))
          return fail(ctx, PQ_ERR_CORRUPT, enc == pqi::ENC_BSS ? "BYTE_STREAM_SPLIT on a BYTE_ARRAY column"
                                                                : "delta string encoding on a fixed-width column");
        const int32_t eff = tc ? static_cast<int32_t>(pqi::ENC_PLAIN) : enc;
        pqi::PlanPage pp{};
        pp.enc = eff;
        pp.page = pid;
        pp.chunk = static_cast<uint32_t>(ch);
        pp.col = static_cast<int32_t>(oc);
        pp.row_lo = static_cast<int32_t>(std::max<int64_t>(rb - p0, 0));
        pp.row_hi = static_cast<int32_t>(std::min<int64_t>(re - p0, pg.num_values));
        pp.out_row = seg.out0 + p0 - rb;
        pp.dict = dict;
        pp.body_len = pg.uncompressed;
        pp.nonnull = -1;
        const uint8_t* stored = cd.base + pg.offset + pg.header_len;
        const bool v2_raw = pg.page_type == pqi::PAGE_DATA_V2 && !pg.v2_compressed;
        if (cd.codec != pqi::CODEC_NONE && !v2_raw) {
          pqi::SnappyJob sj{};
          sj.src = stored;
          sj.src_len = static_cast<uint32_t>(pg.compressed);
          sj.dst_len = static_cast<uint32_t>(pg.uncompressed);
          sj.prefix = pg.page_type == pqi::PAGE_DATA_V2 ? static_cast<uint32_t>(pg.def_len + pg.rep_len) : 0u;
          sj.page = static_cast<int32_t>(pid);
          sj.codec = cd.codec;
          plan_split(sj, plain, &blk_data);
          if (cd.codec == pqi::CODEC_ZSTD) plan->zstd_jobs++;
          data_job_off.push_back(static_cast<int64_t>(scratch));
          plan->snappy_data.push_back(sj);
          if (sj.nsub == 0) {  // (split pages are decompressed by blocks)
            cw.snap_data_max = std::max<uint32_t>(cw.snap_data_max, sj.src_len);
            plan->snap_data_max = std::max<uint32_t>(plan->snap_data_max, sj.src_len);
          }
          pp.body = reinterpret_cast<const uint8_t*>(static_cast<uintptr_t>(scratch));  // rebased below
          pp.pad = 1;  // body is a scratch offset until rebased
          scratch += (static_cast<uint64_t>(pg.uncompressed) + 32 + 15) & ~uint64_t(15);
        } else {
          if (pg.compressed != pg.uncompressed)
            return fail(ctx, PQ_ERR_CORRUPT, "stored page size differs from its uncompressed size");
          pp.body = stored;
        }
        plan->read_bytes += static_cast<uint64_t>(pg.header_len) + static_cast<uint64_t>(pg.compressed);
        if (tc) {
          pqi::TranscodeJob j{};
          j.src = pp.pad == 1 ? nullptr : stored;  // a decompressed body is rebased at upload
          j.src_len = static_cast<uint32_t>(pg.uncompressed);
          j.pp = static_cast<uint32_t>(plan->pps.size());
          j.page = static_cast<int32_t>(pid);
          j.enc = enc;
          j.width = cd.width;
          j.levels = pg.page_type == pqi::PAGE_DATA_V2 ? pg.def_len + pg.rep_len : (cd.max_def ? -1 : 0);
          j.num_values = pg.num_values;
          j.required = cd.max_def ? 0 : 1;
          plan->tc_src_off.push_back(pp.pad == 1 ? static_cast<int64_t>(reinterpret_cast<uintptr_t>(pp.body)) : -1);
          if (enc == pqi::ENC_DELTA_BA && idx->chunk_ba_bytes[ch] < 0)
            return fail(ctx, PQ_ERR_UNSUPPORTED, "DELTA_BYTE_ARRAY chunk without size statistics");
          if (enc == pqi::ENC_DELTA_BA) {
            // the PLAIN size is known only on the device: the page takes a piece
            // of a pool that holds its levels, length words and padding, plus
            // (once per chunk) the chunk's value bytes
            plan->tc_dst_off.push_back(-1);
            tc_pool += (static_cast<uint64_t>(pg.uncompressed) + 4ull * static_cast<uint64_t>(pg.num_values) + 63) &
                       ~uint64_t(15);
            if (!tc_chunk_counted) {
              tc_pool += (static_cast<uint64_t>(idx->chunk_ba_bytes[ch]) + 15) & ~uint64_t(15);
              tc_chunk_counted = true;
            }
          } else {
            const uint64_t cap = static_cast<uint64_t>(pg.uncompressed) +
                                 (enc == pqi::ENC_DELTA_LBA ? 4ull * static_cast<uint64_t>(pg.num_values) : 0);
            if (cap > 0x7fffffffull) return fail(ctx, PQ_ERR_UNSUPPORTED, "transcoded page above 2 GiB");
            j.dst_cap = static_cast<uint32_t>(cap);
            plan->tc_dst_off.push_back(static_cast<int64_t>(scratch));
            scratch += (cap + 32 + 15) & ~uint64_t(15);
          }
          if (enc != pqi::ENC_BSS) {
            // the transcoder records where each value starts, so that the
            // walk need not follow the (length, bytes) chain
            pp.vtab = static_cast<uint32_t>(1 + plan->vpos_rows);
            plan->vpos_rows += static_cast<uint64_t>(pg.num_values) + 1;
          }
          plan->tc_jobs.push_back(j);
        }
        pp.item_begin = static_cast<uint32_t>(plan->n_items);
        if (eff == pqi::ENC_RLE_DICT || eff == pqi::ENC_PLAIN_DICT) cw.dict_pages++;
        const bool plain_fixed = eff == pqi::ENC_PLAIN && cd.ptype != pqi::T_BYTE_ARRAY;
        if (!plain_fixed || cd.max_def) cw.copy_only = false;
        const bool needs_walk = cd.max_def || !plain_fixed;
        if (!cd.max_def) {
          // REQUIRED: the value stream starts after the (empty) levels
          if (pg.page_type == pqi::PAGE_DATA_V2 && (pg.rep_len != 0 || pg.def_len != 0))
            return fail(ctx, PQ_ERR_CORRUPT, "levels in a page of a REQUIRED column");
          pp.values_off = 0;
          pp.nonnull = pg.num_values;
        }
        if (eff == pqi::ENC_DELTA_BP) {
          pp.dtab = static_cast<uint32_t>(plan->delta_blocks);
          plan->delta_blocks += pg.num_values > 1 ? static_cast<uint64_t>(pg.num_values - 2) / 128 + 1 : 1;
          pp.dreg = static_cast<uint32_t>(plan->delta_regions);
          pp.dreg_cap = static_cast<int32_t>(pg.uncompressed / pqi::DELTA_REGION + 2);
          plan->delta_regions += static_cast<uint64_t>(pp.dreg_cap);
          cw.max_regions = std::max(cw.max_regions, pp.dreg_cap);
          plan->delta_pps.push_back(static_cast<uint32_t>(plan->pps.size()));
        }
        if (needs_walk && !plain) {
          plan->walk_pps.push_back(static_cast<uint32_t>(plan->pps.size()));
          walk_cost.push_back(eff == pqi::ENC_DELTA_BP ? pg.num_values / 128 + (cd.max_def ? pg.num_values / 8 : 0)
                              : cd.max_def ? pg.num_values / 8
                              : cd.ptype == pqi::T_BYTE_ARRAY && eff == pqi::ENC_PLAIN ? pg.num_values
                                                                                                 : pg.num_values / 256);
        }
        const int64_t span = pp.row_hi - pp.row_lo;
        // pages with definition levels take the short items (their walks and
        // expands carry a bitmap per item; measured faster for PLAIN too)
        const int64_t per = cd.max_def ? plan->tuning.item_rows_opt : item_rows_max;
        const uint32_t n_it = static_cast<uint32_t>((span + per - 1) / per);
        pp.item_rows = static_cast<int32_t>(per);
        pp.item_count = n_it;
        plan->n_items += n_it;
        plan->pps.push_back(pp);
      }
      const int32_t n_pp = static_cast<int32_t>(plan->pps.size()) - pp_first;
      if (n_pp > 0) {
        plan->chunk_pp.emplace_back(pp_first, n_pp);
        plan->chunk_pp_chunk.push_back(static_cast<int32_t>(ch));
      }
    }
    col.item_count = static_cast<uint32_t>(plan->n_items) - col.item_begin;
    cw.snap_data_n = static_cast<int>(plan->snappy_data.size()) - cw.snap_data_begin;
    cw.snap_dict_n = static_cast<int>(plan->snappy_dict.size()) - cw.snap_dict_begin;
    cw.dict_n = static_cast<int>(plan->dict_jobs.size()) - cw.dict_begin;
    cw.walk_n = static_cast<int>(plan->walk_pps.size()) - cw.walk_begin;
    cw.delta_n = static_cast<int>(plan->delta_pps.size()) - cw.delta_begin;
    cw.tc_n = static_cast<int>(plan->tc_jobs.size()) - cw.tc_begin;
    cw.blk_data_n = blk_data - cw.blk_data_begin;
    cw.blk_dict_n = blk_dict - cw.blk_dict_begin;
    cw.max_fixed_dict = plan->max_fixed_dict_bytes;
    plan->max_fixed_dict_bytes = std::max(max_fixed_before, plan->max_fixed_dict_bytes);
    plan->colwork.push_back(cw);
    sz.chars_bytes = cw.unsized ? 0 : chars;
    if (cw.unsized) plan->needs_sizing = true;
    if (cm.type == pqi::T_BYTE_ARRAY) plan->str_cols.push_back(static_cast<int32_t>(oc));
    plan->decoded_bytes += sz.values_bytes + sz.validity_bytes + sz.chars_bytes;
    plan->outcols.push_back(col);
    plan->sizes.push_back(sz);
  }
  // walk list: inside each column, longest header chains first
  for (const auto& cw : plan->colwork) {
    std::vector<size_t> order(cw.walk_n);
    for (int i = 0; i < cw.walk_n; ++i) order[i] = cw.walk_begin + i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return walk_cost[x] > walk_cost[y]; });
    std::vector<uint32_t> sorted(order.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = plan->walk_pps[order[i]];
    std::copy(sorted.begin(), sorted.end(), plan->walk_pps.begin() + cw.walk_begin);
  }
  // the block list: data pages' blocks, then dictionary pages' blocks
  for (auto& sj : plan->snappy_dict)
    if (sj.nsub > 1) sj.sub += blk_data;
  for (auto& cw : plan->colwork) cw.blk_dict_begin += blk_data;
  plan->snap_blocks = blk_data + blk_dict;
  plan->tc_pool_off = scratch;
  plan->tc_pool_bytes = tc_pool;
  scratch += tc_pool;
  plan->device_bytes = plan_device_bytes(plan.get(), scratch);
  plan->host_scratch = scratch;
  *out = std::move(plan);
  return PQ_OK;
}

static pq_status plan_size_strings(pq_plan* plan);

// Device half: allocations from the context's pool, uploads, work items,
// events, pinned staging.  The uploads go on stream `s` (nullptr: the legacy
// default stream), where the plan's `ready` event is recorded.
pq_status plan_upload(pq_plan* plan, cudaStream_t s) {
  pq_ctx* ctx = plan->ctx;
  const bool plain = (plan->flags & PQ_SCAN_PLAIN) != 0;
  const uint64_t scratch = plan->host_scratch;
  // device arrays
  const size_t npp = plan->pps.size(), nit = plan->n_items;
  plan->d_walk_pps = plan_alloc(uint32_t, plan, plan->walk_pps.size());
  plan->d_delta_pps = plan_alloc(uint32_t, plan, plan->delta_pps.size());
  plan->d_dpos = plan_alloc(uint32_t, plan, plan->delta_blocks);
  plan->d_dbase = plan_alloc(int64_t, plan, plan->delta_blocks);
  plan->d_dregs = plan_alloc(pqi::DeltaRegion, plan, plan->delta_regions);
  plan->d_dreg_lists = plan_alloc(uint32_t, plan, plan->delta_regions * pqi::DELTA_REGION_LIST);
  plan->d_sregs = plan_alloc(pqi::DeltaRegion, plan, plan->dict_regions);
  plan->d_slists = plan_alloc(uint64_t, plan, plan->dict_regions * pqi::STR_REGION_LIST);
  plan->d_pps = plan_alloc(pqi::PlanPage, plan, npp);
  plan->d_items = plan_alloc(pqi::Item, plan, nit);
  plan->d_cols = plan_alloc(pqi::OutCol, plan, plan->outcols.size());
  plan->d_snappy = plan_alloc(pqi::SnappyJob, plan, plan->snappy_data.size() + plan->snappy_dict.size());
  plan->d_snap_blocks = plan_alloc(pqi::SnappyJob, plan, plan->snap_blocks);
  plan->d_vpos = plan_alloc(uint32_t, plan, plan->vpos_rows);
  plan->d_dict_jobs = plan_alloc(pqi::DictJob, plan, plan->dict_jobs.size());
  plan->d_tc_jobs = plan_alloc(pqi::TranscodeJob, plan, plan->tc_jobs.size());
  plan->d_str_cols = plan_alloc(int32_t, plan, plan->str_cols.size());
  plan->d_counter = plan_alloc(uint32_t, plan, 4 + plan->outcols.size());
  plan->d_status = plan_alloc(pqi::DevStatus, plan, 1);
  plan->d_scratch = scratch ? plan_alloc(uint8_t, plan, scratch + 64) : nullptr;
  const uint64_t str_rows = static_cast<uint64_t>(plan->n_rows) * plan->str_cols.size();
  plan->d_str_scratch = str_rows ? plan_alloc(uint64_t, plan, str_rows) : nullptr;
  plan->d_str_items = plan->str_cols.empty() ? nullptr : plan_alloc(uint64_t, plan, nit);
  for (void* p : plan->owned)
    if (!p) {
      free_plan_device(plan);
      return fail(ctx, PQ_ERR_OOM, "plan allocation");
    }
  if ((scratch && !plan->d_scratch) || (str_rows && !plan->d_str_scratch)) {
    free_plan_device(plan);
    return fail(ctx, PQ_ERR_OOM, "plan scratch");
  }
  plan->scratch_bytes = scratch + str_rows * 8 + (plan->d_str_items ? nit * 8 : 0) + plan->delta_blocks * 12 +
                        plan->delta_regions * (sizeof(pqi::DeltaRegion) + 4ull * pqi::DELTA_REGION_LIST);
  // rebase scratch bodies, string scratch per column
  size_t jd = 0;
  for (auto& pp : plan->pps) {
    if (pp.pad == 1) {
      uint8_t* b = plan->d_scratch + reinterpret_cast<uintptr_t>(pp.body);
      pp.body = b;
      plan->snappy_data[jd].dst = b;
      ++jd;
      pp.pad = 0;
    }
  }
  // transcode jobs: sources and destinations in the scratch; the plan page
  // reads the PLAIN body (DELTA_BYTE_ARRAY: its source until the kernel
  // points it at its piece of the pool)
  for (size_t i = 0; i < plan->tc_jobs.size(); ++i) {
    auto& j = plan->tc_jobs[i];
    if (plan->tc_src_off[i] >= 0) j.src = plan->d_scratch + plan->tc_src_off[i];
    j.dst = plan->tc_dst_off[i] >= 0 ? plan->d_scratch + plan->tc_dst_off[i] : nullptr;
    plan->pps[j.pp].body = j.dst ? j.dst : j.src;
  }
  for (size_t i = 0; i < plan->str_cols.size(); ++i) {
    auto& col = plan->outcols[plan->str_cols[i]];
    col.str_scratch = plan->d_str_scratch + static_cast<uint64_t>(plan->n_rows) * i;
    col.str_item_bytes = plan->d_str_items;
  }
  // upload, through one pinned staging block
  std::vector<pqi::SnappyJob> alljobs(plan->snappy_data);
  alljobs.insert(alljobs.end(), plan->snappy_dict.begin(), plan->snappy_dict.end());
  struct Up {
    void* dst;
    const void* src;
    size_t bytes;
  };
  const Up ups[] = {
      {plan->d_pps, plan->pps.data(), sizeof(pqi::PlanPage) * npp},
      {plan->d_snappy, alljobs.data(), sizeof(pqi::SnappyJob) * alljobs.size()},
      {plan->d_dict_jobs, plan->dict_jobs.data(), sizeof(pqi::DictJob) * plan->dict_jobs.size()},
      {plan->d_tc_jobs, plan->tc_jobs.data(), sizeof(pqi::TranscodeJob) * plan->tc_jobs.size()},
      {plan->d_str_cols, plan->str_cols.data(), sizeof(int32_t) * plan->str_cols.size()},
      {plan->d_walk_pps, plan->walk_pps.data(), sizeof(uint32_t) * plan->walk_pps.size()},
      {plan->d_delta_pps, plan->delta_pps.data(), sizeof(uint32_t) * plan->delta_pps.size()},
  };
  size_t up_bytes = 0;
  for (const Up& u : ups) up_bytes += (u.bytes + 15) & ~size_t(15);
  if (!ctx->pinned.take(up_bytes, &plan->h_up)) {
    free_plan_device(plan);
    return fail(ctx, PQ_ERR_OOM, "pinned staging");
  }
  size_t up_off = 0;
  for (const Up& u : ups) {
    if (!u.bytes) continue;
    memcpy(plan->h_up.p + up_off, u.src, u.bytes);
    CK(cudaMemcpyAsync(u.dst, plan->h_up.p + up_off, u.bytes, cudaMemcpyHostToDevice, s));
    up_off += (u.bytes + 15) & ~size_t(15);
  }
  if (nit) pqi::launch_make_items(decode_args(plan), static_cast<int>(npp), s);
  // no host wait: a scan's stream waits on this event (the host arrays are
  // plan members, alive until the plan is freed)
  CK(ctx->events.take(&plan->ready));
  CK(cudaEventRecord(plan->ready, s));
  CK(ctx->events.take(&plan->done));
  if (plan->flags & PQ_SCAN_TIMING)
    for (auto& e : plan->stage_ev) CK(cudaEventCreate(&e));
  CK(ctx->events.take(&plan->fork));
  plan->join.assign(plan->outcols.size(), nullptr);
  for (auto& e : plan->join) CK(ctx->events.take(&e));
  {
    // kernels per scan: prepare, snappy, dictionary (2), walk + expand or one
    // plain launch (+ its snappy) per chunk, strings (2)
    int n = 1;
    const bool any_dict = !plan->dict_jobs.empty();
    if (plain) {
      n += (plan->snappy_dict.empty() ? 0 : (plan->zstd_jobs ? 2 : 1)) + (any_dict ? 2 : 0);
      size_t job = 0;
      for (auto& cp : plan->chunk_pp) {
        int nj = 0;
        for (int q = cp.first; q < cp.first + cp.second; ++q)
          if (job + nj < plan->snappy_data.size() && plan->snappy_data[job + nj].page == static_cast<int32_t>(plan->pps[q].page))
            ++nj;
        n += (nj ? (plan->zstd_jobs ? 2 : 1) : 0) + 1;
        job += nj;
      }
      size_t tcj = 0;
      for (auto& cp : plan->chunk_pp) {
        int ntc = 0;
        while (tcj + ntc < plan->tc_jobs.size() &&
               plan->tc_jobs[tcj + ntc].pp < static_cast<uint32_t>(cp.first + cp.second))
          ++ntc;
        n += ntc ? 1 : 0;
        tcj += ntc;
      }
    } else {
      for (size_t oc = 0; oc < plan->colwork.size(); ++oc) {
        const auto& cw = plan->colwork[oc];
        const int dk = plan->zstd_jobs ? 2 : 1;  // decompression kernels per job list
        // (+2 per job list with split pages: the fragment scan and the blocks)
        n += (cw.snap_dict_n ? dk + (cw.blk_dict_n ? 2 : 0) : 0) + (cw.dict_n ? 2 : 0) +
             (cw.snap_data_n ? dk + (cw.blk_data_n ? 2 : 0) : 0) + (cw.walk_n ? 1 : 0) +
             (cw.delta_n ? 4 : 0) + (cw.tc_n ? 1 : 0) + (plan->outcols[oc].item_count ? 1 : 0);
      }
    }
    for (int32_t sc : plan->str_cols) n += plan->outcols[sc].item_count ? 2 : 0;
    plan->launches = n;
  }
  const int wbps = pqi::walk_blocks_per_sm(), ebps = pqi::expand_blocks_per_sm();
  plan->walk_grid =
      static_cast<int>(std::min<size_t>(std::max<size_t>(plan->walk_pps.size(), 1), size_t(ctx->n_sms) * wbps));
  plan->expand_grid = static_cast<int>(std::min<size_t>(std::max<size_t>((nit + 7) / 8, 1), size_t(ctx->n_sms) * ebps));
  if (!ctx->pinned.take(sizeof(pqi::OutCol) * std::max<size_t>(plan->outcols.size(), 1), &plan->h_cols) ||
      !ctx->pinned.take(sizeof(pqi::DevStatus) + 8 * std::max<size_t>(plan->outcols.size(), 1), &plan->h_out)) {
    free_plan_device(plan);
    return fail(ctx, PQ_ERR_OOM, "pinned staging");
  }
  if (plan->needs_sizing) return plan_size_strings(plan);
  return PQ_OK;
}

// Chars of string columns whose chunks carry no SizeStatistics: one scan
// into temporary outputs without the chars copy (the string offsets pass
// still totals each column), on a private stream, then the totals become
// the plan's chars_bytes.
static pq_status plan_size_strings(pq_plan* plan) {
  pq_ctx* ctx = plan->ctx;
  const size_t nc = plan->outcols.size();
  std::vector<pq_column> outs(nc);
  std::vector<void*> tmp;
  bool oom = false;
  for (size_t i = 0; i < nc; ++i) {
    const auto& sz = plan->sizes[i];
    memset(&outs[i], 0, sizeof outs[i]);
    void* v = ctx->pool.alloc(std::max<uint64_t>(sz.values_bytes, 16));
    tmp.push_back(v);
    outs[i].values = v;
    oom |= !v;
    if (sz.optional) {
      void* m = ctx->pool.alloc(std::max<uint64_t>(sz.validity_bytes, 16));
      tmp.push_back(m);
      outs[i].validity = static_cast<uint32_t*>(m);
      oom |= !m;
    }
  }
  cudaStream_t s = nullptr;
  pq_status st = PQ_OK;
  if (oom) {
    st = fail(ctx, PQ_ERR_OOM, "string sizing buffers");
  } else if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = fail(ctx, PQ_ERR_CUDA, "string sizing stream");
  } else {
    plan->sizing = true;
    st = scan_enqueue(plan, outs.data(), s, &s, 1, false);
    plan->sizing = false;
    if (st == PQ_OK) {
      const cudaError_t e = cudaEventSynchronize(plan->done);
      if (e != cudaSuccess) {
        st = cuda_fail(ctx, e, "string sizing scan");
      } else {
        pqi::DevStatus ds;
        memcpy(&ds, plan->h_out.p, sizeof ds);
        st = status_from_device(ctx, ds);
      }
    }
    cudaStreamDestroy(s);
  }
  if (st == PQ_OK) {
    for (size_t j = 0; j < plan->str_cols.size(); ++j) {
      int64_t v;
      memcpy(&v, plan->h_out.p + sizeof(pqi::DevStatus) + 8 * j, 8);
      auto& sz = plan->sizes[plan->str_cols[j]];
      if (plan->colwork[plan->str_cols[j]].unsized) {
        sz.chars_bytes = static_cast<uint64_t>(v);
        plan->decoded_bytes += static_cast<uint64_t>(v);
      }
    }
  }
  for (void* p : tmp) ctx->pool.free(p);
  return st;
}

uint64_t plan_device_bytes(const pq_plan* plan, uint64_t scratch) {
  const uint64_t npp = plan->pps.size(), nit = plan->n_items;
  const uint64_t str_rows = static_cast<uint64_t>(plan->n_rows) * plan->str_cols.size();
  return npp * sizeof(pqi::PlanPage) + nit * sizeof(pqi::Item) + plan->outcols.size() * sizeof(pqi::OutCol) +
         (plan->snappy_data.size() + plan->snappy_dict.size() + plan->snap_blocks) * sizeof(pqi::SnappyJob) +
         4 * plan->vpos_rows +
         plan->dict_jobs.size() * sizeof(pqi::DictJob) + plan->tc_jobs.size() * sizeof(pqi::TranscodeJob) +
         4 * (plan->walk_pps.size() + plan->delta_pps.size()) +
         plan->delta_blocks * 12 +
         plan->delta_regions * (sizeof(pqi::DeltaRegion) + 4ull * pqi::DELTA_REGION_LIST) +
         plan->dict_regions * (sizeof(pqi::DeltaRegion) + 8ull * pqi::STR_REGION_LIST) + scratch + 64 +
         str_rows * 8 + (plan->str_cols.empty() ? 0 : nit * 8) + 4096;
}

}  // namespace pqe

extern "C" {

pq_status pq_plan_scan(pq_ctx* ctx, pq_index* idx, const pq_request* req, pq_plan** out, pq_out_size* sizes) {
  return pqe::plan_scan_on(ctx, idx, req, nullptr, out, sizes);
}

}  // extern "C"

namespace pqe {

pq_status plan_scan_on(pq_ctx* ctx, pq_index* idx, const pq_request* req, cudaStream_t stream, pq_plan** out,
                       pq_out_size* sizes) {
  if (!ctx || !idx || !req || !out) return fail(ctx, PQ_ERR_INVALID_ARG, "pq_plan_scan: bad arguments");
  *out = nullptr;
  CK(cudaSetDevice(ctx->device));
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::vector<int32_t> cols;
  if (req->columns) {
    for (int i = 0; i < req->n_columns; ++i) {
      if (req->columns[i] < 0 || req->columns[i] >= idx->n_columns)
        return fail(ctx, PQ_ERR_INVALID_ARG, "column id out of range");
      cols.push_back(req->columns[i]);
    }
  } else {
    for (int i = 0; i < idx->n_columns; ++i) cols.push_back(i);
  }
  if (req->row_begin < 0 || req->row_begin > idx->num_rows)
    return fail(ctx, PQ_ERR_INVALID_ARG, "row range outside the indexed rows");
  const int64_t rb = req->row_begin;
  const int64_t re = req->row_count < 0 ? idx->num_rows : rb + req->row_count;
  if (re > idx->num_rows) return fail(ctx, PQ_ERR_INVALID_ARG, "row range outside the indexed rows");
  std::unique_ptr<pq_plan> plan;
  pq_status st = plan_build(ctx, idx, cols, {RowSeg{rb, re, 0}}, re - rb, req->flags, &plan);
  if (st != PQ_OK) return st;
  st = plan_upload(plan.get(), stream);
  if (st != PQ_OK) return st;
  if (sizes)
    for (size_t i = 0; i < plan->sizes.size(); ++i) sizes[i] = plan->sizes[i];
  *out = plan.release();
  return PQ_OK;
}

}  // namespace pqe

extern "C" {

pq_status pq_plan_get_info(const pq_plan* plan, pq_plan_info* out) {
  if (!plan || !out) return PQ_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  out->n_columns = static_cast<int32_t>(plan->cols.size());
  out->n_pages = static_cast<int32_t>(plan->pps.size());
  out->n_dict_pages = static_cast<int32_t>(plan->dict_jobs.size());
  out->n_items = static_cast<int32_t>(plan->n_items);
  out->read_bytes = plan->read_bytes;
  out->decoded_bytes = plan->decoded_bytes;
  out->scratch_bytes = plan->scratch_bytes;
  out->launches_per_scan = plan->launches;
  return PQ_OK;
}

pq_status pq_plan_stage_ms(const pq_plan* plan, float* ms) {
  if (!plan || !ms) return PQ_ERR_INVALID_ARG;
  if (!(plan->flags & PQ_SCAN_TIMING) || !plan->stage_ev[0]) return PQ_ERR_INVALID_ARG;
  for (int i = 0; i < PQ_N_STAGES; ++i) {
    ms[i] = 0.f;
    if (cudaEventElapsedTime(&ms[i], plan->stage_ev[i], plan->stage_ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      return PQ_ERR_CUDA;
    }
  }
  return PQ_OK;
}

// ------------------------------------------------------------------ scan

static int max_str_regions_all(const pq_plan* plan) {
  int m = 0;
  for (const auto& cw : plan->colwork) m = std::max(m, cw.max_str_regions);
  return m;
}

static void enqueue_transcode(pq_plan* plan, int begin, int n, const pqi::DecodeArgs& a, cudaStream_t s) {
  if (n <= 0) return;
  pqi::launch_transcode(plan->d_tc_jobs + begin, n, plan->d_pps, plan->d_scratch + plan->tc_pool_off,
                        plan->tc_pool_bytes, plan->d_counter, plan->d_vpos, a.st, s);
}

// Compressed data pages of at least this many bytes (the tuning's
// snappy_block_kib) are decompressed by a block of 8 warps each (long
// literals copied by all of them); smaller ones by one warp each.
// Dictionary pages always take a block.
static uint32_t coop_snappy_bytes(const pq_plan* plan) {
  return static_cast<uint32_t>(std::min<int64_t>(int64_t(plan->tuning.snappy_block_kib) * 1024, 0xffffffffll));
}

// Decompression of jobs [jobs, jobs + n): the Snappy kernel takes the Snappy
// pages, the Zstandard kernel (launched when the plan has any) the others.
// Split Snappy pages (blocks [blk_begin, blk_begin + blk_n) of the plan's
// block list) are scanned for their fragments first; their blocks are then
// decompressed one warp each.
static void launch_decompress(pq_plan* plan, const pqi::SnappyJob* jobs, int n, uint32_t blk_begin, uint32_t blk_n,
                              bool coop, pqi::DevStatus* st, cudaStream_t s) {
  if (n <= 0) return;
  const int n_sms = plan->ctx->n_sms;
  if (blk_n) pqi::launch_snappy_split(jobs, n, plan->d_snap_blocks, n_sms, st, s);
  pqi::launch_snappy(jobs, n, n_sms, st, s, coop);
  if (plan->zstd_jobs) pqi::launch_zstd(jobs, n, n_sms, st, s);
  if (blk_n) pqi::launch_snappy(plan->d_snap_blocks + blk_begin, static_cast<int>(blk_n), n_sms, st, s, false);
}

// Expansion of one output column: copies (REQUIRED PLAIN fixed width), the
// staged dictionary expand (REQUIRED fixed width with dictionary pages), or
// the general warp decode.
static void launch_column_expand(pq_plan* plan, size_t oc, const pqi::DecodeArgs& a, cudaStream_t s) {
  pq_ctx* ctx = plan->ctx;
  const auto& cw = plan->colwork[oc];
  const auto& col = plan->outcols[oc];
  const int ib = static_cast<int>(col.item_begin), n = static_cast<int>(col.item_count);
  if (cw.copy_only) {
    pqi::launch_copy_items(a, ib, n, static_cast<int>(oc), ctx->n_sms, plan->tuning.expand_ctas_per_sm, s);
    return;
  }
  if (plan->staged_expand && !col.optional && (col.width == 4 || col.width == 8) && col.ptype != pqi::T_BYTE_ARRAY &&
      cw.dict_pages > 0) {
    int bw = 0;
    while (bw < 32 && (int64_t(1) << bw) < cw.max_dict_n) ++bw;
    const uint32_t stage = pqi::dict_expand_stage_bytes(plan->tuning.item_rows, bw);
    uint32_t dict_cap = static_cast<uint32_t>((cw.max_dict_bytes + 15) & ~int64_t(15));
    if (cw.max_dict_bytes > (int64_t(1) << 30) || !pqi::dict_expand_fits(stage, dict_cap)) dict_cap = 0;
    if (pqi::dict_expand_fits(stage, dict_cap)) {
      pqi::launch_dict_expand(a, ib, n, static_cast<int>(oc), ctx->n_sms, col.width, stage, dict_cap, s);
      return;
    }
  }
  pqi::launch_expand(a, ib, n, static_cast<int>(oc), ctx->n_sms, plan->tuning.expand_ctas_per_sm, s);
}

// Kernels of one output column, in order, on one stream.
static void enqueue_column(pq_plan* plan, size_t oc, const pqi::DecodeArgs& a, bool with_dicts, cudaStream_t s) {
  pq_ctx* ctx = plan->ctx;
  const auto& cw = plan->colwork[oc];
  const int n_data_total = static_cast<int>(plan->snappy_data.size());
  if (with_dicts && cw.snap_dict_n)
    launch_decompress(plan, plan->d_snappy + n_data_total + cw.snap_dict_begin, cw.snap_dict_n, cw.blk_dict_begin,
                      cw.blk_dict_n, true, a.st, s);
  if (with_dicts && cw.dict_n)
    pqi::launch_dict(plan->d_dict_jobs + cw.dict_begin, cw.dict_n, cw.max_fixed_dict, cw.max_str_regions,
                     pqi::DictScratch{plan->d_sregs, plan->d_slists}, plan->idx->d_dicts, ctx->n_sms, a.st, s);
  if (cw.snap_data_n)
    launch_decompress(plan, plan->d_snappy + cw.snap_data_begin, cw.snap_data_n, cw.blk_data_begin, cw.blk_data_n,
                      cw.snap_data_max >= coop_snappy_bytes(plan), a.st, s);
  enqueue_transcode(plan, cw.tc_begin, cw.tc_n, a, s);
  const auto& col = plan->outcols[oc];
  pqi::launch_walk(a, cw.walk_begin, cw.walk_n, ctx->n_sms, col.optional != 0, plan->tuning.walk_window, s);
  pqi::launch_delta_bases(a, cw.delta_begin, cw.delta_n, cw.max_regions, s);
  launch_column_expand(plan, oc, a, s);
  if (col.ptype == pqi::T_BYTE_ARRAY)
    pqi::launch_strings(a, static_cast<int>(oc), static_cast<int>(col.item_count), ctx->n_sms, !plan->sizing, s);
}

// Enqueues the kernels of one scan (no host synchronisation).  Default:
// every output column is an independent branch (fork/join through events on
// the context's branch streams), so that the serial header chains of one
// column overlap the bandwidth-bound expansion of the others.  With
// PQ_SCAN_TIMING the stages run one after another over all columns, so that
// each stage can be timed.  PQ_SCAN_PLAIN: per chunk, one launch per stage.
static void enqueue_scan(pq_plan* plan, cudaStream_t s, bool with_dicts, const cudaStream_t* branches,
                         int n_branches) {
  pq_ctx* ctx = plan->ctx;
  pqi::DecodeArgs a = decode_args(plan);
  const int ncols = static_cast<int>(plan->outcols.size());
  const bool timing = (plan->flags & PQ_SCAN_TIMING) != 0;
  auto mark = [&](int i) {
    if (timing) cudaEventRecord(plan->stage_ev[i], s);
  };
  mark(0);
  pqi::launch_prepare(a, ncols, ctx->n_sms * 4, s);
  mark(1);
  const int n_data_jobs = static_cast<int>(plan->snappy_data.size());
  const int n_dict_jobs = static_cast<int>(plan->snappy_dict.size());
  if (plan->flags & PQ_SCAN_PLAIN) {
    // baseline: per chunk, one launch per stage; one page per thread block
    if (with_dicts && n_dict_jobs)
      launch_decompress(plan, plan->d_snappy + n_data_jobs, n_dict_jobs, 0, 0, true, a.st, s);
    mark(2);
    if (with_dicts && !plan->dict_jobs.empty())
      pqi::launch_dict(plan->d_dict_jobs, static_cast<int>(plan->dict_jobs.size()), plan->max_fixed_dict_bytes,
                       max_str_regions_all(plan), pqi::DictScratch{plan->d_sregs, plan->d_slists}, plan->idx->d_dicts,
                       ctx->n_sms, a.st, s);
    mark(3);
    size_t job = 0, tcj = 0;
    for (size_t k = 0; k < plan->chunk_pp.size(); ++k) {
      const int first = plan->chunk_pp[k].first, n = plan->chunk_pp[k].second;
      int nj = 0;
      for (int p = first; p < first + n; ++p)
        if (job + nj < plan->snappy_data.size() && plan->snappy_data[job + nj].page == static_cast<int32_t>(plan->pps[p].page))
          ++nj;
      if (nj) launch_decompress(plan, plan->d_snappy + job, nj, 0, 0, plan->snap_data_max >= coop_snappy_bytes(plan), a.st, s);
      job += nj;
      int ntc = 0;
      while (tcj + ntc < plan->tc_jobs.size() && plan->tc_jobs[tcj + ntc].pp < static_cast<uint32_t>(first + n)) ++ntc;
      enqueue_transcode(plan, static_cast<int>(tcj), ntc, a, s);
      tcj += ntc;
      pqi::launch_plain_pages(a, first, n, s);
    }
    mark(4);
    mark(5);
    for (int32_t sc : plan->str_cols)
      pqi::launch_strings(a, sc, static_cast<int>(plan->outcols[sc].item_count), ctx->n_sms, !plan->sizing, s);
  } else if (timing) {
    for (int oc = 0; oc < ncols; ++oc) {
      const auto& cw = plan->colwork[oc];
      if (with_dicts && cw.snap_dict_n)
        launch_decompress(plan, plan->d_snappy + n_data_jobs + cw.snap_dict_begin, cw.snap_dict_n, cw.blk_dict_begin,
                          cw.blk_dict_n, true, a.st, s);
      if (cw.snap_data_n)
        launch_decompress(plan, plan->d_snappy + cw.snap_data_begin, cw.snap_data_n, cw.blk_data_begin, cw.blk_data_n,
                          cw.snap_data_max >= coop_snappy_bytes(plan), a.st, s);
      enqueue_transcode(plan, cw.tc_begin, cw.tc_n, a, s);
    }
    mark(2);
    for (int oc = 0; oc < ncols; ++oc) {
      const auto& cw = plan->colwork[oc];
      if (with_dicts && cw.dict_n)
        pqi::launch_dict(plan->d_dict_jobs + cw.dict_begin, cw.dict_n, cw.max_fixed_dict, cw.max_str_regions,
                         pqi::DictScratch{plan->d_sregs, plan->d_slists}, plan->idx->d_dicts, ctx->n_sms, a.st, s);
    }
    mark(3);
    for (int oc = 0; oc < ncols; ++oc) {
      const auto& cw = plan->colwork[oc];
      pqi::launch_walk(a, cw.walk_begin, cw.walk_n, ctx->n_sms, plan->outcols[oc].optional != 0,
                       plan->tuning.walk_window, s);
      pqi::launch_delta_bases(a, cw.delta_begin, cw.delta_n, cw.max_regions, s);
    }
    mark(4);
    for (int oc = 0; oc < ncols; ++oc) launch_column_expand(plan, oc, a, s);
    mark(5);
    for (int32_t sc : plan->str_cols)
      pqi::launch_strings(a, sc, static_cast<int>(plan->outcols[sc].item_count), ctx->n_sms, !plan->sizing, s);
  } else {
    cudaEventRecord(plan->fork, s);
    for (int oc = 0; oc < ncols; ++oc) {
      cudaStream_t b = branches[oc % n_branches];
      cudaStreamWaitEvent(b, plan->fork, 0);
      enqueue_column(plan, oc, a, with_dicts, b);
      cudaEventRecord(plan->join[oc], b);
    }
    for (int oc = 0; oc < ncols; ++oc) cudaStreamWaitEvent(s, plan->join[oc], 0);
  }
  mark(6);
  // status and string totals back to pinned host memory
  d2h_small(plan->h_out.p, plan->d_status, sizeof(pqi::DevStatus), s);
  for (size_t i = 0; i < plan->str_cols.size(); ++i) {
    const auto& col = plan->outcols[plan->str_cols[i]];
    d2h_small(plan->h_out.p + sizeof(pqi::DevStatus) + 8 * i, reinterpret_cast<int64_t*>(col.values) + plan->n_rows,
              8, s);
  }
}

}  // extern "C"

namespace pqe {

pq_status scan_enqueue(pq_plan* plan, const pq_column* outs, cudaStream_t s, const cudaStream_t* branches,
                       int n_branches, bool allow_graph) {
  pq_ctx* ctx = plan->ctx;
  // output descriptors
  bool changed = false;
  for (size_t i = 0; i < plan->outcols.size(); ++i) {
    auto& col = plan->outcols[i];
    const auto& sz = plan->sizes[i];
    if (!outs[i].values && sz.values_bytes) return fail(ctx, PQ_ERR_INVALID_ARG, "missing values buffer");
    if (col.optional && !outs[i].validity && sz.n_rows)
      return fail(ctx, PQ_ERR_INVALID_ARG, "missing validity buffer for an OPTIONAL column");
    if (!plan->sizing && col.ptype == pqi::T_BYTE_ARRAY && outs[i].chars_capacity < sz.chars_bytes)
      return fail(ctx, PQ_ERR_CAPACITY, "chars buffer smaller than the plan's chars_bytes");
    if (!plan->sizing && col.ptype == pqi::T_BYTE_ARRAY && !outs[i].chars && sz.chars_bytes)
      return fail(ctx, PQ_ERR_INVALID_ARG, "missing chars buffer");
    uint8_t* v = static_cast<uint8_t*>(outs[i].values);
    uint32_t* m = col.optional ? outs[i].validity : nullptr;
    uint8_t* c = static_cast<uint8_t*>(outs[i].chars);
    changed |= v != col.values || m != col.validity || c != col.chars || outs[i].chars_capacity != col.chars_cap;
    col.values = v;
    col.validity = m;
    col.chars = c;
    col.chars_cap = plan->sizing ? ~uint64_t(0) : outs[i].chars_capacity;
  }
  if (plan->graph && changed && (plan->str_cols.size() > 0)) {
    // the graph reads string totals through baked addresses: rebuild it
    cudaGraphExecDestroy(plan->graph);
    plan->graph = nullptr;
  }
  // the plan's uploads (legacy stream) come before anything of the scan.  A
  // captured stream may not wait on an event recorded outside the capture:
  // callers that capture wait for `ready` before the capture begins.
  if (plan->ready) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cap));
    if (cap == cudaStreamCaptureStatusNone) CK(cudaStreamWaitEvent(s, plan->ready, 0));
  }
  memcpy(plan->h_cols.p, plan->outcols.data(), sizeof(pqi::OutCol) * plan->outcols.size());
  if (!plan->outcols.empty())
    CK(cudaMemcpyAsync(plan->d_cols, plan->h_cols.p, sizeof(pqi::OutCol) * plan->outcols.size(),
                       cudaMemcpyHostToDevice, s));
  // resident dictionaries: decode once, then skip the dictionary stage
  bool with_dicts = true;
  if (plan->flags & PQ_SCAN_RESIDENT_DICT) {
    bool all = true;
    for (int32_t ch : plan->dict_chunks) all = all && plan->idx->dict_resident[ch];
    with_dicts = !all;
  }
  if (allow_graph && (plan->flags & PQ_SCAN_GRAPH) && !(plan->flags & PQ_SCAN_PLAIN)) {
    if (plan->graph && plan->dicts_in_graph != with_dicts) {
      cudaGraphExecDestroy(plan->graph);
      plan->graph = nullptr;
    }
    if (!plan->graph) {
      cudaStream_t cs = s;
      bool own = false;
      if (!cs) {
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        own = true;
      }
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      enqueue_scan(plan, cs, with_dicts, branches, n_branches);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cs, &g);
      if (own) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "graph capture");
      e = cudaGraphInstantiate(&plan->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
      plan->dicts_in_graph = with_dicts;
    }
    CK(cudaGraphLaunch(plan->graph, s));
  } else {
    enqueue_scan(plan, s, with_dicts, branches, n_branches);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(plan->done, s));
  if (plan->flags & PQ_SCAN_RESIDENT_DICT)
    for (int32_t ch : plan->dict_chunks) plan->idx->dict_resident[ch] = 1;
  return PQ_OK;
}

}  // namespace pqe

extern "C" {

pq_status pq_scan_columns(pq_ctx* ctx, pq_plan* plan, const pq_column* outs, void* stream) {
  if (!ctx || !plan || (!outs && !plan->outcols.empty())) return fail(ctx, PQ_ERR_INVALID_ARG, "pq_scan_columns");
  CK(cudaSetDevice(ctx->device));
  const int nb = std::min<int>(std::max<int>(plan->tuning.branches, 1), pq_ctx::kBranches);
  return scan_enqueue(plan, outs, static_cast<cudaStream_t>(stream), ctx->branch, nb, true);
}

pq_status pq_scan_wait(pq_ctx* ctx, pq_plan* plan, void* stream, uint64_t* chars_bytes) {
  if (!ctx || !plan) return fail(ctx, PQ_ERR_INVALID_ARG, "pq_scan_wait");
  (void)stream;
  CK(cudaSetDevice(ctx->device));
  CK(cudaEventSynchronize(plan->done));
  pqi::DevStatus st;
  memcpy(&st, plan->h_out.p, sizeof st);
  if (chars_bytes) {
    size_t j = 0;
    for (size_t i = 0; i < plan->outcols.size(); ++i) {
      if (plan->outcols[i].ptype == pqi::T_BYTE_ARRAY) {
        int64_t v;
        memcpy(&v, plan->h_out.p + sizeof(pqi::DevStatus) + 8 * j, 8);
        chars_bytes[i] = static_cast<uint64_t>(v);
        ++j;
      } else {
        chars_bytes[i] = 0;
      }
    }
  }
  if (st.flags && (plan->flags & PQ_SCAN_RESIDENT_DICT))
    for (int32_t ch : plan->dict_chunks) plan->idx->dict_resident[ch] = 0;
  return status_from_device(ctx, st);
}

}  // extern "C"
