// pq_scan_host: the end-to-end call from host memory — files copied to the
// device, indexed, planned and scanned, columns copied back.
//
// When the requested rows span several row groups whose first rows fall on
// 32-row boundaries of the output (so that validity words do not straddle
// them), the row groups go through a pipeline of four device slots, the
// overlapped reading of the paper's Section 4: row group u+1 is copied in
// while row group u is indexed and decoded and the columns of earlier row
// groups are copied out.  Each slot scans on streams of its own, so the
// scans of consecutive row groups also overlap one another; the host waits
// for a row group only when its slot comes round again, three row groups
// later, so that the copy-out (the host link's slower direction) always has
// row groups queued while slow scans (Snappy pages) are still running.
// Footers are parsed and each row group's page table is walked straight
// from host memory (host_page_walk): the device indexes nothing and reads
// nothing back, so no row group waits for SMs held by an earlier one's
// scan or for a page-table readback queued behind the copy-out.  Files
// with compressed pages of 512 KiB or more take the whole-file path (their
// scans are latency-bound; see scan_pipelined).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "engine.h"
#include "host_pages.h"

using namespace pqe;

namespace {

struct Unit {
  int file, rg;
  int64_t byte0, byte1;  // staged file bytes
  int64_t row0, rows;    // global first row and rows of the row group
  int64_t lo, hi;        // requested rows inside it (row-group relative)
  int64_t out0;          // first output row
};

// A device slot and the row group in flight in it.
struct Slot {
  void* in = nullptr;
  std::vector<pq_column> outs;
  cudaEvent_t h2d = nullptr, scanned = nullptr, d2h = nullptr;
  cudaStream_t sc = nullptr;                        // the slot's scan stream
  cudaStream_t br[pq_ctx::kBranches] = {};          // and its column branches
  int64_t unit = -1;                                // row group in flight, -1 none
  pq_index* idx = nullptr;
  pq_plan* plan = nullptr;
  std::vector<pq_out_size> sz;                      // its planned output sizes
};

struct PipeGuard {
  pq_ctx* ctx;
  cudaStream_t sh = nullptr, sd = nullptr;
  std::vector<void*> blocks;
  static constexpr int kSlots = 4;
  Slot slot[kSlots];
  ~PipeGuard() {
    for (auto& sl : slot)
      if (sl.plan) pq_free_plan(sl.plan);  // waits for its scan
    for (cudaStream_t s : {sh, sd})
      if (s) cudaStreamSynchronize(s);
    for (auto& sl : slot) {
      if (sl.sc) cudaStreamSynchronize(sl.sc);
      if (sl.idx) index_release(sl.idx);
    }
    for (void* b : blocks) ctx->pool.free(b);
    for (auto& sl : slot) {
      for (cudaEvent_t e : {sl.h2d, sl.scanned, sl.d2h})
        if (e) cudaEventDestroy(e);
      if (sl.sc) cudaStreamDestroy(sl.sc);
      for (cudaStream_t b : sl.br)
        if (b) cudaStreamDestroy(b);
    }
    for (cudaStream_t s : {sh, sd})
      if (s) cudaStreamDestroy(s);
  }
  void* alloc(size_t n) {
    void* p = ctx->pool.alloc(std::max<size_t>(n, 16));
    if (p) blocks.push_back(p);
    return p;
  }
};

// Footer of a file in host memory.
pq_status host_footer(pq_ctx* ctx, const pq_file& f, int k, pqh::FileMeta* meta) {
  const uint8_t* b = static_cast<const uint8_t*>(f.data);
  if (!b || f.size < 12 || memcmp(b, "PAR1", 4) || memcmp(b + f.size - 4, "PAR1", 4))
    return fail(ctx, PQ_ERR_CORRUPT, "file " + std::to_string(k) + ": missing PAR1 magic");
  uint32_t flen;
  memcpy(&flen, b + f.size - 8, 4);
  if (static_cast<uint64_t>(flen) + 12 > f.size || flen < 8)
    return fail(ctx, PQ_ERR_CORRUPT, "file " + std::to_string(k) + ": bad footer length");
  std::string err;
  const int rc = pqh::parse_file_metadata(b + f.size - 8 - flen, flen, meta, &err);
  if (rc != pqh::META_OK)
    return fail(ctx, rc == pqh::META_UNSUPPORTED ? PQ_ERR_UNSUPPORTED : PQ_ERR_CORRUPT,
                "file " + std::to_string(k) + ": " + err);
  meta->footer_len = flen;
  return PQ_OK;
}

// The row-group pipeline; returns PQ_ERR_UNSUPPORTED (without side effects)
// when the request does not fit its conditions, so that the caller falls
// back to the whole-file path.
pq_status scan_pipelined(pq_ctx* ctx, const pq_file* host_files, int n_files, const pq_request* req,
                         const pq_column* host_outs) {
  std::vector<pqh::FileMeta> metas(n_files);
  for (int f = 0; f < n_files; ++f) {
    const pq_status st = host_footer(ctx, host_files[f], f, &metas[f]);
    if (st != PQ_OK) return st;
  }
  const int ncol_all = static_cast<int>(metas[0].columns.size());
  std::vector<int32_t> cols;
  if (req->columns) {
    for (int i = 0; i < req->n_columns; ++i) {
      if (req->columns[i] < 0 || req->columns[i] >= ncol_all) return PQ_ERR_UNSUPPORTED;
      cols.push_back(req->columns[i]);
    }
  } else {
    for (int i = 0; i < ncol_all; ++i) cols.push_back(i);
  }
  int64_t total_rows = 0;
  for (const auto& m : metas)
    for (const auto& g : m.rgs) total_rows += g.num_rows;
  const int64_t rb = req->row_begin, re = req->row_count < 0 ? total_rows : rb + req->row_count;
  if (rb < 0 || re > total_rows || rb >= re) return PQ_ERR_UNSUPPORTED;
  // units: requested row groups
  std::vector<Unit> units;
  int64_t row = 0;
  for (int f = 0; f < n_files; ++f) {
    if (metas[f].columns.size() != static_cast<size_t>(ncol_all)) return PQ_ERR_UNSUPPORTED;
    for (int g = 0; g < static_cast<int>(metas[f].rgs.size()); ++g) {
      const auto& rg = metas[f].rgs[g];
      const int64_t r0 = row, r1 = row + rg.num_rows;
      row = r1;
      if (r1 <= rb || r0 >= re) continue;
      Unit u{};
      u.file = f;
      u.rg = g;
      u.row0 = r0;
      u.rows = rg.num_rows;
      u.lo = std::max(rb, r0) - r0;
      u.hi = std::min(re, r1) - r0;
      u.out0 = std::max(rb, r0) - rb;
      int64_t b0 = INT64_MAX, b1 = 0;
      for (const auto& cm : rg.chunks) {
        b0 = std::min(b0, cm.start());
        b1 = std::max(b1, cm.start() + cm.total_compressed);
      }
      if (rg.chunks.empty() || b0 < 4) return PQ_ERR_UNSUPPORTED;
      b1 = std::min<int64_t>(b1 + 64, static_cast<int64_t>(host_files[f].size));
      u.byte0 = b0;
      u.byte1 = b1;
      if (u.out0 % 32) return PQ_ERR_UNSUPPORTED;  // validity words must not straddle units
      units.push_back(u);
    }
  }
  if (units.size() < 2) return PQ_ERR_UNSUPPORTED;
  {
    // Compressed pages of kLongPage or more: one row group's scan then takes
    // as long as its longest page's element chain (about 17 ms at 1 MiB
    // Snappy pages), which the pipeline would pay per row group and the
    // whole-file path pays once; the first row group's pages decide.
    constexpr int32_t kLongPage = 512 * 1024;
    const Unit& u = units[0];
    const uint8_t* hb = static_cast<const uint8_t*>(host_files[u.file].data);
    for (const auto& cm : metas[u.file].rgs[u.rg].chunks) {
      if (cm.codec == pqi::CODEC_NONE || cm.start() < 4 || cm.total_compressed < 0 ||
          static_cast<uint64_t>(cm.start()) + static_cast<uint64_t>(cm.total_compressed) > host_files[u.file].size)
        continue;
      std::vector<pqi::PageDev> pages;
      std::string err;
      if (!host_page_walk(hb + cm.start(), static_cast<uint64_t>(cm.total_compressed), cm.num_values, 0, &pages,
                          &err))
        continue;  // the per-row-group walk reports it
      for (const auto& pg : pages)
        if (pg.page_type != pqi::PAGE_DICT && pg.uncompressed >= kLongPage) return PQ_ERR_UNSUPPORTED;
    }
  }
  // capacities (the largest unit) per column
  int64_t max_bytes = 0, max_rows = 0;
  std::vector<int64_t> max_chars(cols.size(), 0);
  std::vector<int64_t> chars_base(cols.size(), 0);
  for (const auto& u : units) {
    max_bytes = std::max(max_bytes, u.byte1 - u.byte0);
    max_rows = std::max(max_rows, u.hi - u.lo);
    const auto& rg = metas[u.file].rgs[u.rg];
    for (size_t c = 0; c < cols.size(); ++c)
      if (metas[0].columns[cols[c]].type == PQ_TYPE_BYTE_ARRAY) {
        if (rg.chunks[cols[c]].byte_array_bytes < 0) return PQ_ERR_UNSUPPORTED;
        max_chars[c] = std::max(max_chars[c], rg.chunks[cols[c]].byte_array_bytes);
      }
  }
  PipeGuard g{ctx};
  const size_t ns = std::min<size_t>(PipeGuard::kSlots, units.size());  // slots in use
  const int nb = std::min<int>(std::max<int>(ctx->tuning.branches, 1), pq_ctx::kBranches);
  for (cudaStream_t* s : {&g.sh, &g.sd})
    if (cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "stream");
  for (size_t q = 0; q < ns; ++q) {
    Slot& sl = g.slot[q];
    if (cudaStreamCreateWithFlags(&sl.sc, cudaStreamNonBlocking) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "stream");
    for (int b = 0; b < nb; ++b)
      if (cudaStreamCreateWithFlags(&sl.br[b], cudaStreamNonBlocking) != cudaSuccess)
        return fail(ctx, PQ_ERR_CUDA, "stream");
    for (cudaEvent_t* e : {&sl.h2d, &sl.scanned, &sl.d2h})
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "event");
    sl.in = g.alloc(static_cast<size_t>(max_bytes) + 64);
    if (!sl.in) return fail(ctx, PQ_ERR_OOM, "staging buffer");
    sl.outs.assign(cols.size(), pq_column{});
    for (size_t c = 0; c < cols.size(); ++c) {
      const auto& cm = metas[0].columns[cols[c]];
      const bool ba = cm.type == PQ_TYPE_BYTE_ARRAY;
      const int w = ba ? 8 : pqi::type_width(cm.type);
      sl.outs[c].values = g.alloc(static_cast<size_t>(max_rows + 1) * w);
      if (cm.repetition == 1) sl.outs[c].validity = static_cast<uint32_t*>(g.alloc((max_rows + 31) / 32 * 4));
      if (ba) {
        sl.outs[c].chars = static_cast<uint8_t*>(g.alloc(static_cast<size_t>(max_chars[c]) + 16));
        sl.outs[c].chars_capacity = static_cast<uint64_t>(max_chars[c]) + 16;
      }
      if (!sl.outs[c].values || (cm.repetition == 1 && !sl.outs[c].validity) || (ba && !sl.outs[c].chars))
        return fail(ctx, PQ_ERR_OOM, "slot outputs");
    }
  }
  bool any_ba = false;
  for (size_t c = 0; c < cols.size(); ++c) any_ba |= metas[0].columns[cols[c]].type == PQ_TYPE_BYTE_ARRAY;
  auto copy_out = [&](void* host, const void* src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(host, src, bytes, cudaMemcpyDeviceToHost, g.sd) : cudaSuccess;
  };
  // the row group in flight in a slot: waits for its scan (status, chars
  // against the planned sizes, which the copy-out used) and its copy-out
  auto retire = [&](Slot& sl) -> pq_status {
    if (sl.unit < 0) return PQ_OK;
    std::vector<uint64_t> chars(cols.size());
    pq_status st = pq_scan_wait(ctx, sl.plan, sl.sc, chars.data());
    if (st != PQ_OK) return st;
    for (size_t c = 0; c < cols.size(); ++c)
      if (sl.sz[c].type == PQ_TYPE_BYTE_ARRAY && chars[c] != sl.sz[c].chars_bytes)
        return fail(ctx, PQ_ERR_CORRUPT, "row-group chars differ from the chunk's size statistics");
    if (cudaEventSynchronize(sl.d2h) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "slot reuse");
    pq_free_plan(sl.plan);
    sl.plan = nullptr;
    index_release(sl.idx);
    sl.idx = nullptr;
    sl.unit = -1;
    return PQ_OK;
  };
  // copy-in of unit k into its slot, once the slot's previous row group is done
  auto copy_in = [&](size_t k) -> pq_status {
    const Unit& u = units[k];
    Slot& sl = g.slot[k % ns];
    const pq_status st = retire(sl);
    if (st != PQ_OK) return st;
    const uint8_t* hb = static_cast<const uint8_t*>(host_files[u.file].data);
    const cudaError_t e = cudaMemcpyAsync(sl.in, hb + u.byte0, static_cast<size_t>(u.byte1 - u.byte0),
                                          cudaMemcpyHostToDevice, g.sh);
    if (e != cudaSuccess || cudaEventRecord(sl.h2d, g.sh) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "host-to-device copy");
    return PQ_OK;
  };
  pq_status st = copy_in(0);
  if (st != PQ_OK) return st;
  for (size_t k = 0; k < units.size(); ++k) {
    const Unit& u = units[k];
    Slot& sl = g.slot[k % ns];
    if (cudaStreamWaitEvent(sl.sc, sl.h2d, 0) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "event");
    // index of this row group: one file view whose chunk offsets land in the
    // slot, and the page table walked from the host's copy of the chunks
    const auto& rgm = metas[u.file].rgs[u.rg];
    const uint8_t* hb = static_cast<const uint8_t*>(host_files[u.file].data);
    std::vector<pqi::PageDev> pages;
    for (size_t c = 0; c < rgm.chunks.size(); ++c) {
      const auto& cm = rgm.chunks[c];
      if (cm.start() < 4 || cm.total_compressed < 0 ||
          static_cast<uint64_t>(cm.start()) + static_cast<uint64_t>(cm.total_compressed) > host_files[u.file].size)
        return fail(ctx, PQ_ERR_CORRUPT, "chunk byte range outside the file");
      std::string err;
      if (!host_page_walk(hb + cm.start(), static_cast<uint64_t>(cm.total_compressed), cm.num_values,
                          static_cast<uint32_t>(c), &pages, &err))
        return fail(ctx, PQ_ERR_CORRUPT, "row group " + std::to_string(u.rg) + ", column " + std::to_string(c) +
                                             ": " + err);
    }
    auto ix = std::make_unique<pq_index>();
    ix->ctx = ctx;
    pq_file view;
    view.data = static_cast<uint8_t*>(sl.in) - u.byte0;
    view.size = static_cast<uint64_t>(u.byte1);
    ix->files.push_back(view);
    pqh::FileMeta m;
    m.columns = metas[u.file].columns;
    m.rgs.push_back(rgm);
    m.num_rows = u.rows;
    m.footer_len = 0;
    ix->metas.push_back(std::move(m));
    st = index_build(ctx, std::move(ix), false, sl.sc, &sl.idx, &pages);
    if (st != PQ_OK) return st;
    pq_request lr{};
    lr.columns = cols.data();
    lr.n_columns = static_cast<int32_t>(cols.size());
    lr.flags = req->flags & ~(PQ_SCAN_GRAPH | PQ_SCAN_TIMING);
    lr.row_begin = u.lo;
    lr.row_count = u.hi - u.lo;
    sl.sz.assign(cols.size(), pq_out_size{});
    st = plan_scan_on(ctx, sl.idx, &lr, sl.sc, &sl.plan, sl.sz.data());
    if (st != PQ_OK) return st;
    for (size_t c = 0; c < cols.size(); ++c)
      if (sl.sz[c].chars_bytes > sl.outs[c].chars_capacity && sl.sz[c].type == PQ_TYPE_BYTE_ARRAY)
        return fail(ctx, PQ_ERR_CAPACITY, "row-group chars above the chunk's size statistics");
    st = scan_enqueue(sl.plan, sl.outs.data(), sl.sc, sl.br, nb, false);
    if (st != PQ_OK) return st;
    sl.unit = static_cast<int64_t>(k);
    const int64_t n = u.hi - u.lo;
    // chars per string column: the planned sizes are exact for whole row
    // groups; a partial one (the request's first or last) is waited for
    std::vector<uint64_t> chars(cols.size());
    for (size_t c = 0; c < cols.size(); ++c) chars[c] = sl.sz[c].type == PQ_TYPE_BYTE_ARRAY ? sl.sz[c].chars_bytes : 0;
    if (any_ba && (u.lo != 0 || u.hi != u.rows)) {
      st = pq_scan_wait(ctx, sl.plan, sl.sc, chars.data());
      if (st != PQ_OK) return st;
      for (size_t c = 0; c < cols.size(); ++c)
        if (sl.sz[c].type == PQ_TYPE_BYTE_ARRAY) sl.sz[c].chars_bytes = chars[c];
    }
    for (size_t c = 0; c < cols.size(); ++c)
      if (sl.sz[c].type == PQ_TYPE_BYTE_ARRAY)
        pqi::launch_add_offsets(static_cast<int64_t*>(sl.outs[c].values), n + 1, chars_base[c], sl.sc);
    if (cudaEventRecord(sl.scanned, sl.sc) != cudaSuccess || cudaStreamWaitEvent(g.sd, sl.scanned, 0) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "event");
    for (size_t c = 0; c < cols.size(); ++c) {
      const pq_out_size& z = sl.sz[c];
      uint8_t* hv = static_cast<uint8_t*>(host_outs[c].values);
      const bool ba = z.type == PQ_TYPE_BYTE_ARRAY;
      const int64_t w = ba ? 8 : pqi::type_width(z.type);
      cudaError_t e = copy_out(hv + u.out0 * w, sl.outs[c].values, static_cast<size_t>((n + (ba ? 1 : 0)) * w));
      if (e == cudaSuccess && z.optional)
        e = copy_out(reinterpret_cast<uint8_t*>(host_outs[c].validity) + u.out0 / 8, sl.outs[c].validity,
                     static_cast<size_t>((n + 31) / 32 * 4));
      if (e == cudaSuccess && ba && chars[c]) {
        if (static_cast<uint64_t>(chars_base[c]) + chars[c] > host_outs[c].chars_capacity)
          return fail(ctx, PQ_ERR_CAPACITY, "host chars buffer smaller than the scanned chars");
        e = copy_out(static_cast<uint8_t*>(host_outs[c].chars) + chars_base[c], sl.outs[c].chars, chars[c]);
      }
      if (e != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "device-to-host copy");
      chars_base[c] += static_cast<int64_t>(chars[c]);
    }
    if (cudaEventRecord(sl.d2h, g.sd) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "event");
    if (k + 1 < units.size() && (st = copy_in(k + 1)) != PQ_OK) return st;
  }
  // the row groups still in flight, in order
  for (size_t k = units.size() - ns; k < units.size(); ++k)
    if ((st = retire(g.slot[k % ns])) != PQ_OK) return st;
  if (cudaStreamSynchronize(g.sd) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "synchronize");
  return PQ_OK;
}

struct HostScanGuard {
  pq_ctx* ctx;
  cudaStream_t s = nullptr;
  std::vector<void*> blocks;
  pq_index* idx = nullptr;
  pq_plan* plan = nullptr;
  ~HostScanGuard() {
    if (plan) pq_free_plan(plan);
    if (idx) pq_free_index(idx);
    if (s) cudaStreamSynchronize(s);
    for (void* b : blocks) ctx->pool.free(b);
    if (s) cudaStreamDestroy(s);
  }
  void* alloc(size_t n) {
    void* p = ctx->pool.alloc(n);
    if (p) blocks.push_back(p);
    return p;
  }
};

}  // namespace

extern "C" pq_status pq_scan_host(pq_ctx* ctx, const pq_file* host_files, int n_files, const pq_request* req,
                                  const pq_column* host_outs, pq_out_size* sizes) {
  if (!ctx || !host_files || n_files <= 0 || !req) return fail(ctx, PQ_ERR_INVALID_ARG, "pq_scan_host");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "cudaSetDevice");
  if (host_outs && !getenv("PQ_HOST_NO_PIPELINE")) {
    const pq_status st = scan_pipelined(ctx, host_files, n_files, req, host_outs);
    if (st != PQ_ERR_UNSUPPORTED) return st;
  }
  HostScanGuard g{ctx};
  if (cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(ctx, PQ_ERR_CUDA, "stream");
  std::vector<pq_file> dev(n_files);
  for (int f = 0; f < n_files; ++f) {
    if (!host_files[f].data && host_files[f].size) return fail(ctx, PQ_ERR_INVALID_ARG, "null host file");
    void* d = g.alloc(host_files[f].size + 64);
    if (!d) return fail(ctx, PQ_ERR_OOM, "device file buffer");
    if (cudaMemcpyAsync(d, host_files[f].data, host_files[f].size, cudaMemcpyHostToDevice, g.s) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "host-to-device copy");
    dev[f].data = d;
    dev[f].size = host_files[f].size;
  }
  pq_status st = pq_index_chunks(ctx, dev.data(), n_files, g.s, &g.idx);
  if (st != PQ_OK) return st;
  const int ncols = req->columns ? req->n_columns : g.idx->n_columns;
  std::vector<pq_out_size> szs(static_cast<size_t>(std::max(ncols, 1)));
  st = pq_plan_scan(ctx, g.idx, req, &g.plan, szs.data());
  if (st != PQ_OK) return st;
  if (sizes) memcpy(sizes, szs.data(), sizeof(pq_out_size) * ncols);
  if (!host_outs) return PQ_OK;
  std::vector<pq_column> douts(ncols);
  for (int c = 0; c < ncols; ++c) {
    const pq_out_size& z = szs[c];
    douts[c].values = z.values_bytes ? g.alloc(z.values_bytes) : nullptr;
    douts[c].validity = z.validity_bytes ? static_cast<uint32_t*>(g.alloc(z.validity_bytes)) : nullptr;
    douts[c].chars = z.chars_bytes ? g.alloc(z.chars_bytes) : nullptr;
    douts[c].chars_capacity = z.chars_bytes;
    if ((z.values_bytes && !douts[c].values) || (z.validity_bytes && !douts[c].validity) ||
        (z.chars_bytes && !douts[c].chars))
      return fail(ctx, PQ_ERR_OOM, "device output buffers");
    if (host_outs[c].chars_capacity < z.chars_bytes && z.type == PQ_TYPE_BYTE_ARRAY)
      return fail(ctx, PQ_ERR_CAPACITY, "host chars buffer smaller than chars_bytes");
  }
  st = pq_scan_columns(ctx, g.plan, douts.data(), g.s);
  if (st != PQ_OK) return st;
  std::vector<uint64_t> chars(ncols);
  st = pq_scan_wait(ctx, g.plan, g.s, chars.data());
  if (st != PQ_OK) return st;
  for (int c = 0; c < ncols; ++c) {
    const pq_out_size& z = szs[c];
    if (z.values_bytes && cudaMemcpyAsync(host_outs[c].values, douts[c].values, z.values_bytes,
                                          cudaMemcpyDeviceToHost, g.s) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "device-to-host copy");
    if (z.validity_bytes && cudaMemcpyAsync(host_outs[c].validity, douts[c].validity, z.validity_bytes,
                                            cudaMemcpyDeviceToHost, g.s) != cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "device-to-host copy");
    if (chars[c] && cudaMemcpyAsync(host_outs[c].chars, douts[c].chars, chars[c], cudaMemcpyDeviceToHost, g.s) !=
                        cudaSuccess)
      return fail(ctx, PQ_ERR_CUDA, "device-to-host copy");
  }
  if (cudaStreamSynchronize(g.s) != cudaSuccess) return fail(ctx, PQ_ERR_CUDA, "synchronize");
  return PQ_OK;
}
