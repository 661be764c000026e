/*
 * pq.h — C ABI of the GB300 Parquet column-chunk scan engine.
 *
 * The engine implements the GPU scan of Parquet files that the paper
 * "Do GPUs Really Need New Tabular File Formats?" studies: files (already in
 * GPU memory) go in, typed device columns plus validity bitmaps come out.
 * Section 2 of the paper defines the object being scanned: a file holds row
 * groups, a row group holds one column chunk per column, a chunk is split
 * into pages; pages use V1 or V2 encodings and are compressed with the
 * chunk's codec.  Section 3 ("Increase Page Count", Insight 1) is why the
 * engine decodes at a granularity finer than a page, and its effective
 * bandwidth metric (logical decoded bytes / scan time) is what the engine
 * is measured with.
 *
 * Supported subset: flat schemas (REQUIRED or OPTIONAL leaf columns, no
 * repetition), physical types INT32, INT64, DOUBLE and BYTE_ARRAY, data
 * pages V1 and V2, encodings PLAIN, PLAIN_DICTIONARY / RLE_DICTIONARY (with
 * an RLE/bit-packed hybrid index stream), DELTA_BINARY_PACKED, and the other
 * V2 encodings of the paper's Section 3 (Insight 3): BYTE_STREAM_SPLIT
 * (fixed-width columns), DELTA_LENGTH_BYTE_ARRAY and DELTA_BYTE_ARRAY
 * (BYTE_ARRAY columns; DELTA blocks of at most 2048 values), definition
 * levels with the RLE/bit-packed hybrid, codecs UNCOMPRESSED, SNAPPY and ZSTD
 * (the codecs the paper's Section 2 names; Zstandard frames without a
 * dictionary, every block type).
 * Anything else is rejected with PQ_ERR_UNSUPPORTED, never mis-decoded.
 *
 * Conventions for every call:
 *  - every call returns a pq_status; nothing aborts and no device kernel
 *    traps; pq_last_error() gives a one-line reason for the last failure on
 *    a context;
 *  - "device pointer" means memory of the context's CUDA device; "host
 *    pointer" means ordinary or pinned host memory;
 *  - a `stream` argument is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream);
 *  - sizes are in bytes unless a name says rows or values;
 *  - a context is not thread safe: one host thread at a time per context.
 */
#ifndef PQ_H_
#define PQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pq_status {
  PQ_OK = 0,
  PQ_ERR_INVALID_ARG = 1,  /* a NULL handle, a bad column id, a range past the data */
  PQ_ERR_CORRUPT = 2,      /* the file bytes violate the format */
  PQ_ERR_UNSUPPORTED = 3,  /* valid Parquet outside the supported subset */
  PQ_ERR_OOM = 4,          /* device or host allocation failed */
  PQ_ERR_BUDGET = 5,       /* a serving request needs more device memory than the budget */
  PQ_ERR_TIMEOUT = 6,      /* a bounded wait ran out (serving, or a device-side wait) */
  PQ_ERR_CUDA = 7,         /* a CUDA runtime call failed */
  PQ_ERR_CAPACITY = 8      /* a caller buffer is smaller than the plan requires */
} pq_status;

/* Parquet physical types (values as in the format's Type enum). */
typedef enum pq_type {
  PQ_TYPE_BOOLEAN = 0, PQ_TYPE_INT32 = 1, PQ_TYPE_INT64 = 2, PQ_TYPE_INT96 = 3,
  PQ_TYPE_FLOAT = 4, PQ_TYPE_DOUBLE = 5, PQ_TYPE_BYTE_ARRAY = 6,
  PQ_TYPE_FIXED_LEN_BYTE_ARRAY = 7
} pq_type;

typedef struct pq_ctx pq_ctx;
typedef struct pq_index pq_index;
typedef struct pq_plan pq_plan;
typedef struct pq_server pq_server;

/* ------------------------------------------------------------------ context */

/* Creates a context bound to CUDA device `device`.  The context owns a
 * device memory pool for index, plan and scratch buffers (freed by
 * pq_ctx_destroy).  Errors: PQ_ERR_CUDA when the device cannot be used. */
pq_status pq_ctx_create(int device, pq_ctx** out);
void pq_ctx_destroy(pq_ctx* ctx);
/* Last error message of the context ("" if none); valid until the next call. */
const char* pq_last_error(const pq_ctx* ctx);
const char* pq_status_string(pq_status s);
/* Library version string. */
const char* pq_version(void);

/* ------------------------------------------------------------------ files */

/* One Parquet file staged in device memory: `data` is a device pointer to
 * the whole file (magic, chunks, footer), `size` its length in bytes.  The
 * caller owns the buffer; it must stay valid and unchanged while any index,
 * plan or scan built from it is alive. */
typedef struct pq_file {
  const void* data;
  uint64_t size;
} pq_file;

/* ------------------------------------------------------------------ index */

typedef struct pq_index_info {
  int32_t n_files;
  int32_t n_columns;         /* leaf columns (identical schema across files) */
  int32_t n_row_groups;      /* over all files */
  int32_t n_chunks;          /* n_row_groups * n_columns */
  int64_t n_pages;           /* all pages incl. dictionary pages */
  int64_t n_data_pages;
  int64_t num_rows;          /* over all files, in file order */
  uint64_t stored_bytes;     /* sum of chunk bytes as stored (headers + pages) */
  uint64_t uncompressed_bytes; /* sum of page bodies after decompression + headers */
  int32_t used_offset_index; /* 1 when pages were located through OffsetIndex */
  int32_t reserved;
} pq_index_info;

typedef struct pq_column_info {
  char name[64];
  int32_t type;              /* pq_type */
  int32_t optional;          /* 1 = OPTIONAL (definition levels, max level 1) */
  int32_t type_length;       /* bytes per value for fixed-width types, else 0 */
  int32_t reserved;
} pq_column_info;

/* One row of the page table (host copy), for inspection and tests. */
typedef struct pq_page_info {
  int64_t header_offset;     /* in its file */
  int32_t file;
  int32_t chunk;             /* global chunk id: file-major, row group, column */
  int32_t page_type;         /* 0 DATA_PAGE, 2 DICTIONARY_PAGE, 3 DATA_PAGE_V2 */
  int32_t encoding;          /* Parquet Encoding enum value */
  int32_t header_len;
  int32_t uncompressed_size;
  int32_t compressed_size;
  int32_t num_values;        /* rows of a data page (flat schema), entries of a dictionary */
  int32_t num_nulls;         /* V2 header value, -1 for V1 / dictionary pages */
  int32_t def_len;           /* V2 definition-level bytes, 0 otherwise */
  int64_t first_row;         /* first row of the page within its chunk */
} pq_page_info;

/* Builds the page index of `n_files` files staged in device memory.
 *
 * Steps (paper Section 2 hierarchy; Section 3, "Increase Page Count"):
 *  1. host: reads each footer (a small device-to-host copy of the file tail)
 *     and parses FileMetaData (Thrift compact): schema, row groups, chunk
 *     offsets, codecs, types, sizes;
 *  2. device: walks the page headers of every chunk (one thread per chunk,
 *     or one thread per page when the file carries an OffsetIndex) and
 *     builds the device page table.
 * All files must share the leaf schema (names, types, repetition).
 * The index is owned by the library; free it with pq_free_index.  It keeps
 * pointers into the caller's file buffers.  `stream` orders the device work;
 * the call returns after it completed (the host needs the page counts).
 * Errors: PQ_ERR_CORRUPT (bad magic, footer, header, chunk bounds),
 * PQ_ERR_UNSUPPORTED (nested or repeated columns, other codecs/types),
 * PQ_ERR_INVALID_ARG, PQ_ERR_OOM, PQ_ERR_CUDA. */
pq_status pq_index_chunks(pq_ctx* ctx, const pq_file* files, int n_files, void* stream,
                          pq_index** out);
pq_status pq_index_get_info(const pq_index* idx, pq_index_info* out);
pq_status pq_index_get_column(const pq_index* idx, int column, pq_column_info* out);
/* Copies up to `cap` page-table rows (chunk order, pages in file order) to
 * host memory `out`; `*n_out` receives the number of rows available. */
pq_status pq_index_copy_pages(const pq_index* idx, pq_page_info* out, int64_t cap, int64_t* n_out);
void pq_free_index(pq_index* idx);

/* ------------------------------------------------------------------ plan */

/* Scan modes (pq_request.flags). */
#define PQ_SCAN_BATCHED 0u        /* page-walk + persistent expansion kernels (default) */
#define PQ_SCAN_PLAIN 1u          /* baseline: one page per thread block, one launch per
                                     chunk and stage (the grid = pages policy the paper
                                     describes for the reader it measures, Section 3) */
#define PQ_SCAN_GRAPH 2u          /* capture the batched scan into a CUDA graph on first
                                     use; later scans of the same plan replay it */
#define PQ_SCAN_RESIDENT_DICT 4u  /* decode dictionaries once and keep them in the index */
#define PQ_SCAN_TIMING 8u         /* record CUDA events between the scan's stages (see
                                     pq_plan_stage_ms); not combined with PQ_SCAN_GRAPH */

/* A scan request: which columns, which rows.  Rows are numbered over the
 * concatenation of all indexed files in order; the selected range must lie
 * inside [0, num_rows). */
typedef struct pq_request {
  const int32_t* columns;    /* host array of column ids; NULL = all columns */
  int32_t n_columns;         /* entries in `columns` (ignored when NULL) */
  uint32_t flags;            /* PQ_SCAN_* bits */
  int64_t row_begin;
  int64_t row_count;         /* < 0: up to the last row */
} pq_request;

/* Output sizes for one requested column, in request order. */
typedef struct pq_out_size {
  int64_t n_rows;
  int32_t type;              /* pq_type */
  int32_t optional;
  uint64_t values_bytes;     /* fixed width: n_rows * width; BYTE_ARRAY: (n_rows + 1) * 8
                                (int64 offsets) */
  uint64_t validity_bytes;   /* OPTIONAL: ceil(n_rows / 32) * 4, else 0 */
  uint64_t chars_bytes;      /* BYTE_ARRAY: chars capacity the scan needs (exact for whole
                                chunks, an upper bound for partial ones; exact when some
                                chunk carries no SizeStatistics and a sizing scan counted
                                them), else 0 */
} pq_out_size;

typedef struct pq_plan_info {
  int32_t n_columns;
  int32_t n_pages;           /* data pages the scan touches */
  int32_t n_dict_pages;
  int32_t n_items;           /* decode work items */
  uint64_t read_bytes;       /* stored bytes of the touched chunks' pages (headers incl.) */
  uint64_t decoded_bytes;    /* values + validity + offsets + chars the scan writes */
  uint64_t scratch_bytes;    /* device scratch the plan holds */
  int32_t launches_per_scan; /* kernels one pq_scan_columns call launches */
  int32_t reserved;
} pq_plan_info;

/* Plans a scan of `req` over `idx`: selects the pages overlapping the row
 * range, sizes the outputs, splits the pages into decode work items and
 * reserves scratch (decompression buffers, per-item checkpoints).  When
 * `sizes` is not NULL it receives one pq_out_size per requested column.
 * String chars are sized from each chunk's SizeStatistics
 * (unencoded_byte_array_data_bytes).  When a requested BYTE_ARRAY chunk
 * carries none (older writers), planning runs one sizing scan on the device
 * -- every kernel of the scan but the chars copy, into temporary outputs,
 * on a private stream, waited for -- and reports the exact chars bytes of
 * the requested rows.
 * The plan is owned by the library (pq_free_plan); it must not outlive the
 * index.  Errors: PQ_ERR_INVALID_ARG (column id, row range),
 * PQ_ERR_UNSUPPORTED (a DELTA_BYTE_ARRAY chunk without size statistics),
 * PQ_ERR_OOM, and the device errors of the sizing scan (PQ_ERR_CORRUPT ...). */
pq_status pq_plan_scan(pq_ctx* ctx, pq_index* idx, const pq_request* req, pq_plan** out,
                       pq_out_size* sizes);
pq_status pq_plan_get_info(const pq_plan* plan, pq_plan_info* out);
void pq_free_plan(pq_plan* plan);

/* Stages of a scan, in order, for pq_plan_stage_ms. */
#define PQ_STAGE_PREPARE 0     /* reset of bitmaps, counters, error word */
#define PQ_STAGE_SNAPPY 1      /* page decompression (K1), then the rewrite of
                                  BYTE_STREAM_SPLIT / DELTA_(LENGTH_)BYTE_ARRAY
                                  pages into PLAIN bodies */
#define PQ_STAGE_DICT 2        /* dictionary decode (K6) */
#define PQ_STAGE_WALK 3        /* page walk: levels, stream checkpoints */
#define PQ_STAGE_EXPAND 4      /* value expansion of the work items */
#define PQ_STAGE_STRINGS 5     /* string offsets and chars */
#define PQ_N_STAGES 6

/* Device milliseconds of each stage of the last scan of a plan created with
 * PQ_SCAN_TIMING (CUDA events on the scan's stream; call after
 * pq_scan_wait).  `ms` receives PQ_N_STAGES values (0 for skipped stages). */
pq_status pq_plan_stage_ms(const pq_plan* plan, float* ms);

/* ------------------------------------------------------------------ scan */

/* Caller-allocated output buffers of one column (device pointers).
 *  values:   fixed width: n_rows values, little-endian, the file's physical
 *            type (DOUBLE bitwise); null slots are written as 0.
 *            BYTE_ARRAY: n_rows + 1 int64 offsets into `chars`, starting at 0;
 *            a null row has length 0.
 *  validity: OPTIONAL columns only (NULL for REQUIRED): ceil(n_rows/32)
 *            uint32 words, bit i of the bitmap (word i/32, bit i%32) is 1 when
 *            row i is valid (LSB-first).  Bits past n_rows are 0.
 *  chars:    BYTE_ARRAY only: at least pq_out_size.chars_bytes bytes. */
typedef struct pq_column {
  void* values;
  uint32_t* validity;
  void* chars;
  uint64_t chars_capacity;
} pq_column;

/* Enqueues the scan on `stream` (asynchronous).  `outs` holds one entry per
 * requested column, in request order.  The device kernels never write
 * outside the caller's buffers; a format violation found on the device is
 * recorded in the plan's device error word (read by pq_scan_wait).
 * The plan may be scanned again (into the same or other buffers) after the
 * previous scan of it completed.  Errors found on the host before any launch:
 * PQ_ERR_INVALID_ARG, PQ_ERR_CAPACITY, PQ_ERR_CUDA. */
pq_status pq_scan_columns(pq_ctx* ctx, pq_plan* plan, const pq_column* outs, void* stream);

/* Waits for the last scan of `plan` enqueued on `stream` and reports its
 * device status: PQ_OK, PQ_ERR_CORRUPT or PQ_ERR_UNSUPPORTED (with the first
 * failing page in pq_last_error), PQ_ERR_TIMEOUT (a bounded device wait ran
 * out).  When `chars_bytes` is not NULL it receives, per requested column,
 * the chars bytes written (0 for fixed-width columns). */
pq_status pq_scan_wait(pq_ctx* ctx, pq_plan* plan, void* stream, uint64_t* chars_bytes);

/* End-to-end scan from HOST memory: `host_files` point to host memory
 * (pinned for full speed), `host_outs` are host buffers laid out exactly as
 * pq_column describes.  The files are copied to the device, indexed,
 * planned and scanned, and the columns copied back; the call is
 * synchronous.  When `host_outs` is NULL only `sizes` is filled (one entry
 * per requested column), so that the caller can allocate the outputs.
 * `req` as for pq_plan_scan.  Errors as for index/plan/scan.
 * Row groups go through the overlapped reading of the paper's Section 4 (a
 * pipeline of device slots: copy-in, decode and copy-out of different row
 * groups at once, page tables walked on the host) when the request spans
 * several row groups whose first output rows are multiples of 32 and the
 * first row group has no compressed page of 512 KiB or more; otherwise the
 * whole file is copied in, scanned and copied out in turn.  The environment
 * variable PQ_HOST_NO_PIPELINE=1 forces the latter. */
pq_status pq_scan_host(pq_ctx* ctx, const pq_file* host_files, int n_files, const pq_request* req,
                       const pq_column* host_outs, pq_out_size* sizes);

/* ------------------------------------------------------------------ serving */

/* Continuous-batching scan server over a fixed set of indexed files.
 * Requests (column sets + row ranges, rows wrapping cyclically over the
 * indexed rows) are admitted while their planned device bytes fit under
 * `budget_bytes` and one of `slots` CUDA streams is free; admitted requests
 * run concurrently on their streams, and requests that arrive meanwhile are
 * admitted as slots and memory free up.  Page indexes stay resident, and so
 * do decoded dictionaries.  Result buffers are owned by the server until
 * pq_serve_release. */
typedef struct pq_serve_config {
  uint64_t budget_bytes;     /* device bytes for request outputs + scratch */
  int32_t slots;             /* concurrent requests on the device (CUDA streams) */
  int32_t timeout_ms;        /* a queued request older than this fails with PQ_ERR_TIMEOUT
                                (0 = no timeout) */
} pq_serve_config;

typedef struct pq_serve_request {
  const int32_t* columns;    /* host array of column ids (copied at submit) */
  int32_t n_columns;
  int32_t reserved;
  int64_t row_begin;         /* taken modulo the indexed row count */
  int64_t row_count;         /* may exceed the indexed rows: the range wraps */
} pq_serve_request;

typedef struct pq_serve_result {
  pq_status status;
  int32_t n_columns;
  const pq_column* columns;  /* device buffers, server-owned, valid until release */
  const pq_out_size* sizes;
  double queue_ms;           /* submit -> admitted */
  double latency_ms;         /* submit -> completion observed by the server */
  uint64_t decoded_bytes;
  double admit_ms;           /* admission (enqueued on the device), ms since the server was created */
  double done_ms;            /* completion observed, ms since the server was created */
} pq_serve_result;

/* Creates a server over the files of `idx` (the index must outlive it). */
pq_status pq_serve_create(pq_ctx* ctx, pq_index* idx, const pq_serve_config* cfg,
                          pq_server** out);
/* Submits a request; returns at once with a ticket.  Errors:
 * PQ_ERR_INVALID_ARG (bad column), PQ_ERR_BUDGET (the request alone exceeds
 * the budget — it is rejected, not queued). */
pq_status pq_serve_submit(pq_server* srv, const pq_serve_request* req, uint64_t* ticket);
/* Polls a ticket: *done = 1 when finished (then `out` is filled), else 0. */
pq_status pq_serve_poll(pq_server* srv, uint64_t ticket, pq_serve_result* out, int* done);
/* Frees the result buffers of a finished ticket. */
pq_status pq_serve_release(pq_server* srv, uint64_t ticket);
/* Stops the scheduler thread, waits for in-flight work, frees everything. */
void pq_serve_destroy(pq_server* srv);

/* ------------------------------------------------------------------ writer */

/* Column input of the writer (host memory). */
typedef struct pq_write_column {
  const char* name;
  int32_t type;              /* PQ_TYPE_INT32 / INT64 / DOUBLE / BYTE_ARRAY */
  int32_t encoding;          /* Parquet Encoding: 0 PLAIN, 8 RLE_DICTIONARY,
                                5 DELTA_BINARY_PACKED (INT32/INT64), 9 BYTE_STREAM_SPLIT
                                (fixed width), 6 DELTA_LENGTH_BYTE_ARRAY and 7
                                DELTA_BYTE_ARRAY (BYTE_ARRAY); -1: per chunk, every valid
                                encoding of the type is tried and the one with the smallest
                                uncompressed chunk is kept, ties to the earlier of
                                0, 8, 5, 9 (integers), 0, 8, 9 (DOUBLE), 0, 8, 6, 7
                                (BYTE_ARRAY) (paper Section 3, "Encoding Flexibility") */
  int32_t codec;             /* 0 UNCOMPRESSED, 1 SNAPPY, 6 ZSTD (frames of LZ77 sequences
                                under FSE tables fitted per block, Huffman or raw
                                literals; the scan itself reads only UNCOMPRESSED and
                                SNAPPY chunks) */
  int32_t page_version;      /* 1 DATA_PAGE, 2 DATA_PAGE_V2 */
  double compress_threshold; /* < 0: keep the codec's output; else keep it only when the
                                chunk shrinks by more than this fraction (paper Section 3,
                                "No Unnecessary Compression": 0.10) */
  const void* values;        /* fixed width: n_rows values (null slots ignored);
                                BYTE_ARRAY: int64 offsets[n_rows + 1] */
  const uint8_t* chars;      /* BYTE_ARRAY chars */
  const uint8_t* valid;      /* NULL = REQUIRED; else one byte per row, nonzero = valid */
} pq_write_column;

/* Writes a flat table as a Parquet file into host memory — the offline
 * rewriter the paper's Sections 3 and 5 use to choose page size, row-group
 * size, encoding per chunk and selective compression.  Layout rules: row
 * group k holds rows [k*rg_rows, (k+1)*rg_rows); a page holds
 * max(8, floor(page_bytes*8/b) rounded down to a multiple of 8) rows, b
 * being the bits per row (8*width for PLAIN, the index bit width for
 * dictionary indices, +1 for a definition level when OPTIONAL); a REQUIRED
 * DELTA_BINARY_PACKED page holds 1 + 128k values, the most whole 128-value
 * blocks that fit page_bytes; BYTE_ARRAY pages that are not dictionary
 * encoded take rows while their PLAIN encoding fits; BYTE_STREAM_SPLIT pages
 * as PLAIN; dictionary entries in order of first appearance; hybrid runs: a
 * repeated run for >= 8 equal values, else bit-packed runs of <= 63 groups;
 * an OffsetIndex per chunk when `offset_index` is nonzero.
 * `*out` is allocated with malloc (free with pq_write_free); `n_threads`
 * threads encode chunks in parallel (<= 0: hardware threads).  Host code
 * only: needs no GPU.  Errors: PQ_ERR_INVALID_ARG (NULL pointers, sizes,
 * an encoding not valid for the column's type), PQ_ERR_UNSUPPORTED (other
 * types, encodings or codecs), PQ_ERR_OOM. */
pq_status pq_write_table(const pq_write_column* cols, int n_cols, int64_t n_rows, int64_t rg_rows,
                         int64_t page_bytes, int offset_index, int n_threads, uint8_t** out,
                         uint64_t* out_size);
void pq_write_free(uint8_t* buf);

/* ------------------------------------------------------------ tuning */

/* Knobs of the batched scan, per context; plans built afterwards use them
 * (the autotuner in paper_2602_17335_gb300/autotune.py picks them by
 * timing a sample of the workload).  They trade scheduling granularity
 * against per-item overhead: the paper's Section 3 (Insight 1) ties
 * parallelism to page count, this engine to work items of `item_rows`. */
typedef struct pq_tuning {
  int32_t item_rows;          /* rows per work item of pages without definition levels
                                 (REQUIRED columns); 256..65536, a multiple of 32
                                 (default 2048) */
  int32_t item_rows_opt;      /* rows per work item of pages with definition levels
                                 (OPTIONAL columns); 32..512, a multiple of 32
                                 (default 512) */
  int32_t expand_ctas_per_sm; /* cap on resident CTAs per SM of the expansion and copy
                                 kernels; 0 = the occupancy limit (default) */
  int32_t branches;           /* streams the columns of one scan are forked onto, 1..8
                                 (default 8) */
  int32_t walk_window;        /* staging depth of the page walks: bytes of each of the two
                                 shared-memory chain windows a walking block streams its
                                 page through; 0 = chosen by page count (default), else a
                                 power of two in 4096..65536 */
  int32_t snappy_block_kib;   /* compressed data pages of at least this many KiB are
                                 decompressed by a block of 8 warps each, smaller ones by one
                                 warp (dictionary pages always by a block); 1..1048576
                                 (default 256) */
  int32_t staged_expand;      /* 1: REQUIRED fixed-width dictionary columns take the staged
                                 expansion (index bytes bulk-copied to shared memory); 0: the
                                 general warp decode (default 1) */
  int32_t reserved;           /* 0 */
} pq_tuning;

/* Errors: PQ_ERR_INVALID_ARG (NULL, or a knob out of range). */
pq_status pq_ctx_set_tuning(pq_ctx* ctx, const pq_tuning* t);
pq_status pq_ctx_get_tuning(const pq_ctx* ctx, pq_tuning* t);

/* ------------------------------------------------------------ batched scan */

/* A batch groups several plans (typically one per schema of a heterogeneous
 * set of files: the batched workload's thousands of uneven chunks) into one
 * unit of work.  With PQ_SCAN_GRAPH in `flags` the scans of all plans are
 * captured once into a single CUDA graph and each pq_batch_launch is one
 * graph launch; otherwise each launch enqueues the kernels.  Plans run
 * concurrently, each on its own stream, their columns in sequence.
 * `outs[i]` is plan i's output array (as for pq_scan_columns), copied at
 * creation; plans and output buffers must outlive the batch.
 * Errors: PQ_ERR_INVALID_ARG, PQ_ERR_CAPACITY (as pq_scan_columns),
 * PQ_ERR_CUDA. */
typedef struct pq_batch pq_batch;
pq_status pq_batch_create(pq_ctx* ctx, int n_plans, pq_plan* const* plans, const pq_column* const* outs,
                          uint32_t flags, pq_batch** out);
/* Enqueues one run of the batch on `stream` (NULL = legacy default stream). */
pq_status pq_batch_launch(pq_batch* b, void* stream);
/* Waits for the last launch; returns the first device error of any plan
 * (per-plan string sizes: pq_scan_wait on the plan afterwards). */
pq_status pq_batch_wait(pq_batch* b);
void pq_batch_free(pq_batch* b);

/* ---- Allocation-free DELTA stream decode (no counterpart in the paper) ----
 *
 * Decodes one DELTA_BINARY_PACKED value stream of `n_values` INT32 or
 * INT64 values from device memory `d_stream` (`stream_len` bytes, followed
 * by at least 32 readable bytes, which are not used as data) into device
 * memory `d_values` (n_values * 4 or * 8 bytes, little-endian).  The stream
 * is the value part of a REQUIRED data page: header (block size, miniblocks
 * per block, value count, first value) then the blocks; its value count
 * must equal `n_values`.  Same kernels and results as the DELTA path of
 * pq_scan_columns.
 *
 * It allocates nothing: every piece of scratch sits in one fixed device
 * array of about 1.3 MB in the library, so callers that cannot allocate
 * device memory can use it — a host process whose device memory is all
 * reserved by another framework's allocator, or code that must not stall on
 * the device-wide synchronisation a cudaMalloc/cudaFree may cause.
 * Limits: stream_len <= 1 MiB (1048576) and n_values <= 4194305; larger
 * inputs are rejected with PQ_ERR_CAPACITY before anything runs.
 * The first call on a device does the set-up (looks up the array's device
 * address, which may load the library's device code); make that first call
 * before any stream capture.  Every run starts by clearing the status word
 * in the array; nothing else needs to start at zero.  The array is shared by
 * all calls on a device: calls that overlap in time (from several host
 * threads, or on several streams without ordering) race on it and give
 * undefined results.  Synchronous: enqueues on `stream` (NULL = the legacy
 * default stream), then waits for it to read the device status.
 * Errors: PQ_ERR_INVALID_ARG (NULL ctx, pointers, other types),
 * PQ_ERR_CAPACITY (over the limits), PQ_ERR_UNSUPPORTED (stream header
 * outside Parquet's DELTA rules), PQ_ERR_CORRUPT (value count mismatch,
 * malformed blocks), PQ_ERR_TIMEOUT, PQ_ERR_CUDA. */
pq_status pq_delta_decode_static(pq_ctx* ctx, const void* d_stream, uint64_t stream_len, pq_type type,
                                 int64_t n_values, void* d_values, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PQ_H_ */
