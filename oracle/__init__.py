"""CPU oracle for the Parquet column-chunk scan — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct Parquet writer plus an independent reader
for the subset the GPU scan engine supports: the file -> row group ->
column chunk -> page hierarchy with V1 and V2 data pages, PLAIN,
RLE_DICTIONARY (RLE/bit-packed hybrid indices), DELTA_BINARY_PACKED,
definition levels, and per-page Snappy compression (the paper's Section 2
names this hierarchy, the V1/V2 encodings and chunk-level compression; the
byte layouts are those of the public Parquet format, Thrift compact protocol
and Snappy block format definitions).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA engine.

Parity: every function here is pinned by tests that do not go through it
alone — encode/decode round trips against the seeded generator's arrays,
hand-worked byte vectors (``tests/golden/``), brute force over tiny inputs
and, where pyarrow exists, a third-party reader/writer cross-check.
"""
