"""GB300 Parquet column-chunk scan engine.

The compute path is the CUDA library built from ``csrc/`` (sm_103a); this
package holds its ctypes binding (``native``), a small torch-based helper
for device buffers (``scan``) and the build script (``build``).  Importing
the package does not load the library; ``native.lib()`` does, and raises
when it has not been built.
"""
