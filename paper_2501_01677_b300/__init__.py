"""B300-native masked differentiable Gaussian-splat rasterisation for PG-SAG
(arXiv 2501.01677): C-ABI library libpgsag.so (include/pgsag.h) plus a thin
Python binding.  Importing this package does not load the CUDA library; the
first use of `raster` or `_lib.load()` does, and fails if it is missing."""
__all__ = ["raster", "build"]
