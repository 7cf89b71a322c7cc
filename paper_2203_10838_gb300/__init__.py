"""GB300 (sm_103a) implementation of randomized sparse Kaczmarz with averaging
(RSKA; Tondji & Lorenz, arXiv 2203.10838).

The compute path is librska.so (CUDA kernels behind the C ABI declared in
include/rska.h); ``paper_2203_10838_gb300.rska`` is its Python binding.  Build
the library with ``paper_2203_10838_gb300.build.build()``.  Importing this
package does not load the library; using the binding does, and raises if it
is missing.
"""

__all__ = ["rska", "build"]
