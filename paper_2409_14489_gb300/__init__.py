"""GB300-native CB-ESSFM digital backpropagation.

The compute path is the CUDA library ``libcbessfm.so`` (C-ABI declared in ``include/cbessfm.h``)
built for sm_103a from ``csrc/``.  ``paper_2409_14489_gb300.cbessfm`` is the thin Python binding
(ctypes; PyTorch only for device memory and streams).  Importing the binding loads the library
and raises if it is missing: there is no CPU fallback.

Submodules that do not touch the GPU (``cost``, ``build``) import without the library.
"""

__all__ = ["cbessfm", "cost", "build"]
