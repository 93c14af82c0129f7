"""GB300-native screened orbital-space VMC hot path (arXiv:1807.10633).

Submodules: ``systems`` (seeded synthetic inputs), ``build`` (nvcc build of the CUDA library),
``vmc`` (binding of the C ABI in include/vmc.h).  Importing the package loads nothing; the CUDA
library is loaded on first use by ``vmc.lib()`` and its absence is an error.
"""
