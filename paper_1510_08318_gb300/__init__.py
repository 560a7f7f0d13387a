"""GB300-native MOFF imaging step (E-field Parallel Imaging Correlator, arXiv 1510.08318).

The compute path lives in a C-ABI shared library built from `csrc/`; `epic` is its
thin ctypes binding.  Importing this package does not load the library: call
`paper_1510_08318_gb300.epic.load()` (done on first use) or `build.build()`.
"""
