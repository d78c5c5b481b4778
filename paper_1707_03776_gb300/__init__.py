"""GB300-native explicit finite-difference stencils (arXiv 1707.03776).

The compute path is the C-ABI library `libfdgb.so` (CUDA kernels for sm_103a);
`paper_1707_03776_gb300.fd` is its thin ctypes binding.  Importing this package
loads nothing: the library is opened on first use and the binding raises if it
is missing.  `paper_1707_03776_gb300.workloads` holds the seeded synthetic
input generators.
"""

__all__ = ["fd", "workloads"]
