"""FEWHA hot path on B300: CUDA kernels behind a C-ABI library (libfewha.so).

The Python layer only marshals arguments; every step of the reconstruction
runs in the library's kernels.  Import :mod:`paper_2009_00946_b300.fewha` for
the binding (it loads the shared library on first use).
"""
