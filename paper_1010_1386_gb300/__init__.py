"""Exact bivariate resultants Res_y(f, g) in Z[x] on one GB300 (sm_103a).

The compute path lives in the CUDA/C++ library ``librs.so`` (C ABI declared
in ``include/rs.h``); ``paper_1010_1386_gb300.rs`` is its thin ctypes
binding.  Import the binding explicitly; this package ``__init__`` loads
nothing so that the input generators can be used without the library.
"""
