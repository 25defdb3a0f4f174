"""GB300-native local-f_NL a_lm generator (Elsner & Wandelt): C-ABI library + thin binding.

The compute path lives in ``libfnl.so`` (CUDA kernels for sm_103a, built in-tree by
``paper_0909_0009_gb300.build``); ``paper_0909_0009_gb300.fnl`` is the ctypes binding.
"""
from .fnl import (EXPORTS, FNL_BF16X2, FNL_BF16X3, FNL_FP32, FNL_FP64, Cov, FnlError, Shells,  # noqa: F401
                  cholesky_filters, covariance, gauss_legendre, load_library)
