"""Plain FP64 CPU oracle of the local-f_NL shell round trip (test infrastructure).

This package is test infrastructure, not part of the product: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and reference legs
may import it.  It shares no code with the CUDA library and never imports it.

Parity status of each function is stated in ``oracle/fnl_oracle.py`` (the generator, its
adjoint and the output maps) and ``oracle/ksw_oracle.py`` (the cubic estimator) and ``oracle/quadrature_oracle.py`` (the optimal
radial quadrature) and ``oracle/healpix_oracle.py`` (the HEALPix ring grid).
"""
from .fnl_oracle import *  # noqa: F401,F403
from .ksw_oracle import *  # noqa: F401,F403
from .quadrature_oracle import *  # noqa: F401,F403
from .healpix_oracle import *  # noqa: F401,F403
