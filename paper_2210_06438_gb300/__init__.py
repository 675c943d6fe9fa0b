"""GB300-native aggregated hydro RHS (PPM + Kurganov-Tadmor) behind a C ABI.

The computation lives in ``csrc/`` (CUDA for sm_103a, compiled into
``_lib/libhydro.so``); ``binding`` marshals arguments to it.
"""
from .binding import *  # noqa: F401,F403
from .binding import (HydroError, Plan, Server, descriptors, load, now_ns, rhs,  # noqa: F401
                      rhs_per_subgrid, status)
