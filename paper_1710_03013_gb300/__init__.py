"""GB300 (sm_103a) approximate mini-batch kernel k-means.

The library is the C-ABI shared object ``libkkm.so`` (declared in
``include/kkm.h``); ``kkm`` is its Python binding.
"""

from . import kkm  # noqa: F401
from .kkm import (  # noqa: F401
    kkm_assign,
    kkm_cost,
    kkm_debug_kmeanspp,
    kkm_debug_step,
    kkm_fit,
    kkm_kernel_matrix,
    kkm_median_bandwidth,
)
