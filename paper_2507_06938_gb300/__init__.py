"""GB300 (sm_103a) library for the BTA hot path of INLA on spatio-temporal
multivariate Gaussian processes (arXiv 2507.06938).

The numerical work lives in ``libbta.so`` (CUDA kernels behind the C ABI of
``include/bta.h``); ``bta`` is its ctypes binding.  Build with
``paper_2507_06938_gb300._build.build()``.
"""

from . import bta  # noqa: F401
from .bta import (  # noqa: F401
    BTA_FP64, BTA_MIXED, BTA_MIXED_HI, BTA_QC, BTA_QP, BtaContext, BtaError, BtaModel,
)
