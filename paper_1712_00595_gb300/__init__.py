"""GB300 engine for Random Walk with Restart on dynamic graphs (OSP / OSP-T).

The engine is a CUDA library with a C ABI (include/osp.h); ``native`` is its
ctypes binding and ``workloads`` draws seeded synthetic inputs.
"""
from .native import (OSP_EINVAL, OSP_ENOCONV, OSP_ENOTSUP, OSP_ESTATE, OSP_OK,  # noqa: F401
                     OSP_PREC_BF16_ACC64, OSP_PREC_FP32_ACC64, OSP_PREC_FP64, UPDATE_DTYPE,
                     Engine, OspError,
                     load_library)
