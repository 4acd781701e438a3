"""GB300-native generalized FDTD for moving media (arXiv 2304.06586).

The engine is the CUDA library ``libgfdtd.so`` behind the C ABI in
``include/gfdtd.h``; ``binding`` is its thin Python binding and ``workloads``
generates the seeded synthetic inputs shaped like the paper's examples.
"""
from . import binding  # noqa: F401
from .binding import (BF16, F16, F32, F64, FIELD_B, FIELD_D, FIELD_E, FIELD_ESTAR,  # noqa: F401
                      FIELD_H, LAYERS, LINEAR, MATTER, PERTURBATION, GfdtdError, Simulation,
                      stability, use_torch_allocator)
