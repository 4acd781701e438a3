"""FP64 CPU oracle of the generalized FDTD scheme -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and never imports it.

* ``core``: the time-stepping scheme in plain C (FP64), driven through ctypes.
* ``vonneumann``: amplification matrices and their eigenvalues (Sec. 5, App. A).
* ``exact``: closed-form and transfer-matrix scattering results (App. B).
"""
from . import core, exact, vonneumann  # noqa: F401
from .core import Instance, run_many  # noqa: F401
