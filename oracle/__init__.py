"""Oracle for the NEGF selected-inversion path: plain, slow, complex128 CPU code.

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA library never uses it.
"""
from .rgf import *  # noqa: F401,F403
