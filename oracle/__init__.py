"""FP64 CPU oracle of the implicit FE step: TEST INFRASTRUCTURE ONLY.

Imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` and by nothing else.  It shares no code with the CUDA library.
"""
from .fe_oracle import *  # noqa: F401,F403
from . import fe_oracle  # noqa: F401
