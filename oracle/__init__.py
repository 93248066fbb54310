"""CPU FP64 oracle for the ChASE hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (CPU baseline
and reference arm) may import this package.  The product library never
imports, links or executes anything here.
"""
from .chase_ref import *  # noqa: F401,F403
from .chase_ref import __all__  # noqa: F401
