"""GB300-native (sm_103a) Chebyshev-filtered subspace iteration (ChASE).

The compute path lives in the CUDA library ``libchase.so`` behind the C ABI
declared in ``include/chase.h``; ``paper_1805_10121_gb300.chase`` is the thin
ctypes binding to it.  ``synth`` builds seeded synthetic inputs.
"""

__all__ = ["chase", "synth"]
