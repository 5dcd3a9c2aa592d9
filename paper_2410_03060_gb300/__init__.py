"""GB300 (sm_103a) sparsified thin-wire method-of-moments solver for chaff-cloud RCS.

The compute path lives in the CUDA library ``libswm.so`` (sources in ``csrc/``, C ABI in
``include/swm.h``); ``swm`` is its thin ctypes binding.  Import ``paper_2410_03060_gb300.swm`` to
use it.
"""
__all__ = ["swm", "build"]
