"""FP64 CPU oracle for the sparsified thin-wire EFIE method of moments.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check in ``__graft_entry__`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with the CUDA library:
it restates the method from the paper (Sec. II-A and II-B) in plain NumPy, slowly and in float64,
so that the GPU path can be checked against it element by element.

Every function is pinned by the ``-m "not gpu"`` tests against something other than itself
(adaptive quadrature, closed forms, textbook dipole values, reciprocity, the optical theorem,
brute force).  Parity pins and the one unpinned reading are listed in the project's design notes.
"""
from .mom import *  # noqa: F401,F403
