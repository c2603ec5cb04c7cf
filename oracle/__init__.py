"""FP64 CPU oracle for the priorconditioned lagged-diffusivity solver (arXiv 1308.6634).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use this package; the product path (``paper_1308_6634_gb300``)
never imports it.  The arithmetic lives in ``plsqr_oracle.c`` (plain C, double
precision, single threaded); ``oracle.py`` is a ctypes binding taking numpy arrays.

Parity pins (tests/test_oracle_*.py) tie every function here to something other than
itself: closed forms of (1.3)-(1.5), finite differences, dense matrices assembled from
the definitions, scipy's LSQR / CG on the transformed problem (1.10), textbook special
cases (Tikhonov, A = I, P = I), and analytic Radon transforms.
"""
from .oracle import *  # noqa: F401,F403
