"""FP64 CPU oracle for the beta-divergence MM updates (arXiv 2602.14683).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package; the product library never does.  The arithmetic
lives in ``ntf_oracle.c`` (plain loops, FP64); this module only marshals numpy arrays.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, hand-worked fixtures (``tests/golden/``), textbook beta-NMF updates (N = 2),
exact fixed points, brute-force majorizer checks and monotone descent.
"""
from .binding import *  # noqa: F401,F403
