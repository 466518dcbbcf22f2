"""Plain CPU oracle for the PSATD tight-focusing path (test infrastructure only).

This package is the independent, slow, obviously-correct reference that the CUDA
library is checked against.  It is written in numpy, in float64, from the paper
(arXiv:2010.00409) and shares no code, tables or helpers with the CUDA path.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path never
routes through it.
"""
from .psatd_oracle import *  # noqa: F401,F403
