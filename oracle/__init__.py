"""CPU oracle (FP64, NumPy/SciPy) for the multiple-scattering hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import it; the product package never does.
"""
from .msd_oracle import *  # noqa: F401,F403
