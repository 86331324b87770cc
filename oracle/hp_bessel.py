"""High-precision Hankel values H^(1)_l(x) = J_l(x) + i Y_l(x) (mpmath, 40
digits).  TEST INFRASTRUCTURE ONLY: used to write the golden table that the
device Bessel recurrences are checked against."""
from __future__ import annotations


def hankel1_hp(l: int, x: float, dps: int = 40) -> complex:
    import mpmath as mp

    with mp.workdps(dps):
        return complex(mp.besselj(l, x) + 1j * mp.bessely(l, x))
