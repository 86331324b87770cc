"""Writes tests/golden/hankel_hp.json: H^(1)_l(x) for l = 0..2N at the
arguments below, from the oracle's 40-digit mpmath evaluation.  The grid
spans the Miller branch (x <= 20), the asymptotic branch (x > 20), the
crossover, and orders up to 126 (N = 63)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
from oracle.hp_bessel import hankel1_hp  # noqa: E402

GRID = [(0.05, 8), (0.3, 12), (1.0, 20), (3.1, 30), (9.7, 40), (19.9, 44), (20.1, 44), (33.3, 63),
        (77.0, 63), (150.5, 63), (400.0, 63), (886.2, 63), (1500.0, 63)]

if __name__ == "__main__":
    out = []
    for x, N in GRID:
        vals = [hankel1_hp(l, x) for l in range(2 * N + 1)]
        out.append({"x": x, "N": N, "re": [v.real for v in vals], "im": [v.imag for v in vals]})
    with open(os.path.join(HERE, "hankel_hp.json"), "w") as f:
        json.dump({"source": "oracle.hp_bessel.hankel1_hp (mpmath, 40 digits)", "table": out}, f)
    print("wrote", len(out), "arguments")
