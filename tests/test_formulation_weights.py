"""The binding's standard formulations (EFIE, MFIE, CFIE, Brakhage-Werner)
solve the scattering problem: assembled by the oracle with the binding's
weights, each gives the far field of the default rows, and for one
sound-soft disk the Mie series.  (GPU parity feeds the same weights to both
sides, so this CPU check is what ties the weights to the physics.)"""
import numpy as np
import pytest
from scipy import special

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

msd = pytest.importorskip("paper_1409_8186_gb300.msd")
OPS = ("I", "L", "M", "N", "D")


def far_with(cl, weights, betas, th):
    op, rhs, rep = weights
    ow = {c: {OPS[o]: op[c, o] for o in range(5) if op[c, o] != 0} for c in (0, 1)}
    rw = {c: {"U": rhs[c, 0], "dU": rhs[c, 1]} for c in (0, 1)}
    dens = O_.solve_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, ow, rw)
    return O_.farfield_formulation(cl.centres, cl.radii, cl.k, cl.N, dens, th, {"L": rep[0], "M": rep[1]})


@pytest.mark.parametrize("kind", ["efie", "mfie", "cfie", "bwie"])
def test_standard_formulations_solve_the_problem(kind):
    cl = W.small_mixed(seed=3, M=5, N=20, k=2.0)
    if kind == "mfie":
        cl.bc[:] = W.DIRICHLET  # MFIE is stated for sound-soft disks
    th = W.angles(24)
    betas = [0.3]
    rho, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas)
    ref = O_.farfield(cl.centres, cl.radii, cl.k, cl.N, rho, th)
    F = far_with(cl, msd.formulation(kind, k=cl.k), betas, th)
    assert np.abs(F - ref).max() <= 1e-9 * np.abs(ref).max()


def test_default_weights_are_the_default_rows():
    cl = W.small_mixed(seed=3, M=5, N=10, k=2.0)
    op, rhs, rep = msd.formulation("efie")
    ow = {c: {OPS[o]: op[c, o] for o in range(5) if op[c, o] != 0} for c in (0, 1)}
    A = O_.assemble_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, ow)
    assert np.abs(A - O_.assemble(cl.centres, cl.radii, cl.bc, cl.k, cl.N)).max() == 0


def test_eta_is_required_for_combined_formulations():
    with pytest.raises(ValueError):
        msd.formulation("cfie")
    with pytest.raises(ValueError):
        msd.formulation("nonsense")
