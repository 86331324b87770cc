"""The named formulations (EFIE, MFIE, CFIE, Brakhage-Werner; section 3).

The oracle's statement of their weights (standard_formulation) is pinned
by the physics: assembled by the oracle, each formulation gives the far
field of the default rows.  The library forms the same weights itself
(msd_formulation_weights, a host function of libmsd that needs no GPU);
they must equal the oracle's exactly.  (GPU parity of the formulations feeds
the oracle's weights to the oracle and the formulation's name to the
library, so this check ties the two.)"""
import numpy as np
import pytest

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

OPS = ("I", "L", "M", "N", "D")
KINDS = ["efie", "mfie", "cfie", "bwie"]


@pytest.mark.parametrize("kind", KINDS)
def test_standard_formulations_solve_the_problem(kind):
    cl = W.small_mixed(seed=3, M=5, N=20, k=2.0)
    if kind == "mfie":
        cl.bc[:] = W.DIRICHLET  # MFIE is stated for sound-soft disks
    th = W.angles(24)
    betas = [0.3]
    rho, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas)
    ref = O_.farfield(cl.centres, cl.radii, cl.k, cl.N, rho, th)
    ow, rw, pw = O_.standard_formulation(kind, k=cl.k)
    dens = O_.solve_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, ow, rw)
    F = O_.farfield_formulation(cl.centres, cl.radii, cl.k, cl.N, dens, th, pw)
    assert np.abs(F - ref).max() <= 1e-9 * np.abs(ref).max()


def test_efie_weights_are_the_default_rows():
    cl = W.small_mixed(seed=3, M=5, N=10, k=2.0)
    ow, _, _ = O_.standard_formulation("efie")
    A = O_.assemble_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, ow)
    assert np.abs(A - O_.assemble(cl.centres, cl.radii, cl.bc, cl.k, cl.N)).max() == 0


@pytest.mark.parametrize("kind,alpha,eta", [("efie", 0.5, None), ("mfie", 0.5, None), ("cfie", 0.3, None),
                                            ("cfie", 0.7, 0.4 + 2.5j), ("bwie", 0.5, None),
                                            ("bwie", 0.5, -1.0 + 0.8j)])
def test_library_weights_equal_the_oracle_weights(kind, alpha, eta):
    msd = pytest.importorskip("paper_1409_8186_gb300.msd")
    k = 2.7
    op, rhs, rep = msd.msd_formulation_weights(kind, alpha, eta, k)
    ow, rw, pw = O_.standard_formulation(kind, alpha=alpha, eta=eta, k=k)
    for c in (0, 1):
        assert all(op[c, o] == ow[c].get(OPS[o], 0) for o in range(5)), (c, op[c], ow[c])
        assert rhs[c, 0] == rw[c].get("U", 0) and rhs[c, 1] == rw[c].get("dU", 0), (c, rhs[c], rw[c])
    assert rep[0] == pw["L"] and rep[1] == pw["M"]


def test_named_formulation_arguments_are_checked():
    msd = pytest.importorskip("paper_1409_8186_gb300.msd")
    for kind, alpha, eta, k in (("cfie", 1.5, None, 1.0),       # alpha outside [0, 1]
                                ("cfie", 0.5, 2.0, 1.0),        # real eta
                                ("bwie", 0.5, 0.0 + 0.0j, 1.0),
                                ("bwie", 0.5, None, 0.0)):      # eta = i k without k
        with pytest.raises(msd.MsdError) as e:
            msd.msd_formulation_weights(kind, alpha, eta, k)
        assert e.value.status == msd.MSD_ERR_ARG
    with pytest.raises(ValueError):
        msd.formulation("nonsense")
    with pytest.raises(ValueError):
        msd.formulation("cfie")
