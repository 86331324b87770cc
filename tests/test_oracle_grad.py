"""Pins of the oracle's adjoint gradient of the far-field misfit against
centred finite differences of the misfit itself (h = 1e-6), on a small mixed
Dirichlet/Neumann cluster, plus a planted mistake that the pin catches."""
import numpy as np
import pytest

import oracle.msd_grad as G
import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _case():
    cl = W.small_mixed(seed=21, M=4, N=8, k=1.7)
    tgt = W.perturbed_target(cl, seed=40)
    betas = [0.3, 1.4]
    th = W.angles(24)
    rho_t, _ = O_.solve(tgt.centres, tgt.radii, tgt.bc, tgt.k, tgt.N, betas)
    Ft = O_.farfield(tgt.centres, tgt.radii, tgt.k, tgt.N, rho_t, th)
    return cl, betas, th, Ft


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def test_adjoint_gradient_matches_finite_differences():
    cl, betas, th, Ft = _case()
    J, gO, ga, gk, F = G.misfit_and_gradient(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, th, Ft)
    assert abs(J - G.misfit(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, th, Ft)) <= 1e-12 * J
    fO, fa, fk = G.misfit_gradient_fd(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, th, Ft)
    assert _rel(gO, fO) < 1e-6
    assert _rel(ga, fa) < 1e-6
    assert abs(gk - fk) < 1e-6 * abs(fk)


def test_planted_gradient_mistake_is_caught(monkeypatch):
    """Dropping the radius dependence of the far-field coefficients shows up
    in the radius gradient."""
    cl, betas, th, Ft = _case()
    good = G._farfield_matrix_derivs

    def bad(O, a, k, N, thetas):
        C, Cx, Cy, Ca, Ck = good(O, a, k, N, thetas)
        return C, Cx, Cy, 0 * Ca, Ck

    monkeypatch.setattr(G, "_farfield_matrix_derivs", bad)
    _, _, ga, _, _ = G.misfit_and_gradient(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, th, Ft)
    monkeypatch.undo()
    _, fa, _ = G.misfit_gradient_fd(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, th, Ft)
    assert _rel(ga, fa) > 1e-3
