"""Gradient of the far-field misfit on the GPU (adjoint kernels behind
msd_grad_farfield_misfit) against the oracle's analytic adjoint gradient and
against centred finite differences (h = 1e-6) of the GPU misfit.

Tolerances: 1e-7 relative against the oracle (both are adjoint gradients of
the same discrete misfit; the GPU solves to relres 1e-13 here); 1e-5 against
finite differences at full size (the gradient bound of this project: FD
truncation h^2 and solve error / h).
"""
import numpy as np
import pytest

import oracle.msd_grad as G
import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def msd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_8186_gb300 import msd as m
    return m


def _target_far_field_oracle(cl, betas, th):
    tgt = W.perturbed_target(cl, seed=40)
    rho_t, _ = O_.solve(tgt.centres, tgt.radii, tgt.bc, tgt.k, tgt.N, betas)
    return O_.farfield(tgt.centres, tgt.radii, tgt.k, tgt.N, rho_t, th)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.mark.parametrize("case", ["mixed4", "mixed12", "cluster40_k10"])
def test_gradient_matches_oracle(msd, case):
    if case == "mixed4":
        cl = W.small_mixed(seed=21, M=4, N=8, k=1.7)
        betas, th = np.array([0.3, 1.4]), W.angles(24)
    elif case == "mixed12":
        cl = W.small_mixed(seed=5, M=12, N=10, k=2.2, half_side=12.0)
        betas, th = W.angles(3), W.angles(60)
    else:
        cl = W.random_cluster(seed=4, M=40, half_side=14.0, rmin=0.8, rmax=1.2, gap=0.2, k=10.0, N=22)
        betas, th = W.angles(16), W.angles(360)
    Ft = _target_far_field_oracle(cl, betas, th)
    J0, gO0, ga0, gk0, _ = G.misfit_and_gradient(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, th, Ft)
    pb = msd.Problem(cl)
    J, gO, ga, gk = pb.grad_farfield_misfit(betas, th, Ft.reshape(1, len(th), len(betas)), tol=1e-13)
    assert abs(J[0] - J0) <= 1e-9 * J0
    assert _rel(gO, gO0) < 1e-7, _rel(gO, gO0)
    assert _rel(ga, ga0) < 1e-7, _rel(ga, ga0)
    assert abs(gk[0] - gk0) < 1e-7 * abs(gk0)


def test_gradient_full_size_vs_finite_differences(msd):
    """M = 200, k = 10, N = 22, 16 incidences, 360 samples: sampled gradient
    components against centred differences of the GPU misfit (h = 1e-6)."""
    cl = W.cluster_200()
    betas, th = W.angles(16), W.angles(360)
    tgt = W.perturbed_target(cl, seed=40)
    pt = msd.Problem(tgt)
    rt = pt.solve(betas, tol=1e-13, precision=msd.MSD_MIXED)
    Ft = pt.farfield(rt.rho, th).cpu().numpy()
    pt.close()
    pb = msd.Problem(cl)
    J, gO, ga, gk = pb.grad_farfield_misfit(betas, th, Ft, tol=1e-13, precision=msd.MSD_MIXED)

    def misfit(O, a, k):
        pb.update_geometry(O, a, np.array([k]))
        r = pb.solve(betas, tol=1e-13, precision=msd.MSD_MIXED)
        F = pb.farfield(r.rho, th).cpu().numpy()
        return float(np.sum(np.abs(F - Ft) ** 2))

    h = 1e-6
    O, a, k = cl.centres.copy(), cl.radii.copy(), cl.k
    scale = max(np.abs(gO).max(), np.abs(ga).max())
    checks = []
    for p, c in [(0, 0), (57, 1), (143, 0)]:
        Op, Om = O.copy(), O.copy()
        Op[p, c] += h
        Om[p, c] -= h
        checks.append((gO[p, c], (misfit(Op, a, k) - misfit(Om, a, k)) / (2 * h)))
    for p in (11, 190):
        ap, am = a.copy(), a.copy()
        ap[p] += h
        am[p] -= h
        checks.append((ga[p], (misfit(O, ap, k) - misfit(O, am, k)) / (2 * h)))
    gk_fd = (misfit(O, a, k + h) - misfit(O, a, k - h)) / (2 * h)
    for g, fd in checks:
        assert abs(g - fd) <= 1e-5 * max(abs(fd), 1e-3 * scale), (g, fd)
    assert abs(gk[0] - gk_fd) <= 1e-5 * abs(gk_fd), (gk[0], gk_fd)


def test_autograd_function(msd):
    cl = W.small_mixed(seed=5, M=8, N=10, k=2.2, half_side=10.0)
    betas, th = W.angles(2), W.angles(40)
    Ft = _target_far_field_oracle(cl, betas, th).reshape(1, len(th), len(betas))
    pb = msd.Problem(cl)
    cen = torch.tensor(cl.centres, dtype=torch.float64, requires_grad=True)
    rad = torch.tensor(cl.radii, dtype=torch.float64, requires_grad=True)
    kk = torch.tensor([cl.k], dtype=torch.float64, requires_grad=True)
    J = msd.farfield_misfit(pb, cen, rad, kk, betas, th, Ft, tol=1e-13)
    (2.0 * J).backward()
    J1, gO, ga, gk = pb.grad_farfield_misfit(betas, th, Ft, tol=1e-13)
    assert abs(float(J) - J1[0]) <= 1e-12 * J1[0]
    assert np.allclose(cen.grad.numpy(), 2 * gO, rtol=1e-12, atol=0)
    assert np.allclose(rad.grad.numpy(), 2 * ga, rtol=1e-12, atol=0)
    assert np.allclose(kk.grad.numpy(), 2 * gk, rtol=1e-12, atol=0)
