"""Penetrable obstacles (section 7, Example II) through the C-ABI: the
transmission product, solves and exterior far field against the oracle.

Tolerances: FP64 products 1e-11 of the largest entry (two block-Toeplitz
sums of ~M n terms with ~1e-13 Bessel value errors, then 2 x 2 solves).
Solves stop at relres 1e-12 of the preconditioned system, so the densities
and far fields are held to 10 cond(B^-1 A) 1e-12 of their largest entry
(cond from the oracle's matrix: 15 for the 5-disk case, ~4.7e3 for the
70-disk one), FP64 and mixed alike.
"""
import numpy as np
import pytest
from scipy import special

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


def cases():
    c1 = W.small_mixed(seed=5, M=5, N=12, k=1.6)
    c2 = W.random_cluster(seed=8, M=70, half_side=14.0, rmin=0.5, rmax=1.0, gap=0.2, k=1.5, N=8)
    return [(c1, 3.1, np.array([1.0, 0.6, 2.0, 1.0, 1.4])), (c2, 2.2, None)]


def test_product_matches_oracle(msd):
    rng = np.random.default_rng(3)
    for cl, km, mu in cases():
        mu_o = np.ones(cl.M) if mu is None else mu
        P, _ = O_.preconditioned_penetrable(cl.centres, cl.radii, cl.k, km, mu_o, cl.N)
        pb = msd.Problem(cl)
        pb.set_penetrable(km, mu)
        for R in (1, 3):
            x = rng.standard_normal((2 * cl.ntot, R)) + 1j * rng.standard_normal((2 * cl.ntot, R))
            ref = P @ x
            xp = torch.from_numpy(np.ascontiguousarray(x[:cl.ntot])).cuda()
            xm = torch.from_numpy(np.ascontiguousarray(x[cl.ntot:])).cuda()
            yp, ym = pb.penetrable_matvec(xp, xm)
            y = np.concatenate([yp.cpu().numpy(), ym.cpu().numpy()])
            assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max(), (cl.M, R)
        pb.close()


def test_solve_and_far_field(msd):
    th = W.angles(36)
    betas = [0.4, 2.2]
    for cl, km, mu in cases():
        mu_o = np.ones(cl.M) if mu is None else mu
        rp_ref, rm_ref = O_.solve_penetrable(cl.centres, cl.radii, cl.k, km, mu_o, cl.N, betas)
        F_ref = O_.farfield(cl.centres, cl.radii, cl.k, cl.N, rp_ref, th)
        P, _ = O_.preconditioned_penetrable(cl.centres, cl.radii, cl.k, km, mu_o, cl.N)
        tol = 10 * np.linalg.cond(P) * 1e-12
        pb = msd.Problem(cl)
        pb.set_penetrable(km, mu)
        for prec, tol_rho, tol_F in ((msd.MSD_FP64, tol, tol), (msd.MSD_MIXED, tol, tol)):
            rp, rm, res = pb.solve_penetrable(betas, tol=1e-12, precision=prec)
            assert res.status == msd.MSD_OK, (cl.M, prec, res.relres)
            scale = max(np.abs(rp_ref).max(), np.abs(rm_ref).max())
            assert np.abs(rp.cpu().numpy() - rp_ref).max() <= tol_rho * scale
            assert np.abs(rm.cpu().numpy() - rm_ref).max() <= tol_rho * scale
            F = pb.farfield(rp, th).cpu().numpy()[0]
            assert np.abs(F - F_ref).max() <= tol_F * np.abs(F_ref).max(), (cl.M, prec)
        pb.close()


def test_single_disk_transmission_series(msd):
    a, kp, km, mu, beta = 0.9, 1.3, 2.6, 1.7, 0.7
    cl = W.Cluster(np.zeros((1, 2)), np.array([a]), np.array([0], np.int8), kp, 18)
    pb = msd.Problem(cl)
    pb.set_penetrable(km, [mu])
    rp, _, res = pb.solve_penetrable([beta], tol=1e-13)
    th = np.linspace(0, 2 * np.pi, 13)
    F = pb.farfield(rp, th).cpu().numpy()[0, :, 0]
    m = np.arange(-40, 41)
    num = mu * km * special.jvp(m, km * a) * special.jv(m, kp * a) - kp * special.jvp(m, kp * a) * special.jv(m, km * a)
    den = kp * special.h1vp(m, kp * a) * special.jv(m, km * a) - mu * km * special.jvp(m, km * a) * special.hankel1(m, kp * a)
    ref = np.exp(-1j * np.pi / 4) * np.sqrt(2 / (np.pi * kp)) * (np.exp(1j * np.outer(th - beta, m)) @ (num / den))
    assert np.abs(F - ref).max() <= 1e-10 * np.abs(ref).max()
    pb.close()


def test_two_configurations_and_geometry_update(msd):
    c1 = W.small_mixed(seed=5, M=5, N=12, k=1.6)
    c2 = W.small_mixed(seed=6, M=4, N=10, k=2.1)
    pb = msd.Problem([c1, c2])
    pb.set_penetrable([3.1, 1.2])
    betas = [0.4]
    rp, _, res = pb.solve_penetrable(betas, tol=1e-12)
    assert res.status == msd.MSD_OK
    rp = rp.cpu().numpy()
    off = [0, c1.ntot]
    for c, (cl, km) in enumerate(((c1, 3.1), (c2, 1.2))):
        ref, _ = O_.solve_penetrable(cl.centres, cl.radii, cl.k, km, np.ones(cl.M), cl.N, betas)
        got = rp[off[c]:off[c] + cl.ntot]
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), c
    # move every disk by a small shift; the interior-wavenumber data follows
    cen = np.concatenate([c1.centres, c2.centres]) + np.array([0.05, -0.03])
    pb.update_geometry(centres=np.ascontiguousarray(cen))
    rp2, _, res = pb.solve_penetrable(betas, tol=1e-12)
    ref, _ = O_.solve_penetrable(c1.centres + np.array([0.05, -0.03]), c1.radii, c1.k, 3.1, np.ones(c1.M), c1.N, betas)
    assert np.abs(rp2.cpu().numpy()[:c1.ntot] - ref).max() <= 1e-9 * np.abs(ref).max()
    pb.close()


def test_mode_switches(msd):
    cl = W.small_mixed(seed=5, M=5, N=12, k=1.6)
    pb = msd.Problem(cl)
    rho0 = pb.solve([0.3], tol=1e-12).rho.cpu().numpy()
    pb.set_penetrable(2.0)
    with pytest.raises(msd.MsdError):
        pb.set_formulation("cfie")
    pb.set_penetrable(None)
    assert np.abs(pb.solve([0.3], tol=1e-12).rho.cpu().numpy() - rho0).max() <= 1e-12 * np.abs(rho0).max()
    pb.set_formulation("cfie")
    with pytest.raises(msd.MsdError):
        pb.set_penetrable(2.0)
    pb.close()


def test_point_source_solve(msd):
    cl = W.small_mixed(seed=5, M=3, N=14, k=1.6)
    km, mu = 2.4, np.array([1.0, 1.5, 0.7])
    src = np.array([[9.0, -7.5], [-6.0, 8.0]])
    A = O_.assemble_penetrable(cl.centres, cl.radii, cl.k, km, mu, cl.N)
    ref = np.linalg.solve(A, O_.rhs_penetrable_pointsource(cl.centres, cl.radii, cl.k, cl.N, src))
    P, _ = O_.preconditioned_penetrable(cl.centres, cl.radii, cl.k, km, mu, cl.N)
    tol = 10 * np.linalg.cond(P) * 1e-12
    pb = msd.Problem(cl)
    pb.set_penetrable(km, mu)
    rp, rm, res = pb.solve_penetrable(sources=src, tol=1e-12)
    assert res.status == msd.MSD_OK
    got = np.concatenate([rp.cpu().numpy(), rm.cpu().numpy()])
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    pb.close()


def test_interior_field_and_transmission(msd):
    """The interior field u- = L- rho- (msd_penetrable_interior_field) at
    points inside every disk against the oracle's single_layer_potential_inside
    on the oracle's densities (1e-10 of the largest value), and the
    transmission condition u+ + u_inc = u- across each circle: the GPU's
    exterior near field plus the incident wave just outside, and its interior
    field just inside, agree to the truncation level of the solve (the
    oracle's own pointwise residual on this case at N = 12 is 2.2e-6)."""
    cl, km, mu = cases()[0]
    betas = [0.4]
    rp_ref, rm_ref = O_.solve_penetrable(cl.centres, cl.radii, cl.k, km, mu, cl.N, betas)
    pb = msd.Problem(cl)
    pb.set_penetrable(km, mu)
    rng = np.random.default_rng(7)
    pts, owner = [], []
    for p in range(cl.M):
        r = cl.radii[p] * np.sqrt(rng.uniform(0.0, 0.95, 6))
        t = rng.uniform(0, 2 * np.pi, 6)
        pts.append(cl.centres[p] + np.stack([r * np.cos(t), r * np.sin(t)], 1))
        owner += [p] * 6
    pts = np.concatenate(pts + [np.array([[40.0, 40.0]])])   # last point outside every disk
    u = pb.interior_field(torch.from_numpy(rm_ref).cuda(), pts).cpu().numpy()
    ref = np.concatenate([O_.single_layer_potential_inside(cl.centres, cl.radii, km, cl.N, rm_ref,
                                                           pts[i:i + 1], owner[i]) for i in range(len(owner))])
    assert np.abs(u[:-1] - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(u[-1]).max() == 0.0
    # transmission condition from the GPU's own solve
    res_p = torch.empty((cl.ntot, 1), dtype=torch.complex128, device="cuda")
    res_m = torch.empty_like(res_p)
    st = msd.msd_solve_penetrable(pb.handle, 1, np.array([betas]), msd.msd_opts(1e-12, 0, 3000, 0, 0.0, 0, 0),
                                  res_p, res_m)
    assert st == msd.MSD_OK
    th = np.linspace(0.0, 2 * np.pi, 8, endpoint=False)
    for p in range(cl.M):
        e = np.stack([np.cos(th), np.sin(th)], 1)
        out_pts = cl.centres[p] + (cl.radii[p] * (1 + 1e-9)) * e
        in_pts = cl.centres[p] + (cl.radii[p] * (1 - 1e-9)) * e
        us = pb.nearfield(res_p, out_pts).cpu().numpy()[:, 0]
        uinc = np.exp(1j * cl.k * (np.cos(betas[0]) * out_pts[:, 0] + np.sin(betas[0]) * out_pts[:, 1]))
        ui = pb.interior_field(res_m, in_pts).cpu().numpy()[:, 0]
        assert np.abs(us + uinc - ui).max() <= 1e-5 * np.abs(uinc).max(), p
    pb.close()
