"""Near field (Prop. 4.3, kernel K8) against the oracle's single-layer
potential, and the boundary condition through the whole GPU path.

Tolerance: 1e-5 of the largest |u| on the grid -- far point-disk pairs
(k r > 20) evaluate the Hankel functions in FP32 after an FP64 phase
(~1e-6 relative); pairs closer than that are FP64.  The boundary check:
on a sound-soft circle u + u_inc = 0 up to the truncation error of N = 12
(2.8e-9 with the oracle's densities), held to 1e-7.
"""
import numpy as np
import pytest

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


def grid(half, n):
    g = np.linspace(-half, half, n)
    X, Y = np.meshgrid(g, g, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def inside_any(cl, pts):
    d = np.hypot(pts[:, None, 0] - cl.centres[None, :, 0], pts[:, None, 1] - cl.centres[None, :, 1])
    return (d <= cl.radii[None, :]).any(axis=1)


@pytest.mark.parametrize("name", ["four_disks", "rand70"])
def test_nearfield_matches_oracle(msd, name):
    if name == "four_disks":
        cl = W.four_disks()
        pts = grid(5.0, 61)
    else:
        cl = W.random_cluster(seed=8, M=70, half_side=14.0, rmin=0.5, rmax=1.0, gap=0.2, k=2.5, N=12,
                              neumann_fraction=0.3)
        pts = grid(20.0, 45)
    # points just off two disk boundaries (FP64 near path)
    th = np.linspace(0.0, 2 * np.pi, 16, endpoint=False)
    for p in (0, cl.M - 1):
        rr = cl.radii[p] * 1.001
        pts = np.concatenate([pts, cl.centres[p] + rr * np.stack([np.cos(th), np.sin(th)], axis=1)])
    rng = np.random.default_rng(3)
    R = 2
    rho = rng.standard_normal((cl.ntot, R)) + 1j * rng.standard_normal((cl.ntot, R))
    pb = msd.Problem(cl)
    u = pb.nearfield(torch.from_numpy(rho).cuda(), pts).cpu().numpy()
    ins = inside_any(cl, pts)
    assert np.all(u[ins] == 0)
    ref = O_.single_layer_potential(cl.centres, cl.radii, cl.k, cl.N, rho, pts[~ins])
    err = np.abs(u[~ins] - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
    # host buffers give the same values
    u_h = np.zeros_like(u)
    msd.msd_nearfield(pb.handle, 0, rho, R, pts, u_h)
    assert np.array_equal(u_h, u)


def test_boundary_condition_through_gpu_path(msd):
    """Solve on the GPU, then evaluate the scattered field on the four
    sound-soft circles: the total field vanishes there."""
    cl = W.four_disks()
    beta = 0.4
    pb = msd.Problem(cl)
    res = pb.solve([beta], tol=1e-12)
    th = np.linspace(0.0, 2 * np.pi, 32, endpoint=False)
    pts = np.concatenate([cl.centres[p] + cl.radii[p] * (1 + 1e-9) * np.stack([np.cos(th), np.sin(th)], axis=1)
                          for p in range(cl.M)])
    u = pb.nearfield(res.rho, pts).cpu().numpy()[:, 0]
    uinc = np.exp(1j * cl.k * (np.cos(beta) * pts[:, 0] + np.sin(beta) * pts[:, 1]))
    assert np.abs(u + uinc).max() < 1e-7


# ---------------------------------------------------------------- point sources

def test_rhs_pointsource_matches_oracle(msd):
    cl = W.small_mixed(seed=3, M=6, N=10, k=2.0)
    src = np.array([[30.0, -12.0], [0.3, 6.5], [-4.0, -4.2]])
    pb = msd.Problem(cl)
    b = pb.rhs_pointsource(src).cpu().numpy()
    ref = O_.preconditioned_rhs_pointsource(cl.centres, cl.radii, cl.bc, cl.k, cl.N, src)
    assert np.abs(b - ref).max() <= 1e-12 * np.abs(ref).max()


def test_solve_pointsource_boundary_condition(msd):
    """Four sound-soft disks, N = 20, source at the centre of their square:
    GPU solve against the oracle's LU solution, and the total field on the
    circles through the GPU near field (truncation error ~1e-9 at N = 20)."""
    from scipy import special
    c0 = W.four_disks()
    cl = W.Cluster(c0.centres, c0.radii, c0.bc, c0.k, 20)
    s = np.array([0.0, 0.0])
    pb = msd.Problem(cl)
    res = pb.solve_pointsources([s], tol=1e-12)
    assert res.status == msd.MSD_OK
    A = O_.assemble(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
    rho_ref = np.linalg.solve(A, O_.rhs_pointsource(cl.centres, cl.radii, cl.bc, cl.k, cl.N, [s]))
    rho = res.rho.cpu().numpy()
    assert np.abs(rho - rho_ref).max() <= 1e-9 * np.abs(rho_ref).max()
    th = np.linspace(0.0, 2 * np.pi, 24, endpoint=False)
    pts = np.concatenate([cl.centres[p] + cl.radii[p] * (1 + 1e-12) * np.stack([np.cos(th), np.sin(th)], axis=1)
                          for p in range(cl.M)])
    u = pb.nearfield(res.rho, pts).cpu().numpy()[:, 0]
    uinc = 0.25j * special.hankel1(0, cl.k * np.hypot(pts[:, 0] - s[0], pts[:, 1] - s[1]))
    assert np.abs(u + uinc).max() <= 1e-8 * np.abs(uinc).max()
