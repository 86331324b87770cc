"""Per-disk truncation orders (section 5, msd_set_truncation) through the
C ABI against the oracle's ragged system (assemble_ragged, solve_ragged,
farfield_ragged).  The GPU keeps the padded layout of the configuration's N;
the modes |m| > N_p are an identity block with a zero right-hand side.

Checks: products on the kept rows (FP64 1e-11, FP32 1e-5, the CUDA-core
kernels and the shift-GEMM tensor-core kernel) and y = x on the dropped
rows; FP64 and mixed solves against the oracle's LU solution of the ragged
system (within cond * relres) with exact zeros on the dropped rows; far
fields; two configurations of different N in one problem; N_p = N on every
disk reproduces the uniform problem; the orders survive a geometry update;
invalid orders and the excluded combinations are refused."""
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


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def cluster(seed=12, M=9, k=3.0, eps=1e-8):
    """Radii 0.2 .. 1.6 (k a from 0.6 to 4.8), mixed boundary conditions,
    N_p from eq. (Np), N = max N_p."""
    rng = np.random.default_rng(seed)
    O, a = W.random_disks(rng, M, 7.0, 0.2, 1.6, 0.3)
    bc = (rng.uniform(size=M) < 0.5).astype(np.int8)
    Ns = np.array([O_.truncation_order(k * ai, eps) for ai in a])
    return W.Cluster(O, a, bc, k, int(Ns.max()), f"ragged{M}"), Ns


def kept_rows(cl, Ns, row0=0):
    """Padded rows (configuration N) of the ragged unknowns, in ragged order."""
    return np.concatenate([row0 + p * cl.n + cl.N + O_.modes(int(Ns[p])) for p in range(cl.M)])


def test_ragged_products(msd):
    cl, Ns = cluster()
    assert Ns.min() < Ns.max()
    pb = msd.Problem(cl)
    pb.set_truncation(Ns)
    Ar = O_.preconditioned_ragged(cl.centres, cl.radii, cl.bc, cl.k, Ns)
    keep = kept_rows(cl, Ns)
    drop = np.setdiff1d(np.arange(cl.ntot), keep)
    rng = np.random.default_rng(3)
    for R in (1, 8):
        x = rng.standard_normal((cl.ntot, R)) + 1j * rng.standard_normal((cl.ntot, R))
        xk = x.copy()
        xk[drop] = 0.0
        y = pb.matvec(torch.from_numpy(xk).cuda(), msd.MSD_FP64).cpu().numpy()
        ref = Ar @ xk[keep]
        assert relerr(y[keep], ref) < 1e-11, R
        assert np.abs(y[drop]).max() == 0.0
        # arbitrary values on the dropped rows: identity there, no coupling
        y2 = pb.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP64).cpu().numpy()
        assert relerr(y2[keep], ref) < 1e-11 and np.array_equal(y2[drop], x[drop])
        x32 = xk.astype(np.complex64)
        ref32 = Ar @ x32[keep].astype(np.complex128)
        y32 = pb.matvec(torch.from_numpy(x32).cuda(), msd.MSD_FP32).cpu().numpy()
        assert relerr(y32[keep], ref32) < 1e-5, R
    pb.set_tile(8, msd.MSD_FP32, 0, 8)                      # the shift-GEMM tensor-core kernel
    x32 = (rng.standard_normal((cl.ntot, 8)) + 1j * rng.standard_normal((cl.ntot, 8))).astype(np.complex64)
    x32[drop] = 0
    y32 = pb.matvec(torch.from_numpy(x32).cuda(), msd.MSD_FP32).cpu().numpy()
    assert relerr(y32[keep], Ar @ x32[keep].astype(np.complex128)) < 1e-5


def test_ragged_solves_and_far_field(msd):
    cl, Ns = cluster()
    betas = [0.4, 2.2]
    th = W.angles(48)
    Ar = O_.preconditioned_ragged(cl.centres, cl.radii, cl.bc, cl.k, Ns)
    ref = O_.solve_ragged(cl.centres, cl.radii, cl.bc, cl.k, Ns, betas)
    Fref = O_.farfield_ragged(cl.centres, cl.radii, cl.k, Ns, ref, th)
    keep = kept_rows(cl, Ns)
    drop = np.setdiff1d(np.arange(cl.ntot), keep)
    cond = np.linalg.cond(Ar)
    pb = msd.Problem(cl)
    pb.set_truncation(Ns)
    for prec, tol in ((msd.MSD_FP64, 1e-12), (msd.MSD_MIXED, 1e-11)):
        res = pb.solve(betas, tol=tol, precision=prec)
        assert res.status == msd.MSD_OK, (prec, res.relres)
        rho = res.rho.cpu().numpy()
        assert np.abs(rho[drop]).max() == 0.0
        assert relerr(rho[keep], ref) < 10 * cond * tol, prec
        F = pb.farfield(res.rho, th).cpu().numpy()[0]
        assert relerr(F, Fref) < 10 * cond * tol, prec
    # the orders survive a geometry update; N_p = N restores the uniform system
    pb.update_geometry(centres=cl.centres + np.array([0.5, -0.25]))
    moved = O_.solve_ragged(cl.centres + np.array([0.5, -0.25]), cl.radii, cl.bc, cl.k, Ns, betas)
    res = pb.solve(betas, tol=1e-12)
    assert relerr(res.rho.cpu().numpy()[keep], moved) < 10 * cond * 1e-12
    pb.update_geometry(centres=cl.centres)
    pb.set_truncation(None)
    uni, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, method="lu")
    res = pb.solve(betas, tol=1e-12)
    Au = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
    assert relerr(res.rho.cpu().numpy(), uni) < 10 * np.linalg.cond(Au) * 1e-12


def test_ragged_batched_configurations(msd):
    c1, n1 = cluster(seed=12, M=9)
    c2, n2 = cluster(seed=13, M=6, k=1.7)
    pb = msd.Problem([c1, c2])
    pb.set_truncation(np.concatenate([n1, n2]))
    betas = np.array([[0.4, 1.0], [2.0, 3.0]])
    res = pb.solve(betas, tol=1e-12, precision=msd.MSD_MIXED)
    assert res.status == msd.MSD_OK
    rho = res.rho.cpu().numpy()
    for c, (cl, Ns) in enumerate(((c1, n1), (c2, n2))):
        ref = O_.solve_ragged(cl.centres, cl.radii, cl.bc, cl.k, Ns, betas[c])
        Ar = O_.preconditioned_ragged(cl.centres, cl.radii, cl.bc, cl.k, Ns)
        keep = kept_rows(cl, Ns, pb.row_offset(c))
        assert relerr(rho[keep], ref) < 10 * np.linalg.cond(Ar) * 1e-11, c


def test_ragged_errors(msd):
    cl, Ns = cluster()
    pb = msd.Problem(cl)
    bad = Ns.copy()
    bad[0] = cl.N + 1
    with pytest.raises(msd.MsdError) as e:
        pb.set_truncation(bad)
    assert e.value.status == msd.MSD_ERR_ARG
    pb.set_truncation(Ns)
    with pytest.raises(msd.MsdError):
        pb.set_formulation("cfie")
    with pytest.raises(msd.MsdError):
        pb.set_penetrable(2.0)
    with pytest.raises(msd.MsdError):
        pb.grad_farfield_misfit([0.1], W.angles(8), np.zeros((1, 8, 1), np.complex128))
    pb.set_truncation(None)
    pb.set_formulation("cfie")
    with pytest.raises(msd.MsdError):
        pb.set_truncation(Ns)
