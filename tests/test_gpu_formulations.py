"""Integral-equation formulations (sections 3, 4.2, 5) through the C-ABI:
products, right-hand sides, solves, far and near fields of EFIE, MFIE,
CFIE and Brakhage-Werner rows against the oracle.

Tolerances: FP64 products 1e-11 of the largest entry (as for the default
rows: sums of ~M n terms carrying ~1e-13 Bessel value errors); FP32 products
1e-5; far fields of solves to relres 1e-12 against the oracle's LU solution
1e-10 (the formulations are well conditioned); the near field 1e-5 (far
point-disk pairs in FP32 after an FP64 phase).
"""
import numpy as np
import pytest
from scipy import special

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

OPS = ("I", "L", "M", "N", "D")


@pytest.fixture(scope="module")
def msd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_8186_gb300 import msd as m
    return m


def as_dicts(op, rhs, rep):
    """Weight arrays (layout of msd_set_formulation) as the oracle's dictionaries."""
    ow = {c: {OPS[o]: op[c, o] for o in range(5) if op[c, o] != 0} for c in (0, 1)}
    rw = {c: {"U": rhs[c, 0], "dU": rhs[c, 1]} for c in (0, 1)}
    return ow, rw, {"L": rep[0], "M": rep[1]}


def as_arrays(ow, rw, pw):
    """The oracle's weight dictionaries in the layout of msd_set_formulation."""
    op = np.array([[ow[c].get(o, 0) for o in OPS] for c in (0, 1)], np.complex128)
    rhs = np.array([[rw[c].get("U", 0), rw[c].get("dU", 0)] for c in (0, 1)], np.complex128)
    return op, rhs, np.array([pw["L"], pw["M"]], np.complex128)


KINDS = ["efie", "mfie", "cfie", "bwie"]


def clusters():
    return [W.small_mixed(seed=3, M=6, N=10, k=2.0),
            W.random_cluster(seed=8, M=70, half_side=14.0, rmin=0.5, rmax=1.0, gap=0.2, k=2.5, N=8,
                             neumann_fraction=0.3)]


@pytest.mark.parametrize("kind", KINDS)
def test_products_match_oracle(msd, kind):
    rng = np.random.default_rng(5)
    for cl in clusters():
        ow, _, _ = O_.standard_formulation(kind, k=cl.k)
        Ap, _ = O_.preconditioned_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, ow)
        pb = msd.Problem(cl)
        pb.set_formulation(kind)               # by name: the library forms the weights (eta = i k)
        for R in (1, 3, 16):
            x = rng.standard_normal((cl.ntot, R)) + 1j * rng.standard_normal((cl.ntot, R))
            ref = Ap @ x
            y = pb.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP64).cpu().numpy()
            assert np.abs(y - ref).max() <= 1e-11 * np.abs(ref).max(), (kind, cl.M, R)
            x32 = x.astype(np.complex64)
            y32 = pb.matvec(torch.from_numpy(x32).cuda(), msd.MSD_FP32).cpu().numpy()
            ref32 = Ap @ x32.astype(np.complex128)
            assert np.abs(y32 - ref32).max() <= 1e-5 * np.abs(ref32).max(), (kind, cl.M, R)
        pb.close()


def test_efie_weights_reproduce_default_rows(msd):
    cl = clusters()[0]
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal((cl.ntot, 4)) + 1j * rng.standard_normal((cl.ntot, 4))).cuda()
    pb = msd.Problem(cl)
    y0 = pb.matvec(x).cpu().numpy()
    b0 = pb.rhs([0.2, 1.1]).cpu().numpy()
    pb.set_formulation("efie")
    y1 = pb.matvec(x).cpu().numpy()
    b1 = pb.rhs([0.2, 1.1]).cpu().numpy()
    assert np.abs(y1 - y0).max() <= 1e-13 * np.abs(y0).max()
    assert np.abs(b1 - b0).max() <= 1e-14 * np.abs(b0).max()
    pb.set_formulation(None)
    assert np.array_equal(pb.matvec(x).cpu().numpy(), y0)


@pytest.mark.parametrize("kind", KINDS)
def test_rhs_solve_and_fields(msd, kind):
    cl = W.small_mixed(seed=3, M=6, N=14, k=2.0)
    ow, rw, pw = O_.standard_formulation(kind, k=cl.k)
    betas = [0.3, 2.0]
    th = W.angles(48)
    pb = msd.Problem(cl)
    pb.set_formulation(kind)
    _, d = O_.preconditioned_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, ow)
    b_ref = O_.rhs_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, rw) / d[:, None]
    b = pb.rhs(betas).cpu().numpy()
    assert np.abs(b - b_ref).max() <= 1e-12 * np.abs(b_ref).max()
    dens_ref = O_.solve_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, ow, rw)
    F_ref = O_.farfield_formulation(cl.centres, cl.radii, cl.k, cl.N, dens_ref, th, pw)
    for prec, tol in ((msd.MSD_FP64, 1e-10), (msd.MSD_MIXED, 1e-9)):
        res = pb.solve(betas, tol=1e-12, precision=prec)
        assert res.status == msd.MSD_OK, (kind, prec)
        F = pb.farfield(res.rho, th).cpu().numpy()[0]
        assert np.abs(F - F_ref).max() <= tol * np.abs(F_ref).max(), (kind, prec)
        assert np.all(res.true_relres < 1e-9)
    # near field of the formulation's representation
    g = np.linspace(-12.0, 12.0, 25)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    dist = np.hypot(pts[:, None, 0] - cl.centres[None, :, 0], pts[:, None, 1] - cl.centres[None, :, 1])
    pts = pts[(dist > cl.radii[None, :] * 1.01).all(axis=1)]
    res = pb.solve(betas, tol=1e-12)
    u = pb.nearfield(res.rho, pts).cpu().numpy()
    u_ref = O_.potential_formulation(cl.centres, cl.radii, cl.k, cl.N, dens_ref, pts, pw)
    assert np.abs(u - u_ref).max() <= 1e-5 * np.abs(u_ref).max()
    pb.close()


def mie_far(k, a, beta, th, terms=40):
    m = np.arange(-terms, terms + 1)
    c = special.jv(m, k * a) / special.hankel1(m, k * a)
    return -np.exp(-1j * np.pi / 4) * np.sqrt(2 / (np.pi * k)) * (np.exp(1j * np.outer(th - beta, m)) @ c)


def test_dirichlet_resonance(msd):
    """One sound-soft disk at k a = j_{0,1}.  The unpreconditioned EFIE row
    m = 0 vanishes there (pinned on the oracle), but every row is divided by
    its self block, in which the same J_0(k a) cancels: EFIE, CFIE and BWIE
    all give the Mie far field."""
    a = 1.0
    k = special.jn_zeros(0, 1)[0]
    cl = W.Cluster(np.zeros((1, 2)), np.array([a]), np.array([0], np.int8), k, 14)
    pb = msd.Problem(cl)
    th = W.angles(24)
    ref = mie_far(k, a, 0.9, th)
    for kind in ("efie", "cfie", "bwie"):
        pb.set_formulation(kind)
        res = pb.solve([0.9], tol=1e-13)
        assert res.status == msd.MSD_OK
        F = pb.farfield(res.rho, th).cpu().numpy()[0, :, 0]
        assert np.abs(F - ref).max() <= 1e-11 * np.abs(ref).max(), kind
    pb.close()


def test_vanishing_self_block_is_an_error(msd):
    """All weights of the sound-soft rows zero: the self block is 0 and the
    call fails with MSD_ERR_NONFINITE."""
    pb = msd.Problem(W.small_mixed(seed=3, M=6, N=10, k=2.0))
    op, rhs, rep = as_arrays(*O_.standard_formulation("efie"))
    op[msd.MSD_DIRICHLET, :] = 0
    with pytest.raises(msd.MsdError) as e:
        pb.set_formulation(op=op, rhs=rhs, rep=rep)
    assert e.value.status == msd.MSD_ERR_NONFINITE
    pb.close()


def test_time_reversal_is_formulation_independent(msd):
    cl = W.small_mixed(seed=3, M=6, N=14, k=2.0)
    pb = msd.Problem(cl)
    e0, _, _, _ = pb.dort(32, want_F=False, want_T=False)
    pb.set_formulation("bwie")
    e1, _, _, _ = pb.dort(32, want_F=False, want_T=False)
    e0, e1 = e0.cpu().numpy(), e1.cpu().numpy()
    assert np.abs(e1 - e0).max() <= 1e-9 * e0.max()
    pb.close()


def test_default_rows_required(msd):
    cl = W.small_mixed(seed=3, M=6, N=10, k=2.0)
    pb = msd.Problem(cl)
    pb.set_formulation("cfie")
    with pytest.raises(msd.MsdError):
        pb.grad_farfield_misfit([0.1], W.angles(8), np.zeros((1, 8, 1), np.complex128))
    x = torch.zeros((cl.ntot, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(msd.MsdError):
        msd.msd_matvec_noalloc(pb.handle, 1, msd.MSD_FP64, x, torch.empty_like(x))
    pb.set_formulation(None)
    pb.close()


def test_named_formulation_per_configuration_eta(msd):
    """Two configurations with different k set to CFIE and Brakhage-Werner by
    name through the C ABI (msd_set_formulation_kind, eta = i k of each
    configuration; then an explicit eta): products and far fields of solves
    against the oracle's statement of the same formulations."""
    cls = [W.small_mixed(seed=3, M=6, N=12, k=2.0), W.small_mixed(seed=4, M=5, N=12, k=3.1)]
    pb = msd.Problem(cls)
    betas = [0.3, 2.0]
    th = W.angles(40)
    rng = np.random.default_rng(2)
    for kind, alpha, eta in (("cfie", 0.3, None), ("bwie", 0.5, None), ("cfie", 0.6, 0.5 + 1.7j)):
        msd.msd_set_formulation_kind(pb.handle, kind, alpha, eta)
        x = rng.standard_normal((pb.ntot, 2)) + 1j * rng.standard_normal((pb.ntot, 2))
        y = pb.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP64).cpu().numpy()
        res = pb.solve(betas, tol=1e-12)
        assert res.status == msd.MSD_OK, kind
        F = pb.farfield(res.rho, th).cpu().numpy()
        for c, cl in enumerate(cls):
            ow, rw, pw = O_.standard_formulation(kind, alpha=alpha, eta=eta, k=cl.k)
            Ap, _ = O_.preconditioned_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, ow)
            r0 = pb.row_offset(c)
            ref = Ap @ x[r0:r0 + cl.ntot]
            assert np.abs(y[r0:r0 + cl.ntot] - ref).max() <= 1e-11 * np.abs(ref).max(), (kind, c)
            dens = O_.solve_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, ow, rw)
            F_ref = O_.farfield_formulation(cl.centres, cl.radii, cl.k, cl.N, dens, th, pw)
            assert np.abs(F[c] - F_ref).max() <= 1e-10 * np.abs(F_ref).max(), (kind, c)
    with pytest.raises(msd.MsdError) as e:
        msd.msd_set_formulation_kind(pb.handle, "cfie", 0.5, 1.0)       # Im(eta) = 0
    assert e.value.status == msd.MSD_ERR_ARG
    pb.close()
