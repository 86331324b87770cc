"""Products and solves with recomputed generators (MSD_GEN_RECOMPUTE) against
the oracle and against the stored-generator path.

Chunk budgets are chosen to exercise every layout of the chunk plan: one
chunk per problem (default 64 MiB), configurations packed into shared
chunks, and configurations cut into 32-source x 32-target blocks with ragged
source and target tails (later source blocks accumulate into the partial
sums).  Tolerances as for stored generators: FP64 products 1e-11, FP32
products 1e-5 relative to the oracle; the same generator values are summed
in another grouping, so recomputed and stored FP64 products agree to 1e-13.
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


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def rand_x(ntot, R, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ntot, R)) + 1j * rng.standard_normal((ntot, R))


def rand70():
    return W.random_cluster(seed=8, M=70, half_side=14.0, rmin=0.5, rmax=1.0, gap=0.2, k=2.5, N=12,
                            neumann_fraction=0.3)


# budgets for rand70 (N = 12, L = 49): 0 -> one chunk; 40 kB -> 3 x 3 blocks of
# 32 targets x 32 sources (complex128) with tails of 6 sources / 6 targets
BUDGETS = [0, 40_000, 200_000]


@pytest.mark.parametrize("budget", BUDGETS)
@pytest.mark.parametrize("fp64,R", [(True, 1), (True, 3), (False, 1), (False, 8)])
def test_recomputed_product(msd, budget, fp64, R):
    cl = rand70()
    ref_op = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
    x = rand_x(cl.ntot, R, seed=R + 5)
    if not fp64:
        x = x.astype(np.complex64)
    ref = ref_op @ x.astype(np.complex128)
    prec = msd.MSD_FP64 if fp64 else msd.MSD_FP32
    xd = torch.from_numpy(x).cuda()
    ps = msd.Problem(cl)
    ys = ps.matvec(xd, prec).cpu().numpy()
    pr = msd.Problem(cl)
    pr.set_generator_mode(msd.MSD_GEN_RECOMPUTE, budget)
    yr = pr.matvec(xd, prec).cpu().numpy()
    yr2 = pr.matvec(xd, prec).cpu().numpy()
    assert np.array_equal(yr, yr2)  # the chunk buffer is fully rewritten every product
    assert relerr(yr, ref) < (1e-11 if fp64 else 1e-5)
    if fp64:
        assert relerr(yr, ys) < 1e-13


def test_recomputed_product_batched(msd):
    """Three configurations with different N: a 20 kB budget packs the two
    small ones into one chunk and cuts the 70-disk one into blocks."""
    cls = [W.small_mixed(seed=3, M=6, N=10, k=2.0), rand70(), W.four_disks()]
    pr = msd.Problem(cls)
    ps = msd.Problem(cls)
    pr.set_generator_mode(msd.MSD_GEN_RECOMPUTE, 20_000)
    R = 2
    x = rand_x(pr.ntot, R, seed=9)
    xd = torch.from_numpy(x).cuda()
    yr = pr.matvec(xd, msd.MSD_FP64).cpu().numpy()
    ys = ps.matvec(xd, msd.MSD_FP64).cpu().numpy()
    assert relerr(yr, ys) < 1e-13
    off = 0
    for cl in cls:
        A = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
        assert relerr(yr[off:off + cl.ntot], A @ x[off:off + cl.ntot]) < 1e-11
        off += cl.ntot


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_recomputed_solve(msd, precision):
    cl = rand70()
    betas = np.array([0.3, 2.0])
    prec = msd.MSD_FP64 if precision == "fp64" else msd.MSD_MIXED
    pb = msd.Problem(cl)
    rs = pb.solve(betas, tol=1e-12, precision=prec)
    rr = pb.solve(betas, tol=1e-12, precision=prec, gen_mode=msd.MSD_GEN_RECOMPUTE)
    assert (rs.flags == 0).all() and (rr.flags == 0).all()
    rho_ref, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas)
    assert relerr(rr.rho.cpu().numpy(), rho_ref) < 1e-9
    assert relerr(rr.rho.cpu().numpy(), rs.rho.cpu().numpy()) < 1e-9


def test_generator_mode_switch(msd):
    """Streamed -> recompute (stored arrays freed) -> streamed again, with the
    geometry moved in between: every product follows the current geometry."""
    cl = rand70()
    pb = msd.Problem(cl)
    x = rand_x(cl.ntot, 1, seed=3)
    xd = torch.from_numpy(x).cuda()
    y0 = pb.matvec(xd).cpu().numpy()
    pb.set_generator_mode(msd.MSD_GEN_RECOMPUTE, 40_000)
    cen = cl.centres * 1.01  # a dilation changes every b_pq (a translation would not)
    pb.update_geometry(cen, cl.radii, np.array([cl.k]))
    y1 = pb.matvec(xd).cpu().numpy()
    A1 = O_.preconditioned_dense(cen, cl.radii, cl.bc, cl.k, cl.N)
    assert relerr(y1, A1 @ x) < 1e-11
    pb.set_generator_mode(msd.MSD_GEN_STREAMED)
    y2 = pb.matvec(xd).cpu().numpy()
    assert relerr(y2, y1) < 1e-13
    pb.set_generator_mode(msd.MSD_GEN_AUTO)  # small problem: stored
    assert relerr(pb.matvec(xd).cpu().numpy(), y1) < 1e-13
    assert not np.allclose(y0, y1)
    with pytest.raises(msd.MsdError):
        pb.set_generator_mode(7)
