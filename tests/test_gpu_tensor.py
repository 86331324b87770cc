"""The tensor-core (tcgen05, 3xTF32) block-Toeplitz product against the oracle.

Shapes: column tiles TC = 16, 32, 64 (R = 64 admits all three); target tiles
of floor(128 / n) disks restarted at every 32-disk boundary (rand70: n = 25,
5 disks per tile, ragged at 32, 64 and at M = 70); batched configurations of
different N; stored and recomputed generators (chunked, accumulating source
blocks); and an FP32-inner mixed solve running on it.  Tolerance 1e-5
relative, as for the CUDA-core FP32 product.
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
    return (rng.standard_normal((ntot, R)) + 1j * rng.standard_normal((ntot, R))).astype(np.complex64)


def rand70():
    return W.random_cluster(seed=8, M=70, half_side=14.0, rmin=0.5, rmax=1.0, gap=0.2, k=2.5, N=12,
                            neumann_fraction=0.3)


@pytest.mark.parametrize("RC", [16, 32, 64])
def test_tc_product_rand70(msd, RC):
    cl = rand70()
    R = 64
    x = rand_x(cl.ntot, R, seed=RC)
    ref = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N) @ x.astype(np.complex128)
    pb = msd.Problem(cl)
    pb.set_tile(R, msd.MSD_FP32, 0, RC)
    info, _ = pb.plan_info(R, msd.MSD_FP32)
    assert info["RT"] == RC and info["KB"] == 0
    y = pb.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP32).cpu().numpy()
    assert relerr(y, ref) < 1e-5


def test_tc_product_batched_and_recomputed(msd):
    cls = [W.small_mixed(seed=3, M=6, N=10, k=2.0), rand70(), W.four_disks(),
           W.random_cluster(seed=9, M=40, half_side=12.0, rmin=0.6, rmax=1.0, gap=0.2, k=3.0, N=20)]
    R = 16
    ps = msd.Problem(cls)
    x = rand_x(ps.ntot, R, seed=4)
    xd = torch.from_numpy(x).cuda()
    ps.set_tile(R, msd.MSD_FP32, 0, 16)
    ys = ps.matvec(xd, msd.MSD_FP32).cpu().numpy()
    pr = msd.Problem(cls)
    pr.set_tile(R, msd.MSD_FP32, 0, 16)
    pr.set_generator_mode(msd.MSD_GEN_RECOMPUTE, 20_000)  # packed and split chunks
    yr = pr.matvec(xd, msd.MSD_FP32).cpu().numpy()
    off = 0
    for cl in cls:
        A = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
        ref = A @ x[off:off + cl.ntot].astype(np.complex128)
        assert relerr(ys[off:off + cl.ntot], ref) < 1e-5, cl.name
        assert relerr(yr[off:off + cl.ntot], ref) < 1e-5, cl.name
        off += cl.ntot


def test_tc_mixed_solve(msd):
    cl = rand70()
    betas = W.angles(16)
    pb = msd.Problem(cl)
    pb.set_tile(16, msd.MSD_FP32, 0, 16)
    res = pb.solve(betas, tol=1e-12, precision=msd.MSD_MIXED)
    assert (res.flags == 0).all(), res.relres
    rho_ref, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas)
    assert relerr(res.rho.cpu().numpy(), rho_ref) < 1e-9


def test_tc_autotuner_candidates(msd):
    """R = 32 FP32: the tuner times the CUDA-core shapes and the two
    tensor-core shapes (TC = 16, 32) and keeps the fastest."""
    cl = rand70()
    pb = msd.Problem(cl)
    info, ms = pb.plan_info(32, msd.MSD_FP32)
    assert info["candidates"] >= 3 and ms > 0
    x = rand_x(cl.ntot, 32, seed=1)
    ref = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N) @ x.astype(np.complex128)
    y = pb.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP32).cpu().numpy()
    assert relerr(y, ref) < 1e-5


# ---------------------------------------------------------------- shift-GEMM kernel
# KB = 0, RT = 8 pins the shift-GEMM tensor-core kernel (generators streamed
# in their A-operand order, the sources as a slab, one GEMM per shift d = n - m).

@pytest.mark.parametrize("R", [8, 24, 64])
@pytest.mark.parametrize("KB", [0, 1])
def test_shift_gemm_product_rand70(msd, R, KB):
    """rand70 (n = 25: mode blocks of <= 8 grouped two per CTA (KB = 0), or
    blocks of <= 16 one per CTA (KB = 1); M = 70 (one target tile, ragged at
    70; 9 K-steps of 8 sources, ragged at 70; three folds of the
    accumulators), mixed Dirichlet/Neumann."""
    cl = rand70()
    x = rand_x(cl.ntot, R, seed=R)
    ref = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N) @ x.astype(np.complex128)
    pb = msd.Problem(cl)
    pb.set_tile(R, msd.MSD_FP32, KB, 8)
    info, _ = pb.plan_info(R, msd.MSD_FP32)
    assert info["RT"] == 8 and info["KB"] == KB
    y = pb.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP32).cpu().numpy()
    assert relerr(y, ref) < 1e-5


def test_shift_gemm_product_batched_and_two_target_tiles(msd):
    """Batched configurations of different N (n = 3 .. 41) and sizes, one of
    them with 150 disks (two target tiles of 128), 16 columns (two column
    tiles); then a geometry update (generators rebuilt) and a second product."""
    cls = [W.small_mixed(seed=3, M=6, N=10, k=2.0), rand70(), W.four_disks(),
           W.random_cluster(seed=9, M=40, half_side=12.0, rmin=0.6, rmax=1.0, gap=0.2, k=3.0, N=20),
           W.random_cluster(seed=10, M=150, half_side=24.0, rmin=0.4, rmax=0.7, gap=0.2, k=1.5, N=1,
                            neumann_fraction=0.5)]
    R = 16
    pb = msd.Problem(cls)
    pb.set_tile(R, msd.MSD_FP32, 0, 8)
    pw = msd.Problem(cls)
    pw.set_tile(R, msd.MSD_FP32, 1, 8)
    for it in range(2):
        x = rand_x(pb.ntot, R, seed=11 + it)
        y = pb.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP32).cpu().numpy()
        yw = pw.matvec(torch.from_numpy(x).cuda(), msd.MSD_FP32).cpu().numpy()
        off = 0
        for cl in cls:
            A = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
            ref = A @ x[off:off + cl.ntot].astype(np.complex128)
            assert relerr(y[off:off + cl.ntot], ref) < 1e-5, (it, cl.name)
            assert relerr(yw[off:off + cl.ntot], ref) < 1e-5, (it, cl.name, "wide")
            off += cl.ntot
        if it == 0:  # move every disk by the same small offset and rebuild
            for cl in cls:
                cl.centres = cl.centres + np.array([0.05, -0.03])
            cen = np.concatenate([cl.centres for cl in cls])
            pb.update_geometry(centres=cen)
            pw.update_geometry(centres=cen)


def test_shift_gemm_mixed_solve_and_adjoint_fallback(msd):
    """A mixed-precision solve whose FP32 products run on the shift-GEMM
    kernel, and an adjoint (gradient) solve on the same problem, which uses a
    plan without it."""
    cl = rand70()
    betas = W.angles(16)
    pb = msd.Problem(cl)
    pb.set_tile(16, msd.MSD_FP32, 0, 8)
    res = pb.solve(betas, tol=1e-12, precision=msd.MSD_MIXED)
    assert (res.flags == 0).all(), res.relres
    rho_ref, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas)
    assert relerr(res.rho.cpu().numpy(), rho_ref) < 1e-9
    th = W.angles(12)
    J, dO, da, dk = pb.grad_farfield_misfit(betas, th, np.zeros((1, 12, 16), np.complex128), tol=1e-12,
                                            precision=msd.MSD_MIXED)
    J64, dO64, _, _ = pb.grad_farfield_misfit(betas, th, np.zeros((1, 12, 16), np.complex128), tol=1e-12,
                                              precision=msd.MSD_FP64)
    assert abs(J[0] - J64[0]) <= 1e-9 * J64[0]
    assert np.abs(dO - dO64).max() <= 1e-7 * np.abs(dO64).max()


# ---------------------------------------------------------------- converged systems skipped

@pytest.mark.parametrize("precision,KB,RT", [("mixed", 0, 8), ("mixed", 0, 16), ("mixed", 6, 8), ("fp64", None, None)])
def test_converged_configurations_skipped_by_products(msd, precision, KB, RT):
    """Two configurations of very different difficulty in one batched solve:
    four disks converge in a few steps, rand70 needs many more.  After the
    four-disk systems converge, the products of the later Arnoldi steps skip
    their tiles (no active column) and write zero sums there; the solutions of
    both configurations must still equal the oracle's direct solve.  Covers
    the shift-GEMM (KB 0, RT 8), expanded-Toeplitz tensor-core (KB 0, RT 16),
    CUDA-core FP32 and FP64 product kernels."""
    cls = [W.four_disks(), rand70()]
    R = 16
    pb = msd.Problem(cls)
    prec = msd.MSD_MIXED if precision == "mixed" else msd.MSD_FP64
    if KB is not None:
        pb.set_tile(R, msd.MSD_FP32, KB, RT)
    betas = np.stack([W.angles(R), W.angles(R) + 0.05])
    res = pb.solve(betas, tol=1e-12, precision=prec, restart=200)
    assert (res.flags == 0).all(), res.relres
    it = np.asarray(res.iters).reshape(2, R)
    assert it[0].max() < it[1].min(), it          # the skip happened
    rho = res.rho.cpu().numpy()
    for c, cl in enumerate(cls):
        o0 = pb.row_offset(c)
        ref, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas[c], method="lu")
        assert relerr(rho[o0:o0 + cl.ntot], ref) < 1e-9, (c, relerr(rho[o0:o0 + cl.ntot], ref))
    pb.close()
