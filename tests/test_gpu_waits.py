"""The error path of the bounded device waits, made to run by the library's
test hook (msd_test_expire_waits) without any GPU fault: a wait for a
condition that nothing fulfils runs out after ~10 us, the kernel records it,
finishes its own work and returns, the call reports MSD_ERR_CUDA, and the
next call (hook off) gives the right result.

Covered waits: the pipeline wait of the tensor-core product (inside a
mixed-precision solve with 16 columns on the tcgen05 kernel) and the grid
barrier of the time-reversal tridiagonalisation (msd_dort_eigen)."""
import numpy as np
import pytest

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def msd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_8186_gb300 import msd as m
    return m


def test_tensor_core_pipeline_wait_expiry(msd):
    cl = W.random_cluster(seed=3, M=20, half_side=9.0, rmin=0.6, rmax=1.0, gap=0.2, k=2.0, N=10)
    betas = W.angles(16)
    pb = msd.Problem(cl)
    pb.set_tile(16, msd.MSD_FP32, 0, 16)            # FP32 inner products on the tcgen05 kernel
    ref, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, method="lu")
    res = pb.solve(betas, tol=1e-10, precision=msd.MSD_MIXED)
    assert res.status == msd.MSD_OK
    try:
        msd.msd_test_expire_waits(True)
        with pytest.raises(msd.MsdError) as e:
            pb.solve(betas, tol=1e-10, precision=msd.MSD_MIXED)
        assert e.value.status == msd.MSD_ERR_CUDA, e.value
    finally:
        msd.msd_test_expire_waits(False)
    res = pb.solve(betas, tol=1e-10, precision=msd.MSD_MIXED)
    assert res.status == msd.MSD_OK
    rho = res.rho.cpu().numpy()
    assert np.abs(rho - ref).max() <= 1e-9 * np.abs(ref).max()
    pb.close()


def test_time_reversal_grid_barrier_expiry(msd):
    n = 130
    rng = np.random.default_rng(7)
    F = rng.standard_normal((1, n, n)) + 1j * rng.standard_normal((1, n, n))
    ref = O_.dort_eigenvalues(O_.time_reversal_matrix(F[0]))
    pb = msd.Problem(W.four_disks())
    Fd = torch.from_numpy(F).cuda()
    try:
        msd.msd_test_expire_waits(True)
        with pytest.raises(msd.MsdError) as e:
            pb.dort_eigen(Fd)
        assert e.value.status == msd.MSD_ERR_CUDA, e.value
    finally:
        msd.msd_test_expire_waits(False)
    eig = pb.dort_eigen(Fd)[0].cpu().numpy()[0]
    assert np.abs(eig - ref).max() <= 1e-12 * ref[0]
    pb.close()
