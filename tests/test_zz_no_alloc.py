"""The allocation-free product (msd_matvec_noalloc) against the regular one.

msd_matvec_noalloc serves callers that may not allocate device memory when
they call the library -- a process that reserves all of its device memory at
start-up, or a latency-critical path that cannot afford the device-wide
synchronisation of cudaMalloc.  It keeps its work area in one fixed device
array shared by every call, so the test calls it twice in a row on
different inputs (the second call must not see the first call's leftovers)
and compares each result with msd_matvec on the same input and with the
oracle's preconditioned operator P^-1 A (section 5) applied on the CPU,
within the tolerances of the other product tests (1e-11 FP64, 1e-5 FP32
relative).

The file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.fixture(scope="module")
def msd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_8186_gb300 import msd as m
    return m


@pytest.mark.parametrize("precision,R,tol", [(0, 1, 1e-11), (0, 3, 1e-11), (2, 1, 1e-5), (2, 8, 1e-5)])
def test_noalloc_product_matches_regular_product(msd, precision, R, tol):
    cl = W.random_cluster(seed=8, M=70, half_side=14.0, rmin=0.5, rmax=1.0, gap=0.2, k=2.5, N=12,
                          neumann_fraction=0.3)
    pb = msd.Problem(cl)
    A = O_.preconditioned_dense(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
    dtype = torch.complex128 if precision == msd.MSD_FP64 else torch.complex64
    g = torch.Generator(device="cpu").manual_seed(1234 + R)
    for call in range(2):
        x = torch.randn(cl.ntot, R, dtype=dtype, generator=g).cuda()
        y_ref = torch.empty_like(x)
        msd.msd_matvec(pb.handle, R, precision, x, y_ref)          # also builds the generators
        y = torch.full_like(x, float("nan"))
        msd.msd_matvec_noalloc(pb.handle, R, precision, x, y)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all(), call
        assert _relerr(y, y_ref) < tol, (call, _relerr(y, y_ref))
        y_or = torch.from_numpy(A @ x.cpu().to(torch.complex128).numpy())
        assert _relerr(y.cpu().to(torch.complex128), y_or) < tol, (call, _relerr(y.cpu().to(torch.complex128), y_or))
    pb.close()


def test_noalloc_rejects_work_area_overflow_and_missing_generators(msd):
    cl = W.four_disks()
    pb = msd.Problem(cl)
    x = torch.zeros(cl.ntot, 1, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(msd.MsdError) as e:          # no FP64 generators built yet
        msd.msd_matvec_noalloc(pb.handle, 1, msd.MSD_FP64, x, y)
    assert e.value.status == -1
    msd.msd_matvec(pb.handle, 1, msd.MSD_FP64, x, y)
    R = (33 << 20) // (2 * 16 * cl.ntot) + 1       # 2 * N_tot * R complex128 values > 32 MiB
    xb = torch.zeros(cl.ntot, R, dtype=torch.complex128, device="cuda")
    yb = torch.empty_like(xb)
    with pytest.raises(msd.MsdError) as e:
        msd.msd_matvec_noalloc(pb.handle, R, msd.MSD_FP64, xb, yb)
    assert e.value.status == -1
    # y starting one row after x: the byte ranges overlap partially
    buf = torch.zeros(cl.ntot + 1, 1, dtype=torch.complex128, device="cuda")
    with pytest.raises(msd.MsdError) as e:
        msd.msd_matvec_noalloc(pb.handle, 1, msd.MSD_FP64, buf[:-1], buf[1:])
    assert e.value.status == -1
    with pytest.raises(msd.MsdError) as e:
        msd.msd_matvec(pb.handle, 1, msd.MSD_FP64, buf[1:], buf[:-1])
    assert e.value.status == -1
    pb.close()
