"""Time reversal (section 7, DORT) through the C-ABI: far-field matrix F,
T = conj(F)^T F and its eigenvalues against the oracle.

Tolerances.  F comes from a solve to relres 1e-12 (oracle: LU), so F and T
agree to ~1e-11 of their largest entry; an eigenvalue moves by at most
||T_gpu - T_oracle||_2, and Householder plus bisection add a few n eps ||T||:
1e-9 of the largest eigenvalue.  Invariants of the device's own output
(trace and Frobenius norm of T against the sum of the eigenvalues and of
their squares) hold to 1e-12 at any size.
"""
import numpy as np
import pytest
from scipy import special

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


def oracle_dort(cl, n):
    _, F = O_.dort_far_field_matrix(cl.centres, cl.radii, cl.bc, cl.k, cl.N, n)
    T = O_.time_reversal_matrix(F)
    return F, T, O_.dort_eigenvalues(T)


def check_invariants(eig, T):
    for c in range(eig.shape[0]):
        tr = np.trace(T[c]).real
        fro2 = (np.abs(T[c]) ** 2).sum()
        assert abs(eig[c].sum() - tr) <= 1e-12 * abs(tr)
        assert abs((eig[c] ** 2).sum() - fro2) <= 1e-12 * fro2
        assert np.all(np.diff(eig[c]) <= 0)  # largest first


@pytest.mark.parametrize("bc", [0, 1])
def test_single_disk_closed_form(msd, bc):
    """Circulant F: eigenvalues n^2 (2 / (pi k)) |c_m|^2 and zeros."""
    k, a, N, n = 3.1, 0.7, 12, 40
    cl = W.Cluster(np.zeros((1, 2)), np.array([a]), np.array([bc], np.int8), k, N)
    eig, F, T, st = msd.Problem(cl).dort(n)
    assert st == msd.MSD_OK
    m = np.arange(-N, N + 1)
    c = (special.jv(m, k * a) / special.hankel1(m, k * a) if bc == 0
         else special.jvp(m, k * a) / special.h1vp(m, k * a))
    ex = np.sort(np.concatenate([n * n * 2 / (np.pi * k) * np.abs(c) ** 2, np.zeros(n - len(m))]))[::-1]
    e = eig.cpu().numpy()[0]
    assert np.abs(e - ex).max() <= 1e-10 * ex[0]
    check_invariants(eig.cpu().numpy(), T.cpu().numpy())


@pytest.mark.parametrize("n", [1, 2, 3, 33, 64])
def test_parity_small_mixed(msd, n):
    cl = W.small_mixed(seed=3, M=6, N=10, k=2.0)
    eig, F, T, st = msd.Problem(cl).dort(n)
    assert st == msd.MSD_OK
    Fr, Tr, er = oracle_dort(cl, n)
    F, T, e = F.cpu().numpy()[0], T.cpu().numpy()[0], eig.cpu().numpy()[0]
    assert np.abs(F - Fr).max() <= 1e-10 * np.abs(Fr).max()
    assert np.abs(T - Tr).max() <= 1e-10 * np.abs(Tr).max()
    assert np.abs(e - er).max() <= 1e-9 * er[0]
    assert np.abs(F - F.T).max() <= 1e-10 * np.abs(F).max()  # reciprocity
    check_invariants(eig.cpu().numpy(), T[None])


def test_three_small_disks_two_configurations(msd):
    """The example's three small disks, sound-soft and sound-hard, as two
    configurations of one problem, mirror of 512 angles: 3 and 9
    significant eigenvalues, values equal to the oracle's."""
    cs = [W.dort_three_disks(0), W.dort_three_disks(1)]
    n = 512
    eig, F, T, st = msd.Problem(cs).dort(n)
    assert st == msd.MSD_OK
    e = eig.cpu().numpy()
    for c, (cl, count) in enumerate(zip(cs, (3, 9))):
        _, _, er = oracle_dort(cl, n)
        assert np.abs(e[c] - er).max() <= 1e-9 * er[0]
        assert e[c][count] < e[c][count - 1] / 500
    check_invariants(e, T.cpu().numpy())


def test_host_buffers_match_device(msd):
    cl = W.small_mixed(seed=5, M=5, N=9, k=1.7)
    n = 21
    pb = msd.Problem(cl)
    eig, F, T, _ = pb.dort(n)
    e_h = np.zeros((1, n))
    F_h = np.zeros((1, n, n), np.complex128)
    o = msd.msd_opts(1e-12, 0, 3000, 0, 0.0, msd.MSD_FP64, msd.MSD_GEN_AUTO)  # as Problem.dort
    st = msd.msd_dort(pb.handle, n, o, F_h, None, e_h)
    assert st == msd.MSD_OK
    # a second solve (tuned product plan) may differ in the last bits
    e_d, F_d = eig.cpu().numpy(), F.cpu().numpy()
    assert np.abs(e_h - e_d).max() <= 1e-12 * e_d.max()
    assert np.abs(F_h - F_d).max() <= 1e-12 * np.abs(F_d).max()


@pytest.mark.parametrize("n", [1100, 1601])
def test_large_mirror(msd, n):
    """Mirrors beyond one CTA's worth of rows (1601: the update kernel's
    shared memory above 48 KB); four disks, 100 unknowns."""
    cl = W.four_disks()
    eig, F, T, st = msd.Problem(cl).dort(n, want_F=False)
    assert st == msd.MSD_OK
    e = eig.cpu().numpy()
    _, Tr, er = oracle_dort(cl, n)
    assert np.abs(e[0] - er).max() <= 1e-9 * er[0]
    check_invariants(e, T.cpu().numpy())


def test_bad_arguments(msd):
    pb = msd.Problem(W.four_disks())
    e = np.zeros(4)
    for n in (0, msd.MSD_MAX_DORT + 1):
        with pytest.raises(msd.MsdError):
            msd.msd_dort(pb.handle, n, None, None, None, e)


def test_eigen_of_supplied_far_field_matrices(msd):
    """msd_dort_eigen on caller matrices (two configurations): a random
    complex F, a rank-3 F, a unitary F (T = 4 I: every column already
    reduced, eigenvalue of multiplicity n) and a diagonal F (T diagonal)."""
    rng = np.random.default_rng(17)
    pb = msd.Problem([W.four_disks(), W.four_disks()])
    for n in (7, 130, 517):
        G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        Q, _ = np.linalg.qr(G)
        cases = [
            (G, rng.standard_normal((n, 3)) @ rng.standard_normal((3, n)) + 0j),
            (2.0 * Q, np.diag(rng.uniform(0.5, 2.0, n) * np.exp(1j * rng.uniform(0, 6, n)))),
        ]
        for F0, F1 in cases:
            F = np.ascontiguousarray(np.stack([F0, F1]))
            eig, T = pb.dort_eigen(torch.from_numpy(F).cuda(), want_T=True)
            e, Tg = eig.cpu().numpy(), T.cpu().numpy()
            for c in range(2):
                Tr = O_.time_reversal_matrix(F[c])
                er = O_.dort_eigenvalues(Tr)
                assert np.abs(Tg[c] - Tr).max() <= 1e-13 * np.abs(Tr).max()
                assert np.abs(e[c] - er).max() <= 1e-12 * er[0], (n, c)
            check_invariants(e, Tg)
            # host input and output buffers
            e_h = np.zeros((2, n))
            msd.msd_dort_eigen(pb.handle, n, F, None, e_h)
            assert np.array_equal(e_h, e)


# ---------------------------------------------------------------- eigenvectors and Herglotz waves

@pytest.mark.parametrize("n,K", [(3, 3), (7, 4), (130, 6), (517, 5)])
def test_eigenvectors_of_supplied_matrices(msd, n, K):
    """msd_dort_eigenvectors on random far-field matrices (two configurations):
    residual ||T u - lambda u|| <= 1e-10 ||T||, orthonormality 1e-12, and
    agreement up to phase with LAPACK's eigenvectors of the oracle's T
    (|<u, u_ref>| >= 1 - 1e-10; the random spectra are simple)."""
    rng = np.random.default_rng(n)
    F = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    pb = msd.Problem([W.four_disks(), W.four_disks()])
    eig, vec = pb.dort_eigenvectors(torch.from_numpy(F).cuda(), K)
    eig, vec = eig.cpu().numpy(), vec.cpu().numpy()
    for c in range(2):
        T = O_.time_reversal_matrix(F[c])
        lam, V = O_.dort_eigenvectors(T)
        nT = np.linalg.norm(T, 2)
        assert np.abs(eig[c] - lam).max() <= 1e-12 * lam[0]
        U = vec[c].T
        assert np.abs(U.conj().T @ U - np.eye(K)).max() <= 1e-12
        for i in range(K):
            assert np.linalg.norm(T @ U[:, i] - eig[c, i] * U[:, i]) <= 1e-10 * nT, (c, i)
            assert abs(np.vdot(V[:, i], U[:, i])) >= 1 - 1e-10, (c, i)
            j = np.abs(U[:, i]).argmax()
            assert abs(U[j, i].imag) <= 1e-14 and U[j, i].real > 0
    pb.close()


def test_selective_focusing_on_the_three_disks(msd):
    """Section 7 on the GPU: far-field matrix (msd_dort, 512 angles) of the
    three small sound-soft disks, eigenvectors of its three significant
    eigenvalues (msd_dort_eigenvectors) and their Herglotz waves
    (msd_herglotz_wave) on a grid: each wave peaks within a tenth of a
    wavelength of one obstacle, a different one for each, and stays below
    30 % of its peak on the other two; the waves match the oracle's Herglotz
    formula on the same parameters (1e-12) and the eigenvectors match the
    oracle's (LU solve, LAPACK) up to phase."""
    cl = W.dort_three_disks(0)
    n = 512
    pb = msd.Problem(cl)
    _, F, _, st = pb.dort(n, want_T=False)
    assert st == msd.MSD_OK
    eig, vec = pb.dort_eigenvectors(F, 3)
    vec = vec.cpu().numpy()[0]
    alphas, F_ref = O_.dort_far_field_matrix(cl.centres, cl.radii, cl.bc, cl.k, cl.N, n)
    lam, V = O_.dort_eigenvectors(O_.time_reversal_matrix(F_ref))
    for i in range(3):
        assert abs(np.vdot(V[:, i], vec[i])) >= 1 - 1e-8, i
    g = np.linspace(-25, 25, 201)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    u = pb.herglotz_wave(vec, pts).cpu().numpy()
    wavelength = 2 * np.pi / cl.k
    for e in range(3):
        ref = O_.herglotz_wave(cl.k, alphas, vec[e], pts[::97])
        assert np.abs(u[::97, e] - ref).max() <= 1e-12 * np.abs(ref).max()
        ue = np.abs(u[:, e])
        peak = pts[ue.argmax()]
        d = np.hypot(cl.centres[:, 0] - peak[0], cl.centres[:, 1] - peak[1])
        assert d.argmin() == e and d.min() <= 0.1 * wavelength, (e, peak)
        at = np.abs(pb.herglotz_wave(vec[e:e + 1], cl.centres).cpu().numpy()[:, 0])
        assert np.delete(at, e).max() < 0.3 * ue.max(), (e, at / ue.max())
    pb.close()
