"""Pins of the oracle's time-reversal (DORT) functions of section 7 by
quantities they do not use.

* One disk at the origin: the far-field matrix is circulant, so the
  eigenvalues of T = conj(F)^T F are n_alpha^2 |K c_m|^2 (|m| <= N) and zeros,
  with the textbook single-disk series c_m = J_m(ka)/H_m(ka) (sound-soft) or
  J_m'(ka)/H_m'(ka) (sound-hard) and |K|^2 = 2/(pi k): 1e-12 of the largest.
* Reciprocity: with the far field measured opposite to each emitting
  direction, F(alpha_i + pi; alpha_j) = F(alpha_j + pi; alpha_i), so F is
  complex symmetric (mixed boundary conditions, several N).
* The three small disks of the time-reversal example: three significant
  eigenvalues for sound-soft disks (one monopole each) and nine for
  sound-hard disks (monopole and two dipoles each), each within 5 % of its
  isolated-disk value once the mirror resolves the configuration
  (n_alpha = 512), with a gap of more than 500 to the rest.
* T is Hermitian positive semi-definite and its eigenvalues are the squared
  singular values of F.
* The Herglotz waves of the three significant eigenvectors of the example
  focus each on one obstacle (selective focusing).
* Planted mistakes (far field measured in the emitting direction, T without
  the conjugate, the conjugate Herglotz parameter) fail these pins.
"""
import numpy as np
from scipy import special

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W


def single_disk_expected(k, a, N, bc, na):
    m = np.arange(-N, N + 1)
    if bc == 0:
        c = special.jv(m, k * a) / special.hankel1(m, k * a)
    else:
        c = special.jvp(m, k * a) / special.h1vp(m, k * a)
    lam = na ** 2 * (2.0 / (np.pi * k)) * np.abs(c) ** 2
    return np.sort(np.concatenate([lam, np.zeros(na - len(m))]))[::-1]


def test_single_disk_closed_form():
    for bc in (0, 1):
        for (k, a, N, na) in ((3.1, 0.7, 12, 40), (1.2, 1.5, 9, 19)):
            _, F = O_.dort_far_field_matrix(np.zeros((1, 2)), np.array([a]), np.array([bc], np.int8), k, N, na)
            lam = O_.dort_eigenvalues(O_.time_reversal_matrix(F))
            ex = single_disk_expected(k, a, N, bc, na)
            assert np.abs(lam - ex).max() <= 1e-12 * ex[0], (bc, k)


def test_far_field_matrix_is_reciprocal():
    for N in (8, 14):
        cl = W.small_mixed(seed=3, M=6, N=N, k=2.0)
        _, F = O_.dort_far_field_matrix(cl.centres, cl.radii, cl.bc, cl.k, cl.N, 24)
        assert np.abs(F - F.T).max() <= 1e-12 * np.abs(F).max()


def test_planted_measurement_direction_breaks_reciprocity():
    cl = W.small_mixed(seed=3, M=6, N=10, k=2.0)
    alphas = W.angles(24)
    rho, _ = O_.solve(cl.centres, cl.radii, cl.bc, cl.k, cl.N, alphas)
    F = O_.farfield(cl.centres, cl.radii, cl.k, cl.N, rho, alphas)  # mistake: no + pi
    assert np.abs(F - F.T).max() > 1e-2 * np.abs(F).max()


def test_hermitian_psd_and_singular_values():
    cl = W.small_mixed(seed=5, M=5, N=9, k=1.7)
    _, F = O_.dort_far_field_matrix(cl.centres, cl.radii, cl.bc, cl.k, cl.N, 33)
    T = O_.time_reversal_matrix(F)
    lam = O_.dort_eigenvalues(T)
    assert np.abs(T - T.conj().T).max() <= 1e-13 * np.abs(T).max()
    assert lam[-1] >= -1e-12 * lam[0]
    sv = np.linalg.svd(F, compute_uv=False)
    assert np.abs(lam - sv ** 2).max() <= 1e-12 * lam[0]
    # planted mistake: no conjugate
    lam_bad = np.linalg.eigvals(F.T @ F)
    assert np.abs(np.sort(np.abs(lam_bad))[::-1] - lam).max() > 1e-3 * lam[0]


def isolated_values(cl, na):
    """Isolated-disk eigenvalues n^2 |K c_m|^2: m = 0 for sound-soft disks,
    m = 0, +-1 for sound-hard ones (the modes that survive for k a << 1)."""
    ka = cl.k * cl.radii
    K2 = na ** 2 * 2.0 / (np.pi * cl.k)
    if cl.bc[0] == 0:
        v = K2 * np.abs(special.jv(0, ka) / special.hankel1(0, ka)) ** 2
    else:
        v = np.concatenate([K2 * np.abs(special.jvp(m, ka) / special.h1vp(m, ka)) ** 2 for m in (0, 1, -1)])
    return np.sort(v)[::-1]


def test_three_small_disks_significant_eigenvalues():
    na = 512
    for bc, count in ((0, 3), (1, 9)):
        cl = W.dort_three_disks(bc)
        _, F = O_.dort_far_field_matrix(cl.centres, cl.radii, cl.bc, cl.k, cl.N, na)
        lam = O_.dort_eigenvalues(O_.time_reversal_matrix(F))
        ex = isolated_values(cl, na)
        assert len(ex) == count
        assert np.abs(lam[:count] / ex - 1).max() < 0.05, (bc, lam[:count] / ex)
        assert lam[count] < lam[count - 1] / 500, (bc, lam[count] / lam[count - 1])


def test_eigenvectors_focus_on_each_obstacle():
    """Section 7: the Herglotz wave of each of the three significant
    eigenvectors (three small sound-soft disks, 512 angles) peaks on one
    obstacle, a different one for each, largest eigenvalue on the largest
    disk, and stays below 30 % of its peak on the other two.  Planted
    mistake: the conjugate parameter focuses at -O_p, on no obstacle."""
    cl = W.dort_three_disks(0)
    n = 512
    alphas, F = O_.dort_far_field_matrix(cl.centres, cl.radii, cl.bc, cl.k, cl.N, n)
    lam, V = O_.dort_eigenvectors(O_.time_reversal_matrix(F))
    assert np.allclose(lam, O_.dort_eigenvalues(O_.time_reversal_matrix(F)), rtol=0, atol=1e-9 * lam[0])
    g = np.linspace(-25, 25, 201)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    wavelength = 2 * np.pi / cl.k
    for e in range(3):
        u = np.abs(O_.herglotz_wave(cl.k, alphas, V[:, e], pts))
        peak = pts[u.argmax()]
        d = np.hypot(cl.centres[:, 0] - peak[0], cl.centres[:, 1] - peak[1])
        assert d.argmin() == e and d.min() <= 0.1 * wavelength, (e, peak)
        at = np.abs(O_.herglotz_wave(cl.k, alphas, V[:, e], cl.centres))
        others = np.delete(at, e)
        assert others.max() < 0.3 * u.max(), (e, at / u.max())
        u_bad = np.abs(O_.herglotz_wave(cl.k, alphas, V[:, e].conj(), pts))
        bad = pts[u_bad.argmax()]
        assert np.hypot(cl.centres[:, 0] - bad[0], cl.centres[:, 1] - bad[1]).min() > 5 * wavelength
