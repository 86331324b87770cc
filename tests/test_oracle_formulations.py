"""Pins of the oracle's double-layer blocks M, D, its far field and potential,
and of the integral-equation formulations built from I, L, M, N, D
(section 3 equations, section 4.2 blocks, section 5 combinations).

* Off-diagonal M and D blocks against trapezoidal quadrature of the
  Galerkin double integrals with the kernels -d_ny G and -d_nx d_ny G
  (1e-12).
* Jump relations (Prop. 3.2): on every circle the exterior trace of the
  double-layer potential of Prop. 4.3 projects onto (-I/2 + M) lambda and its
  exterior normal derivative onto D lambda; the single-layer potential's
  normal derivative onto (-I/2 + N) rho.  The potential and its gradient are
  summed term by term from the Hankel expansions, independent of the
  addition theorem behind the blocks (1e-11).
* The double-layer far field is the large-r limit of the double-layer
  potential (this fixes the sign of a_M).
* EFIE, MFIE, CFIE and Brakhage-Werner formulations of one mixed cluster
  give the same far field (1e-9), and for one disk the textbook Mie series.
* At k a = j_{0,1} (an interior Dirichlet resonance of one disk) the EFIE
  matrix is singular while CFIE and BWIE solve, with the Mie far field.
* Planted mistakes (the printed sign of a_M, the printed sign of the D
  diagonal, +I/2 on the diagonal of M) fail these pins.
"""
import numpy as np
import pytest
from scipy import special

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

D_, N_ = W.DIRICHLET, W.NEUMANN


def circle(Oc, a, Q):
    t = 2 * np.pi * np.arange(Q) / Q
    return t, Oc[None, :] + a * np.stack([np.cos(t), np.sin(t)], axis=1)


def quad_block(Op, ap, Oq, aq, k, N, kind, Q=160):
    """(K Phi^q_n, Phi^p_m) by the trapezoidal rule on both circles, for the
    kernels of M (-d_ny G) and D (-d_nx d_ny G), G = (i/4) H_0(k|x - y|)."""
    tp, X = circle(Op, ap, Q)
    tq, Y = circle(Oq, aq, Q)
    d = X[:, None, :] - Y[None, :, :]
    r = np.hypot(d[..., 0], d[..., 1])
    nx = np.stack([np.cos(tp), np.sin(tp)], axis=1)[:, None, :]
    ny = np.stack([np.cos(tq), np.sin(tq)], axis=1)[None, :, :]
    dnx, dny = (d * nx).sum(-1), (d * ny).sum(-1)
    H0, H1 = special.hankel1(0, k * r), special.hankel1(1, k * r)
    dG_dny = 0.25j * k * H1 * dny / r  # d/dn_y of (i/4) H_0(k r)
    if kind == "M":
        K = -dG_dny
    else:  # d/dn_x of dG_dny
        K = -0.25j * k * ((k * H0 / r - 2 * H1 / r ** 2) * dnx * dny / r + H1 * (nx * ny).sum(-1) / r)
    m = np.arange(-N, N + 1)
    phq = np.exp(1j * np.outer(tq, m)) / np.sqrt(2 * np.pi * aq) * (aq * 2 * np.pi / Q)
    php = np.exp(1j * np.outer(tp, m)) / np.sqrt(2 * np.pi * ap) * (ap * 2 * np.pi / Q)
    return php.conj().T @ K @ phq


def two_disks():
    return W.Cluster(np.array([[0.3, -0.2], [-1.9, 1.1]]), np.array([0.7, 0.9]),
                     np.array([0, 1], np.int8), 1.3, 6, "two")


@pytest.mark.parametrize("kind", ["M", "D"])
def test_offdiagonal_M_D_blocks_vs_quadrature(kind):
    cl = two_disks()
    O, a, k, N = cl.centres, cl.radii, cl.k, cl.N
    for p, q in [(0, 1), (1, 0)]:
        ref = quad_block(O[p], a[p], O[q], a[q], k, N, kind)
        blk = O_.block_of(kind, O, a, k, N, p, q)
        assert np.abs(blk - ref).max() <= 1e-12 * np.abs(ref).max()


def field_and_gradient(O, a, k, N, coef_rows, x):
    """u(x) = sum_p sum_m c^p_m H_m(k r_p) e^{i m theta_p} and its gradient,
    term by term (c [M, n])."""
    m = O_.modes(N)
    u = np.zeros(len(x), complex)
    g = np.zeros((len(x), 2), complex)
    for p in range(len(a)):
        d = x - O[p][None, :]
        r = np.hypot(d[:, 0], d[:, 1])
        th = np.arctan2(d[:, 1], d[:, 0])
        rh = d / r[:, None]
        tt = np.stack([-rh[:, 1], rh[:, 0]], axis=1)
        H = special.hankel1(m[None, :], k * r[:, None])
        dH = special.h1vp(m[None, :], k * r[:, None])
        E = np.exp(1j * m[None, :] * th[:, None])
        u += (H * E) @ coef_rows[p]
        gr = (k * dH * E) @ coef_rows[p]
        gt = ((1j * m[None, :] / r[:, None]) * H * E) @ coef_rows[p]
        g += gr[:, None] * rh + gt[:, None] * tt
    return u, g


def project(values, a, N, t):
    m = np.arange(-N, N + 1)
    Q = len(t)
    return np.exp(-1j * np.outer(m, t)) @ values * (a * 2 * np.pi / Q) / np.sqrt(2 * np.pi * a)


def test_jump_relations_of_the_blocks():
    cl = W.small_mixed(seed=7, M=4, N=9, k=1.9)
    O, a, k, N = cl.centres, cl.radii, cl.k, cl.N
    M, n = cl.M, cl.n
    rng = np.random.default_rng(2)
    lam = rng.standard_normal(M * n) + 1j * rng.standard_normal(M * n)
    J, dJ, _, _ = O_.bessel_diagonals(a, k, N)
    c_dl = (-0.5j * np.pi * k * a[:, None] * dJ / np.sqrt(2 * np.pi * a[:, None])) * lam.reshape(M, n)
    c_sl = (0.5j * np.pi * a[:, None] * J / np.sqrt(2 * np.pi * a[:, None])) * lam.reshape(M, n)
    allM = np.block([[O_.block_of("M", O, a, k, N, p, q) for q in range(M)] for p in range(M)])
    allD = np.block([[O_.block_of("D", O, a, k, N, p, q) for q in range(M)] for p in range(M)])
    allN = np.block([[O_.block_of("N", O, a, k, N, p, q) for q in range(M)] for p in range(M)])
    tr_M = (-0.5 * lam + allM @ lam).reshape(M, n)
    dn_M = (allD @ lam).reshape(M, n)
    dn_L = (-0.5 * lam + allN @ lam).reshape(M, n)
    Q = 256
    for p in range(M):
        t, x = circle(O[p], a[p] * (1 + 1e-13), Q)
        nrm = np.stack([np.cos(t), np.sin(t)], axis=1)
        u, g = field_and_gradient(O, a, k, N, c_dl, x)
        assert np.abs(project(u, a[p], N, t) - tr_M[p]).max() <= 1e-11 * np.abs(tr_M).max()
        assert np.abs(project((g * nrm).sum(1), a[p], N, t) - dn_M[p]).max() <= 1e-11 * np.abs(dn_M).max()
        u, g = field_and_gradient(O, a, k, N, c_sl, x)
        assert np.abs(project((g * nrm).sum(1), a[p], N, t) - dn_L[p]).max() <= 1e-11 * np.abs(dn_L).max()


def test_printed_diagonal_forms_agree():
    """The two printed diagonal forms of M^pp and N^pp (Wronskian)."""
    a, k, N = np.array([0.8]), 2.7, 12
    J, dJ, H, dH = O_.bessel_diagonals(a, k, N)
    c = 0.5j * np.pi * k * a[0]
    assert np.abs((-0.5 - c * J[0] * dH[0]) - (0.5 - c * dJ[0] * H[0])).max() < 1e-13
    assert np.abs((0.5 + c * J[0] * dH[0]) - (-0.5 + c * dJ[0] * H[0])).max() < 1e-13


def dl_farfield_limit(cl, lam, th, far):
    def scaled(r):
        pts = r * np.stack([np.cos(th), np.sin(th)], 1)
        return O_.double_layer_potential(cl.centres, cl.radii, cl.k, cl.N, lam, pts) * np.exp(-1j * cl.k * r) * np.sqrt(r)
    r = 2.0e6
    est = 2 * scaled(2 * r) - scaled(r)
    return np.abs(est - far).max() / np.abs(far).max()


def test_double_layer_farfield_is_large_r_limit():
    cl = W.small_mixed(seed=5, M=4, N=12, k=1.7)
    rng = np.random.default_rng(4)
    lam = rng.standard_normal(cl.ntot) + 1j * rng.standard_normal(cl.ntot)
    th = np.linspace(0, 2 * np.pi, 9, endpoint=False)
    F = O_.farfield_formulation(cl.centres, cl.radii, cl.k, cl.N, lam, th, {"M": 1.0})[:, 0]
    assert dl_farfield_limit(cl, lam, th, F) <= 1e-6
    # planted mistake: the printed sign
    assert dl_farfield_limit(cl, lam, th, -F) > 1.0


# Formulations of the Dirichlet problem (section 3) and their Neumann rows
def efie():
    return ({D_: {"L": 1}, N_: {"I": -0.5, "N": 1}}, {D_: {"U": 1}, N_: {"dU": 1}}, {"L": 1})


def mfie():
    return ({D_: {"I": 0.5, "N": 1}, N_: {"I": -0.5, "N": 1}}, {D_: {"dU": 1}, N_: {"dU": 1}}, {"L": 1})


def cfie(alpha, eta):
    return ({D_: {"L": alpha * eta, "I": 0.5 * (1 - alpha), "N": 1 - alpha}, N_: {"I": -0.5, "N": 1}},
            {D_: {"U": alpha * eta, "dU": 1 - alpha}, N_: {"dU": 1}}, {"L": 1})


def bwie(eta):
    """u = -(eta L + M) psi: Dirichlet rows (I/2 - eta L - M) psi = -U,
    Neumann rows (eta I/2 - eta N - D) psi = -dU."""
    return ({D_: {"I": 0.5, "L": -eta, "M": -1}, N_: {"I": 0.5 * eta, "N": -eta, "D": -1}},
            {D_: {"U": 1}, N_: {"dU": 1}}, {"L": -eta, "M": -1})


def far(cl, form, betas, th):
    ow, rw, rep = form
    dens = O_.solve_formulation(cl.centres, cl.radii, cl.bc, cl.k, cl.N, betas, ow, rw)
    return O_.farfield_formulation(cl.centres, cl.radii, cl.k, cl.N, dens, th, rep)


def test_formulations_give_the_same_far_field():
    cl = W.small_mixed(seed=3, M=5, N=24, k=2.0)
    th = W.angles(36)
    betas = [0.3, 2.0]
    ref = far(cl, efie(), betas, th)
    k = cl.k
    for form in (cfie(0.5, 1j * k), bwie(1j * k), bwie(-2.0j)):
        F = far(cl, form, betas, th)
        assert np.abs(F - ref).max() <= 1e-9 * np.abs(ref).max()
    cl.bc[:] = D_
    ref = far(cl, efie(), betas, th)
    F = far(cl, mfie(), betas, th)
    assert np.abs(F - ref).max() <= 1e-9 * np.abs(ref).max()


def mie_far(k, a, beta, th, hard=False, terms=40):
    m = np.arange(-terms, terms + 1)
    c = special.jvp(m, k * a) / special.h1vp(m, k * a) if hard else special.jv(m, k * a) / special.hankel1(m, k * a)
    return -np.exp(-1j * np.pi / 4) * np.sqrt(2 / (np.pi * k)) * (np.exp(1j * np.outer(th - beta, m)) @ c)


def test_resonance_efie_singular_cfie_bwie_solve():
    """One sound-soft disk with k a = j_{0,1}: the m = 0 EFIE entry vanishes;
    CFIE and BWIE give the Mie far field."""
    a = 1.0
    k = special.jn_zeros(0, 1)[0] / a
    cl = W.Cluster(np.array([[0.4, -0.3]]), np.array([a]), np.array([D_], np.int8), k, 14)
    A = O_.assemble_formulation(cl.centres, cl.radii, cl.bc, k, cl.N, efie()[0])
    assert np.abs(np.diag(A)).min() < 1e-15
    th = W.angles(24)
    beta = 0.9
    shift = np.exp(-1j * k * (np.cos(th) * 0.4 + np.sin(th) * (-0.3))) * \
        np.exp(1j * k * (np.cos(beta) * 0.4 + np.sin(beta) * (-0.3)))
    ref = shift * mie_far(k, a, beta, th)
    for form in (cfie(0.5, 1j * k), bwie(1j * k)):
        A = O_.assemble_formulation(cl.centres, cl.radii, cl.bc, k, cl.N, form[0])
        assert np.linalg.cond(A) < 10
        F = far(cl, form, [beta], th)[:, 0]
        assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()


def test_planted_M_diagonal_sign_is_caught(monkeypatch):
    cl = W.small_mixed(seed=3, M=5, N=24, k=2.0)
    th = W.angles(36)
    ref = far(cl, efie(), [0.3], th)
    orig = O_.block_M

    def bad(O, a, k, N, p, q):
        B = orig(O, a, k, N, p, q)
        return B + np.eye(2 * N + 1) if p == q else B
    monkeypatch.setattr(O_, "block_M", bad)
    F = far(cl, bwie(2.0j), [0.3], th)
    assert np.abs(F - ref).max() > 1e-3 * np.abs(ref).max()


def test_printed_D_diagonal_sign_is_caught(monkeypatch):
    """With the printed sign of the D diagonal, the Brakhage-Werner rows of
    the sound-hard disks no longer reproduce the far field."""
    cl = W.small_mixed(seed=3, M=5, N=24, k=2.0)
    assert (cl.bc == N_).any()
    th = W.angles(36)
    ref = far(cl, efie(), [0.3], th)
    orig = O_.block_D

    def printed(O, a, k, N, p, q):
        B = orig(O, a, k, N, p, q)
        return -B if p == q else B
    monkeypatch.setattr(O_, "block_D", printed)
    F = far(cl, bwie(1j * cl.k), [0.3], th)
    assert np.abs(F - ref).max() > 1e-3 * np.abs(ref).max()
