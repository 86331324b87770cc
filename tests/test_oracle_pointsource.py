"""Pins of the oracle's point-source right-hand side (the point-source
proposition of section 4.3) by quantities it does not use.

* Trace and normal-derivative trace coefficients against trapezoidal
  quadrature of u_inc = (i/4) H_0(k |x - s|) and of its normal derivative on
  every circle (smooth and periodic, so the quadrature converges
  exponentially): 1e-12.
* A planted mistake (the conjugate phase e^{+i m theta}) fails that pin.
* The whole oracle solve with a point source satisfies the sound-soft
  boundary condition u_scat + u_inc = 0 on every circle (truncation error).
"""
import numpy as np
from scipy import special

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W


def quadrature_coefficients(O, a, k, N, s, K=256):
    """U^p_m = <u_inc, Phi^p_m> and <d_n u_inc, Phi^p_m> on circle p by the
    trapezoidal rule, Phi^p_m = e^{i m theta} / sqrt(2 pi a_p)."""
    th = 2 * np.pi * np.arange(K) / K
    m = O_.modes(N)
    U, dU = [], []
    for p in range(len(a)):
        x = O[p][None, :] + a[p] * np.stack([np.cos(th), np.sin(th)], axis=1)
        d = x - s[None, :]
        r = np.hypot(d[:, 0], d[:, 1])
        u = 0.25j * special.hankel1(0, k * r)
        nrm = np.stack([np.cos(th), np.sin(th)], axis=1)
        du = 0.25j * (-k * special.hankel1(1, k * r)) * (d * nrm).sum(axis=1) / r
        w = a[p] * (2 * np.pi / K) / np.sqrt(2 * np.pi * a[p])
        E = np.exp(-1j * m[:, None] * th[None, :])
        U.append(E @ u * w)
        dU.append(E @ du * w)
    return np.array(U), np.array(dU)


def closed_form(cl, s, conj_phase=False):
    d = O_.pointsource_coefficients(cl.centres, cl.radii, cl.k, cl.N, s)
    if conj_phase:  # planted mistake
        dd = s[None, :] - cl.centres
        th = np.arctan2(dd[:, 1], dd[:, 0])
        d = d * np.exp(2j * O_.modes(cl.N)[None, :] * th[:, None])
    J, dJ, _, _ = O_.bessel_diagonals(cl.radii, cl.k, cl.N)
    return d * J, cl.k * d * dJ


def test_trace_coefficients_match_quadrature():
    cl = W.small_mixed(seed=3, M=6, N=10, k=2.0)
    for s in (np.array([30.0, -12.0]), np.array([0.3, 6.5]), np.array([-4.0, -4.2])):
        U, dU = closed_form(cl, s)
        Uq, dUq = quadrature_coefficients(cl.centres, cl.radii, cl.k, cl.N, s)
        assert np.abs(U - Uq).max() <= 1e-12 * np.abs(Uq).max()
        assert np.abs(dU - dUq).max() <= 1e-12 * np.abs(dUq).max()


def test_planted_phase_mistake_is_caught():
    cl = W.small_mixed(seed=3, M=6, N=10, k=2.0)
    s = np.array([0.3, 6.5])
    U, _ = closed_form(cl, s, conj_phase=True)
    Uq, _ = quadrature_coefficients(cl.centres, cl.radii, cl.k, cl.N, s)
    assert np.abs(U - Uq).max() > 1e-3 * np.abs(Uq).max()


def bc_residual(cl, s, offset=1e-12):
    """max |u_scat + u_inc| / max |u_inc| on the circles, oracle LU solve."""
    b = O_.rhs_pointsource(cl.centres, cl.radii, cl.bc, cl.k, cl.N, [s])
    A = O_.assemble(cl.centres, cl.radii, cl.bc, cl.k, cl.N)
    rho = np.linalg.solve(A, b)
    th = np.linspace(0.0, 2 * np.pi, 24, endpoint=False)
    worst = 0.0
    for p in range(cl.M):
        x = cl.centres[p][None, :] + cl.radii[p] * (1 + offset) * np.stack([np.cos(th), np.sin(th)], axis=1)
        us = O_.single_layer_potential(cl.centres, cl.radii, cl.k, cl.N, rho[:, 0], x)
        ui = 0.25j * special.hankel1(0, cl.k * np.hypot(x[:, 0] - s[0], x[:, 1] - s[1]))
        worst = max(worst, np.abs(us + ui).max() / np.abs(ui).max())
    return worst


def test_rhs_signs_and_sound_soft_boundary_condition():
    """Four sound-soft disks, source at the centre of their square (1.83
    from each circle): the boundary condition holds to the truncation error,
    which falls spectrally with N (the trace of u_inc on a circle decays
    like (a/b)^m)."""
    c0 = W.four_disks()
    s = np.array([0.0, 0.0])
    b = O_.rhs_pointsource(c0.centres, c0.radii, c0.bc, c0.k, c0.N, [s])
    U, _ = closed_form(c0, s)
    assert np.allclose(b[:, 0], -U.reshape(-1), rtol=0, atol=1e-15)
    r12 = bc_residual(W.Cluster(c0.centres, c0.radii, c0.bc, c0.k, 12), s)
    r20 = bc_residual(W.Cluster(c0.centres, c0.radii, c0.bc, c0.k, 20), s)
    assert r20 < 1e-8 and r20 < r12 / 10, (r12, r20)
