"""Pins of the oracle's penetrable (transmission) system (section 7,
Example II) by quantities it does not use.

* One disk at the origin: the far field equals the textbook transmission
  series, b_m = (mu k- J'_m(k- a) J_m(k+ a) - k+ J'_m(k+ a) J_m(k- a)) /
  (k+ H'_m(k+ a) J_m(k- a) - mu k- J'_m(k- a) H_m(k+ a)), for real and
  complex k- and mu != 1 (1e-12).
* A 5-disk cluster: on every circle, the exterior total field
  L+ rho+ + u_inc and the interior field L- rho- (summed term by term from the
  Hankel and Bessel expansions of Prop. 4.3, their gradients likewise)
  satisfy the two transmission conditions once projected on the modes
  -N..N (exactly what the Galerkin system imposes, 1e-11), and pointwise up
  to a truncation error that falls spectrally in N.
* Energy balance (optical theorem) for lossless obstacles (real k-, mu).
* The printed (2, 2) block +(I/2 + N-) fails the single-disk series.
"""
import numpy as np
import pytest
from scipy import special

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def transmission_far(kp, km, mu, a, beta, th, terms=40):
    m = np.arange(-terms, terms + 1)
    num = mu * km * special.jvp(m, km * a) * special.jv(m, kp * a) - kp * special.jvp(m, kp * a) * special.jv(m, km * a)
    den = kp * special.h1vp(m, kp * a) * special.jv(m, km * a) - mu * km * special.jvp(m, km * a) * special.hankel1(m, kp * a)
    return np.exp(-1j * np.pi / 4) * np.sqrt(2 / (np.pi * kp)) * (np.exp(1j * np.outer(th - beta, m)) @ (num / den))


@pytest.mark.parametrize("kp,km,mu", [(1.3, 2.6, 1.0), (2.0, 1.1, 0.5), (1.0, 2.0 + 0.3j, 1.7)])
def test_single_disk_transmission_series(kp, km, mu):
    a, N, beta = 0.9, 18, 0.7
    O = np.zeros((1, 2))
    rp, _ = O_.solve_penetrable(O, np.array([a]), kp, km, mu, N, [beta])
    th = np.linspace(0, 2 * np.pi, 13)
    F = O_.farfield(O, np.array([a]), kp, N, rp, th)[:, 0]
    ref = transmission_far(kp, km, mu, a, beta, th)
    assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()


def test_printed_sign_fails_the_series():
    a, N, beta, kp, km = 0.9, 18, 0.7, 1.3, 2.6
    O = np.zeros((1, 2))
    A = O_.assemble_penetrable(O, np.array([a]), kp, km, 1.0, N)
    Nt = A.shape[0] // 2
    A[Nt:, Nt:] *= -1  # the printed block +(I/2 + N-)
    x = np.linalg.solve(A, O_.rhs_penetrable(O, np.array([a]), kp, N, [beta]))
    th = np.linspace(0, 2 * np.pi, 13)
    F = O_.farfield(O, np.array([a]), kp, N, x[:Nt], th)[:, 0]
    ref = transmission_far(kp, km, 1.0, a, beta, th)
    assert np.abs(F - ref).max() > 0.1 * np.abs(ref).max()


def fields_on_circle(cl, km, rho_p, rho_m, beta, p, t, eps=1e-13):
    """Exterior total field and interior field and their normal derivatives
    at the points of circle p, term by term."""
    O, a, kp, N = cl.centres, cl.radii, cl.k, cl.N
    m = O_.modes(N)
    n = cl.n
    J, _, H, _ = O_.bessel_diagonals(a, kp, N)
    Jm_, _, Hm_, _ = O_.bessel_diagonals(a, km, N)
    nrm = np.stack([np.cos(t), np.sin(t)], axis=1)

    def sum_terms(k, coef, inside_self, x):
        u = np.zeros(len(x), complex)
        g = np.zeros((len(x), 2), complex)
        for q in range(cl.M):
            d = x - O[q][None, :]
            r = np.hypot(d[:, 0], d[:, 1])
            th = np.arctan2(d[:, 1], d[:, 0])
            rh = d / r[:, None]
            tt = np.stack([-rh[:, 1], rh[:, 0]], axis=1)
            if inside_self and q == p:
                Z = special.jv(m[None, :], k * r[:, None])
                dZ = special.jvp(m[None, :], k * r[:, None])
            else:
                Z = special.hankel1(m[None, :], k * r[:, None])
                dZ = special.h1vp(m[None, :], k * r[:, None])
            E = np.exp(1j * m[None, :] * th[:, None])
            c = coef[q]
            u += (Z * E) @ c
            g += ((k * dZ * E) @ c)[:, None] * rh + (((1j * m[None, :] / r[:, None]) * Z * E) @ c)[:, None] * tt
        return u, (g * nrm).sum(1)

    s = 0.5j * np.pi * a[:, None] / np.sqrt(2 * np.pi * a[:, None])
    cp = s * J * rho_p.reshape(cl.M, n)
    cm_out = s * Jm_ * rho_m.reshape(cl.M, n)
    cm_in = cm_out.copy()
    cm_in[p] = s[p] * Hm_[p] * rho_m.reshape(cl.M, n)[p]
    xo = O[p][None, :] + a[p] * (1 + eps) * nrm
    xi = O[p][None, :] + a[p] * (1 - eps) * nrm
    up, dup = sum_terms(kp, cp, False, xo)
    bh = np.array([np.cos(beta), np.sin(beta)])
    ui = np.exp(1j * kp * xo @ bh)
    dui = 1j * kp * (nrm @ bh) * ui
    um, dum = sum_terms(km, cm_in, True, xi)
    return up + ui, dup + dui, um, dum


def project(v, a, N, t):
    m = np.arange(-N, N + 1)
    return np.exp(-1j * np.outer(m, t)) @ v * (a * 2 * np.pi / len(t)) / np.sqrt(2 * np.pi * a)


def test_transmission_conditions_on_every_circle():
    km = 3.1
    beta = 0.4
    worst = {}
    for N in (10, 18):
        cl = W.small_mixed(seed=5, M=5, N=N, k=1.6)
        mu = np.array([1.0, 0.6, 2.0, 1.0, 1.4])
        rp, rm = O_.solve_penetrable(cl.centres, cl.radii, cl.k, km, mu, N, [beta])
        t = 2 * np.pi * np.arange(256) / 256
        point = 0.0
        for p in range(cl.M):
            up, dup, um, dum = fields_on_circle(cl, km, rp[:, 0], rm[:, 0], beta, p, t)
            scale = np.abs(up).max()
            assert np.abs(project(up - um, cl.radii[p], N, t)).max() <= 1e-11 * scale
            assert np.abs(project(dup - mu[p] * dum, cl.radii[p], N, t)).max() <= 1e-11 * scale * cl.k
            point = max(point, np.abs(up - um).max() / scale)
        worst[N] = point
    assert worst[18] < worst[10] / 100, worst


def test_energy_balance_lossless():
    cl = W.small_mixed(seed=5, M=5, N=20, k=1.6)
    km, mu, beta = 2.7, np.array([1.0, 0.6, 2.0, 1.0, 1.4]), 0.4
    rp, _ = O_.solve_penetrable(cl.centres, cl.radii, cl.k, km, mu, cl.N, [beta])
    T = 720
    th = W.angles(T)
    F = O_.farfield(cl.centres, cl.radii, cl.k, cl.N, rp, np.concatenate([th, [beta]]))[:, 0]
    lhs = np.sum(np.abs(F[:T]) ** 2) * 2 * np.pi / T
    rhs = -2 * np.sqrt(2 * np.pi / cl.k) * np.real(np.exp(1j * np.pi / 4) * F[T])
    assert abs(lhs - rhs) <= 1e-10 * lhs


def test_point_source_transmission_conditions():
    """A point source outside a 3-disk cluster: the solution's exterior total
    field (with u_inc = (i/4) H_0(k+|x - s|)) and interior field satisfy the
    projected transmission conditions on every circle."""
    cl = W.small_mixed(seed=5, M=3, N=14, k=1.6)
    km, mu = 2.4, np.array([1.0, 1.5, 0.7])
    src = np.array([9.0, -7.5])
    A = O_.assemble_penetrable(cl.centres, cl.radii, cl.k, km, mu, cl.N)
    x = np.linalg.solve(A, O_.rhs_penetrable_pointsource(cl.centres, cl.radii, cl.k, cl.N, [src]))[:, 0]
    Nt = cl.ntot
    t = 2 * np.pi * np.arange(256) / 256
    for p in range(cl.M):
        nrm = np.stack([np.cos(t), np.sin(t)], axis=1)
        xo = cl.centres[p][None, :] + cl.radii[p] * (1 + 1e-13) * nrm
        xi = cl.centres[p][None, :] + cl.radii[p] * (1 - 1e-13) * nrm
        d = xo - src[None, :]
        r = np.hypot(d[:, 0], d[:, 1])
        ui = 0.25j * special.hankel1(0, cl.k * r)
        up = O_.single_layer_potential(cl.centres, cl.radii, cl.k, cl.N, x[:Nt], xo) + ui
        um = O_.single_layer_potential_inside(cl.centres, cl.radii, km, cl.N, x[Nt:], xi, p)
        assert np.abs(project(up - um, cl.radii[p], cl.N, t)).max() <= 1e-11 * np.abs(up).max()
