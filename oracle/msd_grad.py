"""FP64 CPU oracle for the gradient of a far-field misfit.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper computes fields, not gradients; the misfit and its derivatives are
built here from the paper's formulas by the adjoint method, with every
derivative written out analytically:

    J(O, a, k) = sum_{r, t} |F(theta_t; beta_r) - F*_{t r}|^2,
    F = C rho,   A rho = b   (section 4.4, section 5, Prop. 4.1),
    dJ = 2 Re[ w^H dC rho + lam^H (db - dA rho) ],   A^H lam = C^H w,
    w = F - F*.

Derivatives used (all standard Bessel identities):
  * separation generator G_l(b) = H_l(k|b|) e^{i l alpha(b)}:
      dG_l/db_x = (k/2)(G_{l-1} - G_{l+1}),  dG_l/db_y = (i k/2)(G_{l-1} + G_{l+1}),
      dG_l/dk = |b| H_l'(k|b|) e^{i l alpha};
  * Z'' = -Z'/x - (1 - m^2/x^2) Z for Z = J_m, H_m (Bessel's equation);
  * b_pq = O_p - O_q, so d/dO_p acts as +d/db on block (p, q) and as -d/db on
    block (q, p).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
from scipy import special

from . import msd_oracle as O_

DIRICHLET = O_.DIRICHLET


def _bessel_all(a, k, N):
    """J, J', J'', H, H', H'' at k a_p for m = -N..N ([M, n] each)."""
    m = O_.modes(N)[None, :].astype(float)
    x = k * np.asarray(a, float)[:, None]
    J, dJ, H, dH = O_.bessel_diagonals(a, k, N)
    ddJ = -dJ / x - (1.0 - m * m / (x * x)) * J
    ddH = -dH / x - (1.0 - m * m / (x * x)) * H
    return J, dJ, ddJ, H, dH, ddH


def _row_factor(bc_p, k, a_p, J, dJ, ddJ):
    """(i pi / 2) sqrt(a_p) * left_m and its derivatives in a_p and k, where
    left = J_m (Dirichlet row) or k J'_m (Neumann row), all at k a_p."""
    c = 0.5j * np.pi
    sa = np.sqrt(a_p)
    if bc_p == DIRICHLET:
        left, dl_da, dl_dk = J, k * dJ, a_p * dJ
    else:
        left, dl_da, dl_dk = k * dJ, k * k * ddJ, dJ + k * a_p * ddJ
    f = c * sa * left
    f_a = c * (left / (2.0 * sa) + sa * dl_da)
    f_k = c * sa * dl_dk
    return f, f_a, f_k


def _diag(bc_p, k, a_p, J, dJ, ddJ, H, dH, ddH):
    """Diagonal of A^pp and its derivatives in a_p and k (section 4.2)."""
    c = 0.5j * np.pi
    if bc_p == DIRICHLET:
        d = c * a_p * J * H
        d_a = c * (J * H + a_p * k * (dJ * H + J * dH))
        d_k = c * a_p * a_p * (dJ * H + J * dH)
    else:
        d = c * k * a_p * J * dH
        d_a = c * k * (J * dH + a_p * k * (dJ * dH + J * ddH))
        d_k = c * a_p * (J * dH + k * a_p * (dJ * dH + J * ddH))
    return d, d_a, d_k


def farfield_matrix(O, a, k, N, thetas):
    """C[t, row] = (a_L(theta_t))^p_m of section 4.4."""
    return np.stack([O_.farfield_coefficients(O, a, k, N, t) for t in np.atleast_1d(thetas)])


def _farfield_matrix_derivs(O, a, k, N, thetas):
    """dC/dO_x, dC/dO_y (acting on the disk's own columns), dC/da, dC/dk."""
    O = np.asarray(O, float)
    a = np.asarray(a, float)
    M = len(a)
    n = 2 * N + 1
    th = np.atleast_1d(thetas)[:, None, None]
    C = farfield_matrix(O, a, k, N, thetas).reshape(len(np.atleast_1d(thetas)), M, n)
    dJ = O_.bessel_diagonals(a, k, N)[1]
    proj = np.cos(th) * O[None, :, 0:1] + np.sin(th) * O[None, :, 1:2]      # theta_hat . O_p
    # d/da and d/dk of sqrt(a) J_m(k a) / sqrt(k) e^{-i k theta_hat . O}, written without dividing by J
    K0 = 1j * np.exp(-1j * np.pi / 4) / (2 * np.sqrt(k))
    m = O_.modes(N)[None, None, :]
    E = np.exp(1j * m * (th - np.pi / 2)) * np.exp(-1j * k * proj)
    base_dJ = K0 * np.sqrt(a)[None, :, None] * dJ[None] * E
    C_x = -1j * k * np.cos(th) * C
    C_y = -1j * k * np.sin(th) * C
    C_a = C / (2 * a[None, :, None]) + k * base_dJ
    C_k = -C / (2 * k) - 1j * proj * C + a[None, :, None] * base_dJ
    return C, C_x, C_y, C_a, C_k


def misfit(O, a, bc, k, N, betas, thetas, F_target):
    """J = sum |F - F*|^2 with rho from the dense LU solve."""
    rho, _ = O_.solve(O, a, bc, k, N, betas, method="lu")
    F = O_.farfield(O, a, k, N, rho, thetas)
    return float(np.sum(np.abs(F - F_target) ** 2))


def misfit_and_gradient(O, a, bc, k, N, betas, thetas, F_target):
    """Analytic adjoint gradient of J with respect to the centres [M, 2], the
    radii [M] and k.  Returns (J, gO, ga, gk, F)."""
    O = np.asarray(O, float)
    a = np.asarray(a, float)
    bc = np.asarray(bc)
    M = len(a)
    n = 2 * N + 1
    betas = np.atleast_1d(np.asarray(betas, float))
    R = len(betas)
    A = O_.assemble(O, a, bc, k, N)
    b = O_.rhs_planewave(O, a, bc, k, N, betas)
    lu = sla.lu_factor(A)
    rho = sla.lu_solve(lu, b)
    C, C_x, C_y, C_a, C_k = _farfield_matrix_derivs(O, a, k, N, thetas)
    T = C.shape[0]
    Cm = C.reshape(T, M * n)
    F = Cm @ rho
    w = F - F_target
    J = float(np.sum(np.abs(w) ** 2))
    lam = sla.lu_solve(lu, Cm.conj().T @ w, trans=2)       # A^H lam = C^H w

    RH = rho.reshape(M, n, R)
    LH = lam.reshape(M, n, R)
    gO = np.zeros((M, 2))
    ga = np.zeros(M)
    gk = 0.0

    # far-field term w^H dC rho
    def ff_term(Cd):           # Cd [T, M, n]: per-disk contribution sum_t conj(w) Cd rho
        return np.einsum("tr,tpm,pmr->p", w.conj(), Cd, RH)
    gO[:, 0] += 2 * np.real(ff_term(C_x))
    gO[:, 1] += 2 * np.real(ff_term(C_y))
    ga += 2 * np.real(ff_term(C_a))
    gk += 2 * np.real(ff_term(C_k).sum())

    # right-hand side term lam^H db, b^p_m = -d^p_m left^p_m (Prop. 4.1)
    Jb, dJb, ddJb, Hb, dHb, ddHb = _bessel_all(a, k, N)
    for r, beta in enumerate(betas):
        bh = np.array([np.cos(beta), np.sin(beta)])
        d = O_.planewave_coefficients(O, a, k, N, beta)           # [M, n]
        proj = O @ bh
        for p in range(M):
            if bc[p] == DIRICHLET:
                left, dl_da, dl_dk = Jb[p], k * dJb[p], a[p] * dJb[p]
            else:
                left, dl_da, dl_dk = k * dJb[p], k * k * ddJb[p], dJb[p] + k * a[p] * ddJb[p]
            bp = -d[p] * left
            db_x = 1j * k * bh[0] * bp
            db_y = 1j * k * bh[1] * bp
            db_a = -(d[p] / (2 * a[p]) * left + d[p] * dl_da)
            db_k = -(1j * proj[p] * d[p] * left + d[p] * dl_dk)
            lc = LH[p, :, r].conj()
            gO[p, 0] += 2 * np.real(lc @ db_x)
            gO[p, 1] += 2 * np.real(lc @ db_y)
            ga[p] += 2 * np.real(lc @ db_a)
            gk += 2 * np.real(lc @ db_k)

    # operator term -lam^H dA rho, block by block (section 4.2)
    l_idx = np.arange(-2 * N - 1, 2 * N + 2)                      # one order beyond each end
    m = O_.modes(N)
    idx = (m[None, :] - m[:, None]) + 2 * N + 1                  # (n - m) in the extended range
    sa = np.sqrt(a)
    for p in range(M):
        f, f_a, f_k = _row_factor(bc[p], k, a[p], Jb[p], dJb[p], ddJb[p])
        dg, dg_a, dg_k = _diag(bc[p], k, a[p], Jb[p], dJb[p], ddJb[p], Hb[p], dHb[p], ddHb[p])
        # diagonal block
        t_diag = np.einsum("mr,m,mr->", LH[p].conj(), dg_a, RH[p])
        ga[p] -= 2 * np.real(t_diag)
        gk -= 2 * np.real(np.einsum("mr,m,mr->", LH[p].conj(), dg_k, RH[p]))
        qs = np.array([q for q in range(M) if q != p], dtype=int)
        if not len(qs):
            continue
        bv = O[p][None, :] - O[qs]
        bb = np.hypot(bv[:, 0], bv[:, 1])
        al = np.arctan2(bv[:, 1], bv[:, 0])
        kb = k * bb[:, None]
        G = special.hankel1(l_idx[None, :], kb) * np.exp(1j * l_idx[None, :] * al[:, None])
        Gk = bb[:, None] * special.h1vp(l_idx[None, :], kb) * np.exp(1j * l_idx[None, :] * al[:, None])
        g0 = G[:, 1:-1]                                            # l = -2N..2N
        gx = 0.5 * k * (G[:, :-2] - G[:, 2:])
        gy = 0.5j * k * (G[:, :-2] + G[:, 2:])
        gkk = Gk[:, 1:-1]
        ST = g0[:, idx - 1]                                         # [q, m, n]: g_{n-m}
        STx, STy, STk = gx[:, idx - 1], gy[:, idx - 1], gkk[:, idx - 1]
        rq = sa[qs][:, None] * Jb[qs]                               # sqrt(a_q) J_n(k a_q)
        rq_a = Jb[qs] / (2 * sa[qs][:, None]) + sa[qs][:, None] * k * dJb[qs]
        rq_k = sa[qs][:, None] * a[qs][:, None] * dJb[qs]
        lp = LH[p].conj()                                           # [m, r]
        X = RH[qs]                                                   # [q, n, r]
        # lam^{pH} (dA^{pq}) rho^q summed over r, per q, for each derivative of the block
        def contract(left_vec, S, right):                           # -> [q]
            return np.einsum("mr,m,qmn,qn,qnr->q", lp, left_vec, S, right, X)
        tx = contract(f, STx, rq)
        ty = contract(f, STy, rq)
        # row p: d/dO_p = +d/db; column side: d/dO_q = -d/db
        gO[p, 0] -= 2 * np.real(tx.sum())
        gO[p, 1] -= 2 * np.real(ty.sum())
        np.add.at(gO[:, 0], qs, 2 * np.real(tx))
        np.add.at(gO[:, 1], qs, 2 * np.real(ty))
        # radii: the row factor of p, the column factors of each q
        ga[p] -= 2 * np.real(contract(f_a, ST, rq).sum())
        np.add.at(ga, qs, -2 * np.real(contract(f, ST, rq_a)))
        # wavenumber: row factor, generator, column factor
        gk -= 2 * np.real(contract(f_k, ST, rq).sum() + contract(f, STk, rq).sum()
                          + contract(f, ST, rq_k).sum())
    return J, gO, ga, gk, F


def misfit_gradient_fd(O, a, bc, k, N, betas, thetas, F_target, h=1e-6):
    """Centred finite differences of misfit() in every parameter."""
    O = np.asarray(O, float)
    a = np.asarray(a, float)
    M = len(a)
    gO = np.zeros((M, 2))
    ga = np.zeros(M)
    for p in range(M):
        for c in range(2):
            Op, Om = O.copy(), O.copy()
            Op[p, c] += h
            Om[p, c] -= h
            gO[p, c] = (misfit(Op, a, bc, k, N, betas, thetas, F_target)
                        - misfit(Om, a, bc, k, N, betas, thetas, F_target)) / (2 * h)
        ap, am = a.copy(), a.copy()
        ap[p] += h
        am[p] -= h
        ga[p] = (misfit(O, ap, bc, k, N, betas, thetas, F_target)
                 - misfit(O, am, bc, k, N, betas, thetas, F_target)) / (2 * h)
    gk = (misfit(O, a, bc, k + h, N, betas, thetas, F_target)
          - misfit(O, a, bc, k - h, N, betas, thetas, F_target)) / (2 * h)
    return gO, ga, gk
