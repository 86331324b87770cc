"""FP64 CPU oracle for the Fourier-spectral multiple-scattering method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
executes this module: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path: Bessel and Hankel values come from SciPy (AMOS),
blocks are assembled densely from their printed definitions, systems are
solved by LAPACK LU or by a plain restarted GMRES written here.

Every function cites the part of the paper (mu-diff, arXiv 1409.8186) it
restates.  Notation: disks p = 1..M with centre O_p, radius a_p; Fourier modes
m = -N..N on every disk (n = 2N+1 per disk); b_pq = O_p - O_q is the vector
from O_q to O_p and alpha_pq its polar angle (section 4.1); time dependence
exp(-i omega t) and first-kind Hankel functions (section 2).

Readings of the paper taken here:
  * the Galerkin test uses the hermitian product (section 4.1), so the
    right-hand side of row (p, m) is (u_inc, Phi^p_m) and the system is
    A rho = -U (section 5);
  * the angle alpha_pq of the separation matrix is the polar angle of
    b_pq = O_p - O_q (the printed subscript "alpha_bq" is read as alpha_pq);
  * sound-hard disks use the same single-layer representation u = L rho and
    the exterior normal trace (-I/2 + N) rho = -d_n u_inc (jump relations of
    Prop. 3.2), with the diagonal block (i pi k a_p / 2) J^p H'^p;
  * the single-scattering preconditioner is P = block diagonal part of A
    (section 5), applied on the left; GMRES starts from x0 = 0 and measures
    relres = ||P^-1 (b - A x)|| / ||P^-1 b||;
  * far field: the single-layer coefficient vector of section 4.4 (the a_L
    formula); a_M is not used;
  * other integral equations (sections 3, 4.2, 5): a formulation is a
    linear combination of I, L, M, N, D per boundary condition of the row
    disk, a right-hand side -(w_U U + w_dU dU), and a representation
    u = w_L L dens + w_M M dens for the fields; the diagonal of D is
    -(i pi k^2 a_p / 2) J' H' and the double-layer far-field vector carries
    -i e^{-i pi/4} sqrt(k a_p)/2, the signs the definitions of D and of the
    double-layer potential give (both printed with the opposite sign);
  * penetrable obstacles (section 7, Example II): one interior wavenumber
    k- per configuration and mu per disk; the (2, 2) block of the
    transmission system is -mu (I/2 + N-), the sign the interior normal
    trace of L- rho- (Prop. 3.2) and the transmission condition
    d_n u+ - mu d_n u- = -d_n u_inc give (printed without the minus);
  * time reversal (section 7): the mirror angles are alpha_j = 2 pi j /
    n_alpha from 0, the far field of incidence alpha_j is measured at
    alpha_i + pi (row i of F), and T = conj(F)^T F carries no quadrature
    weight h_alpha (as printed; a weight only scales the eigenvalues).
"""
from __future__ import annotations

import numpy as np
from scipy import special

DIRICHLET = 0
NEUMANN = 1


# --------------------------------------------------------------------------
# Section 4.2: Bessel diagonals and the separation matrix
# --------------------------------------------------------------------------

def modes(N: int) -> np.ndarray:
    """Fourier indices m = -N..N kept on a disk after truncation (section 5)."""
    return np.arange(-N, N + 1)


def bessel_diagonals(a, k: float, N: int):
    """Section 4.2: the diagonal matrices J^p, J'^p, H^p, H'^p with entries
    J_m(k a_p), J_m'(k a_p), H^(1)_m(k a_p), H^(1)_m'(k a_p), m = -N..N.
    Returns four [M, 2N+1] arrays."""
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    m = modes(N)[None, :]
    x = k * a[:, None]
    return (special.jv(m, x), special.jvp(m, x), special.hankel1(m, x),
            special.h1vp(m, x))


def pair_vector(Op, Oq):
    """Section 4.1: b_pq = O_p - O_q (vector from O_q to O_p), its length and
    its polar angle alpha_pq."""
    v = np.asarray(Op, dtype=np.float64) - np.asarray(Oq, dtype=np.float64)
    return v, float(np.hypot(v[0], v[1])), float(np.arctan2(v[1], v[0]))


def separation_generator(Op, Oq, k: float, N: int) -> np.ndarray:
    """Section 4.2: the entries of S^pq depend on m - n only; this returns
    the 4N+1 values H^(1)_l(k b_pq) exp(i l alpha_pq), l = -2N..2N, so that
    S^pq_mn = g[(m - n) + 2N] and (S^pq)^T_mn = g[(n - m) + 2N]."""
    _, b, alpha = pair_vector(Op, Oq)
    l = np.arange(-2 * N, 2 * N + 1)
    return special.hankel1(l, k * b) * np.exp(1j * l * alpha)


def separation_matrix(Op, Oq, k: float, N: int) -> np.ndarray:
    """Section 4.2: S^pq_mn = H^(1)_{m-n}(k b_pq) exp(i (m-n) alpha_pq),
    m, n = -N..N."""
    _, b, alpha = pair_vector(Op, Oq)
    m = modes(N)
    d = m[:, None] - m[None, :]
    return special.hankel1(d, k * b) * np.exp(1j * d * alpha)


# --------------------------------------------------------------------------
# Section 4.2 / section 5: the truncated operator blocks
# --------------------------------------------------------------------------

def block_L(O, a, k, N, p, q) -> np.ndarray:
    """Section 4.2, single-layer block L^pq: (i pi a_p / 2) J^p H^p on the
    diagonal, (i pi sqrt(a_p a_q) / 2) J^p (S^pq)^T J^q off it."""
    J, _, H, _ = bessel_diagonals(a, k, N)
    if p == q:
        return np.diag(0.5j * np.pi * a[p] * J[p] * H[p])
    S = separation_matrix(O[p], O[q], k, N)
    return 0.5j * np.pi * np.sqrt(a[p] * a[q]) * (J[p][:, None] * S.T * J[q][None, :])


def block_N(O, a, k, N, p, q) -> np.ndarray:
    """Section 4.2, block N^pq of the normal-derivative trace of the
    single-layer potential: I/2 + (i pi k a_p / 2) J^p H'^p on the diagonal,
    (i k pi sqrt(a_p a_q) / 2) J'^p (S^pq)^T J^q off it."""
    J, dJ, H, dH = bessel_diagonals(a, k, N)
    if p == q:
        return 0.5 * np.eye(2 * N + 1) + np.diag(0.5j * np.pi * k * a[p] * J[p] * dH[p])
    S = separation_matrix(O[p], O[q], k, N)
    return 0.5j * k * np.pi * np.sqrt(a[p] * a[q]) * (dJ[p][:, None] * S.T * J[q][None, :])


def assemble(O, a, bc, k, N) -> np.ndarray:
    """Section 5: the N_tot x N_tot block matrix.  Dirichlet rows p carry
    the EFIE blocks L^pq; Neumann rows carry (-I/2 + N)^pq, the exterior
    normal trace of the single-layer potential (Prop. 3.2)."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    A = np.zeros((M * n, M * n), dtype=np.complex128)
    for p in range(M):
        for q in range(M):
            if bc[p] == DIRICHLET:
                B = block_L(O, a, k, N, p, q)
            else:
                B = block_N(O, a, k, N, p, q)
                if p == q:
                    B = B - 0.5 * np.eye(n)
            A[p * n:(p + 1) * n, q * n:(q + 1) * n] = B
    return A


# --------------------------------------------------------------------------
# Prop. 4.1: plane-wave right-hand sides
# --------------------------------------------------------------------------

def planewave_coefficients(O, a, k, N, beta) -> np.ndarray:
    """Prop. 4.1: d^p_m = sqrt(2 pi a_p) exp(i k beta_hat . b_p)
    exp(i m (pi/2 - beta)), with b_p = O_p.  Returns [M, 2N+1]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    m = modes(N)[None, :]
    phase = k * (np.cos(beta) * O[:, 0] + np.sin(beta) * O[:, 1])
    return (np.sqrt(2 * np.pi * a)[:, None] * np.exp(1j * phase)[:, None]
            * np.exp(1j * m * (np.pi / 2 - beta)))


def rhs_planewave(O, a, bc, k, N, betas) -> np.ndarray:
    """Prop. 4.1 and section 5: the right-hand side b = -U of A rho = b.
    Dirichlet rows: U^p_m = d^p_m J_m(k a_p); Neumann rows:
    dU^p_m = k d^p_m J_m'(k a_p).  Returns [N_tot, R] (one column per
    incidence angle)."""
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    J, dJ, _, _ = bessel_diagonals(a, k, N)
    cols = []
    for beta in betas:
        d = planewave_coefficients(O, a, k, N, beta)
        U = np.where(np.asarray(bc)[:, None] == DIRICHLET, d * J, k * d * dJ)
        cols.append(-U.reshape(-1))
    return np.stack(cols, axis=1)


def pointsource_coefficients(O, a, k, N, source) -> np.ndarray:
    """Point-source proposition of section 4.3: for u_inc = G(x, s) =
    (i/4) H_0(k |x - s|) the trace coefficients are U^p_m = d'^p_m J_m(k a_p)
    with d'^p_m = (i pi a_p / 2) H_m(k r_p(s)) exp(-i m theta_p(s)) / sqrt(2 pi a_p)
    = (i/4) sqrt(2 pi a_p) H_m(k r_p(s)) exp(-i m theta_p(s)), (r_p, theta_p) the
    polar coordinates of s - O_p (Graf's addition theorem, |s - O_p| > a_p).
    Returns [M, 2N+1]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    s = np.asarray(source, dtype=np.float64)
    m = modes(N)[None, :]
    d = s[None, :] - O
    r = np.hypot(d[:, 0], d[:, 1])
    th = np.arctan2(d[:, 1], d[:, 0])
    return (0.25j * np.sqrt(2 * np.pi * a)[:, None] * special.hankel1(m, k * r[:, None])
            * np.exp(-1j * m * th[:, None]))


def rhs_pointsource(O, a, bc, k, N, sources) -> np.ndarray:
    """b = -U for point sources (one column per source s_r, [R, 2]):
    Dirichlet rows U^p_m = d'^p_m J_m(k a_p), Neumann rows k d'^p_m J_m'(k a_p)."""
    J, dJ, _, _ = bessel_diagonals(a, k, N)
    cols = []
    for src in np.atleast_2d(np.asarray(sources, dtype=np.float64)):
        d = pointsource_coefficients(O, a, k, N, src)
        U = np.where(np.asarray(bc)[:, None] == DIRICHLET, d * J, k * d * dJ)
        cols.append(-U.reshape(-1))
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# Section 5: single-scattering preconditioner, direct and Krylov solves
# --------------------------------------------------------------------------

def diagonal_of_blocks(A, M, n) -> np.ndarray:
    """The diagonal blocks A^pp are diagonal matrices (section 4.2); this
    returns their diagonals as one vector of length N_tot."""
    return np.diag(A).copy()


def precondition(A, b, M, n):
    """Section 5: left single-scattering preconditioning P^-1 A, P^-1 b with
    P the block-diagonal part of A (here a plain diagonal)."""
    P = diagonal_of_blocks(A, M, n)
    return A / P[:, None], b / P[:, None] if b.ndim == 2 else b / P


def solve_lu(A, b) -> np.ndarray:
    """Section 5: direct solve by LU (LAPACK via numpy)."""
    return np.linalg.solve(A, b)


def gmres(matvec, b, restart=50, tol=1e-10, maxit=1000):
    """Restarted GMRES(restart) for one right-hand side, as used in section 6.2
    (x0 = 0).  Arnoldi with modified Gram-Schmidt, Givens rotations on the
    Hessenberg matrix, least-squares update at the end of each cycle.
    Returns x, flag (0 converged, 1 not), relres, total iterations, residual
    history (relative)."""
    b = np.asarray(b, dtype=np.complex128)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0, 0, [0.0]
    resvec = [1.0]
    total = 0
    while total < maxit:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta / nb <= tol:
            return x, 0, beta / nb, total, resvec
        m = restart
        V = np.zeros((len(b), m + 1), dtype=np.complex128)
        Hs = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        j_used = 0
        for j in range(m):
            w = matvec(V[:, j])
            for i in range(j + 1):
                Hs[i, j] = np.vdot(V[:, i], w)
                w = w - Hs[i, j] * V[:, i]
            Hs[j + 1, j] = np.linalg.norm(w)
            if Hs[j + 1, j] != 0:
                V[:, j + 1] = w / Hs[j + 1, j]
            for i in range(j):
                t = cs[i] * Hs[i, j] + sn[i] * Hs[i + 1, j]
                Hs[i + 1, j] = -np.conj(sn[i]) * Hs[i, j] + np.conj(cs[i]) * Hs[i + 1, j]
                Hs[i, j] = t
            den = np.hypot(abs(Hs[j, j]), abs(Hs[j + 1, j]))
            if den == 0:
                cs[j], sn[j] = 1.0, 0.0
            elif abs(Hs[j, j]) == 0:
                cs[j], sn[j] = 0.0, np.conj(Hs[j + 1, j]) / abs(Hs[j + 1, j])
            else:
                ph = Hs[j, j] / abs(Hs[j, j])
                cs[j] = abs(Hs[j, j]) / den
                sn[j] = ph * np.conj(Hs[j + 1, j]) / den
            Hs[j, j] = cs[j] * Hs[j, j] + sn[j] * Hs[j + 1, j]
            Hs[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_used = j + 1
            resvec.append(abs(g[j + 1]) / nb)
            if abs(g[j + 1]) / nb <= tol or total >= maxit:
                break
        y = np.linalg.solve(np.triu(Hs[:j_used, :j_used]), g[:j_used])
        x = x + V[:, :j_used] @ y
    r = b - matvec(x)
    relres = np.linalg.norm(r) / nb
    return x, (0 if relres <= tol else 1), relres, total, resvec


def solve(cluster_O, a, bc, k, N, betas, method="lu", **gm):
    """Assemble, precondition and solve for every incidence angle.
    Returns rho [N_tot, R] and a dict of per-column solver statistics."""
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    A = assemble(cluster_O, a, bc, k, N)
    b = rhs_planewave(cluster_O, a, bc, k, N, betas)
    Ap, bp = precondition(A, b, M, n)
    if method == "lu":
        return solve_lu(Ap, bp), {}
    cols, stats = [], []
    for r in range(b.shape[1]):
        x, flag, relres, it, rv = gmres(lambda v: Ap @ v, bp[:, r], **gm)
        cols.append(x)
        stats.append(dict(flag=flag, relres=relres, iters=it, resvec=rv))
    return np.stack(cols, axis=1), stats


# --------------------------------------------------------------------------
# Matrix-free application of the preconditioned operator to selected rows
# (for clusters whose dense matrix does not fit in host memory)
# --------------------------------------------------------------------------

def preconditioned_block_row(O, a, bc, k, N, p) -> np.ndarray:
    """Row block p of P^-1 A as a dense [2N+1, M(2N+1)] array, built from
    the section 4.2 blocks A^pq (L^pq or N^pq, whose (S^pq)^T factor is read
    from the separation generator) divided by the diagonal of A^pp."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    J, dJ, H, dH = bessel_diagonals(a, k, N)
    m = modes(N)
    idx = (m[None, :] - m[:, None]) + 2 * N      # (n - m) + 2N for entry (m, n)
    if bc[p] == DIRICHLET:
        left = J[p]
        diag = 0.5j * np.pi * a[p] * J[p] * H[p]
    else:
        left = k * dJ[p]
        diag = 0.5j * np.pi * k * a[p] * J[p] * dH[p]
    row = np.zeros((n, M, n), dtype=np.complex128)
    l = np.arange(-2 * N, 2 * N + 1)
    qs = np.array([q for q in range(M) if q != p], dtype=int)
    if len(qs):
        bv = O[p][None, :] - O[qs]
        b = np.hypot(bv[:, 0], bv[:, 1])
        al = np.arctan2(bv[:, 1], bv[:, 0])
        g = special.hankel1(l[None, :], k * b[:, None]) * np.exp(1j * l[None, :] * al[:, None])
        ST = g[:, idx]                                  # [q, m, n] = (S^pq)^T_mn
        coef = 0.5j * np.pi * np.sqrt(a[p] * a[qs])
        blocks = coef[:, None, None] * left[None, :, None] * ST * J[qs][:, None, :]
        row[:, qs, :] = np.transpose(blocks / diag[None, :, None], (1, 0, 2))
    row[:, p, :] = np.eye(n)
    return row.reshape(n, M * n)


def preconditioned_rows(O, a, bc, k, N, x, targets) -> np.ndarray:
    """Rows p in `targets` of (P^-1 A) x (see preconditioned_block_row).
    x is [N_tot, R]; returns [len(targets), 2N+1, R]."""
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[:, None]
    return np.stack([preconditioned_block_row(O, a, bc, k, N, p) @ x for p in targets], axis=0)


def preconditioned_dense(O, a, bc, k, N) -> np.ndarray:
    """P^-1 A assembled block row by block row (same definition as
    precondition(assemble(...)), faster for a few thousand unknowns)."""
    return np.concatenate([preconditioned_block_row(O, a, bc, k, N, p) for p in range(len(a))], axis=0)


def preconditioner_diagonal(a, bc, k, N) -> np.ndarray:
    """The diagonal of the blocks A^pp (section 5), [N_tot]."""
    a = np.asarray(a, dtype=np.float64)
    J, dJ, H, dH = bessel_diagonals(a, k, N)
    return np.where(np.asarray(bc)[:, None] == DIRICHLET,
                    0.5j * np.pi * a[:, None] * J * H,
                    0.5j * np.pi * k * a[:, None] * J * dH).reshape(-1)


def preconditioned_rhs(O, a, bc, k, N, betas) -> np.ndarray:
    """P^-1 b with P the diagonal of the blocks A^pp (section 5)."""
    return rhs_planewave(O, a, bc, k, N, betas) / preconditioner_diagonal(a, bc, k, N)[:, None]


def preconditioned_rhs_pointsource(O, a, bc, k, N, sources) -> np.ndarray:
    """P^-1 b for point sources."""
    return rhs_pointsource(O, a, bc, k, N, sources) / preconditioner_diagonal(a, bc, k, N)[:, None]


# --------------------------------------------------------------------------
# Section 4.4: potentials and far field
# --------------------------------------------------------------------------

def single_layer_potential(O, a, k, N, rho, points) -> np.ndarray:
    """Prop. 4.3: (L rho)(x) = sum_p sum_m rho^p_m (i pi a_p / 2) J_m(k a_p)
    H_m(k r_p(x)) exp(i m theta_p(x)) / sqrt(2 pi a_p), for x outside the
    disks.  rho is [N_tot] or [N_tot, R]; points [P, 2]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    rho = np.asarray(rho)
    squeeze = rho.ndim == 1
    R = rho.reshape(M, n, -1)
    pts = np.asarray(points, dtype=np.float64)
    J = bessel_diagonals(a, k, N)[0]
    m = modes(N)
    u = np.zeros((len(pts), R.shape[2]), dtype=np.complex128)
    for p in range(M):
        d = pts - O[p][None, :]
        r = np.hypot(d[:, 0], d[:, 1])
        th = np.arctan2(d[:, 1], d[:, 0])
        basis = special.hankel1(m[None, :], k * r[:, None]) * np.exp(1j * m[None, :] * th[:, None])
        coef = 0.5j * np.pi * a[p] * J[p] / np.sqrt(2 * np.pi * a[p])
        u += basis @ (coef[:, None] * R[p])
    return u[:, 0] if squeeze else u


def farfield_coefficients(O, a, k, N, theta) -> np.ndarray:
    """Section 4.4: (a_L)^p_m(theta) = i e^{-i pi/4} sqrt(a_p) / (2 sqrt k)
    exp(-i b_p k cos(theta - alpha_p)) J_m(k a_p) exp(i m (theta - pi/2)),
    with b_p = |O_p| and alpha_p its polar angle.  Returns [N_tot]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    J = bessel_diagonals(a, k, N)[0]
    m = modes(N)[None, :]
    bp = np.hypot(O[:, 0], O[:, 1])
    alp = np.arctan2(O[:, 1], O[:, 0])
    c = (1j * np.exp(-1j * np.pi / 4) * np.sqrt(a) / (2 * np.sqrt(k)))[:, None] \
        * np.exp(-1j * bp * k * np.cos(theta - alp))[:, None] * J * np.exp(1j * m * (theta - np.pi / 2))
    return c.reshape(-1)


def farfield(O, a, k, N, rho, thetas) -> np.ndarray:
    """Section 4.4: a_L(theta) = (a_L(theta))^T rho for every sample angle.
    rho [N_tot, R] -> F [T, R]."""
    rho = np.asarray(rho)
    if rho.ndim == 1:
        rho = rho[:, None]
    C = np.stack([farfield_coefficients(O, a, k, N, t) for t in np.atleast_1d(thetas)])
    return C @ rho


def dort_far_field_matrix(O, a, bc, k, N, n_alpha):
    """Section 7 (Example III, far-field time reversal): the mirror emits the
    plane waves of incidence alpha_j = 2 pi j / n_alpha (j = 0..n_alpha-1)
    and measures the far field in the opposite directions alpha_i + pi.
    Column j of F holds that measured far field for incidence alpha_j:
    F[i, j] = a_L(alpha_i + pi; alpha_j) (section 4.4), densities from the
    LU solve of the section 5 system.  Returns (alphas, F [n_alpha, n_alpha])."""
    alphas = 2.0 * np.pi * np.arange(n_alpha) / n_alpha
    rho, _ = solve(O, a, bc, k, N, alphas, method="lu")
    return alphas, farfield(O, a, k, N, rho, alphas + np.pi)


def time_reversal_matrix(F) -> np.ndarray:
    """Section 7: T = conj(F)^T F (Hermitian, positive semi-definite)."""
    F = np.asarray(F)
    return F.conj().T @ F


def dort_eigenvectors(T):
    """Section 7: eigenvalues (largest first) and eigenvectors (columns) of
    the Hermitian T (LAPACK)."""
    lam, V = np.linalg.eigh(T)
    return lam[::-1], V[:, ::-1]


def herglotz_wave(k, alphas, g, points) -> np.ndarray:
    """Section 7: the discrete Herglotz wave of parameter g emitted by the
    mirror, u_I(x) = sum_j h_alpha g_j exp(i k (x1 cos alpha_j + x2 sin alpha_j)),
    h_alpha = 2 pi / n_alpha.  points [P, 2] -> [P]."""
    alphas = np.asarray(alphas, dtype=np.float64)
    pts = np.asarray(points, dtype=np.float64)
    E = np.exp(1j * k * (np.outer(pts[:, 0], np.cos(alphas)) + np.outer(pts[:, 1], np.sin(alphas))))
    return (2 * np.pi / len(alphas)) * (E @ np.asarray(g))


def dort_eigenvalues(T) -> np.ndarray:
    """Section 7: the eigenvalues of T (LAPACK Hermitian solver), largest
    first."""
    return np.linalg.eigvalsh(T)[::-1]


def rcs(F) -> np.ndarray:
    """Section 4.4: RCS = 10 log10(2 pi |a|^2) in dB."""
    return 10.0 * np.log10(2 * np.pi * np.abs(F) ** 2)


# --------------------------------------------------------------------------
# Other integral equations (section 3, "a few boundary integral equations";
# section 4.2 blocks M and D; section 5 linear combinations)
# --------------------------------------------------------------------------

OPERATORS = ("I", "L", "M", "N", "D")


def block_M(O, a, k, N, p, q) -> np.ndarray:
    """Section 4.2, block M^pq of the trace of the double-layer potential:
    -I/2 - (i pi k a_p / 2) J^p H'^p on the diagonal,
    -(i k pi sqrt(a_p a_q) / 2) J^p (S^pq)^T J'^q off it."""
    J, dJ, H, dH = bessel_diagonals(a, k, N)
    if p == q:
        return -0.5 * np.eye(2 * N + 1) - np.diag(0.5j * np.pi * k * a[p] * J[p] * dH[p])
    S = separation_matrix(O[p], O[q], k, N)
    return -0.5j * k * np.pi * np.sqrt(a[p] * a[q]) * (J[p][:, None] * S.T * dJ[q][None, :])


def block_D(O, a, k, N, p, q) -> np.ndarray:
    """Section 4.2, block D^pq of the normal-derivative trace of the
    double-layer potential: -(i pi k^2 a_p / 2) J'^p H'^p on the diagonal,
    -(i k^2 pi sqrt(a_p a_q) / 2) J'^p (S^pq)^T J'^q off it.  The diagonal
    sign is the one the definition D lambda = -d_nx int d_ny G lambda (the
    normal derivative of the double-layer potential of Prop. 4.3, continuous
    across the circle) gives; the printed diagonal has the opposite sign,
    while the printed off-diagonal blocks agree with the definition."""
    J, dJ, H, dH = bessel_diagonals(a, k, N)
    if p == q:
        return np.diag(-0.5j * np.pi * k * k * a[p] * dJ[p] * dH[p])
    S = separation_matrix(O[p], O[q], k, N)
    return -0.5j * k * k * np.pi * np.sqrt(a[p] * a[q]) * (dJ[p][:, None] * S.T * dJ[q][None, :])


def block_of(kind, O, a, k, N, p, q) -> np.ndarray:
    """The block (p, q) of I, L, M, N or D (section 4.2)."""
    if kind == "I":
        return np.eye(2 * N + 1) if p == q else np.zeros((2 * N + 1, 2 * N + 1))
    return {"L": block_L, "M": block_M, "N": block_N, "D": block_D}[kind](O, a, k, N, p, q)


def standard_formulation(kind, alpha=0.5, eta=None, k=None):
    """Section 3 (and the section 5 CFIE system): the weights of the named
    integral equations, as (op_weights, rhs_weights, rep_weights) for
    assemble_formulation / rhs_formulation / farfield_formulation.
    Sound-soft rows:
      "efie"  L rho = -U;
      "mfie"  (I/2 + N) rho = -dU;
      "cfie"  [alpha eta L + (1 - alpha)(I/2 + N)] rho = -(alpha eta U + (1 - alpha) dU);
      "bwie"  (I/2 - eta L - M) psi = -U with u = -(eta L + M) psi.
    Sound-hard rows: (-I/2 + N) rho = -dU for the three single-layer
    representations (u = L rho); for Brakhage-Werner the normal trace of its
    representation, (eta I/2 - eta N - D) psi = -dU.  eta defaults to i k
    (the paper leaves eta free with Im(eta) != 0)."""
    if eta is None and kind in ("cfie", "bwie"):
        eta = 1j * k
    if kind == "bwie":
        return ({DIRICHLET: {"I": 0.5, "L": -eta, "M": -1.0}, NEUMANN: {"I": 0.5 * eta, "N": -eta, "D": -1.0}},
                {DIRICHLET: {"U": 1.0}, NEUMANN: {"dU": 1.0}}, {"L": -eta, "M": -1.0})
    hard_rows, hard_rhs = {"I": -0.5, "N": 1.0}, {"dU": 1.0}
    soft = {"efie": ({"L": 1.0}, {"U": 1.0}),
            "mfie": ({"I": 0.5, "N": 1.0}, {"dU": 1.0}),
            "cfie": ({"L": alpha * eta, "I": 0.5 * (1 - alpha), "N": 1 - alpha},
                     {"U": alpha * eta, "dU": 1 - alpha}) if kind == "cfie" else None}
    if kind not in soft:
        raise ValueError(kind)
    rows, rhs = soft[kind]
    return {DIRICHLET: rows, NEUMANN: hard_rows}, {DIRICHLET: rhs, NEUMANN: hard_rhs}, {"L": 1.0, "M": 0.0}


def assemble_formulation(O, a, bc, k, N, op_weights) -> np.ndarray:
    """Section 5: the matrix of a linear combination of I, L, M, N and D
    (the same block structure for every combination).  op_weights[c] maps
    each operator name to its weight for the rows of disks with boundary
    condition c (DIRICHLET or NEUMANN)."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    A = np.zeros((M * n, M * n), dtype=np.complex128)
    for p in range(M):
        w = op_weights[int(bc[p])]
        for q in range(M):
            B = np.zeros((n, n), dtype=np.complex128)
            for kind in OPERATORS:
                if w.get(kind, 0) != 0:
                    B = B + w[kind] * block_of(kind, O, a, k, N, p, q)
            A[p * n:(p + 1) * n, q * n:(q + 1) * n] = B
    return A


def rhs_formulation(O, a, bc, k, N, betas, rhs_weights) -> np.ndarray:
    """Section 5: b = -(w_U U + w_dU dU) for plane waves (Prop. 4.1),
    rhs_weights[c] = {"U": w_U, "dU": w_dU} for the rows of boundary
    condition c.  [N_tot, R]."""
    a = np.asarray(a, dtype=np.float64)
    J, dJ, _, _ = bessel_diagonals(a, k, N)
    cols = []
    for beta in np.atleast_1d(betas):
        d = planewave_coefficients(O, a, k, N, beta)
        U, dU = d * J, k * d * dJ
        b = np.zeros_like(U)
        for p in range(len(a)):
            w = rhs_weights[int(bc[p])]
            b[p] = -(w.get("U", 0) * U[p] + w.get("dU", 0) * dU[p])
        cols.append(b.reshape(-1))
    return np.stack(cols, axis=1)


def double_layer_potential(O, a, k, N, lam, points) -> np.ndarray:
    """Prop. 4.3: (M lambda)(x) = -sum_p sum_m lambda^p_m (i pi k a_p / 2)
    J'_m(k a_p) H_m(k r_p(x)) exp(i m theta_p(x)) / sqrt(2 pi a_p), for x
    outside the disks."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    lam = np.asarray(lam)
    squeeze = lam.ndim == 1
    R = lam.reshape(M, n, -1)
    pts = np.asarray(points, dtype=np.float64)
    dJ = bessel_diagonals(a, k, N)[1]
    m = modes(N)
    u = np.zeros((len(pts), R.shape[2]), dtype=np.complex128)
    for p in range(M):
        d = pts - O[p][None, :]
        r = np.hypot(d[:, 0], d[:, 1])
        th = np.arctan2(d[:, 1], d[:, 0])
        basis = special.hankel1(m[None, :], k * r[:, None]) * np.exp(1j * m[None, :] * th[:, None])
        coef = -0.5j * np.pi * k * a[p] * dJ[p] / np.sqrt(2 * np.pi * a[p])
        u += basis @ (coef[:, None] * R[p])
    return u[:, 0] if squeeze else u


def farfield_coefficients_M(O, a, k, N, theta) -> np.ndarray:
    """Section 4.4, double-layer far-field vector a_M(theta):
    -i e^{-i pi/4} sqrt(k a_p) / 2 exp(-i b_p k cos(theta - alpha_p))
    J'_m(k a_p) exp(i m (theta - pi/2)).  The sign is the one the large-r
    limit of the double-layer potential of Prop. 4.3 gives (the printed
    vector has the opposite sign).  Returns [N_tot]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    dJ = bessel_diagonals(a, k, N)[1]
    m = modes(N)[None, :]
    bp = np.hypot(O[:, 0], O[:, 1])
    alp = np.arctan2(O[:, 1], O[:, 0])
    c = (-1j * np.exp(-1j * np.pi / 4) * np.sqrt(k * a) / 2)[:, None] \
        * np.exp(-1j * bp * k * np.cos(theta - alp))[:, None] * dJ * np.exp(1j * m * (theta - np.pi / 2))
    return c.reshape(-1)


def farfield_formulation(O, a, k, N, dens, thetas, rep_weights) -> np.ndarray:
    """Section 4.4 for the representation u = w_L L dens + w_M M dens:
    a(theta) = w_L a_L(theta)^T dens + w_M a_M(theta)^T dens.  [T, R]."""
    dens = np.asarray(dens)
    if dens.ndim == 1:
        dens = dens[:, None]
    th = np.atleast_1d(thetas)
    C = np.stack([rep_weights.get("L", 0) * farfield_coefficients(O, a, k, N, t)
                  + rep_weights.get("M", 0) * farfield_coefficients_M(O, a, k, N, t) for t in th])
    return C @ dens


def potential_formulation(O, a, k, N, dens, points, rep_weights) -> np.ndarray:
    """Prop. 4.3: u = w_L L dens + w_M M dens at points outside the disks."""
    u = 0
    if rep_weights.get("L", 0) != 0:
        u = u + rep_weights["L"] * single_layer_potential(O, a, k, N, dens, points)
    if rep_weights.get("M", 0) != 0:
        u = u + rep_weights["M"] * double_layer_potential(O, a, k, N, dens, points)
    return u


def solve_formulation(O, a, bc, k, N, betas, op_weights, rhs_weights) -> np.ndarray:
    """Section 5: LU solve of a formulation's system (no preconditioning
    needed for the direct solve).  [N_tot, R]."""
    A = assemble_formulation(O, a, bc, k, N, op_weights)
    b = rhs_formulation(O, a, bc, k, N, betas, rhs_weights)
    return np.linalg.solve(A, b)


def preconditioned_formulation(O, a, bc, k, N, op_weights):
    """P^-1 A of a formulation, P its diagonal blocks (diagonal matrices for
    every combination of I, L, M, N, D)."""
    A = assemble_formulation(O, a, bc, k, N, op_weights)
    d = np.diag(A).copy()
    M = len(np.asarray(a))
    n = 2 * N + 1
    for p in range(M):
        blk = A[p * n:(p + 1) * n, p * n:(p + 1) * n]
        assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
    return A / d[:, None], d


# --------------------------------------------------------------------------
# Penetrable obstacles (section 7, Example II: the transmission problem)
# --------------------------------------------------------------------------

def assemble_penetrable(O, a, k_plus, k_minus, mu, N) -> np.ndarray:
    """Section 7, transmission system for u+ = L+ rho+ outside and
    u- = L- rho- inside the disks (single layers at k+ and k-):
        [ L+           -L-            ] [rho+]   [ -U  ]
        [ -I/2 + N+    -mu (I/2 + N-) ] [rho-] = [ -dU ],
    rows: the traces u+ - u- = -u_inc and mu-weighted normal traces
    d_n u+ - mu d_n u- = -d_n u_inc on every circle (mu per disk, its row);
    the interior normal trace of L- rho- is (I/2 + N-) rho- (Prop. 3.2), hence
    the minus sign in the (2, 2) block.  [2 N_tot, 2 N_tot]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    mu = np.broadcast_to(np.asarray(mu, dtype=np.complex128), (M,))
    Nt = M * n
    A = np.zeros((2 * Nt, 2 * Nt), dtype=np.complex128)
    for p in range(M):
        rs = slice(p * n, (p + 1) * n)
        rn = slice(Nt + p * n, Nt + (p + 1) * n)
        for q in range(M):
            cp = slice(q * n, (q + 1) * n)
            cm = slice(Nt + q * n, Nt + (q + 1) * n)
            A[rs, cp] = block_L(O, a, k_plus, N, p, q)
            A[rs, cm] = -block_L(O, a, k_minus, N, p, q)
            Bp = block_N(O, a, k_plus, N, p, q)
            Bm = block_N(O, a, k_minus, N, p, q)
            if p == q:
                Bp = Bp - 0.5 * np.eye(n)
                Bm = Bm + 0.5 * np.eye(n)
            A[rn, cp] = Bp
            A[rn, cm] = -mu[p] * Bm
    return A


def rhs_penetrable(O, a, k_plus, N, betas) -> np.ndarray:
    """Section 7: [-U; -dU] of the plane waves at k+ (Prop. 4.1).
    [2 N_tot, R]."""
    a = np.asarray(a, dtype=np.float64)
    J, dJ, _, _ = bessel_diagonals(a, k_plus, N)
    cols = []
    for beta in np.atleast_1d(betas):
        d = planewave_coefficients(O, a, k_plus, N, beta)
        cols.append(np.concatenate([-(d * J).reshape(-1), -(k_plus * d * dJ).reshape(-1)]))
    return np.stack(cols, axis=1)


def rhs_penetrable_pointsource(O, a, k_plus, N, sources) -> np.ndarray:
    """Section 7 with the point-source incident wave of section 4.3:
    [-U; -dU] with U = d' J, dU = k+ d' J' at k+.  [2 N_tot, R]."""
    a = np.asarray(a, dtype=np.float64)
    J, dJ, _, _ = bessel_diagonals(a, k_plus, N)
    cols = []
    for s in np.atleast_2d(np.asarray(sources, dtype=np.float64)):
        d = pointsource_coefficients(O, a, k_plus, N, s)
        cols.append(np.concatenate([-(d * J).reshape(-1), -(k_plus * d * dJ).reshape(-1)]))
    return np.stack(cols, axis=1)


def solve_penetrable(O, a, k_plus, k_minus, mu, N, betas):
    """LU solve of the transmission system; returns (rho+, rho-), each
    [N_tot, R]."""
    A = assemble_penetrable(O, a, k_plus, k_minus, mu, N)
    x = np.linalg.solve(A, rhs_penetrable(O, a, k_plus, N, betas))
    Nt = A.shape[0] // 2
    return x[:Nt], x[Nt:]


def preconditioned_penetrable(O, a, k_plus, k_minus, mu, N):
    """B^-1 A with B the 2 x 2 self blocks of every (disk, mode): the
    trace and normal rows of a mode couple its rho+ and rho- entries
    only, so B is a 2 x 2 matrix per mode.  Returns (B^-1 A, B [N_tot, 2, 2])."""
    A = assemble_penetrable(O, a, k_plus, k_minus, mu, N)
    Nt = A.shape[0] // 2
    i = np.arange(Nt)
    B = np.stack([np.stack([A[i, i], A[i, Nt + i]], -1), np.stack([A[Nt + i, i], A[Nt + i, Nt + i]], -1)], -2)
    Binv = np.linalg.inv(B)
    P = np.zeros_like(A)
    P[i, i], P[i, Nt + i] = Binv[:, 0, 0], Binv[:, 0, 1]
    P[Nt + i, i], P[Nt + i, Nt + i] = Binv[:, 1, 0], Binv[:, 1, 1]
    return P @ A, B


def single_layer_potential_inside(O, a, k, N, rho, points, p) -> np.ndarray:
    """Prop. 4.3 for points x inside disk p: the self term takes the
    interior expansion (i pi a_p/2) H_m(k a_p) J_m(k r_p) exp(i m theta_p)
    / sqrt(2 pi a_p) (Graf's theorem with the roles of x and y exchanged),
    the other disks their exterior expansion."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    M = len(a)
    n = 2 * N + 1
    rho = np.asarray(rho)
    squeeze = rho.ndim == 1
    R = rho.reshape(M, n, -1)
    pts = np.asarray(points, dtype=np.float64)
    J, _, H, _ = bessel_diagonals(a, k, N)
    m = modes(N)
    u = np.zeros((len(pts), R.shape[2]), dtype=np.complex128)
    for q in range(M):
        d = pts - O[q][None, :]
        r = np.hypot(d[:, 0], d[:, 1])
        th = np.arctan2(d[:, 1], d[:, 0])
        if q == p:
            basis = special.jv(m[None, :], k * r[:, None]) * np.exp(1j * m[None, :] * th[:, None])
            coef = 0.5j * np.pi * a[q] * H[q] / np.sqrt(2 * np.pi * a[q])
        else:
            basis = special.hankel1(m[None, :], k * r[:, None]) * np.exp(1j * m[None, :] * th[:, None])
            coef = 0.5j * np.pi * a[q] * J[q] / np.sqrt(2 * np.pi * a[q])
        u += basis @ (coef[:, None] * R[q])
    return u[:, 0] if squeeze else u


# --------------------------------------------------------------------------
# Section 5: truncation rule (eq. Np)
# --------------------------------------------------------------------------

def truncation_order(ka: float, eps: float) -> int:
    """Eq. (Np): N_p = [k a_p + ((1/(2 sqrt 2)) ln(2 sqrt 2 pi k a_p / eps))^(2/3)
    (k a_p)^(1/3) + 1], [.] the integer part."""
    t = (np.log(2 * np.sqrt(2) * np.pi * ka / eps) / (2 * np.sqrt(2))) ** (2.0 / 3.0)
    return int(np.floor(ka + t * ka ** (1.0 / 3.0) + 1))


# --------------------------------------------------------------------------
# Section 5: per-disk truncation orders N_p (blocks of size (2N_p+1) x (2N_q+1))
# --------------------------------------------------------------------------

def ragged_offsets(Ns) -> np.ndarray:
    """Row offset of each disk's modes -N_p..N_p in the ragged unknown vector
    (disk after disk); the last entry is N_tot = sum (2 N_p + 1)."""
    return np.concatenate([[0], np.cumsum(2 * np.asarray(Ns, dtype=int) + 1)])


def assemble_ragged(O, a, bc, k, Ns) -> np.ndarray:
    """Section 5 with a truncation order N_p per disk: the truncated system
    keeps modes -N_p..N_p on disk p, so block (p, q) is (2N_p+1) x (2N_q+1).
    Sound-soft rows: L^pq with entries (i pi sqrt(a_p a_q)/2) J_m(k a_p)
    H_{n-m}(k b_pq) e^{i (n-m) alpha_pq} J_n(k a_q) (section 4.2, (S^pq)^T),
    diagonal (i pi a_p/2) J_m H_m; sound-hard rows: k J'_m(k a_p) in place
    of J_m(k a_p) off the diagonal and (i pi k a_p/2) J_m H'_m on it
    (the exterior trace -I/2 + N, reading of the module header)."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    Ns = np.asarray(Ns, dtype=int)
    off = ragged_offsets(Ns)
    A = np.zeros((off[-1], off[-1]), dtype=np.complex128)
    for p in range(len(a)):
        m = modes(Ns[p])
        Jp, dJp = special.jv(m, k * a[p]), special.jvp(m, k * a[p])
        Hp, dHp = special.hankel1(m, k * a[p]), special.h1vp(m, k * a[p])
        left = Jp if bc[p] == DIRICHLET else k * dJp
        for q in range(len(a)):
            if p == q:
                d = Jp * Hp * 0.5j * np.pi * a[p] if bc[p] == DIRICHLET else 0.5j * np.pi * k * a[p] * Jp * dHp
                A[off[p]:off[p + 1], off[p]:off[p + 1]] = np.diag(d)
                continue
            nn = modes(Ns[q])
            _, b, alpha = pair_vector(O[p], O[q])
            l = nn[None, :] - m[:, None]
            ST = special.hankel1(l, k * b) * np.exp(1j * l * alpha)
            Jq = special.jv(nn, k * a[q])
            A[off[p]:off[p + 1], off[q]:off[q + 1]] = \
                0.5j * np.pi * np.sqrt(a[p] * a[q]) * left[:, None] * ST * Jq[None, :]
    return A


def rhs_ragged(O, a, bc, k, Ns, betas) -> np.ndarray:
    """Prop. 4.1 with N_p modes per disk: -U (sound-soft rows, d^p_m J_m) or
    -dU (sound-hard rows, k d^p_m J'_m), [N_tot, R]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    off = ragged_offsets(Ns)
    b = np.zeros((off[-1], len(np.atleast_1d(betas))), dtype=np.complex128)
    for r, beta in enumerate(np.atleast_1d(betas)):
        for p in range(len(a)):
            m = modes(Ns[p])
            phase = k * (np.cos(beta) * O[p, 0] + np.sin(beta) * O[p, 1])
            d = np.sqrt(2 * np.pi * a[p]) * np.exp(1j * phase) * np.exp(1j * m * (np.pi / 2 - beta))
            trace = special.jv(m, k * a[p]) if bc[p] == DIRICHLET else k * special.jvp(m, k * a[p])
            b[off[p]:off[p + 1], r] = -d * trace
    return b


def solve_ragged(O, a, bc, k, Ns, betas) -> np.ndarray:
    """Section 5: LU solve of the ragged system (the diagonal preconditioner
    does not change the solution)."""
    return np.linalg.solve(assemble_ragged(O, a, bc, k, Ns), rhs_ragged(O, a, bc, k, Ns, betas))


def preconditioned_ragged(O, a, bc, k, Ns) -> np.ndarray:
    """P^-1 A of the ragged system, P its diagonal (section 5)."""
    A = assemble_ragged(O, a, bc, k, Ns)
    return A / np.diag(A)[:, None]


def farfield_ragged(O, a, k, Ns, rho, thetas) -> np.ndarray:
    """Section 4.4 with N_p modes per disk: a_L(theta) = sum_p sum_m
    i e^{-i pi/4} sqrt(a_p)/(2 sqrt k) e^{-i k |O_p| cos(theta - alpha_p)}
    J_m(k a_p) e^{i m (theta - pi/2)} rho^p_m.  rho [N_tot, R] -> [T, R]."""
    O = np.asarray(O, dtype=np.float64)
    a = np.asarray(a, dtype=np.float64)
    off = ragged_offsets(Ns)
    rho = np.asarray(rho)
    if rho.ndim == 1:
        rho = rho[:, None]
    th = np.atleast_1d(np.asarray(thetas, dtype=np.float64))
    F = np.zeros((len(th), rho.shape[1]), dtype=np.complex128)
    for p in range(len(a)):
        m = modes(Ns[p])
        bp, alp = np.hypot(O[p, 0], O[p, 1]), np.arctan2(O[p, 1], O[p, 0])
        c = (1j * np.exp(-1j * np.pi / 4) * np.sqrt(a[p]) / (2 * np.sqrt(k))) \
            * np.exp(-1j * bp * k * np.cos(th - alp))[:, None] * special.jv(m, k * a[p])[None, :] \
            * np.exp(1j * m[None, :] * (th[:, None] - np.pi / 2))
        F += c @ rho[off[p]:off[p + 1]]
    return F
