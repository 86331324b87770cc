"""Pins of the oracle's per-disk truncation (section 5: modes -N_p..N_p on
disk p, blocks of size (2N_p+1) x (2N_q+1)).

* Each rectangular off-diagonal block against brute-force trapezoidal
  quadrature of its Galerkin integral (kernel G for sound-soft rows, d_n G
  for sound-hard rows) with different mode ranges on the two circles (1e-12).
* Equal orders on every disk give the uniform system exactly.
* The ragged system is a consistent discretisation: raising every N_p by
  4 and 8 the far field converges spectrally (more than 20x per 4 modes)
  towards a uniform solve with many more modes.
* The right-hand side and the far field of one disk are the Mie series cut
  at its own N_p.
* Planted mistakes (transposed shift n - m -> m - n; the column Bessel
  factor taken on the target disk) fail the quadrature pin.
"""
import numpy as np
import pytest
from scipy import special

import oracle.msd_oracle as O_
from paper_1409_8186_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def circle(Oc, a, Q):
    t = 2 * np.pi * np.arange(Q) / Q
    return t, Oc[None, :] + a * np.stack([np.cos(t), np.sin(t)], axis=1)


def quadrature_block(Op, ap, Np, Oq, aq, Nq, k, kind, Q=160):
    """(K Phi^q_n, Phi^p_m) for m = -Np..Np, n = -Nq..Nq by the trapezoidal
    rule on both circles (hermitian product, section 4.1); K = G (L) or
    d/dn_x G (N)."""
    tp, X = circle(Op, ap, Q)
    tq, Y = circle(Oq, aq, Q)
    D = X[:, None, :] - Y[None, :, :]
    r = np.hypot(D[..., 0], D[..., 1])
    if kind == "L":
        K = 0.25j * special.hankel1(0, k * r)
    else:
        nx = np.stack([np.cos(tp), np.sin(tp)], axis=1)
        K = -0.25j * k * special.hankel1(1, k * r) * (D[..., 0] * nx[:, None, 0] + D[..., 1] * nx[:, None, 1]) / r
    m, n = np.arange(-Np, Np + 1), np.arange(-Nq, Nq + 1)
    phq = np.exp(1j * np.outer(tq, n)) / np.sqrt(2 * np.pi * aq) * (aq * 2 * np.pi / Q)
    php = np.exp(1j * np.outer(tp, m)) / np.sqrt(2 * np.pi * ap) * (ap * 2 * np.pi / Q)
    return php.conj().T @ K @ phq


def three_disks():
    O = np.array([[0.2, -0.1], [-2.6, 1.3], [1.9, 2.4]])
    a = np.array([0.6, 1.1, 0.4])
    return O, a, np.array([0, 1, 0], np.int8), 1.7, np.array([5, 9, 3])


def ragged_block_errors(assemble):
    O, a, bc, k, Ns = three_disks()
    A = assemble(O, a, bc, k, Ns)
    off = O_.ragged_offsets(Ns)
    worst = 0.0
    for p in range(3):
        for q in range(3):
            if p == q:
                continue
            ref = quadrature_block(O[p], a[p], Ns[p], O[q], a[q], Ns[q], k, "L" if bc[p] == 0 else "N")
            blk = A[off[p]:off[p + 1], off[q]:off[q + 1]]
            worst = max(worst, np.abs(blk - ref).max() / np.abs(ref).max())
    return worst


def test_ragged_blocks_match_quadrature():
    assert ragged_block_errors(O_.assemble_ragged) < 1e-12


def test_equal_orders_give_the_uniform_system():
    O, a, bc, k, _ = three_disks()
    A = O_.assemble_ragged(O, a, bc, k, [7, 7, 7])
    A0 = O_.assemble(O, a, bc, k, 7)
    assert np.abs(A - A0).max() <= 1e-15 * np.abs(A0).max()
    b = O_.rhs_ragged(O, a, bc, k, [7, 7, 7], [0.3, 1.2])
    assert np.abs(b - O_.rhs_planewave(O, a, bc, k, 7, [0.3, 1.2])).max() <= 1e-15 * np.abs(b).max()


def test_ragged_truncation_converges_spectrally():
    rng = np.random.default_rng(12)
    O, a = W.random_disks(rng, 8, 7.0, 0.2, 1.6, 0.3)
    bc = (rng.uniform(size=8) < 0.5).astype(np.int8)
    k, th = 3.0, W.angles(64)
    Ns = np.array([O_.truncation_order(k * ai, 1e-6) for ai in a])
    ref, _ = O_.solve(O, a, bc, k, int(Ns.max()) + 20, [0.4], method="lu")
    Fr = O_.farfield(O, a, k, int(Ns.max()) + 20, ref, th)
    errs = []
    for s in (0, 4, 8):
        rho = O_.solve_ragged(O, a, bc, k, Ns + s, [0.4])
        F = O_.farfield_ragged(O, a, k, Ns + s, rho, th)
        errs.append(np.abs(F - Fr).max() / np.abs(Fr).max())
    assert errs[0] < 1e-4 and errs[1] < errs[0] / 20 and errs[2] < errs[1] / 20, errs


def test_single_disk_ragged_is_the_mie_series():
    a, k, beta = 0.9, 2.2, 0.5
    for bc in (0, 1):
        N = 14
        rho = O_.solve_ragged(np.zeros((1, 2)), np.array([a]), np.array([bc], np.int8), k, [N], [beta])
        th = W.angles(20)
        F = O_.farfield_ragged(np.zeros((1, 2)), np.array([a]), k, [N], rho, th)[:, 0]
        m = np.arange(-40, 41)
        ratio = special.jvp(m, k * a) / special.h1vp(m, k * a) if bc else special.jv(m, k * a) / special.hankel1(m, k * a)
        mie = -np.exp(-1j * np.pi / 4) * np.sqrt(2 / (np.pi * k)) * (np.exp(1j * np.outer(th - beta, m)) @ ratio)
        assert np.abs(F - mie).max() <= 1e-10 * np.abs(mie).max(), bc


def _transposed(O, a, bc, k, Ns):
    """Planted: (S^pq)^T read with n - m replaced by m - n."""
    A = O_.assemble_ragged(O, a, bc, k, Ns)
    off = O_.ragged_offsets(Ns)
    for p in range(len(a)):
        for q in range(len(a)):
            if p == q:
                continue
            m, n = O_.modes(Ns[p]), O_.modes(Ns[q])
            _, b, al = O_.pair_vector(O[p], O[q])
            l = m[:, None] - n[None, :]
            left = special.jv(m, k * a[p]) if bc[p] == 0 else k * special.jvp(m, k * a[p])
            A[off[p]:off[p + 1], off[q]:off[q + 1]] = 0.5j * np.pi * np.sqrt(a[p] * a[q]) * left[:, None] * \
                special.hankel1(l, k * b) * np.exp(1j * l * al) * special.jv(n, k * a[q])[None, :]
    return A


def _wrong_column_disk(O, a, bc, k, Ns):
    """Planted: the column factor J_n evaluated at k a_p instead of k a_q."""
    A = O_.assemble_ragged(O, a, bc, k, Ns)
    off = O_.ragged_offsets(Ns)
    for p in range(len(a)):
        for q in range(len(a)):
            if p == q:
                continue
            n = O_.modes(Ns[q])
            A[off[p]:off[p + 1], off[q]:off[q + 1]] *= (special.jv(n, k * a[p]) / special.jv(n, k * a[q]))[None, :]
    return A


@pytest.mark.parametrize("bad", [_transposed, _wrong_column_disk])
def test_planted_ragged_mistakes_are_caught(bad):
    assert ragged_block_errors(bad) > 1e-3
