"""The seeded workloads draw what their docstrings state (CPU)."""
import numpy as np

from paper_1409_8186_gb300 import workloads as W


def min_gap(cl):
    d = np.hypot(cl.centres[:, None, 0] - cl.centres[None, :, 0], cl.centres[:, None, 1] - cl.centres[None, :, 1])
    d = d - cl.radii[:, None] - cl.radii[None, :]
    np.fill_diagonal(d, np.inf)
    return d.min()


def test_penetrable_lattice():
    cl = W.penetrable_lattice()
    assert cl.M == 400 and cl.k == 1.0 and cl.N == 10
    assert np.all(cl.radii == 1.0)
    assert min_gap(cl) > 0.99  # spacing 3, unit disks
    # the middle row and column are empty: the source at the origin is outside every disk
    assert np.all(cl.centres[:, 0] != 0) and np.all(cl.centres[:, 1] != 0)
    assert np.hypot(cl.centres[:, 0], cl.centres[:, 1]).min() > 4.2
    assert np.allclose(cl.centres.mean(axis=0), 0)


def test_time_reversal_disks():
    for bc in (W.DIRICHLET, W.NEUMANN):
        cl = W.dort_three_disks(bc)
        assert cl.M == 3 and np.all(cl.bc == bc)
        assert np.allclose(cl.k, 2 * np.pi)
        assert (cl.k * cl.radii).max() < 0.13  # small obstacles
        assert min_gap(cl) > 20


def test_random_clusters_do_not_overlap():
    for cl in (W.random_cluster_400(), W.small_mixed(seed=3, M=6, N=10, k=2.0),
               W.random_cluster(seed=8, M=70, half_side=14.0, rmin=0.5, rmax=1.0, gap=0.2, k=2.5, N=8)):
        assert min_gap(cl) >= 0.2 - 1e-12 or cl.M < 10
        assert min_gap(cl) > 0
