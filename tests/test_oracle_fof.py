"""Pins for the friends-of-friends oracle (oracle.fof): brute force on small
sets, chains just inside and outside the linking length, linking across the
periodic boundary, the minimum-size threshold, well-separated clumps, lattices
and relabelling invariance."""
import numpy as np
import pytest

from oracle import fof
from workloads import generators as gen


def _brute_fof(pos, box, link, min_members):
    # O(n^2) pair test and a plain union-find, independent of the k-d tree
    # and of the graph library
    x = np.mod(pos, box)
    n = len(x)
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for i in range(n):
        for j in range(i + 1, n):
            s = 0.0
            for a in range(3):
                d = x[j, a] - x[i, a]
                d = d - box * round(d / box)
                s += d * d
            if s < link * link:
                ri, rj = find(i), find(j)
                if ri != rj:
                    parent[max(ri, rj)] = min(ri, rj)
    roots = np.array([find(i) for i in range(n)])
    return fof.canonical_labels(roots, min_members)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_matches_brute_force(seed):
    L = 6.0
    pos, _, _ = gen.nfw_clustered(400, L, seed, m_lo=20.0, m_hi=150.0)
    for link in (0.15, 0.3):
        lab, sizes = fof.fof(pos, L, link, min_members=5)
        lab_b, sizes_b = _brute_fof(pos, L, link, 5)
        np.testing.assert_array_equal(lab, lab_b)
        np.testing.assert_array_equal(sizes, sizes_b)


def test_chain_inside_and_outside_the_linking_length():
    L, link = 20.0, 0.2
    line = np.zeros((50, 3)) + 5.0
    line[:, 0] = 3.0 + np.arange(50) * 0.99 * link
    lab, sizes = fof.fof(line, L, link, min_members=2)
    assert np.all(lab == 0) and list(sizes) == [50]
    line[:, 0] = 3.0 + np.arange(50) * 1.01 * link
    lab, sizes = fof.fof(line, L, link, min_members=2)
    assert np.all(lab == -1) and len(sizes) == 0


def test_links_across_the_periodic_boundary():
    L, link = 10.0, 0.3
    pts = np.array([[9.9, 5.0, 5.0], [0.1, 5.0, 5.0], [0.35, 5.0, 5.0], [5.0, 9.95, 0.02],
                    [5.0, 0.1, 9.9]])
    lab, sizes = fof.fof(pts, L, link, min_members=2)
    np.testing.assert_array_equal(lab, [0, 0, 0, 1, 1])
    np.testing.assert_array_equal(sizes, [3, 2])


def test_minimum_size_threshold_and_clumps():
    # two dense clumps of 39 and 40 particles in an empty box, far apart
    rng = np.random.default_rng(4)
    L, link = 50.0, 0.2
    a = 10.0 + rng.normal(0.0, 0.02, (39, 3))
    b = 30.0 + rng.normal(0.0, 0.02, (40, 3))
    pos = np.vstack([b, a])
    lab, sizes = fof.fof(pos, L, link, min_members=40)
    assert np.all(lab[:40] == 0) and np.all(lab[40:] == -1) and list(sizes) == [40]
    lab, sizes = fof.fof(pos, L, link, min_members=39)
    assert list(sizes) == [40, 39] and np.all(lab[40:] == 1)


def test_lattice_links_all_or_nothing():
    pos = gen.lattice(8, 8.0)
    lab, _ = fof.fof(pos, 8.0, 0.99, min_members=2)
    assert np.all(lab == -1)
    lab, sizes = fof.fof(pos, 8.0, 1.01, min_members=2)
    assert np.all(lab == 0) and list(sizes) == [512]


def test_relabelling_invariance():
    L = 12.0
    pos, _, _ = gen.nfw_clustered(3000, L, 9, m_lo=40.0, m_hi=600.0)
    lab, sizes = fof.fof(pos, L, 0.2, min_members=20)
    perm = np.random.default_rng(1).permutation(len(pos))
    lab_p, sizes_p = fof.fof(pos[perm], L, 0.2, min_members=20)
    # the same partition (halo ids may be renumbered) and the same sizes
    assert sorted(sizes) == sorted(sizes_p)
    m = lab >= 0
    assert np.array_equal(m[perm], lab_p >= 0)
    pairs = {}
    for a, b in zip(lab[perm][m[perm]], lab_p[m[perm]]):
        assert pairs.setdefault(a, b) == b
