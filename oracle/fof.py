"""Friends-of-friends halo finding (FP64 oracle).

The paper identifies halos with a friends-of-friends (FOF) finder (Sec. 2.2,
Sec. 3.3): two particles are friends when closer than the linking length,
b times the mean inter-particle spacing (b = 0.168 fiducial, 0.2 for the
mass-function runs); halos are the groups of particles connected by
friendship, kept down to 40 particles.  Readings:

- friends iff s < link^2, with d = x_j - x_i after folding both into
  [0, L) (numpy's modulo), d <- d - L round(d / L) per axis (minimum
  image), s = (dx dx + dy dy) + dz dz, each operation rounded in binary64
  in that order (the device path takes the same decision the same way);
- the linking length is an input (the caller forms b * L / N^(1/3));
- a group's tag is its smallest particle index; groups with at least
  min_members particles become halos, numbered 0, 1, ... in increasing
  order of their tags; other particles get label -1.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

from .force import _wrap_for_tree


def friend_pairs(pos, box, link):
    """Index pairs (i < j) of friends, by the exact binary64 predicate."""
    x = _wrap_for_tree(pos, box)
    tree = cKDTree(x, boxsize=box)
    cand = tree.query_pairs(link * (1.0 + 1e-6), output_type="ndarray")   # superset
    if len(cand) == 0:
        return cand.reshape(0, 2)
    i, j = cand[:, 0], cand[:, 1]
    d = x[j] - x[i]
    d = d - box * np.round(d / box)
    s = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
    keep = s < link * link
    return np.stack([np.minimum(i, j)[keep], np.maximum(i, j)[keep]], axis=1)


def canonical_labels(group, min_members):
    """Halo labels from any group assignment: tag = smallest member index,
    halos (>= min_members) numbered by increasing tag, others -1."""
    group = np.asarray(group)
    n = len(group)
    tag_of_group = np.full(group.max() + 1 if n else 0, n, dtype=np.int64)
    np.minimum.at(tag_of_group, group, np.arange(n))
    tag = tag_of_group[group]
    sizes = np.bincount(tag, minlength=n)
    halo_tags = np.flatnonzero(sizes >= min_members)
    halo_id = np.full(n, -1, dtype=np.int64)
    halo_id[halo_tags] = np.arange(len(halo_tags))
    return halo_id[tag], sizes[halo_tags]


def fof(pos, box, link, min_members=40):
    """(labels (n,) int64, halo sizes (n_halos,) int64)."""
    n = len(pos)
    pr = friend_pairs(pos, box, link)
    g = coo_matrix((np.ones(len(pr)), (pr[:, 0], pr[:, 1])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    return canonical_labels(comp, min_members)
