"""Cluster tree (Def 2.1), standard admissibility (§5.1) and block tree (Def 2.2). Oracle; test-only.

Readings of the paper (which only asks for a binary cluster tree, §2.2):

* Geometric bisection: a cluster's tight axis-aligned bounding box is split on its
  longest edge (ties -> lowest axis) at mid = 0.5*(lo+hi); son 0 takes the points with
  coordinate < mid, son 1 those with coordinate >= mid; both keep ascending original
  index.  If one side would be empty, the cluster is split at the median of the
  (coordinate, original index) order instead: son 0 takes the first floor(m/2).
  Clusters with at most ``leaf_size`` points are leaves.
* Clusters are numbered in depth-first pre-order (root 0, son 0's subtree, then son 1).
  The index permutation lists the leaves' points left to right; cluster c covers the
  permuted index range [lo, hi).
* diam = bounding-box diagonal, dist = Euclidean box-to-box distance; admissible iff
  dist > 0 and min(diam_t^2, diam_s^2) <= eta^2 * dist^2 (the printed inequality is
  "<=").  All in FP64 with a fixed operation order.
* Block tree: sons(t, s) is empty if adm(t, s) or either cluster is a leaf, else the
  four pairs of sons.  An admissible leaf is stored low-rank, any other leaf dense.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cluster:
    id: int
    lo: int
    hi: int
    level: int
    bmin: tuple
    bmax: tuple
    sons: list = field(default_factory=list)

    @property
    def size(self) -> int:
        return self.hi - self.lo

    @property
    def is_leaf(self) -> bool:
        return not self.sons


class ClusterTree:
    def __init__(self, points: np.ndarray, leaf_size: int = 64):
        self.points = np.asarray(points, dtype=np.float64)
        self.leaf_size = int(leaf_size)
        self.clusters: list[Cluster] = []
        self.perm: list[int] = []
        n = self.points.shape[0]
        self.root = self._build(list(range(n)), 0)
        self.perm = np.asarray(self.perm, dtype=np.int64)

    def _bbox(self, idx):
        pts = self.points[idx]
        return tuple(float(v) for v in pts.min(axis=0)), tuple(float(v) for v in pts.max(axis=0))

    def _build(self, idx: list, level: int) -> Cluster:
        bmin, bmax = self._bbox(idx)
        c = Cluster(id=len(self.clusters), lo=len(self.perm), hi=-1, level=level,
                    bmin=bmin, bmax=bmax)
        self.clusters.append(c)
        if len(idx) <= self.leaf_size:
            self.perm.extend(idx)
            c.hi = len(self.perm)
            return c
        ext = [bmax[a] - bmin[a] for a in range(3)]
        axis = 0
        for a in (1, 2):
            if ext[a] > ext[axis]:
                axis = a
        mid = 0.5 * (bmin[axis] + bmax[axis])
        coord = self.points[:, axis]
        left = [i for i in idx if coord[i] < mid]
        right = [i for i in idx if not (coord[i] < mid)]
        if not left or not right:
            order = sorted(idx, key=lambda i: (coord[i], i))
            half = len(order) // 2
            left = sorted(order[:half])
            right = sorted(order[half:])
        c.sons = [self._build(left, level + 1), self._build(right, level + 1)]
        c.hi = len(self.perm)
        return c

    @property
    def leaves(self) -> list:
        return [c for c in self.clusters if c.is_leaf]

    def depth(self) -> int:
        return max(c.level for c in self.clusters)


def diam2(c: Cluster) -> float:
    e0 = c.bmax[0] - c.bmin[0]
    e1 = c.bmax[1] - c.bmin[1]
    e2 = c.bmax[2] - c.bmin[2]
    return e0 * e0 + e1 * e1 + e2 * e2


def dist2(t: Cluster, s: Cluster) -> float:
    d = []
    for a in range(3):
        g = max(s.bmin[a] - t.bmax[a], t.bmin[a] - s.bmax[a])
        d.append(g if g > 0.0 else 0.0)
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2]


def admissible(t: Cluster, s: Cluster, eta: float) -> bool:
    """Standard admissibility min(diam t, diam s) <= eta dist(t, s), with dist > 0 (§5.1)."""
    dd = dist2(t, s)
    if not dd > 0.0:
        return False
    return min(diam2(t), diam2(s)) <= (eta * eta) * dd


@dataclass
class Block:
    row: Cluster
    col: Cluster
    adm: bool
    sons: list = field(default_factory=list)   # [[b00, b01], [b10, b11]] when inner

    @property
    def is_leaf(self) -> bool:
        return not self.sons

    @property
    def key(self):
        return (self.row.id, self.col.id)


class BlockTree:
    """Block tree T_{I x I} over one cluster tree (Def 2.2)."""

    def __init__(self, ct: ClusterTree, eta: float = 2.0):
        self.ct = ct
        self.eta = float(eta)
        self.blocks: dict = {}
        self.root = self._build(ct.root, ct.root)

    def _build(self, t: Cluster, s: Cluster) -> Block:
        adm = admissible(t, s, self.eta)
        b = Block(t, s, adm)
        self.blocks[(t.id, s.id)] = b
        if not adm and not t.is_leaf and not s.is_leaf:
            b.sons = [[self._build(t.sons[i], s.sons[j]) for j in range(2)] for i in range(2)]
        return b

    def get(self, t: Cluster, s: Cluster) -> Block:
        return self.blocks[(t.id, s.id)]

    def is_leaf(self, t: Cluster, s: Cluster) -> bool:
        return self.blocks[(t.id, s.id)].is_leaf

    def leaves(self) -> list:
        return [b for b in self.blocks.values() if b.is_leaf]

    def leaves_under(self, b: Block) -> list:
        if b.is_leaf:
            return [b]
        out = []
        for i in range(2):
            for j in range(2):
                out.extend(self.leaves_under(b.sons[i][j]))
        return out
