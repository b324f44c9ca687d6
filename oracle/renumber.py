"""Reverse Cuthill-McKee node renumbering, written out plainly.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle).

Sec. 4 of the paper renumbers the mesh for cache locality (it uses the
Gibbs-Poole-Stockmeyer ordering of Scotch and reports a 17% gain).  The
library renumbers with reverse Cuthill-McKee instead; this is the textbook
statement of that algorithm (Cuthill and McKee 1969; reversal by George
1971) with every tie broken explicitly so that the order is unique:

* the graph is the undirected node graph of the edge list (duplicate
  neighbours and self loops dropped); deg(v) = number of distinct neighbours;
* a component starts from its unvisited node of smallest (degree, id);
* breadth-first search; when a node is taken from the queue its unvisited
  neighbours are appended in increasing (degree, id) order;
* the visit order is reversed: the k-th node of the reversed order gets the
  new id k.

Edges are then relabelled and ordered by (min(i', j'), max(i', j')), ties
kept in input order; each edge keeps its orientation.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def adjacency(num_nodes: int, edge: np.ndarray):
    nbrs = [set() for _ in range(num_nodes)]
    for i, j in np.asarray(edge, dtype=np.int64).tolist():
        if i != j:
            nbrs[i].add(j)
            nbrs[j].add(i)
    return nbrs


def rcm_order(num_nodes: int, edge: np.ndarray) -> np.ndarray:
    """new_of_old: the new id of every node under reverse Cuthill-McKee."""
    nbrs = adjacency(num_nodes, edge)
    deg = [len(s) for s in nbrs]
    visited = [False] * num_nodes
    order = []
    # candidates for component starts, by (degree, id)
    starts = sorted(range(num_nodes), key=lambda v: (deg[v], v))
    si = 0
    while len(order) < num_nodes:
        while visited[starts[si]]:
            si += 1
        s = starts[si]
        visited[s] = True
        queue = deque([s])
        while queue:
            v = queue.popleft()
            order.append(v)
            fresh = sorted((w for w in nbrs[v] if not visited[w]),
                           key=lambda w: (deg[w], w))
            for w in fresh:
                visited[w] = True
                queue.append(w)
    order.reverse()
    new_of_old = np.empty(num_nodes, dtype=np.int64)
    new_of_old[np.array(order, dtype=np.int64)] = np.arange(num_nodes)
    return new_of_old


def rcb_order(xyz: np.ndarray, leaf: int = 1) -> np.ndarray:
    """new_of_old under recursive coordinate bisection.

    The partitioner of Sec. 4 of the paper, used as an ordering: a set of
    more than `leaf` nodes is split along the axis of its largest coordinate
    extent (ties: the lowest axis) into the lower half (the first |set|//2
    nodes in (coordinate, id) order) and the rest; the lower half is
    numbered first; a leaf numbers its nodes in id order.
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    new_of_old = np.empty(xyz.shape[0], dtype=np.int64)
    counter = [0]

    def visit(ids):
        if len(ids) <= leaf:
            for v in sorted(ids):
                new_of_old[v] = counter[0]
                counter[0] += 1
            return
        ext = [max(xyz[v, d] for v in ids) - min(xyz[v, d] for v in ids) for d in range(3)]
        ax = 0
        for d in (1, 2):
            if ext[d] > ext[ax]:
                ax = d
        ordered = sorted(ids, key=lambda v: (xyz[v, ax], v))
        half = len(ids) // 2
        visit(ordered[:half])
        visit(ordered[half:])

    import sys
    sys.setrecursionlimit(max(10000, sys.getrecursionlimit()))
    visit(list(range(xyz.shape[0])))
    return new_of_old


def edge_order(edge: np.ndarray, new_of_old: np.ndarray) -> np.ndarray:
    """Old edge index of each new edge position after relabelling."""
    e = new_of_old[np.asarray(edge, dtype=np.int64)]
    lo, hi = e.min(axis=1), e.max(axis=1)
    return np.lexsort((np.arange(e.shape[0]), hi, lo))


def bandwidth(edge: np.ndarray) -> int:
    e = np.asarray(edge, dtype=np.int64)
    if e.shape[0] == 0:
        return 0
    return int(np.max(np.abs(e[:, 0] - e[:, 1])))
