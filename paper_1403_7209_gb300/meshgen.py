"""Seeded synthetic inputs: periodic jittered lattices and flow states.

This module is the one input source shared by the CUDA path and the CPU
oracle.  It holds none of the method's arithmetic (no flux, gradient,
limiter, time step or update): it only draws the mesh and the state that
the loops consume, following the workload recipe of the paper's test case
stand-in (the NASA Rotor 37 mesh of Sec. 4 is not available, so periodic
lattices with 9 edges per node take its place).

Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): value ``k`` of stream ``s`` under seed ``S`` is the
``(k+1)``-th SplitMix64 output of the state ``mix(S * GAMMA + s)``.
Streams: 0 node-id permutation, 1 coordinate jitter, 2 normal scale,
3 flow state, 4 cell volume, 5 adjoint seed lambda, 6 tangent direction v,
7 finite-difference picks.

Layouts returned here are plain "node-major" numpy arrays (row i = node i);
each consumer converts to its own layout.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA_SM = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_PERM, STREAM_JITTER, STREAM_NORMAL, STREAM_STATE = 0, 1, 2, 3
STREAM_VOLUME, STREAM_LAMBDA, STREAM_V, STREAM_FD = 4, 5, 6, 7

GAMMA_GAS = 1.4  # ratio of specific heats used to turn p into rho*E

# 3 axis + 6 face-diagonal lattice offsets and their dual-face areas.
OFFSETS = np.array(
    [[1, 0, 0], [0, 1, 0], [0, 0, 1],
     [1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]],
    dtype=np.int64)
AREAS = np.array([1.0, 1.0, 1.0, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5])


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix_u64(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Raw 64-bit outputs of stream ``stream`` at counters ``index``."""
    with np.errstate(over="ignore"):
        base = _mix(np.array([seed], dtype=np.uint64) * GAMMA_SM
                    + np.uint64(stream))
        idx = np.asarray(index, dtype=np.uint64)
        return _mix(base + (idx + np.uint64(1)) * GAMMA_SM)


def uniform(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (splitmix_u64(seed, stream, index) >> np.uint64(11)).astype(
        np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform (two uniforms each)."""
    idx = np.asarray(index, dtype=np.uint64)
    u1 = uniform(seed, stream, idx * np.uint64(2))
    u2 = uniform(seed, stream, idx * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class Lattice:
    """A periodic n^3 jittered lattice with 9 edges per node.

    ``edge`` (E, 2) int32 holds (i, j); ``normal`` (E, 3) the dual-face
    normal pointing from i to j; ``dx`` (E, 3) the minimum-image vector
    x_j - x_i; ``coords`` (N, 3); ``volume`` (N,).
    """
    n: int
    coords: np.ndarray
    edge: np.ndarray
    normal: np.ndarray
    dx: np.ndarray
    volume: np.ndarray
    perturbed: bool = True
    seed: int = 0
    new_of_lattice: np.ndarray = field(default=None, repr=False)

    @property
    def num_nodes(self) -> int:
        return self.coords.shape[0]

    @property
    def num_edges(self) -> int:
        return self.edge.shape[0]


def lattice(n: int, seed: int = 0, perturbed: bool = True,
            jitter: float = 0.1, normal_scale: float = 0.05,
            volume_scale: float = 0.1, permute: bool = True) -> Lattice:
    """Build the periodic jittered lattice mesh.

    Nodes (a, b, c) in [0, n)^3 with lattice id a + n*b + n^2*c; coordinates
    are the lattice point plus U[-jitter, jitter] per component.  Edge
    (node, offset o) joins a node to its +o neighbour (mod n).  The normal is
    the unit offset direction times the face area (1 axis, 0.5 diagonal),
    times (1 + U[-normal_scale, normal_scale]) unless ``perturbed`` is False,
    in which case every edge of one offset class has a bit-identical normal.
    Node ids are a random permutation of the lattice ids (seed ``seed``);
    edges keep generation order (node-major, offset-minor), relabelled.
    """
    if n < 3:
        raise ValueError("periodic lattice needs n >= 3 (no duplicate edges)")
    N = n ** 3
    lid = np.arange(N, dtype=np.int64)
    a, b, c = lid % n, (lid // n) % n, lid // (n * n)
    lat = np.stack([a, b, c], axis=1)

    jit = jitter * (2.0 * uniform(seed, STREAM_JITTER,
                                  np.arange(3 * N, dtype=np.uint64)) - 1.0)
    jit = jit.reshape(N, 3)
    coords_lat = lat.astype(np.float64) + jit

    # edges in lattice numbering
    i0 = np.repeat(lid, 9)
    o = np.tile(np.arange(9), N)
    nb = (lat[i0] + OFFSETS[o]) % n
    j0 = nb[:, 0] + n * nb[:, 1] + n * n * nb[:, 2]

    unit = OFFSETS.astype(np.float64) / np.linalg.norm(
        OFFSETS.astype(np.float64), axis=1, keepdims=True)
    cls_normal = unit * AREAS[:, None]          # (9, 3)
    nrm = cls_normal[o]
    if perturbed:
        scale = 1.0 + normal_scale * (2.0 * uniform(
            seed, STREAM_NORMAL, np.arange(9 * N, dtype=np.uint64)) - 1.0)
        nrm = nrm * scale[:, None]
    dxe = OFFSETS[o].astype(np.float64) + jit[j0] - jit[i0]

    vol = 1.0 + volume_scale * (2.0 * uniform(
        seed, STREAM_VOLUME, np.arange(N, dtype=np.uint64)) - 1.0)

    if permute:
        keys = splitmix_u64(seed, STREAM_PERM, np.arange(N, dtype=np.uint64))
        order = np.argsort(keys, kind="stable")       # new id -> lattice id
        new_of_lat = np.empty(N, dtype=np.int64)
        new_of_lat[order] = np.arange(N)
    else:
        order = lid
        new_of_lat = lid
    edge = np.stack([new_of_lat[i0], new_of_lat[j0]], axis=1).astype(np.int32)
    return Lattice(n=n, coords=np.ascontiguousarray(coords_lat[order]),
                   edge=np.ascontiguousarray(edge),
                   normal=np.ascontiguousarray(nrm),
                   dx=np.ascontiguousarray(dxe),
                   volume=np.ascontiguousarray(vol[order]),
                   perturbed=perturbed, seed=seed, new_of_lattice=new_of_lat)


def flow_state(mesh: Lattice, seed: int = 0, gamma: float = GAMMA_GAS,
               uniform_state: bool = False) -> np.ndarray:
    """Conserved state q = (rho, rho u, rho v, rho w, rho E, c) per node.

    rho ~ U[0.9, 1.1]; u = (0.5, 0, 0) + three independent U[-0.3, 0.3];
    p ~ U[0.9, 1.1]; rho E = p/(gamma-1) + rho|u|^2/2; the passive scalar
    c ~ U[0, 1e-3] is stored as the conserved quantity itself.  Draws are
    indexed by lattice id so the physical field does not depend on the node
    numbering.  ``uniform_state`` gives one constant state everywhere
    (freestream).
    """
    N = mesh.num_nodes
    if uniform_state:
        rho = np.full(N, 1.0)
        u = np.tile(np.array([0.5, 0.1, -0.2]), (N, 1))
        p = np.full(N, 1.0)
        cc = np.full(N, 5e-4)
    else:
        idx = np.arange(8 * N, dtype=np.uint64)
        r = uniform(seed, STREAM_STATE, idx).reshape(N, 8)
        rho = 0.9 + 0.2 * r[:, 0]
        u = np.array([0.5, 0.0, 0.0]) + (0.6 * r[:, 1:4] - 0.3)
        p = 0.9 + 0.2 * r[:, 4]
        cc = 1e-3 * r[:, 5]
        # draws are by lattice id: move them to the mesh numbering
        inv = np.empty(N, dtype=np.int64)
        inv[mesh.new_of_lattice] = np.arange(N)
        rho, u, p, cc = rho[inv], u[inv], p[inv], cc[inv]
    q = np.empty((N, 6))
    q[:, 0] = rho
    q[:, 1:4] = rho[:, None] * u
    q[:, 4] = p / (gamma - 1.0) + 0.5 * rho * np.sum(u * u, axis=1)
    q[:, 5] = cc
    return q


def adjoint_seed(num_nodes: int, seed: int = 0, stream: int = STREAM_LAMBDA,
                 dim: int = 6) -> np.ndarray:
    """lambda ~ N(0, 1) per node and component, (N, dim)."""
    return normal(seed, stream, np.arange(num_nodes * dim, dtype=np.uint64)
                  ).reshape(num_nodes, dim)


def fd_picks(count: int, upper: int, seed: int = 0) -> np.ndarray:
    """Distinct-ish random indices in [0, upper) for finite-difference checks."""
    u = uniform(seed, STREAM_FD, np.arange(count, dtype=np.uint64))
    return np.minimum((u * upper).astype(np.int64), upper - 1)


def random_graph_mesh(num_nodes: int, mean_degree: float = 9.0, seed: int = 0,
                      isolated: int = 3) -> Lattice:
    """An irregular edge set on random points, for parity on uneven degrees.

    Points uniform in the unit cube (stream 1).  Each node draws a
    Poisson-like number of partners (0 to about 3x the mean) among nodes
    drawn uniformly (stream 2), so degrees vary widely, some node pairs
    repeat and both orientations occur; the last `isolated` nodes get no
    edges.  Normals: random directions with areas U[0.1, 1] (stream 2);
    dx = x_j - x_i; volumes U[0.5, 1.5] (stream 4).  Not a valid dual
    mesh: for exercising the loops on an uneven graph only.
    """
    N = num_nodes
    coords = uniform(seed, STREAM_JITTER, np.arange(3 * N, dtype=np.uint64)).reshape(N, 3)
    r = uniform(seed, STREAM_NORMAL, np.arange(N, dtype=np.uint64))
    deg = np.minimum((-np.log1p(-r) * mean_degree / 2).astype(np.int64), int(3 * mean_degree))
    live = N - isolated
    deg[live:] = 0
    i = np.repeat(np.arange(N), deg)
    u = uniform(seed, STREAM_NORMAL, np.arange(N, N + i.size, dtype=np.uint64))
    j = np.minimum((u * (live - 1)).astype(np.int64), live - 2)
    j = j + (j >= i)  # never a self loop
    E = i.size
    w = uniform(seed, STREAM_NORMAL, np.arange(N + E, N + 5 * E, dtype=np.uint64)).reshape(E, 4)
    d = 2.0 * w[:, :3] - 1.0
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-3)
    nrm = d * (0.1 + 0.9 * w[:, 3:4])
    edge = np.stack([i, j], axis=1).astype(np.int32)
    vol = 0.5 + uniform(seed, STREAM_VOLUME, np.arange(N, dtype=np.uint64))
    return Lattice(n=0, coords=coords, edge=edge, normal=nrm,
                   dx=coords[j] - coords[i], volume=vol, perturbed=True, seed=seed,
                   new_of_lattice=np.arange(N))


def hand_cube_mesh():
    """The 8-node unit-cube mesh: corners, 12 cube edges, n = edge direction.

    Node id = x + 2y + 4z for corner (x, y, z) in {0,1}^3.  Edges run from
    the lower to the upper corner along each axis; the normal is the unit
    axis vector (area 1) and dx is that same vector.  Non-periodic.
    """
    nodes = [(x, y, z) for z in (0, 1) for y in (0, 1) for x in (0, 1)]
    nid = {p: k for k, p in enumerate(nodes)}
    edges, normals = [], []
    for p in nodes:
        for d in range(3):
            if p[d] == 0:
                qp = list(p)
                qp[d] = 1
                edges.append((nid[p], nid[tuple(qp)]))
                v = [0.0, 0.0, 0.0]
                v[d] = 1.0
                normals.append(v)
    coords = np.array(nodes, dtype=np.float64)
    edge = np.array(edges, dtype=np.int32)
    nrm = np.array(normals)
    return coords, edge, nrm, nrm.copy()
