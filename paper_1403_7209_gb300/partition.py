"""Owner-compute execution of the edge loops over node partitions.

The paper's distributed-memory back-end (Sec. 3.2: an owner-compute model
like OPlus's, whose halo updates Sec. 2 describes) splits the nodes into
parts -- by recursive coordinate bisection in Sec. 4 -- and gives each part
the edges with an owned end; a
cut edge runs in both of its parts.  Before a loop reads node data through
the map, a part refreshes its halo (the non-owned ends of its edges) from
the owners; its INC results are then complete on its owned nodes.

Here every part is one :class:`EdgeSolver` (its own context, sets, maps,
plans and dats) and all parts live on one GPU; the halo refresh is one
library gather kernel per dat over every (importer, owner) pair
(``op2b_exchange_run``).  One explicit second-order stage is

  exchange q -> Green-Gauss + scaling (every part) -> exchange G ->
  flux (every part) -> update (every part)

and on its owned nodes each part then holds exactly what the whole-mesh
solver holds, up to the summation order of the INC.  Halo rows of R, G
(before the G exchange) and of the updated q are partial and are never
read before the next exchange overwrites them.  The partition, the local
meshes and the import / export lists come from the library's host planner
(``op2b_host_partition_rcb``, ``op2b_halo_create``).
"""
from __future__ import annotations

import numpy as np

from . import op2b as L
from .solver import RK5_ALPHA, EdgeSolver


def halo_plan(num_nodes, edge, part, nparts):
    """Local meshes and exchange lists of every part (list of dicts, see
    :func:`op2b.op2b_halo_part`)."""
    h = L.op2b_halo_create(num_nodes, edge, part, nparts)
    try:
        return [L.op2b_halo_part(h, p) for p in range(nparts)]
    finally:
        L.op2b_halo_destroy(h)


def halo_stats(parts):
    """Per-partition figures of the paper's halo table (Sec. 4.2): average
    number of neighbours a part exchanges with, average elements (nodes +
    edges) held per part, and the average share of halo elements (halo
    nodes + redundantly executed cut edges) in them."""
    nb, tot, hshare = [], [], []
    for P in parts:
        z = P["sizes"]
        importers = set(P["nbr"].tolist())
        exporters = set(P["halo_owner"].tolist())
        nb.append(len(importers | exporters))
        t = z["owned"] + z["halo"] + z["edges"]
        tot.append(t)
        hshare.append((z["halo"] + z["halo_edges"]) / max(t, 1))
    return {"parts": len(parts), "avg_neighbours": float(np.mean(nb)),
            "avg_elements": float(np.mean(tot)), "avg_halo_percent": 100.0 * float(np.mean(hshare))}


class PartitionedSolver:
    """The loops of :class:`EdgeSolver` over ``nparts`` owner-compute parts.

    ``edge`` (E, 2), ``normal``/``dx`` (E, 3), ``volume`` (N,), ``q``
    (N, 6), ``coords`` (N, 3) in the caller's numbering; ``part`` (N,)
    overrides the RCB partition.  Each part is renumbered internally with
    ``renumber`` (as :class:`EdgeSolver`).  :meth:`fetch_nodes` assembles
    the owned rows of every part in the caller's numbering.

    With ``concurrent`` the parts' loops run on a pool of up to 16 CUDA
    streams (part p on stream p mod 16), forked from and joined back to
    ``stream`` with events around every halo exchange, which runs on
    ``stream``; small parts then fill the GPU together instead of one
    after another.  Without it every part runs on ``stream`` in turn.
    """

    EXCHANGED = {"q": (6, L.F64), "G": (18, L.F64), "q32": (6, L.F32), "G32": (18, L.F32)}

    def __init__(self, edge, normal, dx, volume, q, coords=None, nparts=2, part=None,
                 device: int = 0, renumber: str = "rcm", mixed: bool = False, stream=None,
                 gamma: float = 1.4, eps_lim: float = 1e-12, concurrent: bool = False):
        import torch
        edge = np.ascontiguousarray(edge, dtype=np.int32)
        normal = np.asarray(normal, dtype=np.float64).reshape(-1, 3)
        dx = np.asarray(dx, dtype=np.float64).reshape(-1, 3)
        volume = np.asarray(volume, dtype=np.float64).reshape(-1)
        q = np.asarray(q, dtype=np.float64).reshape(-1, 6)
        self.N, self.E = volume.shape[0], edge.shape[0]
        if part is None:
            if coords is None:
                raise ValueError("PartitionedSolver needs coords (RCB) or part")
            part = L.op2b_host_partition_rcb(coords, nparts)
        self.part = np.ascontiguousarray(part, dtype=np.int32)
        self.nparts = int(nparts)
        self.mixed = mixed
        self.parts = halo_plan(self.N, edge, self.part, self.nparts)
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.streams = ([torch.cuda.Stream(device=device) for _ in range(min(self.nparts, 16))]
                        if concurrent else [])
        self._fork_ev = torch.cuda.Event()
        self._join_ev = [torch.cuda.Event() for _ in self.streams]
        self.solvers = []
        for p, P in enumerate(self.parts):
            nodes, edges = P["nodes"], P["edges"]
            st = self.streams[p % len(self.streams)] if concurrent else self.stream
            self.solvers.append(EdgeSolver(P["local_map"], normal[edges], dx[edges],
                                           volume[nodes], q[nodes], device=device,
                                           renumber=renumber, mixed=mixed, stream=st,
                                           gamma=gamma, eps_lim=eps_lim))
        # the exchanges launch on `stream` from a context of their own
        self.ctx = L.op2b_init(device, self.stream.cuda_stream)
        self.x = {}
        for name in ("q", "G") + (("q32", "G32") if mixed else ()):
            self.x[name] = self._exchange(name)

    # ------------------------------------------------------- exchanges
    def _exchange(self, name):
        """Exchange of dat `name`: one segment per (importer, owner) pair,
        rows in the library numbering of both parts."""
        dim, type_ = self.EXCHANGED[name]
        src, sld, dst, dld, cnt, si, di = [], [], [], [], [], [], []
        for p, P in enumerate(self.parts):
            sp = self.solvers[p]
            n_own = P["sizes"]["owned"]
            owner = P["halo_owner"]
            for r in np.unique(owner):
                rows = np.nonzero(owner == r)[0]
                so = self.solvers[r]
                src.append(so.t[name].data_ptr())
                sld.append(so.t[name].shape[1])
                dst.append(sp.t[name].data_ptr())
                dld.append(sp.t[name].shape[1])
                cnt.append(rows.size)
                si.append(so.perm[P["halo_src"][rows]])
                di.append(sp.perm[n_own + rows])
        def cat(a):
            return np.concatenate(a) if a else np.zeros(0, np.int64)
        return L.op2b_exchange_create(self.ctx, type_, dim, src, sld, dst, dld, cnt,
                                      cat(si), cat(di))

    def exchange(self, name):
        L.op2b_exchange_run(self.ctx, self.x[name])

    def _fork(self):
        """Part streams wait for the work already queued on `stream`."""
        if self.streams:
            self._fork_ev.record(self.stream)
            for st in self.streams:
                st.wait_event(self._fork_ev)

    def _join(self):
        """`stream` waits for the work queued on the part streams."""
        for st, ev in zip(self.streams, self._join_ev):
            ev.record(st)
            self.stream.wait_event(ev)

    # ------------------------------------------------------------ loops
    def set_strategy(self, loop, prec, strategy, block=0, part=0, staged=0):
        for s in self.solvers:
            s.set_strategy(loop, prec, strategy, block, part, staged)

    def _each(self, fn):
        """fn(solver) for every part, between a fork and a join."""
        self._fork()
        for s in self.solvers:
            fn(s)
        self._join()

    def residual(self, order=2, mixed=False, update_alpha=None):
        """R of the current state on every part's owned nodes (then the
        stage update with `update_alpha`, in the same fork)."""
        sfx = "32" if mixed else ""
        self.exchange("q" + sfx)
        if order == 2:
            self._each(lambda s: s.green_gauss(mixed))
            self.exchange("G" + sfx)

        def flux(s):
            s.flux(order, mixed)
            if update_alpha is not None:
                s.update(update_alpha, mixed)
        self._each(flux)

    def time_step(self, cfl=0.5):
        self.exchange("q")
        self._each(lambda s: s.time_step(cfl))

    def stage(self, alpha, order=2, mixed=False):
        self.residual(order, mixed, update_alpha=alpha)

    def step(self, order=2, mixed=False, stages=5):
        self._each(lambda s: L.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"]))
        for a in RK5_ALPHA[5 - stages:]:
            self.stage(a, order, mixed)

    def sync_shadow(self):
        self._each(lambda s: s.sync_shadow())

    # ------------------------------------------------------------- data
    def fetch_nodes(self, name) -> np.ndarray:
        """(N, dim) float64: every node's row from its owner."""
        self.torch.cuda.synchronize()  # the parts may run on streams of their own
        out = None
        for P, s in zip(self.parts, self.solvers):
            n_own = P["sizes"]["owned"]
            v = s.fetch_nodes(name)[:n_own]
            if out is None:
                out = np.empty((self.N, v.shape[1]), dtype=np.float64)
            out[P["nodes"][:n_own]] = v
        return out

    def launch_count(self):
        return sum(s.launch_count() for s in self.solvers) + L.op2b_launch_count(self.ctx)

    def close(self):
        if self.solvers:
            self.torch.cuda.synchronize()
            for x in self.x.values():
                L.op2b_exchange_destroy(self.ctx, x)
            self.x = {}
            L.op2b_finalize(self.ctx)
            for s in self.solvers:
                s.close()
            self.solvers = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
