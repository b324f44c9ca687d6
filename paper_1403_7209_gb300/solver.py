"""One mesh on one GPU: sets, the edge->node map and the dats of the loops.

A thin layer over :mod:`paper_1403_7209_gb300.op2b`: it owns torch tensors
(device memory) laid out structure-of-arrays, (dim, n) contiguous, declares
them as dats, and calls the loops in the order of one explicit step:

  Green-Gauss edge loop -> gradient scaling -> flux edge loop -> RK update

(Sec. 2 of the paper: Hydra's explicit 5-step Runge-Kutta time march).
All arithmetic runs in the CUDA library; this module only marshals.
"""
from __future__ import annotations

import numpy as np

from . import op2b as L

RK5_ALPHA = (0.25, 1.0 / 6.0, 0.375, 0.5, 1.0)  # Jameson's 5-stage scheme
RENUMBER = {"none": 0, "random": 1, "rcm": 2}  # "rcb" needs coordinates
LIMITERS = {"van_albada": 0, "barth_jespersen": L.LIM_BARTH_JESPERSEN,
            "venkatakrishnan": L.LIM_VENKATAKRISHNAN}


class EdgeSolver:
    """Dats and loops of an edge-based finite-volume mesh.

    ``edge`` (E, 2) int, ``normal``/``dx`` (E, 3), ``volume`` (N,), ``q``
    (N, 6) in the caller's numbering.  ``renumber`` in {"none", "random",
    "rcm", "rcb"} reorders nodes and edges inside the library ("rcb", the
    partition order of recursive coordinate bisection, needs ``coords``
    (N, 3)); :meth:`fetch_nodes` and :meth:`fetch_edges` return data in the
    caller's numbering again.
    ``mixed`` adds the FP32 shadows used by the mixed-precision path;
    ``ff`` the float-float shadows (q, G, n, dx) of the float-float flux,
    whose arithmetic runs on the FP32 units at about FP64 accuracy;
    ``adjoint`` the adjoint and tangent (Jacobian-vector product) dats;
    ``viscous`` = (mu, prandtl, diff) adds the viscous flux to the residual
    (Navier-Stokes instead of Euler).  ``limiter`` picks the second-order
    reconstruction: "van_albada" (per edge, the default), or the node
    limiters "barth_jespersen" and "venkatakrishnan" (``limiter_eps2`` is
    Venkatakrishnan's smoothing constant).  ``precond`` adds the block-Jacobi
    blocks and their inverses for preconditioned steps (``step(sigma=...)``).
    """

    def __init__(self, edge, normal, dx, volume, q=None, device: int = 0,
                 renumber: str = "none", seed: int = 0, mixed: bool = False,
                 adjoint: bool = False, gamma: float = 1.4,
                 eps_lim: float = 1e-12, stream=None, coords=None, viscous=None,
                 limiter: str = "van_albada", limiter_eps2: float = 0.0, ff: bool = False,
                 precond: bool = False):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.gamma, self.eps_lim = gamma, eps_lim
        edge = np.ascontiguousarray(edge, dtype=np.int32)
        self.N = int(np.asarray(volume).shape[0])
        self.E = int(edge.shape[0])
        self.ctx = L.op2b_init(device, self.stream.cuda_stream)
        c = self.ctx
        self.nodes = L.op2b_decl_set(c, self.N, "nodes")
        self.edges = L.op2b_decl_set(c, self.E, "edges")
        self.map = L.op2b_decl_map(c, self.edges, self.nodes, 2, edge.ravel(), "edge2node")
        self.t, self.d = {}, {}

        def node(name, dim, dtype=torch.float64, init=None):
            self._dat(name, self.nodes, self.N, dim, dtype, init)

        def edgd(name, dim, dtype=torch.float64, init=None):
            self._dat(name, self.edges, self.E, dim, dtype, init)

        node("q", 6, init=q)
        node("q0", 6)
        node("R", 6)
        node("G", 18)
        node("V", 1, init=np.asarray(volume).reshape(-1, 1))
        node("lam_s", 1)
        node("dt", 1)
        edgd("n", 3, init=normal)
        edgd("dx", 3, init=dx)
        if coords is not None:
            node("x", 3, init=coords)
        self.mixed = mixed
        if mixed:
            node("q32", 6, torch.float32, init=q)
            node("G32", 18, torch.float32)
            edgd("n32", 3, torch.float32, init=normal)
            edgd("dx32", 3, torch.float32, init=dx)
        if limiter not in LIMITERS:
            raise ValueError("limiter must be one of %s" % sorted(LIMITERS))
        self.limiter, self.limiter_eps2 = limiter, float(limiter_eps2)
        if LIMITERS[limiter]:
            for nm in ("qmin", "qmax", "phi"):
                node(nm, 6)
                if mixed:
                    node(nm + "32", 6, torch.float32)
                if ff:
                    node(nm + "_ff", 6, "ff")
        self.visc = tuple(float(v) for v in viscous) if viscous is not None else None
        if self.visc is not None:
            node("W", 20)
            if mixed:
                node("W32", 20, torch.float32)
        self.ff = ff
        if ff:
            node("q_ff", 6, "ff")
            node("G_ff", 18, "ff")
            edgd("n_ff", 3, "ff")
            edgd("dx_ff", 3, "ff")
            if self.visc is not None:
                node("W_ff", 20, "ff")
        self.precond = precond
        if precond:
            node("M", 36)  # block-Jacobi blocks (row-major 6 x 6 per node)
            node("P", 36)  # their inverses
            node("JS", 4)  # the blocks' factored sums (Lambda, S)
        self.has_adjoint = adjoint
        if adjoint:
            node("lam", 6)
            node("qbar", 6)
            node("Gbar", 18)
            edgd("nbar", 3)
            node("qd", 6)
            node("Gd", 18)
            node("Rd", 6)
            edgd("nd", 3)
            node("qd0", 6)      # tangent march: direction at the step start
            node("sbar", 6)     # march adjoint: adjoint of the current state
            node("qacc", 6)     # march adjoint: per-step accumulator
            edgd("nbar_acc", 3)  # march adjoint: dJ/dn summed over the stages
            if ff:
                node("lam_ff", 6, "ff")  # float-float shadow of the adjoint weights
                node("qd_ff", 6, "ff")   # ... and of the tangent's direction
                node("Gd_ff", 18, "ff")
                edgd("nd_ff", 3, "ff")
        self.perm = np.arange(self.N, dtype=np.int64)   # new id of old node
        self.order = np.arange(self.E, dtype=np.int64)  # old edge of new slot
        if renumber == "rcb":
            if coords is None:
                raise ValueError("renumber='rcb' needs coords")
            perm, order = L.op2b_renumber_rcb(c, self.map, self.d["x"], 1, self.N, self.E)
            self.perm, self.order = perm.astype(np.int64), order
        elif renumber != "none":
            perm, order = L.op2b_renumber(c, self.map, RENUMBER[renumber], seed,
                                          self.N, self.E)
            self.perm, self.order = perm.astype(np.int64), order
        self.edge = L.op2b_fetch_map(c, self.map, 2 * self.E).reshape(-1, 2)
        if ff:
            for nm in ("q", "n", "dx"):
                L.op2b_dat_copy(c, self.d[nm + "_ff"], self.d[nm])
        self._build_args()

    # ------------------------------------------------------------ dats
    def _dat(self, name, set_, n, dim, dtype, init):
        torch = self.torch
        if dtype == "ff":  # float-float: (hi, lo) float pairs, 8 bytes per element
            t = torch.zeros((dim, max(n, 1), 2), dtype=torch.float32, device=self.device)
            self.d[name] = L.op2b_decl_dat(self.ctx, set_, dim, L.FF, t.data_ptr(), t.shape[1],
                                           name)
            self.t[name] = t
            return
        t = torch.zeros((dim, max(n, 1)), dtype=dtype, device=self.device)
        if init is not None and n > 0:
            a = np.asarray(init, dtype=np.float64).reshape(n, dim)
            t[:, :n].copy_(torch.from_numpy(np.ascontiguousarray(a.T)).to(dtype))
        type_ = {torch.float64: L.F64, torch.float32: L.F32}[dtype]
        self.d[name] = L.op2b_decl_dat(self.ctx, set_, dim, type_, t.data_ptr(),
                                       t.shape[1], name)
        self.t[name] = t

    def rebind(self, name, tensor):
        """Make dat `name` use `tensor` (same shape) from now on."""
        assert tensor.shape == self.t[name].shape and tensor.is_contiguous()
        L.op2b_rebind_dat(self.ctx, self.d[name], tensor.data_ptr())
        self.t[name] = tensor

    def _as_f64(self, t, n):
        if t.dim() == 3:  # float-float
            return (t[:, :n, 0].double() + t[:, :n, 1].double()).cpu().numpy()
        return t[:, :n].double().cpu().numpy()

    def fetch_nodes(self, name) -> np.ndarray:
        """(N, dim) float64 in the caller's node numbering."""
        a = self._as_f64(self.t[name], self.N).T
        return np.ascontiguousarray(a[self.perm])

    def fetch_edges(self, name) -> np.ndarray:
        """(E, dim) float64 in the caller's edge order."""
        a = self._as_f64(self.t[name], self.E).T
        out = np.empty_like(a)
        out[self.order] = a
        return out

    def load_nodes(self, name, values):
        """Set dat `name` from (N, dim) values in the caller's numbering."""
        v = np.asarray(values, dtype=np.float64).reshape(self.N, -1)
        a = np.empty_like(v)
        a[self.perm] = v
        t = self.t[name]
        t[:, :self.N].copy_(self.torch.from_numpy(np.ascontiguousarray(a.T)).to(t.dtype))

    def load_edges(self, name, values):
        v = np.asarray(values, dtype=np.float64).reshape(self.E, -1)
        t = self.t[name]
        t[:, :self.E].copy_(self.torch.from_numpy(np.ascontiguousarray(v[self.order].T)).to(t.dtype))

    # ------------------------------------------------------------ loops
    def _build_args(self):
        d, m = self.d, self.map

        def ind(name, idx, acc):
            return (d[name], idx, m, acc)

        def dr(name, acc):
            return (d[name], -1, L.ID, acc)

        R, I, W, RWa = L.READ, L.INC, L.WRITE, L.RW
        self.a_gg = [ind("q", 0, R), ind("q", 1, R), dr("n", R), ind("G", 0, I), ind("G", 1, I)]
        self.a_f1 = [ind("q", 0, R), ind("q", 1, R), dr("n", R), ind("R", 0, I), ind("R", 1, I)]
        self.a_f2 = [ind("q", 0, R), ind("q", 1, R), ind("G", 0, R), ind("G", 1, R),
                     dr("n", R), dr("dx", R), ind("R", 0, I), ind("R", 1, I)]
        self.a_sr = [ind("q", 0, R), ind("q", 1, R), dr("n", R), ind("lam_s", 0, I),
                     ind("lam_s", 1, I)]
        if self.precond:
            self.a_jac = [ind("q", 0, R), ind("q", 1, R), dr("n", R), ind("M", 0, I),
                          ind("M", 1, I)]
            self.a_jsum = [ind("q", 0, R), ind("q", 1, R), dr("n", R), ind("JS", 0, I),
                           ind("JS", 1, I)]
        if self.mixed:
            self.a_gg32 = [ind("q32", 0, R), ind("q32", 1, R), dr("n32", R),
                           ind("G32", 0, I), ind("G32", 1, I)]
            self.a_f1_32 = [ind("q32", 0, R), ind("q32", 1, R), dr("n32", R),
                            ind("R", 0, I), ind("R", 1, I)]
            self.a_f2_32 = [ind("q32", 0, R), ind("q32", 1, R), ind("G32", 0, R),
                            ind("G32", 1, R), dr("n32", R), dr("dx32", R),
                            ind("R", 0, I), ind("R", 1, I)]
        if self.ff:
            self.a_gg_ff = [ind("q_ff", 0, R), ind("q_ff", 1, R), dr("n_ff", R),
                            ind("G_ff", 0, I), ind("G_ff", 1, I)]
            self.a_f2_ff = [ind("q_ff", 0, R), ind("q_ff", 1, R), ind("G_ff", 0, R),
                            ind("G_ff", 1, R), dr("n_ff", R), dr("dx_ff", R),
                            ind("R", 0, I), ind("R", 1, I)]
        if LIMITERS[self.limiter]:
            self.a_f2phi = [ind("q", 0, R), ind("q", 1, R), ind("G", 0, R), ind("G", 1, R),
                            ind("phi", 0, R), ind("phi", 1, R), dr("n", R), dr("dx", R),
                            ind("R", 0, I), ind("R", 1, I)]
            if self.mixed:
                self.a_f2phi32 = [ind("q32", 0, R), ind("q32", 1, R), ind("G32", 0, R),
                                  ind("G32", 1, R), ind("phi32", 0, R), ind("phi32", 1, R),
                                  dr("n32", R), dr("dx32", R), ind("R", 0, I), ind("R", 1, I)]
            if self.ff:
                self.a_f2phi_ff = [ind("q_ff", 0, R), ind("q_ff", 1, R), ind("G_ff", 0, R),
                                   ind("G_ff", 1, R), ind("phi_ff", 0, R), ind("phi_ff", 1, R),
                                   dr("n_ff", R), dr("dx_ff", R), ind("R", 0, I), ind("R", 1, I)]
        if self.visc is not None:
            self.a_vf = [ind("W", 0, R), ind("W", 1, R), dr("n", R), dr("dx", R),
                         ind("R", 0, I), ind("R", 1, I)]
            if self.mixed:
                self.a_vf32 = [ind("W32", 0, R), ind("W32", 1, R), dr("n32", R),
                               dr("dx32", R), ind("R", 0, I), ind("R", 1, I)]
            if self.ff:
                self.a_vf_ff = [ind("W_ff", 0, R), ind("W_ff", 1, R), dr("n_ff", R),
                                dr("dx_ff", R), ind("R", 0, I), ind("R", 1, I)]
        if self.has_adjoint:
            self.a_fa1 = [ind("lam", 0, R), ind("lam", 1, R), ind("q", 0, R), ind("q", 1, R),
                          dr("n", R), ind("qbar", 0, I), ind("qbar", 1, I), dr("nbar", W)]
            self.a_fa2 = [ind("lam", 0, R), ind("lam", 1, R), ind("q", 0, R), ind("q", 1, R),
                          ind("G", 0, R), ind("G", 1, R), dr("n", R), dr("dx", R),
                          ind("qbar", 0, I), ind("qbar", 1, I), ind("Gbar", 0, I),
                          ind("Gbar", 1, I), dr("nbar", W)]
            self.a_ggt = [ind("q", 0, R), ind("q", 1, R), ind("qd", 0, R), ind("qd", 1, R),
                          dr("n", R), dr("nd", R), ind("Gd", 0, I), ind("Gd", 1, I)]
            self.a_ft1 = [ind("q", 0, R), ind("q", 1, R), ind("qd", 0, R), ind("qd", 1, R),
                          dr("n", R), dr("nd", R), ind("Rd", 0, I), ind("Rd", 1, I)]
            self.a_ft2 = [ind("q", 0, R), ind("q", 1, R), ind("qd", 0, R), ind("qd", 1, R),
                          ind("G", 0, R), ind("G", 1, R), ind("Gd", 0, R), ind("Gd", 1, R),
                          dr("n", R), dr("nd", R), dr("dx", R), ind("Rd", 0, I), ind("Rd", 1, I)]
            self.a_gga = [ind("Gbar", 0, R), ind("Gbar", 1, R), ind("q", 0, R), ind("q", 1, R),
                          dr("n", R), ind("qbar", 0, I), ind("qbar", 1, I), dr("nbar", RWa)]
            if self.ff:
                self.a_ft2_ff = [ind("q_ff", 0, R), ind("q_ff", 1, R), ind("qd_ff", 0, R),
                                 ind("qd_ff", 1, R), ind("G_ff", 0, R), ind("G_ff", 1, R),
                                 ind("Gd_ff", 0, R), ind("Gd_ff", 1, R), dr("n_ff", R),
                                 dr("nd_ff", R), dr("dx_ff", R), ind("Rd", 0, I),
                                 ind("Rd", 1, I)]
                self.a_fa2_ff = [ind("lam_ff", 0, R), ind("lam_ff", 1, R), ind("q_ff", 0, R),
                                 ind("q_ff", 1, R), ind("G_ff", 0, R), ind("G_ff", 1, R),
                                 dr("n_ff", R), dr("dx_ff", R), ind("qbar", 0, I),
                                 ind("qbar", 1, I), ind("Gbar", 0, I), ind("Gbar", 1, I),
                                 dr("nbar", W)]

    def set_strategy(self, loop, prec, strategy, block=0, part=0, staged=0):
        L.op2b_set_strategy(self.ctx, loop, prec, strategy, block, part, staged)

    def plan_stats(self, loop, prec=L.PREC_F64):
        return L.op2b_plan_stats(self.ctx, loop, prec, self.map)

    def green_gauss(self, mixed=False, ff=False):
        """G = Graw / V: FP64, FP32 into G32 with ``mixed``, float-float
        (from the float-float shadows of q and n) into G_ff with ``ff``."""
        a = self.a_gg_ff if ff else (self.a_gg32 if mixed else self.a_gg)
        L.op2b_green_gauss_scaled(self.ctx, a, self.d["V"], L.ZERO_INC)

    def node_limiter(self, mixed=False, ff=False):
        """phi from the neighbourhood min/max and the gradients G (FP32 with
        ``mixed``, float-float with ``ff``)."""
        c, d, sfx = self.ctx, self.d, "32" if mixed else ("_ff" if ff else "")
        q, G, dx = ("q" + sfx, "G" + sfx, "dx" + sfx)
        L.op2b_node_minmax(c, self.map, d[q], d["qmin" + sfx], d["qmax" + sfx])
        L.op2b_node_limiter(c, self.map, LIMITERS[self.limiter], self.limiter_eps2, d[q], d[G],
                            d[dx], d["qmin" + sfx], d["qmax" + sfx], d["phi" + sfx])

    def flux(self, order, mixed=False, ff=False):
        """R = sum of edge fluxes (R zeroed first).  ``ff``: the
        second-order flux in float-float arithmetic."""
        if ff:
            if order != 2:
                raise ValueError("the float-float flux is the second-order flux")
            if LIMITERS[self.limiter]:
                self.node_limiter(ff=True)
                L.op2b_edge_flux_limited(self.ctx, self.a_f2phi_ff, self.gamma, L.ZERO_INC)
            else:
                L.op2b_edge_flux(self.ctx, self.a_f2_ff, 2, self.gamma, self.eps_lim, L.ZERO_INC)
            return
        if order == 2 and LIMITERS[self.limiter]:
            self.node_limiter(mixed)
            L.op2b_edge_flux_limited(self.ctx, self.a_f2phi32 if mixed else self.a_f2phi,
                                     self.gamma, L.ZERO_INC)
            return
        if order == 1:
            a = self.a_f1_32 if mixed else self.a_f1
        else:
            a = self.a_f2_32 if mixed else self.a_f2
        L.op2b_edge_flux(self.ctx, a, order, self.gamma, self.eps_lim, L.ZERO_INC)

    def viscous_flux(self, mixed=False, zero=False, ff=False):
        """R -= viscous fluxes (R zeroed first with ``zero``); uses the
        scaled gradients G (G32 with ``mixed``, G_ff in float-float with
        ``ff``)."""
        mu, pr, diff = self.visc
        c = self.ctx
        if ff:
            L.op2b_viscous_prims(c, self.d["q_ff"], self.d["G_ff"], self.d["W_ff"], self.gamma)
            L.op2b_viscous_flux(c, self.a_vf_ff, self.gamma, mu, pr, diff,
                                L.ZERO_INC if zero else 0)
            return
        if mixed:
            L.op2b_viscous_prims(c, self.d["q32"], self.d["G32"], self.d["W32"], self.gamma)
        else:
            L.op2b_viscous_prims(c, self.d["q"], self.d["G"], self.d["W"], self.gamma)
        L.op2b_viscous_flux(c, self.a_vf32 if mixed else self.a_vf, self.gamma, mu, pr, diff,
                            L.ZERO_INC if zero else 0)

    def residual(self, order=2, mixed=False, ff=False):
        """R of the current state: inviscid flux of the given order, plus
        the viscous flux when the solver was built with ``viscous``."""
        if order == 2 or self.visc is not None:
            self.green_gauss(mixed, ff)
        self.flux(order, mixed, ff)
        if self.visc is not None:
            self.viscous_flux(mixed, ff=ff)

    def spectral_radius(self):
        L.op2b_spectral_radius(self.ctx, self.a_sr, self.gamma, L.ZERO_INC)

    def time_step(self, cfl=0.5):
        """Frozen local time step from the current state."""
        self.spectral_radius()
        L.op2b_time_step(self.ctx, self.d["V"], self.d["lam_s"], cfl, self.d["dt"])

    def precondition(self, factored=True):
        """Block-Jacobi preconditioner of the current state: the blocks M
        (diagonal blocks of the first-order residual's Jacobian, wave speeds
        held fixed) and their inverses P.  ``factored``: from the four
        per-node sums (Lambda, sum of signed normals) and one node pass that
        forms and inverts each block; else the 36-value edge loop and the
        inversion loop."""
        if not self.precond:
            raise RuntimeError("EdgeSolver(precond=True) declares the block dats")
        c, d = self.ctx, self.d
        if factored:
            L.op2b_jacobi_sums(c, self.a_jsum, self.gamma, L.ZERO_INC)
            L.op2b_jacobi_from_sums(c, d["q"], d["JS"], d["M"], d["P"], self.gamma)
            return
        L.op2b_jacobi_blocks(c, self.a_jac, self.gamma, L.ZERO_INC)
        L.op2b_block_invert(c, d["M"], d["P"])

    def update(self, alpha, mixed=False, ff=False, sigma=None):
        """q = q0 - alpha (dt/V) R, or with ``sigma`` the block-Jacobi
        preconditioned stage q = q0 - alpha sigma P R (FP64 only)."""
        if sigma is not None:
            if mixed or ff:
                raise NotImplementedError("the preconditioned stage is FP64")
            L.op2b_node_update_precond(self.ctx, self.d["q0"], self.d["q"], self.d["R"],
                                       self.d["P"], alpha * sigma)
            return
        sh = self.d["q32"] if mixed else (self.d["q_ff"] if ff else -1)
        L.op2b_node_update(self.ctx, self.d["q0"], self.d["q"], self.d["R"], self.d["V"],
                           self.d["dt"], alpha, sh)

    def stage(self, alpha, order=2, mixed=False, ff=False, sigma=None):
        self.residual(order, mixed, ff)
        self.update(alpha, mixed, ff, sigma)

    def stage_fused(self, alpha, sync=False, residual=True, gradient=False, store_q0=False,
                    staged=False):
        """One fused FP32-mixed second-order stage (op2b_stage_mixed): q is
        advanced in place; R (with ``residual``) and G32 (with ``gradient``)
        are written too.  ``sync`` re-packs the library's FP32 records from
        q (needed after q was changed by anything but this call); ``staged``
        asks for the shared-memory staged form of the passes."""
        if self.visc is not None or LIMITERS[self.limiter]:
            raise NotImplementedError("the fused stage is the inviscid van Albada scheme")
        d = self.d
        flags = ((L.STAGE_SYNC if sync else 0) | (L.STAGE_STORE_Q0 if store_q0 else 0)
                 | (L.STAGE_STAGED if staged else 0))
        L.op2b_stage_mixed(self.ctx, self.map, d["q0"], d["q"], d["V"], d["dt"], d["n"], d["dx"],
                           d["R"] if residual else -1, d["G32"] if gradient else -1, alpha,
                           self.gamma, self.eps_lim, flags)

    def step(self, order=2, mixed=False, stages=5, ff=False, sigma=None, fused=False,
             staged=False):
        """One explicit RK step (q0 <- q, then `stages` stages).  With
        ``sigma``: block-Jacobi preconditioned, the blocks formed from the
        step's initial state and kept for its stages.  With ``fused`` (the
        second-order FP32-mixed scheme only): every stage is one
        op2b_stage_mixed call, the first re-packing the records from q."""
        L.op2b_dat_copy(self.ctx, self.d["q0"], self.d["q"])
        if fused:
            if order != 2 or ff or sigma is not None:
                raise ValueError("the fused stage is the second-order FP32-mixed scheme")
            for k, a in enumerate(RK5_ALPHA[5 - stages:]):
                self.stage_fused(a, sync=(k == 0), residual=False, staged=staged)
            return
        if sigma is not None:
            self.precondition()
        for a in RK5_ALPHA[5 - stages:]:
            self.stage(a, order, mixed, ff, sigma)

    def sync_shadow(self, ff=False):
        """q32 <- q (FP32 shadow of the state), or q_ff <- q with ``ff``."""
        L.op2b_dat_copy(self.ctx, self.d["q_ff" if ff else "q32"], self.d["q"])

    def _inviscid_only(self, what):
        if self.visc is not None or LIMITERS[self.limiter]:
            raise NotImplementedError(what + " loops cover the inviscid residual with the van "
                                      "Albada limiter only")

    def adjoint(self, order=2, recompute_gradient=True, ff=False):
        """qbar = dJ/dq (dat qbar) and nbar = dJ/dn (dat nbar) of J = lam . R.

        The edge states are recomputed from the node data.  With
        ``recompute_gradient=False`` the dat G must still hold the gradient
        of the current q and n (as the forward residual left it; G_ff with
        ``ff``).  ``ff``: the flux adjoint in float-float arithmetic from
        the float-float shadows of lam, q, G, n and dx (q_ff must match q);
        the scaling and Green-Gauss adjoints stay FP64."""
        self._inviscid_only("adjoint")
        c = self.ctx
        if ff:
            if order != 2:
                raise ValueError("the float-float adjoint is the second-order one")
            if recompute_gradient:
                self.green_gauss(ff=True)
            L.op2b_dat_copy(c, self.d["lam_ff"], self.d["lam"])
            L.op2b_edge_flux_adjoint(c, self.a_fa2_ff, 2, self.gamma, self.eps_lim, L.ZERO_INC)
            L.op2b_grad_scale_adjoint(c, self.d["Gbar"], self.d["V"])
            L.op2b_green_gauss_adjoint(c, self.a_gga, 0)
            return
        if order == 1:
            L.op2b_edge_flux_adjoint(c, self.a_fa1, 1, self.gamma, self.eps_lim, L.ZERO_INC)
            return
        if recompute_gradient:
            self.green_gauss()
        L.op2b_edge_flux_adjoint(c, self.a_fa2, 2, self.gamma, self.eps_lim, L.ZERO_INC)
        L.op2b_grad_scale_adjoint(c, self.d["Gbar"], self.d["V"])
        L.op2b_green_gauss_adjoint(c, self.a_gga, 0)

    def tangent(self, order=2, recompute_gradient=True, ff=False):
        """Rd = dR/dq . qd + dR/dn . nd (dats qd, nd in, Rd out).

        With ``recompute_gradient=False`` the dat G must hold the gradient of
        the current q and n (G_ff with ``ff``).  ``ff``: the flux tangent in
        float-float arithmetic from the float-float shadows (q_ff must match
        q); the Green-Gauss tangent and its scaling stay FP64."""
        self._inviscid_only("tangent")
        c = self.ctx
        if ff:
            if order != 2:
                raise ValueError("the float-float tangent is the second-order one")
            if recompute_gradient:
                self.green_gauss(ff=True)
            L.op2b_green_gauss_tangent(c, self.a_ggt, L.ZERO_INC)
            L.op2b_grad_scale(c, self.d["Gd"], self.d["V"])
            for nm in ("qd", "Gd", "nd"):
                L.op2b_dat_copy(c, self.d[nm + "_ff"], self.d[nm])
            L.op2b_edge_flux_tangent(c, self.a_ft2_ff, 2, self.gamma, self.eps_lim, L.ZERO_INC)
            return
        if order == 1:
            L.op2b_edge_flux_tangent(c, self.a_ft1, 1, self.gamma, self.eps_lim, L.ZERO_INC)
            return
        if recompute_gradient:
            self.green_gauss()
        L.op2b_green_gauss_tangent(c, self.a_ggt, L.ZERO_INC)
        L.op2b_grad_scale(c, self.d["Gd"], self.d["V"])
        L.op2b_edge_flux_tangent(c, self.a_ft2, 2, self.gamma, self.eps_lim, L.ZERO_INC)

    # ------------------------------------------------ march derivatives
    def march_tangent(self, steps, order=2, stages=5):
        """Advance q and its tangent qd together by `steps` RK steps with
        the fixed local time step in dat dt: on return qd holds
        dq_N/dq_0 . qd + dq_N/dn . nd (dats qd, nd on entry)."""
        self._inviscid_only("tangent")
        c, d = self.ctx, self.d
        for _ in range(steps):
            L.op2b_dat_copy(c, d["q0"], d["q"])
            L.op2b_dat_copy(c, d["qd0"], d["qd"])
            for a in RK5_ALPHA[5 - stages:]:
                self.residual(order)
                self.tangent(order, recompute_gradient=False)
                L.op2b_node_update(c, d["qd0"], d["qd"], d["Rd"], d["V"], d["dt"], a, -1)
                L.op2b_node_update(c, d["q0"], d["q"], d["R"], d["V"], d["dt"], a, -1)

    def march_adjoint(self, steps, order=2, stages=5, keep_gradients=True):
        """Reverse of `steps` RK steps with the fixed dt (dat dt) for
        J = g . q_N.  On entry dat sbar holds g and q holds q_0; on return
        sbar holds dJ/dq_0, nbar_acc dJ/dn, and q holds q_N.

        The forward march keeps the input state of every stage resident
        (steps * stages + 1 states of 6 N doubles) and, with
        ``keep_gradients`` (order 2), the gradient of every stage (18 N
        doubles each) instead of recomputing it in the reverse sweep: the
        stage loops read and write the stored slices directly (the dats
        are rebound), so nothing is copied."""
        self._inviscid_only("adjoint")
        torch, c, d, t = self.torch, self.ctx, self.d, self.t
        K = steps * stages
        ld = t["q"].shape[1]
        S = torch.empty((K + 1, 6, ld), dtype=torch.float64, device=self.device)
        GS = (torch.empty((max(K, 1), 18, ld), dtype=torch.float64, device=self.device)
              if keep_gradients and order == 2 else None)
        q_t, q0_t, G_t = t["q"], t["q0"], t["G"]
        alphas = RK5_ALPHA[5 - stages:]
        try:
            self.rebind("q0", S[0])
            L.op2b_dat_copy(c, d["q0"], d["q"])
            for st in range(steps):
                self.rebind("q0", S[st * stages])
                for k, a in enumerate(alphas):
                    idx = st * stages + k
                    self.rebind("q", S[idx])
                    if GS is not None:
                        self.rebind("G", GS[idx])
                    self.residual(order)
                    self.rebind("q", S[idx + 1])
                    L.op2b_node_update(c, d["q0"], d["q"], d["R"], d["V"], d["dt"], a, -1)
            L.op2b_dat_fill(c, d["nbar_acc"], 0.0)
            for st in reversed(range(steps)):
                L.op2b_dat_fill(c, d["qacc"], 0.0)
                for k in reversed(range(stages)):
                    idx = st * stages + k
                    L.op2b_node_update_adjoint(c, d["sbar"], d["qacc"], d["lam"], d["V"],
                                               d["dt"], alphas[k])
                    self.rebind("q", S[idx])
                    if GS is not None:
                        self.rebind("G", GS[idx])
                    self.adjoint(order, recompute_gradient=GS is None)
                    L.op2b_dat_axpy(c, d["nbar_acc"], 1.0, d["nbar"])
                    sb, qb = t["sbar"], t["qbar"]  # sbar <- qbar by swapping buffers
                    self.rebind("sbar", qb)
                    self.rebind("qbar", sb)
                L.op2b_dat_axpy(c, d["sbar"], 1.0, d["qacc"])
            self.rebind("q0", S[K])
        finally:
            self.rebind("q", q_t)
            self.rebind("G", G_t)
        L.op2b_dat_copy(c, d["q"], d["q0"])
        self.rebind("q0", q0_t)

    def reduce(self, name, op):
        """Per-component reduction of dat `name` (op: op2b.RED_*), as a
        device tensor (asynchronous)."""
        out = self.torch.empty(self.t[name].shape[0], dtype=self.torch.float64,
                               device=self.device)
        L.op2b_dat_reduce(self.ctx, self.d[name], op, out.data_ptr())
        return out

    def launch_count(self):
        return L.op2b_launch_count(self.ctx)

    def close(self):
        if self.ctx is not None:
            L.op2b_finalize(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
