"""Benchmark of the edge-loop hot path on one GB300 (or N replicas).

One step = one explicit second-order Runge-Kutta stage in FP64 on the
200^3 periodic jittered lattice (8,000,000 nodes, 72,000,000 edges, RCM
numbering, every loop's strategy autotuned): Green-Gauss edge loop with the
gradient scaling, limited Rusanov flux edge loop, node update.  value =
edges / stage time (whole job over all ranks).  Also reported on the same
mesh: the per-loop times, the roofline of the dominant kernel, the
FP32-mixed stage, the adjoint sweep, 50-step marches, an end-to-end figure
through host buffers; on the 100^3 lattice (1M nodes, 9M edges) the same
stage under RCM and random numbering and the other loops of the library;
and the CPU oracle's rate on a bounded sample, with its 50-step march on
the 40^3 lattice as the reference of the GPU marches.

``--impl reference`` times the CPU oracle instead (serial FP64 C) on a
bounded sample of the same workload.  With N > 1 (torchrun) every rank runs
its own replica of the mesh: the edge loops have no exchange step on one
mesh per GPU.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s & HBM GB/s (FP64, FP32-mixed, adjoint) vs oracle; fraction of roofline"

# Algorithmic (compulsory) bytes per edge of each loop: edge data read once
# (map 8 B, n and dx 3 values each), node data read once and INC targets
# written once, node bytes spread over the 9 edges per node.  "gg": the
# Green-Gauss loop with the gradient scaling (q, n and V read, G written
# once, as the fused pass does).
BYTES_PER_EDGE = {"gg": 8 + 24 + (48 + 8 + 144) / 9, "flux2": 8 + 24 + 24 + (48 + 144 + 48) / 9,
                  "scale": 296 / 9, "update": 160 / 9}
BYTES_PER_EDGE_F32 = {"gg": 8 + 12 + (24 + 8 + 72) / 9, "flux2": 8 + 12 + 12 + (24 + 72 + 48) / 9,
                      "scale": 148 / 9, "update": 184 / 9}
# FP64 operations per edge of the flux2 definition (reconstruction 198 +
# Rusanov 97), each add, multiply, divide and square root counted once.
FLOPS_PER_EDGE_FLUX2 = 295.0
# Viscous flux edge loop: per edge the map (8), n and dx (48), and per node
# (9 edges per node) W read (160) and R read + write (96); the node pass
# reads q and G (192) and writes W (160) per node.  FP64 operations per
# edge of the loop body as written (multiply-add = 2, the reciprocal = 1).
BYTES_PER_EDGE_VISC = {"prims": 352 / 9, "visc": 8 + 48 + (160 + 96) / 9}
BYTES_PER_EDGE_VISC_F32 = {"prims": 176 / 9, "visc": 8 + 24 + (80 + 96) / 9}
FLOPS_PER_EDGE_VISC = 146.0
VISC_COEFFS = (1.0e-3, 0.72, 1.0e-3)  # mu, Prandtl number, scalar diffusivity
# DRAM bytes per edge of the FP64 flux2 kernel (atomic strategy, 128 threads)
# from an ncu capture on the 60^3 lattice (dram__bytes_read.sum +
# dram__bytes_write.sum = 170.81 MB over 1,944,000 edges;
# profiles/ncu_flux_gg_kernels_n60.md), scaled to a launch by its edge
# count.  Traffic grows in proportion to the edges.
DRAM_BYTES_PER_EDGE_FLUX2_ATOMIC = 170.809088e6 / 1944000
# FP64 instructions per edge of the same kernel in the same capture
# (smsp__sass_thread_inst_executed_op_{dfma,dmul,dadd}_pred_on per cycle x
# cycles / edges: 106.6 DFMA + 85.8 DMUL + 31.0 DADD)
FP64_INSTR_PER_EDGE_FLUX2 = 223.5
# FP64 instruction peak: 152 SMs x 2 per clock x 2.07 GHz
FP64_PEAK_GINSTR = 152 * 2 * 2.07


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 ALU peak: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons while timing.

    The sampler starts before the warm-up (``start()``), a reader thread
    stamps every line with the host time it arrived, and ``summary()`` keeps
    the samples that arrived between ``mark_begin()`` and ``mark_end()`` (the
    timed region), so that a short timed region still gets its own samples.
    """

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.samples = []  # (host time, line)
        self.t_begin = self.t_end = None
        self._thread = None

    def _reader(self):
        for line in self.proc.stdout:
            if line.strip():
                self.samples.append((time.perf_counter(), line))

    def start(self, wait_s=3.0):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        self._thread = threading.Thread(target=self._reader, daemon=True)
        self._thread.start()
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < wait_s:
            time.sleep(0.01)
        return self

    def mark_begin(self):
        self.t_begin = time.perf_counter()

    def mark_end(self):
        # the last period's sample may still be on its way
        time.sleep(2 * self.PERIOD_MS / 1e3)
        self.t_end = time.perf_counter()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self._thread is not None:
                self._thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = self.t_begin if self.t_begin is not None else -1e300
        hi = self.t_end if self.t_end is not None else 1e300
        for t, l in list(self.samples):
            if not lo <= t <= hi:
                continue
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": self.PERIOD_MS}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def build_mesh(n, numbering=None):
    from paper_1403_7209_gb300 import meshgen
    m = meshgen.lattice(n)
    q = meshgen.flow_state(m)
    return m, q


# The oracle's bounded sample of a lattice: the first 1/8 of the edges in
# generation order (those leaving the lowest eighth of the lattice's planes,
# n^3 / 8 nodes: a slab of the same mesh) and the nodes they touch, renumbered
# compactly.  Same per-edge work, same state distribution, 1/8 of the edges.
SAMPLE_FRACTION = 8


def sample_submesh(m, q, frac=SAMPLE_FRACTION):
    E = m.num_edges // frac
    e = m.edge[:E]
    nodes, inv = np.unique(e.ravel(), return_inverse=True)
    return (inv.reshape(-1, 2).astype(np.int32), np.ascontiguousarray(q[nodes]),
            np.ascontiguousarray(m.normal[:E]), np.ascontiguousarray(m.dx[:E]),
            np.ascontiguousarray(m.volume[nodes]))


def cpu_baseline_run(m, q, stages, warmup=0, n=0):
    """CPU-baseline leg: time the oracle (as it stands) on `stages`
    second-order RK stages of the bounded sample of the mesh, after
    `warmup` untimed ones.  Returns (edges/s, seconds, sample text)."""
    import oracle
    oracle.build()
    edge, qs, nrm, dx, V = sample_submesh(m, q)
    lam = oracle.spectral_radius(edge, qs, nrm)
    dt = oracle.time_step(V, lam, 0.5)
    qq = qs
    for k in range(warmup):
        R, _ = oracle.residual(2, edge, qq, nrm, dx, V)
        qq = oracle.rk_update(qs, R, V, dt, 0.25)
    t0 = time.perf_counter()
    for k in range(stages):
        R, _ = oracle.residual(2, edge, qq, nrm, dx, V)
        qq = oracle.rk_update(qs, R, V, dt, 0.25)
    t = time.perf_counter() - t0
    sample = ("second-order RK stages (Green-Gauss, scaling, flux, update) of the oracle on the "
              "first 1/%d of the %d^3 lattice's edges (%d edges, %d nodes: a slab of the same "
              "mesh), serial C on one host core" % (SAMPLE_FRACTION, n, edge.shape[0], V.shape[0]))
    return edge.shape[0] * stages / t, t, sample


def cpu_baseline_march_child(n, steps):
    """CPU-baseline leg, run in a spawned process while the GPU works: the
    oracle's 50-step march on the n^3 lattice (cached on disk by
    oracle.march_cache), the reference of the GPU marches."""
    sys.path.insert(0, ROOT)
    from oracle import march_cache
    march_cache.oracle_march(n, steps)


def run_reference(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return 0
    m, q = build_mesh(args.n)
    steps = max(1, args.steps)
    rate, t, sample = cpu_baseline_run(m, q, steps, warmup=args.warmup, n=args.n)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "edges/s",
        "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, m),
        "cpu_baseline": {"value": rate, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": "%d timed (after %d untimed) %s" % (steps, args.warmup, sample)},
        "e2e": {"value": rate, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(args, m):
    return {"workload": "second-order FP64 explicit RK stage (Green-Gauss + gradient scaling + "
                        "van Albada-limited Rusanov flux + node update) on the %d^3 periodic "
                        "jittered lattice" % args.n,
            "nodes": m.num_nodes, "edges": m.num_edges, "numbering": args.numbering,
            "l2": "inputs larger than L2 (node + edge data %.0f MB vs 129 MB L2)" %
                  ((m.num_nodes * (6 * 4 + 18 + 3) * 8 + m.num_edges * (6 * 8 + 8)) / 1e6),
            "parallelism": "replicas (one mesh per GPU)"}


def reduce_max_ms(ms, dist, device=None):
    """Max over ranks of the per-rank step time: the slowest replica sets
    the job's time."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(edges_per_rank, world_size, ms):
    """Whole-job edges per second: all ranks' edges over the max step time."""
    return world_size * edges_per_rank / (ms * 1e-3)


def timed(torch, fn, steps, stream):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(steps):
        fn()
    ev[1].record(stream)
    torch.cuda.synchronize()
    return ev[0].elapsed_time(ev[1]) / steps


def loop_events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def mixed_extra(torch, L, s, args, stream, ms64, E, N):
    """FP32-mixed stage: per-loop times, speed-up and residual error."""
    s.sync_shadow()
    names = ["gg32", "flux2_32", "update"]

    def stage(ev=None):
        if ev: ev[0].record(stream)
        L.op2b_green_gauss_scaled(s.ctx, s.a_gg32, s.d["V"], L.ZERO_INC)
        if ev: ev[1].record(stream)
        L.op2b_edge_flux(s.ctx, s.a_f2_32, 2, s.gamma, s.eps_lim, L.ZERO_INC)
        if ev: ev[2].record(stream)
        L.op2b_node_update(s.ctx, s.d["q0"], s.d["q"], s.d["R"], s.d["V"], s.d["dt"], 0.25,
                           s.d["q32"])
        if ev: ev[3].record(stream)
    for _ in range(args.warmup):
        stage()
    evs = [loop_events(torch, 4) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0, t1 = loop_events(torch, 2)
    t0.record(stream)
    for k in range(args.steps):
        stage(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    mms = t0.elapsed_time(t1) / args.steps
    loops = {nm: statistics.mean(evs[k][j].elapsed_time(evs[k][j + 1]) for k in range(args.steps))
             for j, nm in enumerate(names)}
    bpe = {"gg32": BYTES_PER_EDGE_F32["gg"], "flux2_32": BYTES_PER_EDGE_F32["flux2"],
           "update": BYTES_PER_EDGE_F32["update"]}
    strat = {"gg32": L.STRATEGY_NAMES[s.plan_stats(L.LOOP_GREEN_GAUSS, 1)["strategy"]],
             "flux2_32": L.STRATEGY_NAMES[s.plan_stats(L.LOOP_FLUX2, 1)["strategy"]]}
    hbm, _ = read_peaks()
    out_loops = {nm: {"ms": loops[nm], "gbs": bpe[nm] * E / (loops[nm] * 1e-3) / 1e9,
                      "hbm_frac": bpe[nm] * E / (loops[nm] * 1e-3) / 1e9 / hbm,
                      "strategy": strat.get(nm, "direct")} for nm in names}
    # residual error of the mixed path against the FP64 path on one state
    s.sync_shadow()
    s.residual(2)
    R64 = s.t["R"][:, :N].clone()
    s.residual(2, mixed=True)
    R32 = s.t["R"][:, :N].clone()
    rerr = ((R32 - R64).abs().amax(dim=1) / R64.abs().amax(dim=1)).cpu().tolist()
    out = {"ms_per_stage": mms, "edges_per_s": E / (mms * 1e-3), "speedup_vs_fp64": ms64 / mms,
           "loops": out_loops, "residual_rel_err_per_component": rerr}
    out["fused"] = fused_extra(torch, L, s, args, stream, ms64, E, N, R64)
    return out


# Algorithmic bytes per node of the FP32-mixed stage: the Green-Gauss loop
# with its scaling, the flux loop and the update (BYTES_PER_EDGE_F32, nine
# edges per node), the unit of the fused stage's HBM roofline.
BYTES_PER_NODE_MIXED_STAGE = 9 * (BYTES_PER_EDGE_F32["gg"] + BYTES_PER_EDGE_F32["flux2"]
                                  + BYTES_PER_EDGE_F32["update"])
# DRAM bytes per node the fused stage's two passes move (ncu, 60^3 lattice:
# Green-Gauss 86.5 + 2.5 MB, flux + update 164.1 + 10.3 MB for 216,000 nodes)
DRAM_BYTES_PER_NODE_FUSED = (86.5e6 + 2.5e6 + 164.1e6 + 10.3e6) / 216000


def fused_extra(torch, L, s, args, stream, ms64, E, N, R64):
    """The fused FP32-mixed stage (op2b_stage_mixed: a Green-Gauss node pass
    and a flux + update node pass over packed FP32 records): stage time,
    fraction of the HBM roofline of the stage's algorithmic bytes, residual
    error against the FP64 path."""
    L.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.stage_fused(0.25, sync=True, residual=False)
    for _ in range(args.warmup):
        s.stage_fused(0.25, residual=False)
    ms = timed(torch, lambda: s.stage_fused(0.25, residual=False), args.steps, stream)
    ms_r = timed(torch, lambda: s.stage_fused(0.25), args.steps, stream)
    hbm, src = read_peaks()
    gbs = BYTES_PER_NODE_MIXED_STAGE * N / (ms * 1e-3) / 1e9
    # the residual of the step's state against the FP64 path's
    L.op2b_dat_copy(s.ctx, s.d["q"], s.d["q0"])
    s.stage_fused(0.0, sync=True)
    Rf = s.t["R"][:, :N].clone()
    rerr = ((Rf - R64).abs().amax(dim=1) / R64.abs().amax(dim=1)).cpu().tolist()
    dram = DRAM_BYTES_PER_NODE_FUSED * N / (ms * 1e-3) / 1e9
    return {"ms_per_stage": ms, "ms_per_stage_writing_R": ms_r,
            "edges_per_s": E / (ms * 1e-3), "speedup_vs_fp64": ms64 / ms,
            "algorithmic_bytes_per_node": BYTES_PER_NODE_MIXED_STAGE,
            "gbs": gbs, "hbm_frac": gbs / hbm, "hbm_peak_source": src,
            "dram_bytes_per_node": DRAM_BYTES_PER_NODE_FUSED, "dram_gbs": dram,
            "dram_frac": dram / hbm,
            "dram_note": "DRAM bytes per node of the two passes from their 60^3 ncu captures "
                         "(read + write, the stage without R): the per-end records are streamed "
                         "rather than gathered, 1.35x the algorithmic bytes",
            "residual_rel_err_per_component": rerr}


def ff_extra(torch, L, s, args, stream, ms64, E, N):
    """Float-float stage: Green-Gauss (node gather) and scaling in
    float-float from the float-float shadows of q and n, the second-order
    flux in float-float arithmetic (FP32 units, FP64 residual), the FP64
    update that also writes the float-float shadow of q; per-loop times,
    speed-up over the FP64 stage and the residual's difference from the
    FP64 path's."""
    names = ["gg_ff", "flux2_ff", "update"]
    s.set_strategy(L.LOOP_FLUX2, L.PREC_FF, L.STRAT_AUTO)
    s.sync_shadow(ff=True)

    def stage(ev=None):
        if ev: ev[0].record(stream)
        L.op2b_green_gauss_scaled(s.ctx, s.a_gg_ff, s.d["V"], L.ZERO_INC)
        if ev: ev[1].record(stream)
        L.op2b_edge_flux(s.ctx, s.a_f2_ff, 2, s.gamma, s.eps_lim, L.ZERO_INC)
        if ev: ev[2].record(stream)
        L.op2b_node_update(s.ctx, s.d["q0"], s.d["q"], s.d["R"], s.d["V"], s.d["dt"], 0.25,
                           s.d["q_ff"])
        if ev: ev[3].record(stream)
    for _ in range(args.warmup):
        stage()
    evs = [loop_events(torch, 4) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0, t1 = loop_events(torch, 2)
    t0.record(stream)
    for k in range(args.steps):
        stage(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    fms = t0.elapsed_time(t1) / args.steps
    loops = {nm: statistics.mean(evs[k][j].elapsed_time(evs[k][j + 1]) for k in range(args.steps))
             for j, nm in enumerate(names)}
    fl = loops["flux2_ff"]
    hbm, _ = read_peaks()
    # difference from the FP64 path on one state (same q, same G)
    s.sync_shadow(ff=True)
    s.residual(2)
    R64 = s.t["R"][:, :N].clone()
    s.residual(2, ff=True)
    Rff = s.t["R"][:, :N].clone()
    diff = ((Rff - R64).abs().amax(dim=1) / R64.abs().amax(dim=1)).tolist()
    return {"ms_per_stage": fms, "edges_per_s": E / (fms * 1e-3), "speedup_vs_fp64": ms64 / fms,
            "loops": {nm: {"ms": loops[nm]} for nm in names},
            "flux2_ff": {"ms": fl, "edges_per_s": E / (fl * 1e-3),
                         "strategy": L.STRATEGY_NAMES[s.plan_stats(L.LOOP_FLUX2, L.PREC_FF)["strategy"]],
                         "fp64_equivalent_tflops": FLOPS_PER_EDGE_FLUX2 * E / (fl * 1e-3) / 1e12,
                         "vs_fp64_peak": FLOPS_PER_EDGE_FLUX2 * E / (fl * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "gbs": BYTES_PER_EDGE["flux2"] * E / (fl * 1e-3) / 1e9,
                         "hbm_frac": BYTES_PER_EDGE["flux2"] * E / (fl * 1e-3) / 1e9 / hbm},
            "residual_max_diff_vs_fp64_path_per_component": diff}


def adjoint_extra(torch, L, s, args, stream, E):
    """Reverse sweep (flux adjoint, scaling adjoint, Green-Gauss adjoint;
    edge states recomputed, G kept from the forward pass) against the
    forward residual (Green-Gauss, scaling, flux) it differentiates."""
    s.t["lam"].normal_()
    s.residual(2)
    for _ in range(max(1, args.warmup)):
        s.adjoint(2, recompute_gradient=False)
    ams = timed(torch, lambda: s.adjoint(2, recompute_gradient=False), args.steps, stream)
    rms = timed(torch, lambda: s.adjoint(2), args.steps, stream)
    fms = timed(torch, lambda: s.residual(2), args.steps, stream)
    out = {"ms": ams, "forward_residual_ms": fms, "ratio_to_forward": ams / fms,
           "ms_with_gradient_recompute": rms, "edges_per_s": E / (ams * 1e-3)}
    if s.ff:  # the flux adjoint in float-float (scaling and Green-Gauss adjoints FP64)
        s.sync_shadow(ff=True)
        s.residual(2, ff=True)
        for _ in range(max(1, args.warmup)):
            s.adjoint(2, recompute_gradient=False, ff=True)
        fams = timed(torch, lambda: s.adjoint(2, recompute_gradient=False, ff=True), args.steps,
                     stream)
        ffms = timed(torch, lambda: s.residual(2, ff=True), args.steps, stream)
        out["float_float"] = {"ms": fams, "forward_residual_ms": ffms,
                              "ratio_to_forward": fams / ffms, "speedup_vs_fp64_adjoint": ams / fams,
                              "strategy": L.STRATEGY_NAMES[
                                  s.plan_stats(L.LOOP_FLUX2_ADJ, L.PREC_FF)["strategy"]]}
    return out


def tangent_extra(torch, L, s, args, stream, E):
    """Jacobian-vector product (tangent loops, G kept from the forward pass)."""
    s.t["qd"].normal_()
    s.t["nd"].normal_()
    s.residual(2)
    for _ in range(max(1, args.warmup)):
        s.tangent(2, recompute_gradient=False)
    tms = timed(torch, lambda: s.tangent(2, recompute_gradient=False), args.steps, stream)
    fms = timed(torch, lambda: s.residual(2), args.steps, stream)
    out = {"ms": tms, "forward_residual_ms": fms, "ratio_to_forward": tms / fms,
           "edges_per_s": E / (tms * 1e-3)}
    if s.ff:  # the flux tangent in float-float (Green-Gauss tangent and scaling FP64)
        s.sync_shadow(ff=True)
        s.residual(2, ff=True)
        for _ in range(max(1, args.warmup)):
            s.tangent(2, recompute_gradient=False, ff=True)
        ftms = timed(torch, lambda: s.tangent(2, recompute_gradient=False, ff=True), args.steps,
                     stream)
        out["float_float"] = {"ms": ftms, "speedup_vs_fp64_tangent": tms / ftms,
                              "strategy": L.STRATEGY_NAMES[
                                  s.plan_stats(L.LOOP_FLUX2_TAN, L.PREC_FF)["strategy"]]}
    return out


def viscous_extra(torch, L, m, q, args, stream, device, E):
    """Navier-Stokes residual: the viscous node pass and edge loop alone
    (FP64, FP32-mixed and float-float) and the whole stage with them
    (Green-Gauss, scaling, limited inviscid flux, viscous flux, update)."""
    from paper_1403_7209_gb300.solver import EdgeSolver
    sv = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, device=device,
                    renumber=args.numbering, mixed=True, stream=stream, viscous=VISC_COEFFS,
                    ff=True)
    if args.tune_cache and os.path.exists(args.tune_cache):
        L.op2b_load_tuning(sv.ctx, args.tune_cache)
    for loop in range(L.NUM_LOOPS):
        for prec in range(L.NUM_PREC):
            sv.set_strategy(loop, prec, L.STRAT_AUTO)
    sv.time_step(0.5)
    L.op2b_dat_copy(sv.ctx, sv.d["q0"], sv.d["q"])
    sv.sync_shadow()
    mu, pr, diff = VISC_COEFFS
    out = {"coefficients": {"mu": mu, "prandtl": pr, "diff": diff}}
    hbm, _ = read_peaks()
    for tag, mixed, ff in (("fp64", False, False), ("mixed", True, False),
                           ("float_float", False, True)):
        sv.residual(2, mixed=mixed, ff=ff)  # tunes every loop of the stage
        q_, G_, W_ = ("q32", "G32", "W32") if mixed else (
            ("q_ff", "G_ff", "W_ff") if ff else ("q", "G", "W"))
        args_v = sv.a_vf32 if mixed else (sv.a_vf_ff if ff else sv.a_vf)
        prec = L.PREC_F32 if mixed else (L.PREC_FF if ff else L.PREC_F64)

        def prims():
            L.op2b_viscous_prims(sv.ctx, sv.d[q_], sv.d[G_], sv.d[W_], sv.gamma)

        def visc():
            L.op2b_viscous_flux(sv.ctx, args_v, sv.gamma, mu, pr, diff, 0)
        for _ in range(max(1, args.warmup)):
            prims()
            visc()
        pms = timed(torch, prims, args.steps, stream)
        vms = timed(torch, visc, args.steps, stream)
        sms = timed(torch, lambda: sv.stage(0.25, 2, mixed=mixed, ff=ff), args.steps, stream)
        bpe = BYTES_PER_EDGE_VISC_F32 if mixed else BYTES_PER_EDGE_VISC
        r = {"prims_ms": pms, "visc_ms": vms, "ns_stage_ms": sms,
             "ns_stage_edges_per_s": E / (sms * 1e-3),
             "visc_strategy": L.STRATEGY_NAMES[sv.plan_stats(L.LOOP_VISCOUS, prec)["strategy"]],
             "visc_gbs": bpe["visc"] * E / (vms * 1e-3) / 1e9,
             "visc_hbm_frac": bpe["visc"] * E / (vms * 1e-3) / 1e9 / hbm,
             "prims_gbs": bpe["prims"] * E / (pms * 1e-3) / 1e9}
        if not mixed:  # FP64-equivalent for float-float
            ach = FLOPS_PER_EDGE_VISC * E / (vms * 1e-3) / 1e12
            r["visc_fp64_tflops"] = ach
            r["visc_fp64_frac"] = ach / FP64_PEAK_TFLOPS
        out[tag] = r
    # error of the mixed viscous loop against the FP64 one on one state
    sv.load_nodes("q", q)
    sv.sync_shadow()
    sv.green_gauss()
    sv.viscous_flux(zero=True)
    R64 = sv.t["R"][:, :sv.N].clone()
    sv.green_gauss(mixed=True)
    sv.viscous_flux(mixed=True, zero=True)
    R32 = sv.t["R"][:, :sv.N].clone()
    out["mixed_visc_rel_err_per_component"] = (
        (R32 - R64)[1:].abs().amax(dim=1) / R64[1:].abs().amax(dim=1)).cpu().tolist()
    sv.sync_shadow(ff=True)
    sv.green_gauss(ff=True)
    sv.viscous_flux(zero=True, ff=True)
    Rff = sv.t["R"][:, :sv.N].clone()
    out["float_float_visc_max_diff_vs_fp64_per_component"] = (
        (Rff - R64)[1:].abs().amax(dim=1) / R64[1:].abs().amax(dim=1)).cpu().tolist()
    out["fp64_ns_stage_vs_euler_stage"] = None
    sv.close()
    return out


def limiter_extra(torch, L, m, q, args, stream, device, E, ms_va):
    """Node-limited second-order scheme: neighbourhood min/max, the
    Barth-Jespersen and Venkatakrishnan limiters, the node-limited flux, and
    the whole stage with them against the van Albada stage."""
    from paper_1403_7209_gb300.solver import EdgeSolver
    sl = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, device=device,
                    renumber=args.numbering, mixed=True, stream=stream,
                    limiter="barth_jespersen", ff=True)
    if args.tune_cache and os.path.exists(args.tune_cache):
        L.op2b_load_tuning(sl.ctx, args.tune_cache)
    for loop in range(L.NUM_LOOPS):
        for prec in range(L.NUM_PREC):
            sl.set_strategy(loop, prec, L.STRAT_AUTO)
    sl.time_step(0.5)
    L.op2b_dat_copy(sl.ctx, sl.d["q0"], sl.d["q"])
    sl.sync_shadow()
    sl.sync_shadow(ff=True)
    c, d = sl.ctx, sl.d
    out = {}
    for tag, mixed, ff in (("fp64", False, False), ("mixed", True, False),
                           ("float_float", False, True)):
        sfx = "32" if mixed else ("_ff" if ff else "")
        qn, Gn, dxn = "q" + sfx, "G" + sfx, "dx" + sfx
        prec = L.PREC_F32 if mixed else (L.PREC_FF if ff else L.PREC_F64)
        sl.residual(2, mixed=mixed, ff=ff)  # tunes
        for _ in range(max(1, args.warmup)):
            sl.stage(0.25, 2, mixed=mixed, ff=ff)

        def mm():
            L.op2b_node_minmax(c, sl.map, d[qn], d["qmin" + sfx], d["qmax" + sfx])

        def lim(kind):
            L.op2b_node_limiter(c, sl.map, kind, 0.0, d[qn], d[Gn], d[dxn], d["qmin" + sfx],
                                d["qmax" + sfx], d["phi" + sfx])

        def fl():
            L.op2b_edge_flux_limited(c, sl.a_f2phi32 if mixed else (sl.a_f2phi_ff if ff else
                                                                     sl.a_f2phi), sl.gamma,
                                     L.ZERO_INC)
        r = {"minmax_ms": timed(torch, mm, args.steps, stream),
             "limiter_bj_ms": timed(torch, lambda: lim(L.LIM_BARTH_JESPERSEN), args.steps, stream),
             "limiter_venkat_ms": timed(torch, lambda: lim(L.LIM_VENKATAKRISHNAN), args.steps,
                                        stream),
             "flux_limited_ms": timed(torch, fl, args.steps, stream),
             "stage_ms": timed(torch, lambda: sl.stage(0.25, 2, mixed=mixed, ff=ff), args.steps,
                               stream),
             "flux_strategy": L.STRATEGY_NAMES[sl.plan_stats(L.LOOP_FLUX2_PHI, prec)["strategy"]]}
        r["stage_edges_per_s"] = E / (r["stage_ms"] * 1e-3)
        out[tag] = r
    out["fp64"]["stage_vs_van_albada_stage"] = out["fp64"]["stage_ms"] / ms_va
    sl.close()
    return out


def block_jacobi_extra(torch, L, m, q, args, stream, device, E):
    """Block-Jacobi preconditioning (FP64): the factored blocks (edge loop
    of four sums, one node pass forming and inverting the blocks) and the
    direct form (36-value edge loop, inversion loop), each tuned; the
    preconditioned update, and a preconditioned step (blocks and inverses of
    the step's initial state, five stages) against a plain step."""
    from paper_1403_7209_gb300.solver import EdgeSolver
    sj = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, device=device,
                    renumber=args.numbering, stream=stream, precond=True)
    if args.tune_cache and os.path.exists(args.tune_cache):
        L.op2b_load_tuning(sj.ctx, args.tune_cache)
    for loop in range(L.NUM_LOOPS):
        for prec in range(L.NUM_PREC):
            sj.set_strategy(loop, prec, L.STRAT_AUTO)
    sj.time_step(0.5)
    c, d = sj.ctx, sj.d
    sj.precondition(factored=False)  # tunes both blocks' loops
    sj.precondition()
    sj.residual(2)
    L.op2b_dat_copy(c, d["q0"], d["q"])
    nb = max(2, args.steps // 4)
    out = {
        "sums_ms": timed(torch, lambda: L.op2b_jacobi_sums(c, sj.a_jsum, sj.gamma, L.ZERO_INC),
                         nb, stream),
        "sums_strategy": L.STRATEGY_NAMES[sj.plan_stats(L.LOOP_JACOBI_SUMS)["strategy"]],
        "form_and_invert_ms": timed(torch, lambda: L.op2b_jacobi_from_sums(
            c, d["q"], d["JS"], -1, d["P"], sj.gamma), nb, stream),
        "direct_blocks_ms": timed(torch, lambda: L.op2b_jacobi_blocks(c, sj.a_jac, sj.gamma,
                                                                      L.ZERO_INC), nb, stream),
        "direct_blocks_strategy": L.STRATEGY_NAMES[sj.plan_stats(L.LOOP_JACOBI)["strategy"]],
        "invert_ms": timed(torch, lambda: L.op2b_block_invert(c, d["M"], d["P"]), nb, stream),
        "update_precond_ms": timed(torch, lambda: L.op2b_node_update_precond(
            c, d["q0"], d["q"], d["R"], d["P"], 0.1), nb, stream),
    }
    q_keep = sj.t["q"].clone()
    out["precond_step_ms"] = timed(torch, lambda: sj.step(order=2, sigma=0.25), nb, stream)
    sj.t["q"].copy_(q_keep)
    out["step_ms"] = timed(torch, lambda: sj.step(order=2), nb, stream)
    out["precond_step_over_step"] = out["precond_step_ms"] / out["step_ms"]
    sj.close()
    return out


def march_adjoint_extra(torch, L, s, q, args, stream, E, steps=10):
    """Reverse sweep of a 10-step march (50 stages, dt fixed) with every
    stage's state and gradient kept in HBM, against the forward march."""
    N = s.N
    g = torch.randn((6, s.t["q"].shape[1]), dtype=torch.float64, device=s.device)

    def fwd():
        for _ in range(steps):
            s.step(order=2)

    def rev(keep):
        s.t["sbar"].copy_(g)
        s.march_adjoint(steps, order=2, keep_gradients=keep)
    s.load_nodes("q", q)
    s.time_step(0.5)
    rev(True)  # warm-up: tunes the loops, allocates the stage storage
    torch.cuda.synchronize()
    f_ms = timed(torch, fwd, 1, stream)
    s.load_nodes("q", q)
    r_ms = timed(torch, lambda: rev(True), 1, stream)
    s.load_nodes("q", q)
    rr_ms = timed(torch, lambda: rev(False), 1, stream)
    stored = (steps * 5 + 1) * 6 * N * 8 + steps * 5 * 18 * N * 8
    return {"steps": steps, "stages": 5 * steps, "forward_march_ms": f_ms,
            "adjoint_march_ms": r_ms, "ratio_to_forward": r_ms / f_ms,
            "adjoint_march_includes": "the forward march that stores every stage, then the "
                                      "reverse sweep",
            "adjoint_march_recompute_gradients_ms": rr_ms,
            "stored_gb": stored / 1e9, "edges_per_s_per_stage": E * 5 * steps / (r_ms * 1e-3)}


def lattice16_extra(torch, L, args):
    """First-order Rusanov residual on the 16^3 lattice (random numbering),
    the correctness configuration; launch-bound at 36,864 edges, so timed
    as a captured CUDA graph of 100 loop calls."""
    from paper_1403_7209_gb300 import meshgen
    from paper_1403_7209_gb300.solver import EdgeSolver
    m = meshgen.lattice(16)
    q = meshgen.flow_state(m)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, stream=st)
        s.set_strategy(L.LOOP_FLUX1, 0, L.STRAT_AUTO)
        for _ in range(3):
            s.flux(1)
        torch.cuda.synchronize()
        eager = timed(torch, lambda: s.flux(1), 100, st)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for _ in range(100):
                s.flux(1)
        g.replay()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(st)
        for _ in range(5):
            g.replay()
        ev[1].record(st)
        torch.cuda.synchronize()
        graph_ms = ev[0].elapsed_time(ev[1]) / 500
        strat = L.STRATEGY_NAMES[s.plan_stats(L.LOOP_FLUX1)["strategy"]]
        s.close()
    return {"mesh": "16^3 lattice, 4,096 nodes, 36,864 edges, random numbering",
            "loop": "first-order flux (R zeroed + edge loop)", "strategy": strat,
            "eager_us": eager * 1e3, "graph_us": graph_ms * 1e3,
            "edges_per_s_graph": m.num_edges / (graph_ms * 1e-3)}


def march_extra(torch, L, s, q, args, stream, steps=50):
    """50-step explicit march in FP64, in FP32-mixed and in float-float from
    the same state; relative max-norm state difference per component from
    the FP64 march after it."""
    N = s.N

    def run(mixed, ff=False):
        s.load_nodes("q", q)
        if mixed:
            s.sync_shadow()
        if ff:
            s.sync_shadow(ff=True)
        s.time_step(0.5)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(steps):
            s.step(order=2, mixed=mixed, ff=ff)
        torch.cuda.synchronize()
        return s.t["q"][:, :N].clone(), time.perf_counter() - t

    def rel(a, b):
        return ((a - b).abs().amax(dim=1) / b.abs().amax(dim=1)).cpu().tolist()
    q64, t64 = run(False)
    q32, t32 = run(True)
    s.load_nodes("q", q)
    s.time_step(0.5)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        s.step(fused=True)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t
    qf = s.t["q"][:, :N].clone()
    out = {"steps": steps, "stages_per_step": 5, "fp64_s": t64, "mixed_s": t32,
           "mixed_state_rel_err_per_component": rel(q32, q64),
           "fused_mixed_s": tf, "fused_mixed_state_rel_err_per_component": rel(qf, q64),
           "fp64_finite": bool(torch.isfinite(q64).all().item())}
    if s.ff:
        qff, tff = run(False, ff=True)
        out["float_float_s"] = tff
        out["float_float_state_rel_diff_per_component"] = rel(qff, q64)
    return out


def cpu_baseline_march_result(n, steps):
    """CPU-baseline leg: the oracle march's final state from the cache the
    spawned child wrote (computed here if the child could not)."""
    from oracle import march_cache
    q, status, t = march_cache.oracle_march(n, steps)
    return q, status


def march_oracle_extra(torch, L, args, stream, device, q_ora, n, steps):
    """50-step marches (250 stages) on the n^3 lattice in FP64 and in
    FP32-mixed against the oracle's march of the same mesh: normwise state
    error per component (max |q - q_oracle| / max |q_oracle|); the fused
    march also replayed from a CUDA graph (bitwise the eager march)."""
    from paper_1403_7209_gb300.solver import EdgeSolver
    m, q = build_mesh(n)
    out = {"mesh": "%d^3 lattice, %d nodes, %d edges, RCM" % (n, m.num_nodes, m.num_edges),
           "steps": steps, "stages_per_step": 5}
    for tag, mixed, fused in (("fp64", False, False), ("mixed", True, False),
                              ("fused_mixed", True, True)):
        # the fused march runs on a side stream, so that its steps can also be
        # captured in a CUDA graph below (same solver, same time step)
        st = torch.cuda.Stream(device=device) if fused else stream
        with torch.cuda.stream(st):
            s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, device=device, renumber="rcm",
                           mixed=mixed, stream=st)
            prec = L.PREC_F32 if mixed else L.PREC_F64
            for loop in range(L.NUM_LOOPS):
                s.set_strategy(loop, prec, L.STRAT_AUTO)
            s.time_step(0.5)
            s.residual(2, mixed=mixed)  # tunes the loops before the timed march
            torch.cuda.synchronize()
            t = time.perf_counter()
            for _ in range(steps):
                s.step(order=2, mixed=mixed, fused=fused)
            torch.cuda.synchronize()
            t = time.perf_counter() - t
            qg = s.fetch_nodes("q")
            err = (np.max(np.abs(qg - q_ora), axis=0) / np.max(np.abs(q_ora), axis=0)).tolist()
            out[tag] = {"state_err_vs_oracle_per_component": err, "gpu_march_s": t}
            if fused:
                # the same march, every step one replay of a CUDA graph captured
                # from a step (the launches of this small mesh's stages dominate)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=st):
                    s.step(fused=True)
                s.load_nodes("q", q)
                st.synchronize()
                t = time.perf_counter()
                for _ in range(steps):
                    g.replay()
                st.synchronize()
                t = time.perf_counter() - t
                out["fused_mixed_graph"] = {
                    "gpu_march_s": t,
                    "bitwise_equal_to_eager": bool(np.array_equal(s.fetch_nodes("q"), qg))}
            s.close()
    out["mixed_state_err_vs_oracle"] = max(out["mixed"]["state_err_vs_oracle_per_component"])
    out["fused_mixed_state_err_vs_oracle"] = max(
        out["fused_mixed"]["state_err_vs_oracle_per_component"])
    out["fp64_state_err_vs_oracle"] = max(out["fp64"]["state_err_vs_oracle_per_component"])
    out["bars"] = {"fp64": 1e-12, "mixed": 1e-5}
    return out


def numbering_extra(torch, L, m, q, args, stream, ms_rcm, device):
    """The same FP64 stage (and FP32-mixed stage) under a random node
    numbering and under the partition order of recursive coordinate
    bisection, against RCM."""
    from paper_1403_7209_gb300.solver import EdgeSolver
    out = {"rcm_ms": ms_rcm}
    for name in ("random", "rcb"):
        r = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, device=device, renumber=name,
                       seed=1, stream=stream, coords=m.coords, mixed=True)
        for loop in range(L.NUM_LOOPS):
            for prec in (0, 1):
                r.set_strategy(loop, prec, L.STRAT_AUTO)
        r.time_step(0.5)
        L.op2b_dat_copy(r.ctx, r.d["q0"], r.d["q"])
        for _ in range(args.warmup):
            r.stage(0.25)
        ms = timed(torch, lambda: r.stage(0.25), args.steps, stream)
        r.sync_shadow()
        for _ in range(args.warmup):
            r.stage(0.25, 2, mixed=True)
        mms = timed(torch, lambda: r.stage(0.25, 2, mixed=True), args.steps, stream)
        out[name] = {"ms": ms, "edges_per_s": m.num_edges / (ms * 1e-3),
                     "rcm_speedup": ms / ms_rcm, "mixed_ms": mms,
                     "strategies": {nm: L.STRATEGY_NAMES[r.plan_stats(lp, pr)["strategy"]]
                                    for nm, lp, pr in (("gg", L.LOOP_GREEN_GAUSS, 0),
                                                       ("flux2", L.LOOP_FLUX2, 0),
                                                       ("gg32", L.LOOP_GREEN_GAUSS, 1),
                                                       ("flux2_32", L.LOOP_FLUX2, 1))}}
        r.close()
    return out


def partition_extra(torch, L, m, q, args, stream, ms_whole, device, strat):
    """Owner-compute execution on one GPU: the FP64 stage over P parts (RCB,
    each part RCM-numbered, halo of q and G refreshed by the exchange
    kernel; the parts one after another, or on concurrent streams) against
    the whole mesh, with the halo statistics of the paper's table of halo
    sizes for the same partitions."""
    from paper_1403_7209_gb300.partition import PartitionedSolver, halo_stats
    out = {"whole_mesh_ms": ms_whole}
    for P, conc in ((8, False), (64, False), (64, True)):
        ps = PartitionedSolver(m.edge, m.normal, m.dx, m.volume, q, coords=m.coords, nparts=P,
                               device=device, renumber="rcm", stream=stream, concurrent=conc)
        for loop, nm in ((L.LOOP_GREEN_GAUSS, "gg"), (L.LOOP_FLUX2, "flux2")):
            z = strat[nm]
            ps.set_strategy(loop, 0, z["strategy"], z["block"], z["part"], z["staged"])
        ps.set_strategy(L.LOOP_SPECTRAL, 0, L.STRAT_ATOMIC, 256)
        ps.time_step(0.5)
        ps._each(lambda sv: L.op2b_dat_copy(sv.ctx, sv.d["q0"], sv.d["q"]))
        for _ in range(args.warmup):
            ps.stage(0.25)
        ms = timed(torch, lambda: ps.stage(0.25), args.steps, stream)
        ex = timed(torch, lambda: (ps.exchange("q"), ps.exchange("G")), args.steps, stream)
        st = halo_stats(ps.parts)
        executed = sum(P_["sizes"]["edges"] for P_ in ps.parts)
        out["parts_%d%s" % (P, "_concurrent" if conc else "")] = {
                               "ms": ms, "edges_per_s": m.num_edges / (ms * 1e-3),
                               "vs_whole_mesh": ms / ms_whole,
                               "exchange_q_and_G_ms": ex,
                               "executed_edges_over_mesh_edges": executed / m.num_edges,
                               "halo": st}
        ps.close()
    return out


def stage_fn(L, s, stream, mixed=False):
    """One second-order RK stage through the C ABI (per-loop events
    optional): Green-Gauss with the scaling, flux, update."""
    a_gg, a_f2 = (s.a_gg32, s.a_f2_32) if mixed else (s.a_gg, s.a_f2)

    def stage(ev=None):
        if ev: ev[0].record(stream)
        L.op2b_green_gauss_scaled(s.ctx, a_gg, s.d["V"], L.ZERO_INC)
        if ev: ev[1].record(stream)
        L.op2b_edge_flux(s.ctx, a_f2, 2, s.gamma, s.eps_lim, L.ZERO_INC)
        if ev: ev[2].record(stream)
        L.op2b_node_update(s.ctx, s.d["q0"], s.d["q"], s.d["R"], s.d["V"], s.d["dt"], 0.25,
                           s.d["q32"] if mixed else -1)
        if ev: ev[3].record(stream)
    return stage


def tuned_solver(L, m, q, args, stream, device, **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, device=device, renumber=args.numbering,
                   stream=stream, **kw)
    if args.tune_cache and os.path.exists(args.tune_cache):
        L.op2b_load_tuning(s.ctx, args.tune_cache)
    for loop in range(L.NUM_LOOPS):
        for prec in range(L.NUM_PREC):
            s.set_strategy(loop, prec, L.STRAT_AUTO)
    s.time_step(0.5)
    L.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    return s


def lattice100_extra(torch, L, args, stream, device):
    """The 100^3 lattice (1M nodes, 9M edges): the FP64 stage with per-loop
    times, the FP32-mixed stage, the adjoint at 1M nodes, and the library's
    other loops (tangent, viscous, march adjoint, node limiters,
    block-Jacobi, numberings, partitions) on this mesh."""
    m, q = build_mesh(args.extras_n)
    E, N = m.num_edges, m.num_nodes
    s = tuned_solver(L, m, q, args, stream, device, mixed=True, adjoint=True, ff=True)
    stage = stage_fn(L, s, stream)
    for _ in range(args.warmup):
        stage()
    names = ["gg", "flux2", "update"]
    evs = [loop_events(torch, 4) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0, t1 = loop_events(torch, 2)
    t0.record(stream)
    for k in range(args.steps):
        stage(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    loops = {nm: statistics.mean(evs[k][j].elapsed_time(evs[k][j + 1]) for k in range(args.steps))
             for j, nm in enumerate(names)}
    strat = {nm: L.STRATEGY_NAMES[s.plan_stats(lp)["strategy"]] for nm, lp in
             (("gg", L.LOOP_GREEN_GAUSS), ("flux2", L.LOOP_FLUX2))}
    out = {"mesh": "%d^3 lattice, %d nodes, %d edges, RCM" % (args.extras_n, N, E),
           "ms_per_stage": ms, "edges_per_s": E / (ms * 1e-3),
           "loops": {nm: {"ms": loops[nm], "edges_per_s": E / (loops[nm] * 1e-3),
                          "gbs": BYTES_PER_EDGE[nm] * E / (loops[nm] * 1e-3) / 1e9,
                          "strategy": strat.get(nm, "direct")} for nm in names}}
    out["mixed"] = mixed_extra(torch, L, s, args, stream, ms, E, N)
    out["float_float"] = ff_extra(torch, L, s, args, stream, ms, E, N)
    out["adjoint"] = adjoint_extra(torch, L, s, args, stream, E)
    out["tangent"] = tangent_extra(torch, L, s, args, stream, E)
    out["viscous"] = viscous_extra(torch, L, m, q, args, stream, device, E)
    out["viscous"]["fp64_ns_stage_vs_euler_stage"] = out["viscous"]["fp64"]["ns_stage_ms"] / ms
    out["march_adjoint"] = march_adjoint_extra(torch, L, s, q, args, stream, E)
    out["limiters"] = limiter_extra(torch, L, m, q, args, stream, device, E, ms)
    out["block_jacobi"] = block_jacobi_extra(torch, L, m, q, args, stream, device, E)
    if args.numbering == "rcm":
        out["numbering"] = numbering_extra(torch, L, m, q, args, stream, ms, device)
    out["partitions"] = partition_extra(
        torch, L, m, q, args, stream, ms, device,
        {"gg": s.plan_stats(L.LOOP_GREEN_GAUSS), "flux2": s.plan_stats(L.LOOP_FLUX2)})
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="op2b", choices=["op2b", "reference"])
    ap.add_argument("--n", type=int, default=200, help="lattice size per side")
    ap.add_argument("--extras-n", type=int, default=100,
                    help="lattice size of the second mesh (the other loops, numberings)")
    ap.add_argument("--oracle-march-n", type=int, default=40,
                    help="lattice of the 50-step marches checked against the oracle's")
    ap.add_argument("--numbering", default="rcm", choices=["rcm", "random", "none"])
    ap.add_argument("--cpu-stages", type=int, default=5, help="oracle sample size (stages, about 2.5 s each on one host core)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--tune-cache", default="",
                    help="JSON strategy table: loaded if present, written after tuning")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    ws, rank, local = dist_setup()
    child = None
    if rank == 0 and not args.no_extras:
        # the CPU-baseline leg's oracle march runs in a spawned process
        # (started before the first GPU call) while the GPU works
        import multiprocessing as mp
        child = mp.get_context("spawn").Process(
            target=cpu_baseline_march_child, args=(args.oracle_march_n, 50), daemon=True)
        child.start()

    import torch
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1403_7209_gb300 import op2b as L
    L.load(build_if_missing=False)

    m, q = build_mesh(args.n)
    stream = torch.cuda.current_stream()
    s = tuned_solver(L, m, q, args, stream, local, mixed=not args.no_extras,
                     adjoint=not args.no_extras, ff=not args.no_extras)

    # per-loop events inside each timed step
    names = ["gg", "flux2", "update"]
    stage = stage_fn(L, s, stream)

    clk = Clocks(local).start()
    for _ in range(args.warmup):
        stage()
    torch.cuda.synchronize()
    if args.tune_cache and rank == 0:
        L.op2b_save_tuning(s.ctx, args.tune_cache)
    def timed_region():
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        n_launch0 = s.launch_count()
        clk.mark_begin()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(args.steps):
            stage(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
        return evs, s.launch_count() - n_launch0, t0.elapsed_time(t1) / args.steps, clk.summary()

    evs, launches, ms, clocks = timed_region()
    if set(clocks["reasons"]) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}:
        # a throttled measurement is not kept: take it once more
        first = clocks
        evs, launches, ms, clocks = timed_region()
        clocks["remeasured_after"] = first["reasons"]
    clk.stop()
    if dist is not None:
        ms = reduce_max_ms(ms, dist, device="cuda")
        dist.barrier()
    loop_ms = {nm: statistics.mean(evs[k][j].elapsed_time(evs[k][j + 1]) for k in range(args.steps))
               for j, nm in enumerate(names)}
    E, N = m.num_edges, m.num_nodes
    value = job_value(E, ws, ms)
    hbm, hbm_src = read_peaks()
    fl_ms = loop_ms["flux2"]
    achieved = FLOPS_PER_EDGE_FLUX2 * E / (fl_ms * 1e-3) / 1e12
    strat = {nm: L.STRATEGY_NAMES[s.plan_stats(lp)["strategy"]] for nm, lp in
             (("gg", L.LOOP_GREEN_GAUSS), ("flux2", L.LOOP_FLUX2))}
    line = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, m),
        "roofline": {"kernel": "flux2 edge loop (FP64, %s)" % strat["flux2"], "bound": "alu",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": (DRAM_BYTES_PER_EDGE_FLUX2_ATOMIC * E
                                 if strat["flux2"] == "atomic" else None),
                     "traffic_note": "bytes per launch, scaled by edge count from the "
                                     "60^3 ncu capture of the same kernel",
                     "peak_source": "FP64 FMA units x clock (152 SMs x 2/clk x 2 flop x 2.07 GHz)",
                     "hbm_frac": BYTES_PER_EDGE["flux2"] * E / (fl_ms * 1e-3) / 1e9 / hbm,
                     "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src,
                     "fp64_pipe": {
                         "instr_per_edge": FP64_INSTR_PER_EDGE_FLUX2,
                         "achieved_ginstr_s": FP64_INSTR_PER_EDGE_FLUX2 * E / (fl_ms * 1e-3) / 1e9,
                         "peak_ginstr_s": FP64_PEAK_GINSTR,
                         "frac": FP64_INSTR_PER_EDGE_FLUX2 * E / (fl_ms * 1e-3) / 1e9
                                 / FP64_PEAK_GINSTR,
                         "note": "FP64 instructions per edge from the ncu capture of this kernel; "
                                 "frac above is algorithmic flops (FMA = 2) over the FP64 flop "
                                 "peak, lower because 52% of the instructions are not FMAs"}},
        "gpu_launches": launches,
        "clocks": clocks,
        "loops": {nm: {"ms": loop_ms[nm], "edges_per_s": E / (loop_ms[nm] * 1e-3),
                       "gbs": BYTES_PER_EDGE[nm] * E / (loop_ms[nm] * 1e-3) / 1e9,
                       "strategy": strat.get(nm, "direct")} for nm in names},
    }

    # End to end through host memory, right after the device-only timing (the
    # same GPU state).  Every step copies its input state from pinned host
    # memory and reads back its result, the residual's L2 norm per component
    # (the convergence monitor of an explicit solver).  The input is
    # double-buffered: the next step's host-to-device copy runs on a copy
    # stream while the current step computes.
    q_host = torch.empty((6, N), dtype=torch.float64).pin_memory()
    q_host.copy_(s.t["q"][:, :N].cpu())
    norm_dev = torch.empty(6, dtype=torch.float64, device=s.device)
    norm_host = torch.empty(6, dtype=torch.float64).pin_memory()
    q_orig = s.t["q"]
    bufs = [q_orig.clone(), q_orig.clone()]
    copy_stream = torch.cuda.Stream(device=s.device)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]

    def issue_copy(k, after=None):
        b = k % 2
        with torch.cuda.stream(copy_stream):
            if after is not None:
                copy_stream.wait_event(after)
            copy_stream.wait_event(consumed[b])  # the buffer's previous step is done
            bufs[b][:, :N].copy_(q_host, non_blocking=True)
            copied[b].record(copy_stream)

    def e2e_step(k):
        b = k % 2
        stream.wait_event(copied[b])
        s.rebind("q", bufs[b])
        stage()
        L.op2b_dat_reduce(s.ctx, s.d["R"], L.RED_L2, norm_dev.data_ptr())
        norm_host.copy_(norm_dev, non_blocking=True)
        consumed[b].record(stream)

    def e2e_run(steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        issue_copy(0, after=ev[0])
        for k in range(steps):
            if k + 1 < steps:
                issue_copy(k + 1)
            e2e_step(k)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / steps
    e2e_run(3)
    ems = e2e_run(args.steps)
    s.rebind("q", q_orig)
    line["e2e"] = {"value": ws * E / (ems * 1e-3), "unit": "edges/s",
                   "h2d_bytes_per_step": int(q_host.numel() * 8),
                   "d2h_bytes_per_step": int(norm_host.numel() * 8),
                   "result": "residual L2 norm per component",
                   "ms_per_step": ems}

    # the same, reading back the whole new state and without the overlap
    out_host = torch.empty((6, N), dtype=torch.float64).pin_memory()

    def roundtrip_step():
        s.t["q"][:, :N].copy_(q_host, non_blocking=True)
        stage()
        out_host.copy_(s.t["q"][:, :N], non_blocking=True)
    for _ in range(3):
        roundtrip_step()
    rms = timed(torch, roundtrip_step, args.steps, stream)
    line["e2e_state_roundtrip"] = {"value": ws * E / (rms * 1e-3), "unit": "edges/s",
                                   "h2d_bytes_per_step": int(q_host.numel() * 8),
                                   "d2h_bytes_per_step": int(out_host.numel() * 8),
                                   "ms_per_step": rms}
    del bufs, out_host, q_host

    if not args.no_extras:
        # the same mesh: the FP32-mixed stage, the adjoint at 8M nodes, the
        # 50-step marches
        line["mixed"] = mixed_extra(torch, L, s, args, stream, ms, E, N)
        line["float_float"] = ff_extra(torch, L, s, args, stream, ms, E, N)
        line["adjoint"] = adjoint_extra(torch, L, s, args, stream, E)
        line["march"] = march_extra(torch, L, s, q, args, stream)
        L.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
        line["lattice_100"] = lattice100_extra(torch, L, args, stream, local)
        line["lattice_16"] = lattice16_extra(torch, L, args)
        if child is not None:
            child.join()
            q_ora, st = cpu_baseline_march_result(args.oracle_march_n, 50)
            line["march_vs_oracle"] = march_oracle_extra(torch, L, args, stream, local, q_ora,
                                                         args.oracle_march_n, 50)
            line["march_vs_oracle"]["oracle_status"] = st

    if rank == 0:
        rate, t, sample = cpu_baseline_run(m, q, args.cpu_stages, n=args.n)
        line["cpu_baseline"] = {"value": rate, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                "sample": "%d %s (%.1f s)" % (args.cpu_stages, sample, t)}
        if "march_vs_oracle" in line:
            line["cpu_baseline"]["march"] = {
                "mesh": line["march_vs_oracle"]["mesh"], "steps": 50,
                "note": "the oracle's 50-step march, run in a spawned process during the GPU "
                        "work; its final state is the reference of march_vs_oracle"}
        print(json.dumps(line))
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
