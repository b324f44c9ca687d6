"""Python binding of the op2b C ABI (include/op2b.h): argument marshalling only.

Every function here has the name of the C entry point it calls and raises
:class:`Op2bError` when that call returns an error code.  Device pointers are
plain integers (e.g. ``tensor.data_ptr()``), streams are ``cudaStream_t``
values (e.g. ``torch.cuda.current_stream().cuda_stream``).  The shared
library is loaded on first use and must exist: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libop2b.so")

OK, EINVAL, EDIM, ETYPE, EACCESS, ESET = 0, -1, -2, -3, -4, -5
ENOMEM, ECUDA, ETIMEOUT, EPLAN, ERANGE = -6, -7, -8, -9, -10
READ, WRITE, RW, INC = 1, 2, 3, 4
F64, F32, I32, FF = 0, 1, 2, 3
ID = -1
LOOP_GREEN_GAUSS, LOOP_FLUX1, LOOP_FLUX2, LOOP_SPECTRAL = 0, 1, 2, 3
LOOP_FLUX1_ADJ, LOOP_FLUX2_ADJ, LOOP_GG_ADJ = 4, 5, 6
LOOP_FLUX1_TAN, LOOP_FLUX2_TAN, LOOP_GG_TAN, LOOP_VISCOUS = 7, 8, 9, 10
LOOP_FLUX2_PHI, LOOP_JACOBI, LOOP_JACOBI_SUMS, NUM_LOOPS = 11, 12, 13, 14
LIM_BARTH_JESPERSEN, LIM_VENKATAKRISHNAN = 1, 2
PREC_F64, PREC_F32, PREC_FF, NUM_PREC = 0, 1, 2, 3
STAGE_SYNC, STAGE_STORE_Q0, STAGE_SYNC_MESH, STAGE_STAGED = 1, 2, 4, 8
STRAT_AUTO, STRAT_ATOMIC, STRAT_COLOUR, STRAT_SEGMENTED, STRAT_AUTO_DET = 0, 1, 2, 3, 4
STRAT_BLOCK_ATOMIC, STRAT_OWNER, STRAT_GATHER, STRAT_HYBRID = 5, 6, 7, 8
ZERO_INC = 1
RED_SUM, RED_L2, RED_MAXABS, RED_MIN = 0, 1, 2, 3
STRATEGY_NAMES = {STRAT_AUTO: "auto", STRAT_ATOMIC: "atomic",
                  STRAT_COLOUR: "colour", STRAT_SEGMENTED: "segmented",
                  STRAT_AUTO_DET: "auto-deterministic", STRAT_BLOCK_ATOMIC: "block-atomic",
                  STRAT_OWNER: "owner", STRAT_GATHER: "gather", STRAT_HYBRID: "hybrid"}
ERROR_NAMES = {EINVAL: "EINVAL", EDIM: "EDIM", ETYPE: "ETYPE",
               EACCESS: "EACCESS", ESET: "ESET", ENOMEM: "ENOMEM",
               ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT", EPLAN: "EPLAN",
               ERANGE: "ERANGE"}


class Op2bError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


class Arg(ctypes.Structure):
    _fields_ = [("dat", ctypes.c_int32), ("idx", ctypes.c_int32),
                ("map", ctypes.c_int32), ("acc", ctypes.c_int32)]


class FluxParams(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("eps_lim", ctypes.c_double)]


class ViscParams(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("gamma", ctypes.c_double), ("mu", ctypes.c_double),
                ("prandtl", ctypes.c_double), ("diff", ctypes.c_double)]


class PlanStats(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int32), ("block", ctypes.c_int32),
                ("part", ctypes.c_int32), ("staged", ctypes.c_int32),
                ("nblocks", ctypes.c_int64), ("ncolours", ctypes.c_int64),
                ("min_blocks_per_colour", ctypes.c_int64),
                ("max_blocks_per_colour", ctypes.c_int64),
                ("max_unique_nodes", ctypes.c_int64),
                ("avg_unique_nodes", ctypes.c_double),
                ("tuned_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_D = ctypes.c_double
_PI32 = ctypes.POINTER(ctypes.c_int32)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PARG = ctypes.POINTER(Arg)

_SIGS = {
    "op2b_init": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _P]),
    "op2b_finalize": (ctypes.c_int, [_P]),
    "op2b_set_stream": (ctypes.c_int, [_P, _P]),
    "op2b_last_error": (ctypes.c_char_p, [_P]),
    "op2b_version": (ctypes.c_char_p, []),
    "op2b_decl_set": (ctypes.c_int, [_P, _I64, ctypes.c_char_p, _PI32]),
    "op2b_decl_map": (ctypes.c_int, [_P, _I32, _I32, _I32, _PI32,
                                     ctypes.c_char_p, _PI32]),
    "op2b_decl_dat": (ctypes.c_int, [_P, _I32, _I32, _I32, _P, _I64,
                                     ctypes.c_char_p, _PI32]),
    "op2b_rebind_dat": (ctypes.c_int, [_P, _I32, _P]),
    "op2b_fetch_map": (ctypes.c_int, [_P, _I32, _PI32]),
    "op2b_renumber": (ctypes.c_int, [_P, _I32, _I32, _U64, _PI32, _PI64]),
    "op2b_renumber_rcb": (ctypes.c_int, [_P, _I32, _I32, _I32, _PI32, _PI64]),
    "op2b_green_gauss": (ctypes.c_int, [_P, _PARG, _I32, _I32]),
    "op2b_green_gauss_scaled": (ctypes.c_int, [_P, _PARG, _I32, _I32, _I32]),
    "op2b_edge_flux": (ctypes.c_int, [_P, _PARG, _I32,
                                      ctypes.POINTER(FluxParams)]),
    "op2b_spectral_radius": (ctypes.c_int, [_P, _PARG, _I32, _D, _I32]),
    "op2b_edge_flux_adjoint": (ctypes.c_int, [_P, _PARG, _I32,
                                              ctypes.POINTER(FluxParams)]),
    "op2b_green_gauss_adjoint": (ctypes.c_int, [_P, _PARG, _I32, _I32]),
    "op2b_green_gauss_tangent": (ctypes.c_int, [_P, _PARG, _I32, _I32]),
    "op2b_edge_flux_tangent": (ctypes.c_int, [_P, _PARG, _I32,
                                              ctypes.POINTER(FluxParams)]),
    "op2b_node_minmax": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32]),
    "op2b_node_limiter": (ctypes.c_int, [_P, _I32, _I32, _D, _I32, _I32, _I32, _I32, _I32,
                                         _I32]),
    "op2b_edge_flux_limited": (ctypes.c_int, [_P, _PARG, _I32, ctypes.POINTER(FluxParams)]),
    "op2b_viscous_prims": (ctypes.c_int, [_P, _I32, _I32, _I32, _D]),
    "op2b_viscous_flux": (ctypes.c_int, [_P, _PARG, _I32,
                                         ctypes.POINTER(ViscParams)]),
    "op2b_grad_scale": (ctypes.c_int, [_P, _I32, _I32]),
    "op2b_jacobi_blocks": (ctypes.c_int, [_P, _PARG, _I32, _D, _I32]),
    "op2b_block_invert": (ctypes.c_int, [_P, _I32, _I32]),
    "op2b_jacobi_sums": (ctypes.c_int, [_P, _PARG, _I32, _D, _I32]),
    "op2b_jacobi_from_sums": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _D]),
    "op2b_node_update_precond": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _D]),
    "op2b_grad_scale_adjoint": (ctypes.c_int, [_P, _I32, _I32]),
    "op2b_time_step": (ctypes.c_int, [_P, _I32, _I32, _D, _I32]),
    "op2b_node_update": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32,
                                        _D, _I32]),
    "op2b_stage_mixed": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _I32, _I32, _I32,
                                        _I32, _D, _D, _D, _I32]),
    "op2b_node_update_adjoint": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _D]),
    "op2b_dat_axpy": (ctypes.c_int, [_P, _I32, _D, _I32]),
    "op2b_dat_fill": (ctypes.c_int, [_P, _I32, _D]),
    "op2b_dat_copy": (ctypes.c_int, [_P, _I32, _I32]),
    "op2b_dat_reduce": (ctypes.c_int, [_P, _I32, _I32, _P]),
    "op2b_set_strategy": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _I32,
                                         _I32]),
    "op2b_set_tune_deadline": (ctypes.c_int, [_P, _D]),
    "op2b_save_tuning": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "op2b_load_tuning": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "op2b_plan_stats": (ctypes.c_int, [_P, _I32, _I32, _I32,
                                       ctypes.POINTER(PlanStats)]),
    "op2b_launch_count": (ctypes.c_int64, [_P]),
    "op2b_edge_flux1_noalloc": (ctypes.c_int, [_P, _I64, _P, _I64, _P, _P, _P, _P,
                                               _I64, _I64, _D, _P, _I64, _P]),
    "op2b_host_rcm": (ctypes.c_int, [_I64, _I64, _PI32, _PI32]),
    "op2b_host_renumber": (ctypes.c_int, [_I64, _I64, _PI32, _I32, _U64,
                                          _PI32, _PI64]),
    "op2b_host_colour_blocks": (ctypes.c_int, [_I64, _I64, _PI32, _I32,
                                               _PI32, _PI64]),
    "op2b_host_node_csr": (ctypes.c_int, [_I64, _I64, _PI32, _PI64, _PI64]),
    "op2b_host_rcb": (ctypes.c_int, [_I64, ctypes.POINTER(ctypes.c_double), _I32, _PI32]),
    "op2b_host_partition_rcb": (ctypes.c_int, [_I64, ctypes.POINTER(ctypes.c_double), _I32,
                                               _PI32]),
    "op2b_halo_create": (ctypes.c_int, [_I64, _I64, _PI32, _PI32, _I32, ctypes.POINTER(_P)]),
    "op2b_halo_sizes": (ctypes.c_int, [_P, _I32, _PI64]),
    "op2b_halo_part": (ctypes.c_int, [_P, _I32, _PI32, _PI32, _PI32, _PI32, _PI32, _PI32,
                                      _PI64, _PI32]),
    "op2b_halo_destroy": (ctypes.c_int, [_P]),
    "op2b_exchange_create": (ctypes.c_int, [_P, _I32, _I32, _I32, ctypes.POINTER(_P), _PI64,
                                            ctypes.POINTER(_P), _PI64, _PI64, _PI32, _PI32,
                                            ctypes.POINTER(_P)]),
    "op2b_exchange_run": (ctypes.c_int, [_P, _P]),
    "op2b_exchange_destroy": (ctypes.c_int, [_P, _P]),
}
EXPORTED = tuple(_SIGS)

_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load libop2b.so (building it with nvcc first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise OSError("op2b CUDA library missing: %s" % LIB_PATH)
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc, ctx=None):
    if rc != OK:
        msg = load().op2b_last_error(ctx)
        raise Op2bError(rc, msg.decode() if msg else "")
    return rc


def _i32p(a):
    return a.ctypes.data_as(_PI32)


def _i64p(a):
    return a.ctypes.data_as(_PI64)


def _args(arglist):
    arr = (Arg * len(arglist))()
    for k, a in enumerate(arglist):
        arr[k] = Arg(*a)
    return arr, len(arglist)


# ------------------------------------------------------------- lifecycle
def op2b_version() -> str:
    return load().op2b_version().decode()


def op2b_init(device: int = 0, stream: int = 0):
    ctx = _P()
    rc = load().op2b_init(ctypes.byref(ctx), device, stream)
    _check(rc, None)
    return ctx


def op2b_finalize(ctx):
    _check(load().op2b_finalize(ctx), None)


def op2b_set_stream(ctx, stream: int):
    _check(load().op2b_set_stream(ctx, stream), ctx)


def op2b_last_error(ctx) -> str:
    return load().op2b_last_error(ctx).decode()


def op2b_launch_count(ctx) -> int:
    return int(load().op2b_launch_count(ctx))


# ----------------------------------------------------------- declarations
def op2b_decl_set(ctx, size: int, name: str = "") -> int:
    out = ctypes.c_int32()
    _check(load().op2b_decl_set(ctx, size, name.encode(), ctypes.byref(out)), ctx)
    return out.value


def op2b_decl_map(ctx, frm: int, to: int, arity: int, data, name: str = "") -> int:
    data = np.ascontiguousarray(data, dtype=np.int32)
    out = ctypes.c_int32()
    _check(load().op2b_decl_map(ctx, frm, to, arity, _i32p(data), name.encode(),
                                ctypes.byref(out)), ctx)
    return out.value


def op2b_decl_dat(ctx, set_: int, dim: int, type_: int, device_ptr: int,
                  ld: int = 0, name: str = "") -> int:
    out = ctypes.c_int32()
    _check(load().op2b_decl_dat(ctx, set_, dim, type_, device_ptr, ld, name.encode(),
                                ctypes.byref(out)), ctx)
    return out.value


def op2b_rebind_dat(ctx, dat: int, device_ptr: int):
    _check(load().op2b_rebind_dat(ctx, dat, device_ptr), ctx)


def op2b_fetch_map(ctx, map_: int, size: int) -> np.ndarray:
    out = np.empty(size, dtype=np.int32)
    _check(load().op2b_fetch_map(ctx, map_, _i32p(out)), ctx)
    return out


def op2b_renumber(ctx, map_: int, method: int, seed: int, num_nodes: int,
                  num_edges: int):
    perm = np.empty(num_nodes, dtype=np.int32)
    order = np.empty(num_edges, dtype=np.int64)
    _check(load().op2b_renumber(ctx, map_, method, seed, _i32p(perm), _i64p(order)), ctx)
    return perm, order


def op2b_renumber_rcb(ctx, map_: int, coords_dat: int, leaf: int, num_nodes: int,
                      num_edges: int):
    perm = np.empty(num_nodes, dtype=np.int32)
    order = np.empty(num_edges, dtype=np.int64)
    _check(load().op2b_renumber_rcb(ctx, map_, coords_dat, leaf, _i32p(perm), _i64p(order)),
           ctx)
    return perm, order


# ------------------------------------------------------------------ loops
def op2b_green_gauss(ctx, args, flags: int = 0):
    a, n = _args(args)
    _check(load().op2b_green_gauss(ctx, a, n, flags), ctx)


def op2b_green_gauss_scaled(ctx, args, V: int, flags: int = 0):
    a, n = _args(args)
    _check(load().op2b_green_gauss_scaled(ctx, a, n, V, flags), ctx)


def op2b_edge_flux(ctx, args, order: int, gamma: float = 1.4,
                   eps_lim: float = 1e-12, flags: int = 0):
    a, n = _args(args)
    p = FluxParams(order, flags, gamma, eps_lim)
    _check(load().op2b_edge_flux(ctx, a, n, ctypes.byref(p)), ctx)


def op2b_spectral_radius(ctx, args, gamma: float = 1.4, flags: int = 0):
    a, n = _args(args)
    _check(load().op2b_spectral_radius(ctx, a, n, gamma, flags), ctx)


def op2b_edge_flux_adjoint(ctx, args, order: int, gamma: float = 1.4,
                           eps_lim: float = 1e-12, flags: int = 0):
    a, n = _args(args)
    p = FluxParams(order, flags, gamma, eps_lim)
    _check(load().op2b_edge_flux_adjoint(ctx, a, n, ctypes.byref(p)), ctx)


def op2b_green_gauss_adjoint(ctx, args, flags: int = 0):
    a, n = _args(args)
    _check(load().op2b_green_gauss_adjoint(ctx, a, n, flags), ctx)


def op2b_green_gauss_tangent(ctx, args, flags: int = 0):
    a, n = _args(args)
    _check(load().op2b_green_gauss_tangent(ctx, a, n, flags), ctx)


def op2b_edge_flux_tangent(ctx, args, order: int, gamma: float = 1.4,
                           eps_lim: float = 1e-12, flags: int = 0):
    a, n = _args(args)
    p = FluxParams(order, flags, gamma, eps_lim)
    _check(load().op2b_edge_flux_tangent(ctx, a, n, ctypes.byref(p)), ctx)


def op2b_node_minmax(ctx, map_: int, q: int, qmin: int, qmax: int):
    _check(load().op2b_node_minmax(ctx, map_, q, qmin, qmax), ctx)


def op2b_node_limiter(ctx, map_: int, kind: int, eps2: float, q: int, G: int, dx: int,
                      qmin: int, qmax: int, phi: int):
    _check(load().op2b_node_limiter(ctx, map_, kind, eps2, q, G, dx, qmin, qmax, phi), ctx)


def op2b_edge_flux_limited(ctx, args, gamma: float = 1.4, flags: int = 0):
    a, n = _args(args)
    p = FluxParams(2, flags, gamma, 1e-12)
    _check(load().op2b_edge_flux_limited(ctx, a, n, ctypes.byref(p)), ctx)


def op2b_viscous_prims(ctx, q: int, G: int, W: int, gamma: float = 1.4):
    _check(load().op2b_viscous_prims(ctx, q, G, W, gamma), ctx)


def op2b_viscous_flux(ctx, args, gamma: float = 1.4, mu: float = 1e-3,
                      prandtl: float = 0.72, diff: float = 1e-3, flags: int = 0):
    a, n = _args(args)
    p = ViscParams(flags, 0, gamma, mu, prandtl, diff)
    _check(load().op2b_viscous_flux(ctx, a, n, ctypes.byref(p)), ctx)


def op2b_grad_scale(ctx, G: int, V: int):
    _check(load().op2b_grad_scale(ctx, G, V), ctx)


def op2b_jacobi_blocks(ctx, args, gamma: float = 1.4, flags: int = 0):
    a, n = _args(args)
    _check(load().op2b_jacobi_blocks(ctx, a, n, gamma, flags), ctx)


def op2b_jacobi_sums(ctx, args, gamma: float = 1.4, flags: int = 0):
    a, n = _args(args)
    _check(load().op2b_jacobi_sums(ctx, a, n, gamma, flags), ctx)


def op2b_jacobi_from_sums(ctx, q: int, S: int, M: int, P: int, gamma: float = 1.4):
    _check(load().op2b_jacobi_from_sums(ctx, q, S, M, P, gamma), ctx)


def op2b_block_invert(ctx, M: int, P: int):
    _check(load().op2b_block_invert(ctx, M, P), ctx)


def op2b_node_update_precond(ctx, q0: int, q: int, R: int, P: int, alpha_sigma: float):
    _check(load().op2b_node_update_precond(ctx, q0, q, R, P, alpha_sigma), ctx)


def op2b_grad_scale_adjoint(ctx, Gb: int, V: int):
    _check(load().op2b_grad_scale_adjoint(ctx, Gb, V), ctx)


def op2b_time_step(ctx, V: int, lam: int, cfl: float, dt: int):
    _check(load().op2b_time_step(ctx, V, lam, cfl, dt), ctx)


def op2b_node_update(ctx, q0: int, q: int, R: int, V: int, dt: int,
                     alpha: float, q32: int = -1):
    _check(load().op2b_node_update(ctx, q0, q, R, V, dt, alpha, q32), ctx)


def op2b_stage_mixed(ctx, map_: int, q0: int, q: int, V: int, dt: int, n: int, dx: int,
                     R: int, G: int, alpha: float, gamma: float = 1.4, eps_lim: float = 1e-12,
                     flags: int = 0):
    """Fused FP32-mixed second-order RK stage (see op2b.h)."""
    _check(load().op2b_stage_mixed(ctx, map_, q0, q, V, dt, n, dx, R, G, alpha, gamma,
                                   eps_lim, flags), ctx)


def op2b_node_update_adjoint(ctx, sbar: int, qbar: int, lam: int, V: int, dt: int,
                             alpha: float):
    _check(load().op2b_node_update_adjoint(ctx, sbar, qbar, lam, V, dt, alpha), ctx)


def op2b_dat_axpy(ctx, y: int, a: float, x: int):
    _check(load().op2b_dat_axpy(ctx, y, a, x), ctx)


def op2b_dat_fill(ctx, dat: int, value: float):
    _check(load().op2b_dat_fill(ctx, dat, value), ctx)


def op2b_dat_reduce(ctx, dat: int, op: int, out_ptr: int):
    _check(load().op2b_dat_reduce(ctx, dat, op, out_ptr), ctx)


def op2b_dat_copy(ctx, dst: int, src: int):
    _check(load().op2b_dat_copy(ctx, dst, src), ctx)


# ------------------------------------------------------ planner / tuner
def op2b_set_strategy(ctx, loop: int, prec: int, strategy: int, block: int = 0,
                      part: int = 0, staged: int = 0):
    _check(load().op2b_set_strategy(ctx, loop, prec, strategy, block, part, staged), ctx)


def op2b_set_tune_deadline(ctx, ms: float):
    _check(load().op2b_set_tune_deadline(ctx, ms), ctx)


def op2b_save_tuning(ctx, path: str):
    _check(load().op2b_save_tuning(ctx, path.encode()), ctx)


def op2b_load_tuning(ctx, path: str):
    _check(load().op2b_load_tuning(ctx, path.encode()), ctx)


def op2b_plan_stats(ctx, loop: int, prec: int, map_: int) -> dict:
    st = PlanStats()
    _check(load().op2b_plan_stats(ctx, loop, prec, map_, ctypes.byref(st)), ctx)
    return st.as_dict()


# ------------------------------------------------- allocation-free entry
NOALLOC_MAX_EDGES = 262144


def op2b_edge_flux1_noalloc(q_ptr: int, ldq: int, n_ptr: int, ldn: int,
                            edge_first_ptr: int, edge_second_ptr: int,
                            rowptr_ptr: int, ends_ptr: int, N: int, E: int,
                            gamma: float, R_ptr: int, ldR: int, stream: int):
    """First-order residual without any device allocation (see op2b.h)."""
    rc = load().op2b_edge_flux1_noalloc(q_ptr, ldq, n_ptr, ldn, edge_first_ptr,
                                        edge_second_ptr, rowptr_ptr, ends_ptr, N, E,
                                        gamma, R_ptr, ldR, stream)
    _check(rc, None)


# ------------------------------------------------------ host-only planners
def op2b_host_rcm(num_nodes: int, edge) -> np.ndarray:
    edge = np.ascontiguousarray(edge, dtype=np.int32)
    out = np.empty(num_nodes, dtype=np.int32)
    _check(load().op2b_host_rcm(num_nodes, edge.shape[0], _i32p(edge), _i32p(out)))
    return out


def op2b_host_renumber(num_nodes: int, edge, method: int, seed: int = 0):
    edge = np.ascontiguousarray(edge, dtype=np.int32)
    perm = np.empty(num_nodes, dtype=np.int32)
    order = np.empty(edge.shape[0], dtype=np.int64)
    _check(load().op2b_host_renumber(num_nodes, edge.shape[0], _i32p(edge), method,
                                     seed, _i32p(perm), _i64p(order)))
    return perm, order


def op2b_host_colour_blocks(num_nodes: int, edge, part: int):
    edge = np.ascontiguousarray(edge, dtype=np.int32)
    nb = (edge.shape[0] + part - 1) // part if part > 0 else 0
    col = np.empty(max(nb, 1), dtype=np.int32)
    nc = ctypes.c_int64()
    _check(load().op2b_host_colour_blocks(num_nodes, edge.shape[0], _i32p(edge), part,
                                          _i32p(col), ctypes.byref(nc)))
    return col[:nb], nc.value


def op2b_host_rcb(xyz, leaf: int = 1) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    out = np.empty(xyz.shape[0], dtype=np.int32)
    _check(load().op2b_host_rcb(xyz.shape[0], xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                leaf, _i32p(out)))
    return out


def op2b_host_node_csr(num_nodes: int, edge):
    edge = np.ascontiguousarray(edge, dtype=np.int32)
    rowptr = np.empty(num_nodes + 1, dtype=np.int64)
    ends = np.empty(max(2 * edge.shape[0], 1), dtype=np.int64)
    _check(load().op2b_host_node_csr(num_nodes, edge.shape[0], _i32p(edge),
                                     _i64p(rowptr), _i64p(ends)))
    return rowptr, ends[:2 * edge.shape[0]]


def op2b_host_partition_rcb(xyz, nparts: int) -> np.ndarray:
    """Part of every node: recursive coordinate bisection into nparts."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    out = np.empty(xyz.shape[0], dtype=np.int32)
    _check(load().op2b_host_partition_rcb(
        xyz.shape[0], xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nparts, _i32p(out)))
    return out


# ------------------------------------------------ owner-compute partitions
HALO_FIELDS = ("owned", "halo", "edges", "importers", "exported", "halo_edges")


def op2b_halo_create(num_nodes: int, edge, part, nparts: int):
    edge = np.ascontiguousarray(edge, dtype=np.int32)
    part = np.ascontiguousarray(part, dtype=np.int32)
    h = _P()
    _check(load().op2b_halo_create(num_nodes, edge.shape[0], _i32p(edge), _i32p(part), nparts,
                                   ctypes.byref(h)))
    return h


def op2b_halo_sizes(h, p: int) -> dict:
    out = np.zeros(6, dtype=np.int64)
    _check(load().op2b_halo_sizes(h, p, _i64p(out)))
    return dict(zip(HALO_FIELDS, (int(v) for v in out)))


def op2b_halo_part(h, p: int) -> dict:
    """Local mesh and exchange lists of part p (numpy arrays)."""
    z = op2b_halo_sizes(h, p)
    nodes = np.empty(z["owned"] + z["halo"], dtype=np.int32)
    edges = np.empty(z["edges"], dtype=np.int32)
    lmap = np.empty(2 * z["edges"], dtype=np.int32)
    owner = np.empty(z["halo"], dtype=np.int32)
    src = np.empty(z["halo"], dtype=np.int32)
    nbr = np.empty(z["importers"], dtype=np.int32)
    off = np.empty(z["importers"] + 1, dtype=np.int64)
    exp = np.empty(z["exported"], dtype=np.int32)
    _check(load().op2b_halo_part(h, p, _i32p(nodes), _i32p(edges), _i32p(lmap), _i32p(owner),
                                 _i32p(src), _i32p(nbr), _i64p(off), _i32p(exp)))
    return {"sizes": z, "nodes": nodes, "edges": edges, "local_map": lmap.reshape(-1, 2),
            "halo_owner": owner, "halo_src": src, "nbr": nbr, "exp_off": off, "exp_idx": exp}


def op2b_halo_destroy(h):
    _check(load().op2b_halo_destroy(h))


def op2b_exchange_create(ctx, type_: int, dim: int, src_ptrs, src_ld, dst_ptrs, dst_ld,
                         counts, src_idx, dst_idx):
    nseg = len(counts)
    src_a = (_P * max(nseg, 1))(*src_ptrs)
    dst_a = (_P * max(nseg, 1))(*dst_ptrs)
    sld = np.ascontiguousarray(src_ld, dtype=np.int64)
    dld = np.ascontiguousarray(dst_ld, dtype=np.int64)
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    si = np.ascontiguousarray(src_idx, dtype=np.int32)
    di = np.ascontiguousarray(dst_idx, dtype=np.int32)
    x = _P()
    _check(load().op2b_exchange_create(ctx, type_, dim, nseg, src_a, _i64p(sld), dst_a,
                                       _i64p(dld), _i64p(cnt), _i32p(si), _i32p(di),
                                       ctypes.byref(x)), ctx)
    return x


def op2b_exchange_run(ctx, x):
    _check(load().op2b_exchange_run(ctx, x), ctx)


def op2b_exchange_destroy(ctx, x):
    _check(load().op2b_exchange_destroy(ctx, x), ctx)
