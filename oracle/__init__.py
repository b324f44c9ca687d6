"""CPU oracle of the edge loops (serial FP64).  TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import this package.  It shares no code with the CUDA library
and never imports it.  ``oracle.c`` holds the arithmetic; this wrapper
compiles it with gcc (plain ``-O2``, no FMA contraction, no fast-math) and
marshals numpy arrays in the oracle's node-major layout:
q (N, 6), G (N, 18) with column 3k+d = dq_k/dx_d, n and dx (E, 3),
edge (E, 2) int32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .renumber import rcm_order, rcb_order, bandwidth  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAMMA = 1.4
EPS_LIM = 1e-12
RK_ALPHA = (0.25, 1.0 / 6.0, 0.375, 0.5, 1.0)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            I = ctypes.c_int
            sig = {
                "ora_euler_flux": [P, P, D, P],
                "ora_wave_speed": [P, P, D],
                "ora_rusanov": [P, P, P, D, P],
                "ora_van_albada": [D, D, D],
                "ora_reconstruct": [P, P, P, P, P, D, P, P],
                "ora_flux1": [I64, I64, P, P, P, D, P, P],
                "ora_green_gauss": [I64, I64, P, P, P, P, P],
                "ora_grad_scale": [I64, P, P, P],
                "ora_flux2": [I64, I64, P, P, P, P, P, D, D, P, P],
                "ora_residual": [I, I64, I64, P, P, P, P, P, D, D, P, P, P],
                "ora_spectral_radius": [I64, I64, P, P, P, D, P],
                "ora_time_step": [I64, P, P, D, P],
                "ora_rk_update": [I64, P, P, P, P, D, P],
                "ora_flux_jacobian": [P, P, D, P],
                "ora_jacobi_blocks": [I64, I64, P, P, P, D, P],
                "ora_block_invert": [I64, P, P],
                "ora_precond_update": [I64, P, P, P, D, P],
                "ora_check_state": [I64, P, D],
                "ora_march": [I, I, I, I64, I64, P, P, P, P, P, D, D, D,
                              P, P, P, P, P],
                "ora_residual_tangent": [I, I64, I64, P, P, P, P, P, D, D,
                                         P, P, P, P, P],
                "ora_residual_reverse": [I, I64, I64, P, P, P, P, P, D, D,
                                         P, P, P, P, P],
                "ora_kink_margin": [I, I64, I64, P, P, P, P, P, D, D, P, P],
                "ora_reduce": [I64, I, P, I, P],
                "ora_viscous_flux": [P, P, P, P, P, P, D, D, D, D, P],
                "ora_march_dt": [I, I, I, I64, I64, P, P, P, P, P, D, D, P, P, P, P],
                "ora_march_tangent": [I, I, I, I64, I64, P, P, P, P, P, D, D, P, P, P,
                                      P, P, P, P, P, P],
                "ora_march_reverse": [I, I, I, I64, I64, P, P, P, P, P, D, D, P, P, P,
                                      P, P, P, P, P, P, P, P, P],
                "ora_viscous": [I64, I64, P, P, P, P, P, D, D, D, D, P, P],
                "ora_minmax": [I64, I64, P, P, P, P],
                "ora_limiter_edge": [I, D, D, D],
                "ora_limiter": [I, I64, I64, P, P, P, P, P, P, D, P],
                "ora_flux2_phi": [I64, I64, P, P, P, P, P, P, D, P, P],
                "ora_residual_limited": [I, I64, I64, P, P, P, P, P, D, D, P, P, P, P, P,
                                         P],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None
            lib.ora_wave_speed.restype = D
            lib.ora_van_albada.restype = D
            lib.ora_check_state.restype = I64
            lib.ora_march.restype = I64
            lib.ora_march_dt.restype = I64
            lib.ora_limiter_edge.restype = D
            lib.ora_block_invert.restype = I64
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


# ------------------------------------------------------------ per-state parts
def euler_flux(q, n, gamma=GAMMA):
    q, n = _f64(q, (6,)), _f64(n, (3,))
    f = np.empty(6)
    _load().ora_euler_flux(_p(q), _p(n), gamma, _p(f))
    return f


def wave_speed(q, n, gamma=GAMMA):
    q, n = _f64(q, (6,)), _f64(n, (3,))
    return _load().ora_wave_speed(_p(q), _p(n), gamma)


def rusanov(qL, qR, n, gamma=GAMMA):
    qL, qR, n = _f64(qL, (6,)), _f64(qR, (6,)), _f64(n, (3,))
    F = np.empty(6)
    _load().ora_rusanov(_p(qL), _p(qR), _p(n), gamma, _p(F))
    return F


def van_albada(a, b, eps=EPS_LIM):
    return _load().ora_van_albada(float(a), float(b), float(eps))


def reconstruct(qi, qj, Gi, Gj, dx, eps=EPS_LIM):
    qi, qj = _f64(qi, (6,)), _f64(qj, (6,))
    Gi, Gj, dx = _f64(Gi, (18,)), _f64(Gj, (18,)), _f64(dx, (3,))
    qL, qR = np.empty(6), np.empty(6)
    _load().ora_reconstruct(_p(qi), _p(qj), _p(Gi), _p(Gj), _p(dx), eps,
                            _p(qL), _p(qR))
    return qL, qR


# ------------------------------------------------------------------ loops
def flux1(edge, q, n, gamma=GAMMA, with_abs=False):
    edge, q, n = _i32(edge), _f64(q), _f64(n)
    N, E = q.shape[0], edge.shape[0]
    R = np.empty((N, 6))
    Ra = np.empty((N, 6)) if with_abs else None
    _load().ora_flux1(N, E, _p(edge), _p(q), _p(n), gamma, _p(R), _p(Ra))
    return (R, Ra) if with_abs else R


def green_gauss(edge, q, n, with_abs=False):
    """Unscaled Green-Gauss sums Graw (N, 18)."""
    edge, q, n = _i32(edge), _f64(q), _f64(n)
    N, E = q.shape[0], edge.shape[0]
    G = np.empty((N, 18))
    Ga = np.empty((N, 18)) if with_abs else None
    _load().ora_green_gauss(N, E, _p(edge), _p(q), _p(n), _p(G), _p(Ga))
    return (G, Ga) if with_abs else G


def grad_scale(Graw, V):
    Graw, V = _f64(Graw), _f64(V)
    G = np.empty_like(Graw)
    _load().ora_grad_scale(Graw.shape[0], _p(Graw), _p(V), _p(G))
    return G


def flux2(edge, q, G, n, dx, gamma=GAMMA, eps=EPS_LIM, with_abs=False):
    edge, q, G, n, dx = _i32(edge), _f64(q), _f64(G), _f64(n), _f64(dx)
    N, E = q.shape[0], edge.shape[0]
    R = np.empty((N, 6))
    Ra = np.empty((N, 6)) if with_abs else None
    _load().ora_flux2(N, E, _p(edge), _p(q), _p(G), _p(n), _p(dx), gamma,
                      eps, _p(R), _p(Ra))
    return (R, Ra) if with_abs else R


def residual(order, edge, q, n, dx, V, gamma=GAMMA, eps=EPS_LIM,
             with_abs=False):
    """R(q, n); for order 2 also returns the scaled gradient G."""
    edge, q, n, dx, V = _i32(edge), _f64(q), _f64(n), _f64(dx), _f64(V)
    N, E = q.shape[0], edge.shape[0]
    G = np.empty((N, 18))
    R = np.empty((N, 6))
    Ra = np.empty((N, 6)) if with_abs else None
    _load().ora_residual(order, N, E, _p(edge), _p(q), _p(n), _p(dx), _p(V),
                         gamma, eps, _p(G), _p(R), _p(Ra))
    out = (R, G) if order == 2 else (R, None)
    return out + (Ra,) if with_abs else out


def spectral_radius(edge, q, n, gamma=GAMMA):
    edge, q, n = _i32(edge), _f64(q), _f64(n)
    lam = np.empty(q.shape[0])
    _load().ora_spectral_radius(q.shape[0], edge.shape[0], _p(edge), _p(q),
                                _p(n), gamma, _p(lam))
    return lam


def time_step(V, lam, cfl=0.5):
    V, lam = _f64(V), _f64(lam)
    dt = np.empty_like(V)
    _load().ora_time_step(V.shape[0], _p(V), _p(lam), cfl, _p(dt))
    return dt


def rk_update(q0, R, V, dt, alpha):
    q0, R, V, dt = _f64(q0), _f64(R), _f64(V), _f64(dt)
    q = np.empty_like(q0)
    _load().ora_rk_update(q0.shape[0], _p(q0), _p(R), _p(V), _p(dt), alpha,
                          _p(q))
    return q


def flux_jacobian(q, n, gamma=GAMMA):
    """A = d(f(q).n)/dq, 6 x 6 (row = flux component)."""
    q, n = _f64(q), _f64(n)
    A = np.empty((6, 6))
    _load().ora_flux_jacobian(_p(q), _p(n), gamma, _p(A))
    return A


def jacobi_blocks(edge, q, n, gamma=GAMMA):
    """Block-Jacobi blocks M (N x 6 x 6): the diagonal blocks of the
    first-order Rusanov residual's Jacobian, wave speeds held fixed."""
    edge, q, n = _i32(edge), _f64(q), _f64(n)
    N = q.shape[0]
    M = np.empty((N, 6, 6))
    _load().ora_jacobi_blocks(N, edge.shape[0], _p(edge), _p(q), _p(n), gamma, _p(M))
    return M


def block_invert(M):
    """(P, number of singular blocks): P_i = M_i^{-1} by Gauss-Jordan with
    partial pivoting."""
    M = _f64(M)
    P = np.empty_like(M)
    bad = int(_load().ora_block_invert(M.shape[0], _p(M), _p(P)))
    return P, bad


def precond_update(q0, R, P, alpha_sigma):
    """q = q0 - alpha sigma P R per node."""
    q0, R, P = _f64(q0), _f64(R), _f64(P)
    q = np.empty_like(q0)
    _load().ora_precond_update(q0.shape[0], _p(q0), _p(R), _p(P), alpha_sigma, _p(q))
    return q


def check_state(q, gamma=GAMMA):
    q = _f64(q)
    return int(_load().ora_check_state(q.shape[0], _p(q), gamma))


def march(order, steps, edge, q, n, dx, V, stages=5, gamma=GAMMA,
          eps=EPS_LIM, cfl=0.5):
    """Explicit RK march; returns (q, status) with status 0 or -(1+stage)."""
    edge, n, dx, V = _i32(edge), _f64(n), _f64(dx), _f64(V)
    q = _f64(q).copy()
    N, E = q.shape[0], edge.shape[0]
    q0, R = np.empty((N, 6)), np.empty((N, 6))
    G, lam, dt = np.empty((N, 18)), np.empty(N), np.empty(N)
    st = _load().ora_march(order, steps, stages, N, E, _p(edge), _p(q), _p(n),
                           _p(dx), _p(V), gamma, eps, cfl, _p(q0), _p(R),
                           _p(G), _p(lam), _p(dt))
    return q, int(st)


def residual_tangent(order, edge, q, n, dx, V, qd, nd, gamma=GAMMA,
                     eps=EPS_LIM):
    edge, q, n, dx, V = _i32(edge), _f64(q), _f64(n), _f64(dx), _f64(V)
    qd, nd = _f64(qd), _f64(nd)
    N, E = q.shape[0], edge.shape[0]
    G, Gd, Rd = np.empty((N, 18)), np.empty((N, 18)), np.empty((N, 6))
    _load().ora_residual_tangent(order, N, E, _p(edge), _p(q), _p(n), _p(dx),
                                 _p(V), gamma, eps, _p(qd), _p(nd), _p(G),
                                 _p(Gd), _p(Rd))
    return Rd


def residual_reverse(order, edge, q, n, dx, V, lam, gamma=GAMMA,
                     eps=EPS_LIM):
    """Returns (qbar (N, 6), nbar (E, 3)) of J = lam . R(q, n)."""
    edge, q, n, dx, V = _i32(edge), _f64(q), _f64(n), _f64(dx), _f64(V)
    lam = _f64(lam)
    N, E = q.shape[0], edge.shape[0]
    G, Gb = np.empty((N, 18)), np.empty((N, 18))
    qb, nb = np.empty((N, 6)), np.empty((E, 3))
    _load().ora_residual_reverse(order, N, E, _p(edge), _p(q), _p(n), _p(dx),
                                 _p(V), gamma, eps, _p(lam), _p(G), _p(Gb),
                                 _p(qb), _p(nb))
    return qb, nb


def march_dt(order, steps, edge, q, n, dx, V, dt, stages=5, gamma=GAMMA, eps=EPS_LIM):
    """March with the given fixed local time step dt (N,); returns (q, status)."""
    edge, n, dx, V, dt = _i32(edge), _f64(n), _f64(dx), _f64(V), _f64(dt)
    q = _f64(q).copy()
    N, E = q.shape[0], edge.shape[0]
    q0, R, G = np.empty((N, 6)), np.empty((N, 6)), np.empty((N, 18))
    st = _load().ora_march_dt(order, steps, stages, N, E, _p(edge), _p(q), _p(n), _p(dx),
                              _p(V), gamma, eps, _p(dt), _p(q0), _p(R), _p(G))
    return q, int(st)


def march_tangent(order, steps, edge, q, n, dx, V, dt, qd, nd, stages=5, gamma=GAMMA,
                  eps=EPS_LIM):
    """Tangent of the fixed-dt march: returns (q_final, qd_final)."""
    edge, n, dx, V, dt = _i32(edge), _f64(n), _f64(dx), _f64(V), _f64(dt)
    q, qd, nd = _f64(q).copy(), _f64(qd).copy(), _f64(nd)
    N, E = q.shape[0], edge.shape[0]
    w6 = [np.empty((N, 6)) for _ in range(4)]
    w18 = [np.empty((N, 18)) for _ in range(2)]
    _load().ora_march_tangent(order, steps, stages, N, E, _p(edge), _p(q), _p(n), _p(dx),
                              _p(V), gamma, eps, _p(dt), _p(qd), _p(nd),
                              *[_p(w) for w in w6], *[_p(w) for w in w18])
    return q, qd


def march_reverse(order, steps, edge, q, n, dx, V, dt, g, stages=5, gamma=GAMMA,
                  eps=EPS_LIM, with_states=False):
    """Reverse of the fixed-dt march for J = g . q_final: returns (qbar0,
    nbar) and, with ``with_states``, the input state of every stage
    (steps * stages, N, 6)."""
    edge, n, dx, V, dt = _i32(edge), _f64(n), _f64(dx), _f64(V), _f64(dt)
    q, g = _f64(q), _f64(g).copy()
    N, E = q.shape[0], edge.shape[0]
    nbar = np.empty((E, 3))
    S = np.empty((max(steps * stages, 1), N, 6))
    w6 = [np.empty((N, 6)) for _ in range(5)]
    w18 = [np.empty((N, 18)) for _ in range(2)]
    nb = np.empty((E, 3))
    _load().ora_march_reverse(order, steps, stages, N, E, _p(edge), _p(q), _p(n), _p(dx),
                              _p(V), gamma, eps, _p(dt), _p(g), _p(nbar), _p(S),
                              *[_p(w) for w in w6], *[_p(w) for w in w18], _p(nb))
    return (g, nbar, S[:steps * stages]) if with_states else (g, nbar)


LIM_BJ, LIM_VENKAT = 1, 2


def minmax(edge, q):
    """(qmin, qmax): per node and variable, over the node and its neighbours."""
    edge, q = _i32(edge), _f64(q)
    N, E = q.shape[0], edge.shape[0]
    lo, hi = np.empty((N, 6)), np.empty((N, 6))
    _load().ora_minmax(N, E, _p(edge), _p(q), _p(lo), _p(hi))
    return lo, hi


def limiter_edge(kind, d1, d2, eps2=0.0):
    """phi of one edge end (Barth-Jespersen: kind 1, Venkatakrishnan: 2)."""
    return _load().ora_limiter_edge(kind, float(d1), float(d2), float(eps2))


def limiter(kind, edge, q, G, dx, qmin, qmax, eps2=0.0):
    """Node limiter phi (N, 6)."""
    edge, q, G, dx = _i32(edge), _f64(q), _f64(G), _f64(dx)
    qmin, qmax = _f64(qmin), _f64(qmax)
    N, E = q.shape[0], edge.shape[0]
    phi = np.empty((N, 6))
    _load().ora_limiter(kind, N, E, _p(edge), _p(q), _p(G), _p(dx), _p(qmin), _p(qmax),
                        eps2, _p(phi))
    return phi


def flux2_phi(edge, q, G, phi, n, dx, gamma=GAMMA, with_abs=False):
    edge, q, G, phi, n, dx = _i32(edge), _f64(q), _f64(G), _f64(phi), _f64(n), _f64(dx)
    N, E = q.shape[0], edge.shape[0]
    R = np.empty((N, 6))
    Ra = np.empty((N, 6)) if with_abs else None
    _load().ora_flux2_phi(N, E, _p(edge), _p(q), _p(G), _p(phi), _p(n), _p(dx), gamma,
                          _p(R), _p(Ra))
    return (R, Ra) if with_abs else R


def residual_limited(kind, edge, q, n, dx, V, eps2=0.0, gamma=GAMMA, with_abs=False):
    """Node-limited second-order residual; returns dict R, G, qmin, qmax,
    phi (and Rabs with ``with_abs``)."""
    edge, q, n, dx, V = _i32(edge), _f64(q), _f64(n), _f64(dx), _f64(V)
    N, E = q.shape[0], edge.shape[0]
    out = {k: np.empty((N, 6)) for k in ("R", "qmin", "qmax", "phi")}
    out["G"] = np.empty((N, 18))
    out["Rabs"] = np.empty((N, 6)) if with_abs else None
    _load().ora_residual_limited(kind, N, E, _p(edge), _p(q), _p(n), _p(dx), _p(V), gamma,
                                 eps2, _p(out["G"]), _p(out["qmin"]), _p(out["qmax"]),
                                 _p(out["phi"]), _p(out["R"]), _p(out["Rabs"]))
    return out


def viscous_flux(qi, qj, Gi, Gj, n, dx, gamma=GAMMA, mu=1e-3, prandtl=0.72,
                 diff=1e-3):
    """Viscous flux Fv of one edge (see oracle.c)."""
    qi, qj = _f64(qi, (6,)), _f64(qj, (6,))
    Gi, Gj = _f64(Gi, (18,)), _f64(Gj, (18,))
    n, dx = _f64(n, (3,)), _f64(dx, (3,))
    F = np.empty(6)
    _load().ora_viscous_flux(_p(qi), _p(qj), _p(Gi), _p(Gj), _p(n), _p(dx), gamma, mu,
                             prandtl, diff, _p(F))
    return F


def viscous(edge, q, G, n, dx, gamma=GAMMA, mu=1e-3, prandtl=0.72, diff=1e-3,
            with_abs=False):
    """Viscous residual: R_i -= Fv, R_j += Fv over the edges."""
    edge, q, G, n, dx = _i32(edge), _f64(q), _f64(G), _f64(n), _f64(dx)
    N, E = q.shape[0], edge.shape[0]
    R = np.empty((N, 6))
    Ra = np.empty((N, 6)) if with_abs else None
    _load().ora_viscous(N, E, _p(edge), _p(q), _p(G), _p(n), _p(dx), gamma, mu, prandtl,
                        diff, _p(R), _p(Ra))
    return (R, Ra) if with_abs else R


def reduce(x, op):
    """Per-component sum (op 0), L2 norm (1), max |x| (2) or min (3) of an
    (n, dim) array."""
    x = _f64(x)
    if x.ndim == 1:
        x = x.reshape(-1, 1)
    out = np.empty(x.shape[1])
    _load().ora_reduce(x.shape[0], x.shape[1], _p(x), op, _p(out))
    return out


def kink_margin(order, edge, q, n, dx, V, gamma=GAMMA, eps=EPS_LIM):
    edge, q, n, dx, V = _i32(edge), _f64(q), _f64(n), _f64(dx), _f64(V)
    N, E = q.shape[0], edge.shape[0]
    G, m = np.empty((N, 18)), np.empty(E)
    _load().ora_kink_margin(order, N, E, _p(edge), _p(q), _p(n), _p(dx),
                            _p(V), gamma, eps, _p(G), _p(m))
    return m
