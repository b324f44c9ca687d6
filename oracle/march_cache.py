"""The oracle's explicit march on a seeded lattice, cached on disk.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests and the
benchmark's CPU-baseline leg use it as the reference for marches on the GPU.
It calls nothing but the oracle (``oracle.march``, Sec. 2's multi-stage
Runge-Kutta march with local time stepping) on inputs drawn by the shared
input generator, and stores the final state, FP64, node-major (N, 6), in
the mesh's own node numbering.

The cache key hashes the lattice size, the input seed, the march settings
and the oracle's C source, so a change to the oracle's arithmetic never
reuses an old result.  Cache directory: ``$OP2B_ORACLE_CACHE``, else
``.oracle_cache/`` at the repository root (untracked).

    python -m oracle.march_cache --n 40 --steps 50
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)


def cache_dir() -> str:
    return os.environ.get("OP2B_ORACLE_CACHE") or os.path.join(_ROOT, ".oracle_cache")


def key(n: int, steps: int, order: int = 2, seed: int = 0, stages: int = 5,
        cfl: float = 0.5) -> str:
    with open(os.path.join(_HERE, "oracle.c"), "rb") as fh:
        src = hashlib.sha256(fh.read()).hexdigest()[:16]
    desc = json.dumps({"n": n, "seed": seed, "steps": steps, "order": order, "stages": stages,
                       "cfl": cfl, "oracle_c": src}, sort_keys=True)
    return "march_n%d_s%d_o%d_%s" % (n, steps, order, hashlib.sha256(desc.encode()).hexdigest()[:16])


def oracle_march(n: int, steps: int, order: int = 2, seed: int = 0, stages: int = 5,
                 cfl: float = 0.5, use_cache: bool = True):
    """Final state (N, 6) of the oracle's march on the n^3 lattice (mesh and
    state of seed `seed`), its status (0, or -(1 + stage) at the first
    non-physical state) and the seconds the march took (0.0 from cache)."""
    import oracle
    from paper_1403_7209_gb300 import meshgen  # inputs only
    path = os.path.join(cache_dir(), key(n, steps, order, seed, stages, cfl) + ".npz")
    if use_cache and os.path.exists(path):
        d = np.load(path)
        return d["q"], int(d["status"]), 0.0
    m = meshgen.lattice(n, seed=seed)
    q = meshgen.flow_state(m, seed=seed)
    t = time.perf_counter()
    qf, st = oracle.march(order, steps, m.edge, q, m.normal, m.dx, m.volume, stages=stages,
                          cfl=cfl)
    t = time.perf_counter() - t
    if use_cache:
        os.makedirs(cache_dir(), exist_ok=True)
        tmp = path + ".tmp.%d.npz" % os.getpid()
        np.savez(tmp, q=qf, status=st)
        os.replace(tmp, path)
    return qf, st, t


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=40)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    q, st, t = oracle_march(a.n, a.steps, a.order, a.seed)
    print("n=%d steps=%d status=%d  %.1f s  -> %s" % (a.n, a.steps, st, t, cache_dir()))
    return 0 if st == 0 else 1


if __name__ == "__main__":
    if _ROOT not in sys.path:
        sys.path.insert(0, _ROOT)
    sys.exit(main())
