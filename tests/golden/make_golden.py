"""Write oracle reference data for full-size parity checks.

Runs only the FP64 CPU oracle (``oracle/``) on a seeded workload and stores a
compact sample of its output under tests/golden/:

  <name>.npz   idx (sampled node indices), u (oracle values there), labels
               (full label map, int8), gap (a* best-vs-second gap at the
               sampled nodes), phimax (max_j phi^j at the sampled nodes),
               tie (bit-packed mask over every node: the tie nodes of the
               label comparison, see tests/_labels.py), astar_full (the
               coarse feedback index at every node, 255 where undefined),
               meta (JSON: sizes, sweeps,
               per-patch node counts, reachable count, max u, E1/E_inf of the
               patchy solution against the global one when computed).

Usage:  python tests/golden/make_golden.py sincos2d 0 [--global]
        python tests/golden/make_golden.py sin3d 0 --n=129 --nc=33
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from tests._labels import tie_mask  # noqa: E402  (the tie rule of the label comparison)

HERE = os.path.dirname(os.path.abspath(__file__))


def make(family: str, seed: int, with_global: bool, samples: int = 20000, **kw):
    p = getattr(W, family)(seed, **kw)
    t0 = time.time()
    r = oracle.patchy_solve(p, tol=1e-10, keep_phi=True)
    t1 = time.time()
    rng = np.random.default_rng(1234 + seed)
    fin = np.nonzero(np.isfinite(r.u))[0]
    idx = np.sort(rng.choice(fin, size=min(samples, fin.size), replace=False))
    meta = {
        "family": family, "seed": seed, "kw": kw, "n": list(p.n), "n_coarse": list(p.n_coarse),
        "tol_oracle": 1e-10, "seconds_patchy": t1 - t0, "stats": r.stats,
        "reachable": int(np.isfinite(r.u).sum()), "max_u": float(r.u[fin].max()),
        "label_counts": {int(k): int(v) for k, v in zip(*np.unique(r.labels, return_counts=True))},
    }
    tie = tie_mask(r, p)
    meta["tie_nodes"] = int(tie.sum())
    out = {"idx": idx, "u": r.u[idx], "labels": r.labels, "gap": r.gap[idx],
           "phimax": r.phi.max(axis=0)[idx], "astar": r.astar[idx], "tie": np.packbits(tie),
           "astar_full": np.where(r.astar >= 0, r.astar, 255).astype(np.uint8)}
    if with_global:
        t2 = time.time()
        g = oracle.global_solve(p.with_(n_coarse=None), tol=1e-10)
        meta["seconds_global"] = time.time() - t2
        meta["global_sweeps"] = g.sweeps
        e1, einf = oracle.patchy_error(r.u, g.u)
        meta["E1"], meta["Einf"] = e1, einf
        out["u_global"] = g.u[idx]
    name = f"{family}_n{p.n[0]}_s{seed}"
    np.savez_compressed(os.path.join(HERE, name + ".npz"), meta=json.dumps(meta, default=float), **out)
    print(name, json.dumps({k: meta[k] for k in meta if k != "stats"}, default=float))


if __name__ == "__main__":
    fam = sys.argv[1]
    seed = int(sys.argv[2])
    kw = {}
    for a in sys.argv[3:]:
        if a.startswith("--n="):
            kw["n"] = int(a[4:])
        if a.startswith("--nc="):
            kw["n_coarse"] = int(a[5:])
    make(fam, seed, "--global" in sys.argv, **kw)
