"""Write oracle_counts.json: iteration counts and solution samples of full oracle solves.

Runs only the CPU oracle (oracle.cg) on the synthetic workloads.  For each
workload it records the outer/inner iteration counts, the status and true
relative residual, ||x_oracle|| and ``x_sample``: the oracle's x at
``x_sample_idx`` (4096 row indices drawn without replacement, sorted, by
numpy's PCG64 with ``x_sample_seed``), so that the full-size GPU tests can
check ||x_gpu - x_oracle|| / ||x_oracle|| on a seeded sample of rows.
bench.py's CPU-baseline legs divide their timed samples by these counts.
Usage:
    python tests/golden/make_oracle_counts.py [--no-hscg] [workload ...]
(--no-hscg keeps the HSCG fields already stored for a workload.)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cg  # noqa: E402
from oracle.operators import as_matrix  # noqa: E402
from sscg_inputs import generators as gen  # noqa: E402

WORKLOADS = {
    "varcoef3d_160": dict(smax=16, basis="newton", tol=1e-10),
    "poisson2d_64": dict(smax=8, basis="chebyshev", tol=1e-10),
    "rgg_2m": dict(smax=16, basis="newton", tol=1e-10),
    "rgg_2m_fp32": dict(smax=16, basis="newton", tol=1e-10, y_fp32=True, base="rgg_2m", hscg=False),
}

X_SAMPLES = 4096
X_SAMPLE_SEED = 20240


def x_sample_indices(n: int, seed: int = X_SAMPLE_SEED, count: int = X_SAMPLES) -> np.ndarray:
    """The sampled rows: `count` distinct indices below n, sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


def main(argv):
    no_hscg = "--no-hscg" in argv
    names = [a for a in argv if not a.startswith("--")] or list(WORKLOADS)
    path = os.path.join(HERE, "oracle_counts.json")
    for name in names:
        cfg = WORKLOADS[name]
        op, b, x0, _ = gen.config_problem(cfg.get("base", name))
        A = as_matrix(op)
        t = time.time()
        x, info = cg.sstep_cg(A, b, x0, cfg["tol"], cg.Options(smax=cfg["smax"], basis=cfg["basis"],
                                                              y_fp32=cfg.get("y_fp32", False)))
        ts = time.time() - t
        idx = x_sample_indices(len(x))
        rec = dict(sstep_outer=info["outer"], sstep_inner=info["inner"], sstep_status=info["status"],
                   sstep_relres=info["relres_true"], sstep_seconds=ts, cpu_count=os.cpu_count(),
                   x_norm=float(np.sqrt(x @ x)), x_sample_seed=X_SAMPLE_SEED,
                   x_sample_idx=[int(i) for i in idx], x_sample=[float(v) for v in x[idx]], **cfg)
        if "fp32_replacements" in info:
            rec["fp32_replacements"] = info["fp32_replacements"]
        out = json.load(open(path)) if os.path.exists(path) else {}
        old = out.get(name, {})
        if cfg.get("hscg", True):
            if no_hscg and "hscg_iters" in old:
                rec.update(hscg_iters=old["hscg_iters"], hscg_seconds=old["hscg_seconds"])
            else:
                t = time.time()
                _, h = cg.hscg(A, b, x0, cfg["tol"])
                rec.update(hscg_iters=h["iters"], hscg_seconds=time.time() - t)
        out = json.load(open(path)) if os.path.exists(path) else {}   # merge with concurrent writers
        out[name] = rec
        json.dump(out, open(path, "w"), indent=1, sort_keys=True)
        print(name, {k: v for k, v in rec.items() if not k.startswith("x_sample")}, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
