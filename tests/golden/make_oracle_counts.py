"""Write oracle_counts.json: outer/inner iteration counts of full oracle solves.

Runs only the CPU oracle (oracle.cg) on the synthetic workloads; bench.py's
CPU-baseline legs time a bounded sample of outer loops and divide by these
counts to express the oracle's speed in solves/s.  Usage:
    python tests/golden/make_oracle_counts.py [workload ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

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


def main(names):
    path = os.path.join(HERE, "oracle_counts.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        cfg = WORKLOADS[name]
        op, b, x0, _ = gen.config_problem(cfg.get("base", name))
        A = as_matrix(op)
        t = time.time()
        x, info = cg.sstep_cg(A, b, x0, cfg["tol"], cg.Options(smax=cfg["smax"], basis=cfg["basis"],
                                                              y_fp32=cfg.get("y_fp32", False)))
        ts = time.time() - t
        rec = dict(sstep_outer=info["outer"], sstep_inner=info["inner"], sstep_status=info["status"],
                   sstep_relres=info["relres_true"], sstep_seconds=ts, cpu_count=os.cpu_count(), **cfg)
        if "fp32_replacements" in info:
            rec["fp32_replacements"] = info["fp32_replacements"]
        if cfg.get("hscg", True):
            t = time.time()
            _, h = cg.hscg(A, b, x0, cfg["tol"])
            rec.update(hscg_iters=h["iters"], hscg_seconds=time.time() - t)
        out[name] = rec
        json.dump(out, open(path, "w"), indent=1, sort_keys=True)
        print(name, out[name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
