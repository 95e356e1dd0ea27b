"""Benchmark: converged adaptive s-step CG solves/s on one GB300 (and HSCG beside it).

Workload (default): FP64 3D 7-point variable-coefficient diffusion on a 160^3
grid (N = 4,096,000), per-face conductivities exp(g) with g ~ N(0, 1) i.i.d.,
b ~ N(0, 1), x0 = 0, sigma = 16, Newton basis with Leja-ordered shifts from the
running Ritz estimates, tol = 1e-10 (relative true residual).  One step = one
complete solve through the C ABI (every kernel of the method), inputs resident
in HBM.  Plain Hestenes-Stiefel CG (Algorithm 1) on the same GPU is timed
beside it.  Synthetic, seeded data.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 (torchrun), every rank solves its own copy (replicas: the method has
no data-parallel exchange on one system), value = total solves / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s & HBM GB/s at rel. residual 1e-10: s-step CG vs plain HSCG, one GB300"
WORKLOADS = {
    "varcoef3d_160": dict(desc="FP64 3D 7-pt var-coef diffusion 160^3 (N=4,096,000), k=exp(N(0,1)) per face, "
                               "b~N(0,1), x0=0", smax=16, basis="newton", tol=1e-10),
    "poisson2d_64": dict(desc="FP64 2D 5-pt Poisson 64x64 CSR (N=4096), b=A x*, x*~U(-1,1), x0=0",
                         smax=8, basis="chebyshev", tol=1e-10, gram_mode=0),
    "rgg_2m": dict(desc="FP64 CSR: Laplacian of a 3D random geometric graph, N=2,000,000, ~27 nnz/row, RCM order, "
                        "+1e-4*mean-degree*I, diagonal scaling 10^U(0,3); FP64 basis vs FP32-stored basis",
                   smax=16, basis="newton", tol=1e-10),
    "batched_256": dict(desc="256 independent 2D/3D log-normal-coefficient Poisson systems, N log-uniform in "
                             "[1e3, 2.6e5], 1-8 right-hand sides each, one graph launch, sigma per system by the "
                             "autotuner", smax=16, basis="newton", tol=1e-10),
    "adjoint2d_512": dict(desc="differentiable solve: 2D 5-pt var-coef Poisson 512^2 (N=262,144), theta=exp(g) per "
                               "edge, loss ||x(theta)-x_t||^2; forward s-step solve + adjoint s-step solve + "
                               "face-gradient gather", smax=16, basis="newton", tol=1e-10),
    # a smaller graph of the same family, used for kernel profiles
    "rgg_400k": dict(desc="FP64 CSR: Laplacian of a 3D random geometric graph, N=400,000 (the 2M workload's "
                          "recipe at a smaller size), for kernel profiles", smax=16, basis="newton", tol=1e-10,
                     base="rgg_2m", scale=400_000),
    # the forward solve of the differentiable workload's operator, with and
    # without a stored basis (recompute_y, NEXT row f4)
    "varcoef2d_512": dict(desc="FP64 2D 5-pt var-coef Poisson 512^2 (N=262,144), theta=exp(g) per edge, b~N(0,1), "
                               "x0=0; stored basis against recompute-Y (no stored basis)", smax=16, basis="newton",
                          tol=1e-10, base="adjoint2d_512", gram_mode=0),
    # a smaller grid of the same stencil family, used for kernel profiles
    "varcoef3d_96": dict(desc="FP64 3D 7-pt var-coef diffusion 96^3 (N=884,736), k=exp(N(0,1)) per face, "
                              "b~N(0,1), x0=0", smax=16, basis="newton", tol=1e-10, base="varcoef3d_160",
                         scale=96),
}
def _hbm_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0   # fallback: one earlier GB300 copy measurement


HBM_PEAK_GBS = _hbm_peak_gbs()
L2_BYTES = 129 * 2 ** 20
L2_FLUSH_BYTES = 256 * 2 ** 20
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz
FP32_PEAK_TINST = 152 * 128 * 2.070e9 / 1e12  # 152 SMs x 128 binary32 lanes/clk x 2070 MHz


def _bf16_peak_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


BF16_PEAK_TFLOPS, BF16_PEAK_SRC = _bf16_peak_tflops()   # f16 has the same nominal dense rate


def dg_tiles(ncols):
    """m16n8 tiles the gram_mode 2 kernel runs for ncols columns (the
    diagonal-only last tile row of ncols = 16 m + 1 is summed in binary64)."""
    mt_n, nt_n = (ncols + 15) // 16, (ncols + 7) // 8
    rows = mt_n - 1 if ncols % 16 == 1 else mt_n
    return sum(nt_n - 2 * a for a in range(rows))


DG_MMA_FLOP_PER_ROW_TILE = 78 * 16 * 8 * 16 * 2 // 16   # 78 f16 m16n8k16 MMAs per 16 rows and tile
# gram_mode 3: tcgen05.mma of M = 128, K = 16 per 16 rows (columns 0..31)
TC_MMA_FLOP_PER_ROW = (2 * 128 * 128 + 2 * 128 * 64) * 16 * 2 // 16   # per 16 rows: two N = 128, two N = 64 MMAs
FF_OPS_PER_PRODUCT = 13                       # binary32 instructions per pair and row (gram_mode 1)
# binary64 lane operations per cell of one 3D matrix-powers level (both chains,
# stencil_mpk_grid_kernel): 17 (Newton and monomial, mu = 0), 19 (Chebyshev)
MPK_FP64_OPS_PER_CELL = {"newton": 17, "monomial": 17, "chebyshev": 19}
FP64_PEAK_TOPS = 152 * 4 * 32 / 64 * 2.070e9 / 1e12   # binary64 lane ops/s: 4 sub-partitions x 32 lanes / 64 cycles
# DRAM bytes per cell and level of stencil_mpk_hybrid_kernel (read + write),
# from a one-pass ncu capture (dram__bytes_read.sum + dram__bytes_write.sum)
# of four steady-state levels of the 160^3 case: 197.27 MB read and
# 44.3-48.6 MB written per launch, 243.6 MB / 4,096,000 cells
MPK_DRAM_BYTES_PER_CELL = 59.48
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="varcoef3d_160", choices=sorted(WORKLOADS))
    ap.add_argument("--hscg-steps", type=int, default=3)
    ap.add_argument("--cpu-outer", type=int, default=3, help="outer loops in the oracle sample")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--gram64-steps", type=int, default=2,
                    help="solves timed with the binary64 FMA Gram beside the line (0: skip)")
    ap.add_argument("--max-outer", type=int, default=0, help="cap outer loops (profiling runs only)")
    ap.add_argument("--s-max", type=int, default=0,
                    help="override the workload's s_max (sigma) for studies; 0 keeps the configuration's")
    ap.add_argument("--gram-mode", type=int, default=None,
                    help="0: binary64 Gram (the method as written); 1: binary32-pair products on the FP32 pipes; "
                         "2: exact 5-bit digit products on the f16 tensor cores (mma.sync); 3: the same digit "
                         "products by tcgen05.mma into tensor memory.  Default: the workload's (3, except 0 for "
                         "the 64^2 Poisson case, where the tensor-core kernels' fixed cost per launch exceeds "
                         "the binary64 kernel's time)")
    return ap.parse_args()


def load_inputs(name):
    from sscg_inputs import generators as gen
    cfg = WORKLOADS[name]
    return gen.config_problem(cfg.get("base", name), scale=cfg.get("scale"))


def oracle_counts(name):
    path = os.path.join(ROOT, "tests", "golden", "oracle_counts.json")
    if os.path.exists(path):
        d = json.load(open(path))
        if name in d:
            return d[name]
    return None


def time_oracle_sample(op, b, x0, cfg, n_outer):
    """Time the CPU oracle (as it stands) for n_outer outer loops of the workload."""
    from oracle import cg
    from oracle.operators import as_matrix
    A = as_matrix(op)
    opts = cg.Options(smax=cfg["smax"], basis=cfg["basis"], max_outer=n_outer)
    t = time.perf_counter()
    _, info = cg.sstep_cg(A, b, x0, cfg["tol"], opts)
    el = time.perf_counter() - t
    return el, info["outer"], info["inner"]


def measure_fp64_peak(torch, dev):
    """FP64 peak of this GPU measured in this run: cuBLAS DGEMM 4096^3 (best of
    5, CUDA events).  GB300's FP64 tensor path (DMMA) and its FP64 FMA share one
    FP64 unit per sub-partition, so DGEMM's rate is the part's FP64 ceiling."""
    m = 4096
    a = torch.randn(m, m, dtype=torch.float64, device=dev)
    bm = torch.randn(m, m, dtype=torch.float64, device=dev)
    c = a @ bm
    torch.cuda.synchronize()
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ bm
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    del a, bm, c
    tf = 2.0 * m ** 3 / best / 1e12
    return tf, f"measured in this run: cuBLAS DGEMM {m}^3, best of 5 ({tf:.3f} TFLOP/s)"


def oracle_full_solve_rates(reps=5):
    """Full oracle solves of the 64^2 Poisson workload (the small configuration
    the oracle finishes in well under a second), timed on the host cores in a
    fresh interpreter: single-thread (BLAS/OpenMP pinned to one thread) and on
    all cores.  Returns {mode: {value (solves/s), cores, seconds per solve}}."""
    code = ("import json, sys, time\n"
            f"sys.path.insert(0, {ROOT!r})\n"
            "from oracle import cg\n"
            "from oracle.operators import as_matrix\n"
            "from sscg_inputs import generators as gen\n"
            "op, b, x0, _ = gen.config_problem('poisson2d_64')\n"
            "A = as_matrix(op)\n"
            "o = cg.Options(smax=8, basis='chebyshev')\n"
            "cg.sstep_cg(A, b, x0, 1e-10, o)\n"
            "ts = []\n"
            f"for _ in range({reps}):\n"
            "    t = time.perf_counter(); x, info = cg.sstep_cg(A, b, x0, 1e-10, o); ts.append(time.perf_counter() - t)\n"
            "ts.sort()\n"
            "print(json.dumps(dict(seconds=ts[len(ts) // 2], outer=info['outer'], inner=info['inner'], "
            "status=info['status'])))\n")
    out = {}
    for mode, threads in (("single_thread", 1), ("all_cores", os.cpu_count() or 1)):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
        try:
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
            d = json.loads(r.stdout.strip().splitlines()[-1])
            out[mode] = {"value": 1.0 / d["seconds"], "unit": "solves/s", "cores": threads,
                         "seconds_per_solve": d["seconds"], "outer_loops": d["outer"], "inner_iters": d["inner"],
                         "status": d["status"], "sample": f"median of {reps} complete solves"}
        except (OSError, ValueError, IndexError, KeyError, subprocess.TimeoutExpired) as e:
            out[mode] = {"value": None, "error": repr(e)[:200]}
    return out


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={SMI_FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def aggregate_ranks(elapsed_s, steps, dist=None, device=None):
    """Whole-job throughput of a replicas run: every rank solved `steps` systems
    in `elapsed_s` seconds; the job's time is the slowest rank's (all-reduce
    MAX), and the value is the total number of solves over that time."""
    import torch
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    worst = float(t.item())
    return world * steps / worst, worst


def algorithmic_bytes_per_outer(n, s, bytes_a):
    """Bytes the method must move per outer loop (A once, 2s-1 new basis columns
    written once, 2s+1 columns read once by the recombination, x/r/p)."""
    return bytes_a + 8.0 * n * (4 * s + 6)


def run_reference(args, cfg):
    """The oracle as it stands, on the host cores: a bounded sample per step."""
    op, b, x0, _ = load_inputs(args.workload)
    counts = oracle_counts(args.workload)
    n_outer = args.cpu_outer
    times = []
    for i in range(args.warmup + args.steps):
        el, outer, inner = time_oracle_sample(op, b, x0, cfg, n_outer)
        if i >= args.warmup:
            times.append(el / max(outer, 1))
    per_outer = statistics.median(times)
    full_outer = counts["sstep_outer"] if counts else None
    value = 1.0 / (per_outer * full_outer) if full_outer else None
    sample = (f"PROJECTED, not timed solves: each step times {n_outer} outer loops of the full-size oracle "
              f"solve, scaled by the oracle's own full-solve outer-loop count ({full_outer}, "
              f"tests/golden/oracle_counts.json); complete solves of the small 64^2 case are timed in "
              f"full_solves_64x64_poisson")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_outer * (full_outer or 0) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"], "s_max": cfg["smax"], "basis": cfg["basis"], "tol": cfg["tol"]},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample, "full_solves_64x64_poisson": oracle_full_solve_rates()},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_rgg(args, cfg, pkg, torch, dev):
    """FP64-stored vs FP32-stored basis on the CSR random-geometric-graph workload."""
    import numpy as np
    op, b_np, x0_np, _ = load_inputs(args.workload)
    n = b_np.size
    solver = pkg.Solver.csr(op.rowptr, op.col, op.val)
    b = torch.tensor(b_np, dtype=torch.float64, device=dev)
    out = {}
    for y32 in (0, 1):
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            x.zero_()
            solver.solve(b, x, tol=cfg["tol"], s_max=cfg["smax"], basis=cfg["basis"], y_fp32=y32,
                         gram_mode=args.gram_mode)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        sts = []
        for _ in range(args.steps):
            x.zero_()
            sts.append(solver.solve(b, x, tol=cfg["tol"], s_max=cfg["smax"], basis=cfg["basis"], y_fp32=y32,
                                    hist_cap=20000, gram_mode=args.gram_mode))
        e1.record()
        torch.cuda.synchronize()
        el = e0.elapsed_time(e1) / 1e3
        st = sts[-1]
        h = pkg.sscg.history(st)
        # one more solve, untimed, with direct launches and per-phase events
        xp = torch.zeros(n, dtype=torch.float64, device=dev)
        sp = solver.solve(b, xp, tol=cfg["tol"], s_max=cfg["smax"], basis=cfg["basis"], y_fp32=y32, profile=1,
                          gram_mode=args.gram_mode)
        phases = {k: getattr(sp, "t_" + k + "_ms") for k in ("mpk", "gram", "kappa", "control", "recombine", "other")}
        out[y32] = dict(value=args.steps / el, ms_per_step=el / args.steps * 1e3, outer=st.outer_iters,
                        inner=st.inner_iters, status=st.status, true_relres=st.true_relres,
                        mean_sk=float(np.mean([r["sk"] for r in h])) if h else None,
                        fp32_replacements=st.fp32_replacements, phase_ms_profiled_solve=phases, x=x.clone())
    err = float(torch.linalg.norm(out[1]["x"] - out[0]["x"]) / torch.linalg.norm(out[0]["x"]))
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t = time.perf_counter()
    hs = solver.hscg(b, x, tol=cfg["tol"])
    torch.cuda.synchronize()
    th = time.perf_counter() - t
    for d in out.values():
        d.pop("x")
    line = {"metric": METRIC, "value": out[0]["value"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out[0]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"], "s_max": cfg["smax"], "basis": cfg["basis"], "tol": cfg["tol"],
                       "nnz": int(op.val.size), "gram_mode": args.gram_mode},
            "fp64_basis": out[0], "fp32_basis": out[1], "fp32_vs_fp64_solution_rel_diff": err,
            "hscg": {"value": 1.0 / th, "unit": "solves/s", "iters": hs.inner_iters, "status": hs.status,
                     "true_relres": hs.true_relres}}
    print(json.dumps(line))


def run_batched(args, cfg, pkg, torch, dev):
    """The batched workload: autotune sigma per size class, then one batched solve per step."""
    import numpy as np
    from sscg_inputs import generators as gen
    systems = gen.batched_stencils(256, 1003)
    solvers = [pkg.Solver.stencil(st.kx, st.ky, st.kz) for st, _ in systems]
    nrhs = [B.shape[0] for _, B in systems]
    b_np = np.concatenate([B.ravel() for _, B in systems])
    b = torch.tensor(b_np, dtype=torch.float64, device=dev)
    # autotuner: one trial per size class (dimension, N to the nearest power of 4)
    classes = {}
    t_tune = time.perf_counter()
    for i, (st, B) in enumerate(systems):
        key = (st.dim, int(round(math.log(st.n, 4))))
        if key not in classes:
            bi = torch.tensor(B[0], dtype=torch.float64, device=dev)
            best, _ = pkg.sscg.sscg_autotune(solvers[i].h, bi, cfg["tol"], [4, 8, 12, 16], trial_outer=12,
                                             basis=cfg["basis"])
            classes[key] = best
    s_max = [classes[(st.dim, int(round(math.log(st.n, 4))))] for st, _ in systems]
    # autotuner, tile shapes and Gram: rows per work chunk and per Gram block,
    # and the binary64 or the tcgen05 Gram, by timed trial batches
    tiles = [(1024, 1024), (2048, 2048), (4096, 4096), (8192, 8192), (2048, 8192)]
    grams = [0, 3] if args.gram_mode == 3 else [0]
    shapes = [(c, g, m) for m in grams for c, g in tiles]
    ib, shape_us = pkg.sscg.sscg_autotune_batch([s.h for s in solvers], nrhs, b, cfg["tol"], s_max, shapes,
                                                trial_outer=20, basis=cfg["basis"])
    batch_gram = shapes[ib][2]
    opts = pkg.sscg.sscg_opts_default(batch_chunk_rows=shapes[ib][0], batch_gram_rows=shapes[ib][1],
                                      gram_mode=batch_gram)
    t_tune = time.perf_counter() - t_tune
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        x.zero_()
        pkg.sscg.sscg_solve_batch([s.h for s in solvers], nrhs, b, x, cfg["tol"], s_max, cfg["basis"], opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        x.zero_()
        rc, stats = pkg.sscg.sscg_solve_batch([s.h for s in solvers], nrhs, b, x, cfg["tol"], s_max, cfg["basis"],
                                              opts)
    e1.record()
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    pairs = sum(nrhs)
    # HSCG on the same GPU: every pair solved by the library's HSCG (one graph
    # launch per pair; there is no batched HSCG)
    hs_el = None
    if args.hscg_steps > 0:
        xh = torch.zeros_like(b)
        hs_iters, hs_conv = 0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        off = 0
        for solver, (st, B) in zip(solvers, systems):
            for k in range(B.shape[0]):
                r = solver.hscg(b[off:off + st.n], xh[off:off + st.n], tol=cfg["tol"])
                hs_iters += r.inner_iters
                hs_conv += int(r.status == 0)
                off += st.n
        torch.cuda.synchronize()
        hs_el = time.perf_counter() - t0
        # the same solves from 16 host threads, each driving its own systems'
        # handles (private streams), so that the GPU overlaps the pairs
        import concurrent.futures as cf
        offs, o = [], 0
        for st, B in systems:
            offs.append(o)
            o += B.shape[0] * st.n
        xc = torch.zeros_like(b)

        def run_systems(idx):
            torch.cuda.set_device(dev)
            it = 0
            for i in idx:
                st, B = systems[i]
                for k in range(B.shape[0]):
                    a = offs[i] + k * st.n
                    it += solvers[i].hscg(b[a:a + st.n], xc[a:a + st.n], tol=cfg["tol"]).inner_iters
            return it

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(16) as ex:
            hc_iters = sum(ex.map(run_systems, [list(range(t, len(systems), 16)) for t in range(16)]))
        torch.cuda.synchronize()
        hc_el = time.perf_counter() - t0
        # batched HSCG: all pairs in lock-step in one graph launch, like the s-step batch
        xh.zero_()
        pkg.sscg.sscg_solve_batch_hscg([s.h for s in solvers], nrhs, b, xh, cfg["tol"])  # warm-up
        xh.zero_()
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record()
        hrc, hst = pkg.sscg.sscg_solve_batch_hscg([s.h for s in solvers], nrhs, b, xh, cfg["tol"])
        h1.record()
        torch.cuda.synchronize()
        hb_el = h0.elapsed_time(h1) / 1e3
        hb = {"value": pairs / hb_el, "unit": "system-rhs solves/s", "seconds": hb_el, "status": hrc,
              "converged": hst["converged"], "iters_total": hst["inner_iters"], "max_iters": hst["max_iters"],
              "note": "sscg_solve_batch_hscg: plain CG for every pair in lock-step, one graph launch"}
    line = {"metric": METRIC, "value": pairs * args.steps / el, "unit": "system-rhs solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"], "systems": len(systems), "pairs": pairs,
                       "unknowns": int(b_np.size), "sigma_by_class": {f"{k[0]}d_4^{k[1]}": v for k, v in classes.items()},
                       "tile_rows": {"chunk": shapes[ib][0], "gram": shapes[ib][1]},
                       "tile_us_per_inner": {f"{c}x{g} gram_mode {m}": t for (c, g, m), t in zip(shapes, shape_us)},
                       "gram_mode": batch_gram,
                       "autotune_s": t_tune},
            "status": rc, "converged": stats["converged"], "outer_loops": stats["outer_loops"],
            "inner_iters_total": stats["inner_iters"], "max_true_relres": stats["max_true_relres"],
            "graph_launches": stats["graph_launches"], "host_syncs": stats["host_syncs"],
            "gpu_launches": stats["kernel_launches"]}
    if hs_el is not None:
        line["hscg_per_pair"] = {"value": pairs / hs_el, "unit": "system-rhs solves/s", "seconds": hs_el,
                                 "iters_total": hs_iters, "converged": hs_conv,
                                 "note": "each pair by sscg_solve_hscg (one graph launch and one host wait per pair), "
                                         "host-timed"}
        line["hscg_batched"] = hb
        line["hscg_concurrent"] = {"value": pairs / hc_el, "unit": "system-rhs solves/s", "seconds": hc_el,
                                   "iters_total": hc_iters,
                                   "note": "the same per-pair HSCG solves from 16 host threads (systems dealt "
                                           "round-robin, each handle on its private stream), host-timed"}
    print(json.dumps(line))


def run_adjoint(args, cfg, pkg, torch, dev):
    """Forward + backward of the differentiable solve (autograd through the C ABI)."""
    from paper_1908_04081_gb300 import autograd as ag
    from paper_1908_04081_gb300.autograd import stencil_solve
    op, b_np, x0_np, extra = load_inputs(args.workload)
    kx = torch.tensor(op.kx, device=dev)
    ky = torch.tensor(op.ky, device=dev)
    b = torch.tensor(b_np, device=dev)
    xt = torch.tensor(extra["x_target"], device=dev)

    def step():
        kxr, kyr = kx.clone().requires_grad_(), ky.clone().requires_grad_()
        x = stencil_solve(kxr, kyr, None, b, tol=cfg["tol"], s_max=cfg["smax"], basis=cfg["basis"],
                          gram_mode=args.gram_mode)
        loss = ((x - xt) ** 2).sum()
        loss.backward()
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the working set (basis 69 MB) fits in L2: flush it between timed steps, outside the events
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    evs = []
    for _ in range(args.steps):
        flush.add_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        loss = step()
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    el = sum(a.elapsed_time(b_) for a, b_ in evs) / 1e3
    line = {"metric": METRIC, "value": args.steps / el, "unit": "forward+backward/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"], "s_max": cfg["smax"], "basis": cfg["basis"], "tol": cfg["tol"],
                       "l2": f"L2 flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)",
                       "gram_mode": args.gram_mode},
            "loss": float(loss.item())}
    for k in ("forward", "adjoint"):
        st = ag.last_stats.get(k)
        if st is not None:
            line[k] = {"outer_loops": st.outer_iters, "inner_iters": st.inner_iters, "true_relres": st.true_relres}
    print(json.dumps(line))


def run_recompute(args, cfg, pkg, torch, dev):
    """Converged solves/s of a 2D stencil with the stored basis (binary64 Gram)
    and without it (recompute_y = 1: the basis formed tile by tile twice per
    outer loop), the same right-hand side and tolerance."""
    op, b_np, _, _ = load_inputs(args.workload)
    n = b_np.size
    solver = pkg.Solver.stencil(op.kx, op.ky, None)
    b = torch.tensor(b_np, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    out = {}
    for rcy in (0, 1):
        def solve(profile=0):
            x.zero_()
            return solver.solve(b, x, tol=cfg["tol"], s_max=cfg["smax"], basis=cfg["basis"], gram_mode=0,
                                recompute_y=rcy, profile=profile)
        for _ in range(args.warmup):
            solve()
        evs, sts = [], []
        with ClockSampler(0) as clk:
            for _ in range(args.steps):
                flush.add_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                sts.append(solve())
                e1.record()
                evs.append((e0, e1))
            torch.cuda.synchronize()
        el = sum(a.elapsed_time(b_) for a, b_ in evs) / 1e3
        sp = solve(profile=1)
        torch.cuda.synchronize()
        ol = max(sp.outer_iters, 1)
        st = sts[-1]
        out[rcy] = {"value": args.steps / el, "ms_per_step": el / args.steps * 1e3, "outer_loops": st.outer_iters,
                    "inner_iters": st.inner_iters, "true_relres": st.true_relres,
                    "converged": all(s.status == 0 and s.true_relres <= cfg["tol"] for s in sts),
                    "basis_bytes": 0 if rcy else 8 * n * (2 * cfg["smax"] + 1),
                    "ms_per_outer_loop_profiled": {k: getattr(sp, "t_" + k + "_ms") / ol
                                                   for k in ("mpk", "gram", "kappa", "control", "recombine",
                                                             "other")},
                    "clocks": clk.summary()}
    line = {"metric": METRIC, "value": out[0]["value"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": out[0]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"], "s_max": cfg["smax"], "basis": cfg["basis"], "tol": cfg["tol"],
                       "l2": f"L2 flushed between timed solves ({L2_FLUSH_BYTES >> 20} MB write)", "gram_mode": 0,
                       "timing": "CUDA events around each solve (graph path); phases from one profiled solve"},
            "stored_basis": out[0], "recompute_y": out[1],
            "note": "recompute_y: the (2 s + 1) N basis is not stored; the Gram phase forms the basis and G, the "
                    "recombine phase forms it again for x, r, p"}
    print(json.dumps(line))


def main():
    args = parse_args()
    cfg = dict(WORKLOADS[args.workload])
    if args.gram_mode is None:
        args.gram_mode = cfg.get("gram_mode", 3)
    if args.s_max > 0:
        cfg["smax"] = args.s_max
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, cfg)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1908_04081_gb300 as pkg

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    if args.workload in ("rgg_2m", "rgg_400k", "batched_256", "adjoint2d_512", "varcoef2d_512"):
        if rank == 0:
            {"rgg_2m": run_rgg, "rgg_400k": run_rgg, "batched_256": run_batched,
             "adjoint2d_512": run_adjoint, "varcoef2d_512": run_recompute}[args.workload](
                args, cfg, pkg, torch, dev)
        if world > 1:
            dist.destroy_process_group()
        return

    op, b_np, x0_np, _ = load_inputs(args.workload)
    n = b_np.size
    if hasattr(op, "kx"):
        solver = pkg.Solver.stencil(op.kx, op.ky, op.kz)
        bytes_a = 8.0 * (op.kx.size + op.ky.size + (op.kz.size if op.kz is not None else 0) + n)
    else:
        solver = pkg.Solver.csr(op.rowptr, op.col, op.val)
        bytes_a = 12.0 * op.val.size + 8.0 * (n + 1)
    b = torch.tensor(b_np, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def solve(profile=0, gram_mode=None):
        x.zero_()
        extra = {"max_outer": args.max_outer} if args.max_outer > 0 else {}
        gm = args.gram_mode if gram_mode is None else gram_mode
        if gm:
            extra["gram_mode"] = gm
        return solver.solve(b, x, tol=cfg["tol"], s_max=cfg["smax"], basis=cfg["basis"], hist_cap=20000,
                            profile=profile, **extra)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()

    # ---- timed region: K complete solves on the production path (one CUDA
    # graph launch per solve, the loop decided on the device, one host wait).
    # A working set below twice the L2 (129 MB) would stay cached from one
    # solve to the next, so then L2 is flushed (a 256 MB write) between the
    # timed solves, outside the events.
    y_bytes = 8.0 * n * (2 * cfg["smax"] + 1)
    flush = None
    if y_bytes + bytes_a < 2 * L2_BYTES:
        flush = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
        l2_note = f"L2 flushed between timed solves ({L2_FLUSH_BYTES >> 20} MB write); working set " \
                  f"{(y_bytes + bytes_a) / 1e6:.1f} MB"
    else:
        l2_note = f"inputs larger than L2 (basis Y {y_bytes / 1e9:.2f} GB, operator {bytes_a / 1e6:.0f} MB)"
    stats = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        evs = []
        for _ in range(args.steps):
            if flush is not None:
                flush.add_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(solve())
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    value, elapsed = aggregate_ranks(sum(a.elapsed_time(b_) for a, b_ in evs) / 1e3, args.steps,
                                     dist if world > 1 else None, dev)
    clocks = clk.summary()
    ok = all(s.status == 0 and s.true_relres <= cfg["tol"] for s in stats)
    ms_per_step = elapsed / args.steps * 1e3
    st0 = stats[-1]
    hist = pkg.sscg.history(st0)
    alg_bytes = sum(algorithmic_bytes_per_outer(n, h["sbar"], bytes_a) for h in hist)
    hbm_gbs = alg_bytes / (ms_per_step / 1e3) / 1e9
    launches = sum(s.kernel_launches for s in stats)

    # ---- one more solve, untimed by the line's value: direct launches with
    # CUDA events on the library's stream around every phase (the per-kernel
    # durations of the rooflines below come from it)
    if flush is not None:
        flush.add_(1)
    sp = solve(profile=1)
    torch.cuda.synchronize()
    hist_p = pkg.sscg.history(sp)
    phase_ms = {k: getattr(sp, "t_" + k + "_ms") for k in ("mpk", "gram", "kappa", "control", "recombine", "other")}
    t_gram = sp.t_gram_ms / 1e3
    f_gram = sp.gram_flops
    n_gram = sp.n_gram_launches
    gram_tflops = f_gram / t_gram / 1e12 if t_gram > 0 else None
    fp64_peak, fp64_note = measure_fp64_peak(torch, dev)
    gram_traffic = None
    if hist_p and hasattr(op, "kx"):
        gram_traffic = sum(8.0 * n * (2 * h["sbar"] + 1) + 3.4e6 for h in hist_p) / len(hist_p)
    traffic_src = ("scaled from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same kernel "
                   "on a smaller or earlier case, by the rows and columns each launch processes; not measured "
                   "in this run")
    # the matrix-powers phase: binary64 issue bound (stencil workloads)
    mpk_roof = None
    if hasattr(op, "kx") and op.kz is not None and phase_ms["mpk"] > 0:
        ops = MPK_FP64_OPS_PER_CELL.get(cfg["basis"], 17)
        # s-bar levels per outer loop; the last one advances the P chain only
        lane_ops = sum(n * ops * (h["sbar"] - 0.5) for h in hist_p)
        levels = sum(h["sbar"] for h in hist_p)
        mpk_tops = lane_ops / (phase_ms["mpk"] / 1e3) / 1e12
        peak_ops = fp64_peak / 2.0   # one FMA = 2 flop = one lane operation
        # algorithmic HBM bytes of the phase: per level the operator (diag and
        # the three face arrays, 32 B per cell) and P_l, R_l read, P_{l+1},
        # R_{l+1} written (the last level of a block advances P only)
        mpk_bytes = sum(n * (32.0 * h["sbar"] + 32.0 * (h["sbar"] - 0.5)) for h in hist_p)
        mpk_gbs = mpk_bytes / (phase_ms["mpk"] / 1e3) / 1e9
        mpk_roof = {"bound": "alu", "kernel": "stencil_mpk_hybrid_kernel (one matrix-powers level, both chains; "
                                              "cells split between binary64 FMAs and exact integer products)",
                    "achieved": mpk_tops, "peak": peak_ops, "unit": "T binary64 lane-ops/s",
                    "frac": mpk_tops / peak_ops,
                    "traffic": (MPK_DRAM_BYTES_PER_CELL * n) if MPK_DRAM_BYTES_PER_CELL else None,
                    "traffic_source": "an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of this "
                                      "kernel at 160^3 (four steady-state levels), bytes per cell times the "
                                      "cells of a launch; not measured in this run",
                    "launches": levels,
                    "algorithmic": f"{ops} binary64 operations per cell and level (formed by the FP64 unit or, in "
                                   f"the integer warps, exactly by the integer pipes)",
                    "peak_note": fp64_note + " (as lane operations: TFLOP/s / 2); the integer warps add work "
                                 "beyond the FP64 unit, so frac can exceed 1",
                    "hbm": {"achieved_gbs": mpk_gbs, "peak_gbs": HBM_PEAK_GBS, "frac": mpk_gbs / HBM_PEAK_GBS,
                            "algorithmic": "64 B per cell and level (operator 32, two columns read, two written)"},
                    "timing": "CUDA events around the matrix-powers phase of a profiled solve"}
    if args.gram_mode == 0:
        roofline = {"bound": "alu", "kernel": "gram_partial+gram_reduce (G = Y^T Y, FP64)",
                    "achieved": gram_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": (gram_tflops / fp64_peak) if gram_tflops else None,
                    "traffic": gram_traffic, "traffic_source": traffic_src, "launches": n_gram,
                    "peak_note": fp64_note}
    elif args.gram_mode == 3:
        # executed tcgen05 f16 MMA flops (per 16 rows: 128 x 128 x 16 twice, 128 x 64 x 16 twice)
        tc_flop = sum(n * TC_MMA_FLOP_PER_ROW for h in hist_p)
        tc_tf = tc_flop / t_gram / 1e12 if t_gram > 0 else None
        roofline = {"bound": "tensor", "kernel": "gram_chunk_exp+gram_partial_tc+gram_reduce (G = Y^T Y, exact "
                                                  "6-bit digit products by tcgen05.mma into tensor memory)",
                    "achieved": tc_tf, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": (tc_tf / BF16_PEAK_TFLOPS) if tc_tf else None,
                    "traffic": gram_traffic, "traffic_source": traffic_src, "launches": n_gram,
                    "gram_fp64_equiv_tflops": gram_tflops,
                    "peak_note": f"{BF16_PEAK_SRC} bf16 burst {BF16_PEAK_TFLOPS:.0f} TFLOP/s (same nominal dense rate "
                                 "as f16)"}
    elif args.gram_mode == 2:
        # digit Gram: executed f16 MMA flops (tiles x 78 MMAs per 16 rows) per
        # second of the Gram phase (which includes the chunk-exponent pass)
        dg_flop = sum(n * dg_tiles(2 * h["sbar"] + 1) * DG_MMA_FLOP_PER_ROW_TILE for h in hist_p)
        dg_tf = dg_flop / t_gram / 1e12 if t_gram > 0 else None
        roofline = {"bound": "tensor", "kernel": "gram_chunk_exp+gram_partial_dg+gram_reduce (G = Y^T Y, "
                                                  "exact 5-bit digit products on f16 tensor cores)",
                    "achieved": dg_tf, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": (dg_tf / BF16_PEAK_TFLOPS) if dg_tf else None,
                    "traffic": gram_traffic, "traffic_source": traffic_src, "launches": n_gram,
                    "gram_fp64_equiv_tflops": gram_tflops,
                    "peak_note": f"{BF16_PEAK_SRC} bf16 burst {BF16_PEAK_TFLOPS:.0f} TFLOP/s (same nominal dense rate "
                                 "as f16); mma.sync f16 measured 604 TFLOP/s on this part"}
    else:
        # binary32-pair Gram: 13 binary32 instructions per unique (i <= j) pair and row
        # (one binary64 FMA is 2 flop, so gram_flops / 2 is pairs x rows)
        tinst = FF_OPS_PER_PRODUCT * (f_gram / 2) / t_gram / 1e12 if t_gram > 0 else None
        roofline = {"bound": "alu", "kernel": "gram_partial_ff+gram_reduce (G = Y^T Y, binary32 pairs)",
                    "achieved": tinst, "peak": FP32_PEAK_TINST, "unit": "T binary32 inst/s",
                    "frac": (tinst / FP32_PEAK_TINST) if tinst else None,
                    "traffic": gram_traffic, "traffic_source": traffic_src, "launches": n_gram,
                    "gram_fp64_equiv_tflops": gram_tflops,
                    "peak_note": "derived: 152 SMs x 128 binary32 lanes/clk x 2070 MHz"}
    # report the dominant phase's kernel; the other one beside it
    gram_roof = roofline
    if mpk_roof is not None and phase_ms["mpk"] > phase_ms["gram"]:
        roofline = dict(mpk_roof, secondary=gram_roof)
    elif mpk_roof is not None:
        roofline = dict(gram_roof, secondary=mpk_roof)

    # ---- the same solve with the binary64 FMA Gram (the method as written)
    gram64 = None
    if args.gram_mode != 0 and args.gram64_steps > 0:
        solve(gram_mode=0)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        gs = [solve(gram_mode=0) for _ in range(args.gram64_steps)]
        g1.record(stream)
        torch.cuda.synchronize()
        gel = g0.elapsed_time(g1) / 1e3
        gram64 = {"value": args.gram64_steps / gel, "unit": "solves/s", "steps": args.gram64_steps,
                  "outer_loops": gs[-1].outer_iters, "inner_iters": gs[-1].inner_iters,
                  "true_relres": gs[-1].true_relres, "converged": all(g.status == 0 for g in gs),
                  "note": "gram_mode 0: G = Y^T Y by binary64 FMAs, graph path"}

    # ---- HSCG on the same GPU: with binary64 FMA chains in its SpMV (the
    # comparator as written) and, for stencils, with the SpMV split between
    # FMA chains and exact integer products like the s-step matrix powers
    def time_hscg(split):
        solver.hscg(b, x.zero_(), tol=cfg["tol"], spmv_fp64_per16=split)
        torch.cuda.synchronize()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        hs = []
        h0.record(stream)
        for _ in range(args.hscg_steps):
            x.zero_()
            hs.append(solver.hscg(b, x, tol=cfg["tol"], spmv_fp64_per16=split))
        h1.record(stream)
        torch.cuda.synchronize()
        hscg_el = h0.elapsed_time(h1) / 1e3
        return {"value": args.hscg_steps / hscg_el, "unit": "solves/s", "ms_per_step": hscg_el / args.hscg_steps * 1e3,
                "iters": hs[-1].inner_iters, "true_relres": hs[-1].true_relres,
                "converged": all(h.status == 0 for h in hs),
                "hbm_gbs_alg": (hs[-1].inner_iters * (bytes_a + 8.0 * n * 9)) / (hscg_el / args.hscg_steps) / 1e9}

    hscg = hscg_split = None
    if args.hscg_steps > 0:
        hscg = time_hscg(16)
        if hasattr(op, "kx"):
            hscg_split = time_hscg(-1)
            hscg_split["note"] = ("sscg_solve_hscg_ex: the SpMV's warps split between binary64 FMA chains and "
                                  "exact integer products, the library's default share (as the s-step levels)")

    # ---- end to end through the C ABI with host buffers (copies inside)
    pin_b = torch.tensor(b_np, dtype=torch.float64).pin_memory()
    pin_x = torch.zeros(n, dtype=torch.float64).pin_memory()
    bn, xn = pin_b.numpy(), pin_x.numpy()
    e2e_steps = max(0, min(args.steps, args.e2e_steps))
    e2e = None
    if e2e_steps > 0:
        torch.cuda.synchronize()
        te = time.perf_counter()
        for _ in range(e2e_steps):
            xn[:] = 0.0
            solver.solve_host(bn, xn, tol=cfg["tol"], s_max=cfg["smax"], basis=cfg["basis"],
                              **({"gram_mode": args.gram_mode} if args.gram_mode else {}))
        te = time.perf_counter() - te
        e2e = {"value": world * e2e_steps / te, "unit": "solves/s", "h2d_bytes_per_step": 16 * n,
               "d2h_bytes_per_step": 8 * n, "steps": e2e_steps}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        el, outer, _ = time_oracle_sample(op, b_np, x0_np, cfg, args.cpu_outer)
        per_outer = el / max(outer, 1)
        cpu = {"value": 1.0 / (per_outer * st0.outer_iters), "unit": "solves/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"PROJECTED, not a timed solve: the first {outer} outer loops of the full-size oracle "
                         f"solve ({el:.1f} s), scaled by the GPU solve's {st0.outer_iters} outer loops; "
                         f"numpy/OpenBLAS Gram on all cores, scipy SpMV single-threaded",
               "full_solves_64x64_poisson": oracle_full_solve_rates()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["desc"], "s_max": cfg["smax"], "basis": cfg["basis"], "tol": cfg["tol"],
                       "parallelism": "replicas" if world > 1 else "single-gpu",
                       "l2": l2_note,
                       "timing": "CUDA events around K solves on the production path (one graph launch and "
                                 "one host wait per solve); the phase split and kernel rooflines come from one "
                                 "extra profiled solve (direct launches, CUDA events around each phase)",
                       "gram": {0: "binary64 FMA", 1: "binary32-pair products, binary64 accumulation",
                                2: "G at binary64 normwise accuracy or better: every value written as 12 5-bit "
                                   "digits (exact within 2^7 of its column's largest, else rounded at 2^-60 of "
                                   "it), digit products exact on the f16 tensor cores, exact binary32 sums over "
                                   "1024 rows, binary64 across blocks (normwise error below binary64 FMAs')",
                                3: "G at binary64 normwise accuracy or better: the digit arithmetic of mode 2 as "
                                   "tcgen05.mma with f32 accumulators in tensor memory (one plane pair each, exact "
                                   "binary32 sums over 4096 rows); the 33rd column by binary64 FMAs"}
                       [args.gram_mode]},
            "converged": ok, "true_relres": max(s.true_relres for s in stats),
            "outer_loops": st0.outer_iters, "inner_iters": st0.inner_iters, "host_syncs": st0.host_syncs,
            "ms_per_outer_loop": ms_per_step / st0.outer_iters,
            "hbm_gbs_alg": hbm_gbs, "hbm_frac_alg": hbm_gbs / HBM_PEAK_GBS,
            "hbm_peak_note": "measured copy peak (MEASURED_PEAKS.json); algorithmic bytes per outer loop: "
                             "the operator once plus 8 N (4 s-bar + 6)",
            "phase_ms_profiled_solve": phase_ms,
            "profiled_solve": {"outer_loops": sp.outer_iters, "inner_iters": sp.inner_iters,
                               "ms": sum(phase_ms.values()), "host_syncs": sp.host_syncs},
            "gram_binary64": gram64,
            "hscg": hscg,
            "hscg_split_spmv": hscg_split,
            "roofline": roofline,
            "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
