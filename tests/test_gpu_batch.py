"""GPU parity of the batched solve (many systems x right-hand sides, one graph launch).

Every (system, right-hand side) pair of a seeded batch of uneven 2D/3D
variable-coefficient systems must converge (true residual <= tol, checked here
with the oracle's sparse matrix) and match the oracle's run of Algorithm 5 on
that pair within 1e-8 in the solution.  Outer and inner counts are within 10 %
of the oracle's summed over the batch, and per pair within max(2, 20 %): the
pairs are small (30-60 outer loops), where one rounding-driven decision moves a
count by more than 10 %.  The graph-driven batch must equal the host-polled
batch bitwise (same kernels, same order).
"""
import numpy as np
import pytest

from oracle import cg
from oracle.operators import as_matrix
from sscg_inputs import generators as gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1908_04081_gb300 as p
    p.load_library()
    return p


def build(pkg, count, seed, n_lo, n_hi, max_rhs):
    systems = gen.batched_stencils(count, seed, n_lo=n_lo, n_hi=n_hi, max_rhs=max_rhs)
    solvers = [pkg.Solver.stencil(st.kx, st.ky, st.kz) for st, _ in systems]
    nrhs = [B.shape[0] for _, B in systems]
    b = np.concatenate([B.ravel() for _, B in systems])
    return systems, solvers, nrhs, b


def split(systems, v):
    out, off = [], 0
    for st, B in systems:
        for k in range(B.shape[0]):
            out.append((st, B[k], v[off:off + st.n]))
            off += st.n
    return out


@pytest.mark.parametrize("gram_mode,mpk_split", [(0, -1), (3, -1), (0, 0), (3, 16)])
def test_batch_matches_oracle_per_pair(pkg, gram_mode, mpk_split):
    """With the binary64 Gram and with the tcgen05 digit Gram (one thread block
    per 2048-row Gram block of a pair, its scales computed over its rows), and
    with the matrix-powers rows split between binary64 FMA chains and exact
    integer products by default (-1), on integer products alone (0) and on
    FMA chains alone (16)."""
    systems, solvers, nrhs, b = build(pkg, 7, 1003, 300, 9000, 3)
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    s_max = [8 if st.dim == 2 else 12 for st, _ in systems]
    rc, stats = pkg.sscg.sscg_solve_batch([s.h for s in solvers], nrhs, bt, xt, 1e-10, s_max, "newton",
                                          pkg.sscg.sscg_opts_default(gram_mode=gram_mode,
                                                                     mpk_fp64_per16=mpk_split))
    assert pkg.sscg.sscg_wait_failures() == 0
    assert rc == 0 and stats["converged"] == stats["npairs"] == sum(nrhs)
    assert stats["graph_launches"] == 1 and stats["host_syncs"] == 1
    x = xt.cpu().numpy()
    sig_of_pair = [s for s, (_, B) in zip(s_max, systems) for _ in range(B.shape[0])]
    tot = np.zeros(4)
    for j, (st, bj, xj) in enumerate(split(systems, x)):
        A = as_matrix(st)
        assert np.linalg.norm(bj - A @ xj) / np.linalg.norm(bj) <= 1e-10
        xo, info = cg.sstep_cg(A, bj, np.zeros(st.n), 1e-10, cg.Options(smax=sig_of_pair[j], basis="newton"))
        assert info["status"] == 0
        go, gi = stats["pair_outer"][j], stats["pair_inner"][j]
        assert abs(go - info["outer"]) <= max(2, 0.2 * info["outer"]), (j, go, info["outer"])
        assert abs(gi - info["inner"]) <= max(2, 0.2 * info["inner"]), (j, gi, info["inner"])
        tot += (go, info["outer"], gi, info["inner"])
        assert np.linalg.norm(xj - xo) <= 1e-8 * np.linalg.norm(xo)
    assert abs(tot[0] - tot[1]) <= 0.1 * tot[1] and abs(tot[2] - tot[3]) <= 0.1 * tot[3], tot


def test_batch_graph_equals_host_polling_and_zero_rhs_counts(pkg):
    systems, solvers, nrhs, b = build(pkg, 5, 77, 200, 4000, 2)
    nrhs[1] = 0                                   # a system with no right-hand side
    b = np.concatenate([B[:k].ravel() for (_, B), k in zip(systems, nrhs)])
    bt = torch.tensor(b, device="cuda")
    s_max = [6] * len(systems)
    x1 = torch.zeros_like(bt)
    rc1, st1 = pkg.sscg.sscg_solve_batch([s.h for s in solvers], nrhs, bt, x1, 1e-10, s_max, "chebyshev")
    o = pkg.sscg.sscg_opts_default(use_graph=0, check_every=3)
    x2 = torch.zeros_like(bt)
    rc2, st2 = pkg.sscg.sscg_solve_batch([s.h for s in solvers], nrhs, bt, x2, 1e-10, s_max, "chebyshev", o)
    assert rc1 == rc2 == 0
    assert torch.equal(x1, x2)
    assert st1["pair_outer"] == st2["pair_outer"] and st1["pair_inner"] == st2["pair_inner"]
    assert st2["host_syncs"] > 1 and st1["host_syncs"] == 1


def test_autotune_picks_a_candidate(pkg):
    st = gen.varcoef_stencil((40, 40, 40), seed=5)
    s = pkg.Solver.stencil(st.kx, st.ky, st.kz)
    b = torch.tensor(gen.random_rhs(st.n, 1), device="cuda")
    best, times = pkg.sscg.sscg_autotune(s.h, b, 1e-10, [4, 8, 16], trial_outer=10, basis="newton")
    assert best in (4, 8, 16)
    assert all(t > 0 for t in times)
    assert times[[4, 8, 16].index(best)] == min(times)


def test_batch_tile_shapes_and_their_autotuner(pkg):
    """The batch's rows per work chunk and per Gram block are runtime choices:
    every shape converges every pair to tol (independent residual) with the
    same solutions to within 1e-8 (only summation orders change), the shape
    autotuner returns one of its candidates with the least time, and
    out-of-range shapes are rejected."""
    systems, solvers, nrhs, b = build(pkg, 6, 2024, 300, 20000, 2)
    bt = torch.tensor(b, device="cuda")
    hs = [s.h for s in solvers]
    s_max = [8] * len(systems)
    xs = []
    for chunk, gram in ((2048, 2048), (256, 512), (8192, 128)):
        o = pkg.sscg.sscg_opts_default(batch_chunk_rows=chunk, batch_gram_rows=gram)
        xt = torch.zeros_like(bt)
        rc, stats = pkg.sscg.sscg_solve_batch(hs, nrhs, bt, xt, 1e-10, s_max, "newton", o)
        assert rc == 0 and stats["converged"] == stats["npairs"]
        assert stats["device_ms"] > 0.0
        x = xt.cpu().numpy()
        for st, bj, xj in split(systems, x):
            A = as_matrix(st)
            assert np.linalg.norm(bj - A @ xj) <= 1e-10 * np.linalg.norm(bj)
        xs.append(x)
    for x in xs[1:]:
        for (_, _, x0j), (_, _, xj) in zip(split(systems, xs[0]), split(systems, x)):
            assert np.linalg.norm(xj - x0j) <= 1e-8 * np.linalg.norm(x0j)
    shapes = [(1024, 1024), (2048, 2048), (4096, 8192)]
    best, times = pkg.sscg.sscg_autotune_batch(hs, nrhs, bt, 1e-10, s_max, shapes, trial_outer=8)
    assert 0 <= best < len(shapes)
    assert all(t > 0 for t in times) and times[best] == min(times)
    # the Gram as a third dimension of the candidates (binary64 or tcgen05)
    cands = [(2048, 2048, 0), (2048, 2048, 3), (1024, 1024, 3)]
    best, times = pkg.sscg.sscg_autotune_batch(hs, nrhs, bt, 1e-10, s_max, cands, trial_outer=8)
    assert 0 <= best < len(cands)
    assert all(t > 0 for t in times) and times[best] == min(times)
    with pytest.raises(pkg.sscg.SscgError):
        pkg.sscg.sscg_autotune_batch(hs, nrhs, bt, 1e-10, s_max, [(2048, 2048, 2)], trial_outer=2)
    with pytest.raises(pkg.sscg.SscgError):
        pkg.sscg.sscg_solve_batch(hs, nrhs, bt, torch.zeros_like(bt), 1e-10, s_max, "newton",
                                  pkg.sscg.sscg_opts_default(batch_chunk_rows=64))
    for mode in (1, 2):  # the batch has neither the binary32-pair nor the mma.sync digit Gram
        with pytest.raises(pkg.sscg.SscgError):
            pkg.sscg.sscg_solve_batch(hs, nrhs, bt, torch.zeros_like(bt), 1e-10, s_max, "newton",
                                      pkg.sscg.sscg_opts_default(gram_mode=mode))
    # the tcgen05 Gram sums at most 16384 rows per thread block
    with pytest.raises(pkg.sscg.SscgError):
        pkg.sscg.sscg_solve_batch(hs, nrhs, bt, torch.zeros_like(bt), 1e-10, s_max, "newton",
                                  pkg.sscg.sscg_opts_default(gram_mode=3, batch_gram_rows=32768))


def test_batched_hscg_matches_per_pair_hscg(pkg):
    """The batched HSCG comparator (one graph launch over all pairs) takes each
    pair through the iterations of the single-system HSCG (its kernels sum in
    another order: counts within 2, solutions within 1e-8), every pair to tol
    (independent residual), and the oracle's HSCG count within 2 per pair."""
    systems, solvers, nrhs, b = build(pkg, 6, 77, 300, 9000, 3)
    bt = torch.tensor(b, device="cuda")
    xb = torch.zeros_like(bt)
    rc, stats = pkg.sscg.sscg_solve_batch_hscg([s.h for s in solvers], nrhs, bt, xb, 1e-10)
    assert rc == 0 and stats["converged"] == stats["npairs"] == sum(nrhs)
    assert stats["graph_launches"] == 1 and stats["device_ms"] > 0.0
    x = xb.cpu().numpy()
    off, j = 0, 0
    for solver, (st, B) in zip(solvers, systems):
        A = as_matrix(st)
        for k in range(B.shape[0]):
            xs = torch.zeros(st.n, dtype=torch.float64, device="cuda")
            r = solver.hscg(torch.tensor(B[k], device="cuda"), xs, tol=1e-10)
            xj = x[off:off + st.n]
            assert r.status == 0 and abs(stats["pair_iters"][j] - r.inner_iters) <= 2
            assert np.linalg.norm(xj - xs.cpu().numpy()) <= 1e-8 * np.linalg.norm(xj)
            assert np.linalg.norm(B[k] - A @ xj) <= 1e-10 * np.linalg.norm(B[k])
            _, h = cg.hscg(A, B[k], np.zeros(st.n), 1e-10)
            assert abs(h["iters"] - stats["pair_iters"][j]) <= 2
            off += st.n
            j += 1
