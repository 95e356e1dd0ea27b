"""GPU parity of the differentiable solve (the adjoint pattern).

Small grids: gradients against the oracle's dense adjoint (1e-7 relative to the
largest entry; forward and adjoint solves at tol 1e-12).  Full size (512^2,
N = 262144): 32 seeded face conductivities, gradient against central finite
differences of the forward map with h = 1e-6 k_f, each perturbed solve done as a
correction solve from x(k) so that x+ - x- is resolved (agreement 1e-4).
"""
import numpy as np
import pytest

from oracle import adjoint as oadj
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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("gram_mode", [0, 2])
@pytest.mark.parametrize("shape", [(16, 16), (6, 5, 7)])
def test_gradients_match_dense_adjoint(pkg, shape, gram_mode):
    from paper_1908_04081_gb300.autograd import stencil_solve
    st = gen.varcoef_stencil(shape, seed=5)
    b = gen.random_rhs(st.n, 1)
    xt = gen.random_rhs(st.n, 2)
    L, x_o, lam_o, gkx_o, gky_o, gkz_o = oadj.face_gradients(st, b, xt)
    kx = dev(st.kx).requires_grad_()
    ky = dev(st.ky).requires_grad_()
    kz = dev(st.kz).requires_grad_() if st.kz is not None else None
    bt = dev(b).requires_grad_()
    x = stencil_solve(kx, ky, kz, bt, tol=1e-12, s_max=8, basis="newton", gram_mode=gram_mode)
    loss = ((x - dev(xt)) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - L) <= 1e-9 * L
    pairs = [(kx.grad, gkx_o), (ky.grad, gky_o), (bt.grad, lam_o)]
    if kz is not None:
        pairs.append((kz.grad, gkz_o))
    for g, ref in pairs:
        g = g.cpu().numpy().reshape(ref.shape)
        assert np.max(np.abs(g - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_full_size_gradient_vs_finite_differences(pkg):
    from paper_1908_04081_gb300.autograd import stencil_solve
    op, b, x0, extra = gen.config_problem("adjoint2d_512")
    xt = extra["x_target"]
    kx = dev(op.kx).requires_grad_()
    ky = dev(op.ky).requires_grad_()
    bt = dev(b)
    xtt = dev(xt)
    # the benchmark's configuration: the tensor-core digit Gram
    x = stencil_solve(kx, ky, None, bt, tol=1e-10, s_max=16, basis="newton", gram_mode=2)
    loss = ((x - xtt) ** 2).sum()
    loss.backward()
    x = x.detach()
    rng = np.random.default_rng(1004)
    checked = 0
    rel_errors = []
    gscale = float(np.mean(np.abs(kx.grad.cpu().numpy())) + np.mean(np.abs(ky.grad.cpu().numpy()))) / 2
    for _ in range(32):
        which = rng.integers(0, 2)
        arr = op.kx if which == 0 else op.ky
        g = (kx.grad if which == 0 else ky.grad).cpu().numpy()
        idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
        h = 1e-6 * arr[idx]
        xs = []
        for sign in (1.0, -1.0):
            kxp, kyp = op.kx.copy(), op.ky.copy()
            (kxp if which == 0 else kyp)[idx] += sign * h
            s = pkg.Solver.stencil(kxp, kyp, None)
            r = torch.zeros_like(bt)
            s.spmv(x, r)
            r = bt - r                          # residual of x(k) for the perturbed operator
            d = torch.zeros_like(bt)
            st = s.solve(r.contiguous(), d, tol=1e-10, s_max=16, basis="newton")
            assert st.status == 0
            xs.append(x + d)
            s.close()
        xp, xm = xs
        fd = float(((xp - xm) * (xp + xm - 2 * xtt)).sum()) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-3 * abs(fd) + 1e-4 * gscale, (which, idx, fd, g[idx])
        rel_errors.append(abs(fd - g[idx]) / abs(fd))
        checked += 1
    assert checked == 32
    assert float(np.median(rel_errors)) <= 1e-4, np.median(rel_errors)
