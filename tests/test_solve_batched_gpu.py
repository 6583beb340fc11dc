"""Batched solves (vsie_solve_batched): every column of a block of plane-wave right-hand
sides reaches the FP64 residual tolerance measured with the oracle's matrix, in the mixed
mode (tensor-core FP32 inner apply, FP64 multi-RHS residuals) and the FP64 mode; and the
FP64 multi-RHS apply against the oracle."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return torch, B


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SMALL = {
    "ball12_k2": lambda: W.single_ball(12, 3, 2.0),
    "layered10_k5": lambda: W.layered_ball(10, 2, 2, 5.0),
}


@pytest.fixture(scope="module", params=sorted(SMALL))
def case(request):
    _setup()
    w = SMALL[request.param]()
    D = O.Discretisation.from_workload(w)
    return request.param, w, D, D.assemble()


def test_fp64_batched_apply_matches_oracle(case):
    torch, B = _setup()
    name, w, D, A = case
    op = B.Operator.from_workload(w)
    X = np.stack([W.random_vector(D.n, 60 + r) for r in range(7)])
    Y = op.apply_batched(torch.from_numpy(X).cuda(), precision=64).cpu().numpy()
    ref = X @ A.T
    for r in range(7):
        assert _rel(Y[r], ref[r]) <= 1e-12, (name, r, _rel(Y[r], ref[r]))
    # two blocks of 64 columns (ragged second block) against the single-column FP64 apply
    X2 = torch.from_numpy(np.stack([W.random_vector(D.n, 200 + r) for r in range(70)])).cuda()
    Y2 = op.apply_batched(X2, precision=64)
    Yc = op.apply(X2, precision=64)
    for r in (0, 63, 64, 69):
        assert float(torch.linalg.norm(Y2[r] - Yc[r]) / torch.linalg.norm(Yc[r])) <= 1e-13


@pytest.mark.parametrize("mode", [32, 64])
def test_batched_solve_reaches_fp64_residual(case, mode):
    torch, B = _setup()
    name, w, D, A = case
    op = B.Operator.from_workload(w)
    dirs = W.fibonacci_dirs(6)
    b = op.plane_wave_rhs(dirs)                       # (6, n) on the device
    b = torch.cat([b, torch.zeros_like(b[:1])])       # a zero column: x = 0 at once
    x, infos = op.solve_batched(b.contiguous(), mode=mode, tol=1e-8, max_iters=400)
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    for c in range(6):
        res = np.linalg.norm(bh[c] - A @ xh[c]) / np.linalg.norm(bh[c])
        assert res <= 1.5e-8, (name, mode, c, res, infos[c])
        assert infos[c].rel_residual <= 1e-8
        assert _rel(xh[c], np.linalg.solve(A, bh[c])) <= 1e-6
        if mode == 32:
            assert infos[c].fp32_applies > infos[c].fp64_applies
        else:
            assert infos[c].fp32_applies == 0
    assert np.all(xh[6] == 0) and infos[6].rel_residual == 0.0


def test_batched_solve_more_than_one_block():
    """70 columns: two blocks of the multi-RHS kernels per apply, columns converging at
    different steps leave the active set; every column agrees with the single-RHS solver."""
    torch, B = _setup()
    w = W.single_ball(12, 3, 2.0)
    op = B.Operator.from_workload(w)
    D = O.Discretisation.from_workload(w)
    A = D.assemble()
    b = op.plane_wave_rhs(W.fibonacci_dirs(70)).contiguous()
    x, infos = op.solve_batched(b, mode=32, tol=1e-8, max_iters=300)
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    worst = max(np.linalg.norm(bh[c] - A @ xh[c]) / np.linalg.norm(bh[c]) for c in range(70))
    assert worst <= 1.5e-8, worst
    for c in (0, 35, 69):
        xs, _ = op.solve(b[c].contiguous(), mode=64, tol=1e-10, max_iters=400)
        assert _rel(xh[c], xs.cpu().numpy()) <= 1e-6


def test_batched_solve_rejects_adjoint_and_bad_options():
    torch, B = _setup()
    w = W.single_ball(6, 1, 2.0)
    op = B.Operator.from_workload(w)
    b = op.plane_wave_rhs(W.fibonacci_dirs(2)).contiguous()
    with pytest.raises(B.VsieError) as e:
        op.solve_batched(b, mode=16)
    assert e.value.status == 1
    with pytest.raises(B.VsieError) as e:
        op.solve_batched(b, restart=2000, max_iters=5000)
    assert e.value.status == 1


def test_batched_solve_nested24_matches_single_solves():
    """Mid-size nested k0 = 10 workload, 8 plane waves: the mixed batched solve reaches the
    tolerance (FP64 residual) and agrees with per-column mixed solves."""
    torch, B = _setup()
    w = W.nested_k10(24, 4, 10.0)
    op = B.Operator.from_workload(w)
    b = op.plane_wave_rhs(W.fibonacci_dirs(8)).contiguous()
    x, infos = op.solve_batched(b, mode=32, tol=1e-8, max_iters=1000)
    for c in range(8):
        assert infos[c].rel_residual <= 1e-8
    # residuals re-measured with the FP64 multi-RHS and single-column applies
    r64 = b - op.apply_batched(x, precision=64)
    r1 = b[3] - op.apply(x[3], precision=64)
    for c in range(8):
        assert float(torch.linalg.norm(r64[c]) / torch.linalg.norm(b[c])) <= 1.5e-8
    assert float(torch.linalg.norm(r1) / torch.linalg.norm(b[3])) <= 1.5e-8
    for c in (0, 7):
        xs, _ = op.solve(b[c].contiguous(), mode=32, tol=1e-8)
        assert float(torch.linalg.norm(x[c] - xs) / torch.linalg.norm(xs)) <= 1e-6
