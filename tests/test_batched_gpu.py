"""The tensor-core multi-RHS apply (vsie_apply_batched) against the FP64 oracle and against
the per-column FP32 apply.  Tolerance per right-hand side: relative L2 <= 1e-5."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return torch, B


def _block(n, nrhs, seed):
    return np.stack([W.random_vector(n, seed + r) for r in range(nrhs)])


@pytest.mark.parametrize("maker,nrhs", [
    (lambda: W.single_ball(12, 3, 2.0), 3),       # 4-point volume rule, one padded block
    (lambda: W.smooth_density_ball(8, 2, 1, 3.0), 5),  # heterogeneous density (F class too)
    (lambda: W.layered_ball(10, 2, 2, 5.0), 70),  # two blocks of 64 columns, ragged tail
])
def test_batched_matches_oracle(maker, nrhs):
    torch, B = _setup()
    w = maker()
    D = O.Discretisation.from_workload(w)
    A = D.assemble()
    op = B.Operator.from_workload(w)
    X = _block(D.n, nrhs, 40)
    ref = X @ A.T
    Y = op.apply_batched(torch.from_numpy(X).cuda()).cpu().numpy()
    errs = [float(np.linalg.norm(Y[r] - ref[r]) / np.linalg.norm(ref[r])) for r in range(nrhs)]
    assert max(errs) <= TOL, max(errs)
    # the tensor-core path is as accurate as the per-column FP32 apply (accumulator error
    # compensated), not merely inside the tolerance
    Y32 = op.apply(torch.from_numpy(X[:3]).cuda(), precision=32).cpu().numpy()
    e32 = max(float(np.linalg.norm(Y32[r] - ref[r]) / np.linalg.norm(ref[r])) for r in range(min(3, nrhs)))
    assert max(errs) <= 3.0 * e32 + 1e-7, (max(errs), e32)


def test_batched_matches_per_column_apply_mid_size():
    torch, B = _setup()
    w = W.nested_k10(24, 4, 10.0)
    op = B.Operator.from_workload(w)
    X = torch.from_numpy(_block(op.n, 64, 7)).cuda()
    Y = op.apply_batched(X)
    Yc = op.apply(X, precision=32)
    for r in (0, 17, 63):
        e = float(torch.linalg.norm(Y[r] - Yc[r]) / torch.linalg.norm(Yc[r]))
        assert e <= TOL, (r, e)
    # the same call twice gives identical results (deterministic reduction order)
    assert torch.equal(op.apply_batched(X), Y)


def test_batched_oracle_rows_nested24_k10():
    """Mid-size nested k0 = 10 workload (2,048-source work items, target tiles split over
    CTAs): sampled rows of eight right-hand sides against the oracle, at the accuracy of
    the per-column FP32 apply."""
    torch, B = _setup()
    w = W.nested_k10(24, 4, 10.0)
    op = B.Operator.from_workload(w)
    D = O.Discretisation.from_workload(w)
    rows = np.sort(np.random.default_rng(0).choice(w.n, 16, replace=False))
    X = _block(op.n, 64, 100)
    Xd = torch.from_numpy(X).cuda()
    Y = op.apply_batched(Xd).cpu().numpy()
    ref = D.matrix_rows(rows) @ X[:8].T
    errs = [float(np.linalg.norm(Y[r, rows] - ref[:, r]) / np.linalg.norm(ref[:, r])) for r in range(8)]
    Y32 = op.apply(Xd[:8], precision=32).cpu().numpy()
    e32 = max(float(np.linalg.norm(Y32[r, rows] - ref[:, r]) / np.linalg.norm(ref[:, r])) for r in range(8))
    assert max(errs) <= TOL, max(errs)
    assert max(errs) <= 3.0 * e32 + 1e-7, (max(errs), e32)


def test_expired_wait_reports_error_and_context_survives():
    """Failure path without a fault: the issuing warp withholds its bulk copies, every
    bounded mbarrier wait expires (2 s), the call returns VSIE_ERR_CUDA, and the device
    context keeps working for the next operator."""
    torch, B = _setup()
    import time
    w = W.single_ball(6, 1, 2.0)
    op = B.Operator.from_workload(w, debug_flags=1)
    X = torch.from_numpy(_block(op.n, 2, 1)).cuda()
    t0 = time.time()
    with pytest.raises(B.VsieError) as e:
        op.apply_batched(X)
    assert e.value.status == 3 and "wait expired" in str(e.value)
    assert time.time() - t0 < 60
    op.close()
    good = B.Operator.from_workload(w)
    Y = good.apply_batched(X)
    Yc = good.apply(X, precision=32)
    assert float(torch.linalg.norm(Y - Yc) / torch.linalg.norm(Yc)) <= TOL


def test_batched_16_rhs_at_k25_full_size():
    """The large workload at full size (128^3 grid, 6,594,816 tetrahedra, two ico-7 spheres,
    k0 = 25, 7,250,176 unknowns, 8,560,896 far-field source points) with 16 right-hand
    sides (plane waves) through the tensor-core multi-RHS apply: every column against the
    oracle on seeded rows (volume rows, both interfaces)."""
    torch, B = _setup()
    w = W.nested_k25(128, 7, 25.0)
    op = B.Operator.from_workload(w)
    X = op.plane_wave_rhs(W.fibonacci_dirs(16)).contiguous()
    Y = op.apply_batched(X)
    D = O.Discretisation.from_workload(w)
    rng = np.random.default_rng(128)
    rows = np.sort(np.concatenate([rng.choice(w.n_tet, 3, replace=False),
                                   w.n_tet + rng.choice(w.n_tri, 2, replace=False)]))
    ref = D.apply_rows(X.cpu().numpy().T, rows)                  # (rows, 16)
    got = Y.cpu().numpy()[:, rows].T
    errs = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert errs.max() <= TOL, errs.max()
    op.close()
