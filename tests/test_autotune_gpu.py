"""Autotuning of the persistent kernels' work shapes (vsie_autotune) on the mid-size nested
k0 = 10 workload: the chosen shapes come from the candidate sets, the chosen shape is never
slower than the built-in default on the tuning sample, and after tuning the single-column
and batched applies still match the FP64 oracle (only the summation order changed)."""
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


def test_autotune_choices_and_parity_after_tuning():
    torch, B = _setup()
    w = W.nested_k10(24, 4, 10.0)
    op = B.Operator.from_workload(w)
    D = O.Discretisation.from_workload(w)
    rows = np.sort(np.random.default_rng(2).choice(w.n, 12, replace=False))
    X = np.stack([W.random_vector(w.n, 300 + r) for r in range(8)])
    Xd = torch.from_numpy(X).cuda()
    y0 = op.apply(Xd[0], precision=32).cpu().numpy()
    yb0 = op.apply_batched(Xd).cpu().numpy()

    rep = op.autotune()
    assert rep["candidates"] >= 2 * 4 + 4
    assert set(rep["far"]) == {"G", "K"}            # no heterogeneous-volume sources here
    for r in rep["far"].values():
        assert r["chunk"] in (512, 1024, 2048, 4096) and r["blocks_per_sm"] >= 1
        assert r["ms"] <= r["default_ms"] * (1 + 1e-6)
    assert rep["batched"]["chunk_tiles"] in (16, 32, 64, 128)
    assert rep["batched"]["ms"] <= rep["batched"]["default_ms"] * (1 + 1e-6)

    y1 = op.apply(Xd[0], precision=32).cpu().numpy()
    yb1 = op.apply_batched(Xd).cpu().numpy()
    assert _rel(y1, y0) <= 1e-6 and _rel(yb1, yb0) <= 1e-6
    M = D.matrix_rows(rows)
    for c in (0, 7):
        ref = M @ X[c]
        assert _rel(yb1[c, rows], ref) <= 1e-5
    assert _rel(y1[rows], M @ X[0]) <= 1e-5
    # the tuned shapes stay deterministic
    assert np.array_equal(op.apply(Xd[0], precision=32).cpu().numpy(), y1)


@pytest.mark.parametrize("split", [(1, 7), (4, 4), (6, 2)])
def test_concurrent_g_and_k_sums_match_sequential_and_oracle(split):
    """The G and K sums on two streams at once (vsie_set_tuning's gk_blocks_per_sm) give the
    sequential result up to the summation order, and the oracle's rows, for any split of the
    resident blocks; a mixed-precision solve through them converges to the same solution."""
    torch, B = _setup()
    w = W.nested_k10(24, 4, 10.0)
    op = B.Operator.from_workload(w)
    D = O.Discretisation.from_workload(w)
    x = W.random_vector(w.n, 41)
    xd = torch.from_numpy(x).cuda()
    y_seq = op.apply(xd, precision=32).cpu().numpy()
    op.set_tuning(gk_blocks_per_sm=split)
    t = op.get_tuning()
    assert t["gk_blocks_per_sm"] == list(split)
    y_con = op.apply(xd, precision=32).cpu().numpy()
    assert _rel(y_con, y_seq) <= 1e-6
    rows = np.sort(np.random.default_rng(5).choice(w.n, 16, replace=False))
    assert _rel(y_con[rows], D.matrix_rows(rows) @ x) <= 1e-5
    assert np.array_equal(op.apply(xd, precision=32).cpu().numpy(), y_con)   # deterministic
    # other precisions do not take the concurrent path
    y64 = op.apply(xd, precision=64).cpu().numpy()
    assert _rel(y64[rows], D.matrix_rows(rows) @ x) <= 1e-11
    b = op.plane_wave_rhs([1.0, 0.0, 0.0])[0].contiguous()
    p_con, info = op.solve(b, mode=32, tol=1e-8)
    op.set_tuning()
    assert op.get_tuning()["gk_blocks_per_sm"] == [0, 0]
    p_seq, _ = op.solve(b, mode=32, tol=1e-8)
    assert _rel(p_con.cpu().numpy(), p_seq.cpu().numpy()) <= 1e-7


def test_concurrent_sums_with_heterogeneous_volume_sources():
    """With the least-squares density gradient the F class follows G on the main stream
    while K runs concurrently; rows against the oracle."""
    torch, B = _setup()
    w = W.nested_perturbed(10, 2, 6.0, lsq=True)
    op = B.Operator.from_workload(w)
    assert op.n_far_sources > 0
    D = O.Discretisation.from_workload(w)
    x = W.random_vector(w.n, 43)
    xd = torch.from_numpy(x).cuda()
    y_seq = op.apply(xd, precision=32).cpu().numpy()
    op.set_tuning(gk_blocks_per_sm=(3, 5))
    y_con = op.apply(xd, precision=32).cpu().numpy()
    assert _rel(y_con, y_seq) <= 1e-6
    rows = np.sort(np.random.default_rng(6).choice(w.n, 24, replace=False))
    assert _rel(y_con[rows], D.matrix_rows(rows) @ x) <= 1e-5


def test_set_tuning_rejects_out_of_range_values_and_keeps_the_shapes():
    torch, B = _setup()
    w = W.nested_k10(16, 3, 10.0)
    op = B.Operator.from_workload(w)
    op.set_tuning(far_chunk=(2048, 1024, 0), far_blocks_per_sm=(6, 4, 0), batch_chunk_tiles=32,
                  gk_blocks_per_sm=(5, 3))
    before = op.get_tuning()
    assert before == {"far_chunk": [2048, 1024, 0], "far_blocks_per_sm": [6, 4, 0],
                      "batch_chunk_tiles": 32, "gk_blocks_per_sm": [5, 3]}
    for bad in (dict(far_chunk=(100, 0, 0)), dict(far_blocks_per_sm=(0, 65, 0)),
                dict(batch_chunk_tiles=-1), dict(gk_blocks_per_sm=(4, 0))):
        with pytest.raises(B.VsieError):
            op.set_tuning(**bad)
        assert op.get_tuning() == before
    x = torch.from_numpy(W.random_vector(w.n, 7)).cuda()
    D = O.Discretisation.from_workload(w)
    rows = np.arange(0, w.n, max(1, w.n // 20))
    y = op.apply(x, precision=32).cpu().numpy()
    assert _rel(y[rows], D.matrix_rows(rows) @ x.cpu().numpy()) <= 1e-5


def test_concurrent_sums_are_captured_in_a_cuda_graph():
    """The fork/join of the concurrent G and K sums (a second stream, two events) records
    into a CUDA graph like any other launch sequence: replays equal the direct apply bit
    for bit, and no allocation happens during capture."""
    torch, B = _setup()
    w = W.nested_k10(16, 3, 10.0)
    op = B.Operator.from_workload(w)
    op.set_tuning(gk_blocks_per_sm=(5, 3))
    x = torch.from_numpy(W.random_vector(w.n, 17)).cuda()
    y = torch.empty_like(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        op.apply(x, y, precision=32)      # warm: every buffer of the path exists
    torch.cuda.synchronize()
    ref = y.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        op.apply(x, y, precision=32)
    y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    x.copy_(torch.from_numpy(W.random_vector(w.n, 18)).cuda())
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, op.apply(x, precision=32))
