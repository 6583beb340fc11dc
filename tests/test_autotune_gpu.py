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
