"""Several frequencies on one mesh (the nested k0 in [6, 12] multi-frequency workload at
mid size): one persistent tensor-core launch per source class for all operators
(vsie_apply_batched_multi) and its CUDA-graph plan, per right-hand side against the FP64
oracle, against the single-operator batched apply, and replayed bit for bit."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu

FREQS = np.linspace(6.0, 12.0, 8)
NDIR = 64


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return torch, B


@pytest.fixture(scope="module")
def multi():
    torch, B = _setup()
    ws = [W.nested_k10(24, 4, float(k)) for k in FREQS]
    ops = [B.Operator.from_workload(w) for w in ws]
    dirs = W.fibonacci_dirs(NDIR)
    xs = [op.plane_wave_rhs(dirs).contiguous() for op in ops]
    ys = B.apply_batched_multi(ops, xs)
    yield ws, ops, xs, ys
    for op in ops:
        op.close()


def test_multi_frequency_matches_oracle_per_rhs(multi):
    ws, ops, xs, ys = multi
    rng = np.random.default_rng(5)
    for p, (w, op) in enumerate(zip(ws, ops)):
        D = O.Discretisation.from_workload(w)
        rows = np.sort(rng.choice(w.n, 8, replace=False))
        M = D.matrix_rows(rows)
        X = xs[p].cpu().numpy()
        Y = ys[p].cpu().numpy()
        for c in (0, NDIR - 1):
            ref = M @ X[c]
            e = float(np.linalg.norm(Y[c, rows] - ref) / np.linalg.norm(ref))
            y32 = op.apply(xs[p][c], precision=32).cpu().numpy()[rows]
            e32 = float(np.linalg.norm(y32 - ref) / np.linalg.norm(ref))
            assert e <= 1e-5, (FREQS[p], c, e)
            assert e <= 3.0 * e32 + 1e-7, (FREQS[p], c, e, e32)


def test_multi_frequency_matches_single_operator_batched(multi):
    torch, B = _setup()
    ws, ops, xs, ys = multi
    for p in (0, 3, 7):
        y1 = ops[p].apply_batched(xs[p])
        # same sums, different split of the work over the CTAs: FP32-accumulation level
        d = float(torch.linalg.norm(y1 - ys[p]) / torch.linalg.norm(y1))
        assert d <= 1e-6, (p, d)


def test_graph_plan_replays_bit_for_bit(multi):
    torch, B = _setup()
    ws, ops, xs, ys = multi
    outs = [torch.full_like(x, float("nan")) for x in xs]
    g = B.BatchedGraph(ops, xs, outs)
    assert g.nodes > 2 * len(ops)
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    g.launch()
    torch.cuda.synchronize()
    for p in range(len(ops)):
        assert torch.equal(outs[p], first[p])
        assert torch.equal(outs[p], ys[p])  # the same launches as the direct multi apply
    g.close()


def test_multi_rejects_operators_of_different_meshes():
    torch, B = _setup()
    a = B.Operator.from_workload(W.nested_k10(12, 2, 6.0))
    b = B.Operator.from_workload(W.nested_k10(14, 2, 6.0))
    x = a.plane_wave_rhs(W.fibonacci_dirs(2)).contiguous()
    xb = b.plane_wave_rhs(W.fibonacci_dirs(2)).contiguous()
    with pytest.raises(B.VsieError) as e:
        B.apply_batched_multi([a, b], [x, xb])
    assert e.value.status == 1
    with pytest.raises(B.VsieError) as e:
        B.apply_batched_multi([a, a], [x, x.clone()])
    assert e.value.status == 1


def test_multi_frequency_full_size_vs_oracle():
    """The batched workload at full size: the 80^3 nested mesh at 8 wavenumbers in [6, 12]
    with 64 Fibonacci plane waves each (512 right-hand sides), all operators in one graph
    plan (one persistent tensor-core launch per source class); the first and last
    direction of every wavenumber against the oracle on seeded rows."""
    torch, B = _setup()
    ws = [W.nested_k10(80, 6, float(k)) for k in FREQS]
    ops = [B.Operator.from_workload(w) for w in ws]
    dirs = W.fibonacci_dirs(NDIR)
    xs = [op.plane_wave_rhs(dirs).contiguous() for op in ops]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    g = B.BatchedGraph(ops, xs, ys)
    for y in ys:
        y.fill_(float("nan"))
    g.launch()
    torch.cuda.synchronize()
    rng = np.random.default_rng(80)
    worst = 0.0
    for p, w in enumerate(ws):
        D = O.Discretisation.from_workload(w)
        rows = np.sort(rng.choice(w.n, 6, replace=False))
        X = xs[p][[0, NDIR - 1]].cpu().numpy().T
        ref = D.apply_rows(X, rows)
        got = ys[p][[0, NDIR - 1]].cpu().numpy()[:, rows].T
        e = float((np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)).max())
        worst = max(worst, e)
        assert e <= 1e-5, (FREQS[p], e)
        del D
    g.close()
    for op in ops:
        op.close()
    assert worst <= 1e-5
