"""Parity of the CUDA library (through the C ABI) with the FP64 CPU oracle.

Tolerances: relative L2 error <= 1e-5 for the FP32 far-field path and <= 1e-12 for the
FP64 path and the double-float path (precision 48) (full vectors on the small workloads,
seeded sampled rows at full size)."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _op(w, **kw):
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return B.Operator.from_workload(w, **kw)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _cuda(v):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


SMALL = {
    "ball12_k2": lambda: W.single_ball(12, 3, 2.0),
    "smooth8_k3": lambda: W.smooth_density_ball(8, 2, 1, 3.0),
    "layered10_k5": lambda: W.layered_ball(10, 2, 2, 5.0),
}


@pytest.fixture(scope="module", params=sorted(SMALL))
def small_case(request):
    _torch()
    w = SMALL[request.param]()
    D = O.Discretisation.from_workload(w)
    A = D.assemble()
    return request.param, w, D, A


def test_apply_full_vector(small_case):
    name, w, D, A = small_case
    op = _op(w)
    assert op.n == D.n
    x = W.random_vector(D.n, 7)
    ref = A @ x
    xd = _cuda(x)
    y64 = op.apply(xd, precision=64).cpu().numpy()
    y48 = op.apply(xd, precision=48).cpu().numpy()
    y32 = op.apply(xd, precision=32).cpu().numpy()
    assert rel(y64, ref) <= TOL64, (name, rel(y64, ref))
    assert rel(y48, ref) <= TOL64, (name, rel(y48, ref))  # double-float sums
    assert rel(y32, ref) <= TOL32, (name, rel(y32, ref))
    # repeat: deterministic launch configuration gives bitwise-identical results
    y32b = op.apply(xd, precision=32).cpu().numpy()
    assert np.array_equal(y32, y32b)


def test_apply_multi_rhs_and_host_path(small_case):
    name, w, D, A = small_case
    op = _op(w)
    X = np.stack([W.random_vector(D.n, s) for s in (11, 12, 13)])
    ref = X @ A.T
    Y = op.apply(_cuda(X), precision=64).cpu().numpy()
    assert rel(Y, ref) <= TOL64
    Yh = op.apply_host(X, precision=32)
    assert rel(Yh, ref) <= TOL32


def test_adjoint_full_vector(small_case):
    name, w, D, A = small_case
    op = _op(w)
    lam = W.random_vector(D.n, 21)
    ref = A.conj().T @ lam
    x64 = op.adjoint_apply(_cuda(lam), precision=64).cpu().numpy()
    x32 = op.adjoint_apply(_cuda(lam), precision=32).cpu().numpy()
    assert rel(x64, ref) <= TOL64, rel(x64, ref)
    assert rel(x32, ref) <= TOL32, rel(x32, ref)


def test_plane_wave_and_far_field(small_case):
    name, w, D, A = small_case
    op = _op(w)
    dirs = W.fibonacci_dirs(5)
    b = op.plane_wave_rhs(dirs).cpu().numpy()
    for i, d in enumerate(dirs):
        assert rel(b[i], D.plane_wave(d)) <= 1e-13
    p = W.random_vector(D.n, 3)
    ff = op.far_field(_cuda(p), W.fibonacci_dirs(16)).cpu().numpy()
    assert rel(ff, D.far_field(p, W.fibonacci_dirs(16))) <= 1e-12


@pytest.mark.parametrize("mode", [64, 32])
def test_solve_reaches_fp64_residual(small_case, mode):
    name, w, D, A = small_case
    op = _op(w)
    b = D.plane_wave([0.0, 0.0, 1.0])
    x, info = op.solve(_cuda(b), mode=mode, tol=1e-8, max_iters=400)
    x = x.cpu().numpy()
    # residual measured by the oracle
    res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert res <= 1.5e-8, (name, mode, res, info)
    assert info.rel_residual <= 1e-8
    xs = np.linalg.solve(A, b)
    assert rel(x, xs) <= 1e-6
    if mode == 32:
        assert info.fp32_applies > info.fp64_applies


# ----------------------------------------------------------------- sampled rows at size

def _sample_rows(w, count, seed):
    rng = np.random.default_rng(seed)
    n = w.n
    rows = set(rng.choice(n, size=count, replace=False).tolist())
    rows |= {0, n - 1, w.n_tet - 1, w.n_tet}
    g2 = np.nonzero(w.tri_iface == 2)[0]
    if g2.size:
        rows |= {int(w.n_tet + g2[0]), int(w.n_tet + g2[-1])}
    return np.array(sorted(rows))


@pytest.mark.parametrize("maker,count", [(lambda: W.nested_k10(24, 4, 10.0), 96),
                                         (lambda: W.nested_perturbed(20, 3, 6.0), 64)])
def test_apply_sampled_rows_mid_size(maker, count):
    _torch()
    w = maker()
    op = _op(w)
    D = O.Discretisation.from_workload(w)
    rows = _sample_rows(w, count, 3)
    x = W.random_vector(w.n, 5)
    ref = D.apply_rows(x, rows)
    xd = _cuda(x)
    assert rel(op.apply(xd, precision=64).cpu().numpy()[rows], ref) <= TOL64
    assert rel(op.apply(xd, precision=48).cpu().numpy()[rows], ref) <= TOL64
    assert rel(op.apply(xd, precision=32).cpu().numpy()[rows], ref) <= TOL32


def test_apply_sampled_rows_nested80_k10():
    """The full-size nested k0 = 10 workload in the launch configuration the benchmark
    times: FP32 apply vs the oracle on seeded rows (incl. both interfaces)."""
    _torch()
    w = W.nested_k10(80, 6, 10.0)
    op = _op(w)
    D = O.Discretisation.from_workload(w)
    rows = _sample_rows(w, 24, 9)
    x = W.random_vector(w.n, 17)
    y = op.apply(_cuda(x), precision=32).cpu().numpy()
    ref = D.apply_rows(x, rows)
    assert rel(y[rows], ref) <= TOL32, rel(y[rows], ref)


# ----------------------------------------------------------------- edge cases

def test_single_voxel_no_surface():
    _torch()
    vert, tet, h = W.voxel_ball(1, 1.0)  # the single voxel's centre is the origin
    w = W.Workload("voxel", vert, tet, np.zeros((0, 3), np.int32), np.zeros(0, np.int8),
                   np.full(6, 1.3), np.full(6, 0.8), None, np.zeros(0), np.zeros(0), k0=2.0,
                   tet_far_points=1, near_radius=2.0 * h)
    D = O.Discretisation.from_workload(w)
    A = D.assemble()
    op = _op(w)
    x = W.random_vector(6, 1)
    assert rel(op.apply(_cuda(x), precision=64).cpu().numpy(), A @ x) <= TOL64
    assert rel(op.apply(_cuda(x), precision=32).cpu().numpy(), A @ x) <= TOL32


def test_surface_only():
    _torch()
    v, f = W.icosphere(2, 1.0)
    w = W.Workload("shell", v, np.zeros((0, 4), np.int32), f, np.ones(f.shape[0], np.int8),
                   np.zeros(0), np.zeros(0), None, np.full(f.shape[0], 2.0),
                   np.ones(f.shape[0]), k0=3.0, tri_near_radius=0.4)
    D = O.Discretisation.from_workload(w)
    A = D.assemble()
    op = _op(w)
    x = W.random_vector(D.n, 2)
    assert rel(op.apply(_cuda(x), precision=64).cpu().numpy(), A @ x) <= TOL64
    assert rel(op.apply(_cuda(x), precision=32).cpu().numpy(), A @ x) <= TOL32


def test_invalid_mesh_reports_error():
    _torch()
    from paper_2607_06429_b300 import binding as B
    w = W.single_ball(4, 1, 2.0)
    w.tet = w.tet.copy()
    w.tet[3, 2] = w.vert.shape[0] + 5
    with pytest.raises(B.VsieError) as e:
        _op(w)
    assert e.value.status == 2
    w = W.single_ball(4, 1, 2.0)
    w.rho = w.rho.copy()
    w.rho[0] = -1.0
    with pytest.raises(B.VsieError):
        _op(w)


@pytest.mark.parametrize("name,count", [("perturbed40_k6", 24), ("perturbed40_k6_lsq", 16),
                                         ("nested128_k25", 12)])
def test_apply_sampled_rows_full_size(name, count):
    """Full-size workloads (k0 = 6 with per-element contrast, with grad(alpha) = 0 and with
    the least-squares density gradient, which puts every tetrahedron in the heterogeneous
    class; k0 = 25 with 7.25M unknowns and 8.56M far-field source points): FP32 apply vs the
    oracle on seeded rows."""
    _torch()
    w = W.CONFIGS[name]()
    op = _op(w)
    D = O.Discretisation.from_workload(w)
    rows = _sample_rows(w, count, 21)
    x = W.random_vector(w.n, 23)
    xd = _cuda(x)
    y = op.apply(xd, precision=32).cpu().numpy()
    ref = D.apply_rows(x, rows)
    assert rel(y[rows], ref) <= TOL32, rel(y[rows], ref)
    if name.startswith("perturbed40"):  # per-element contrast: the double-float sums at full size
        y48 = op.apply(xd, precision=48).cpu().numpy()
        assert rel(y48[rows], ref) <= TOL64, rel(y48[rows], ref)


# ----------------------------------------------------------------- row ranges

def test_apply_rows_small(small_case):
    """vsie_apply_rows on ragged, empty, single-row and full ranges (volume rows, the
    volume/interface boundary, interface rows) against the oracle's rows, all precisions."""
    name, w, D, A = small_case
    from paper_2607_06429_b300 import binding as B
    op = _op(w)
    x = W.random_vector(D.n, 31)
    ref = A @ x
    xd = _cuda(x)
    nt = w.n_tet
    ranges = [(0, D.n), (0, 1), (D.n - 1, D.n), (5, 5), (3, 700), (max(nt - 37, 0), min(nt + 41, D.n)),
              (nt, D.n)]
    for r0, r1 in ranges:
        for prec, tol in ((64, TOL64), (48, TOL64), (32, TOL32)):
            y = op.apply_rows(xd, r0, r1, precision=prec).cpu().numpy()
            assert y.shape == (r1 - r0,)
            if r1 > r0:
                assert rel(y, ref[r0:r1]) <= tol, (name, r0, r1, prec, rel(y, ref[r0:r1]))
    for r0, r1 in ((-1, 3), (4, 2), (0, D.n + 1)):
        with pytest.raises(B.VsieError) as e:
            op.apply_rows(xd, r0, r1, precision=32)
        assert e.value.status == 1


@pytest.mark.parametrize("name", ["nested80_k10", "nested128_k25"])
def test_apply_rows_fp64_and_double_float_full_size(name):
    """FP64 and double-float parity at full size on contiguous row blocks (volume rows deep
    inside, the volume/interface boundary and the last interface rows), where a full
    FP64 apply would take minutes: each row sums over every far-field source point."""
    _torch()
    w = W.CONFIGS[name]()
    op = _op(w)
    D = O.Discretisation.from_workload(w)
    x = W.random_vector(w.n, 41)
    xd = _cuda(x)
    nt = w.n_tet
    blocks = [(nt // 2, nt // 2 + 24), (nt - 12, nt + 12), (w.n - 16, w.n)]
    for r0, r1 in blocks:
        ref = D.apply_rows(x, np.arange(r0, r1))
        y64 = op.apply_rows(xd, r0, r1, precision=64).cpu().numpy()
        y48 = op.apply_rows(xd, r0, r1, precision=48).cpu().numpy()
        y32 = op.apply_rows(xd, r0, r1, precision=32).cpu().numpy()
        assert rel(y64, ref) <= TOL64, (name, r0, rel(y64, ref))
        assert rel(y48, ref) <= TOL64, (name, r0, rel(y48, ref))
        assert rel(y32, ref) <= TOL32, (name, r0, rel(y32, ref))
