"""The paper's own cuboid discretisation (vsie_create_cuboid) through the C ABI: parity
with the cuboid oracle, and the sphere benchmark of Sec. 3 reproduced on the GPU.

Parity: full vectors on small grids (no faces; matched nested cubes; random per-cell
material with jump faces of every orientation), relative L2 <= 1e-12 for the FP64 and
double-float applies, <= 1e-5 for FP32, and the adjoint.  Benchmark: the sphere r = 2.5
in the cube [-3, 3]^3 (c2 = 5/6, lambda0 = 2), solved with the mixed solver at 4, 8 and 16
cells per interior wavelength; relative errors on the z = 0 slice of cell centres against
the Mie series below 3% at 8 cells per wavelength in both norms, and about second-order
convergence in the number of cells per dimension."""
import math

import numpy as np
import pytest

from oracle import cuboid_oracle as CO
from oracle import series as S
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _op(w):
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return B.Operator.from_cuboid(w)


def _cuda(v):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


SMALL = {
    "sphere_cube9": lambda: W.sphere_in_cube(9),
    "nested_cubes_h1": lambda: W.nested_cubes(1.0),
    "random_6x5x7": lambda: W.random_cuboids((6, 5, 7), seed=11),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_cuboid_apply_matches_oracle(name):
    _torch()
    w = SMALL[name]()
    op = _op(w)
    D = CO.CuboidDiscretisation.from_workload(w)
    assert op.n == D.n
    A = D.assemble()
    X = np.stack([W.random_vector(D.n, s) for s in (3, 4)])
    ref = X @ A.T
    Xd = _cuda(X)
    for prec, tol in ((64, TOL64), (48, TOL64), (32, TOL32)):
        got = op.apply(Xd, precision=prec).cpu().numpy()
        assert rel(got, ref) <= tol, (name, prec, rel(got, ref))
    lam = W.random_vector(D.n, 9)
    xa = op.adjoint_apply(_cuda(lam), precision=64).cpu().numpy()
    assert rel(xa, A.conj().T @ lam) <= TOL64
    # the multi-right-hand-side applies (tensor cores; FP64-accurate CUDA cores)
    assert rel(op.apply_batched(Xd, precision=32).cpu().numpy(), ref) <= TOL32
    assert rel(op.apply_batched(Xd, precision=64).cpu().numpy(), ref) <= TOL64


def test_cuboid_face_count_and_exterior_field():
    """Matched nested cubes: the unknowns are the cells plus the 6 x 25 faces of the inner
    cube (rho1 = rho0, so the outer cube has none); the scattered field at exterior points
    (midpoint rule, no near rows on a cuboid handle) against the oracle."""
    _torch()
    w = W.nested_cubes(1.0)
    op = _op(w)
    D = CO.CuboidDiscretisation.from_workload(w)
    assert D.n_face == 150 and op.n == 343 + 150
    x = W.random_vector(D.n, 21)
    pts = 6.0 * W.fibonacci_dirs(20)
    got = op.scattered_field(_cuda(x), pts, precision=64).cpu().numpy()
    assert rel(got, D.scattered_field(x, pts)) <= TOL64


def _slice_error(N):
    from paper_2607_06429_b300 import binding as B  # noqa: F401
    w = W.sphere_in_cube(N)
    op = _op(w)
    d = np.array([1.0, 0.0, 0.0])
    b = op.plane_wave_rhs(d)[0]
    x, info = op.solve(b, mode=32, tol=1e-8)
    assert info.rel_residual <= 1e-8
    p = x.cpu().numpy()
    ctr = w.centres()
    sl = np.abs(ctr[:, 2]) < 1e-12
    ref = S.layered_sphere_field(ctr[sl], d, w.k0, [2.5], [1.0], [5.0 / 6.0])
    e2 = np.linalg.norm(p[sl] - ref) / np.linalg.norm(ref)
    einf = np.max(np.abs(p[sl] - ref)) / np.max(np.abs(ref))
    per_lambda = (5.0 / 3.0) / (6.0 / N)
    print(f"sphere benchmark N={N} ({per_lambda:.2f} cells per interior wavelength, n={op.n}): "
          f"E2={e2:.4e} Einf={einf:.4e} iterations={info.iterations}")
    return e2, einf


def test_sphere_benchmark_reproduction():
    """Sec. 3: below 3% at 8 cells per interior wavelength (N = 29), both norms; second-order
    convergence over N = 15, 29, 57."""
    _torch()
    e15 = _slice_error(15)
    e29 = _slice_error(29)
    e57 = _slice_error(57)
    assert e29[0] < 0.03 and e29[1] < 0.03, e29
    assert e57[0] < e29[0] < e15[0]
    order = math.log(e15[0] / e57[0]) / math.log(57.0 / 15.0)
    print(f"sphere benchmark: observed order {order:.2f} over N = 15..57")
    assert order > 1.5, order


def test_cuboid_far_field_matches_oracle():
    _torch()
    w = W.nested_cubes(1.0)
    op = _op(w)
    D = CO.CuboidDiscretisation.from_workload(w)
    x = W.random_vector(D.n, 13)
    dirs = W.fibonacci_dirs(32)
    got = op.far_field(_cuda(x), dirs).cpu().numpy()
    assert rel(got, D.far_field(x, dirs)) <= TOL64


def _far_pattern(op, d, dirs):
    b = op.plane_wave_rhs(d)[0]
    x, info = op.solve(b, mode=32, tol=1e-8)
    assert info.rel_residual <= 1e-8
    return op.far_field(x, dirs).cpu().numpy(), info.iterations


def test_nested_cubes_two_discretisations_converge():
    """Sec. 3 density benchmark (cubes of 7 and 5 mm, rho2 = rho0/2, c1 = c2 = c0/1.2,
    lambda0 = 3 mm), where the paper compares with a BEM: here the cuboid discretisation
    against the tetrahedral one (Kuhn tetrahedra, near rules, triangle interfaces) on
    matched grids of spacing h.  Their far-field patterns (64 directions) approach each
    other as h shrinks."""
    from paper_2607_06429_b300 import binding as B
    _torch()
    d = np.array([1.0, 0.0, 0.0])
    dirs = W.fibonacci_dirs(64)
    diffs = {}
    for h in (1.0, 0.5, 0.25):
        fc, itc = _far_pattern(_op(W.nested_cubes(h)), d, dirs)
        ft, itt = _far_pattern(B.Operator.from_workload(W.nested_cube_tets(h)), d, dirs)
        diffs[h] = rel(fc, ft)
        print(f"nested cubes h={h} mm: cuboid vs tetrahedral far field {diffs[h]:.4e} "
              f"(iterations {itc} / {itt})")
    fc2, _ = _far_pattern(_op(W.nested_cubes(0.125)), d, dirs)
    fc1, _ = _far_pattern(_op(W.nested_cubes(0.25)), d, dirs)
    print(f"nested cubes: cuboid h=0.25 vs h=0.125 far field {rel(fc1, fc2):.4e}")
    assert diffs[0.25] < diffs[0.5] < diffs[1.0]
    assert diffs[0.25] < 0.08


def test_cuboid_gradient_channels_match_oracle():
    """The gradient channels at the cuboid handle's source points (cell centres, then face
    centres) against the oracle's channel sums over the cuboid collocation points."""
    from oracle import vsie_oracle as O
    _torch()
    w = W.random_cuboids((4, 5, 3), seed=5)
    op = _op(w)
    D = CO.CuboidDiscretisation.from_workload(w)
    pts, owner, _ = op.source_points()
    assert np.array_equal(np.sort(owner), np.arange(D.n))
    lam = W.random_vector(D.n, 17)
    for prec, tol in ((64, TOL64), (32, TOL32)):
        phi, psi = op.gradient_channels(_cuda(lam), precision=prec)
        rphi, rpsi = O.gradient_channels(D, lam, pts)
        assert rel(phi.cpu().numpy(), rphi) <= tol
        assert rel(psi.cpu().numpy(), rpsi) <= tol


def _oracle_misfit(w, c, dirs, target, d):
    import dataclasses
    D = CO.CuboidDiscretisation.from_workload(dataclasses.replace(w, c=c.reshape(w.shape)))
    p = np.linalg.solve(D.assemble(), D.plane_wave(d))
    return 0.5 * float(np.sum(np.abs(D.far_field(p, dirs) - target) ** 2))


def test_cuboid_sound_speed_gradient_against_oracle_finite_differences():
    """dL/dc of the far-field misfit on a cuboid grid (autograd through the library, FP64
    solves) against central finite differences of the oracle's misfit, on cells with and
    without contrast (s_e = 0 outside the inclusion)."""
    import torch
    from paper_2607_06429_b300 import autograd as AG
    _torch()
    w = W.sphere_in_cube(7, R=2.2)
    w.rho[2:5, 2:5, 2:5] = 1.3           # an interior density block: faces take part
    c0 = w.c.reshape(-1).copy()
    dirs = W.fibonacci_dirs(12)
    d = np.array([0.0, 0.6, 0.8])
    rng = np.random.default_rng(3)
    ct = c0 * (1.0 + 0.05 * rng.standard_normal(c0.shape))
    import dataclasses
    Dt = CO.CuboidDiscretisation.from_workload(dataclasses.replace(w, c=ct.reshape(w.shape)))
    target = Dt.far_field(np.linalg.solve(Dt.assemble(), Dt.plane_wave(d)), dirs)
    c = torch.tensor(c0, dtype=torch.float64, requires_grad=True)
    L = AG.cuboid_far_field_misfit(c, w, dirs, target, direction=d, mode=64, tol=1e-12)
    L.backward()
    grad = c.grad.numpy()
    L_or = _oracle_misfit(w, c0, dirs, target, d)
    assert abs(L.item() - L_or) <= 1e-9 * L_or
    inside = np.nonzero(c0 < 1.0)[0]
    outside = np.nonzero(c0 == 1.0)[0]
    cells = np.concatenate([inside[:4], outside[:4]])
    assert outside.size and inside.size
    for e in cells:
        h = 1e-6 * c0[e]
        cp, cm = c0.copy(), c0.copy()
        cp[e] += h
        cm[e] -= h
        fd = (_oracle_misfit(w, cp, dirs, target, d) - _oracle_misfit(w, cm, dirs, target, d)) / (2 * h)
        assert abs(grad[e] - fd) <= 1e-5 * np.max(np.abs(grad)) + 1e-6 * abs(fd), (e, grad[e], fd)
