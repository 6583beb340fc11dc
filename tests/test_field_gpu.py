"""Scattered field at exterior points (Eq. vsie with the mass function 1 outside the
scatterer: p_s(X) = -(integral row at X) p) through the C ABI against the FP64 oracle.

Points: a shell at 1.5-3 scatterer radii (far rule only) and points just outside the
surface (1.01-1.12 radii), inside the near radii of surface triangles and, where the
volume near rule is on, of boundary tetrahedra, so that the near rows built for the field
points are exercised.  Tolerances as for the operator: relative L2 <= 1e-12 for the FP64
and double-float paths, <= 1e-5 for the FP32 far sums."""
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


def _op(w):
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return B.Operator.from_workload(w)


def _cuda(v):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _points(w, m_far, m_near, seed):
    """Seeded exterior points: m_far on the shell 1.5-3 R, m_near at 1.01-1.12 R, with R the
    largest vertex radius (every tetrahedron lies inside the ball of radius R)."""
    R = float(np.max(np.linalg.norm(w.vert, axis=1)))
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(m_far + m_near, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = np.concatenate([rng.uniform(1.5, 3.0, m_far), rng.uniform(1.01, 1.12, m_near)]) * R
    return d * r[:, None]


def _near_count(D, pts):
    """Points within the triangle near radius of some triangle centroid."""
    if D.tri_near_radius <= 0.0 or D.n_tri == 0:
        return 0
    d2 = ((pts[:, None, :] - D.tri_cen[None, :, :]) ** 2).sum(-1)
    return int((d2.min(axis=1) < D.tri_near_radius ** 2).sum())


SMALL = {
    "ball12_k2": lambda: W.single_ball(12, 3, 2.0),
    "smooth8_k3": lambda: W.smooth_density_ball(8, 2, 1, 3.0),
    "layered10_k5": lambda: W.layered_ball(10, 2, 2, 5.0),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_scattered_field_matches_oracle(name):
    _torch()
    w = SMALL[name]()
    op = _op(w)
    D = O.Discretisation.from_workload(w)
    pts = _points(w, 40, 40, 3)
    assert _near_count(D, pts) >= 10  # the near rows take part
    P = np.stack([W.random_vector(D.n, s) for s in (31, 32, 33)])  # (nrhs, n)
    ref = O.scattered_field(D, P.T, pts).T  # (nrhs, m)
    Pd = _cuda(P)
    for prec, tol in ((64, TOL64), (48, TOL64), (32, TOL32)):
        got = op.scattered_field(Pd, pts, precision=prec).cpu().numpy()
        assert got.shape == ref.shape
        assert rel(got, ref) <= tol, (name, prec, rel(got, ref))
    # one column, one point: the (m,) form and a single-target launch
    one = op.scattered_field(Pd[1], pts[-1:], precision=64).cpu().numpy()
    assert one.shape == (1,)
    assert abs(one[0] - ref[1, -1]) <= TOL64 * max(abs(ref[1, -1]), 1e-300) * 10


def test_scattered_field_of_solution_and_far_field_limit():
    """Solve the plane-wave problem, then: the field just outside and far away matches the
    oracle's field of the same solution, and R e^{-ik0 R} p_s(R xhat) approaches the
    library's own far-field pattern (O(k0 |y|^2 / R) apart at R = 1e4)."""
    _torch()
    w = W.single_ball(12, 3, 2.0)
    op = _op(w)
    D = O.Discretisation.from_workload(w)
    d = np.array([0.0, 0.0, 1.0])
    b = op.plane_wave_rhs(d)[0]
    x, info = op.solve(b, mode=64, tol=1e-12)
    assert info.rel_residual <= 1e-12
    p = x.cpu().numpy()
    pts = _points(w, 16, 16, 5)
    ref = O.scattered_field(D, p, pts)
    got = op.scattered_field(x, pts, precision=64).cpu().numpy()
    assert rel(got, ref) <= TOL64
    xhat = W.fibonacci_dirs(24)
    R = 1.0e4
    far = op.scattered_field(x, R * xhat, precision=64).cpu().numpy() * R * np.exp(-1j * w.k0 * R)
    pinf = op.far_field(x, xhat).cpu().numpy()
    assert rel(far, pinf) < 1e-3


def test_scattered_field_mid_size_sampled():
    """nested24_k10 (two interfaces, per-element sound speed): 24 points, half of them just
    outside the outer sphere, in all three precisions."""
    _torch()
    w = W.nested_k10(24, 4, 10.0)
    op = _op(w)
    D = O.Discretisation.from_workload(w)
    pts = _points(w, 12, 12, 7)
    assert _near_count(D, pts) >= 4
    x = W.random_vector(w.n, 41)
    ref = O.scattered_field(D, x, pts)
    xd = _cuda(x)
    for prec, tol in ((64, TOL64), (48, TOL64), (32, TOL32)):
        got = op.scattered_field(xd, pts, precision=prec).cpu().numpy()
        assert rel(got, ref) <= tol, (prec, rel(got, ref))


def test_scattered_field_rejects_bad_arguments():
    from paper_2607_06429_b300 import binding as B
    _torch()
    w = W.single_ball(6, 1, 2.0)
    op = _op(w)
    x = _cuda(W.random_vector(op.n, 1))
    with pytest.raises(B.VsieError) as e:
        op.scattered_field(x, np.zeros((0, 3)))
    assert e.value.status == 1
    with pytest.raises(B.VsieError):
        op.scattered_field(x, np.array([[2.0, 0.0, 0.0]]), precision=16)
    with pytest.raises(B.VsieError):
        op.scattered_field(x, np.array([[np.nan, 0.0, 3.0]]))
