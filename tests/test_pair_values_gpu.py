"""Single pair coefficients of the far-field kernels, read through the field entry point:
with p the unit vector of one element, the field at a point X is minus that element's
integral-row entry at X, i.e. one pair (or one element's quadrature points) of the G, K or
F class.  Random pairs with k0 r up to 60, against the oracles, per pair.

Tolerances per pair: FP64 and double-float 1e-12 relative.  FP32: the phase is formed from
FP32 coordinates kappa x (kappa = k0/2pi, in revolutions), so a pair at |kappa x| <= P
carries a phase error up to about 2 pi ulp(P) ~ 2 pi 2^-23 P radians on top of a few ulp
of arithmetic; the bound used is 4 (2 pi 2^-24 (P + 1)) + 2e-6.  The denominator has a
floor of 1e-3 times the element's largest value, for points where the double-layer
cosine (d . n) nearly vanishes."""
import math

import numpy as np
import pytest

from oracle import cuboid_oracle as CO
from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _binding():
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return B


def _pair_err(got, ref):
    floor = 1e-3 * np.max(np.abs(ref), axis=1, keepdims=True)
    return np.abs(got - ref) / (np.abs(ref) + floor)


def _points(centre, rmin, rmax, m, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = np.exp(rng.uniform(math.log(rmin), math.log(rmax), m))
    return centre + d * r[:, None]


def test_pair_values_cell_and_faces():
    """One cell (density 2, speed 0.7) at k0 = 10: its G source point and its six K face
    points, 256 points at 0.005 <= r <= 6 (k0 r up to 60)."""
    torch = _torch()
    B = _binding()
    e = np.array([-0.1, 0.1])
    w = W.CuboidWorkload("one_cell", e, e.copy(), e.copy(), np.full((1, 1, 1), 2.0),
                         np.full((1, 1, 1), 0.7), k0=10.0)
    op = B.Operator.from_cuboid(w)
    D = CO.CuboidDiscretisation.from_workload(w)
    assert op.n == 7
    pts = _points(np.zeros(3), 0.005, 6.0, 256, 1)
    ref = D.scattered_field(np.eye(7), pts).T  # (element, point)
    P = torch.eye(7, dtype=torch.complex128, device="cuda")
    kap = w.k0 / (2 * math.pi)
    tol32 = 4 * (2 * math.pi * 2.0 ** -24 * (kap * 6.2 + 1)) + 2e-6
    for prec, tol in ((64, 1e-12), (48, 1e-12), (32, tol32)):
        got = op.scattered_field(P, pts, precision=prec).cpu().numpy()
        err = _pair_err(got, ref)
        assert err.max() <= tol, (prec, float(err.max()), tol)
    # a point on the cell's own source point: the coincident pair contributes 0
    z = op.scattered_field(P[0], np.zeros((1, 3)), precision=64).cpu().numpy()
    assert z[0] == D.scattered_field(np.eye(7)[0], np.zeros((1, 3)))[0]


def test_pair_values_heterogeneous_volume_class():
    """Tetrahedra with grad(alpha) != 0 (the F class, both weights) of the smooth-density
    ball at k0 = 3, centroid far rule: 64 points beyond the near radii (r up to 8)."""
    torch = _torch()
    B = _binding()
    w = W.smooth_density_ball(8, 2, 1, 3.0)
    op = B.Operator.from_workload(w)
    D = O.Discretisation.from_workload(w)
    assert w.tet_far_points == 1
    cols = np.nonzero(np.any(w.grad_alpha != 0.0, axis=1))[0][:6]
    assert cols.size == 6
    pts = _points(np.zeros(3), 1.0 + w.near_radius + 0.05, 8.0, 64, 2)
    E = np.zeros((cols.size, D.n), dtype=np.complex128)
    E[np.arange(cols.size), cols] = 1.0
    ref = O.scattered_field(D, E.T, pts).T
    kap = w.k0 / (2 * math.pi)
    tol32 = 4 * (2 * math.pi * 2.0 ** -24 * (kap * 8.2 + 1)) + 2e-6
    Ed = torch.from_numpy(E).cuda()
    for prec, tol in ((64, 1e-12), (48, 1e-12), (32, tol32)):
        got = op.scattered_field(Ed, pts, precision=prec).cpu().numpy()
        err = _pair_err(got, ref)
        assert err.max() <= tol, (prec, float(err.max()), tol)
