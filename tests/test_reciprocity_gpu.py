"""Reciprocity p_inf(xhat; d) = p_inf(-d; -xhat) of the library's solves and far fields.
Exact for the density-1 cuboid grid (the discrete system is symmetric up to the diagonal
weights), so there it holds to the solve tolerance; at discretisation level for the
tetrahedral penetrable ball."""
import numpy as np
import pytest

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


def _pinf(op, xhat, d, mode, tol):
    b = op.plane_wave_rhs(d)[0]
    x, info = op.solve(b, mode=mode, tol=tol)
    assert info.rel_residual <= tol
    return op.far_field(x, xhat[None]).cpu().numpy()[0]


def test_reciprocity_cuboid_lippmann_schwinger():
    _torch()
    B = _binding()
    op = B.Operator.from_cuboid(W.sphere_in_cube(15))
    dirs = W.fibonacci_dirs(6)
    for a, b in ((0, 3), (1, 4), (2, 5)):
        f1 = _pinf(op, dirs[a], dirs[b], 64, 1e-12)
        f2 = _pinf(op, -dirs[b], -dirs[a], 64, 1e-12)
        assert abs(f1 - f2) <= 1e-9 * abs(f1), (a, b, f1, f2)


def test_reciprocity_tetrahedral_ball():
    _torch()
    B = _binding()
    op = B.Operator.from_workload(W.single_ball(12, 3, 2.0))
    dirs = W.fibonacci_dirs(6)
    for a, b in ((0, 3), (1, 4), (2, 5)):
        f1 = _pinf(op, dirs[a], dirs[b], 32, 1e-10)
        f2 = _pinf(op, -dirs[b], -dirs[a], 32, 1e-10)
        assert abs(f1 - f2) <= 0.01 * abs(f1), (a, b, f1, f2)
