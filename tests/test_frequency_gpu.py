"""vsie_set_frequency: an operator moved to a new k0 equals a fresh create at that k0
(bitwise, same arithmetic) and the oracle at that k0 (relative L2 <= 1e-12 FP64, <= 1e-5
FP32), for the tetrahedral and the cuboid discretisations; a rejected k0 leaves the
operator as it was."""
import dataclasses

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


def _cuda(v):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(v)).to("cuda")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_set_frequency_tetrahedral():
    _torch()
    B = _binding()
    w = W.layered_ball(10, 2, 2, 2.0)
    op = B.Operator.from_workload(w)
    x = W.random_vector(op.n, 5)
    xd = _cuda(x)
    y_before = op.apply(xd, precision=64).cpu().numpy()
    op.set_frequency(4.5)
    w2 = dataclasses.replace(w, k0=4.5)
    fresh = B.Operator.from_workload(w2)
    D = O.Discretisation.from_workload(w2)
    ref = D.apply_rows(x, np.arange(D.n))
    for prec, tol in ((64, 1e-12), (48, 1e-12), (32, 1e-5)):
        got = op.apply(xd, precision=prec).cpu().numpy()
        assert rel(got, ref) <= tol, (prec, rel(got, ref))
        assert np.array_equal(got, fresh.apply(xd, precision=prec).cpu().numpy())
    assert rel(y_before, ref) > 1e-2  # the operator did change
    # back to the first frequency: the first result again, bit for bit
    op.set_frequency(2.0)
    assert np.array_equal(op.apply(xd, precision=64).cpu().numpy(), y_before)
    with pytest.raises(B.VsieError) as e:
        op.set_frequency(-1.0)
    assert e.value.status == 1
    assert np.array_equal(op.apply(xd, precision=64).cpu().numpy(), y_before)


def test_set_frequency_cuboid():
    _torch()
    B = _binding()
    w = W.random_cuboids((5, 6, 4), seed=2, k0=2.0)
    op = B.Operator.from_cuboid(w)
    x = W.random_vector(op.n, 8)
    op.set_frequency(5.0)
    D = CO.CuboidDiscretisation.from_workload(dataclasses.replace(w, k0=5.0))
    ref = D.assemble() @ x
    xd = _cuda(x)
    assert rel(op.apply(xd, precision=64).cpu().numpy(), ref) <= 1e-12
    assert rel(op.apply(xd, precision=32).cpu().numpy(), ref) <= 1e-5
