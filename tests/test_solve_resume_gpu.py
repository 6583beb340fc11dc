"""Resume and failure statuses of vsie_solve.

Resume (checkpoint/restart of the refinement): a solve stopped at its iteration limit
returns VSIE_ERR_NOT_CONVERGED with x written; handing that x back as the starting iterate
finishes the solve to the same tolerance, and a converged x is accepted after one
residual evaluation with no iterations.  A non-finite right-hand side returns
VSIE_ERR_NAN."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("mode", [32, 64])
def test_resume_from_a_stopped_solve(mode):
    torch = _torch()
    B = _binding()
    w = W.layered_ball(10, 2, 2, 5.0)
    op = B.Operator.from_workload(w)
    D = O.Discretisation.from_workload(w)
    b = op.plane_wave_rhs([1.0, 0.0, 0.0])[0]
    x_part, info = op.solve(b, mode=mode, tol=1e-10, max_iters=6, raise_on_fail=False)
    assert info.status == 5 and info.iterations == 6 and info.rel_residual > 1e-6
    x_saved = x_part.cpu()                               # the checkpoint
    x, info2 = op.solve(b, mode=mode, tol=1e-10, x0=x_saved.to("cuda"))
    assert info2.status == 0 and info2.rel_residual <= 1e-10
    A = D.assemble()
    bh = b.cpu().numpy()
    res = np.linalg.norm(bh - A @ x.cpu().numpy()) / np.linalg.norm(bh)
    assert res <= 1.5e-10, res
    # x0 is copied, not modified
    assert torch.equal(x_saved, x_part.cpu())
    # a converged iterate: one residual evaluation, no iterations
    x3, info3 = op.solve(b, mode=mode, tol=1e-9, x0=x)
    assert info3.iterations == 0 and info3.fp64_applies == 1 and info3.rel_residual <= 1e-9
    assert torch.equal(x3, x)


def test_solve_failure_statuses():
    torch = _torch()
    B = _binding()
    op = B.Operator.from_workload(W.single_ball(6, 1, 2.0))
    b = op.plane_wave_rhs([0.0, 0.0, 1.0])[0]
    with pytest.raises(B.VsieError) as e:
        op.solve(b, mode=64, tol=1e-12, max_iters=2)
    assert e.value.status == 5
    bad = b.clone()
    bad[3] = complex(float("nan"), 0.0)
    with pytest.raises(B.VsieError) as e:
        op.solve(bad, mode=32)
    assert e.value.status == 7
    # b = 0: x = 0 whatever the starting iterate
    z = torch.zeros_like(b)
    x, info = op.solve(z, mode=32, x0=b)
    assert info.status == 0 and float(x.abs().max()) == 0.0
