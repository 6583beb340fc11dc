"""The allocation-free apply (vsie_apply_noalloc) against the oracle and the regular apply
(vsie_apply).

vsie_apply_noalloc serves callers that may not allocate device memory after set-up (an
application that owns all device memory through its own pool, or a loop that must not
pay cudaMalloc's implicit synchronisation).  It keeps the source-split partial sums in a
fixed device array instead of a buffer grown on demand.  This file is collected last so
that a failure here never hides the other tests; it passes alone and after them."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {32: 1e-5, 48: 1e-12, 64: 1e-12}


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


def _load_device_code(torch, B):
    """Runs every precision of the call once on a throwaway operator, so that the device
    code the calls use is loaded (with lazy module loading the driver loads a module, and
    reserves device memory for its code, on first use) before free memory is compared."""
    op = B.Operator.from_workload(W.single_ball(4, 1, 2.0))
    x = torch.from_numpy(W.random_vector(op.n, 1)).cuda()
    y = torch.empty_like(x)
    for prec in (32, 48, 64):
        op.apply_noalloc(x, y, precision=prec)
    torch.cuda.synchronize()
    op.close()


@pytest.mark.parametrize("maker", [lambda: W.single_ball(12, 3, 2.0),
                                   lambda: W.smooth_density_ball(8, 2, 1, 3.0)])
def test_noalloc_matches_oracle_and_apply_on_two_calls(maker):
    torch, B = _setup()
    _load_device_code(torch, B)
    w = maker()
    A = O.Discretisation.from_workload(w).assemble()
    op = B.Operator.from_workload(w)   # fresh: the handle's own split buffer does not exist yet
    for prec in (32, 48, 64):
        for call in range(2):  # two calls in a row share (and reuse) the fixed scratch
            x = torch.from_numpy(W.random_vector(op.n, 100 + call)).cuda()
            y = torch.full_like(x, complex(np.nan, np.nan))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            op.apply_noalloc(x, y, precision=prec)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0     # nothing allocated by the call
            got = y.cpu().numpy()
            assert np.all(np.isfinite(got))
            ref = A @ x.cpu().numpy()
            assert _rel(got, ref) <= TOL[prec], (prec, call, _rel(got, ref))
            reg = op.apply(x, precision=prec).cpu().numpy()  # the regular apply after it
            assert _rel(got, reg) <= TOL[prec], (prec, call, _rel(got, reg))


def test_noalloc_two_columns():
    torch, B = _setup()
    w = W.smooth_density_ball(8, 2, 1, 3.0)
    op = B.Operator.from_workload(w)
    X = torch.from_numpy(np.stack([W.random_vector(op.n, s) for s in (7, 8)])).cuda()
    for prec in (32, 48):
        Y = torch.full_like(X, complex(np.nan, np.nan))
        op.apply_noalloc(X, Y, precision=prec)
        ref = op.apply(X, precision=prec)
        for c in range(2):
            assert _rel(Y[c].cpu().numpy(), ref[c].cpu().numpy()) <= TOL[prec]


def test_noalloc_rejects_a_launch_shape_beyond_its_scratch():
    """A launch shape whose source-split partial sums exceed the fixed array (forced here by
    a grid override of 4,096 blocks on a mesh with more work items than that) is rejected
    with VSIE_ERR_ARG before any device work; y stays untouched and vsie_apply still works."""
    torch, B = _setup()
    w = W.nested_k10(24, 4, 10.0)
    op = B.Operator.from_workload(w, tile_override=4096)
    x = torch.from_numpy(W.random_vector(op.n, 3)).cuda()
    y = torch.full_like(x, complex(np.nan, np.nan))
    with pytest.raises(B.VsieError) as e:
        op.apply_noalloc(x, y, precision=32)
    assert e.value.status == 1 and "scratch" in str(e.value)
    assert torch.isnan(y.real).all()
    assert torch.isfinite(op.apply(x, precision=32).real).all()
