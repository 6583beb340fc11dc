"""The allocation-free apply (vsie_apply_noalloc) against the regular apply (vsie_apply).

vsie_apply_noalloc serves callers that may not allocate device memory after set-up (an
application that owns all device memory through its own pool, or a loop that must not
pay cudaMalloc's implicit synchronisation).  It keeps the source-split partial sums in a
fixed device array instead of a buffer grown on demand.  This file is collected last so
that a failure here never hides the other tests; it passes alone and after them."""
import numpy as np
import pytest

from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("maker", [lambda: W.single_ball(12, 3, 2.0),
                                   lambda: W.smooth_density_ball(8, 2, 1, 3.0)])
def test_noalloc_matches_apply_on_two_calls(maker):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    w = maker()
    op = B.Operator.from_workload(w)
    for prec, tol in ((32, 1e-5), (64, 1e-12)):
        for call in range(2):  # two calls in a row share (and reuse) the fixed scratch
            x = torch.from_numpy(W.random_vector(op.n, 100 + call)).cuda()
            ref = op.apply(x, precision=prec).cpu().numpy()
            y = torch.full_like(x, complex(np.nan, np.nan))
            op.apply_noalloc(x, y, precision=prec)
            got = y.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert _rel(got, ref) <= tol, (prec, call, _rel(got, ref))
