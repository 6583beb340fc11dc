"""Gradient of the far-field misfit through the library (torch.autograd.Function with the
adjoint solve and adjoint apply) against the oracle's adjoint gradient and against central
finite differences of the library's own loss."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    from paper_2607_06429_b300 import autograd as AG
    return torch, AG


def _case():
    w = W.nested_perturbed(8, 2, 3.0)
    dirs = W.fibonacci_dirs(32)
    rng = np.random.default_rng(4)
    t = rng.normal(size=32) + 1j * rng.normal(size=32)
    return w, dirs, t


@pytest.mark.parametrize("mode", [32, 64])
def test_gradient_matches_oracle(mode):
    torch, AG = _setup()
    w, dirs, t = _case()
    L0, grho0, gc0, _ = O.misfit_and_gradient(w, dirs, t, [1.0, 0.0, 0.0])
    rho = torch.tensor(w.rho, dtype=torch.float64, requires_grad=True)
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    L = AG.far_field_misfit(rho, c, w, dirs, t, mode=mode, tol=1e-11)
    L.backward()
    tol = 1e-5 if mode == 32 else 1e-9
    assert abs(L.item() - L0) <= tol * L0
    gc = c.grad.numpy()
    assert np.linalg.norm(gc - gc0) <= tol * np.linalg.norm(gc0), np.linalg.norm(gc - gc0) / np.linalg.norm(gc0)
    assert np.max(np.abs(rho.grad.numpy())) <= 1e-6 * np.max(np.abs(gc0))


def test_gradient_matches_finite_differences():
    torch, AG = _setup()
    w, dirs, t = _case()
    rho = torch.tensor(w.rho, dtype=torch.float64)
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    L = AG.far_field_misfit(rho, c, w, dirs, t, mode=64, tol=1e-13)
    L.backward()
    g = c.grad.numpy()
    rng = np.random.default_rng(7)
    for e in rng.choice(w.n_tet, size=4, replace=False):
        h = 1e-6 * w.c[e]
        cp, cm = c.detach().clone(), c.detach().clone()
        cp[e] += h
        cm[e] -= h
        Lp = AG.far_field_misfit(rho, cp, w, dirs, t, mode=64, tol=1e-13).item()
        Lm = AG.far_field_misfit(rho, cm, w, dirs, t, mode=64, tol=1e-13).item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * np.max(np.abs(g)), (e, fd, g[e])
