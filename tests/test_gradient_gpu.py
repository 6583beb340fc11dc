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


# ----------------------------------------------------------------- least-squares density gradient

def _case_lsq():
    w = W.nested_perturbed(8, 2, 3.0, lsq=True)
    dirs = W.fibonacci_dirs(32)
    rng = np.random.default_rng(4)
    t = rng.normal(size=32) + 1j * rng.normal(size=32)
    return w, dirs, t


def test_library_lsq_stencil_matches_oracle():
    torch, AG = _setup()
    from paper_2607_06429_b300 import binding as B
    w = W.nested_perturbed(8, 2, 3.0, lsq=True)
    alpha = w.rho0 / w.rho - 1.0
    g_o, W_o = O.lsq_grad_alpha(w.vert, w.tet, w.tet_domain, alpha)
    g = B.lsq_grad_alpha(w.vert, w.tet, w.tet_domain, alpha)
    assert np.abs(g - g_o).max() <= 1e-12 * np.abs(g_o).max()
    rng = np.random.default_rng(5)
    d = rng.normal(size=(w.n_tet, 3))
    a_t = B.lsq_grad_alpha_adjoint(w.vert, w.tet, w.tet_domain, d)
    assert np.abs(a_t - W_o.T @ d.ravel()).max() <= 1e-12 * np.abs(a_t).max()


@pytest.mark.parametrize("mode", [64, 32])
def test_lsq_density_gradient_matches_oracle(mode):
    """With the least-squares density gradient, dL/drho no longer vanishes; both
    gradients match the oracle's dense adjoint gradient."""
    torch, AG = _setup()
    w, dirs, t = _case_lsq()
    L0, grho0, gc0, _ = O.misfit_and_gradient(w, dirs, t, [1.0, 0.0, 0.0])
    rho = torch.tensor(w.rho, dtype=torch.float64, requires_grad=True)
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    L = AG.far_field_misfit(rho, c, w, dirs, t, mode=mode, tol=1e-11)
    L.backward()
    tol = 1e-5 if mode == 32 else 1e-9
    assert abs(L.item() - L0) <= tol * L0
    for g, g0 in ((rho.grad.numpy(), grho0), (c.grad.numpy(), gc0)):
        assert np.linalg.norm(g - g0) <= tol * np.linalg.norm(g0), np.linalg.norm(g - g0) / np.linalg.norm(g0)
    assert np.abs(grho0).max() > 1e-3 * np.abs(gc0).max()


def test_lsq_density_gradient_matches_finite_differences():
    torch, AG = _setup()
    w, dirs, t = _case_lsq()
    rho = torch.tensor(w.rho, dtype=torch.float64, requires_grad=True)
    c = torch.tensor(w.c, dtype=torch.float64)
    L = AG.far_field_misfit(rho, c, w, dirs, t, mode=64, tol=1e-13)
    L.backward()
    g = rho.grad.numpy()
    rng = np.random.default_rng(9)
    for e in rng.choice(w.n_tet, size=4, replace=False):
        h = 1e-6 * w.rho[e]
        rp, rm = rho.detach().clone(), rho.detach().clone()
        rp[e] += h
        rm[e] -= h
        Lp = AG.far_field_misfit(rp, c, w, dirs, t, mode=64, tol=1e-13).item()
        Lm = AG.far_field_misfit(rm, c, w, dirs, t, mode=64, tol=1e-13).item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * np.abs(g).max() + 1e-6 * abs(g[e]), (e, fd, g[e])
