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


# ----------------------------------------------------------------- elements without contrast

def test_gradient_covers_elements_without_contrast():
    """Elements with c_e = c0 carry no single-layer weight (s_e = 0); the gradient with
    respect to their sound speed comes from the unit-weight operator, not from a division
    by s_e, and matches the oracle's adjoint gradient there as elsewhere."""
    torch, AG = _setup()
    w, dirs, t = _case()
    w.c = w.c.copy()
    w.c[::5] = w.c0                                  # every fifth element without contrast
    L0, grho0, gc0, _ = O.misfit_and_gradient(w, dirs, t, [1.0, 0.0, 0.0])
    rho = torch.tensor(w.rho, dtype=torch.float64, requires_grad=True)
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    L = AG.far_field_misfit(rho, c, w, dirs, t, mode=64, tol=1e-11)
    L.backward()
    gc = c.grad.numpy()
    assert np.all(np.isfinite(gc))
    assert np.abs(gc0[::5]).max() > 1e-3 * np.abs(gc0).max()        # those elements matter
    assert np.linalg.norm(gc - gc0) <= 1e-9 * np.linalg.norm(gc0)
    assert np.abs(gc[::5] - gc0[::5]).max() <= 1e-9 * np.abs(gc0).max()


# ----------------------------------------------------------------- the k0 = 6 workload at size

def test_gradient_vs_oracle_on_the_largest_dense_mesh():
    """The k0 = 6 perturbed nested workload on a 12^3 grid (n ~ 6,800, the largest the dense
    oracle handles in seconds): mixed-precision autograd gradient against the oracle's
    adjoint gradient."""
    torch, AG = _setup()
    w = W.nested_perturbed(12, 3, 6.0)
    dirs = W.fibonacci_dirs(128)
    rng = np.random.default_rng(12)
    t = rng.normal(size=128) + 1j * rng.normal(size=128)
    L0, _, gc0, _ = O.misfit_and_gradient(w, dirs, t, [1.0, 0.0, 0.0])
    rho = torch.tensor(w.rho, dtype=torch.float64)
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    L = AG.far_field_misfit(rho, c, w, dirs, t, mode=32, tol=1e-11)
    L.backward()
    assert abs(L.item() - L0) <= 1e-6 * L0
    gc = c.grad.numpy()
    assert np.linalg.norm(gc - gc0) <= 1e-5 * np.linalg.norm(gc0), np.linalg.norm(gc - gc0) / np.linalg.norm(gc0)


def test_gradient_vs_central_differences_at_full_size():
    """The differentiation workload at full size (40^3 grid, 201,312 tetrahedra, k0 = 6, 128
    far-field directions, seeded target): the autograd gradient against central finite
    differences (h = 1e-6 relative) on 32 seeded elements.

    L(c +- h c_e e_e) is evaluated exactly without a fresh solve per perturbation: c_e
    enters only column e of A and of the far-field map F, through its single-layer weight
    s_e (Eqs. alpha, beta), so A_+- = A + d_+- u e_e^T with u = dA/ds_e (column e of the
    unit-weight operator of the same mesh, minus its unit mass) and d_+- the change of s_e;
    by the Sherman-Morrison identity p_+- = p - g_+- z with z = A^{-1} u (one batched solve
    for the 32 elements) and g_+- = d_+- p_e / (1 + d_+- z_e), and F_+- p_+- = F p_+- +
    d_+- (p_+-)_e F_u e_e.  The perturbed losses therefore carry only the solve error of z,
    not that of two full solves, which at 2e5 unknowns would swamp a one-element
    difference; their difference is formed from the perturbations (no cancellation)."""
    torch, AG = _setup()
    from paper_2607_06429_b300 import binding as B
    w = W.nested_perturbed(40, 5, 6.0)
    dirs = W.fibonacci_dirs(128)
    rng = np.random.default_rng(40)
    nt = w.n_tet
    t = 0.05 * (rng.normal(size=128) + 1j * rng.normal(size=128))
    rho = torch.tensor(w.rho, dtype=torch.float64)
    c = torch.tensor(w.c, dtype=torch.float64, requires_grad=True)
    L = AG.far_field_misfit(rho, c, w, dirs, t, mode=32, tol=1e-12)
    L.backward()
    g = c.grad.numpy()
    op = B.Operator.from_workload(w)
    b = op.plane_wave_rhs([[1.0, 0.0, 0.0]])[0].contiguous()
    p, _ = op.solve(b, mode=32, tol=1e-12, max_iters=3000, inner_tol=1e-4, max_refinements=30)
    a = op.far_field(p, dirs).cpu().numpy() - t                 # F p - t
    assert abs(0.5 * np.sum(np.abs(a) ** 2) - L.item()) <= 1e-9 * L.item()
    elems = np.sort(rng.choice(nt, size=32, replace=False))
    # unit-weight operator: s = 1 on every tetrahedron, rho = rho0 (unit mass), no jumps
    cu = np.full(nt, w.c0 / np.sqrt(1.0 + 1.0 / w.k0 ** 2))
    U = B.Operator(w.vert, w.tet, w.tri, np.full(nt, w.rho0), cu, np.full(w.n_tri, w.rho0),
                   np.full(w.n_tri, w.rho0), w.k0, w.rho0, w.c0, None, w.tet_far_points,
                   w.near_radius, w.tri_near_radius)
    E = torch.zeros((32, op.n), dtype=torch.complex128, device="cuda")
    E[torch.arange(32), torch.as_tensor(elems)] = 1.0
    Ucols = (U.apply(E, precision=32) - E).contiguous()          # dA/ds_e, one row per element
    fu = U.far_field(E, dirs).cpu().numpy()                      # dF/ds_e
    Z, _ = op.solve_batched(Ucols, mode=32, tol=1e-10, max_iters=1000, restart=500)
    FZ = op.far_field(Z, dirs).cpu().numpy()
    Z = Z.cpu().numpy()
    ph = p.cpu().numpy()

    def s_of(ce, e):
        return w.k0 ** 2 * (w.rho0 / w.rho[e]) * ((w.c0 / ce) ** 2 - 1.0)

    h = 1e-6
    fds = np.empty(32)
    for q, e in enumerate(elems):
        dl = []
        for sg in (1.0, -1.0):
            d = s_of(w.c[e] * (1.0 + sg * h), e) - s_of(w.c[e], e)
            gam = d * ph[e] / (1.0 + d * Z[q, e])
            delta = -gam * FZ[q] + d * (ph[e] - gam * Z[q, e]) * fu[q]   # F_+- p_+- - F p
            dl.append(float(np.real(np.vdot(a, delta))) + 0.5 * float(np.sum(np.abs(delta) ** 2)))
        fds[q] = (dl[0] - dl[1]) / (2.0 * h * w.c[e])
    err = np.abs(fds - g[elems]).max() / np.abs(g[elems]).max()
    assert err <= 1e-5, err
    U.close()
    op.close()
