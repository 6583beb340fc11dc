"""Host-only parts of the library, run through the C ABI without a GPU: the least-squares
density-gradient stencil (vsie_lsq_grad_alpha and its adjoint are host code) against the
oracle's independent pseudo-inverse, the adjoint identity, and the error path."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import binding as B
from paper_2607_06429_b300 import build as BUILD
from paper_2607_06429_b300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load_library()


def test_lsq_stencil_matches_oracle_on_the_cpu(lib):
    w = W.nested_perturbed(8, 2, 3.0, lsq=True)
    alpha = w.rho0 / w.rho - 1.0
    g_o, W_o = O.lsq_grad_alpha(w.vert, w.tet, w.tet_domain, alpha)
    g = B.lsq_grad_alpha(w.vert, w.tet, w.tet_domain, alpha)
    assert np.max(np.abs(g - g_o)) <= 1e-12 * np.max(np.abs(g_o))
    d = np.random.default_rng(2).normal(size=(w.n_tet, 3))
    a_t = B.lsq_grad_alpha_adjoint(w.vert, w.tet, w.tet_domain, d)
    assert np.max(np.abs(a_t - W_o.T @ d.reshape(-1))) <= 1e-12 * np.max(np.abs(a_t))
    # <W a, d> = <a, W^T d> through the library alone
    a = np.random.default_rng(3).normal(size=w.n_tet)
    lhs = float(np.sum(B.lsq_grad_alpha(w.vert, w.tet, w.tet_domain, a) * d))
    rhs = float(np.dot(a, a_t))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_lsq_stencil_rejects_bad_vertex_index(lib):
    w = W.nested_perturbed(4, 1, 3.0, lsq=True)
    tet = w.tet.copy()
    tet[3, 2] = w.vert.shape[0]
    with pytest.raises(B.VsieError) as e:
        B.lsq_grad_alpha(w.vert, tet, w.tet_domain, np.zeros(w.n_tet))
    assert e.value.status == 2
