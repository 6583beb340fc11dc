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


def _face_cases():
    w1 = W.random_cuboids((5, 4, 6), seed=9)
    w2 = W.nested_cubes(1.0)
    w3 = W.sphere_in_cube(7)
    w3.rho = w3.rho.copy()
    w3.rho[1:4, 2:6, 0:3] = 1.7
    return [w1, w2, w3]


def test_cuboid_faces_match_the_oracle_bit_for_bit(lib):
    """The library's face enumeration (the one vsie_create_cuboid uses) against the
    oracle's independent one: count, order, centres, normals, areas, omega and mass."""
    from oracle import cuboid_oracle as CO
    for w in _face_cases():
        D = CO.CuboidDiscretisation.from_workload(w)
        f = B.cuboid_faces(w)
        assert f["centres"].shape[0] == D.n_face
        assert np.array_equal(f["centres"], D.face_cen)
        assert np.array_equal(np.eye(3)[f["axis"]], D.face_nrm)
        assert np.array_equal(f["area"], D.face_area)
        assert np.array_equal(f["omega"], D.face_omega)
        assert np.array_equal(f["mass"], D.mass[D.n_cell:])


def test_cuboid_faces_errors(lib):
    import ctypes
    w = W.random_cuboids((3, 3, 3), seed=1)
    ex = np.ascontiguousarray(w.x_edges)
    rho = np.ascontiguousarray(w.rho.reshape(-1))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    grid = B._CuboidGrid(3, 3, 3, P(ex), P(ex), P(ex))
    n = ctypes.c_int64()
    assert lib.vsie_cuboid_faces(ctypes.byref(grid), P(rho), 1.0, 0, ctypes.byref(n), None, None, None, None,
                                 None) == 0
    assert n.value > 0
    buf = np.empty(3 * n.value)
    # too little room for the arrays given
    assert lib.vsie_cuboid_faces(ctypes.byref(grid), P(rho), 1.0, n.value - 1, ctypes.byref(n), P(buf),
                                 None, None, None, None) == 1
    bad = ex.copy()
    bad[2] = bad[1]
    grid = B._CuboidGrid(3, 3, 3, P(bad), P(ex), P(ex))
    assert lib.vsie_cuboid_faces(ctypes.byref(grid), P(rho), 1.0, 0, ctypes.byref(n), None, None, None, None,
                                 None) == 2
    grid = B._CuboidGrid(3, 3, 3, P(ex), P(ex), P(ex))
    r2 = rho.copy()
    r2[5] = -1.0
    assert lib.vsie_cuboid_faces(ctypes.byref(grid), P(r2), 1.0, 0, ctypes.byref(n), None, None, None, None,
                                 None) == 2
