"""Pins of the cuboid-grid oracle (the paper's own discretisation, Sec. 2.3.4) to things
other than itself: the face bookkeeping written out by hand for a one-cell inclusion, the
symmetry that the midpoint rule gives the Lippmann-Schwinger case, the sphere benchmark of
Sec. 3 against the Mie series with its second-order mesh convergence, and the
tetrahedral oracle on the same cube (two discretisations of one continuous problem)."""
import math

import numpy as np

from oracle import cuboid_oracle as CO
from oracle import series as S
from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W


def test_face_bookkeeping_of_a_single_inclusion():
    """3 x 3 x 3 unit cells with density 2 in the centre cell only: exactly its six faces
    are interfaces, in the order x (a = 1, 2), y, z; omega = alpha_in - alpha_out and the
    mean mass function, by hand."""
    e = np.array([0.0, 1.0, 2.0, 3.0])
    rho = np.ones((3, 3, 3))
    rho[1, 1, 1] = 2.0
    D = CO.CuboidDiscretisation(e, e, e, rho, np.ones((3, 3, 3)), k0=1.0)
    assert D.n_cell == 27 and D.n_face == 6 and D.n == 33
    want_cen = [(1.0, 1.5, 1.5), (2.0, 1.5, 1.5), (1.5, 1.0, 1.5), (1.5, 2.0, 1.5),
                (1.5, 1.5, 1.0), (1.5, 1.5, 2.0)]
    assert np.array_equal(D.face_cen, np.array(want_cen))
    assert np.array_equal(D.face_nrm, np.repeat(np.eye(3), 2, axis=0))
    assert np.array_equal(D.face_area, np.ones(6))
    # below the first face of each axis: density 1 (alpha 0), above: 2 (alpha -1/2)
    assert np.array_equal(D.face_omega, np.array([0.5, -0.5] * 3))
    assert np.array_equal(D.mass[27:], np.full(6, 0.75))
    assert D.mass[(1 * 3 + 1) * 3 + 1] == 0.5 and D.mass[0] == 1.0
    # the centre cell is (1, 1, 1) at index 13
    assert np.array_equal(D.cell_cen[13], np.array([1.5, 1.5, 1.5]))
    # a grid whose boundary cells differ from the exterior gets boundary faces too
    D2 = CO.CuboidDiscretisation(e[:2], e[:2], e[:2], np.full((1, 1, 1), 3.0), np.ones((1, 1, 1)), k0=1.0)
    assert D2.n_face == 6
    assert np.allclose(D2.face_omega, [1.0 - 1.0 / 3.0, 1.0 / 3.0 - 1.0] * 3)


def test_lippmann_schwinger_symmetry():
    """Density 1 everywhere: no faces, and off the diagonal A_ij = -G(x_i, x_j) s_j V_j,
    so A_ij / (s_j V_j) is symmetric (a weight taken from the wrong index breaks it); the
    diagonal is m - s S(a) with S the ball integral, S(a) -> a^2/2 + i k a^3/3 as k a -> 0."""
    w = W.random_cuboids((4, 3, 5), seed=3, k0=2.0)
    w.rho[:] = 1.0
    D = CO.CuboidDiscretisation.from_workload(w)
    assert D.n_face == 0
    A = D.assemble()
    sv = D.sdens * D.cell_vol
    B = (A - np.diag(np.diag(A))) / sv[None, :]
    assert np.allclose(B, B.T, rtol=1e-13, atol=1e-15)
    r = np.linalg.norm(D.cell_cen[0] - D.cell_cen[1])
    assert abs(B[0, 1] + np.exp(1j * w.k0 * r) / (4 * math.pi * r)) < 1e-14
    # the diagonal, at a tiny wavenumber, against the static ball integral a^2/2
    D0 = CO.CuboidDiscretisation(w.x_edges, w.y_edges, w.z_edges, w.rho, w.c * 1e6, k0=1e-4)
    diag = np.array([D0.matrix_rows([i])[0, i] for i in range(3)])
    self_term = (diag - D0.mass[:3]) / (-D0.sdens[:3])  # the ball integral S(a_e)
    a = D0.a_eq[:3]
    # the ball integral of e^{ikr}/(4 pi r) = a^2/2 + i k a^3/3 + O(k^2 a^4)
    assert np.allclose(self_term, a ** 2 / 2.0 + 1j * 1e-4 * a ** 3 / 3.0, rtol=1e-5)
    assert np.allclose(D0.a_eq ** 3 * 4.0 * math.pi / 3.0, D0.cell_vol, rtol=1e-14)


def _sphere_error(N):
    w = W.sphere_in_cube(N)
    D = CO.CuboidDiscretisation.from_workload(w)
    d = np.array([1.0, 0.0, 0.0])
    p = np.linalg.solve(D.assemble(), D.plane_wave(d))
    sl = np.abs(D.cell_cen[:, 2]) < 1e-12  # the z = 0 slice of cell centres (N odd)
    ref = S.layered_sphere_field(D.cell_cen[sl], d, w.k0, [2.5], [1.0], [5.0 / 6.0])
    return (np.linalg.norm(p[sl] - ref) / np.linalg.norm(ref),
            np.max(np.abs(p[sl] - ref)) / np.max(np.abs(ref)))


def test_sphere_benchmark_against_mie_with_second_order_convergence():
    """Sec. 3 sphere benchmark (r = 2.5 in [-3, 3]^3, c2 = 5/6, lambda0 = 2) on coarse grids
    (3.6 and 4.7 cells per interior wavelength): relative slice errors against the Mie
    series at the staircase level, decreasing at about second order in N."""
    e13 = _sphere_error(13)
    e17 = _sphere_error(17)
    assert e13[0] < 0.13 and e17[0] < 0.08 and e17[1] < 0.07
    order = math.log(e13[0] / e17[0]) / math.log(17.0 / 13.0)
    assert 1.5 < order < 2.5, order


def test_density_jump_cube_against_the_tetrahedral_oracle():
    """A cube with density 2 and speed 0.8 (interfaces on all six sides): the scattered
    field at radius 3 from the cuboid discretisation approaches that of the tetrahedral
    one (four-point rule, singularity-subtracted triangles) as the grid is refined; with
    the interface weight's sign flipped it is off by O(1)."""
    d = np.array([0.3, 0.4, math.sqrt(0.75)])
    pts = 3.0 * W.fibonacci_dirs(32)
    wt = W.cube_tets(6, 1.0, 2.0, 0.8, 2.0)
    T = O.Discretisation.from_workload(wt)
    ref = O.scattered_field(T, np.linalg.solve(T.assemble(), T.plane_wave(d)), pts)
    errs = []
    for N in (6, 12):
        e = np.linspace(-1.0, 1.0, N + 1)
        C = CO.CuboidDiscretisation(e, e, e, np.full((N,) * 3, 2.0), np.full((N,) * 3, 0.8), 2.0)
        p = np.linalg.solve(C.assemble(), C.plane_wave(d))
        errs.append(np.linalg.norm(C.scattered_field(p, pts) - ref) / np.linalg.norm(ref))
        if N == 6:
            C.face_omega = -C.face_omega
            pf = np.linalg.solve(C.assemble(), C.plane_wave(d))
            assert np.linalg.norm(C.scattered_field(pf, pts) - ref) / np.linalg.norm(ref) > 1.0
    assert errs[1] < 0.06 and errs[1] < 0.7 * errs[0], errs


def test_far_field_is_the_large_radius_limit_of_the_exterior_field():
    """R e^{-ik0 R} p_s(R xhat) -> p_inf(xhat) with an O(k0 |y|^2 / R) error, for a grid with
    interface faces of every orientation (both sums of the far-field formula)."""
    w = W.random_cuboids((4, 5, 3), seed=4, k0=2.5)
    D = CO.CuboidDiscretisation.from_workload(w)
    assert D.n_face > 20
    p = W.random_vector(D.n, 3)
    xhat = W.fibonacci_dirs(16)
    R = 1.0e5
    lim = D.scattered_field(p, R * xhat) * R * np.exp(-1j * w.k0 * R)
    pinf = D.far_field(p, xhat)
    assert np.linalg.norm(lim - pinf) / np.linalg.norm(pinf) < 1e-4
    # each part on its own (cells only, faces only)
    for sl in (slice(0, D.n_cell), slice(D.n_cell, D.n)):
        q = np.zeros_like(p)
        q[sl] = p[sl]
        lim = D.scattered_field(q, R * xhat) * R * np.exp(-1j * w.k0 * R)
        assert np.linalg.norm(lim - D.far_field(q, xhat)) / np.linalg.norm(D.far_field(q, xhat)) < 1e-4


def test_reciprocity_exact_for_the_lippmann_schwinger_grid():
    """Reciprocity p_inf(xhat; d) = p_inf(-d; -xhat).  With density 1 the cuboid system is
    A = m - G S with G symmetric (midpoint rule, centroid collocation, symmetric self terms)
    and S = diag(s V) also the far-field weights, so the discrete far field
    u(-xhat)^T S A^{-1} u(d) / 4pi is reciprocal exactly (push-through identity), to
    rounding (density jumps add the unsymmetric face terms: discretisation level only)."""
    w = W.random_cuboids((5, 4, 6), seed=7, k0=2.0)
    w.rho[:] = 1.0
    D = CO.CuboidDiscretisation.from_workload(w)
    A = D.assemble()
    dirs = W.fibonacci_dirs(6)

    def pinf(xhat, d):
        p = np.linalg.solve(A, D.plane_wave(d))
        return D.far_field(p, xhat[None])[0]

    for a in range(3):
        for b in range(3, 6):
            f1, f2 = pinf(dirs[a], dirs[b]), pinf(-dirs[b], -dirs[a])
            assert abs(f1 - f2) <= 1e-11 * abs(f1), (a, b, f1, f2)
    # the sign of the far-field phase matters: with the exponent's sign flipped the
    # identity fails
    xh, d = dirs[0], dirs[4]
    p = np.linalg.solve(A, D.plane_wave(d))
    wrong = np.sum(np.exp(+1j * w.k0 * (D.cell_cen @ xh)) * D.sdens * D.cell_vol * p[:D.n_cell]) / (4 * math.pi)
    assert abs(wrong - pinf(-d, -xh)) > 1e-3 * abs(pinf(-d, -xh))


def test_reciprocity_of_the_tetrahedral_penetrable_ball(ball12_lu):
    """The tetrahedral discretisation (collocation at centroids, four-point sources) is not
    symmetric, so reciprocity holds at discretisation level: within 1% for the 12^3 ball
    over 9 direction pairs (0.26% measured)."""
    w, D, fac = ball12_lu
    dirs = W.fibonacci_dirs(6)
    lu = __import__("scipy.linalg", fromlist=["lu_solve"])
    worst = 0.0
    for a in range(3):
        for b in range(3, 6):
            f1 = D.far_field(lu.lu_solve(fac, D.plane_wave(dirs[b])), dirs[a][None])[0]
            f2 = D.far_field(lu.lu_solve(fac, D.plane_wave(-dirs[a])), -dirs[b][None])[0]
            worst = max(worst, abs(f1 - f2) / abs(f1))
    assert worst < 0.01, worst
