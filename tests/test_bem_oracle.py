"""Pins of the PMCHWT boundary element oracle (oracle/bem_oracle.py) against facts that do
not come from it: exactness of the quadrature rule, brute-force integration of the
closed-form triangle potentials, the spectrum of the boundary operators on a sphere
(spherical Bessel closed forms), the symmetries of the Galerkin matrices, the
layered-sphere series of the transmission problem (oracle/series.py), and the absence of
scattering when every medium is the same.  Planted mistakes (a sign, a dropped term, a
wrong normal derivative of the incident field, an inverted density) must fail the series
pin.  (Two mistakes are invisible to it by symmetry and are pinned elsewhere: flipping
the sign of the blocks coupling two interfaces flips the inner interface's unknowns and
leaves the exterior field unchanged; and K' = K on a sphere's nearly uniform mesh is
close to K' = K^T, which the transpose tests check exactly.)"""
import functools
import math

import numpy as np
import pytest
from scipy.special import spherical_jn, spherical_yn

from oracle import bem_oracle as BO
from oracle import series
from paper_2607_06429_b300.workloads import fibonacci_dirs, icosphere


def _nested(subdiv, radii, k0, rho, c, **kw):
    return BO.BemDiscretisation.nested([icosphere(sd, R) for sd, R in zip(subdiv, radii)], k0, rho, c, **kw)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_triangle_rule_is_exact_to_degree_2n_minus_2(n):
    lam, w = BO.triangle_rule(n)
    assert abs(w.sum() - 1.0) < 1e-14 and (w > 0).all()
    s, t = lam[:, 1], lam[:, 2]
    for p in range(2 * n - 1):
        for q in range(2 * n - 1 - p):
            exact = 2.0 * math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
            assert abs((w * s ** p * t ** q).sum() - exact) < 1e-14
    # and not to degree 2n - 1: t^(2n-1) is missed
    exact = 2.0 * math.factorial(2 * n - 1) / math.factorial(2 * n + 1)
    assert abs((w * t ** (2 * n - 1)).sum() - exact) > 1e-8


def _subdivided(x, a, b, c, n=40):
    """S0, S1, D0, D1 by a 6x6 collapsed rule on each of n^2 congruent sub-triangles."""
    lam, w = BO.triangle_rule(6)
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
    P, W = [], []
    for i in range(n):
        for j in range(n - i):
            p0 = a + (b - a) * i / n + (c - a) * j / n
            p1 = p0 + (b - a) / n
            p2 = p0 + (c - a) / n
            P.append(lam @ np.stack([p0, p1, p2]))
            W.append(w * area / n ** 2)
            if j < n - i - 1:
                q0 = p1 + (c - a) / n
                P.append(lam @ np.stack([q0, p2, p1]))
                W.append(w * area / n ** 2)
    P, W = np.concatenate(P), np.concatenate(W)
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    h = (x - a) @ nrm
    rho = x - h * nrm
    R = np.linalg.norm(x - P, axis=1)
    return ((W / R).sum(), ((P - rho) * (W / R)[:, None]).sum(0), (W * h / R ** 3).sum(),
            ((P - rho) * (W * h / R ** 3)[:, None]).sum(0))


def _duffy_in_plane(x, a, b, c, n=80):
    """S0, S1 for x in the triangle's plane: the triangle as three signed triangles with
    apex x, each mapped from the unit square by y = x + u (p + v (q - p)) so that the
    Jacobian cancels 1/|y - x|."""
    g, wg = BO.gauss_legendre01(n)
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    S0, S1 = 0.0, np.zeros(3)
    for p, q in ((a, b), (b, c), (c, a)):
        e0, e1 = p - x, q - p
        twoA = np.dot(nrm, np.cross(p - x, q - x))       # signed
        wv = e0[None, :] + g[:, None] * e1[None, :]       # (n, 3)
        L = np.linalg.norm(wv, axis=1)
        S0 += twoA * (wg / L).sum()                       # u-integral of 1 over [0, 1]
        S1 += twoA * 0.5 * ((wg / L)[:, None] * wv).sum(0)   # u-integral of u = 1/2
    return S0, S1


TRI = (np.array([0.1, 0.0, 0.05]), np.array([1.0, 0.2, -0.1]), np.array([0.3, 0.9, 0.2]))


@pytest.mark.parametrize("x", [[0.4, 0.3, 0.8], [2.0, -1.0, 0.3], [0.5, 0.4, 0.2], [0.45, 0.35, 0.1],
                               [1.2, 1.1, 0.3], [-0.3, 0.2, -0.1]])
def test_triangle_potentials_match_subdivided_quadrature(x):
    x = np.array(x)
    got = BO.triangle_potentials(x, *TRI)
    ref = _subdivided(x, *TRI)
    for g, r in zip(got[:4], ref):
        assert np.max(np.abs(np.asarray(g) - np.asarray(r))) <= 1e-9 * max(1e-3, np.max(np.abs(r)))


@pytest.mark.parametrize("bary", [(0.3, 0.3, 0.4), (0.8, 0.1, 0.1), (0.05, 0.05, 0.9), (1.4, -0.2, -0.2),
                                  (-0.5, 0.9, 0.6)])
def test_triangle_potentials_in_plane_match_duffy(bary):
    a, b, c = TRI
    x = bary[0] * a + bary[1] * b + bary[2] * c
    S0, S1, D0, D1, h, rho, n = BO.triangle_potentials(x, a, b, c)
    r0, r1 = _duffy_in_plane(x, a, b, c)
    assert abs(h) < 1e-15
    assert abs(S0 - r0) <= 1e-11 * abs(r0)
    assert np.max(np.abs(S1 - r1)) <= 1e-11 * np.max(np.abs(r1))
    assert np.max(np.abs(D1)) < 1e-14
    if min(bary) < 0:                      # outside the triangle: no solid angle
        assert abs(D0) < 1e-12


def test_linear_potentials_partition_of_unity_and_first_moment():
    a, b, c = TRI
    X = np.array([[0.4, 0.3, 0.8], [0.2, 0.7, -0.4], [1.5, 0.1, 0.1]])
    IV, IK = BO.linear_potentials(X, a, b, c)
    for i, x in enumerate(X):
        S0, S1, D0, D1, h, rho, n = BO.triangle_potentials(x, a, b, c)
        assert abs(IV[i].sum() - S0) < 1e-13 * abs(S0)
        assert abs(IK[i].sum() - D0) < 1e-13 * max(abs(D0), 1e-3)
        # sum_j lambda_j(y) v_j = y: sum_j IV_j v_j = int y/R = S1 + rho S0
        mom = IV[i, 0] * a + IV[i, 1] * b + IV[i, 2] * c
        assert np.max(np.abs(mom - (S1 + rho * S0))) < 1e-12


def _h1(n, z, d=False):
    return spherical_jn(n, z, d) + 1j * spherical_yn(n, z, d)


def _sphere_eigenvalues(n, k, R):
    """V, K (= K'), W on the spherical harmonics of degree n (addition theorem of G):
    V = ik R^2 j_n h_n, K = ik^2 R^2 j_n h_n' + 1/2, W = -ik^3 R^2 j_n' h_n' at kR."""
    z = k * R
    return (1j * k * R ** 2 * spherical_jn(n, z) * _h1(n, z),
            1j * k ** 2 * R ** 2 * spherical_jn(n, z) * _h1(n, z, True) + 0.5,
            -1j * k ** 3 * R ** 2 * spherical_jn(n, z, True) * _h1(n, z, True))


def _sphere_errors(subdiv, k=1.5, R=1.0):
    v, t = icosphere(subdiv, R)
    D = BO.BemDiscretisation([(v, t)], [{"k": k, "rho": 1.0, "sides": {0: -1}}], far_order=3, near_order=3)
    V, K, Kp, W = D.operator_blocks(0, 0, k)
    M = D.S[0].mass()
    z = v[:, 2] / R
    errs = []
    for n, f in enumerate([np.ones(len(v)), z, 1.5 * z ** 2 - 0.5]):
        ev, ek, ew = _sphere_eigenvalues(n, k, R)
        for X, lam in ((V, ev), (K, ek), (Kp, ek), (W, ew)):
            errs.append(_rel(X @ f, lam * (M @ f)))
    return np.array(errs), (V, K, Kp, W)


def test_operators_on_a_sphere_converge_to_the_spherical_harmonic_spectrum():
    e1, _ = _sphere_errors(1)
    e2, (V, K, Kp, W) = _sphere_errors(2)
    assert e2.max() < 0.05
    assert (e1 / e2).min() > 2.5 and np.median(e1 / e2) > 3.5   # second order in the mesh size
    # Galerkin symmetries: V, W complex symmetric, K' = K^T on one surface
    assert np.abs(V - V.T).max() < 1e-13 * np.abs(V).max()
    assert np.abs(W - W.T).max() < 1e-13 * np.abs(W).max()
    assert np.abs(Kp - K.T).max() < 1e-13 * np.abs(K).max()


def test_cross_surface_blocks_are_transposes():
    D = _nested((1, 1), [1.0, 0.5], 3.0, [1.5, 3.0], [0.8, 0.6])
    k1 = D.domains[1]["k"]
    V01, K01, Kp01, W01 = D.operator_blocks(0, 1, k1)
    V10, K10, Kp10, W10 = D.operator_blocks(1, 0, k1)
    for X, Y in ((V01, V10.T), (W01, W10.T), (Kp01, K10.T), (K01, Kp10.T)):
        assert np.abs(X - Y).max() < 1e-13 * np.abs(Y).max()


RADII, RHO, C, K0 = [1.0, 0.5], [1.5, 3.0], [0.8, 0.6], 3.0


def _series_error(D, dirs):
    ref = series.layered_sphere_far_field(dirs, [1, 0, 0], K0, RADII, RHO, C)
    return _rel(D.far_field(D.solve([1, 0, 0]), dirs), ref)


def test_pmchwt_converges_to_the_layered_sphere_series():
    dirs = fibonacci_dirs(32)
    e11 = _series_error(_nested((1, 1), RADII, K0, RHO, C), dirs)
    e21 = _series_error(_nested((2, 1), RADII, K0, RHO, C), dirs)
    assert e11 < 0.2 and e21 < 0.08 and e11 / e21 > 2.0


def test_identical_media_do_not_scatter():
    D = _nested((1, 1), RADII, K0, [1.0, 1.0], [1.0, 1.0])
    y = D.solve([1, 0, 0])
    ff = D.far_field(y, fibonacci_dirs(32))
    ref = series.layered_sphere_far_field(fibonacci_dirs(32), [1, 0, 0], K0, RADII, RHO, C)
    assert np.abs(ff).max() < 0.05 * np.abs(ref).max()
    # and the traces are those of the incident field: u = p_inc at the vertices
    S = D.S[0]
    pinc = np.exp(1j * K0 * S.vert[:, 0])
    assert _rel(y[:S.n_vert], pinc) < 0.15           # k0 h ~ 2 on this coarse mesh


@functools.lru_cache(maxsize=1)
def _base_error():
    return _series_error(_nested((1, 1), RADII, K0, RHO, C), fibonacci_dirs(32))


@pytest.mark.parametrize("mistake", ["w_without_k2_term", "k_sign", "dn_sign_in_rhs", "rho_in_v"])
def test_planted_mistakes_fail_the_series_pin(mistake, monkeypatch):
    dirs = fibonacci_dirs(32)
    D = _nested((1, 1), RADII, K0, RHO, C)
    base = _base_error()
    orig_blocks = BO.BemDiscretisation.operator_blocks

    def blocks(self, m, l, k):
        V, K, Kp, W = orig_blocks(self, m, l, k)
        if mistake == "w_without_k2_term":
            W = W + k ** 2 * _normal_block(self, m, l, k)
        elif mistake == "k_sign":
            K = -K
        return V, K, Kp, W

    def _normal_block(self, m, l, k):
        # the k^2 (n.n') V part of W, rebuilt from V with unit-curl terms removed: take the
        # operator at the same k with curls zeroed
        A, B = self.S[m], self.S[l]
        ca, cb = A.curl, B.curl
        A.curl = np.zeros_like(ca)
        B.curl = np.zeros_like(cb)
        try:
            _, _, _, Wn = orig_blocks(self, m, l, k)
        finally:
            A.curl, B.curl = ca, cb
        return Wn / k ** 2

    monkeypatch.setattr(BO.BemDiscretisation, "operator_blocks", blocks)
    if mistake == "dn_sign_in_rhs":
        orig_rhs = BO.BemDiscretisation.rhs

        def rhs(self, direction, lumped=True):
            b = orig_rhs(self, direction, lumped)
            nv = self.S[0].n_vert
            b[nv:2 * nv] *= -1.0
            return b
        monkeypatch.setattr(BO.BemDiscretisation, "rhs", rhs)
    if mistake == "rho_in_v":
        for dom in D.domains:
            dom["rho"] = 1.0 / dom["rho"] if dom is not D.domains[0] else dom["rho"]
    bad = _series_error(D, dirs)
    assert base < 0.2
    assert bad > 2.0 * base and bad > 0.25


def test_single_interface_converges_to_the_one_layer_series():
    """One penetrable ball (exterior and one layer, no inner interface): the same
    formulation with a single interface against the series with one radius."""
    dirs = fibonacci_dirs(32)
    k0, R, rho, c = 2.0, 1.0, 1.5, 0.8
    ref = series.layered_sphere_far_field(dirs, [1, 0, 0], k0, [R], [rho], [c])
    errs = []
    for sd in (1, 2):
        D = _nested((sd,), [R], k0, [rho], [c])
        assert [d["sides"] for d in D.domains] == [{0: -1}, {0: +1}]
        errs.append(_rel(D.far_field(D.solve([1, 0, 0]), dirs), ref))
    assert errs[1] < 0.04 and errs[0] / errs[1] > 2.5


def test_lumped_mass_is_the_row_sum_of_the_mass_matrix():
    v, t = icosphere(2, 0.7)
    S = BO.Surface(v, t)
    M = S.mass()
    assert np.allclose(M.sum(axis=1), S.lumped_mass(), rtol=1e-14, atol=0)
    assert abs(S.lumped_mass().sum() - S.area.sum()) < 1e-13 * S.area.sum()
    # the area of the inscribed polyhedron approaches the sphere's from below
    assert S.area.sum() < 4 * np.pi * 0.7 ** 2 and S.area.sum() > 0.97 * 4 * np.pi * 0.7 ** 2


@pytest.mark.parametrize("n", [1, 3, 6])
def test_cube_surface_is_a_closed_outward_triangulation(n):
    from collections import Counter
    from paper_2607_06429_b300.workloads import cube_surface
    v, t = cube_surface(n, 2.5)
    assert t.shape == (12 * n * n, 3) and v.shape == (6 * n * n + 2, 3)
    edges = Counter()
    for a, b, c in t:
        for x, y in ((a, b), (b, c), (c, a)):
            edges[(x, y)] += 1
    assert all(k == 1 for k in edges.values()) and all((y, x) in edges for (x, y) in edges)
    S = BO.Surface(v, t)
    assert abs(S.area.sum() - 6 * 5.0 ** 2) < 1e-12
    assert np.all(np.einsum("ij,ij->i", S.nrm, S.cen) > 0)          # outward
    assert len(v) - len(edges) // 2 + len(t) == 2                    # Euler characteristic


def test_near_pairs_are_symmetric_and_contain_every_touching_pair():
    D = _nested((2, 1), RADII, K0, RHO, C)
    S = D.S[0]
    T, Tp = D.near_pairs(0, 0)
    pairs = set(zip(T.tolist(), Tp.tolist()))
    assert all((b, a) in pairs for a, b in pairs)
    touching = {(a, b) for a in range(S.n_tri) for b in range(S.n_tri)
                if set(S.tri[a].tolist()) & set(S.tri[b].tolist())}
    assert touching <= pairs
    d2 = ((S.cen[T] - S.cen[Tp]) ** 2).sum(1)
    far_ok = d2 < D.near_factor ** 2 * np.maximum(S.diam2[T], S.diam2[Tp])
    assert all(far_ok[i] or (T[i], Tp[i]) in touching for i in range(T.size))
    # across the two interfaces (r = 1 and 0.5, closer than two outer diameters here) the
    # pairs found from either side are the same set
    a, b = D.near_pairs(0, 1)
    c, d = D.near_pairs(1, 0)
    assert a.size > 0 and set(zip(a.tolist(), b.tolist())) == set(zip(d.tolist(), c.tolist()))
