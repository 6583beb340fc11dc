"""Pins of the oracle's centroid-far / four-point-near volume rule (``tet_far_points == 1``
with a near radius), the rule of the nested k0 = 10, k0 = 25 and perturbed k0 = 6
workloads.

The reading (Sec. 2.3.4 gives the midpoint rule; the workloads ask for a four-point rule
within two voxel widths): a tetrahedron whose centroid lies within two voxel widths h of
the collocation point is integrated by the degree-2 four-point rule, every other one by
its centroid with weight |e|; its own collocation point takes the equal-volume-ball
single-layer term and nothing else.  Tetrahedron centroids of the Kuhn-split voxel grid
sit on a lattice of spacing h/4, so the squared centroid distances between volume
collocation points are integer multiples of h^2/16 and the cut lies at (4 + 1/32) h^2,
between the occupied shells 64 h^2/16 (exactly two widths: near) and 66 h^2/16 (far).

Each entry of a row is recomputed here, one scalar at a time with ``cmath``, from the
mesh and material arrays (vertices, tetrahedra, rho, c, grad alpha), with the rule chosen
by that cut, and compared with the oracle's row.  Planted mistakes (a cut inside the 2h
shell, the radius compared with a squared distance, the near rule everywhere or nowhere,
a self pair that also receives the four-point sum) each break the comparison.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import series as S
from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

CUT16 = 64.5        # (4 + 1/32) h^2 in units of h^2/16


def _four_point_bary():
    a = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    b = (5.0 - math.sqrt(5.0)) / 20.0
    return [[a if j == q else b for j in range(4)] for q in range(4)]


def _coef(x, y, s, v, k):
    """-G s + grad_x G . v for one source point with G = e^{ikr}/(4 pi r)."""
    d = [x[0] - y[0], x[1] - y[1], x[2] - y[2]]
    r = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
    if r == 0.0:
        return 0j
    G = cmath.exp(1j * k * r) / (4.0 * math.pi * r)
    dv = d[0] * v[0] + d[1] * v[1] + d[2] * v[2]
    return G * (-s + (1j * k * r - 1.0) * dv / (r * r))


def _volume_entries(w, target, row, cut2):
    """Expected volume columns of one row, element by element.  Returns (values, shell)
    with shell the squared centroid distance in units of h^2/16."""
    k = w.k0
    rho = np.asarray(w.rho, dtype=np.float64)
    c = np.asarray(w.c, dtype=np.float64)
    # single-layer weight beta - k0^2 alpha = k0^2 (rho0/rho) ((c0/c)^2 - 1) (Eqs. alpha, beta)
    sw = k * k * (w.rho0 / rho) * ((w.c0 / c) ** 2 - 1.0)
    ga = np.zeros((w.n_tet, 3)) if w.grad_alpha is None else np.asarray(w.grad_alpha).reshape(-1, 3)
    bary = _four_point_bary()
    vals = np.zeros(w.n_tet, dtype=np.complex128)
    shell = np.zeros(w.n_tet)
    for e in range(w.n_tet):
        P = w.vert[w.tet[e]]
        vol = abs(np.dot(P[1] - P[0], np.cross(P[2] - P[0], P[3] - P[0]))) / 6.0
        cen = P.sum(axis=0) / 4.0
        dc = target - cen
        dist2 = float(dc @ dc)
        shell[e] = dist2 * 16.0 / (w.h * w.h)
        if e == row:
            a = (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
            vals[e] = -sw[e] * O.ball_green_integral(a, k)
        elif dist2 < cut2:
            acc = 0j
            for lam in bary:
                y = lam[0] * P[0] + lam[1] * P[1] + lam[2] * P[2] + lam[3] * P[3]
                acc += _coef(target, y, sw[e] * vol / 4.0, ga[e] * vol / 4.0, k)
            vals[e] = acc
        else:
            vals[e] = _coef(target, cen, sw[e] * vol, ga[e] * vol, k)
    return vals, shell


def _triangle_entries(w, D, target, row):
    """Expected interface columns of one row: the three-point rule with v = -omega n w
    beyond the triangle near radius, omega times the singularity-subtracted integral
    (pinned separately against refined quadrature) within it, 0 on its own centroid."""
    k = w.k0
    om = w.rho0 / np.asarray(w.tri_rho_in) - w.rho0 / np.asarray(w.tri_rho_out)
    vals = np.zeros(w.n_tri, dtype=np.complex128)
    near = np.zeros(w.n_tri, dtype=bool)
    for t in range(w.n_tri):
        P = w.vert[w.tri[t]]
        cr = np.cross(P[1] - P[0], P[2] - P[0])
        area = 0.5 * float(np.linalg.norm(cr))
        nrm = cr / np.linalg.norm(cr)
        cen = P.sum(axis=0) / 3.0
        if row == w.n_tet + t:
            near[t] = True
            continue
        dc = target - cen
        if float(dc @ dc) < w.tri_near_radius ** 2:
            near[t] = True
            vals[t] = om[t] * O.double_layer_near(target, P, nrm, area, k)
            continue
        acc = 0j
        for q in range(3):
            lam = [1.0 / 6.0] * 3
            lam[q] = 2.0 / 3.0
            y = lam[0] * P[0] + lam[1] * P[1] + lam[2] * P[2]
            acc += _coef(target, y, 0.0, -om[t] * (area / 3.0) * nrm, k)
        vals[t] = acc
    return vals, near


@pytest.fixture(scope="module")
def smooth():
    """8^3 grid (h = 1/4), both interfaces, linear alpha in both layers: single layer,
    adjoint double layer and double layer all active on the centroid-far branch."""
    w = W.smooth_density_ball(8, 2, 1)
    assert w.tet_far_points == 1 and w.near_radius > 0
    return w, O.Discretisation.from_workload(w)


def _rows(w):
    cen = w.vert[w.tet].mean(axis=1)
    r = np.linalg.norm(cen, axis=1)
    pick = [int(np.argmin(r)), int(np.argmin(np.abs(r - 0.5))), int(np.argmax(r))]
    pick += [int(i) for i in np.random.default_rng(11).choice(w.n_tet, 3, replace=False)]
    return pick


def _deviation(w, A_rows, rows, cut2):
    dev = 0.0
    shells = []
    for a, i in zip(A_rows, rows):
        vals, shell = _volume_entries(w, w.vert[w.tet[i]].mean(axis=0), i, cut2)
        scale = np.abs(vals).max()
        dev = max(dev, float(np.abs(a[:w.n_tet] - vals).max() / scale))
        shells.append(shell)
    return dev, np.concatenate(shells)


def test_volume_rows_follow_the_two_width_cut(smooth):
    w, D = smooth
    rows = _rows(w)
    A = D.matrix_rows(np.array(rows))
    mass = np.asarray(D.mass)[rows]
    A[np.arange(len(rows)), rows] -= mass
    dev, shells = _deviation(w, A, rows, CUT16 * w.h ** 2 / 16.0)
    assert dev <= 1e-13, dev
    # both sides of the cut are exercised: the exact 2h shell (near) and the next one (far)
    assert np.any(np.isclose(shells, 64.0)) and np.any(np.isclose(shells, 66.0))
    assert not np.any((shells > 64.0 + 1e-9) & (shells < 66.0 - 1e-9))


def test_triangle_targets_and_interface_columns(smooth):
    """Interface collocation points (off the lattice) use the same volume cut; their
    interface columns switch to the near rule within the triangle near radius."""
    w, D = smooth
    tc = w.vert[w.tri].mean(axis=1)
    rows = [w.n_tet + int(t) for t in (0, w.n_tri // 2, w.n_tri - 1)]
    A = D.matrix_rows(np.array(rows))
    A[np.arange(len(rows)), rows] -= np.asarray(D.mass)[rows]
    n_near = 0
    for a, i in zip(A, rows):
        x = tc[i - w.n_tet]
        vals, _ = _volume_entries(w, x, i, CUT16 * w.h ** 2 / 16.0)
        assert np.abs(a[:w.n_tet] - vals).max() <= 1e-13 * np.abs(vals).max()
        tv, near = _triangle_entries(w, D, x, i)
        assert np.abs(a[w.n_tet:] - tv).max() <= 1e-13 * np.abs(tv).max()
        assert a[i] == 0.0                      # flat triangle on its own centroid
        n_near += int(near.sum())
    assert n_near > 3 * 3                       # the near triangle rule is exercised


@pytest.mark.parametrize("mistake", ["cut_inside_2h_shell", "radius_not_squared", "near_everywhere",
                                     "near_nowhere", "self_plus_four_point"])
def test_planted_cut_mistakes_are_caught(smooth, mistake):
    """Rows of an oracle carrying one plausible mistake deviate from the hand-built rows."""
    w, D = smooth
    rows = _rows(w)
    h = w.h
    radius = {"cut_inside_2h_shell": h * math.sqrt(4.0 - 1.0 / 32.0),
              # comparing the distance (not its square) with R^2 = a cut at sqrt(R)
              "radius_not_squared": math.sqrt(w.near_radius),
              "near_everywhere": 100.0, "near_nowhere": 0.0}.get(mistake, w.near_radius)
    Dm = O.Discretisation(w.vert, w.tet, w.tri, w.rho, w.c, w.grad_alpha, w.tri_rho_in,
                          w.tri_rho_out, w.k0, w.rho0, w.c0, 1, radius, w.tri_near_radius)
    A = Dm.matrix_rows(np.array(rows))
    A[np.arange(len(rows)), rows] -= np.asarray(Dm.mass)[rows]
    if mistake == "self_plus_four_point":
        for j, i in enumerate(rows):
            P = w.vert[w.tet[i]]
            x = P.mean(axis=0)
            vol = O.tet_volumes(P[None])[0]
            A[j, i] += sum(_coef(x, sum(l * P[m] for m, l in enumerate(lam)),
                                 Dm.sdens[i] * vol / 4.0, Dm.grad_alpha[i] * vol / 4.0, w.k0)
                           for lam in _four_point_bary())
    dev, _ = _deviation(w, A, rows, CUT16 * h ** 2 / 16.0)
    assert dev > 1e-6, (mistake, dev)


def test_centroid_far_branch_converges_to_newton_potential():
    """The volume single layer of the centroid-far / four-point-near rule applied to the
    constant 1 (rho = rho0, beta = 1) tends to the closed-form Newton potential of the
    ball as the grid is refined (Eq. vsie with only the V term)."""
    k = 2.0
    c1 = k / math.sqrt(k * k + 1.0)
    errs = []
    for N in (12, 20, 28):
        w = W.nested_sphere(N, 1.0, 0.0, 2, None, k, lambda x, d: np.ones(x.shape[0]),
                            lambda x, d: np.full(x.shape[0], c1), tet_far_points=1)
        D = O.Discretisation.from_workload(w)
        assert D.far_points == 1 and D.near_radius > 2.0 * w.h
        r = np.linalg.norm(D.tet_cen, axis=1)
        rows = np.random.default_rng(5).choice(np.nonzero(r < 0.6)[0], size=60, replace=False)
        p = np.concatenate([np.ones(D.n_tet), np.zeros(D.n_tri)])
        u = -(D.apply_rows(p, rows) - D.mass[rows])
        ref = S.ball_newton_potential(np.linalg.norm(D.targets[rows], axis=1), 1.0, k)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert errs[0] < 0.01 and errs[2] < 0.5 * errs[0], errs


def test_layered_sphere_vs_series_centroid_far_branch():
    """The constant-layer nested ball on the centroid-far / four-point-near rule against the
    layered-sphere series (density jumps on both interfaces)."""
    k, d = 3.0, np.array([1.0, 0.0, 0.0])
    w = W.layered_ball(12, 3, 2, k, R2=0.5, rho1=1.2, c1=0.8, rho2=3.0, c2=0.5, tet_far_points=1)
    D = O.Discretisation.from_workload(w)
    assert D.far_points == 1 and D.near_radius > 0
    x = np.linalg.solve(D.assemble(), D.plane_wave(d))
    r = np.linalg.norm(D.tet_cen, axis=1)
    m = (r < 0.8) & (np.abs(r - 0.5) > 0.15)
    args = (d, k, [1.0, 0.5], [1.2, 3.0], [0.8, 0.5])
    ref_v = S.layered_sphere_field(D.tet_cen[m], *args)
    dirs = W.fibonacci_dirs(32)
    ref_f = S.layered_sphere_far_field(dirs, *args)
    ev = np.linalg.norm(x[:D.n_tet][m] - ref_v) / np.linalg.norm(ref_v)
    ef = np.linalg.norm(D.far_field(x, dirs) - ref_f) / np.linalg.norm(ref_f)
    assert ev < 0.06 and ef < 0.06, (ev, ef)
