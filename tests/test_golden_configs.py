"""The benchmark workloads carry the parameters the paper prints (tests/golden/*.json,
each fixture citing its section): the sphere benchmark grid and the nested-cubes grid,
as generated for both the oracle pins and the GPU reproduction tests."""
import json
import math
import os

import numpy as np

from paper_2607_06429_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_sphere_benchmark_workload_matches_the_paper():
    g = _load("sphere_benchmark.json")
    c2 = g["c2_numerator"] / g["c2_denominator"]
    N = 29
    w = W.sphere_in_cube(N)
    assert np.allclose([w.x_edges[0], w.x_edges[-1]], g["cube"])
    assert np.array_equal(w.x_edges, w.y_edges) and np.array_equal(w.x_edges, w.z_edges)
    assert np.all(w.rho == g["density"]) and w.rho0 == g["density"]
    assert w.c0 == g["c0"]
    assert math.isclose(w.k0, 2 * math.pi / g["lambda0"], rel_tol=1e-15)
    ctr = w.centres()
    inside = np.linalg.norm(ctr, axis=1) < g["sphere_radius"]
    cc = w.c.reshape(-1)
    assert np.all(cc[inside] == c2) and np.all(cc[~inside] == g["c1"])
    assert w.layers["radii"] == [g["sphere_radius"]] and w.layers["c"] == [c2]
    # N = 29 is the grid with 8 cells per interior wavelength
    lam2 = g["lambda0"] * c2 / g["c0"]
    h = (g["cube"][1] - g["cube"][0]) / N
    assert math.floor(lam2 / h) == g["cells_per_interior_wavelength"]
    # N odd: a layer of cell centres lies on the z = 0 slice where the error is measured
    assert np.any(np.abs(ctr[:, 2]) < 1e-12)


def test_nested_cubes_workload_matches_the_paper():
    g = _load("nested_cubes_benchmark.json")
    for h in (1.0, 0.5, 0.25):
        w = W.nested_cubes(h)
        a, b = g["side_outer_mm"] / 2, g["side_inner_mm"] / 2
        e = w.x_edges
        assert math.isclose(e[0], -a) and math.isclose(e[-1], a)
        assert np.any(np.isclose(e, -b)) and np.any(np.isclose(e, b))  # matched interfaces
        assert np.max(np.diff(e)) <= h + 1e-12
        assert w.rho0 == g["rho0"] and w.c0 == g["c0"]
        ctr = w.centres()
        inner = np.max(np.abs(ctr), axis=1) < b
        rr = w.rho.reshape(-1)
        assert np.all(rr[inner] == g["rho2"]) and np.all(rr[~inner] == g["rho1"])
        assert np.allclose(w.c, g["c0"] / g["speed_ratio_c0_over_c"])
        assert math.isclose(w.c.reshape(-1)[0] / g["c0"], g["c1_over_c0"], rel_tol=1e-12)
        assert math.isclose(w.k0, 2 * math.pi / g["lambda0_mm"], rel_tol=1e-15)
        t = W.nested_cube_tets(h)
        tin = t.tet_domain == 2
        assert np.all(t.rho[tin] == g["rho2"]) and np.all(t.rho[~tin] == g["rho1"])
        assert np.all(t.tri_rho_in == g["rho2"]) and np.all(t.tri_rho_out == g["rho1"])
