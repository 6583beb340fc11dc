"""Seeded synthetic workloads for the nested-sphere Helmholtz transmission problem.

This module only *generates inputs*: tetrahedral volume meshes of a voxelised ball
(each kept voxel Kuhn-split into six tetrahedra), icosphere interface meshes, and the
material fields rho(x), c(x) sampled per element.  It contains none of the VSIE
method's arithmetic (no quadrature, no Green's function, no operator weights), so it
can feed both the CUDA library and the FP64 CPU oracle without coupling them.

Geometry follows the nested layout of Sec. 2.1 (Fig. 1): Omega_2 inside Omega_1 inside
the homogeneous exterior Omega_0, interfaces Gamma_1 (outer) and Gamma_2 (inner), every
interface triangle oriented so that its normal points out of the subdomain it encloses.

Mesh conventions handed to the library:
  * ``vert``      float64 (n_vert, 3)
  * ``tet``       int32 (n_tet, 4) vertex indices
  * ``tri``       int32 (n_tri, 3) vertex indices, (b-a)x(c-a) points outward
  * ``tri_iface`` int8 (n_tri,) 1 for Gamma_1, 2 for Gamma_2
Material conventions:
  * ``rho``, ``c``  float64 per tetrahedron
  * ``grad_alpha``  float64 (n_tet, 3) or None (piecewise-constant density)
  * ``tri_rho_in``  density limit on the side the triangle normal points away from
  * ``tri_rho_out`` density limit on the side the normal points into
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    vert: np.ndarray
    tet: np.ndarray
    tri: np.ndarray
    tri_iface: np.ndarray
    rho: np.ndarray
    c: np.ndarray
    grad_alpha: Optional[np.ndarray]
    tri_rho_in: np.ndarray
    tri_rho_out: np.ndarray
    k0: float
    rho0: float = 1.0
    c0: float = 1.0
    tet_far_points: int = 1
    near_radius: float = 0.0
    tri_near_radius: float = 0.0
    h: float = 0.0
    R1: float = 1.0
    R2: float = 0.0
    layers: dict = dataclasses.field(default_factory=dict)
    tet_domain: Optional[np.ndarray] = None  # subdomain (1 outer, 2 inner) of every tetrahedron
    grad_alpha_lsq: bool = False             # grad(alpha) from the least-squares reading (consumers compute it)

    @property
    def n_tet(self) -> int:
        return int(self.tet.shape[0])

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n(self) -> int:
        return self.n_tet + self.n_tri

    def n_far_sources(self) -> int:
        return self.n_tet * self.tet_far_points + 3 * self.n_tri


# ----------------------------------------------------------------------------- meshes

_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def voxel_ball(n_grid: int, R1: float = 1.0):
    """Voxel grid on [-R1, R1]^3 with n_grid cells per axis; a voxel is kept iff its
    centre lies strictly inside the ball |x| < R1.  Each kept voxel is split into the six
    Kuhn tetrahedra sharing its main diagonal.  Returns (vert, tet, h)."""
    N = int(n_grid)
    h = 2.0 * R1 / N
    ctr = -R1 + (np.arange(N) + 0.5) * h
    cx, cy, cz = np.meshgrid(ctr, ctr, ctr, indexing="ij")
    keep = cx * cx + cy * cy + cz * cz < R1 * R1
    vi, vj, vk = (a.astype(np.int64) for a in np.nonzero(keep))
    nv = vi.shape[0]
    M = N + 1

    def node(i, j, k):
        return (i * M + j) * M + k

    unit = np.eye(3, dtype=np.int64)
    tets = np.empty((nv, 6, 4), dtype=np.int64)
    base = np.stack([vi, vj, vk], axis=1)
    for t, perm in enumerate(_KUHN_PERMS):
        p0 = base
        p1 = p0 + unit[perm[0]]
        p2 = p1 + unit[perm[1]]
        p3 = p0 + 1
        for q, pq in enumerate((p0, p1, p2, p3)):
            tets[:, t, q] = node(pq[:, 0], pq[:, 1], pq[:, 2])
    tets = tets.reshape(-1, 4)
    used, inv = np.unique(tets, return_inverse=True)
    tet = inv.reshape(-1, 4).astype(np.int32)
    ii = used // (M * M)
    jj = (used // M) % M
    kk = used % M
    vert = np.stack([-R1 + ii * h, -R1 + jj * h, -R1 + kk * h], axis=1).astype(np.float64)
    return vert, tet, h


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(subdiv: int, radius: float):
    """Icosphere of the given radius: the icosahedron refined ``subdiv`` times by edge
    midpoints projected back to the sphere (20 * 4^subdiv triangles), every triangle
    oriented outward.  Returns (vert, tri)."""
    v, f = _icosahedron()
    for _ in range(int(subdiv)):
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        ue, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[ue[:, 0]] + v[ue[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        nf = f.shape[0]
        mab = inv[:nf] + v.shape[0]
        mbc = inv[nf:2 * nf] + v.shape[0]
        mca = inv[2 * nf:] + v.shape[0]
        v = np.concatenate([v, mid], axis=0)
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate([
            np.stack([a, mab, mca], 1), np.stack([b, mbc, mab], 1),
            np.stack([c, mca, mbc], 1), np.stack([mab, mbc, mca], 1)], axis=0)
    v = v * radius
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    outward = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) > 0
    f[~outward] = f[~outward][:, [0, 2, 1]]
    return v, f.astype(np.int32)


def cube_surface(n: int, half: float):
    """Closed triangulation of the surface of the cube [-half, half]^3: an n x n grid of
    squares on every face, each split into two triangles, vertices shared along the edges,
    every triangle oriented outward.  Returns (vert, tri)."""
    n = int(n)
    idx = -np.ones((n + 1,) * 3, dtype=np.int64)
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    on = (I == 0) | (I == n) | (J == 0) | (J == n) | (K == 0) | (K == n)
    idx[on] = np.arange(int(on.sum()))
    vert = np.stack([I[on], J[on], K[on]], axis=1).astype(np.float64) * (2.0 * half / n) - half
    tris = []
    for axis in range(3):
        for side in (0, n):
            a, b = [d for d in range(3) if d != axis]
            for i in range(n):
                for j in range(n):
                    corner = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        c = [0, 0, 0]
                        c[axis], c[a], c[b] = side, i + di, j + dj
                        corner.append(idx[tuple(c)])
                    tris.append([corner[0], corner[1], corner[2]])
                    tris.append([corner[0], corner[2], corner[3]])
    tri = np.array(tris, dtype=np.int64)
    p0, p1, p2 = vert[tri[:, 0]], vert[tri[:, 1]], vert[tri[:, 2]]
    outward = np.einsum("ij,ij->i", np.cross(p1 - p0, p2 - p0), p0 + p1 + p2) > 0
    tri[~outward] = tri[~outward][:, [0, 2, 1]]
    return vert, tri.astype(np.int32)


def _centroids(vert, idx):
    return vert[idx].mean(axis=1)


# ----------------------------------------------------------------------------- builders

def nested_sphere(n_grid: int, R1: float, R2: float, subdiv1: int, subdiv2: Optional[int],
                  k0: float, rho_fn: Callable, c_fn: Callable,
                  grad_alpha_fn: Optional[Callable] = None,
                  tet_far_points: int = 1, near_factor: float = 2.0,
                  tri_near_factor: float = 2.0,
                  rho0: float = 1.0, c0: float = 1.0, name: str = "nested",
                  layers: Optional[dict] = None) -> Workload:
    """Nested (or, with R2 = 0, single) penetrable ball.

    ``rho_fn(x, dom)`` and ``c_fn(x, dom)`` give the material of subdomain ``dom`` (1 or
    2) at points ``x`` (m, 3); ``grad_alpha_fn(x, dom)`` the gradient of
    alpha = rho0/rho - 1 where the density varies smoothly.  A tetrahedron belongs to
    Omega_2 iff its centroid satisfies |x| < R2.  Targets closer than
    ``tri_near_factor`` times the longest interface edge to a triangle's centroid use the
    accurate near rule for that triangle.
    """
    vert, tet, h = voxel_ball(n_grid, R1)
    cen = _centroids(vert, tet)
    dom = np.where(np.linalg.norm(cen, axis=1) < R2, 2, 1).astype(np.int8)
    rho = np.empty(tet.shape[0])
    c = np.empty(tet.shape[0])
    ga = None if grad_alpha_fn is None else np.zeros((tet.shape[0], 3))
    for d in (1, 2):
        m = dom == d
        if not m.any():
            continue
        rho[m] = rho_fn(cen[m], d)
        c[m] = c_fn(cen[m], d)
        if ga is not None:
            ga[m] = grad_alpha_fn(cen[m], d)

    verts = [vert]
    tris = []
    iface = []
    rin = []
    rout = []
    off = vert.shape[0]
    max_edge = 0.0
    shells = [(1, R1, subdiv1)]
    if R2 > 0 and subdiv2 is not None:
        shells.append((2, R2, subdiv2))
    for g, R, s in shells:
        sv, sf = icosphere(s, R)
        tc = sv[sf].mean(axis=1)
        for q in range(3):
            max_edge = max(max_edge, float(np.max(np.linalg.norm(
                sv[sf[:, q]] - sv[sf[:, (q + 1) % 3]], axis=1))))
        verts.append(sv)
        tris.append(sf + off)
        iface.append(np.full(sf.shape[0], g, dtype=np.int8))
        if g == 1:
            rin.append(rho_fn(tc, 1))
            rout.append(np.full(sf.shape[0], rho0))
        else:
            rin.append(rho_fn(tc, 2))
            rout.append(rho_fn(tc, 1))
        off += sv.shape[0]
    # Near-field cut: "within near_factor voxel widths".  Tetrahedron centroids sit on a
    # lattice of spacing h/4, so squared centroid distances are multiples of h^2/16; the
    # cut is placed halfway between the shell (near_factor*h)^2 and the next one, so
    # rounding of coordinates can never flip an inclusion decision.
    near = 0.0
    if tet_far_points == 1 and near_factor > 0:
        near = h * math.sqrt(near_factor ** 2 + 1.0 / 32.0)
    return Workload(
        name=name, vert=np.concatenate(verts, axis=0).astype(np.float64), tet=tet,
        tri=np.concatenate(tris, axis=0).astype(np.int32),
        tri_iface=np.concatenate(iface), rho=rho, c=c, grad_alpha=ga,
        tri_rho_in=np.concatenate(rin).astype(np.float64),
        tri_rho_out=np.concatenate(rout).astype(np.float64),
        k0=float(k0), rho0=rho0, c0=c0, tet_far_points=int(tet_far_points),
        near_radius=near, tri_near_radius=tri_near_factor * max_edge, h=h, R1=R1, R2=R2, layers=layers or {},
        tet_domain=dom)


def _const(v1, v2=None):
    def f(x, dom):
        return np.full(x.shape[0], v1 if dom == 1 else v2, dtype=np.float64)
    return f


def single_ball(n_grid=12, subdiv=3, k0=2.0, rho1=1.5, c1=0.7) -> Workload:
    """Single penetrable unit ball, homogeneous inside, all tetrahedra on the 4-point rule
    (the small FP64 workload; its exterior/interior field has the Mie series)."""
    return nested_sphere(n_grid, 1.0, 0.0, subdiv, None, k0, _const(rho1), _const(c1),
                         tet_far_points=4, name=f"ball{n_grid}_k{k0:g}",
                         layers=dict(rho1=rho1, c1=c1))


def layered_ball(n_grid, subdiv1, subdiv2, k0, R2=0.5, rho1=1.2, c1=0.8, rho2=3.0, c2=0.5,
                 tet_far_points=1) -> Workload:
    """Nested balls with constant layers (the layered-sphere series applies)."""
    return nested_sphere(n_grid, 1.0, R2, subdiv1, subdiv2, k0, _const(rho1, rho2),
                         _const(c1, c2), tet_far_points=tet_far_points,
                         name=f"layered{n_grid}_k{k0:g}",
                         layers=dict(rho1=rho1, c1=c1, rho2=rho2, c2=c2))


def shell_x0(seed: int = 0, r_in: float = 0.5, r_out: float = 1.0) -> np.ndarray:
    """Seeded point uniform in the spherical shell r_in < |x| < r_out."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    r = (rng.uniform(r_in ** 3, r_out ** 3)) ** (1.0 / 3.0)
    return d * r


def nested_k10(n_grid=80, subdiv=6, k0=10.0, seed=0) -> Workload:
    """Nested spheres r=1 / r=0.5 at k0=10: shell rho=1.2 with a Gaussian sound-speed bump
    c = 0.8 + 0.2 exp(-|x-x0|^2/0.1) (x0 seeded in the shell), core rho=3, c=0.5;
    centroid rule in the far field, 4-point rule within two voxel widths."""
    x0 = shell_x0(seed)

    def rho_fn(x, dom):
        return np.full(x.shape[0], 1.2 if dom == 1 else 3.0)

    def c_fn(x, dom):
        if dom == 2:
            return np.full(x.shape[0], 0.5)
        return 0.8 + 0.2 * np.exp(-np.sum((x - x0) ** 2, axis=1) / 0.1)

    return nested_sphere(n_grid, 1.0, 0.5, subdiv, subdiv, k0, rho_fn, c_fn,
                         tet_far_points=1, name=f"nested{n_grid}_k{k0:g}",
                         layers=dict(rho1=1.2, rho2=3.0, c2=0.5, x0=x0.tolist()))


def nested_k25(n_grid=128, subdiv=7, k0=25.0, seed=0) -> Workload:
    """Nested spheres r=1 / r=0.6 at k0=25 with the layer densities of the k0=10 case and
    a seeded random-phase sound speed c = 1 + 0.3 * mean_m cos(g_m.x + phi_m), |g_m| = k0/2,
    which stays inside [0.7, 1.3]."""
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(8, 3))
    g *= (k0 / 2.0) / np.linalg.norm(g, axis=1, keepdims=True)
    phi = rng.uniform(0, 2 * np.pi, size=8)

    def rho_fn(x, dom):
        return np.full(x.shape[0], 1.2 if dom == 1 else 3.0)

    def c_fn(x, dom):
        return 1.0 + 0.3 * np.mean(np.cos(x @ g.T + phi), axis=1)

    return nested_sphere(n_grid, 1.0, 0.6, subdiv, subdiv, k0, rho_fn, c_fn,
                         tet_far_points=1, name=f"nested{n_grid}_k{k0:g}")


def nested_perturbed(n_grid=40, subdiv=5, k0=6.0, seed=0, sigma=0.05, lsq=False) -> Workload:
    """Nested spheres r=1 / r=0.5 at k0=6 with per-element multiplicative perturbations
    rho_e = rho_layer (1 + d_rho), c_e = c_layer (1 + d_c), d ~ N(0, sigma^2) seeded.
    lsq: grad(alpha) from the least-squares reading over face neighbours (computed by the
    consumers from rho), else element-wise constant density (grad(alpha) = 0)."""
    w = nested_k10(n_grid, subdiv, k0, seed)
    w.grad_alpha_lsq = bool(lsq)
    rng_r = np.random.default_rng(seed)
    rng_c = np.random.default_rng(seed + 1)
    w.rho = w.rho * (1.0 + sigma * rng_r.normal(size=w.n_tet))
    w.c = w.c * (1.0 + sigma * rng_c.normal(size=w.n_tet))
    w.name = f"perturbed{n_grid}_k{k0:g}"
    return w


def smooth_density_ball(n_grid=8, subdiv1=2, subdiv2=1, k0=3.0, R2=0.5) -> Workload:
    """Small nested case with a smooth linear density perturbation in both layers, so that
    all three operator kinds (volume single layer, volume adjoint double layer, interface
    double layer on both interfaces) are active.  alpha = rho0/rho - 1 is linear:
    alpha = a_d + g.x in layer d, with analytic gradient g."""
    g = np.array([0.15, -0.1, 0.05])
    a = {1: -0.2, 2: -0.5}

    def rho_fn(x, dom):
        return 1.0 / (1.0 + a[dom] + x @ g)

    def c_fn(x, dom):
        return np.full(x.shape[0], 0.9 if dom == 1 else 0.7)

    def ga_fn(x, dom):
        return np.tile(g, (x.shape[0], 1))

    return nested_sphere(n_grid, 1.0, R2, subdiv1, subdiv2, k0, rho_fn, c_fn, ga_fn,
                         tet_far_points=1, name=f"smooth{n_grid}_k{k0:g}")


def random_vector(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    """Seeded complex test vector(s), column-major (n, nrhs) when nrhs > 1."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, nrhs)) + 1j * rng.normal(size=(n, nrhs))
    return v[:, 0].copy() if nrhs == 1 else np.asfortranarray(v)


def fibonacci_dirs(m: int) -> np.ndarray:
    """m unit vectors on the golden-angle (Fibonacci) spiral."""
    i = np.arange(m) + 0.5
    z = 1.0 - 2.0 * i / m
    r = np.sqrt(1.0 - z * z)
    th = np.pi * (3.0 - math.sqrt(5.0)) * np.arange(m)
    return np.stack([r * np.cos(th), r * np.sin(th), z], axis=1)


CONFIGS = {
    "ball12_k2": lambda: single_ball(12, 3, 2.0),
    "nested24_k10": lambda: nested_k10(24, 4, 10.0),
    "nested80_k10": lambda: nested_k10(80, 6, 10.0),
    "perturbed40_k6": lambda: nested_perturbed(40, 5, 6.0),
    "perturbed40_k6_lsq": lambda: nested_perturbed(40, 5, 6.0, lsq=True),
    "nested128_k25": lambda: nested_k25(128, 7, 25.0),
}


# ----------------------------------------------------------------------------- cuboid grids

@dataclasses.dataclass
class CuboidWorkload:
    """A nonuniform cuboid grid (the paper's own mesh type) with per-cell material: cell
    (i, j, k) spans [x_edges[i], x_edges[i+1]] x [y_edges[j], ...] x [z_edges[k], ...];
    ``rho`` and ``c`` are (nx, ny, nz) arrays; the exterior (and everything outside the
    grid) has rho0, c0."""
    name: str
    x_edges: np.ndarray
    y_edges: np.ndarray
    z_edges: np.ndarray
    rho: np.ndarray
    c: np.ndarray
    k0: float
    rho0: float = 1.0
    c0: float = 1.0
    layers: dict = dataclasses.field(default_factory=dict)

    @property
    def shape(self):
        return self.rho.shape

    @property
    def n_cells(self) -> int:
        return int(self.rho.size)

    def centres(self) -> np.ndarray:
        """Cell centres (n_cells, 3) in the cell order (i, j, k), k fastest."""
        cx = 0.5 * (self.x_edges[1:] + self.x_edges[:-1])
        cy = 0.5 * (self.y_edges[1:] + self.y_edges[:-1])
        cz = 0.5 * (self.z_edges[1:] + self.z_edges[:-1])
        X, Y, Z = np.meshgrid(cx, cy, cz, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def sphere_in_cube(n_cells: int, R: float = 2.5, half: float = 3.0, c2: float = 5.0 / 6.0,
                   lambda0: float = 2.0) -> CuboidWorkload:
    """The sphere benchmark of Sec. 3 ("Verification with spherical harmonics"): a uniform
    n^3 cuboid grid on the cube [-half, half]^3 (Omega_1, with the exterior material), the
    sphere |x| < R (Omega_2) with speed of sound c2, density 1 everywhere, exterior
    wavelength lambda0.  A cell takes c2 iff its centre lies inside the sphere (the
    staircase interface)."""
    e = np.linspace(-half, half, int(n_cells) + 1)
    w = CuboidWorkload(name=f"sphere_cube{n_cells}", x_edges=e, y_edges=e.copy(), z_edges=e.copy(),
                       rho=np.ones((n_cells,) * 3), c=np.ones((n_cells,) * 3),
                       k0=2.0 * math.pi / lambda0,
                       layers={"radii": [R], "rho": [1.0], "c": [c2]})
    ctr = w.centres()
    inside = (np.linalg.norm(ctr, axis=1) < R).reshape(w.shape)
    w.c[inside] = c2
    return w


def _matched_edges(breaks, h):
    """Edges of a nonuniform 1-D grid through every break point: each interval between
    consecutive breaks is split into ceil(length / h) equal cells."""
    out = [float(breaks[0])]
    for a, b in zip(breaks[:-1], breaks[1:]):
        m = max(1, int(math.ceil((b - a) / h - 1e-9)))
        out.extend(list(np.linspace(a, b, m + 1)[1:]))
    return np.asarray(out, dtype=np.float64)


def nested_cubes(h: float, side1: float = 7.0, side2: float = 5.0, rho0: float = 1000.0,
                 rho2: float = 500.0, c0: float = 1482.3, speed_ratio: float = 1.2,
                 lambda0: float = 3.0) -> CuboidWorkload:
    """The piecewise-constant density benchmark of Sec. 3: concentric cubes of sides side1
    (Omega_1) and side2 (Omega_2) centred at the origin (lengths in mm), rho1 = rho0,
    rho2, c1 = c2 = c0/speed_ratio, exterior wavelength lambda0.  A nonuniform grid whose
    faces match both interfaces, cells at most h wide."""
    a, b = 0.5 * side1, 0.5 * side2
    e = _matched_edges([-a, -b, b, a], h)
    n = e.shape[0] - 1
    w = CuboidWorkload(name=f"nested_cubes_h{h:g}", x_edges=e, y_edges=e.copy(), z_edges=e.copy(),
                       rho=np.full((n,) * 3, rho0), c=np.full((n,) * 3, c0 / speed_ratio),
                       k0=2.0 * math.pi / lambda0, rho0=rho0, c0=c0)
    ctr = w.centres()
    inner = (np.max(np.abs(ctr), axis=1) < b).reshape(w.shape)
    w.rho[inner] = rho2
    return w


def random_cuboids(shape, seed: int, k0: float = 3.0, jump_fraction: float = 0.5) -> CuboidWorkload:
    """Seeded nonuniform grid on [-1, 1]^3 with random cell widths and per-cell material:
    about ``jump_fraction`` of the cells take a random density in [0.5, 2] (the rest the
    exterior density 1), every cell a random speed of sound in [0.7, 1.3]; many density
    jumps between neighbouring cells, so every face orientation carries unknowns."""
    rng = np.random.default_rng(seed)

    def edges(n):
        w = rng.uniform(0.5, 1.5, n)
        return np.concatenate([[0.0], np.cumsum(w)]) / w.sum() * 2.0 - 1.0

    nx, ny, nz = shape
    rho = np.where(rng.random(shape) < jump_fraction, rng.uniform(0.5, 2.0, shape), 1.0)
    return CuboidWorkload(name=f"random_cuboids{nx}x{ny}x{nz}_s{seed}", x_edges=edges(nx), y_edges=edges(ny),
                          z_edges=edges(nz), rho=rho, c=rng.uniform(0.7, 1.3, shape), k0=float(k0))


def nested_cube_tets(h: float, side1: float = 7.0, side2: float = 5.0, rho0: float = 1000.0,
                     rho2: float = 500.0, c0: float = 1482.3, speed_ratio: float = 1.2,
                     lambda0: float = 3.0, near_factor: float = 2.0,
                     tri_near_factor: float = 2.0) -> Workload:
    """The nested-cubes density benchmark of Sec. 3 as a tetrahedral workload (a second,
    independent discretisation of the problem that ``nested_cubes`` grids with cuboids): a
    uniform grid of spacing h (h must divide both half-sides) on the outer cube, every
    voxel Kuhn-split into six tetrahedra, tetrahedra whose centroid lies in the inner cube
    in Omega_2; the inner cube's boundary squares, two outward triangles each, form
    Gamma_2 (rho_in = rho2, rho_out = rho1 = rho0, so Gamma_1 carries no jump and no
    elements).  Centroid far rule, four-point rule within near_factor voxel widths,
    singularity-subtracted triangles within tri_near_factor edge lengths."""
    a, b = 0.5 * side1, 0.5 * side2
    n = int(round(2 * a / h))
    m_in = int(round((a - b) / h))
    assert abs(n * h - 2 * a) < 1e-9 and abs(m_in * h - (a - b)) < 1e-9, "h must divide both half-sides"
    M = n + 1

    def node(i, j, k):
        return (i * M + j) * M + k

    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    unit = np.eye(3, dtype=np.int64)
    tets = np.empty((base.shape[0], 6, 4), dtype=np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        p1 = base + unit[perm[0]]
        p2 = p1 + unit[perm[1]]
        for q, pq in enumerate((base, p1, p2, base + 1)):
            tets[:, t, q] = node(pq[:, 0], pq[:, 1], pq[:, 2])
    tet = tets.reshape(-1, 4)
    g = np.arange(M)
    GI, GJ, GK = np.meshgrid(g, g, g, indexing="ij")
    vert = np.stack([GI.ravel(), GJ.ravel(), GK.ravel()], axis=1) * h - a
    cen = vert[tet].mean(axis=1)
    inner = np.max(np.abs(cen), axis=1) < b
    rho = np.where(inner, rho2, rho0)
    c = np.full(tet.shape[0], c0 / speed_ratio)
    lo, hi = m_in, n - m_in  # inner cube in node indices
    tris = []
    for ax in range(3):
        b1, b2 = (ax + 1) % 3, (ax + 2) % 3
        for side, sgn in ((lo, -1.0), (hi, 1.0)):
            for u in range(lo, hi):
                for v in range(lo, hi):
                    def p(du, dv):
                        q = [0, 0, 0]
                        q[ax], q[b1], q[b2] = side, u + du, v + dv
                        return node(*q)
                    a0, a1, a2, a3 = p(0, 0), p(1, 0), p(1, 1), p(0, 1)
                    tris.extend([(a0, a1, a2), (a0, a2, a3)] if sgn > 0 else [(a0, a2, a1), (a0, a3, a2)])
    tri = np.asarray(tris, dtype=np.int32)
    near = h * math.sqrt(near_factor ** 2 + 1.0 / 32.0)
    dom = np.where(inner, 2, 1).astype(np.int8)
    return Workload(name=f"nested_cube_tets_h{h:g}", vert=vert.astype(np.float64), tet=tet.astype(np.int32),
                    tri=tri, tri_iface=np.full(tri.shape[0], 2, dtype=np.int8), rho=rho, c=c, grad_alpha=None,
                    tri_rho_in=np.full(tri.shape[0], rho2), tri_rho_out=np.full(tri.shape[0], rho0),
                    k0=2.0 * math.pi / lambda0, rho0=rho0, c0=c0, tet_far_points=1, near_radius=near,
                    tri_near_radius=tri_near_factor * h * math.sqrt(2.0), h=h, R1=a, tet_domain=dom)


def cube_tets(n: int, half: float, rho1: float, c1: float, k0: float, rho0: float = 1.0, c0: float = 1.0,
              tet_far_points: int = 4, tri_near_factor: float = 2.0) -> Workload:
    """The cube [-half, half]^3 with constant material as a tetrahedral workload: the n^3
    voxels Kuhn-split into six tetrahedra each, every boundary square split into two
    outward-oriented triangles (Gamma_1)."""
    h = 2.0 * half / n
    M = n + 1

    def node(i, j, k):
        return (i * M + j) * M + k

    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    unit = np.eye(3, dtype=np.int64)
    tets = np.empty((base.shape[0], 6, 4), dtype=np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        p1 = base + unit[perm[0]]
        p2 = p1 + unit[perm[1]]
        for q, pq in enumerate((base, p1, p2, base + 1)):
            tets[:, t, q] = node(pq[:, 0], pq[:, 1], pq[:, 2])
    g = np.arange(M)
    GI, GJ, GK = np.meshgrid(g, g, g, indexing="ij")
    vert = np.stack([GI.ravel(), GJ.ravel(), GK.ravel()], axis=1) * h - half
    tris = []
    for ax in range(3):
        b1, b2 = (ax + 1) % 3, (ax + 2) % 3
        for side, sgn in ((0, -1.0), (n, 1.0)):
            for u in range(n):
                for v in range(n):
                    def p(du, dv):
                        q = [0, 0, 0]
                        q[ax], q[b1], q[b2] = side, u + du, v + dv
                        return node(*q)
                    a, b, c, d = p(0, 0), p(1, 0), p(1, 1), p(0, 1)
                    # (b1, b2, ax) is right-handed: a->b->c is counter-clockwise about +ax
                    quad = [(a, b, c), (a, c, d)] if sgn > 0 else [(a, c, b), (a, d, c)]
                    tris.extend(quad)
    tri = np.asarray(tris, dtype=np.int32)
    nt = tets.shape[0] * 6
    return Workload(name=f"cube_tets{n}", vert=vert.astype(np.float64), tet=tets.reshape(-1, 4).astype(np.int32),
                    tri=tri, tri_iface=np.ones(tri.shape[0], dtype=np.int8), rho=np.full(nt, rho1),
                    c=np.full(nt, c1), grad_alpha=None, tri_rho_in=np.full(tri.shape[0], rho1),
                    tri_rho_out=np.full(tri.shape[0], rho0), k0=float(k0), rho0=rho0, c0=c0,
                    tet_far_points=tet_far_points, tri_near_radius=tri_near_factor * h * math.sqrt(2.0), h=h,
                    R1=half)
