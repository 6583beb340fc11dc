"""FP64 CPU oracle of the paper's own discretisation on cuboid grids.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library never does.  It shares no code
with the library: it receives the grid edges and the per-cell material and recomputes
everything from the paper's definitions.

What it computes (Sec. 2.3.4, "Computational domain" and "Discrete representation"):

* P0 unknowns on every cell of an nx x ny x nz cuboid grid and on every rectangular
  cell face across which the density jumps (the interfaces, matched by the grid);
* point collocation at the cell and face centroids;
* every integral by the midpoint rule: a cell contributes its integrand at its centre
  times its volume, a face at its centre times its area;
* the weakly singular self term of a cell, -(beta - k0^2 alpha)_e times the integral of G
  over the ball of equal volume; the double-layer self term of a flat face is 0, since
  (x - y).n vanishes on the face;
* Eqs. (alpha), (beta), (mass_function) for the weights and the mass function, the
  interface weight omega = alpha_in - alpha_out (Eq. vsie; "in" the side the face normal
  leaves).

Reading: with a per-cell density, every face between cells of different density is an
interface face (the distributional gradient of a piecewise-constant alpha), so the
adjoint double layer of the volume vanishes.  For the paper's benchmarks, whose density
is constant in each subdomain, those faces are exactly Gamma_1 and Gamma_2.

Unknown order: the cells (i, j, k) at (i ny + j) nz + k; then the jump faces normal to x
(face a between cells a-1 and a, a = 0..nx, the exterior density outside the grid) in the
order (a, j, k); then those normal to y in the order (i, b, k); then those normal to z in
the order (i, j, c).  A face's normal is the +axis direction.

Pins: tests/test_oracle_cuboid.py.
"""
from __future__ import annotations

import math

import numpy as np

from oracle.vsie_oracle import ball_green_integral

FOUR_PI = 4.0 * math.pi


def green(d, k):
    """G = e^{ikr}/(4 pi r) for difference vectors d (..., 3); 0 where r = 0."""
    r = np.linalg.norm(d, axis=-1)
    rs = np.where(r > 0.0, r, 1.0)
    return np.where(r > 0.0, np.exp(1j * k * r) / (FOUR_PI * rs), 0.0)


def green_dny(d, nrm, k):
    """Normal derivative of G in the source point, dG/dn_y = grad_y G . n, for d = x - y:
    grad_y G = -G (ikr - 1) d / r^2.  0 where r = 0."""
    r = np.linalg.norm(d, axis=-1)
    rs = np.where(r > 0.0, r, 1.0)
    g = np.exp(1j * k * rs) / (FOUR_PI * rs)
    dn = np.einsum("...i,...i->...", d, np.broadcast_to(nrm, d.shape))
    return np.where(r > 0.0, -g * (1j * k * rs - 1.0) * dn / (rs * rs), 0.0)


class CuboidDiscretisation:
    """All per-element quantities of the cuboid collocation system, in FP64."""

    def __init__(self, x_edges, y_edges, z_edges, rho, c, k0, rho0=1.0, c0=1.0):
        E = [np.asarray(e, dtype=np.float64) for e in (x_edges, y_edges, z_edges)]
        rho = np.asarray(rho, dtype=np.float64)
        c = np.asarray(c, dtype=np.float64)
        N = tuple(len(e) - 1 for e in E)
        assert rho.shape == N and c.shape == N
        self.k0, self.rho0, self.c0 = float(k0), float(rho0), float(c0)
        omega = self.k0 * self.c0
        ctr = [0.5 * (e[1:] + e[:-1]) for e in E]
        wid = [np.diff(e) for e in E]

        # cells, in the order (i, j, k)
        X, Y, Z = np.meshgrid(*ctr, indexing="ij")
        self.cell_cen = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        WX, WY, WZ = np.meshgrid(*wid, indexing="ij")
        self.cell_vol = (WX * WY * WZ).ravel()
        r = rho.ravel()
        cc = c.ravel()
        self.alpha = self.rho0 / r - 1.0                                        # Eq. (alpha)
        self.beta = (self.rho0 / r) * (omega / cc) ** 2 - (omega / self.c0) ** 2  # Eq. (beta)
        self.sdens = self.beta - self.k0 ** 2 * self.alpha
        self.a_eq = (3.0 * self.cell_vol / FOUR_PI) ** (1.0 / 3.0)
        self.n_cell = r.shape[0]

        # jump faces: axis by axis, lattice order
        cen, nrm, area, om, mass_f = [], [], [], [], []
        pad = np.full(tuple(n + 2 for n in N), self.rho0)
        pad[1:-1, 1:-1, 1:-1] = rho
        for ax in range(3):
            shape = [N[0], N[1], N[2]]
            shape[ax] += 1
            for idx in np.ndindex(*shape):
                lo = [i + 1 for i in idx]
                lo[ax] -= 1                      # the cell below (padded index)
                hi = [i + 1 for i in idx]        # the cell above (padded index)
                rin, rout = pad[tuple(lo)], pad[tuple(hi)]
                if rin == rout:
                    continue
                p = np.empty(3)
                for d in range(3):
                    p[d] = E[d][idx[d]] if d == ax else ctr[d][idx[d]]
                a = 1.0
                for d in range(3):
                    if d != ax:
                        a *= wid[d][idx[d]]
                n = np.zeros(3)
                n[ax] = 1.0
                cen.append(p)
                nrm.append(n)
                area.append(a)
                om.append(self.rho0 / rin - self.rho0 / rout)           # alpha_in - alpha_out
                mass_f.append(0.5 * (self.rho0 / rin + self.rho0 / rout))  # Eq. (mass_function)
        self.n_face = len(cen)
        self.face_cen = np.asarray(cen, dtype=np.float64).reshape(-1, 3)
        self.face_nrm = np.asarray(nrm, dtype=np.float64).reshape(-1, 3)
        self.face_area = np.asarray(area, dtype=np.float64)
        self.face_omega = np.asarray(om, dtype=np.float64)
        self.n = self.n_cell + self.n_face
        self.mass = np.concatenate([self.rho0 / r, np.asarray(mass_f, dtype=np.float64)])
        self.targets = np.concatenate([self.cell_cen, self.face_cen], axis=0)

    @classmethod
    def from_workload(cls, w):
        return cls(w.x_edges, w.y_edges, w.z_edges, w.rho, w.c, w.k0, w.rho0, w.c0)

    # -------------------------------------------------------------- operator rows
    def integral_rows(self, X, rows=None) -> np.ndarray:
        """The integral terms of Eq. (vsie) at the points X (m, 3) by the midpoint rule, as
        rows (m, n); the self terms when X are the collocation points ``rows``."""
        X = np.asarray(X, dtype=np.float64)
        k = self.k0
        A = np.empty((X.shape[0], self.n), dtype=np.complex128)
        d = X[:, None, :] - self.cell_cen[None, :, :]
        A[:, :self.n_cell] = -green(d, k) * (self.sdens * self.cell_vol)[None, :]
        d = X[:, None, :] - self.face_cen[None, :, :]
        A[:, self.n_cell:] = green_dny(d, self.face_nrm[None, :, :], k) * \
            (self.face_omega * self.face_area)[None, :]
        if rows is not None:
            rows = np.asarray(rows, dtype=np.int64)
            own = np.nonzero(rows < self.n_cell)[0]
            e = rows[own]
            A[own, e] = -self.sdens[e] * ball_green_integral(self.a_eq[e], k)
            fo = np.nonzero(rows >= self.n_cell)[0]
            A[fo, rows[fo]] = 0.0  # flat face on its own centre
        return A

    def matrix_rows(self, rows) -> np.ndarray:
        rows = np.asarray(rows, dtype=np.int64)
        A = self.integral_rows(self.targets[rows], rows)
        A[np.arange(rows.shape[0]), rows] += self.mass[rows]
        return A

    def assemble(self) -> np.ndarray:
        """The dense collocation matrix (n, n); small grids only."""
        out = np.empty((self.n, self.n), dtype=np.complex128)
        step = max(1, int(2.0e6 // max(self.n, 1)))
        for r0 in range(0, self.n, step):
            rows = np.arange(r0, min(self.n, r0 + step))
            out[rows] = self.matrix_rows(rows)
        return out

    def apply_rows(self, x, rows) -> np.ndarray:
        return self.matrix_rows(rows) @ x

    def plane_wave(self, direction) -> np.ndarray:
        """Eq. (planewave) at the collocation points."""
        d = np.asarray(direction, dtype=np.float64)
        return np.exp(1j * self.k0 * (self.targets @ d))

    def far_field(self, p, dirs) -> np.ndarray:
        """Far-field pattern p_inf(xhat) with p_s(R xhat) ~ e^{ikR}/R p_inf(xhat): the limit
        of the representation formula, where G(x, y) -> e^{ikR}/(4 pi R) e^{-ik xhat.y} and
        dG/dn_y -> e^{ikR}/(4 pi R) (-ik xhat.n) e^{-ik xhat.y}:
            p_inf = (1/4pi) [sum_cells e^{-ik xhat.y} s V p + ik sum_faces e^{-ik xhat.y} (xhat.n) omega A p].
        p: (n,) or (n, nrhs); dirs: (m, 3) unit vectors."""
        k = self.k0
        X = np.asarray(dirs, dtype=np.float64)
        Ec = np.exp(-1j * k * (X @ self.cell_cen.T)) * (self.sdens * self.cell_vol)[None, :]
        Ef = np.exp(-1j * k * (X @ self.face_cen.T)) * (1j * k) * (X @ self.face_nrm.T) * \
            (self.face_omega * self.face_area)[None, :]
        return np.concatenate([Ec, Ef], axis=1) @ p / FOUR_PI

    def scattered_field(self, p, points) -> np.ndarray:
        """Representation formula (Eq. vsie with m = 1) at exterior points: -(rows) p."""
        return -(self.integral_rows(points) @ p)
