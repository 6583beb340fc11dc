"""FP64 CPU oracle for the discretised nested volume-surface integral equation (VSIE).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the library never does, and the oracle shares
no code, constants or preprocessing with the library (it receives the same mesh and
material arrays and recomputes everything from the paper's definitions).

What it computes, in the paper's notation:

* Eqs. (alpha), (beta): alpha = rho0/rho - 1, beta = (rho0/rho)(omega/c)^2 - (omega/c0)^2,
  omega = k0 c0.
* Eq. (vsie), Theorem "VSIE": for every collocation point x_i
      m(x_i) p_i - sum_e int_e G (beta - k0^2 alpha) p_e
                 + sum_e div_x int_e G grad(alpha) p_e
                 + sum_t int_t dG/dn_y  omega_t p_t  = p_inc(x_i)
  with G = exp(i k0 r)/(4 pi r) (Eq. greens_function) and m from Eq. (mass_function);
  omega_t = alpha_1 on Gamma_1 and alpha_2 - alpha_1 on Gamma_2.
* Sec. 2.3.4: P0 unknowns, collocation at element centroids, the 4x4 block system of the
  "Linear system" subsection ordered [tets | triangles]; weakly singular self terms from
  the integral of G over the ball of equal volume.

Discretisation readings where the paper is silent (the paper uses cuboids; these are
tetrahedra and flat triangles):
* far-field volume rule: the centroid (1 point, weight |e|) or the degree-2 four-point
  rule on every tetrahedron; interface triangles always use the degree-2 three-point
  interior rule;
* near rule: a tetrahedron whose centroid lies within ``near_radius`` of the target uses
  the four-point rule;
* self term of a tetrahedron on its own centroid: -(beta - k0^2 alpha)_e * S(a_e), with
  S(a) = int_{|y|<a} G dy and a the equal-volume radius; the adjoint-double-layer self
  term vanishes by symmetry; the double-layer self term of a flat triangle vanishes since
  (x - y).n = 0;
* near rule for interface triangles: for a target within ``tri_near_radius`` of a
  triangle's centroid, the Laplace part of the double layer is integrated exactly
  (solid angle) and only the bounded Helmholtz remainder uses the three-point rule;
* coincident points (r = 0) that are not a self pair contribute zero.

Pins (tests/test_oracle_*.py) tie every function here to something other than itself.
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi


# ------------------------------------------------------------------ quadrature rules

def tet_rule4_points(P: np.ndarray) -> np.ndarray:
    """Degree-2 four-point rule on tetrahedra (Keast/Hammer-Stroud): barycentric
    coordinates (a, b, b, b) and permutations, a = (5 + 3 sqrt5)/20, b = (5 - sqrt5)/20,
    each weight |e|/4.  P: (m, 4, 3) vertex coordinates -> (m, 4, 3) points."""
    a = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    b = (5.0 - math.sqrt(5.0)) / 20.0
    out = np.empty_like(P)
    for q in range(4):
        lam = np.full(4, b)
        lam[q] = a
        out[:, q, :] = np.einsum("v,mvx->mx", lam, P)
    return out


def tri_rule3_points(P: np.ndarray) -> np.ndarray:
    """Degree-2 three-point interior rule on triangles: barycentric (2/3, 1/6, 1/6) and
    rotations, each weight |t|/3.  P: (m, 3, 3) -> (m, 3, 3)."""
    out = np.empty_like(P)
    for q in range(3):
        lam = np.full(3, 1.0 / 6.0)
        lam[q] = 2.0 / 3.0
        out[:, q, :] = np.einsum("v,mvx->mx", lam, P)
    return out


def tet_volumes(P: np.ndarray) -> np.ndarray:
    d1 = P[:, 1] - P[:, 0]
    d2 = P[:, 2] - P[:, 0]
    d3 = P[:, 3] - P[:, 0]
    return np.abs(np.einsum("ij,ij->i", d1, np.cross(d2, d3))) / 6.0


# ------------------------------------------------------------------ Green's function

def green(r: np.ndarray, k: float) -> np.ndarray:
    """G_k(r) = exp(i k r) / (4 pi r)  (Eq. greens_function)."""
    return np.exp(1j * k * r) / (FOUR_PI * r)


def pair_kernel(d: np.ndarray, s: np.ndarray, v: np.ndarray, k: float) -> np.ndarray:
    """Coefficient of p_e for one source point y with weights (s, v), target x, d = x - y:

        C = -G s + grad_x G . v,     grad_x G = G (i k r - 1) d / r^2,

    i.e. the single-layer term of Eq. (vsie) (s = (beta - k0^2 alpha) w), the adjoint
    double-layer term (v = grad(alpha) w) and the double-layer term, whose normal
    derivative dG/dn_y = -grad_x G . n gives v = -omega n w.  r = 0 contributes 0."""
    r2 = np.einsum("...i,...i->...", d, d)
    ok = r2 > 0.0
    r = np.sqrt(np.where(ok, r2, 1.0))
    G = green(r, k)
    dv = np.einsum("...i,...i->...", d, v)
    val = G * (-s + (1j * k * r - 1.0) * dv / (r * r))
    return np.where(ok, val, 0.0)


def solid_angle(A, B, C, x):
    """Signed solid angle subtended at x by the flat triangle (A, B, C), the sign of
    (A-x).((B-x)x(C-x)) (Van Oosterom & Strackee, IEEE TBME 1983):
    tan(Omega/2) = a.(b x c) / (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|).
    Equals int_t (y - x).n / |y - x|^3 dS_y with n along (B-A)x(C-A)."""
    a = A - x
    b = B - x
    c = C - x
    la = np.linalg.norm(a, axis=-1)
    lb = np.linalg.norm(b, axis=-1)
    lc = np.linalg.norm(c, axis=-1)
    num = np.einsum("...i,...i->...", a, np.cross(b, c))
    den = (la * lb * lc + np.einsum("...i,...i->...", a, b) * lc
           + np.einsum("...i,...i->...", a, c) * lb + np.einsum("...i,...i->...", b, c) * la)
    return 2.0 * np.arctan2(num, den)


def double_layer_near(x, P, nrm, area, k: float):
    """int_t dG_k/dn_y dS_y for a target x near the flat triangle t with vertices P.

    Singularity subtraction: G_k = G_0 + g with G_0 = 1/(4 pi r) and
    g = (e^{ikr} - 1)/(4 pi r), whose derivative g'(r) stays bounded as r -> 0.
    The Laplace part is exact: int_t dG_0/dn_y = -Omega(x)/(4 pi) (solid angle above);
    the remainder dg/dn_y = -g'(r) (x - y).n / r uses the three-point rule."""
    lap = -solid_angle(P[..., 0, :], P[..., 1, :], P[..., 2, :], x) / FOUR_PI
    pts = tri_rule3_points(P.reshape(-1, 3, 3)).reshape(P.shape)
    acc = np.zeros(lap.shape, dtype=np.complex128)
    for q in range(3):
        d = x - pts[..., q, :]
        r = np.linalg.norm(d, axis=-1)
        ok = r > 0
        rs = np.where(ok, r, 1.0)
        eikr = np.exp(1j * k * rs)
        gp = (1j * k * rs * eikr - eikr + 1.0) / (FOUR_PI * rs * rs)
        dn = np.einsum("...i,...i->...", d, nrm)
        acc += np.where(ok, -gp * dn / rs, 0.0)
    return lap + acc * (area / 3.0)


def ball_green_integral(a, k: float):
    """S(a) = int_{|y|<a} G_k(|y|) dy = [exp(i k a)(1 - i k a) - 1] / k^2: the analytic
    self integral over the sphere of equal volume (Sec. 2.3.4).  k -> 0 limit a^2/2."""
    a = np.asarray(a, dtype=np.float64)
    if k == 0.0:
        return a * a / 2.0 + 0j
    return (np.exp(1j * k * a) * (1.0 - 1j * k * a) - 1.0) / (k * k)


# ------------------------------------------------------------------ density gradient

def face_neighbours(tet, dom):
    """For every tetrahedron the tetrahedra that share one of its faces and lie in the
    same subdomain."""
    tet = np.asarray(tet, dtype=np.int64)
    owner = {}
    for e in range(tet.shape[0]):
        for f in range(4):
            key = tuple(sorted(int(v) for j, v in enumerate(tet[e]) if j != f))
            owner.setdefault(key, []).append(e)
    nb = [[] for _ in range(tet.shape[0])]
    for es in owner.values():
        if len(es) == 2 and dom[es[0]] == dom[es[1]]:
            nb[es[0]].append(es[1])
            nb[es[1]].append(es[0])
    return nb


def lsq_grad_alpha(vert, tet, dom, alpha):
    """grad(alpha) of an element-wise alpha by least squares over face neighbours in the
    same subdomain (the reading for per-element density): g_e minimises
    sum_f (alpha_f - alpha_e - g . (c_f - c_e))^2, c the centroids; the minimum-norm
    minimiser (numpy pseudo-inverse, singular values below 1e-6 of the largest dropped)
    when the neighbours span fewer than three directions, 0 without neighbours.  g is linear in alpha: returns (g (n_tet, 3), W) with W the
    sparse (3 n_tet) x n_tet matrix, g.ravel() = W alpha."""
    import scipy.sparse as sp
    vert = np.asarray(vert, dtype=np.float64)
    tet = np.asarray(tet, dtype=np.int64)
    cen = vert[tet].mean(axis=1)
    nb = face_neighbours(tet, dom)
    alpha = np.asarray(alpha, dtype=np.float64)
    g = np.zeros((tet.shape[0], 3))
    rows, cols, vals = [], [], []
    for e in range(tet.shape[0]):
        if not nb[e]:
            continue
        Dm = cen[nb[e]] - cen[e]                      # (k, 3)
        P = np.linalg.pinv(Dm, rcond=1e-6)            # (3, k): g = P (alpha_f - alpha_e)
        g[e] = P @ (alpha[nb[e]] - alpha[e])
        for c in range(3):
            for q, f in enumerate(nb[e]):
                rows.append(3 * e + c)
                cols.append(f)
                vals.append(P[c, q])
            rows.append(3 * e + c)
            cols.append(e)
            vals.append(-P[c].sum())
    W = sp.csr_matrix((vals, (rows, cols)), shape=(3 * tet.shape[0], tet.shape[0]))
    return g, W


# ------------------------------------------------------------------ discretisation

class Discretisation:
    """All per-element quantities of the collocation system, in FP64."""

    def __init__(self, vert, tet, tri, rho, c, grad_alpha, tri_rho_in, tri_rho_out,
                 k0, rho0=1.0, c0=1.0, tet_far_points=1, near_radius=0.0,
                 tri_near_radius=0.0):
        vert = np.asarray(vert, dtype=np.float64)
        tet = np.asarray(tet, dtype=np.int64)
        tri = np.asarray(tri, dtype=np.int64).reshape(-1, 3)
        self.k0 = float(k0)
        self.rho0 = float(rho0)
        self.c0 = float(c0)
        self.far_points = int(tet_far_points)
        self.near_radius = float(near_radius)
        self.tri_near_radius = float(tri_near_radius)
        self.n_tet = tet.shape[0]
        self.n_tri = tri.shape[0]
        self.n = self.n_tet + self.n_tri

        # volume elements
        PT = vert[tet]
        self.tet_cen = PT.mean(axis=1)
        self.tet_vol = tet_volumes(PT)
        self.tet_pts = tet_rule4_points(PT)
        rho = np.asarray(rho, dtype=np.float64)
        c = np.asarray(c, dtype=np.float64)
        omega = self.k0 * self.c0                                # omega = k0 c0
        alpha = self.rho0 / rho - 1.0                             # Eq. (alpha)
        beta = (self.rho0 / rho) * (omega / c) ** 2 - (omega / self.c0) ** 2  # Eq. (beta)
        self.alpha = alpha
        self.beta = beta
        self.sdens = beta - self.k0 ** 2 * alpha                  # weight of the V term
        if grad_alpha is None:
            self.grad_alpha = np.zeros((self.n_tet, 3))
        else:
            self.grad_alpha = np.asarray(grad_alpha, dtype=np.float64).reshape(-1, 3)
        self.a_eq = (3.0 * self.tet_vol / FOUR_PI) ** (1.0 / 3.0)

        # interface elements
        PS = vert[tri]
        self.tri_P = PS
        self.tri_cen = PS.mean(axis=1)
        cr = np.cross(PS[:, 1] - PS[:, 0], PS[:, 2] - PS[:, 0])
        nrm = np.linalg.norm(cr, axis=1)
        self.tri_area = 0.5 * nrm
        self.tri_nrm = cr / np.where(nrm > 0, nrm, 1.0)[:, None]
        self.tri_pts = tri_rule3_points(PS)
        rin = np.asarray(tri_rho_in, dtype=np.float64)
        rout = np.asarray(tri_rho_out, dtype=np.float64)
        # omega_t = alpha_in - alpha_out: alpha_1 on Gamma_1 (alpha_0 = 0), alpha_2 - alpha_1
        # on Gamma_2 (Eq. vsie); written with rho directly since alpha = rho0/rho - 1.
        self.tri_omega = self.rho0 / rin - self.rho0 / rout

        # mass function, Eq. (mass_function)
        self.mass = np.concatenate([self.rho0 / rho,
                                    0.5 * (self.rho0 / rin + self.rho0 / rout)])
        self.targets = np.concatenate([self.tet_cen, self.tri_cen], axis=0)

    @classmethod
    def from_workload(cls, w):
        ga = w.grad_alpha
        if getattr(w, "grad_alpha_lsq", False):
            ga, _ = lsq_grad_alpha(w.vert, w.tet, w.tet_domain, w.rho0 / np.asarray(w.rho) - 1.0)
        return cls(w.vert, w.tet, w.tri, w.rho, w.c, ga, w.tri_rho_in,
                   w.tri_rho_out, w.k0, w.rho0, w.c0, w.tet_far_points, w.near_radius,
                   w.tri_near_radius)

    # -------------------------------------------------------------- operator rows
    def matrix_rows(self, rows) -> np.ndarray:
        """Rows ``rows`` of the collocation matrix A (len(rows), n), from the plain
        element-by-element definition (no far/near splitting, no correction matrix)."""
        rows = np.asarray(rows, dtype=np.int64)
        A = self.integral_rows(self.targets[rows], rows)
        A[np.arange(rows.shape[0]), rows] += self.mass[rows]
        return A

    def integral_rows(self, X, rows=None) -> np.ndarray:
        """The integral terms of Eq. (vsie) at the points X (m, 3) as rows (m, n): the far
        rule, the near rules for elements within the near radii of a point, and, when X are
        the collocation points ``rows``, the self terms; no mass term."""
        X = np.asarray(X, dtype=np.float64)
        R = X.shape[0]
        k = self.k0
        A = np.zeros((R, self.n), dtype=np.complex128)

        # volume columns
        s4 = self.sdens * self.tet_vol / 4.0
        g4 = self.grad_alpha * (self.tet_vol / 4.0)[:, None]
        if self.far_points == 4:
            for q in range(4):
                d = X[:, None, :] - self.tet_pts[None, :, q, :]
                A[:, :self.n_tet] += pair_kernel(d, s4[None, :], g4[None, :, :], k)
        else:
            d = X[:, None, :] - self.tet_cen[None, :, :]
            A[:, :self.n_tet] = pair_kernel(d, (self.sdens * self.tet_vol)[None, :],
                                            (self.grad_alpha * self.tet_vol[:, None])[None],
                                            k)
            if self.near_radius > 0.0:
                dist2 = np.einsum("rei,rei->re", d, d)
                rr, ee = np.nonzero(dist2 < self.near_radius ** 2)
                acc = np.zeros(rr.shape[0], dtype=np.complex128)
                for q in range(4):
                    dq = X[rr] - self.tet_pts[ee, q, :]
                    acc += pair_kernel(dq, s4[ee], g4[ee], k)
                A[rr, ee] = acc
        # self terms: sphere of equal volume for the single layer; adjoint double layer 0
        own = rows < self.n_tet if rows is not None else np.zeros(R, dtype=bool)
        if own.any():
            e = rows[own]
            A[np.nonzero(own)[0], e] = -self.sdens[e] * ball_green_integral(self.a_eq[e], k)

        # interface columns: three-point rule, v = -omega n w
        if self.n_tri:
            w3 = self.tri_area / 3.0
            vt = -(self.tri_omega * w3)[:, None] * self.tri_nrm
            zero = np.zeros(self.n_tri)
            acc = np.zeros((R, self.n_tri), dtype=np.complex128)
            for q in range(3):
                d = X[:, None, :] - self.tri_pts[None, :, q, :]
                acc += pair_kernel(d, zero[None, :], vt[None, :, :], k)
            if self.tri_near_radius > 0.0:
                d = X[:, None, :] - self.tri_cen[None, :, :]
                dist2 = np.einsum("rti,rti->rt", d, d)
                rr, tt = np.nonzero(dist2 < self.tri_near_radius ** 2)
                acc[rr, tt] = self.tri_omega[tt] * double_layer_near(
                    X[rr], self.tri_P[tt], self.tri_nrm[tt], self.tri_area[tt], k)
                # a triangle on its own centroid: principal value 0 (the jump -1/2 is
                # part of the mass function, Eqs. jump_g1, jump_g2)
                if rows is not None:
                    own_t = rows[rr] == self.n_tet + tt
                    acc[rr[own_t], tt[own_t]] = 0.0
            A[:, self.n_tet:] = acc
        return A

    def matrix_columns(self, cols) -> np.ndarray:
        """Columns ``cols`` of the collocation matrix A (n, len(cols)) from the same
        element-by-element definition as ``matrix_rows``, read down a column: the integral
        of element e at every collocation point (the far rule, or the near rule at points
        within the near radius of e, the self term at e's own point), plus the mass on the
        diagonal.  Serves entries of A^H lam = conj(A)^T lam at large sizes."""
        cols = np.asarray(cols, dtype=np.int64)
        X = self.targets
        k = self.k0
        out = np.zeros((self.n, cols.shape[0]), dtype=np.complex128)
        for c, e in enumerate(cols):
            if e < self.n_tet:
                s = self.sdens[e] * self.tet_vol[e]
                g = self.grad_alpha[e] * self.tet_vol[e]
                if self.far_points == 4:
                    for q in range(4):
                        out[:, c] += pair_kernel(X - self.tet_pts[e, q], np.full(self.n, s / 4.0),
                                                 np.tile(g / 4.0, (self.n, 1)), k)
                else:
                    d = X - self.tet_cen[e]
                    out[:, c] = pair_kernel(d, np.full(self.n, s), np.tile(g, (self.n, 1)), k)
                    if self.near_radius > 0.0:
                        near = np.nonzero(np.einsum("ri,ri->r", d, d) < self.near_radius ** 2)[0]
                        acc = np.zeros(near.shape[0], dtype=np.complex128)
                        for q in range(4):
                            acc += pair_kernel(X[near] - self.tet_pts[e, q], np.full(near.shape[0], s / 4.0),
                                               np.tile(g / 4.0, (near.shape[0], 1)), k)
                        out[near, c] = acc
                out[e, c] = -self.sdens[e] * ball_green_integral(self.a_eq[e], k)
            else:
                t = e - self.n_tet
                w3 = self.tri_area[t] / 3.0
                vt = -(self.tri_omega[t] * w3) * self.tri_nrm[t]
                for q in range(3):
                    out[:, c] += pair_kernel(X - self.tri_pts[t, q], np.zeros(self.n),
                                             np.tile(vt, (self.n, 1)), k)
                if self.tri_near_radius > 0.0:
                    d = X - self.tri_cen[t]
                    near = np.nonzero(np.einsum("ri,ri->r", d, d) < self.tri_near_radius ** 2)[0]
                    out[near, c] = self.tri_omega[t] * double_layer_near(
                        X[near], np.broadcast_to(self.tri_P[t], (near.shape[0], 3, 3)),
                        np.broadcast_to(self.tri_nrm[t], (near.shape[0], 3)),
                        np.full(near.shape[0], self.tri_area[t]), k)
                    out[e, c] = 0.0
            out[e, c] += self.mass[e]
        return out

    def _chunk(self) -> int:
        pts = self.n_tet * (4 if self.far_points == 4 else 1) + 3 * self.n_tri
        return max(1, int(3.0e6 // max(pts, 1)))

    def apply_rows(self, p: np.ndarray, rows) -> np.ndarray:
        """(A p)[rows]; p may be (n,) or (n, nrhs)."""
        rows = np.asarray(rows, dtype=np.int64)
        out = np.empty((rows.shape[0],) + p.shape[1:], dtype=np.complex128)
        ch = self._chunk()
        for s in range(0, rows.shape[0], ch):
            out[s:s + ch] = self.matrix_rows(rows[s:s + ch]) @ p
        return out

    def apply(self, p: np.ndarray) -> np.ndarray:
        return self.apply_rows(p, np.arange(self.n))

    def adjoint_apply(self, lam: np.ndarray) -> np.ndarray:
        """A^H lam, accumulated from the same rows."""
        out = np.zeros((self.n,) + lam.shape[1:], dtype=np.complex128)
        ch = self._chunk()
        for s in range(0, self.n, ch):
            rows = np.arange(s, min(s + ch, self.n))
            out += self.matrix_rows(rows).conj().T @ lam[rows]
        return out

    def assemble(self) -> np.ndarray:
        return self.matrix_rows(np.arange(self.n))

    # -------------------------------------------------------------- right-hand sides
    def plane_wave(self, direction) -> np.ndarray:
        """f_i = p_inc(x_i) = exp(i k0 x_i . d) (Eq. planewave)."""
        d = np.asarray(direction, dtype=np.float64)
        d = d / np.linalg.norm(d)
        return np.exp(1j * self.k0 * (self.targets @ d))

    def far_field(self, p: np.ndarray, dirs) -> np.ndarray:
        """Far-field pattern of the scattered field, from Eq. (vsie) used as a
        representation formula in Omega_0 (m = 1): p_s(x) = -sum_j C(x, y_j) p_e(j), and
        as |x| -> inf, G -> e^{ik|x|}/(4 pi |x|) e^{-ik xhat.y}, grad_x G -> i k xhat G, so
        p_inf(xhat) = (1/4pi) sum_j e^{-ik xhat.y_j} (s_j - i k xhat.v_j) p_e(j),
        with the far-field source points (no near rule applies at infinity)."""
        dirs = np.asarray(dirs, dtype=np.float64)
        k = self.k0
        if self.far_points == 4:
            Y = self.tet_pts.reshape(-1, 3)
            S = np.repeat(self.sdens * self.tet_vol / 4.0, 4)
            V = np.repeat(self.grad_alpha * (self.tet_vol / 4.0)[:, None], 4, axis=0)
            own = np.repeat(np.arange(self.n_tet), 4)
        else:
            Y = self.tet_cen
            S = self.sdens * self.tet_vol
            V = self.grad_alpha * self.tet_vol[:, None]
            own = np.arange(self.n_tet)
        w3 = self.tri_area / 3.0
        vt = -(self.tri_omega * w3)[:, None] * self.tri_nrm
        Y = np.concatenate([Y, self.tri_pts.reshape(-1, 3)])
        S = np.concatenate([S, np.zeros(3 * self.n_tri)])
        V = np.concatenate([V, np.repeat(vt, 3, axis=0)])
        own = np.concatenate([own, self.n_tet + np.repeat(np.arange(self.n_tri), 3)])
        ph = np.exp(-1j * k * (dirs @ Y.T))
        amp = S[None, :] - 1j * k * (dirs @ V.T)
        return (ph * amp) @ p[own] / FOUR_PI


# ------------------------------------------------------------------ GMRES

def gmres(matvec, b: np.ndarray, tol: float = 1e-5, maxiter: int = 1000):
    """Unrestarted, unpreconditioned GMRES with x0 = 0 (Sec. 3.1 settings): Arnoldi with
    modified Gram-Schmidt, least-squares solve of the Hessenberg system at each step.
    Returns (x, iterations, relative residual estimate)."""
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    V = [b / bn]
    H = np.zeros((maxiter + 1, maxiter), dtype=np.complex128)
    rel = 1.0
    y = np.zeros(0, dtype=np.complex128)
    j = 0
    for j in range(maxiter):
        w = matvec(V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2, dtype=np.complex128)
        e1[0] = bn
        y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)
        rel = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / bn
        if rel <= tol or H[j + 1, j] == 0.0:
            break
        V.append(w / H[j + 1, j])
    x = np.zeros_like(b)
    for i in range(y.shape[0]):
        x = x + y[i] * V[i]
    return x, j + 1, rel


# ------------------------------------------------------------------ far-field misfit gradient

def scattered_field(D, p, points):
    """Scattered pressure at points of the exterior domain Omega_0, from Eq. (vsie) read as a
    representation formula with m = 1 outside the body (the mass function of Omega_0):
    p(x) + sum_e [integral terms of column e at x] p_e = p_inc(x), so
    p_s(x) = p(x) - p_inc(x) = -(integral rows at x) p.  p: (n,) or (n, nrhs)."""
    return -(D.integral_rows(points) @ p)


def far_field_matrix(D: Discretisation, dirs) -> np.ndarray:
    """F with (F p)_d = p_inf(xhat_d) of ``Discretisation.far_field``: columns summed over the
    far-field points of each element."""
    n = D.n
    dirs = np.asarray(dirs, dtype=np.float64)
    k = D.k0
    F = np.zeros((dirs.shape[0], n), dtype=np.complex128)
    if D.far_points == 4:
        for q in range(4):
            y = D.tet_pts[:, q, :]
            amp = (D.sdens * D.tet_vol / 4.0)[None, :] - 1j * k * (dirs @ (D.grad_alpha * (D.tet_vol / 4.0)[:, None]).T)
            F[:, :D.n_tet] += np.exp(-1j * k * (dirs @ y.T)) * amp
    else:
        amp = (D.sdens * D.tet_vol)[None, :] - 1j * k * (dirs @ (D.grad_alpha * D.tet_vol[:, None]).T)
        F[:, :D.n_tet] = np.exp(-1j * k * (dirs @ D.tet_cen.T)) * amp
    w3 = D.tri_area / 3.0
    vt = -(D.tri_omega * w3)[:, None] * D.tri_nrm
    for q in range(3):
        y = D.tri_pts[:, q, :]
        F[:, D.n_tet:] += np.exp(-1j * k * (dirs @ y.T)) * (-1j * k * (dirs @ vt.T))
    return F / FOUR_PI


def far_source_points(D):
    """The far-rule source points y_j of the discretisation and their owning unknowns:
    tetrahedron centroids (or the four points of the degree-2 rule when far_points == 4),
    then the three interior points of every interface triangle."""
    if D.far_points == 4:
        tp = D.tet_pts.reshape(-1, 3)
        town = np.repeat(np.arange(D.n_tet), 4)
    else:
        tp = D.tet_cen
        town = np.arange(D.n_tet)
    sp = D.tri_pts.reshape(-1, 3)
    sown = D.n_tet + np.repeat(np.arange(D.n_tri), 3)
    return np.concatenate([tp, sp], axis=0), np.concatenate([town, sown])


def gradient_channels(D, lam, points):
    """Derivative channels of the operator's columns with respect to the source weights,
    for an adjoint state lam: at every point y_j
        Phi_j = sum_i conj(G(x_i, y_j)) lam_i,   Psi_j = sum_i conj(grad_x G(x_i, y_j)) lam_i,
    over all collocation points x_i (terms with x_i = y_j vanish), G = e^{ikr}/(4 pi r)
    (Eq. greens_function), grad_x G = G (i k r - 1)(x - y)/r^2.  With the pair coefficient
    C = -G s + grad_x G . v of a source point (pair_kernel), sum_i conj(dC/ds) lam_i = -Phi
    and sum_i conj(dC/dv) lam_i = Psi.  Returns (Phi (m,), Psi (m, 3))."""
    points = np.asarray(points, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.complex128)
    k = D.k0
    m = points.shape[0]
    phi = np.zeros(m, dtype=np.complex128)
    psi = np.zeros((m, 3), dtype=np.complex128)
    step = max(1, int(2.0e6 // max(D.n, 1)))
    for a in range(0, m, step):
        Y = points[a:a + step]
        d = D.targets[None, :, :] - Y[:, None, :]          # x_i - y_j
        r2 = np.einsum("jil,jil->ji", d, d)
        ok = r2 > 0.0
        r = np.sqrt(np.where(ok, r2, 1.0))
        G = np.where(ok, green(r, k), 0.0)
        phi[a:a + step] = np.conj(G) @ lam
        g = np.where(ok, G * (1j * k * r - 1.0) / (r * r), 0.0)
        psi[a:a + step] = np.einsum("ji,jil,i->jl", np.conj(g), d, lam)
    return phi, psi


def misfit_and_gradient(w, dirs, target, direction):
    """L = 1/2 sum_d |p_inf(xhat_d) - t_d|^2 for the solution of A p = p_inc, and dL/drho_e,
    dL/dc_e for every tetrahedron (element-wise density, interface densities fixed; with
    w.grad_alpha_lsq the density gradient of the least-squares reading, which carries
    rho into neighbouring columns), by the adjoint method:
        A^H lam = F^H r,  r = F p - t,
        dL/dtheta = Re[r^H (dF/dtheta) p] - Re[lam^H (dA/dtheta) p].
    A and F depend on (rho_e, c_e) only through the single-layer weight
    s_e = beta_e - k0^2 alpha_e of column e (linear in s_e) and the mass m_e = rho0/rho_e,
    so dA/ds_e = A_unit[:, e] (the operator assembled with unit weight and no mass) and
    dF/ds_e = F_unit[:, e].  Dense (tiny meshes only).  Returns (L, dL/drho, dL/dc, p)."""
    D = Discretisation.from_workload(w)
    A = D.assemble()
    F = far_field_matrix(D, dirs)
    b = D.plane_wave(direction)
    p = np.linalg.solve(A, b)
    r = F @ p - target
    L = 0.5 * float(np.vdot(r, r).real)
    lam = np.linalg.solve(A.conj().T, F.conj().T @ r)
    # unit-weight single layer: sdens = 1 on every tetrahedron, no interface term, no mass
    U = Discretisation.from_workload(w)
    U.sdens = np.ones_like(U.sdens)
    U.grad_alpha = np.zeros_like(U.grad_alpha)
    U.tri_omega = np.zeros_like(U.tri_omega)
    U.mass = np.zeros_like(U.mass)
    Au = U.assemble()[:, :D.n_tet]
    Fu = far_field_matrix(U, dirs)[:, :D.n_tet]
    pt = p[:D.n_tet]
    dLds = ((np.conj(r) @ Fu) * pt).real - ((np.conj(lam) @ Au) * pt).real
    dLdm = -(np.conj(lam[:D.n_tet]) * pt).real
    rho = np.asarray(w.rho, dtype=np.float64)
    c = np.asarray(w.c, dtype=np.float64)
    k0, rho0, c0 = D.k0, D.rho0, D.c0
    # s = beta - k0^2 alpha = k0^2 (rho0/rho) ((c0/c)^2 - 1),  m = rho0/rho
    ds_drho = -D.sdens / rho
    ds_dc = -2.0 * k0 ** 2 * (rho0 / rho) * c0 ** 2 / c ** 3
    dm_drho = -rho0 / rho ** 2
    dLdrho = dLds * ds_drho + dLdm * dm_drho
    if getattr(w, "grad_alpha_lsq", False):
        # grad(alpha) = W alpha (least squares over face neighbours) depends on rho through
        # alpha = rho0/rho - 1: dL/dalpha = W^T dL/dgrad(alpha), with dA/dgrad(alpha)_{e,c}
        # the column of the operator assembled with unit grad(alpha) along axis c
        _, Wst = lsq_grad_alpha(w.vert, w.tet, w.tet_domain, rho0 / rho - 1.0)
        gv = np.zeros((D.n_tet, 3))
        for ax in range(3):
            V = Discretisation.from_workload(w)
            V.sdens = np.zeros_like(V.sdens)
            V.grad_alpha = np.zeros_like(V.grad_alpha)
            V.grad_alpha[:, ax] = 1.0
            V.tri_omega = np.zeros_like(V.tri_omega)
            V.mass = np.zeros_like(V.mass)
            Av = V.assemble()[:, :D.n_tet]
            Fv = far_field_matrix(V, dirs)[:, :D.n_tet]
            gv[:, ax] = ((np.conj(r) @ Fv) * pt).real - ((np.conj(lam) @ Av) * pt).real
        dLdrho = dLdrho + (Wst.T @ gv.ravel()) * (-rho0 / rho ** 2)
    return L, dLdrho, dLds * ds_dc, p
