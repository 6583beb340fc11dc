"""FP64 oracle of the nested PMCHWT boundary element method (test infrastructure only).

The paper compares its VSIE with the standard PMCHWT boundary integral formulation for
nested domains with piecewise-constant material (Sec. 2.4, "Boundary Element Method";
benchmark 2 of Table "benchmarks"), discretised with piecewise-linear (P1) Galerkin
elements on triangulated interfaces and solved by GMRES with mass-matrix preconditioning
(Sec. 3.1, computational settings).  This module writes that formulation out as a dense
matrix.  Nothing here is shared with, or calls, the CUDA library.

Formulation (derived from the Calderon identities of each subdomain).  Interfaces
Gamma_m with fixed normals n (pointing away from the centre); subdomain j (wavenumber
k_j, density rho_j) is bounded by the interfaces in ``domains[j]["sides"]``, with
sigma_{jm} = +1 if n points out of Omega_j on Gamma_m and -1 otherwise.  The unknowns on
every interface are the traces u = p and v = (1/rho) dp/dn, both continuous across it
(Eqs. transmission_pressure, transmission_velocity).  With the boundary operators of
wavenumber k on the interfaces,

    V phi(x)  = int G(x,y) phi(y) dy,          K psi(x)  = int dG/dn_y psi(y) dy,
    K' phi(x) = d/dn_x int G(x,y) phi(y) dy,   W psi(x)  = -d/dn_x int dG/dn_y psi(y) dy,

G(x, y) = e^{ik|x-y|}/(4 pi |x-y|) (Eq. greens_function), the Cauchy data X_j of Omega_j
(taken with Omega_j's outward normal) satisfy A_j X_j = X_j/2 with A_j = [[-K, V], [W, K']]
(the exterior one for the scattered field).  Writing X_j = diag(1, sigma rho_j) (u, v),
multiplying the rows on Gamma_m by diag(sigma_{jm}, 1/rho_j) and summing over j cancels
the identity terms on every interface, and the incident field (an entire solution) moves
to the right-hand side:

    sum_j sigma_{jm} sigma_{jl} [[-K_j, rho_j V_j], [W_j/rho_j, K'_j]]_{m <- l} (u_l, v_l)
        = (p_inc, (1/rho_0) dp_inc/dn) on the outermost interface, 0 elsewhere.

Discretisation.  P1 (continuous piecewise-linear) trial and test functions for u and v on
flat triangles; Galerkin entries with the hypersingular form written through surface
curls (integration by parts on a closed surface):
    <phi_a, W phi_b> = int int G [curl phi_a . curl phi_b - k^2 (n_x . n_y) phi_a phi_b].
<phi_a, K' phi_b> equals <phi_b, K phi_a> for Galerkin matrices (G is symmetric), so K' is
the transpose of K with test and trial surfaces swapped.  Quadrature:
  * every triangle pair: the "far rule", a collapsed Gauss product rule with q x q points
    on each triangle (point pairs at zero distance contribute nothing);
  * near pairs (sharing a vertex, or centroid distance below near_factor times the larger
    diameter) replace that by: a q_n x q_n collapsed rule on the test triangle, and on the
    trial triangle the static part 1/(4 pi r) integrated in closed form (potentials of
    linear densities on a flat triangle: line integrals over its edges, and the solid
    angle) plus the smooth remainder G - 1/(4 pi r) on a q_n x q_n rule; the V block of a
    pair is the mean of its two orders (test/trial swapped), so V and W are symmetric.
Left preconditioning by the lumped P1 mass matrix (diagonal, the row sums of the mass
matrix) scales every row by 1/m_a; the right-hand side is scaled alike.

Far-field pattern (p_s ~ e^{ik0 R}/R p_inf) from the exterior representation
p_s = DL(u) - SL(rho_0 v) on the outermost interface:
    p_inf(xhat) = (1/4 pi) int e^{-i k0 xhat.y} [-i k0 (xhat . n_y) u(y) - rho_0 v(y)] dy.
"""
from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi


# ------------------------------------------------------------------ quadrature

def gauss_legendre01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(int(n))
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(n: int):
    """Collapsed (Duffy) Gauss product rule on a triangle: (u, v) in [0,1]^2 maps to the
    point with barycentric coordinates (1 - s - t, s, t), s = u, t = (1 - u) v, weight
    w_u w_v (1 - u), normalised to sum 1 (multiply by the triangle's area).  Exact for
    polynomials of degree 2n - 2 (the Jacobian adds one degree in u).  Returns
    (lam (n^2, 3), w (n^2,))."""
    u, wu = gauss_legendre01(n)
    v, wv = gauss_legendre01(n)
    s = np.repeat(u, n)
    t = (1.0 - s) * np.tile(v, n)
    w = 2.0 * np.repeat(wu, n) * np.tile(wv, n) * (1.0 - s)
    lam = np.stack([1.0 - s - t, s, t], axis=1)
    return lam, w


# ------------------------------------------------------------------ surfaces

class Surface:
    """A closed triangulated surface, triangles oriented so that the right-hand normal
    points outward."""

    def __init__(self, vert, tri):
        self.vert = np.asarray(vert, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        a, b, c = (self.vert[self.tri[:, i]] for i in range(3))
        cr = np.cross(b - a, c - a)
        nn = np.linalg.norm(cr, axis=1)
        self.area = 0.5 * nn
        self.nrm = cr / nn[:, None]
        self.cen = (a + b + c) / 3.0
        e2 = np.stack([((b - a) ** 2).sum(1), ((c - b) ** 2).sum(1), ((a - c) ** 2).sum(1)], 1)
        self.diam2 = e2.max(axis=1)
        # gradients of the barycentric functions (constant per triangle) and surface curls
        twoA = (2.0 * self.area)[:, None]
        g0 = np.cross(self.nrm, c - b) / twoA
        g1 = np.cross(self.nrm, a - c) / twoA
        g2 = np.cross(self.nrm, b - a) / twoA
        self.grad = np.stack([g0, g1, g2], axis=1)                     # (nt, 3 vertices, 3)
        self.curl = np.cross(self.nrm[:, None, :], self.grad)          # n x grad lambda
        self.n_vert = self.vert.shape[0]
        self.n_tri = self.tri.shape[0]

    def points(self, lam, w):
        """Quadrature points (nt, Q, 3) and weights times area (nt, Q)."""
        P = np.einsum("qi,tid->tqd", lam, self.vert[self.tri])
        return P, self.area[:, None] * w[None, :]

    def lumped_mass(self):
        """Row sums of the P1 mass matrix: sum of A_T / 3 over the triangles at a vertex."""
        m = np.zeros(self.n_vert)
        np.add.at(m, self.tri.reshape(-1), np.repeat(self.area / 3.0, 3))
        return m

    def mass(self):
        """Consistent P1 mass matrix (dense): A_T/12 (1 + delta_ij)."""
        M = np.zeros((self.n_vert, self.n_vert))
        loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
        for t in range(self.n_tri):
            idx = self.tri[t]
            M[np.ix_(idx, idx)] += self.area[t] * loc
        return M


# ------------------------------------------------------------------ closed-form potentials

def _edge_log(lm, lp, R0sq, Rm, Rp):
    """ln((R+ + l+)/(R- + l-)) = int_{l-}^{l+} dl / sqrt(l^2 + R0^2), written without
    cancellation for either sign of l-, l+."""
    with np.errstate(divide="ignore", invalid="ignore"):
        pos = np.log((Rp + lp) / (Rm + lm))            # l- >= 0
        neg = np.log((Rm - lm) / (Rp - lp))            # l+ <= 0
        mid = np.log((Rp + lp) * (Rm - lm) / R0sq)     # l- < 0 < l+
    return np.where(lm >= 0.0, pos, np.where(lp <= 0.0, neg, mid))


def triangle_potentials(x, a, b, c):
    """For points x and flat triangles (a, b, c) (arrays broadcast over leading axes; the
    triangle oriented by its right-hand normal n), with rho the projection of x on the
    triangle's plane and h = n.(x - a):
        S0 = int 1/R dS,  S1 = int (y - rho)/R dS,  D0 = int h/R^3 dS,  D1 = int h (y - rho)/R^3 dS,
    R = |x - y|.  S1 = sum_e u_e int_e R dl and D1 = -h sum_e u_e int_e dl/R follow from the
    gradient theorem in the plane (u_e: the edge's outward in-plane normal); S0 from
    integrating in polar coordinates about rho; D0 is the solid angle of the triangle seen
    from x, signed with h.  Returns (S0, S1, D0, D1, h, rho, n)."""
    x, a, b, c = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (x, a, b, c)))
    n = np.cross(b - a, c - a)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    h = np.einsum("...d,...d->...", x - a, n)
    rho = x - h[..., None] * n
    ah = np.abs(h)
    S0 = np.zeros(h.shape)
    S1 = np.zeros(x.shape)
    D1 = np.zeros(x.shape)
    for p, q in ((a, b), (b, c), (c, a)):
        L = q - p
        ll = np.linalg.norm(L, axis=-1, keepdims=True)
        lhat = L / ll
        uhat = np.cross(lhat, n)
        lm = np.einsum("...d,...d->...", p - rho, lhat)
        lp = np.einsum("...d,...d->...", q - rho, lhat)
        P0 = np.einsum("...d,...d->...", p - rho, uhat)
        R0sq = P0 * P0 + h * h
        Rm = np.sqrt(lm * lm + R0sq)
        Rp = np.sqrt(lp * lp + R0sq)
        f = np.where(R0sq > 0.0, _edge_log(lm, lp, R0sq, Rm, Rp), 0.0)
        with np.errstate(divide="ignore", invalid="ignore"):
            at = np.arctan2(P0 * lp, R0sq + ah * Rp) - np.arctan2(P0 * lm, R0sq + ah * Rm)
        S0 += P0 * f - ah * at
        S1 += 0.5 * uhat * (R0sq * f + lp * Rp - lm * Rm)[..., None]
        D1 += -h[..., None] * uhat * f[..., None]
    A, B, C = a - x, b - x, c - x
    nA, nB, nC = (np.linalg.norm(v, axis=-1) for v in (A, B, C))
    num = np.einsum("...d,...d->...", A, np.cross(B, C))
    den = (nA * nB * nC + np.einsum("...d,...d->...", A, B) * nC
           + np.einsum("...d,...d->...", A, C) * nB + np.einsum("...d,...d->...", B, C) * nA)
    D0 = -2.0 * np.arctan2(num, den)
    return S0, S1, D0, D1, h, rho, n


def linear_potentials(x, a, b, c):
    """int lambda_j(y)/R dy and int lambda_j(y) (x - y).n/R^3 dy for the three
    barycentric functions of triangle (a, b, c) (last axis j): lambda_j is linear, so
    lambda_j(y) = lambda_j(rho) + grad lambda_j . (y - rho)."""
    S0, S1, D0, D1, h, rho, n = triangle_potentials(x, a, b, c)
    a_, b_, c_ = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (a, b, c)))
    twoA = np.linalg.norm(np.cross(b_ - a_, c_ - a_), axis=-1)[..., None]
    grads = [np.cross(n, c_ - b_) / twoA, np.cross(n, a_ - c_) / twoA, np.cross(n, b_ - a_) / twoA]
    verts = [a_, b_, c_]
    IV, IK = [], []
    for j in range(3):
        lr = 1.0 + np.einsum("...d,...d->...", grads[j], rho - verts[j])
        IV.append(lr * S0 + np.einsum("...d,...d->...", grads[j], S1))
        IK.append(lr * D0 + np.einsum("...d,...d->...", grads[j], D1))
    return np.stack(IV, axis=-1), np.stack(IK, axis=-1)


# ------------------------------------------------------------------ kernels

def green(r, k):
    """G = e^{ikr}/(4 pi r), 0 where r = 0 (point pairs at zero distance are dropped)."""
    rr = np.where(r > 0.0, r, 1.0)
    return np.where(r > 0.0, np.exp(1j * k * rr) / (FOUR_PI * rr), 0.0)


def green_dny(d, ny, k):
    """dG/dn_y for d = x - y: (ikr - 1) e^{ikr} (y - x).n_y/(4 pi r^3); 0 where r = 0."""
    r = np.linalg.norm(d, axis=-1)
    rr = np.where(r > 0.0, r, 1.0)
    val = (1j * k * rr - 1.0) * np.exp(1j * k * rr) * (-np.einsum("...d,...d->...", d, ny)) / (FOUR_PI * rr ** 3)
    return np.where(r > 0.0, val, 0.0)


def green_smooth(r, k):
    """G - 1/(4 pi r) = (e^{ikr} - 1)/(4 pi r), bounded (-> ik/(4 pi) at r = 0):
    e^{ikr} - 1 = -2 sin^2(kr/2) + i sin kr."""
    rr = np.where(r > 0.0, r, 1.0)
    em1 = -2.0 * np.sin(0.5 * k * rr) ** 2 + 1j * np.sin(k * rr)
    return np.where(r > 0.0, em1 / (FOUR_PI * rr), 1j * k / FOUR_PI)


def green_smooth_dny(d, ny, k):
    """d/dn_y [G - 1/(4 pi r)] = [(ikr - 1) e^{ikr} + 1] (y - x).n_y/(4 pi r^3), bounded
    (-> -k^2 (y - x).n_y/(8 pi r)); with c = cos kr, s = sin kr the bracket is
    (2 sin^2(kr/2) - kr s) + i (kr c - s)."""
    r = np.linalg.norm(d, axis=-1)
    rr = np.where(r > 0.0, r, 1.0)
    kr = k * rr
    br = (2.0 * np.sin(0.5 * kr) ** 2 - kr * np.sin(kr)) + 1j * (kr * np.cos(kr) - np.sin(kr))
    val = br * (-np.einsum("...d,...d->...", d, ny)) / (FOUR_PI * rr ** 3)
    return np.where(r > 0.0, val, 0.0)


# ------------------------------------------------------------------ Galerkin blocks

class BemDiscretisation:
    """P1 Galerkin PMCHWT on nested interfaces.

    surfaces: list of (vert, tri), outermost first.  domains: list of dicts
    {"k": k_j, "rho": rho_j, "sides": {m: sigma_jm}}, domain 0 the exterior."""

    def __init__(self, surfaces, domains, far_order=3, near_order=4, near_factor=2.0, rho0=None):
        self.S = [Surface(v, t) for v, t in surfaces]
        self.domains = domains
        self.far_order, self.near_order, self.near_factor = int(far_order), int(near_order), float(near_factor)
        self.lam_f, self.w_f = triangle_rule(far_order)
        self.lam_n, self.w_n = triangle_rule(near_order)
        self.offsets = np.concatenate([[0], np.cumsum([2 * s.n_vert for s in self.S])])
        self.n = int(self.offsets[-1])
        self.rho0 = domains[0]["rho"] if rho0 is None else rho0
        self.k0 = domains[0]["k"]

    @classmethod
    def nested(cls, surfaces, k0, rho, c, rho0=1.0, c0=1.0, **kw):
        """Nested closed interfaces (list of (vert, tri), outermost first) with homogeneous
        layers: (rho[l], c[l]) inside interface l, down to the next; exterior (rho0, c0)."""
        omega = k0 * c0
        L = len(surfaces)
        domains = [{"k": k0, "rho": rho0, "sides": {0: -1}}]
        for l in range(L):
            sides = {l: +1}
            if l + 1 < L:
                sides[l + 1] = -1
            domains.append({"k": omega / c[l], "rho": rho[l], "sides": sides})
        return cls(surfaces, domains, rho0=rho0, **kw)

    # -- near pairs
    def near_pairs(self, m, l):
        """(T, T') index arrays of the near pairs between test surface m and trial surface
        l: a shared vertex (same surface) or |c_T - c_T'|^2 < near_factor^2 max(d_T^2, d_T'^2)."""
        A, B = self.S[m], self.S[l]
        d2 = ((A.cen[:, None, :] - B.cen[None, :, :]) ** 2).sum(-1)
        lim = self.near_factor ** 2 * np.maximum(A.diam2[:, None], B.diam2[None, :])
        near = d2 < lim
        if m == l:
            share = (A.tri[:, None, :, None] == B.tri[None, :, None, :]).any(axis=(2, 3))
            near |= share
        return np.nonzero(near)

    # -- far rule, all pairs: point-level matrices
    def _far_points(self, m):
        S = self.S[m]
        P, W = S.points(self.lam_f, self.w_f)
        return P.reshape(-1, 3), W.reshape(-1), np.repeat(np.arange(S.n_tri), len(self.w_f))

    def _point_to_vertex(self, m, weights):
        """Sparse map (n_points, n_vert): weights[T, q, i] on vertex T_i."""
        import scipy.sparse as sp
        S = self.S[m]
        Q = len(self.w_f)
        rows = np.tile(np.arange(S.n_tri * Q), 3)
        cols = np.concatenate([np.repeat(S.tri[:, i], Q) for i in range(3)])
        vals = np.concatenate([weights[:, :, i].reshape(-1) for i in range(3)])
        return sp.csr_matrix((vals, (rows, cols)), shape=(S.n_tri * Q, S.n_vert))

    def far_blocks(self, m, l, k):
        """V, K, K', W of test surface m, trial surface l, wavenumber k with the far rule on
        every triangle pair (the near correction is added separately)."""
        A, B = self.S[m], self.S[l]
        Px, Wx, Tx = self._far_points(m)
        Py, Wy, Ty = self._far_points(l)
        Q = len(self.w_f)
        lamx = np.broadcast_to(self.lam_f[None], (A.n_tri, Q, 3))
        lamy = np.broadcast_to(self.lam_f[None], (B.n_tri, Q, 3))
        Lx = self._point_to_vertex(m, lamx * Wx.reshape(A.n_tri, Q)[:, :, None])
        Ly = self._point_to_vertex(l, lamy * Wy.reshape(B.n_tri, Q)[:, :, None])
        Cx = [self._point_to_vertex(m, np.broadcast_to(A.curl[:, None, :, d], (A.n_tri, Q, 3))
                                    * Wx.reshape(A.n_tri, Q)[:, :, None]) for d in range(3)]
        Cy = [self._point_to_vertex(l, np.broadcast_to(B.curl[:, None, :, d], (B.n_tri, Q, 3))
                                    * Wy.reshape(B.n_tri, Q)[:, :, None]) for d in range(3)]
        Nx = [Lx.multiply(np.repeat(A.nrm[:, d], Q)[:, None]).tocsr() for d in range(3)]
        Ny = [Ly.multiply(np.repeat(B.nrm[:, d], Q)[:, None]).tocsr() for d in range(3)]
        nx = np.repeat(A.nrm, Q, axis=0)
        ny = np.repeat(B.nrm, Q, axis=0)
        V = np.zeros((A.n_vert, B.n_vert), dtype=np.complex128)
        K = np.zeros_like(V)
        Kp = np.zeros_like(V)
        W = np.zeros_like(V)

        def sandwich(Lt, M, R):
            return Lt.T @ (R.T @ M.T).T

        step = max(1, int(1e7 // max(1, Py.shape[0])))
        for s in range(0, Px.shape[0], step):
            e = min(Px.shape[0], s + step)
            dx = Px[s:e, None, 0] - Py[None, :, 0]
            dy = Px[s:e, None, 1] - Py[None, :, 1]
            dz = Px[s:e, None, 2] - Py[None, :, 2]
            r = np.sqrt(dx * dx + dy * dy + dz * dz)
            G = green(r, k)
            rr = np.where(r > 0.0, r, 1.0)
            # dG/dr / r = (ikr - 1) G / r^2; dG/dn_y = that * (y - x).n_y, dG/dn_x = that * (x - y).n_x
            E = (1j * k * rr - 1.0) * G / (rr * rr)
            dny = -(dx * ny[None, :, 0] + dy * ny[None, :, 1] + dz * ny[None, :, 2])
            dnx = dx * nx[s:e, None, 0] + dy * nx[s:e, None, 1] + dz * nx[s:e, None, 2]
            Lxs = Lx[s:e]
            V += sandwich(Lxs, G, Ly)
            K += sandwich(Lxs, E * dny, Ly)
            Kp += sandwich(Lxs, E * dnx, Ly)
            for dd in range(3):
                W += sandwich(Cx[dd][s:e], G, Cy[dd]) - k ** 2 * sandwich(Nx[dd][s:e], G, Ny[dd])
        return V, K, Kp, W

    # -- near pairs: exact minus far rule, as 3 x 3 blocks
    def _pair_blocks(self, A, B, T, Tp, k, lam_o, w_o, lam_i, w_i, exact):
        """V3[p, i, j] and K3[p, i, j] for test triangles T (surface A) and trial
        triangles Tp (surface B): outer rule (lam_o, w_o) on T; on Tp the closed-form static
        part plus the smooth remainder on (lam_i, w_i) if exact, else the plain rule
        (lam_i, w_i) with the full kernel."""
        va = A.vert[A.tri[T]]                      # (p, 3, 3)
        vb = B.vert[B.tri[Tp]]
        X = np.einsum("qi,pid->pqd", lam_o, va)    # (p, Qo, 3)
        WX = A.area[T][:, None] * w_o[None, :]
        Y = np.einsum("si,pid->psd", lam_i, vb)    # (p, Qi, 3)
        WY = B.area[Tp][:, None] * w_i[None, :]
        ny = B.nrm[Tp][:, None, None, :]
        d = X[:, :, None, :] - Y[:, None, :, :]    # (p, Qo, Qi, 3)
        r = np.linalg.norm(d, axis=-1)
        if exact:
            g = green_smooth(r, k)
            dg = green_smooth_dny(d, ny, k)
        else:
            g = green(r, k)
            dg = green_dny(d, ny, k)
        VI = np.einsum("pqs,ps,si->pqi", g, WY, lam_i)
        KI = np.einsum("pqs,ps,si->pqi", dg, WY, lam_i)
        if exact:
            IV, IK = linear_potentials(X, vb[:, None, 0, :], vb[:, None, 1, :], vb[:, None, 2, :])
            # a flat triangle's double-layer kernel (x - y).n_y vanishes on its own plane:
            # for coincident pairs the static part is exactly 0 (the solid angle would give
            # the one-sided limit +-2 pi at points in the plane, up to rounding of h)
            same = (T == Tp) & (A is B)
            IK = np.where(same[:, None, None], 0.0, IK)
            VI = VI + IV / FOUR_PI
            KI = KI + IK / FOUR_PI
        V3 = np.einsum("pq,qi,pqj->pij", WX, lam_o, VI)
        K3 = np.einsum("pq,qi,pqj->pij", WX, lam_o, KI)
        return V3, K3

    def near_blocks(self, m, l, k):
        """Per near pair (T, T') of test surface m and trial surface l: the correction
        (near rule - far rule) of the 3 x 3 V, K, K', W blocks.  V is the mean of the pair
        and its swap; K' is the swap's K transposed."""
        A, B = self.S[m], self.S[l]
        T, Tp = self.near_pairs(m, l)
        out = {"T": T, "Tp": Tp}
        if T.size == 0:
            return out
        args_e = (self.lam_n, self.w_n, self.lam_n, self.w_n, True)
        args_f = (self.lam_f, self.w_f, self.lam_f, self.w_f, False)
        Ve, Ke = self._pair_blocks(A, B, T, Tp, k, *args_e)
        Vs, Ks = self._pair_blocks(B, A, Tp, T, k, *args_e)          # swapped roles
        Vf, Kf = self._pair_blocks(A, B, T, Tp, k, *args_f)
        _, Ksf = self._pair_blocks(B, A, Tp, T, k, *args_f)
        dV = 0.5 * (Ve + np.swapaxes(Vs, 1, 2)) - Vf
        dK = Ke - Kf
        dKp = np.swapaxes(Ks - Ksf, 1, 2)
        cc = np.einsum("pid,pjd->pij", A.curl[T], B.curl[Tp])
        nn = np.einsum("pd,pd->p", A.nrm[T], B.nrm[Tp])
        dW = cc * dV.sum(axis=(1, 2))[:, None, None] - k ** 2 * nn[:, None, None] * dV
        out.update(V=dV, K=dK, Kp=dKp, W=dW)
        return out

    def operator_blocks(self, m, l, k):
        """Galerkin V, K, K', W (n_vert_m x n_vert_l) of wavenumber k."""
        V, K, Kp, W = self.far_blocks(m, l, k)
        nb = self.near_blocks(m, l, k)
        A, B = self.S[m], self.S[l]
        for p in range(nb["T"].size):
            ia = A.tri[nb["T"][p]]
            ib = B.tri[nb["Tp"][p]]
            ix = np.ix_(ia, ib)
            V[ix] += nb["V"][p]
            K[ix] += nb["K"][p]
            Kp[ix] += nb["Kp"][p]
            W[ix] += nb["W"][p]
        return V, K, Kp, W

    # -- the PMCHWT system
    def assemble(self, lumped=True):
        """The PMCHWT matrix on [u_1, v_1, u_2, v_2, ...] (rows scaled by 1/m_a if lumped)."""
        A = np.zeros((self.n, self.n), dtype=np.complex128)
        for dom in self.domains:
            k, rho = dom["k"], dom["rho"]
            for m, sm in dom["sides"].items():
                for l, sl in dom["sides"].items():
                    V, K, Kp, W = self.operator_blocks(m, l, k)
                    s = sm * sl
                    nm, nl = self.S[m].n_vert, self.S[l].n_vert
                    om, ol = self.offsets[m], self.offsets[l]
                    A[om:om + nm, ol:ol + nl] += -s * K
                    A[om:om + nm, ol + nl:ol + 2 * nl] += s * rho * V
                    A[om + nm:om + 2 * nm, ol:ol + nl] += s * W / rho
                    A[om + nm:om + 2 * nm, ol + nl:ol + 2 * nl] += s * Kp
        if lumped:
            A /= self.lumped_scale()[:, None]
        return A

    def lumped_scale(self):
        """m_a per unknown (u and v of each interface share the vertex's lumped mass)."""
        return np.concatenate([np.tile(s.lumped_mass(), 2) for s in self.S])

    def rhs(self, direction, lumped=True):
        """(int phi_a p_inc, int phi_a (1/rho_0) dp_inc/dn) on the outermost interface,
        p_inc = exp(i k0 x.d) (Eq. planewave), with the far rule."""
        d = np.asarray(direction, dtype=np.float64)
        d = d / np.linalg.norm(d)
        S = self.S[0]
        P, W = S.points(self.lam_f, self.w_f)
        pinc = np.exp(1j * self.k0 * (P @ d))
        dn = 1j * self.k0 * (S.nrm @ d)[:, None] * pinc / self.rho0
        b = np.zeros(self.n, dtype=np.complex128)
        for i in range(3):
            np.add.at(b, S.tri[:, i], (W * self.lam_f[None, :, i] * pinc).sum(1))
            np.add.at(b, S.n_vert + S.tri[:, i], (W * self.lam_f[None, :, i] * dn).sum(1))
        if lumped:
            b /= self.lumped_scale()
        return b

    def far_field(self, y, dirs):
        """p_inf(xhat) from the outermost interface's (u, v), far rule."""
        dirs = np.asarray(dirs, dtype=np.float64)
        S = self.S[0]
        P, W = S.points(self.lam_f, self.w_f)
        u = np.einsum("qi,ti->tq", self.lam_f, y[:S.n_vert][S.tri])
        v = np.einsum("qi,ti->tq", self.lam_f, y[S.n_vert:2 * S.n_vert][S.tri])
        k = self.k0
        ph = np.exp(-1j * k * np.einsum("md,tqd->mtq", dirs, P))
        xn = dirs @ S.nrm.T                                         # (m, t)
        amp = -1j * k * xn[:, :, None] * u[None] - self.rho0 * v[None]
        return (ph * amp * W[None]).sum(axis=(1, 2)) / FOUR_PI

    def solve(self, direction):
        return np.linalg.solve(self.assemble(), self.rhs(direction))
