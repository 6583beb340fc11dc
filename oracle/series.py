"""Closed-form and series solutions used to pin the oracle (test infrastructure only).

Everything here is derived from the Helmholtz transmission problem of Sec. 2.1
(Eqs. helmholtz_exterior ... sommerfeld, time convention e^{-i omega t}, outgoing
e^{+ikr}) and from the Green's function of Eq. (greens_function), independently of the
discretised operator in ``vsie_oracle``.

* ``ball_newton_potential``: u(x) = int_{|y|<a} G_k(x, y) dy (Newton potential, Sec. 2.2,
  Eq. theorem_convolution, with unit density), from the addition theorem
  G = i k sum_n j_n(k r<) h_n(k r>) sum_m Y_nm Y_nm^*: only n = 0 survives.
* ``sphere_double_layer_of_one``: int_{|y|=a} dG/dn_y dS_y, n outward (the double-layer
  operator of Eq. vsie applied to the constant 1).
* ``layered_sphere_field``: spherical-harmonic series for a plane wave hitting concentric
  homogeneous layers (the analytic benchmark of Sec. 3.2 generalised to a density jump
  and to two layers): continuity of p and of (1/rho) dp/dr on every interface
  (Eqs. transmission_pressure, transmission_velocity).
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def ball_newton_potential(r, a: float, k: float):
    """Newton potential of the unit density on the ball |y| < a at distance r from the
    centre.  Inside: [e^{ika}(1 - ika) j0(kr) - 1]/k^2.  Outside:
    (sin ka - ka cos ka)/k^3 * e^{ikr}/r."""
    r = np.asarray(r, dtype=np.float64)
    ka = k * a
    inside = (np.exp(1j * ka) * (1.0 - 1j * ka) * spherical_jn(0, k * r) - 1.0) / k ** 2
    rr = np.where(r > 0, r, 1.0)
    outside = (np.sin(ka) - ka * np.cos(ka)) / k ** 3 * np.exp(1j * k * rr) / rr
    return np.where(r < a, inside, outside)


def ball_newton_potential_grad_r(r, a: float, k: float):
    """d/dr of the interior Newton potential (r < a):
    e^{ika}(1 - ika)/k^2 * d/dr j0(kr) = -e^{ika}(1 - ika) j1(kr)/k."""
    r = np.asarray(r, dtype=np.float64)
    ka = k * a
    return -np.exp(1j * ka) * (1.0 - 1j * ka) * spherical_jn(1, k * r) / k


def sphere_double_layer_of_one(r, a: float, k: float):
    """int_{|y|=a} dG_k(x,y)/dn_y dS_y for |x| = r.  Inside: j0(kr) e^{ika} (ika - 1)
    (-> -1 as k -> 0, Gauss).  Outside: e^{ikr} (ka cos ka - sin ka)/(kr) (-> 0)."""
    r = np.asarray(r, dtype=np.float64)
    ka = k * a
    inside = spherical_jn(0, k * r) * np.exp(1j * ka) * (1j * ka - 1.0)
    rr = np.where(r > 0, r, 1.0)
    outside = np.exp(1j * k * rr) * (ka * np.cos(ka) - np.sin(ka)) / (k * rr)
    return np.where(r < a, inside, outside)


def _h1(n, z, derivative=False):
    return spherical_jn(n, z, derivative) + 1j * spherical_yn(n, z, derivative)


def layered_sphere_coefficients(k0: float, radii, rho, c, rho0=1.0, c0=1.0, nmax=None):
    """Coefficients for concentric homogeneous layers.

    radii: decreasing interface radii [R_1, R_2, ...]; layer l (1-based) lies between
    R_{l+1} and R_l with density rho[l-1] and speed c[l-1].  Incident plane wave
    sum_n (2n+1) i^n j_n(k0 r) P_n(cos g).  Field representation:
      exterior   : (2n+1) i^n j_n(k0 r) + A_n h_n(k0 r)
      layer l < L: D_ln j_n(k_l r) + E_ln y_n(k_l r)
      innermost  : D_Ln j_n(k_L r)
    Unknowns solved per order n from 2 conditions per interface."""
    radii = list(radii)
    L = len(radii)
    omega = k0 * c0
    ks = [omega / cl for cl in c]
    if nmax is None:
        nmax = int(max([k0 * radii[0]] + [ks[i] * radii[i] for i in range(L)])) + 25
    coefs = []
    for n in range(nmax + 1):
        inc = (2 * n + 1) * (1j ** n)
        nu = 1 + 2 * (L - 1) + 1          # A, (D,E) per inner non-core layer, D core
        M = np.zeros((2 * L, nu), dtype=np.complex128)
        rhs = np.zeros(2 * L, dtype=np.complex128)

        def cols(layer):
            # column indices of (D, E) of layer ``layer`` (1-based); core has only D
            base = 1 + 2 * (layer - 1)
            return (base, base + 1) if layer < L else (base, None)

        for i, R in enumerate(radii):
            outer = i          # layer outside interface i (0 = exterior)
            inner = i + 1
            row_p, row_v = 2 * i, 2 * i + 1
            # outer side
            if outer == 0:
                z = k0 * R
                rhs[row_p] -= inc * spherical_jn(n, z)
                rhs[row_v] -= inc * (k0 / rho0) * spherical_jn(n, z, True)
                M[row_p, 0] += _h1(n, z)
                M[row_v, 0] += (k0 / rho0) * _h1(n, z, True)
            else:
                kk, rr = ks[outer - 1], rho[outer - 1]
                z = kk * R
                cd, ce = cols(outer)
                M[row_p, cd] += spherical_jn(n, z)
                M[row_v, cd] += (kk / rr) * spherical_jn(n, z, True)
                M[row_p, ce] += spherical_yn(n, z)
                M[row_v, ce] += (kk / rr) * spherical_yn(n, z, True)
            # inner side (moved to the left with a minus sign)
            kk, rr = ks[inner - 1], rho[inner - 1]
            z = kk * R
            cd, ce = cols(inner)
            M[row_p, cd] -= spherical_jn(n, z)
            M[row_v, cd] -= (kk / rr) * spherical_jn(n, z, True)
            if ce is not None:
                M[row_p, ce] -= spherical_yn(n, z)
                M[row_v, ce] -= (kk / rr) * spherical_yn(n, z, True)
        coefs.append(np.linalg.solve(M, rhs))
    return dict(coefs=coefs, ks=ks, radii=radii, k0=k0, L=L)


def layered_sphere_field(x, direction, k0: float, radii, rho, c, rho0=1.0, c0=1.0,
                         nmax=None):
    """Total pressure at points x (m, 3) for the incident plane wave exp(i k0 x.d)."""
    cf = layered_sphere_coefficients(k0, radii, rho, c, rho0, c0, nmax)
    x = np.asarray(x, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    r = np.linalg.norm(x, axis=1)
    cosg = np.where(r > 0, (x @ d) / np.where(r > 0, r, 1.0), 1.0)
    radii = cf["radii"]
    L = cf["L"]
    layer = np.zeros(r.shape[0], dtype=np.int64)
    for i, R in enumerate(radii):
        layer[r < R] = i + 1
    out = np.zeros(r.shape[0], dtype=np.complex128)
    for n, co in enumerate(cf["coefs"]):
        P = eval_legendre(n, cosg)
        m0 = layer == 0
        if m0.any():
            z = k0 * r[m0]
            out[m0] += ((2 * n + 1) * (1j ** n) * spherical_jn(n, z) + co[0] * _h1(n, z)) * P[m0]
        for l in range(1, L + 1):
            ml = layer == l
            if not ml.any():
                continue
            z = cf["ks"][l - 1] * r[ml]
            base = 1 + 2 * (l - 1)
            val = co[base] * spherical_jn(n, z)
            if l < L:
                val = val + co[base + 1] * spherical_yn(n, z)
            out[ml] += val * P[ml]
    return out


def layered_sphere_far_field(xhat, direction, k0: float, radii, rho, c, rho0=1.0, c0=1.0,
                             nmax=None):
    """Far-field pattern p_inf with p_s ~ e^{ik0 R}/R p_inf(xhat): since
    h_n(z) ~ (-i)^{n+1} e^{iz}/z, p_inf = sum_n A_n (-i)^{n+1}/k0 P_n(xhat.d)."""
    cf = layered_sphere_coefficients(k0, radii, rho, c, rho0, c0, nmax)
    xhat = np.asarray(xhat, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    cosg = xhat @ d
    out = np.zeros(xhat.shape[0], dtype=np.complex128)
    for n, co in enumerate(cf["coefs"]):
        out += co[0] * ((-1j) ** (n + 1)) / k0 * eval_legendre(n, cosg)
    return out
