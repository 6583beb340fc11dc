"""Differentiable far-field misfit of the nested VSIE (torch.autograd.Function).

For per-tetrahedron density rho_e and sound speed c_e (geometry, exterior medium and
interface densities fixed) the forward pass solves A(rho, c) p = p_inc with the library's
GMRES, evaluates the far-field pattern u = F(rho, c) p on a set of directions and returns
L = 1/2 sum_d |u_d - t_d|^2.  The backward pass is the adjoint method:

    A^H lam = F^H r,   r = u - t,
    dL/dtheta = Re[r^H (dF/dtheta) p] - Re[lam^H (dA/dtheta) p].

A and F depend on (rho_e, c_e) through the single-layer weight
s_e = beta_e - k0^2 alpha_e = k0^2 (rho0/rho_e)((c0/c_e)^2 - 1) of column e (Eqs. alpha, beta,
vsie; every entry of that column is linear in s_e) and the mass m_e = rho0/rho_e
(Eq. mass_function).  Column e is s_e times the single-layer column of unit weight, so
dA/ds_e and dF/ds_e are the columns of an operator A_u (and its far-field map F_u) of the
same mesh with s = 1 on every tetrahedron, no interface jump and rho = rho0 (unit mass):
    dL/ds_e = Re[conj(F_u^H r - (A_u^H lam - lam))_e p_e],    dL/dm_e = -Re[conj(lam_e) p_e],
from the library's adjoint apply and far-field adjoint on A_u (near and self corrections
included), and the chain rule through s_e(rho_e, c_e) and m_e(rho_e) gives the gradients.
No division by s_e occurs, so elements without contrast (c_e = c0, s_e = 0) and elements
near it are covered.

Without a density-gradient term (piecewise-constant density per element, grad(alpha) = 0)
the column of element e scales as 1/rho_e as a whole, so p_e absorbs rho_e and the far field
does not depend on it: dL/drho vanishes identically in this discrete model.

With the least-squares density gradient (workload flag grad_alpha_lsq), grad(alpha) = W alpha
over face neighbours (the library's stencil), so rho_e also enters the adjoint double layer
of its neighbours.  The backward pass then takes per-unit-weight channels from operators of
the same mesh carrying one unit weight (s = 1, or grad(alpha) along one axis) on every
tetrahedron: every column is linear in its element's weights, so their adjoint applies and
far-field adjoints give dL/ds_e and dL/dgrad(alpha)_e exactly (near and self corrections
included), and dL/dalpha = W^T dL/dgrad(alpha) (vsie_lsq_grad_alpha_adjoint).
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class FarFieldMisfit(torch.autograd.Function):
    """L(rho, c) for a workload's geometry; rho, c: CPU float64 tensors of length n_tet."""

    @staticmethod
    def forward(ctx, rho, c, workload, dirs, target, direction, solve_kw):
        w = workload
        lsq = bool(getattr(w, "grad_alpha_lsq", False))
        rho_np = rho.detach().numpy()
        ga = B.lsq_grad_alpha(w.vert, w.tet, w.tet_domain, w.rho0 / rho_np - 1.0) if lsq else None
        op = B.Operator(w.vert, w.tet, w.tri, rho_np, c.detach().numpy(), w.tri_rho_in,
                        w.tri_rho_out, w.k0, w.rho0, w.c0, ga, w.tet_far_points, w.near_radius,
                        w.tri_near_radius)
        b = op.plane_wave_rhs([direction])[0].contiguous()
        p, _ = op.solve(b, **solve_kw)
        u = op.far_field(p, dirs)
        t = torch.as_tensor(np.asarray(target), dtype=torch.complex128, device=u.device)
        r = (u - t).contiguous()
        loss = 0.5 * float((r.abs() ** 2).sum().item())
        ctx.op, ctx.p, ctx.r, ctx.dirs, ctx.solve_kw = op, p, r, dirs, solve_kw
        ctx.k0, ctx.rho0, ctx.c0, ctx.n_tet = w.k0, w.rho0, w.c0, w.n_tet
        ctx.w, ctx.lsq = w, lsq
        ctx.save_for_backward(rho, c)
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_loss):
        rho, c = ctx.saved_tensors
        op, p, r, nt = ctx.op, ctx.p, ctx.r, ctx.n_tet
        g = op.far_field_adjoint(r, ctx.dirs)
        lam, _ = op.solve(g.contiguous(), adjoint=True, **ctx.solve_kw)
        prec = 64 if ctx.solve_kw.get("mode", 32) == 64 else 32
        rho_d = rho.to(device=p.device)
        c_d = c.to(device=p.device)
        m = ctx.rho0 / rho_d
        s = ctx.k0 ** 2 * (ctx.rho0 / rho_d) * ((ctx.c0 / c_d) ** 2 - 1.0)
        dLdm = -(torch.conj(lam[:nt]) * p[:nt]).real
        ds_drho = -s / rho_d
        ds_dc = -2.0 * ctx.k0 ** 2 * (ctx.rho0 / rho_d) * ctx.c0 ** 2 / c_d ** 3
        dm_drho = -ctx.rho0 / rho_d ** 2
        if not ctx.lsq:
            dLds = _unit_channels(ctx.w, lam, r, p, ctx.dirs, prec, density_axes=False)[0]
            grad_rho = dLds * ds_drho + dLdm * dm_drho
        else:
            chans = _unit_channels(ctx.w, lam, r, p, ctx.dirs, prec)
            dLds = chans[0]
            dLdga = torch.stack(chans[1:], dim=1).cpu().numpy()          # dL/dgrad(alpha)
            dLda = B.lsq_grad_alpha_adjoint(ctx.w.vert, ctx.w.tet, ctx.w.tet_domain, dLdga)
            dLda = torch.as_tensor(dLda, dtype=torch.float64, device=p.device)
            grad_rho = dLds * ds_drho + dLdm * dm_drho + dLda * dm_drho    # d alpha/d rho = d m/d rho
        grad_c = (dLds * ds_dc).cpu() * grad_loss
        grad_rho = grad_rho.cpu() * grad_loss
        op.close()
        return grad_rho, grad_c, None, None, None, None, None


def _unit_channels(w, lam, r, p, dirs, prec, density_axes=True):
    """Per-unit-weight derivative channels Re[conj(F_u^H r - (A_u^H lam - lam)) p] on the
    tetrahedra for the unit single-layer weight (s = 1) and, with density_axes, the unit
    density gradient along x, y, z: A_u, F_u are the operator and far-field map of the same
    mesh with that unit weight on every tetrahedron, no interface jump and unit mass
    (rho = rho0), so that every column carries exactly d(column)/d(weight), near and self
    corrections included."""
    import torch
    nt = w.n_tet
    one = np.full(nt, w.rho0)
    tri_one = np.full(w.n_tri, w.rho0)
    c_s = np.full(nt, w.c0 / np.sqrt(1.0 + 1.0 / w.k0 ** 2))   # s = k0^2((c0/c)^2 - 1) = 1
    variants = [(c_s, None)]
    for ax in (range(3) if density_axes else ()):
        ga = np.zeros((nt, 3))
        ga[:, ax] = 1.0
        variants.append((np.full(nt, w.c0), ga))                 # s = 0, grad(alpha) = e_ax
    out = []
    for cv, ga in variants:
        u = B.Operator(w.vert, w.tet, w.tri, one, cv, tri_one, tri_one, w.k0, w.rho0, w.c0, ga,
                       w.tet_far_points, w.near_radius, w.tri_near_radius)
        wu = u.adjoint_apply(lam, precision=prec) - lam
        gu = u.far_field_adjoint(r, dirs)
        out.append((torch.conj(gu[:nt] - wu[:nt]) * p[:nt]).real)
        u.close()
    return out


def far_field_misfit(rho, c, workload, dirs, target, direction=(1.0, 0.0, 0.0), **solve_kw):
    """Differentiable L(rho, c); solve_kw go to Operator.solve (default: mixed mode,
    tolerance 1e-10)."""
    kw = dict(mode=32, tol=1e-10, max_iters=2000, inner_tol=1e-4, max_refinements=30)
    kw.update(solve_kw)
    return FarFieldMisfit.apply(rho, c, workload, np.asarray(dirs, dtype=np.float64), target,
                                tuple(direction), kw)


class CuboidFarFieldMisfit(torch.autograd.Function):
    """L(c) on a cuboid grid (the paper's discretisation) for per-cell sound speed c; the
    density (and with it the interface faces, which exist where the density jumps) stays
    fixed.  c enters only the cell weights s_e = (rho0/rho_e)((omega/c_e)^2 - k0^2) (Eqs.
    alpha, beta), every entry of a cell's column (self term included) and of its far-field
    column being linear in s_e.  dL/ds_e comes from an operator of the same grid with s = 1
    on every cell (c_u = omega / sqrt(k0^2 + rho_e/rho0), same density, so the same faces and
    mass): dL/ds_e = Re[conj(F_u^H r - (A_u^H lam - m lam))_e p_e], which also covers cells
    without contrast (s_e = 0)."""

    @staticmethod
    def forward(ctx, c, workload, dirs, target, direction, solve_kw):
        w = workload
        cw = _with_c(w, c.detach().numpy())
        op = B.Operator.from_cuboid(cw)
        b = op.plane_wave_rhs([direction])[0].contiguous()
        p, _ = op.solve(b, **solve_kw)
        u = op.far_field(p, dirs)
        t = torch.as_tensor(np.asarray(target), dtype=torch.complex128, device=u.device)
        r = (u - t).contiguous()
        loss = 0.5 * float((r.abs() ** 2).sum().item())
        ctx.op, ctx.p, ctx.r, ctx.dirs, ctx.solve_kw, ctx.w = op, p, r, dirs, solve_kw, w
        ctx.save_for_backward(c)
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_loss):
        (c,) = ctx.saved_tensors
        op, p, r, w = ctx.op, ctx.p, ctx.r, ctx.w
        nc = w.n_cells
        g_adj = op.far_field_adjoint(r, ctx.dirs)
        lam, _ = op.solve(g_adj.contiguous(), adjoint=True, **ctx.solve_kw)
        prec = 64 if ctx.solve_kw.get("mode", 32) == 64 else 32
        rho = np.asarray(w.rho, dtype=np.float64).reshape(-1)
        omega = w.k0 * w.c0
        unit = B.Operator.from_cuboid(_with_c(w, (omega / np.sqrt(w.k0 ** 2 + rho / w.rho0)).reshape(w.shape)))
        m = torch.as_tensor(w.rho0 / rho, dtype=torch.float64, device=p.device)
        wu = unit.adjoint_apply(lam, precision=prec)[:nc] - m * lam[:nc]
        gu = unit.far_field_adjoint(r, ctx.dirs)[:nc]
        dLds = (torch.conj(gu - wu) * p[:nc]).real
        cc = c.to(device=p.device, dtype=torch.float64)
        ds_dc = -2.0 * m * omega ** 2 / cc ** 3
        unit.close()
        op.close()
        return (dLds * ds_dc).cpu() * grad_loss, None, None, None, None, None


def _with_c(w, c):
    import dataclasses
    return dataclasses.replace(w, c=np.asarray(c, dtype=np.float64).reshape(w.shape))


def cuboid_far_field_misfit(c, workload, dirs, target, direction=(1.0, 0.0, 0.0), **solve_kw):
    """Differentiable L(c) on a cuboid grid; c: CPU float64 tensor of the n_cells sound
    speeds in cell order; solve_kw go to Operator.solve (default: mixed mode, 1e-10)."""
    kw = dict(mode=32, tol=1e-10, max_iters=2000, inner_tol=1e-4, max_refinements=30)
    kw.update(solve_kw)
    return CuboidFarFieldMisfit.apply(c, workload, np.asarray(dirs, dtype=np.float64), target,
                                      tuple(direction), kw)
