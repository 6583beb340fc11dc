"""The nested PMCHWT boundary element path of the library (vsie_bem_*) against the FP64
oracle (oracle/bem_oracle.py): the preconditioned operator applied to seeded vectors
(every entry of the result), the near-pair lists, the right-hand side, the far field and
the solution; on finer meshes, against the layered-sphere series."""
import numpy as np
import pytest

from oracle import bem_oracle as BO
from oracle import series
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu

RADII, RHO, C, K0 = [1.0, 0.5], [1.5, 3.0], [0.8, 0.6], 3.0


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return torch, B


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


CASES = {
    "nested_ico2_ico1": dict(subdiv=(2, 1), radii=RADII, rho=RHO, c=C),
    "single_ico2": dict(subdiv=(2,), radii=[1.0], rho=[1.5], c=[0.8]),
    "nested_ico1_far2_near5": dict(subdiv=(1, 1), radii=RADII, rho=RHO, c=C, far_order=2, near_order=5,
                                   near_factor=1.5),
}


def _pair(case):
    torch, B = _setup()
    p = dict(CASES[case])
    kw = {k: p.pop(k) for k in ("far_order", "near_order", "near_factor") if k in p}
    op = B.BemOperator.nested_spheres(p["subdiv"], p["radii"], K0, p["rho"], p["c"], **kw)
    D = BO.BemDiscretisation.nested([W.icosphere(sd, R) for sd, R in zip(p["subdiv"], p["radii"])], K0,
                                    p["rho"], p["c"], **kw)
    return torch, B, op, D


@pytest.mark.parametrize("case", list(CASES))
def test_bem_apply_matches_the_oracle_matrix(case):
    torch, B, op, D = _pair(case)
    assert op.n == D.n
    A = D.assemble()
    for seed in (1, 2):
        x = W.random_vector(D.n, 700 + seed)
        ref = A @ x
        xd = torch.from_numpy(x).cuda()
        y64 = op.apply(xd, precision=64).cpu().numpy()
        y48 = op.apply(xd, precision=48).cpu().numpy()
        y32 = op.apply(xd, precision=32).cpu().numpy()
        assert _rel(y64, ref) <= 1e-11
        assert _rel(y48, ref) <= 1e-11
        assert _rel(y32, ref) <= 2e-6
        # entry by entry: the largest error relative to the row scale
        assert np.max(np.abs(y64 - ref)) <= 1e-10 * np.max(np.abs(ref))
        assert np.max(np.abs(y48 - ref)) <= 1e-10 * np.max(np.abs(ref))
    # deterministic
    assert torch.equal(op.apply(xd, precision=32), op.apply(xd, precision=32))


@pytest.mark.parametrize("case", list(CASES))
def test_bem_near_pairs_rhs_and_far_field_match_the_oracle(case):
    torch, B, op, D = _pair(case)
    n_near = 0
    for m in range(len(D.S)):
        for l in range(len(D.S)):
            if any(m in dom["sides"] and l in dom["sides"] for dom in D.domains):
                n_near += D.near_pairs(m, l)[0].size
    assert op.n_near_pairs == n_near
    b = op.rhs([1.0, 0.3, -0.2]).cpu().numpy()
    assert _rel(b, D.rhs([1.0, 0.3, -0.2])) <= 1e-13
    dirs = W.fibonacci_dirs(24)
    x = W.random_vector(D.n, 9)
    ff = op.far_field(torch.from_numpy(x).cuda(), dirs).cpu().numpy()
    assert _rel(ff, D.far_field(x, dirs)) <= 1e-13


def test_bem_solve_matches_the_oracle_solution_and_the_series():
    torch, B, op, D = _pair("nested_ico2_ico1")
    y_ref = D.solve([1.0, 0.0, 0.0])
    b = op.rhs([1.0, 0.0, 0.0])
    x64, info64 = op.solve(b, mode=64, tol=1e-12, max_iters=800)
    x32, info32 = op.solve(b, mode=32, tol=1e-10, max_iters=800)
    assert info64.rel_residual <= 1e-12 and info32.rel_residual <= 1e-10
    assert info32.refinements >= 1 and info32.fp32_applies > info32.fp64_applies
    assert _rel(x64.cpu().numpy(), y_ref) <= 1e-9
    assert _rel(x32.cpu().numpy(), y_ref) <= 1e-8
    dirs = W.fibonacci_dirs(32)
    ff = op.far_field(x32, dirs).cpu().numpy()
    ref = series.layered_sphere_far_field(dirs, [1, 0, 0], K0, RADII, RHO, C)
    e_gpu, e_oracle = _rel(ff, ref), _rel(D.far_field(y_ref, dirs), ref)
    assert abs(e_gpu - e_oracle) <= 1e-6 and e_gpu < 0.08


def test_bem_converges_to_the_layered_sphere_series_on_finer_meshes():
    torch, B = _setup()
    dirs = W.fibonacci_dirs(64)
    ref = series.layered_sphere_far_field(dirs, [1, 0, 0], K0, RADII, RHO, C)
    errs, iters = [], []
    for sub in ((3, 2), (4, 3)):
        op = B.BemOperator.nested_spheres(sub, RADII, K0, RHO, C)
        x, info = op.solve(op.rhs([1.0, 0.0, 0.0]), mode=32, tol=1e-6, max_iters=2000)
        errs.append(_rel(op.far_field(x, dirs).cpu().numpy(), ref))
        iters.append(info.iterations)
        op.close()
    assert errs[0] < 0.02 and errs[1] < 0.006 and errs[0] / errs[1] > 3.0


def test_bem_errors_are_reported_without_device_faults():
    torch, B = _setup()
    v, t = W.icosphere(1, 1.0)
    v = np.array(v)
    v[t[3, 1]] = v[t[3, 0]]                 # collapse one triangle to zero area
    with pytest.raises(B.VsieError) as e:
        B.BemOperator([(v, t)], 2.0, [1.5], [0.8])
    assert e.value.status == 2 and "zero area" in str(e.value)
    op = B.BemOperator.nested_spheres((1,), [1.0], 2.0, [1.5], [0.8])
    x = torch.from_numpy(W.random_vector(op.n, 3)).cuda()
    with pytest.raises(B.VsieError):
        op.apply(x, precision=33)
    with pytest.raises(B.VsieError):
        op.apply(x, y=x, precision=32)     # aliased
    with pytest.raises(B.VsieError):
        op.rhs([0.0, 0.0, 0.0])
    # the handle still works after the rejected calls
    y = op.apply(x, precision=64)
    assert torch.isfinite(torch.view_as_real(y)).all()


def test_vsie_and_bem_agree_on_the_same_layered_ball():
    """The paper's comparison for piecewise-constant layers (its benchmark 2): the VSIE on
    a tetrahedral layered ball and the PMCHWT BEM on icosphere interfaces solve the same
    transmission problem; their far fields agree to within their discretisation errors,
    which both shrink against the layered-sphere series."""
    torch, B = _setup()
    dirs = W.fibonacci_dirs(64)
    ref = series.layered_sphere_far_field(dirs, [1, 0, 0], K0, RADII, RHO, C)
    bem = B.BemOperator.nested_spheres((4, 3), RADII, K0, RHO, C)
    xb, _ = bem.solve(bem.rhs([1.0, 0.0, 0.0]), mode=32, tol=1e-6, max_iters=2000)
    ff_bem = bem.far_field(xb, dirs).cpu().numpy()
    bem.close()
    w = W.layered_ball(32, 4, 3, K0, R2=RADII[1], rho1=RHO[0], c1=C[0], rho2=RHO[1], c2=C[1])
    op = B.Operator.from_workload(w)
    p, _ = op.solve(op.plane_wave_rhs([1.0, 0.0, 0.0])[0].contiguous(), mode=32, tol=1e-6)
    ff_vsie = op.far_field(p, dirs).cpu().numpy()
    op.close()
    e_bem, e_vsie, d = _rel(ff_bem, ref), _rel(ff_vsie, ref), _rel(ff_vsie, ff_bem)
    assert e_bem < 0.006 and e_vsie < 0.03
    assert d < 0.02


def test_bem_and_cuboid_vsie_agree_on_the_papers_nested_cubes():
    """The paper's density benchmark (Sec. 3: cubes of 7 and 5 mm, rho2 = rho0/2,
    c1 = c2 = c0/1.2, lambda0 = 3 mm), where it compares its VSIE with a BEM: the library's
    cuboid VSIE (the paper's discretisation) against its PMCHWT BEM on triangulated cube
    surfaces.  Only ratios of densities and speeds enter, so the BEM takes them scaled to
    rho0 = c0 = 1.  As both refine, their far fields approach each other."""
    torch, B = _setup()
    d = [1.0, 0.0, 0.0]
    dirs = W.fibonacci_dirs(64)
    k0 = 2.0 * np.pi / 3.0
    ff_vsie = {}
    for h in (0.25, 0.125):
        op = B.Operator.from_cuboid(W.nested_cubes(h))
        x, info = op.solve(op.plane_wave_rhs(np.array(d))[0], mode=32, tol=1e-8)
        assert info.rel_residual <= 1e-8
        ff_vsie[h] = op.far_field(x, dirs).cpu().numpy()
        op.close()
    ff_bem = {}
    for n1, n2 in ((14, 10), (28, 20)):
        bem = B.BemOperator([W.cube_surface(n1, 3.5), W.cube_surface(n2, 2.5)], k0, [1.0, 0.5],
                            [1.0 / 1.2, 1.0 / 1.2], rho0=1.0, c0=1.0)
        xb, info = bem.solve(bem.rhs(d), mode=32, tol=1e-6, max_iters=3000)
        assert info.rel_residual <= 1e-6
        ff_bem[n1] = bem.far_field(xb, dirs).cpu().numpy()
        bem.close()
    coarse, fine = _rel(ff_bem[14], ff_vsie[0.125]), _rel(ff_bem[28], ff_vsie[0.125])
    print(f"nested cubes: BEM (h = 0.5 / 0.25 mm) vs cuboid VSIE (h = 0.125 mm) far field "
          f"{coarse:.4e} / {fine:.4e}; VSIE h = 0.25 vs 0.125 {_rel(ff_vsie[0.25], ff_vsie[0.125]):.4e}; "
          f"BEM coarse vs fine {_rel(ff_bem[14], ff_bem[28]):.4e}")
    assert fine < coarse and fine < 0.03
