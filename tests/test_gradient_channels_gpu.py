"""Gradient channels (vsie_gradient_channels) against the oracle on the small workloads:
the library's far-field source points are matched to the oracle's far-rule points by
owner and position, then Phi and Psi are compared point by point (FP64 path <= 1e-12,
FP32 path <= 1e-5, relative L2)."""
import numpy as np
import pytest

from oracle import vsie_oracle as O
from paper_2607_06429_b300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = {
    "ball12_k2": lambda: W.single_ball(12, 3, 2.0),        # four-point rule, G and K points
    "smooth8_k3": lambda: W.smooth_density_ball(8, 2, 1, 3.0),  # grad(alpha) != 0: F points
    "layered10_k5": lambda: W.layered_ball(10, 2, 2, 5.0),  # centroid rule, two interfaces
}


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_06429_b300 import binding as B
    from paper_2607_06429_b300 import build as BUILD
    BUILD.build()
    return torch, B


def _order(xyz, own):
    return np.lexsort((np.round(xyz[:, 2], 12), np.round(xyz[:, 1], 12), np.round(xyz[:, 0], 12), own))


@pytest.mark.parametrize("name", sorted(SMALL))
def test_gradient_channels_match_oracle(name):
    torch, B = _setup()
    w = SMALL[name]()
    D = O.Discretisation.from_workload(w)
    op = B.Operator.from_workload(w)
    pts_o, own_o = O.far_source_points(D)
    xyz, own, cls = op.source_points()
    assert xyz.shape == pts_o.shape
    io, ig = _order(pts_o, own_o), _order(xyz, own)
    assert np.array_equal(own_o[io], own[ig])
    assert np.abs(pts_o[io] - xyz[ig]).max() <= 1e-13
    rng = np.random.default_rng(11)
    lam = rng.normal(size=D.n) + 1j * rng.normal(size=D.n)
    phi_o, psi_o = O.gradient_channels(D, lam, pts_o)
    lam_d = torch.from_numpy(lam).cuda()
    for prec, tol in ((64, 1e-12), (32, 1e-5)):
        phi, psi = op.gradient_channels(lam_d, precision=prec)
        phi, psi = phi.cpu().numpy()[ig], psi.cpu().numpy()[ig]
        e_phi = np.linalg.norm(phi - phi_o[io]) / np.linalg.norm(phi_o)
        e_psi = np.linalg.norm(psi - psi_o[io]) / np.linalg.norm(psi_o)
        assert e_phi <= tol and e_psi <= tol, (name, prec, e_phi, e_psi)
    if name == "smooth8_k3":
        assert set(np.unique(cls)) == {0, 1, 2} or set(np.unique(cls)) == {1, 2}
