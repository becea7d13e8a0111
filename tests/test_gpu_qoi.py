"""The quantity-of-interest sweeps of Sec. 3.6 on the GPU: every parameter
value a geometry of one batch, solved together (batch_heat_setup with an
infinite time step: the steady problem Lap u = 3, u = 0 on the ellipse) and
reduced by batch_weighted_sum; checked against the oracle's direct solves
(rel <= 1e-8 with the GPU at rtol 1e-11: kappa ~ 1/h^2 ~ 1e4 bounds the
solution error), the closed forms and the mirror symmetries."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import eb_inputs as ei
from oracle import eb as oeb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _sweep(cases, weight_fn):
    import paper_2204_06083_gb300 as eb
    grids = [g for g, _ in cases]
    lss = [l for _, l in cases]
    B = eb.Batch(grids, lss)
    B.heat_setup([math.inf] * len(cases), theta=1.0)
    f = B.zeros()
    w = B.zeros()
    for g, gr in enumerate(grids):
        B.view(f, g).fill_(ei.QOI_F)
        B.view(w, g).copy_(torch.tensor(weight_fn(gr)))
    ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device="cuda")
    b = B.rhs(f, ug)
    u = B.zeros()
    st = B.heat_step(u, b, rtol=1e-11, maxit=1000, allow_noconv=True)
    assert all(s.converged for s in st), [(s.iterations, s.rel_residual, s.true_rel_residual) for s in st]
    q = B.weighted_sum(w, u).cpu().numpy()
    ref = []
    for gr, ls in cases:
        s = oeb.build(gr, ls)
        bb = oeb.rhs(s, np.full(gr.shape(), ei.QOI_F), np.zeros(s.cut_cp.size))
        x = spla.spsolve(s.A.tocsc(), bb)
        ref.append(float(s.to_grid(x).reshape(-1) @ weight_fn(gr).reshape(-1)))
    return q, np.array(ref)


def test_ellipse_sweep_u00():
    a = np.exp(np.linspace(math.log(0.5), math.log(2.0), 9))
    a = np.concatenate([a[:4], [1.0], a[5:]])
    cases = [ei.qoi_ellipse(p, 1.0 / p) for p in a] + [ei.qoi_ellipse(1.0 / p, p) for p in a]
    q, ref = _sweep(cases, lambda gr: ei.qoi_point_weights(gr, 0.0, 0.0))
    assert np.all(np.abs(q - ref) <= 1e-8 * np.abs(ref))
    k = len(a)
    assert np.all(np.abs(q[:k] - q[k:]) <= 1e-8 * np.abs(q[:k]))      # u(0,0) for a and 1/a
    assert int(np.argmin(q[:k])) == 4                                 # extreme at the circle
    exact = np.array([ei.qoi_ellipse_exact(p, 1.0 / p) for p in a])
    assert np.all(np.abs(q[:k] - exact) <= 2e-3 * np.abs(exact))


def test_rotated_ellipse_sweep_integral():
    th = np.linspace(0.0, 2.0 * math.pi, 8, endpoint=False) + 0.1
    cases = [ei.qoi_rotated(t) for t in th] + [ei.qoi_rotated(-t) for t in th]
    q, ref = _sweep(cases, ei.qoi_rect_weights)
    assert np.all(np.abs(q - ref) <= 1e-8 * np.abs(ref))
    k = len(th)
    assert np.all(np.abs(q[:k] - q[k:]) <= 1e-8 * np.abs(q[:k]))      # theta and -theta
    exact = np.array([ei.qoi_rotated_exact(t) for t in th])
    assert np.all(np.abs(q[:k] - exact) <= 0.03 * np.abs(exact))
