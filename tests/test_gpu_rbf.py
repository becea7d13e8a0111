"""GPU parity of the mixed and RBF-based closures (Sec. 2.2-2.3, Algorithm 2)
against the oracle, through the C ABI (eb_build_ex, eb_rbf_cuts).

The nearest points come from sampling and Newton's method on the boundary
curve with the device's sin / cos, whose last-ulp results differ from the
host's: points within 1e-12 (domain units), weights within 1e-9 (the 6 x 6
saddle systems amplify the points' rounding by their condition number), the
diagonal and the right-hand side within 1e-9 relative; the RBF cut list and
Algorithm 2's branch identical; solutions within 1e-9 when both sides solve
to rtol 1e-13.
"""
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


CASES = {
    "star258_01": lambda: (ei.box_grid(2, 258), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])),
    "star402_02": lambda: ei.helmholtz_star(402),
    "ellipse200": lambda: (ei.box_grid(2, 200), ei.ellipsoid((0.013, -0.021), (0.8, 0.35), np.array(
        [[np.cos(0.4), np.sin(0.4), 0], [-np.sin(0.4), np.cos(0.4), 0], [0, 0, 1]]))),
}


def _pair(name, closure):
    import paper_2204_06083_gb300 as eb
    grid, ls = CASES[name]()
    mode = {"mixed": eb.EB_CLOSURE_MIXED, "rbf": eb.EB_CLOSURE_RBF}[closure]
    h = eb.EB(grid, ls, closure=mode)
    ref = oeb.build(grid, ls, closure=closure)
    return eb, grid, ls, h, ref


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("closure", ["mixed", "rbf"])
def test_rbf_build_parity(name, closure):
    eb, grid, ls, h, ref = _pair(name, closure)
    assert h.info.num_cut == ref.cut_cp.size and h.info.num_rbf == ref.rbf_cut.size
    assert h.info.num_rbf_rotated == int(ref.rbf_rot.sum())
    idx, xg2, w, rot = h.rbf_cuts()
    assert np.array_equal(idx.cpu().numpy(), ref.rbf_cut)
    assert np.array_equal(rot.cpu().numpy().astype(bool), ref.rbf_rot)
    assert np.abs(xg2.cpu().numpy() - ref.rbf_xg2).max() <= 1e-12
    _, _, delta, xg = h.cuts()
    assert np.abs(xg.cpu().numpy() - ref.cut_xg).max() <= 1e-12
    w = w.cpu().numpy()
    assert np.abs(w[:, 1] - ref.cut_w1[ref.rbf_cut]).max() <= 1e-9
    assert np.abs(w[:, 2] - ref.rbf_w2).max() <= 1e-9
    assert np.abs((1.0 - w[:, 0]) - ref.cut_c[ref.rbf_cut]).max() <= 1e-9
    _, diag = h.cp_data()
    assert np.abs(diag.cpu().numpy() - ref.diag).max() <= 1e-9
    assert abs(h.info.min_dominance_margin - oeb.dominance_margin(ref)) <= 1e-9
    X, Y = ei.grid_points(grid)
    pts = ref.sample_points()
    ug = ei.u_k1(pts[:, 0], pts[:, 1])
    b = h.rhs(torch.tensor(ei.f_k1(X, Y), device="cuda"), torch.tensor(ug, device="cuda")).cpu().numpy()
    b_ref = oeb.rhs(ref, ei.f_k1(X, Y), ug)
    assert np.abs(ref.from_grid(b) - b_ref).max() <= 1e-9 * np.abs(b_ref).max()


@pytest.mark.parametrize("name", ["star258_01", "star402_02"])
def test_mixed_closure_solution_parity_and_accuracy(name):
    eb, grid, ls, h, ref = _pair(name, "mixed")
    X, Y = ei.grid_points(grid)
    pts = h.sample_points().cpu().numpy()
    b = h.rhs(torch.tensor(ei.f_k1(X, Y), device="cuda"), torch.tensor(ei.u_k1(pts[:, 0], pts[:, 1]), device="cuda"))
    x, st = eb.AMG(h, 0.0).solve(b, rtol=1e-13, maxit=500)
    pr = ref.sample_points()
    b_ref = oeb.rhs(ref, ei.f_k1(X, Y), ei.u_k1(pr[:, 0], pr[:, 1]))
    x_ref = spla.spsolve(ref.A.tocsc(), b_ref)
    got = ref.from_grid(x.cpu().numpy())
    assert np.linalg.norm(got - x_ref) / np.linalg.norm(x_ref) <= 1e-9
    err = np.abs(got - ei.u_k1(X, Y).reshape(-1)[ref.cp_nodes]).max()
    print(f"{name}: mixed closure, {h.info.num_rbf} RBF cuts, max error {err:.2e}")


def test_mixed_closure_with_beta():
    import paper_2204_06083_gb300 as eb
    grid, ls = CASES["star258_01"]()
    betas = ei.beta_half_points(grid, ei.beta_bone)
    h = eb.EB(grid, ls, closure=eb.EB_CLOSURE_MIXED)
    h.set_beta(betas)
    ref = oeb.build(grid, ls, beta=betas, closure="mixed")
    _, diag = h.cp_data()
    assert np.abs(diag.cpu().numpy() - ref.diag).max() <= 1e-9
    X, Y = ei.grid_points(grid)
    pts = ref.sample_points()
    ug = np.cos(pts[:, 0]) + pts[:, 1]
    b = h.rhs(torch.tensor(np.sin(X), device="cuda"), torch.tensor(ug, device="cuda")).cpu().numpy()
    b_ref = oeb.rhs(ref, np.sin(X), ug)
    assert np.abs(ref.from_grid(b) - b_ref).max() <= 1e-9 * np.abs(b_ref).max()


def test_rbf_closure_rejections():
    import paper_2204_06083_gb300 as eb
    grid, ls = ei.ellipsoid_k3(34, seed=0)
    with pytest.raises(eb.EBError):
        eb.EB(grid, ls, closure=eb.EB_CLOSURE_MIXED)
    g2 = ei.box_grid(2, 66)
    with pytest.raises(eb.EBError):
        eb.EB(g2, ei.sampled(ei.circle_distance_values(g2, (0.02, 0.01), 0.5)), closure=eb.EB_CLOSURE_RBF)
