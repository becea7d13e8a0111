"""GPU parity of the classical (Ruge-Stueben) hierarchy and of the W-cycle
(amg_opts.coarsening = EB_AMG_RS, amg_opts.cycle = 2; Sec. 3) against the
oracle's sequential implementation of the same rules.

* C/F splitting identical (amg_level_copy which = 2: coarse index of C
  points, -1 for F points), every level's size and pattern identical, P and
  A_l within 1e-13 of the row maximum;
* one V- or W-cycle on the same input: rel-L2 <= 1e-12;
* AMG-PCG with RS + W: solution within 1e-10 of the oracle's, iteration
  counts equal within 1; W-cycle counts flat over the sizes (Sec. 3.1).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import eb_inputs as ei
from oracle import amg as oamg
from oracle import eb as oeb
from oracle import solvers as osol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


CASES = {
    "circle256": lambda: ei.circle_k1(256),
    "star258": lambda: (ei.box_grid(2, 258), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])),
    "ellipsoid48": lambda: ei.ellipsoid_k3(48, seed=0),
}


def _csr(rp, ci, v, n, m):
    return sp.csr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(n, m))


def _close_rows(M, R, tol):
    assert np.array_equal(M.indptr, R.indptr)
    assert np.array_equal(M.indices, R.indices)
    rowmax = np.maximum.reduceat(np.abs(R.data), R.indptr[:-1]) if R.nnz else np.zeros(0)
    scale = np.repeat(rowmax, np.diff(R.indptr))
    assert np.all(np.abs(M.data - R.data) <= tol * scale)


def _setup(name, cycle=1):
    import paper_2204_06083_gb300 as eb
    grid, ls = CASES[name]()
    ref = oeb.build(grid, ls)
    H = oamg.setup(ref.A, "rs")
    h = eb.EB(grid, ls)
    g = eb.AMG(h, 0.0, coarsening=eb.EB_AMG_RS, cycle=cycle)
    return eb, grid, ref, H, h, g


@pytest.mark.parametrize("name", list(CASES))
def test_rs_hierarchy_matches_oracle(name):
    eb, grid, ref, H, h, g = _setup(name)
    assert g.num_levels == len(H.levels) >= 3
    for l, lev in enumerate(H.levels):
        n = lev.A.shape[0]
        assert g.rows[l] == n and g.nnz[l] == lev.A.nnz
        rp, ci, v = g.level(l, 0)
        _close_rows(_csr(rp, ci, v, n, n), lev.A, 1e-13)
        if l < len(H.levels) - 1:
            assert np.array_equal(g.level(l, 2).cpu().numpy(), lev.agg), l
            rp, ci, v = g.level(l, 1)
            _close_rows(_csr(rp, ci, v, n, lev.P.shape[1]), lev.P, 1e-13)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("cycle", [1, 2])
def test_rs_cycle_matches_oracle(name, cycle):
    eb, grid, ref, H, h, g = _setup(name, cycle)
    r = np.random.default_rng(5).standard_normal(grid.shape())
    z = g.vcycle(torch.tensor(r, device="cuda")).cpu().numpy()
    z_ref = oamg.vcycle(H, ref.from_grid(r), gamma=cycle)
    got = ref.from_grid(z)
    assert np.linalg.norm(got - z_ref) / np.linalg.norm(z_ref) <= 1e-12


@pytest.mark.parametrize("coarsening", ["sa", "rs"])
def test_w_cycle_pcg_matches_oracle(coarsening):
    import paper_2204_06083_gb300 as eb
    grid, ls = ei.circle_k1(256)
    ref = oeb.build(grid, ls)
    H = oamg.setup(ref.A, coarsening)
    h = eb.EB(grid, ls)
    g = eb.AMG(h, 0.0, coarsening=eb.EB_AMG_RS if coarsening == "rs" else eb.EB_AMG_SA, cycle=2)
    X, Y = ei.grid_points(grid)
    f = ei.f_k1(X, Y)
    ug = ei.u_k1(ref.cut_xg[:, 0], ref.cut_xg[:, 1])
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda"))
    b_ref = oeb.rhs(ref, f, ug)
    x, st = g.solve(b, rtol=1e-12, maxit=300)
    x_ref, st_ref = osol.pcg(ref.A, b_ref, M=lambda r: oamg.vcycle(H, r, gamma=2), rtol=1e-12)
    got = ref.from_grid(x.cpu().numpy())
    assert np.linalg.norm(got - x_ref) / np.linalg.norm(x_ref) <= 1e-10
    assert abs(st.iterations - st_ref.iterations) <= 1


def test_rs_w_iterations_flat_over_sizes():
    import paper_2204_06083_gb300 as eb
    its = []
    for n in (256, 512, 1024, 2048):
        grid, ls = ei.circle_k1(n)
        h = eb.EB(grid, ls)
        X, Y = ei.grid_points(grid)
        _, _, _, xg = h.cuts()
        xg = xg.cpu().numpy()
        b = h.rhs(torch.tensor(ei.f_k1(X, Y), device="cuda"), torch.tensor(ei.u_k1(xg[:, 0], xg[:, 1]), device="cuda"))
        g = eb.AMG(h, 0.0, coarsening=eb.EB_AMG_RS, cycle=2)
        _, st = g.solve(b, rtol=1e-12, maxit=300)
        assert st.converged
        its.append(st.iterations)
    print("RS W-cycle iterations at n = 256..2048:", its)
    assert max(its) - min(its) <= 3, its
