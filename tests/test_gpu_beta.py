"""GPU parity of the variable-coefficient operator (eq. 3 with beta at the half
points, the beta-weighted closure of Sec. 2.1) against the oracle, through the
C ABI (eb_set_beta).

Tolerances (GPU vs oracle): D_k, the right-hand side (quadric geometries) and
the dominance margin bit-exact (the same IEEE operations); FP64 apply rel-L2
<= 1e-14; AMG aggregates identical and level values within 1e-13 of the row
maximum; PCG solutions within rel-L2 1e-10 when both sides solve to 1e-13;
Crank-Nicolson heat steps (Sec. 3.4) within 1e-10 of exact (sparse LU) oracle
steps; leapfrog with beta within 1e-11 after 25 steps.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
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


def _eb():
    import paper_2204_06083_gb300 as eb
    return eb


CASES = {
    "circle130_bone": lambda: (*ei.circle_k1(130), ei.beta_bone),
    "star258_bone": lambda: (ei.box_grid(2, 258), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0]), ei.beta_bone),
    "disk128_heat": lambda: (*ei.heat_disk(128), ei.beta_heat_disk),
    "ellipsoid42_lin": lambda: (*ei.ellipsoid_k3(42, seed=0), lambda x, y, z: 1.5 + 0.4 * x - 0.3 * y + 0.2 * z),
}


def _pair(name):
    eb = _eb()
    grid, ls, bfun = CASES[name]()
    betas = ei.beta_half_points(grid, bfun)
    h = eb.EB(grid, ls)
    h.set_beta(betas)
    ref = oeb.build(grid, ls, beta=betas)
    return h, ref, grid, ls


@pytest.mark.parametrize("name", list(CASES))
def test_beta_build_parity(name):
    h, ref, grid, ls = _pair(name)
    nodes, diag = h.cp_data()
    assert np.array_equal(nodes.cpu().numpy().astype(np.int64), ref.cp_nodes)
    d = diag.cpu().numpy()
    if ls.kind == ei.LS_QUADRIC:
        assert np.array_equal(d, ref.diag)
        assert h.info.min_dominance_margin == oeb.dominance_margin(ref)
    else:
        assert np.abs(d - ref.diag).max() <= 1e-12 / grid.h
        assert abs(h.info.min_dominance_margin - oeb.dominance_margin(ref)) <= 1e-12
    # the public codes keep the beta = 1 layout (0x80 | BP-direction mask)
    code = h.classes().cpu().numpy().reshape(-1)
    assert np.all(code[ref.cp_nodes] & 0x40 == 0)
    pts = ei.grid_points(grid)
    f = np.sin(pts[0]) + 0.5
    ug = np.cos(ref.cut_xg[:, 0])
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda")).cpu().numpy()
    b_ref = oeb.rhs(ref, f, ug)
    got = ref.from_grid(b)
    if ls.kind == ei.LS_QUADRIC:
        assert np.array_equal(got, b_ref)
    else:
        assert np.abs(got - b_ref).max() <= 1e-11 * np.abs(b_ref).max()


@pytest.mark.parametrize("name", list(CASES))
def test_beta_apply_parity(name):
    h, ref, grid, _ = _pair(name)
    x = np.random.default_rng(1).standard_normal(grid.shape())
    y_ref = ref.A @ ref.from_grid(x)
    for dtype, tol in ((torch.float64, 1e-14), (torch.float32, 1e-6)):
        y = h.apply(torch.tensor(x, device="cuda").to(dtype)).double().cpu().numpy()
        got = ref.from_grid(y)
        assert np.linalg.norm(got - y_ref) / np.linalg.norm(y_ref) <= tol, dtype
        off = np.ones(y.size, bool)
        off[ref.cp_nodes] = False
        assert np.all(y.reshape(-1)[off] == 0.0)


def _csr(rp, ci, v, n, m):
    return sp.csr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(n, m))


@pytest.mark.parametrize("name", ["circle130_bone", "disk128_heat", "ellipsoid42_lin"])
def test_beta_hierarchy_and_pcg_parity(name):
    eb = _eb()
    h, ref, grid, _ = _pair(name)
    H = oamg.setup(ref.A)
    g = eb.AMG(h, 0.0)
    assert g.num_levels == len(H.levels)
    for l, lev in enumerate(H.levels):
        n = lev.A.shape[0]
        rp, ci, v = g.level(l, 0)
        M = _csr(rp, ci, v, n, n)
        assert np.array_equal(M.indptr, lev.A.indptr) and np.array_equal(M.indices, lev.A.indices)
        rowmax = np.repeat(np.maximum.reduceat(np.abs(lev.A.data), lev.A.indptr[:-1]), np.diff(lev.A.indptr))
        assert np.all(np.abs(M.data - lev.A.data) <= 1e-13 * rowmax)
        if l < len(H.levels) - 1:
            assert np.array_equal(g.level(l, 2).cpu().numpy(), lev.agg)
    b_cp = np.random.default_rng(2).standard_normal(ref.num_cp)
    b = torch.tensor(ref.to_grid(b_cp), device="cuda")
    x_ref = spla.spsolve(ref.A.tocsc(), b_cp)
    for prec in (eb.EB_F64, eb.EB_F32):
        gp = g if prec == eb.EB_F64 else eb.AMG(h, 0.0, vcycle_prec=prec)
        x, st = gp.solve(b, rtol=1e-13, maxit=800)
        got = ref.from_grid(x.cpu().numpy())
        assert np.linalg.norm(got - x_ref) / np.linalg.norm(x_ref) <= 1e-10, prec
        _, st1 = gp.solve(b, rtol=1e-10, maxit=800)
        _, st1_ref = osol.pcg(ref.A, b_cp, M=lambda r: oamg.vcycle(H, r), rtol=1e-10)
        if prec == eb.EB_F64:
            assert abs(st1.iterations - st1_ref.iterations) <= 1


def test_beta_linear_exactness_on_gpu():
    """beta and u linear: the discrete solution is u at every CP (the oracle's
    exactness pin), reproduced through eb_set_beta / eb_rhs / AMG-PCG."""
    eb = _eb()
    grid, ls = ei.star_wave(258)
    bfun = lambda x, y: 1.5 + 0.4 * x - 0.3 * y
    h = eb.EB(grid, ls)
    h.set_beta(ei.beta_half_points(grid, bfun))
    u = lambda x, y: 0.3 + 0.7 * x - 1.1 * y
    fconst = 0.7 * 0.4 + (-1.1) * (-0.3)
    _, _, _, xg = h.cuts()
    xg = xg.cpu().numpy()
    b = h.rhs(torch.full(h.shape(), fconst, dtype=torch.float64, device="cuda"),
              torch.tensor(u(xg[:, 0], xg[:, 1]), device="cuda"))
    x, st = eb.AMG(h, 0.0).solve(b, rtol=1e-13, maxit=500)
    X, Y = ei.grid_points(grid)
    nodes, _ = h.cp_data()
    nodes = nodes.cpu().numpy()
    err = np.abs(x.cpu().numpy().reshape(-1)[nodes] - u(X, Y).reshape(-1)[nodes]).max()
    assert err <= 1e-9, err


def test_crank_nicolson_heat_disk_matches_oracle():
    """Sec. 3.4: theta = 1/2, dt = h, the disk with beta = 0.25 - r^2 and its
    manufactured solution: five GPU heat steps (AMG on sigma I + A, sigma =
    1/(theta dt), warm start, rtol 1e-13) against exact oracle steps."""
    eb = _eb()
    grid, ls = ei.heat_disk(130)
    betas = ei.beta_half_points(grid, ei.beta_heat_disk)
    h = eb.EB(grid, ls)
    h.set_beta(betas)
    ref = oeb.build(grid, ls, beta=betas)
    X, Y = ei.grid_points(grid)
    dt, theta = grid.h, 0.5
    g = eb.AMG(h, 1.0 / (theta * dt))
    lhs = (sp.identity(ref.num_cp, format="csc") / dt + theta * ref.A).tocsc()
    lu = spla.splu(lhs)
    u = torch.tensor(ei.u_heat_disk(X, Y, 0.0), device="cuda")
    u_ref = ref.from_grid(ei.u_heat_disk(X, Y, 0.0))
    zeros_cut = np.zeros(ref.cut_cp.size)

    def b_at(t):
        F = -ei.f_heat_disk(X, Y, t)
        return F, oeb.rhs(ref, F, zeros_cut)

    F0, b0_ref = b_at(0.0)
    b0 = h.rhs(torch.tensor(F0, device="cuda"), torch.zeros(max(ref.cut_cp.size, 1), dtype=torch.float64,
                                                               device="cuda"))
    for k in range(5):
        F1, b1_ref = b_at((k + 1) * dt)
        b1 = h.rhs(torch.tensor(F1, device="cuda"), torch.zeros(max(ref.cut_cp.size, 1), dtype=torch.float64,
                                                                   device="cuda"))
        st = g.heat_step(u, b1, dt, theta=theta, b0=b0, rtol=1e-13, maxit=300)
        assert st.converged
        r = u_ref / dt - (1.0 - theta) * (ref.A @ u_ref) + theta * b1_ref + (1.0 - theta) * b0_ref
        u_ref = lu.solve(r)
        b0, b0_ref = b1, b1_ref
        got = ref.from_grid(u.cpu().numpy())
        assert np.linalg.norm(got - u_ref) / np.linalg.norm(u_ref) <= 1e-10, k


def test_leapfrog_with_beta_matches_oracle():
    eb = _eb()
    grid, ls = ei.star_wave(258)
    betas = ei.beta_half_points(grid, ei.beta_bone)
    h = eb.EB(grid, ls)
    h.set_beta(betas)
    ref = oeb.build(grid, ls, beta=betas)
    X, Y = ei.grid_points(grid)
    c, w = ei.pulse_params(1)
    u0 = ref.from_grid(ei.pulse(X, Y, c, 4 * w))
    dt = 0.5 * grid.h / math.sqrt(2.0) / math.sqrt(3.0)   # beta <= 3
    u1 = u0 - 0.5 * dt * dt * (ref.A @ u0)
    a, b = osol.leapfrog(ref.A, u0, u1, dt, 25)
    ua = torch.tensor(ref.to_grid(u0), device="cuda")
    ub = torch.tensor(ref.to_grid(u1), device="cuda")
    h.wave_step(ua, ub, dt, 25)
    got = ref.from_grid(ub.cpu().numpy())
    assert np.linalg.norm(got - b) / np.linalg.norm(b) <= 1e-11


def test_beta_rejections():
    eb = _eb()
    grid, ls = ei.circle_k1(66)
    h = eb.EB(grid, ls)
    bad = ei.beta_half_points(grid, lambda x, y: 1.0 - 3.0 * np.abs(x))   # negative inside
    with pytest.raises(eb.EBError):
        h.set_beta(bad)
    h2 = eb.EB(grid, ls)
    h2.set_beta(ei.beta_half_points(grid, ei.beta_bone))
    with pytest.raises(eb.EBError):
        h2.set_beta(ei.beta_half_points(grid, ei.beta_bone))
