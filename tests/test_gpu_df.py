"""The double-float (DF) outer iteration of pcg_solve (pcg_opts.outer_prec =
EB_DF64) against the oracle and against the FP64 outer iteration.

* Solutions: DF solves to rtol 1e-12 (the FP64 true residual confirms it)
  match the oracle's AMG-PCG solution at rtol 1e-13 within rel-L2 1e-8
  (kappa times the residual; DF carries about 48 bits).
* Iterations to 1e-10 equal those of the FP64 outer iteration within 1.
* The loop forms (device-side loop, captured chunks, direct launches) and the
  profiling modes give the same x bit for bit (every reduction has a fixed
  order).
* Exact power-of-two scaling: b 2^-100 and b 2^100 give x 2^-100 and x 2^100
  bit for bit (the DF image of b is rescaled to a unit root mean square).
* A warm start, b = 0, and the cases DF does not cover (Jacobi, an FP64
  V-cycle, a bad outer_prec).
* A variable coefficient (eq. 3): DF solves against the exact oracle solve;
  Crank-Nicolson heat steps and theta-scheme wave steps through the solver's
  default outer precision (amg_set_outer_prec) against the FP64 outer
  iteration.
"""
import numpy as np
import pytest
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
    "circle128": lambda: ei.circle_k1(128),
    "star258": lambda: (ei.box_grid(2, 258), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])),
    "ellipsoid64": lambda: ei.ellipsoid_k3(64, seed=2),
}


def _problem(name):
    grid, ls = CASES[name]()
    ref = oeb.build(grid, ls)
    pts = ei.grid_points(grid)
    ufun, ffun = (ei.u_k1, ei.f_k1) if grid.dim == 2 else (ei.u_k3, ei.f_k3)
    f = ffun(*pts)
    ug = ufun(*[ref.cut_xg[:, a] for a in range(grid.dim)])
    return grid, ls, ref, f, ug


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_df_pcg_matches_oracle(name, prec):
    eb = _eb()
    grid, ls, ref, f, ug = _problem(name)
    h = eb.EB(grid, ls)
    g = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32 if prec == "f32" else eb.EB_BF16)
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda"))
    b_ref = oeb.rhs(ref, f, ug)
    x, st = g.solve(b, rtol=1e-12, maxit=500, outer=eb.EB_DF64)
    H = oamg.setup(ref.A)
    x_ref, _ = osol.pcg(ref.A, b_ref, M=lambda q: oamg.vcycle(H, q), rtol=1e-13)
    got = ref.from_grid(x.cpu().numpy())
    err = np.linalg.norm(got - x_ref) / np.linalg.norm(x_ref)
    print(f"{name} {prec}: DF its {st.iterations}, true rel res {st.true_rel_residual:.2e}, rel-L2 vs oracle {err:.2e}")
    assert st.converged and st.true_rel_residual <= 1e-12
    assert err <= 1e-8
    # entries off the CPs stay zero
    full = x.cpu().numpy().ravel()
    mask = np.zeros(full.size, bool)
    mask[ref.cp_nodes] = True
    assert np.all(full[~mask] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_df_iterations_match_fp64_outer(name):
    eb = _eb()
    grid, ls, ref, f, ug = _problem(name)
    h = eb.EB(grid, ls)
    g = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda"))
    x64, s64 = g.solve(b, rtol=1e-10, maxit=500)
    xdf, sdf = g.solve(b, rtol=1e-10, maxit=500, outer=eb.EB_DF64)
    print(f"{name}: its FP64 outer {s64.iterations}, DF {sdf.iterations}; true rel res {s64.true_rel_residual:.2e} "
          f"{sdf.true_rel_residual:.2e}")
    assert abs(sdf.iterations - s64.iterations) <= 1
    assert sdf.converged and sdf.true_rel_residual <= 1e-10
    d = torch.linalg.norm(xdf - x64) / torch.linalg.norm(x64)
    assert d.item() <= 1e-7


def test_df_loop_forms_and_profiling_agree():
    eb = _eb()
    grid, ls, ref, f, ug = _problem("ellipsoid64")
    h = eb.EB(grid, ls)
    g = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda"))
    x0, st0 = g.solve(b, rtol=1e-10, outer=eb.EB_DF64)
    for kw in ({"use_graph": 0}, {"use_graph": 2, "check_every": 3}, {"profile": 1}, {"profile": 3},
               {"profile": 4}, {"profile": 5}):
        x, st = g.solve(b, rtol=1e-10, outer=eb.EB_DF64, **kw)
        assert st.iterations == st0.iterations, kw
        assert torch.equal(x, x0), kw


def test_df_power_of_two_scaling_is_exact():
    eb = _eb()
    grid, ls, ref, f, ug = _problem("circle128")
    h = eb.EB(grid, ls)
    g = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda"))
    x0, st0 = g.solve(b, rtol=1e-10, outer=eb.EB_DF64)
    for k in (-100, 100):
        x, st = g.solve(b * 2.0 ** k, rtol=1e-10, outer=eb.EB_DF64)
        assert st.iterations == st0.iterations
        assert torch.equal(x, x0 * 2.0 ** k), k


def test_df_warm_start_and_zero_rhs():
    eb = _eb()
    grid, ls, ref, f, ug = _problem("star258")
    h = eb.EB(grid, ls)
    g = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda"))
    xs, st = g.solve(b, rtol=1e-10, outer=eb.EB_DF64)
    x0 = xs + 1e-3 * torch.tensor(np.random.default_rng(1).standard_normal(h.shape()), device="cuda")
    x, st2 = g.solve(b, x=x0, rtol=1e-10, outer=eb.EB_DF64)
    assert st2.converged and st2.true_rel_residual <= 1e-10
    z, st3 = g.solve(torch.zeros_like(b), rtol=1e-10, outer=eb.EB_DF64)
    assert st3.converged and st3.iterations == 0 and torch.count_nonzero(z).item() == 0


def test_df_rejects_what_it_does_not_cover():
    eb = _eb()
    grid, ls = ei.circle_k1(64)
    h = eb.EB(grid, ls)
    b = torch.ones(h.shape(), dtype=torch.float64, device="cuda")
    g64 = eb.AMG(h, 0.0)
    with pytest.raises(eb.EBError) as e:
        g64.solve(b, outer=eb.EB_DF64)
    assert e.value.code == eb.EB_ERR_NOT_IMPLEMENTED
    g32 = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
    with pytest.raises(eb.EBError) as e:
        g32.solve(b, precond=eb.EB_PC_JACOBI, outer=eb.EB_DF64)
    assert e.value.code == eb.EB_ERR_NOT_IMPLEMENTED
    with pytest.raises(eb.EBError) as e:
        g32.solve(b, outer=7)
    assert e.value.code == eb.EB_ERR_INVALID
    with pytest.raises(eb.EBError) as e:
        g32.set_outer(5)
    assert e.value.code == eb.EB_ERR_INVALID


BETA_CASES = {
    "circle130_bone": lambda: (*ei.circle_k1(130), ei.beta_bone),
    "disk128_heat": lambda: (*ei.heat_disk(128), ei.beta_heat_disk),
    "ellipsoid42_lin": lambda: (*ei.ellipsoid_k3(42, seed=0), lambda x, y, z: 1.5 + 0.4 * x - 0.3 * y + 0.2 * z),
}


@pytest.mark.parametrize("name", list(BETA_CASES))
def test_df_pcg_variable_beta_matches_oracle(name):
    """The DF outer iteration with a variable coefficient (eq. 3): beta at the
    half points and D_k enter through DF copies; solutions to rtol 1e-12 match
    the exact oracle solve within rel-L2 1e-8, and the iteration count to
    1e-10 equals the FP64 outer iteration's within 1."""
    import scipy.sparse.linalg as spla
    eb = _eb()
    grid, ls, bfun = BETA_CASES[name]()
    betas = ei.beta_half_points(grid, bfun)
    h = eb.EB(grid, ls)
    h.set_beta(betas)
    ref = oeb.build(grid, ls, beta=betas)
    b_cp = np.random.default_rng(3).standard_normal(ref.num_cp)
    b = torch.tensor(ref.to_grid(b_cp), device="cuda")
    x_ref = spla.spsolve(ref.A.tocsc(), b_cp)
    g = eb.AMG(h, 0.0, vcycle_prec=eb.EB_F32)
    x, st = g.solve(b, rtol=1e-12, maxit=800, outer=eb.EB_DF64)
    got = ref.from_grid(x.cpu().numpy())
    err = np.linalg.norm(got - x_ref) / np.linalg.norm(x_ref)
    print(f"{name}: DF its {st.iterations}, true rel res {st.true_rel_residual:.2e}, rel-L2 vs exact {err:.2e}")
    assert st.converged and st.true_rel_residual <= 1e-12
    assert err <= 1e-8
    _, s64 = g.solve(b, rtol=1e-10, maxit=800)
    _, sdf = g.solve(b, rtol=1e-10, maxit=800, outer=eb.EB_DF64)
    assert abs(s64.iterations - sdf.iterations) <= 1


def test_df_crank_nicolson_and_theta_wave_match_fp64():
    """amg_set_outer_prec(EB_DF64): heat_step (Crank-Nicolson on the Sec. 3.4
    disk with beta = 0.25 - r^2) and wave_theta_step run their solves in
    double-float; after 5 steps the fields match those of the FP64 outer
    iteration within rel-L2 1e-9 (both solve to 1e-11), with iteration totals
    within 1 per step (heat); a single-level hierarchy runs FP64."""
    eb = _eb()
    grid, ls = ei.heat_disk(130)
    betas = ei.beta_half_points(grid, ei.beta_heat_disk)
    h = eb.EB(grid, ls)
    h.set_beta(betas)
    X, Y = ei.grid_points(grid)
    dt, theta = grid.h, 0.5
    zc = torch.zeros(max(h.info.num_cut, 1), dtype=torch.float64, device="cuda")
    out = {}
    for outer in (eb.EB_F64, eb.EB_DF64):
        g = eb.AMG(h, 1.0 / (theta * dt), vcycle_prec=eb.EB_F32)
        g.set_outer(outer)
        u = torch.tensor(ei.u_heat_disk(X, Y, 0.0), device="cuda")
        b0 = h.rhs(torch.tensor(-ei.f_heat_disk(X, Y, 0.0), device="cuda"), zc)
        its = []
        for k in range(5):
            b1 = h.rhs(torch.tensor(-ei.f_heat_disk(X, Y, (k + 1) * dt), device="cuda"), zc)
            st = g.heat_step(u, b1, dt, theta=theta, b0=b0, rtol=1e-11, maxit=300)
            assert st.converged and st.true_rel_residual <= 1e-11
            its.append(st.iterations)
            b0 = b1
        out[outer] = (u, its)
    u64, udf = out[eb.EB_F64][0], out[eb.EB_DF64][0]
    assert (torch.linalg.norm(udf - u64) / torch.linalg.norm(u64)).item() <= 1e-9
    assert all(abs(a - b) <= 1 for a, b in zip(out[eb.EB_F64][1], out[eb.EB_DF64][1]))
    # theta-scheme wave steps (theta = 1/4, dt = 2h: a shift that leaves the
    # hierarchy two levels deep) on the same disk
    dtw, th = 2.0 * grid.h, 0.25
    wout = {}
    for outer in (eb.EB_F64, eb.EB_DF64):
        g = eb.AMG(h, 1.0 / (th * dtw * dtw), vcycle_prec=eb.EB_F32)
        g.set_outer(outer)
        ua = torch.tensor(np.exp(-40.0 * (X ** 2 + Y ** 2)), device="cuda")
        ub = ua.clone()
        st = g.wave_theta_step(ua, ub, dtw, th, 5, rtol=1e-11)
        assert st.converged
        wout[outer] = (ub.clone(), st.iterations)
    w64, wdf = wout[eb.EB_F64][0], wout[eb.EB_DF64][0]
    assert (torch.linalg.norm(wdf - w64) / torch.linalg.norm(w64)).item() <= 1e-9
    assert abs(wout[eb.EB_F64][1] - wout[eb.EB_DF64][1]) <= 5
    # theta = 1/12, dt = 0.85 h: the shift leaves one level, where the default
    # outer precision falls back to FP64 -- the same result bit for bit
    dtw, th = 0.85 * grid.h, 1.0 / 12.0
    res = []
    for outer in (eb.EB_F64, eb.EB_DF64):
        g = eb.AMG(h, 1.0 / (th * dtw * dtw), vcycle_prec=eb.EB_F32)
        assert g.num_levels == 1
        g.set_outer(outer)
        ua = torch.tensor(np.exp(-40.0 * (X ** 2 + Y ** 2)), device="cuda")
        ub = ua.clone()
        g.wave_theta_step(ua, ub, dtw, th, 3, rtol=1e-11)
        res.append(ub)
    assert torch.equal(res[0], res[1])
