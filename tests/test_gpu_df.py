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
* A warm start, b = 0, and the cases DF does not cover (variable beta, Jacobi,
  an FP64 V-cycle, a bad outer_prec).
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
    hb = eb.EB(grid, ls)
    hb.set_beta(ei.beta_half_points(grid, ei.beta_bone))
    gb = eb.AMG(hb, 0.0, vcycle_prec=eb.EB_F32)
    with pytest.raises(eb.EBError) as e:
        gb.solve(b, outer=eb.EB_DF64)
    assert e.value.code == eb.EB_ERR_NOT_IMPLEMENTED
