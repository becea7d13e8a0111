"""GPU parity of eb_build / eb_rhs / eb_apply against the FP64 oracle, through
the C ABI.

Tolerances (GPU vs oracle):
* node classes and the cut list (CP, direction): bit-exact.
* quadric geometries: delta, c_s, D_k and b are computed by the same IEEE
  operations in the same order on both sides: bit-exact.
* star geometries: psi uses sin / atan2, whose last-ulp results differ between
  the CUDA and host libraries; a psi error of a few ulp of O(1) values moves a
  grid-line root by ~eps / |dpsi/dt|.  Bound used: |d delta| <= 1e-12 (absolute,
  domain units), i.e. ~2e-9 h at n = 4096 for grazing crossings.
* apply in FP64: rel-L2 <= 1e-14 (different rounding order of the stencil sum).
* apply in FP32 / BF16: the error against FP64 is stated: rel-L2 <= 1e-6 (FP32)
  and <= 1e-2 (BF16 storage, FP32 accumulation).
"""
import numpy as np
import pytest
import torch

import eb_inputs as ei
from oracle import eb as oeb

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
    "circle130": lambda: ei.circle_k1(130),
    "circle128": lambda: ei.circle_k1(128),
    "star_k2_258": lambda: (ei.box_grid(2, 258), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])),
    "randstar_300": lambda: (ei.box_grid(2, 300), ei.random_star(3)),
    "ellipsoid42": lambda: ei.ellipsoid_k3(42, seed=0),
    "ellipsoid64": lambda: ei.ellipsoid_k3(64, seed=5),
    "sphere3_38": lambda: (ei.box_grid(3, 38), ei.sphere((0.013, -0.021, 0.017), 0.6)),
}


def _compare_build(grid, ls, exact):
    eb = _eb()
    ref = oeb.build(grid, ls)
    h = eb.EB(grid, ls)
    assert h.info.num_cp == ref.num_cp
    assert h.info.num_cut == ref.cut_cp.size
    assert h.info.num_bp == int((ref.cls == 1).sum())
    code = h.classes().cpu().numpy()
    want = np.where(ref.cls == 2, 0x80, np.where(ref.cls == 1, 0x40, 0))
    assert np.array_equal(code & 0xC0, want)
    nodes, diag = h.cp_data()
    assert np.array_equal(nodes.cpu().numpy().astype(np.int64), ref.cp_nodes)
    cp, d, delta, xg = h.cuts()
    assert np.array_equal(cp.cpu().numpy(), ref.cut_cp)
    assert np.array_equal(d.cpu().numpy(), ref.cut_dir)
    delta = delta.cpu().numpy()
    diag = diag.cpu().numpy()
    if exact:
        assert np.array_equal(delta, ref.cut_delta)
        assert np.array_equal(diag, ref.diag)
        assert np.array_equal(xg.cpu().numpy(), ref.cut_xg)
    else:
        assert np.abs(delta - ref.cut_delta).max() <= 1e-12
        assert np.abs(diag - ref.diag).max() <= 1e-12 / grid.h
    # BP-neighbour direction masks agree with the cut list
    masks = np.zeros(ref.num_cp, dtype=np.int64)
    np.bitwise_or.at(masks, ref.cut_cp, 1 << ref.cut_dir)
    assert np.array_equal(code.reshape(-1)[ref.cp_nodes] & 0x3F, masks)
    return h, ref


@pytest.mark.parametrize("name", list(CASES))
def test_build_parity(name):
    grid, ls = CASES[name]()
    h, ref = _compare_build(grid, ls, exact=(ls.kind == ei.LS_QUADRIC))
    margin = oeb.dominance_margin(ref)
    if ls.kind == ei.LS_QUADRIC:
        assert h.info.min_dominance_margin == margin
    else:
        assert abs(h.info.min_dominance_margin - margin) <= 1e-12
    assert h.info.min_dominance_margin > 0


def _sampled_cases():
    """Level sets known only at the nodes (Sec. 3.3): psi values are inputs, so
    both sides run the same IEEE operations on the same numbers."""
    g2 = ei.box_grid(2, 258)
    g3 = ei.box_grid(3, 66)
    g2b = ei.box_grid(2, 1026)
    star_vals = lambda g: (np.hypot(*(p - c for p, c in zip(ei.grid_points(g), ei.STAR_CENTER)))
                           - (0.5 + 0.1 * np.sin(5 * np.arctan2(ei.grid_points(g)[1] - ei.STAR_CENTER[1],
                                                                  ei.grid_points(g)[0] - ei.STAR_CENTER[0]))))
    return {
        "circle_sdf_258": (g2, ei.sampled(ei.circle_distance_values(g2, (0.02, 0.01), 0.5))),
        "diamond_258": (g2, ei.sampled(ei.diamond_values(g2, (0.0123, 0.0071), 0.71))),
        "sphere_sdf_66": (g3, ei.sampled(ei.circle_distance_values(g3, (0.013, -0.021, 0.017), 0.6))),
        "star_samples_1026": (g2b, ei.sampled(star_vals(g2b))),
    }


@pytest.mark.parametrize("name", list(_sampled_cases()))
def test_sampled_levelset_build_parity(name):
    """EB_LS_SAMPLED: classes, cuts, delta (linear ratio), D_k, crossing points
    and the dominance margin bit-exact against the oracle; then a solve on the
    sampled geometry against the oracle's."""
    grid, ls = _sampled_cases()[name]
    h, ref = _compare_build(grid, ls, exact=True)
    assert h.info.min_dominance_margin == oeb.dominance_margin(ref)
    eb = _eb()
    rng = np.random.default_rng(11)
    b = rng.standard_normal(grid.shape())
    x_ref = __import__("scipy.sparse.linalg", fromlist=["spsolve"]).spsolve(ref.A.tocsc(), ref.from_grid(b))
    solver = eb.AMG(h, 0.0)
    x, st = solver.solve(torch.tensor(b, device="cuda"), rtol=1e-13, maxit=500)
    err = np.linalg.norm(ref.from_grid(x.cpu().numpy()) - x_ref) / np.linalg.norm(x_ref)
    assert err <= 1e-10, err


def test_sampled_levelset_requires_values():
    import ctypes as C
    eb = _eb()
    L = eb.load()
    grid = ei.box_grid(2, 66)
    g = eb.make_grid(grid)
    ls = eb.eb_levelset()
    ls.kind = eb.EB_LS_SAMPLED
    out = C.c_void_p()
    rc = L.eb_build(C.byref(g), C.byref(ls), C.byref(out), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == eb.EB_ERR_INVALID


@pytest.mark.parametrize("name", ["circle130", "randstar_300", "ellipsoid42"])
def test_rhs_parity(name):
    grid, ls = CASES[name]()
    eb = _eb()
    h = eb.EB(grid, ls)
    ref = oeb.build(grid, ls)
    pts = ei.grid_points(grid)
    ufun, ffun = (ei.u_k1, ei.f_k1) if grid.dim == 2 else (ei.u_k3, ei.f_k3)
    f = ffun(*pts)
    ug = ufun(*[ref.cut_xg[:, a] for a in range(grid.dim)])
    b = h.rhs(torch.tensor(f, device="cuda"), torch.tensor(ug, device="cuda")).cpu().numpy()
    b_ref = oeb.rhs(ref, f, ug)
    got = ref.from_grid(b)
    if ls.kind == ei.LS_QUADRIC:
        assert np.array_equal(got, b_ref)
    else:
        assert np.abs(got - b_ref).max() <= 1e-11 * np.abs(b_ref).max()
    # zero at every non-CP node of the grid
    bf = b.reshape(-1)
    mask = np.ones(bf.size, bool)
    mask[ref.cp_nodes] = False
    assert np.all(bf[mask] == 0.0)


@pytest.mark.parametrize("name", ["circle130", "star_k2_258", "ellipsoid42", "sphere3_38"])
def test_apply_parity_all_precisions(name):
    grid, ls = CASES[name]()
    eb = _eb()
    h = eb.EB(grid, ls)
    ref = oeb.build(grid, ls)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(grid.shape())
    # non-CP entries must be ignored: fill them with garbage
    y_ref = ref.A @ ref.from_grid(x)
    xt = torch.tensor(x, device="cuda")
    y = h.apply(xt).cpu().numpy()
    got = ref.from_grid(y)
    assert np.linalg.norm(got - y_ref) / np.linalg.norm(y_ref) <= 1e-14
    off = np.ones(y.size, bool)
    off[ref.cp_nodes] = False
    assert np.all(y.reshape(-1)[off] == 0.0)
    y32 = ref.from_grid(h.apply(xt.float()).double().cpu().numpy())
    e32 = np.linalg.norm(y32 - y_ref) / np.linalg.norm(y_ref)
    assert e32 <= 1e-6, e32
    y16 = ref.from_grid(h.apply(xt.bfloat16()).double().cpu().numpy())
    # bf16 input rounding (2^-9 relative) amplified by the stencil's cancellation
    xr = ref.from_grid(xt.bfloat16().double().cpu().numpy())
    y16_ref = ref.A @ xr
    e16 = np.linalg.norm(y16 - y16_ref) / np.linalg.norm(y16_ref)
    assert e16 <= 1e-2, e16


@pytest.mark.parametrize("name", ["circle130", "ellipsoid42"])
def test_apply_write_set_and_timer(name):
    """eb_apply writes A x at the CPs and 0 at the other node of every x-pair
    (2j, 2j + 1) holding a CP, and nothing else; eb_time_apply leaves the same
    y and reports a positive time."""
    grid, ls = CASES[name]()
    eb = _eb()
    h = eb.EB(grid, ls)
    ref = oeb.build(grid, ls)
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.standard_normal(grid.shape()), device="cuda")
    for dt in (torch.float64, torch.float32):
        xd = x.to(dt)
        fill = torch.full_like(xd, 7.0)
        y = h.apply(xd, out=fill.clone()).reshape(-1).double().cpu().numpy()
        cp = np.zeros(y.size, bool)
        cp[ref.cp_nodes] = True
        pair = cp.reshape(-1, 2).any(axis=1).repeat(2)
        assert np.all(y[~pair] == 7.0)
        assert np.all(y[pair & ~cp] == 0.0)
        y_ref = ref.A @ ref.from_grid(x.cpu().numpy())
        tol = 1e-14 if dt == torch.float64 else 1e-6
        assert np.linalg.norm(y[ref.cp_nodes] - y_ref) / np.linalg.norm(y_ref) <= tol
        y2 = fill.clone()
        us = h.time_apply_us(xd, y2, launches=3, clear_bytes=1 << 20)
        assert us > 0.0
        assert np.array_equal(y2.reshape(-1).double().cpu().numpy(), y)


def test_full_size_wave_geometry_star_4096():
    """The star of the wave workload at its full 4096^2 size: classes, cut list,
    diagonal; apply on sampled outputs."""
    grid, ls = ei.star_wave(4096)
    h, ref = _compare_build(grid, ls, exact=False)
    assert h.info.min_abs_psi > 1e-12
    rng = np.random.default_rng(1)
    x = rng.standard_normal(grid.shape())
    y = h.apply(torch.tensor(x, device="cuda")).cpu().numpy().reshape(-1)
    k = rng.choice(ref.num_cp, 20000, replace=False)
    xc = ref.from_grid(x)
    y_ref = ref.A[k] @ xc
    got = y[ref.cp_nodes[k]]
    assert np.abs(got - y_ref).max() <= 1e-13 * np.abs(y_ref).max()


def test_full_size_ellipsoid_256():
    grid, ls = ei.ellipsoid_k3(256, seed=0)
    h, ref = _compare_build(grid, ls, exact=True)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(grid.shape())
    y = h.apply(torch.tensor(x, device="cuda")).cpu().numpy().reshape(-1)
    y_ref = ref.A @ ref.from_grid(x)
    got = y[ref.cp_nodes]
    assert np.linalg.norm(got - y_ref) / np.linalg.norm(y_ref) <= 1e-14


def test_geometry_errors():
    eb = _eb()
    grid = ei.box_grid(2, 64)
    with pytest.raises(eb.EBError) as e:
        eb.EB(grid, ei.sphere((0.0, 0.0), 1.5))       # covers the border ring
    assert e.value.code == eb.EB_ERR_GEOMETRY
    with pytest.raises(eb.EBError) as e:
        eb.EB(grid, ei.sphere((0.0, 0.0), 0.01))      # no computational point
    assert e.value.code == eb.EB_ERR_GEOMETRY
    bad = ei.box_grid(2, 63)                          # odd n0
    with pytest.raises(eb.EBError) as e:
        eb.EB(bad, ei.sphere((0.0, 0.0), 0.5))
    assert e.value.code == eb.EB_ERR_INVALID
