"""Tile shapes and the autotuner on the GPU.

* eb_apply (FP64 / FP32 / BF16) and the leapfrog step give bit-identical
  results at the CPs with every candidate tile shape (each node's arithmetic
  does not depend on how nodes are grouped into CTAs).
* AMG-PCG after a retile (its captured iteration is rebuilt): same iteration
  count within 1, solutions within 1e-12 relative (the reduction partials
  are grouped by tile, so the rounding of the dot products differs).
* eb_autotune / amg_autotune / batch_autotune time every candidate, leave the
  fastest shape in use, and the batched heat step still matches its own
  result with the default shape.
* invalid shapes are rejected with EB_ERR_INVALID.
"""
import math

import numpy as np
import pytest
import torch

import eb_inputs as ei

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def _pkg():
    import paper_2204_06083_gb300 as eb
    return eb


SHAPES2 = [(32, 8, 1), (64, 4, 1), (16, 16, 1), (128, 2, 1), (8, 32, 1), (2, 128, 1)]
SHAPES3 = [(16, 4, 4), (32, 4, 2), (8, 8, 4), (16, 8, 2), (32, 2, 4), (64, 2, 2), (8, 4, 8), (16, 2, 8),
           (32, 8, 1), (2, 8, 16)]


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_apply_and_leapfrog_independent_of_tile_shape(case):
    eb = _pkg()
    if case == "2d":
        grid, ls = ei.box_grid(2, 250), ei.random_star(5)
        shapes = SHAPES2
    else:
        grid, ls = ei.ellipsoid_k3(66, seed=3)
        shapes = SHAPES3
    h = eb.EB(grid, ls)
    rng = np.random.default_rng(1)
    x = torch.from_numpy(rng.standard_normal(h.shape())).cuda()
    refs = {}
    for dt in (torch.float64, torch.float32, torch.bfloat16):
        refs[dt] = h.apply(x.to(dt))
    # the leapfrog writes the nodes of the active tiles only (0 off the CPs),
    # and which tiles are active depends on the shape: compare the CPs
    cp = (h.classes() & eb.CODE_CP) != 0
    dtw = 0.5 * grid.h / math.sqrt(grid.dim)
    ua, ub = x.clone(), x.clone() * 0.5
    h.wave_step(ua, ub, dtw, 7)
    for shape in shapes:
        h.retile(shape)
        assert h.info.tile == shape
        for dt, ref in refs.items():
            assert torch.equal(h.apply(x.to(dt)), ref), (shape, dt)
        va, vb = x.clone(), x.clone() * 0.5
        h.wave_step(va, vb, dtw, 7)
        assert torch.equal(va[cp], ua[cp]) and torch.equal(vb[cp], ub[cp]), shape


def test_pcg_after_retile():
    eb = _pkg()
    grid, ls = ei.ellipsoid_k3(80, seed=1)
    h = eb.EB(grid, ls)
    amg = eb.AMG(h, vcycle_prec=eb.EB_F32)
    b = torch.from_numpy(np.random.default_rng(2).standard_normal(h.shape())).cuda()
    x0, st0 = amg.solve(b, rtol=1e-12)
    for shape in [(32, 4, 2), (8, 8, 4), (16, 4, 4)]:
        h.retile(shape)
        x1, st1 = amg.solve(b, rtol=1e-12)
        assert abs(st1.iterations - st0.iterations) <= 1
        assert torch.linalg.norm(x1 - x0) <= 1e-10 * torch.linalg.norm(x0)


def test_invalid_shapes_rejected():
    eb = _pkg()
    h = eb.EB(ei.box_grid(2, 64), ei.random_star(3))
    for bad in [(16, 8, 1), (32, 8, 2), (1, 256, 1), (256, 1, 1), (24, 8, 1)]:
        with pytest.raises(eb.EBError) as e:
            h.retile(bad)
        assert e.value.code == eb.EB_ERR_INVALID
    assert h.info.tile == (32, 8, 1)


def test_autotuners():
    eb = _pkg()
    grid, ls = ei.ellipsoid_k3(96, seed=0)
    h = eb.EB(grid, ls)
    res = h.autotune(eb.EB_F32, reps=5)
    assert len(res.shapes) == 10
    resw = h.autotune(eb.EB_F32, reps=2, op=eb.EB_TUNE_LEAPFROG)
    assert h.info.tile == resw.shape and min(resw.us) == resw.us[resw.best]
    res = h.autotune(eb.EB_F32, reps=5)
    assert h.info.tile == res.shape and min(res.us) == res.us[res.best] and all(u > 0 for u in res.us)
    amg = eb.AMG(h, vcycle_prec=eb.EB_F32)
    b = torch.from_numpy(np.random.default_rng(3).standard_normal(h.shape())).cuda()
    x0, st0 = amg.solve(b, rtol=1e-11)
    res2 = amg.autotune(reps=3)
    assert h.info.tile == res2.shape
    x1, st1 = amg.solve(b, rtol=1e-11)
    assert abs(st1.iterations - st0.iterations) <= 1
    assert torch.linalg.norm(x1 - x0) <= 1e-9 * torch.linalg.norm(x0)


def test_batch_autotune_keeps_results():
    eb = _pkg()
    grids = [ei.box_grid(2, n) for n in (96, 160, 130)]
    lss = [ei.random_star(s) for s in (41, 42, 43)]
    dts = [g.h for g in grids]
    outs = []
    for tune in (False, True):
        B = eb.Batch(grids, lss)
        B.heat_setup(dts, 1.0, vcycle_prec=eb.EB_F32)
        if tune:
            res = B.autotune(reps=3)
            assert len(res.shapes) == 5 and min(res.us) == res.us[res.best]
        u = B.zeros()
        for g, gr in enumerate(grids):
            X, Y = ei.grid_points(gr)
            B.view(u, g).copy_(torch.tensor(ei.u_heat(X, Y, 0.0)))
        f = B.zeros()
        for g, gr in enumerate(grids):
            X, Y = ei.grid_points(gr)
            B.view(f, g).copy_(torch.tensor(-ei.f_heat(X, Y, 0.0)))
        ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device="cuda")
        b1 = B.rhs(f, ug)
        for _ in range(3):
            B.heat_step(u, b1, rtol=1e-12)
        # the CPs of every geometry (nodes outside the active tiles are not written)
        outs.append(torch.cat([B.view(u, g)[(B.geometry(g).classes() & eb.CODE_CP) != 0]
                               for g in range(len(grids))]))
    assert torch.linalg.norm(outs[1] - outs[0]) <= 1e-10 * torch.linalg.norm(outs[0])


def test_amg_on_batch_geometry_outlives_batch_variable():
    """An AMG hierarchy built on a geometry borrowed from a batch keeps the
    batch alive after the last direct reference to the batch is dropped."""
    import gc
    eb = _pkg()
    grids = [ei.box_grid(2, n) for n in (64, 96)]
    B = eb.Batch(grids, [ei.random_star(s) for s in (1, 2)])
    amg = eb.AMG(B.geometry(1), 1.0 / grids[1].h)
    del B
    gc.collect()
    b = torch.ones(amg.eb.shape(), dtype=torch.float64, device="cuda")
    x, st = amg.solve(b, rtol=1e-10)
    assert st.converged
    del amg
    gc.collect()


def test_csr_group_tuning_keeps_results():
    eb = _pkg()
    grid, ls = ei.ellipsoid_k3(80, seed=2)
    h = eb.EB(grid, ls)
    amg = eb.AMG(h, vcycle_prec=eb.EB_F32)
    b = torch.from_numpy(np.random.default_rng(9).standard_normal(h.shape())).cuda()
    z0 = amg.vcycle(b)
    x0, st0 = amg.solve(b, rtol=1e-11)
    best, us = amg.tune_csr(reps=3)
    assert best in (1, 2, 4, 8) and min(us.values()) == us[best]
    z1 = amg.vcycle(b)
    assert torch.linalg.norm(z1 - z0) <= 1e-5 * torch.linalg.norm(z0)   # FP32 sums regrouped
    x1, st1 = amg.solve(b, rtol=1e-11)
    assert abs(st1.iterations - st0.iterations) <= 1
    assert torch.linalg.norm(x1 - x0) <= 1e-9 * torch.linalg.norm(x0)
    # a cached choice is applied without timing; other values are rejected
    other = 8 if best != 8 else 1
    amg.set_csr_epl(other)
    x2, st2 = amg.solve(b, rtol=1e-11)
    assert abs(st2.iterations - st0.iterations) <= 1
    assert torch.linalg.norm(x2 - x0) <= 1e-9 * torch.linalg.norm(x0)
    with pytest.raises(eb.EBError) as e:
        amg.set_csr_epl(3)
    assert e.value.code == eb.EB_ERR_INVALID


def test_handles_destroyed_in_any_order():
    """Cycle collection finalizes objects in any order: a hierarchy destroyed
    after its grid must not touch the grid."""
    eb = _pkg()
    h = eb.EB(ei.box_grid(2, 96), ei.random_star(7))
    amg = eb.AMG(h)
    eb.load().eb_destroy(h.handle)   # the grid first ...
    h._h = type(h._h)()
    amg.close()                      # ... then the hierarchy
