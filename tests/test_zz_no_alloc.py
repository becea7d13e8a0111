"""wave_step_noalloc against wave_step, through the C ABI.

wave_step_noalloc serves callers that cannot allocate memory while they run
(loops with a fixed memory budget, programs whose device memory belongs to
another framework's pool): it keeps the state of its grid-wide barrier in a
fixed device array of the library instead of allocating anything.  It must
give the same fields as wave_step.  Two calls in a row check that the shared
array, which keeps the previous call's contents, is cleared correctly.  This
file is collected last so that a run stopping at its first failure has run
every other test before it.
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import eb_inputs as ei

pytestmark = pytest.mark.gpu

# Both entry points run the same per-node expression (one shared device
# function, the same compiled contraction), so the fields must agree bit for bit.


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2204_06083_gb300 as eb
    return eb


def _fields(eb, h, grid, dtype):
    X, Y = ei.grid_points(grid)
    c, w = ei.pulse_params(2)
    u0 = torch.tensor(ei.pulse(X, Y, c, max(w, 4 * grid.h)), device="cuda", dtype=dtype)
    code = h.classes()
    u0 = torch.where((code & eb.CODE_CP) != 0, u0, torch.zeros_like(u0))
    dt = 0.9 * grid.h / math.sqrt(2.0)
    u1 = u0 - 0.5 * dt * dt * h.apply(u0)
    return u0.contiguous(), u1.contiguous(), dt


def _call(eb, fn, h, dtype, ua, ub, dt, nsteps):
    prec = eb.EB_F64 if dtype == torch.float64 else eb.EB_F32
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(h.handle, prec, C.c_double(dt), C.c_void_p(ua.data_ptr()), C.c_void_p(ub.data_ptr()), nsteps, stream)
    assert rc == eb.EB_OK, eb.load().eb_last_error().decode()


def _same(a, b):
    return bool(torch.equal(a, b))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_wave_step_twice(lib, dtype):
    eb = lib
    L = eb.load()
    grid, ls = ei.box_grid(2, 258), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])
    h = eb.EB(grid, ls)
    u0, u1, dt = _fields(eb, h, grid, dtype)
    ref_a, ref_b = u0.clone(), u1.clone()
    new_a, new_b = u0.clone(), u1.clone()
    for nsteps in (37, 12):   # odd then even step counts; the second call continues the first
        _call(eb, L.wave_step, h, dtype, ref_a, ref_b, dt, nsteps)
        _call(eb, L.wave_step_noalloc, h, dtype, new_a, new_b, dt, nsteps)
        torch.cuda.synchronize()
        assert _same(new_b, ref_b)
        assert _same(new_a, ref_a)


def test_noalloc_3d_and_invalid_arguments(lib):
    eb = lib
    L = eb.load()
    grid, ls = ei.ellipsoid_k3(34, seed=1)
    h = eb.EB(grid, ls)
    rng = np.random.default_rng(0)
    code = h.classes()
    u0 = torch.tensor(rng.standard_normal(h.shape()), device="cuda")
    u0 = torch.where((code & eb.CODE_CP) != 0, u0, torch.zeros_like(u0)).contiguous()
    u1 = (0.99 * u0).contiguous()
    dt = 0.5 * grid.h / math.sqrt(3.0)
    ra, rb, na, nb = u0.clone(), u1.clone(), u0.clone(), u1.clone()
    _call(eb, L.wave_step, h, torch.float64, ra, rb, dt, 9)
    _call(eb, L.wave_step_noalloc, h, torch.float64, na, nb, dt, 9)
    torch.cuda.synchronize()
    assert _same(nb, rb) and _same(na, ra)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.wave_step_noalloc(h.handle, eb.EB_BF16, C.c_double(dt), C.c_void_p(na.data_ptr()),
                             C.c_void_p(nb.data_ptr()), 1, stream)
    assert rc == eb.EB_ERR_INVALID
    rc = L.wave_step_noalloc(h.handle, eb.EB_F64, C.c_double(dt), C.c_void_p(na.data_ptr()),
                             C.c_void_p(na.data_ptr()), 1, stream)
    assert rc == eb.EB_ERR_INVALID


@pytest.mark.parametrize("nsteps", [1, 2])
def test_noalloc_short_runs_clear_non_cp_entries(lib, nsteps):
    """One or two steps from fields whose non-CP entries hold arbitrary values:
    both entry points must ignore those inputs and leave the same fields (a
    single step never writes the older field, so its non-CP entries must be
    cleared explicitly)."""
    eb = lib
    L = eb.load()
    grid, ls = ei.box_grid(2, 130), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])
    h = eb.EB(grid, ls)
    u0, u1, dt = _fields(eb, h, grid, torch.float64)
    rng = np.random.default_rng(7)
    cp = (h.classes() & eb.CODE_CP) != 0
    junk0 = torch.tensor(rng.standard_normal(h.shape()), device="cuda")
    junk1 = torch.tensor(rng.standard_normal(h.shape()), device="cuda")
    u0 = torch.where(cp, u0, junk0).contiguous()
    u1 = torch.where(cp, u1, junk1).contiguous()
    ra, rb, na, nb = u0.clone(), u1.clone(), u0.clone(), u1.clone()
    _call(eb, L.wave_step, h, torch.float64, ra, rb, dt, nsteps)
    _call(eb, L.wave_step_noalloc, h, torch.float64, na, nb, dt, nsteps)
    torch.cuda.synchronize()
    assert _same(na, ra) and _same(nb, rb)
