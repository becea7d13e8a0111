"""GPU parity of the batched form: several stars of uneven size advanced by
one batch_heat_step per time step (per-geometry PCG recurrences, one AMG
hierarchy on the block-diagonal operator), against the oracle doing the same
steps geometry by geometry with the hierarchy of the same block-diagonal
matrix.  Tolerance: both sides solve to rtol 1e-13; solutions within rel-L2
1e-10 per geometry (kappa_hat * rtol bound of the shifted operators)."""
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


def _case(sizes, seeds):
    grids = [ei.box_grid(2, n) for n in sizes]
    lss = [ei.random_star(s) for s in seeds]
    return grids, lss


def _oracle_batch(grids, lss, dts, theta):
    refs = [oeb.build(g, l) for g, l in zip(grids, lss)]
    blocks = [oeb.assemble_unit(r, g.h ** 2 / (theta * dt)) for r, g, dt in zip(refs, grids, dts)]
    H = oamg.setup(sp.block_diag(blocks, format="csr"))
    offs = np.cumsum([0] + [r.num_cp for r in refs])
    return refs, blocks, H, offs


def _run(vprec, sizes=(64, 96, 130), seeds=(21, 22, 23), nsteps=3, outer=0, rtol=1e-13, tol=1e-10):
    import paper_2204_06083_gb300 as eb
    grids, lss = _case(sizes, seeds)
    dts = [g.h for g in grids]
    theta = 1.0
    B = eb.Batch(grids, lss)
    B.heat_setup(dts, theta=theta, vcycle_prec=vprec)
    B.set_outer(outer)
    refs, blocks, H, offs = _oracle_batch(grids, lss, dts, theta)
    ntot = offs[-1]

    def M_block(g):
        def M(r):
            full = np.zeros(ntot)
            full[offs[g]:offs[g + 1]] = r
            return oamg.vcycle(H, full)[offs[g]:offs[g + 1]]
        return M

    u = B.zeros()
    u_ref = []
    for g, (gr, r) in enumerate(zip(grids, refs)):
        X, Y = ei.grid_points(gr)
        B.view(u, g).copy_(torch.tensor(ei.u_heat(X, Y, 0.0)))
        u_ref.append(r.from_grid(ei.u_heat(X, Y, 0.0)))
    iters = []
    for k in range(nsteps):
        t1 = (k + 1) * np.array(dts)
        mf = B.zeros()
        ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device="cuda")
        b1_ref = []
        for g, (gr, r) in enumerate(zip(grids, refs)):
            X, Y = ei.grid_points(gr)
            F = -ei.f_heat(X, Y, t1[g])
            ugc = ei.u_heat(r.cut_xg[:, 0], r.cut_xg[:, 1], t1[g])
            B.view(mf, g).copy_(torch.tensor(F))
            ug[B.cut_off[g]:B.cut_off[g + 1]] = torch.tensor(ugc)
            b1_ref.append(oeb.rhs(r, F, ugc))
        b1 = B.rhs(mf, ug)
        for g, r in enumerate(refs):
            got = r.from_grid(B.view(b1, g).cpu().numpy())
            assert np.abs(got - b1_ref[g]).max() <= 1e-11 * np.abs(b1_ref[g]).max()
        st = B.heat_step(u, b1, rtol=rtol, maxit=300)
        iters.append([s.iterations for s in st])
        for g, (gr, r) in enumerate(zip(grids, refs)):
            h2 = gr.h ** 2
            rhs = h2 * (u_ref[g] / dts[g] + b1_ref[g])
            u_ref[g], _ = osol.pcg(blocks[g], rhs, x0=u_ref[g], M=M_block(g), rtol=1e-14, maxit=500)
    for g, r in enumerate(refs):
        got = r.from_grid(B.view(u, g).cpu().numpy())
        e = np.linalg.norm(got - u_ref[g]) / np.linalg.norm(u_ref[g])
        assert e <= tol, (g, e)
    return iters


def test_batched_heat_df_outer_matches_oracle():
    """The batched PCG in double-float (batch_set_outer_prec EB_DF64): solved
    to rtol 1e-12 (DF carries about 48 bits; the exit test is the FP64 true
    residual), per-geometry rel-L2 <= 1e-9 against the oracle's steps."""
    import paper_2204_06083_gb300 as eb
    _run(eb.EB_F32, outer=eb.EB_DF64, rtol=1e-12, tol=1e-9)


def test_batched_df_outer_against_fp64_outer():
    """Same batch, one step to 1e-10 with the FP64 and the DF outer iteration:
    per-geometry iteration counts within 1, solutions within rel-L2 1e-8; the
    device-side loop and the host-checked loop (profiling on) of the DF
    iteration give the same solution bit for bit; an FP64 V-cycle or an
    unknown precision is refused."""
    import paper_2204_06083_gb300 as eb
    grids, lss = _case((64, 96, 130, 80), (31, 32, 33, 34))
    dts = [g.h for g in grids]
    B = eb.Batch(grids, lss)
    B.heat_setup(dts, theta=1.0, vcycle_prec=eb.EB_F32)
    u0 = B.zeros()
    mf = B.zeros()
    ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device="cuda")
    for g, gr in enumerate(grids):
        X, Y = ei.grid_points(gr)
        B.view(u0, g).copy_(torch.tensor(ei.u_heat(X, Y, 0.0)))
        B.view(mf, g).copy_(torch.tensor(-ei.f_heat(X, Y, dts[g])))
        xg = B.geometry(g).cuts()[3].cpu().numpy()
        ug[B.cut_off[g]:B.cut_off[g + 1]] = torch.tensor(ei.u_heat(xg[:, 0], xg[:, 1], dts[g]))
    b1 = B.rhs(mf, ug)
    out = {}
    for outer in (eb.EB_F64, eb.EB_DF64):
        B.set_outer(outer)
        u = u0.clone()
        st = B.heat_step(u, b1, rtol=1e-10, maxit=300)
        assert all(s.converged and s.true_rel_residual <= 1e-10 for s in st)
        out[outer] = (u, [s.iterations for s in st])
    print("iterations FP64 / DF outer:", out[eb.EB_F64][1], out[eb.EB_DF64][1])
    for a, b in zip(out[eb.EB_F64][1], out[eb.EB_DF64][1]):
        assert abs(a - b) <= 1
    for g in range(B.count):
        x64, xdf = B.view(out[eb.EB_F64][0], g), B.view(out[eb.EB_DF64][0], g)
        assert (torch.linalg.norm(xdf - x64) / torch.linalg.norm(x64)).item() <= 1e-8
    B.set_outer(eb.EB_DF64)
    B.set_profile(True)
    u = u0.clone()
    B.heat_step(u, b1, rtol=1e-10, maxit=300)
    B.set_profile(False)
    assert torch.equal(u, out[eb.EB_DF64][0])
    with pytest.raises(eb.EBError) as e:
        B.set_outer(7)
    assert e.value.code == eb.EB_ERR_INVALID
    B64 = eb.Batch(grids[:2], lss[:2])
    B64.heat_setup(dts[:2], theta=1.0)
    B64.set_outer(eb.EB_DF64)
    uu = B64.zeros()
    with pytest.raises(eb.EBError) as e:
        B64.heat_step(uu, B64.zeros(), rtol=1e-10, maxit=10)
    assert e.value.code == eb.EB_ERR_NOT_IMPLEMENTED


def test_batched_heat_fp64_vcycle_matches_oracle():
    its = _run(0)
    assert max(max(i) for i in its) < 40


def test_batched_heat_fp32_vcycle_matches_oracle():
    import paper_2204_06083_gb300 as eb
    _run(eb.EB_F32)


def test_batch_geometry_handles_and_layout():
    import paper_2204_06083_gb300 as eb
    grids, lss = _case((64, 128), (31, 32))
    B = eb.Batch(grids, lss)
    assert B.count == 2 and B.stride == 128
    assert B.node_off[1] == 64 * 128 and B.node_off[2] == 64 * 128 + 128 * 128
    for g in range(2):
        h = B.geometry(g)
        ref = oeb.build(grids[g], lss[g])
        assert h.info.num_cp == ref.num_cp
        assert B.cp_off[g + 1] - B.cp_off[g] == ref.num_cp


def test_full_size_batch_64_stars_matches_oracle():
    """The batched workload at its full size: the 64 seeded stars of 128^2 to
    1024^2 nodes (about 5M unknowns), FP32 V-cycle on the block-diagonal
    hierarchy with per-geometry flexible FP64 PCG as the benchmark runs it,
    two backward-Euler steps (dt = h per geometry, warm start) of the
    manufactured heat solution solved to rtol 1e-13.  The oracle solves the
    same steps geometry by geometry with a sparse LU factorisation of each
    h^2 (I/dt + A) block; per-geometry rel-L2 <= 1e-10 (kappa * rtol of the
    shifted operators, kappa ~ 1/h); the double-float outer iteration of the
    same batch to rtol 1e-12, per-geometry rel-L2 <= 1e-9."""
    import scipy.sparse.linalg as spla
    import paper_2204_06083_gb300 as eb
    cfg = ei.star_batch(64, 0)
    grids = [ei.box_grid(2, n) for n, _ in cfg]
    lss = [ls for _, ls in cfg]
    dts = [g.h for g in grids]
    B = eb.Batch(grids, lss)
    B.heat_setup(dts, theta=1.0, vcycle_prec=eb.EB_F32)
    refs = [oeb.build(g, l) for g, l in zip(grids, lss)]
    assert [B.cp_off[g + 1] - B.cp_off[g] for g in range(64)] == [r.num_cp for r in refs]
    lus = [spla.splu(oeb.assemble_unit(r, g.h ** 2 / dt).tocsc()) for r, g, dt in zip(refs, grids, dts)]
    # the FP64 and the double-float outer iteration (batch_set_outer_prec), the
    # latter to rtol 1e-12 (its exit test is the FP64 true residual)
    for outer, rtol, tol in ((eb.EB_F64, 1e-13, 1e-10), (eb.EB_DF64, 1e-12, 1e-9)):
        B.set_outer(outer)
        u = B.zeros()
        u_ref = []
        for g, (gr, r) in enumerate(zip(grids, refs)):
            X, Y = ei.grid_points(gr)
            B.view(u, g).copy_(torch.tensor(ei.u_heat(X, Y, 0.0)))
            u_ref.append(r.from_grid(ei.u_heat(X, Y, 0.0)))
        for k in range(2):
            mf = B.zeros()
            ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device="cuda")
            b1_ref = []
            for g, (gr, r) in enumerate(zip(grids, refs)):
                t1 = (k + 1) * dts[g]
                X, Y = ei.grid_points(gr)
                F = -ei.f_heat(X, Y, t1)
                ugc = ei.u_heat(r.cut_xg[:, 0], r.cut_xg[:, 1], t1)
                B.view(mf, g).copy_(torch.tensor(F))
                ug[B.cut_off[g]:B.cut_off[g + 1]] = torch.tensor(ugc)
                b1_ref.append(oeb.rhs(r, F, ugc))
            b1 = B.rhs(mf, ug)
            st = B.heat_step(u, b1, rtol=rtol, maxit=400)
            assert all(s.converged for s in st)
            for g, gr in enumerate(grids):
                u_ref[g] = lus[g].solve(gr.h ** 2 * (u_ref[g] / dts[g] + b1_ref[g]))
        worst = 0.0
        for g, r in enumerate(refs):
            got = r.from_grid(B.view(u, g).cpu().numpy())
            e = np.linalg.norm(got - u_ref[g]) / np.linalg.norm(u_ref[g])
            worst = max(worst, e)
            assert e <= tol, (outer, g, grids[g].n[0], e)
        print(f"64-star batch, 2 steps, outer {outer}: worst per-geometry rel-L2 {worst:.2e}")


def test_batch_level0_tensor_copy_step_bit_identical():
    """The level-0 Chebyshev steps fed by tensor copies (batch_set_level0_tma,
    the default for FP32 batched V-cycles with tiles 16-128 nodes wide and a
    row stride that is a multiple of 16 nodes) give the same heat step, bit
    for bit, as the per-thread sweep kernel: the default 32 x 8 tiles, then
    whatever shape the batch autotuner picks; also in double-float."""
    import paper_2204_06083_gb300 as eb
    grids, lss = _case((96, 128, 160, 112), (41, 42, 43, 44))
    dts = [g.h for g in grids]
    B = eb.Batch(grids, lss)
    assert B.stride % 16 == 0
    B.heat_setup(dts, theta=1.0, vcycle_prec=eb.EB_F32)
    u0 = B.zeros()
    mf = B.zeros()
    ug = torch.zeros(max(B.num_cut, 1), dtype=torch.float64, device="cuda")
    for g, gr in enumerate(grids):
        X, Y = ei.grid_points(gr)
        B.view(u0, g).copy_(torch.tensor(ei.u_heat(X, Y, 0.0)))
        B.view(mf, g).copy_(torch.tensor(-ei.f_heat(X, Y, dts[g])))
        xg = B.geometry(g).cuts()[3].cpu().numpy()
        ug[B.cut_off[g]:B.cut_off[g + 1]] = torch.tensor(ei.u_heat(xg[:, 0], xg[:, 1], dts[g]))
    b1 = B.rhs(mf, ug)

    def run():
        out = {}
        for on in (True, False):
            B.set_level0_tma(on)
            u = u0.clone()
            st = B.heat_step(u, b1, rtol=1e-10, maxit=300)
            assert all(s.converged for s in st)
            out[on] = (u, [s.iterations for s in st])
        assert out[True][1] == out[False][1]
        assert torch.equal(out[True][0], out[False][0])

    run()
    B.set_outer(eb.EB_DF64)
    run()
    B.set_outer(eb.EB_F64)
    B.autotune(reps=3)
    run()
