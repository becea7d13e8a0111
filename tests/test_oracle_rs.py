"""Pins of the oracle's classical (Ruge-Stueben) coarsening and of the
W-cycle, the paper's AMG variants (Sec. 3), CPU only.

* strength: the row-max criterion, checked entry by entry on a dense copy;
* PMIS splitting: every F point that influences others strongly depends on a
  C point; C points chosen in one round are not strongly connected;
* direct interpolation: C rows inject; on rows of zero row sum (interior CPs)
  the weights sum to 1, so P reproduces constants there; weights positive for
  an M-matrix; the Galerkin product checked densely;
* the W-cycle is a symmetric operator; with two levels it equals the V-cycle;
* iteration counts (Sec. 3.1: W-cycle iterations independent of the size, the
  V-cycle's growing slowly, O(DOF^0.19)): W-cycle counts within +-2 over n =
  128..512 and a V-cycle growth exponent below 0.25 on the K1 circle.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import eb_inputs as ei
from oracle import amg, eb, solvers


def _sys(n=64):
    grid, ls = ei.circle_k1(n)
    return grid, eb.build(grid, ls)


def test_strength_row_max_criterion_dense():
    _, s = _sys(40)
    A = s.A.toarray()
    S = amg.strength_rs(s.A).toarray() > 0
    for i in range(A.shape[0]):
        off = [j for j in range(A.shape[0]) if j != i and A[i, j] != 0]
        m = max(-A[i, j] for j in off) if off else 0.0
        for j in off:
            want = m > 0 and np.float32(-A[i, j]) >= np.float32(0.25 * m)
            assert S[i, j] == want
        assert not S[i, i]


def test_pmis_splitting_properties():
    _, s = _sys(96)
    S = amg.strength_rs(s.A)
    cf = amg.pmis(S)
    lam = np.diff(S.T.tocsr().indptr)
    Sd = S.tocsr()
    for i in np.flatnonzero(cf == 0):
        if lam[i] > 0:
            deps = Sd.indices[Sd.indptr[i]:Sd.indptr[i + 1]]
            assert (cf[deps] == 1).any(), i
    assert 0.1 < cf.mean() < 0.6


def test_direct_interpolation_properties_and_galerkin():
    grid, s = _sys(48)
    A = s.A
    S = amg.strength_rs(A)
    cf = amg.pmis(S)
    P = amg.direct_interpolation(A, S, cf).toarray()
    cidx = np.cumsum(cf) - 1
    for i in np.flatnonzero(cf == 1):
        row = np.zeros(P.shape[1])
        row[cidx[i]] = 1.0
        assert np.array_equal(P[i], row)
    Ad = A.toarray()
    rowsum = Ad.sum(axis=1)
    interior = (np.abs(rowsum) < 1e-12 * np.abs(np.diag(Ad))) & (cf == 0)
    has = P.sum(axis=1) != 0
    assert np.allclose(P[interior & has].sum(axis=1), 1.0, rtol=0, atol=1e-13)
    assert (P >= 0).all()
    old = amg.COARSE_MAX
    try:
        amg.COARSE_MAX = 10
        H = amg.setup(A, "rs")
    finally:
        amg.COARSE_MAX = old
    Ac = P.T @ Ad @ P
    assert np.abs(H.levels[1].A.toarray() - Ac).max() <= 1e-12 * np.abs(Ac).max()
    assert np.linalg.eigvalsh(Ac)[0] > 0


@pytest.mark.parametrize("coarsening", ["sa", "rs"])
def test_w_cycle_symmetric_and_two_level_equals_v(coarsening):
    grid, s = _sys(256)
    H = amg.setup(s.A, coarsening)
    assert len(H.levels) >= 3
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(s.num_cp), rng.standard_normal(s.num_cp)
    Mx, My = amg.vcycle(H, x, gamma=2), amg.vcycle(H, y, gamma=2)
    assert abs(Mx @ y - x @ My) <= 1e-12 * abs(Mx @ y)
    assert x @ Mx > 0
    H2 = amg.Hierarchy(levels=H.levels[:2], coarse_chol=None)
    import scipy.linalg as sla
    H2.coarse_chol = sla.cho_factor(H.levels[1].A.toarray(), lower=True)
    assert np.array_equal(amg.vcycle(H2, x, gamma=2), amg.vcycle(H2, x, gamma=1))


def test_iteration_counts_w_flat_v_slow_growth():
    w_its, v_its, dofs = [], [], []
    for n in (128, 256, 512):
        grid, s = _sys(n)
        X, Y = ei.grid_points(grid)
        b = eb.rhs(s, ei.f_k1(X, Y), ei.u_k1(s.cut_xg[:, 0], s.cut_xg[:, 1]))
        H = amg.setup(s.A, "rs")
        _, sw = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r, gamma=2), rtol=1e-12)
        _, sv = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r, gamma=1), rtol=1e-12)
        w_its.append(sw.iterations)
        v_its.append(sv.iterations)
        dofs.append(s.num_cp)
    assert max(w_its) - min(w_its) <= 2, w_its
    expo = math.log(v_its[-1] / v_its[0]) / math.log(dofs[-1] / dofs[0])
    assert expo < 0.25, (v_its, expo)
