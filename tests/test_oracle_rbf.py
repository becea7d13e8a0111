"""Pins of the oracle's RBF closure (Sec. 2.2, eqs. 7-9, Algorithm 2) and of
the mixed method (Sec. 2.3), CPU only.

* the cubic-RBF-plus-linear interpolant's weights reproduce constants and
  linear functions at x_BP (the polynomial augmentation), and give (1, 0, 0)
  when x_BP is the interior point itself;
* closest points lie on Gamma, the segment to them is normal to Gamma, and no
  dense sample of Gamma is nearer;
* Algorithm 2: with the mixed method the two boundary points are always
  distinct for eps = 0.025 (the paper's observation, Sec. 2.3); with RBF
  everywhere the rotated branch occurs, its G2 lies on Gamma at pi/4 from G1;
* a harmonic linear u is reproduced exactly by the mixed and RBF-based
  methods on a non-convex star;
* on the star r = 0.5 + 0.1 sin 5 phi the mixed method is second order in the
  max norm (the line-by-line-only closure with far crossings is first order);
* the matrix stays symmetric and every segment meets Lemma 1 (Sec. 2.4).
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import eb_inputs as ei
from oracle import eb, geometry


def _star(n=96, amp=0.1):
    return ei.box_grid(2, n), ei.star(ei.STAR_CENTER, 0.5, [5], [amp], [0.0])


def test_rbf_weights_reproduce_linear_functions():
    rng = np.random.default_rng(0)
    h = 0.01
    for _ in range(20):
        x_bp = rng.uniform(-1, 1, 2)
        x_ij = x_bp + np.array([h, 0.0])
        g1 = x_bp + rng.uniform(-1.5, 0.2, 2) * h
        g2 = x_bp + rng.uniform(-0.5, 1.5, 2) * h
        w = np.array(eb.rbf_weights(x_ij, g1, g2, x_bp, h))
        pts = np.array([x_ij, g1, g2])
        assert abs(w.sum() - 1.0) < 1e-12
        assert abs(w @ pts[:, 0] - x_bp[0]) < 1e-12 and abs(w @ pts[:, 1] - x_bp[1]) < 1e-12
    w = eb.rbf_weights((0.3, 0.2), (0.25, 0.21), (0.31, 0.15), (0.3, 0.2), 0.01)
    assert np.allclose(w, (1.0, 0.0, 0.0), atol=1e-12)


@pytest.mark.parametrize("shape", ["star", "ellipse"])
def test_closest_point(shape):
    ls = ei.star(ei.STAR_CENTER, 0.5, [5], [0.2], [0.0]) if shape == "star" else \
        ei.ellipsoid((0.02, 0.01), (0.7, 0.4), ei.random_rotation(3))
    ts = np.linspace(0, 2 * np.pi, 200001)
    (gx, gy), _, _ = geometry.curve(ls, ts)
    rng = np.random.default_rng(1)
    for _ in range(10):
        p = rng.uniform(-0.3, 0.3, 2)
        x, y, t = geometry.closest_point(ls, p)
        psi = geometry.psi_points(ls, 2, [np.array([x]), np.array([y])])[0]
        assert abs(psi) < 1e-12
        _, (tx, ty), _ = geometry.curve(ls, t)
        assert abs((x - p[0]) * tx + (y - p[1]) * ty) < 1e-10 * math.hypot(tx, ty)
        d = math.hypot(x - p[0], y - p[1])
        assert d <= np.min(np.hypot(gx - p[0], gy - p[1])) + 1e-9


def test_algorithm2_branches():
    grid, ls = _star(160, 0.2)
    mixed = eb.build(grid, ls, closure="mixed")
    assert mixed.rbf_cut.size > 0 and not mixed.rbf_rot.any()
    full = eb.build(grid, ls, closure="rbf")
    assert full.rbf_rot.any()
    for r in np.flatnonzero(full.rbf_rot):
        j = full.rbf_cut[r]
        node = full.cp_nodes[full.cut_cp[j]]
        ax, sg = full.cut_dir[j] // 2, (1 if full.cut_dir[j] % 2 else -1)
        ij = [node % grid.n[0], node // grid.n[0]]
        ij[ax] += sg
        x_bp = np.array([grid.lo[0] + ij[0] * grid.h, grid.lo[1] + ij[1] * grid.h])
        v1, v2 = full.cut_xg[j] - x_bp, full.rbf_xg2[r] - x_bp
        ang = math.atan2(v1[0] * v2[1] - v1[1] * v2[0], v1 @ v2)
        assert abs(ang - math.pi / 4) < 1e-9
        psi = geometry.psi_points(ls, 2, [np.array([full.rbf_xg2[r][0]]), np.array([full.rbf_xg2[r][1]])])[0]
        assert abs(psi) < 1e-12


@pytest.mark.parametrize("closure", ["mixed", "rbf"])
def test_linear_u_exact_nonconvex(closure):
    grid, ls = _star(128, 0.2)
    s = eb.build(grid, ls, closure=closure)
    u = lambda x, y: 0.4 - 1.3 * x + 0.8 * y
    pts = s.sample_points()
    b = eb.rhs(s, np.zeros(grid.shape()), u(pts[:, 0], pts[:, 1]))
    x = spla.spsolve(s.A.tocsc(), b)
    X, Y = ei.grid_points(grid)
    ue = u(X, Y).reshape(-1)[s.cp_nodes]
    assert np.abs(x - ue).max() < 1e-10


def test_mixed_closure_second_order_in_max_norm():
    def run(closure):
        out = []
        for n in (64, 128, 256, 512):
            grid, ls = _star(n)
            s = eb.build(grid, ls, closure=closure)
            pts = s.sample_points()
            X, Y = ei.grid_points(grid)
            b = eb.rhs(s, ei.f_k1(X, Y), ei.u_k1(pts[:, 0], pts[:, 1]))
            x = spla.spsolve(s.A.tocsc(), b)
            out.append(np.abs(x - ei.u_k1(X, Y).reshape(-1)[s.cp_nodes]).max())
        return out
    mixed, line = run("mixed"), run("line")
    assert math.log2(mixed[0] / mixed[-1]) / 3 > 1.7, mixed
    assert math.log2(line[0] / line[-1]) / 3 < 1.3, line
    assert mixed[-1] < line[-1] / 10


@pytest.mark.parametrize("closure", ["mixed", "rbf"])
def test_rbf_matrix_symmetric_and_lemma1(closure):
    grid, ls = _star(96, 0.2)
    s = eb.build(grid, ls, closure=closure)
    D = (s.A - s.A.T).tocsr()
    assert D.nnz == 0 or np.all(D.data == 0.0)
    for ax, n, a, b in eb.line_segments(s):
        assert eb.lemma1_holds(n, a, b)
    assert np.linalg.eigvalsh(s.A.toarray())[0] > 0
