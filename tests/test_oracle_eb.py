"""Pins of the oracle's discretisation against what the paper and mathematics
fix (CPU only).

P1  exact symmetry, off-diagonals -1/h^2, c_s in (0,1), strict diagonal
    dominance on cut rows (Sec. 2.1: only the diagonal changes, |g| <= 1)
P2  multilinear exactness: a harmonic, grid-line-linear u is reproduced
P3  second order in l2 on manufactured solutions (Sec. 3.1-3.3: O(h^2))
P7  spectrum: lambda_max(h^2 A) <= 4 dim (the periodic maximum, 8 in 2D); lambda_min -> j01^2 / R^2 (disk)
P8  Lemma 1 / Corollary 1 on every segment; Theorem 2 decomposition
    ghost-point negative control: small cells blow up lambda_max (Sec. 1)
    brute-force classification on a tiny grid
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import eb_inputs as ei
from oracle import eb, geometry, solvers


def _geoms():
    return {
        "circle": ei.circle_k1(48),
        "star": (ei.box_grid(2, 64), ei.star(ei.STAR_CENTER, 0.5, [5], [0.1], [0.0])),
        "randstar": (ei.box_grid(2, 80), ei.random_star(7)),
        "ellipsoid": ei.ellipsoid_k3(24, seed=0),
        "sphere3": (ei.box_grid(3, 20), ei.sphere((0.013, -0.021, 0.017), 0.6)),
    }


@pytest.mark.parametrize("name", list(_geoms().keys()))
def test_p1_structure(name):
    grid, ls = _geoms()[name]
    s = eb.build(grid, ls)
    A = s.A
    # bitwise symmetric
    D = (A - A.T).tocsr()
    assert D.nnz == 0 or np.all(D.data == 0.0)
    h2 = grid.h * grid.h
    off = A - __import__("scipy.sparse", fromlist=["diags"]).diags(A.diagonal())
    off = off.tocsr()
    off.eliminate_zeros()
    assert np.all(off.data == -1.0 / h2)
    assert np.all((s.cut_c > 0.0) & (s.cut_c < 1.0))
    # interior rows have 2*dim on the diagonal of h^2 A, cut rows strictly dominant
    diag = s.diag
    nnz_off = np.diff(off.indptr)
    assert np.all(diag <= 2 * grid.dim)
    cut_rows = np.unique(s.cut_cp)
    assert np.all(diag[cut_rows] > nnz_off[cut_rows])
    others = np.setdiff1d(np.arange(s.num_cp), cut_rows)
    assert np.all(diag[others] == 2 * grid.dim)
    assert np.all(nnz_off[others] == 2 * grid.dim)


def test_classification_brute_force():
    """Sec. 2 definitions of BP and CP, checked node by node in plain loops."""
    grid, ls = ei.box_grid(2, 14), ei.star((0.031, -0.017), 0.55, [3], [0.15], [0.4])
    s = eb.build(grid, ls)
    n = grid.n[0]
    xs = grid.axis_coords(0)
    ys = grid.axis_coords(1)

    def m(i, j):
        return 1 if geometry.psi_points(ls, 2, [np.array([xs[i]]), np.array([ys[j]])])[0] < 0 else 0

    for j in range(1, n - 1):
        for i in range(1, n - 1):
            inside = m(i, j)
            cnt = m(i + 1, j) + m(i - 1, j) + m(i, j + 1) + m(i, j - 1)
            want = 0 if not inside else (2 if cnt == 4 else 1)
            assert s.cls[j, i] == want


def test_quadric_root_is_on_boundary():
    grid, ls = ei.ellipsoid_k3(32, seed=3)
    s = eb.build(grid, ls)
    pts = [s.cut_xg[:, a] for a in range(3)]
    psi = geometry.psi_points(ls, 3, pts)
    assert np.abs(psi).max() < 1e-13
    assert np.all(s.cut_delta > 0)


def test_star_root_is_on_boundary():
    grid, ls = ei.box_grid(2, 200), ei.random_star(3)
    s = eb.build(grid, ls)
    psi = geometry.psi_points(ls, 2, [s.cut_xg[:, 0], s.cut_xg[:, 1]])
    assert np.abs(psi).max() < 1e-14
    # the crossing is the first one walking outward: no sign change before it
    for k in range(0, s.cut_cp.size, 37):
        ax, sg = divmod(int(s.cut_dir[k]), 2)
        sgn = 1.0 if sg else -1.0
        bp = s.cut_xg[k].copy()
        bp[ax] -= sgn * s.cut_delta[k]
        ts = np.linspace(0.0, s.cut_delta[k] * (1 - 1e-9), 50)
        q = [np.full(ts.size, bp[0]), np.full(ts.size, bp[1])]
        q[ax] = bp[ax] + sgn * ts
        assert np.all(geometry.psi_points(ls, 2, q) < 0)


@pytest.mark.parametrize("name", ["circle", "star", "randstar", "ellipsoid", "sphere3"])
def test_p2_multilinear_exactness(name):
    """u = a + bx + cy + dxy (+ z terms) is harmonic, linear along every grid
    line (so the line-by-line interpolant is exact) and differenced exactly:
    the discrete solution equals u at every CP up to round-off."""
    grid, ls = _geoms()[name]
    s = eb.build(grid, ls)
    pts = ei.grid_points(grid)
    f = np.zeros(grid.shape())
    xg = [s.cut_xg[:, a] for a in range(grid.dim)]
    ug = ei.u_bilinear(*xg)
    b = eb.rhs(s, f, ug)
    x = solvers.dense_cholesky_solve(s.A, b) if s.num_cp < 4000 else spla.spsolve(s.A.tocsc(), b)
    ue = ei.u_bilinear(*pts).reshape(-1)[s.cp_nodes]
    assert np.abs(x - ue).max() < 1e-10 * max(1.0, np.abs(ue).max())


def _errors(grid, ls, ufun, ffun):
    s = eb.build(grid, ls)
    pts = ei.grid_points(grid)
    b = eb.rhs(s, ffun(*pts), ufun(*[s.cut_xg[:, a] for a in range(grid.dim)]))
    x = spla.spsolve(s.A.tocsc(), b)
    e = x - ufun(*pts).reshape(-1)[s.cp_nodes]
    return math.sqrt(grid.h ** grid.dim * float(e @ e)), float(np.abs(e).max()), s


def test_p3_order_2d_circle():
    res = [_errors(*ei.circle_k1(n), ei.u_k1, ei.f_k1) for n in (64, 128, 256, 512)]
    l2 = np.array([r[0] for r in res])
    li = np.array([r[1] for r in res])
    # successive halvings of h (n-1 = 63, 127, 255, 511)
    hs = np.array([2.0 / (n - 1) for n in (64, 128, 256, 512)])
    p_l2 = np.polyfit(np.log(hs), np.log(l2), 1)[0]
    p_li = np.polyfit(np.log(hs), np.log(li), 1)[0]
    assert p_l2 > 1.7, p_l2
    # far intersections (delta > h near grazing rows) cost one order in max norm
    assert p_li > 0.85, p_li


def test_p3_order_3d_ellipsoid():
    ns = (24, 48, 96)
    res = [_errors(*ei.ellipsoid_k3(n, seed=0), ei.u_k3, ei.f_k3) for n in ns]
    hs = np.array([2.0 / (n - 1) for n in ns])
    l2 = np.array([r[0] for r in res])
    p_l2 = np.polyfit(np.log(hs), np.log(l2), 1)[0]
    assert p_l2 > 1.6, p_l2


def test_p7_spectrum_bounds():
    grid, ls = ei.circle_k1(96)
    s = eb.build(grid, ls)
    lmin, lmax = solvers.extreme_eigs(s.A)
    assert lmax * grid.h ** 2 <= 8.0 + 1e-12
    assert lmin > 0.0
    # first Dirichlet eigenvalue of the disk of radius R = 0.5: (j01 / R)^2
    j01 = 2.404825557695773
    exact = (j01 / 0.5) ** 2
    assert abs(lmin - exact) / exact < 0.02


def test_p7_lambda_min_converges():
    j01 = 2.404825557695773
    exact = (j01 / 0.5) ** 2
    errs = []
    for n in (48, 96, 192):
        s = eb.build(*ei.circle_k1(n))
        lmin, _ = solvers.extreme_eigs(s.A)
        errs.append(abs(lmin - exact))
    assert errs[2] < errs[0] / 2.5


@pytest.mark.parametrize("name", ["circle", "star", "randstar", "ellipsoid"])
def test_p8_lemma1_segments(name):
    grid, ls = _geoms()[name]
    s = eb.build(grid, ls)
    segs = eb.line_segments(s)
    assert len(segs) > 0
    for ax, n, a, b in segs:
        assert eb.lemma1_holds(n, a, b)
        if n >= 2:
            assert a > 1.0 and b > 1.0        # Corollary 1
        if n <= 40:
            M = eb.tridiag_segment(n, a, b)
            np.linalg.cholesky(M)              # SPD, independently of Lemma 1


def test_p8_theorem2_decomposition():
    """h^2 A is the sum of the per-axis line operators (Theorem 2)."""
    grid, ls = _geoms()["ellipsoid"]
    s = eb.build(grid, ls)
    parts = eb.directional_parts(s)
    tot = parts[0] + parts[1] + parts[2]
    diff = (tot - s.A * grid.h ** 2).tocsr()
    assert np.abs(diff.data).max() < 1e-12


def test_lemma1_statement_against_eigenvalues():
    """Lemma 1's condition is sufficient: sample (n, a, b) satisfying it and
    confirm SPD by eigenvalues; a = b = (n-2)/(n-1) - eps must fail at n >= 3."""
    rng = np.random.default_rng(0)
    for _ in range(300):
        n = int(rng.integers(1, 12))
        a, b = rng.uniform(0.01, 2.5, size=2)
        M = eb.tridiag_segment(n, a, b)
        if eb.lemma1_holds(n, a, b):
            assert np.linalg.eigvalsh(M)[0] > 0
    for n in range(3, 10):
        r = (n - 2) / (n - 1)
        assert not eb.lemma1_holds(n, r - 1e-3, r - 1e-3)
        assert np.linalg.eigvalsh(eb.tridiag_segment(n, r - 1e-3, r - 1e-3))[0] < 0


def test_ghost_point_negative_control():
    """The exterior ghost-point closure puts 1/theta on the diagonal; with a
    small cut cell lambda_max(h^2 A) exceeds the periodic bound 8 by far, while
    the interior-boundary-point closure never does."""
    worst = 0.0
    for n in (40, 41, 42, 43, 44, 45, 46, 47):
        grid, ls = ei.circle_k1(n)
        G = eb.ghost_point_operator(grid, ls)
        lmax = solvers.extreme_eigs(G)[1] * grid.h ** 2
        worst = max(worst, lmax)
        s = eb.build(grid, ls)
        assert solvers.extreme_eigs(s.A)[1] * grid.h ** 2 <= 8.0 + 1e-12
    assert worst > 16.0


def test_rhs_sign_convention():
    """For u = x^2 + y^2 (lap u = 4), b = -4 + boundary terms and A u_exact
    matches b up to the O(1) closure truncation at cut rows only."""
    grid, ls = ei.circle_k1(40)
    s = eb.build(grid, ls)
    X, Y = ei.grid_points(grid)
    u = X * X + Y * Y
    b = eb.rhs(s, np.full(grid.shape(), 4.0), s.cut_xg[:, 0] ** 2 + s.cut_xg[:, 1] ** 2)
    r = s.A @ u.reshape(-1)[s.cp_nodes] - b
    interior = np.setdiff1d(np.arange(s.num_cp), s.cut_cp)
    assert np.abs(r[interior]).max() < 1e-9


def test_unit_operator_is_scaled_operator():
    grid, ls = ei.box_grid(2, 70), ei.random_star(12)
    s = eb.build(grid, ls)
    sig = 3.7
    U = eb.assemble_unit(s, sig * grid.h ** 2)
    ref = (s.A * grid.h ** 2 + sig * grid.h ** 2 * __import__("scipy.sparse", fromlist=["identity"]).identity(s.num_cp)).tocsr()
    assert np.abs((U - ref).toarray()).max() < 1e-12
    off = U - __import__("scipy.sparse", fromlist=["diags"]).diags(U.diagonal())
    off = off.tocsr()
    off.eliminate_zeros()
    assert np.all(off.data == -1.0)


# ------------------------------------------------ sampled level set (Sec. 3.3)

def test_sampled_distance_is_second_order():
    """psi given only at the nodes (signed distance to the K1 circle): the
    linear-ratio distance of Sec. 3.3 approaches the exact crossing (closed
    form of the same circle) as O(h^2) where the grid line crosses Gamma at an
    angle, with the interpolation bound h^2 max|psi''| / (8 |psi'|), psi'' <= 1/rho
    along a line; classes and cuts are those of the analytic circle.  Near
    tangency |psi'| -> 0 and the error is larger (bounded here by h^1.5)."""
    c, R = (0.02, 0.01), 0.5
    errs, errs_all = [], []
    for n in (64, 128, 256, 512):
        grid = ei.box_grid(2, n)
        h = grid.h
        s_exact = eb.build(grid, ei.sphere(c, R))
        s_samp = eb.build(grid, ei.sampled(ei.circle_distance_values(grid, c, R)))
        assert np.array_equal(s_exact.cls, s_samp.cls)
        assert np.array_equal(s_exact.cut_cp, s_samp.cut_cp) and np.array_equal(s_exact.cut_dir, s_samp.cut_dir)
        err = np.abs(s_samp.cut_delta - s_exact.cut_delta)
        ax = s_exact.cut_dir // 2
        normal_ax = np.abs(s_exact.cut_xg[np.arange(ax.size), ax] - np.asarray(c)[ax]) / R   # |psi'| along the line
        steep = normal_ax >= 0.5
        assert steep.mean() > 0.6
        assert err[steep].max() <= h * h / (8.0 * (R - 2 * h) * 0.5)
        errs.append(err[steep].max())
        errs_all.append(err.max())
        assert err.max() <= 2.0 * h ** 1.5
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > 1.8, (errs, rates)


def _diamond_exact_delta(s, center, R):
    """Exact BP -> Gamma distance of every cut of the diamond sum |x_a - c_a| = R
    and whether the linear-ratio segment holds no kink (last inside node and
    first outside node on the same side of the diamond's axis)."""
    grid = s.grid
    dim, h = grid.dim, grid.h
    ax = s.cut_dir // 2
    sgn = np.where(s.cut_dir % 2 == 1, 1.0, -1.0)
    bp = s.cut_xg.copy()
    bp[np.arange(bp.shape[0]), ax] -= sgn * s.cut_delta
    other = np.zeros(bp.shape[0])
    for a in range(dim):
        other += np.where(ax == a, 0.0, np.abs(bp[:, a] - center[a]))
    x_bp = bp[np.arange(bp.shape[0]), ax]
    c_ax = np.asarray(center)[ax]
    x_gamma = c_ax + sgn * (R - other)          # the crossing on the outward side
    exact = np.abs(x_gamma - x_bp)
    last_in = x_bp + sgn * (np.floor(s.cut_delta / h + 1e-12) * h)
    first_out = last_in + sgn * h
    no_kink = np.sign(last_in - c_ax) == np.sign(first_out - c_ax)
    return exact, no_kink


@pytest.mark.parametrize("dim,n", [(2, 96), (3, 40)])
def test_sampled_distance_exact_where_psi_is_linear(dim, n):
    """On the diamond psi = sum |x_a - c_a| - R, psi is linear along a grid line
    between two nodes on the same side of the axis: there the linear-ratio
    distance is the exact crossing (round-off only)."""
    grid = ei.box_grid(dim, n)
    center = (0.0123, 0.0071, -0.0047)[:dim]
    s = eb.build(grid, ei.sampled(ei.diamond_values(grid, center, 0.71)))
    exact, ok = _diamond_exact_delta(s, center, 0.71)
    assert ok.mean() > 0.9
    assert np.abs(s.cut_delta[ok] - exact[ok]).max() < 1e-13


def test_sampled_diamond_multilinear_exactness():
    """P2 on the sampled diamond: every cut's segment is kink-free here (a BP
    next to a CP leaves at least two inside nodes on its line), so every
    crossing is exact and the discrete solution equals a grid-line-linear
    harmonic u at every CP up to round-off."""
    grid = ei.box_grid(2, 96)
    center = (0.0123, 0.0071)
    s = eb.build(grid, ei.sampled(ei.diamond_values(grid, center, 0.71)))
    exact, ok = _diamond_exact_delta(s, center, 0.71)
    assert ok.all()
    xg = s.cut_xg
    ug = ei.u_bilinear(xg[:, 0], xg[:, 1])
    b = eb.rhs(s, np.zeros(grid.shape()), ug)
    x = spla.spsolve(s.A.tocsc(), b)
    X, Y = ei.grid_points(grid)
    ue = ei.u_bilinear(X, Y).reshape(-1)[s.cp_nodes]
    assert np.abs(x - ue).max() < 1e-10 * np.abs(ue).max()


def test_dominance_margin_matches_rows():
    """The reported margin is the smallest D_k - sum_j |off-diagonal| over the
    cut rows of h^2 A, computed here from the assembled matrix."""
    for grid, ls in (ei.circle_k1(64), (ei.box_grid(2, 80), ei.random_star(7)), ei.ellipsoid_k3(24, seed=0)):
        s = eb.build(grid, ls)
        H = (s.A * grid.h ** 2).tocsr()
        d = H.diagonal()
        off = np.asarray(abs(H).sum(axis=1)).ravel() - np.abs(d)
        cut_rows = np.unique(s.cut_cp)
        want = (d - off)[cut_rows].min()
        got = eb.dominance_margin(s)
        assert got > 0 and abs(got - want) < 1e-14
        assert np.all((d - off)[np.setdiff1d(np.arange(s.num_cp), cut_rows)] == 0.0)
