"""Pins of the quantity-of-interest sweeps of Sec. 3.6 on the oracle (CPU).

Both examples solve Lap u = 3 with u = 0 on an ellipse, whose exact solution
is a quadratic: the QOIs have closed forms.  Pinned: the discrete QOIs
converge to them, the mirror symmetries the paper reports hold on the
symmetric grid (u(0,0) equal for a and 1/a; the rotated integral equal for
theta and -theta and for theta and theta + pi), and u(0,0) is extreme at the
circle a = 1.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import eb_inputs as ei
from oracle import eb


def _qoi(grid, ls, w):
    s = eb.build(grid, ls)
    b = eb.rhs(s, np.full(grid.shape(), ei.QOI_F), np.zeros(s.cut_cp.size))
    x = spla.spsolve(s.A.tocsc(), b)
    return float(s.to_grid(x).reshape(-1) @ w.reshape(-1))


def test_ellipse_point_qoi_closed_form_symmetry_and_minimum():
    vals = {}
    for a in (0.5, 0.8, 1.0, 1.25, 2.0):
        p, q = a, 1.0 / a
        grid, ls = ei.qoi_ellipse(p, q)
        vals[a] = _qoi(grid, ls, ei.qoi_point_weights(grid, 0.0, 0.0))
        assert abs(vals[a] - ei.qoi_ellipse_exact(p, q)) < 2e-3 * abs(ei.qoi_ellipse_exact(p, q)), a
        # the mirror a -> 1/a: exactly swapped semi-axes, the transposed grid problem
        grid2, ls2 = ei.qoi_ellipse(q, p)
        v2 = _qoi(grid2, ls2, ei.qoi_point_weights(grid2, 0.0, 0.0))
        assert abs(v2 - vals[a]) <= 1e-11 * abs(vals[a])
    assert min(vals, key=vals.get) == 1.0     # u(0,0) is most negative for the circle


def test_ellipse_qoi_second_order():
    errs = []
    for n in (128, 256, 512):
        grid, ls = ei.qoi_ellipse(1.6, 1.0 / 1.6, n=n)
        errs.append(abs(_qoi(grid, ls, ei.qoi_point_weights(grid, 0.0, 0.0)) - ei.qoi_ellipse_exact(1.6, 1 / 1.6)))
    assert math.log2(errs[0] / errs[2]) / 2 > 1.5, errs


def test_rotated_ellipse_integral_closed_form_and_symmetry():
    for th in (0.3, 1.1):
        grid, ls = ei.qoi_rotated(th)
        w = ei.qoi_rect_weights(grid)
        v = _qoi(grid, ls, w)
        exact = ei.qoi_rotated_exact(th)
        assert abs(v - exact) < 0.03 * abs(exact), (th, v, exact)
        grid2, ls2 = ei.qoi_rotated(-th)
        v2 = _qoi(grid2, ls2, w)
        assert abs(v2 - v) <= 1e-9 * abs(v)
