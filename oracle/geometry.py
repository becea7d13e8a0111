"""Level sets, the node mask and grid-line / boundary intersections (oracle).

Sec. 2: the mask m_ij is 1 inside Omega and 0 outside, read off the sign of the
level set psi.  Reading of the sign convention: inside <=> psi < 0 strictly
(psi = 0 counts as outside).

Two descriptor families:

* quadric   psi = sum_a (y_a / s_a)^2 - 1,  y = Q^T (x - c)   (circle, sphere,
            rotated ellipsoid).  Evaluated in the fixed operation order
            t_d = x_d - c_d;  y_a = (Q[0][a] t_0 + Q[1][a] t_1) + Q[2][a] t_2;
            w_a = y_a / s_a;  psi = ((w_0 w_0 + w_1 w_1) + w_2 w_2) - 1,
            every operation an IEEE-rounded FP64 operation.
* star2d    psi = rho - r(phi), rho = |x - c|, phi = atan2(y - c_y, x - c_x),
            r(phi) = r0 + sum_k a_k sin(k phi + p_k) (summed in list order).

Grid-line roots (Sec. 2.1: psi(xi_Gamma, y_j) = 0, "found by a root-finding
algorithm such as the secant method"):

* quadric: psi along the line x(t) = p + sign t e_axis is the quadratic
  alpha t^2 + beta t + gamma, solved in closed form for its root t > 0
  (p inside, gamma < 0, so exactly one positive root).
* star2d: Illinois (safeguarded secant) iteration on the bracket
  [last inside node, first outside node].
"""
from __future__ import annotations

import numpy as np

import eb_inputs as ei


def quadric_parts(ls: ei.LevelSet, dim: int):
    Q = np.asarray(ls.rot, dtype=np.float64).reshape(3, 3)
    c = np.asarray(ls.center, dtype=np.float64)
    s = np.asarray(ls.semi, dtype=np.float64)
    return Q, c, s


def psi_points(ls: ei.LevelSet, dim: int, pts):
    """psi at points; ``pts`` is a list of ``dim`` coordinate arrays."""
    if ls.kind == ei.LS_QUADRIC:
        Q, c, s = quadric_parts(ls, dim)
        t = [pts[d] - c[d] for d in range(dim)]
        w = []
        for a in range(dim):
            y = Q[0][a] * t[0] + Q[1][a] * t[1]
            if dim == 3:
                y = y + Q[2][a] * t[2]
            w.append(y / s[a])
        acc = w[0] * w[0] + w[1] * w[1]
        if dim == 3:
            acc = acc + w[2] * w[2]
        return acc - 1.0
    if ls.kind == ei.LS_STAR2D:
        dx = pts[0] - ls.center[0]
        dy = pts[1] - ls.center[1]
        rho = np.sqrt(dx * dx + dy * dy)
        phi = np.arctan2(dy, dx)
        r = np.full_like(rho, ls.r0)
        for k, a, p in zip(ls.ks, ls.amps, ls.phases):
            r = r + a * np.sin(k * phi + p)
        return rho - r
    raise ValueError("unknown level-set kind")


def psi_nodes(grid: ei.Grid, ls: ei.LevelSet) -> np.ndarray:
    """psi on the full grid, numpy shape grid.shape() (x fastest)."""
    if ls.kind == ei.LS_SAMPLED:
        psi = np.asarray(ls.psi, dtype=np.float64)
        if psi.shape != grid.shape():
            raise ValueError("sampled level set: psi must have the grid's shape")
        return psi.copy()
    pts = ei.grid_points(grid)
    return psi_points(ls, grid.dim, list(pts))


def sampled_line_distance(psi_in, psi_out, steps_in, h):
    """Distance from a BP to Gamma along its grid line when psi is known only at
    the nodes (Sec. 3.3, the linear-ratio distance of two grid points that
    border x_Gamma): psi is taken linear between the last inside node psi_in
    < 0, which lies steps_in nodes beyond the BP (0: the BP itself), and the
    next node psi_out >= 0, so the crossing lies psi_in / (psi_in - psi_out) h
    beyond the last inside node: delta = steps_in h + psi_in / (psi_in -
    psi_out) h.  Second-order accurate for a smooth psi, exact where psi is
    linear between the two nodes."""
    psi_in = np.asarray(psi_in, dtype=np.float64)
    psi_out = np.asarray(psi_out, dtype=np.float64)
    steps = np.asarray(steps_in).astype(np.float64)
    return steps * h + (psi_in / (psi_in - psi_out)) * h


def quadric_line_root(ls: ei.LevelSet, dim: int, p, axis: int, sign):
    """Positive root t of psi(p + sign t e_axis) = 0 for a quadric (p inside).

    alpha = sum_a u_a^2 with u_a = Q[axis][a] / s_a;
    beta  = 2 sign sum_a w_a u_a with w_a = y_a(p) / s_a;
    gamma = psi(p) < 0.
    t = -2 gamma / (beta + sqrt(disc)) if beta >= 0 else (sqrt(disc) - beta) / (2 alpha),
    disc = beta^2 - 4 alpha gamma (the two cancellation-free forms of the root).
    Vectorised over the points in ``p`` (list of coordinate arrays), with
    ``axis`` an integer array and ``sign`` an array of +-1.0.
    """
    Q, c, s = quadric_parts(ls, dim)
    t = [p[d] - c[d] for d in range(dim)]
    w = []
    for a in range(dim):
        y = Q[0][a] * t[0] + Q[1][a] * t[1]
        if dim == 3:
            y = y + Q[2][a] * t[2]
        w.append(y / s[a])
    u = [Q[axis, a] / s[a] for a in range(dim)]
    alpha = u[0] * u[0] + u[1] * u[1]
    dot = w[0] * u[0] + w[1] * u[1]
    gamma = w[0] * w[0] + w[1] * w[1]
    if dim == 3:
        alpha = alpha + u[2] * u[2]
        dot = dot + w[2] * u[2]
        gamma = gamma + w[2] * w[2]
    gamma = gamma - 1.0
    beta = 2.0 * (sign * dot)
    disc = beta * beta - 4.0 * alpha * gamma
    sq = np.sqrt(disc)
    with np.errstate(divide="ignore", invalid="ignore"):
        t_pos = (-2.0 * gamma) / (beta + sq)
        t_neg = (sq - beta) / (2.0 * alpha)
    return np.where(beta >= 0.0, t_pos, t_neg)


def star_line_root(ls: ei.LevelSet, p, axis, sign, ta, tb, h, maxit: int = 100):
    """Root of g(t) = psi(p + sign t e_axis) in [ta, tb], g(ta) < 0 <= g(tb).

    Illinois variant of regula falsi: the secant point of the current bracket
    replaces the end with the same sign of g; when the same end is kept twice
    in a row, the kept end's g value is halved.  Stops when g(t) == 0 or when
    the iterate moves by at most 1e-15 h; vectorised over the cuts.
    """
    p = [np.asarray(v, dtype=np.float64) for v in p]

    def g(t):
        q = [p[0].copy(), p[1].copy()]
        for a in (0, 1):
            m = axis == a
            q[a] = np.where(m, p[a] + sign * t, p[a])
        return psi_points(ls, 2, q)

    ta = np.asarray(ta, dtype=np.float64).copy()
    tb = np.asarray(tb, dtype=np.float64).copy()
    fa = g(ta)
    fb = g(tb)
    t = tb.copy()
    done = fb == 0.0
    side = np.zeros_like(ta)
    told = ta.copy()
    for _ in range(maxit):
        act = ~done
        if not act.any():
            break
        tn = (ta * fb - tb * fa) / (fb - fa)
        tn = np.where(act, tn, t)
        ft = g(tn)
        t = np.where(act, tn, t)
        hit0 = act & (ft == 0.0)
        lower = act & (ft < 0.0)
        upper = act & (ft > 0.0)
        # keep bracket [ta, tb] with g(ta) < 0 < g(tb)
        fb = np.where(lower & (side == -1), 0.5 * fb, fb)
        fa = np.where(upper & (side == 1), 0.5 * fa, fa)
        ta = np.where(lower, tn, ta)
        fa = np.where(lower, ft, fa)
        tb = np.where(upper, tn, tb)
        fb = np.where(upper, ft, fb)
        side = np.where(lower, -1.0, np.where(upper, 1.0, side))
        conv = act & (np.abs(tn - told) <= 1e-15 * h)
        told = np.where(act, tn, told)
        done = done | hit0 | conv
    return t


# ------------------------------------------------ the boundary as a curve (2D)
# Sec. 2.2 (RBF closure) needs points ON Gamma nearest to given points and the
# intersection of a rotated line with Gamma.  Both 2D descriptor families are
# parameterised curves: the quadric y = Q^T (x - c) has y(t) = (s0 cos t,
# s1 sin t); the star has x(phi) = c + r(phi) (cos phi, sin phi).

def curve(ls: ei.LevelSet, t):
    """Gamma(t), Gamma'(t), Gamma''(t) as (x, y) pairs of arrays."""
    t = np.asarray(t, dtype=np.float64)
    if ls.kind == ei.LS_QUADRIC:
        Q, c, s = quadric_parts(ls, 2)
        # y = Q2^T (x - c) for the leading 2 x 2 block Q2, so x = c + M y with M = (Q2^T)^-1
        M = np.linalg.inv(Q[:2, :2].T)
        y = (s[0] * np.cos(t), s[1] * np.sin(t))
        y1 = (-s[0] * np.sin(t), s[1] * np.cos(t))
        y2 = (-y[0], -y[1])
        f = lambda v, off: (off[0] + M[0][0] * v[0] + M[0][1] * v[1], off[1] + M[1][0] * v[0] + M[1][1] * v[1])
        return f(y, c[:2]), f(y1, (0.0, 0.0)), f(y2, (0.0, 0.0))
    if ls.kind == ei.LS_STAR2D:
        r = np.full_like(t, ls.r0)
        r1 = np.zeros_like(t)
        r2 = np.zeros_like(t)
        for k, a, p in zip(ls.ks, ls.amps, ls.phases):
            r = r + a * np.sin(k * t + p)
            r1 = r1 + a * k * np.cos(k * t + p)
            r2 = r2 - a * k * k * np.sin(k * t + p)
        ct, st = np.cos(t), np.sin(t)
        g = (ls.center[0] + r * ct, ls.center[1] + r * st)
        g1 = (r1 * ct - r * st, r1 * st + r * ct)
        g2 = (r2 * ct - 2.0 * r1 * st - r * ct, r2 * st + 2.0 * r1 * ct - r * st)
        return g, g1, g2
    raise ValueError("the RBF closure needs a quadric or star boundary (2D)")


def closest_point(ls: ei.LevelSet, p, n_guess: int = 256, maxit: int = 60):
    """The point of Gamma nearest to p (Sec. 3.3's procedure for parametric
    curves): the nearest of n_guess uniform parameter samples, then Newton's
    method on (Gamma(t) - p) . Gamma'(t) = 0 with steps limited to one sample
    spacing.  Returns (x, y, t)."""
    ts = 2.0 * np.pi * np.arange(n_guess) / n_guess
    (gx, gy), _, _ = curve(ls, ts)
    t = float(ts[int(np.argmin((gx - p[0]) ** 2 + (gy - p[1]) ** 2))])
    dmax = 2.0 * np.pi / n_guess
    for _ in range(maxit):
        (x, y), (x1, y1), (x2, y2) = curve(ls, t)
        g = (x - p[0]) * x1 + (y - p[1]) * y1
        dg = x1 * x1 + y1 * y1 + (x - p[0]) * x2 + (y - p[1]) * y2
        step = -g / dg if dg > 0 else -np.sign(g) * dmax
        step = float(np.clip(step, -dmax, dmax))
        t = t + step
        if abs(step) <= 1e-15:
            break
    (x, y), _, _ = curve(ls, t)
    return float(x), float(y), t


def ray_boundary(ls: ei.LevelSet, p, d, h):
    """First crossing of Gamma on the ray p + s d (s > 0, |d| = 1, p inside):
    march in steps of h/4 to the first point with psi >= 0, then the Illinois
    iteration of star_line_root's kind on that bracket."""
    def psi_at(s):
        return float(psi_points(ls, 2, [np.array([p[0] + s * d[0]]), np.array([p[1] + s * d[1]])])[0])
    step = 0.25 * h
    s0, f0 = 0.0, psi_at(0.0)
    s1 = step
    f1 = psi_at(s1)
    n = 0
    while f1 < 0.0:
        s0, f0 = s1, f1
        s1 = s1 + step
        f1 = psi_at(s1)
        n += 1
        if n > 10 ** 6:
            raise RuntimeError("ray does not leave the domain")
    if f1 == 0.0:
        return s1
    a, fa, b, fb = s0, f0, s1, f1
    side, told, t = 0, a, b
    for _ in range(100):
        t = (a * fb - b * fa) / (fb - fa)
        ft = psi_at(t)
        if ft == 0.0:
            break
        if ft < 0.0:
            if side == -1:
                fb = 0.5 * fb
            a, fa, side = t, ft, -1
        else:
            if side == 1:
                fa = 0.5 * fa
            b, fb, side = t, ft, 1
        if abs(t - told) <= 1e-15 * h:
            break
        told = t
    return t
