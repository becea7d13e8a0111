"""Line-by-line embedded-boundary discretisation of the Laplacian (oracle).

Follows Algorithm 1 of the paper:
  step 1  mask, boundary points (BP) and computational points (CP)  (Sec. 2)
  step 2  central differences (eq. 3, beta = 1) at the CPs only
  step 3  line-by-line interpolation at each BP neighbour (Sec. 2.1, eqs. 4-6)

Readings of the paper taken here:

* Unknowns are the CPs only, ordered lexicographically (x fastest); the BP
  values are eliminated through the interpolant of eq. (6) (Algorithm 1).
* A = -L is assembled (the SPD sign), interior rows (1/h^2)[2 dim, -1 ...].
* Closure of one CP k towards a BP neighbour in direction s: the interpolant
  through (xi_Gamma, u_Gamma) and (xi_1 = x_k, u_k) evaluated at the BP gives
  u_BP = g_Gamma u_Gamma + g_1 u_k with g_Gamma = h/(h+delta), g_1 =
  delta/(h+delta), where delta = |x_BP - x_Gamma| (Sec. 2.1).  Substituted in
  (u_BP - u_k)/h^2 this leaves c_s = g_Gamma = h/(h+delta) on the diagonal of
  h^2 A and +c_s u_Gamma / h^2 on the right-hand side.
* When the node beyond the BP is also inside, the paper switches to RBF
  interpolation (Algorithm 1 step 3).  The line-by-line-only reading used here
  walks outward from the BP along the grid line to the first node that is not
  inside and takes the first crossing of Gamma there; delta may then exceed h
  but c_s stays in (0, 1), so symmetry and strict diagonal dominance hold.
* The outermost ring of grid nodes must lie outside Omega (the paper assumes
  the geometry is contained in the grid), otherwise GeometryError.
* Right-hand side: b = -f + sum_s c_s u_Gamma,s / h^2 for div(grad u) = f.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

import eb_inputs as ei
from . import geometry as geo

OUTSIDE, BOUNDARY, COMPUTATIONAL = 0, 1, 2


class GeometryError(ValueError):
    pass


@dataclass
class EBSystem:
    grid: ei.Grid
    ls: ei.LevelSet
    psi: np.ndarray          # full grid
    cls: np.ndarray          # uint8 full grid: 0 outside, 1 BP, 2 CP
    cp_nodes: np.ndarray     # int64 [N_C], linear node index of CP k (ascending)
    cp_of_node: np.ndarray   # int64 full grid (flattened), -1 off CP
    cut_cp: np.ndarray       # int64 [n_cut], CP index of each cut
    cut_dir: np.ndarray      # int64 [n_cut], 2*axis + (0 for -, 1 for +)
    cut_delta: np.ndarray    # float64 [n_cut], distance BP -> Gamma
    cut_xg: np.ndarray       # float64 [n_cut, dim], intersection point
    cut_c: np.ndarray        # float64 [n_cut], c_s = h/(h+delta)
    diag: np.ndarray         # float64 [N_C], D_k = sum_s beta_s c_s (h^2 units)
    A: sp.csr_matrix         # [N_C, N_C], A = -L
    beta: tuple = None       # None (beta = 1) or per axis a full-grid array: beta at node + h/2 e_axis
    cut_beta: np.ndarray = None  # float64 [n_cut], beta at the half point between the CP and its BP
    cut_w1: np.ndarray = None    # float64 [n_cut], right-hand-side weight of the first boundary value
    rbf_cut: np.ndarray = None   # int64 [n_rbf], the cuts closed by RBF interpolation (ascending)
    rbf_xg2: np.ndarray = None   # float64 [n_rbf, 2], their second boundary point G2
    rbf_w2: np.ndarray = None    # float64 [n_rbf], its weight
    rbf_rot: np.ndarray = None   # bool [n_rbf], G2 from the rotated line (Algorithm 2's second branch)

    @property
    def num_samples(self) -> int:
        """Boundary values the right-hand side needs: one per cut, then the
        second point of every RBF cut."""
        return int(self.cut_cp.size + (0 if self.rbf_cut is None else self.rbf_cut.size))

    def sample_points(self) -> np.ndarray:
        """The boundary points of the right-hand side's values, in order."""
        if self.rbf_cut is None or self.rbf_cut.size == 0:
            return self.cut_xg
        return np.concatenate([self.cut_xg, self.rbf_xg2], axis=0)

    @property
    def num_cp(self) -> int:
        return int(self.cp_nodes.size)

    def to_grid(self, v: np.ndarray) -> np.ndarray:
        out = np.zeros(self.grid.num_nodes, dtype=np.float64)
        out[self.cp_nodes] = v
        return out.reshape(self.grid.shape())

    def from_grid(self, g: np.ndarray) -> np.ndarray:
        return np.asarray(g, dtype=np.float64).reshape(-1)[self.cp_nodes]


def strides(grid: ei.Grid):
    return (1, grid.n[0], grid.n[0] * grid.n[1])


def classify(grid: ei.Grid, psi: np.ndarray) -> np.ndarray:
    """Mask and BP / CP classes (Sec. 2): a BP is inside with fewer than 2*dim
    inside nearest neighbours, a CP is inside with all of them inside."""
    inside = psi < 0.0
    border = np.zeros_like(inside)
    if grid.dim == 2:
        border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
    else:
        border[0] = border[-1] = True
        border[:, 0] = border[:, -1] = True
        border[:, :, 0] = border[:, :, -1] = True
    if (inside & border).any():
        raise GeometryError("the geometry touches the outermost ring of grid nodes")
    cnt = np.zeros(inside.shape, dtype=np.int32)
    m = inside.astype(np.int32)
    for ax in range(grid.dim):
        npax = grid.dim - 1 - ax          # numpy axis of grid axis ax
        cnt += np.roll(m, 1, axis=npax) + np.roll(m, -1, axis=npax)
    cls = np.zeros(inside.shape, dtype=np.uint8)
    cls[inside] = BOUNDARY
    cls[inside & (cnt == 2 * grid.dim)] = COMPUTATIONAL
    return cls


def half_point_beta(eb_or_beta, grid, cp_nodes, ax, sgn):
    """beta at the half point between each CP and its neighbour in direction
    (ax, sgn): beta_{i+1/2} is stored at node i (eq. 3), so the -x half point
    of node i is beta_x[i - 1]."""
    b = np.asarray(eb_or_beta[ax], dtype=np.float64).reshape(-1)
    st = strides(grid)[ax]
    return b[cp_nodes] if sgn > 0 else b[cp_nodes - st]


RBF_EPS = 0.025   # Algorithm 2's tolerance (Sec. 2.3: distinct points for eps = 0.025)


def rbf_weights(x_ij, x_g1, x_g2, x_bp, h):
    """Weights (w_ij, w_1, w_2) of u_BP = w_ij u_ij + w_1 u_G1 + w_2 u_G2 from
    the cubic polyharmonic RBF interpolant with linear augmentation of eqs.
    (7)-(9): B c = (phi_BP; pi_BP), B = [[Phi, Pi^T], [Pi, 0]], phi(r) = r^3
    (Sec. 3).  Coordinates are taken relative to x_BP and scaled by 1/h (the
    interpolant is invariant under translation and scaling)."""
    pts = np.array([x_ij, x_g1, x_g2], dtype=np.float64)
    loc = (pts - np.asarray(x_bp, dtype=np.float64)[None, :]) / h
    B = np.zeros((6, 6))
    for a in range(3):
        for b in range(3):
            B[a, b] = np.linalg.norm(loc[a] - loc[b]) ** 3
    B[3, :3] = 1.0
    B[4, :3] = loc[:, 0]
    B[5, :3] = loc[:, 1]
    B[:3, 3:] = B[3:, :3].T
    rhs = np.zeros(6)
    rhs[:3] = np.linalg.norm(loc, axis=1) ** 3
    rhs[3] = 1.0                      # pi_BP = (1, 0, 0) at the local origin
    c = np.linalg.solve(B, rhs)
    return c[0], c[1], c[2]


def rbf_points(ls, x_ij, x_bp, h, eps=RBF_EPS):
    """Algorithm 2: x_G1 nearest to x_BP on Gamma, x_G2 nearest to x_ij if the
    two are more than eps h apart, else the crossing of Gamma with the line
    x_BP -> x_G1 turned counterclockwise by pi/4 about x_BP.  Returns
    (x_G1, x_G2, rotated)."""
    g1 = geo.closest_point(ls, x_bp)[:2]
    g2 = geo.closest_point(ls, x_ij)[:2]
    if math.hypot(g1[0] - g2[0], g1[1] - g2[1]) > eps * h:
        return g1, g2, False
    v = (g1[0] - x_bp[0], g1[1] - x_bp[1])
    nv = math.hypot(*v)
    c, s_ = math.cos(math.pi / 4.0), math.sin(math.pi / 4.0)
    d = ((c * v[0] - s_ * v[1]) / nv, (s_ * v[0] + c * v[1]) / nv)
    t = geo.ray_boundary(ls, x_bp, d, h)
    return g1, (x_bp[0] + t * d[0], x_bp[1] + t * d[1]), True


def build(grid: ei.Grid, ls: ei.LevelSet, beta=None, closure: str = "line", rbf_eps: float = RBF_EPS) -> EBSystem:
    """Algorithm 1, steps 1-3.  beta: None for beta = 1, else one full-grid
    array per axis holding beta at the half points node + h/2 e_axis (eq. 3).
    With beta the stencil of eq. 3 weights each neighbour difference by the
    beta of its half point; the closure of Sec. 2.1 then leaves beta_s c_s on
    the diagonal and beta_s c_s u_Gamma / h^2 on the right-hand side.
    closure: "line" (line-by-line everywhere, the far crossing beyond the BP
    when the node past it is inside), "mixed" (Sec. 2.3: line-by-line where
    the node past the BP is outside, the RBF interpolation of Sec. 2.2
    otherwise) or "rbf" (RBF everywhere); the RBF forms are 2D."""
    dim, h = grid.dim, grid.h
    psi = geo.psi_nodes(grid, ls)
    cls = classify(grid, psi)
    flat_cls = cls.reshape(-1)
    flat_psi = psi.reshape(-1)
    cp_nodes = np.flatnonzero(flat_cls == COMPUTATIONAL).astype(np.int64)
    if cp_nodes.size == 0:
        raise GeometryError("no computational point")
    cp_of_node = np.full(flat_cls.size, -1, dtype=np.int64)
    cp_of_node[cp_nodes] = np.arange(cp_nodes.size)
    st = strides(grid)

    # node coordinates of every node, per axis (x_i = lo + i h)
    idx = [None] * dim
    rem = cp_nodes.copy()
    for ax in range(dim):
        idx[ax] = rem % grid.n[ax]
        rem = rem // grid.n[ax]

    cut_cp, cut_dir, cut_delta, cut_xg, cut_far = [], [], [], [], []
    diag = np.zeros(cp_nodes.size, dtype=np.float64)
    cs_per_dir = []
    for ax in range(dim):
        for sgn_bit, sgn in ((0, -1), (1, 1)):
            nb = cp_nodes + sgn * st[ax]
            is_bp = flat_cls[nb] == BOUNDARY
            cs = np.ones(cp_nodes.size, dtype=np.float64)
            k = np.flatnonzero(is_bp)
            if k.size:
                bp = nb[k]
                # walk outward from the BP to the first node that is not inside
                m = np.ones(k.size, dtype=np.int64)
                cur = bp + sgn * st[ax]
                active = flat_psi[cur] < 0.0
                while active.any():
                    m = np.where(active, m + 1, m)
                    cur = np.where(active, cur + sgn * st[ax], cur)
                    active = flat_psi[cur] < 0.0
                # BP coordinates
                p = []
                for a2 in range(dim):
                    ia = idx[a2][k] + (sgn if a2 == ax else 0)
                    p.append(grid.lo[a2] + ia.astype(np.float64) * h)
                if ls.kind == ei.LS_QUADRIC:
                    delta = geo.quadric_line_root(ls, dim, p, ax, float(sgn))
                elif ls.kind == ei.LS_SAMPLED:
                    delta = geo.sampled_line_distance(flat_psi[cur - sgn * st[ax]], flat_psi[cur], m - 1, h)
                else:
                    ta = (m - 1).astype(np.float64) * h
                    tb = m.astype(np.float64) * h
                    axes = np.full(k.size, ax)
                    delta = geo.star_line_root(ls, p, axes, np.full(k.size, float(sgn)), ta, tb, h)
                c = h / (h + delta)
                cs[k] = c
                xg = np.stack(p, axis=1)
                xg[:, ax] = p[ax] + sgn * delta
                cut_cp.append(k)
                cut_dir.append(np.full(k.size, 2 * ax + sgn_bit))
                cut_delta.append(delta)
                cut_xg.append(xg)
                cut_far.append(m > 1)
            if beta is not None:
                cs = half_point_beta(beta, grid, cp_nodes, ax, sgn) * cs
            cs_per_dir.append(cs)
    # D_k = sum_s (beta_s) c_s, summed in direction order (-x, +x, -y, +y, -z, +z)
    for cs in cs_per_dir:
        diag = diag + cs

    if cut_cp:
        cut_cp_a = np.concatenate(cut_cp)
        cut_dir_a = np.concatenate(cut_dir)
        cut_delta_a = np.concatenate(cut_delta)
        cut_xg_a = np.concatenate(cut_xg, axis=0)
        cut_far_a = np.concatenate(cut_far)
        order = np.lexsort((cut_dir_a, cut_cp_a))
        cut_cp_a, cut_dir_a = cut_cp_a[order], cut_dir_a[order]
        cut_delta_a, cut_xg_a = cut_delta_a[order], cut_xg_a[order]
        cut_far_a = cut_far_a[order]
    else:
        cut_cp_a = np.zeros(0, np.int64)
        cut_dir_a = np.zeros(0, np.int64)
        cut_delta_a = np.zeros(0)
        cut_xg_a = np.zeros((0, dim))
        cut_far_a = np.zeros(0, dtype=bool)
    cut_c_a = h / (h + cut_delta_a)
    # the RBF closure (Sec. 2.2, Algorithm 2) of the selected cuts: u_BP = w_ij
    # u_ij + w_1 u_G1 + w_2 u_G2 leaves 1 - w_ij on the diagonal (in h^2 units)
    # and w_1 u_G1 + w_2 u_G2 on the right-hand side; the cut's crossing
    # becomes G1, its distance |x_BP - G1|, and G2 a second boundary sample
    cut_w1 = cut_c_a.copy()
    rbf_cut = np.zeros(0, dtype=np.int64)
    rbf_xg2 = np.zeros((0, dim))
    rbf_w2 = np.zeros(0)
    rbf_rot = np.zeros(0, dtype=bool)
    if closure not in ("line", "mixed", "rbf"):
        raise ValueError("closure must be line, mixed or rbf")
    if closure != "line":
        if dim != 2:
            raise ValueError("the RBF closure is two-dimensional (Sec. 2.2)")
        sel = np.flatnonzero(cut_far_a if closure == "mixed" else np.ones(cut_cp_a.size, dtype=bool))
        rbf_cut = sel
        rbf_xg2 = np.zeros((sel.size, 2))
        rbf_w2 = np.zeros(sel.size)
        rbf_rot = np.zeros(sel.size, dtype=bool)
        for r, j in enumerate(sel):
            node = cp_nodes[cut_cp_a[j]]
            ax, sg = cut_dir_a[j] // 2, (1 if cut_dir_a[j] % 2 else -1)
            ij = [int(node % grid.n[0]), int(node // grid.n[0])]
            x_ij = (grid.lo[0] + float(ij[0]) * h, grid.lo[1] + float(ij[1]) * h)
            ij[ax] += sg
            x_bp = (grid.lo[0] + float(ij[0]) * h, grid.lo[1] + float(ij[1]) * h)
            g1, g2, rot = rbf_points(ls, x_ij, x_bp, h, rbf_eps)
            w_ij, w1, w2 = rbf_weights(x_ij, g1, g2, x_bp, h)
            cut_c_a[j] = 1.0 - w_ij
            cut_w1[j] = w1
            cut_xg_a[j] = g1
            cut_delta_a[j] = math.hypot(g1[0] - x_bp[0], g1[1] - x_bp[1])
            rbf_xg2[r] = g2
            rbf_w2[r] = w2
            rbf_rot[r] = rot
        # D_k = sum_s beta_s c_s again, with the RBF diagonal contributions
        cdir = np.ones((cp_nodes.size, 2 * dim))
        cdir[cut_cp_a, cut_dir_a] = cut_c_a
        diag = np.zeros(cp_nodes.size)
        for sdir in range(2 * dim):
            w = cdir[:, sdir]
            if beta is not None:
                w = half_point_beta(beta, grid, cp_nodes, sdir // 2, 1 if sdir % 2 else -1) * w
            diag = diag + w
    cut_beta = np.ones(cut_cp_a.size)
    if beta is not None:
        beta = tuple(np.ascontiguousarray(b, dtype=np.float64).reshape(grid.shape()) for b in beta)
        for ax in range(dim):
            for sgn_bit, sgn in ((0, -1), (1, 1)):
                m = cut_dir_a == 2 * ax + sgn_bit
                cut_beta[m] = half_point_beta(beta, grid, cp_nodes[cut_cp_a[m]], ax, sgn)

    A = assemble(grid, cp_nodes, cp_of_node, flat_cls, diag, beta)
    return EBSystem(grid, ls, psi, cls, cp_nodes, cp_of_node, cut_cp_a, cut_dir_a,
                    cut_delta_a, cut_xg_a, cut_c_a, diag, A, beta, cut_beta, cut_w1, rbf_cut, rbf_xg2,
                    rbf_w2, rbf_rot)


def assemble(grid, cp_nodes, cp_of_node, flat_cls, diag, beta=None) -> sp.csr_matrix:
    """Eq. (3) at the CPs (Algorithm 1 step 2); BP neighbours are dropped from
    the off-diagonal pattern (their value is eliminated by the closure, step
    3), CP neighbours give -beta_{half point}/h^2 (-1/h^2 for beta = 1)."""
    h2 = grid.h * grid.h
    st = strides(grid)
    rows = [np.arange(cp_nodes.size)]
    cols = [np.arange(cp_nodes.size)]
    vals = [diag / h2]
    for ax in range(grid.dim):
        for sgn in (-1, 1):
            nb = cp_nodes + sgn * st[ax]
            j = cp_of_node[nb]
            k = np.flatnonzero(j >= 0)
            rows.append(k)
            cols.append(j[k])
            if beta is None:
                vals.append(np.full(k.size, -1.0 / h2))
            else:
                vals.append(-half_point_beta(beta, grid, cp_nodes[k], ax, sgn) / h2)
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    A = sp.csr_matrix((v, (r, c)), shape=(cp_nodes.size, cp_nodes.size))
    A.sort_indices()
    return A


def dominance_margin(eb: EBSystem) -> float:
    """Smallest strict diagonal-dominance margin of the cut rows of h^2 A:
    D_k - sum_j |h^2 a_kj| = sum of c_s over the BP directions of CP k (Sec.
    2.1: only the diagonal changes and |g| <= 1).  Positive for the line-by-
    line closure (every c_s lies in (0, 1)); interior rows have margin 0."""
    if eb.cut_cp.size == 0:
        return 0.0
    acc = np.zeros(eb.num_cp)
    has = np.zeros(eb.num_cp, dtype=bool)
    w = eb.cut_c if eb.beta is None else eb.cut_beta * eb.cut_c
    for s in range(2 * eb.grid.dim):   # direction order, as D_k is summed
        m = eb.cut_dir == s
        acc[eb.cut_cp[m]] += w[m]
        has[eb.cut_cp[m]] = True
    return float(acc[has].min())


def rhs(eb: EBSystem, f_nodes: np.ndarray, ugamma: np.ndarray) -> np.ndarray:
    """b = -f + sum_s c_s u_Gamma,s / h^2 (Sec. 2.1, the g_Gamma u_Gamma term;
    Algorithm 1 step 3 correction of b)."""
    h2 = eb.grid.h * eb.grid.h
    b = -eb.from_grid(f_nodes)
    add = np.zeros(eb.num_cp)
    w1 = eb.cut_c if eb.cut_w1 is None else eb.cut_w1
    w = w1 if eb.beta is None else eb.cut_beta * w1
    ugamma = np.asarray(ugamma, dtype=np.float64)
    nc = eb.cut_cp.size
    np.add.at(add, eb.cut_cp, w * ugamma[:nc] / h2)
    if eb.rbf_cut is not None and eb.rbf_cut.size:
        j = eb.rbf_cut
        w2 = eb.rbf_w2 if eb.beta is None else eb.cut_beta[j] * eb.rbf_w2
        np.add.at(add, eb.cut_cp[j], w2 * ugamma[nc:nc + j.size] / h2)
    return b + add


def apply(eb: EBSystem, x: np.ndarray) -> np.ndarray:
    return eb.A @ x


# ------------------------------------------------ Lemma 1 / Theorem 2

def line_segments(eb: EBSystem):
    """Split every grid line of CPs into segments of consecutive CPs and return
    (axis, n, a, b) per segment, a / b the first / last diagonal entry of
    h^2 D_xx (resp. D_yy, D_zz) on that segment (Sec. 2.3, eqs. 11-12)."""
    grid = eb.grid
    st = strides(grid)
    flat_cls = eb.cls.reshape(-1)
    # per-direction c_s for every CP
    cdir = np.ones((eb.num_cp, 2 * grid.dim))
    cdir[eb.cut_cp, eb.cut_dir] = eb.cut_c
    out = []
    for ax in range(grid.dim):
        is_cp = flat_cls == COMPUTATIONAL
        nodes = eb.cp_nodes
        prev_cp = is_cp[nodes - st[ax]]
        next_cp = is_cp[nodes + st[ax]]
        starts = nodes[~prev_cp]
        for s in starts:
            n = 1
            cur = s
            while is_cp[cur + st[ax]]:
                cur += st[ax]
                n += 1
            k0 = eb.cp_of_node[s]
            k1 = eb.cp_of_node[cur]
            lo_c = cdir[k0, 2 * ax]
            hi_c = cdir[k1, 2 * ax + 1]
            if n == 1:
                a = lo_c + hi_c
                b = a
            else:
                a = 1.0 + lo_c
                b = 1.0 + hi_c
            out.append((ax, n, a, b))
        del prev_cp, next_cp
    return out


def lemma1_holds(n: int, a: float, b: float) -> bool:
    """The three conditions of Lemma 1 for D^(n)(a, b) to be SPD."""
    if n == 1:
        return a > 0
    if n == 2:
        return a > 0 and a * b > 1
    r = (n - 2) / (n - 1)
    return a > r and b > r and a > ((n - 2) * b - (n - 3)) / ((n - 1) * b - (n - 2))


def tridiag_segment(n: int, a: float, b: float) -> np.ndarray:
    """The matrix D^(n)(a, b) of eq. (11)."""
    M = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    M[0, 0] = a
    M[-1, -1] = b if n > 1 else a
    return M


def directional_parts(eb: EBSystem):
    """h^2 A split as the sum over axes of the 1D operators (Theorem 2):
    returns one CSR per axis with diagonal c_lo + c_hi and -1 to CP neighbours."""
    grid = eb.grid
    st = strides(grid)
    cdir = np.ones((eb.num_cp, 2 * grid.dim))
    cdir[eb.cut_cp, eb.cut_dir] = eb.cut_c
    parts = []
    for ax in range(grid.dim):
        r = [np.arange(eb.num_cp)]
        c = [np.arange(eb.num_cp)]
        v = [cdir[:, 2 * ax] + cdir[:, 2 * ax + 1]]
        for sgn in (-1, 1):
            j = eb.cp_of_node[eb.cp_nodes + sgn * st[ax]]
            k = np.flatnonzero(j >= 0)
            r.append(k)
            c.append(j[k])
            v.append(-np.ones(k.size))
        parts.append(sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))),
                                   shape=(eb.num_cp, eb.num_cp)))
    return parts


# ------------------------------------------------ ghost-point negative control

def ghost_point_operator(grid: ei.Grid, ls: ei.LevelSet) -> sp.csr_matrix:
    """Exterior ghost-point closure (Sec. 1, Sec. 2.1 right panel of Fig. 3):
    every inside node is an unknown; an outside neighbour at distance theta h
    from the boundary (theta in (0, 1]) is extrapolated linearly, which puts
    1/theta on the diagonal of h^2 A.  Used only as the negative control of the
    small-cell-stiffness tests."""
    dim, h = grid.dim, grid.h
    psi = geo.psi_nodes(grid, ls)
    inside = (psi < 0.0).reshape(-1)
    nodes = np.flatnonzero(inside)
    idx_of = np.full(inside.size, -1, dtype=np.int64)
    idx_of[nodes] = np.arange(nodes.size)
    st = strides(grid)
    ii = []
    rem = nodes.copy()
    for ax in range(dim):
        ii.append(rem % grid.n[ax])
        rem //= grid.n[ax]
    diag = np.zeros(nodes.size)
    rows, cols, vals = [], [], []
    for ax in range(dim):
        for sgn in (-1, 1):
            nb = nodes + sgn * st[ax]
            j = idx_of[nb]
            inn = j >= 0
            k = np.flatnonzero(inn)
            rows.append(k)
            cols.append(j[k])
            vals.append(-np.ones(k.size))
            diag[k] += 1.0
            k2 = np.flatnonzero(~inn)
            if k2.size:
                p = [grid.lo[a] + ii[a][k2].astype(np.float64) * h for a in range(dim)]
                if ls.kind == ei.LS_QUADRIC:
                    t = geo.quadric_line_root(ls, dim, p, ax, float(sgn))
                else:
                    t = geo.star_line_root(ls, p, np.full(k2.size, ax), np.full(k2.size, float(sgn)),
                                           np.zeros(k2.size), np.full(k2.size, h), h)
                theta = np.maximum(t / h, 1e-300)
                diag[k2] += 1.0 / theta
    rows.append(np.arange(nodes.size))
    cols.append(np.arange(nodes.size))
    vals.append(diag)
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nodes.size, nodes.size)) / (h * h)
    return M


def assemble_unit(eb: EBSystem, shift: float) -> sp.csr_matrix:
    """h^2 (sigma I + A) written with unit spacing: off-diagonals -1 towards CP
    neighbours, diagonal D_k + shift with shift = sigma h^2 (eq. 3 multiplied
    by h^2; used for batches of grids with different h)."""
    n = eb.num_cp
    st = strides(eb.grid)
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [eb.diag + shift]
    for ax in range(eb.grid.dim):
        for sgn in (-1, 1):
            j = eb.cp_of_node[eb.cp_nodes + sgn * st[ax]]
            k = np.flatnonzero(j >= 0)
            rows.append(k)
            cols.append(j[k])
            vals.append(np.full(k.size, -1.0))
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    M.sort_indices()
    return M
