"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the embedded-boundary method itself: it only
describes grids and geometries (as plain parameters), draws the seeded random
parameters the workloads use, and evaluates the manufactured exact solutions and
source terms at points a caller gives it.  Both the CPU oracle (``oracle/``) and
the CUDA library's Python binding consume these descriptors; neither imports the
other.

Workloads (the paper works in 2D; the 3D case is the dimension-by-dimension
extension of the 5-point stencil to 7 points):

* ``circle_k1``      2D Poisson, [-1,1]^2, circle R=0.5 at (0.02, 0.01),
                     u = sin(2x) cos(3y).
* ``star_wave``      2D wave, [-1,1]^2, star r(phi) = 0.5 + 0.1 sin(5 phi) about
                     (0.02 sqrt5, 0.02 sqrt5) (the star centre of Sec. 3.4),
                     Gaussian pulse with seeded centre and width.
* ``ellipsoid_k3``   3D Poisson, [-1,1]^3, ellipsoid semi-axes (0.7, 0.5, 0.4)
                     with a seeded rotation, u = exp(x) sin(y + z).
* ``star_batch``     64 seeded stars r = 0.5 + sum_{k=2..6} a_k sin(k phi + p_k).
* ``bessel_disk``    unit disk in [-1.1,1.1]^2, standing mode J_7(kappa r) cos 7
                     theta cos kappa t (Sec. 3.5, Table 1).

Grid convention: ``n`` nodes per axis, node i at lo + i*h, h = (hi-lo)/(n-1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# level-set kinds (values match the C enum eb_ls_kind)
LS_QUADRIC = 0   # (rotated) ellipsoid / sphere / circle: sum_a (y_a/s_a)^2 - 1
LS_STAR2D = 1    # rho - r(phi), r(phi) = r0 + sum_k a_k sin(k phi + p_k)
LS_SAMPLED = 2   # psi given at every grid node (full-grid array)


@dataclass
class Grid:
    dim: int
    n: Tuple[int, int, int]          # nodes per axis (unused axes = 1)
    lo: Tuple[float, float, float]
    h: float

    @property
    def num_nodes(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def shape(self) -> Tuple[int, ...]:
        """numpy shape of a full-grid array, x fastest: (ny, nx) or (nz, ny, nx)."""
        if self.dim == 2:
            return (self.n[1], self.n[0])
        return (self.n[2], self.n[1], self.n[0])

    def axis_coords(self, axis: int) -> np.ndarray:
        """Node coordinates lo + i*h along one axis (two IEEE operations)."""
        i = np.arange(self.n[axis], dtype=np.float64)
        return self.lo[axis] + i * self.h


def box_grid(dim: int, n: int, lo: float = -1.0, hi: float = 1.0) -> Grid:
    h = (hi - lo) / (n - 1)
    nn = (n, n, n if dim == 3 else 1)
    ll = (lo, lo, lo if dim == 3 else 0.0)
    return Grid(dim=dim, n=nn, lo=ll, h=h)


@dataclass
class LevelSet:
    """Descriptor of the level set psi (psi < 0 strictly inside)."""
    kind: int
    center: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    semi: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    rot: Tuple[float, ...] = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)  # Q, row-major
    r0: float = 0.5
    ks: List[int] = field(default_factory=list)
    amps: List[float] = field(default_factory=list)
    phases: List[float] = field(default_factory=list)
    psi: Optional[np.ndarray] = None   # LS_SAMPLED: psi at the nodes, shape Grid.shape()


def sphere(center: Sequence[float], radius: float) -> LevelSet:
    c = tuple(center) + (0.0,) * (3 - len(center))
    return LevelSet(kind=LS_QUADRIC, center=c, semi=(radius, radius, radius))


def ellipsoid(center, semi, rot) -> LevelSet:
    c = tuple(center) + (0.0,) * (3 - len(center))
    s = tuple(semi) + (1.0,) * (3 - len(semi))
    return LevelSet(kind=LS_QUADRIC, center=c, semi=s, rot=tuple(float(v) for v in np.asarray(rot).ravel()))


def star(center, r0, ks, amps, phases) -> LevelSet:
    c = tuple(center) + (0.0,) * (3 - len(center))
    return LevelSet(kind=LS_STAR2D, center=c, r0=float(r0), ks=[int(k) for k in ks],
                    amps=[float(a) for a in amps], phases=[float(p) for p in phases])


def sampled(psi_nodes) -> LevelSet:
    """A level set known only through its values at the grid nodes."""
    return LevelSet(kind=LS_SAMPLED, psi=np.ascontiguousarray(psi_nodes, dtype=np.float64))


def circle_distance_values(grid: "Grid", center, radius: float) -> np.ndarray:
    """Signed distance |x - c| - R to a circle (2D) or sphere (3D), sampled at
    the nodes: a smooth level set for the sampled-psi path."""
    pts = grid_points(grid)
    r2 = sum((pts[a] - center[a]) ** 2 for a in range(grid.dim))
    return np.sqrt(r2) - radius


def diamond_values(grid: "Grid", center, radius: float) -> np.ndarray:
    """|x - c_x| + |y - c_y| (+ |z - c_z|) - R sampled at the nodes: linear
    along every grid line except where the line crosses the diamond's axis."""
    pts = grid_points(grid)
    return sum(np.abs(pts[a] - center[a]) for a in range(grid.dim)) - radius


# ---------------------------------------------------------------- workloads

def circle_k1(n: int = 128) -> Tuple[Grid, LevelSet]:
    return box_grid(2, n), sphere((0.02, 0.01), 0.5)


STAR_CENTER = (0.02 * math.sqrt(5.0), 0.02 * math.sqrt(5.0))


def star_wave(n: int = 4096) -> Tuple[Grid, LevelSet]:
    return box_grid(2, n), star(STAR_CENTER, 0.5, [5], [0.1], [0.0])


def random_rotation(seed: int) -> np.ndarray:
    """Rotation Q (det +1) from the QR factorisation of a seeded Gaussian 3x3."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def ellipsoid_k3(n: int = 256, seed: int = 0) -> Tuple[Grid, LevelSet]:
    return box_grid(3, n), ellipsoid((0.0, 0.0, 0.0), (0.7, 0.5, 0.4), random_rotation(seed))


def star_batch(count: int = 64, seed: int = 0):
    """Seeded batch of stars: returns a list of (n_b, LevelSet)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nb = 32 * int(math.ceil(rng.uniform(4.0, 32.0)))
        amps = rng.uniform(0.0, 0.05, size=5)
        phases = rng.uniform(0.0, 2.0 * math.pi, size=5)
        out.append((nb, star((0.02, 0.01), 0.5, [2, 3, 4, 5, 6], amps, phases)))
    return out


def random_star(seed: int) -> LevelSet:
    rng = np.random.default_rng(seed)
    amps = rng.uniform(0.0, 0.05, size=5)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=5)
    return star((0.02, 0.01), 0.5, [2, 3, 4, 5, 6], amps, phases)


def disk_bessel(n: int) -> Tuple[Grid, LevelSet]:
    """Unit disk on [-1.1,1.1]^2 with n nodes per axis (Sec. 3.5)."""
    return box_grid(2, n, -1.1, 1.1), sphere((0.0, 0.0), 1.0)


# ------------------------------------------------- manufactured solutions

def u_k1(x, y):
    return np.sin(2.0 * x) * np.cos(3.0 * y)


def f_k1(x, y):
    """Laplacian of u_k1 (the paper's convention: div(grad u) = f)."""
    return -13.0 * np.sin(2.0 * x) * np.cos(3.0 * y)


def u_k3(x, y, z):
    return np.exp(x) * np.sin(y + z)


def f_k3(x, y, z):
    return -np.exp(x) * np.sin(y + z)


def u_bilinear(x, y, z=None, coef=(0.3, -1.2, 0.7, 2.1, 0.5, -0.4, 0.9, 0.25)):
    """Multilinear harmonic function a + bx + cy + dxy (+ z terms in 3D)."""
    a, b, c, d, e, f_, g, k = coef
    if z is None:
        return a + b * x + c * y + d * x * y
    return a + b * x + c * y + d * x * y + e * z + f_ * x * z + g * y * z + k * x * y * z


def u_heat(x, y, t):
    return math.exp(-t) * np.sin(2.0 * x) * np.cos(3.0 * y)


def f_heat(x, y, t):
    """Source F of u_t = lap u + F for u_heat: F = u_t - lap u = 12 u."""
    return 12.0 * math.exp(-t) * np.sin(2.0 * x) * np.cos(3.0 * y)


# ------------------------------------------- variable coefficient beta (eq. 3)

def beta_half_points(grid: "Grid", beta_fn):
    """beta at the half points of eq. 3: one full-grid array per axis a whose
    entry at node i is beta(x_i + h/2 e_a) (the beta_{i+1/2} of that axis)."""
    pts = grid_points(grid)
    out = []
    for a in range(grid.dim):
        shifted = [p + (0.5 * grid.h if b == a else 0.0) for b, p in enumerate(pts)]
        out.append(np.ascontiguousarray(beta_fn(*shifted), dtype=np.float64))
    return out


def beta_bone(x, y, z=None):
    """beta = 2 + sin(x y) (the bone-shaped example of Sec. 3.3.1)."""
    return 2.0 + np.sin(x * y)


def heat_disk(n: int) -> Tuple["Grid", LevelSet]:
    """The heat example of Sec. 3.4: disk of radius 0.5 about the origin in
    [-1,1]^2 (psi = x^2 + y^2 - 0.25 < 0 inside)."""
    return box_grid(2, n), sphere((0.0, 0.0), 0.5)


def beta_heat_disk(x, y):
    """beta = 0.25 - x^2 - y^2 (Sec. 3.4), positive inside the disk."""
    return 0.25 - x * x - y * y


def u_heat_disk(x, y, t):
    """u = exp(-t) (x^2 + y^2 - 0.25): zero on the circle (Sec. 3.4)."""
    return math.exp(-t) * (x * x + y * y - 0.25)


def f_heat_disk(x, y, t):
    """Source F of u_t = div(beta grad u) + F for u_heat_disk and
    beta_heat_disk: F = u_t - div(beta grad u) = exp(-t) (7 r^2 - 0.75)."""
    return math.exp(-t) * (7.0 * (x * x + y * y) - 0.75)


# ------------------------------------------------- Helmholtz (Sec. 3.3.2)

HELMHOLTZ_OMEGA = 50.0
HELMHOLTZ_SOURCE = (-0.375, 0.125)


def helmholtz_star(n: int) -> Tuple["Grid", LevelSet]:
    """The Helmholtz example of Sec. 3.3.2: star r = 0.5 + 0.2 sin(5 theta)
    about (0.02 sqrt5, 0.02 sqrt5) in [-1,1]^2, n nodes per axis."""
    return box_grid(2, n), star(STAR_CENTER, 0.5, [5], [0.2], [0.0])


def hat_source(grid: "Grid", center=HELMHOLTZ_SOURCE, amplitude: float = 1000.0, width_h: float = 2.0):
    """amplitude times a 2D hat function of unit integral about center:
    phi(dx / e) phi(dy / e) / e^2 with phi(t) = max(0, 1 - |t|) and e = width_h h
    (the approximate delta of Sec. 3.3.2)."""
    X, Y = grid_points(grid)
    e = width_h * grid.h
    phi = lambda t: np.maximum(0.0, 1.0 - np.abs(t))
    return amplitude * phi((X - center[0]) / e) * phi((Y - center[1]) / e) / (e * e)


# ------------------------------------ quantities of interest (Sec. 3.6)

QOI_F = 3.0   # the source of both examples: Lap u = 3, u = 0 on the boundary


def qoi_ellipse(semi_x: float, semi_y: float, n: int = 256, L: float = 2.25) -> Tuple["Grid", LevelSet]:
    """First example of Sec. 3.6: the ellipse x^2/a^2 + y^2 a^2 = 1 (semi-axes
    a and 1/a, area pi) in [-L, L]^2; the semi-axes are given explicitly so that
    a parameter and its mirror 1/a can use exactly swapped values."""
    return box_grid(2, n, -L, L), ellipsoid((0.0, 0.0), (semi_x, semi_y), np.eye(3))


def qoi_rotated(theta: float, n: int = 502) -> Tuple["Grid", LevelSet]:
    """Second example of Sec. 3.6: the ellipse (x cos t - y sin t)^2/16 +
    (x sin t + y cos t)^2/4 < 1 in [-5, 5]^2 (the paper's 501^2 grid; n even
    here)."""
    c, s = math.cos(theta), math.sin(theta)
    Q = np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])
    return box_grid(2, n, -5.0, 5.0), ellipsoid((0.0, 0.0), (4.0, 2.0), Q)


def qoi_point_weights(grid: "Grid", x0: float, y0: float) -> np.ndarray:
    """Bilinear interpolation weights of the point (x0, y0) on the grid nodes."""
    w = np.zeros(grid.shape())
    fx = (x0 - grid.lo[0]) / grid.h
    fy = (y0 - grid.lo[1]) / grid.h
    i, j = int(math.floor(fx)), int(math.floor(fy))
    tx, ty = fx - i, fy - j
    w[j, i] = (1 - tx) * (1 - ty)
    w[j, i + 1] = tx * (1 - ty)
    w[j + 1, i] = (1 - tx) * ty
    w[j + 1, i + 1] = tx * ty
    return w


def qoi_rect_weights(grid: "Grid", xr=(-1.0, 1.0), yr=(-0.5, 0.5)) -> np.ndarray:
    """h^2 at the nodes inside the rectangle: the sum of u times these is the
    integral of u over it (node rule)."""
    X, Y = grid_points(grid)
    inside = (X >= xr[0]) & (X <= xr[1]) & (Y >= yr[0]) & (Y <= yr[1])
    return np.where(inside, grid.h * grid.h, 0.0)


def qoi_ellipse_exact(semi_x: float, semi_y: float) -> float:
    """u(0, 0) of Lap u = 3 in an ellipse with u = 0 on it: u = C (x^2/p^2 +
    y^2/q^2 - 1) with 2 C (1/p^2 + 1/q^2) = 3."""
    return -QOI_F / (2.0 * (1.0 / semi_x ** 2 + 1.0 / semi_y ** 2))


def qoi_rotated_exact(theta: float) -> float:
    """The integral of u over [-1,1] x [-0.5,0.5] for the rotated ellipse:
    u = C (x'^2/16 + y'^2/4 - 1), C = 3 / (2 (1/16 + 1/4)) = 4.8; over the
    rectangle the mixed moment vanishes, int x^2 = 2/3, int y^2 = 1/6, area 2."""
    c2, s2 = math.cos(theta) ** 2, math.sin(theta) ** 2
    C = QOI_F / (2.0 * (1.0 / 16.0 + 1.0 / 4.0))
    ix = c2 * (2.0 / 3.0) + s2 / 6.0
    iy = s2 * (2.0 / 3.0) + c2 / 6.0
    return C * (ix / 16.0 + iy / 4.0 - 2.0)


KAPPA_77 = 31.4227941922


def bessel_mode(x, y, t, m: int = 7, kappa: float = KAPPA_77):
    from scipy.special import jv
    r = np.sqrt(x * x + y * y)
    th = np.arctan2(y, x)
    return jv(m, kappa * r) * np.cos(m * th) * math.cos(kappa * t)


def pulse_params(seed: int = 0, center=STAR_CENTER):
    """Gaussian pulse: centre uniform in the disk of radius 0.25 about the star
    centre, width uniform in [0.02, 0.05]."""
    rng = np.random.default_rng(seed)
    rr = 0.25 * math.sqrt(rng.uniform())
    th = rng.uniform(0.0, 2.0 * math.pi)
    c = (center[0] + rr * math.cos(th), center[1] + rr * math.sin(th))
    w = rng.uniform(0.02, 0.05)
    return c, w


def pulse(x, y, c, w):
    return np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2) / (w * w))


def grid_points(grid: Grid):
    """Full-grid coordinate arrays (x fastest) for evaluating inputs at nodes."""
    xs = [grid.axis_coords(a) for a in range(grid.dim)]
    if grid.dim == 2:
        Y, X = np.meshgrid(xs[1], xs[0], indexing="ij")
        return X, Y
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return X, Y, Z
