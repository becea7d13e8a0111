"""Learned correction stage of the preconditioner (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper has no learned component; this stage is an extension of its AMG-PCG
(Algorithm 1 step 4).  What it computes, stated here once and followed by the
functions below:

Network N (6 layers, zero-padded 3x3 cross-correlations, 32 hidden channels):
    a1 = ReLU(conv(x0; W1, b1))            x0 = (s_hat, m): 2 channels
    a_{l+1} = ReLU(conv(a_l; W_l, b_l))    l = 1..4, 32 -> 32 channels
    y6 = conv(a5; W6, b6)                  32 -> 1 channel
    N(s_hat, m) = m * y6                   output kept on the CPs only
  conv(x; W, b)[co, i, j] = b[co] + sum_{d, ci} W[co, d, ci] x[ci, i+dy, j+dx]
  with tap d = 3 (dy + 1) + (dx + 1), dy, dx in {-1, 0, 1}, i the row (y) and
  j the column (x) of the grid (x fastest, as the grid's node numbering), and
  x = 0 outside the image.

Flat parameter vector theta (float):
    W1 [32][9][2], b1 [32], then for l = 1..4: W_l [32][9][32], b_l [32],
    then W6 [9][32], b6 [1]                               (NPARAM = 37,889).

Training pairs (the solver's own residual / error pairs).  For an SPD operator
A (shift included), right-hand side b, its solution x* and the V-cycle V:
    x_0 = 0,  x_k = x_{k-1} + V(b - A x_{k-1}),  e_k = x* - x_k
    t_k = h^2 A e_k (the unit-spacing operator A~ applied to e_k)
    rho_k = rms of t_k over the CPs
    s_hat_k = t_k / rho_k,  e_hat_k = e_k / rho_k,  c_k = e_hat_k' s_hat_k
so A~ e_hat_k = s_hat_k exactly: e_hat_k is what the network should return
for the input s_hat_k, the residual left after a V-cycle correction.

Loss (relative energy norm of the error of the correction):
    L(o) = ||o - e_hat||_A~^2 / ||e_hat||_A~^2 = (o'A~o - 2 o's_hat + c) / c
    dL/do = 2 (A~ o - s_hat) / c        on the CPs
A batch loss is the mean of L over its images.

Preconditioner stage (flexible PCG): z1 = V(r); s = r - A z1;
    z = z1 + omega h^2 rms(s) N(s / rms(s), m)
with omega = 1 (mode "plain") or the energy-optimal step of stage() (mode
"energy").

Adam (Kingma & Ba, 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and the
bias corrections 1 - beta^t.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import amg as amg_mod
from . import eb as ebm

NC = 32
NMID = 4
LAYER_IO = [(2, NC)] + [(NC, NC)] * NMID + [(NC, 1)]


def layer_sizes():
    """(weight count, bias count) of the six layers in theta order."""
    return [(co * 9 * ci, co) for ci, co in LAYER_IO]


NPARAM = sum(w + b for w, b in layer_sizes())


def unpack(theta: np.ndarray):
    """theta -> [(W [co, 9, ci], b [co]) for the six layers]."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == NPARAM
    out, o = [], 0
    for ci, co in LAYER_IO:
        W = theta[o:o + co * 9 * ci].reshape(co, 9, ci)
        o += co * 9 * ci
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.reshape(-1), b.reshape(-1)]) for W, b in layers])


def init_params(seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, seeded."""
    rng = np.random.default_rng(seed)
    layers = []
    for ci, co in LAYER_IO:
        W = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=(co, 9, ci))
        layers.append((W, np.zeros(co)))
    return pack(layers)


def tap(d: int):
    return d // 3 - 1, d % 3 - 1


def shifted(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """out[..., i, j] = x[..., i+dy, j+dx], zero outside the image."""
    H, W = x.shape[-2:]
    out = np.zeros_like(x)
    i0, i1 = max(0, -dy), min(H, H - dy)
    j0, j1 = max(0, -dx), min(W, W - dx)
    if i0 < i1 and j0 < j1:
        out[..., i0:i1, j0:j1] = x[..., i0 + dy:i1 + dy, j0 + dx:j1 + dx]
    return out


def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3 cross-correlation: x [ci, H, W], W [co, 9, ci], b [co]."""
    out = np.broadcast_to(b[:, None, None], (W.shape[0],) + x.shape[1:]).astype(np.float64).copy()
    for d in range(9):
        dy, dx = tap(d)
        out += np.einsum("oc,chw->ohw", W[:, d, :], shifted(x, dy, dx))
    return out


def conv3x3_transpose(g: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 in x: out[ci, p] = sum_{d, co} W[co, d, ci] g[co, p - off(d)]."""
    out = np.zeros((W.shape[2],) + g.shape[1:])
    for d in range(9):
        dy, dx = tap(d)
        out += np.einsum("oc,ohw->chw", W[:, d, :], shifted(g, -dy, -dx))
    return out


def conv3x3_wgrad(x: np.ndarray, g: np.ndarray):
    """Gradient of sum(g * conv3x3(x; W, b)) in W [co, 9, ci] and b [co]."""
    dW = np.zeros((g.shape[0], 9, x.shape[0]))
    for d in range(9):
        dy, dx = tap(d)
        dW[:, d, :] = np.einsum("ohw,chw->oc", g, shifted(x, dy, dx))
    return dW, g.sum(axis=(1, 2))


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta: np.ndarray, s_hat: np.ndarray, mask: np.ndarray, storage: str = "f64"):
    """N(s_hat, m) on one image [H, W]; returns (output [H, W], cache).

    storage = "bf16" rounds what a BF16 implementation stores (the hidden
    activations a1..a5 and the weights of the four 32 -> 32 layers) to
    bfloat16, every sum still in float64."""
    layers = unpack(theta)
    rnd = bf16 if storage == "bf16" else (lambda v: v)
    x0 = np.stack([np.asarray(s_hat, np.float64), np.asarray(mask, np.float64)])
    acts = [x0]
    a = x0
    for l in range(5):
        W, b = layers[l]
        if 1 <= l <= 4:
            W = rnd(W)
        a = rnd(np.maximum(conv3x3(a, W, b), 0.0))
        acts.append(a)
    W6, b6 = layers[5]
    y6 = conv3x3(a, W6, b6)[0]
    return mask * y6, {"acts": acts, "mask": np.asarray(mask, np.float64), "storage": storage}


def backward(theta: np.ndarray, cache, dout: np.ndarray) -> np.ndarray:
    """Gradient of sum(dout * N(s_hat, m)) in theta (reverse of forward).

    After a forward with storage = "bf16" the gradients of the five hidden
    layers' outputs are rounded to bfloat16 as a BF16 implementation stores
    them, and their propagation through the four 32 -> 32 layers uses the
    bf16 weights."""
    layers = unpack(theta)
    acts = cache["acts"]
    rnd = bf16 if cache.get("storage") == "bf16" else (lambda v: v)
    grads = [None] * 6
    g = (dout * cache["mask"])[None]
    dW, db = conv3x3_wgrad(acts[5], g)
    grads[5] = (dW, db)
    ga = conv3x3_transpose(g, layers[5][0])
    for l in range(4, -1, -1):
        g = rnd(ga * (acts[l + 1] > 0))      # through ReLU of layer l
        dW, db = conv3x3_wgrad(acts[l], g)
        grads[l] = (dW, db)
        if l > 0:
            ga = conv3x3_transpose(g, rnd(layers[l][0]))
    return pack(grads)


def unit_operator(eb: ebm.EBSystem) -> sp.csr_matrix:
    """A~ = h^2 A over the CPs (lexicographic order)."""
    return ebm.assemble_unit(eb, 0.0)


def loss(eb: ebm.EBSystem, o: np.ndarray, s_hat: np.ndarray, c: float):
    """(L, dL/do) for one image; o, s_hat full-grid [H, W] arrays."""
    At = unit_operator(eb)
    ov = eb.from_grid(o)
    sv = eb.from_grid(s_hat)
    Ao = At @ ov
    L = (ov @ Ao - 2.0 * ov @ sv + c) / c
    return L, eb.to_grid(2.0 * (Ao - sv) / c)


def cp_mask(eb: ebm.EBSystem) -> np.ndarray:
    return (eb.cls == ebm.COMPUTATIONAL).astype(np.float64).reshape(eb.grid.shape())


def pairs(eb: ebm.EBSystem, A: sp.csr_matrix, H: amg_mod.Hierarchy, b: np.ndarray, x_star: np.ndarray,
          count: int):
    """The first `count` training pairs of the V-cycle iteration (header):
    returns lists of full-grid s_hat_k, e_hat_k and the scalars c_k.  A is the
    operator the hierarchy H was built for (over the CPs), b, x_star CP
    vectors."""
    h2 = eb.grid.h ** 2
    x = np.zeros_like(b)
    S, E, C = [], [], []
    for _ in range(count):
        x = x + amg_mod.vcycle(H, b - A @ x)
        e = x_star - x
        t = h2 * (A @ e)
        rho = np.sqrt(np.mean(t * t))
        sh, eh = t / rho, e / rho
        S.append(eb.to_grid(sh))
        E.append(eb.to_grid(eh))
        C.append(float(eh @ sh))
    return S, E, C


def adam(theta, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def stage(eb: ebm.EBSystem, A: sp.csr_matrix, H: amg_mod.Hierarchy, theta: np.ndarray, r: np.ndarray,
          mode: str = "plain"):
    """Preconditioner with the learned stage on a CP vector r (header).

    mode "energy" scales the correction by omega = (o's_hat) / (o'A~o) with
    A~ = h^2 A (shift included): the step along o that minimises the energy
    norm of the remaining error A^-1 s - step, so the stage never increases
    it; a network returning exactly A~^-1 s_hat gives omega = 1."""
    z1 = amg_mod.vcycle(H, r)
    s = r - A @ z1
    rms = np.sqrt(np.mean(s * s))
    if rms == 0.0:
        return z1
    sh = s / rms
    o, _ = forward(theta, eb.to_grid(sh), cp_mask(eb))
    ov = eb.from_grid(o)
    h2 = eb.grid.h ** 2
    omega = 1.0
    if mode == "energy":
        den = ov @ (h2 * (A @ ov))
        omega = (ov @ sh) / den if den > 0.0 else 0.0
    return z1 + h2 * rms * omega * ov


def fpcg(A: sp.csr_matrix, b: np.ndarray, M, rtol=1e-10, maxit=500):
    """Flexible PCG (Polak-Ribiere beta = r_{k+1}'(z_{k+1} - z_k) / r_k'z_k);
    returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= rtol * bn:
            return x, it
        zn = M(r)
        beta = (r @ (zn - z)) / rz
        rz = r @ zn
        z = zn
        p = z + beta * p
    return x, maxit
