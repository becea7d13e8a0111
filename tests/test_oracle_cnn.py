"""Pins of the oracle's learned stage (CPU only).

P11 (oracle side)
  * the 3x3 convolution equals scipy.signal.correlate2d summed over channels
  * a network whose every layer is a one-tap shift has the closed-form output
    m * (ReLU(s_hat) shifted by the sum of the taps) + b6
  * the transposed convolution is the adjoint of the convolution
  * backward() equals central finite differences of forward()
  * the loss is 1 at o = 0, 0 at the exact error (sparse direct solve), and
    its gradient equals finite differences
  * training pairs follow the closed form e_k = (I - M A)^k x* with M the
    V-cycle as a dense matrix; A~ e_hat_k = s_hat_k; rms(s_hat_k) = 1
  * Adam's first step is -lr g / (|g| + eps); Adam minimises a quadratic
  * flexible PCG with the stage converges to the direct solution; with a zero
    network it reproduces plain AMG-PCG
  * the energy-optimal step never leaves more error energy than the V-cycle
    alone, and is 1 for a network returning the exact error
  * bf16() rounds to nearest even and agrees with torch's conversion
"""
import numpy as np
import pytest
import scipy.signal as ss
import scipy.sparse.linalg as spla

import eb_inputs as ei
from oracle import amg, cnn, eb, solvers


def _small_system(n=40, seed=3):
    grid = ei.box_grid(2, n)
    s = eb.build(grid, ei.random_star(seed))
    return s


def test_conv_matches_scipy_correlate2d():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 9, 13))
    W = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, W, b)
    for co in range(4):
        ref = np.full((9, 13), b[co])
        for ci in range(3):
            k = W[co, :, ci].reshape(3, 3)     # k[dy + 1, dx + 1]
            ref += ss.correlate2d(x[ci], k, mode="same", boundary="fill", fillvalue=0.0)
        assert np.allclose(y[co], ref, rtol=0, atol=1e-12)


def test_shift_network_closed_form():
    rng = np.random.default_rng(1)
    H, W = 11, 14
    s_hat = rng.standard_normal((H, W))
    mask = (rng.random((H, W)) < 0.6).astype(float)
    # (dy, dx) = (0,1) (1,0) (0,1) (0,0) (1,1) (0,1): never back, so zero padding
    # between layers only drops what later taps would not bring back
    taps = [5, 7, 5, 4, 8, 5]
    layers = []
    for (ci, co), d in zip(cnn.LAYER_IO, taps):
        Wl = np.zeros((co, 9, ci))
        Wl[0, d, 0] = 1.0
        layers.append((Wl, np.zeros(co)))
    layers[5] = (layers[5][0], np.array([0.25]))
    theta = cnn.pack(layers)
    o, _ = cnn.forward(theta, s_hat, mask)
    sy = sum(cnn.tap(d)[0] for d in taps)
    sx = sum(cnn.tap(d)[1] for d in taps)
    ref = np.zeros((H, W))
    r = np.maximum(s_hat, 0.0)
    ref[:H - sy, :W - sx] = r[sy:, sx:]
    assert (sy, sx) == (2, 4)
    assert np.array_equal(o, mask * (ref + 0.25))


def test_transpose_is_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 8, 7))
    g = rng.standard_normal((6, 8, 7))
    W = rng.standard_normal((6, 9, 5))
    lhs = np.sum(cnn.conv3x3(x, W, np.zeros(6)) * g)
    rhs = np.sum(x * cnn.conv3x3_transpose(g, W))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(4)
    H, W = 7, 6
    s_hat = rng.standard_normal((H, W))
    mask = (rng.random((H, W)) < 0.7).astype(float)
    theta = cnn.init_params(5)
    layers = cnn.unpack(theta)
    layers = [(Wl, rng.uniform(0.05, 0.2, size=b.shape)) for Wl, b in layers]
    theta = cnn.pack(layers)
    dout = rng.standard_normal((H, W))

    def f(t):
        return float(np.sum(dout * cnn.forward(t, s_hat, mask)[0]))

    o, cache = cnn.forward(theta, s_hat, mask)
    g = cnn.backward(theta, cache, dout)
    eps = 1e-6
    # a few coordinates of every layer
    offs = np.cumsum([0] + [w + b for w, b in cnn.layer_sizes()])
    idx = np.concatenate([rng.choice(np.arange(offs[l], offs[l + 1]), size=12, replace=False) for l in range(6)])
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = eps
        fd = (f(theta + e) - f(theta - e)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
    v = rng.standard_normal(theta.size)
    fd = (f(theta + eps * v) - f(theta - eps * v)) / (2 * eps)
    assert abs(fd - g @ v) <= 1e-6 * abs(g @ v)


def test_loss_values_and_gradient():
    s = _small_system()
    rng = np.random.default_rng(6)
    At = cnn.unit_operator(s)
    sv = rng.standard_normal(s.num_cp)
    sv /= np.sqrt(np.mean(sv * sv))
    ev = spla.spsolve(At.tocsc(), sv)
    c = float(ev @ sv)
    s_hat = s.to_grid(sv)
    L0, _ = cnn.loss(s, np.zeros_like(s_hat), s_hat, c)
    assert L0 == 1.0
    L1, g1 = cnn.loss(s, s.to_grid(ev), s_hat, c)
    assert abs(L1) < 1e-10 and np.abs(g1).max() < 1e-10 * np.abs(s_hat).max() / c
    o = s.to_grid(rng.standard_normal(s.num_cp))
    L, g = cnn.loss(s, o, s_hat, c)
    # off-CP entries of the gradient vanish
    assert np.all(g.reshape(-1)[s.cls.reshape(-1) != eb.COMPUTATIONAL] == 0.0)
    for k in rng.choice(s.cp_nodes, size=8, replace=False):
        e = np.zeros(s.grid.num_nodes)
        e[k] = 1e-5
        e = e.reshape(o.shape)
        fd = (cnn.loss(s, o + e, s_hat, c)[0] - cnn.loss(s, o - e, s_hat, c)[0]) / 2e-5
        assert abs(fd - g.reshape(-1)[k]) <= 1e-6 * max(1.0, abs(fd))


def test_pairs_closed_form():
    s = eb.build(ei.box_grid(2, 84), ei.random_star(7))
    H = amg.setup(s.A)
    assert len(H.levels) >= 2   # V is not the exact inverse
    n = s.num_cp
    rng = np.random.default_rng(8)
    b = rng.standard_normal(n)
    x_star = solvers.dense_cholesky_solve(s.A, b)
    S, E, C = cnn.pairs(s, s.A, H, b, x_star, 4)
    M = np.column_stack([amg.vcycle(H, np.eye(n)[:, i]) for i in range(n)])
    G = np.eye(n) - M @ s.A.toarray()
    At = cnn.unit_operator(s)
    ek = x_star.copy()
    prev = np.inf
    for k in range(4):
        ek = G @ ek
        sv, evh = s.from_grid(S[k]), s.from_grid(E[k])
        rho = np.linalg.norm(ek) / np.linalg.norm(evh)
        assert np.allclose(evh * rho, ek, rtol=0, atol=1e-10 * np.abs(ek).max())
        assert np.abs(At @ evh - sv).max() <= 1e-9 * np.abs(sv).max()
        assert abs(np.sqrt(np.mean(sv * sv)) - 1.0) < 1e-12
        assert abs(C[k] - evh @ (At @ evh)) <= 1e-10 * C[k]
        energy = ek @ (s.A @ ek)
        assert energy < prev
        prev = energy


def test_adam_first_step_and_quadratic():
    rng = np.random.default_rng(9)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    t1, m, v = cnn.adam(th, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    target = rng.standard_normal(50)
    x, m, v = np.zeros(50), np.zeros(50), np.zeros(50)
    for t in range(1, 3001):
        x, m, v = cnn.adam(x, 2 * (x - target), m, v, t, 1e-2)
    assert np.abs(x - target).max() < 1e-3


def test_fpcg_with_stage_converges_and_reduces_to_pcg():
    s = _small_system(48, 11)
    H = amg.setup(s.A)
    rng = np.random.default_rng(12)
    b = rng.standard_normal(s.num_cp)
    xd = solvers.dense_cholesky_solve(s.A, b)
    theta = cnn.init_params(13) * 0.1
    x, it = cnn.fpcg(s.A, b, lambda r: cnn.stage(s, s.A, H, theta, r), rtol=1e-12)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    zero = np.zeros(cnn.NPARAM)
    x0, it0 = cnn.fpcg(s.A, b, lambda r: cnn.stage(s, s.A, H, zero, r), rtol=1e-10)
    x1, st = solvers.pcg(s.A, b, M=lambda r: amg.vcycle(H, r), rtol=1e-10)
    assert it0 == st.iterations
    assert np.linalg.norm(x0 - x1) <= 1e-9 * np.linalg.norm(x1)


def test_bf16_rounding():
    one = 1.0
    assert cnn.bf16(np.array([one + 2.0 ** -8]))[0] == 1.0            # tie to even (down)
    assert cnn.bf16(np.array([one + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie to even (up)
    assert cnn.bf16(np.array([one + 2.0 ** -8 + 2.0 ** -20]))[0] == 1.0 + 2.0 ** -7
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(10).standard_normal(4096).astype(np.float32) * 100
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(x), ref)


def test_energy_step_never_increases_error_energy():
    s = _small_system(84, 14)
    H = amg.setup(s.A)
    assert len(H.levels) >= 2   # V is not the exact inverse
    rng = np.random.default_rng(15)
    A = s.A
    Ad = A.toarray()
    for trial in range(4):
        r = rng.standard_normal(s.num_cp)
        delta = np.linalg.solve(Ad, r)             # exact error of the preconditioning step
        z1 = amg.vcycle(H, r)
        theta = cnn.init_params(20 + trial) * (0.5 + trial)
        z = cnn.stage(s, A, H, theta, r, mode="energy")
        e1, e2 = delta - z1, delta - z
        assert e2 @ (A @ e2) <= e1 @ (A @ e1) * (1 + 1e-12)
    # a "network" equal to the exact correction: omega = 1, zero error left
    r = rng.standard_normal(s.num_cp)
    z1 = amg.vcycle(H, r)
    res = r - A @ z1
    exact = np.linalg.solve(Ad, res)
    ov = exact * s.grid.h ** -2 / np.sqrt(np.mean(res * res))
    sh = res / np.sqrt(np.mean(res * res))
    omega = (ov @ sh) / (ov @ (s.grid.h ** 2 * (A @ ov)))
    assert abs(omega - 1.0) < 1e-10
