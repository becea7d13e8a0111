"""The PCG recurrences of the GPU path, restated in numpy, against the oracle's
textbook PCG (Algorithm 1 step 4), on the CPU.

The GPU iteration reorganises the textbook steps without changing the iterates
in exact arithmetic: q holds B p with B = h^2 (sigma I + A) (the unit stencil)
and is updated as q = B z + beta q in the same pass as p = z + beta p; alpha is
formed from p'q with that q and x takes the step alpha h^2; with the flexible
(Polak-Ribiere) beta, the term r_{k+1}'z_k is summed right after the r update,
from the z of the iteration ending.  With a fixed SPD preconditioner (the FP64
V-cycle) r_{k+1}'z_k = 0, so the flexible beta equals the textbook one and both
variants must reproduce the oracle's iterates to rounding; a mistake in the
reorganisation (a wrong z in r'zold, a missing h^2, a stale q) does not.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import eb_inputs as ei
from oracle import amg, eb, solvers


def _gpu_order_pcg(A, B, h2, b, M, iters, flexible):
    """x_1 .. x_iters in the order the GPU kernels compute them."""
    x = np.zeros_like(b)
    r = b - A @ x
    z = M(r)
    rz = float(r @ z)
    p = z.copy()
    q = B @ z
    xs = []
    for _ in range(iters):
        alpha = rz / float(p @ q)
        x = x + (alpha * h2) * p
        r = r - alpha * q
        rzo = float(r @ z) if flexible else 0.0
        z = M(r)
        rz_new = float(r @ z)
        beta = (rz_new - rzo) / rz
        rz = rz_new
        p = z + beta * p
        q = B @ z + beta * q
        xs.append(x.copy())
    return xs


# two-level hierarchies (N_C above the coarsest size), so the preconditioner is
# not an exact solve and the iterates differ from step to step
CASES = {
    "circle128": (lambda: ei.circle_k1(128), 0.0),
    "circle128_heat": (lambda: ei.circle_k1(128), 40.0),
    "ellipsoid40": (lambda: ei.ellipsoid_k3(40, seed=1), 0.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("flexible", [False, True])
def test_gpu_order_matches_textbook_pcg(name, flexible):
    make, sigma = CASES[name]
    grid, ls = make()
    E = eb.build(grid, ls)
    h2 = grid.h * grid.h
    A = (E.A + sigma * sp.identity(E.num_cp, format="csr")).tocsr()
    B = eb.assemble_unit(E, sigma * h2)
    assert abs(B - h2 * A).max() <= 1e-12 * abs(B).max()
    H = amg.setup(A)
    assert len(H.levels) >= 2
    M = lambda v: amg.vcycle(H, v)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(E.num_cp)
    iters = 8
    xs = _gpu_order_pcg(A, B, h2, b, M, iters, flexible)
    for k in range(1, iters + 1):
        x_ref, st = solvers.pcg(A, b, M=M, rtol=1e-300, maxit=k)
        assert st.iterations == k
        err = np.linalg.norm(xs[k - 1] - x_ref) / np.linalg.norm(x_ref)
        assert err <= 1e-9, (k, err)


def test_wrong_rzold_is_caught():
    """The pin has teeth: taking r_{k+1}'z_{k+1} for the r'zold term (the z after
    the preconditioner instead of before it) makes beta 0 and the iterates leave
    the textbook ones."""
    grid, ls = ei.circle_k1(128)
    E = eb.build(grid, ls)
    h2 = grid.h * grid.h
    A = E.A.tocsr()
    B = eb.assemble_unit(E, 0.0)
    H = amg.setup(A)
    assert len(H.levels) >= 2
    M = lambda v: amg.vcycle(H, v)
    b = np.random.default_rng(5).standard_normal(E.num_cp)
    x = np.zeros_like(b)
    r = b.copy()
    z = M(r)
    rz = float(r @ z)
    p, q = z.copy(), B @ z
    for _ in range(4):
        alpha = rz / float(p @ q)
        x = x + (alpha * h2) * p
        r = r - alpha * q
        z = M(r)
        rz_new = float(r @ z)
        beta = (rz_new - float(r @ z)) / rz   # the mistake
        rz = rz_new
        p = z + beta * p
        q = B @ z + beta * q
    x_ref, _ = solvers.pcg(A, b, M=M, rtol=1e-300, maxit=4)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) > 1e-3
