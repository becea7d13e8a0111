"""Pins of the oracle's preconditioned MINRES (the solver of the Helmholtz
example, Sec. 3.3.2), CPU only.

* its iterates equal those of scipy's independent MINRES implementation,
  with and without the AMG V-cycle as preconditioner;
* on an SPD matrix its residual norm never exceeds CG's at the same
  iteration (MINRES minimises it over the same Krylov space) and both reach
  the same solution;
* on the indefinite Helmholtz operator of Sec. 3.3.2 (omega = 50, star
  r = 0.5 + 0.2 sin 5 theta, hat-function source) it converges to the sparse
  direct solution, and the hat source has unit integral times its amplitude.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import eb_inputs as ei
from oracle import amg, eb, solvers


def _helmholtz(n):
    grid, ls = ei.helmholtz_star(n)
    s = eb.build(grid, ls)
    K = (s.A - ei.HELMHOLTZ_OMEGA ** 2 * sp.identity(s.num_cp, format="csr")).tocsr()
    f = ei.hat_source(grid)
    b = eb.rhs(s, f, np.zeros(s.cut_cp.size))   # omega^2 u + Lap u = f  <=>  (A - omega^2) u = -f
    return grid, s, K, b, f


@pytest.mark.parametrize("precond", [False, True])
def test_minres_iterates_match_scipy(precond):
    grid, s, K, b, _ = _helmholtz(96)
    H = amg.setup(s.A)
    M = (lambda r: amg.vcycle(H, r)) if precond else None
    Mop = spla.LinearOperator(K.shape, matvec=lambda r: amg.vcycle(H, r)) if precond else None
    ref = []
    spla.minres(K, b, M=Mop, rtol=1e-300, maxiter=8, callback=lambda xk: ref.append(xk.copy()))
    for k in (1, 3, 8):
        x, st = solvers.minres(K, b, M=M, rtol=1e-300, maxit=k)
        assert st.iterations == k
        assert np.linalg.norm(x - ref[k - 1]) <= 1e-10 * np.linalg.norm(ref[k - 1])


def test_minres_residual_below_cg_on_spd():
    grid, ls = ei.circle_k1(64)
    s = eb.build(grid, ls)
    b = np.random.default_rng(0).standard_normal(s.num_cp)
    for k in (2, 5, 10, 20):
        xm, _ = solvers.minres(s.A, b, rtol=1e-300, maxit=k)
        xc, _ = solvers.pcg(s.A, b, rtol=1e-300, maxit=k)
        assert np.linalg.norm(b - s.A @ xm) <= np.linalg.norm(b - s.A @ xc) * (1 + 1e-12)
    xm, st = solvers.minres(s.A, b, rtol=1e-12)
    xd = spla.spsolve(s.A.tocsc(), b)
    assert st.converged and np.linalg.norm(xm - xd) <= 1e-9 * np.linalg.norm(xd)


def test_helmholtz_star_minres_converges_to_direct_solution():
    grid, s, K, b, f = _helmholtz(160)
    assert abs(f.sum() * grid.h ** 2 - 1000.0) < 1e-9 * 1000.0      # unit-integral hat
    xd = spla.spsolve(K.tocsc(), b)
    H = amg.setup(s.A)
    x, st = solvers.minres(K, b, M=lambda r: amg.vcycle(H, r), rtol=1e-12, maxit=5000)
    assert st.converged and st.true_rel_residual < 1e-9
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    # indefinite: a smooth vector has a negative Rayleigh quotient, a
    # grid-scale checkerboard a positive one
    smooth = np.ones(s.num_cp)
    idx = s.cp_nodes
    checker = np.where(((idx % grid.n[0]) + (idx // grid.n[0])) % 2 == 0, 1.0, -1.0)
    assert smooth @ (K @ smooth) < 0 < checker @ (K @ checker)
