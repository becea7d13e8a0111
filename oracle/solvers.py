"""Krylov solvers, dense reference solves, spectra and time stepping (oracle).

* CG / PCG: Algorithm 1 step 4 (CG with an AMG preconditioner, Sec. 3
  preamble).  Reading of "relative residual": ||b - A x_k||_2 / ||b||_2 on the
  recurrence residual; at exit the true residual is recomputed and the
  iteration continues if it does not meet the tolerance.
* Dense Cholesky: the textbook solve used to pin CG / PCG on tiny grids.
* Lanczos extremes (ARPACK through scipy): the spectrum statements of Sec. 1
  and Sec. 3.1 (eigenvalues bounded like the periodic problem).
* Leapfrog: the theta-scheme of Sec. 3.5 at theta = 0,
  u^{n+1} = 2 u^n - u^{n-1} - dt^2 A u^n (homogeneous Dirichlet data).
* theta-scheme for the wave equation (Sec. 3.5) with theta > 0; the printed
  scheme lacks the Laplacian on its (1 - 2 theta) term, read as
  (I + theta dt^2 A) u^{n+1} = 2 u^n - (1 - 2 theta) dt^2 A u^n - u^{n-1}
  - theta dt^2 A u^{n-1}  (A = -L; theta = 0 is the leapfrog).
* theta-method heat step (Sec. 3.4 uses Crank-Nicolson, theta = 1/2; theta = 1
  is backward Euler):
  (I/dt + theta A) u^{n+1} = (I/dt - (1-theta) A) u^n + theta b^{n+1}
  + (1-theta) b^n, with b the right-hand side of -L u = b for the source F and
  the boundary data at that time (b = F + sum_s c_s u_Gamma / h^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class SolveStats:
    iterations: int
    rel_residual: float
    true_rel_residual: float
    converged: bool


def pcg(A, b, x0=None, M=None, rtol=1e-10, maxit=10000):
    """Preconditioned CG; ``M`` maps r -> z (None = identity)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros_like(b), SolveStats(0, 0.0, 0.0, True)
    r = b - A @ x
    it = 0
    while True:
        if np.linalg.norm(r) / bnorm <= rtol:
            break
        z = r if M is None else M(r)
        p = z.copy()
        rz = float(r @ z)
        conv = False
        while it < maxit:
            q = A @ p
            pq = float(p @ q)
            alpha = rz / pq
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            if np.linalg.norm(r) / bnorm <= rtol:
                conv = True
                break
            z = r if M is None else M(r)
            rz_new = float(r @ z)
            beta = rz_new / rz
            p = z + beta * p
            rz = rz_new
        r = b - A @ x
        if not conv or np.linalg.norm(r) / bnorm <= rtol or it >= maxit:
            break
    tr = float(np.linalg.norm(b - A @ x)) / bnorm
    return x, SolveStats(it, float(np.linalg.norm(r)) / bnorm, tr, tr <= rtol)


def dense_cholesky_solve(A, b):
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    c = sla.cho_factor(Ad, lower=True)
    return sla.cho_solve(c, b)


def extreme_eigs(A):
    """(lambda_min, lambda_max) of the SPD matrix A."""
    n = A.shape[0]
    if n <= 2000:
        w = np.linalg.eigvalsh(A.toarray())
        return float(w[0]), float(w[-1])
    lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False, tol=1e-10)[0]
    lmin = spla.eigsh(A, k=1, sigma=0.0, which="LM", return_eigenvectors=False, tol=1e-10)[0]
    return float(lmin), float(lmax)


def leapfrog(A, u_prev, u_cur, dt, nsteps):
    """Returns (u^{N-1}, u^N) after ``nsteps`` steps from (u^{-1}, u^0)."""
    a, b = np.array(u_prev, dtype=np.float64), np.array(u_cur, dtype=np.float64)
    dt2 = dt * dt
    for _ in range(nsteps):
        a, b = b, 2.0 * b - a - dt2 * (A @ b)
    return a, b


def leapfrog_energy(A, u_n, u_np1, dt):
    """Discrete energy ||(u^{n+1}-u^n)/dt||^2 + <u^{n+1}, A u^n>, conserved
    exactly by the leapfrog recursion for symmetric A."""
    v = (u_np1 - u_n) / dt
    return float(v @ v + u_np1 @ (A @ u_n))


def theta_heat_step(A, u, dt, theta, b_next, b_cur, M=None, rtol=1e-10, maxit=1000):
    """One theta-method step; warm start from u^n."""
    n = A.shape[0]
    I = sp.identity(n, format="csr")
    lhs = (I / dt + theta * A).tocsr()
    r = u / dt - (1.0 - theta) * (A @ u) + theta * b_next + (1.0 - theta) * b_cur
    return pcg(lhs, r, x0=u, M=M, rtol=rtol, maxit=maxit)


def theta_wave(A, u_prev, u_cur, dt, theta, nsteps, solve=None):
    """nsteps of the theta-scheme of Sec. 3.5 (theta > 0, homogeneous
    Dirichlet data) from (u^{-1}, u^0); returns (u^{N-1}, u^N).  solve(rhs,
    guess) solves (I + theta dt^2 A) x = rhs; default: a sparse LU
    factorisation computed once."""
    n = A.shape[0]
    dt2 = dt * dt
    M = (sp.identity(n, format="csc") + (theta * dt2) * A).tocsc()
    if solve is None:
        lu = spla.splu(M)
        solve = lambda rhs, guess: lu.solve(rhs)
    a, b = np.array(u_prev, dtype=np.float64), np.array(u_cur, dtype=np.float64)
    for _ in range(nsteps):
        rhs = 2.0 * b - (1.0 - 2.0 * theta) * dt2 * (A @ b) - a - theta * dt2 * (A @ a)
        a, b = b, solve(rhs, 2.0 * b - a)
    return a, b


def minres(A, b, x0=None, M=None, rtol=1e-10, maxit=10000):
    """Preconditioned MINRES for symmetric (indefinite) A with a symmetric
    positive definite preconditioner M (M maps r -> M^-1 r; None = identity):
    the Lanczos process in the M-inner product with Givens rotations (Paige &
    Saunders 1975; the three-term form of Elman, Silvester & Wathen, Finite
    Elements and Fast Iterative Solvers, ch. 6).  Sec. 3.3.2 solves the
    Helmholtz problem with MINRES.  Stops when the M^-1-norm of the residual
    |eta| drops below rtol times its initial value gamma_1; returns (x, stats)
    with the true relative residual ||b - A x|| / ||b|| at exit."""
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros(n), SolveStats(0, 0.0, 0.0, True)
    Mi = (lambda r: r.copy()) if M is None else M
    v_prev = np.zeros(n)
    v = b - A @ x
    z = Mi(v)
    gamma = math.sqrt(float(z @ v))
    gamma1, gamma_prev = gamma, 1.0
    eta = gamma
    c_prev, c, s_prev, s = 1.0, 1.0, 0.0, 0.0
    w_prev, w = np.zeros(n), np.zeros(n)
    it = 0
    conv = gamma == 0.0
    while not conv and it < maxit:
        z = z / gamma
        Az = A @ z
        delta = float(Az @ z)
        v_next = Az - (delta / gamma) * v - (gamma / gamma_prev) * v_prev
        z_next = Mi(v_next)
        gamma_next = math.sqrt(max(float(z_next @ v_next), 0.0))
        a0 = c * delta - c_prev * s * gamma
        a1 = math.sqrt(a0 * a0 + gamma_next * gamma_next)
        a2 = s * delta + c_prev * c * gamma
        a3 = s_prev * gamma
        c_prev, s_prev = c, s
        c, s = a0 / a1, gamma_next / a1
        w_next = (z - a3 * w_prev - a2 * w) / a1
        x = x + (c * eta) * w_next
        eta = -s * eta
        w_prev, w = w, w_next
        v_prev, v = v, v_next
        z = z_next
        gamma_prev, gamma = gamma, gamma_next
        it += 1
        conv = abs(eta) <= rtol * gamma1 or gamma == 0.0
    tr = float(np.linalg.norm(b - A @ x)) / bnorm
    return x, SolveStats(it, abs(eta) / gamma1 if gamma1 else 0.0, tr, conv)
