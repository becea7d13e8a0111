"""Deterministic smoothed-aggregation AMG preconditioner (oracle).

The paper preconditions CG with classical AMG from a Julia package and gives no
parameters (Sec. 3 preamble).  This reading replaces it by a smoothed-
aggregation hierarchy whose every decision is a fixed function of the matrix,
so that a parallel implementation can reproduce it exactly:

* strength       j != i is a strong neighbour of i iff |a_ij| >= theta
                 sqrt(a_ii a_jj), theta = 0.02 (with 0.08 the first coarse
                 level of the 3D operator has most couplings just below the
                 threshold, aggregation degenerates to singletons and the
                 operator complexity exceeds 10).
* MIS-2 roots    synchronous rounds over the strength graph.  Every node has
                 the 64-bit key (state << 62) | (hash32(i) << 30) | i with state
                 2 = root, 1 = undecided, 0 = removed; a round takes the key
                 maximum over the closed neighbourhood twice (distance 2); an
                 undecided node whose distance-2 maximum is its own key becomes
                 a root, an undecided node whose distance-2 maximum is a root
                 becomes removed.  hash32 is Wellons' "lowbias32" integer hash.
* aggregates     roots are numbered in index order; a node with a strong root
                 neighbour joins it (at most one exists); every other node
                 joins the aggregate of the strong neighbour (assigned in the
                 first pass) with the largest |a_ij| (compared rounded to
                 single precision), ties to the lowest aggregate id.  The
                 single-precision comparison is part of this specification:
                 below the finest level the entries are Galerkin sums whose
                 summation order is an implementation choice, and near-equal
                 couplings (symmetric stencils, mirrored cut cells) are common;
                 comparing them at 24 bits makes the choice independent of
                 the last FP64 bits, so that any correct summation order
                 builds the same aggregates except for weights that straddle
                 an FP32 rounding boundary.
* prolongation   P_hat = normalised constant vector per aggregate
                 (1/sqrt(|agg|)); P = (I - omega D^-1 A) P_hat with omega =
                 4/(3 rho), rho = max_i sum_j |a_ij| / a_ii (Gershgorin bound of
                 D^-1 A).  The sparsity pattern of P is that of |A| |P_hat| and
                 of A_c = P^T A P that of |P|^T |A| |P|: entries that cancel to
                 zero stay in the pattern.
* levels         coarsen until n <= 1024 (or 25 levels, or no reduction); the
                 coarsest level is solved by a dense Cholesky factorisation.
* smoother       Chebyshev polynomial of degree 2 for D^-1 A on
                 [rho/30, 1.1 rho], one sweep before and one after the coarse
                 correction (same polynomial, so the V-cycle is symmetric).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

STRENGTH_THETA = 0.02
COARSE_MAX = 1024
MAX_LEVELS = 25
CHEB_LO_FRAC = 1.0 / 30.0
CHEB_HI_FRAC = 1.1

MASK30 = np.uint64((1 << 30) - 1)


def hash32(i: np.ndarray) -> np.ndarray:
    """lowbias32 (C. Wellons): x ^= x>>16; x *= 0x7feb352d; x ^= x>>15;
    x *= 0x846ca68b; x ^= x>>16, all modulo 2^32."""
    x = np.asarray(i, dtype=np.uint32).copy()
    x ^= x >> np.uint32(16)
    x *= np.uint32(0x7FEB352D)
    x ^= x >> np.uint32(15)
    x *= np.uint32(0x846CA68B)
    x ^= x >> np.uint32(16)
    return x


def strength_graph(A: sp.csr_matrix) -> sp.csr_matrix:
    """Strong off-diagonal entries, values |a_ij| (pattern sorted per row)."""
    A = A.tocsr()
    d = A.diagonal()
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    cols = A.indices
    v = A.data
    keep = (rows != cols) & (np.abs(v) >= STRENGTH_THETA * np.sqrt(d[rows] * d[cols]))
    S = sp.csr_matrix((np.abs(v[keep]), (rows[keep], cols[keep])), shape=A.shape)
    S.sort_indices()
    return S


def _closed_max(S: sp.csr_matrix, key: np.ndarray) -> np.ndarray:
    out = key.copy()
    nnz = np.diff(S.indptr)
    rows = np.flatnonzero(nnz > 0)
    if rows.size:
        red = np.maximum.reduceat(key[S.indices], S.indptr[rows])
        out[rows] = np.maximum(out[rows], red)
    return out


def mis2(S: sp.csr_matrix) -> np.ndarray:
    """Boolean root mask of the distance-2 maximal independent set."""
    n = S.shape[0]
    idx = np.arange(n, dtype=np.uint64)
    hv = hash32(np.arange(n)).astype(np.uint64)
    state = np.ones(n, dtype=np.uint64)
    while (state == 1).any():
        key = (state << np.uint64(62)) | (hv << np.uint64(30)) | idx
        k2 = _closed_max(S, _closed_max(S, key))
        und = state == 1
        win = und & ((k2 & MASK30) == idx)
        lose = und & ~win & ((k2 >> np.uint64(62)) == 2)
        state[win] = 2
        state[lose] = 0
    return state == 2


def aggregate(A: sp.csr_matrix):
    """Aggregate id per node and the number of aggregates."""
    S = strength_graph(A)
    return aggregate_from_roots(S, mis2(S))


def aggregate_from_roots(S: sp.csr_matrix, roots: np.ndarray):
    """The two aggregation passes around given roots on the strength graph S
    (values |a_ij|): aggregate id per node and the number of aggregates."""
    n = S.shape[0]
    agg = np.full(n, -1, dtype=np.int64)
    agg[roots] = np.arange(int(roots.sum()))
    rows = np.repeat(np.arange(n), np.diff(S.indptr))
    cols = S.indices
    w = S.data
    # pass 1: strong neighbour that is a root
    m = (~roots[rows]) & roots[cols]
    first = np.full(n, -1, dtype=np.int64)
    first[rows[m]] = agg[cols[m]]
    agg1 = np.where(agg >= 0, agg, first)
    # pass 2: strongest strong neighbour assigned in pass 1, ties -> lowest id
    un = agg1 < 0
    cand = un[rows] & (agg1[cols] >= 0)
    # weights compared after rounding to single precision: a last-ulp difference
    # in the matrix (e.g. from a different libm) cannot break a tie differently
    r2, c2, w2 = rows[cand], agg1[cols[cand]], w[cand].astype(np.float32)
    order = np.lexsort((c2, -w2, r2))
    r2, c2 = r2[order], c2[order]
    firsts = np.ones(r2.size, dtype=bool)
    firsts[1:] = r2[1:] != r2[:-1]
    agg2 = agg1.copy()
    agg2[r2[firsts]] = c2[firsts]
    if (agg2 < 0).any():
        raise RuntimeError("aggregation left a node unassigned")
    return agg2, int(roots.sum())


def _on_pattern(pattern: sp.csr_matrix, values: sp.csr_matrix) -> sp.csr_matrix:
    """Values of ``values`` on the (sorted) sparsity pattern of ``pattern``;
    positions absent from ``values`` hold 0."""
    pattern = pattern.tocsr()
    pattern.sort_indices()
    values = values.tocsr()
    values.sort_indices()
    ncol = pattern.shape[1]
    pr = np.repeat(np.arange(pattern.shape[0], dtype=np.int64), np.diff(pattern.indptr))
    pk = pr * ncol + pattern.indices
    vr = np.repeat(np.arange(values.shape[0], dtype=np.int64), np.diff(values.indptr))
    vk = vr * ncol + values.indices
    pos = np.searchsorted(pk, vk)
    out = np.zeros(pk.size)
    out[pos] = values.data
    return sp.csr_matrix((out, pattern.indices.copy(), pattern.indptr.copy()), shape=pattern.shape)


def _abs(M):
    M = M.tocsr().copy()
    M.data = np.ones_like(M.data)
    return M


@dataclass
class Level:
    A: sp.csr_matrix
    dinv: np.ndarray
    rho: float
    agg: np.ndarray = None
    P: sp.csr_matrix = None
    R: sp.csr_matrix = None


@dataclass
class Hierarchy:
    levels: List[Level]
    coarse_chol: tuple


def gershgorin_rho(A: sp.csr_matrix) -> float:
    d = A.diagonal()
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    s = np.zeros(A.shape[0])
    np.add.at(s, rows, np.abs(A.data))
    return float(np.max(s / d))


# ---------------------------------------------- classical (Ruge-Stueben) AMG
# The paper's preconditioner is classical AMG (Ruge & Stueben) from a library,
# with V and W cycles (Sec. 3).  Its sequential first-pass C/F splitting is
# replaced by the parallel independent-set form of the same coarsening
# (PMIS, De Sterck, Yang & Heys 2006), with the strength, measure and direct
# interpolation of the classical method (Stueben 2001, "A review of algebraic
# multigrid", Sec. 4):
#   strength    j in S_i iff -a_ij >= theta_rs max_{k != i} (-a_ik), theta_rs = 0.25
#               (both sides rounded to single precision before comparing)
#   measure     lambda_i = |S_i^T| (how many points depend strongly on i);
#               key_i = (lambda_i << 32) | hash32(i): distinct, a fixed order
#   splitting   points no one depends on are F; then synchronous rounds over
#               the undecided set U: i in U becomes C if its key exceeds the
#               keys of every undecided j with j in S_i or i in S_j; then every
#               undecided point with a C point in its S becomes F
#   interpolation (direct) for an F point i with strong C neighbours P_i:
#               w_ij = -alpha_i a_ij / a_ii (a_ij < 0), -beta_i a_ij / a_ii
#               (a_ij > 0), alpha_i = sum_{k != i} a_ik^- / sum_{j in P_i}
#               a_ij^-, beta_i likewise for the positive parts; positive
#               couplings with no positive entry in P_i are added to a_ii.
#               C points inject (w = 1); an F point without strong C
#               neighbours gets an empty row.
RS_THETA = 0.25


def strength_rs(A: sp.csr_matrix) -> sp.csr_matrix:
    """Boolean CSR of the classical strength S (row i: the j in S_i)."""
    A = A.tocsr()
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    off = rows != A.indices
    neg = np.where(off, -A.data, -np.inf)
    mrow = np.full(n, -np.inf)
    np.maximum.at(mrow, rows, neg)
    # compared in single precision, as the aggregation weights: coarse-level
    # entries are sums whose rounding order is an implementation choice
    lhs = (-A.data).astype(np.float32)
    rhs = (RS_THETA * mrow[rows]).astype(np.float32)
    keep = off & (mrow[rows] > 0) & (lhs >= rhs)
    S = sp.csr_matrix((np.ones(int(keep.sum())), (rows[keep], A.indices[keep])), shape=A.shape)
    S.sort_indices()
    return S


def pmis(S: sp.csr_matrix) -> np.ndarray:
    """C/F splitting: 1 = C, 0 = F."""
    n = S.shape[0]
    ST = S.T.tocsr()
    lam = np.diff(ST.indptr).astype(np.uint64)          # |S_i^T|
    key = (lam << np.uint64(32)) | hash32(np.arange(n)).astype(np.uint64)
    N = ((S + ST) > 0).tocsr()                          # j in S_i or i in S_j
    N.setdiag(0)
    N.eliminate_zeros()
    state = np.full(n, -1, dtype=np.int64)              # -1 undecided, 1 C, 0 F
    state[lam == 0] = 0
    rows = np.repeat(np.arange(n), np.diff(N.indptr))
    srows = np.repeat(np.arange(n), np.diff(S.indptr))
    while (state < 0).any():
        und = state < 0
        nbmax = np.zeros(n, dtype=np.uint64)
        m = und[N.indices]
        np.maximum.at(nbmax, rows[m], key[N.indices[m]])
        newc = und & (key > nbmax)
        state[newc] = 1
        dep = np.zeros(n, dtype=bool)
        mc = state[S.indices] == 1
        dep[srows[mc]] = True
        state[(state < 0) & dep] = 0
        if not newc.any() and not (dep & und).any():
            raise RuntimeError("PMIS made no progress")
    return state.astype(np.int8)


def direct_interpolation(A: sp.csr_matrix, S: sp.csr_matrix, cf: np.ndarray) -> sp.csr_matrix:
    A = A.tocsr()
    n = A.shape[0]
    cidx = np.cumsum(cf) - 1
    nc = int(cf.sum())
    rows, cols, vals = [], [], []
    for i in range(n):
        if cf[i] == 1:
            rows.append(i); cols.append(cidx[i]); vals.append(1.0)
            continue
        a = A.data[A.indptr[i]:A.indptr[i + 1]]
        c = A.indices[A.indptr[i]:A.indptr[i + 1]]
        sc = set(S.indices[S.indptr[i]:S.indptr[i + 1]].tolist())
        aii = 0.0
        sneg = spos = pneg = ppos = 0.0
        for j, v in zip(c, a):
            if j == i:
                aii = v
                continue
            if v < 0:
                sneg += v
            else:
                spos += v
            if j in sc and cf[j] == 1:
                if v < 0:
                    pneg += v
                else:
                    ppos += v
        if ppos == 0.0:
            aii = aii + spos
        alpha = sneg / pneg if pneg != 0.0 else 0.0
        beta = spos / ppos if ppos != 0.0 else 0.0
        for j, v in zip(c, a):
            if j != i and j in sc and cf[j] == 1:
                w = -(alpha if v < 0 else beta) * v / aii
                rows.append(i); cols.append(cidx[j]); vals.append(w)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))
    P.sort_indices()
    return P


def setup(A0: sp.csr_matrix, coarsening: str = "sa") -> Hierarchy:
    """The hierarchy of A0: smoothed aggregation ("sa", the default) or
    classical Ruge-Stueben coarsening with direct interpolation ("rs")."""
    levels = []
    A = A0.tocsr()
    A.sort_indices()
    while True:
        d = A.diagonal()
        lev = Level(A=A, dinv=1.0 / d, rho=gershgorin_rho(A))
        levels.append(lev)
        n = A.shape[0]
        if n <= COARSE_MAX or len(levels) >= MAX_LEVELS:
            break
        if coarsening == "rs":
            S = strength_rs(A)
            cf = pmis(S)
            nc = int(cf.sum())
            if nc >= n or nc == 0:
                break
            P = direct_interpolation(A, S, cf)
            lev.agg = np.where(cf == 1, np.cumsum(cf) - 1, -1)
            AP = A @ P
            Ac_val = P.T.tocsr() @ AP
            Ac = _on_pattern(_abs(P).T.tocsr() @ _abs(A) @ _abs(P), Ac_val)
            lev.P, lev.R = P, P.T.tocsr()
            A = Ac
            continue
        agg, nc = aggregate(A)
        if nc >= n:
            break
        sizes = np.bincount(agg, minlength=nc).astype(np.float64)
        Phat = sp.csr_matrix((1.0 / np.sqrt(sizes[agg]), (np.arange(n), agg)), shape=(n, nc))
        omega = 4.0 / (3.0 * lev.rho)
        Pval = Phat - omega * (sp.diags(lev.dinv) @ (A @ Phat))
        P = _on_pattern(_abs(A) @ _abs(Phat), Pval)
        AP = A @ P
        Ac_val = P.T.tocsr() @ AP
        Ac = _on_pattern(_abs(P).T.tocsr() @ _abs(A) @ _abs(P), Ac_val)
        lev.agg, lev.P, lev.R = agg, P, P.T.tocsr()
        A = Ac
    Ad = levels[-1].A.toarray()
    chol = sla.cho_factor(Ad, lower=True)
    return Hierarchy(levels=levels, coarse_chol=chol)


def chebyshev(lev: Level, b: np.ndarray, x: np.ndarray, degree: int = 2) -> np.ndarray:
    """Chebyshev iteration for D^-1 A x = D^-1 b on [rho/30, 1.1 rho]
    (three-term recurrence, e.g. Saad, Iterative Methods, Alg. 12.1)."""
    lo = CHEB_LO_FRAC * lev.rho
    hi = CHEB_HI_FRAC * lev.rho
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho_old = 1.0 / sigma
    r = lev.dinv * (b - lev.A @ x)
    d = r / theta
    x = x + d
    for _ in range(degree - 1):
        rho_new = 1.0 / (2.0 * sigma - rho_old)
        r = lev.dinv * (b - lev.A @ x)
        d = (rho_new * rho_old) * d + (2.0 * rho_new / delta) * r
        x = x + d
        rho_old = rho_new
    return x


def vcycle(H: Hierarchy, b: np.ndarray, level: int = 0, gamma: int = 1, x0: np.ndarray = None) -> np.ndarray:
    """One symmetric cycle M^-1 b: a V-cycle (gamma = 1) or a W-cycle (gamma =
    2: the coarse-grid correction of every level is itself two cycles, the
    second starting from the first one's result); x0: initial guess (zero)."""
    if level == len(H.levels) - 1:
        return sla.cho_solve(H.coarse_chol, b)
    lev = H.levels[level]
    x = chebyshev(lev, b, np.zeros_like(b) if x0 is None else x0)
    r = b - lev.A @ x
    bc = lev.R @ r
    e = vcycle(H, bc, level + 1, gamma)
    if gamma == 2 and level + 1 < len(H.levels) - 1:
        e = vcycle(H, bc, level + 1, gamma, x0=e)
    x = x + lev.P @ e
    x = chebyshev(lev, b, x)
    return x


def operator_complexity(H: Hierarchy) -> float:
    return sum(l.A.nnz for l in H.levels) / H.levels[0].A.nnz
