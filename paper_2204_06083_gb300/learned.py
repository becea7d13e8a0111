"""Training of the learned preconditioner stage on the device.

Control flow only: every step runs in the library's kernels (nn_pairs,
nn_geometry, nn_train_step, pcg_solve, ...), called through the binding.

A pair store holds, for G geometries of one grid size (height x width nodes),
the node codes and diagonals of each geometry and P training pairs (s_hat, c)
with the geometry each came from.  Pairs come from the solver itself: for each
geometry a seeded white-noise right-hand side b on the CPs, its solution x* by
AMG-PCG to 1e-12, and the first `per_geo` iterates of the V-cycle iteration
x_k = x_{k-1} + V(b - A x_{k-1}) (nn_pairs).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from . import AMG, EB, Net, nn_geometry, nn_pairs


LAYER_IO = [(2, 32), (32, 32), (32, 32), (32, 32), (32, 32), (32, 1)]


def init_params(seed: int, last_scale: float = 0.01) -> np.ndarray:
    """Seeded initial parameters in the flat layout of nn_set_params: He-normal
    weights (std sqrt(2 / (9 c_in))), zero biases, the output layer scaled by
    last_scale so that the untrained stage starts close to the plain V-cycle."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (ci, co) in enumerate(LAYER_IO):
        w = rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=co * 9 * ci)
        if l == len(LAYER_IO) - 1:
            w *= last_scale
        parts += [w, np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


@dataclass
class PairStore:
    s_hat: "object"    # torch float32 [P, H, W]
    c: "object"        # torch float64 [P]
    geo_of: "object"   # torch int32 [P]
    code: "object"     # torch uint8 [G, H, W]
    diag: "object"     # torch float32 [G, H, W]
    pcg_iterations: List[int]

    @property
    def num_pairs(self) -> int:
        return int(self.s_hat.shape[0])


def make_pairs(geometries: Sequence, per_geo: int, seed: int, rtol: float = 1e-12) -> PairStore:
    """geometries: (grid, levelset) descriptors of one 2D grid size."""
    import torch
    if not geometries:
        raise ValueError("no geometries")
    g0 = geometries[0][0]
    H, W = int(g0.n[1]), int(g0.n[0])
    G, P = len(geometries), len(geometries) * per_geo
    s_hat = torch.zeros((P, H, W), dtype=torch.float32, device="cuda")
    c = torch.zeros(P, dtype=torch.float64, device="cuda")
    code = torch.zeros((G, H, W), dtype=torch.uint8, device="cuda")
    diag = torch.zeros((G, H, W), dtype=torch.float32, device="cuda")
    geo_of = torch.arange(G, dtype=torch.int32, device="cuda").repeat_interleave(per_geo)
    rng = np.random.default_rng(seed)
    iters = []
    for gi, (grid, ls) in enumerate(geometries):
        if grid.dim != 2 or (int(grid.n[1]), int(grid.n[0])) != (H, W):
            raise ValueError("all geometries of a pair store share one 2D grid size")
        eb = EB(grid, ls)
        amg = AMG(eb)
        b = torch.from_numpy(rng.standard_normal((H, W))).cuda()
        x, st = amg.solve(b, rtol=rtol, maxit=500)
        iters.append(st.iterations)
        nn_pairs(amg, b, x, per_geo, s_hat[gi * per_geo:(gi + 1) * per_geo], c[gi * per_geo:(gi + 1) * per_geo])
        nn_geometry(eb, code[gi], diag[gi])
        amg.close()
        eb.close()
    torch.cuda.synchronize()
    return PairStore(s_hat, c, geo_of, code, diag, iters)


def train(net: Net, store: PairStore, steps: int, batch: int, lr: float, seed: int, log_every: int = 50):
    """Adam steps on random batches (an epoch is a seeded permutation of the
    store); returns [(step, mean batch loss before the step)] every log_every
    steps and at the last one."""
    import torch
    rng = np.random.default_rng(seed)
    P = store.num_pairs
    if batch > P:
        raise ValueError("batch larger than the pair store")
    order = rng.permutation(P)
    pos = 0
    loss = torch.zeros(batch + 1, dtype=torch.float32, device="cuda")
    picks = []
    for _ in range(steps):
        if pos + batch > P:
            order = rng.permutation(P)
            pos = 0
        picks.append(order[pos:pos + batch])
        pos += batch
    pick_dev = torch.from_numpy(np.asarray(picks, dtype=np.int32)).cuda()
    log = []
    for t in range(steps):
        net.train_step(store.s_hat, store.c, store.geo_of, store.code, store.diag, pick_dev[t], lr, loss)
        if (t + 1) % log_every == 0 or t == steps - 1:
            log.append((t + 1, float(loss[batch].item())))
    return log
