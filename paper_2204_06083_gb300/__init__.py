"""Python binding of the GB300 embedded-boundary Laplacian library.

Thin ctypes layer over the C ABI of ``include/eb.h`` (``_lib/libeb.so``, built
by ``build.py``): argument marshalling only.  Every step of the method runs in
the library's CUDA kernels; vectors are ``torch`` CUDA tensors passed by their
device pointers together with torch's current CUDA stream.  Importing the
package does not load the library; the first call does, and raises if the
library is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libeb.so")

EB_OK, EB_ERR_INVALID, EB_ERR_GEOMETRY, EB_ERR_CUDA, EB_ERR_NONFINITE = 0, 1, 2, 3, 4
EB_ERR_NO_CONVERGENCE, EB_ERR_BREAKDOWN, EB_ERR_TIMEOUT, EB_ERR_OOM, EB_ERR_NOT_IMPLEMENTED = 5, 6, 7, 8, 9
EB_F64, EB_F32, EB_BF16, EB_DF64 = 0, 1, 2, 3
EB_PC_AMG, EB_PC_JACOBI, EB_PC_NONE, EB_PC_AMG_NN = 0, 1, 2, 3
EB_NN_PLAIN, EB_NN_ENERGY = 0, 1
EB_TUNE_APPLY, EB_TUNE_LEAPFROG = 0, 1
EB_TK_SMOOTH_STEP = 0
STAR_MAX = 16

CODE_BP = 0x40
CODE_CP = 0x80


def time_copy_us(nbytes: int, launches: int = 20, clear_bytes: int = 0, stream=None) -> float:
    """Microseconds per launch of a plain copy moving nbytes (half read, half
    written), timed like amg_time_kernel (eb_time_copy)."""
    out = C.c_double()
    _check(load().eb_time_copy(int(nbytes), int(launches), int(clear_bytes), C.byref(out), _stream(stream)))
    return out.value


def fp64_peak_tflops(reps: int = 20, stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s."""
    out = C.c_double()
    _check(load().eb_fp64_peak(int(reps), C.byref(out), _stream(stream)))
    return out.value


class EBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[eb status {code}] {msg}")
        self.code = code


class eb_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("h", C.c_double)]


class eb_levelset(C.Structure):
    _fields_ = [("kind", C.c_int), ("center", C.c_double * 3), ("semi", C.c_double * 3), ("rot", C.c_double * 9),
                ("r0", C.c_double), ("nk", C.c_int), ("k", C.c_int * STAR_MAX), ("a", C.c_double * STAR_MAX),
                ("p", C.c_double * STAR_MAX), ("psi", C.c_void_p)]


class eb_info_t(C.Structure):
    _fields_ = [("num_nodes", C.c_int64), ("num_cp", C.c_int64), ("num_bp", C.c_int64), ("num_cut", C.c_int64),
                ("num_far", C.c_int64), ("num_tiles", C.c_int64), ("tile", C.c_int * 3),
                ("max_delta_over_h", C.c_double), ("min_abs_psi", C.c_double),
                ("min_dominance_margin", C.c_double), ("num_rbf", C.c_int64), ("num_rbf_rotated", C.c_int64)]


class eb_build_opts(C.Structure):
    _fields_ = [("closure", C.c_int), ("rbf_eps", C.c_double)]


EB_CLOSURE_LINE, EB_CLOSURE_MIXED, EB_CLOSURE_RBF = 0, 1, 2


class amg_opts(C.Structure):
    _fields_ = [("max_levels", C.c_int), ("coarse_max", C.c_int), ("strength", C.c_double),
                ("cheb_degree", C.c_int), ("vcycle_prec", C.c_int), ("coarsening", C.c_int), ("cycle", C.c_int)]


EB_AMG_SA, EB_AMG_RS = 0, 1


class amg_info_t(C.Structure):
    _fields_ = [("num_levels", C.c_int), ("rows", C.c_int64 * 32), ("nnz", C.c_int64 * 32),
                ("operator_complexity", C.c_double), ("setup_ms", C.c_double)]


class pcg_opts(C.Structure):
    _fields_ = [("precond", C.c_int), ("check_every", C.c_int), ("use_graph", C.c_int), ("profile", C.c_int),
                ("outer_prec", C.c_int)]


class pcg_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("true_rel_residual", C.c_double),
                ("solve_ms", C.c_double), ("converged", C.c_int), ("prof_kernel_ms", C.c_double),
                ("prof_launches", C.c_int), ("launches", C.c_int64)]


class eb_tune_t(C.Structure):
    _fields_ = [("count", C.c_int), ("tile", (C.c_int * 3) * 16), ("us", C.c_double * 16), ("best", C.c_int)]


@dataclass
class TuneResult:
    shapes: list
    us: list
    best: int

    @property
    def shape(self):
        return self.shapes[self.best]


def _tune_result(t: eb_tune_t) -> TuneResult:
    return TuneResult([tuple(t.tile[i]) for i in range(t.count)], [t.us[i] for i in range(t.count)], t.best)


_P = C.c_void_p
_SIGS = {
    "eb_build": (C.c_int, [C.POINTER(eb_grid), C.POINTER(eb_levelset), C.POINTER(_P), _P]),
    "eb_destroy": (None, [_P]),
    "eb_build_ex": (C.c_int, [C.POINTER(eb_grid), C.POINTER(eb_levelset), C.POINTER(eb_build_opts), C.POINTER(_P),
                              _P]),
    "eb_rbf_cuts": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "eb_info": (C.c_int, [_P, C.POINTER(eb_info_t)]),
    "eb_classes": (C.c_int, [_P, _P, _P]),
    "eb_cp_data": (C.c_int, [_P, _P, _P, _P]),
    "eb_cuts": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "eb_rhs": (C.c_int, [_P, _P, _P, _P, _P]),
    "eb_apply": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "eb_retile": (C.c_int, [_P, _P, _P]),
    "eb_autotune": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(eb_tune_t), _P]),
    "amg_autotune": (C.c_int, [_P, C.c_int, C.POINTER(eb_tune_t), _P]),
    "amg_tune_csr": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "amg_time_kernel": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int64, _P, _P]),
    "amg_set_csr_epl": (C.c_int, [_P, C.c_int]),
    "batch_autotune": (C.c_int, [_P, C.c_int, C.POINTER(eb_tune_t), _P]),
    "amg_setup": (C.c_int, [_P, C.c_double, C.POINTER(amg_opts), C.POINTER(_P), _P]),
    "amg_destroy": (None, [_P]),
    "amg_info": (C.c_int, [_P, C.POINTER(amg_info_t)]),
    "amg_level_copy": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, _P]),
    "amg_vcycle": (C.c_int, [_P, _P, _P, _P]),
    "amg_set_outer_prec": (C.c_int, [_P, C.c_int]),
    "pcg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.POINTER(pcg_opts), C.POINTER(pcg_stats), _P]),
    "heat_step": (C.c_int, [_P, C.c_double, C.c_double, _P, _P, _P, C.c_double, C.c_int, C.POINTER(pcg_stats), _P]),
    "wave_step": (C.c_int, [_P, C.c_int, C.c_double, _P, _P, C.c_int, _P]),
    "wave_step_noalloc": (C.c_int, [_P, C.c_int, C.c_double, _P, _P, C.c_int, _P]),
    "batch_build": (C.c_int, [_P, _P, C.c_int, C.POINTER(_P), _P]),
    "batch_destroy": (None, [_P]),
    "batch_info": (C.c_int, [_P, _P]),
    "batch_offsets": (C.c_int, [_P, _P, _P, _P]),
    "batch_geometry": (_P, [_P, C.c_int]),
    "batch_rhs": (C.c_int, [_P, _P, _P, _P, _P]),
    "batch_heat_setup": (C.c_int, [_P, _P, C.c_double, C.POINTER(amg_opts), _P]),
    "batch_heat_step": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_int, _P, _P]),
    "batch_set_profile": (C.c_int, [_P, C.c_int]),
    "batch_set_outer_prec": (C.c_int, [_P, C.c_int]),
    "batch_set_level0_tma": (C.c_int, [_P, C.c_int]),
    "nn_create": (C.c_int, [C.POINTER(_P), _P]),
    "nn_destroy": (None, [_P]),
    "nn_num_params": (C.c_int, []),
    "nn_status": (C.c_int, [_P, _P]),
    "nn_set_profile": (C.c_int, [_P, C.c_int]),
    "nn_set_fused": (C.c_int, [_P, C.c_int]),
    "nn_profile": (C.c_int, [_P, _P, _P, _P]),
    "nn_set_params": (C.c_int, [_P, _P, _P]),
    "nn_get_params": (C.c_int, [_P, _P, _P, _P]),
    "nn_forward": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "nn_backward": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "nn_pairs": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P, _P]),
    "nn_geometry": (C.c_int, [_P, _P, _P, _P]),
    "nn_train_step": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, C.c_float, _P, _P]),
    "nn_precondition": (C.c_int, [_P, _P, C.c_int, _P, _P, _P]),
    "pcg_solve_nn": (C.c_int, [_P, _P, C.c_int, _P, _P, C.c_double, C.c_int, C.POINTER(pcg_opts),
                               C.POINTER(pcg_stats), _P]),
    "eb_fp64_peak": (C.c_int, [C.c_int, _P, _P]),
    "eb_set_beta": (C.c_int, [_P, _P, _P, _P, _P]),
    "eb_time_copy": (C.c_int, [C.c_int64, C.c_int, C.c_int64, _P, _P]),
    "eb_time_apply": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.c_int64, _P, _P]),
    "batch_weighted_sum": (C.c_int, [_P, _P, _P, _P, _P]),
    "minres_solve": (C.c_int, [_P, C.c_double, C.c_int, _P, _P, C.c_double, C.c_int, C.POINTER(pcg_stats), _P]),
    "wave_theta_step": (C.c_int, [_P, C.c_double, C.c_double, _P, _P, C.c_int, C.c_double, C.c_int,
                                  C.POINTER(pcg_stats), _P]),
    "eb_last_error": (C.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return LIB_PATH


def load(path: Optional[str] = None) -> C.CDLL:
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: run paper_2204_06083_gb300.build.build() first")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS.keys())


def _check(code: int, allow=()):
    if code != EB_OK and code not in allow:
        raise EBError(code, load().eb_last_error().decode())
    return code


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def make_grid(g) -> eb_grid:
    """eb_grid from an ``eb_inputs.Grid``-like object (dim, n, lo, h)."""
    out = eb_grid()
    out.dim = g.dim
    for a in range(3):
        out.n[a] = int(g.n[a])
        out.lo[a] = float(g.lo[a])
    out.h = float(g.h)
    return out


EB_LS_QUADRIC, EB_LS_STAR2D, EB_LS_SAMPLED = 0, 1, 2


def sampled_psi_on_device(ls):
    """The node values of a sampled level set as a contiguous CUDA float64
    tensor (the caller keeps it alive while eb_build / batch_build run)."""
    import numpy as np
    import torch
    if getattr(ls, "psi", None) is None:
        raise ValueError("sampled level set without psi values")
    psi = ls.psi
    if not isinstance(psi, torch.Tensor):
        psi = torch.from_numpy(np.ascontiguousarray(psi, dtype=np.float64))
    return psi.to(device="cuda", dtype=torch.float64).contiguous()


def make_levelset(ls, psi_dev=None) -> eb_levelset:
    """eb_levelset from an ``eb_inputs.LevelSet``-like descriptor; psi_dev: the
    CUDA tensor of node values of a sampled level set."""
    out = eb_levelset()
    out.kind = int(ls.kind)
    for a in range(3):
        out.center[a] = float(ls.center[a])
        out.semi[a] = float(ls.semi[a])
    for a in range(9):
        out.rot[a] = float(ls.rot[a])
    out.r0 = float(ls.r0)
    if len(ls.ks) > STAR_MAX:
        raise ValueError("too many star terms")
    out.nk = len(ls.ks)
    for j, (k, a, p) in enumerate(zip(ls.ks, ls.amps, ls.phases)):
        out.k[j] = int(k)
        out.a[j] = float(a)
        out.p[j] = float(p)
    if int(ls.kind) == EB_LS_SAMPLED:
        if psi_dev is None:
            raise ValueError("sampled level set: pass its node values on the device")
        out.psi = C.c_void_p(psi_dev.data_ptr())
    return out


@dataclass
class Info:
    num_nodes: int
    num_cp: int
    num_bp: int
    num_cut: int
    num_far: int
    num_tiles: int
    tile: tuple
    max_delta_over_h: float
    min_abs_psi: float
    min_dominance_margin: float
    num_rbf: int = 0
    num_rbf_rotated: int = 0


class EB:
    """Handle of eb_build: the classified grid, cuts and diagonal."""

    def __init__(self, grid, levelset, stream=None, closure=EB_CLOSURE_LINE, rbf_eps=0.025):
        lib = load()
        self._h = C.c_void_p()
        self.grid = grid
        self.dim = grid.dim
        g = make_grid(grid)
        psi_dev = sampled_psi_on_device(levelset) if int(levelset.kind) == EB_LS_SAMPLED else None
        ls = make_levelset(levelset, psi_dev)
        o = eb_build_opts(int(closure), float(rbf_eps))
        _check(lib.eb_build_ex(C.byref(g), C.byref(ls), C.byref(o), C.byref(self._h), _stream(stream)))
        inf = eb_info_t()
        _check(lib.eb_info(self._h, C.byref(inf)))
        self.info = Info(inf.num_nodes, inf.num_cp, inf.num_bp, inf.num_cut, inf.num_far, inf.num_tiles,
                         tuple(inf.tile), inf.max_delta_over_h, inf.min_abs_psi, inf.min_dominance_margin,
                         inf.num_rbf, inf.num_rbf_rotated)

    def close(self):
        if self._h:
            load().eb_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def shape(self):
        g = self.grid
        return (g.n[1], g.n[0]) if g.dim == 2 else (g.n[2], g.n[1], g.n[0])

    def classes(self, stream=None):
        import torch
        out = torch.empty(self.info.num_nodes, dtype=torch.uint8, device="cuda")
        _check(load().eb_classes(self._h, _ptr(out), _stream(stream)))
        return out.view(self.shape())

    def cp_data(self, stream=None):
        import torch
        n = self.info.num_cp
        nodes = torch.empty(n, dtype=torch.int32, device="cuda")
        diag = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(load().eb_cp_data(self._h, _ptr(nodes), _ptr(diag), _stream(stream)))
        return nodes, diag

    def cuts(self, stream=None):
        import torch
        n = self.info.num_cut
        cp = torch.empty(n, dtype=torch.int32, device="cuda")
        d = torch.empty(n, dtype=torch.int32, device="cuda")
        delta = torch.empty(n, dtype=torch.float64, device="cuda")
        xg = torch.empty((n, self.dim), dtype=torch.float64, device="cuda")
        _check(load().eb_cuts(self._h, _ptr(cp), _ptr(d), _ptr(delta), _ptr(xg), _stream(stream)))
        return cp, d, delta, xg

    def rbf_cuts(self, stream=None):
        """(cut index, G2 [n, 2], weights (w_ij, w_1, w_2) [n, 3], rotated) of the RBF cuts."""
        import torch
        n = self.info.num_rbf
        idx = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        xg2 = torch.empty((max(n, 1), 2), dtype=torch.float64, device="cuda")
        w = torch.empty((max(n, 1), 3), dtype=torch.float64, device="cuda")
        rot = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        _check(load().eb_rbf_cuts(self._h, _ptr(idx), _ptr(xg2), _ptr(w), _ptr(rot), _stream(stream)))
        return idx[:n], xg2[:n], w[:n], rot[:n]

    def sample_points(self, stream=None):
        """The boundary points whose values eb_rhs takes, in its order: each
        cut's crossing, then the second point of every RBF cut."""
        import torch
        _, _, _, xg = self.cuts(stream)
        if self.info.num_rbf == 0:
            return xg
        return torch.cat([xg, self.rbf_cuts(stream)[1]], dim=0)

    def rhs(self, f, ugamma, out=None, stream=None):
        import torch
        if out is None:
            out = torch.zeros(self.shape(), dtype=torch.float64, device="cuda")
        _check(load().eb_rhs(self._h, _ptr(f), _ptr(ugamma), _ptr(out), _stream(stream)))
        return out

    def apply(self, x, out=None, stream=None):
        import torch
        prec = {torch.float64: EB_F64, torch.float32: EB_F32, torch.bfloat16: EB_BF16}[x.dtype]
        if out is None:
            out = torch.zeros_like(x)
        _check(load().eb_apply(self._h, prec, _ptr(x), _ptr(out), _stream(stream)))
        return out

    def time_apply_us(self, x, out, launches: int = 20, clear_bytes: int = 0, stream=None) -> float:
        """Microseconds per eb_apply launch on x -> out, launches captured in one
        graph, each after a read of clear_bytes when > 0 (eb_time_apply)."""
        import torch
        prec = {torch.float64: EB_F64, torch.float32: EB_F32, torch.bfloat16: EB_BF16}[x.dtype]
        us = C.c_double()
        _check(load().eb_time_apply(self._h, prec, _ptr(x), _ptr(out), int(launches), int(clear_bytes),
                                    C.byref(us), _stream(stream)))
        return us.value

    def set_beta(self, betas, stream=None):
        """Variable coefficient of eq. 3: betas = one full-grid array per axis
        (numpy or torch), beta at node + h/2 e_axis (eb_set_beta)."""
        import numpy as np
        import torch
        dev = []
        for b in betas:
            t = b if isinstance(b, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(b, dtype=np.float64))
            dev.append(t.to(device="cuda", dtype=torch.float64).contiguous())
        ptrs = [_ptr(t) for t in dev] + [None] * (3 - len(dev))
        _check(load().eb_set_beta(self._h, ptrs[0], ptrs[1], ptrs[2], _stream(stream)))
        self._refresh_info()

    def _refresh_info(self):
        inf = eb_info_t()
        _check(load().eb_info(self._h, C.byref(inf)))
        self.info = Info(inf.num_nodes, inf.num_cp, inf.num_bp, inf.num_cut, inf.num_far, inf.num_tiles,
                         tuple(inf.tile), inf.max_delta_over_h, inf.min_abs_psi, inf.min_dominance_margin,
                         inf.num_rbf, inf.num_rbf_rotated)

    def retile(self, shape, stream=None):
        t = (C.c_int * 3)(*[int(v) for v in shape])
        _check(load().eb_retile(self._h, C.cast(t, C.c_void_p), _stream(stream)))
        self._refresh_info()

    def autotune(self, prec=EB_F64, reps=20, op=EB_TUNE_APPLY, stream=None) -> TuneResult:
        """Times eb_apply (or 16 leapfrog steps) for every candidate tile shape and keeps the fastest."""
        t = eb_tune_t()
        _check(load().eb_autotune(self._h, int(op), int(prec), int(reps), C.byref(t), _stream(stream)))
        self._refresh_info()
        return _tune_result(t)

    def wave_step(self, u_prev, u_cur, dt, nsteps, stream=None):
        import torch
        prec = {torch.float64: EB_F64, torch.float32: EB_F32}[u_cur.dtype]
        return _check(load().wave_step(self._h, prec, float(dt), _ptr(u_prev), _ptr(u_cur), int(nsteps),
                                       _stream(stream)))


class AMG:
    """Handle of amg_setup: AMG hierarchy (or Jacobi only) for sigma I + A."""

    def __init__(self, eb: EB, shift: float = 0.0, max_levels: int = 25, coarse_max: int = 1024,
                 strength: float = 0.02, cheb_degree: int = 2, vcycle_prec: int = EB_F64, coarsening: int = EB_AMG_SA,
                 cycle: int = 1, stream=None):
        lib = load()
        self.eb = eb
        self.shift = shift
        self.vcycle_prec = vcycle_prec
        o = amg_opts(max_levels, coarse_max, strength, cheb_degree, vcycle_prec, coarsening, cycle)
        self._h = C.c_void_p()
        _check(lib.amg_setup(eb.handle, float(shift), C.byref(o), C.byref(self._h), _stream(stream)))
        inf = amg_info_t()
        _check(lib.amg_info(self._h, C.byref(inf)))
        self.num_levels = inf.num_levels
        self.rows = [inf.rows[i] for i in range(inf.num_levels)]
        self.nnz = [inf.nnz[i] for i in range(inf.num_levels)]
        self.operator_complexity = inf.operator_complexity
        self.setup_ms = inf.setup_ms

    def close(self):
        if self._h:
            load().amg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level(self, level: int, which: int):
        """CSR of A_l (which=0) or P_l (which=1) as torch tensors; which=2: aggregates."""
        import torch
        if which == 2:
            agg = torch.empty(self.rows[level], dtype=torch.int32, device="cuda")
            _check(load().amg_level_copy(self._h, level, 2, None, _ptr(agg), None, _stream()))
            return agg
        nrow = self.rows[level]
        if which == 0:
            nnz = self.nnz[level]
        else:
            nnz = self._p_nnz(level)
        rp = torch.empty(nrow + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
        _check(load().amg_level_copy(self._h, level, which, _ptr(rp), _ptr(col), _ptr(val), _stream()))
        return rp, col[:nnz], val[:nnz]

    def _p_nnz(self, level):
        import torch
        rp = torch.empty(self.rows[level] + 1, dtype=torch.int32, device="cuda")
        _check(load().amg_level_copy(self._h, level, 1, _ptr(rp), None, None, _stream()))
        return int(rp[-1].item())

    def vcycle(self, r, out=None, stream=None):
        import torch
        if out is None:
            out = torch.zeros_like(r)
        _check(load().amg_vcycle(self._h, _ptr(r), _ptr(out), _stream(stream)))
        return out

    def solve(self, b, x=None, rtol=1e-10, maxit=1000, precond=None, check_every=1, use_graph=1,
              stream=None, allow_noconv=False, profile=False, outer=EB_F64):
        """pcg_solve; outer = EB_DF64 keeps the outer iteration in double-float."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        o = pcg_opts(EB_PC_AMG if (precond is None and self.num_levels > 0) else
                     (EB_PC_JACOBI if precond is None else precond), check_every, use_graph, int(profile), int(outer))
        st = pcg_stats()
        _check(load().pcg_solve(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit), C.byref(o), C.byref(st),
                                _stream(stream)), allow=(EB_ERR_NO_CONVERGENCE,) if allow_noconv else ())
        return x, st

    def set_outer(self, prec):
        """amg_set_outer_prec: the outer precision of heat_step, wave_theta_step and option-less solves."""
        _check(load().amg_set_outer_prec(self._h, int(prec)))

    def autotune(self, reps=20, stream=None) -> TuneResult:
        """Times V-cycles for every candidate tile shape of the grid and keeps the fastest."""
        t = eb_tune_t()
        _check(load().amg_autotune(self._h, int(reps), C.byref(t), _stream(stream)))
        self.eb._refresh_info()
        return _tune_result(t)

    def tune_csr(self, reps=20, stream=None):
        """Times V-cycles with 1, 2, 4, 8 entries per lane in the CSR kernels; keeps the fastest.
        Returns (chosen entries per lane, {entries per lane: microseconds})."""
        us = (C.c_double * 4)()
        best = C.c_int()
        _check(load().amg_tune_csr(self._h, int(reps), C.cast(us, C.c_void_p), C.byref(best), _stream(stream)))
        return best.value, {e: us[i] for i, e in enumerate((1, 2, 4, 8))}

    def set_csr_epl(self, epl):
        """Entries per lane of the CSR row groups (1, 2, 4 or 8), e.g. a cached tuning result."""
        _check(load().amg_set_csr_epl(self._h, int(epl)))

    def time_smoother_step(self, level, launches=50, clear_bytes=0, stream=None):
        """Microseconds per launch of level `level`'s Chebyshev smoothing step
        timed on its own (amg_time_kernel); clear_bytes > 0 clears L2 before
        every launch.  Overwrites the level's smoother vectors."""
        us = C.c_double()
        _check(load().amg_time_kernel(self._h, EB_TK_SMOOTH_STEP, int(level), int(launches), int(clear_bytes),
                                      C.byref(us), _stream(stream)))
        return us.value

    def minres(self, b, sigma, x=None, rtol=1e-10, maxit=5000, precond=EB_PC_AMG, stream=None, allow_noconv=False):
        """(sigma I + A) x = b by preconditioned MINRES (sigma = -omega^2: Helmholtz)."""
        import torch
        if x is None:
            x = torch.zeros_like(b)
        st = pcg_stats()
        _check(load().minres_solve(self._h, float(sigma), int(precond), _ptr(b), _ptr(x), float(rtol), int(maxit),
                                   C.byref(st), _stream(stream)),
               allow=(EB_ERR_NO_CONVERGENCE,) if allow_noconv else ())
        return x, st

    def wave_theta_step(self, u_prev, u_cur, dt, theta, nsteps, rtol=1e-10, maxit=1000, stream=None):
        """nsteps implicit theta-scheme wave steps (the hierarchy's shift must be
        1 / (theta dt^2)); (u_prev, u_cur) advanced in place."""
        st = pcg_stats()
        _check(load().wave_theta_step(self._h, float(dt), float(theta), _ptr(u_prev), _ptr(u_cur), int(nsteps),
                                      float(rtol), int(maxit), C.byref(st), _stream(stream)))
        return st

    def heat_step(self, u, b1, dt, theta=1.0, b0=None, rtol=1e-10, maxit=1000, stream=None):
        st = pcg_stats()
        _check(load().heat_step(self._h, float(dt), float(theta), _ptr(b1), _ptr(b0), _ptr(u), float(rtol),
                                int(maxit), C.byref(st), _stream(stream)))
        return st


class batch_info_t(C.Structure):
    _fields_ = [("count", C.c_int), ("stride", C.c_int64), ("num_nodes", C.c_int64), ("num_cp", C.c_int64),
                ("num_cut", C.c_int64), ("num_tiles", C.c_int64)]


class _Borrowed(EB):
    """EB view of a geometry owned by a batch (never destroyed here).  It keeps
    the batch alive, so that handles built on it (an AMG hierarchy reads its
    geometry when destroyed) never outlive the geometry."""

    def __init__(self, handle, grid, owner):
        self._owner = owner
        self._h = C.c_void_p(handle)
        self.grid = grid
        self.dim = grid.dim
        inf = eb_info_t()
        _check(load().eb_info(self._h, C.byref(inf)))
        self.info = Info(inf.num_nodes, inf.num_cp, inf.num_bp, inf.num_cut, inf.num_far, inf.num_tiles,
                         tuple(inf.tile), inf.max_delta_over_h, inf.min_abs_psi, inf.min_dominance_margin,
                         inf.num_rbf, inf.num_rbf_rotated)

    def close(self):
        self._h = C.c_void_p()


class Batch:
    """Handle of batch_build: many 2D geometries in one batch layout."""

    def __init__(self, grids, levelsets, stream=None):
        lib = load()
        n = len(grids)
        G = (eb_grid * n)(*[make_grid(g) for g in grids])
        psis = [sampled_psi_on_device(l) if int(l.kind) == EB_LS_SAMPLED else None for l in levelsets]
        L = (eb_levelset * n)(*[make_levelset(l, p) for l, p in zip(levelsets, psis)])
        self._h = C.c_void_p()
        self.grids = list(grids)
        _check(lib.batch_build(C.cast(G, C.c_void_p), C.cast(L, C.c_void_p), n, C.byref(self._h), _stream(stream)))
        inf = batch_info_t()
        _check(lib.batch_info(self._h, C.cast(C.byref(inf), C.c_void_p)))
        self.count, self.stride, self.num_nodes = inf.count, inf.stride, inf.num_nodes
        self.num_cp, self.num_cut, self.num_tiles = inf.num_cp, inf.num_cut, inf.num_tiles
        no, co, po = (C.c_int64 * (n + 1))(), (C.c_int64 * (n + 1))(), (C.c_int64 * (n + 1))()
        _check(lib.batch_offsets(self._h, C.cast(no, C.c_void_p), C.cast(co, C.c_void_p), C.cast(po, C.c_void_p)))
        self.node_off, self.cut_off, self.cp_off = list(no), list(co), list(po)

    def close(self):
        if self._h:
            load().batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def geometry(self, g):
        h = load().batch_geometry(self._h, g)
        if not h:
            raise EBError(EB_ERR_INVALID, load().eb_last_error().decode())
        return _Borrowed(h, self.grids[g], self)

    def view(self, v, g):
        """Geometry g's (n1, n0) grid inside a batch-layout vector."""
        gr = self.grids[g]
        a = v[self.node_off[g]:self.node_off[g + 1]].view(gr.n[1], self.stride)
        return a[:, :gr.n[0]]

    def zeros(self, dtype=None):
        import torch
        return torch.zeros(self.num_nodes, dtype=dtype or torch.float64, device="cuda")

    def rhs(self, f_all, ug_all, out=None, stream=None):
        if out is None:
            out = self.zeros()
        _check(load().batch_rhs(self._h, _ptr(f_all), _ptr(ug_all), _ptr(out), _stream(stream)))
        return out

    def heat_setup(self, dt, theta=1.0, max_levels=25, coarse_max=1024, strength=0.02, cheb_degree=2,
                   vcycle_prec=EB_F64, stream=None):
        d = (C.c_double * self.count)(*[float(v) for v in dt])
        o = amg_opts(max_levels, coarse_max, strength, cheb_degree, vcycle_prec, EB_AMG_SA, 1)
        _check(load().batch_heat_setup(self._h, C.cast(d, C.c_void_p), float(theta), C.byref(o), _stream(stream)))

    def heat_step(self, u_all, b1_all, b0_all=None, rtol=1e-10, maxit=500, stream=None, allow_noconv=False):
        st = (pcg_stats * self.count)()
        _check(load().batch_heat_step(self._h, _ptr(b1_all), _ptr(b0_all), _ptr(u_all), float(rtol), int(maxit),
                                      C.cast(st, C.c_void_p), _stream(stream)),
               allow=(EB_ERR_NO_CONVERGENCE,) if allow_noconv else ())
        return list(st)

    def set_profile(self, on: bool):
        _check(load().batch_set_profile(self._h, int(bool(on))))

    def set_outer(self, prec):
        """batch_set_outer_prec: EB_DF64 runs the batched PCG in double-float, EB_F64 in FP64."""
        _check(load().batch_set_outer_prec(self._h, int(prec)))

    def set_level0_tma(self, on: bool):
        """batch_set_level0_tma: level-0 smoothing steps fed by tensor copies (default) or per-thread loads."""
        _check(load().batch_set_level0_tma(self._h, int(bool(on))))

    def weighted_sum(self, w_all, u_all, stream=None):
        """Per-geometry sum of w u (batch_weighted_sum): a device tensor of count doubles."""
        import torch
        out = torch.empty(self.count, dtype=torch.float64, device="cuda")
        _check(load().batch_weighted_sum(self._h, _ptr(w_all), _ptr(u_all), _ptr(out), _stream(stream)))
        return out

    def autotune(self, reps=10, stream=None) -> TuneResult:
        """Times batch V-cycles for every candidate 2D tile shape and keeps the fastest."""
        t = eb_tune_t()
        _check(load().batch_autotune(self._h, int(reps), C.byref(t), _stream(stream)))
        return _tune_result(t)


class Net:
    """Handle of nn_create: the learned preconditioner stage (a 6-layer BF16
    convolutional network on the 2D grid), its training and its use in the
    flexible PCG."""

    def __init__(self, params=None, stream=None):
        lib = load()
        self._h = C.c_void_p()
        _check(lib.nn_create(C.byref(self._h), _stream(stream)))
        self.num_params = lib.nn_num_params()
        if params is not None:
            self.set_params(params, stream)

    def close(self):
        if self._h:
            load().nn_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_params(self, params, stream=None):
        """params: numpy-convertible vector of num_params floats (host)."""
        import numpy as np
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if a.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {a.size}")
        _check(load().nn_set_params(self._h, a.ctypes.data_as(C.c_void_p), _stream(stream)))

    def params(self, stream=None):
        import numpy as np
        p = np.empty(self.num_params, dtype=np.float32)
        g = np.empty(self.num_params, dtype=np.float32)
        _check(load().nn_get_params(self._h, p.ctypes.data_as(C.c_void_p), g.ctypes.data_as(C.c_void_p),
                                    _stream(stream)))
        return p, g

    def forward(self, inp, out=None, stream=None):
        """inp: float32 [images, height, width, 2] (s_hat, m); returns [images, height, width]."""
        import torch
        if inp.dim() == 3:
            inp = inp.unsqueeze(0)
        nimg, h, w, two = inp.shape
        if two != 2 or inp.dtype != torch.float32:
            raise ValueError("expected a float32 [images, height, width, 2] tensor")
        if out is None:
            out = torch.empty((nimg, h, w), dtype=torch.float32, device="cuda")
        _check(load().nn_forward(self._h, w, h, nimg, _ptr(inp), _ptr(out), _stream(stream)))
        return out

    def set_profile(self, on: bool):
        _check(load().nn_set_profile(self._h, int(bool(on))))

    def set_fused(self, on: bool):
        """nn_set_fused: the one-launch forward (default) or the layer-by-layer launches."""
        _check(load().nn_set_fused(self._h, int(bool(on))))

    def profile(self, stream=None):
        """(summed ms, launches) of the timed launches since the last call: the
        32 -> 32 convolutions of a layer-by-layer forward, the one fused launch
        of a fused forward."""
        ms = C.c_double()
        n = C.c_int()
        _check(load().nn_profile(self._h, C.byref(ms), C.byref(n), _stream(stream)))
        return ms.value, n.value

    def status(self, stream=None):
        """Raises if a tensor-core wait gave up since the last check."""
        _check(load().nn_status(self._h, _stream(stream)))

    def backward(self, inp, dout, stream=None):
        """Gradient of sum(dout * N(inp)) in the parameters (read with params())."""
        if inp.dim() == 3:
            inp = inp.unsqueeze(0)
        nimg, h, w, _ = inp.shape
        _check(load().nn_backward(self._h, w, h, nimg, _ptr(inp), _ptr(dout), _stream(stream)))

    def train_step(self, s_hat, c, geo_of, code, diag, pick, lr, loss=None, stream=None):
        """One Adam step over the pairs pick[] of a pair store (nn_train_step).
        s_hat [n_pairs, height, width] float32, c [n_pairs] float64, geo_of
        [n_pairs] int32, code [n_geo, height, width] uint8, diag [n_geo,
        height, width] float32, pick [batch] int32, all on the device; loss:
        optional float32 [batch + 1] device tensor."""
        batch = pick.numel()
        h, w = s_hat.shape[1], s_hat.shape[2]
        _check(load().nn_train_step(self._h, w, h, batch, _ptr(s_hat), _ptr(c), _ptr(geo_of), _ptr(code),
                                    _ptr(diag), _ptr(pick), float(lr), _ptr(loss), _stream(stream)))
        return loss


def nn_geometry(eb: EB, code_out, diag_out, stream=None):
    _check(load().nn_geometry(eb.handle, _ptr(code_out), _ptr(diag_out), _stream(stream)))


def nn_pairs(amg: AMG, b, x_star, count, s_out, c_out, e_out=None, stream=None):
    """The first count training pairs of the V-cycle iteration (nn_pairs)."""
    _check(load().nn_pairs(amg._h, _ptr(b), _ptr(x_star), int(count), _ptr(s_out), _ptr(c_out), _ptr(e_out),
                           _stream(stream)))


def precondition_nn(amg: AMG, net: Net, r, out=None, mode=EB_NN_PLAIN, stream=None):
    """z = V(r) followed by the learned stage (nn_precondition)."""
    import torch
    if out is None:
        out = torch.zeros_like(r)
    _check(load().nn_precondition(amg._h, net.handle, int(mode), _ptr(r), _ptr(out), _stream(stream)))
    return out


def solve_nn(amg: AMG, net: Net, b, x=None, rtol=1e-10, maxit=1000, mode=EB_NN_PLAIN, check_every=1, use_graph=1,
             stream=None, allow_noconv=False, profile=0):
    """Flexible PCG with the V-cycle followed by the learned stage (pcg_solve_nn);
    profile 2 times the stage's 32 -> 32 convolution launches."""
    import torch
    if x is None:
        x = torch.zeros_like(b)
    o = pcg_opts(EB_PC_AMG_NN, check_every, use_graph, int(profile))
    st = pcg_stats()
    _check(load().pcg_solve_nn(amg._h, net.handle, int(mode), _ptr(b), _ptr(x), float(rtol), int(maxit), C.byref(o),
                               C.byref(st), _stream(stream)), allow=(EB_ERR_NO_CONVERGENCE,) if allow_noconv else ())
    return x, st

