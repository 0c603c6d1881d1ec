"""Thin ctypes binding of the C ABI in ``include/pp_cweno.h``.

Argument marshalling only: every step of the scheme runs in the CUDA library
``_build/libppcweno.so``.  Device arrays are passed as torch CUDA tensors
(their ``data_ptr()``), host arrays as numpy float64 arrays.  There is no CPU
fallback: if the library has not been built, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PP_OK, PP_ERR_ARG, PP_ERR_STATE, PP_ERR_NONPHYSICAL, PP_ERR_STEPS, PP_ERR_TIMEOUT, \
    PP_ERR_CUDA, PP_ERR_UNSUPPORTED = range(8)
PREC_FP64, PREC_MIXED = 0, 1
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE = 0, 1, 2
FLUX_HLLC, FLUX_LLF = 0, 1
RECON_COMPONENT, RECON_CHARACTERISTIC = 0, 1


class Config(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64),
        ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
        ("gamma", C.c_double), ("cfl", C.c_double), ("bc", C.c_int * 4),
        ("precision", C.c_int), ("gl_weight", C.c_double), ("eps_weno", C.c_double),
        ("eps_pos", C.c_double), ("cfl_positivity_cap", C.c_int), ("limiter", C.c_int),
        ("flux", C.c_int), ("recon", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64), ("stages", C.c_int64), ("theta1_active", C.c_int64),
        ("theta2_active", C.c_int64), ("violations", C.c_int64), ("first_bad_cell", C.c_int64),
        ("t", C.c_double), ("last_dt", C.c_double), ("max_rate", C.c_double),
        ("min_rho", C.c_double), ("rejected", C.c_int64),
    ]


# every entry point declared in include/pp_cweno.h
EXPORTS = [
    "pp_cweno_config_default", "pp_cweno_create", "pp_cweno_create_batch", "pp_cweno_set_state",
    "pp_cweno_get_state", "pp_cweno_step", "pp_cweno_advance", "pp_cweno_enqueue_steps",
    "pp_cweno_operator", "pp_cweno_stats", "pp_cweno_problem_stats", "pp_cweno_num_problems",
    "pp_cweno_problem_cells",
    "pp_cweno_rows_per_chunk",
    "pp_cweno_launches_per_step", "pp_cweno_profile_step", "pp_cweno_fma_peak",
    "pp_cweno_operator_noalloc", "pp_cweno_destroy", "pp_cweno_strerror",
]

_lib = None


class PPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


def lib(build_if_missing: bool = False):
    """Load libppcweno.so (raises if it is missing and build_if_missing is False)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libppcweno.so not built ({path}); run __graft_entry__.build()")
        _build.build()
    L = C.CDLL(path)
    vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
    dp = C.POINTER(C.c_double)
    cfgp = C.POINTER(Config)
    L.pp_cweno_config_default.argtypes = [cfgp]
    L.pp_cweno_create.argtypes = [cfgp, vp, C.POINTER(vp)]
    L.pp_cweno_create_batch.argtypes = [cfgp, C.c_int64, vp, C.POINTER(vp)]
    L.pp_cweno_set_state.argtypes = [vp, vp, C.c_int, C.c_double]
    L.pp_cweno_get_state.argtypes = [vp, vp, C.c_int, dp, i64p]
    L.pp_cweno_step.argtypes = [vp, C.c_double, dp]
    L.pp_cweno_advance.argtypes = [vp, C.c_double, C.c_int64, i64p]
    L.pp_cweno_enqueue_steps.argtypes = [vp, C.c_int64]
    L.pp_cweno_operator.argtypes = [vp, vp, vp, C.c_double]
    L.pp_cweno_stats.argtypes = [vp, C.POINTER(Stats)]
    L.pp_cweno_problem_stats.argtypes = [vp, C.c_int64, C.POINTER(Stats)]
    L.pp_cweno_num_problems.argtypes = [vp, i64p]
    L.pp_cweno_problem_cells.argtypes = [vp, C.c_int64, i64p]
    L.pp_cweno_launches_per_step.argtypes = [vp, i64p]
    L.pp_cweno_rows_per_chunk.argtypes = [vp, C.POINTER(C.c_int)]
    L.pp_cweno_profile_step.argtypes = [vp, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]
    L.pp_cweno_fma_peak.argtypes = [C.c_int, dp]
    L.pp_cweno_operator_noalloc.argtypes = [cfgp, vp, vp, C.c_double, vp]
    L.pp_cweno_destroy.argtypes = [vp]
    L.pp_cweno_strerror.argtypes = [C.c_int]
    L.pp_cweno_strerror.restype = C.c_char_p
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().pp_cweno_strerror(code).decode()
    except Exception:  # library absent: still give a message
        return f"error {code}"


def _check(rc: int, where: str, ok=(PP_OK,)):
    if rc not in ok:
        raise PPError(rc, where)
    return rc


def make_config(ndim=1, nx=200, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, cfl=0.5,
                bc=(0, 0, 0, 0), precision=PREC_FP64, gl_weight=1.0 / 12.0, eps_weno=1e-13,
                eps_pos=1e-13, cfl_positivity_cap=False, limiter=True, flux=FLUX_HLLC,
                recon=RECON_COMPONENT) -> Config:
    c = Config()
    lib().pp_cweno_config_default(C.byref(c))
    c.ndim, c.nx, c.ny = ndim, nx, (ny if ndim == 2 else 1)
    c.x0, c.x1, c.y0, c.y1 = x0, x1, y0, y1
    c.gamma, c.cfl = gamma, cfl
    for k in range(4):
        c.bc[k] = int(bc[k]) if k < len(bc) else 0
    c.precision = int(precision)
    c.gl_weight, c.eps_weno, c.eps_pos = gl_weight, eps_weno, eps_pos
    c.cfl_positivity_cap, c.limiter = int(cfl_positivity_cap), int(limiter)
    c.flux = int(flux)
    c.recon = int(recon)
    return c


def config_from_problem(p, precision=PREC_FP64, **kw) -> Config:
    """Config of a :class:`workloads.Problem`."""
    bc = tuple(p.bc) + (0,) * (4 - len(p.bc))
    return make_config(p.ndim, p.nx, p.ny, p.x0, p.x1, p.y0, p.y1, p.gamma, p.cfl, bc,
                       precision, **kw)


def fma_peak(fp64: bool) -> float:
    """measured FMA throughput of the CUDA cores, GFLOP/s"""
    g = C.c_double()
    _check(lib().pp_cweno_fma_peak(int(fp64), C.byref(g)), "fma_peak")
    return g.value


def operator_noalloc(cfg, U_dev, L_dev, eps: float = 0.0, stream=None) -> None:
    """L = L(U) of one FP64 problem using the library's fixed device scratch
    (no allocation); asynchronous on the given stream."""
    pu, du = _ptr(U_dev)
    pl, dl = _ptr(L_dev)
    assert du and dl, "operator_noalloc() takes device tensors"
    st = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
    _check(lib().pp_cweno_operator_noalloc(C.byref(cfg), pu, pl, eps, st), "operator_noalloc")


def _ptr(a):
    """(pointer, on_device) of a torch CUDA tensor or a numpy float64 array."""
    if hasattr(a, "data_ptr"):
        assert a.dtype.__str__() == "torch.float64" and a.is_contiguous()
        return C.c_void_p(a.data_ptr()), int(a.is_cuda)
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data), 0


class Solver:
    """One handle of the C ABI (single problem or batch)."""

    def __init__(self, cfg, stream=None, batch: list | None = None):
        L = lib()
        h = C.c_void_p()
        st = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))
        if batch is None:
            _check(L.pp_cweno_create(C.byref(cfg), st, C.byref(h)), "pp_cweno_create")
            self.nv = 4 if cfg.ndim == 2 else 3
        else:
            arr = (Config * len(batch))(*batch)
            _check(L.pp_cweno_create_batch(arr, len(batch), st, C.byref(h)), "pp_cweno_create_batch")
            self.nv = 4 if batch[0].ndim == 2 else 3
        self.h = h
        n = C.c_int64()
        _check(L.pp_cweno_num_problems(h, C.byref(n)), "num_problems")
        self.nprob = n.value
        cells = []
        for k in range(self.nprob):
            _check(L.pp_cweno_problem_cells(h, k, C.byref(n)), "problem_cells")
            cells.append(n.value)
        self.cells = cells
        self.size = self.nv * sum(cells)

    def close(self):
        if self.h:
            lib().pp_cweno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, U, t0: float = 0.0, check=True):
        p, dev = _ptr(U)
        rc = lib().pp_cweno_set_state(self.h, p, dev, t0)
        return _check(rc, "set_state") if check else rc

    def get_state(self, out=None):
        if out is None:
            out = np.zeros(self.size)
        p, dev = _ptr(out)
        t = C.c_double()
        s = C.c_int64()
        _check(lib().pp_cweno_get_state(self.h, p, dev, C.byref(t), C.byref(s)), "get_state")
        return out, t.value, s.value

    def step(self, dt_max: float = float("inf")):
        dt = C.c_double()
        rc = lib().pp_cweno_step(self.h, dt_max if dt_max < float("inf") else 1e300, C.byref(dt))
        _check(rc, "step")
        return dt.value

    def advance(self, t_final: float, max_steps: int = 2**62, check=True):
        n = C.c_int64()
        rc = lib().pp_cweno_advance(self.h, t_final, max_steps, C.byref(n))
        if check:
            _check(rc, "advance")
        return n.value, rc

    def enqueue_steps(self, nsteps: int):
        _check(lib().pp_cweno_enqueue_steps(self.h, nsteps), "enqueue_steps")

    def operator(self, U_dev, L_dev, eps: float = 0.0):
        pu, du = _ptr(U_dev)
        pl, dl = _ptr(L_dev)
        assert du and dl, "operator() takes device tensors"
        _check(lib().pp_cweno_operator(self.h, pu, pl, eps), "operator")

    def stats(self) -> Stats:
        s = Stats()
        _check(lib().pp_cweno_stats(self.h, C.byref(s)), "stats")
        return s

    def problem_stats(self, k: int) -> Stats:
        """steps, time, limiter counts and violations of problem k of a batch"""
        s = Stats()
        _check(lib().pp_cweno_problem_stats(self.h, k, C.byref(s)), "problem_stats")
        return s

    def profile_step(self) -> list[float]:
        """per-kernel durations (ms) of one step, launch by launch"""
        ms = (C.c_float * 32)()
        nk = C.c_int()
        _check(lib().pp_cweno_profile_step(self.h, ms, 32, C.byref(nk)), "profile_step")
        return [ms[i] for i in range(nk.value)]

    def rows_per_chunk(self) -> int:
        m = C.c_int()
        _check(lib().pp_cweno_rows_per_chunk(self.h, C.byref(m)), "rows_per_chunk")
        return m.value

    def launches_per_step(self) -> int:
        n = C.c_int64()
        _check(lib().pp_cweno_launches_per_step(self.h, C.byref(n)), "launches_per_step")
        return n.value
