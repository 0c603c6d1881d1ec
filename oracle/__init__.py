"""FP64 CPU oracle of the positivity-preserving FV compact-WENO scheme.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never loads it, and the two share no code.

The arithmetic lives in plain C (``pp_oracle.c`` for the scheme,
``riemann_exact.c`` for the exact Riemann solver used as a test reference);
this module compiles it with gcc and wraps it with ctypes.  Arrays are numpy
float64 in the structure-of-arrays layout ``U[v][j][i]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["pp_oracle.c", "riemann_exact.c"]
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE = 0, 1, 2


class Grid(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("nx", C.c_long), ("ny", C.c_long),
        ("dx", C.c_double), ("dy", C.c_double), ("gamma", C.c_double),
        ("bc", C.c_int * 4), ("gl_weight", C.c_double), ("eps_weno", C.c_double),
        ("eps_pos", C.c_double), ("limiter", C.c_int), ("linear_weights", C.c_int),
        ("flux", C.c_int), ("recon", C.c_int), ("face_cfl", C.c_double),
    ]


class Counters(C.Structure):
    _fields_ = [("theta1_active", C.c_long), ("theta2_active", C.c_long),
                ("bad_cells", C.c_long), ("face_rate", C.c_double), ("rejected", C.c_long)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, FP64,
    no FMA contraction so that x86 and Arm hosts round identically)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "pp_oracle.h")
    newest = max(os.path.getmtime(p) for p in srcs + [hdr])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fopenmp", *srcs, "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            gp = C.POINTER(Grid)
            cp = C.POINTER(Counters)
            L.orc_smoothness.argtypes = [dp, dp]
            L.orc_wenoz_weights.argtypes = [dp, dp, C.c_double, dp]
            L.orc_thomas.argtypes = [C.c_long, dp, dp, dp, dp, dp, C.c_int]
            L.orc_cyclic.argtypes = [C.c_long, dp, dp, dp, dp, dp, C.c_int]
            L.orc_recon_scalar.argtypes = [C.c_long, dp, C.c_int, C.c_double, C.c_int, dp, dp]
            L.orc_hllc.argtypes = [C.c_int, C.c_double, dp, dp, dp]
            L.orc_roe_eigen.argtypes = [C.c_int, C.c_double, dp, dp, dp, dp]
            L.orc_block_thomas.argtypes = [C.c_long, C.c_int, dp, dp, dp, dp, C.c_int, dp, C.c_int]
            L.orc_block_cyclic.argtypes = [C.c_long, C.c_int, dp, dp, dp, dp, dp, C.c_int]
            L.orc_recon_char.argtypes = [C.c_int, C.c_long, dp, C.c_int, C.c_double, C.c_double,
                                         C.c_int, dp, dp]
            L.orc_llf.argtypes = [C.c_int, C.c_double, dp, dp, dp]
            L.orc_flux.argtypes = [C.c_int, C.c_double, dp, dp]
            L.orc_hllc_batch.argtypes = [C.c_int, C.c_double, C.c_long, dp, dp, dp]
            L.orc_limit_cell.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, dp, dp, dp]
            L.orc_operator.argtypes = [gp, dp, dp, C.c_double, cp]
            lp = C.POINTER(C.c_long)
            L.orc_operator_lines.argtypes = [gp, dp, C.c_double, C.c_long, lp, C.c_long, lp, dp, dp]
            L.orc_max_rate.argtypes = [gp, dp]
            L.orc_max_rate.restype = C.c_double
            L.orc_min_rho.argtypes = [gp, dp]
            L.orc_min_rho.restype = C.c_double
            L.orc_rk3_step.argtypes = [gp, dp, C.c_double, cp]
            L.orc_advance.argtypes = [gp, dp, C.c_double, C.c_double, C.c_double, C.c_long,
                                      dp, C.POINTER(C.c_long), dp, cp]
            L.orc_riemann_star.argtypes = [C.c_double, dp, dp, dp, dp, C.POINTER(C.c_int),
                                           C.POINTER(C.c_int)]
            L.orc_riemann_star_bisect.argtypes = [C.c_double, dp, dp]
            L.orc_riemann_star_bisect.restype = C.c_double
            L.orc_riemann_sample.argtypes = [C.c_double, dp, dp, C.c_double, dp]
            L.orc_riemann_cell_averages.argtypes = [C.c_double, dp, dp, C.c_double, C.c_double,
                                                    C.c_long, C.c_double, C.c_double, C.c_int, dp]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def make_grid(ndim: int, nx: int, ny: int = 1, dx: float = 1.0, dy: float = 1.0,
              gamma: float = 1.4, bc=(0, 0, 0, 0), gl_weight: float = 1.0 / 12.0,
              eps_weno: float = 1e-13, eps_pos: float = 1e-13, limiter: bool = True,
              linear_weights: bool = False, flux: int = 0, recon: int = 0,
              face_cfl: float = 0.0) -> Grid:
    """face_cfl > 0: check eq. (CFL-CD) on the limited face values of every
    stage (bound omega_hat_1) and redo a failing step with a smaller dt."""
    g = Grid()
    g.ndim, g.nx, g.ny = ndim, nx, (ny if ndim == 2 else 1)
    g.dx, g.dy, g.gamma = dx, dy, gamma
    for k in range(4):
        g.bc[k] = int(bc[k])
    g.gl_weight, g.eps_weno, g.eps_pos = gl_weight, eps_weno, eps_pos
    g.limiter, g.linear_weights = int(limiter), int(linear_weights)
    g.flux = int(flux)
    g.recon = int(recon)
    g.face_cfl = float(face_cfl)
    return g


# ---------------------------------------------------------------- scalar pieces
def smoothness(u5) -> np.ndarray:
    u5, b = _f64(u5), np.zeros(3)
    lib().orc_smoothness(_p(u5), _p(b))
    return b


def wenoz_weights(beta3, c3=(0.2, 0.5, 0.3), eps=1e-13) -> np.ndarray:
    beta3, c3, w = _f64(beta3), _f64(c3), np.zeros(3)
    lib().orc_wenoz_weights(_p(beta3), _p(c3), eps, _p(w))
    return w


def thomas(sub, diag, sup, rhs, reverse=False) -> np.ndarray:
    sub, diag, sup, rhs = map(_f64, (sub, diag, sup, rhs))
    x = np.zeros_like(rhs)
    rc = lib().orc_thomas(len(rhs), _p(sub), _p(diag), _p(sup), _p(rhs), _p(x), int(reverse))
    if rc:
        raise ArithmeticError("zero pivot")
    return x


def cyclic(sub, diag, sup, rhs, reverse=False) -> np.ndarray:
    sub, diag, sup, rhs = map(_f64, (sub, diag, sup, rhs))
    x = np.zeros_like(rhs)
    rc = lib().orc_cyclic(len(rhs), _p(sub), _p(diag), _p(sup), _p(rhs), _p(x), int(reverse))
    if rc:
        raise ArithmeticError("singular cyclic system")
    return x


def recon_scalar(ext, periodic: bool, eps_weno=1e-13, linear=False):
    """ext: n+4 cell averages (two ghosts per side). Returns (u^-_{j+1/2}, u^+_{j-1/2})."""
    ext = _f64(ext)
    n = len(ext) - 4
    um, up = np.zeros(n), np.zeros(n)
    rc = lib().orc_recon_scalar(n, _p(ext), int(periodic), eps_weno, int(linear), _p(um), _p(up))
    if rc:
        raise ArithmeticError("reconstruction failed")
    return um, up


def roe_eigen(Ua, Ub, gamma=1.4):
    """(L, R): left / right eigenvector matrices at the Roe average, Sec. 2.3"""
    Ua, Ub = _f64(Ua), _f64(Ub)
    nv = len(Ua)
    Lm, Rm = np.zeros((nv, nv)), np.zeros((nv, nv))
    lib().orc_roe_eigen(nv, gamma, _p(Ua), _p(Ub), _p(Lm), _p(Rm))
    return Lm, Rm


def block_thomas(A, B, C_, r, reverse=False) -> np.ndarray:
    """A, B, C_: [n, m, m]; r: [n, m] or [n, m, ncol]"""
    A, B, C_, r = map(_f64, (A, B, C_, r))
    n, m = B.shape[0], B.shape[1]
    ncol = 1 if r.ndim == 2 else r.shape[2]
    x = np.zeros_like(r)
    rc = lib().orc_block_thomas(n, m, _p(A), _p(B), _p(C_), _p(r), ncol, _p(x), int(reverse))
    if rc:
        raise ArithmeticError("singular pivot block")
    return x


def block_cyclic(A, B, C_, r, reverse=False) -> np.ndarray:
    A, B, C_, r = map(_f64, (A, B, C_, r))
    n, m = B.shape[0], B.shape[1]
    x = np.zeros_like(r)
    rc = lib().orc_block_cyclic(n, m, _p(A), _p(B), _p(C_), _p(r), _p(x), int(reverse))
    if rc:
        raise ArithmeticError("singular cyclic block system")
    return x


def recon_char(ext, periodic: bool, gamma=1.4, eps_weno=1e-13, linear=False):
    """ext: [nv, n+4] conserved averages with two ghosts per side.  Returns
    (U^-_{j+1/2}, U^+_{j-1/2}) as [nv, n] arrays."""
    ext = _f64(ext)
    nv, n = ext.shape[0], ext.shape[1] - 4
    um, up = np.zeros((nv, n)), np.zeros((nv, n))
    rc = lib().orc_recon_char(nv, n, _p(ext), int(periodic), gamma, eps_weno, int(linear),
                              _p(um), _p(up))
    if rc:
        raise ArithmeticError("reconstruction failed")
    return um, up


def hllc(Ul, Ur, gamma=1.4) -> np.ndarray:
    Ul, Ur = _f64(Ul), _f64(Ur)
    F = np.zeros(len(Ul))
    lib().orc_hllc(len(Ul), gamma, _p(Ul), _p(Ur), _p(F))
    return F


def llf(Ul, Ur, gamma=1.4) -> np.ndarray:
    Ul, Ur = _f64(Ul), _f64(Ur)
    F = np.zeros(len(Ul))
    lib().orc_llf(len(Ul), gamma, _p(Ul), _p(Ur), _p(F))
    return F


def hllc_batch(Ul, Ur, gamma=1.4) -> np.ndarray:
    """Ul, Ur: [n, nv] face states."""
    Ul, Ur = _f64(Ul), _f64(Ur)
    F = np.zeros_like(Ul)
    lib().orc_hllc_batch(Ul.shape[1], gamma, Ul.shape[0], _p(Ul), _p(Ur), _p(F))
    return F


def flux(U, gamma=1.4) -> np.ndarray:
    U = _f64(U)
    F = np.zeros(len(U))
    lib().orc_flux(len(U), gamma, _p(U), _p(F))
    return F


def limit_cell(ubar, um, up, eps, gamma=1.4, wgl=1.0 / 12.0):
    ubar, um, up = _f64(ubar), _f64(um).copy(), _f64(up).copy()
    flags = lib().orc_limit_cell(len(ubar), gamma, wgl, eps, _p(ubar), _p(um), _p(up))
    return um, up, flags


# ---------------------------------------------------------------- whole grid
def operator(g: Grid, U: np.ndarray, eps: float | None = None):
    U = _f64(U)
    L = np.zeros_like(U)
    if eps is None:
        eps = min(g.eps_pos, float(lib().orc_min_rho(C.byref(g), _p(U))))
    cnt = Counters()
    rc = lib().orc_operator(C.byref(g), _p(U), _p(L), eps, C.byref(cnt))
    if rc:
        raise ArithmeticError("operator failed")
    return L, cnt


def operator_lines(g: Grid, U: np.ndarray, eps: float, rows, cols):
    """(Lx on rows [nr, nv, nx], Ly on cols [nc, nv, ny]) -- sampled operator."""
    U = _f64(U)
    nv = 4 if g.ndim == 2 else 3
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    Lx = np.zeros((len(rows), nv, g.nx))
    Ly = np.zeros((len(cols), nv, g.ny))
    lp = C.POINTER(C.c_long)
    rc = lib().orc_operator_lines(C.byref(g), _p(U), eps, len(rows), rows.ctypes.data_as(lp),
                                  len(cols), cols.ctypes.data_as(lp), _p(Lx), _p(Ly))
    if rc:
        raise ArithmeticError("operator_lines failed")
    return Lx, Ly


def min_rho(g: Grid, U: np.ndarray) -> float:
    return float(lib().orc_min_rho(C.byref(g), _p(_f64(U))))


def max_rate(g: Grid, U: np.ndarray) -> float:
    return float(lib().orc_max_rate(C.byref(g), _p(_f64(U))))


def rk3_step(g: Grid, U: np.ndarray, dt: float) -> np.ndarray:
    U = _f64(U).copy()
    cnt = Counters()
    rc = lib().orc_rk3_step(C.byref(g), _p(U), dt, C.byref(cnt))
    if rc:
        raise ArithmeticError("rk3 step failed")
    return U


def advance(g: Grid, U: np.ndarray, cfl: float, t_final: float, t0: float = 0.0,
            max_steps: int = 10**9):
    """Returns (U, t, steps, dt_last, counters, rc)."""
    U = _f64(U).copy()
    t = C.c_double(0.0)
    steps = C.c_long(0)
    dtl = C.c_double(0.0)
    cnt = Counters()
    rc = lib().orc_advance(C.byref(g), _p(U), cfl, t0, t_final, max_steps, C.byref(t),
                           C.byref(steps), C.byref(dtl), C.byref(cnt))
    return U, t.value, steps.value, dtl.value, cnt, rc


# ---------------------------------------------------------------- exact Riemann
def riemann_star(WL, WR, gamma=1.4):
    WL, WR = _f64(WL), _f64(WR)
    ps, us = C.c_double(), C.c_double()
    vac, it = C.c_int(), C.c_int()
    rc = lib().orc_riemann_star(gamma, _p(WL), _p(WR), C.byref(ps), C.byref(us),
                                C.byref(vac), C.byref(it))
    return ps.value, us.value, bool(vac.value), it.value, rc


def riemann_star_bisect(WL, WR, gamma=1.4) -> float:
    WL, WR = _f64(WL), _f64(WR)
    return float(lib().orc_riemann_star_bisect(gamma, _p(WL), _p(WR)))


def riemann_sample(WL, WR, xi, gamma=1.4) -> np.ndarray:
    WL, WR = _f64(WL), _f64(WR)
    W = np.zeros(3)
    lib().orc_riemann_sample(gamma, _p(WL), _p(WR), float(xi), _p(W))
    return W


def riemann_cell_averages(WL, WR, x0, x1, n, xd, t, gamma=1.4, nsub=4) -> np.ndarray:
    WL, WR = _f64(WL), _f64(WR)
    U = np.zeros(3 * n)
    lib().orc_riemann_cell_averages(gamma, _p(WL), _p(WR), x0, x1, n, xd, t, nsub, _p(U))
    return U.reshape(3, n)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))
