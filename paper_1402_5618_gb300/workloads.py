"""Seeded synthetic inputs shaped like the paper's test problems.

This module holds initial data only (cell averages of closed-form or
piecewise-constant states) and none of the scheme's arithmetic.  Both the
CUDA path and the CPU oracle are fed from it, so they see identical inputs.

Every random draw uses numpy's counter-based Philox generator keyed by the
master seed 14025618 plus a per-workload stream id.

State layout: float64 structure of arrays ``U[v][j][i]`` (x fastest);
1-D: (rho, m, E); 2-D: (rho, m_x, m_y, E).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 14025618

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE = 0, 1, 2


def rng(stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=MASTER_SEED + stream))


def prim_to_cons_1d(rho, u, p, gamma):
    rho, u, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, p))
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


def prim_to_cons_2d(rho, u, v, p, gamma):
    rho, u, v, p = (np.asarray(a, dtype=np.float64) for a in (rho, u, v, p))
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


@dataclass
class Problem:
    """One problem: grid, boundary conditions and initial cell averages."""
    ndim: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    gamma: float
    bc: tuple
    cfl: float
    t_final: float
    U0: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny if self.ndim == 2 else 1.0

    @property
    def ncell(self) -> int:
        return self.nx * (self.ny if self.ndim == 2 else 1)


# ------------------------------------------------------------------ 1-D problems
def density_wave(n: int, gamma: float = 1.4, cfl_coef: float = 0.6) -> Problem:
    """Advection of a density perturbation on [0, 2], periodic (paper Ex. 3.1):
    rho = 1 + 0.2 sin(pi x), u = 1, p = 1.  Exact cell averages (rho, m, E are
    affine in rho).  dt = cfl_coef * h^(5/3) / max(|u|+a), expressed as
    cfl = cfl_coef * h^(2/3) in dt = cfl * h / max(|u|+a)."""
    h = 2.0 / n
    xf = np.arange(n + 1, dtype=np.float64) * h
    rho = 1.0 + 0.2 * (np.cos(np.pi * xf[:-1]) - np.cos(np.pi * xf[1:])) / (np.pi * h)
    U = np.stack([rho, rho, np.full(n, 1.0 / (gamma - 1.0)) + 0.5 * rho])
    return Problem(1, n, 1, 0.0, 2.0, 0.0, 1.0, gamma, (BC_PERIODIC,) * 4,
                   cfl_coef * h ** (2.0 / 3.0), 2.0, np.ascontiguousarray(U),
                   name=f"density_wave_{n}")


def density_wave_exact(n: int, t: float) -> np.ndarray:
    """Exact cell averages of rho = 1 + 0.2 sin(pi (x - t)) on [0, 2]."""
    h = 2.0 / n
    xf = np.arange(n + 1, dtype=np.float64) * h - t
    return 1.0 + 0.2 * (np.cos(np.pi * xf[:-1]) - np.cos(np.pi * xf[1:])) / (np.pi * h)


def riemann_1d(n: int, WL, WR, x0: float = 0.0, x1: float = 1.0, xd: float = 0.5,
               gamma: float = 1.4, bc=(BC_TRANSMISSIVE, BC_TRANSMISSIVE), cfl: float = 0.5,
               t_final: float = 0.15, name: str = "riemann") -> Problem:
    """Piecewise-constant Riemann data; exact cell averages (the cell holding
    the jump is mixed in proportion)."""
    s = (xd - x0) / (x1 - x0) * n        # jump position in cell units
    frac_left = np.clip(s - np.arange(n, dtype=np.float64), 0.0, 1.0)
    UL = prim_to_cons_1d(*WL, gamma)[:, None]
    UR = prim_to_cons_1d(*WR, gamma)[:, None]
    U = frac_left[None, :] * UL + (1.0 - frac_left[None, :]) * UR
    return Problem(1, n, 1, x0, x1, 0.0, 1.0, gamma, (bc[0], bc[1], 0, 0), cfl, t_final,
                   np.ascontiguousarray(U), name=name,
                   meta={"WL": tuple(map(float, WL)), "WR": tuple(map(float, WR)), "xd": xd})


def riemann_batch(nprob: int = 4096, n_lo: int = 256, n_hi: int = 8192, stream: int = 2,
                  gamma: float = 1.4) -> list[Problem]:
    """Batch of independent 1-D Riemann problems on [0, 1], jump at 0.5,
    transmissive, CFL 0.5 to t = 0.15.  N log-uniform in [n_lo, n_hi];
    rho log-U[0.1, 10], u U[-3, 3], p log-U[0.01, 10] per side; 10% forced
    double rarefactions rho = 1, p = 0.4, u = -/+ s with s ~ U[2, 4]."""
    g = rng(stream)
    out = []
    for k in range(nprob):
        n = int(round(float(np.exp(g.uniform(np.log(n_lo), np.log(n_hi))))))
        rl, rr = np.exp(g.uniform(np.log(0.1), np.log(10.0), 2))
        ul, ur = g.uniform(-3.0, 3.0, 2)
        pl, pr = np.exp(g.uniform(np.log(0.01), np.log(10.0), 2))
        forced = g.uniform() < 0.1
        s = g.uniform(2.0, 4.0)
        if forced:
            rl = rr = 1.0
            pl = pr = 0.4
            ul, ur = -s, s
        out.append(riemann_1d(n, (rl, ul, pl), (rr, ur, pr), gamma=gamma,
                              name=f"riemann_{k}", cfl=0.5, t_final=0.15))
        out[-1].meta["forced_vacuum"] = bool(forced)
    return out


def opens_vacuum(q: Problem) -> bool:
    """True when the 1-D Riemann data of q generate a vacuum in the exact
    solution: u_R - u_L >= 2 (a_L + a_R) / (gamma - 1) between the end states."""
    g = q.gamma
    ends = []
    for c in (0, q.nx - 1):
        rho, m, E = q.U0[:, c]
        u = m / rho
        pr = (g - 1.0) * (E - 0.5 * rho * u * u)
        ends.append((u, np.sqrt(g * pr / rho)))
    (ul, al), (ur, ar) = ends
    return bool(ur - ul >= 2.0 * (al + ar) / (g - 1.0))


# paper Sec. 3 examples used as Riemann instances (domain, jump, t_final, BC)
PAPER_RIEMANN = {
    "lax": dict(WL=(0.445, 0.698, 3.528), WR=(0.5, 0.0, 0.571), x0=-5.0, x1=5.0, xd=0.0, t=1.4),
    # textbook Sod states; the printed states are garbled (equal p and u)
    "sod": dict(WL=(1.0, 0.0, 1.0), WR=(0.125, 0.0, 0.1), x0=-5.0, x1=5.0, xd=0.0, t=2.0),
    "123": dict(WL=(1.0, -2.0, 0.4), WR=(1.0, 2.0, 0.4), x0=0.0, x1=1.0, xd=0.5, t=0.1),
    "strong_shock": dict(WL=(1.0, 0.0, 1e10), WR=(0.125, 0.0, 0.1), x0=0.0, x1=1.0, xd=0.5,
                         t=2.5e-6),
    # the printed right state repeats the left one; the double rarefaction
    # described in the text needs u_R = +1
    "double_rarefaction": dict(WL=(7.0, -1.0, 0.2), WR=(7.0, 1.0, 0.2), x0=-1.0, x1=1.0,
                               xd=0.0, t=0.6),
}


def paper_riemann(name: str, n: int, gamma: float = 1.4, cfl: float = 1.0 / 12.0) -> Problem:
    d = PAPER_RIEMANN[name]
    return riemann_1d(n, d["WL"], d["WR"], d["x0"], d["x1"], d["xd"], gamma=gamma,
                      cfl=cfl, t_final=d["t"], name=name)


def leblanc(n: int, cfl: float = 1.0 / 12.0) -> Problem:
    """LeBlanc tube on [0, 9], gamma = 5/3, (rho, u, e) = (1, 0, 0.1) | (1e-3, 0, 1e-7)
    with the jump at x = 3, t = 6."""
    gamma = 5.0 / 3.0
    pl = (gamma - 1.0) * 1.0 * 0.1
    pr = (gamma - 1.0) * 1e-3 * 1e-7
    return riemann_1d(n, (1.0, 0.0, pl), (1e-3, 0.0, pr), 0.0, 9.0, 3.0, gamma=gamma, cfl=cfl,
                      t_final=6.0, name="leblanc")


def sedov_1d(h: float = 0.005, cfl: float = 1.0 / 12.0) -> Problem:
    """Planar Sedov blast on [0, 4]: p = 4e-13 except 2.56e8 in the centre cell."""
    gamma = 1.4
    n = int(round(4.0 / h))
    rho = np.ones(n)
    p = np.full(n, 4e-13)
    p[n // 2] = 2.56e8   # centre cell (n even: the cell just right of x = 2)
    U = prim_to_cons_1d(rho, np.zeros(n), p, gamma)
    return Problem(1, n, 1, 0.0, 4.0, 0.0, 1.0, gamma, (BC_TRANSMISSIVE,) * 2 + (0, 0), cfl,
                   0.001, np.ascontiguousarray(U), name="sedov_1d")


def blastwave_wc(n: int, cfl: float = 1.0 / 12.0) -> Problem:
    """Woodward-Colella interacting blast waves on [0, 1], reflective walls."""
    gamma = 1.4
    h = 1.0 / n
    xc = (np.arange(n) + 0.5) * h
    p = np.where(xc < 0.1, 1000.0, np.where(xc < 0.9, 0.01, 100.0))
    U = prim_to_cons_1d(np.ones(n), np.zeros(n), p, gamma)
    return Problem(1, n, 1, 0.0, 1.0, 0.0, 1.0, gamma, (BC_REFLECTIVE, BC_REFLECTIVE, 0, 0), cfl,
                   0.038, np.ascontiguousarray(U), name="blastwave_wc")


# ------------------------------------------------------------------ 2-D problems
def _gauss(nq: int):
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * x, 0.5 * w   # on [-1/2, 1/2], weights sum to 1


def vortex_prim(x, y, gamma=1.4, strength=5.0, xc=5.0, yc=5.0):
    dxv, dyv = x - xc, y - yc
    r2 = dxv * dxv + dyv * dyv
    f = strength / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = 1.0 - f * dyv
    v = 1.0 + f * dxv
    T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    return rho, u, v, p


def vortex_2d(n: int, gamma: float = 1.4, nq: int = 3, t: float = 0.0,
              cfl: float = 0.5, t_final: float = 10.0) -> Problem:
    """Isentropic vortex (strength 5 at (5, 5), background (1, 1, 1, 1)) on the
    periodic square [0, 10]^2; nq x nq Gauss-Legendre cell averages of the
    conserved variables.  The exact solution translates by (t, t)."""
    L = 10.0
    h = L / n
    qx, qw = _gauss(nq)
    U = np.zeros((4, n, n))
    xc = (np.arange(n) + 0.5) * h
    cx, cy = (5.0 + t) % L, (5.0 + t) % L
    for a in range(nq):
        ya = xc + qx[a] * h
        for b in range(nq):
            xb = xc + qx[b] * h
            X, Y = np.meshgrid(xb, ya)           # Y varies along rows (j), X along i
            # nearest periodic image of the vortex centre
            DX = (X - cx + 0.5 * L) % L - 0.5 * L
            DY = (Y - cy + 0.5 * L) % L - 0.5 * L
            rho, u, v, p = vortex_prim(DX, DY, gamma, xc=0.0, yc=0.0)
            U += qw[a] * qw[b] * prim_to_cons_2d(rho, u, v, p, gamma)
    return Problem(2, n, n, 0.0, L, 0.0, L, gamma, (BC_PERIODIC,) * 4, cfl, t_final,
                   np.ascontiguousarray(U), name=f"vortex_{n}")


def blast_2d(n: int = 4096, gamma: float = 1.4, cfl: float = 0.5, t_final: float = 1.0) -> Problem:
    """Sedov-type blast in the corner of [0, 1.1]^2: rho = 1, u = v = 0,
    E = 1e-10 everywhere (p = 1e-10 (gamma - 1)) except E = 0.244816 / (dx dy)
    in cell (0, 0).  Reflective x-lo / y-lo walls, transmissive x-hi / y-hi."""
    L = 1.1
    h = L / n
    U = np.zeros((4, n, n))
    U[0] = 1.0
    U[3] = 1e-10
    U[3, 0, 0] = 0.244816 / (h * h)
    return Problem(2, n, n, 0.0, L, 0.0, L, gamma,
                   (BC_REFLECTIVE, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_TRANSMISSIVE), cfl,
                   t_final, np.ascontiguousarray(U), name=f"blast_{n}")


def quadrant_2d(n: int, states, gamma: float = 1.4, cfl: float = 0.5, t_final: float = 0.25,
                name: str = "quadrant") -> Problem:
    """Four-quadrant Riemann data on [0, 1]^2 split at (0.5, 0.5); states are
    (rho, u, v, p) for quadrants (x>.5,y>.5), (x<.5,y>.5), (x<.5,y<.5), (x>.5,y<.5).
    Cells are aligned with the split when n is even; odd n mixes the straddling
    cells in proportion."""
    h = 1.0 / n
    lo = np.arange(n) * h
    fx = np.clip((0.5 - lo) / h, 0.0, 1.0)    # fraction of the cell with x < 0.5
    fy = fx
    Uq = [prim_to_cons_2d(*s, gamma) for s in states]
    FXl, FYl = np.meshgrid(fx, fy)
    U = ((1 - FXl) * (1 - FYl))[None] * Uq[0][:, None, None] \
        + (FXl * (1 - FYl))[None] * Uq[1][:, None, None] \
        + (FXl * FYl)[None] * Uq[2][:, None, None] \
        + ((1 - FXl) * FYl)[None] * Uq[3][:, None, None]
    return Problem(2, n, n, 0.0, 1.0, 0.0, 1.0, gamma, (BC_TRANSMISSIVE,) * 4, cfl, t_final,
                   np.ascontiguousarray(U), name=name, meta={"states": states})


def quadrant_batch(nprob: int = 256, n_lo: int = 128, n_hi: int = 1024, stream: int = 5,
                   gamma: float = 1.4) -> list[Problem]:
    """Batch of four-quadrant problems: n log-uniform in [n_lo, n_hi]; per
    quadrant rho log-U[0.1, 2], u, v U[-1, 1], p log-U[0.02, 2]."""
    g = rng(stream)
    out = []
    for k in range(nprob):
        n = int(round(float(np.exp(g.uniform(np.log(n_lo), np.log(n_hi))))))
        states = []
        for _ in range(4):
            rho = float(np.exp(g.uniform(np.log(0.1), np.log(2.0))))
            u, v = (float(a) for a in g.uniform(-1.0, 1.0, 2))
            p = float(np.exp(g.uniform(np.log(0.02), np.log(2.0))))
            states.append((rho, u, v, p))
        out.append(quadrant_2d(n, states, gamma, name=f"quadrant_{k}"))
    return out


def random_smooth_1d(n: int, stream: int, periodic: bool = True, gamma: float = 1.4,
                     amp: float = 0.3) -> Problem:
    """Random smooth periodic data (a few Fourier modes) for parity tests."""
    g = rng(stream)
    x = (np.arange(n) + 0.5) / n
    def field_(base, a):
        k = g.integers(1, 4, 3)
        ph = g.uniform(0, 2 * np.pi, 3)
        c = g.uniform(-a, a, 3)
        return base + sum(c[i] * np.sin(2 * np.pi * k[i] * x + ph[i]) for i in range(3))
    rho = field_(1.0, amp)
    u = field_(0.0, amp)
    p = field_(1.0, amp)
    U = prim_to_cons_1d(rho, u, p, gamma)
    bc = (BC_PERIODIC,) * 4 if periodic else (BC_TRANSMISSIVE, BC_REFLECTIVE, 0, 0)
    return Problem(1, n, 1, 0.0, 1.0, 0.0, 1.0, gamma, bc, 0.4, 0.05,
                   np.ascontiguousarray(U), name=f"smooth_{n}")


def random_jumps_2d(nx: int, ny: int, stream: int, bc=None, gamma: float = 1.4) -> Problem:
    """Random piecewise-constant blocks plus noise (2-D parity tests with
    discontinuities in both directions and ragged sizes)."""
    g = rng(stream)
    nb = 4
    bx = np.sort(g.integers(1, nx, nb - 1))
    by = np.sort(g.integers(1, ny, nb - 1))
    ix = np.searchsorted(bx, np.arange(nx), side="right")
    iy = np.searchsorted(by, np.arange(ny), side="right")
    rho_b = np.exp(g.uniform(np.log(0.2), np.log(5.0), (nb, nb)))
    p_b = np.exp(g.uniform(np.log(0.05), np.log(5.0), (nb, nb)))
    u_b = g.uniform(-1.0, 1.0, (nb, nb))
    v_b = g.uniform(-1.0, 1.0, (nb, nb))
    I, J = np.meshgrid(ix, iy)
    rho, p, u, v = rho_b[J, I], p_b[J, I], u_b[J, I], v_b[J, I]
    U = prim_to_cons_2d(rho, u, v, p, gamma)
    if bc is None:
        bc = (BC_REFLECTIVE, BC_TRANSMISSIVE, BC_TRANSMISSIVE, BC_REFLECTIVE)
    return Problem(2, nx, ny, 0.0, nx / max(nx, ny), 0.0, ny / max(nx, ny), gamma, tuple(bc),
                   0.4, 0.02, np.ascontiguousarray(U), name=f"jumps_{nx}x{ny}")
