"""Integration pins of the FP64 oracle: whole runs against what the paper
prints (Table 1, the Sec. 3 minima) and against exact properties of the
scheme (conservation, free stream, mirror symmetry, 2-D/1-D reduction,
positivity under the limiter, exact Riemann solutions)."""
import os

import numpy as np
import pytest

import oracle
from paper_1402_5618_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid(p: W.Problem, **kw):
    return oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc, **kw)


def _run(p: W.Problem, **kw):
    U, t, steps, dtl, cnt, rc = oracle.advance(_grid(p, **kw), p.U0, p.cfl, p.t_final)
    assert rc == 0 and t == p.t_final
    return U, steps, cnt


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------- P1: Table 1
def test_table1_density_wave_errors_and_order():
    """Paper Table 1: the L1 errors (normalised h * sum |e|) at N = 40, 80, 160
    within 40% of the printed values and the observed order at least 4.8.
    The paper's own dt constant is omega_1, ours 0.6 (the benchmark's
    configuration); the spatial error dominates at these N."""
    table = {int(r[0]): (float(r[1]), float(r[2])) for r in _read_table("table1_density_wave.txt")}
    l1 = {}
    for n in (40, 80, 160):
        p = W.density_wave(n)
        U, steps, cnt = _run(p)
        err = np.abs(U[0] - W.density_wave_exact(n, 2.0))
        l1[n] = p.dx * err.sum()
        linf = err.max()
        assert 0.6 < l1[n] / table[n][0] < 1.4, (n, l1[n], table[n][0])
        assert 0.5 < linf / table[n][1] < 1.5, (n, linf, table[n][1])
        assert cnt.theta1_active == 0 and cnt.theta2_active == 0
    assert np.log2(l1[40] / l1[80]) > 4.8 and np.log2(l1[80] / l1[160]) > 4.8


# ---------------------------------------------- P4 / P9: conservation, smooth
def test_conservation_periodic_1d_and_smooth_never_limits():
    p = W.random_smooth_1d(96, stream=21)
    g_on = _grid(p)
    U_on, t, steps, _, cnt, rc = oracle.advance(g_on, p.U0, p.cfl, p.t_final)
    assert rc == 0 and steps > 10
    tot0, tot1 = p.U0.sum(axis=1), U_on.sum(axis=1)
    scale = np.abs(p.U0).sum(axis=1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale)
    # no limiter activity on smooth data: the run with the limiter switched
    # off is bit-identical
    assert cnt.theta1_active == 0 and cnt.theta2_active == 0
    U_off, *_ = oracle.advance(_grid(p, limiter=False), p.U0, p.cfl, p.t_final)
    assert np.array_equal(U_on, U_off)


def test_conservation_periodic_2d_with_jumps():
    p = W.random_jumps_2d(24, 20, stream=33, bc=(0, 0, 0, 0))
    U, t, steps, _, cnt, rc = oracle.advance(_grid(p), p.U0, p.cfl, 0.01)
    assert rc == 0
    tot0, tot1 = p.U0.reshape(4, -1).sum(1), U.reshape(4, -1).sum(1)
    scale = np.abs(p.U0).reshape(4, -1).sum(1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale)


# ---------------------------------------------------------- P10: free stream
@pytest.mark.parametrize("ndim", [1, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (2, 1, 1, 2)])
def test_free_stream_preserved(ndim, bc):
    gamma = 1.4
    if ndim == 1:
        U0 = np.ascontiguousarray(np.tile(np.array([[1.3], [0.0 if 2 in bc[:2] else 0.5 * 1.3], [2.7]]), (1, 17)))
        g = oracle.make_grid(1, 17, dx=0.1, bc=bc)
    else:
        vx = 0.0 if 2 in bc[:2] else 0.4
        vy = 0.0 if 2 in bc[2:] else -0.3
        U0 = np.zeros((4, 13, 11))
        U0[0], U0[1], U0[2], U0[3] = 0.8, 0.8 * vx, 0.8 * vy, 1.9
        g = oracle.make_grid(2, 11, 13, 0.1, 0.12, gamma, bc)
    U = U0.copy()
    for _ in range(5):
        U = oracle.rk3_step(g, U, 0.01)
    assert np.max(np.abs(U - U0)) <= 1e-14 * np.abs(U0).max()


# -------------------------------------------------------- P11: mirror symmetry
def test_mirror_symmetry_1d():
    """x -> -x (reverse the cells, negate the momentum) commutes with the
    scheme: this ties the plus-side reconstruction to the minus side."""
    p = W.riemann_1d(40, (1.0, 0.3, 1.0), (0.2, -0.6, 0.15), bc=(2, 1), t_final=0.05)
    pm = W.riemann_1d(40, (0.2, 0.6, 0.15), (1.0, -0.3, 1.0), bc=(1, 2), t_final=0.05)
    assert np.allclose(pm.U0, p.U0[:, ::-1] * np.array([1, -1, 1])[:, None], rtol=0, atol=1e-15)
    U, *_ = _run(p)
    Um, *_ = _run(pm)
    mir = Um[:, ::-1] * np.array([1, -1, 1])[:, None]
    assert np.max(np.abs(U - mir)) <= 1e-12 * np.abs(U).max()


def test_transpose_symmetry_2d_corner_blast():
    """Corner blast with reflective walls on both low sides: U(i, j) equals
    the x<->y swapped U(j, i) (the x and y sweeps are mirror images)."""
    n = 24
    p = W.blast_2d(n, t_final=0.06)
    p.U0[3] = 1e-3       # milder background so the short run moves the front
    p.U0[3, 0, 0] = 5.0 / (p.dx * p.dy) * 1e-3
    U, steps, cnt = _run(p)
    UT = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    assert steps > 3
    assert np.max(np.abs(U - UT)) <= 1e-13 * np.abs(U).max()


# --------------------------------------------------- P12: 2-D reduces to 1-D
def test_2d_y_invariant_equals_1d():
    p1 = W.random_smooth_1d(32, stream=41, periodic=False)
    ny = 6
    U2 = np.zeros((4, ny, p1.nx))
    U2[0], U2[1], U2[3] = p1.U0[0], p1.U0[1], p1.U0[2]
    g1 = oracle.make_grid(1, p1.nx, dx=p1.dx, bc=p1.bc)
    g2 = oracle.make_grid(2, p1.nx, ny, p1.dx, 0.05, 1.4, (p1.bc[0], p1.bc[1], 0, 0))
    Ua, Ub = p1.U0.copy(), U2.copy()
    for _ in range(4):
        Ua = oracle.rk3_step(g1, Ua, 0.002)
        Ub = oracle.rk3_step(g2, Ub, 0.002)
    for j in range(ny):
        assert np.max(np.abs(Ub[[0, 1, 3], j] - Ua)) <= 1e-13 * np.abs(Ua).max()
    assert np.max(np.abs(Ub[2])) <= 1e-13


# ------------------------------------------------------ P13: vortex closed form
def test_vortex_translation_converges():
    """Isentropic vortex moving with (1, 1): error vs the translated closed
    form decreases under refinement (the 2-D extension is dimension by
    dimension with mid-face fluxes, formally second order)."""
    errs = []
    for n in (24, 48):
        p = W.vortex_2d(n, t_final=0.5)
        U, steps, cnt = _run(p)
        ex = W.vortex_2d(n, t=0.5).U0
        errs.append(np.mean(np.abs(U[0] - ex[0])))
    assert errs[1] < errs[0] / 3.0, errs


# ------------------------------------------------ P5 / P14: positivity, minima
def _prim(U, gamma):
    rho = U[0]
    e = U[-1] / rho - 0.5 * np.sum(U[1:-1] ** 2, axis=0) / rho ** 2
    return rho, e, (gamma - 1) * rho * e


POSITIVITY_CASES = {
    "123": lambda: W.paper_riemann("123", 400, cfl=1 / 24),
    "strong_shock": lambda: W.paper_riemann("strong_shock", 200, cfl=1 / 24),
    "double_rarefaction": lambda: W.paper_riemann("double_rarefaction", 400, cfl=1 / 24),
    "leblanc": lambda: W.leblanc(400, cfl=1 / 24),
}


@pytest.mark.parametrize("name", sorted(POSITIVITY_CASES))
def test_positivity_and_paper_minima(name):
    """At CFL omega_1/2 (the limiter theorem's bound combined with the
    half-CFL first-order bound pinned above) densities and internal energies
    stay positive, and the minima match the paper's printed values to within
    an order of magnitude (the paper used characteristic variables for these
    runs, the oracle conservative ones)."""
    minima = {r[0]: (r[1], float(r[2]), float(r[3])) for r in _read_table("positivity_minima.txt")}
    p = POSITIVITY_CASES[name]()
    U, steps, cnt = _run(p)
    rho, e, pr = _prim(U, p.gamma)
    assert np.all(rho > 0) and np.all(e > 0)
    q, rho_min, q_min = minima[name]
    got_q = e.min() if q == "e" else pr.min()
    # the double rarefaction is critical (its exact solution touches vacuum
    # at x = 0), so its minima depend on the scheme's dissipation; a wider
    # band applies there
    band = 30.0 if name == "double_rarefaction" else 10.0
    assert 1 / band < rho.min() / rho_min < band, (rho.min(), rho_min)
    assert 1 / band < got_q / q_min < band, (got_q, q_min)


@pytest.mark.slow
def test_sedov_1d_positivity():
    p = W.sedov_1d(cfl=1 / 24)
    U, steps, cnt = _run(p)
    rho, e, pr = _prim(U, p.gamma)
    assert np.all(rho > 0) and np.all(e > 0)
    assert 0.1 < rho.min() / 4.731e-3 < 10
    assert cnt.theta2_active > 0


def test_riemann_problem_converges_to_exact():
    """Sod data: L1 error against the exact cell averages decreases with N."""
    errs = []
    for n in (50, 100):
        p = W.paper_riemann("sod", n, cfl=0.4)
        U, steps, cnt = _run(p)
        d = W.PAPER_RIEMANN["sod"]
        ex = oracle.riemann_cell_averages(d["WL"], d["WR"], d["x0"], d["x1"], n, d["xd"], d["t"])
        errs.append(p.dx * np.abs(U[0] - ex[0]).sum())
    assert errs[1] < 0.75 * errs[0] and errs[1] < 0.1, errs


# ------------------------------------------- Sec. 3 remark: Lax-Friedrichs flux
def test_llf_density_wave_fifth_order():
    """With the local Lax-Friedrichs flux at the faces the scheme is still
    fifth order on the smooth density wave (the face flux is consistent and
    Lipschitz; the order comes from the reconstruction).  The wave is a pure
    contact (u = 1, p = 1), which HLLC resolves without dissipation while LLF
    damps the O(h^5) face jumps with alpha = |u| + a, so LLF's errors are
    larger than HLLC's but by a bounded factor (2.1 measured)."""
    l1 = {}
    for n in (40, 80):
        p = W.density_wave(n)
        Ul, *_ = _run(p, flux=1)
        Uh, *_ = _run(p)
        ex = W.density_wave_exact(n, 2.0)
        l1[n] = p.dx * np.abs(Ul[0] - ex).sum()
        lh = p.dx * np.abs(Uh[0] - ex).sum()
        assert 1.0 < l1[n] / lh < 3.0, (n, l1[n], lh)
        assert not np.array_equal(Ul, Uh)
    assert np.log2(l1[40] / l1[80]) > 4.8, l1


@pytest.mark.parametrize("name", ["123", "leblanc"])
def test_llf_positivity(name):
    """Positivity under the limiter at CFL omega_1/2 with the Lax-Friedrichs
    face flux (its first-order scheme is positive up to CFL 1, pinned above,
    so the limiter theorem's bound holds a fortiori)."""
    p = POSITIVITY_CASES[name]()
    U, steps, cnt = _run(p, flux=1)
    rho, e, pr = _prim(U, p.gamma)
    assert np.all(rho > 0) and np.all(e > 0)
    assert np.all(np.isfinite(U))


def test_llf_123_central_deviation_not_larger():
    """Sec. 3, double rarefaction (123) example: the paper attributes the
    oscillations of velocity and internal energy in the near-vacuum centre
    to the less dissipative HLLC flux and names the Lax-Friedrichs flux as
    the way to control them, without showing results.  Measured form of that
    remark: on the paper's 400 cells, the largest deviation from the exact
    solution of u and of e over the central quarter of the domain is no
    larger with LLF than with HLLC (the oracle reconstructs conservative
    variables, the paper characteristic ones, so the effect is small:
    about 5% here)."""
    d = W.PAPER_RIEMANN["123"]
    p = POSITIVITY_CASES["123"]()
    ex = oracle.riemann_cell_averages(d["WL"], d["WR"], d["x0"], d["x1"], p.nx, d["xd"], d["t"])
    uex = ex[1] / ex[0]
    eex = ex[2] / ex[0] - 0.5 * uex ** 2
    c = slice(3 * p.nx // 8, 5 * p.nx // 8)
    dev = {}
    for flux in (0, 1):
        U, *_ = _run(p, flux=flux)
        u = U[1] / U[0]
        e = U[2] / U[0] - 0.5 * u ** 2
        dev[flux] = (np.abs(u - uex)[c].max(), np.abs(e - eex)[c].max())
    assert dev[1][0] <= dev[0][0] and dev[1][1] <= dev[0][1], dev
