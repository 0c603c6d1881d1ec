"""Pins of the time-step reading behind the positivity theorem (Sec. 2.4,
eq. (CFL-CD)) on the seeded 4096-problem Riemann batch.

The theorem bounds lambda * max(|u| + a) by omega_hat_1 over the states the
first-order steps of its proof act on: the limited face values U^-, U^+ of
every stage.  A time step taken from the cell averages alone does not bound
them: after theta_1 pulls a face density towards epsilon without touching
its energy, the face's sound speed can exceed the averages' by orders of
magnitude.  Two seeded non-vacuum problems of the batch leave G that way at
half the theorem's CFL; with the check on the face values and a step redone
from U^n when it fails (the oracle's face_cfl), every problem of the batch,
including the ones whose exact solution opens a vacuum, stays in G."""
import numpy as np
import pytest

import oracle
from paper_1402_5618_gb300 import workloads as W

W1 = 1.0 / 12.0          # omega_hat_1, the bound of eq. (CFL-CD)
CFL = W1 / 2.0           # the first-order positivity factor 1/2 (brute force, Sec. 2.4 remark)


def _in_G(U):
    rho = U[0]
    e = U[2] / rho - 0.5 * (U[1] / rho) ** 2
    return bool(np.all(np.isfinite(U)) and np.all(rho > 0) and np.all(e > 0))


def _grid(q, face_cfl=0.0):
    return oracle.make_grid(1, q.nx, 1, q.dx, 1.0, q.gamma, q.bc, face_cfl=face_cfl)


def _face_speed_cfl(q, U, dt):
    """lambda max(|u| + a) over the limited face values of U (component-wise
    reconstruction with two copied ghosts per side, Sec. 2.4 limiter)."""
    ext = np.concatenate([U[:, :1], U[:, :1], U, U[:, -1:], U[:, -1:]], axis=1)
    um, up = np.zeros_like(U), np.zeros_like(U)
    for v in range(3):
        um[v], up[v] = oracle.recon_scalar(ext[v], False)
    eps = min(1e-13, float(U[0].min()))
    for j in range(q.nx):
        um[:, j], up[:, j], _ = oracle.limit_cell(U[:, j], um[:, j], up[:, j], eps, q.gamma)
    s = 0.0
    for F in (um, up):
        rho, u = F[0], F[1] / F[0]
        p = (q.gamma - 1.0) * (F[2] - 0.5 * rho * u * u)
        s = max(s, float(np.max(np.abs(u) + np.sqrt(np.maximum(q.gamma * p / rho, 0.0)))))
    return dt / q.dx * s


def test_average_cfl_does_not_bound_the_face_values():
    """Problem 491 of the seeded batch (890 cells, a strong non-vacuum double
    rarefaction): with dt from the cell averages at CFL omega_1/2, some
    state reached before step 21 has limited face values at lambda max(|u|+a)
    far beyond omega_1, and the step after it leaves G."""
    q = W.riemann_batch()[491]
    g = _grid(q)
    U = np.ascontiguousarray(q.U0)
    worst = 0.0
    left_G = False
    for _ in range(23):
        dt = CFL / oracle.max_rate(g, U)
        worst = max(worst, _face_speed_cfl(q, U, dt))
        U = oracle.rk3_step(g, U, dt)
        if not _in_G(U):
            left_G = True
            break
    assert left_G
    assert worst > 10.0 * W1, worst


@pytest.mark.parametrize("k", [491, 1630])
def test_face_check_keeps_the_failing_problems_in_G(k):
    """The two seeded non-vacuum problems that leave G with dt from the cell
    averages stay in G with eq. (CFL-CD) checked on the face values."""
    q = W.riemann_batch()[k]
    U, t, steps, _, cnt, rc = oracle.advance(_grid(q), q.U0, CFL, 1e9, max_steps=23)
    assert not _in_G(U)
    U, t, steps, _, cnt, rc = oracle.advance(_grid(q, W1), q.U0, CFL, 1e9, max_steps=23)
    assert rc == -2 and steps == 23 and _in_G(U)
    assert cnt.face_rate > 0.0


def test_face_check_bounds_every_accepted_step():
    """Every accepted step satisfies dt * (face rate of each of its stages)
    <= omega_1: the accepted step recomputed stage by stage (eq. (RK3)) with
    the check off is bitwise the accepted state, and each stage's face rate,
    from the operator's own count, obeys the bound."""
    q = W.riemann_batch()[491]
    g_on, g_off = _grid(q, W1), _grid(q)
    U = np.ascontiguousarray(q.U0)
    t = 0.0
    rejected = 0
    for _ in range(23):
        Un, t1, steps, dt, cnt, rc = oracle.advance(g_on, U, CFL, 1e9, t0=t, max_steps=1)
        assert rc == -2 and steps == 1
        rejected += cnt.rejected
        rates = []
        V = U
        for k in range(3):
            L, c = oracle.operator(g_off, V, min(1e-13, float(V[0].min())))
            rates.append(c.face_rate)
            if k == 0:
                V = U + dt * L
            elif k == 1:
                V = 0.75 * U + 0.25 * V + 0.25 * dt * L
            else:
                V = U / 3.0 + 2.0 / 3.0 * V + 2.0 / 3.0 * dt * L
        assert np.array_equal(V, Un)
        assert dt * max(rates) <= W1, (dt, rates)
        U, t = Un, t1
    assert _in_G(U)
    assert rejected > 0   # dt from the averages alone fails somewhere in these steps


@pytest.mark.slow
def test_vacuum_subset_stays_in_G():
    """P5 on the batch's vacuum subset: the problems whose data open an exact
    vacuum (u_R - u_L >= 2 (a_L + a_R) / (gamma - 1), 168 of 4096) stay in G
    for 40 steps at CFL omega_1/2 with the face check; none of them fails a
    step."""
    probs = W.riemann_batch()
    vac = [q for q in probs if W.opens_vacuum(q)]
    assert len(vac) == 168
    for q in vac:
        U, t, steps, _, cnt, rc = oracle.advance(_grid(q, W1), q.U0, CFL, 1e9, max_steps=40)
        assert rc == -2 and steps == 40, q.name
        assert _in_G(U), q.name


def test_face_check_stalls_at_a_floor_face_value():
    """The cost of the face check near a vacuum: on problem 44 of the set (a
    double rarefaction whose centre cell holds rho = 0.02) the limited face
    values include one of density ~1e-9 that keeps its energy as kinetic
    energy, so |u| = sqrt(2 E / rho) ~ 1e4 - 1e5; the checked dt then
    collapses while every cell average stays tame.  Without the check the
    same problem leaves G (a stage produces a cell outside it): the scheme
    as read either stalls or loses positivity here."""
    q = W.riemann_batch()[44]
    g = oracle.make_grid(1, q.nx, 1, q.dx, 1.0, q.gamma, q.bc, face_cfl=W1)
    U, t, steps, dt, cnt, rc = oracle.advance(g, q.U0, W1 / 2, 0.15, max_steps=300)
    assert rc == -2 and steps == 300
    assert t < 1e-3 and dt < 1e-8 and cnt.face_rate > 1e6
    assert _in_G(U) and U[0].min() > 0.02
    # the averages' rate alone: orders of magnitude below the face rate
    assert oracle.max_rate(g, U) < 1e4
    # the limited face values: one near the floor whose energy is kinetic
    ext = np.concatenate([U[:, :1], U[:, :1], U, U[:, -1:], U[:, -1:]], axis=1)
    um, up = np.zeros_like(U), np.zeros_like(U)
    for v in range(3):
        um[v], up[v] = oracle.recon_scalar(ext[v], False)
    eps = min(1e-13, float(U[0].min()))
    for j in range(q.nx):
        um[:, j], up[:, j], _ = oracle.limit_cell(U[:, j], um[:, j], up[:, j], eps, q.gamma)
    F = np.concatenate([um, up], axis=1)
    rho = F[0]
    pr = (q.gamma - 1.0) * (F[2] - 0.5 * F[1] ** 2 / rho)
    k = int(np.argmin(rho))
    assert rho[k] < 1e-8 and pr[k] > 0 and abs(F[1, k] / rho[k]) > 1e4
    assert abs(F[1, k] / rho[k]) > 100 * np.sqrt(q.gamma * pr[k] / rho[k])
    g0 = _grid(q)
    U0, t0, s0, *_, rc0 = oracle.advance(g0, q.U0, W1 / 2, 0.01)
    assert rc0 == -1 and t0 < 0.01
