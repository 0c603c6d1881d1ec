"""The 2-D four-quadrant batch workload run as its configuration states it,
to t = 0.25, on a seeded subset: the 16 first problems of the 256-problem
set with at most 256^2 cells (transmissive boundaries, states of density
0.1-2, velocities in [-1, 1], pressures 0.02-2), at the positivity cap
(CFL omega_1/2 with the face check of eq. (CFL-CD)), in both arithmetics.
Every problem stays in G; the problems that reach t = 0.25 within a step
budget of three times their initial estimate (the face check can stall a
problem near a vacuum) are compared mixed against FP64.  The four-quadrant
problems have no closed form; their shear layers amplify rounding, so the
mixed form is held to agreement in L1, not to the FP64 rounding level."""
import numpy as np
import pytest

from paper_1402_5618_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1 = 1.0 / 12.0


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5618_gb300 import binding
    binding.lib()
    return binding


def _budget(probs, t_final):
    est = 0.0
    for q in probs:
        rho, mx, my, E = q.U0
        u, v = mx / rho, my / rho
        a = np.sqrt(q.gamma * (q.gamma - 1.0) * (E - 0.5 * rho * (u * u + v * v)) / rho)
        rate = np.max(np.abs(u) + a) / q.dx + np.max(np.abs(v) + a) / q.dy
        est = max(est, t_final * rate / (W1 / 2))
    return int(3 * est) + 2000


def _run(B, probs, precision, t_final, cap):
    s = B.Solver(None, batch=[B.config_from_problem(q, precision, cfl_positivity_cap=True)
                              for q in probs])
    s.set_state(np.concatenate([np.ascontiguousarray(q.U0).ravel() for q in probs]))
    n, rc = s.advance(t_final, cap, check=False)
    U = s.get_state()[0]
    per = [s.problem_stats(k) for k in range(len(probs))]
    s.close()
    out, off = [], 0
    for q in probs:
        out.append(U[off:off + q.U0.size].reshape(q.U0.shape))
        off += q.U0.size
    return out, rc, per


def test_quadrant_batch_to_final_time(B):
    probs = [q for q in W.quadrant_batch() if q.nx <= 256][:16]
    t = 0.25
    cap = _budget(probs, t)
    o32, rc32, p32 = _run(B, probs, B.PREC_MIXED, t, cap)
    o64, rc64, p64 = _run(B, probs, B.PREC_FP64, t, cap)
    rels = []
    for q, a, b, s32, s64 in zip(probs, o32, o64, p32, p64):
        for U in (a, b):
            rho = U[0]
            e = U[3] / rho - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho ** 2
            assert np.all(np.isfinite(U)) and np.all(rho > 0) and np.all(e > 0), q.name
        assert s32.violations == 0 and s64.violations == 0
        if s32.t == t and s64.t == t:
            rels.append(np.abs(a[0] - b[0]).sum() / np.abs(b[0]).sum())
    done = sum(1 for s in p32 if s.t == t)
    rels = np.array(rels)
    print(f"quadrant batch to t = 0.25, {len(probs)} problems of {min(q.nx for q in probs)}^2-"
          f"{max(q.nx for q in probs)}^2, budget {cap} steps: {done} reach t (mixed), "
          f"{sum(1 for s in p64 if s.t == t)} (FP64); density rel-L1 mixed vs FP64 median "
          f"{np.median(rels):.2e} max {rels.max():.2e}; redone steps "
          f"{sum(s.rejected for s in p32)} / {sum(s.rejected for s in p64)}")
    assert done >= 15
    assert np.median(rels) < 1e-3 and rels.max() < 5e-2
