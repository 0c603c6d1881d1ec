"""Eq. (CFL-CD) checked on the limited face values through the CUDA path
(pp_cweno_config.cfl_positivity_cap): the seeded 4096-problem Riemann batch,
which includes two non-vacuum problems that leave G when dt comes from the
cell averages alone (problems 491 and 1630) and 168 problems whose exact
solution opens a vacuum, run as one batch in both arithmetics.  FP64
problems match the oracle's checked run (same steps, same redone steps);
every problem of the batch stays in G."""
import numpy as np
import pytest

import oracle
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


def _rel(A, Bm):
    return np.array([np.abs(A[v] - Bm[v]).sum() / max(np.abs(Bm[v]).sum(), 1e-300)
                     for v in range(A.shape[0])])


def _in_G(U):
    rho = U[0]
    e = U[2] / rho - 0.5 * (U[1] / rho) ** 2
    return bool(np.all(np.isfinite(U)) and np.all(rho > 0) and np.all(e > 0))


def _batch(B, probs, precision, steps):
    cfgs = [B.config_from_problem(p, precision, cfl_positivity_cap=True) for p in probs]
    s = B.Solver(None, batch=cfgs)
    s.set_state(np.concatenate([np.ascontiguousarray(p.U0).ravel() for p in probs]))
    n, rc = s.advance(1e9, steps, check=False)
    U = s.get_state()[0]
    per = [s.problem_stats(k) for k in range(len(probs))]
    st = s.stats()
    s.close()
    out, off = [], 0
    for p in probs:
        out.append(U[off:off + p.U0.size].reshape(p.U0.shape))
        off += p.U0.size
    return out, rc, st, per


def _subset():
    probs = W.riemann_batch()
    vac = [k for k, q in enumerate(probs) if W.opens_vacuum(q)]
    ks = [491, 1630] + vac[:6]
    sub = [probs[k] for k in ks]
    for q in sub:
        q.cfl = W1 / 2
    return ks, sub


def test_checked_batch_matches_oracle(B):
    """FP64: the two problems that leave G without the check and six
    vacuum-opening ones, 23 steps as one checked batch, each against the
    oracle's checked run on it alone: identical step and redo counts,
    relative L1 per variable within max(1e-11, 8 d_ref) (d_ref: the
    oracle's own change under a 1e-16 relative perturbation of its input),
    and in G."""
    ks, sub = _subset()
    outs, rc, st, per = _batch(B, sub, B.PREC_FP64, 23)
    assert rc == B.PP_ERR_STEPS and st.violations == 0
    rej_o = 0
    for k, q, Ug, ps in zip(ks, sub, outs, per):
        g = oracle.make_grid(1, q.nx, 1, q.dx, 1.0, q.gamma, q.bc, face_cfl=W1)
        Uo, to, so, _, cnt, rco = oracle.advance(g, q.U0, q.cfl, 1e9, max_steps=23)
        Up, *_ = oracle.advance(g, q.U0 * (1 + 1e-16 * W.rng(77).standard_normal(q.U0.shape)),
                                q.cfl, 1e9, max_steps=23)
        assert rco == -2 and so == 23 and ps.steps == 23
        assert ps.rejected == cnt.rejected, (k, ps.rejected, cnt.rejected)
        rej_o += cnt.rejected
        rel, tol = _rel(Ug, Uo), np.maximum(1e-11, 8 * _rel(Up, Uo))
        print(f"problem {k}: n={q.nx} redone={ps.rejected} rel-L1={rel} bound={tol}")
        assert np.all(rel <= tol), (k, rel, tol)
        assert _in_G(Ug)
    assert st.rejected == rej_o and rej_o > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_riemann_batch_stays_in_G(B, precision):
    """P5 on the whole seeded batch (4096 problems of 256-8192 cells, the
    168 vacuum-opening ones included) at CFL omega_1/2 with the check: 40
    steps, no cell average outside G in any problem."""
    probs = W.riemann_batch()
    for q in probs:
        q.cfl = W1 / 2
    prec = B.PREC_FP64 if precision == "fp64" else B.PREC_MIXED
    outs, rc, st, per = _batch(B, probs, prec, 40)
    print(f"{precision}: redone steps {st.rejected} in "
          f"{sum(1 for ps in per if ps.rejected)} problems")
    assert rc == B.PP_ERR_STEPS and st.violations == 0
    assert all(ps.steps == 40 and ps.violations == 0 for ps in per)
    assert all(_in_G(U) for U in outs)


def test_checked_step_api_redoes_until_accepted(B):
    """pp_cweno_step with the check: problem 491 stepped one call at a time
    matches the oracle's checked run step for step (each call ends with an
    accepted step)."""
    q = W.riemann_batch()[491]
    q.cfl = W1 / 2
    s = B.Solver(B.config_from_problem(q, B.PREC_FP64, cfl_positivity_cap=True))
    s.set_state(np.ascontiguousarray(q.U0).ravel())
    g = oracle.make_grid(1, q.nx, 1, q.dx, 1.0, q.gamma, q.bc, face_cfl=W1)
    Uo, to, so, _, cnt, rco = oracle.advance(g, q.U0, q.cfl, 1e9, max_steps=23)
    for _ in range(23):
        s.step()
    Ug, tg, sg = s.get_state()
    st = s.stats()
    s.close()
    assert sg == 23 and st.violations == 0 and st.rejected == cnt.rejected
    assert abs(tg - to) <= 1e-12 * to
    assert np.all(_rel(Ug.reshape(q.U0.shape), Uo) <= 1e-9)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checked_graph_replay_equals_single_steps(B, precision):
    """Checked steps alternate the two state buffers; a graph replay that
    runs past the step limit (21 steps from graphs of 16) must leave the
    same state as 21 single pp_cweno_step calls, bit for bit, on the 2-D
    corner blast (the mixed form also keeps its transposed planes)."""
    p = W.blast_2d(64, cfl=0.5, t_final=1e9)
    prec = B.PREC_FP64 if precision == "fp64" else B.PREC_MIXED
    res = []
    for mode in ("advance", "step"):
        s = B.Solver(B.config_from_problem(p, prec, cfl_positivity_cap=True))
        s.set_state(np.ascontiguousarray(p.U0).ravel())
        if mode == "advance":
            s.advance(1e9, 21, check=False)
        else:
            for _ in range(21):
                s.step()
        U, t, steps = s.get_state()
        st = s.stats()
        s.close()
        assert steps == 21 and st.violations == 0
        res.append((U, t, st.rejected))
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]
    assert np.array_equal(res[0][0], res[1][0])
