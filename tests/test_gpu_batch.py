"""Batched problems of uneven size through pp_cweno_create_batch: every
problem keeps its own time step and step count, and each one matches the
FP64 oracle run on it alone (same bounds as the single-problem tests)."""
import numpy as np
import pytest

import oracle
from paper_1402_5618_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5618_gb300 import binding
    binding.lib()
    return binding


def _grid(p):
    return oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc)


def _rel(A, Bm):
    return np.array([np.abs(A[v] - Bm[v]).sum() / max(np.abs(Bm[v]).sum(), 1e-300)
                     for v in range(A.shape[0])])


def _batch_run(B, probs, precision, t_final=None, max_steps=10**9):
    cfgs = [B.config_from_problem(p, precision) for p in probs]
    s = B.Solver(None, batch=cfgs)
    U0 = np.concatenate([np.ascontiguousarray(p.U0).ravel() for p in probs])
    s.set_state(U0)
    tf = min(p.t_final for p in probs) if t_final is None else t_final
    n, rc = s.advance(tf, max_steps, check=False)
    U, t, steps = s.get_state()
    st = s.stats()
    s.close()
    out, off = [], 0
    for p in probs:
        sz = p.U0.size
        out.append(U[off:off + sz].reshape(p.U0.shape))
        off += sz
    return out, rc, st


def test_batch_1d_ragged_matches_oracle(B):
    probs = [W.riemann_1d(n, (1.0, 0.2 * k, 1.0 + k), (0.3, -0.1 * k, 0.2), bc=(1, 2 if k % 2 else 1),
                          t_final=0.04, cfl=0.4)
             for k, n in enumerate([100, 700, 1500, 3000, 64])]
    outs, rc, st = _batch_run(B, probs, B.PREC_FP64)
    assert rc == 0 and st.violations == 0
    noise_key = 999
    for p, Ug in zip(probs, outs):
        g = _grid(p)
        Uo, to, so, *_ = oracle.advance(g, p.U0, p.cfl, 0.04)
        Up, *_ = oracle.advance(g, p.U0 * (1 + 1e-16 * W.rng(noise_key).standard_normal(p.U0.shape)),
                                p.cfl, 0.04)
        tol = np.maximum(1e-11, 8 * _rel(Up, Uo))
        print(f"PARITY batch n={p.nx}: rel-L1 {_rel(Ug, Uo)} d_ref {_rel(Up, Uo)} bound {tol}")
        assert np.all(_rel(Ug, Uo) <= tol), (p.nx, _rel(Ug, Uo), tol)


def test_batch_2d_quadrants_match_oracle(B):
    probs = [W.quadrant_2d(n, s, t_final=0.02) for n, s in
             zip([40, 130, 600], [[(1.0, 0.1, 0.0, 1.0), (0.5, 0.0, 0.2, 0.4),
                                   (0.2, -0.1, 0.0, 0.1), (0.8, 0.0, -0.2, 0.6)]] * 3)]
    outs, rc, st = _batch_run(B, probs, B.PREC_FP64, max_steps=12)
    assert rc in (0, B.PP_ERR_STEPS) and st.violations == 0
    for p, Ug in zip(probs, outs):
        g = _grid(p)
        Uo, to, so, *_ = oracle.advance(g, p.U0, p.cfl, 0.02, max_steps=12)
        Up, *_ = oracle.advance(g, p.U0 * (1 + 1e-16 * W.rng(5).standard_normal(p.U0.shape)),
                                p.cfl, 0.02, max_steps=12)
        tol = np.maximum(1e-11, 8 * _rel(Up, Uo))
        print(f"PARITY batch n={p.nx}: rel-L1 {_rel(Ug, Uo)} d_ref {_rel(Up, Uo)} bound {tol}")
        assert np.all(_rel(Ug, Uo) <= tol), (p.nx, _rel(Ug, Uo), tol)


def test_batch_mixed_runs_and_tracks_fp64(B):
    """The 1-D Riemann batch workload (small seeded subset) in the mixed
    form: no violations, and close to the FP64 batch."""
    probs = W.riemann_batch(nprob=24, n_lo=256, n_hi=2048)
    for p in probs:
        p.cfl = 1.0 / 12.0
    o64, rc64, st64 = _batch_run(B, probs, B.PREC_FP64, t_final=0.02)
    o32, rc32, st32 = _batch_run(B, probs, B.PREC_MIXED, t_final=0.02)
    assert rc64 == 0 and rc32 == 0 and st64.violations == 0 and st32.violations == 0
    for a, b in zip(o32, o64):
        assert _rel(a, b)[0] < 1e-4


def test_batch_mixed_2d_transposed_path(B):
    """Mixed 2-D batch (transposed y rows, batched stage combination) of
    uneven problems -- partial tiles, sides that are not multiples of 4, a
    periodic vortex beside transmissive quadrants: no violations, each
    problem close to the FP64 batch, and to the same problem run alone."""
    st4 = [(1.0, 0.1, 0.0, 1.0), (0.5, 0.0, 0.2, 0.4), (0.2, -0.1, 0.0, 0.1), (0.8, 0.0, -0.2, 0.6)]
    probs = [W.quadrant_2d(n, st4, t_final=0.02) for n in (40, 130, 600)]
    probs.append(W.vortex_2d(96, t_final=0.02))
    for p in probs:
        p.cfl = 1.0 / 12.0
    o64, rc64, s64 = _batch_run(B, probs, B.PREC_FP64, max_steps=12)
    o32, rc32, s32 = _batch_run(B, probs, B.PREC_MIXED, max_steps=12)
    assert rc32 in (0, B.PP_ERR_STEPS) and s32.violations == 0 and s64.violations == 0
    for p, a, b in zip(probs, o32, o64):
        assert np.all(_rel(a, b) < 1e-5), (p.nx, _rel(a, b))
        s = B.Solver(B.config_from_problem(p, B.PREC_MIXED))
        s.set_state(np.ascontiguousarray(p.U0).ravel())
        s.advance(p.t_final, 12, check=False)
        one = s.get_state()[0].reshape(p.U0.shape)
        s.close()
        assert np.all(_rel(a, one) < 1e-5), (p.nx, _rel(a, one))


def test_batch_problem_stats(B):
    """Per-problem statistics of a batch: each problem's own step count (the
    oracle's, run alone), time and violations; an index out of range is an
    argument error."""
    probs = [W.riemann_1d(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), t_final=0.02) for n in (64, 300, 1000)]
    s = B.Solver(None, batch=[B.config_from_problem(p, B.PREC_FP64) for p in probs])
    s.set_state(np.concatenate([np.ascontiguousarray(p.U0).ravel() for p in probs]))
    s.advance(0.02)
    for k, p in enumerate(probs):
        st = s.problem_stats(k)
        Uo, to, so, *_ = oracle.advance(_grid(p), p.U0, p.cfl, 0.02)
        assert st.steps == so and st.t == 0.02 and st.violations == 0 and st.first_bad_cell == -1
    with pytest.raises(B.PPError) as e:
        s.problem_stats(len(probs))
    assert e.value.code == B.PP_ERR_ARG
    s.close()


def test_batch_rows_per_chunk_tuned_and_results_unchanged(B):
    """The autotuner times both chunk lengths on the batch's own lines at the
    first set_state and keeps one; a batch handle reports 8 or 16, and its
    steps match the same problems run one by one (each single-problem handle
    tunes its own length) within the FP64 run bound."""
    probs = [W.riemann_1d(n, (1.0, 0.3, 1.0), (0.2, -0.2, 0.1), bc=(1, 1), t_final=0.01)
             for n in (300, 2500, 6000)]
    cfgs = [B.config_from_problem(p, B.PREC_FP64) for p in probs]
    s = B.Solver(None, batch=cfgs)
    s.set_state(np.concatenate([np.ascontiguousarray(p.U0).ravel() for p in probs]))
    assert s.rows_per_chunk() in (8, 16)
    s.advance(0.01)
    U = s.get_state()[0]
    s.close()
    off = 0
    for p in probs:
        one = B.Solver(B.config_from_problem(p, B.PREC_FP64))
        one.set_state(np.ascontiguousarray(p.U0).ravel())
        one.advance(0.01)
        Uo = one.get_state()[0]
        one.close()
        got = U[off:off + p.U0.size]
        off += p.U0.size
        rel = np.abs(got - Uo).sum() / np.abs(Uo).sum()
        assert rel < 1e-12, (p.nx, rel)
