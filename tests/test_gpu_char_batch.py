"""Batches in the characteristic-wise form (Sec. 2.3) through
pp_cweno_create_batch: problems of uneven size, boundary kind and dimension
advanced together, each against the oracle's characteristic run on it alone
(FP64: identical step counts, relative L1 within max(1e-11, 8 d_ref) as for
single problems), and the mixed form against the FP64 batch and against the
same problem run alone."""
import numpy as np
import pytest

import oracle
from paper_1402_5618_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHAR = 1
W1 = 1.0 / 12.0


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5618_gb300 import binding
    binding.lib()
    return binding


def _grid(p, **kw):
    return oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc, recon=CHAR, **kw)


def _rel(A, Bm):
    return np.array([np.abs(A[v] - Bm[v]).sum() / max(np.abs(Bm[v]).sum(), 1e-300)
                     for v in range(A.shape[0])])


def _batch_run(B, probs, precision, t_final, max_steps=10**9, **kw):
    cfgs = [B.config_from_problem(p, precision, recon=B.RECON_CHARACTERISTIC, **kw) for p in probs]
    s = B.Solver(None, batch=cfgs)
    s.set_state(np.concatenate([np.ascontiguousarray(p.U0).ravel() for p in probs]))
    n, rc = s.advance(t_final, max_steps, check=False)
    U = s.get_state()[0]
    per = [s.problem_stats(k) for k in range(len(probs))]
    st = s.stats()
    s.close()
    out, off = [], 0
    for p in probs:
        out.append(U[off:off + p.U0.size].reshape(p.U0.shape))
        off += p.U0.size
    return out, rc, st, per


def _single_run(B, p, precision, t_final, max_steps=10**9):
    s = B.Solver(B.config_from_problem(p, precision, recon=B.RECON_CHARACTERISTIC))
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    s.advance(t_final, max_steps, check=False)
    U = s.get_state()[0].reshape(p.U0.shape)
    s.close()
    return U


def _riemann_mix():
    probs = [W.riemann_1d(n, (1.0, 0.2 * k, 1.0 + k), (0.3, -0.1 * k, 0.2), bc=(1, 2 if k % 2 else 1),
                          t_final=0.04, cfl=0.4)
             for k, n in enumerate([100, 700, 1500, 3000, 64])]
    probs.append(W.density_wave(200))   # periodic: a group of its own
    return probs


def test_char_batch_1d_matches_oracle(B):
    """FP64: five bounded Riemann problems of 64-3000 cells (transmissive
    and reflective ends) and a periodic density wave in one batch, to
    t = 0.04, each against the oracle's characteristic run."""
    probs = _riemann_mix()
    outs, rc, st, per = _batch_run(B, probs, B.PREC_FP64, 0.04)
    assert rc == 0 and st.violations == 0
    for k, (p, Ug, ps) in enumerate(zip(probs, outs, per)):
        g = _grid(p)
        Uo, to, so, *_ = oracle.advance(g, p.U0, p.cfl, 0.04)
        Up, *_ = oracle.advance(g, p.U0 * (1 + 1e-16 * W.rng(300 + k).standard_normal(p.U0.shape)),
                                p.cfl, 0.04)
        tol = np.maximum(1e-11, 8 * _rel(Up, Uo))
        print(f"PARITY char batch {p.name} n={p.nx}: rel-L1 {_rel(Ug, Uo)} d_ref {_rel(Up, Uo)}")
        assert ps.steps == so, (p.name, ps.steps, so)
        assert np.all(_rel(Ug, Uo) <= tol), (p.name, _rel(Ug, Uo), tol)


def test_char_batch_2d_matches_oracle(B):
    """FP64 2-D: transmissive four-quadrant problems of 40^2 and 130^2 and a
    periodic vortex of 48^2 in one batch (x and y line groups, bounded and
    periodic), 8 steps, each against the oracle's characteristic run."""
    st4 = [(1.0, 0.1, 0.0, 1.0), (0.5, 0.0, 0.2, 0.4), (0.2, -0.1, 0.0, 0.1), (0.8, 0.0, -0.2, 0.6)]
    probs = [W.quadrant_2d(n, st4, t_final=0.02) for n in (40, 130)]
    probs.append(W.vortex_2d(48, t_final=0.02))
    outs, rc, st, per = _batch_run(B, probs, B.PREC_FP64, 0.02, max_steps=8)
    assert rc in (0, B.PP_ERR_STEPS) and st.violations == 0
    for k, (p, Ug) in enumerate(zip(probs, outs)):
        g = _grid(p)
        Uo, *_ = oracle.advance(g, p.U0, p.cfl, 0.02, max_steps=8)
        Up, *_ = oracle.advance(g, p.U0 * (1 + 1e-16 * W.rng(310 + k).standard_normal(p.U0.shape)),
                                p.cfl, 0.02, max_steps=8)
        tol = np.maximum(1e-11, 8 * _rel(Up, Uo))
        print(f"PARITY char batch {p.name}: rel-L1 {_rel(Ug, Uo)} d_ref {_rel(Up, Uo)}")
        assert np.all(_rel(Ug, Uo) <= tol), (p.name, _rel(Ug, Uo), tol)


def test_char_batch_mixed_1d_tracks_fp64_and_single(B):
    """Mixed form, the same 1-D mix: in G, close to the FP64 batch, and
    equal to each problem run alone."""
    probs = _riemann_mix()
    o64, rc64, s64, _ = _batch_run(B, probs, B.PREC_FP64, 0.04)
    o32, rc32, s32, _ = _batch_run(B, probs, B.PREC_MIXED, 0.04)
    assert rc64 == 0 and rc32 == 0 and s32.violations == 0
    for p, a, b in zip(probs, o32, o64):
        r = _rel(a, b)
        print(f"char batch mixed vs FP64 {p.name}: {r}")
        assert np.all(r < 1e-4), (p.name, r)   # FP32 face values: 1e-5 on the momentum of shocked lines
        one = _single_run(B, p, B.PREC_MIXED, 0.04)
        assert np.all(_rel(a, one) < 1e-6), (p.name, _rel(a, one))


def test_char_batch_mixed_2d_transposed_path(B):
    """Mixed 2-D characteristic batch: y lines as rows of the transposed
    planes; uneven sizes, one periodic problem; close to the FP64 batch and
    to each problem run alone."""
    st4 = [(1.0, 0.1, 0.0, 1.0), (0.5, 0.0, 0.2, 0.4), (0.2, -0.1, 0.0, 0.1), (0.8, 0.0, -0.2, 0.6)]
    probs = [W.quadrant_2d(n, st4, t_final=0.02) for n in (40, 130, 300)]
    probs.append(W.vortex_2d(96, t_final=0.02))
    for p in probs:
        p.cfl = W1
    o64, rc64, s64, _ = _batch_run(B, probs, B.PREC_FP64, 0.02, max_steps=12)
    o32, rc32, s32, _ = _batch_run(B, probs, B.PREC_MIXED, 0.02, max_steps=12)
    assert s32.violations == 0 and s64.violations == 0
    for p, a, b in zip(probs, o32, o64):
        r = _rel(a, b)
        print(f"char batch mixed 2-D vs FP64 {p.name}: {r}")
        assert np.all(r < 1e-5), (p.name, r)
        one = _single_run(B, p, B.PREC_MIXED, 0.02, max_steps=12)
        assert np.all(_rel(a, one) < 1e-6), (p.name, _rel(a, one))


def test_char_batch_riemann_positivity(B):
    """The 1-D Riemann batch workload in the characteristic form with the
    positivity cap (eq. (CFL-CD) checked on the face values): the two
    problems that leave G without the check and 30 vacuum-opening ones,
    both arithmetics, 40 steps, every problem in G."""
    probs = W.riemann_batch()
    vac = [k for k, q in enumerate(probs) if W.opens_vacuum(q)]
    sub = [probs[k] for k in [491, 1630] + vac[:30]]
    for q in sub:
        q.cfl = W1 / 2
    for prec in (B.PREC_FP64, B.PREC_MIXED):
        outs, rc, st, per = _batch_run(B, sub, prec, 1e9, max_steps=40, cfl_positivity_cap=True)
        assert rc == B.PP_ERR_STEPS and st.violations == 0
        for q, U in zip(sub, outs):
            rho = U[0]
            e = U[2] / rho - 0.5 * (U[1] / rho) ** 2
            assert np.all(np.isfinite(U)) and np.all(rho > 0) and np.all(e > 0), (prec, q.name)
