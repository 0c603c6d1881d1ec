"""The local Lax-Friedrichs face flux (the alternative Sec. 3 names for the
near-vacuum double rarefaction) through the C ABI, against the oracle run
with the same flux.

Tolerances are those of the HLLC parity tests: one FP64 operator evaluation
element-wise within 1e-12 of the variable's flux scale; whole FP64 runs with
an identical step count and relative L1 within max(1e-11, 8 d_ref), d_ref
the oracle's own sensitivity to a 1e-16 relative perturbation of the input;
the mixed form's operator within its stated FP32 accuracy (2e-6 of the flux
scale on smooth data, 1e-4 with jumps)."""
import numpy as np
import pytest

import oracle
from paper_1402_5618_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LLF = 1


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5618_gb300 import binding
    binding.lib()
    return binding


def _grid(p):
    return oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc, flux=LLF)


def _scale(p, U):
    nv = U.shape[0]
    flat = U.reshape(nv, -1)
    rho = flat[0]
    vel = np.sqrt(np.sum(flat[1:nv - 1] ** 2, axis=0)) / rho
    pr = (p.gamma - 1) * (flat[nv - 1] - 0.5 * rho * vel ** 2)
    smax = np.max(vel + np.sqrt(p.gamma * np.maximum(pr, 0) / rho))
    mom = np.abs(rho * vel * vel + pr).max()
    F = [np.abs(rho * vel).max(), mom] + ([mom] if nv == 4 else [])
    F.append(np.abs(vel * (flat[nv - 1] + pr)).max())
    h = min(p.dx, p.dy) if p.ndim == 2 else p.dx
    return np.array([(F[v] + np.abs(flat[v]).max() * smax) / h for v in range(nv)])


def _gpu_operator(B, p, U, eps, precision):
    s = B.Solver(B.config_from_problem(p, precision, flux=B.FLUX_LLF))
    Ud = torch.from_numpy(np.ascontiguousarray(U).ravel()).cuda()
    Ld = torch.zeros_like(Ud)
    s.operator(Ud, Ld, eps)
    s.close()
    return Ld.cpu().numpy().reshape(U.shape)


OPERATOR_CASES = [
    ("smooth_periodic_1500", lambda: W.random_smooth_1d(1500, stream=52), 2e-6),
    ("riemann_1300", lambda: W.riemann_1d(1300, (1.0, 0.75, 1.0), (0.125, -0.3, 0.1), bc=(2, 1)), 1e-4),
    ("riemann_vacuum_517", lambda: W.riemann_1d(517, (1.0, -3.5, 0.4), (1.0, 3.5, 0.4)), 1e-4),
    ("riemann_bounded_8192", lambda: W.riemann_1d(8192, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)), 1e-4),
    ("vortex_64", lambda: W.vortex_2d(64), 2e-6),
    ("jumps_600x530", lambda: W.random_jumps_2d(600, 530, stream=61), 1e-4),
    ("jumps_periodic_1100x600", lambda: W.random_jumps_2d(1100, 600, stream=64, bc=(0, 0, 0, 0)), 1e-4),
]


@pytest.mark.parametrize("name,make,tol32", OPERATOR_CASES, ids=[c[0] for c in OPERATOR_CASES])
def test_llf_operator_parity(B, name, make, tol32):
    p = make()
    eps = min(1e-13, p.U0[0].min())
    Lo, _ = oracle.operator(_grid(p), p.U0, eps)
    Lh, _ = oracle.operator(oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc),
                            p.U0, eps)
    scale = _scale(p, p.U0)
    L64 = _gpu_operator(B, p, p.U0, eps, B.PREC_FP64)
    L32 = _gpu_operator(B, p, p.U0, eps, B.PREC_MIXED)
    for v in range(p.U0.shape[0]):
        assert np.abs(L64[v] - Lo[v]).max() <= 1e-12 * scale[v], (v, np.abs(L64[v] - Lo[v]).max())
        assert np.abs(L32[v] - Lo[v]).max() <= tol32 * scale[v], (v, np.abs(L32[v] - Lo[v]).max())
    # the flux switch is live: with jumps in the data the LLF operator
    # differs from the HLLC one (on smooth data the face jumps are O(h^5)
    # and the two agree to rounding)
    if tol32 > 2e-6:
        assert np.abs(Lo - Lh).max() > 1e-6 * scale.max()


def _rel_l1(A, Bm):
    return np.array([np.abs(A[v] - Bm[v]).sum() / max(np.abs(Bm[v]).sum(), 1e-300)
                     for v in range(A.shape[0])])


RUN_CASES = [
    ("123_400", lambda: W.paper_riemann("123", 400, cfl=1 / 12), 10**9),
    ("lax_200", lambda: W.paper_riemann("lax", 200, cfl=0.4), 10**9),
    ("blast_64_cfl_1_12", lambda: W.blast_2d(64, cfl=1 / 12, t_final=0.05), 40),
]


@pytest.mark.parametrize("name,make,max_steps", RUN_CASES, ids=[c[0] for c in RUN_CASES])
def test_llf_run_parity_fp64(B, name, make, max_steps):
    p = make()
    g = _grid(p)
    Uo, to, so, _, cnt, rc = oracle.advance(g, p.U0, p.cfl, p.t_final, max_steps=max_steps)
    noise = W.rng(999).standard_normal(p.U0.shape)
    Ub, *_ = oracle.advance(g, p.U0 * (1 + 1e-16 * noise), p.cfl, p.t_final, max_steps=max_steps)
    tol = np.maximum(1e-11, 8 * _rel_l1(Ub, Uo))
    s = B.Solver(B.config_from_problem(p, flux=B.FLUX_LLF))
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    n, rcg = s.advance(p.t_final, max_steps, check=False)
    Ug, tg, sg = s.get_state()
    st = s.stats()
    s.close()
    assert rc in (0, -2) and rcg in (0, B.PP_ERR_STEPS)
    assert sg == so
    rel = _rel_l1(Ug.reshape(p.U0.shape), Uo)
    print(f"PARITY llf run {name}: rel-L1 {rel} d_ref {_rel_l1(Ub, Uo)} bound {tol}")
    assert np.all(rel <= tol), (rel, tol)
    assert st.violations == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_llf_123_positivity(B, prec):
    """The paper's double rarefaction (400 cells) at the positivity CFL with
    the LLF flux: every stage stays in G, and the minima agree with the
    oracle's LLF run."""
    p = W.paper_riemann("123", 400, cfl=1 / 24)
    Uo, *_ = oracle.advance(_grid(p), p.U0, p.cfl, p.t_final)
    P = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED
    s = B.Solver(B.config_from_problem(p, P, flux=B.FLUX_LLF))
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    n, rc = s.advance(p.t_final, check=False)
    U = s.get_state()[0].reshape(p.U0.shape)
    st = s.stats()
    s.close()
    assert rc == 0 and st.violations == 0
    rho = U[0]
    e = U[2] / rho - 0.5 * (U[1] / rho) ** 2
    eo = Uo[2] / Uo[0] - 0.5 * (Uo[1] / Uo[0]) ** 2
    assert np.all(rho > 0) and np.all(e > 0)
    tol = 1e-8 if prec == "fp64" else 5e-2
    assert abs(rho.min() / Uo[0].min() - 1) <= tol
    assert abs(e.min() / eo.min() - 1) <= tol

