"""The characteristic-wise reconstruction (Sec. 2.3) through the C ABI,
against the oracle run with recon = 1 on the same seeded inputs.

FP64 tolerances, as for the component-wise form: one operator evaluation
element-wise within 1e-12 of the variable's flux scale (max |F_v| + max |U_v|
max(|u|+a)) / h; whole runs with an identical step count and relative L1
within max(1e-11, 8 d_ref), d_ref the oracle's own change under a 1e-16
relative perturbation of the input (the WENO-Z weights amplify rounding
near jumps).  The GPU walks each line's block system in the same
elimination order as the oracle with the same partial pivoting; the
arithmetic differs in rounding only (reciprocals instead of divisions, the
Woodbury matrix G taken at the first row of the walk)."""
import numpy as np
import pytest

import oracle
from paper_1402_5618_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHAR = 1


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_5618_gb300 import binding
    binding.lib()
    return binding


def _grid(p):
    return oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc, recon=CHAR)


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


def _gpu_operator(B, p, U, eps, precision=0, **kw):
    s = B.Solver(B.config_from_problem(p, precision, recon=B.RECON_CHARACTERISTIC, **kw))
    Ud = torch.from_numpy(np.ascontiguousarray(U).ravel()).cuda()
    Ld = torch.zeros_like(Ud)
    s.operator(Ud, Ld, eps)
    s.close()
    return Ld.cpu().numpy().reshape(U.shape)


OPERATOR_CASES = [
    ("smooth_periodic_200", lambda: W.random_smooth_1d(200, stream=51)),
    ("smooth_bounded_1100", lambda: W.random_smooth_1d(1100, stream=53, periodic=False)),
    ("riemann_1300", lambda: W.riemann_1d(1300, (1.0, 0.75, 1.0), (0.125, -0.3, 0.1), bc=(2, 1))),
    ("riemann_vacuum_517", lambda: W.riemann_1d(517, (1.0, -3.5, 0.4), (1.0, 3.5, 0.4))),
    ("leblanc_1000", lambda: W.leblanc(1000)),
    ("n8_periodic", lambda: W.random_smooth_1d(8, stream=54)),
    ("n8_bounded", lambda: W.random_smooth_1d(8, stream=55, periodic=False)),
    ("smooth_periodic_8192", lambda: W.random_smooth_1d(8192, stream=56)),
    ("vortex_64", lambda: W.vortex_2d(64)),
    ("jumps_600x530", lambda: W.random_jumps_2d(600, 530, stream=61)),
    ("jumps_periodic_96x40", lambda: W.random_jumps_2d(96, 40, stream=62, bc=(0, 0, 0, 0))),
    ("blast_96", lambda: W.blast_2d(96)),
    ("jumps_periodic_1100x600", lambda: W.random_jumps_2d(1100, 600, stream=64, bc=(0, 0, 0, 0))),
]


@pytest.mark.parametrize("name,make", OPERATOR_CASES, ids=[c[0] for c in OPERATOR_CASES])
def test_char_operator_parity(B, name, make):
    p = make()
    eps = min(1e-13, p.U0[0].min())
    Lo, _ = oracle.operator(_grid(p), p.U0, eps)
    Lg = _gpu_operator(B, p, p.U0, eps)
    scale = _scale(p, p.U0)
    for v in range(p.U0.shape[0]):
        err = np.abs(Lg[v] - Lo[v]).max()
        assert err <= 1e-12 * scale[v], (v, err / scale[v])


def test_char_operator_with_llf(B):
    """The two choices combine: characteristic reconstruction with the
    Lax-Friedrichs face flux."""
    p = W.random_jumps_2d(300, 200, stream=65)
    eps = min(1e-13, p.U0[0].min())
    g = oracle.make_grid(2, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc, recon=CHAR, flux=1)
    Lo, _ = oracle.operator(g, p.U0, eps)
    Lg = _gpu_operator(B, p, p.U0, eps, flux=B.FLUX_LLF)
    scale = _scale(p, p.U0)
    for v in range(4):
        assert np.abs(Lg[v] - Lo[v]).max() <= 1e-12 * scale[v]


def _rel_l1(A, Bm):
    return np.array([np.abs(A[v] - Bm[v]).sum() / max(np.abs(Bm[v]).sum(), 1e-300)
                     for v in range(A.shape[0])])


RUN_CASES = [
    ("sod_100", lambda: W.paper_riemann("sod", 100, cfl=0.4), 10**9),
    ("lax_200", lambda: W.paper_riemann("lax", 200, cfl=0.4), 10**9),
    # at CFL omega_1 = 1/12 the oracle itself leaves G on this problem from
    # inputs perturbed by 1e-16 (4 of 4 seeds, near step 170); at omega_1/2
    # it stays inside on every seed
    ("123_400", lambda: W.paper_riemann("123", 400, cfl=1 / 24), 10**9),
    ("density_wave_56", lambda: W.density_wave(56), 10**9),
    ("vortex_48", lambda: W.vortex_2d(48, t_final=0.5), 40),
    ("blast_64_cfl_1_12", lambda: W.blast_2d(64, cfl=1 / 12, t_final=0.05), 40),
]


@pytest.mark.parametrize("name,make,max_steps", RUN_CASES, ids=[c[0] for c in RUN_CASES])
def test_char_run_parity(B, name, make, max_steps):
    p = make()
    g = _grid(p)
    Uo, to, so, _, cnt, rc = oracle.advance(g, p.U0, p.cfl, p.t_final, max_steps=max_steps)
    noise = W.rng(999).standard_normal(p.U0.shape)
    Ub, *_ = oracle.advance(g, p.U0 * (1 + 1e-16 * noise), p.cfl, p.t_final, max_steps=max_steps)
    tol = np.maximum(1e-11, 8 * _rel_l1(Ub, Uo))
    s = B.Solver(B.config_from_problem(p, recon=B.RECON_CHARACTERISTIC))
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    n, rcg = s.advance(p.t_final, max_steps, check=False)
    Ug, tg, sg = s.get_state()
    st = s.stats()
    s.close()
    assert rc in (0, -2) and rcg in (0, B.PP_ERR_STEPS)
    assert sg == so
    rel = _rel_l1(Ug.reshape(p.U0.shape), Uo)
    print(f"PARITY char run {name}: rel-L1 {rel} d_ref {_rel_l1(Ub, Uo)} bound {tol}")
    assert np.all(rel <= tol), (rel, tol)
    assert st.violations == 0


def test_char_123_positivity(B):
    """The paper's double rarefaction (400 cells) at the positivity CFL in
    the characteristic form: every stage stays in G and the minima agree
    with the oracle's to 1e-2 (the oracle's own minima move by up to 1e-3
    relative when its input is perturbed by 1e-16: the near-vacuum centre
    amplifies rounding)."""
    p = W.paper_riemann("123", 400, cfl=1 / 24)
    Uo, *_ = oracle.advance(_grid(p), p.U0, p.cfl, p.t_final)
    s = B.Solver(B.config_from_problem(p, recon=B.RECON_CHARACTERISTIC))
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    n, rc = s.advance(p.t_final, check=False)
    U = s.get_state()[0].reshape(p.U0.shape)
    st = s.stats()
    s.close()
    assert rc == 0 and st.violations == 0
    e = U[2] / U[0] - 0.5 * (U[1] / U[0]) ** 2
    eo = Uo[2] / Uo[0] - 0.5 * (Uo[1] / Uo[0]) ** 2
    assert np.all(U[0] > 0) and np.all(e > 0)
    assert abs(U[0].min() / Uo[0].min() - 1) <= 1e-2
    assert abs(e.min() / eo.min() - 1) <= 1e-2


def test_char_full_size_sampled_operator_4096(B):
    """The benchmark's grid size (4096^2, lines of 8 CTAs) on random jump
    data: GPU L at the intersections of sampled rows and columns equals the
    oracle's L_x(row) + L_y(column)."""
    p = W.random_jumps_2d(4096, 4096, stream=91)
    g = _grid(p)
    eps = 1e-13
    Lg = _gpu_operator(B, p, p.U0, eps)
    rng = W.rng(93)
    rows = np.sort(rng.choice(4096, 8, replace=False))
    cols = np.sort(rng.choice(4096, 8, replace=False))
    Lx, Ly = oracle.operator_lines(g, p.U0, eps, rows, cols)
    scale = _scale(p, p.U0)
    for a, j in enumerate(rows):
        for b, i in enumerate(cols):
            Lo = Lx[a, :, i] + Ly[b, :, j]
            assert np.all(np.abs(Lg[:, j, i] - Lo) <= 1e-12 * scale), (j, i)



# ------------------------------------------------------------ mixed form
MIXED_CASES = [
    ("smooth_1d_1500", lambda: W.random_smooth_1d(1500, stream=52), 2e-6),
    ("riemann_1300", lambda: W.riemann_1d(1300, (1.0, 0.75, 1.0), (0.125, -0.3, 0.1), bc=(2, 1)), 1e-4),
    ("smooth_periodic_8192", lambda: W.random_smooth_1d(8192, stream=56), 2e-6),
    # the FP32 WENO-Z floor 2^20 (u s)^2 (s the size of the characteristic
    # sums) linearises the weights on the vortex's outer indicators, which
    # the oracle's 1e-13 leaves nonlinear: 2.2e-6 of the flux scale
    ("vortex_64", lambda: W.vortex_2d(64), 4e-6),
    ("jumps_600x530", lambda: W.random_jumps_2d(600, 530, stream=61), 1e-4),
    ("jumps_periodic_1100x600", lambda: W.random_jumps_2d(1100, 600, stream=64, bc=(0, 0, 0, 0)), 1e-4),
]


@pytest.mark.parametrize("name,make,tol", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_char_mixed_operator_close_to_oracle(B, name, make, tol):
    """The mixed form (FP32 line arithmetic on the hi parts, the same block
    solve) within the mixed component-wise form's stated bounds: 2e-6 of
    the flux scale on smooth data, 1e-4 with jumps (where the WENO-Z weights
    react to the FP32 rounding of the averages)."""
    p = make()
    eps = min(1e-13, p.U0[0].min())
    Lo, _ = oracle.operator(_grid(p), p.U0, eps)
    Lg = _gpu_operator(B, p, p.U0, eps, precision=B.PREC_MIXED)
    scale = _scale(p, p.U0)
    for v in range(p.U0.shape[0]):
        err = np.abs(Lg[v] - Lo[v]).max()
        assert err <= tol * scale[v], (v, err / scale[v])


def _run_gpu(B, p, prec, max_steps=10**9):
    s = B.Solver(B.config_from_problem(p, prec, recon=B.RECON_CHARACTERISTIC))
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    n, rc = s.advance(p.t_final, max_steps, check=False)
    U, t, steps = s.get_state()
    st = s.stats()
    s.close()
    return U.reshape(p.U0.shape), steps, rc, st


@pytest.mark.parametrize("n", [64, 128])
def test_char_mixed_vortex_error_within_2x_fp64(B, n):
    """Smooth data: the mixed characteristic form's L1 density error against
    the translated closed-form vortex within 2x of the FP64 form's."""
    p = W.vortex_2d(n, t_final=1.0)
    ex = W.vortex_2d(n, t=1.0).U0
    U64, s64, rc64, _ = _run_gpu(B, p, B.PREC_FP64)
    U32, s32, rc32, st = _run_gpu(B, p, B.PREC_MIXED)
    assert rc64 == 0 and rc32 == 0 and st.violations == 0
    e64 = np.mean(np.abs(U64[0] - ex[0]))
    e32 = np.mean(np.abs(U32[0] - ex[0]))
    assert e32 <= 2.0 * e64, (e32, e64)


def test_char_mixed_blast_positivity_symmetry(B):
    """Corner blast at CFL omega_1/2: no cell leaves G, the state stays
    exactly symmetric about the diagonal (the x sweep and the y sweep over
    the transposed planes run the same arithmetic), and it stays close to
    the FP64 characteristic form."""
    p = W.blast_2d(128, cfl=1 / 24, t_final=1e-3)
    U32, s32, rc32, st32 = _run_gpu(B, p, B.PREC_MIXED, max_steps=60)
    U64, s64, rc64, st64 = _run_gpu(B, p, B.PREC_FP64, max_steps=60)
    assert st32.violations == 0 and st64.violations == 0
    sym = np.stack([U32[0].T, U32[2].T, U32[1].T, U32[3].T])
    assert np.array_equal(U32, sym)
    rel = np.abs(U32[0] - U64[0]).sum() / np.abs(U64[0]).sum()
    assert rel < 1e-3, rel


def test_char_mixed_123_positivity(B):
    """The double rarefaction in the mixed characteristic form: every stage
    in G.  Its near-vacuum minimum is not a stable quantity of this form:
    the oracle's own run gives min rho 0.0074 from the exact data and 0.0122
    / 0.0151 from data perturbed by 1e-7 (the component-wise form stays at
    0.01516 under the same perturbations), so the FP32 run is compared to
    the oracle within that spread (a factor 3)."""
    p = W.paper_riemann("123", 400, cfl=1 / 24)
    Uo, *_ = oracle.advance(_grid(p), p.U0, p.cfl, p.t_final)
    U, steps, rc, st = _run_gpu(B, p, B.PREC_MIXED)
    assert rc == 0 and st.violations == 0
    e = U[2] / U[0] - 0.5 * (U[1] / U[0]) ** 2
    eo = Uo[2] / Uo[0] - 0.5 * (Uo[1] / Uo[0]) ** 2
    assert np.all(U[0] > 0) and np.all(e > 0)
    assert 1 / 3 < U[0].min() / Uo[0].min() < 3
    assert 1 / 3 < e.min() / eo.min() < 3


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_char_lax_fewer_oscillations_on_gpu(B, prec):
    """Sec. 3, the remark after Table 3, through the CUDA path: on the Lax
    shock tube (200 cells) the characteristic form's total variation of rho,
    u and p is below the component-wise form's and within 3% of the exact
    solution's (the oracle shows the same: 1.87 / 2.40 / 3.01 against
    1.86 / 2.36 / 2.96 exact, 2.01 / 2.92 / 3.82 component-wise)."""
    p = W.paper_riemann("lax", 200, cfl=0.4)
    d = W.PAPER_RIEMANN["lax"]
    ex = oracle.riemann_cell_averages(d["WL"], d["WR"], d["x0"], d["x1"], p.nx, d["xd"], d["t"])
    P = B.PREC_FP64 if prec == "fp64" else B.PREC_MIXED

    def tv3(U):
        rho = U[0]
        u = U[1] / rho
        pr = (p.gamma - 1) * (U[2] - 0.5 * rho * u * u)
        return [np.abs(np.diff(q)).sum() for q in (rho, u, pr)]

    out = {}
    for recon in (0, 1):
        s = B.Solver(B.config_from_problem(p, P, recon=recon))
        s.set_state(np.ascontiguousarray(p.U0).ravel())
        n, rc = s.advance(p.t_final, check=False)
        U = s.get_state()[0].reshape(p.U0.shape)
        st = s.stats()
        s.close()
        assert rc == 0 and st.violations == 0
        out[recon] = tv3(U)
    tex = tv3(ex)
    for q in range(3):
        assert out[1][q] < out[0][q], (q, out)
        assert out[1][q] < 1.03 * tex[q], (q, out[1], tex)
