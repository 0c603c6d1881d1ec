"""pp_cweno_operator_noalloc: the operator evaluated with the library's fixed
device scratch instead of allocated memory, for callers that cannot call
cudaMalloc.  It must give what pp_cweno_operator gives and what the oracle's
operator gives (same tolerance as the other operator tests), on two calls in
a row sharing the scratch array.

This file is collected last on purpose."""
import numpy as np
import pytest

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


def _handle_operator(B, p, Ud, eps):
    s = B.Solver(B.config_from_problem(p))
    L = torch.zeros_like(Ud)
    s.operator(Ud, L, eps)
    s.close()
    return L.cpu().numpy().reshape(p.U0.shape)


@pytest.mark.parametrize("name,make,eps", [
    ("jumps_2d_300x200", lambda: W.random_jumps_2d(300, 200, stream=71), 1e-13),
    ("vortex_2d_64_device_eps", lambda: W.vortex_2d(64), 0.0),
    ("riemann_1d_1300", lambda: W.riemann_1d(1300, (1.0, 0.4, 1.0), (0.2, -0.2, 0.1), bc=(2, 1)), 1e-13),
])
def test_noalloc_operator_matches_handle_operator_twice(B, name, make, eps):
    p = make()
    Ud = torch.from_numpy(np.ascontiguousarray(p.U0).ravel()).cuda()
    cfg = B.config_from_problem(p)
    ref = _handle_operator(B, p, Ud, eps if eps > 0 else min(cfg.eps_pos, p.U0[0].min()))
    scale = _scale(p, p.U0)
    for _ in range(2):
        L = torch.full_like(Ud, float("nan"))
        B.operator_noalloc(cfg, Ud, L, eps)
        torch.cuda.synchronize()
        got = L.cpu().numpy().reshape(p.U0.shape)
        for v in range(p.U0.shape[0]):
            assert np.abs(got[v] - ref[v]).max() <= 1e-12 * scale[v], (name, v)


@pytest.mark.parametrize("name,make,eps", [
    ("jumps_2d_300x200", lambda: W.random_jumps_2d(300, 200, stream=72), 1e-13),
    ("riemann_1d_1300_device_eps", lambda: W.riemann_1d(1300, (1.0, 0.4, 1.0), (0.2, -0.2, 0.1),
                                                        bc=(2, 1)), 0.0),
])
def test_noalloc_operator_matches_oracle(B, name, make, eps):
    """The allocation-free operator against the oracle's operator directly,
    element-wise within 1e-12 of each variable's flux scale."""
    import oracle
    p = make()
    Ud = torch.from_numpy(np.ascontiguousarray(p.U0).ravel()).cuda()
    cfg = B.config_from_problem(p)
    L = torch.full_like(Ud, float("nan"))
    B.operator_noalloc(cfg, Ud, L, eps)
    torch.cuda.synchronize()
    got = L.cpu().numpy().reshape(p.U0.shape)
    g = oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc)
    ref = oracle.operator(g, p.U0, eps if eps > 0 else min(cfg.eps_pos, p.U0[0].min()))
    ref = ref[0] if isinstance(ref, tuple) else ref
    scale = _scale(p, p.U0)
    err = [np.abs(got[v] - ref[v]).max() / scale[v] for v in range(p.U0.shape[0])]
    print(f"PARITY noalloc vs oracle {name}: max |dL| / flux scale {np.max(err):.2e}")
    assert max(err) <= 1e-12, (name, err)


def test_noalloc_rejects_oversized_and_mixed(B):
    big = B.make_config(ndim=2, nx=2048, ny=2048, bc=(1, 1, 1, 1))
    U = torch.zeros(4 * 2048 * 2048, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PPError) as e:
        B.operator_noalloc(big, U, U)
    assert e.value.code == B.PP_ERR_UNSUPPORTED
    mixed = B.make_config(ndim=1, nx=64, precision=B.PREC_MIXED)
    u = torch.zeros(3 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PPError) as e:
        B.operator_noalloc(mixed, u, u)
    assert e.value.code == B.PP_ERR_UNSUPPORTED


def test_noalloc_state_outside_G_gives_nan(B):
    """With eps <= 0 the device takes the limiter epsilon from the state; a
    state with one cell outside G is not evaluated and L comes back NaN
    (the call itself does not synchronise and returns PP_OK)."""
    p = W.riemann_1d(300, (1.0, 0.4, 1.0), (0.2, -0.2, 0.1), bc=(2, 1))
    U = np.ascontiguousarray(p.U0).copy()
    U[2, 150] = 0.5 * U[1, 150] ** 2 / U[0, 150] * 0.5   # E below the kinetic energy: e < 0
    Ud = torch.from_numpy(U.ravel()).cuda()
    L = torch.zeros_like(Ud)
    B.operator_noalloc(B.config_from_problem(p), Ud, L, 0.0)
    torch.cuda.synchronize()
    assert torch.isnan(L).all()
    # the same call on the admissible state writes finite values again
    Ud = torch.from_numpy(np.ascontiguousarray(p.U0).ravel()).cuda()
    B.operator_noalloc(B.config_from_problem(p), Ud, L, 0.0)
    torch.cuda.synchronize()
    assert torch.isfinite(L).all()


def test_noalloc_rejects_characteristic_form(B):
    """The characteristic-wise form needs the handle's block-solve scratch:
    PP_ERR_UNSUPPORTED, with real device buffers."""
    cfg = B.make_config(ndim=1, nx=64, recon=B.RECON_CHARACTERISTIC)
    u = torch.zeros(3 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PPError) as e:
        B.operator_noalloc(cfg, u, u)
    assert e.value.code == B.PP_ERR_UNSUPPORTED
