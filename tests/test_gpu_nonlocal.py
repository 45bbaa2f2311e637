"""Nonlocal pseudopotential projectors (Sec. 2.1, V_nloc u = sum_p <xi_p, u> xi_p), through the C-ABI.

The oracle takes the projectors on the grid (``Config.xi``, from
``projectors_gaussian``); the library takes centres, widths and amplitudes
(``pou_set_projectors``) and builds its own per-axis tables.  Tolerances as in
the local-potential parity tests.
"""
import numpy as np
import pytest

from oracle import pou_oracle as O
from paper_1510_07230_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1510_07230_gb300 import pou
    return pou


def _projectors(R, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    widths = rng.uniform(0.6, 0.9, len(R))
    amps = scale * rng.uniform(0.5, 1.5, len(R))
    return R, widths, amps


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order,n", [(2, (20, 12, 10)), (4, (20, 12, 10)), (4, (5, 6, 8))])
def test_energy_and_h_apply_with_projectors(P, precision, order, n):
    L, N = (6.0, 5.0, 4.0), 3
    cfg0 = O.Config(n=n, L=L, order=order, N=N)
    R = np.array([[1.8, 2.0, 2.4], [4.5, 1.0, 0.4], [3.0, 4.5, 1.8]])
    Z = np.array([3.0, 2.0, 4.0])
    c, wd, am = _projectors(R, 3)
    xi = O.projectors_gaussian(cfg0, c, wd, am)
    cfg = O.Config(n=n, L=L, order=order, N=N, xi=xi)
    U = inputs.random_orbitals(9, N, n)
    if precision == 1:
        U = U.astype(np.float32).astype(np.float64)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = P.Solver(n, L, N, order=order, precision=precision)
    s.set_atoms(R, Z, 0.8)
    s.set_projectors(c, wd, am)
    got = s.evaluate(U)
    ref = O.energy_terms(U, vext, cfg)
    tol = 1e-11 if precision == 0 else 2e-6
    for k in ("kinetic", "external", "hartree", "exchange"):
        assert abs(got[k] - getattr(ref, k)) <= tol * max(1.0, abs(getattr(ref, k))), k
    tdt = torch.float64 if precision == 0 else torch.float32
    Ud = torch.as_tensor(U, dtype=tdt, device="cuda")
    out = torch.empty_like(Ud)
    s.backward(Ud, 1.0 / (2 * O.F_OCC * cfg.dV), out)
    ref_h = O.apply_h(U, O.total_potential(O.density(U), vext, cfg), cfg)
    np.testing.assert_allclose(out.double().cpu().numpy(), ref_h,
                               atol=(1e-11 if precision == 0 else 2e-5) * np.max(np.abs(ref_h)))
    s.close()


def _l10_with_projectors(P, precision, **kw):
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    c, wd, am = _projectors(R, 5, scale=2.0)
    cfg0 = O.cubic(w.n, w.L, order=w.order, N=w.N)
    xi = O.projectors_gaussian(cfg0, c, wd, am)
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N, xi=xi, **kw)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    s = P.Solver(w.n, w.L, w.N, order=w.order, precision=precision, **kw)
    s.set_atoms(R, Z, w.width)
    s.set_projectors(c, wd, am)
    return w, cfg, vext, U0, s


@pytest.mark.parametrize("kw,steps", [({}, 80), ({"n_diag": 20}, 60)])
def test_fp64_trajectory_with_projectors(P, kw, steps):
    w, cfg, vext, U0, s = _l10_with_projectors(P, P.FP64, **kw)
    ref = O.run(U0, vext, cfg, steps)
    Eo = np.array([h.energy for h in ref.history])
    s.set_orbitals(U0)
    s.iterate(steps)
    E, _ = s.history()
    assert np.max(np.abs(E - Eo)) < 1e-9
    W = s.get_orbitals()
    HW = O.apply_h(W, O.total_potential(O.density(W), vext, cfg), cfg)
    g = O.gradient_residual(W, HW, cfg)
    assert abs(s.gradient_norm() - g) <= 1e-8 * g + 1e-12
    s.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_converged_energy_with_projectors(P, precision, tol):
    """Both forms reach the oracle's converged energy with projectors."""
    w, cfg, vext, U0, s = _l10_with_projectors(P, precision)
    ref = O.run(U0, vext, cfg, 3000, e_tol=1e-15)
    s.set_orbitals(U0)
    s.iterate(3000)
    e = s.energy()["total"]
    assert abs(e - ref.E) <= tol, (e, ref.E)
    W = s.get_orbitals()
    assert abs(O.energy(W, vext, cfg) - e) <= 1e-7 * abs(e)
    s.close()


def test_mixed_n128_13pt_with_projectors(P):
    """The bench's kernel configuration with 32 projectors: the first steps
    follow the oracle; the returned orbitals carry the reported energy."""
    n, L, N = 40, 16.0, 128
    R, Z = inputs.atoms(71, 32, L, "uniform26")
    c, wd, am = _projectors(R, 8)
    cfg0 = O.cubic(n, L, order=4, N=N)
    cfg = O.cubic(n, L, order=4, N=N, xi=O.projectors_gaussian(cfg0, c, wd, am))
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    U = inputs.random_orbitals(71, N, (n, n, n)).astype(np.float32)
    s = P.Solver(n, L, N, order=4, precision=P.FP32)
    s.set_atoms(R, Z, 0.8)
    s.set_projectors(c, wd, am)
    s.set_orbitals(U)
    steps = 5
    s.iterate(steps)
    Eg, _ = s.history()
    ref = O.run(U.astype(np.float64), vext, cfg, steps)
    Eo = np.array([h.energy for h in ref.history])
    np.testing.assert_allclose(Eg[:steps], Eo[:steps], rtol=2e-6)
    W = s.get_orbitals().astype(np.float64)
    e = s.energy()["total"]
    assert abs(O.energy(W, vext, cfg) - e) <= 1e-7 * abs(e)
    s.close()


def test_resume_with_projectors_is_bit_exact(P):
    w, cfg, vext, U0, a = _l10_with_projectors(P, P.FP64)
    a.set_orbitals(U0)
    a.iterate(30)
    blob = a.get_state()
    a.iterate(20)
    Ea, _ = a.history()
    _, _, _, _, b = _l10_with_projectors(P, P.FP64)
    b.set_state(blob)
    b.iterate(20)
    Eb, _ = b.history()
    assert np.array_equal(Ea, Eb)
    a.close()
    b.close()


def test_projector_arguments(P):
    s = P.Solver(16, 6.0, 2, solver=1)
    with pytest.raises(P.PouError):
        s.set_projectors([[1.0, 1.0, 1.0]], [0.8], [1.0])
    s.close()
    s = P.Solver(16, 6.0, 2)
    with pytest.raises(P.PouError):
        s.set_projectors([[1.0, 1.0, 1.0]], [0.0], [1.0])
    with pytest.raises(P.PouError):
        s.set_projectors(np.zeros((257, 3)), np.ones(257), np.ones(257))
    s.set_projectors(np.zeros((0, 3)), [], [])  # removes them
    s.close()
