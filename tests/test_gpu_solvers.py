"""Per-orbital step sizes and the conjugate-gradient subproblem solver, through the C-ABI.

tau_mode = 1: each orbital takes its own Barzilai-Borwein step tau_i (the
tau_i of Sec. 3.2), all scaled by delta^s when backtracking.  solver = 1:
conjugate-gradient directions with each orbital's Newton step along them (one
of the solvers Sec. 3.1 lists).  The oracle restates both
(``pou_oracle.Config(tau_mode=1)`` and ``Config(solver=1)``).

Step-by-step comparison horizons, from the oracle against itself with U0
perturbed by 1e-15: per-orbital BB steps agree to 7e-12 Ha over 40 steps (they
are chaotic like every BB iteration); the Newton steps of the CG solver are not
chaotic (5e-12 Ha over 160 steps), so 100 steps are compared.
"""
import json
import os

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


def _golden(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", "converged_energies.json")) as f:
        return json.load(f)[name]["E_converged"]


MODES = {"tau_i": ({"tau_mode": 1}, 40), "cg": ({"solver": 1}, 100)}


@pytest.mark.parametrize("mode", list(MODES))
def test_fp64_trajectory_matches_oracle(P, mode):
    kw, steps = MODES[mode]
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N, **kw)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    ref = O.run(U0, vext, cfg, steps)
    Eo = np.array([h.energy for h in ref.history])
    to = np.array([h.tau for h in ref.history])
    s = P.Solver(w.n, w.L, w.N, order=w.order, precision=P.FP64, **kw)
    s.set_atoms(R, Z, w.width)
    s.set_orbitals(U0)
    rep = s.iterate(steps)
    assert rep["iterations"] == steps
    E, tau = s.history()
    assert np.max(np.abs(E - Eo)) < 1e-9
    np.testing.assert_allclose(tau, to, rtol=1e-6)
    W = s.get_orbitals()
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(w.N))) < 1e-12
    s.close()


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_reaches_the_minimum(P, mode, precision, tol):
    kw, _ = MODES[mode]
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    s = P.Solver(w.n, w.L, w.N, order=w.order, precision=precision, **kw)
    s.set_atoms(R, Z, w.width)
    s.set_orbitals(U0)
    s.iterate(4000)
    e = s.energy()["total"]
    Estar = _golden("l10_g32_n4")
    assert abs(e - Estar) <= tol, (e, Estar)
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N)
    W = s.get_orbitals()
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(w.N))) < (1e-12 if precision == 0 else 1e-7)
    s.close()


@pytest.mark.parametrize("mode", list(MODES))
def test_mixed_n128_13pt_first_steps(P, mode):
    """The bench's kernel configuration (mixed form, N = 128, 13-point
    stencil) with per-orbital steps on the tensor-core trial kernels: the first
    steps follow the oracle; the returned orbitals are orthonormal and carry
    the reported energy."""
    kw, _ = MODES[mode]
    n, L, N = 40, 16.0, 128
    R, Z = inputs.atoms(71, 32, L, "uniform26")
    U = inputs.random_orbitals(71, N, (n, n, n)).astype(np.float32)
    cfg = O.cubic(n, L, order=4, N=N, **kw)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = P.Solver(n, L, N, order=4, precision=P.FP32, **kw)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U)
    steps = 5
    s.iterate(steps)
    Eg, _ = s.history()
    ref = O.run(U.astype(np.float64), vext, cfg, steps)
    Eo = np.array([h.energy for h in ref.history])
    np.testing.assert_allclose(Eg[:steps], Eo[:steps], rtol=2e-6)
    W = s.get_orbitals().astype(np.float64)
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(N))) < 2e-6
    e = s.energy()["total"]
    assert abs(O.energy(W, vext, cfg) - e) <= 1e-7 * abs(e)
    s.close()


@pytest.mark.parametrize("mode", list(MODES))
def test_resume_is_bit_exact(P, mode):
    kw, _ = MODES[mode]
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    a = P.Solver(w.n, w.L, w.N, order=w.order, precision=P.FP64, **kw)
    a.set_atoms(R, Z, w.width)
    a.set_orbitals(U0)
    a.iterate(25)
    blob = a.get_state()
    a.iterate(15)
    Ea, _ = a.history()
    b = P.Solver(w.n, w.L, w.N, order=w.order, precision=P.FP64, **kw)
    b.set_atoms(R, Z, w.width)
    b.set_state(blob)
    b.iterate(15)
    Eb, _ = b.history()
    assert np.array_equal(Ea, Eb)
    a.close()
    b.close()


def test_invalid_combinations(P):
    for kw in ({"tau_mode": 1, "solver": 1}, {"tau_mode": 1, "direction": 1}, {"solver": 1, "n_diag": 10},
               {"solver": 1, "n_org": 2}, {"tau_mode": 2}, {"solver": 2}):
        with pytest.raises(P.PouError):
            P.Solver(16, 6.0, 2, **kw)
