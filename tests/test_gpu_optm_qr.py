"""OptM-QR, the comparison method of Table 1 (Sec. 3.1), through the C-ABI.

The direction uses the full Lagrange-multiplier matrix, Z = HW - W Sigma,
Sigma = <W^T H W>, with the Barzilai-Borwein differences Y = Z - Z' of its own
directions; everything else (nonmonotone backtracking, Cholesky-QR, density
and Hartree potential) is the iteration of Algorithm E.  The oracle restates it
as ``pou_oracle.run(..., full_sigma=True)``.

Tolerances as in the Opt-Par parity tests: the FP64 trajectory step by step
over its first 80 steps (a 1e-15 perturbation of U0 moves the oracle's own
OptM-QR energies by < 1e-11 there), converged energies to 1e-8 Ha (FP64) and
1e-6 Ha (mixed), and Table 1's claim that both directions reach the same
minimum.
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


def _solver(P, w, precision, **kw):
    return P.Solver(w.n, w.L, w.N, order=w.order, precision=precision, direction=P.OPTM_QR, **kw)


def test_optm_qr_fp64_trajectory_matches_oracle(P):
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    ref = O.run(U0, vext, cfg, 80, full_sigma=True)
    Eo = np.array([h.energy for h in ref.history])
    to = np.array([h.tau for h in ref.history])
    s = _solver(P, w, P.FP64)
    s.set_atoms(R, Z, w.width)
    s.set_orbitals(U0)
    rep = s.iterate(80)
    assert rep["iterations"] == 80
    E, tau = s.history()
    assert np.max(np.abs(E - Eo)) < 1e-9
    np.testing.assert_allclose(tau, to, rtol=1e-6)
    W = s.get_orbitals()
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(w.N))) < 1e-12
    assert abs(O.energy(W, vext, cfg) - s.energy()["total"]) < 1e-10
    s.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_optm_qr_reaches_the_opt_par_minimum(P, precision, tol):
    """Table 1: Opt-Par and OptM-QR reach the same energy."""
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    s = _solver(P, w, precision)
    s.set_atoms(R, Z, w.width)
    s.set_orbitals(U0)
    s.iterate(3000)
    Estar = _golden("l10_g32_n4")
    e = s.energy()["total"]
    assert abs(e - Estar) <= tol, (e, Estar)
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N)
    W = s.get_orbitals()
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(w.N))) < (1e-12 if precision == 0 else 1e-7)
    s.close()


def test_optm_qr_mixed_n128_13pt_first_steps(P):
    """The mixed form at N = 128 with the 13-point stencil (the tensor-core
    trial Gram and rotation on w - tau z): the first steps follow the oracle's
    OptM-QR trajectory, the returned orbitals are orthonormal and carry the
    reported energy."""
    n, L, N = 40, 16.0, 128
    R, Z = inputs.atoms(71, 32, L, "uniform26")
    U = inputs.random_orbitals(71, N, (n, n, n)).astype(np.float32)
    cfg = O.cubic(n, L, order=4, N=N)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = P.Solver(n, L, N, order=4, precision=P.FP32, direction=P.OPTM_QR)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U)
    steps = 6
    s.iterate(steps)
    Eg, _ = s.history()
    ref = O.run(U.astype(np.float64), vext, cfg, steps, full_sigma=True)
    Eo = np.array([h.energy for h in ref.history])
    np.testing.assert_allclose(Eg[:steps], Eo[:steps], rtol=2e-6)
    W = s.get_orbitals().astype(np.float64)
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(N))) < 2e-6
    e = s.energy()["total"]
    assert abs(O.energy(W, vext, cfg) - e) <= 1e-7 * abs(e)
    s.close()


def test_optm_qr_resume_is_bit_exact(P):
    """Checkpoint / resume keeps the previous iterate and direction of OptM-QR."""
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    a = _solver(P, w, P.FP64)
    a.set_atoms(R, Z, w.width)
    a.set_orbitals(U0)
    a.iterate(30)
    blob = a.get_state()
    a.iterate(20)
    Ea, _ = a.history()
    b = _solver(P, w, P.FP64)
    b.set_atoms(R, Z, w.width)
    b.set_state(blob)
    b.iterate(20)
    Eb, _ = b.history()
    assert np.array_equal(Ea, Eb)
    a.close()
    b.close()


def test_optm_qr_needs_algorithm_e(P):
    for kw in ({"n_org": 2}, {"n_diag": 10}, {"direction": 2}):
        args = {"direction": P.OPTM_QR}
        args.update(kw)
        with pytest.raises(P.PouError):
            P.Solver(16, 6.0, 2, **args)
