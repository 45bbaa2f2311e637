"""GPU-vs-oracle parity for every step of the hot path, through the C-ABI.

Tolerances.  FP64 form: the kernels reorder FP64 sums, so results agree to a
few ulps times the condition of each quantity; energies to 1e-8 Ha over a
200-step trajectory (the target bound).  FP32 form: inputs are rounded to
FP32 first and the oracle runs on the rounded values, so the remaining error
is FP32 arithmetic (2^-24 relative per operation, random sign, summed in FP64
at the block level): 1e-5 relative for pointwise fields, 1e-6 Ha for energies.
"""
import math

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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def ocfg(n, L, N, order=2, hartree=1, exchange=1, **kw):
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    L = (L, L, L) if np.isscalar(L) else tuple(L)
    return O.Config(n=n, L=L, order=order, N=N, hartree=hartree, exchange=exchange, **kw)


def solver(P, n, L, N, order=2, precision=0, **kw):
    return P.Solver(n, L, N, order=order, precision=precision, **kw)


# ------------------------------------------------------------------ a3: Gram
@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("N,ng", [(1, 37), (5, 2160), (64, 20000), (100, 50000), (128, 4099)])
def test_gram_op(P, dt, N, ng):
    rng = np.random.default_rng(N * 7 + ng)
    A = rng.standard_normal((N, ng))
    tdt = torch.float64 if dt == "f64" else torch.float32
    Ad = dev(A, tdt)
    code = P.DT_F64 if dt == "f64" else P.DT_F32
    ws = torch.empty(P.gram_workspace_bytes(code, ng, N) // 8 + 1, dtype=torch.float64, device="cuda")
    S = torch.empty((N, N), dtype=torch.float64, device="cuda")
    dV = 0.37
    P.gram(Ad, dV, S, ws)
    Ar = Ad.double().cpu().numpy()
    ref = dV * Ar @ Ar.T
    scale = dV * np.sqrt(np.outer(np.sum(Ar * Ar, 1), np.sum(Ar * Ar, 1)))
    err = np.max(np.abs(S.cpu().numpy() - ref) / scale)
    assert err < (1e-13 if dt == "f64" else 2e-6), err


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("N,ng", [(16, 40000), (128, 160 ** 3 // 8)])
def test_gram_op_coherent_sums(P, dt, N, ng):
    # rows sharing one positive component: every off-diagonal entry is a sum
    # of products of one sign, the case where a biased accumulation shows
    rng = np.random.default_rng(N + 3 * ng)
    A = 1.0 + 0.3 * rng.standard_normal((N, ng)) + 0.2 * rng.random((N, 1))
    tdt = torch.float64 if dt == "f64" else torch.float32
    Ad = dev(A, tdt)
    code = P.DT_F64 if dt == "f64" else P.DT_F32
    ws = torch.empty(P.gram_workspace_bytes(code, ng, N) // 8 + 1, dtype=torch.float64, device="cuda")
    S = torch.empty((N, N), dtype=torch.float64, device="cuda")
    P.gram(Ad, 1.0 / ng, S, ws)
    Ar = Ad.double().cpu().numpy()
    ref = (Ar @ Ar.T) / ng
    err = np.max(np.abs(S.cpu().numpy() - ref) / np.abs(ref))
    assert err < (1e-13 if dt == "f64" else 1e-6), err
    d = np.abs(np.diag(S.cpu().numpy()) - np.diag(ref)) / np.diag(ref)
    assert np.max(d) < (1e-13 if dt == "f64" else 1e-9), np.max(d)


# ------------------------------------------------------------------ a4: Cholesky / inverse
@pytest.mark.parametrize("N", [1, 7, 64, 100, 128])
def test_cholinv_op(P, N):
    rng = np.random.default_rng(N)
    B = rng.standard_normal((N, N)) * 0.1
    S = np.eye(N) + B @ B.T
    Sd = dev(S)
    Rinv = torch.empty_like(Sd)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.cholinv(Sd, Rinv, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    import scipy.linalg as sl
    R = sl.cholesky(S, lower=False)
    np.testing.assert_allclose(Rinv.cpu().numpy(), np.linalg.inv(R), atol=1e-12 * np.linalg.cond(R))
    np.testing.assert_allclose(np.tril(Rinv.cpu().numpy(), -1), 0.0)


def test_cholinv_reports_non_spd(P):
    N = 6
    S = np.eye(N)
    S[3, 3] = -1.0
    Rinv = torch.empty((N, N), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.cholinv(dev(S), Rinv, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 4


# ------------------------------------------------------------------ a5: rotation + density
@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("N,ng", [(1, 100), (5, 2160), (64, 6000), (128, 4099)])
def test_rotate_op(P, dt, N, ng):
    rng = np.random.default_rng(N + ng)
    A = rng.standard_normal((N, ng))
    Bm = rng.standard_normal((N, N)) * 0.05
    R = np.linalg.cholesky(np.eye(N) + Bm @ Bm.T).T
    Rinv = np.linalg.inv(R)
    tdt = torch.float64 if dt == "f64" else torch.float32
    Ad = dev(A, tdt)
    Bd = torch.empty_like(Ad)
    rho = torch.empty(ng, dtype=torch.float64, device="cuda")
    P.rotate(Ad, dev(Rinv), Bd, rho)
    Ar = Ad.double().cpu().numpy()
    ref = Rinv.T @ Ar  # rows of A Rinv (columns)
    tol = 1e-12 if dt == "f64" else 3e-6
    np.testing.assert_allclose(Bd.double().cpu().numpy(), ref, atol=tol * np.max(np.abs(ref)))
    np.testing.assert_allclose(rho.cpu().numpy(), 2.0 * np.sum(ref * ref, 0), rtol=tol * 10, atol=tol)


@pytest.mark.parametrize("N,ng", [(128, 64 * 1000), (37, 64 * 300 + 11)])
def test_rotate_op_off_diagonal_sum_is_unbiased(P, N, ng):
    # positive block and positive off-diagonal R^-1: every output's
    # off-diagonal sum has terms of one sign, so a rounding that always goes
    # one way (such as a truncating accumulator) shows as a mean error
    rng = np.random.default_rng(5 * N + ng)
    A = 1.0 + 0.25 * rng.random((N, ng))
    Rinv = np.triu(0.02 * rng.random((N, N)), 1) + np.eye(N)
    Ad = dev(A, torch.float32)
    Bd = torch.empty_like(Ad)
    rho = torch.empty(ng, dtype=torch.float64, device="cuda")
    P.rotate(Ad, dev(Rinv), Bd, rho)
    Ar = Ad.double().cpu().numpy()
    ref = Rinv.T @ Ar
    off = (Rinv - np.diag(np.diag(Rinv))).T @ Ar
    got = Bd.double().cpu().numpy()
    rows = np.arange(1, N)  # row 0 has no off-diagonal part
    bias = np.mean(got[rows] - ref[rows]) / np.mean(off[rows])
    spread = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print("rotation off-diagonal bias", bias, "max rel err", spread)
    assert abs(bias) < 3e-7, bias
    assert spread < 3e-7, spread
    np.testing.assert_allclose(rho.cpu().numpy(), 2.0 * np.sum(ref * ref, 0), rtol=1e-6)


# ------------------------------------------------------------------ N > 128 (FP32 form)
@pytest.mark.parametrize("N,ng", [(129, 4099), (256, 20000), (300, 6001), (512, 9000)])
def test_gram_op_block_pairs(P, N, ng):
    """Tensor-core Gram over 128 x 128 block pairs: ragged last block, odd Ng."""
    rng = np.random.default_rng(N * 11 + ng)
    A = rng.standard_normal((N, ng))
    Ad = dev(A, torch.float32)
    ws = torch.empty(P.gram_workspace_bytes(P.DT_F32, ng, N) // 8 + 1, dtype=torch.float64, device="cuda")
    S = torch.empty((N, N), dtype=torch.float64, device="cuda")
    dV = 0.21
    P.gram(Ad, dV, S, ws)
    Ar = Ad.double().cpu().numpy()
    ref = dV * Ar @ Ar.T
    scale = dV * np.sqrt(np.outer(np.sum(Ar * Ar, 1), np.sum(Ar * Ar, 1)))
    Sg = S.cpu().numpy()
    assert np.max(np.abs(Sg - ref) / scale) < 2e-6
    assert np.array_equal(Sg, Sg.T)


def test_gram_op_block_pairs_coherent_sums(P):
    N, ng = 384, 40000
    rng = np.random.default_rng(17)
    A = 1.0 + 0.3 * rng.standard_normal((N, ng)) + 0.2 * rng.random((N, 1))
    Ad = dev(A, torch.float32)
    ws = torch.empty(P.gram_workspace_bytes(P.DT_F32, ng, N) // 8 + 1, dtype=torch.float64, device="cuda")
    S = torch.empty((N, N), dtype=torch.float64, device="cuda")
    P.gram(Ad, 1.0 / ng, S, ws)
    Ar = Ad.double().cpu().numpy()
    ref = (Ar @ Ar.T) / ng
    err = (S.cpu().numpy() - ref) / np.abs(ref)
    assert np.max(np.abs(err)) < 1e-6, np.max(np.abs(err))
    # the tensor core truncates at each of the 12-16 accumulations of a
    # promotion period (64 points): a mean error of about -3e-7 of these
    # coherent sums, the same on diagonal and off-diagonal blocks
    assert abs(np.mean(err)) < 5e-7, np.mean(err)


@pytest.mark.parametrize("N", [129, 200, 512])
def test_cholinv_op_large(P, N):
    rng = np.random.default_rng(N)
    B = rng.standard_normal((N, N)) * 0.05
    S = np.eye(N) + B @ B.T
    Rinv = torch.empty((N, N), dtype=torch.float64, device="cuda")
    info = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    P.cholinv(dev(S), Rinv, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    import scipy.linalg as sl
    R = sl.cholesky(S, lower=False)
    np.testing.assert_allclose(Rinv.cpu().numpy(), np.linalg.inv(R), atol=1e-12 * np.linalg.cond(R))
    np.testing.assert_allclose(np.tril(Rinv.cpu().numpy(), -1), 0.0)


def test_cholinv_op_large_reports_non_spd(P):
    N = 300
    S = np.eye(N)
    S[250, 250] = -1.0
    Rinv = torch.empty((N, N), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    P.cholinv(dev(S), Rinv, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 251


@pytest.mark.parametrize("N,ng", [(129, 4099), (256, 6000), (300, 2561), (512, 4096)])
def test_rotate_op_large(P, N, ng):
    """Chunked tensor-core rotation: output chunks of 128, R^-1 streamed per atom."""
    rng = np.random.default_rng(N * 3 + ng)
    A = rng.standard_normal((N, ng))
    Bm = rng.standard_normal((N, N)) * 0.03
    R = np.linalg.cholesky(np.eye(N) + Bm @ Bm.T).T
    Rinv = np.linalg.inv(R)
    Ad = dev(A, torch.float32)
    Bd = torch.empty_like(Ad)
    rho = torch.empty(ng, dtype=torch.float64, device="cuda")
    P.rotate(Ad, dev(Rinv), Bd, rho)
    Ar = Ad.double().cpu().numpy()
    ref = Rinv.T @ Ar
    np.testing.assert_allclose(Bd.double().cpu().numpy(), ref, atol=3e-6 * np.max(np.abs(ref)))
    np.testing.assert_allclose(rho.cpu().numpy(), 2.0 * np.sum(ref * ref, 0), rtol=3e-5, atol=3e-6)


def test_rotate_op_fp64_large_n_is_einval(P):
    N, ng = 200, 1000
    A = torch.zeros((N, ng), dtype=torch.float64, device="cuda")
    with pytest.raises(P.PouError):
        P.rotate(A, torch.eye(N, dtype=torch.float64, device="cuda"), torch.empty_like(A))


def _large_n_system(N):
    n, L = (16, 16, 18), (6.0, 6.0, 7.0)
    R, Z, _ = _system(n, L, 1, 23, M=3)
    U = inputs.random_orbitals(29, N, n)
    return n, L, R, Z, U


def test_iteration_large_n_fp32(P):
    """N = 192 (two 128-row blocks, the chunked rotation and the multi-kernel
    Cholesky inside the iteration): the first steps follow the FP64 oracle's
    trajectory, and the energy and density the library reports are those of
    the FP32 orbitals it returns, which stay orthonormal."""
    N = 192
    n, L, R, Z, U = _large_n_system(N)
    cfg = ocfg(n, L, N)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = solver(P, n, L, N, precision=1)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U.astype(np.float32))
    s.iterate(6)
    Eg, _ = s.history()
    st = O.run(U.astype(np.float32).astype(np.float64), vext, cfg, 6)
    Eo = np.array([h.energy for h in st.history])
    np.testing.assert_allclose(Eg[:len(Eo)], Eo[:len(Eg)], rtol=2e-6)
    s.iterate(40)
    W = s.get_orbitals()
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(N))) < 2e-6
    e = s.energy()["total"]
    assert abs(O.energy(W, vext, cfg) - e) < 1e-7 * abs(e)
    np.testing.assert_allclose(s.get_density(), O.density(W), rtol=1e-6, atol=1e-9)
    E, _ = s.history()
    assert np.all(np.isfinite(E)) and E[-1] < E[5]
    # residual norm of Eq. (gra) over two 128-orbital blocks of Sigma
    HW = O.apply_h(W, O.total_potential(O.density(W), vext, cfg), cfg)
    ref = O.gradient_residual(W, HW, cfg)
    assert abs(s.gradient_norm() - ref) <= 3e-3 * ref + 2e-5
    s.close()


def test_iteration_large_n_single_tf32(P):
    """POU_FP32_TF32 with N = 192 (two 128-row blocks: the single TF32
    product on the diagonal and the off-diagonal block pairs of the
    tensor-core Gram): the first steps follow the FP64 oracle to the form's
    averaged rounding, the orbitals stay orthonormal to it and carry the
    reported energy."""
    N = 192
    n, L, R, Z, U = _large_n_system(N)
    cfg = ocfg(n, L, N)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = solver(P, n, L, N, precision=P.FP32_TF32)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U.astype(np.float32))
    s.iterate(6)
    Eg, _ = s.history()
    st = O.run(U.astype(np.float32).astype(np.float64), vext, cfg, 6)
    Eo = np.array([h.energy for h in st.history])
    np.testing.assert_allclose(Eg[:len(Eo)], Eo[:len(Eg)], rtol=1e-5)
    W = s.get_orbitals().astype(np.float64)
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(N))) < 2e-5
    e = s.energy()["total"]
    assert abs(O.energy(W, vext, cfg) - e) <= 1e-6 * abs(e)
    s.close()


def test_large_n_fp64_form_is_einval(P):
    with pytest.raises(P.PouError):
        solver(P, (16, 16, 18), (6.0, 6.0, 7.0), 192, precision=0)
    with pytest.raises(P.PouError):
        solver(P, (16, 16, 18), (6.0, 6.0, 7.0), 192, precision=1, n_diag=50)
    with pytest.raises(P.PouError):
        solver(P, (16, 16, 18), (6.0, 6.0, 7.0), 192, precision=2, n_diag=50)


def test_full_size_160_energy_and_h_apply(P):
    """The bench's workload at full size (160^3 grid, N = 128, 13-point
    stencil, mixed form): the energy terms of an orthonormal block and
    H(rho) W on sampled orbitals (through the adjoint, dE/dU = 2 f dV H U)
    against the oracle.  The oracle orthonormalises the seeded start in FP64;
    both sides then work on the same FP32-rounded block."""
    w, R, Z, U0 = inputs.workload_inputs("l30_g160_n128")
    cfg = ocfg(w.n, w.L, w.N, order=w.order)
    W, _, _ = O.cholesky_qr(U0, cfg)
    del U0
    W = np.ascontiguousarray(W.astype(np.float32).astype(np.float64))
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    s = solver(P, w.n, w.L, w.N, order=w.order, precision=1)
    s.set_atoms(R, Z, w.width)
    got = s.evaluate(W)
    ref = O.energy_terms(W, vext, cfg)
    for k in ("kinetic", "external", "hartree", "exchange"):
        assert abs(got[k] - getattr(ref, k)) <= 2e-6 * max(1.0, abs(getattr(ref, k))), k
    out = np.empty(W.shape)
    s.backward(W, 1.0 / (2 * O.F_OCC * cfg.dV), out)
    idx = [0, 77, 127]
    ref_h = O.apply_h(W[idx], O.total_potential(O.density(W), vext, cfg), cfg)
    np.testing.assert_allclose(out[idx].astype(np.float64), ref_h, atol=2e-5 * np.max(np.abs(ref_h)))
    s.close()


@pytest.mark.parametrize("n,L", [((40, 40, 40), (16.0, 16.0, 16.0)), ((64, 64, 32), (24.0, 24.0, 12.0))])
def test_bench_kernel_configuration_mixed_n128_13pt(P, n, L):
    """The launch configuration the bench times (mixed form, N = 128, 13-point
    stencil: the tensor-core trial Gram over one 128 x 128 block, the
    tensor-core rotation with all four 32-orbital atoms of R^-1, the one-CTA
    Cholesky) on grids the oracle steps through in seconds, with equal
    spacings in the three directions as on the 160^3 workload (one kinetic
    sum): 64 x 64 x 32 tiles exactly like 160^3 (whole 32 x 16 tiles), 40^3
    leaves ragged tiles.  The first steps follow the FP64 oracle's
    trajectory from the same FP32-rounded start (on 40^3 at least one of them
    takes the second Cholesky-QR pass); the returned orbitals are
    orthonormal, and the energy, density and residual norm the library
    reports are those the oracle computes from them."""
    N = 128
    R, Z = inputs.atoms(71, 32, L[0], "uniform26")
    R[:, 2] *= L[2] / L[0]
    U = inputs.random_orbitals(71, N, n).astype(np.float32)
    cfg = ocfg(n, L, N, order=4)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = solver(P, n, L, N, order=4, precision=1)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U)
    steps = 8
    rep = s.iterate(steps)
    assert rep["iterations"] == steps
    if n[0] == 40:
        assert rep["second_passes"] >= 1
    Eg, _ = s.history()
    st = O.run(U.astype(np.float64), vext, cfg, steps)
    Eo = np.array([h.energy for h in st.history])
    np.testing.assert_allclose(Eg[:steps], Eo[:steps], rtol=2e-6)
    W = s.get_orbitals().astype(np.float64)
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(N))) < 2e-6
    e = s.energy()
    ref = O.energy_terms(W, vext, cfg)
    assert abs(ref.total - e["total"]) <= 1e-7 * abs(ref.total)
    for k in ("kinetic", "external", "hartree", "exchange"):
        assert abs(e[k] - getattr(ref, k)) <= 2e-7 * max(1.0, abs(getattr(ref, k))), k
    np.testing.assert_allclose(s.get_density(), O.density(W), rtol=1e-6, atol=1e-9)
    HW = O.apply_h(W, O.total_potential(O.density(W), vext, cfg), cfg)
    g_ref = O.gradient_residual(W, HW, cfg)
    assert abs(s.gradient_norm() - g_ref) <= 3e-3 * g_ref + 2e-5
    s.close()


@pytest.mark.parametrize("order", [2, 4])
def test_mixed_trajectory_non_cubic_grid(P, order):
    """The mixed form on a grid with three different spacings (the FP32
    H-apply keeps per-axis kinetic sums, the step's Barzilai-Borwein terms
    included): the first steps follow the oracle."""
    n, L, N = (64, 32, 16), (12.0, 7.0, 3.5), 8
    R, Z, U = _system(n, L, N, 21, M=3)
    U = U.astype(np.float32)
    cfg = ocfg(n, L, N, order=order)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = solver(P, n, L, N, order=order, precision=1)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U)
    steps = 8
    s.iterate(steps)
    Eg, tg = s.history()
    st = O.run(U.astype(np.float64), vext, cfg, steps)
    Eo = np.array([h.energy for h in st.history])
    np.testing.assert_allclose(Eg[:steps], Eo[:steps], rtol=2e-6)
    W = s.get_orbitals().astype(np.float64)
    e = s.energy()["total"]
    assert abs(O.energy(W, vext, cfg) - e) <= 1e-7 * abs(e)
    s.close()


def test_full_size_160_reported_energy_after_200_steps(P):
    """The bench's workload (160^3, N = 128, 13-point, mixed form) after the
    200 steps the bench takes before timing: the energy the library reports
    is the oracle's energy of the orbitals it returns, which are orthonormal
    (checked on a sample of 16 orbitals against the whole block)."""
    w, R, Z, U0 = inputs.workload_inputs("l30_g160_n128")
    cfg = ocfg(w.n, w.L, w.N, order=w.order)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    s = solver(P, w.n, w.L, w.N, order=w.order, precision=1)
    s.set_atoms(R, Z, w.width)
    s.set_orbitals(U0)
    del U0
    rep = s.iterate(200)
    assert rep["iterations"] == 200
    W = s.get_orbitals().astype(np.float64)
    e = s.energy()["total"]
    s.close()
    idx = np.arange(0, w.N, 8)
    G = cfg.dV * (W[idx].reshape(len(idx), -1) @ W.reshape(w.N, -1).T)
    G[np.arange(len(idx)), idx] -= 1.0
    assert np.max(np.abs(G)) < 2e-6
    ref = O.energy(W, vext, cfg)
    assert abs(ref - e) <= 1e-6 * abs(ref), (ref, e)


def test_full_size_512_orbitals(P):
    """The 192^3 grid with N = 512 (14.5 GB per FP32 block), in the launch
    configuration the bench times: properties that hold at any size, checked
    with plain PyTorch FP64 on the returned orbitals (the oracle cannot run
    at this size): orthonormality of the whole block, the density at sampled
    points, and an energy that goes down."""
    w, R, Z, U0 = inputs.workload_inputs("l40_g192_n512")
    s = solver(P, w.n, w.L, w.N, order=w.order, precision=1, bb_variant=3)
    s.set_atoms(R, Z, w.width)
    s.set_orbitals(U0)
    del U0
    E0 = s.energy()["total"]
    rep = s.iterate(4)
    assert rep["status"] == P.OK and rep["iterations"] == 4
    E, _ = s.history()
    assert np.all(np.isfinite(E)) and E[-1] < E0
    ng = w.n ** 3
    dV = (w.L / w.n) ** 3
    W = torch.empty((w.N, ng), dtype=torch.float32, device="cuda")
    s.get_orbitals(W)
    G = torch.zeros((w.N, w.N), dtype=torch.float64, device="cuda")
    for a in range(0, ng, 1 << 20):
        Wc = W[:, a:a + (1 << 20)].double()
        G += Wc @ Wc.T
        del Wc
    G *= dV
    ortho = (G - torch.eye(w.N, dtype=torch.float64, device="cuda")).abs().max().item()
    assert ortho < 2e-6, ortho
    rho = s.get_density()
    idx = np.random.default_rng(3).choice(ng, 4096, replace=False)
    Ws = W[:, torch.as_tensor(idx, device="cuda")].double()
    ref = (2.0 * (Ws * Ws).sum(0)).cpu().numpy()
    np.testing.assert_allclose(rho.reshape(-1)[idx], ref, rtol=1e-6)
    s.close()


# ------------------------------------------------------------------ a6: Hartree
@pytest.mark.parametrize("n,L", [((20, 12, 15), (7.0, 5.0, 6.0)), ((32, 32, 32), (10.0,) * 3),
                                 ((16, 10, 9), (4.0, 3.0, 3.3)), ((96, 6, 5), (20.0, 2.0, 2.0))])
def test_hartree_op(P, n, L):
    cfg = ocfg(n, L, 1)
    rho = inputs.random_field(sum(n), n, 0.0, 1.0)
    ref = O.hartree_potential(rho, cfg)
    rd = dev(rho)
    vh = torch.empty_like(rd)
    ws = torch.empty(P.hartree_workspace_bytes(n) // 8, dtype=torch.float64, device="cuda")
    P.hartree(n, L, rd, vh, ws)
    np.testing.assert_allclose(vh.cpu().numpy(), ref, atol=1e-12 * np.max(np.abs(ref)))


# ------------------------------------------------------------------ a1, a7: evaluation
def _system(n, L, N, seed, M=2):
    cfg = ocfg(n, L, N)
    Lv = cfg.L
    R = np.array([[0.3 * Lv[0], 0.4 * Lv[1], 0.6 * Lv[2]], [0.75 * Lv[0], 0.2 * Lv[1], 0.1 * Lv[2]],
                  [0.5 * Lv[0], 0.9 * Lv[1], 0.45 * Lv[2]]])[:M]
    Z = np.array([3.0, 2.0, 4.0])[:M]
    U = inputs.random_orbitals(seed, N, cfg.n)
    return R, Z, U


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order", [2, 4])
def test_evaluate_energy_terms(P, precision, order):
    n, L, N = (20, 12, 10), (7.0, 5.0, 4.5), 3
    R, Z, U = _system(n, L, N, 5)
    if precision == 1:
        U = U.astype(np.float32).astype(np.float64)
    cfg = ocfg(n, L, N, order=order)
    s = solver(P, n, L, N, order=order, precision=precision)
    s.set_atoms(R, Z, 0.8)
    got = s.evaluate(U)
    ref = O.energy_terms(U, O.vext_gaussians(cfg, R, Z, 0.8), cfg)
    tol = 1e-11 if precision == 0 else 2e-6
    for k in ("kinetic", "external", "hartree", "exchange"):
        assert abs(got[k] - getattr(ref, k)) <= tol * max(1.0, abs(getattr(ref, k))), k
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order,n", [(2, (20, 12, 10)), (4, (20, 12, 10)), (4, (5, 6, 8)), (2, (27, 9, 4)),
                                     (4, (64, 32, 12)), (2, (32, 48, 5)), (4, (32, 16, 3)), (4, (18, 12, 10))])
def test_apply_h_through_adjoint(P, precision, order, n):
    """a1: HW = -1/2 Lap_h W + V W, read through dE/dU = 2 f dV H U with g = 1/(2 f dV).
    The grids cover whole and ragged 32 x 16 tiles of the FP32 kernel, nx
    even but not a multiple of 4 (the paired kernel), odd nx (the scalar
    kernel) and fewer planes than the stencil's reach in z."""
    L, N = (6.0, 5.0, 4.0), 2
    R, Z, U = _system(n, L, N, 9)
    if precision == 1:
        U = U.astype(np.float32).astype(np.float64)
    cfg = ocfg(n, L, N, order=order)
    s = solver(P, n, L, N, order=order, precision=precision)
    s.set_atoms(R, Z, 0.8)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    tdt = torch.float64 if precision == 0 else torch.float32
    Ud = dev(U, tdt)
    out = torch.empty_like(Ud)
    g = 1.0 / (2 * O.F_OCC * cfg.dV)
    s.backward(Ud, g, out)
    ref = O.apply_h(U, O.total_potential(O.density(U), vext, cfg), cfg)
    tol = 1e-11 if precision == 0 else 2e-5
    np.testing.assert_allclose(out.double().cpu().numpy(), ref, atol=tol * np.max(np.abs(ref)))
    s.close()


@pytest.mark.parametrize("offset_in,offset_out", [(1, 0), (0, 1), (1, 1), (2, 2)])
def test_apply_h_unaligned_caller_blocks(P, offset_in, offset_out):
    """A caller's FP32 block or output that starts off the 16-byte boundary
    (a view into a larger buffer) takes a kernel whose accesses it allows;
    the result is the oracle's either way."""
    n, L, N, order = (32, 16, 12), (6.0, 5.0, 4.0), 3, 4
    R, Z, U = _system(n, L, N, 9)
    U = U.astype(np.float32).astype(np.float64)
    cfg = ocfg(n, L, N, order=order)
    s = solver(P, n, L, N, order=order, precision=1)
    s.set_atoms(R, Z, 0.8)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    size = U.size
    bufu = torch.zeros(size + 4, dtype=torch.float32, device="cuda")
    bufo = torch.zeros(size + 4, dtype=torch.float32, device="cuda")
    Ud = bufu[offset_in:offset_in + size].view(U.shape)
    Ud.copy_(dev(U, torch.float32))
    out = bufo[offset_out:offset_out + size].view(U.shape)
    g = 1.0 / (2 * O.F_OCC * cfg.dV)
    s.backward(Ud, g, out)
    ref = O.apply_h(U, O.total_potential(O.density(U), vext, cfg), cfg)
    np.testing.assert_allclose(out.double().cpu().numpy(), ref, atol=2e-5 * np.max(np.abs(ref)))
    # the energy of the same block through the same kernels
    e = s.evaluate(Ud)
    refE = O.energy_terms(U, vext, cfg)
    assert abs(e["kinetic"] - refE.kinetic) <= 2e-6 * abs(refE.kinetic)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_set_orbitals_orthonormalises(P, precision):
    n, L, N = (24, 20, 16), (8.0, 7.0, 6.0), 5
    R, Z, U = _system(n, L, N, 3, M=3)
    cfg = ocfg(n, L, N)
    s = solver(P, n, L, N, precision=precision)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U if precision == 0 else U.astype(np.float32))
    Uin = U if precision == 0 else U.astype(np.float32).astype(np.float64)
    W, _, _ = O.cholesky_qr(Uin, cfg)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    tol = 1e-11 if precision == 0 else 3e-6
    got = s.get_orbitals()
    np.testing.assert_allclose(got, W, atol=tol * np.max(np.abs(W)))
    rho = O.density(W)
    np.testing.assert_allclose(s.get_density(), rho, atol=tol * np.max(rho))
    Vref = O.total_potential(rho, vext, cfg)
    np.testing.assert_allclose(s.get_potential(), Vref, atol=tol * np.max(np.abs(Vref)))
    e = s.energy()
    # the reported energy is that of the returned orbitals
    ref = O.energy(got, vext, cfg)
    assert abs(e["total"] - ref) < (1e-10 if precision == 0 else 1e-8) * max(1.0, abs(ref))
    s.close()


# ------------------------------------------------------------------ whole iteration, FP64
def _workload_solver(P, name, precision=0, **kw):
    w, R, Z, U0 = inputs.workload_inputs(name)
    s = solver(P, w.n, w.L, w.N, order=w.order, precision=precision, **kw)
    s.set_atoms(R, Z, w.width)
    return w, R, Z, U0, s


def test_fp64_trajectory_matches_oracle_l10_g32_n4(P):
    """Workload L=10, 32^3, N=4, FP64: the same trajectory as the oracle.

    The Barzilai-Borwein iteration amplifies rounding differences: a 1e-15
    relative perturbation of U0 changes the oracle's own energies by more
    than 1e-8 after about 120 steps (test_bb_trajectory_is_chaotic pins this).
    So energies are compared step by step over the first 80 steps (1e-9 Ha,
    where a 1e-15 perturbation stays below 1e-10), and the 200 steps of the
    workload are checked for validity: every accepted step satisfies Eq.
    (ene-de) and the iterate stays orthonormal.
    """
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4")
    s.set_orbitals(U0)
    rep = s.iterate(w.iterations)
    assert rep["iterations"] == w.iterations
    Eg, taug = s.history()
    cfg = ocfg(w.n, w.L, w.N, order=w.order)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    st = O.run(U0, vext, cfg, 80)
    Eo = np.array([h.energy for h in st.history])
    to = np.array([h.tau for h in st.history])
    assert np.max(np.abs(Eg[:80] - Eo)) <= 1e-9, np.max(np.abs(Eg[:80] - Eo))
    np.testing.assert_allclose(taug[:80], to, rtol=1e-6)
    # Eq. (ene-de) along the whole GPU trajectory: E^(l+1) <= C^l - rho1 tau ||Z^l||^2 < C^l
    E0 = O.energy(O.cholesky_qr(U0, cfg)[0], vext, cfg)
    C, Q = E0, 1.0
    for E in Eg:
        assert E <= C + 1e-10
        Qn = cfg.eta * Q + 1.0
        C, Q = (cfg.eta * Q * C + E) / Qn, Qn
    Wg = s.get_orbitals()
    ortho = np.max(np.abs(O.inner_matrix(Wg, Wg, cfg) - np.eye(w.N)))
    assert ortho < 1e-12, ortho
    # the energy reported is the energy of the returned orbitals, and rho is theirs
    assert abs(O.energy(Wg, vext, cfg) - Eg[-1]) < 1e-10
    np.testing.assert_allclose(s.get_density(), O.density(Wg), atol=1e-12 * np.max(O.density(Wg)))
    s.close()


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "converged_energies.json")) as f:
        return json.load(f)[name]["E_converged"]


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_converged_energy_matches_oracle_l10_g32_n4(P, precision, tol):
    """Both forms reach the oracle's converged energy (1e-8 Ha FP64, 1e-6 Ha mixed)."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", precision=precision, bb_variant=3)
    s.set_orbitals(U0)
    s.iterate(4000)
    E, _ = s.history()
    Estar = _golden("l10_g32_n4")
    e = s.energy()["total"]
    assert abs(e - Estar) <= tol, (e, Estar)
    # never below the minimum by more than the tolerance (normalisation errors
    # would show here).  The bound for single steps of the mixed form leaves
    # room for transients at large Barzilai-Borwein steps (tau ~ 10-45), where
    # the trial block is furthest from orthonormal; the last 500 steps must
    # stay within the target, where a systematic normalisation error would show.
    assert np.min(E) >= Estar - (tol if precision == 0 else 2e-6)
    if precision == 1:
        assert np.min(E[-500:]) >= Estar - tol  # no persistent dip near convergence
    W = s.get_orbitals()
    cfg = ocfg(w.n, w.L, w.N, order=w.order)
    ortho = np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(w.N)))
    assert ortho < (1e-12 if precision == 0 else 1e-7), ortho
    s.close()


def test_iterate_in_chunks_equals_one_call(P):
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4")
    s.set_orbitals(U0)
    s.iterate(30)
    s.iterate(1)
    s.iterate(19)
    E1, _ = s.history()
    s.set_orbitals(U0)
    s.iterate(50)
    E2, _ = s.history()
    assert np.array_equal(E1, E2)
    s.close()


def test_state_resume_is_bit_exact(P):
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4")
    s.set_orbitals(U0)
    s.iterate(40)
    blob = s.get_state()
    s.iterate(25)
    E_ref, _ = s.history()
    W_ref = s.get_orbitals()
    s2 = solver(P, w.n, w.L, w.N, order=w.order)
    s2.set_atoms(R, Z, w.width)
    s2.set_state(blob)
    s2.iterate(25)
    E2, _ = s2.history()
    assert np.array_equal(E_ref, E2)
    assert np.array_equal(W_ref, s2.get_orbitals())
    s.close()
    s2.close()


def test_energy_criterion_stops(P):
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", bb_variant=3)
    s.set_orbitals(U0)
    rep = s.iterate(5000, e_tol=1e-11)
    assert rep["converged"] == 1 and rep["status"] == P.OK
    assert rep["df_mean3"] < 1e-11
    s.close()


# ------------------------------------------------------------------ a10: Kohn-Sham residual
def _oracle_gradient(W, R, Z, w):
    cfg = ocfg(w.n, w.L, w.N, order=w.order)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    HW = O.apply_h(W, O.total_potential(O.density(W), vext, cfg), cfg)
    return O.gradient_residual(W, HW, cfg)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("steps", [0, 40, 400])
def test_gradient_norm_matches_oracle(P, precision, steps):
    """|HW - W Sigma|_F (Eq. gra) of the current orbitals, from random start to
    near convergence.  The oracle runs on the returned orbitals; in the FP32
    form HW is rounded to FP32 (2^-24 |HW| per point), which bounds the
    absolute error by about 1e-6 |HW|_F."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", precision=precision)
    s.set_orbitals(U0)
    if steps:
        s.iterate(steps)
    W = s.get_orbitals()
    got, ref = s.gradient_norm(), _oracle_gradient(W, R, Z, w)
    tol = 1e-9 * max(1.0, ref) if precision == 0 else 3e-3 * ref + 2e-5
    assert abs(got - ref) <= tol, (got, ref)
    s.close()


def test_gradient_norm_odd_sizes_and_128_orbitals(P):
    """Ragged point chunks (ng not a multiple of 64) and the largest block."""
    for n, N in [((5, 6, 3), 3), ((12, 10, 9), 128)]:
        L = (5.0, 4.0, 3.5)
        cfg = ocfg(n, L, N)
        R = np.array([[1.0, 1.5, 2.0]])
        Z = np.array([2.0])
        s = solver(P, n, L, N)
        s.set_atoms(R, Z, 0.8)
        s.set_orbitals(inputs.random_orbitals(7, N, cfg.n))
        W = s.get_orbitals()
        vext = O.vext_gaussians(cfg, R, Z, 0.8)
        HW = O.apply_h(W, O.total_potential(O.density(W), vext, cfg), cfg)
        ref = O.gradient_residual(W, HW, cfg)
        assert abs(s.gradient_norm() - ref) <= 1e-10 * ref
        s.close()


def test_iterate_gradient_criterion_stops(P):
    """grad_tol: iterate stops once |grad E| < tol (checked every 10 steps)."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4")
    s.set_orbitals(U0)
    rep = s.iterate(5000, grad_tol=1e-4)
    assert rep["converged"] == 2 and rep["status"] == P.OK  # 2: the gradient criterion
    assert rep["grad_norm"] < 1e-4
    g = s.gradient_norm()
    assert g < 1e-4
    assert abs(g - _oracle_gradient(s.get_orbitals(), R, Z, w)) < 1e-9
    s.close()


# ------------------------------------------------------------------ Algorithm M: subspace diagonalisation
def test_subspace_diagonalisation_fp64_matches_oracle(P):
    """n_diag = 20 (Sec. 3.3): three rotations W <- W P within the first 70 steps."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", n_diag=20)
    s.set_orbitals(U0)
    s.iterate(70)
    Eg, _ = s.history()
    cfg = ocfg(w.n, w.L, w.N, order=w.order, n_diag=20)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    st = O.run(U0, vext, cfg, 70)
    Eo = np.array([h.energy for h in st.history])
    assert np.max(np.abs(Eg - Eo)) <= 1e-9, np.max(np.abs(Eg - Eo))
    W = s.get_orbitals()
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(w.N))) < 1e-12
    s.close()


# steps inside the chaos horizon: with U0 perturbed by 1e-15 the oracle's own
# energies stay within 1e-11 for these many steps (n_org = 3: 3.7e-12 at 30
# steps, 1.3e-8 at 36; n_org = 2: 4.6e-12 at 70)
@pytest.mark.parametrize("n_org,n_diag,steps", [(2, 0, 70), (3, 0, 30), (2, 20, 70)])
def test_algorithm_m_n_org_fp64_matches_oracle(P, n_org, n_diag, steps):
    """Algorithm M with Orth every n_org steps (Sec. 3.3): the steps in
    between take W - tau Z as it is; the energies of the orthonormalised steps
    and the NaN entries of the others follow the oracle's trajectory."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", n_org=n_org, n_diag=n_diag)
    s.set_orbitals(U0)
    s.iterate(steps)
    Eg, taug = s.history()
    cfg = ocfg(w.n, w.L, w.N, order=w.order, n_org=n_org, n_diag=n_diag)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    st = O.run(U0, vext, cfg, steps)
    Eo = np.array([h.energy for h in st.history])
    assert np.array_equal(np.isnan(Eg), np.isnan(Eo))
    assert np.sum(np.isnan(Eo)) == steps - (steps + n_org - 1) // n_org
    fin = ~np.isnan(Eo)
    assert np.max(np.abs(Eg[fin] - Eo[fin])) <= 1e-9, np.max(np.abs(Eg[fin] - Eo[fin]))
    np.testing.assert_allclose(taug, np.array([h.tau for h in st.history]), rtol=1e-6)
    s.close()


def test_algorithm_m_n_org_mixed_form(P):
    """n_org = 2 in the mixed form: the orthonormalised steps reach the
    oracle's converged energy region and the returned orbitals (taken after an
    orthonormalised step) are orthonormal and carry the reported energy."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", precision=1, n_org=2)
    s.set_orbitals(U0)
    s.iterate(2001)  # step l is orthonormalised when l % 2 == 0: the last one (l = 2000) is
    E, _ = s.history()
    fin = E[~np.isnan(E)]
    assert len(fin) == 1001 and np.all(np.isfinite(fin))
    Estar = _golden("l10_g32_n4")
    assert abs(fin[-1] - Estar) < 1e-4  # the oracle is 2.0e-5 above E* after these 1000 Orth steps
    W = s.get_orbitals()
    cfg = ocfg(w.n, w.L, w.N, order=w.order)
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(w.N))) < 1e-6
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    assert abs(O.energy(W, vext, cfg) - s.energy()["total"]) < 1e-7
    s.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_algorithm_m_converged_energy(P, precision, tol):
    """Algorithm M (n_diag = 100, the paper's setting): both forms reach E*."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", precision=precision, n_diag=100)
    s.set_orbitals(U0)
    s.iterate(3000)
    E, _ = s.history()
    Estar = _golden("l10_g32_n4")
    assert abs(s.energy()["total"] - Estar) <= tol
    # single-step transients of the mixed form, see the Algorithm E test above
    assert np.min(E) >= Estar - (tol if precision == 0 else 2e-6)
    s.close()


# ------------------------------------------------------------------ a8: mixed precision
def test_mixed_form_energy_of_returned_orbitals(P):
    """The mixed form reports the energy of the FP32 orbitals it returns (FP64 oracle)."""
    w, R, Z, U0, s = _workload_solver(P, "l10_g32_n4", precision=1)
    s.set_orbitals(U0)
    s.iterate(300)
    W = s.get_orbitals()
    cfg = ocfg(w.n, w.L, w.N, order=w.order)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    assert abs(O.energy(W, vext, cfg) - s.energy()["total"]) < 1e-7
    np.testing.assert_allclose(s.get_density(), O.density(W), rtol=1e-6, atol=1e-9)
    s.close()


# ------------------------------------------------------------------ a9: adjoint and forces
@pytest.mark.parametrize("precision", [0, 1])
def test_atom_gradients_match_oracle(P, precision):
    n, L, N = (24, 20, 25), (7.0, 6.0, 6.5), 3
    R, Z, U = _system(n, L, N, 17, M=3)
    cfg = ocfg(n, L, N)
    W = np.ascontiguousarray(O.cholesky_qr(U, cfg)[0])
    if precision == 1:
        W = W.astype(np.float32).astype(np.float64)
    s = solver(P, n, L, N, precision=precision)
    s.set_atoms(R, Z, 0.8)
    _, dR, dZ = s.backward(W, 1.0, None, atoms=True)
    rR, rZ = O.energy_gradient_atoms(W, cfg, R, Z, 0.8)
    tol = 1e-10 if precision == 0 else 1e-6
    np.testing.assert_allclose(dR, rR, atol=tol * max(1.0, np.max(np.abs(rR))))
    np.testing.assert_allclose(dZ, rZ, atol=tol * max(1.0, np.max(np.abs(rZ))))
    s.close()


def test_autograd_function_matches_oracle_and_fd(P):
    from paper_1510_07230_gb300.autograd import kohn_sham_energy
    n, L, N = (16, 15, 12), (6.0, 5.5, 5.0), 2
    R, Z, U = _system(n, L, N, 23)
    cfg = ocfg(n, L, N, order=4)
    s = solver(P, n, L, N, order=4)
    Ut = dev(0.3 * U).requires_grad_(True)
    Rt = torch.tensor(R, dtype=torch.float64, requires_grad=True)
    Zt = torch.tensor(Z, dtype=torch.float64, requires_grad=True)
    E = kohn_sham_energy(Ut, Rt, Zt, s)
    E.backward()
    Un = 0.3 * U
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    assert abs(E.item() - O.energy(Un, vext, cfg)) < 1e-10
    gU = O.energy_gradient_orbitals(Un, vext, cfg)
    np.testing.assert_allclose(Ut.grad.cpu().numpy(), gU, atol=1e-11 * np.max(np.abs(gU)))
    rR, rZ = O.energy_gradient_atoms(Un, cfg, R, Z, 0.8)
    np.testing.assert_allclose(Rt.grad.numpy(), rR, atol=1e-10 * max(1, np.max(np.abs(rR))))
    np.testing.assert_allclose(Zt.grad.numpy(), rZ, atol=1e-10 * max(1, np.max(np.abs(rZ))))
    # central finite differences of the GPU energy itself (step 1e-4 bohr)
    eps = 1e-4
    for I, a in [(0, 0), (1, 2)]:
        Rp, Rm = R.copy(), R.copy()
        Rp[I, a] += eps
        Rm[I, a] -= eps
        s.set_atoms(Rp, Z, 0.8)
        ep = s.evaluate(Un)["total"]
        s.set_atoms(Rm, Z, 0.8)
        em = s.evaluate(Un)["total"]
        fd = (ep - em) / (2 * eps)
        assert abs(fd - Rt.grad[I, a].item()) < 1e-6 * max(1.0, abs(fd))
    s.close()


# ------------------------------------------------------------------ failure statuses
def test_rank_deficient_orbitals_report_not_spd(P):
    n, L, N = 12, 5.0, 3
    U = inputs.random_orbitals(1, N, (n, n, n))
    U[2] = U[0]
    s = solver(P, n, L, N)
    with pytest.raises(P.PouError) as ei:
        s.set_orbitals(U)
    assert ei.value.status == P.ENOTSPD
    s.set_orbitals(inputs.random_orbitals(2, N, (n, n, n)))  # the context stays usable
    s.iterate(3)
    s.close()


def test_nan_potential_reports_enan(P):
    n, L, N = 12, 5.0, 2
    v = np.zeros((n, n, n))
    v[3, 4, 5] = np.nan
    s = solver(P, n, L, N)
    s.set_vext(v)
    with pytest.raises(P.PouError) as ei:
        s.set_orbitals(inputs.random_orbitals(1, N, (n, n, n)))
    assert ei.value.status == P.ENAN
    s.close()


def test_iterate_without_orbitals_is_einval(P):
    s = solver(P, 12, 5.0, 2)
    with pytest.raises(P.PouError) as ei:
        s.iterate(1)
    assert ei.value.status == P.EINVAL
    s.close()


# ------------------------------------------------------------------ edge cases
def test_single_orbital_and_tiny_grid(P):
    n, L, N = (5, 4, 6), (3.0, 2.5, 3.5), 1
    R, Z, U = _system(n, L, N, 31, M=1)
    cfg = ocfg(n, L, N, order=4)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = solver(P, n, L, N, order=4)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U)
    s.iterate(40)
    st = O.run(U, vext, cfg, 40)
    Eg, _ = s.history()
    assert np.max(np.abs(Eg - np.array([h.energy for h in st.history]))) < 1e-9
    s.close()


def test_max_orbitals_128(P):
    n, L, N = (24, 24, 24), (9.0,) * 3, 128
    cfg = ocfg(n, L, N)
    R, Z = inputs.atoms(77, 8, 9.0, "uniform26")
    U = inputs.random_orbitals(77, N, cfg.n)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = solver(P, n, L, N)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U)
    s.iterate(3)
    st = O.run(U, vext, cfg, 3)
    Eg, _ = s.history()
    assert np.max(np.abs(Eg - np.array([h.energy for h in st.history]))) < 1e-8
    W = s.get_orbitals()
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(N))) < 1e-11
    s.close()


def test_device_orbitals_and_stream(P):
    """Orbitals passed as CUDA tensors, on torch's current stream."""
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    st_ptr = torch.cuda.current_stream().cuda_stream
    s = P.Solver(w.n, w.L, w.N, order=w.order, stream=st_ptr)
    s.set_atoms(R, Z, w.width)
    s.set_orbitals(dev(U0))
    s.iterate(10)
    out = torch.empty((w.N, w.n, w.n, w.n), dtype=torch.float32, device="cuda")
    s.get_orbitals(out)
    s2 = P.Solver(w.n, w.L, w.N, order=w.order)
    s2.set_atoms(R, Z, w.width)
    s2.set_orbitals(U0)
    s2.iterate(10)
    np.testing.assert_allclose(out.double().cpu().numpy(), s2.get_orbitals().astype(np.float32), atol=0)
    assert s.launch_count() > 10 * 7
    s.close()
    s2.close()


def test_single_product_tf32_gram_form(P):
    """POU_FP32_TF32 (one TF32 product in the iteration's Gram matrices) in
    the bench's kernel configuration: the first steps follow the oracle, the
    returned orbitals are orthonormal to the Gram's averaged rounding and carry
    the reported energy."""
    n, L, N = 40, 16.0, 128
    R, Z = inputs.atoms(71, 32, L, "uniform26")
    U = inputs.random_orbitals(71, N, (n, n, n)).astype(np.float32)
    cfg = ocfg(n, L, N, order=4)
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    s = solver(P, n, L, N, order=4, precision=P.FP32_TF32)
    s.set_atoms(R, Z, 0.8)
    s.set_orbitals(U)
    steps = 8
    s.iterate(steps)
    Eg, _ = s.history()
    st = O.run(U.astype(np.float64), vext, cfg, steps)
    Eo = np.array([h.energy for h in st.history])
    np.testing.assert_allclose(Eg[:steps], Eo[:steps], rtol=1e-5)
    W = s.get_orbitals().astype(np.float64)
    ortho = np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(N)))
    assert ortho < 2e-5, ortho
    e = s.energy()["total"]
    assert abs(O.energy(W, vext, cfg) - e) <= 1e-6 * abs(e)
    s.close()


def test_bounded_barrier_wait_gives_up_and_the_device_stays_usable(P):
    """A tensor-core kernel's barrier wait on an arrival that never comes
    gives up after its limit and reports it (no hang, no trap); the next
    tensor-core Gram on the same device is correct."""
    import time
    t0 = time.time()
    assert P.selftest_wait_timeout(0.05)
    assert time.time() - t0 < 30.0
    rng = np.random.default_rng(4)
    A = torch.as_tensor(rng.standard_normal((64, 5000)), dtype=torch.float32, device="cuda")
    S = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    ws = torch.empty(P.gram_workspace_bytes(P.DT_F32, 5000, 64) // 8 + 1, dtype=torch.float64, device="cuda")
    P.gram(A, 0.5, S, ws)
    Ar = A.double().cpu().numpy()
    ref = 0.5 * (Ar @ Ar.T)
    d = np.sum(Ar * Ar, 1)
    assert np.max(np.abs(S.cpu().numpy() - ref) / (0.5 * np.sqrt(np.outer(d, d)))) < 2e-6
