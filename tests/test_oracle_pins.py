"""Pins of the FP64 CPU oracle against facts the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (plane-wave symbols of the stencils, the Hartree cosine, Gaussian
integrals), textbook or library routines built independently (explicit DFT
matrices, numpy QR, scipy sparse eigensolvers), brute-force finite
differences, and invariants of the method (Sec. 2-3 of the paper).
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import pou_oracle as O
from paper_1510_07230_gb300 import inputs


def _plane(cfg, m, phase=0.0):
    x, y, z = O.grid_coords(cfg)
    Lx, Ly, Lz = cfg.L
    arg = (2 * math.pi * m[0] * x[None, None, :] / Lx + 2 * math.pi * m[1] * y[None, :, None] / Ly
           + 2 * math.pi * m[2] * z[:, None, None] / Lz)
    return np.cos(arg + phase)


def _symbol(order, m, n, h):
    """Eigenvalue of -Lap_h on exp(2 pi i m x / L) for one axis (Fourier analysis)."""
    th = 2 * math.pi * m / n
    if order == 2:
        return 4.0 * math.sin(th / 2) ** 2 / h ** 2
    return (30.0 - 32.0 * math.cos(th) + 2.0 * math.cos(2 * th)) / (12.0 * h ** 2)


@pytest.mark.parametrize("order", [2, 4])
def test_laplacian_plane_wave_symbol(order):
    cfg = O.Config(n=(12, 10, 9), L=(6.0, 5.5, 4.0), order=order)
    for m in [(1, 0, 0), (0, 2, 0), (3, 1, 4), (6, 5, 4)]:
        u = _plane(cfg, m, 0.3)
        lam = sum(_symbol(order, m[a], cfg.n[a], cfg.h[a]) for a in range(3))
        np.testing.assert_allclose(-O.laplacian(u, cfg), lam * u, atol=1e-10 * lam)


@pytest.mark.parametrize("order", [2, 4])
def test_lambda_max_brute_force(order):
    cfg = O.Config(n=(4, 5, 3), L=(2.0, 2.5, 1.5), order=order)
    Ng = cfg.Ng
    A = np.zeros((Ng, Ng))
    for k in range(Ng):
        e = np.zeros(Ng)
        e[k] = 1.0
        A[:, k] = (-0.5 * O.laplacian(e.reshape(cfg.shape), cfg)).ravel()
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    # max over all discrete modes of the closed-form symbol
    best = max(0.5 * sum(_symbol(order, m[a], cfg.n[a], cfg.h[a]) for a in range(3))
               for m in itertools.product(*(range(v) for v in cfg.n)))
    assert abs(lam[-1] - best) < 1e-10 * best
    # lambda_max_kinetic is the Nyquist value, an upper bound reached for even n
    assert O.lambda_max_kinetic(cfg) >= lam[-1] - 1e-9


def test_vext_single_well_closed_form():
    L, n, w = 16.0, 32, 0.8
    cfg = O.cubic(n, L)
    R = np.array([[8.0, 8.0, 8.0]])
    V = O.vext_gaussians(cfg, R, np.array([3.0]), w)
    x, y, z = O.grid_coords(cfg)
    d2 = (z[:, None, None] - 8) ** 2 + (y[None, :, None] - 8) ** 2 + (x[None, None, :] - 8) ** 2
    np.testing.assert_allclose(V, -3.0 * np.exp(-d2 / (2 * w * w)), atol=1e-14)
    # integral of a Gaussian: -Z (2 pi w^2)^(3/2); the periodic trapezoid rule is exact here
    assert abs(cfg.dV * V.sum() + 3.0 * (2 * math.pi * w * w) ** 1.5) < 1e-10


def test_vext_periodic_images():
    cfg = O.Config(n=(20, 16, 12), L=(8.0, 7.0, 6.0))
    R = np.array([[0.1, 6.9, 3.0], [4.0, 0.2, 5.9]])
    Z = np.array([2.0, 5.0])
    V1 = O.vext_gaussians(cfg, R, Z, 0.8)
    V2 = O.vext_gaussians(cfg, R + np.array([[8.0, -7.0, 6.0], [-8.0, 7.0, -6.0]]), Z, 0.8)
    # shifting an atom by one box length changes only which images are summed (all ~1e-10 level)
    np.testing.assert_allclose(V1, V2, atol=1e-9)
    # integral: -sum Z (2 pi w^2)^(3/2), up to the far images not summed
    assert abs(cfg.dV * V1.sum() + Z.sum() * (2 * math.pi * 0.64) ** 1.5) < 1e-6


def test_vext_product_form_equals_literal_image_sum():
    cfg = O.Config(n=(14, 12, 10), L=(6.0, 5.0, 4.5))
    R = np.array([[0.2, 4.9, 2.0], [3.1, 2.2, 4.4], [5.8, 0.1, 0.05]])
    Z = np.array([2.0, 5.5, 3.0])
    np.testing.assert_allclose(O.vext_gaussians(cfg, R, Z, 0.8), O.vext_gaussians_literal(cfg, R, Z, 0.8),
                               atol=1e-13)


def test_random_orbitals_prefix_is_the_same_draw():
    a = inputs.random_orbitals(4, 6, (5, 4, 3))
    b = inputs.random_orbitals(4, 6, (5, 4, 3), count=2)
    assert np.array_equal(a[:2], b)


def test_random_orbitals_float32_draw():
    """The float32 draw (for blocks too large to draw in float64) is seeded,
    orbital by orbital, so a prefix is the same draw, and it is a standard
    normal sample."""
    a = inputs.random_orbitals(7, 5, (9, 8, 7), dtype=np.float32)
    b = inputs.random_orbitals(7, 5, (9, 8, 7), dtype=np.float32)
    c = inputs.random_orbitals(7, 5, (9, 8, 7), count=2, dtype=np.float32)
    assert a.dtype == np.float32 and a.shape == (5, 7, 8, 9)
    assert np.array_equal(a, b) and np.array_equal(a[:2], c)
    assert abs(float(np.mean(a))) < 0.05 and abs(float(np.std(a)) - 1.0) < 0.05


def test_hartree_cosine_closed_form():
    cfg = O.Config(n=(16, 12, 10), L=(7.0, 6.0, 5.0))
    x, y, z = O.grid_coords(cfg)
    A, rbar = 0.3, 1.1
    for axis, coord, Lax in ((0, x[None, None, :], 7.0), (1, y[None, :, None], 6.0), (2, z[:, None, None], 5.0)):
        rho = rbar + A * np.cos(2 * math.pi * coord / Lax) + 0 * np.zeros(cfg.shape)
        VH = O.hartree_potential(rho, cfg)
        exact = A * Lax ** 2 / math.pi * np.cos(2 * math.pi * coord / Lax) + 0 * np.zeros(cfg.shape)
        np.testing.assert_allclose(VH, exact, atol=1e-12)
        EH = 0.5 * cfg.dV * np.sum(rho * VH)
        vol = 7.0 * 6.0 * 5.0
        assert abs(EH - A * A * Lax ** 2 * vol / (4 * math.pi)) < 1e-10
    # constant density: neutralising background gives V_H = 0
    assert np.max(np.abs(O.hartree_potential(np.full(cfg.shape, 2.5), cfg))) < 1e-13


def test_hartree_against_explicit_dft_matrices():
    cfg = O.Config(n=(4, 3, 5), L=(3.0, 2.0, 4.0))
    rng = np.random.default_rng(0)
    rho = rng.uniform(0, 1, cfg.shape)

    def dft(n):
        j = np.arange(n)
        return np.exp(-2j * math.pi * np.outer(j, j) / n)

    nx, ny, nz = cfg.n
    Fx, Fy, Fz = dft(nx), dft(ny), dft(nz)
    rh = np.einsum("az,by,cx,zyx->abc", Fz, Fy, Fx, rho)
    # |G|^2 with m folded to the symmetric range (|m| = n/2 at Nyquist)
    def g(n, L):
        m = np.array([k if k <= n // 2 else k - n for k in range(n)], dtype=float)
        return 2 * math.pi * m / L
    gx, gy, gz = g(nx, 3.0), g(ny, 2.0), g(nz, 4.0)
    G2 = gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2
    K = np.where(G2 > 0, 4 * math.pi / np.where(G2 > 0, G2, 1), 0.0)
    vh = np.einsum("za,yb,xc,abc->zyx", np.conj(Fz), np.conj(Fy), np.conj(Fx), rh * K).real / cfg.Ng
    np.testing.assert_allclose(O.hartree_potential(rho, cfg), vh, atol=1e-12)


def test_exchange_closed_form_and_derivative():
    assert abs(O.exchange_energy_density(np.array(1.0)) + 0.75 * (3 / math.pi) ** (1 / 3)) < 1e-15
    rho = np.array([1e-3, 0.05, 0.7, 3.0])
    eps = 1e-6 * rho
    fd = (O.exchange_energy_density(rho + eps) - O.exchange_energy_density(rho - eps)) / (2 * eps)
    np.testing.assert_allclose(O.exchange_potential(rho), fd, rtol=1e-8)
    assert O.exchange_potential(np.array(0.0)) == 0.0


def test_cholesky_qr_matches_numpy_qr():
    cfg = O.Config(n=(6, 5, 4), L=(3.0, 2.5, 2.0), N=5)
    U = inputs.random_orbitals(3, 5, cfg.n)
    W, S, R = O.cholesky_qr(U, cfg)
    X = math.sqrt(cfg.dV) * U.reshape(5, -1).T  # columns = orbitals, unit-weight inner product
    Qm, Rm = np.linalg.qr(X)
    sgn = np.sign(np.diag(Rm))
    Qm, Rm = Qm * sgn[None, :], Rm * sgn[:, None]
    np.testing.assert_allclose(W.reshape(5, -1).T * math.sqrt(cfg.dV), Qm, atol=1e-12)
    np.testing.assert_allclose(R, Rm, rtol=1e-12, atol=1e-12)
    assert np.max(np.abs(O.inner_matrix(W, W, cfg) - np.eye(5))) < 1e-12


def test_energy_plane_wave_and_rotation_invariance():
    cfg = O.cubic(8, 5.0, N=1, hartree=0, exchange=0)
    u = _plane(cfg, (1, 0, 0))
    u /= math.sqrt(cfg.dV * np.sum(u * u))
    e = O.energy(u[None], np.zeros(cfg.shape), cfg)
    lam = 0.5 * _symbol(2, 1, 8, cfg.h[0])
    assert abs(e - 2 * lam) < 1e-12
    # E(UP) = E(U) for orthogonal P (Sec. 2.2), interacting case
    cfg2 = O.cubic(8, 6.0, N=3)
    R, Z = inputs.atoms(5, 2, 6.0, "const4")
    vext = O.vext_gaussians(cfg2, R, Z, 0.8)
    W, _, _ = O.cholesky_qr(inputs.random_orbitals(5, 3, cfg2.n), cfg2)
    P, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))
    WP = (P.T @ W.reshape(3, -1)).reshape(W.shape)
    assert abs(O.energy(W, vext, cfg2) - O.energy(WP, vext, cfg2)) < 1e-11
    assert abs(cfg2.dV * O.density(W).sum() - 2 * 3) < 1e-11


@pytest.mark.parametrize("order", [2, 4])
def test_gradient_residual_two_plane_waves(order):
    """Eq. gra on w = a phi_1 + b phi_2 (free particle, eigenvalues e_1, e_2 of
    H = -1/2 Lap_h): Sigma = a^2 e_1 + b^2 e_2 and |G| = |a b| |e_1 - e_2|;
    any rotation of (phi_1, phi_2) spans an invariant subspace, so G = 0."""
    cfg = O.Config(n=(12, 10, 9), L=(6.0, 5.5, 4.0), order=order, N=1, hartree=0, exchange=0)
    m1, m2 = (1, 0, 0), (0, 2, 1)
    e = [0.5 * sum(_symbol(order, m[a], cfg.n[a], cfg.h[a]) for a in range(3)) for m in (m1, m2)]
    phis = []
    for m in (m1, m2):
        u = _plane(cfg, m)
        phis.append(u / math.sqrt(cfg.dV * np.sum(u * u)))
    V0 = np.zeros(cfg.shape)
    a, b = 0.6, -0.8
    w = (a * phis[0] + b * phis[1])[None]
    g = O.gradient_residual(w, O.apply_h(w, V0, cfg), cfg)
    assert abs(g - abs(a * b) * abs(e[0] - e[1])) < 1e-12 * max(e)
    W = np.stack([a * phis[0] + b * phis[1], -b * phis[0] + a * phis[1]])
    assert O.gradient_residual(W, O.apply_h(W, V0, cfg), cfg) < 1e-12 * max(e)


def test_gradient_residual_is_the_projected_norm():
    """For orthonormal W and symmetric H, G = (I - W W^T) H W, so
    |G|^2 = |HW|^2 - |Sigma|^2 (Pythagoras on the projector)."""
    cfg = O.Config(n=(10, 9, 8), L=(5.0, 4.5, 4.0), order=4, N=4)
    W, _, _ = O.cholesky_qr(inputs.random_orbitals(21, 4, cfg.n), cfg)
    V = np.random.default_rng(3).standard_normal(cfg.shape)
    HW = O.apply_h(W, V, cfg)
    hw2 = cfg.dV * float(np.sum(HW * HW))
    sig = cfg.dV * (W.reshape(4, -1) @ HW.reshape(4, -1).T)
    exact = math.sqrt(hw2 - float(np.sum(sig * sig)))
    assert abs(O.gradient_residual(W, HW, cfg) - exact) < 1e-10 * exact


def _free_levels(cfg, N):
    lv = sorted(0.5 * sum(_symbol(cfg.order, m[a], cfg.n[a], cfg.h[a]) for a in range(3))
                for m in itertools.product(*(range(v) for v in cfg.n)))
    return lv[:N]


@pytest.mark.parametrize("order,N", [(2, 1), (2, 7), (4, 7)])
def test_free_particle_closed_shells(order, N):
    cfg = O.cubic(8, 6.0, order=order, N=N, hartree=0, exchange=0)
    vext = np.zeros(cfg.shape)
    U0 = inputs.random_orbitals(11, N, cfg.n)
    st = O.run(U0, vext, cfg, 600, e_tol=1e-15)
    exact = 2.0 * sum(_free_levels(cfg, N))
    assert abs(st.E - exact) < 1e-9 * max(1.0, abs(exact))


@pytest.mark.parametrize("N", [1, 7])
def test_jellium_with_exchange(N):
    L = 6.0
    cfg = O.cubic(8, L, order=2, N=N, hartree=1, exchange=1)
    st = O.run(inputs.random_orbitals(12, N, cfg.n), np.zeros(cfg.shape), cfg, 800, e_tol=1e-15)
    rbar = 2.0 * N / L ** 3
    ex = -0.75 * (3 / math.pi) ** (1 / 3) * rbar ** (4 / 3) * L ** 3
    exact = 2.0 * sum(_free_levels(cfg, N)) + ex
    assert abs(st.E - exact) < 1e-8
    assert np.max(np.abs(st.rho - rbar)) < 1e-5


def _sparse_h(cfg, vext):
    """FD Hamiltonian built from 1-D periodic difference matrices by Kronecker sums."""
    def d2(n, h, order):
        if order == 2:
            c = {0: -2.0, 1: 1.0, -1: 1.0}
            s = 1.0 / h ** 2
        else:
            c = {0: -30.0, 1: 16.0, -1: 16.0, 2: -1.0, -2: -1.0}
            s = 1.0 / (12 * h ** 2)
        M = np.zeros((n, n))
        for i in range(n):
            for k, v in c.items():
                M[i, (i + k) % n] += v * s
        return sp.csr_matrix(M)
    nx, ny, nz = cfg.n
    hx, hy, hz = cfg.h
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    lap = (sp.kron(sp.kron(Iz, Iy), d2(nx, hx, cfg.order))
           + sp.kron(sp.kron(Iz, d2(ny, hy, cfg.order)), Ix)
           + sp.kron(sp.kron(d2(nz, hz, cfg.order), Iy), Ix))
    return (-0.5 * lap + sp.diags(vext.ravel())).tocsr()


@pytest.mark.parametrize("order,N", [(2, 1), (2, 4), (4, 3)])
def test_noninteracting_well_vs_eigsh(order, N):
    cfg = O.cubic(12, 8.0, order=order, N=N, hartree=0, exchange=0)
    R = np.array([[3.1, 4.2, 3.7], [5.3, 3.5, 4.9]])
    vext = O.vext_gaussians(cfg, R, np.array([4.0, 3.0]), 0.8)
    ev = spla.eigsh(_sparse_h(cfg, vext), k=N + 2, which="SA", tol=1e-13)[0]
    exact = 2.0 * np.sort(ev)[:N].sum()
    st = O.run(inputs.random_orbitals(13, N, cfg.n), vext, cfg, 2000, e_tol=1e-16)
    assert abs(st.E - exact) < 1e-8


def test_self_consistency_subspace():
    cfg = O.cubic(8, 6.0, order=2, N=3)
    R, Z = inputs.atoms(21, 2, 6.0, "const4")
    Z = np.array([3.0, 3.0])
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    st = O.run(inputs.random_orbitals(21, 3, cfg.n), vext, cfg, 3000, e_tol=1e-16)
    H = _sparse_h(cfg, st.V).toarray()
    lam, vec = np.linalg.eigh(H)
    Pv = vec[:, :3]  # lowest three eigenvectors, unit Euclidean norm
    Wn = st.W.reshape(3, -1).T * math.sqrt(cfg.dV)
    s = np.linalg.svd(Pv.T @ Wn, compute_uv=False)
    assert np.min(s) > 1 - 1e-10  # cos of the largest principal angle
    assert lam[2] < lam[3] - 1e-3  # the occupied subspace is well separated


def test_orbital_gradient_finite_differences():
    cfg = O.Config(n=(6, 5, 6), L=(4.0, 3.5, 4.5), order=4, N=2)
    R = np.array([[1.0, 1.2, 2.0], [3.0, 2.5, 0.7]])
    vext = O.vext_gaussians(cfg, R, np.array([2.0, 4.0]), 0.8)
    U = 0.3 * inputs.random_orbitals(7, 2, cfg.n)
    g = O.energy_gradient_orbitals(U, vext, cfg)
    rng = np.random.default_rng(2)
    idx = [tuple(rng.integers(0, s) for s in U.shape) for _ in range(25)]
    eps = 1e-5
    for ix in idx:
        Up, Um = U.copy(), U.copy()
        Up[ix] += eps
        Um[ix] -= eps
        fd = (O.energy(Up, vext, cfg) - O.energy(Um, vext, cfg)) / (2 * eps)
        assert abs(fd - g[ix]) <= 1e-7 * max(1.0, np.max(np.abs(g))) , (ix, fd, g[ix])


def test_atom_gradient_finite_differences():
    cfg = O.Config(n=(10, 9, 8), L=(5.0, 4.5, 4.0), order=2, N=2)
    R = np.array([[1.0, 1.2, 2.0], [3.9, 2.5, 0.3]])
    Z = np.array([2.0, 4.0])
    U = inputs.random_orbitals(8, 2, cfg.n)
    U, _, _ = O.cholesky_qr(U, cfg)
    dR, dZ = O.energy_gradient_atoms(U, cfg, R, Z, 0.8)
    eps = 1e-5

    def E(Rv, Zv):
        return O.energy(U, O.vext_gaussians(cfg, Rv, Zv, 0.8), cfg)
    for I in range(2):
        for a in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[I, a] += eps
            Rm[I, a] -= eps
            fd = (E(Rp, Z) - E(Rm, Z)) / (2 * eps)
            assert abs(fd - dR[I, a]) < 1e-8 * max(1.0, abs(fd))
        Zp, Zm = Z.copy(), Z.copy()
        Zp[I] += eps
        Zm[I] -= eps
        fd = (E(R, Zp) - E(R, Zm)) / (2 * eps)
        assert abs(fd - dZ[I]) < 1e-8 * max(1.0, abs(fd))


def test_invariants_along_trajectory():
    cfg = O.cubic(10, 7.0, order=2, N=4)
    R, Z = inputs.atoms(31, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    st = O.initial_state(inputs.random_orbitals(31, 4, cfg.n), vext, cfg)
    for _ in range(60):
        C, Q = st.C, st.Q
        O.iterate(st, vext, cfg)
        rec = st.history[-1]
        assert np.max(np.abs(O.inner_matrix(st.W, st.W, cfg) - np.eye(4))) < 1e-12
        assert abs(cfg.dV * st.rho.sum() - 8.0) < 1e-10
        if not rec.forced:
            assert rec.energy <= C - cfg.rho1 * rec.tau * rec.znorm2 + 1e-12
        assert st.Q == pytest.approx(cfg.eta * Q + 1)


def test_monotone_when_eta_zero():
    cfg = O.cubic(10, 7.0, order=2, N=4, eta=0.0)
    R, Z = inputs.atoms(32, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    st = O.run(inputs.random_orbitals(32, 4, cfg.n), vext, cfg, 80)
    E = [O.initial_state(inputs.random_orbitals(32, 4, cfg.n), vext, cfg).E] + [h.energy for h in st.history]
    assert all(b <= a + 1e-12 for a, b in zip(E, E[1:]))


def test_bb_steps_cauchy_schwarz_and_scalar_case():
    cfg = O.cubic(4, 2.0, N=2)
    rng = np.random.default_rng(4)
    S = rng.standard_normal((2,) + cfg.shape)
    Y = rng.standard_normal((2,) + cfg.shape)
    t1 = O.bb_step(S, Y, O.Config(n=cfg.n, L=cfg.L, bb_variant=1), 0)
    t2 = O.bb_step(S, Y, O.Config(n=cfg.n, L=cfg.L, bb_variant=2), 0)
    assert t1 >= t2 > 0
    # Y = c S (a quadratic with Hessian c I): both steps equal 1/c
    for v in (1, 2):
        assert O.bb_step(S, 2.5 * S, O.Config(n=cfg.n, L=cfg.L, bb_variant=v), 0) == pytest.approx(0.4, rel=1e-14)


def test_optm_qr_and_opt_par_agree():
    """Table 1 claim: Opt-Par reaches the same energy as OptM-QR (full Sigma)."""
    cfg = O.cubic(10, 7.0, order=2, N=4)
    R, Z = inputs.atoms(41, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    U0 = inputs.random_orbitals(41, 4, cfg.n)
    a = O.run(U0, vext, cfg, 3000, e_tol=1e-16)
    b = O.run(U0, vext, cfg, 3000, e_tol=1e-16, full_sigma=True)
    assert abs(a.E - b.E) < 1e-8


def test_algorithm_m_variants_reach_same_energy():
    cfg = O.cubic(10, 7.0, order=2, N=4)
    R, Z = inputs.atoms(41, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    U0 = inputs.random_orbitals(41, 4, cfg.n)
    a = O.run(U0, vext, cfg, 3000, e_tol=1e-16)
    cfgm = O.cubic(10, 7.0, order=2, N=4, n_diag=20)
    b = O.run(U0, vext, cfgm, 3000, e_tol=1e-16)
    assert abs(a.E - b.E) < 1e-8


@pytest.mark.parametrize("n_org", [2, 3])
def test_algorithm_m_n_org_same_minimum_and_structure(n_org):
    """Algorithm M with Orth every n_org steps (Sec. 3.3) reaches the minimum
    Algorithm E reaches; only steps l = 0 mod n_org are orthonormalised (their
    iterates are orthonormal, the others carry no energy)."""
    cfg = O.cubic(10, 7.0, order=2, N=4)
    R, Z = inputs.atoms(41, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    U0 = inputs.random_orbitals(41, 4, cfg.n)
    a = O.run(U0, vext, cfg, 3000, e_tol=1e-16)
    cfgm = O.cubic(10, 7.0, order=2, N=4, n_org=n_org)
    b = O.run(U0, vext, cfgm, 6000, e_tol=1e-16)
    assert abs(b.E - a.E) < 1e-10
    E = np.array([h.energy for h in b.history])
    assert np.array_equal(np.isfinite(E), np.arange(len(E)) % n_org == 0)
    st = O.initial_state(U0, vext, cfgm)
    for l in range(3 * n_org):
        O.iterate(st, vext, cfgm)
        if st.l % n_org == 1 or n_org == 1:  # the step just taken (l - 1) was orthonormalised
            assert np.max(np.abs(O.inner_matrix(st.W, st.W, cfgm) - np.eye(4))) < 1e-12


def test_trial_gram_is_near_identity():
    """Fig. 2: the Gram matrix <Wt^T Wt> of the trial point stays close to the
    identity, and so diagonally dominant, away from the first steps; the
    exceptions are single large Barzilai-Borwein steps."""
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    st = O.run(U0, vext, cfg, 300)
    g = np.array([h.gram_offdiag for h in st.history])[100:]
    assert np.median(g) < 1e-3
    assert np.percentile(g, 90) < 1e-2
    assert np.mean(g < 1.0 / w.N) > 0.95  # max |S - I| < 1/N: S diagonally dominant


@pytest.mark.slow
def test_bb_trajectory_is_chaotic():
    """A 1e-15 relative change of U0 moves the oracle's energy by > 1e-8 within 200 steps
    but by < 1e-10 over the first 80: the horizon over which two correct
    implementations can be compared step by step."""
    w, R, Z, U0 = inputs.workload_inputs("l10_g32_n4")
    cfg = O.cubic(w.n, w.L, order=w.order, N=w.N)
    vext = O.vext_gaussians(cfg, R, Z, w.width)
    a = O.run(U0, vext, cfg, 200)
    rng = np.random.default_rng(0)
    b = O.run(U0 * (1 + 1e-15 * rng.standard_normal(U0.shape)), vext, cfg, 200)
    d = np.abs(np.array([h.energy for h in a.history]) - np.array([h.energy for h in b.history]))
    assert np.max(d[:80]) < 1e-10
    assert np.max(d) > 1e-8


def test_subspace_rotation_diagonalises_sigma():
    """Sec. 3.3 subspace diagonalisation, checked on what it must produce
    rather than on E (every orthogonal rotation leaves E unchanged): after
    W <- W P, Sigma = <W^T H W> is diagonal, its diagonal ascends and carries
    the spectrum of the Sigma before the rotation (same trace, same sum of
    squares, same ordered eigenvalues), the span and rho are unchanged, and
    W stays orthonormal.  A transposed P leaves P Sigma P^T, which is not
    diagonal; unsorted eigenpairs fail the ordering."""
    cfg = O.cubic(10, 7.0, order=4, N=5)
    R, Z = inputs.atoms(51, 3, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    st = O.run(inputs.random_orbitals(51, 5, cfg.n), vext, cfg, 25)
    W0, rho0, E0 = st.W.copy(), st.rho.copy(), st.E
    H0 = O.apply_h(W0, st.V, cfg)
    Sig0 = cfg.dV * (W0.reshape(5, -1) @ H0.reshape(5, -1).T)
    off0 = np.max(np.abs(Sig0 - np.diag(np.diag(Sig0))))
    assert off0 > 1e-3  # far from diagonal before: the check below is not vacuous
    O.subspace_diagonalise(st, vext, cfg)
    W1 = st.W
    H1 = O.apply_h(W1, st.V, cfg)
    Sig1 = cfg.dV * (W1.reshape(5, -1) @ H1.reshape(5, -1).T)
    d = np.diag(Sig1)
    scale = np.max(np.abs(Sig0))
    assert np.max(np.abs(Sig1 - np.diag(d))) < 1e-12 * scale
    assert np.all(np.diff(d) > 0)
    # invariants of an orthogonal similarity: trace and Frobenius norm
    assert abs(d.sum() - np.trace(Sig0)) < 1e-12 * scale
    assert abs(np.sum(d * d) - np.sum((0.5 * (Sig0 + Sig0.T)) ** 2)) < 1e-11 * scale ** 2
    # the ordered eigenvalues of the symmetric 5 x 5 matrix, from its characteristic polynomial
    lam = np.sort(np.roots(np.poly(0.5 * (Sig0 + Sig0.T))).real)
    np.testing.assert_allclose(d, lam, atol=1e-9 * scale)
    # span, orthonormality, density and energy unchanged
    M = cfg.dV * (W0.reshape(5, -1) @ W1.reshape(5, -1).T)
    assert abs(np.sum(M * M) - 5.0) < 1e-12
    assert np.max(np.abs(O.inner_matrix(W1, W1, cfg) - np.eye(5))) < 1e-12
    np.testing.assert_allclose(O.density(W1), rho0, atol=1e-12 * np.max(rho0))
    assert abs(O.energy(W1, vext, cfg) - E0) < 1e-11
    # the step after the rotation uses the Barzilai-Borwein step of the pair
    # before it (traces are invariant under the rotation of both iterates)
    assert st.tau_next is not None and st.W_prev is None


def test_nonmonotone_reference_closed_form():
    """Eq. (ene-de): Q^(l+1) = eta Q^l + 1, C^(l+1) = (eta Q^l C^l + E^(l+1)) / Q^(l+1)
    with C^0 = E^0, Q^0 = 1.  Unrolling, Q^l C^l = sum_k eta^(l-k) E^k and
    Q^l = sum_k eta^(l-k), so C^l is the eta-weighted mean of E^0..E^l.  The
    oracle's C and Q along an eta = 0.85 trajectory must equal that closed
    form, and every accepted (not forced) step must satisfy the test with C
    taken from it."""
    eta = 0.85
    cfg = O.cubic(10, 7.0, order=2, N=4, eta=eta)
    R, Z = inputs.atoms(33, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    st = O.initial_state(inputs.random_orbitals(33, 4, cfg.n), vext, cfg)
    E = [st.E]
    C_seen, Q_seen = [st.C], [st.Q]
    backtracked = 0
    for _ in range(30):
        O.iterate(st, vext, cfg)
        E.append(st.history[-1].energy)
        C_seen.append(st.C)
        Q_seen.append(st.Q)
        backtracked += st.history[-1].backtracks
    E = np.array(E)
    for l in range(len(E)):
        wts = eta ** np.arange(l, -1, -1, dtype=float)  # eta^(l-k), k = 0..l
        Cl = float(np.dot(wts, E[: l + 1]) / wts.sum())
        assert abs(C_seen[l] - Cl) < 1e-12 * abs(Cl)
        assert abs(Q_seen[l] - wts.sum()) < 1e-13 * wts.sum()
        if l > 0:
            rec = st.history[l - 1]
            wp = eta ** np.arange(l - 1, -1, -1, dtype=float)
            Cprev = float(np.dot(wp, E[:l]) / wp.sum())
            if not rec.forced:
                assert E[l] <= Cprev - cfg.rho1 * rec.tau * rec.znorm2 + 1e-12
    # C is a weighted mean, not the last energy: it lags above E on a descending run
    assert np.sum(np.array(C_seen[1:]) > E[1:] + 1e-9) > 10


def test_converged_forces_match_fd_of_reconverged_energies():
    """Sec. 2.1: at the minimum over orthonormal U the derivative of the
    converged energy E*(R) equals the explicit dE/dR at fixed U (the U-gradient
    H u_i lies in the span, so the orbitals' response does not enter).  The
    analytic gradient of the converged orbitals must match central differences
    of energies re-converged at R +- 1e-4 bohr, to 1e-5 Ha/bohr."""
    cfg = O.cubic(8, 6.0, order=2, N=2)
    R = np.array([[1.3, 2.1, 2.6], [3.9, 3.4, 4.2]])
    Zc = np.array([3.0, 2.0])
    U0 = inputs.random_orbitals(61, 2, cfg.n)

    def converge(Rv, U):
        vext = O.vext_gaussians(cfg, Rv, Zc, 0.8)
        st = O.run(U, vext, cfg, 4000, e_tol=1e-16)
        return st

    st = converge(R, U0)
    dR, _ = O.energy_gradient_atoms(st.W, cfg, R, Zc, 0.8)
    assert np.max(np.abs(dR)) > 1e-2  # the atoms feel a real force
    h = 1e-4
    for I in range(2):
        for a in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[I, a] += h
            Rm[I, a] -= h
            Ep = converge(Rp, st.W).E
            Em = converge(Rm, st.W).E
            fd = (Ep - Em) / (2 * h)
            assert abs(fd - dR[I, a]) < 1e-5, (I, a, fd, dR[I, a])


def test_per_orbital_bb_steps_on_separate_quadratics():
    """tau_i of Sec. 3.2 taken orbital by orbital: when y_i = k_i s_i (orbital
    i on its own quadratic with Hessian k_i I) both quotients give 1/k_i, and
    the common step of the traces lies between the smallest and largest."""
    cfg = O.cubic(6, 3.0, N=3)
    rng = np.random.default_rng(7)
    S = rng.standard_normal((3,) + cfg.shape)
    k = np.array([0.5, 2.0, 8.0])
    Y = k[:, None, None, None] * S
    for v in (1, 2):
        c = O.Config(n=cfg.n, L=cfg.L, bb_variant=v)
        np.testing.assert_allclose(O.bb_step_per_orbital(S, Y, c, 0), 1.0 / k, rtol=1e-14)
        t = O.bb_step(S, Y, c, 0)
        assert 1.0 / k.max() <= t <= 1.0 / k.min()


def _rayleigh(u, V, cfg):
    return float(np.sum(u * O.apply_h(u[None], V, cfg)[0]) / np.sum(u * u))


def test_newton_step_is_minus_first_over_second_derivative():
    """The CG step of each orbital is the Newton step of its Rayleigh quotient
    R(t) = <u, H u> / <u, u>, u = w_i - t d_i (potential frozen): checked
    against -R'(0) / R''(0) from central differences of R itself."""
    cfg = O.Config(n=(10, 9, 8), L=(5.0, 4.5, 4.0), order=4, N=3)
    R, Zc = inputs.atoms(9, 2, 4.0, "const4")
    vext = O.vext_gaussians(cfg, R, Zc, 0.8)
    W, _, _ = O.cholesky_qr(inputs.random_orbitals(9, 3, cfg.n), cfg)
    V = O.total_potential(O.density(W), vext, cfg)
    HW = O.apply_h(W, V, cfg)
    Zd, sigma = O.search_direction(W, HW, cfg)
    rng = np.random.default_rng(3)
    D = Zd + 0.3 * rng.standard_normal(W.shape) * np.max(np.abs(Zd))
    w2 = W.reshape(3, -1)
    D = (D.reshape(3, -1) - (cfg.dV * np.sum(w2 * D.reshape(3, -1), 1))[:, None] * w2).reshape(W.shape)
    t = O.newton_steps(D, Zd, V, sigma, cfg)
    h = 1e-4
    for i in range(3):
        r = [_rayleigh(W[i] - s * D[i], V, cfg) for s in (-h, 0.0, h)]
        d1 = (r[2] - r[0]) / (2 * h)
        d2 = (r[2] - 2 * r[1] + r[0]) / (h * h)
        assert abs(t[i] - (-d1 / d2)) < 1e-5 * abs(t[i]), (i, t[i], -d1 / d2)


def test_cg_direction_structure():
    """d_i = z_i on the first step; otherwise d_i - z_i is a non-negative
    multiple of the previous direction with its w_i component removed, beta_i
    is zero when z_i = z_i', and every orbital keeps <z_i, d_i> >= <z_i, z_i>/2."""
    cfg = O.cubic(6, 3.0, N=4)
    rng = np.random.default_rng(11)
    W, _, _ = O.cholesky_qr(rng.standard_normal((4,) + cfg.shape), cfg)
    Zc = rng.standard_normal(W.shape)
    Zp = rng.standard_normal(W.shape)
    Dp = rng.standard_normal(W.shape)
    assert np.array_equal(O.cg_direction(W, Zc, None, None, cfg), Zc)
    D = O.cg_direction(W, Zc, Zp, Dp, cfg).reshape(4, -1)
    z, w, dp = Zc.reshape(4, -1), W.reshape(4, -1), Dp.reshape(4, -1)
    dpp = dp - (cfg.dV * np.sum(w * dp, 1))[:, None] * w
    for i in range(4):
        diff = D[i] - z[i]
        beta = float(np.dot(diff, dpp[i]) / np.dot(dpp[i], dpp[i]))
        assert beta >= 0.0 and np.allclose(diff, beta * dpp[i], atol=1e-12 * np.max(np.abs(z)))
        assert np.dot(z[i], D[i]) >= 0.5 * np.dot(z[i], z[i]) - 1e-9
    # identical gradients: the Polak-Ribiere numerator vanishes
    assert np.allclose(O.cg_direction(W, Zc, Zc, Dp, cfg), Zc)


@pytest.mark.parametrize("kw", [{"tau_mode": 1}, {"solver": 1}])
def test_per_orbital_steps_and_cg_reach_the_minimum(kw):
    """Both additions to the subproblem solver reach the minimum Algorithm E
    reaches (steepest descent with one Barzilai-Borwein step, run to
    convergence), and every accepted step passes Eq. (ene-de) with the
    decrease of the step actually taken (here: E never above C)."""
    cfg0 = O.cubic(16, 7.0, order=4, N=3)
    R, Z = inputs.atoms(14, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg0, R, Z, 0.8)
    U0 = inputs.random_orbitals(14, 3, cfg0.n)
    ref = O.run(U0, vext, cfg0, 4000, e_tol=1e-16)
    cfg = O.cubic(16, 7.0, order=4, N=3, **kw)
    st = O.initial_state(U0, vext, cfg)
    for _ in range(60):
        C = st.C
        O.iterate(st, vext, cfg)
        rec = st.history[-1]
        if not rec.forced:
            assert rec.energy <= C + 1e-12
    st = O.run(None, vext, cfg, 4000, e_tol=1e-16, st=st)
    assert abs(st.E - ref.E) < 1e-9, (st.E - ref.E, len(st.history))


def test_projectors_product_form_and_integral():
    """Nonlocal projectors (Sec. 2.1's xi_l): the per-axis image product equals
    the literal 27-image sum, and a projector integrates to a (2 pi s^2)^(3/2)."""
    cfg = O.Config(n=(18, 16, 14), L=(7.0, 6.0, 5.5))
    c = np.array([[0.3, 5.8, 2.0], [3.5, 2.5, 5.4]])
    s = np.array([0.7, 0.9])
    a = np.array([1.5, -0.8])
    xi = O.projectors_gaussian(cfg, c, s, a)
    x, y, z = O.grid_coords(cfg)
    for p in range(2):
        lit = np.zeros(cfg.shape)
        for i, j, k in itertools.product((-1, 0, 1), repeat=3):
            d2 = ((z[:, None, None] - c[p, 2] - k * 5.5) ** 2 + (y[None, :, None] - c[p, 1] - j * 6.0) ** 2
                  + (x[None, None, :] - c[p, 0] - i * 7.0) ** 2)
            lit += a[p] * np.exp(-d2 / (2 * s[p] ** 2))
        np.testing.assert_allclose(xi[p], lit, atol=1e-13)
        assert abs(cfg.dV * xi[p].sum() - a[p] * (2 * math.pi * s[p] ** 2) ** 1.5) < 1e-6


def test_nonlocal_rank_one_lifts_the_constant_mode():
    """Free particles with one projector xi = alpha phi_0, phi_0 the normalised
    constant mode (eigenvalue 0 of -1/2 Lap_h): H = -1/2 Lap_h + alpha^2 |phi_0><phi_0|
    lifts that mode to alpha^2 and leaves the plane waves.  With alpha^2 above the
    second shell, the 6 lowest states are the first shell: E = 2 * 6 * e_1."""
    n, L = 8, 6.0
    cfg0 = O.cubic(n, L, order=2, N=6, hartree=0, exchange=0)
    e = sorted(0.5 * sum(_symbol(2, m[a], n, L / n) for a in range(3))
               for m in itertools.product(range(n), repeat=3))
    e1, e2 = e[1], e[7]
    alpha = math.sqrt(3.0 * e2)
    xi = (alpha / math.sqrt(L ** 3)) * np.ones((1,) + cfg0.shape)
    cfg = O.cubic(n, L, order=2, N=6, hartree=0, exchange=0, xi=xi)
    st = O.run(inputs.random_orbitals(17, 6, cfg.n), np.zeros(cfg.shape), cfg, 1500, e_tol=1e-15)
    assert abs(st.E - 2 * 6 * e1) < 1e-9
    # the constant mode itself carries alpha^2 in the energy
    phi0 = np.ones((1,) + cfg.shape) / math.sqrt(L ** 3)
    cfg1 = O.cubic(n, L, order=2, N=1, hartree=0, exchange=0, xi=xi)
    assert abs(O.energy(phi0, np.zeros(cfg.shape), cfg1) - 2 * alpha ** 2) < 1e-12


def test_nonlocal_well_vs_eigsh():
    """Non-interacting well plus two Gaussian projectors: the converged energy
    is twice the sum of the lowest eigenvalues of the sparse FD Hamiltonian
    plus the rank-2 term sum_p dV xi_p xi_p^T, from scipy's eigsh."""
    cfg0 = O.cubic(12, 8.0, order=4, N=3, hartree=0, exchange=0)
    R = np.array([[3.1, 4.2, 3.7], [5.3, 3.5, 4.9]])
    vext = O.vext_gaussians(cfg0, R, np.array([4.0, 3.0]), 0.8)
    xi = O.projectors_gaussian(cfg0, R, np.array([0.7, 0.9]), np.array([1.2, 0.6]))
    cfg = O.cubic(12, 8.0, order=4, N=3, hartree=0, exchange=0, xi=xi)
    H0 = _sparse_h(cfg0, vext)
    X = xi.reshape(2, -1)
    op = spla.LinearOperator(H0.shape, matvec=lambda v: H0 @ v + cfg.dV * (X.T @ (X @ v)), dtype=float)
    ev = np.sort(spla.eigsh(op, k=5, which="SA", tol=1e-13)[0])
    st = O.run(inputs.random_orbitals(13, 3, cfg.n), vext, cfg, 3000, e_tol=1e-16)
    assert abs(st.E - 2.0 * ev[:3].sum()) < 1e-8


def test_nonlocal_gradient_finite_differences():
    cfg0 = O.Config(n=(6, 5, 6), L=(4.0, 3.5, 4.5), order=4, N=2)
    R = np.array([[1.0, 1.2, 2.0], [3.0, 2.5, 0.7]])
    vext = O.vext_gaussians(cfg0, R, np.array([2.0, 4.0]), 0.8)
    xi = O.projectors_gaussian(cfg0, R, np.array([0.8, 0.6]), np.array([1.0, 0.7]))
    cfg = O.Config(n=(6, 5, 6), L=(4.0, 3.5, 4.5), order=4, N=2, xi=xi)
    U = 0.3 * inputs.random_orbitals(7, 2, cfg.n)
    g = O.energy_gradient_orbitals(U, vext, cfg)
    rng = np.random.default_rng(5)
    eps = 1e-5
    for _ in range(20):
        ix = tuple(rng.integers(0, s) for s in U.shape)
        Up, Um = U.copy(), U.copy()
        Up[ix] += eps
        Um[ix] -= eps
        fd = (O.energy(Up, vext, cfg) - O.energy(Um, vext, cfg)) / (2 * eps)
        assert abs(fd - g[ix]) <= 1e-7 * max(1.0, np.max(np.abs(g)))


def test_trial_without_positive_definite_gram_is_refused():
    """A rank-deficient trial block has no Cholesky-QR: try_cholesky_qr
    refuses it (the iteration then shrinks the step), and agrees with
    cholesky_qr on a well-conditioned block."""
    cfg = O.cubic(6, 3.0, N=3)
    U = inputs.random_orbitals(4, 3, cfg.n)
    W, S, R = O.cholesky_qr(U, cfg)
    W2, S2, R2 = O.try_cholesky_qr(U, cfg)
    assert np.array_equal(W, W2) and np.array_equal(R, R2)
    Ud = U.copy()
    Ud[2] = 0.5 * Ud[0] - 2.0 * Ud[1]
    assert O.try_cholesky_qr(Ud, cfg) is None
    Ud[2] += 1e-9 * U[2]  # numerically singular: pivot ~1e-18 of S_max
    assert O.try_cholesky_qr(Ud, cfg) is None


def test_search_directions_are_tangent_gradients():
    """Sec. 3.1-3.2: OptM-QR's direction Z = HW - W Sigma is the gradient of E
    on the orthonormality constraint (tangent: <W^T Z> + <Z^T W> = 0; along
    every tangent direction the derivative of E is 2 f dV sum <z_i, d_i>/dV),
    and Opt-Par's z_i = H w_i - sigma_ii w_i is the gradient of E in orbital i
    on its own sphere (<w_i, z_i> = 0; the same derivative along a d_i with
    <w_i, d_i> = 0).  Derivatives by central finite differences of the energy."""
    cfg = O.Config(n=(6, 5, 6), L=(4.0, 3.5, 4.5), order=4, N=3)
    R = np.array([[1.0, 1.2, 2.0], [3.0, 2.5, 0.7]])
    vext = O.vext_gaussians(cfg, R, np.array([2.0, 4.0]), 0.8)
    W, _, _ = O.cholesky_qr(inputs.random_orbitals(3, 3, cfg.n), cfg)
    HW = O.apply_h(W, O.total_potential(O.density(W), vext, cfg), cfg)
    Zf, _ = O.search_direction(W, HW, cfg, full=True)
    Zp, sig = O.search_direction(W, HW, cfg)
    M = O.inner_matrix(W, Zf, cfg)
    assert np.max(np.abs(M + M.T)) < 1e-12
    assert np.max(np.abs(np.diag(O.inner_matrix(W, Zp, cfg)))) < 1e-12
    rng = np.random.default_rng(8)
    eps = 1e-5

    def dE(D):
        return (O.energy(W + eps * D, vext, cfg) - O.energy(W - eps * D, vext, cfg)) / (2 * eps)

    for _ in range(4):
        X = rng.standard_normal(W.shape)
        # tangent part of X on the constraint <W^T W> = I
        S = O.inner_matrix(W, X, cfg)
        D = X - np.einsum("ij,i...->j...", 0.5 * (S + S.T), W)
        assert abs(dE(D) - 2 * O.F_OCC * cfg.dV * np.sum(Zf * D)) <= 1e-7 * max(1.0, abs(dE(D)))
        # one orbital on its own sphere
        i = int(rng.integers(0, 3))
        Di = np.zeros_like(W)
        Di[i] = X[i] - cfg.dV * np.sum(W[i] * X[i]) * W[i]
        assert abs(dE(Di) - 2 * O.F_OCC * cfg.dV * np.sum(Zp[i] * Di[i])) <= 1e-7 * max(1.0, abs(dE(Di)))


def test_energy_criterion_stops_at_the_first_qualifying_step():
    """Sec. 4.2's stopping rule on a real trajectory: df^l is the change of
    the energy relative to |E^(l-1)| + 1, and the run stops at the first l
    whose average of df^l, df^(l-1), df^(l-2) is below the tolerance."""
    cfg = O.cubic(10, 7.0, order=2, N=4)
    R, Z = inputs.atoms(33, 2, 7.0, "const4")
    vext = O.vext_gaussians(cfg, R, Z, 0.8)
    U0 = inputs.random_orbitals(33, 4, cfg.n)
    E0 = O.initial_state(U0, vext, cfg).E
    free = O.run(U0, vext, cfg, 150)
    E = np.array([E0] + [h.energy for h in free.history])
    df = np.abs(np.diff(E)) / (np.abs(E[:-1]) + 1.0)
    avg = (df[2:] + df[1:-1] + df[:-2]) / 3.0
    tol = float(np.sort(avg)[len(avg) // 2])  # a tolerance met part way through
    first = int(np.nonzero(avg < tol)[0][0]) + 3  # steps taken when it is first met
    st = O.run(U0, vext, cfg, 150, e_tol=tol)
    assert st.l == first
    np.testing.assert_allclose(st.df, df[:first], rtol=0, atol=0)
