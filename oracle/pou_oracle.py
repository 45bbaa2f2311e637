"""Plain, slow, FP64 CPU oracle for the parallel orbital-updating method.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The GPU library never
calls it and shares no code with it.

Paper: Dai, Liu, Zhang, Zhou, "A Parallel Orbital-updating Based Optimization
Method for Electronic Structure Calculations" (arXiv 1510.07230).

Discrete model (uniform periodic grid, n = (nx, ny, nz), box L = (Lx, Ly, Lz),
h_a = L_a / n_a, dV = hx*hy*hz; arrays are (N, nz, ny, nx), x fastest):

* inner product  <a, b> = dV * sum_r a(r) b(r)      (L2 product of Sec. 2.2)
* density        rho = f * sum_i w_i^2, f = 2        (Sec. 2.1, double occupancy)
* energy         E = f sum_i <w_i, -1/2 Lap_h w_i> + dV sum rho Vext
                     + 1/2 dV sum rho V_H + dV sum eps_x(rho) rho   (Eq. energy)
* Hamiltonian    H = -1/2 Lap_h + Vext + V_H + v_x                 (Sec. 2.1)
* Hartree        -Lap V_H = 4 pi (rho - mean rho), solved spectrally
* exchange       Slater LDA: eps_x = -3/4 (3/pi)^(1/3) rho^(1/3),
                 v_x = -(3/pi)^(1/3) rho^(1/3)
* Lap_h          periodic 7-point (order 2) or 13-point (order 4) stencil

Iteration (Algorithm E, i.e. Algorithm M with n_org = 1 and no subspace
diagonalisation; Sec. 3.2):

1. HW = H(rho_W) W, sigma_ii = <H w_i, w_i>, z_i = H w_i - sigma_ii w_i
2. Barzilai-Borwein step from S = W^l - W^(l-1), Y = Z^l - Z^(l-1):
   tau1 = tr<S^T S> / |tr<S^T Y>|,  tau2 = |tr<S^T Y>| / tr<Y^T Y>
3. nonmonotone backtracking (Eq. ene-de): tau = tau_BB * delta^s with the
   smallest s such that E(W(tau)) <= C^l - rho1 * tau * ||Z^l||_F^2,
   W(tau) = Orth(W - tau Z), Orth = Cholesky-based QR
4. Q^(l+1) = eta Q^l + 1, C^(l+1) = (eta Q^l C^l + E^(l+1)) / Q^(l+1)

Algorithm M options (Sec. 3.3): n_org > 1 orthonormalises only the steps
l = 0 mod n_org (the others take W - tau Z as it is, without the Eq. (ene-de)
test; C, Q and E are kept); n_diag > 0 rotates W to the eigenvectors of
Sigma = <W^T H W> after every n_diag-th orthonormalised step.

Readings where the paper is silent (also listed in the design notes):
the two BB steps ("tau1 or tau2") alternate by default, tau1 on even l;
tau at l = 0 and when tr<S^T Y> = 0 is 1 / lambda_max(-1/2 Lap_h); tau is
clamped to [1e-12, 1e3]; after ``max_backtrack`` reductions the last trial
is accepted and counted; the Hartree kernel is 4 pi / |G|^2 with G = 2 pi m / L,
m in FFT order, G = 0 set to zero; Gaussian wells are summed over the 27
nearest periodic images.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np
from scipy.linalg import cholesky, solve_triangular

F_OCC = 2.0  # double occupancy (reading of Sec. 2.1 rho = sum |u_i|^2 with f = 2)
CX = (3.0 / math.pi) ** (1.0 / 3.0)


# --------------------------------------------------------------------------
# configuration
# --------------------------------------------------------------------------
@dataclass
class Config:
    n: Sequence[int]  # (nx, ny, nz)
    L: Sequence[float]  # (Lx, Ly, Lz)
    order: int = 2  # 2: 7-point, 4: 13-point Laplacian
    N: int = 1
    hartree: int = 1
    exchange: int = 1
    bb_variant: int = 3  # 1: tau1, 2: tau2, 3: alternate (tau1 on even l, tau2 on odd l)
    rho1: float = 1e-4  # Sec. 3.2 constants
    delta: float = 0.1
    eta: float = 0.85
    max_backtrack: int = 10
    tau0: float = 0.0  # 0 -> 1 / lambda_max(-1/2 Lap_h)
    tau_min: float = 1e-12
    tau_max: float = 1e3
    n_org: int = 1  # Algorithm M: orthonormalise every n_org steps
    n_diag: int = 0  # Algorithm M: subspace diagonalisation every n_diag steps (0 = off)
    tau_mode: int = 0  # 0: one Barzilai-Borwein step for all orbitals, 1: tau_i per orbital
    solver: int = 0  # per-orbital subproblem solver: 0 steepest descent, 1 conjugate gradient
    xi: Optional[np.ndarray] = None  # nonlocal projectors xi_p on the grid, (P, nz, ny, nx); None: none

    @property
    def h(self):
        return tuple(float(self.L[a]) / int(self.n[a]) for a in range(3))

    @property
    def dV(self):
        hx, hy, hz = self.h
        return hx * hy * hz

    @property
    def Ng(self):
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    @property
    def shape(self):
        return (int(self.n[2]), int(self.n[1]), int(self.n[0]))


def cubic(n: int, L: float, **kw) -> Config:
    return Config(n=(n, n, n), L=(L, L, L), **kw)


# --------------------------------------------------------------------------
# discrete operators (Sec. 2.3: real-space finite differences)
# --------------------------------------------------------------------------
def laplacian(u: np.ndarray, cfg: Config) -> np.ndarray:
    """Periodic finite-difference Laplacian along the last three axes.

    order 2: sum_a (u[+1] - 2u + u[-1]) / h_a^2
    order 4: sum_a (-u[+2] + 16u[+1] - 30u + 16u[-1] - u[-2]) / (12 h_a^2)
    """
    hx, hy, hz = cfg.h
    out = np.zeros_like(u)
    for axis, h in ((-1, hx), (-2, hy), (-3, hz)):
        p1 = np.roll(u, -1, axis)
        m1 = np.roll(u, 1, axis)
        if cfg.order == 2:
            out += (p1 - 2.0 * u + m1) / (h * h)
        elif cfg.order == 4:
            p2 = np.roll(u, -2, axis)
            m2 = np.roll(u, 2, axis)
            out += (-p2 + 16.0 * p1 - 30.0 * u + 16.0 * m1 - m2) / (12.0 * h * h)
        else:
            raise ValueError("order must be 2 or 4")
    return out


def lambda_max_kinetic(cfg: Config) -> float:
    """Largest eigenvalue of -1/2 Lap_h (reached at the Nyquist mode).

    Per axis -Lap_h has largest symbol 4/h^2 (order 2) and 16/(3 h^2) (order 4).
    """
    c = 4.0 if cfg.order == 2 else 16.0 / 3.0
    return 0.5 * sum(c / (h * h) for h in cfg.h)


def grid_coords(cfg: Config):
    hx, hy, hz = cfg.h
    nx, ny, nz = (int(v) for v in cfg.n)
    return np.arange(nx) * hx, np.arange(ny) * hy, np.arange(nz) * hz


def vext_gaussians(cfg: Config, R: np.ndarray, Z: np.ndarray, width: float) -> np.ndarray:
    """Local wells V(r) = -sum_I Z_I sum_images exp(-|r - R_I - nL|^2 / (2 width^2)).

    Stands in for the local pseudopotential of Sec. 2.1; the sum runs over the
    27 nearest periodic images n in {-1, 0, 1}^3 of the position wrapped into
    [0, L) (so every grid point sees its nearest image of every atom).
    Because exp(-|d|^2/(2 w^2)) is a product over the three axes, the 27-term
    image sum equals the product of the three per-axis sums over n_a in
    {-1, 0, 1} (distributivity); it is evaluated in that form.  The literal
    27-term sum is ``vext_gaussians_literal``.
    """
    x, y, z = grid_coords(cfg)
    Lx, Ly, Lz = (float(v) for v in cfg.L)
    R = wrap_positions(R, cfg)
    V = np.zeros(cfg.shape)
    two_s2 = 2.0 * width * width
    for I in range(len(Z)):
        gx = sum(np.exp(-(x - R[I, 0] - a * Lx) ** 2 / two_s2) for a in (-1, 0, 1))
        gy = sum(np.exp(-(y - R[I, 1] - b * Ly) ** 2 / two_s2) for b in (-1, 0, 1))
        gz = sum(np.exp(-(z - R[I, 2] - c * Lz) ** 2 / two_s2) for c in (-1, 0, 1))
        V -= Z[I] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return V


def vext_gaussians_literal(cfg: Config, R: np.ndarray, Z: np.ndarray, width: float) -> np.ndarray:
    """The same wells as ``vext_gaussians``, summed image by image (27 terms per atom)."""
    x, y, z = grid_coords(cfg)
    Lx, Ly, Lz = (float(v) for v in cfg.L)
    R = wrap_positions(R, cfg)
    V = np.zeros(cfg.shape)
    two_s2 = 2.0 * width * width
    for I in range(len(Z)):
        for a, b, c in itertools.product((-1, 0, 1), repeat=3):
            dx = x - R[I, 0] - a * Lx
            dy = y - R[I, 1] - b * Ly
            dz = z - R[I, 2] - c * Lz
            d2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
            V -= Z[I] * np.exp(-d2 / two_s2)
    return V


def wrap_positions(R: np.ndarray, cfg: Config) -> np.ndarray:
    """Atom positions folded into the periodic box [0, L)."""
    L = np.asarray(cfg.L, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    return R - L[None, :] * np.floor(R / L[None, :])


def projectors_gaussian(cfg: Config, centres: np.ndarray, widths: np.ndarray, amps: np.ndarray) -> np.ndarray:
    """Synthetic nonlocal projectors xi_p(r) = a_p sum_n exp(-|r - c_p - nL|^2 / (2 s_p^2))
    on the grid (the xi_l of the pseudopotential's nonlocal part, Sec. 2.1),
    summed over the 27 nearest periodic images of c_p folded into [0, L),
    evaluated as the product of three per-axis image sums (distributivity)."""
    x, y, z = grid_coords(cfg)
    Lx, Ly, Lz = (float(v) for v in cfg.L)
    C = wrap_positions(centres, cfg)
    P = len(amps)
    xi = np.zeros((P,) + cfg.shape)
    for p in range(P):
        t = 2.0 * widths[p] ** 2
        gx = sum(np.exp(-(x - C[p, 0] - a * Lx) ** 2 / t) for a in (-1, 0, 1))
        gy = sum(np.exp(-(y - C[p, 1] - b * Ly) ** 2 / t) for b in (-1, 0, 1))
        gz = sum(np.exp(-(z - C[p, 2] - c * Lz) ** 2 / t) for c in (-1, 0, 1))
        xi[p] = amps[p] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return xi


def projections(W: np.ndarray, cfg: Config) -> np.ndarray:
    """C_pi = <xi_p, w_i> (P x N)."""
    N = W.shape[0]
    P = cfg.xi.shape[0]
    return cfg.dV * (cfg.xi.reshape(P, -1) @ W.reshape(N, -1).T)


def apply_nonlocal(W: np.ndarray, cfg: Config) -> np.ndarray:
    """V_nloc w_i = sum_p <xi_p, w_i> xi_p (Sec. 2.1)."""
    N = W.shape[0]
    P = cfg.xi.shape[0]
    C = projections(W, cfg)
    return (C.T @ cfg.xi.reshape(P, -1)).reshape(W.shape)


def density(W: np.ndarray) -> np.ndarray:
    """rho = f * sum_i w_i^2 (Sec. 2.1 with double occupancy)."""
    return F_OCC * np.sum(W * W, axis=0)


def hartree_potential(rho: np.ndarray, cfg: Config) -> np.ndarray:
    """Solve -Lap V_H = 4 pi (rho - mean rho) spectrally on the periodic box.

    V_H_hat(G) = 4 pi rho_hat(G) / |G|^2 with G = 2 pi m / L (m in FFT order,
    |m| = n/2 at Nyquist), and V_H_hat(0) = 0 (neutralising background).
    """
    nx, ny, nz = (int(v) for v in cfg.n)
    Lx, Ly, Lz = (float(v) for v in cfg.L)
    gx = 2.0 * math.pi * np.fft.fftfreq(nx, 1.0 / nx) / Lx
    gy = 2.0 * math.pi * np.fft.fftfreq(ny, 1.0 / ny) / Ly
    gz = 2.0 * math.pi * np.fft.fftfreq(nz, 1.0 / nz) / Lz
    G2 = gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2
    kernel = np.zeros_like(G2)
    nz_mask = G2 > 0
    kernel[nz_mask] = 4.0 * math.pi / G2[nz_mask]
    return np.real(np.fft.ifftn(np.fft.fftn(rho) * kernel))


def exchange_potential(rho: np.ndarray) -> np.ndarray:
    """v_x = d(rho eps_x)/d rho = -(3/pi)^(1/3) rho^(1/3) (Slater LDA exchange)."""
    return -CX * np.cbrt(rho)


def exchange_energy_density(rho: np.ndarray) -> np.ndarray:
    """eps_x(rho) rho = -3/4 (3/pi)^(1/3) rho^(4/3)."""
    return -0.75 * CX * np.cbrt(rho) * rho


@dataclass
class EnergyTerms:
    kinetic: float
    external: float
    hartree: float
    exchange: float

    @property
    def total(self) -> float:
        return self.kinetic + self.external + self.hartree + self.exchange


def energy_terms(W: np.ndarray, vext: np.ndarray, cfg: Config) -> EnergyTerms:
    """Discrete Kohn-Sham energy of Eq. (energy); W need not be orthonormal.
    The external term holds the local part dV sum rho Vext and, with
    projectors, the nonlocal part f sum_i sum_p <xi_p, w_i>^2 (both are parts
    of V_ext in Sec. 2.1)."""
    dV = cfg.dV
    rho = density(W)
    ekin = F_OCC * dV * float(np.sum(W * (-0.5 * laplacian(W, cfg))))
    eext = dV * float(np.sum(rho * vext))
    if cfg.xi is not None:
        eext += F_OCC * float(np.sum(projections(W, cfg) ** 2))
    eh = 0.0
    if cfg.hartree:
        eh = 0.5 * dV * float(np.sum(rho * hartree_potential(rho, cfg)))
    ex = 0.0
    if cfg.exchange:
        ex = dV * float(np.sum(exchange_energy_density(rho)))
    return EnergyTerms(ekin, eext, eh, ex)


def energy(W: np.ndarray, vext: np.ndarray, cfg: Config) -> float:
    return energy_terms(W, vext, cfg).total


def total_potential(rho: np.ndarray, vext: np.ndarray, cfg: Config) -> np.ndarray:
    """V = Vext + V_H(rho) + v_x(rho), the local part of H(rho) (Sec. 2.1)."""
    V = vext.copy()
    if cfg.hartree:
        V = V + hartree_potential(rho, cfg)
    if cfg.exchange:
        V = V + exchange_potential(rho)
    return V


def apply_h(W: np.ndarray, V: np.ndarray, cfg: Config) -> np.ndarray:
    """H(rho) w_i = -1/2 Lap_h w_i + V w_i (+ V_nloc w_i with projectors) for
    every orbital (E_{u_i} = H u_i, Sec. 2.1)."""
    out = -0.5 * laplacian(W, cfg) + V[None] * W
    if cfg.xi is not None:
        out = out + apply_nonlocal(W, cfg)
    return out


def inner_matrix(A: np.ndarray, B: np.ndarray, cfg: Config) -> np.ndarray:
    """<A^T B> = (<a_i, b_j>)_ij (Sec. 2.2)."""
    N = A.shape[0]
    return cfg.dV * (A.reshape(N, -1) @ B.reshape(B.shape[0], -1).T)


def cholesky_qr(Wt: np.ndarray, cfg: Config):
    """Orth by Cholesky-based QR (Sec. 3.2): S = <Wt^T Wt>, S = R^T R, W = Wt R^-1.

    Returns (W, S, R); R is upper triangular with positive diagonal.
    """
    N = Wt.shape[0]
    X = Wt.reshape(N, -1)
    S = cfg.dV * (X @ X.T)
    R = cholesky(S, lower=False)
    # rows of W are the columns of Wt R^-1, i.e. W_rows = R^-T X
    Xn = solve_triangular(R, X, trans="T", lower=False)
    return Xn.reshape(Wt.shape), S, R


PIVOT_REL = 1e-13  # a Cholesky pivot below this fraction of max S_ii counts as singular
TAU_SPREAD = 10.0  # per-orbital steps stay within this factor of the common step


def try_cholesky_qr(Wt: np.ndarray, cfg: Config):
    """Cholesky-QR of a trial block, or None when its Gram matrix is not
    numerically positive definite: a pivot (R_kk^2) at or below PIVOT_REL
    times the largest diagonal entry of S, or a failed factorisation.  The
    iteration rejects such a trial like one failing Eq. (ene-de)."""
    N = Wt.shape[0]
    X = Wt.reshape(N, -1)
    S = cfg.dV * (X @ X.T)
    try:
        R = cholesky(S, lower=False)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(R)) or np.min(np.diag(R)) ** 2 <= PIVOT_REL * np.max(np.diag(S)):
        return None
    Xn = solve_triangular(R, X, trans="T", lower=False)
    return Xn.reshape(Wt.shape), S, R


def gradient_residual(W: np.ndarray, HW: np.ndarray, cfg: Config) -> float:
    """||grad E||_F = sqrt(tr<G^T G>), G = HW - W Sigma, Sigma = <(HW)^T W> (Eq. gra)."""
    N = W.shape[0]
    Sig = inner_matrix(HW, W, cfg)
    G = HW.reshape(N, -1) - Sig.T @ W.reshape(N, -1)
    return math.sqrt(cfg.dV * float(np.sum(G * G)))


# --------------------------------------------------------------------------
# the optimiser (Algorithms E and M)
# --------------------------------------------------------------------------
@dataclass
class IterRecord:
    energy: float
    tau: float
    backtracks: int
    forced: bool
    gram_offdiag: float  # max |<Wt^T Wt> - I| of the accepted trial (Fig. 2 diagnostic)
    znorm2: float


@dataclass
class State:
    W: np.ndarray
    rho: np.ndarray
    V: np.ndarray
    E: float
    C: float
    Q: float = 1.0
    l: int = 0
    W_prev: Optional[np.ndarray] = None
    Z_prev: Optional[np.ndarray] = None
    tau_prev: float = 0.0
    tau_next: Optional[float] = None
    D_prev: Optional[np.ndarray] = None  # conjugate-gradient direction of the previous step
    history: List[IterRecord] = field(default_factory=list)
    df: List[float] = field(default_factory=list)


def initial_state(U0: np.ndarray, vext: np.ndarray, cfg: Config) -> State:
    """Initialisation of Algorithm B: orthonormalise U0, then C^0 = E(W^0), Q^0 = 1 (Sec. 3.2)."""
    W, _, _ = cholesky_qr(np.asarray(U0, dtype=np.float64), cfg)
    rho = density(W)
    V = total_potential(rho, vext, cfg)
    E = energy(W, vext, cfg)
    return State(W=W, rho=rho, V=V, E=E, C=E, Q=1.0)


def bb_step(S: np.ndarray, Y: np.ndarray, cfg: Config, l: int) -> float:
    """Barzilai-Borwein step shared by all orbitals (Sec. 3.2).

    tau1 = tr<S^T S> / |tr<S^T Y>|, tau2 = |tr<S^T Y>| / tr<Y^T Y>.
    """
    dV = cfg.dV
    ss = dV * float(np.sum(S * S))
    sy = abs(dV * float(np.sum(S * Y)))
    yy = dV * float(np.sum(Y * Y))
    variant = cfg.bb_variant
    if variant == 3:
        variant = 1 if (l % 2 == 0) else 2
    if variant == 1:
        tau = ss / sy if sy > 0 else float("nan")
    else:
        tau = sy / yy if yy > 0 else float("nan")
    return tau


def bb_step_per_orbital(S: np.ndarray, Y: np.ndarray, cfg: Config, l: int) -> np.ndarray:
    """Barzilai-Borwein step of each orbital (the tau_i of Sec. 3.2, whose
    diagonal elements "can be done in parallel for each orbital"):
    tau_i^1 = <s_i,s_i> / |<s_i,y_i>|, tau_i^2 = |<s_i,y_i>| / <y_i,y_i>;
    tau_0 where a quotient is not a positive number, then clamped."""
    N = S.shape[0]
    dV = cfg.dV
    ss = dV * np.sum((S * S).reshape(N, -1), axis=1)
    sy = np.abs(dV * np.sum((S * Y).reshape(N, -1), axis=1))
    yy = dV * np.sum((Y * Y).reshape(N, -1), axis=1)
    variant = cfg.bb_variant
    if variant == 3:
        variant = 1 if (l % 2 == 0) else 2
    with np.errstate(divide="ignore", invalid="ignore"):
        tau = ss / sy if variant == 1 else sy / yy
    tau = np.where(np.isfinite(tau) & (tau > 0), tau, default_tau0(cfg))
    return np.clip(tau, cfg.tau_min, cfg.tau_max)


def cg_direction(W: np.ndarray, Z: np.ndarray, Z_prev: Optional[np.ndarray], D_prev: Optional[np.ndarray],
                 cfg: Config) -> np.ndarray:
    """Conjugate-gradient direction of each orbital's subproblem (Sec. 3.1
    names conjugate gradients among the solvers): d_i = z_i + beta_i d_i'',
    d_i'' = d_i' - <w_i, d_i'> w_i (the previous direction without its w_i
    component), with the Polak-Ribiere coefficient
    beta_i = max(0, <z_i, z_i - z_i'>) / <z_i', z_i'> (zero on the first step),
    capped so that <z_i, d_i> >= <z_i, z_i> / 2 (every orbital keeps a descent
    direction)."""
    if D_prev is None or Z_prev is None:
        return Z.copy()
    N = Z.shape[0]
    w = W.reshape(N, -1)
    z = Z.reshape(N, -1)
    zp = Z_prev.reshape(N, -1)
    dp = D_prev.reshape(N, -1)
    gamma = cfg.dV * np.sum(w * dp, axis=1)
    dpp = dp - gamma[:, None] * w
    zz = np.sum(z * z, axis=1)
    den = np.sum(zp * zp, axis=1)
    beta = np.where(den > 0, np.maximum(zz - np.sum(z * zp, axis=1), 0.0) / np.where(den > 0, den, 1.0), 0.0)
    zd = np.sum(z * dpp, axis=1)
    cap = np.where(zd < 0, 0.5 * zz / np.where(zd < 0, -zd, 1.0), np.inf)
    beta = np.minimum(beta, cap)
    return (z + beta[:, None] * dpp).reshape(Z.shape)


def newton_steps(D: np.ndarray, Z: np.ndarray, V: np.ndarray, sigma: np.ndarray, cfg: Config) -> np.ndarray:
    """Per-orbital Newton step along d_i of the Rayleigh quotient of orbital i
    with the potential frozen: for a tangent direction d_i (<w_i, d_i> = 0)
    the quotient at w_i - t d_i is sigma_ii - 2 t <z_i, d_i> +
    t^2 <d_i, (H - sigma_ii) d_i> to second order, minimised at
    t_i = <z_i, d_i> / <d_i, (H - sigma_ii) d_i>; tau_0 where that is not a
    positive number; clamped."""
    N = D.shape[0]
    dV = cfg.dV
    HD = apply_h(D, V, cfg)
    d = D.reshape(N, -1)
    zd = dV * np.sum(Z.reshape(N, -1) * d, axis=1)
    den = dV * (np.sum(d * HD.reshape(N, -1), axis=1) - sigma * np.sum(d * d, axis=1))
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where((den > 0) & (zd > 0), zd / den, default_tau0(cfg))
    t = np.where(np.isfinite(t) & (t > 0), t, default_tau0(cfg))
    return np.clip(t, cfg.tau_min, cfg.tau_max)


def default_tau0(cfg: Config) -> float:
    return cfg.tau0 if cfg.tau0 > 0 else 1.0 / lambda_max_kinetic(cfg)


def search_direction(W: np.ndarray, HW: np.ndarray, cfg: Config, full: bool = False):
    """z_i = H w_i - sigma_ii w_i (Sec. 3.2); full=True gives OptM-QR's HW - W Sigma."""
    N = W.shape[0]
    if full:
        Sig = inner_matrix(HW, W, cfg)
        Z = HW.reshape(N, -1) - Sig.T @ W.reshape(N, -1)
        return Z.reshape(W.shape), np.diag(Sig).copy()
    sigma = cfg.dV * np.sum((HW * W).reshape(N, -1), axis=1)
    return HW - sigma[:, None, None, None] * W, sigma


def iterate(st: State, vext: np.ndarray, cfg: Config, full_sigma: bool = False) -> State:
    """One step l of Algorithm M (= Algorithm E when n_org = 1, n_diag = 0).

    With cfg.tau_mode = 1 each orbital takes its own Barzilai-Borwein step
    tau_i (backtracking scales them all by delta^s); with cfg.solver = 1 the
    orbitals move along conjugate-gradient directions D instead of Z, each
    with its Newton step (``newton_steps``; tau is their mean).  The descent
    test of Eq. (ene-de) then uses the first-order decrease of the step
    actually taken, sum_i tau_i <z_i, d_i> (= tau ||Z||_F^2 for one
    steepest-descent step).
    """
    W = st.W
    HW = apply_h(W, st.V, cfg)
    Z, sigma = search_direction(W, HW, cfg, full=full_sigma)
    dV = cfg.dV
    N = W.shape[0]
    D = cg_direction(W, Z, st.Z_prev, st.D_prev, cfg) if cfg.solver == 1 else Z
    zd = dV * np.sum((Z * D).reshape(N, -1), axis=1)  # <z_i, d_i>
    znorm2 = float(np.sum(zd))
    tau0 = default_tau0(cfg)
    if st.tau_next is not None:
        tau = st.tau_next  # computed before a subspace rotation (see subspace_diagonalise)
        st.tau_next = None
    elif st.W_prev is None:
        tau = tau0
    else:
        tau = bb_step(W - st.W_prev, Z - st.Z_prev, cfg, st.l)
    if not math.isfinite(tau) or tau <= 0:
        tau = tau0
    tau = min(max(tau, cfg.tau_min), cfg.tau_max)
    # relative per-orbital steps: tau_i = tau * fac_i
    fac = np.ones(N)
    if cfg.solver == 1:
        # conjugate gradients: each orbital's Newton step; tau is their mean
        tsteps = newton_steps(D, Z, st.V, sigma, cfg)
        tau = float(np.mean(tsteps))
        fac = tsteps / tau
    elif cfg.tau_mode == 1 and st.W_prev is not None:
        # each orbital's own quotient, kept within TAU_SPREAD of the common step
        fac = np.clip(bb_step_per_orbital(W - st.W_prev, Z - st.Z_prev, cfg, st.l) / tau,
                      1.0 / TAU_SPREAD, TAU_SPREAD)

    orth_step = (st.l % max(cfg.n_org, 1)) == 0
    if not orth_step:
        # Algorithm M, intermediate step: plain update, no Orth, no backtracking
        Wn = W - tau * fac[:, None, None, None] * D
        rho = density(Wn)
        V = total_potential(rho, vext, cfg)
        st.W_prev, st.Z_prev, st.D_prev = W, Z, D
        st.W, st.rho, st.V = Wn, rho, V
        st.l += 1
        st.history.append(IterRecord(float("nan"), tau, 0, False, float("nan"), znorm2))
        return st
    decrease = float(np.sum(fac * zd))  # sum_i fac_i <z_i, d_i>

    backtracks = 0
    forced = False
    while True:
        t = tau * cfg.delta ** backtracks
        Wt = W - t * fac[:, None, None, None] * D
        orth = try_cholesky_qr(Wt, cfg)
        if orth is None:
            # a trial without a positive definite Gram matrix is rejected like
            # one failing Eq. (ene-de); past max_backtrack it is a breakdown
            if backtracks >= cfg.max_backtrack:
                raise np.linalg.LinAlgError("trial Gram matrix not positive definite")
            backtracks += 1
            continue
        Wn, Sg, _ = orth
        En = energy(Wn, vext, cfg)
        if En <= st.C - cfg.rho1 * t * decrease:
            break
        if backtracks >= cfg.max_backtrack:
            forced = True
            break
        backtracks += 1
    gram_off = float(np.max(np.abs(Sg - np.eye(Sg.shape[0]))))
    Qn = cfg.eta * st.Q + 1.0
    Cn = (cfg.eta * st.Q * st.C + En) / Qn
    rho = density(Wn)
    V = total_potential(rho, vext, cfg)
    st.W_prev, st.Z_prev, st.D_prev = W, Z, D
    E_old = st.E
    st.W, st.rho, st.V, st.E, st.C, st.Q = Wn, rho, V, En, Cn, Qn
    st.tau_prev = t
    st.l += 1
    st.df.append(abs(E_old - En) / (abs(E_old) + 1.0))
    st.history.append(IterRecord(En, t, backtracks, forced, gram_off, znorm2))
    if cfg.n_diag > 0 and st.l % cfg.n_diag == 0:
        subspace_diagonalise(st, vext, cfg, full_sigma)
    return st


def subspace_diagonalise(st: State, vext: np.ndarray, cfg: Config, full_sigma: bool = False) -> None:
    """Sec. 3.3: P^T Sigma P = Gamma, W <- W P (rho, H and E unchanged).

    Reading: the Barzilai-Borwein step of the next step is taken from S and Y
    of the orbitals before the rotation, so it is computed here, first.  The
    rotated orbitals then serve as W^(l) for the step after.
    """
    W = st.W
    N = W.shape[0]
    HW = apply_h(W, st.V, cfg)
    Zn, _ = search_direction(W, HW, cfg, full=full_sigma)
    st.tau_next = bb_step(W - st.W_prev, Zn - st.Z_prev, cfg, st.l)
    Sig = inner_matrix(W, HW, cfg)
    Sig = 0.5 * (Sig + Sig.T)
    _, P = np.linalg.eigh(Sig)
    st.W = (P.T @ W.reshape(N, -1)).reshape(W.shape)
    st.W_prev = None
    st.Z_prev = None
    st.D_prev = None


def converged_df(df: List[float], e_tol: float) -> bool:
    """Sec. 4.2 criterion: (df^l + df^(l-1) + df^(l-2)) / 3 < e_tol."""
    return e_tol > 0 and len(df) >= 3 and (df[-1] + df[-2] + df[-3]) / 3.0 < e_tol


def run(U0: np.ndarray, vext: np.ndarray, cfg: Config, max_iter: int,
        e_tol: float = 0.0, grad_tol: float = 0.0, full_sigma: bool = False,
        st: Optional[State] = None) -> State:
    """Algorithm E/M inner loop from U0 for at most max_iter steps."""
    if st is None:
        st = initial_state(U0, vext, cfg)
    for _ in range(max_iter):
        if grad_tol > 0:
            HW = apply_h(st.W, st.V, cfg)
            if gradient_residual(st.W, HW, cfg) < grad_tol:
                break
        iterate(st, vext, cfg, full_sigma=full_sigma)
        if converged_df(st.df, e_tol):
            break
    return st


# --------------------------------------------------------------------------
# derivatives (differentiation form)
# --------------------------------------------------------------------------
def energy_gradient_orbitals(U: np.ndarray, vext: np.ndarray, cfg: Config) -> np.ndarray:
    """dE/dU with respect to the raw array entries: 2 f dV H(rho_U) U.

    Follows from E_{u_i} = H(rho) u_i (Sec. 2.1) with occupation f and the
    quadrature weight dV of the discrete integrals.
    """
    rho = density(U)
    V = total_potential(rho, vext, cfg)
    return 2.0 * F_OCC * cfg.dV * apply_h(U, V, cfg)


def energy_gradient_atoms(U: np.ndarray, cfg: Config, R: np.ndarray, Z: np.ndarray,
                          width: float):
    """dE/dR_I and dE/dZ_I at fixed orbitals.

    Only E_ext = dV sum rho Vext depends on the atoms.  With d = r - R_I - nL,
    g = exp(-|d|^2 / (2 width^2)):
      dVext/dR_I = -Z_I sum_n g d / width^2,  dVext/dZ_I = -sum_n g.
    """
    rho = density(U)
    x, y, z = grid_coords(cfg)
    Lx, Ly, Lz = (float(v) for v in cfg.L)
    R = wrap_positions(R, cfg)
    M = len(Z)
    dR = np.zeros((M, 3))
    dZ = np.zeros(M)
    two_s2 = 2.0 * width * width
    s2 = width * width
    dV = cfg.dV
    for I in range(M):
        for a, b, c in itertools.product((-1, 0, 1), repeat=3):
            dx = (x - R[I, 0] - a * Lx)[None, None, :]
            dy = (y - R[I, 1] - b * Ly)[None, :, None]
            dz = (z - R[I, 2] - c * Lz)[:, None, None]
            g = np.exp(-(dx * dx + dy * dy + dz * dz) / two_s2)
            rg = rho * g
            dZ[I] -= dV * float(np.sum(rg))
            dR[I, 0] -= dV * Z[I] * float(np.sum(rg * dx)) / s2
            dR[I, 1] -= dV * Z[I] * float(np.sum(rg * dy)) / s2
            dR[I, 2] -= dV * Z[I] * float(np.sum(rg * dz)) / s2
    return dR, dZ
