"""Seeded synthetic inputs for the average spectrum method.

This module builds the *inputs* of the problem only: imaginary-time grids,
real-frequency grids with their Riemann weights, the fermionic and bosonic
imaginary-time kernels, synthetic true spectra, data with (correlated) Gaussian
noise, the covariance of that noise and the block partitions.  It contains none
of the sampling method's arithmetic, and it is the only module shared by the
CPU oracle and the CUDA path.

Readings of the paper used here (Ghanem & Koch, arXiv:1912.01379):
  * Discretisation g = K fbar with fbar_n = f(x_n) w_n (Sec. V.B, Eq. Riemann).
  * Non-uniform grids x_n = P^{-1}((n - 1/2)/N) from a density rho and weights
    w_n = 1/(N rho(x_n)) (Sec. V.B).  A Gaussian density on a finite interval is
    read as the normal density truncated to that interval.
  * Uniform grids use the interval midpoints omega_n = a + (n - 1/2) d_omega, so
    w_n = d_omega (Sec. V.A, Fig. cutoff_dependence).
  * Fermionic imaginary-time kernel e^{-tau w}/(1 + e^{-beta w}) (Sec. II) with
    the -1/(2 pi) prefactor dropped so that K > 0.  Bosonic kernel in the
    tau <-> beta - tau symmetric form w (e^{-tau w} + e^{-(beta - tau) w}) /
    (1 - e^{-beta w}) on w >= 0, with its limit 2/beta at w = 0.
  * Data G = K fbar_true + L z, z ~ N(0, I) from numpy PCG64(seed), where
    C = L L^T is the covariance of the mean passed to the method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import special


# --------------------------------------------------------------------------
# kernels (stable forms)
# --------------------------------------------------------------------------

def fermionic_kernel(tau: np.ndarray, omega: np.ndarray, beta: float) -> np.ndarray:
    """K(tau, w) = e^{-tau w} / (1 + e^{-beta w}), evaluated without overflow."""
    t = np.asarray(tau, dtype=np.float64)[:, None]
    w = np.asarray(omega, dtype=np.float64)[None, :]
    pos = w >= 0
    wp = np.where(pos, w, 0.0)
    wn = np.where(pos, 0.0, w)
    k_pos = np.exp(-t * wp) / (1.0 + np.exp(-beta * wp))
    k_neg = np.exp((beta - t) * wn) / (1.0 + np.exp(beta * wn))
    return np.where(pos, k_pos, k_neg)


def bosonic_kernel(tau: np.ndarray, omega: np.ndarray, beta: float) -> np.ndarray:
    """K(tau, w) = w (e^{-tau w} + e^{-(beta - tau) w}) / (1 - e^{-beta w}), w >= 0."""
    t = np.asarray(tau, dtype=np.float64)[:, None]
    w = np.asarray(omega, dtype=np.float64)[None, :]
    if np.any(w < 0):
        raise ValueError("bosonic kernel is defined on omega >= 0")
    small = w < 1e-12
    ws = np.where(small, 1.0, w)
    k = ws * (np.exp(-t * ws) + np.exp(-(beta - t) * ws)) / (-np.expm1(-beta * ws))
    return np.where(small, 2.0 / beta, k)


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------

def uniform_grid(a: float, b: float, n: int):
    """Midpoints of n equal intervals on [a, b] and their widths."""
    d = (b - a) / n
    omega = a + (np.arange(n) + 0.5) * d
    return omega, np.full(n, d)


def gaussian_grid(a: float, b: float, n: int, sigma: float, center: float = 0.0):
    """Grid from a normal density truncated to [a, b]: x_n = P^{-1}((n-1/2)/N)."""
    za, zb = (a - center) / sigma, (b - center) / sigma
    pa, pb = special.ndtr(za), special.ndtr(zb)
    z = (np.arange(n) + 0.5) / n
    omega = center + sigma * special.ndtri(pa + z * (pb - pa))
    rho = np.exp(-0.5 * ((omega - center) / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi) * (pb - pa))
    return omega, 1.0 / (n * rho)


def tau_grid(beta: float, m: int) -> np.ndarray:
    return np.linspace(0.0, beta, m)


# --------------------------------------------------------------------------
# spectra and noise
# --------------------------------------------------------------------------

def gauss_pdf(x, c, s):
    return np.exp(-0.5 * ((x - c) / s) ** 2) / (s * math.sqrt(2 * math.pi))


def lorentz_pdf(x, c, g):
    return (g / math.pi) / ((x - c) ** 2 + g * g)


def exp_decay_covariance(tau: np.ndarray, amp: float, length: float) -> np.ndarray:
    d = np.abs(tau[:, None] - tau[None, :])
    return amp * np.exp(-d / length)


def contiguous_blocks(n: int, sizes) -> np.ndarray:
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int32)
    assert int(np.sum(sizes)) == n
    return starts


def equal_blocks(n: int, nb: int) -> np.ndarray:
    """nb contiguous blocks of sizes floor(n/nb) or ceil(n/nb)."""
    edges = np.floor(np.arange(nb + 1) * n / nb).astype(np.int64)
    return edges[:-1].astype(np.int32)


@dataclass
class Problem:
    """One continuation problem, all FP64 / int32 host arrays."""
    name: str
    K: np.ndarray            # M x N, kernel acting on fbar
    G: np.ndarray            # M, data
    C: np.ndarray            # M x M, covariance of the data mean
    omega: np.ndarray        # N grid points
    w: np.ndarray            # N Riemann weights, A = fbar / w
    levels: list             # list of int32 arrays of block starts (each begins at 0)
    fbar_true: np.ndarray    # N, the spectrum the data were generated from
    chains: int = 16
    burn_in: int = 100
    sweeps: int = 1000
    extra: dict = field(default_factory=dict)

    @property
    def M(self):
        return self.K.shape[0]

    @property
    def N(self):
        return self.K.shape[1]


def _make(name, K, fbar, C, omega, w, levels, rng, **kw):
    L = np.linalg.cholesky(C)
    G = K @ fbar + L @ rng.standard_normal(K.shape[0])
    return Problem(name, K, G, C, omega, w, [np.asarray(l, np.int32) for l in levels], fbar, **kw)


# --------------------------------------------------------------------------
# the five synthetic workloads
# --------------------------------------------------------------------------

def plain_modes_problem(seed: int = 1001) -> Problem:
    """Plain global modes: fermionic, beta=10, N_tau=20, N_omega=50 on [-5,5],
    two Gaussians at +-1.5 (width 0.5, weight 0.5 each), iid noise 1e-3,
    one level with one block, 16 chains x 1e4 sweeps after 1e3 burn-in."""
    rng = np.random.Generator(np.random.PCG64(seed))
    beta, M, N = 10.0, 20, 50
    tau = tau_grid(beta, M)
    omega, w = uniform_grid(-5.0, 5.0, N)
    A = 0.5 * gauss_pdf(omega, -1.5, 0.5) + 0.5 * gauss_pdf(omega, 1.5, 0.5)
    K = fermionic_kernel(tau, omega, beta)
    C = np.eye(M) * 1e-3 ** 2
    return _make("plain_modes_b10_M20_N50", K, A * w, C, omega, w, [[0]], rng,
                 chains=16, burn_in=1000, sweeps=10000)


def blocked_modes_problem(seed: int = 1002, chains: int = 1024) -> Problem:
    """Blocked modes, one problem: fermionic, beta=20, N_tau=100, N_omega=400 on a
    Gaussian-density grid (sigma=3) on [-8,8], 8 blocks of 50, quasiparticle
    peak at 0 (width 0.2, weight 0.3) plus Hubbard bands at +-3 (width 1,
    weight 0.35 each), covariance 1e-4 exp(-|tau-tau'|/0.5), 1024 chains."""
    rng = np.random.Generator(np.random.PCG64(seed))
    beta, M, N = 20.0, 100, 400
    tau = tau_grid(beta, M)
    omega, w = gaussian_grid(-8.0, 8.0, N, 3.0)
    A = 0.3 * gauss_pdf(omega, 0.0, 0.2) + 0.35 * gauss_pdf(omega, -3.0, 1.0) + 0.35 * gauss_pdf(omega, 3.0, 1.0)
    K = fermionic_kernel(tau, omega, beta)
    C = exp_decay_covariance(tau, 1e-4, 0.5)
    levels = [[0], equal_blocks(N, 8)]
    return _make("blocked_modes_b20_M100_N400", K, A * w, C, omega, w, levels, rng,
                 chains=chains, burn_in=1000, sweeps=10000)


def batch_problems(seed: int = 1003, n_problems: int = 256, chains: int = 64):
    """Batching workload: independent problems with N_omega ~ U{100..1000},
    N_tau ~ U{50..200}, beta ~ U[5,40], fermionic or bosonic kernel, blocks of
    25-100 points, 1-3 Gaussian peaks, iid noise sigma log-uniform in
    [1e-5, 1e-3], 64 chains per problem."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for p in range(n_problems):
        N = int(rng.integers(100, 1001))
        M = int(rng.integers(50, 201))
        beta = float(rng.uniform(5.0, 40.0))
        bos = bool(rng.integers(0, 2))
        a, b = (0.0, 8.0) if bos else (-8.0, 8.0)
        omega, w = uniform_grid(a, b, N)
        tau = tau_grid(beta, M)
        K = bosonic_kernel(tau, omega, beta) if bos else fermionic_kernel(tau, omega, beta)
        npk = int(rng.integers(1, 4))
        span = b - a
        cs = rng.uniform(a + 0.2 * span, b - 0.2 * span, npk)
        ss = rng.uniform(0.1, 1.0, npk)
        ws = rng.dirichlet(np.ones(npk))
        A = sum(ws[i] * gauss_pdf(omega, cs[i], ss[i]) for i in range(npk))
        sig = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-3))))
        sizes = []
        rem = N
        while rem > 0:
            s = int(rng.integers(25, 101))
            s = min(s, rem)
            sizes.append(s)
            rem -= s
        if len(sizes) > 1 and sizes[-1] < 25:   # a short tail joins its neighbour, in two halves if > 100
            joined = sizes.pop() + sizes.pop()
            sizes += [joined] if joined <= 100 else [joined // 2, joined - joined // 2]
        levels = [[0], contiguous_blocks(N, sizes)]
        C = np.eye(M) * sig * sig
        out.append(_make(f"batch{p}_{'bos' if bos else 'fer'}_M{M}_N{N}", K, A * w, C, omega, w,
                         levels, rng, chains=chains, burn_in=500, sweeps=5000,
                         extra={"beta": beta, "bosonic": bos, "sigma": sig}))
    return out


def differentiation_problem(seed: int = 1004, chains: int = 4096) -> Problem:
    """Differentiation workload: N_tau=64, N_omega=200 uniform on [-6,6], beta=16,
    three random Gaussians, iid noise 1e-4, global level plus 8 blocks of 25."""
    rng = np.random.Generator(np.random.PCG64(seed))
    beta, M, N = 16.0, 64, 200
    tau = tau_grid(beta, M)
    omega, w = uniform_grid(-6.0, 6.0, N)
    cs = rng.uniform(-4.0, 4.0, 3)
    ss = rng.uniform(0.2, 1.0, 3)
    ws = rng.dirichlet(np.ones(3))
    A = sum(ws[i] * gauss_pdf(omega, cs[i], ss[i]) for i in range(3))
    K = fermionic_kernel(tau, omega, beta)
    C = np.eye(M) * 1e-4 ** 2
    levels = [[0], equal_blocks(N, 8)]
    return _make("differentiation_b16_M64_N200", K, A * w, C, omega, w, levels, rng,
                 chains=chains, burn_in=500, sweeps=5000)


def grid_sweep_problem(N: int, density: str = "uniform", seed: int = 1005, chains: int = 8192) -> Problem:
    """Grid-size sweep: N_tau=400, beta=50, N_omega in {250,500,1000,2000} on
    [-10,10], uniform or Gaussian-density (sigma=4), metallic spectrum
    (Lorentzian HWHM 0.1 weight 0.2 plus Gaussian bands at +-4, width 1.5,
    weight 0.4 each) renormalised on [-10,10], covariance
    1e-5 exp(-|tau-tau'|/1.0), 16 blocks, 8192 chains."""
    rng = np.random.Generator(np.random.PCG64(seed + N))
    beta, M = 50.0, 400
    tau = tau_grid(beta, M)
    if density == "uniform":
        omega, w = uniform_grid(-10.0, 10.0, N)
    else:
        omega, w = gaussian_grid(-10.0, 10.0, N, 4.0)
    A = 0.2 * lorentz_pdf(omega, 0.0, 0.1) + 0.4 * gauss_pdf(omega, -4.0, 1.5) + 0.4 * gauss_pdf(omega, 4.0, 1.5)
    A = A / np.sum(A * w)
    K = fermionic_kernel(tau, omega, beta)
    C = exp_decay_covariance(tau, 1e-5, 1.0)
    levels = [[0], equal_blocks(N, 16)]
    return _make(f"grid_sweep_{density}_N{N}", K, A * w, C, omega, w, levels, rng,
                 chains=chains, burn_in=500, sweeps=5000)


# --------------------------------------------------------------------------
# the paper's own test case (Sec. III): optical conductivity on bosonic
# Matsubara frequencies
# --------------------------------------------------------------------------

def optical_conductivity(omega, model: int = 2):
    """sigma(omega) of the paper's test models (Eq. model): a cutoff factor
    1/(1 + (omega/4)^6) times a Drude peak (weight 0.3, width 0.3 for model 1,
    0.6 for model 2) and two Lorentzians of weight 0.2 and width 1.2 at +-3."""
    omega = np.asarray(omega, dtype=np.float64)
    g0 = 0.3 if model == 1 else 0.6
    peaks = 0.3 / (1.0 + (omega / g0) ** 2)
    for sgn in (1.0, -1.0):
        peaks = peaks + 0.2 / (1.0 + ((omega + sgn * 3.0) / 1.2) ** 2)
    return peaks / (1.0 + (omega / 4.0) ** 6)


def matsubara_kernel(omega_m, omega):
    """K(i omega_m, omega) = (2/pi) omega^2 / (omega_m^2 + omega^2) (Eq. optcond) on omega > 0."""
    om = np.asarray(omega_m, dtype=np.float64)[:, None]
    w = np.asarray(omega, dtype=np.float64)[None, :]
    return (2.0 / math.pi) * w * w / (om * om + w * w)


def matsubara_data(omega_m, model: int = 2):
    """Pi(i omega_m) = (2/pi) int_0^inf omega^2/(omega_m^2 + omega^2) sigma(omega) d omega by
    adaptive quadrature (the integrand is smooth; tolerance 1e-13)."""
    from scipy import integrate
    out = np.empty(len(omega_m))
    for i, om in enumerate(omega_m):
        f = lambda x, om=om: (2.0 / math.pi) * x * x / (om * om + x * x) * optical_conductivity(x, model)
        v = 0.0
        for a, b in ((0.0, 2.0), (2.0, 6.0), (6.0, 20.0), (20.0, np.inf)):
            v += integrate.quad(f, a, b, epsabs=1e-14, epsrel=1e-13, limit=400)[0]
        out[i] = v
    return out


def half_line_grid(kind: str, N: int, param: float):
    """Grids on [0, inf) from a density rho (Sec. V.B table): x_n = x(z_n), z_n = (n-1/2)/N,
    weights w_n = (1/N) dx/dz.  kind: 'gaussian' (alpha), 'exponential' (beta),
    'lorentzian' (gamma)."""
    z = (np.arange(N) + 0.5) / N
    if kind == "gaussian":
        e = special.erfinv(z)
        x = math.sqrt(2.0) * param * e
        dxdz = math.sqrt(2.0 * math.pi) * param / 2.0 / np.exp(-e * e)
    elif kind == "exponential":
        x = -param * np.log1p(-z)
        dxdz = param / (1.0 - z)
    elif kind == "lorentzian":
        x = param * np.tan(math.pi * z / 2.0)
        dxdz = math.pi * param / 2.0 / np.cos(math.pi * z / 2.0) ** 2
    else:
        raise ValueError(kind)
    return x, dxdz / N


def paper_problem(model: int = 2, noise: float = 1e-3, grid: str = "uniform", N: int = 64,
                  d_omega: float = 0.25, seed: int = 1006, chains: int = 1024, grid_param=None) -> Problem:
    """The paper's test case: optical conductivity model 1 or 2 continued from
    Pi(i omega_m) (1 + r_m) on the first 60 bosonic Matsubara frequencies at
    beta = 15, relative noise r_m of standard deviation `noise` (reading of the
    paper's sigma_Pi), on a uniform grid omega_n = (n - 1/2) d_omega or a
    Gaussian (alpha = 4), exponential (beta = 3) or Lorentzian (gamma = 2.5)
    grid of N points (grid_param overrides alpha, beta or gamma).  Levels: the
    whole grid only (callers add blocks)."""
    kinds = {"uniform": 0, "gaussian": 1, "exponential": 2, "lorentzian": 3}
    rng = np.random.Generator(np.random.PCG64(seed + 7 * N + 1000 * kinds[grid] + 100000 * model))
    beta, M = 15.0, 60
    om = 2.0 * math.pi * np.arange(M) / beta
    if grid == "uniform":
        omega = (np.arange(N) + 0.5) * d_omega
        w = np.full(N, d_omega)
    else:
        param = grid_param if grid_param is not None else {"gaussian": 4.0, "exponential": 3.0, "lorentzian": 2.5}[grid]
        omega, w = half_line_grid(grid, N, param)
    K = matsubara_kernel(om, omega)
    pi_m = matsubara_data(om, model)
    G = pi_m * (1.0 + noise * rng.standard_normal(M))
    C = np.diag((noise * pi_m) ** 2)
    fbar = optical_conductivity(omega, model) * w
    return Problem(f"paper_model{model}_{grid}_N{N}", K, G, C, omega, w, [np.array([0], np.int32)], fbar,
                   chains=chains, burn_in=500, sweeps=5000,
                   extra={"beta": beta, "omega_m": om, "pi_exact": pi_m, "noise": noise, "model": model})


# --------------------------------------------------------------------------
# small cases for tests
# --------------------------------------------------------------------------

def small_problem(M: int, N: int, seed: int, levels=None, noise: float = 1e-3,
                  beta: float = 10.0, offset: float = 0.0, bosonic: bool = False) -> Problem:
    """A small random fermionic (or bosonic) problem for parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tau = tau_grid(beta, M)
    if bosonic:
        omega, w = uniform_grid(0.0, 6.0, N)
        K = bosonic_kernel(tau, omega, beta)
    else:
        omega, w = uniform_grid(-5.0, 5.0, N)
        K = fermionic_kernel(tau, omega, beta)
    A = 0.5 * gauss_pdf(omega, -1.2, 0.6) + 0.5 * gauss_pdf(omega, 1.5, 0.4) + offset
    C = np.eye(M) * noise * noise
    if levels is None:
        levels = [[0]]
    return _make(f"small_M{M}_N{N}_s{seed}", K, A * w, C, omega, w, levels, rng)


def levels_flat(levels) -> tuple[np.ndarray, np.ndarray]:
    """Pack a list of per-level block-start arrays as (level_nblocks, block_start)."""
    nb = np.array([len(l) for l in levels], dtype=np.int32)
    bs = np.concatenate([np.asarray(l, dtype=np.int32) for l in levels]).astype(np.int32)
    return nb, bs


# --------------------------------------------------------------------------
# grid-density (default-model) parameters theta for the differentiation
# workload: a mixture of three Gaussians truncated to [a, b]
#   theta = (c1, c2, c3, log s1, log s2, log s3, a2, a3), weights softmax(0, a2, a3)
# grid x_n = P^{-1}((n - 1/2)/N), weights w_n = 1/(N rho(x_n)) (Sec. V.B).
# --------------------------------------------------------------------------

THETA0 = np.array([-3.0, 0.0, 3.0, np.log(2.0), np.log(2.0), np.log(2.0), 0.0, 0.0])


def _mixture(theta):
    c = np.asarray(theta[:3], dtype=np.float64)
    s = np.exp(np.asarray(theta[3:6], dtype=np.float64))
    a = np.array([0.0, theta[6], theta[7]])
    pi = np.exp(a - a.max())
    return c, s, pi / pi.sum()


def mixture_cdf_pdf(x, theta, a=-6.0, b=6.0):
    """CDF and density of the truncated mixture at x."""
    c, s, pi = _mixture(theta)
    x = np.asarray(x, dtype=np.float64)[..., None]
    Z = np.sum(pi * (special.ndtr((b - c) / s) - special.ndtr((a - c) / s)))
    cdf = np.sum(pi * (special.ndtr((x - c) / s) - special.ndtr((a - c) / s)), axis=-1) / Z
    pdf = np.sum(pi * np.exp(-0.5 * ((x - c) / s) ** 2) / (s * math.sqrt(2 * math.pi)), axis=-1) / Z
    return cdf, pdf


def mixture_grid(theta, N, a=-6.0, b=6.0):
    """x_n = P^{-1}((n - 1/2)/N) by bisection then Newton, and w_n = 1/(N rho(x_n))."""
    z = (np.arange(N) + 0.5) / N
    lo, hi = np.full(N, a), np.full(N, b)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        cm, _ = mixture_cdf_pdf(mid, theta, a, b)
        lo, hi = np.where(cm < z, mid, lo), np.where(cm < z, hi, mid)
    x = 0.5 * (lo + hi)
    for _ in range(3):
        cm, pm = mixture_cdf_pdf(x, theta, a, b)
        x = x - (cm - z) / pm
    _, pm = mixture_cdf_pdf(x, theta, a, b)
    return x, 1.0 / (N * pm)


def fermionic_kernel_domega(tau, omega, beta):
    """dK/d omega of the fermionic kernel: K (-tau + beta / (1 + e^{beta omega}))."""
    K = fermionic_kernel(tau, omega, beta)
    t = np.asarray(tau, dtype=np.float64)[:, None]
    w = np.asarray(omega, dtype=np.float64)[None, :]
    return K * (-t + beta * special.expit(-beta * w))


def theta_problem(theta=None, N=200, M=64, beta=16.0, noise=1e-4, seed=1004, offset=0.0,
                  levels=None, h=1e-6):
    """The differentiation workload on the theta-grid: K(theta) acting on fbar,
    w(theta), dK/dtheta (P x M x N), dw/dtheta (P x N).  The data G are made
    once from the true spectrum on a fine grid, so they do not depend on theta."""
    theta = THETA0.copy() if theta is None else np.asarray(theta, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    cs = rng.uniform(-4.0, 4.0, 3)
    ss = rng.uniform(0.2, 1.0, 3)
    ws = rng.dirichlet(np.ones(3))
    A = lambda om: sum(ws[i] * gauss_pdf(om, cs[i], ss[i]) for i in range(3)) + offset
    tau = tau_grid(beta, M)
    fine, dfine = uniform_grid(-6.0, 6.0, 24000)
    G0 = fermionic_kernel(tau, fine, beta) @ (A(fine) * dfine)
    C = np.eye(M) * noise * noise
    G = G0 + np.linalg.cholesky(C) @ rng.standard_normal(M)
    x, w = mixture_grid(theta, N)
    K = fermionic_kernel(tau, x, beta)
    P = len(theta)
    dx = np.zeros((P, N))
    dw = np.zeros((P, N))
    for p_ in range(P):
        e = np.zeros(P)
        e[p_] = h
        xp, wp = mixture_grid(theta + e, N)
        xm, wm = mixture_grid(theta - e, N)
        dx[p_] = (xp - xm) / (2 * h)
        dw[p_] = (wp - wm) / (2 * h)
    dK = fermionic_kernel_domega(tau, x, beta)[None, :, :] * dx[:, None, :]
    if levels is None:
        levels = [[0], equal_blocks(N, 8)] if N >= 16 else [[0]]
    prob = Problem(f"theta_grid_N{N}_M{M}", K, G, C, x, w, [np.asarray(l, np.int32) for l in levels],
                   A(x) * w, chains=4096, burn_in=500, sweeps=5000)
    prob.extra.update({"theta": theta, "dK_dtheta": dK, "dw_dtheta": dw, "dx_dtheta": dx, "beta": beta,
                       "tau": tau})
    return prob
