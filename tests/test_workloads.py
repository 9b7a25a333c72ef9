"""Pins of the seeded synthetic inputs (paper_1912_01379_gb300/workloads.py)
against what the workload recipes state and what the mathematics fixes,
independently of the generator's own formulas:

* kernels (Sec. II): the fermionic kernel against its plain expression where
  that does not overflow, its particle-hole symmetry K(beta - tau, w) = K(tau, -w)
  and finite values at |beta w| = 1600; the bosonic kernel against its plain
  expression, its tau <-> beta - tau symmetry and its limit 2/beta at w -> 0;
* grids (Sec. V.A-B): midpoints and widths of the uniform grid; the
  Gaussian-density grid puts the mass fraction (n - 1/2)/N of the truncated
  normal (scipy.stats.truncnorm) below x_n, and its weights add up to the
  length of the interval;
* every workload: sizes, levels, covariance, a non-negative true spectrum of
  unit weight, and data whose whitened residual against the true spectrum is a
  plausible chi^2 draw with M degrees of freedom (the noise is drawn from the
  covariance handed to the method, not from a scaled copy of it).
"""
import numpy as np
import pytest
from scipy import stats

from paper_1912_01379_gb300 import workloads as W


def _chi2_z(p):
    """(chi^2 - M) / sqrt(2 M) of the data against the true spectrum."""
    r = p.G - p.K @ p.fbar_true
    return (r @ np.linalg.solve(p.C, r) - p.M) / np.sqrt(2.0 * p.M)


def _exp_cov(tau, amp, length):
    return np.array([[amp * np.exp(-abs(a - b) / length) for b in tau] for a in tau])


# ---------------------------------------------------------------- kernels

def test_fermionic_kernel_expression_and_symmetry():
    beta = 10.0
    tau = np.linspace(0.0, beta, 7)
    omega = np.linspace(-5.0, 5.0, 11)
    K = W.fermionic_kernel(tau, omega, beta)
    plain = np.array([[np.exp(-t * w) / (1.0 + np.exp(-beta * w)) for w in omega] for t in tau])
    assert np.allclose(K, plain, rtol=1e-14, atol=0)
    assert np.allclose(W.fermionic_kernel(beta - tau, omega, beta), W.fermionic_kernel(tau, -omega, beta),
                       rtol=1e-13, atol=0)
    far = W.fermionic_kernel(tau, np.array([-160.0, 160.0]), beta)
    assert np.all(np.isfinite(far)) and np.all(far >= 0)


def test_bosonic_kernel_expression_symmetry_and_limit():
    beta = 15.0
    tau = np.linspace(0.0, beta, 9)
    omega = np.linspace(0.1, 8.0, 12)
    K = W.bosonic_kernel(tau, omega, beta)
    plain = np.array([[w * (np.exp(-t * w) + np.exp(-(beta - t) * w)) / (1.0 - np.exp(-beta * w))
                       for w in omega] for t in tau])
    assert np.allclose(K, plain, rtol=1e-13, atol=0)
    assert np.allclose(W.bosonic_kernel(beta - tau, omega, beta), K, rtol=1e-13, atol=0)
    small = W.bosonic_kernel(tau, np.array([0.0, 1e-7]), beta)
    assert np.allclose(small, 2.0 / beta, rtol=1e-6, atol=0)
    with pytest.raises(ValueError):
        W.bosonic_kernel(tau, np.array([-1.0]), beta)


# ---------------------------------------------------------------- grids

def test_uniform_grid_midpoints():
    omega, w = W.uniform_grid(-5.0, 5.0, 50)
    assert omega[0] == pytest.approx(-4.9) and omega[-1] == pytest.approx(4.9)
    assert np.allclose(np.diff(omega), 0.2) and np.allclose(w, 0.2)
    assert w.sum() == pytest.approx(10.0)


@pytest.mark.parametrize("a,b,n,sigma", [(-8.0, 8.0, 400, 3.0), (-10.0, 10.0, 2000, 4.0)])
def test_gaussian_grid_quantiles_and_weights(a, b, n, sigma):
    omega, w = W.gaussian_grid(a, b, n, sigma)
    cdf = stats.truncnorm(a / sigma, b / sigma, scale=sigma).cdf(omega)
    assert np.abs(cdf - (np.arange(n) + 0.5) / n).max() < 1e-12
    assert np.all(np.diff(omega) > 0) and omega[0] > a and omega[-1] < b
    # midpoint rule for the integral of dx over [a, b] in the quantile variable
    assert abs(w.sum() - (b - a)) < 0.005 * (b - a)


# ---------------------------------------------------------------- workloads

def test_plain_modes_workload():
    p = W.plain_modes_problem()
    assert (p.M, p.N) == (20, 50)
    assert p.omega.min() > -5.0 and p.omega.max() < 5.0 and np.allclose(p.w, 0.2)
    assert len(p.levels) == 1 and list(p.levels[0]) == [0]
    assert np.allclose(p.C, np.eye(20) * 1e-6, rtol=0, atol=1e-20)
    assert (p.chains, p.burn_in, p.sweeps) == (16, 1000, 10000)
    assert np.all(p.fbar_true >= 0) and p.fbar_true.sum() == pytest.approx(1.0, abs=1e-6)
    assert abs(_chi2_z(p)) < 6.0


def test_blocked_modes_workload():
    p = W.blocked_modes_problem()
    assert (p.M, p.N, p.chains) == (100, 400, 1024)
    tau = np.linspace(0.0, 20.0, 100)
    assert np.allclose(p.C, _exp_cov(tau, 1e-4, 0.5), rtol=1e-13, atol=0)
    assert list(p.levels[0]) == [0] and list(p.levels[1]) == list(range(0, 400, 50))
    assert p.omega.min() > -8.0 and p.omega.max() < 8.0
    assert np.all(p.fbar_true >= 0) and p.fbar_true.sum() == pytest.approx(1.0, abs=1e-3)
    assert abs(_chi2_z(p)) < 6.0


def test_differentiation_workload():
    p = W.differentiation_problem()
    assert (p.M, p.N, p.chains) == (64, 200, 4096)
    assert np.allclose(p.w, 12.0 / 200) and p.omega.min() > -6.0 and p.omega.max() < 6.0
    assert np.allclose(p.C, np.eye(64) * 1e-8, rtol=0, atol=1e-24)
    assert np.all(p.fbar_true >= 0) and p.fbar_true.sum() == pytest.approx(1.0, abs=1e-3)
    assert abs(_chi2_z(p)) < 6.0


@pytest.mark.parametrize("N", [250, 500, 1000, 2000])
@pytest.mark.parametrize("density", ["uniform", "gaussian"])
def test_grid_sweep_workload(N, density):
    p = W.grid_sweep_problem(N, density, chains=16)
    assert (p.M, p.N) == (400, N)
    tau = np.linspace(0.0, 50.0, 400)
    assert np.allclose(p.C, _exp_cov(tau, 1e-5, 1.0), rtol=1e-13, atol=0)
    assert len(p.levels) == 2 and len(p.levels[1]) == 16
    sizes = np.diff(np.append(p.levels[1], N))
    assert sizes.min() >= N // 16 and sizes.max() <= -(-N // 16)
    assert p.omega.min() > -10.0 and p.omega.max() < 10.0
    assert np.all(p.fbar_true >= 0) and p.fbar_true.sum() == pytest.approx(1.0, abs=1e-12)
    assert abs(_chi2_z(p)) < 6.0


def test_batch_workload():
    ps = W.batch_problems()
    assert len(ps) == 256
    for p in ps:
        assert 100 <= p.N <= 1000 and 50 <= p.M <= 200 and p.chains == 64
        beta, sig = p.extra["beta"], p.extra["sigma"]
        assert 5.0 <= beta <= 40.0 and 1e-5 <= sig <= 1e-3
        assert np.allclose(p.C, np.eye(p.M) * sig * sig, rtol=1e-14, atol=0)
        sizes = np.diff(np.append(p.levels[1], p.N))
        assert list(p.levels[0]) == [0] and sizes.min() >= 25 and sizes.max() <= 100, p.name
        if p.extra["bosonic"]:
            assert p.omega.min() > 0.0 and p.omega.max() < 8.0
        # peaks centred in the middle 60 % of the window with widths <= 1: most of the weight is inside
        assert np.all(p.fbar_true >= 0) and 0.85 < p.fbar_true.sum() < 1.0 + 1e-9
        assert abs(_chi2_z(p)) < 6.0, p.name
    assert 0 < sum(p.extra["bosonic"] for p in ps) < 256
