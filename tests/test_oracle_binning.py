"""The oracle's binning estimate of the Monte Carlo error, pinned against an
AR(1) series x_t = rho x_{t-1} + sqrt(1 - rho^2) e_t (unit variance), whose
error of the mean over n steps is exactly known: n Var(mean) -> (1 + rho)/(1 - rho)
(integrated autocorrelation time tau_int = (1 + rho)/(2 (1 - rho))), while
uncorrelated data (rho = 0) give 1 at every binning level."""
import numpy as np
import pytest

from oracle import oracle as O


def _ar1(rho, chains, T, N, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.empty((chains, T, N))
    x[:, 0] = rng.standard_normal((chains, N))
    s = np.sqrt(1.0 - rho * rho)
    for t in range(1, T):
        x[:, t] = rho * x[:, t - 1] + s * rng.standard_normal((chains, N))
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9, 0.98])
def test_binning_plateau_matches_ar1(rho):
    chains, T, N = 64, 8192, 4
    x = _ar1(rho, chains, T, N, seed=int(rho * 1000) + 7)
    sig2, counts = O.binning(x, 0, 0)
    n = chains * T
    exact = (1.0 + rho) / (1.0 - rho) / n
    # the level-0 bins (64 steps) already exceed the correlation time for rho <= 0.9; the
    # plateau levels (bins >= 16 tau_int, >= 64 bins in all) agree within their own noise
    tau = (1.0 + rho) / (2.0 * (1.0 - rho))
    for k in range(len(counts)):
        L = O.BIN_SWEEPS * 2 ** k
        nbins = chains * counts[k]
        if L >= 16 * tau and nbins >= 256:
            rel = np.sqrt(2.0 / (nbins - 1))   # standard error of a variance estimate
            assert np.all(np.abs(sig2[k] / exact - 1.0) < 5 * rel + 2 * tau / L), (rho, k, sig2[k] / exact)


def test_binning_bins_are_aligned_and_kept_only():
    # sweeps 10..409 recorded, burn-in ends at 100: bins [128,192), ..., [320,384) are complete
    chains, T, N = 3, 400, 2
    x = np.zeros((chains, T, N))
    sweep0, burn = 10, 100
    for t in range(T):
        x[:, t, :] = sweep0 + t          # the state equals its absolute sweep index
    sig2, counts = O.binning(x, sweep0, burn)
    assert counts[0] == 4                # 128, 192, 256, 320
    # level-0 bin means 159.5, 223.5, 287.5, 351.5 in each chain: variance over 12 bins / 12
    means = np.repeat([159.5, 223.5, 287.5, 351.5], chains)
    assert np.allclose(sig2[0], means.var(ddof=1) / means.size)
    assert counts[1] == 2 and counts[2] == 1


def test_mc_error_never_below_chain_spread():
    x = _ar1(0.95, 32, 2048, 3, seed=3)
    S1 = x.sum(axis=1)
    S2 = (x * x).sum(axis=1)
    r = O.mc_error(x, 0, 0, S1, S2, 2048)
    s = O.summarize(S1, S2, 2048)
    assert np.all(r["sigma2"] >= s["sem_fbar"] ** 2 * (1 - 1e-12))
