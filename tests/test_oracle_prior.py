"""The oracle's gamma prior prod f_n^(a_n - 1) (Eq. compat, Sec. V.C), pinned on
* Eq. refine: halving every interval of a grid whose kernel is constant on each
  pair of halves, flat sampling of the halves gives their sums the density of
  shape 2 on the coarse grid -- so the coarse grid sampled with a_n = 2 must
  reproduce the fine grid's pair sums;
* brute-force quadrature of the posterior mean with a gamma prior on one- and
  two-point grids."""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_1912_01379_gb300 import workloads as W


def _z(a, b):
    return np.abs(a["mean_fbar"] - b["mean_fbar"]) / np.hypot(a["sem_fbar"], b["sem_fbar"])


def test_pair_sums_equal_shape_two_prior():
    c = W.small_problem(12, 8, seed=7, levels=[[0]], noise=3e-3)
    Kf = np.repeat(c.K, 2, axis=1)                       # two equal columns per coarse interval
    fine = O.OracleProblem(Kf, c.G, c.C, [[0]])
    coarse = O.OracleProblem(c.K, c.G, c.C, [[0]], prior_shape=np.full(c.N, 2.0))
    burn, sweeps, seed = 2000, 6000, 11
    rf = fine.run(256, burn, sweeps, seed=seed)
    rc = coarse.run(256, burn, sweeps, seed=seed + 1)
    sf = O.summarize(rf["S1"][:, 0::2] + rf["S1"][:, 1::2], None if rf["S2"] is None else
                     (rf["S2"][:, 0::2] + rf["S2"][:, 1::2]), sweeps)   # S2 of the sums is not needed
    sc = O.summarize(rc["S1"], rc["S2"], sweeps)
    assert np.max(_z(sf, sc)) < 4.0, _z(sf, sc)


def _quad_mean_1d(k, g, s2, a):
    w = lambda f: f ** (a - 1) * np.exp(-0.5 * (g - k * f) ** 2 / s2)
    hi = (g + 12 * np.sqrt(s2)) / k
    return integrate.quad(lambda f: f * w(f), 0, hi, limit=400)[0] / integrate.quad(w, 0, hi, limit=400)[0]


@pytest.mark.parametrize("a", [1.5, 2.0, 4.0])
def test_one_point_posterior_mean(a):
    K = np.array([[1.0], [0.5]])
    G = np.array([0.3, 0.1])
    C = np.eye(2) * 0.2 ** 2
    op = O.OracleProblem(K, G, C, [[0]], prior_shape=np.array([a]))
    r = op.run(512, 200, 4000, seed=3)
    s = O.summarize(r["S1"], r["S2"], 4000)
    # the fit of one value: g = K^T C^-1 G / K^T C^-1 K with variance 1 / K^T C^-1 K
    prec = float(K[:, 0] @ K[:, 0]) / 0.04
    gbar = float(K[:, 0] @ G) / 0.04 / prec
    exact = _quad_mean_1d(1.0, gbar, 1.0 / prec, a)
    assert abs(s["mean_fbar"][0] - exact) < 4 * s["sem_fbar"][0], (s["mean_fbar"][0], exact)


def test_two_point_posterior_mean():
    K = np.array([[1.0, 0.3], [0.2, 1.0], [0.5, 0.5]])
    G = np.array([0.4, 0.2, 0.25])
    s2 = 0.15 ** 2
    a = np.array([2.0, 3.0])
    op = O.OracleProblem(K, G, np.eye(3) * s2, [[0]], prior_shape=a)
    r = op.run(512, 200, 4000, seed=4)
    s = O.summarize(r["S1"], r["S2"], 4000)
    dens = lambda f1, f0: f0 ** (a[0] - 1) * f1 ** (a[1] - 1) * np.exp(-0.5 * np.sum((G - K @ [f0, f1]) ** 2) / s2)
    Z = integrate.dblquad(dens, 0, 3, 0, 3)[0]
    m0 = integrate.dblquad(lambda f1, f0: f0 * dens(f1, f0), 0, 3, 0, 3)[0] / Z
    m1 = integrate.dblquad(lambda f1, f0: f1 * dens(f1, f0), 0, 3, 0, 3)[0] / Z
    assert np.all(np.abs(s["mean_fbar"] - [m0, m1]) < 4 * s["sem_fbar"]), (s["mean_fbar"], m0, m1)


def test_shapes_below_one_are_rejected():
    p = W.small_problem(6, 4, seed=1, levels=[[0]])
    with pytest.raises(ValueError):
        O.OracleProblem(p.K, p.G, p.C, p.levels, prior_shape=np.array([1.0, 0.5, 1.0, 1.0]))
