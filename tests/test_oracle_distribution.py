"""Distributional pins of the oracle, against routes that share nothing with it:

- its inverse-CDF draw of the truncated normal (reading R1, Sec. IV.A-B)
  against Robert's (1995) rejection sampler and against the exact CDF and
  moments of the truncated normal, over intervals from the centre of the
  Gaussian to its far tails and from narrow to half-infinite;
- a two-point chain (Sec. IV.B modes, Sec. IV.A components) against its exact
  density exp(-chi^2/2) on the positive quadrant (Eq. chi2), by a Pearson
  chi-square test on a 2-D histogram of independent chain end points, with
  positivity binding and, for M = 1, a flat direction;
- the second moments <f f^T> of a two-point chain against brute-force
  quadrature of the same density;
- reading R2 (sign-changing modes with d <= d_1 max(M,n) 2^-40 sampled flat)
  against the plain numerical-zero rule (2^-52) on the blocked-modes and
  Matsubara problems: the averages agree within the binned Monte Carlo error.
"""
import mpmath as mp
import numpy as np
import pytest
from scipy import integrate, special, stats

from oracle import oracle as O
from paper_1912_01379_gb300 import workloads as W

# -- truncated normal -------------------------------------------------------
INTERVALS = [(-1.0, 2.0), (0.5, 3.0), (-5.0, 5.0), (5.0, np.inf), (30.0, 31.0), (1000.0, np.inf),
             (-np.inf, -7.0), (-1e-3, 1e-3), (4.9, 5.1), (-3.0, np.inf), (0.0, np.inf),
             (6.0, 6.000001), (-40.0, -39.9), (-np.inf, 0.3)]
NDRAW = 20000


def _exact_cdf(x, a, b):
    """P(a <= X <= x) / P(a <= X <= b) for X ~ N(0,1), in forms that keep
    their accuracy in the tails (scipy's log_ndtr)."""
    x = np.asarray(x, dtype=np.float64)
    if b <= 0:
        return 1.0 - _exact_cdf(-x, -b, -a)
    if a >= 0:
        lq = lambda t: special.log_ndtr(-t)
        num = -np.expm1(lq(x) - lq(a))
        den = -np.expm1(lq(b) - lq(a)) if np.isfinite(b) else 1.0
        return num / den
    return (special.ndtr(x) - special.ndtr(a)) / (special.ndtr(b) - special.ndtr(a))


def _exact_moments(a, b):
    """Mean and variance of N(0,1) on [a, b] (40 digits)."""
    mp.mp.dps = 40
    A, B = mp.mpf(a), (mp.mpf(b) if np.isfinite(b) else mp.inf)
    if not np.isfinite(a):
        A = -mp.inf
    phi = lambda t: mp.mpf(0) if mp.isinf(t) else mp.exp(-t * t / 2) / mp.sqrt(2 * mp.pi)
    tphi = lambda t: mp.mpf(0) if mp.isinf(t) else t * phi(t)
    Z = (mp.ncdf(B) - mp.ncdf(A)) if a < 0 else (mp.erfc(A / mp.sqrt(2)) - mp.erfc(B / mp.sqrt(2))) / 2
    m = (phi(A) - phi(B)) / Z
    v = 1 + (tphi(A) - tphi(B)) / Z - m * m
    return float(m), float(v)


def _inverse_cdf_draws(a, b, n, seed):
    # the sampler's uniforms lie on the grid (k + 1/2) 2^-52
    r = np.random.default_rng(seed).random(n)
    u = (np.floor(r * 2.0**52) + 0.5) * 2.0**-52
    return np.array([O.truncnorm(0.0, 1.0, a, b, x) for x in u])


@pytest.mark.parametrize("a,b", INTERVALS)
def test_robert_sampler_against_exact_distribution(a, b):
    """Robert's rejection sampler, written from its published description, is
    an independent route to the truncated normal: its draws pass a KS test
    against the exact CDF and match the exact mean."""
    x, tries = O.truncnorm_robert(a, b, NDRAW, seed=11, stream=7)
    assert np.all((x >= a) & (x <= b))
    assert tries >= NDRAW
    assert stats.kstest(x, lambda t: _exact_cdf(t, a, b)).pvalue > 1e-4
    m, v = _exact_moments(a, b)
    assert abs(x.mean() - m) <= 4.5 * np.sqrt(v / NDRAW)


@pytest.mark.parametrize("a,b", INTERVALS)
def test_inverse_cdf_and_robert_agree_in_distribution(a, b):
    """The oracle's inverse-CDF draw at random uniforms and Robert's sampler
    give the same distribution (two-sample KS), and both the exact mean and
    variance."""
    x = _inverse_cdf_draws(a, b, NDRAW, seed=INTERVALS.index((a, b)) + 3)
    y, _ = O.truncnorm_robert(a, b, NDRAW, seed=5, stream=1)
    assert np.all((x >= a) & (x <= b))
    assert stats.ks_2samp(x, y).pvalue > 1e-4
    m, v = _exact_moments(a, b)
    for s in (x, y):
        assert abs(s.mean() - m) <= 4.5 * np.sqrt(v / NDRAW)
        # sample variance: standard error about v sqrt(2/n) for near-Gaussian shapes, wider for others
        assert abs(s.var() - v) <= 0.06 * v


# -- two-point chains against their exact density ---------------------------
def _two_point_problem(M):
    K = np.array([[1.0, 0.5], [0.3, 1.0], [0.7, 0.8]])[:M]
    sig = 0.2
    ftrue = np.array([0.6, 0.05])
    G = K @ ftrue + sig * np.array([0.3, -1.1, 0.4])[:M]
    return K, G, np.eye(M) * sig * sig, K / sig, G / sig


class _Density:
    """exp(-chi^2(x, y)/2) on x, y >= 0 with chi^2 = |g - K [x, y]|^2 quadratic:
    integrals over y in closed form (a Gaussian CDF difference), over x by
    adaptive quadrature."""

    def __init__(self, Kt, gt):
        self.Kt, self.gt = Kt, gt
        k2 = Kt[:, 1]
        self.a = k2 @ k2
        # shift: chi^2 at its minimum over the quadrant keeps the exponentials in range
        xs = np.linspace(0, 10, 2001)
        self.c0 = min(self._cmin(x) for x in xs)

    def _cmin(self, x):
        r = self.gt - self.Kt[:, 0] * x
        b = -2.0 * self.Kt[:, 1] @ r
        c = r @ r
        m = max(-b / (2 * self.a), 0.0)
        return self.a * m * m + b * m + c

    def _y_moments(self, x, y0, y1):
        """int_{y0}^{y1} y^k exp(-(chi^2 - c0)/2) dy for k = 0, 1, 2."""
        r = self.gt - self.Kt[:, 0] * x
        b = -2.0 * self.Kt[:, 1] @ r
        c = r @ r
        m = -b / (2 * self.a)
        s = 1.0 / np.sqrt(self.a)
        e = np.exp(-0.5 * (c - b * b / (4 * self.a) - self.c0))
        z0, z1 = (y0 - m) / s, (y1 - m) / s
        P = special.ndtr(z1) - special.ndtr(z0)
        p0 = np.exp(-0.5 * z0 * z0) if np.isfinite(z0) else 0.0
        p1 = np.exp(-0.5 * z1 * z1) if np.isfinite(z1) else 0.0
        t0p0 = z0 * p0 if np.isfinite(z0) else 0.0
        t1p1 = z1 * p1 if np.isfinite(z1) else 0.0
        g = s * np.sqrt(2 * np.pi)
        I0 = g * P
        I1 = m * I0 + s * s * (p0 - p1)
        I2 = (m * m + s * s) * I0 + 2 * m * s * s * (p0 - p1) + s ** 3 * (t0p0 - t1p1)
        return e * I0, e * I1, e * I2

    def mass(self, x0, x1, y0, y1):
        return integrate.quad(lambda x: self._y_moments(x, y0, y1)[0], x0, x1, epsabs=0, epsrel=1e-10,
                              limit=400)[0]

    def moments(self, xmax):
        q = lambda g: integrate.quad(g, 0, xmax, epsabs=0, epsrel=1e-11, limit=400)[0]
        Z = q(lambda x: self._y_moments(x, 0, np.inf)[0])
        ex = q(lambda x: x * self._y_moments(x, 0, np.inf)[0]) / Z
        ey = q(lambda x: self._y_moments(x, 0, np.inf)[1]) / Z
        exx = q(lambda x: x * x * self._y_moments(x, 0, np.inf)[0]) / Z
        exy = q(lambda x: x * self._y_moments(x, 0, np.inf)[1]) / Z
        eyy = q(lambda x: self._y_moments(x, 0, np.inf)[2]) / Z
        return np.array([ex, ey]), np.array([[exx, exy], [exy, eyy]]), Z


@pytest.mark.parametrize("M,levels", [(3, [[0]]), (3, [[0, 1]]), (1, [[0]]), (1, [[0], [0, 1]])])
def test_two_point_chain_histogram(M, levels):
    """Independent chain end points (4000 chains after 300 sweeps) fall into
    the cells of a 2-D grid with the probabilities of the exact density
    (Pearson chi-square).  M = 1 leaves a flat direction along which only
    f >= 0 bounds the chain (a zero mode, Sec. IV.B)."""
    K, G, C, Kt, gt = _two_point_problem(M)
    dens = _Density(Kt, gt)
    xmax = 10.0
    _, _, Z = dens.moments(xmax)
    # cell edges at quantiles of the exact marginals (fixed before looking at samples)
    def marg_q(which, q):
        if which == 0:
            F = lambda t: dens.mass(0, t, 0, np.inf) / Z
        else:
            F = lambda t: dens.mass(0, xmax, 0, t) / Z
        lo, hi = 0.0, xmax
        for _ in range(50):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if F(mid) < q else (lo, mid)
        return 0.5 * (lo + hi)
    qs = [0.12, 0.25, 0.4, 0.55, 0.7, 0.85, 0.95]
    ex = [0.0] + [marg_q(0, q) for q in qs] + [np.inf]
    ey = [0.0] + [marg_q(1, q) for q in qs] + [np.inf]
    expect = np.array([[dens.mass(ex[i], min(ex[i + 1], xmax), ey[j], ey[j + 1]) / Z
                        for j in range(len(ey) - 1)] for i in range(len(ex) - 1)])
    assert expect.sum() == pytest.approx(1.0, abs=1e-8)
    op = O.OracleProblem(K, G, C, levels)
    chains = 4000
    r = op.run(chains, 0, 300, seed=29 + M, threads=8)
    f = r["f_final"]
    assert np.all(f >= 0)
    obs, _, _ = np.histogram2d(f[:, 0], f[:, 1], bins=[ex, ey])
    E = expect * chains
    keep = E >= 5
    stat = np.sum((obs[keep] - E[keep]) ** 2 / E[keep])
    rest_o, rest_e = obs[~keep].sum(), E[~keep].sum()
    dof = keep.sum() - 1
    if rest_e > 0:
        stat += (rest_o - rest_e) ** 2 / rest_e
        dof += 1
    assert stats.chi2.sf(stat, dof) > 1e-4, (stat, dof)


@pytest.mark.parametrize("M,levels", [(3, [[0]]), (3, [[0, 1]]), (1, [[0]])])
def test_two_point_second_moments_by_quadrature(M, levels):
    """<f> and <f f^T> of the chain against brute-force quadrature of the same
    density, within 4.5 standard errors from independent chain means."""
    K, G, C, Kt, gt = _two_point_problem(M)
    mean, mom2, _ = _Density(Kt, gt).moments(10.0)
    op = O.OracleProblem(K, G, C, levels)
    chains, burn, sweeps = 64, 200, 3000
    r = op.run(chains, burn, sweeps, seed=41 + M, threads=8, trace_chains=chains)
    tr = r["trace"][:, burn:, :]
    per_chain = np.stack([tr[..., 0], tr[..., 1], tr[..., 0] ** 2, tr[..., 0] * tr[..., 1],
                          tr[..., 1] ** 2], axis=-1).mean(axis=1)
    est = per_chain.mean(axis=0)
    sem = per_chain.std(axis=0, ddof=1) / np.sqrt(chains)
    want = np.array([mean[0], mean[1], mom2[0, 0], mom2[0, 1], mom2[1, 1]])
    z = (est - want) / sem
    assert np.all(np.abs(z) < 4.5), (est, want, z)


# -- reading R2 -------------------------------------------------------------
@pytest.mark.parametrize("case", ["blocked_modes", "matsubara"])
def test_flat_rule_does_not_move_the_average(case):
    """Sampling the sign-changing modes with d_1 max(M,n) 2^-52 < d <= d_1
    max(M,n) 2^-40 flat (reading R2) instead of Gaussian leaves <fbar> within
    4.5 combined binned standard errors, on the two problems where the rule
    turns modes flat (same level schedule, disjoint chain ids)."""
    from paper_1912_01379_gb300 import asm
    if case == "blocked_modes":
        p = W.blocked_modes_problem(chains=4)
        levels, burn, sweeps = p.levels, 512, 1024
    else:
        p = W.paper_problem(2, 1e-3, "gaussian", 64)
        levels, burn, sweeps = asm.partition_hierarchy(p.N), 1536, 1536
    chains = 32
    res = {}
    for e in (40, 52):
        op = O.OracleProblem(p.K, p.G, p.C, levels, flat_exp=e)
        res[e] = {"flat": int((op.decomposition().d == 0).sum())}
        r = op.run(chains, burn, sweeps, seed=77, threads=8, chain_offset=0 if e == 40 else chains,
                   trace_chains=chains)
        me = O.mc_error(r["trace"][:, burn:, :], burn, burn, r["S1"], r["S2"], sweeps)
        res[e]["mean"] = O.summarize(r["S1"], r["S2"], sweeps)["mean_fbar"]
        res[e]["sem"] = np.sqrt(me["sigma2"])
    assert res[40]["flat"] > res[52]["flat"]   # the rule is in force on this problem
    z = (res[40]["mean"] - res[52]["mean"]) / np.hypot(res[40]["sem"], res[52]["sem"])
    assert np.max(np.abs(z)) < 4.5, float(np.max(np.abs(z)))
