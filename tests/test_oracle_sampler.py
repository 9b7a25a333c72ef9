"""Pins of the oracle's sampler against what the paper and the mathematics fix:
the whitened chi^2 (Sec. IV), the components conditional (Eq. CompChi), the
1-D conditional along any mode (a quadratic in the step), the bounds of
Eq. modeLimits, the unconstrained Gaussian limit (Sec. IV.B), brute-force
quadrature on 2- and 3-point grids, the no-data limit (Eq. def), and the
W-invariance of Eq. Itrafo."""
import numpy as np
import pytest
from scipy import integrate, optimize, special

from oracle import oracle as O
from paper_1912_01379_gb300 import workloads as W


def _whiten(p):
    L = np.linalg.cholesky(p.C)
    Kt = np.linalg.solve(L, p.K)
    gt = np.linalg.solve(L, p.G)
    return Kt, gt


def test_whitening_preserves_chi2():
    p = W.blocked_modes_problem(chains=4)
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    dec = op.decomposition()
    Cinv = np.linalg.inv(p.C)
    rng = np.random.default_rng(0)
    for _ in range(3):
        f = np.abs(rng.standard_normal(p.N)) * 1e-3
        r = p.G - p.K @ f
        chi2 = r @ Cinv @ r                                  # Eq. chi2, unwhitened
        assert op.chi2(f) == pytest.approx(chi2, rel=1e-9)
        assert np.sum((dec.gt - dec.Kt @ f) ** 2) == pytest.approx(chi2, rel=1e-9)


def test_block_factors_reconstruct_whitened_kernel():
    p = W.blocked_modes_problem(chains=4)
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    dec = op.decomposition()
    Kt, _ = _whiten(p)
    assert np.allclose(dec.Kt, Kt, rtol=1e-10, atol=1e-10 * np.abs(Kt).max())
    od = ov = ou = 0
    for (l, b, s, n) in op.blocks():
        npr = min(p.M, n)
        d = dec.d[od:od + n]; od += n
        V = dec.V[ov:ov + n * n].reshape(n, n).T; ov += n * n      # columns = modes
        U = dec.U[ou:ou + npr * p.M].reshape(npr, p.M).T; ou += npr * p.M
        Kb = dec.Kt[:, s:s + n]
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
        rec = U @ np.diag(d[:npr]) @ V[:, :npr].T
        sv = np.linalg.svd(Kb, compute_uv=False)
        # modes at or below d_1 max(M, n) 2^-40 may be flat (R2): the reconstruction misses
        # at most sqrt(n) such singular values
        assert np.abs(rec - Kb).max() <= 1e-10 * np.abs(Kb).max() + np.sqrt(n) * max(p.M, n) * 2.0 ** -40 * sv[0]
        keep = d[:npr] > 0
        assert np.allclose(d[:npr][keep], sv[:npr][keep], rtol=1e-8, atol=1e-12 * sv[0])


def test_components_conditional_matches_eq_compchi():
    """A level of one-point blocks is components sampling: the step of f_n is a
    Gaussian of width 1/|K~_n| centred at K~_n^T r~ / |K~_n|^2, cut at -f_n."""
    p = W.small_problem(12, 9, seed=5)
    lev = [np.arange(p.N, dtype=np.int32)]
    op = O.OracleProblem(p.K, p.G, p.C, lev)
    Kt, gt = _whiten(p)
    rng = np.random.default_rng(1)
    f = np.abs(rng.standard_normal(p.N)) * 0.05
    r = gt - Kt @ f
    for n in range(p.N):
        mu, sg, lo, hi = op.conditional(0, n, 0, f)
        kn = Kt[:, n]
        assert sg == pytest.approx(1.0 / np.linalg.norm(kn), rel=1e-12)
        assert mu == pytest.approx(kn @ r / (kn @ kn), rel=1e-9, abs=1e-12 * abs(f[n]) + 1e-15)
        assert lo == pytest.approx(-f[n], rel=1e-15)
        assert hi == np.inf


@pytest.mark.parametrize("levels", [[[0]], [[0, 7, 15]], [[0, 4, 9, 13, 18]]])
def test_mode_conditional_is_the_chi2_line(levels):
    """Along any mode V_j of any block, chi^2(f + t V_j) is the quadratic
    (t - mu)^2 / sigma^2 + const (flat for zero modes), and [lo, hi] is the
    largest interval with f + t V_j >= 0."""
    p = W.small_problem(10, 22, seed=11, levels=levels)
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    dec = op.decomposition()
    Kt, gt = dec.Kt, dec.gt
    rng = np.random.default_rng(2)
    f = np.abs(rng.standard_normal(p.N)) * 0.02
    f[rng.integers(0, p.N, 4)] = 0.0
    chi2 = lambda x: float(np.sum((gt - Kt @ x) ** 2))
    ov = od = 0
    for (l, b, s, n) in op.blocks():
        V = dec.V[ov:ov + n * n].reshape(n, n); ov += n * n
        d1 = dec.d[od]; od += n
        for j in range(n):
            mu, sg, lo, hi = op.conditional(l, b, j, f)
            v = np.zeros(p.N); v[s:s + n] = V[j]
            h = sg if sg > 0 else 1e-2     # the mode's own length scale
            c0, cp, cm = chi2(f), chi2(f + h * v), chi2(f - h * v)
            a2 = (cp + cm - 2 * c0) / (2 * h * h)   # coefficient of t^2
            a1 = (cp - cm) / (2 * h)                # coefficient of t
            scale = max(abs(cp), abs(c0)) / (h * h)
            if sg > 0 and 1.0 / sg >= 1e-7 * d1:
                # (weaker modes sit within rounding of the zero-mode cut-off:
                # there K~ V_j itself is not known to better than ~1e-3)
                assert a2 == pytest.approx(1.0 / sg**2, rel=1e-5, abs=1e-7 * scale)
                assert -a1 / (2 * a2) == pytest.approx(mu, rel=1e-4, abs=1e-6 * sg + 1e-9 * abs(mu))
            elif sg == 0:
                assert abs(a2) <= 1e-6 * scale
            assert lo <= 0.0 <= hi
            for t, away in ((lo, -1.0), (hi, 1.0)):
                if np.isfinite(t):
                    x = f + t * v
                    assert x.min() >= -1e-12 * max(f.max(), 1e-300)
                    assert np.min(np.abs(x[s:s + n])) <= 1e-12 * max(f.max(), 1e-300)
                    # a little further and some component turns negative
                    y = f + (t + away * 1e-9 * max(abs(t), f.max())) * v
                    assert y.min() < 0


def _run_stats(op, chains, burn, sweeps, seed, w=None, threads=8):
    r = op.run(chains, burn, sweeps, seed=seed, threads=threads)
    assert r["stats"][0] == 0, "positivity violated"
    s = O.summarize(r["S1"], r["S2"], r["kept"], w)
    return r, s


def test_unconstrained_gaussian_limit():
    """N <= M and the posterior far from f = 0: the average is the least-squares
    solution and the covariance is (K~^T K~)^{-1} (Sec. IV.B)."""
    M, N = 20, 4
    tau = W.tau_grid(10.0, M)
    omega, w = W.uniform_grid(-5, 5, N)
    K = W.fermionic_kernel(tau, omega, 10.0)
    fbar = np.array([2.0, 3.0, 2.5, 1.5])
    C = np.eye(M) * 1e-3 ** 2
    G = K @ fbar + np.random.default_rng(7).standard_normal(M) * 1e-3
    Kt = K / 1e-3
    gt = G / 1e-3
    P = np.linalg.inv(Kt.T @ Kt)
    mean = P @ Kt.T @ gt
    assert np.min(mean / np.sqrt(np.diag(P))) >= 10     # positivity inactive
    for levels in ([[0]], [[0, 2]], [np.arange(N)]):
        op = O.OracleProblem(K, G, C, levels)
        r, s = _run_stats(op, 32, 200, 3000, seed=21)
        z = (s["mean_fbar"] - mean) / s["sem_fbar"]
        assert np.all(np.abs(z) < 4.5), (levels, z)
        assert np.allclose(s["var_fbar"], np.diag(P), rtol=0.1)


def _quad_mean(Kt, gt, box):
    """<f> over the positive orthant weighted by exp(-chi^2/2).  The last
    coordinate is integrated in closed form (chi^2 is a quadratic a t^2 + b t + c
    in it, so its integral over t >= 0 is a Gaussian tail); the others by
    adaptive quadrature on [0, box]."""
    N = Kt.shape[1]
    kl = Kt[:, -1]
    a = kl @ kl
    sg = 1.0 / np.sqrt(a)
    fmin = optimize.minimize(lambda f: np.sum((gt - Kt @ f) ** 2), np.full(N, 0.1),
                             bounds=[(0, None)] * N).fun

    def inner(*x):
        r = gt - Kt[:, :-1] @ np.array(x)
        b = -2.0 * kl @ r
        c = r @ r
        m = -b / (2 * a)
        e = np.exp(-0.5 * (c - b * b / (4 * a) - fmin))
        z0 = e * sg * np.sqrt(2 * np.pi) * special.ndtr(m / sg)
        z1 = e * (m * sg * np.sqrt(2 * np.pi) * special.ndtr(m / sg) + sg * sg * np.exp(-0.5 * (m / sg) ** 2))
        return z0, z1

    if N == 2:
        q = lambda g: integrate.quad(g, 0, box[0], epsabs=0, epsrel=1e-11, limit=400)[0]
        Z = q(lambda x: inner(x)[0])
        m0 = q(lambda x: x * inner(x)[0])
        m1 = q(lambda x: inner(x)[1])
        return np.array([m0, m1]) / Z
    q = lambda g: integrate.dblquad(g, 0, box[0], 0, box[1], epsabs=0, epsrel=1e-9)[0]
    Z = q(lambda y, x: inner(x, y)[0])
    m0 = q(lambda y, x: x * inner(x, y)[0])
    m1 = q(lambda y, x: y * inner(x, y)[0])
    m2 = q(lambda y, x: inner(x, y)[1])
    return np.array([m0, m1, m2]) / Z


@pytest.mark.parametrize("M,N,levels", [(3, 2, [[0]]), (3, 2, [[0, 1]]), (2, 3, [[0], [0, 1, 2]])])
def test_brute_force_quadrature(M, N, levels):
    """The average over the positive orthant by quadrature, with positivity
    binding (and, for N > M, a flat direction bounded only by f >= 0)."""
    rng = np.random.default_rng(M * 10 + N)
    K = np.abs(rng.standard_normal((M, N))) + 0.3
    ftrue = np.array([0.6, 0.05, 0.3][:N])
    sig = 0.2
    G = K @ ftrue + sig * rng.standard_normal(M)
    C = np.eye(M) * sig * sig
    Kt, gt = K / sig, G / sig
    box = [2.5 * max(G.max(), 0.5) / K.min()] * N
    exact = _quad_mean(Kt, gt, box)
    op = O.OracleProblem(K, G, C, levels)
    r, s = _run_stats(op, 64, 200, 4000, seed=5)
    z = (s["mean_fbar"] - exact) / s["sem_fbar"]
    assert np.all(np.abs(z) < 4.5), (exact, s["mean_fbar"], z)


def test_no_data_limit_grid_density_is_default_model():
    """Only a sum rule in the data: all fbar_n share the same average <F>/N
    (Eq. def) and Dirichlet(1,...,1) second moments."""
    N, sig = 5, 0.02
    K = np.ones((1, N))
    G = np.array([1.0])
    C = np.array([[sig * sig]])
    F = np.linspace(0, 1.5, 20001)
    dens = F ** (N - 1) * np.exp(-0.5 * ((F - 1) / sig) ** 2)
    Z = np.trapezoid(dens, F)
    EF = np.trapezoid(F * dens, F) / Z
    EF2 = np.trapezoid(F * F * dens, F) / Z
    op = O.OracleProblem(K, G, C, [[0], [0, 2]])
    r = op.run(64, 100, 4000, seed=9, threads=8)
    s = O.summarize(r["S1"], r["S2"], r["kept"])
    z = (s["mean_fbar"] - EF / N) / s["sem_fbar"]
    assert np.all(np.abs(z) < 4.5), z
    m2 = r["S2"].sum(0) / (64 * r["kept"])
    assert np.allclose(m2, 2 * EF2 / (N * (N + 1)), rtol=0.03)


def test_w_invariance_step_by_step():
    """Components sampling of fbar with K equals components sampling of f with
    K W, fbar = W f, draw by draw (Eq. Itrafo with the same random numbers)."""
    p = W.small_problem(15, 10, seed=3)
    w = np.linspace(0.5, 2.0, p.N)
    lev = [np.arange(p.N, dtype=np.int32)]
    a = O.OracleProblem(p.K, p.G, p.C, lev)
    b = O.OracleProblem(p.K * w[None, :], p.G, p.C, lev)
    f0 = a.initial_f()
    ra = a.run(4, 0, 30, seed=4, trace_chains=4, f_start=f0)
    rb = b.run(4, 0, 30, seed=4, trace_chains=4, f_start=f0 / w)
    ta, tb = ra["trace"], rb["trace"] * w[None, None, :]
    assert np.allclose(ta, tb, rtol=1e-10, atol=1e-14)


def test_all_levels_sample_the_same_average():
    """Modes, blocked modes, components and a random mix of levels are all valid
    Gibbs schemes for the same target: same average within the MC error."""
    p = W.small_problem(10, 12, seed=8)
    res = []
    for levels in ([[0]], [[0, 4, 8]], [np.arange(12)], [[0], [0, 6], [0, 3, 6, 9], np.arange(12)]):
        op = O.OracleProblem(p.K, p.G, p.C, levels)
        r, s = _run_stats(op, 32, 500, 4000, seed=13)
        res.append(s)
    for s in res[1:]:
        z = (s["mean_fbar"] - res[0]["mean_fbar"]) / np.hypot(s["sem_fbar"], res[0]["sem_fbar"])
        assert np.all(np.abs(z) < 4.5), z


def test_chain_means_standard_error():
    """The SEM estimate from independent chain means matches 1/sqrt(C K) for iid
    unit-variance samples."""
    rng = np.random.default_rng(0)
    C, K, N = 256, 100, 50
    x = rng.standard_normal((C, K, N))
    S1, S2 = x.sum(1), (x * x).sum(1)
    s = O.summarize(S1, S2, K)
    assert np.allclose(s["sem_fbar"], 1 / np.sqrt(C * K), rtol=0.2)
    assert np.allclose(s["ess"], C * K, rtol=0.4)


def test_setup_rejects_bad_inputs():
    p = W.small_problem(6, 8, seed=1)
    with pytest.raises(ValueError, match="SPD"):
        O.OracleProblem(p.K, p.G, -p.C, p.levels)
    G = p.G.copy(); G[0] = np.nan
    with pytest.raises(ValueError, match="non-finite"):
        O.OracleProblem(p.K, G, p.C, p.levels)
    with pytest.raises(ValueError, match="shape"):
        O.OracleProblem(p.K, p.G, p.C, [[1, 3]])
    # a zero mode along which f >= 0 gives no bound: two identical columns of
    # opposite sign make (1, 1)/sqrt2 a single-signed null vector
    K = np.ones((2, 2)); K[:, 1] = -1.0
    with pytest.raises(ValueError, match="improper"):
        O.OracleProblem(K, np.ones(2), np.eye(2), [[0]])
