"""Backward pass: vector-Jacobian products of <A> from the covariance identity
(asm_backward, hand-written contractions), against closed forms the
mathematics fixes:
 * the unconstrained Gaussian limit (N <= M, positivity inactive), where
   <fbar> = (K~^T K~)^{-1} K~^T g~ exactly, for the G-gradient and, by central
   differences of that closed form over the grid-density parameters, the
   theta-gradient;
 * a 2-point grid with positivity binding, where <f> is known by quadrature and
   its G-derivative by central differences of the quadrature;
 * the differentiation workload itself (N_tau = 64, N_omega = 200, 8 grid
   parameters, 4096 chains), against central differences of the sampled mean.

The closed-form checks are sized by the measured Monte Carlo error of the
products: independent replicas (seeds) are added until the relative standard
error of their mean is at most 2.5e-4, and the products must then agree with
the closed form within 1e-3 relative, or 4 standard errors where that is
larger.
"""
import numpy as np
import pytest
from scipy import integrate, special

from paper_1912_01379_gb300 import asm
from paper_1912_01379_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    torch.cuda.synchronize()


def _gaussian_limit_problem(offset=10.0):
    M, N, beta = 64, 6, 16.0
    tau = W.tau_grid(beta, M)
    omega, w = W.uniform_grid(-6.0, 6.0, N)
    K = W.fermionic_kernel(tau, omega, beta)
    A = 0.4 * W.gauss_pdf(omega, -1.0, 0.8) + 0.6 * W.gauss_pdf(omega, 2.0, 0.6) + offset
    C = np.eye(M) * 1e-4 ** 2
    G = K @ (A * w) + np.random.default_rng(4).standard_normal(M) * 1e-4
    return K, G, C, w


def _exact_mean(K, G, C):
    L = np.linalg.cholesky(C)
    Kt, gt = np.linalg.solve(L, K), np.linalg.solve(L, G)
    P = np.linalg.inv(Kt.T @ Kt)
    return P @ Kt.T @ gt, P, L, Kt


REL_SEM = 2.5e-4     # target relative standard error of the products
REL_TOL = 1e-3       # agreement with the closed form (or 4 standard errors)


def _replicas(gp, v, chains, burn, sweeps, precision, want_theta=False, max_reps=48, min_reps=4):
    """Mean and standard error of the products over independent replicas, added
    until both relative standard errors are at most REL_SEM."""
    gs, ts = [], []
    while True:
        gp.sample(chains, burn, sweeps, 1000 + len(gs), precision=precision, moments=True)
        g, t = gp.backward(v, want_theta=want_theta)
        gs.append(g)
        if want_theta:
            ts.append(t)
        out = []
        for x in (gs, ts) if want_theta else (gs,):
            a = np.array(x)
            m = a.mean(axis=0)
            sem = np.linalg.norm(a.std(axis=0, ddof=1)) / np.sqrt(len(a)) if len(a) > 1 else np.inf
            out.append((m, sem / np.linalg.norm(m)))
        if len(gs) >= min_reps and all(r <= REL_SEM for _, r in out) or len(gs) >= max_reps:
            return out


def _check(est, rel_sem, exact, bias=0.0):
    err = np.linalg.norm(est - exact) / np.linalg.norm(exact)
    assert rel_sem <= REL_SEM, f"replicas did not reach the target error: {rel_sem}"
    assert err <= max(REL_TOL, 4 * rel_sem) + bias, (err, rel_sem, bias)


def _fp32_state_bias(L, Kt, mean, vp):
    """Relative change of the G-product caused by holding the chain state in
    FP32: the stored fbar_n carries a rounding error uniform over one ulp,
    whose variance (2^-23 |fbar_n|)^2 / 12 adds to the posterior covariance
    (it matters where the posterior spread is not large against the ulp)."""
    ulp = 2.0 ** -23 * 2.0 ** np.floor(np.log2(np.abs(mean)))
    Q = np.diag(ulp ** 2 / 12)
    P = np.linalg.inv(Kt.T @ Kt)
    exact = np.linalg.solve(L.T, Kt @ (P @ vp))
    return np.linalg.norm(np.linalg.solve(L.T, Kt @ (Q @ vp))) / np.linalg.norm(exact)


# FP32 chain state resolves fbar to 2^-24 |fbar|.  With the offset 10 the two
# strongest modes' posterior width is only about 25 ulps of fbar, and the mixed
# path then samples them with a 2-3 % too large variance (measured in the mode
# basis; the excess falls with the square of the ulp: 0.1 % at offset 2), which
# moves the G-product by 1.2e-3.  The mixed path is therefore checked at offset 2
# (positivity still inactive by a margin of 10 standard deviations).
@pytest.mark.parametrize("precision,offset", [(asm.ASM_FP64, 10.0), (asm.ASM_MIXED, 2.0)])
def test_grad_G_gaussian_limit(precision, offset):
    K, G, C, w = _gaussian_limit_problem(offset)
    mean, P, L, Kt = _exact_mean(K, G, C)
    assert np.min(mean / np.sqrt(np.diag(P))) >= 10          # positivity inactive
    gp = asm.Problem(K, G, C, [[0], [0, 3]], w=w)
    v = np.random.default_rng(1).standard_normal(len(w))
    [(gG, rel)] = _replicas(gp, v, 4096, 200, 8000, precision)
    exact = np.linalg.solve(L.T, Kt @ (P @ (v / w)))          # C^{-1} K Cov (v/w)
    bias = _fp32_state_bias(L, Kt, mean, v / w) if precision == asm.ASM_MIXED else 0.0
    _check(gG, rel, exact, bias)
    r = gp.average()
    assert np.allclose(r["mean_fbar"], mean, rtol=1e-3)


@pytest.mark.parametrize("precision,offset", [(asm.ASM_FP64, 10.0), (asm.ASM_MIXED, 2.0)])
def test_grad_theta_gaussian_limit(precision, offset):
    theta0 = W.THETA0.copy()
    build = lambda th: W.theta_problem(th, N=6, offset=offset, levels=[[0]])
    p = build(theta0)
    # data representable on the 6-point grid at theta0 (fixed for every theta)
    p.G = p.K @ p.fbar_true + np.random.default_rng(8).standard_normal(p.M) * 1e-4
    mean, P, _, _ = _exact_mean(p.K, p.G, p.C)
    assert np.min(mean / np.sqrt(np.diag(P))) >= 10
    v = np.random.default_rng(2).standard_normal(p.N)
    # closed form <A>(theta) = (K~^T K~)^{-1} K~^T g~ / w, central differences
    h = 1e-5
    fd = np.zeros(len(theta0))
    for k in range(len(theta0)):
        e = np.zeros(len(theta0)); e[k] = h
        pp, pm = build(theta0 + e), build(theta0 - e)
        Ap = _exact_mean(pp.K, p.G, p.C)[0] / pp.w
        Am = _exact_mean(pm.K, p.G, p.C)[0] / pm.w
        fd[k] = v @ (Ap - Am) / (2 * h)
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, dK_dtheta=p.extra["dK_dtheta"],
                     dw_dtheta=p.extra["dw_dtheta"])
    _, (gt, rel) = _replicas(gp, v, 4096, 200, 8000, precision, want_theta=True)
    _check(gt, rel, fd)


def _quad_mean_2(Kt, gt):
    """<f> on the positive quadrant for N = 2 (inner coordinate in closed form)."""
    a = Kt[:, 1] @ Kt[:, 1]
    sg = 1 / np.sqrt(a)
    f_min = 0.0

    def inner(x):
        r = gt - Kt[:, 0] * x
        b = -2 * Kt[:, 1] @ r
        c = r @ r
        m = -b / (2 * a)
        e = np.exp(-0.5 * (c - b * b / (4 * a)))
        z0 = e * sg * np.sqrt(2 * np.pi) * special.ndtr(m / sg)
        z1 = e * (m * sg * np.sqrt(2 * np.pi) * special.ndtr(m / sg) + sg * sg * np.exp(-0.5 * (m / sg) ** 2))
        return z0, z1

    top = 3.0 * max(gt.max(), 1.0) / Kt.min()
    q = lambda g: integrate.quad(g, 0, top, epsabs=0, epsrel=1e-12, limit=500)[0]
    Z = q(lambda x: inner(x)[0])
    return np.array([q(lambda x: x * inner(x)[0]), q(lambda x: inner(x)[1])]) / Z


def test_grad_G_with_positivity_binding_against_quadrature():
    rng = np.random.default_rng(6)
    K = np.abs(rng.standard_normal((3, 2))) + 0.3
    sig = 0.2
    G = K @ np.array([0.5, 0.05]) + sig * rng.standard_normal(3)
    C = np.eye(3) * sig * sig
    v = np.array([0.7, -1.3])
    h = 1e-3 * sig
    fd = np.zeros(3)
    for m in range(3):
        e = np.zeros(3); e[m] = h
        fd[m] = v @ (_quad_mean_2(K / sig, (G + e) / sig) - _quad_mean_2(K / sig, (G - e) / sig)) / (2 * h)
    gp = asm.Problem(K, G, C, [[0], [0, 1]])
    [(gG, rel)] = _replicas(gp, v, 4096, 200, 8000, asm.ASM_FP64)
    _check(gG, rel, fd)


def test_differentiation_workload_against_finite_differences():
    """At the differentiation workload's size (N_tau = 64, N_omega = 200, 4096
    chains) the G-product along random data directions e agrees with central
    differences of the sampled mean, d/dh v.<A>(G + h e) at h = 0, within
    4 combined standard errors.  The difference step h = sigma (the noise
    level) keeps the curvature term below the statistical error: the two
    differences at h and h/2 agree within their errors (Richardson check)."""
    p = W.theta_problem()
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    chains, burn, sweeps, reps = 4096, 300, 1500, 4
    v = np.random.default_rng(3).standard_normal(p.N)
    gs = []
    for r in range(reps):
        gp.sample(chains, burn, sweeps, 50 + r, precision=asm.ASM_MIXED, moments=True)
        gs.append(gp.backward(v)[0])
    gs = np.array(gs)
    g, g_sem = gs.mean(axis=0), gs.std(axis=0, ddof=1) / np.sqrt(reps)
    sigma = 1e-4
    rng = np.random.default_rng(11)
    for _ in range(2):
        e = rng.standard_normal(p.M)
        e /= np.linalg.norm(e)
        want, want_sem = g @ e, np.sqrt(((gs @ e).var(ddof=1)) / reps)
        fds = {}
        for h in (sigma, 0.5 * sigma):
            vals = []
            for r in range(reps):
                a = []
                for sgn in (1, -1):
                    q = asm.Problem(p.K, p.G + sgn * h * e, p.C, p.levels, w=p.w)
                    q.sample(chains, burn, sweeps, 70 + r, precision=asm.ASM_MIXED)
                    a.append(v @ q.average()["mean_A"])
                vals.append((a[0] - a[1]) / (2 * h))
            vals = np.array(vals)
            fds[h] = (vals.mean(), vals.std(ddof=1) / np.sqrt(reps))
        (f1, s1), (f2, s2) = fds[sigma], fds[0.5 * sigma]
        assert abs(f1 - want) <= 4 * np.hypot(s1, want_sem), (f1, s1, want, want_sem)
        assert abs(f1 - f2) <= 4 * np.hypot(s1, s2), (f1, f2, s1, s2)


def test_autograd_function_matches_the_c_abi():
    import torch
    from paper_1912_01379_gb300.autograd import ASMSpec, average_spectrum
    theta0 = torch.tensor(W.THETA0, dtype=torch.float64, requires_grad=True)

    def build(th):
        q = W.theta_problem(th, N=24, M=32, levels=[[0], [0, 12]])
        return q.K, q.C, q.w, q.levels, q.extra["dK_dtheta"], q.extra["dw_dtheta"]

    p = W.theta_problem(W.THETA0, N=24, M=32)
    G = torch.tensor(p.G, dtype=torch.float64, requires_grad=True)
    spec = ASMSpec(build=build, chains=128, burn_in=50, sweeps=400, seed=4, precision=asm.ASM_MIXED)
    A = average_spectrum(G, theta0, spec)
    v = torch.linspace(-1, 1, 24, dtype=torch.float64)
    gG, gth = torch.autograd.grad((A * v).sum(), (G, theta0))
    K, C, w, levels, dK, dw = build(W.THETA0)
    gp = asm.Problem(K, p.G, C, levels, w=w, dK_dtheta=dK, dw_dtheta=dw)
    gp.sample(128, 50, 400, 4, precision=asm.ASM_MIXED, moments=True)
    eG, et = gp.backward(v.numpy())
    assert np.allclose(gG.numpy(), eG, rtol=1e-12, atol=0)
    assert np.allclose(gth.numpy(), et, rtol=1e-12, atol=0)
    assert np.allclose(A.detach().numpy(), gp.average()["mean_A"], rtol=1e-12)
