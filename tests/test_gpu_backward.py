"""Backward pass: vector-Jacobian products of <A> from the covariance identity
(asm_backward), against closed forms the mathematics fixes:
 * the unconstrained Gaussian limit (N <= M, positivity inactive), where
   <fbar> = (K~^T K~)^{-1} K~^T g~ exactly, for the G-gradient and, by central
   differences of that closed form over the grid-density parameters, the
   theta-gradient;
 * a 2-point grid with positivity binding, where <f> is known by quadrature and
   its G-derivative by central differences of the quadrature.
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


def _gaussian_limit_problem():
    M, N, beta = 64, 6, 16.0
    tau = W.tau_grid(beta, M)
    omega, w = W.uniform_grid(-6.0, 6.0, N)
    K = W.fermionic_kernel(tau, omega, beta)
    A = 0.4 * W.gauss_pdf(omega, -1.0, 0.8) + 0.6 * W.gauss_pdf(omega, 2.0, 0.6) + 10.0
    C = np.eye(M) * 1e-4 ** 2
    G = K @ (A * w) + np.random.default_rng(4).standard_normal(M) * 1e-4
    return K, G, C, w


def _exact_mean(K, G, C):
    L = np.linalg.cholesky(C)
    Kt, gt = np.linalg.solve(L, K), np.linalg.solve(L, G)
    P = np.linalg.inv(Kt.T @ Kt)
    return P @ Kt.T @ gt, P, L, Kt


@pytest.mark.parametrize("precision,tol", [(asm.ASM_FP64, 0.02), (asm.ASM_MIXED, 0.05)])
def test_grad_G_gaussian_limit(precision, tol):
    K, G, C, w = _gaussian_limit_problem()
    mean, P, L, Kt = _exact_mean(K, G, C)
    assert np.min(mean / np.sqrt(np.diag(P))) >= 10          # positivity inactive
    gp = asm.Problem(K, G, C, [[0], [0, 3]], w=w)
    gp.sample(256, 200, 4000, 3, precision=precision, moments=True)
    v = np.random.default_rng(1).standard_normal(len(w))
    gG, _ = gp.backward(v)
    exact = np.linalg.solve(L.T, Kt @ (P @ (v / w)))          # C^{-1} K Cov (v/w)
    assert np.linalg.norm(gG - exact) <= tol * np.linalg.norm(exact)
    r = gp.average()
    assert np.allclose(r["mean_fbar"], mean, rtol=1e-3)


def test_grad_theta_gaussian_limit():
    theta0 = W.THETA0.copy()
    build = lambda th: W.theta_problem(th, N=6, offset=10.0, levels=[[0]])
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
    gp.sample(256, 200, 4000, 5, precision=asm.ASM_FP64, moments=True)
    _, gt = gp.backward(v)
    assert np.linalg.norm(gt - fd) <= 0.03 * np.linalg.norm(fd), (gt, fd)


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
    gp.sample(512, 200, 8000, 9, precision=asm.ASM_FP64, moments=True)
    gG, _ = gp.backward(v)
    assert np.linalg.norm(gG - fd) <= 0.03 * np.linalg.norm(fd), (gG, fd)


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
