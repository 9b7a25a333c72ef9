"""CPU checks of the grid-density inputs of the theta-gradient: the grid
inverts the mixture CDF, the weights integrate the interval, and dK/dtheta,
dw/dtheta agree with finite differences taken with another step."""
import numpy as np

from paper_1912_01379_gb300 import workloads as W


def test_mixture_grid_and_derivatives():
    p = W.theta_problem(N=40, M=16)
    th = p.extra["theta"]
    cdf, pdf = W.mixture_cdf_pdf(p.omega, th)
    assert np.allclose(cdf, (np.arange(40) + 0.5) / 40, atol=1e-13)
    assert np.allclose(p.w, 1 / (40 * pdf), rtol=1e-13)
    assert abs(p.w.sum() - 12.0) < 0.5                       # Riemann weights span [-6, 6]
    for k in range(len(th)):
        e = np.zeros(len(th)); e[k] = 3e-4
        xp, wp = W.mixture_grid(th + e, 40)
        xm, wm = W.mixture_grid(th - e, 40)
        Kp = W.fermionic_kernel(p.extra["tau"], xp, p.extra["beta"])
        Km = W.fermionic_kernel(p.extra["tau"], xm, p.extra["beta"])
        dK = (Kp - Km) / 6e-4
        assert np.abs(dK - p.extra["dK_dtheta"][k]).max() <= 1e-5 * np.abs(dK).max() + 1e-14
        assert np.allclose((wp - wm) / 6e-4, p.extra["dw_dtheta"][k], rtol=1e-5, atol=1e-9)
