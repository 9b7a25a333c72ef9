"""Inputs of the paper's own test case (Sec. III): the optical-conductivity
models on bosonic Matsubara frequencies.  Pins: the kernel's m = 0 row is the
sum rule 2/pi; the Riemann sum K fbar_true on each grid (Eq. Riemann) agrees
with the data computed by adaptive quadrature of Eq. optcond, two independent
discretisations of the same integral; the half-line grids are increasing and
positive with the widths of their density (Sec. V.B table)."""
import math

import numpy as np
import pytest

from paper_1912_01379_gb300 import workloads as W


def test_sum_rule_row():
    K = W.matsubara_kernel(np.array([0.0, 1.0]), np.array([0.1, 1.0, 10.0]))
    assert np.allclose(K[0], 2.0 / math.pi)
    assert np.allclose(K[1], 2.0 / math.pi * np.array([0.01 / 1.01, 0.5, 100.0 / 101.0]))


@pytest.mark.parametrize("grid,N,tol", [("uniform", 64, 1e-3), ("uniform", 256, 1e-3), ("gaussian", 64, 1e-3),
                                        ("exponential", 64, 1e-3), ("lorentzian", 64, 1e-3)])
@pytest.mark.parametrize("model", [1, 2])
def test_riemann_sum_matches_quadrature(grid, N, tol, model):
    p = W.paper_problem(model, 1e-3, grid, N)
    rel = np.abs(p.K @ p.fbar_true - p.extra["pi_exact"]) / p.extra["pi_exact"]
    assert rel.max() < tol, rel.max()
    assert p.K.shape == (60, N) and np.all(p.K > 0)


@pytest.mark.parametrize("kind,param", [("gaussian", 4.0), ("exponential", 3.0), ("lorentzian", 2.5)])
def test_half_line_grids(kind, param):
    x, w = W.half_line_grid(kind, 64, param)
    assert np.all(x > 0) and np.all(np.diff(x) > 0) and np.all(w > 0)
    # w_n = 1 / (N rho(x_n)) with the density of the table
    rho = {"gaussian": lambda t: np.exp(-t * t / (2 * param ** 2)) / (math.sqrt(2 * math.pi) * param / 2),
           "exponential": lambda t: np.exp(-t / param) / param,
           "lorentzian": lambda t: (2 / (math.pi * param)) / (1 + (t / param) ** 2)}[kind]
    assert np.allclose(w, 1.0 / (64 * rho(x)), rtol=1e-10)
