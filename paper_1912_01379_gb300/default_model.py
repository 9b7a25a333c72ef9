"""Choosing the grid density, which acts as the default model of the average
spectrum (Sec. VI, "Practical method"): the default optical conductivity
sigma_def(omega) = pi Pi(0) rho(omega) / 2 of a grid density rho has the
imaginary-axis values

    Pi_def(omega_m) = Pi(0) (1 - int_0^inf rho(omega) / (1 + (omega/omega_m)^2) d omega),

and a family's parameter is chosen to minimise sum_m (Pi(omega_m) - Pi_def(omega_m))^2,
the misfit of the default model to the data.  Host code (scipy quadrature and a
bounded scalar search); the chosen density then gives the grid of
workloads.half_line_grid.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

# densities on [0, inf) of the grid families (Sec. V.B table), normalised
FAMILIES = {
    "gaussian": lambda a: (lambda x: np.exp(-x * x / (2.0 * a * a)) / (math.sqrt(2.0 * math.pi) * a / 2.0)),
    "exponential": lambda b: (lambda x: np.exp(-x / b) / b),
    "lorentzian": lambda g: (lambda x: (2.0 / (math.pi * g)) / (1.0 + (x / g) ** 2)),
}


def pi_default(rho, omega_m, pi0):
    """Pi_def(omega_m) of the density rho (a callable on [0, inf)) for the
    Matsubara frequencies omega_m, given Pi(0) = pi0 (the sum rule)."""
    out = np.empty(len(omega_m))
    for i, om in enumerate(omega_m):
        if om == 0.0:
            out[i] = pi0
            continue
        f = lambda x, om=om: rho(x) / (1.0 + (x / om) ** 2)
        out[i] = pi0 * (1.0 - integrate.quad(f, 0.0, np.inf, limit=200, epsabs=1e-14, epsrel=1e-12)[0])
    return out


def misfit(kind, param, omega_m, data):
    """sum_m (Pi(omega_m) - Pi_def(omega_m))^2 for family `kind` with parameter `param`;
    Pi(0) is taken from the data at omega_m = 0."""
    pi0 = float(np.asarray(data)[np.asarray(omega_m) == 0.0][0])
    return float(np.sum((np.asarray(data) - pi_default(FAMILIES[kind](param), omega_m, pi0)) ** 2))


def fit_grid_density(kind, omega_m, data, bounds=(0.2, 20.0)):
    """The family parameter (Gaussian alpha, exponential beta or Lorentzian
    gamma) whose default model fits the data best; returns (param, misfit)."""
    res = optimize.minimize_scalar(lambda t: misfit(kind, t, omega_m, data), bounds=bounds, method="bounded",
                                   options={"xatol": 1e-6})
    return float(res.x), float(res.fun)
