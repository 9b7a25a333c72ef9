"""Default-model selection by fitting the grid density to the data (Sec. VI):
the fitted Gaussian width for the paper's optical-conductivity test case
matches the value the paper reads off its fit (tests/golden/default_model_fit.txt),
Pi_def has the sum rule at omega_m = 0 and tends to 0 at large omega_m for every
family, and the paper's Lorentzian grid of width 2.5 misfits the data far more
than the fitted densities (the paper finds that grid far from representing the data)."""
import math
import os

import numpy as np
import pytest

from paper_1912_01379_gb300 import default_model as D
from paper_1912_01379_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
OM = 2.0 * math.pi * np.arange(60) / 15.0


def _golden():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "default_model_fit.txt")) if l.strip() and l[0] != "#"]
    return [(r[0], float(r[1]), float(r[2])) for r in rows]


@pytest.mark.parametrize("kind,value,tol", _golden())
def test_fitted_density_matches_paper(kind, value, tol):
    data = W.matsubara_data(OM, model=2)
    p, _ = D.fit_grid_density(kind, OM, data)
    assert abs(p - value) <= tol, p


@pytest.mark.parametrize("kind", sorted(D.FAMILIES))
def test_pi_default_limits(kind):
    pd = D.pi_default(D.FAMILIES[kind](2.0), np.array([0.0, 1e-3, 1e4]), 0.5)
    assert pd[0] == 0.5
    assert abs(pd[1] - 0.5) < 0.5 * 1e-2     # omega_m -> 0: the whole density counts
    assert abs(pd[2]) < 0.5 * 1e-2           # omega_m -> inf: nothing left


def test_lorentzian_2p5_misfits():
    data = W.matsubara_data(OM, model=2)
    bad = D.misfit("lorentzian", 2.5, OM, data)
    for kind in ("gaussian", "exponential", "lorentzian"):
        _, best = D.fit_grid_density(kind, OM, data)
        assert bad > 3.0 * best
