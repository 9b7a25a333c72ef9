"""Pins of the oracle's numerical building blocks against things other than
itself: published known-answer vectors, numpy/scipy library routines and
80-digit mpmath evaluations of the exact definitions."""
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import special

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answer():
    with open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for r in rows:
        ctr = [int(x, 16) for x in r[0:4]]
        key = [int(x, 16) for x in r[4:6]]
        want = [int(x, 16) for x in r[7:11]]
        assert list(map(int, O.philox4x64_10(ctr, key))) == want


@pytest.mark.parametrize("ctr,key", [([5, 7, 11, 13], [123456789, 987654321]),
                                     ([2**64 - 1, 3, 0, 9], [42, 0]),
                                     ([1, 2**63, 2**40 + 5, 77], [2**64 - 1, 2**32])])
def test_philox_matches_numpy(ctr, key):
    # numpy's Philox (the 4x64-10 variant) adds one to the counter before each
    # block, so start it one below.
    c = list(ctr)
    c0 = (c[0] - 1) % 2**64
    c1 = (c[1] - (1 if c[0] == 0 else 0)) % 2**64
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array([c0, c1, c[2], c[3]], dtype=np.uint64))
    assert list(map(int, O.philox4x64_10(ctr, key))) == list(map(int, bg.random_raw(4)))


def test_norm_quantile_and_erfcx_match_scipy():
    for p in [1e-300, 1e-100, 1e-20, 1e-5, 0.01, 0.3, 0.5 - 1e-9, 0.7, 0.999999]:
        assert O.norm_quantile(p) == pytest.approx(special.ndtri(p), rel=4e-16, abs=4e-16)
    xs = np.concatenate([np.linspace(0, 3, 61), np.geomspace(3, 1e6, 80)])
    for x in xs:
        assert O.erfcx(x) == pytest.approx(special.erfcx(x), rel=2e-15)
    for x in [0.0, 1.0, 5.0, 40.0, 1e3]:
        want = float(mp.log(mp.erfc(mp.mpf(x) / mp.sqrt(2)) / 2))
        assert O.log_q(x) == pytest.approx(want, rel=1e-14, abs=1e-14)


# ---------------------------------------------------------------------------
# truncated normal: the draw IS the inverse CDF of the truncated normal, so a
# draw can be checked exactly against an 80-digit root of the definition.
# ---------------------------------------------------------------------------
mp.mp.dps = 80


def _q(x):
    return mp.erfc(x / mp.sqrt(2)) / 2


def _p(x):
    return mp.erfc(-x / mp.sqrt(2)) / 2


def _exact_std(a, b, u):
    u = mp.mpf(u)
    if a >= 0:
        tgt = (1 - u) * _q(a) + (u * _q(b) if np.isfinite(b) else 0)
        lo, hi = mp.mpf(a), mp.mpf(b if np.isfinite(b) else a + 60)
        for _ in range(260):
            m = (lo + hi) / 2
            lo, hi = (m, hi) if _q(m) > tgt else (lo, m)
        return (lo + hi) / 2
    if b <= 0:
        return -_exact_std(-b, -a, 1 - u)
    tgt = (1 - u) * _p(a) + u * _p(b)
    lo, hi = mp.mpf(max(a, -60)), mp.mpf(min(b, 60))
    for _ in range(260):
        m = (lo + hi) / 2
        lo, hi = (m, hi) if _p(m) < tgt else (lo, m)
    return (lo + hi) / 2


INTERVALS = [(-1, 2), (0.5, 3), (5, np.inf), (30, 31), (1000, np.inf), (-np.inf, -7),
             (-40, -39.9), (-400, -300), (-1e-3, 1e-3), (4.9, 5.1), (-3, np.inf), (0, np.inf),
             (-np.inf, 0), (-np.inf, np.inf), (6, 6.000001), (1e6, np.inf),
             (1000, 1000 + 1e-7), (-50 - 1e-6, -50), (7, 7.5)]
US = [2.0**-53, 1e-9, 0.01, 0.37, 0.5, 0.93, 1 - 1e-9, 1 - 2.0**-53]


def _grid(u):
    # uniforms the sampler sees are (k + 1/2) 2^-52
    if u in (2.0**-53, 1 - 2.0**-53):
        return u
    return float((np.floor(u * 2**52) + 0.5) * 2.0**-52)


@pytest.mark.parametrize("lo,hi", INTERVALS)
def test_truncnorm_is_exact_inverse_cdf(lo, hi):
    for u in US:
        u = _grid(u)
        x = O.truncnorm(0.0, 1.0, lo, hi, u)
        e = _exact_std(lo, hi, u)
        assert lo <= x <= hi
        err_ulps = float(abs(mp.mpf(x) - e) / (max(abs(e), 1) * mp.mpf(2) ** -52))
        assert err_ulps <= 16, (lo, hi, u, x, float(e))


def test_truncnorm_location_scale_and_monotone():
    # N(mu, s^2) on [lo, hi] is mu + s * N(0,1) on [(lo-mu)/s, (hi-mu)/s]
    for mu, s, lo, hi in [(3.0, 0.01, -1.0, 0.0), (-2.0, 5.0, 0.0, 1.0), (0.1, 1e-6, -1.0, 1.0)]:
        prev = -np.inf
        for u in np.linspace(0.001, 0.999, 57):
            u = _grid(u)
            x = O.truncnorm(mu, s, lo, hi, u)
            e = mu + s * float(_exact_std((lo - mu) / s, (hi - mu) / s, u))
            assert x == pytest.approx(e, rel=1e-12, abs=1e-14 * max(abs(lo), abs(hi)))
            assert x >= prev
            prev = x


def test_truncnorm_moments():
    # stratified uniforms give the exact mean of the truncated normal up to O(1/n^2)
    n = 20000
    us = (np.arange(n) + 0.5) / n
    for a, b in [(-1.0, 2.0), (2.0, 4.0), (8.0, np.inf), (-0.5, 0.5)]:
        xs = np.array([O.truncnorm(0.0, 1.0, a, b, u) for u in us])
        Z = _p(b) - _p(a) if np.isfinite(b) else _q(a)
        phi = lambda t: mp.exp(-mp.mpf(t) ** 2 / 2) / mp.sqrt(2 * mp.pi)
        mean = (phi(a) - (phi(b) if np.isfinite(b) else 0)) / Z
        assert xs.mean() == pytest.approx(float(mean), abs=2e-6)


# ---------------------------------------------------------------------------
# linear algebra against numpy
# ---------------------------------------------------------------------------
def test_cholesky_matches_numpy():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 30))
    C = A @ A.T + 30 * np.eye(30)
    assert np.allclose(O.cholesky(C), np.linalg.cholesky(C), rtol=1e-13, atol=1e-13)
    with pytest.raises(ValueError):
        O.cholesky(-np.eye(3))


@pytest.mark.parametrize("m,n", [(20, 50), (50, 20), (7, 7), (1, 5), (100, 50)])
def test_jacobi_svd(m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n)) * np.geomspace(1, 1e-6, n)[None, :]
    s, U, V = O.jacobi_svd(A)
    k = min(m, n)
    sn = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s[:k], sn, rtol=1e-12, atol=1e-14 * sn[0])
    assert np.all(np.diff(s) <= 0)
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)
    assert np.allclose(A @ V, U * s[None, :], atol=1e-13 * sn[0])
    if n > m:
        assert np.abs(A @ V[:, m:]).max() <= 1e-13 * sn[0]
    # sign convention: largest |component| of each V_j is positive
    for j in range(n):
        i = np.argmax(np.abs(V[:, j]))
        assert V[i, j] > 0


def _exact_offset(a, w, u):
    """t in [0, w] with int_0^t e^{-a s - s^2/2} = u int_0^w (80 digits)."""
    a, w, u = mp.mpf(a), mp.mpf(w), mp.mpf(u)
    r2 = mp.sqrt(2)
    if a >= 0:   # erfc differences: no cancellation against 1 in the tails
        I = lambda t: mp.exp(a * a / 2) * mp.sqrt(mp.pi / 2) * (mp.erfc(a / r2) - mp.erfc((a + t) / r2))
    else:
        I = lambda t: mp.exp(a * a / 2) * mp.sqrt(mp.pi / 2) * (mp.erfc(-(a + t) / r2) - mp.erfc(-a / r2))
    tgt = u * I(w)
    lo, hi = mp.mpf(0), w
    for _ in range(300):
        m = (lo + hi) / 2
        lo, hi = (m, hi) if I(m) < tgt else (lo, m)
    return (lo + hi) / 2


@pytest.mark.parametrize("a", [-3.0, -0.2, 0.0, 0.3, 2.0, 10.0, 1e3, 1e6, -1e6])
def test_truncnorm_narrow_intervals_keep_relative_accuracy(a):
    """On intervals much narrower than sigma (weak modes), delta - lo must stay
    accurate relative to hi - lo: lo = 0 and mu = -a put the interval at
    [a, a + w] in standard units with delta = t exactly representable."""
    for w in [1e-14, 1e-9, 1e-5, 1e-2, 0.3, 2.0]:
        if w * (abs(a) + w) > 5.0:
            continue
        for u in [1e-9, 0.2, 0.5, 0.97]:
            u = _grid(u)
            t = O.truncnorm(-a, 1.0, 0.0, w, u)
            e = _exact_offset(a, w, u)
            assert abs(mp.mpf(t) - e) <= 64 * mp.mpf(2) ** -52 * w, (a, w, u, t, float(e))
