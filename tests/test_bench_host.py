"""CPU checks of bench.py's host-side accounting.

The roofline's algorithmic work per step depends on the levels the sampler
draws (one per sweep, shared by all chains: word 0 of Philox4x64-10 at counter
{2^64 - 1, sweep, 0, problem}, Sec. IV.C).  bench.py replays that schedule with
numpy's Philox, whose generator advances its counter before each block; here
it is compared with the oracle's own Philox4x64-10 (plain C, pinned against the
published known-answer vector), draw by draw.
"""
import numpy as np
import pytest

import bench
from oracle import oracle as O


def _oracle_levels(seed, n_sweeps, n_levels, problem_id):
    out = np.empty(n_sweeps, dtype=np.int64)
    for s in range(n_sweeps):
        w0 = int(O.philox4x64_10([2**64 - 1, s, 0, problem_id], [seed, 0])[0])
        u = ((w0 >> 12) + 0.5) * 2.0 ** -52
        out[s] = min(int(u * n_levels), n_levels - 1)
    return out


@pytest.mark.parametrize("seed,n_levels,problem_id", [(1, 2, 0), (2024, 10, 3), (2**63 + 5, 3, 7)])
def test_level_schedule_matches_the_oracle(seed, n_levels, problem_id):
    got = bench._level_sequence(seed, 300, n_levels, problem_id)
    ref = _oracle_levels(seed, 300, n_levels, problem_id)
    assert np.array_equal(got, ref)
    assert set(np.unique(got)) == set(range(n_levels))   # every level is drawn over 300 sweeps


def test_ops_per_level_adds_blocks():
    """Block work adds over the blocks of a level: the whole grid as one block
    has more pass elements than the same grid cut in two (n^2 per block), and a
    level of one-point blocks has N pass elements and 2 M N projection FMAs."""
    class P:
        M, N = 20, 60
        levels = [np.array([0]), np.array([0, 30]), np.arange(60)]
    elems, fmas = bench._ops_per_level(P)
    assert elems[0] > elems[1] > 0
    assert elems[0] == 60 * 60 and elems[1] == 2 * 30 * 30
    assert elems[2] == 60 and fmas[2] == 2 * 20 * 60
    assert fmas[0] == 2 * 20 * 20 and fmas[1] == 2 * (2 * 20 * 20)


def test_roofline_peak_is_the_weighted_harmonic_mean():
    """The peak is the rate of the same work at the measured rates: all-pass
    work peaks at 6 x the pass rate, all-FMA work at the FMA rate, and a mix
    lies between them."""
    ceil = {"pass_f32": {"rate": 1e12}, "ffma": {"rate": 3e13}}
    a, pk = bench.roofline(np.float64(1e9), np.float64(0.0), 1.0, ceil, "f32")
    assert pk == pytest.approx(6e12 / 1e12) and a == pytest.approx(6e9 / 1e12)
    _, pk = bench.roofline(np.float64(0.0), np.float64(1e9), 1.0, ceil, "f32")
    assert pk == pytest.approx(3e13 / 1e12)
    _, pk = bench.roofline(np.float64(1e9), np.float64(1e9), 1.0, ceil, "f32")
    assert 6.0 < pk < 30.0
    assert pk == pytest.approx(7e9 / (1e9 / 1e12 + 1e9 / 3e13) / 1e12)
