"""GPU parity of the CUDA sampler (through the C ABI) against the FP64 CPU oracle.

* FP64 path, same singular vectors (the oracle's factors given to the library)
  and the same Philox stream: chain states after every sweep of a short run
  agree with the oracle's within 1e-9 relative (element by element).  A short
  run is the window over which the oracle reproduces itself from a start one
  ulp away (the sampler's map amplifies rounding differences each sweep).
* Invariants: fbar >= 0 after every sweep; the residual the kernel tracks
  incrementally equals |g~ - K~ f|^2 recomputed in FP64 within 1e-10 relative.
* One mixed-precision sweep from the same start with the same stream: every
  element within a multiple of the oracle's own divergence when each of its
  conditional means is moved by one rounding at FP32 resolution.
* Long runs with the library's own factorisation (cuSOLVER): <fbar> agrees with
  the oracle's within 4 combined Monte Carlo standard errors (the library's
  binned error, asm_mc_error; the spread of the oracle's independent chain
  means), in FP64 and in the mixed FP32/FP64 path; the blocked-modes run has
  the benchmark workload's 1000 burn-in and 10^4 kept sweeps.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_01379_gb300 import asm
from paper_1912_01379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_RTOL = 1e-9     # FP64 step-by-step tolerance (relative to the chain's max |f|)
CHI2_RTOL = 1e-10    # tracked vs recomputed chi^2
Z_MAX = 4.0          # long-run agreement in combined standard errors


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    torch.cuda.synchronize()


def _gpu_problem(p, factors=None, team=None):
    old = os.environ.get("ASM_TEAM_LANES")
    if team is not None:
        os.environ["ASM_TEAM_LANES"] = str(team)
    try:
        return asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, factors=factors)
    finally:
        if team is not None:
            if old is None:
                os.environ.pop("ASM_TEAM_LANES", None)
            else:
                os.environ["ASM_TEAM_LANES"] = old


def _step_cases():
    yield "plain_modes", W.plain_modes_problem()
    # several levels, ragged blocks spanning more than one register tile,
    # N > M (zero modes), a components level
    yield "ragged_levels", W.small_problem(30, 150, seed=21, levels=[[0], [0, 37, 87], np.arange(150)[::10],
                                                                    np.arange(150)])
    yield "tall_M_gt_N", W.small_problem(40, 12, seed=22, levels=[[0], [0, 5]])
    yield "bosonic", W.small_problem(25, 70, seed=23, levels=[[0], [0, 20, 45]], bosonic=True)


def _short_run_window(op, chains, sweeps, seed, f0):
    """Sweeps over which FP64 trajectories are reproducible at all: the oracle
    is run again from a start perturbed by one ulp, and the window ends at the
    first sweep where its own two trajectories differ by more than 1e-11
    (relative).  The Gibbs map of blocked modes sampling amplifies rounding
    differences by ~1e2-1e4 per sweep, so later sweeps of two correct FP64
    implementations differ by more than any fixed tolerance."""
    a = op.run(chains, 0, sweeps, seed=seed, trace_chains=chains, f_start=f0)["trace"]
    b = op.run(chains, 0, sweeps, seed=seed, trace_chains=chains, f_start=f0 * (1 + 2.0**-52))["trace"]
    sens = (np.abs(a - b) / np.abs(a).max(axis=2, keepdims=True)).max(axis=(0, 2))
    n = 0
    while n < sweeps and sens[n] <= 1e-11:
        n += 1
    return max(n, 1), a


@pytest.mark.parametrize("team", [32, 8])
@pytest.mark.parametrize("case", list(range(4)))
def test_fp64_matches_oracle_step_by_step(case, team):
    name, p = list(_step_cases())[case]
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    dec = op.decomposition()
    chains, sweeps, seed = 7, 6, 1234 + case
    window, ref = _short_run_window(op, chains, sweeps, seed, op.initial_f())
    gp = _gpu_problem(p, factors=dec, team=team)
    for s in range(sweeps):
        gp.sample(chains, 0, 1, seed, precision=asm.ASM_FP64, cont=s > 0)
        f, chi2 = gp.chain_state()
        if s < window:
            want = ref[:, s, :]
            err = np.abs(f - want) / np.abs(want).max(axis=1, keepdims=True)
            assert err.max() <= STEP_RTOL, (name, team, s, err.max())
        # invariants hold on every sweep: A >= 0 and the tracked residual
        assert f.min() >= 0.0
        exact = np.sum((dec.gt[None, :] - f @ dec.Kt.T) ** 2, axis=1)
        assert np.allclose(chi2, exact, rtol=CHI2_RTOL, atol=0), (name, s)
    st = gp.status()
    assert st["nonfinite_moves"] == 0


def test_fp64_full_size_sampled_chains():
    """The blocked-modes workload at full size (N=400, M=100, 1024 chains) in the
    launch configuration of the benchmark: sampled chains match the oracle over
    the reproducible window (one sweep here)."""
    p = W.blocked_modes_problem()
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    dec = op.decomposition()
    chains, seed = 1024, 77
    idx = [0, 1, 333, 511, 512, 777, 1022, 1023]
    ref = op.run(chains, 0, 1, seed=seed, threads=0)
    gp = _gpu_problem(p, factors=dec)
    gp.sample(chains, 0, 1, seed, precision=asm.ASM_FP64)
    f, chi2 = gp.chain_state()
    want = ref["f_final"][idx]
    err = np.abs(f[idx] - want) / np.abs(want).max(axis=1, keepdims=True)
    assert err.max() <= STEP_RTOL, err.max()
    assert np.allclose(chi2[idx], ref["chi2"][idx], rtol=1e-9)
    assert f.min() >= 0.0
    # and beyond the window the invariants still hold at full size
    gp.sample(chains, 0, 20, seed, precision=asm.ASM_FP64, cont=True)
    f, chi2 = gp.chain_state()
    assert f.min() >= 0.0
    exact = np.sum((dec.gt[None, :] - f[idx] @ dec.Kt.T) ** 2, axis=1)
    assert np.allclose(chi2[idx], exact, rtol=CHI2_RTOL)


# The mixed path rounds its chain state, residual, bounds and draw arithmetic to
# FP32 (unit roundoff 2^-24).  Its distance from the FP64 oracle after one sweep
# is measured against the oracle's own divergence from a run in which every
# move's conditional mean and interval ends are moved by one FP32 rounding
# (ora_set_jitter at 2^-24; the largest difference over JITTER_PATTERNS sets of
# rounding directions, so that one lucky set does not make a chain look
# insensitive): the mixed path commits O(M) such roundings per move where the
# probe commits one (c_j and the residual are sums over the M data points), and
# their sum grows like sqrt(M) for independent roundings.  The bound is
# MIXED_ENV sqrt(M) times that envelope (the chain's largest element
# difference), plus 2^-22 of the chain's largest element for the rounding of
# the stored state itself.
MIXED_ENV = 4.0
JITTER_PATTERNS = 4


@pytest.mark.parametrize("case", list(range(4)))
def test_mixed_precision_tracks_fp64_over_one_sweep(case):
    name, p = list(_step_cases())[case]
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    dec = op.decomposition()
    chains, seed = 16, 5
    ref = op.run(chains, 0, 1, seed=seed)["f_final"]
    env = np.zeros((chains, 1))
    for pattern in range(JITTER_PATTERNS):
        op.set_jitter(True, unit_exp=24, pattern=pattern)
        probe = op.run(chains, 0, 1, seed=seed)["f_final"]
        env = np.maximum(env, np.abs(probe - ref).max(axis=1, keepdims=True))
    op.set_jitter(False)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    gp = _gpu_problem(p, factors=dec)
    gp.sample(chains, 0, 1, seed, precision=asm.ASM_MIXED)
    f, _ = gp.chain_state()
    assert f.min() >= 0.0
    bound = MIXED_ENV * np.sqrt(p.K.shape[0]) * env + 2.0**-22 * scale
    excess = np.abs(f - ref) / bound
    assert excess.max() <= 1.0, (name, float(excess.max()), float(np.median(np.abs(f - ref) / scale)))


_ORACLE_RUNS = {}


def _oracle_long(p, key, chains_cpu, burn, sweeps, seed, chain0):
    # the same oracle run serves the FP64 and the mixed comparison
    k = (key, chains_cpu, burn, sweeps, seed, chain0)
    if k not in _ORACLE_RUNS:
        op = O.OracleProblem(p.K, p.G, p.C, p.levels)
        r = op.run(chains_cpu, burn, sweeps, seed=seed, threads=0, chain_offset=chain0)
        _ORACLE_RUNS[k] = O.summarize(r["S1"], r["S2"], r["kept"], p.w)
    return _ORACLE_RUNS[k]


def _long_run(p, key, chains_gpu, chains_cpu, burn, sweeps, precision, seed):
    # the same level schedule (seed, problem id) with chain ids disjoint from the GPU's: all chains
    # of a run share the level of each sweep, so runs under different schedules differ by a
    # schedule-dependent burn-in transient that the spread of the chain means does not measure
    so = _oracle_long(p, key, chains_cpu, burn, sweeps, seed, chains_gpu)
    gp = _gpu_problem(p)                   # library's own cuSOLVER factors
    gp.sample(chains_gpu, burn, sweeps, seed, precision=precision)
    sg = gp.average()
    me = gp.mc_error()                     # binned error (or the chain-mean spread, if larger)
    assert np.all(me["sem_fbar"] >= sg["sem_fbar"] * (1 - 1e-12))
    z = (sg["mean_fbar"] - so["mean_fbar"]) / np.hypot(me["sem_fbar"], so["sem_fbar"])
    return z, sg, so, gp.status()


@pytest.mark.parametrize("precision", [asm.ASM_FP64, asm.ASM_MIXED])
def test_long_run_plain_modes(precision):
    p = W.plain_modes_problem()
    z, sg, so, st = _long_run(p, "plain", 256, 64, 1000, 10000, precision, seed=11)
    assert np.all(np.abs(z) < Z_MAX), np.abs(z).max()
    assert st["nonfinite_moves"] == 0
    assert np.allclose(sg["mean_A"], sg["mean_fbar"] / p.w)


@pytest.mark.parametrize("precision", [asm.ASM_FP64, asm.ASM_MIXED])
def test_long_run_blocked_modes(precision):
    """The benchmark workload as it is timed (1024 chains, 1000 + 10^4 sweeps)
    against 256 oracle chains of the same length."""
    p = W.blocked_modes_problem()
    z, sg, so, st = _long_run(p, "blocked", 1024, 256, 1000, 10000, precision, seed=12)
    assert np.all(np.abs(z) < Z_MAX), np.abs(z).max()
    assert st["nonfinite_moves"] == 0
    assert st["max_resync_drift"] < (1e-8 if precision == asm.ASM_FP64 else 1e-2)


def test_edge_cases_and_errors():
    p = W.small_problem(10, 9, seed=3, levels=[[0], [0, 1, 8]])
    gp = _gpu_problem(p)
    gp.sample(1, 0, 3, 1, precision=asm.ASM_FP64)           # a single chain
    f, _ = gp.chain_state()
    assert f.shape == (1, 9) and f.min() >= 0
    gp.sample(33, 2, 3, 1, precision=asm.ASM_MIXED)          # ragged last warp
    r = gp.average()
    assert np.all(np.isfinite(r["mean_A"]))
    with pytest.raises(asm.ASMError):                        # continue with other chains
        gp.sample(34, 0, 1, 1, precision=asm.ASM_MIXED, cont=True)
    with pytest.raises(asm.ASMError, match="symmetric positive"):
        asm.Problem(p.K, p.G, -p.C, p.levels)
    with pytest.raises(asm.ASMError, match="partition"):
        asm.Problem(p.K, p.G, p.C, [[2, 5]])
    K = np.ones((2, 2)); K[:, 1] = -1.0
    with pytest.raises(asm.ASMError, match="improper"):
        asm.Problem(K, np.ones(2), np.eye(2), [[0]])
    G = p.G.copy(); G[1] = np.inf
    with pytest.raises(asm.ASMError, match="non-finite"):
        asm.Problem(p.K, G, p.C, p.levels)
    import torch
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(asm.ASMError, match="workspace"):
        gp.sample(4, 0, 1, 1, workspace=small)


def test_shards_reproduce_the_unsharded_run_chain_by_chain():
    """Replicas: chains keyed by global id, so two shards equal one run."""
    p = W.small_problem(16, 40, seed=9, levels=[[0], [0, 13, 29]])
    whole = _gpu_problem(p)
    whole.sample(20, 5, 30, 77, precision=asm.ASM_MIXED)
    fw, _ = whole.chain_state()
    parts = []
    for off, n in [(0, 12), (12, 8)]:
        gp = _gpu_problem(p)
        gp.set_stream_ids(0, off)
        gp.sample(n, 5, 30, 77, precision=asm.ASM_MIXED)
        parts.append(gp.chain_state()[0])
    assert np.array_equal(np.concatenate(parts), fw)


@pytest.mark.parametrize("precision", [asm.ASM_FP64, asm.ASM_MIXED])
def test_checkpoint_restore_continues_bit_for_bit(precision):
    p = W.small_problem(16, 40, seed=10, levels=[[0], [0, 13, 29]])
    ref = _gpu_problem(p)
    ref.sample(9, 10, 130, 5, precision=precision)          # crosses a refresh boundary
    f_ref, chi_ref = ref.chain_state()
    avg_ref = ref.average()
    a = _gpu_problem(p)
    a.sample(9, 10, 50, 5, precision=precision)
    blob = a.checkpoint()
    del a
    b = _gpu_problem(p)
    b.restore(blob, 9, precision=precision)
    b.sample(9, 0, 80, 5, precision=precision, cont=True)
    f_b, chi_b = b.chain_state()
    assert np.array_equal(f_b, f_ref)
    assert np.array_equal(chi_b, chi_ref)
    assert np.array_equal(b.average()["mean_fbar"], avg_ref["mean_fbar"])
    # the bins of the Monte Carlo error continue too: the restored run keeps the start of
    # the kept sweeps, so the bin that holds burn-in sweeps stays out on both sides
    me_b, me_ref = b.mc_error(), ref.mc_error()
    assert np.array_equal(me_b["bins_per_chain"], me_ref["bins_per_chain"])
    assert np.array_equal(me_b["sigma2_levels"], me_ref["sigma2_levels"], equal_nan=True)
    assert np.array_equal(me_b["ess"], me_ref["ess"], equal_nan=True)
