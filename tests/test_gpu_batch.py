"""Batched sampling (asm_setup_batch): many independent problems with uneven
N_omega, N_tau and block counts in the same persistent launches.

* Problem k of a batch keys its Philox stream with problem id k, so it must
  reproduce, bit for bit, a single handle of that problem with problem id k:
  the work-item order, the CTA that runs a chain group and the launch shape
  change no arithmetic.  The same holds for the launch shape picked by the
  autotuner (lanes per chain, chain warps per CTA), and for whole refresh
  periods replayed from the CUDA graph versus launched one by one.
* FP64 batch against the oracle over a short window (same factors, same
  stream): 1e-9 relative; a long mixed-precision batch run agrees with the
  oracle's long runs within 4 combined standard errors for every problem.
  Both runs share the level schedule (same seed and problem id) and use
  disjoint chain ids: all chains of a run share the level drawn for each
  sweep, so runs with different schedules differ by a schedule-dependent
  burn-in transient that the spread of the chain means does not measure.
* The full-size batching workload (256 problems, 64 chains each) runs without
  timeouts or non-finite moves and matches single-problem runs on sampled
  problems.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_01379_gb300 import asm
from paper_1912_01379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

Z_MAX = 4.0


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    torch.cuda.synchronize()


def _spec(p, factors=None):
    return dict(K=p.K, G=p.G, C=p.C, levels=p.levels, w=p.w, factors=factors)


def _uneven_small():
    """Small problems with different M, N, level and block structure."""
    return [
        W.small_problem(20, 60, seed=31, levels=[[0], [0, 25, 40]]),
        W.small_problem(35, 130, seed=32, levels=[[0], [0, 30, 70, 100], np.arange(130)[::13]]),
        W.small_problem(12, 40, seed=33, levels=[[0]]),
        W.small_problem(28, 90, seed=34, levels=[[0], [0, 45]], bosonic=True),
        W.small_problem(50, 25, seed=35, levels=[[0], [0, 10]]),
    ]


def _assert_status_clean(st):
    assert st["timeouts"] == 0
    assert st["nonfinite_moves"] == 0


@pytest.mark.parametrize("prec", [asm.ASM_FP64, asm.ASM_MIXED])
def test_batch_equals_single_problems(prec):
    probs = _uneven_small()
    b = asm.Batch([_spec(p) for p in probs])
    assert len(b) == len(probs)
    chains, burn, sweeps, seed = 37, 10, 190, 77   # ragged chain groups; whole periods replayed
    b.sample(chains, burn, sweeps, seed, precision=prec)
    st = b.status()
    _assert_status_clean(st)
    assert st["graph_replays"] >= 2
    assert st["work_items"] >= len(probs)
    for k, p in enumerate(probs):
        got = b.average(k)
        one = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
        one.set_stream_ids(k, 0)
        one.sample(chains, burn, sweeps, seed, precision=prec)
        ref = one.average()
        assert np.array_equal(got["mean_fbar"], ref["mean_fbar"]), k
        assert np.array_equal(got["sem_fbar"], ref["sem_fbar"]), k


def test_batch_problem_ids_offset_by_handle_id():
    probs = _uneven_small()[:2]
    b = asm.Batch([_spec(p) for p in probs])
    b.set_stream_ids(40, 0)
    b.sample(16, 0, 20, 5, precision=asm.ASM_FP64)
    one = asm.Problem(probs[1].K, probs[1].G, probs[1].C, probs[1].levels, w=probs[1].w)
    one.set_stream_ids(41, 0)
    one.sample(16, 0, 20, 5, precision=asm.ASM_FP64)
    assert np.array_equal(b.average(1)["mean_fbar"], one.average()["mean_fbar"])


def test_graph_replay_equals_direct_launches():
    p = W.small_problem(30, 150, seed=21, levels=[[0], [0, 37, 87], np.arange(150)[::10]])
    a = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    a.sample(40, 0, 300, 9, precision=asm.ASM_MIXED)                 # graph replays
    sa = a.status()
    assert sa["graph_replays"] >= 4
    b = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    b.sample(40, 0, 300, 9, precision=asm.ASM_MIXED, timing=True)    # every launch direct
    sb = b.status()
    assert sb["graph_replays"] == 0 and sb["timed_launches"] == sb["sweep_launches"]
    assert np.array_equal(a.average()["mean_fbar"], b.average()["mean_fbar"])
    fa, ca = a.chain_state()
    fb, cb = b.chain_state()
    assert np.array_equal(fa, fb) and np.array_equal(ca, cb)
    # continuing replays the kept graph
    a.sample(40, 0, 128, 9, precision=asm.ASM_MIXED, cont=True)
    b.sample(40, 0, 128, 9, precision=asm.ASM_MIXED, cont=True, timing=True)
    assert np.array_equal(a.average()["mean_fbar"], b.average()["mean_fbar"])


@pytest.mark.parametrize("prec", [asm.ASM_FP64, asm.ASM_MIXED])
def test_tuned_shape_changes_no_result(prec):
    probs = _uneven_small()
    b = asm.Batch([_spec(p) for p in probs])
    b.sample(64, 0, 70, 3, precision=prec)
    ref = [b.average(k)["mean_fbar"] for k in range(len(probs))]
    team, cons, minb = b.tune(64, precision=prec)
    assert team in (8, 16, 32) and cons in (0, 2, 3, 4, 5, 6, 7) and minb in (1, 2)
    with pytest.raises(asm.ASMError):   # the trial chains replaced the state
        b.sample(64, 0, 1, 3, precision=prec, cont=True)
    b.sample(64, 0, 70, 3, precision=prec)
    st = b.status()
    assert st["team_lanes"] == team and st["min_blocks"] == minb
    for k in range(len(probs)):
        assert np.array_equal(b.average(k)["mean_fbar"], ref[k]), (k, team, cons)


def test_batch_fp64_short_window_against_oracle():
    probs = _uneven_small()[:3]
    facs = [O.OracleProblem(p.K, p.G, p.C, p.levels) for p in probs]
    b = asm.Batch([_spec(p, op.decomposition()) for p, op in zip(probs, facs)])
    chains, seed = 8, 123
    b.sample(chains, 0, 1, seed, precision=asm.ASM_FP64)   # one sweep: inside every problem's parity window
    for k, (p, op) in enumerate(zip(probs, facs)):
        r = op.run(chains, 0, 1, seed=seed, problem_id=k)
        ref = O.summarize(r["S1"], r["S2"], 1)["mean_fbar"]
        got = b.average(k)["mean_fbar"]
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref)), k


def test_batch_long_run_against_oracle():
    probs = _uneven_small()[:3]
    chains, burn, sweeps = 64, 200, 2000
    b = asm.Batch([_spec(p) for p in probs])
    b.sample(chains, burn, sweeps, 2024, precision=asm.ASM_MIXED)
    _assert_status_clean(b.status())
    for k, p in enumerate(probs):
        op = O.OracleProblem(p.K, p.G, p.C, p.levels)
        # same seed and problem id (the level schedule all chains share), disjoint chain ids
        r = op.run(32, burn, sweeps, seed=2024, problem_id=k, chain_offset=chains)
        ref = O.summarize(r["S1"], r["S2"], sweeps)
        got = b.average(k)
        z = np.abs(got["mean_fbar"] - ref["mean_fbar"]) / np.sqrt(got["sem_fbar"] ** 2 + ref["sem_fbar"] ** 2)
        assert np.nanmax(z) < Z_MAX, (k, float(np.nanmax(z)))


def test_batch_rejects_single_problem_calls():
    b = asm.Batch([_spec(p) for p in _uneven_small()[:2]])
    b.sample(8, 0, 4, 1, precision=asm.ASM_MIXED)
    L = asm.load()
    z = np.zeros(1000)
    assert L.asm_average(b._h, asm._dptr(z), asm._dptr(z), asm._dptr(z), asm._dptr(z)) == -7
    assert L.asm_chain_state(b._h, asm._dptr(z), asm._dptr(z)) == -7
    with pytest.raises(asm.ASMError):
        b.sample(8, 0, 4, 1, precision=asm.ASM_MIXED, moments=True)
    assert L.asm_average_at(b._h, 2, asm._dptr(z), asm._dptr(z), asm._dptr(z), asm._dptr(z)) == -7


def test_full_size_batch_workload():
    probs = W.batch_problems()
    chains = probs[0].chains
    b = asm.Batch([_spec(p) for p in probs])
    b.sample(chains, 0, 128, 1003, precision=asm.ASM_MIXED)
    st = b.status()
    _assert_status_clean(st)
    assert st["sweeps_done"] == 128 and st["graph_replays"] == 2
    for k in (0, 101, 255):
        p = probs[k]
        got = b.average(k)["mean_fbar"]
        assert np.all(got >= 0) and np.all(np.isfinite(got))
        one = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
        one.set_stream_ids(k, 0)
        one.sample(chains, 0, 128, 1003, precision=asm.ASM_MIXED)
        assert np.array_equal(got, one.average()["mean_fbar"]), k
