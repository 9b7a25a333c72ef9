"""Blocked modes sampling over the full partition hierarchy (asm_partition_hierarchy:
whole grid, halved blocks with every other level shifted, single points) through
the C ABI against the FP64 oracle on the same levels.

* FP64 with the oracle's factors and Philox stream: one sweep of every chain
  within 1e-9 (relative to the chain's largest value) -- a sweep draws one level
  at random, so the sampled chains pass through different levels.
* Mixed precision with the library's own factors: <fbar> within 4 combined
  standard errors of the oracle's long run (same level schedule, disjoint chain
  ids, as in the other long-run tests)."""
import numpy as np
import pytest

from oracle import oracle as O
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


def _problem():
    p = W.small_problem(24, 64, seed=41, levels=[[0]])
    return p, asm.partition_hierarchy(p.N)


def test_hierarchy_fp64_one_sweep_against_oracle():
    p, levels = _problem()
    assert len(levels) == 7
    op = O.OracleProblem(p.K, p.G, p.C, levels)
    dec = op.decomposition()
    gp = asm.Problem(p.K, p.G, p.C, levels, w=p.w, factors=dec)
    for seed in (5, 6, 7, 8):   # several level draws
        chains = 16
        ref = op.run(chains, 0, 1, seed=seed)["f_final"]
        gp.sample(chains, 0, 1, seed, precision=asm.ASM_FP64)
        f, _ = gp.chain_state()
        err = np.abs(f - ref) / np.abs(ref).max(axis=1, keepdims=True)
        assert err.max() <= 1e-9, (seed, err.max())
        assert f.min() >= 0.0


def test_hierarchy_mixed_long_run_against_oracle():
    p, levels = _problem()
    chains_gpu, chains_cpu, burn, sweeps, seed = 1024, 128, 300, 3000, 17
    gp = asm.Problem(p.K, p.G, p.C, levels, w=p.w)
    gp.sample(chains_gpu, burn, sweeps, seed, precision=asm.ASM_MIXED)
    st = gp.status()
    assert st["timeouts"] == 0 and st["nonfinite_moves"] == 0
    sg = gp.average()
    op = O.OracleProblem(p.K, p.G, p.C, levels)
    r = op.run(chains_cpu, burn, sweeps, seed=seed, threads=0, chain_offset=chains_gpu)
    so = O.summarize(r["S1"], r["S2"], sweeps, p.w)
    z = np.abs(sg["mean_fbar"] - so["mean_fbar"]) / np.hypot(sg["sem_fbar"], so["sem_fbar"])
    assert np.max(z) < 4.0, float(np.max(z))
