"""Grid-size sweep workload (N_tau = 400, beta = 50, 16 blocks, correlated noise
1e-5 exp(-|dtau|)): the mixed path -- FP32 chain state, FP64 accumulators and
the 3xTF32 tensor-core residual refresh over two M_tau tiles -- against the
FP64 oracle at N_omega = 250 on the uniform and the Gaussian-density grid.

Both runs share the level schedule (same seed, problem id 0) on disjoint chain
ids; <fbar> must agree within 4 combined standard errors at every grid point
(the library's binned error, asm_mc_error, and the spread of 128 independent
oracle chain means, so that each standard error is itself estimated to a few
per cent).  The relative L2 error of <A> is checked against the same combined
error.  The largest grid, N_omega = 2000, is compared the same way, with the
4-sigma rule applied per point (at most the two points that chance allows
beyond 4 in 2000, none beyond 5) and the distribution of the z-scores checked
as well (mean square near 1, no more than 1 % beyond 3).
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


def _compare(n_omega, density, chains_gpu, chains_cpu, burn, sweeps, seed, oracle_factors=False):
    p = W.grid_sweep_problem(n_omega, density, chains=chains_gpu)
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, factors=op.decomposition() if oracle_factors else None)
    gp.sample(chains_gpu, burn, sweeps, seed, precision=asm.ASM_MIXED)
    st = gp.status()
    assert st["tc_refreshes"] >= (burn + sweeps) // 64 and st["timeouts"] == 0 and st["nonfinite_moves"] == 0
    sg = gp.average()
    sem_gpu = gp.mc_error()["sem_fbar"]
    r = op.run(chains_cpu, burn, sweeps, seed=seed, threads=0, chain_offset=chains_gpu)
    so = O.summarize(r["S1"], r["S2"], sweeps, p.w)
    se = np.hypot(sem_gpu, so["sem_fbar"])
    z = np.abs(sg["mean_fbar"] - so["mean_fbar"]) / se
    l2 = np.linalg.norm(sg["mean_A"] - so["mean_A"]) / np.linalg.norm(so["mean_A"])
    l2_se = np.linalg.norm(se / p.w) / np.linalg.norm(so["mean_A"])
    return z, l2, l2_se


@pytest.mark.parametrize("density", ["uniform", "gaussian"])
def test_grid_sweep_mixed_against_oracle(density):
    # enough chains on both sides that the standard errors themselves are well estimated
    z, l2, l2_se = _compare(250, density, 1024, 128, 200, 1000, 55)
    assert np.max(z) < Z_MAX, float(np.max(z))
    assert l2 < 3.0 * l2_se, (l2, l2_se)


def test_grid_sweep_largest_grid_against_oracle():
    """N_omega = 2000 (the largest grid of the sweep): 1024 GPU chains against
    128 oracle chains, 200 burn-in + 300 kept sweeps each, the library given
    the oracle's factors.  At this size 200 sweeps do not reach equilibrium:
    runs in two mode bases (the library's SVD and the oracle's) are two Markov
    chains with the same stationary law but different transients, which the
    standard errors do not measure (runs on different level schedules differ by
    tens of standard errors here); in the oracle's basis and on its level
    schedule both sides run the same chain."""
    z, l2, l2_se = _compare(2000, "uniform", 1024, 128, 200, 300, 56, oracle_factors=True)
    # 4 standard errors per point over 2000 points: independent normal z-scores exceed 4 at
    # 0.13 points on average (a max-over-the-grid test would fail a correct sampler about one
    # run in eight), so at most two points may, and none may exceed 5 (2000 points x P(|z| > 5)
    # = 1e-3); the 128 oracle chain means are skewed where the spectrum peaks, which fattens
    # the tails a little
    assert np.sum(z > Z_MAX) <= 2, (int(np.sum(z > Z_MAX)), float(np.max(z)))
    assert np.max(z) < 5.0, float(np.max(z))
    assert 0.75 < np.mean(z ** 2) < 1.33, float(np.mean(z ** 2))
    assert np.mean(z > 3.0) <= 0.01, float(np.mean(z > 3.0))
    assert l2 < 3.0 * l2_se, (l2, l2_se)
