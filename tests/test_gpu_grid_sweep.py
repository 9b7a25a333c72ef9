"""Grid-size sweep workload (N_tau = 400, beta = 50, 16 blocks, correlated noise
1e-5 exp(-|dtau|)): the mixed path -- FP32 chain state, FP64 accumulators and
the 3xTF32 tensor-core residual refresh over two M_tau tiles -- against the
FP64 oracle at N_omega = 250 on the uniform and the Gaussian-density grid.

Both runs share the level schedule (same seed, problem id 0) on disjoint chain
ids; <fbar> must agree within 4 combined standard errors at every grid point
(1024 GPU and 128 oracle chains, so that the spread of the chain means
estimates each standard error to a few per cent).
The relative L2 error of <A> is checked against the same combined error.
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


@pytest.mark.parametrize("density", ["uniform", "gaussian"])
def test_grid_sweep_mixed_against_oracle(density):
    p = W.grid_sweep_problem(250, density, chains=1024)
    # enough chains on both sides that the standard errors themselves are well estimated
    chains_gpu, chains_cpu, burn, sweeps, seed = 1024, 128, 200, 1000, 55
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    gp.sample(chains_gpu, burn, sweeps, seed, precision=asm.ASM_MIXED)
    st = gp.status()
    assert st["tc_refreshes"] >= (burn + sweeps) // 64 and st["timeouts"] == 0 and st["nonfinite_moves"] == 0
    sg = gp.average()
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    r = op.run(chains_cpu, burn, sweeps, seed=seed, threads=0, chain_offset=chains_gpu)
    so = O.summarize(r["S1"], r["S2"], sweeps, p.w)
    se = np.hypot(sg["sem_fbar"], so["sem_fbar"])
    z = np.abs(sg["mean_fbar"] - so["mean_fbar"]) / se
    assert np.max(z) < Z_MAX, float(np.max(z))
    l2 = np.linalg.norm(sg["mean_A"] - so["mean_A"]) / np.linalg.norm(so["mean_A"])
    l2_se = np.linalg.norm(se / p.w) / np.linalg.norm(so["mean_A"])
    assert l2 < 3.0 * l2_se, (l2, l2_se)
