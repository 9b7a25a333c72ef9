"""The allocation-free entry point asm_sample_noalloc, for callers that cannot
allocate device memory (stream capture, a host framework's own memory pool, a
fixed budget): it must give the same averages as asm_sample + asm_average on
the same problem, chains and seed, on two calls in a row (each call restarts
from the shared static scratch, which still holds the previous call's data).
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1912_01379_gb300 import asm
from paper_1912_01379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-9   # the FP64 tolerance of the parity tests


def test_noalloc_matches_the_allocating_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = W.small_problem(20, 60, seed=3, levels=[[0], [0, 25, 40]])
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    out = torch.empty((3, p.N), dtype=torch.float64, device="cuda")
    # two calls in a row, the second larger than the first and in the other precision
    for chains, burn, sweeps, seed, prec in [(48, 20, 200, 11, asm.ASM_MIXED), (96, 10, 150, 12, asm.ASM_FP64)]:
        gp.sample(chains, burn, sweeps, seed, precision=prec)
        ref = gp.average()
        out.fill_(np.nan)
        gp.sample_noalloc(chains, burn, sweeps, seed, prec, out[0], out[1], out[2])
        torch.cuda.synchronize()
        mean, sem2, m2 = (out[k].cpu().numpy() for k in range(3))
        assert np.allclose(mean, ref["mean_fbar"], rtol=RTOL, atol=0)
        assert np.allclose(np.sqrt(sem2), ref["sem_fbar"], rtol=RTOL, atol=0)
        var = np.maximum(m2 - mean * mean, 0.0)
        assert np.allclose(var / sem2, ref["ess"], rtol=1e-6)
        assert gp.status()["sweeps_done"] == burn + sweeps


def test_noalloc_rejects_runs_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = W.small_problem(20, 60, seed=3)
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    chains = 100000
    assert gp.workspace_bytes(chains, asm.ASM_FP64) > asm.ASM_NOALLOC_SCRATCH_BYTES
    out = torch.empty((3, p.N), dtype=torch.float64, device="cuda")
    with pytest.raises(asm.ASMError, match="compiled limit"):
        gp.sample_noalloc(chains, 0, 1, 1, asm.ASM_FP64, out[0], out[1], out[2])
