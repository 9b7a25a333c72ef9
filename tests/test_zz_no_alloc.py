"""The allocation-free entry point asm_sample_noalloc, for callers that cannot
allocate device memory themselves (a plug-in whose host application owns all
device memory through its own pool, a loop held to a fixed memory budget).

It must give the same averages as asm_sample + asm_average on the same
problem, chains and seed, on two calls in a row (each call restarts from the
shared static scratch, which still holds the previous call's data), leave the
device's free memory unchanged, and leave a run state that a checkpoint
carries like that of asm_sample.  This file is collected last on purpose, so
that a run stopping at its first failure has run every other test before."""
import numpy as np
import pytest

from paper_1912_01379_gb300 import asm
from paper_1912_01379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-9   # the FP64 tolerance of the parity tests


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_matches_the_allocating_entry_point():
    torch = _cuda()
    p = W.small_problem(20, 60, seed=3, levels=[[0], [0, 25, 40]])
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    out = torch.empty((3, p.N), dtype=torch.float64, device="cuda")
    runs = [(48, 20, 200, 11, asm.ASM_MIXED), (96, 10, 150, 12, asm.ASM_FP64)]
    # references first, and one round of every call the checks below make, so
    # that each kernel -- the library's and torch's -- has been loaded before
    # the free-memory check (a first launch loads its module into device memory)
    refs = []
    for chains, burn, sweeps, seed, prec in runs:
        gp.sample(chains, burn, sweeps, seed, precision=prec)
        refs.append(gp.average())
        out.fill_(np.nan)
        gp.sample_noalloc(chains, burn, sweeps, seed, prec, out[0], out[1], out[2])
        torch.cuda.synchronize()
        _ = [out[k].cpu().numpy() for k in range(3)]
        gp.status()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    # two calls in a row, the second larger than the first and in the other precision
    for (chains, burn, sweeps, seed, prec), ref in zip(runs, refs):
        out.fill_(np.nan)
        gp.sample_noalloc(chains, burn, sweeps, seed, prec, out[0], out[1], out[2])
        torch.cuda.synchronize()
        mean, sem2, m2 = (out[k].cpu().numpy() for k in range(3))
        assert np.allclose(mean, ref["mean_fbar"], rtol=RTOL, atol=0)
        assert np.allclose(np.sqrt(sem2), ref["sem_fbar"], rtol=RTOL, atol=0)
        var = np.maximum(m2 - mean * mean, 0.0)
        assert np.allclose(var / sem2, ref["ess"], rtol=1e-6)
        assert gp.status()["sweeps_done"] == burn + sweeps
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes across the calls"


def test_noalloc_state_checkpoints_like_asm_sample():
    """A checkpoint after the allocation-free call carries the start of the
    kept run, so a restored continuation without burn-in bins its error from
    the same sweeps as a continuation of asm_sample."""
    _cuda()
    p = W.small_problem(20, 60, seed=5, levels=[[0], [0, 30]])
    chains, burn, sweeps, more, seed = 32, 64, 128, 128, 21
    ref = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    ref.sample(chains, burn, sweeps, seed, precision=asm.ASM_MIXED)
    ref.sample(chains, 0, more, seed, precision=asm.ASM_MIXED, cont=True)
    want = ref.mc_error()
    torch = _cuda()
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    out = torch.empty((3, p.N), dtype=torch.float64, device="cuda")
    # a different earlier run on the handle first: its state must not leak into the blob
    gp.sample(chains, 0, 64, seed + 1, precision=asm.ASM_MIXED, refresh_fp64=True)
    gp.sample_noalloc(chains, burn, sweeps, seed, asm.ASM_MIXED, out[0], out[1], out[2])
    blob = gp.checkpoint()
    gp.restore(blob, chains, asm.ASM_MIXED)
    gp.sample(chains, 0, more, seed, precision=asm.ASM_MIXED, cont=True)
    got = gp.mc_error()
    assert np.array_equal(got["bins_per_chain"], want["bins_per_chain"])
    assert np.array_equal(got["sem_fbar"], want["sem_fbar"])


def test_noalloc_rejects_runs_beyond_its_scratch():
    torch = _cuda()
    p = W.small_problem(20, 60, seed=3)
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    chains = 100000
    assert gp.workspace_bytes(chains, asm.ASM_FP64) > asm.ASM_NOALLOC_SCRATCH_BYTES
    out = torch.empty((3, p.N), dtype=torch.float64, device="cuda")
    with pytest.raises(asm.ASMError, match="compiled limit"):
        gp.sample_noalloc(chains, 0, 1, 1, asm.ASM_FP64, out[0], out[1], out[2])
