"""Binned Monte Carlo error (asm_mc_error) through the C ABI.

* Cascade identity: with 2^j complete bins per chain, level j has one bin per
  chain, whose mean is the chain's mean, so its error equals the spread of the
  chain means (asm_average's error) to rounding; a wrong pairing or weighting
  in the merge fails it.
* Bins count only whole 64-sweep blocks after the burn-in, aligned to the
  absolute sweep index, and continue across continued runs.
* Against the oracle's binning of traced chains (plain numpy doubling
  analysis, pinned on AR(1) series): the integrated autocorrelation time
  tau = n sigma^2 / (2 var) at the plateau levels agrees within the statistical
  noise of the two estimates (median over the grid).
* A batch problem's error equals the single handle's with the same problem id.
"""
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


def _p():
    return W.small_problem(20, 60, seed=3, levels=[[0], [0, 25, 40]])


@pytest.mark.parametrize("prec", [asm.ASM_FP64, asm.ASM_MIXED])
def test_single_bin_level_equals_chain_spread(prec):
    p = _p()
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    gp.sample(48, 0, 64 * 16, 7, precision=prec)
    e = gp.mc_error()
    assert list(e["bins_per_chain"]) == [16, 8, 4, 2, 1, 0, 0, 0]
    sem_chains = gp.average()["sem_fbar"]
    assert np.allclose(e["sigma2_levels"][4], sem_chains ** 2, rtol=1e-10, atol=0)
    assert np.all(np.isnan(e["sigma2_levels"][5:]))
    # the reported error is the largest level with two or more bins per chain, or the chain spread
    want = np.fmax(np.nanmax(e["sigma2_levels"][:4], axis=0), sem_chains ** 2)
    assert np.allclose(e["sem_fbar"] ** 2, want, rtol=1e-12)
    assert np.all(e["ess"] <= gp.average()["ess"] * (1 + 1e-12))


def test_bins_follow_burn_in_and_continuation():
    p = _p()
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    gp.sample(8, 100, 412, 3, precision=asm.ASM_MIXED)          # sweeps 0..511, kept from 100
    assert list(gp.mc_error()["bins_per_chain"])[:3] == [6, 3, 1]   # bins from 128 on
    gp.sample(8, 0, 128, 3, precision=asm.ASM_MIXED, cont=True)   # sweeps 512..639
    assert gp.mc_error()["bins_per_chain"][0] == 8
    gp.sample(8, 0, 30, 3, precision=asm.ASM_MIXED, cont=True)    # 640..669: no boundary
    assert gp.mc_error()["bins_per_chain"][0] == 8
    gp.sample(8, 0, 34, 3, precision=asm.ASM_MIXED, cont=True)    # ..703: bin [640, 704) closes
    assert gp.mc_error()["bins_per_chain"][0] == 9


def test_tau_matches_oracle_binning():
    p = _p()
    chains_gpu, chains_cpu, sweeps, seed = 512, 64, 4096, 21
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    gp.sample(chains_gpu, 0, sweeps, seed, precision=asm.ASM_FP64)
    e = gp.mc_error()
    var = gp.average()["ess"] * gp.average()["sem_fbar"] ** 2            # posterior variance
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    r = op.run(chains_cpu, 0, sweeps, seed=seed, trace_chains=chains_cpu, chain_offset=chains_gpu)
    so = O.binning(r["trace"], 0, 0)
    s = O.summarize(r["S1"], r["S2"], sweeps)
    for k in (2, 3):   # bins of 256 and 512 sweeps: 16 and 8 per chain
        tau_gpu = e["sigma2_levels"][k] * chains_gpu * sweeps / (2 * var)
        tau_cpu = so[0][k] * chains_cpu * sweeps / (2 * s["var_fbar"])
        ratio = np.median(tau_gpu / tau_cpu)
        assert 0.75 < ratio < 1.33, (k, ratio)


def test_batch_problem_error_equals_single_handle():
    probs = [_p(), W.small_problem(30, 90, seed=4, levels=[[0], [0, 45]])]
    b = asm.Batch([dict(K=q.K, G=q.G, C=q.C, levels=q.levels, w=q.w) for q in probs])
    b.sample(16, 64, 256, 9, precision=asm.ASM_MIXED)
    one = asm.Problem(probs[1].K, probs[1].G, probs[1].C, probs[1].levels, w=probs[1].w)
    one.set_stream_ids(1, 0)
    one.sample(16, 64, 256, 9, precision=asm.ASM_MIXED)
    eb, eo = b.mc_error(1), one.mc_error()
    assert np.array_equal(eb["sem_fbar"], eo["sem_fbar"]) and np.array_equal(eb["ess"], eo["ess"])


def test_new_burn_in_inside_an_open_block():
    """A continuation that starts a new burn-in inside a 64-sweep block: kept
    sweeps 0..9, then 54 burn-in sweeps and 64 kept ones, so the one complete bin
    is sweeps 64..127.  The mixed path keeps the open block's sums in FP32 until
    the block closes; they must reach the FP64 sums before the bin starts, or
    the bin would also hold sweeps 0..9 and its mean come out (74/64) too large.
    The level-0 bin variance over the chain-mean variance is then the same in the
    mixed and the FP64 path (1.08 here for both)."""
    p = W.small_problem(16, 40, seed=10, levels=[[0], [0, 13, 29]])
    ratio = {}
    for prec in (asm.ASM_MIXED, asm.ASM_FP64):
        gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
        gp.sample(512, 0, 10, 5, precision=prec)
        gp.sample(512, 54, 64, 5, precision=prec, cont=True)
        e, a = gp.mc_error(), gp.average()
        assert e["bins_per_chain"][0] == 1 and e["bins_per_chain"][1] == 0
        assert np.all(np.isfinite(a["mean_A"]))
        ratio[prec] = float(np.nanmean(e["sigma2_levels"][0] / a["sem_fbar"] ** 2))
    assert abs(ratio[asm.ASM_MIXED] - ratio[asm.ASM_FP64]) < 0.1, ratio
