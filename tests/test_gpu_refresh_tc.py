"""The residual refresh of the mixed path on the tensor cores (3xTF32 tcgen05
GEMM over all chains, FP64 difference and chi^2) against the same quantity
recomputed in FP64 on the host from the chain states.

The kernel takes the product of the centred states A = f - fref (fref the
problem's mean chain state, summed in FP32) and subtracts it from
r_ref = g~ - K~ fref formed in FP64.  Error model: each of the N products
K~_mn A_n carries the split-precision error of 3xTF32 (the dropped A_lo K_lo
term and the rounding of both low parts to TF32, about 3 2^-22 relative) and
the FP32 accumulation in tensor memory adds about 2^-24 sqrt(N/8) of the running
sum over one part of the k range (the parts are added in FP64), so
|r~_m - r~_m,exact| <= 2^-18 S_m with S_m = sum_n |K~_mn| |f_n - fref_n|
bounds both with room; the test bounds |f_n - fref_n| by |f_n - mean_n| +
1e-3 |mean_n| (fref is an FP32 sum of the chains).  r~ is stored in FP32 (the
precision of the chain state), which adds 2^-24 |r_m|, and chi^2 read back
from the stored r~ then differs from the exact value by at most
2 sum_m |r_m| d_m + sum_m d_m^2.  Without the centring S_m would be
sum_n |K~_mn f_n| ~ |g~_m|, up to 1e5 times larger on accurate data.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_01379_gb300 import asm
from paper_1912_01379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REL = 2.0 ** -18


@pytest.fixture(autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    torch.cuda.synchronize()


def _check_refresh(p, chains, seed):
    op = O.OracleProblem(p.K, p.G, p.C, p.levels)
    dec = op.decomposition()
    gp = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, factors=dec)
    gp.sample(chains, 0, 64, seed, precision=asm.ASM_MIXED)   # the refresh runs after sweep 64
    st = gp.status()
    assert st["tc_refreshes"] >= 1 and st["timeouts"] == 0
    f, chi2 = gp.chain_state()
    r = dec.gt[None, :] - f @ dec.Kt.T                         # exact residual of the stored states
    exact = np.sum(r * r, axis=1)
    # per-component bound, plus the FP32 storage of r~ (chi^2 is read back from it)
    mean = f.mean(axis=0)
    dev = np.abs(f - mean[None, :]) + 1e-3 * np.abs(mean)[None, :]
    d = REL * (dev @ np.abs(dec.Kt).T) + 2.0 ** -24 * np.abs(r)
    bound = 2 * np.sum(np.abs(r) * d, axis=1) + np.sum(d * d, axis=1)
    err = np.abs(chi2 - exact)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and the FP64 CUDA-core refresh of the same states is exact up to the FP32 storage of r~
    gq = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, factors=dec)
    gq.sample(chains, 0, 64, seed, precision=asm.ASM_MIXED, refresh_fp64=True)
    assert gq.status()["tc_refreshes"] == 0
    fq, cq = gq.chain_state()
    rq = dec.gt[None, :] - fq @ dec.Kt.T
    assert np.allclose(cq, np.sum(rq * rq, axis=1), rtol=2.0 ** -22, atol=0)
    return float(np.max(err / np.maximum(exact, 1e-300)))


def test_tc_refresh_blocked_modes_full_size():
    """M = 100 (one M tile), N = 400, 1024 chains: the benchmark's workload."""
    _check_refresh(W.blocked_modes_problem(), 1024, 31)


def test_tc_refresh_two_m_tiles_ragged():
    """M = 400 (two M tiles of 208), N = 250 (ragged last k tile), 300 chains
    (ragged last chain tile)."""
    _check_refresh(W.grid_sweep_problem(250, "uniform", chains=300), 300, 32)


def test_tc_refresh_small_edges():
    """M = 12 (MMA N = 16), N = 40 (two k tiles, the second ragged), 5 chains."""
    _check_refresh(W.small_problem(12, 40, seed=33, levels=[[0], [0, 17]]), 5, 33)


def test_tc_refresh_largest_grid_relative_chi2():
    """The largest grid of the grid-size sweep (N_tau = 400, N_omega = 2000, the
    accurate data of noise 1e-5): besides the per-component bound, chi^2 of the
    tensor-core refresh within 1e-6 relative of its FP64 value.  3xTF32 with both
    parts rounded to TF32 keeps about 3 2^-22 of every product K~_mn A_n, and the
    k range in 16 parts added in FP64 keeps the FP32 accumulation short;
    measured: 5.6e-7.  One part with the low parts left to the MMA's truncation
    gave 1.3e-6, the uncentred product 1e-4."""
    p = W.grid_sweep_problem(2000, "uniform", chains=512)
    err = _check_refresh(p, 512, 34)
    assert err <= 1e-6, err
