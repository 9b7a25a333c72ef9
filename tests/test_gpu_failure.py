"""Failure detection on the GPU without a fault: with ASM_FLAG_TEST_STALL the
sweep kernel's record producer withholds every move record, so the consumer
warps' bounded mbarrier waits run out (a barrier that nothing completes); the
kernel counts the timeouts and returns with nothing in flight, the result calls
report ASM_ERR_TIMEOUT, and the same context then runs a normal problem."""
import time

import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", [asm.ASM_FP64, asm.ASM_MIXED])
def test_stalled_records_time_out_and_the_context_survives(prec):
    import torch
    p = W.small_problem(20, 60, seed=3, levels=[[0], [0, 25, 40]])
    bad = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, flags=asm.ASM_FLAG_TEST_STALL)
    t0 = time.time()
    bad.sample(8, 0, 1, 1, precision=prec)          # asynchronous: returns before the waits run out
    with pytest.raises(asm.ASMError) as err:
        bad.average()
    assert err.value.code == asm.ASM_ERR_TIMEOUT
    assert bad.status()["timeouts"] > 0
    assert time.time() - t0 < 60.0
    torch.cuda.synchronize()                         # no error is pending on the context
    good = asm.Problem(p.K, p.G, p.C, p.levels, w=p.w)
    good.sample(8, 0, 16, 1, precision=prec)
    r = good.average()
    assert good.status()["timeouts"] == 0 and np.all(np.isfinite(r["mean_fbar"]))


def test_unknown_flags_rejected():
    p = W.small_problem(20, 60, seed=3)
    with pytest.raises(asm.ASMError):
        asm.Problem(p.K, p.G, p.C, p.levels, w=p.w, flags=1)
