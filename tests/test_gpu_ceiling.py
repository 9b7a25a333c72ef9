"""The measured arithmetic ceilings of the chain kernel's instruction mix
(asm_measure_ceiling), the denominators of its roofline: each rate must be
physically possible for the GPU it ran on (at most one warp instruction per
cycle per SM sub-partition, i.e. 128 lanes per SM per cycle at the clock seen
during the launch), and the five-instruction pass cannot run faster than one
of its instructions alone."""
import pytest

from paper_1912_01379_gb300 import asm

pytestmark = pytest.mark.gpu


def _sms():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_ceilings_are_physical():
    sms = _sms()
    got = {k: asm.measure_ceiling(k, 20.0) for k in asm.CEILING_KINDS}
    for k, r in got.items():
        assert r["rate"] > 0 and r["ms"] > 5.0, k
        assert 500.0 < r["sm_mhz"] < 2300.0, (k, r["sm_mhz"])
        per_sm_clk = r["rate"] / (sms * r["sm_mhz"] * 1e6)
        # lanes (elements or instructions) per SM per cycle: at most 4 x 32
        assert per_sm_clk <= 128 * 1.05, (k, per_sm_clk)
    # the pass issues five instructions per element: at most a fifth of the issue rate
    assert got["pass_f32"]["rate"] / (sms * got["pass_f32"]["sm_mhz"] * 1e6) <= 128 / 5 * 1.05
    assert got["pass_f32"]["rate"] < got["ffma"]["rate"]
    assert got["pass_f64"]["rate"] < got["dfma"]["rate"]
    # the FP32 FMA reaches a useful fraction of the issue rate (the kernel is not folded away)
    assert got["ffma"]["rate"] / (sms * got["ffma"]["sm_mhz"] * 1e6) > 32


def test_ceiling_rejects_bad_arguments():
    _sms()
    L = asm.load()
    import ctypes as ct
    x = ct.c_double(0)
    assert L.asm_measure_ceiling(99, 10.0, ct.byref(x), None, None) == -7
    assert L.asm_measure_ceiling(0, 0.0, ct.byref(x), None, None) == -7
    assert L.asm_measure_ceiling(0, 10.0, None, None, None) == -7
