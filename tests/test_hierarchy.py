"""The partition hierarchy of blocked modes sampling (asm_partition_hierarchy,
host code of the library; Sec. IV.C and Fig. blocks of the paper): from the
whole grid (modes sampling) down to one grid point per block (components
sampling), blocks halved from level to level, every other level shifted by half
a block width so that not every level has a boundary at the centre.

Checked against closed forms on power-of-two grids (exact block widths N/2^l,
half-width edge blocks on shifted levels) and against invariants for any N."""
import numpy as np
import pytest

from paper_1912_01379_gb300 import asm


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 9])
def test_power_of_two_grids_closed_form(k):
    N = 2 ** k
    lv = asm.partition_hierarchy(N)
    assert len(lv) == k + 1
    assert list(lv[0]) == [0] and list(lv[-1]) == list(range(N))
    for l in range(1, k):
        w = N >> l
        if l % 2 == 1:   # unshifted: 2^l blocks of width w
            assert list(lv[l]) == list(range(0, N, w)), l
        else:            # shifted by w/2: half blocks at both edges, full ones between
            assert list(lv[l]) == [0] + list(range(w // 2, N, w)), l


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 25, 50, 99, 100, 400, 1000, 2000])
def test_invariants_any_grid(N):
    lv = asm.partition_hierarchy(N)
    assert list(lv[0]) == [0]
    if N > 1:
        assert list(lv[-1]) == list(range(N))
    depth = int(np.ceil(np.log2(N))) if N > 1 else 0
    assert len(lv) <= depth + 1
    sizes = [len(l) for l in lv]
    assert sizes == sorted(set(sizes))            # strictly more blocks at every level
    for l, starts in enumerate(lv):
        starts = np.asarray(starts)
        assert starts[0] == 0 and np.all(np.diff(starts) > 0) and starts[-1] < N
        if 0 < l < len(lv) - 1:
            w = N / 2 ** l
            widths = np.diff(np.append(starts, N))
            inner = widths[1:-1] if l % 2 == 0 else widths
            assert np.all(np.abs(inner - w) <= 1.0), (l, w, widths)


@pytest.mark.parametrize("N", [16, 100, 400, 1000])
def test_shifted_levels_avoid_the_centre(N):
    lv = asm.partition_hierarchy(N)
    for l in range(1, len(lv) - 1):
        centre_is_boundary = (N // 2) in set(int(b) for b in lv[l])
        if l % 2 == 1:
            assert centre_is_boundary
        elif N / 2 ** l >= 2:
            assert not centre_is_boundary, l


def test_rejects_bad_arguments():
    L = asm.load()
    import ctypes as ct
    nl, tot = ct.c_int(0), ct.c_int(0)
    nb = (ct.c_int * 64)()
    assert L.asm_partition_hierarchy(0, ct.byref(nl), nb, None, ct.byref(tot)) == -7
    assert L.asm_partition_hierarchy(8, None, nb, None, ct.byref(tot)) == -7
