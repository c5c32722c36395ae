"""Host logic of the apply launches (no GPU): the block tiling returned by
fem_fft_apply_tiling and the thread map of every block returned by
fem_fft_apply_block_map -- computed by the decode the apply kernels
themselves run -- must give every (outer index, position, element) triple
of the axis to exactly one thread of one block, with the thread's element
slot inside the block (256 threads, TW positions x 256 / TW elements)."""

import ctypes

import numpy as np
import pytest

NT = 256


def _tiling(inner, outer, K):
    from paper_1701_03967_gb300 import _lib
    tw = ctypes.c_int()
    blocks = ctypes.c_int64()
    rc = _lib.lib().fem_fft_apply_tiling(inner, outer, K, ctypes.byref(tw), ctypes.byref(blocks))
    assert rc == 0
    return tw.value, blocks.value


def _block_map(inner, outer, K, bx):
    from paper_1701_03967_gb300 import _lib
    o = np.empty(NT, np.int64)
    w = np.empty(NT, np.int64)
    e = np.empty(NT, np.int64)
    p = ctypes.POINTER(ctypes.c_int64)
    rc = _lib.lib().fem_fft_apply_block_map(inner, outer, K, bx, o.ctypes.data_as(p), w.ctypes.data_as(p),
                                            e.ctypes.data_as(p))
    assert rc == 0
    return o, w, e


def _cover(inner, outer, K):
    TW, B = _tiling(inner, outer, K)
    assert 1 <= TW <= 32 and NT % TW == 0
    lines = inner == 1 and TW > 1
    npos = outer if lines else inner
    nouter = 1 if lines else outer
    seen = np.zeros((nouter, npos, K), np.int32)
    for bx in range(B):
        o, w, e = _block_map(inner, outer, K, bx)
        has = e >= 0
        assert np.all((o[has] >= 0) & (o[has] < nouter))
        assert np.all((w[has] >= 0) & (w[has] < npos))
        assert np.all((e[has] >= 0) & (e[has] < K))
        assert np.all((o[~has] == -1) & (w[~has] == -1))
        np.add.at(seen, (o[has], w[has], e[has]), 1)
    assert np.all(seen == 1)
    return TW, lines


@pytest.mark.parametrize("inner,outer,K", [(1, 1, 64), (1, 7, 64), (1, 100, 16), (1, 3, 2), (1, 33, 512),
                                           (1, 5, 1024), (577, 1, 64), (9217, 2, 4), (3, 5, 6), (40, 3, 300)])
def test_every_element_has_exactly_one_thread(inner, outer, K):
    TW, lines = _cover(inner, outer, K)
    if inner == 1 and K <= NT // 2 and outer >= 2:
        assert lines      # short lines share blocks
    if inner == 1 and K >= NT:
        assert TW == 1    # long lines fill a block on their own


def test_lines_mode_keeps_threads_busy():
    """On the contiguous axis with short lines (the 3D K = 64 and batched K =
    16 cases) most element slots of a block hold an element."""
    for K, outer in [(64, 577 * 577), (16, 1000), (48, 4096)]:
        TW, _ = _tiling(1, outer, K)
        assert K / (NT // TW) >= 0.5


def test_rejects_non_positive_sizes_and_blocks_outside_the_launch():
    from paper_1701_03967_gb300 import _lib
    for args in [(0, 1, 8), (1, 0, 8), (1, 1, 0), (-1, 1, 8)]:
        assert _lib.lib().fem_fft_apply_tiling(*args, None, None) != 0
    _, B = _tiling(3, 5, 6)
    o = np.empty(NT, np.int64)
    p = o.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    for bx in (-1, B):
        assert _lib.lib().fem_fft_apply_block_map(3, 5, 6, bx, p, p, p) != 0
    assert _lib.lib().fem_fft_apply_block_map(3, 5, 6, 0, None, p, p) != 0
