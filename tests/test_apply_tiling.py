"""Host logic of the apply launches (no GPU): the block tiling returned by
fem_fft_apply_tiling, run through the thread -> (position, element) mapping
the apply kernels use, must give every (position, element) pair of the axis
to exactly one thread, and every thread's element slots must fit the block
(256 threads, TW positions x 256 / TW elements).

Mapping of a block bx (the kernels' decode): element tile et = bx mod
etiles, then position tile and outer index.  Normal tiling: positions are
the `inner` positions after the axis, thread t -> (t mod TW, t div TW).
Lines mode (inner == 1, TW > 1): positions are the `outer` lines, thread t
-> (t div TE, t mod TE), one element tile row per line."""

import ctypes

import pytest

NT = 256


def _tiling(inner, outer, K):
    from paper_1701_03967_gb300 import _lib
    tw = ctypes.c_int()
    blocks = ctypes.c_int64()
    rc = _lib.lib().fem_fft_apply_tiling(inner, outer, K, ctypes.byref(tw), ctypes.byref(blocks))
    assert rc == 0
    return tw.value, blocks.value


def _cover(inner, outer, K):
    TW, B = _tiling(inner, outer, K)
    assert 1 <= TW <= 32 and NT % TW == 0
    TE = NT // TW
    lines = inner == 1 and TW > 1
    npos = outer if lines else inner
    etiles = (K + TE - 1) // TE
    wtiles = (npos + TW - 1) // TW
    assert B == (1 if lines else outer) * wtiles * etiles
    seen = {}
    for bx0 in range(B):
        et, bx = bx0 % etiles, bx0 // etiles
        wt, o = bx % wtiles, (0 if lines else bx // wtiles)
        for t in range(NT):
            tw, te = (t // TE, t % TE) if lines else (t % TW, t // TW)
            w, e = wt * TW + tw, et * TE + te
            if w < npos and e < K:
                key = (o, w, e)
                seen[key] = seen.get(key, 0) + 1
    want = (1 if lines else outer) * npos * K
    assert len(seen) == want and all(v == 1 for v in seen.values())
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


def test_rejects_non_positive_sizes():
    from paper_1701_03967_gb300 import _lib
    for args in [(0, 1, 8), (1, 0, 8), (1, 1, 0), (-1, 1, 8)]:
        assert _lib.lib().fem_fft_apply_tiling(*args, None, None) != 0
