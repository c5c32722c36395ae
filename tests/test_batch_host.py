"""Host logic of the batched solver (no GPU): the level order of the work
list.  Every item's dependency (the previous step of the same problem) must
carry a smaller ticket, which is what makes the ticket-ordered schedule
deadlock-free; the order must contain every step exactly once."""

import random

import pytest

pytest.importorskip("ctypes")


def _order(nsteps, work=None):
    from paper_1701_03967_gb300 import batch_order
    return batch_order(nsteps, work)


@pytest.mark.parametrize("seed", range(5))
def test_level_order_puts_dependencies_first(seed):
    g = random.Random(seed)
    nprob = g.randint(1, 60)
    nsteps = [g.randint(0, 27) for _ in range(nprob)]
    work = [g.random() for _ in range(nprob)]
    order = _order(nsteps, work)
    assert sorted(order) == sorted((p, s) for p in range(nprob) for s in range(nsteps[p]))
    pos = {ps: i for i, ps in enumerate(order)}
    for (p, s), i in pos.items():
        if s > 0:
            assert pos[(p, s - 1)] < i
    # level order: steps never decrease along the list
    levels = [s for _, s in order]
    assert levels == sorted(levels)
    # within a level, problems by decreasing work
    for lvl in set(levels):
        probs = [p for p, s in order if s == lvl]
        assert [work[p] for p in probs] == sorted((work[p] for p in probs), reverse=True)


def test_level_order_edge_cases():
    assert _order([]) == []
    assert _order([0, 0]) == []
    assert _order([1]) == [(0, 0)]
    assert _order([2, 1]) == [(0, 0), (1, 0), (0, 1)]


def test_level_order_rejects_negative_counts():
    from paper_1701_03967_gb300 import FemFftError
    with pytest.raises(FemFftError):
        _order([1, -1])
