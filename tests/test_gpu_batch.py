"""Batched solves (one graph launch for many problems of uneven N, n, K and
right-hand-side counts) against the FP64 oracle and the stand-alone plans.

Tolerance: relative L2 1e-10 per problem (the mixed path after its default
two refinement steps).  Also: repeated launches give identical bits, a change
of buffers rewrites the step tables, the bounded dependency waits report
FEM_FFT_ERR_TIMEOUT when a step can never start, and the autotune cache
round-trips.  Plans on algorithm (b) of Section 4 batch as well."""

import json
import os

import numpy as np
import pytest

from oracle import solve as osolve
from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# orders 1..9, N = 1..3, K with factors 2 and 3, several right-hand sides,
# two problems of the same order
SMALL = [
    dict(n=2, K=(16, 16), a=(1.0, 1.0), c=0.0, nrhs=2),
    dict(n=3, K=(12, 8), X=(1.0, 1.5), a=(1.5, 0.7), c=0.3, nrhs=1),
    dict(n=9, K=(16, 32), X=(1.0, 2.0), a=(1.0, 2.5), c=1.0, nrhs=1),
    dict(n=5, K=(48,), a=(2.0,), c=1.0, nrhs=3),
    dict(n=1, K=(8, 8, 8), nrhs=2),
    dict(n=4, K=(8, 6, 12), a=(1.0, 3.0, 0.5), c=0.5, nrhs=1),
    dict(n=7, K=(16, 16), a=(0.6, 1.2), c=2.0, nrhs=1),
    dict(n=2, K=(6, 24, 8), nrhs=2),
    dict(n=8, K=(32,), nrhs=1),
    dict(n=6, K=(12, 16), a=(1.0, 4.0), c=0.1, nrhs=4),
]


def _plans(cases, precision="mixed"):
    from paper_1701_03967_gb300 import Plan
    return [Plan(c["n"], c["K"], c.get("X"), c.get("a"), c.get("c", 0.0), precision, max_nrhs=c["nrhs"])
            for c in cases]


def _rhs(cases, cfg):
    out = []
    for pid, c in enumerate(cases):
        M = tuple(c["n"] * k - 1 for k in c["K"])
        out.append(synth.normal_batch(c["nrhs"], M, cfg, pid))
    return out


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.fixture(scope="module")
def small_batch():
    from paper_1701_03967_gb300 import Batch
    plans = _plans(SMALL)
    batch = Batch(plans, [c["nrhs"] for c in SMALL])
    rhs = _rhs(SMALL, synth.CFG_TEST)
    b = batch.pack(rhs)
    return batch, rhs, b


def test_small_batch_matches_oracle(small_batch):
    batch, rhs, b = small_batch
    u = batch.solve(b, check=True)
    for c, bp, up in zip(SMALL, rhs, batch.views(u)):
        prob = osolve.Problem(c["n"], c["K"], c.get("X"), c.get("a"), c.get("c", 0.0))
        want = osolve.solve(prob, bp)
        rel = _rel(up.cpu().numpy(), want)
        assert rel <= 1e-10, (c, rel)


@pytest.mark.parametrize("nstreams", [1, 3])
def test_stream_mode_matches_oracle_and_graph_mode(small_batch, nstreams):
    """Stream mode (every problem by its own plan on nstreams streams) gives
    the same solutions as the graph launch, to the mixed bar against the
    oracle."""
    batch, rhs, b = small_batch
    ug = batch.solve(b, check=True).clone()
    try:
        batch.set_mode("streams", nstreams)
        us = batch.solve(b)
        torch.cuda.synchronize()
    finally:
        batch.set_mode("graph")
    for c, bp, up, gp in zip(SMALL, rhs, batch.views(us), batch.views(ug)):
        prob = osolve.Problem(c["n"], c["K"], c.get("X"), c.get("a"), c.get("c", 0.0))
        want = osolve.solve(prob, bp)
        assert _rel(up.cpu().numpy(), want) <= 1e-10, c
        assert _rel(up.cpu().numpy(), gp.cpu().numpy()) <= 1e-10, c


def test_replay_is_bitwise_stable_and_buffers_relocate(small_batch):
    batch, rhs, b = small_batch
    u1 = batch.solve(b, check=True).clone()
    u2 = batch.solve(b, check=True)
    assert torch.equal(u1, u2)
    b2 = b.clone()
    out = torch.full_like(b, float("nan"))
    u3 = batch.solve(b2, out=out, check=True)
    assert u3.data_ptr() == out.data_ptr()
    assert torch.equal(u1, u3)
    assert torch.equal(b, b2)     # the right-hand sides are not modified


def test_bounded_wait_reports_timeout_then_recovers(small_batch):
    from paper_1701_03967_gb300 import FemFftError
    batch, rhs, b = small_batch
    ref = batch.solve(b, check=True).clone()
    last = batch.n_steps - 1           # the last step of the last order: it has a predecessor
    batch.set_wait_limit(0.05)
    batch.hold_step(last)
    batch.solve(b)
    code, where = batch.status()
    assert code == -5 and where == last
    with pytest.raises(FemFftError):
        batch.check()
    batch.hold_step(-1)
    batch.set_wait_limit(2.0)
    u = batch.solve(b, check=True)
    assert torch.equal(u, ref)


def test_batch_with_algorithm_b_plans():
    """Plans set to algorithm (b) (every N >= 2 problem but one) share a batch
    with algorithm (a) plans: the three phases of the band solve run as batch
    steps.  Every problem against the oracle at the mixed path's bar."""
    from paper_1701_03967_gb300 import Batch
    plans = _plans(SMALL)
    algos = []
    for i, (c, pl) in enumerate(zip(SMALL, plans)):
        algo = "b" if len(c["K"]) >= 2 and i != 1 else "a"
        if algo == "b":
            pl.set_algorithm("b")
        algos.append(algo)
    assert algos.count("b") >= 6
    batch = Batch(plans, [c["nrhs"] for c in SMALL])
    rhs = _rhs(SMALL, synth.CFG_TEST)
    u = batch.solve(batch.pack(rhs), check=True)
    for c, algo, bp, up in zip(SMALL, algos, rhs, batch.views(u)):
        prob = osolve.Problem(c["n"], c["K"], c.get("X"), c.get("a"), c.get("c", 0.0))
        rel = _rel(up.cpu().numpy(), osolve.solve(prob, bp))
        assert rel <= 1e-10, (c, algo, rel)


def test_tuning_cache_round_trip(tmp_path):
    from paper_1701_03967_gb300 import Batch
    cases = SMALL[:4]
    plans = _plans(cases)
    path = str(tmp_path / "tune.json")
    b1 = Batch(plans, [c["nrhs"] for c in cases], tune=True, tune_cache=path)
    t1 = b1.tuning()
    assert os.path.exists(path)
    doc = json.load(open(path))
    assert doc["gpu"] == torch.cuda.get_device_name() and len(doc["entries"]) >= len(t1)
    for e in t1:
        assert e["W"] >= 1 and e["V"] >= 2 and e["us_per_pencil"] > 0
    b1.close()
    b2 = Batch(plans, [c["nrhs"] for c in cases], tune=False, tune_cache=path)
    key = lambda e: (e["n"], e["K"], e["strided"], e["mode"])
    assert sorted(map(key, t1)) == sorted(map(key, b2.tuning()))
    assert {key(e): (e["W"], e["V"], e["split"]) for e in t1} == \
        {key(e): (e["W"], e["V"], e["split"]) for e in b2.tuning()}
    # the cached schedule solves as well as the tuned one
    rhs = _rhs(cases, synth.CFG_TEST)
    u = b2.solve(b2.pack(rhs), check=True)
    for c, bp, up in zip(cases, rhs, b2.views(u)):
        prob = osolve.Problem(c["n"], c["K"], c.get("X"), c.get("a"), c.get("c", 0.0))
        assert _rel(up.cpu().numpy(), osolve.solve(prob, bp)) <= 1e-10


def test_batch_rejects_fp64_and_repeated_plans():
    from paper_1701_03967_gb300 import Batch, FemFftError
    p64 = _plans(SMALL[:1], "fp64")
    with pytest.raises(FemFftError):
        Batch(p64, [1])
    pm = _plans(SMALL[:1])
    with pytest.raises(FemFftError):
        Batch([pm[0], pm[0]], [1, 1])
    with pytest.raises(FemFftError):
        Batch(pm, [SMALL[0]["nrhs"] + 1])      # more right-hand sides than max_nrhs


@pytest.mark.parametrize("algo", ["a", "b"])
def test_batched_workload_256_problems(algo):
    """The batched workload: 256 seeded problems (N in {2,3}, n in 2..8, K_i in
    {16,32,48,96,128,384,512}, 1-8 right-hand sides), every plan on algorithm
    (a) or every plan on algorithm (b).  Every problem against the stand-alone
    FP64 plan (itself held to 1e-12 of the oracle by the other parity tests)
    and the four smallest against the oracle directly."""
    from paper_1701_03967_gb300 import Batch, Plan
    specs = synth.batched_problems()
    plans = _plans(specs)
    for pl in plans:
        pl.set_algorithm(algo)
    batch = Batch(plans, [s["nrhs"] for s in specs])
    b = torch.empty(batch.total_len, dtype=torch.float64, device="cuda")
    for pid, (s, v) in enumerate(zip(specs, batch.views(b))):
        M = tuple(s["n"] * k - 1 for k in s["K"])
        v.copy_(torch.from_numpy(synth.normal_batch(s["nrhs"], M, synth.CFG_BATCHED, pid)))
    u = batch.solve(b, check=True)
    torch.cuda.synchronize()
    worst = 0.0
    for s, pl, bv, uv in zip(specs, plans, batch.views(b), batch.views(u)):
        p64 = Plan(s["n"], s["K"], s["X"], s["a"], s["c"], "fp64", max_nrhs=s["nrhs"])
        ref = p64.solve(bv)
        p64.close()
        rel = float(torch.linalg.vector_norm(uv - ref) / torch.linalg.vector_norm(ref))
        worst = max(worst, rel)
        assert rel <= 1e-10, (s, rel)
    dofs = [s["nrhs"] * pl.dof for s, pl in zip(specs, plans)]
    for pid in np.argsort(dofs)[:4]:
        s = specs[pid]
        prob = osolve.Problem(s["n"], s["K"], s["X"], s["a"], s["c"])
        want = osolve.solve(prob, batch.views(b)[pid].cpu().numpy())
        assert _rel(batch.views(u)[pid].cpu().numpy(), want) <= 1e-10
    print(f"algorithm ({algo}): 256 problems, {batch.total_len} DOF x rhs, {batch.n_steps} steps, {batch.n_items} items; "
          f"worst rel vs FP64 plan {worst:.3e}")
