"""Status reporting of fem_fft_solve through the C ABI: non-finite right-hand
sides (flagged by the first pass without a synchronisation, reported by
fem_fft_last_info), the residual guard of rtol > 0 (FEM_FFT_ERR_NOT_CONVERGED
when the final iterate misses rtol), and that a clean solve clears both."""

import numpy as np
import pytest

from oracle import solve as osolve
from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NONFINITE, NOT_CONVERGED = -7, -6

# register-radix passes (K a power of two in [16, 1024]) and the shared-memory
# Stockham passes (K = 12, 48), float32 and float64
CASES = [dict(n=3, K=(16, 32), c=0.5), dict(n=2, K=(12, 48), c=0.0), dict(n=4, K=(8, 16, 16), c=1.0)]


def _ids(c):
    return f"n{c['n']}_K{'x'.join(map(str, c['K']))}"


@pytest.mark.parametrize("case", CASES, ids=_ids)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_right_hand_side_is_reported(case, precision, bad):
    from paper_1701_03967_gb300 import FemFftError, Plan
    plan = Plan(case["n"], case["K"], None, None, case["c"], precision, max_nrhs=2)
    b = synth.normal_batch(2, plan.M, synth.CFG_TEST, 400)
    b[1].reshape(-1)[b[1].size // 3] = bad          # one value of the second right-hand side
    bt = torch.from_numpy(b).cuda()
    u = plan.solve(bt)                               # asynchronous: no status yet
    with pytest.raises(FemFftError) as ei:
        plan.last_info()
    assert ei.value.code == NONFINITE
    # the same plan with a finite right-hand side: the flag is cleared
    b[1].reshape(-1)[b[1].size // 3] = 0.0
    bt = torch.from_numpy(b).cuda()
    u = plan.solve(bt)
    plan.last_info()
    prob = osolve.Problem(case["n"], case["K"], None, None, case["c"])
    want = osolve.solve(prob, b)
    tol = 1e-12 if precision == "fp64" else 1e-10
    assert np.linalg.norm(u.cpu().numpy() - want) / np.linalg.norm(want) <= tol
    # with rtol > 0 the mixed solve synchronises and returns the status itself
    if precision == "mixed":
        plan.set_refinement(1e-9, 4)
        b[0].reshape(-1)[7] = bad
        with pytest.raises(FemFftError) as ei:
            plan.solve(torch.from_numpy(b).cuda())
        assert ei.value.code == NONFINITE
    plan.close()


@pytest.mark.parametrize("case", CASES[:2], ids=_ids)
def test_residual_guard(case):
    """rtol unreachable in the steps allowed -> FEM_FFT_ERR_NOT_CONVERGED with
    the last iterate in u; a reachable rtol stops early and solves to the
    mixed bar."""
    from paper_1701_03967_gb300 import FemFftError, Plan
    prob = osolve.Problem(case["n"], case["K"], None, None, case["c"])
    b = synth.normal_field(prob.M, synth.CFG_TEST, 401)
    want = osolve.solve(prob, b)
    bt = torch.from_numpy(b).cuda()
    plan = Plan(case["n"], case["K"], None, None, case["c"], "mixed")
    plan.set_refinement(1e-30, 1)
    u = torch.empty_like(bt)
    with pytest.raises(FemFftError) as ei:
        plan.solve(bt, out=u)
    assert ei.value.code == NOT_CONVERGED
    with pytest.raises(FemFftError):
        plan.last_info()
    got = u.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-6   # one refinement step taken
    plan.set_refinement(1e-9, 6)
    plan.solve(bt, out=u)
    iters, rel = plan.last_info()
    assert 1 <= iters <= 6 and 0.0 <= rel <= 1e-9
    assert np.linalg.norm(u.cpu().numpy() - want) / np.linalg.norm(want) <= 1e-10
    plan.close()
