"""Differentiation (torch.autograd through the C-ABI solver) against the FP64
oracle's gradient and FP64 central finite differences.

Loss = ||u - u_target||^2 with u = L(a, c)^{-1} f; gradients with respect to
f, a and c.  The adjoint reuses the fast solve (L is symmetric) and the
coefficient gradients are float64 matrix-free bilinear forms."""

import numpy as np
import pytest

from oracle import solve as osolve
from paper_1701_03967_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grads(plan, f, ut, a, c):
    from paper_1701_03967_gb300 import fem_solve
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    at = torch.tensor(a, dtype=torch.float64, requires_grad=True)
    ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    u = fem_solve(plan, ft, at, ct)
    loss = torch.sum((u - torch.from_numpy(ut).cuda()) ** 2)
    loss.backward()
    return float(loss.detach()), ft.grad.cpu().numpy(), at.grad.numpy(), float(ct.grad)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradients_small_vs_oracle_and_finite_differences(precision):
    from paper_1701_03967_gb300 import Plan
    n, K, X = 2, (8, 8, 8), (1.0, 1.0, 1.0)
    a, c = (1.0, 1.3, 0.8), 0.4
    prob = osolve.Problem(n, K, X, a, c)
    f = synth.normal_field(prob.M, synth.CFG_GRAD, 1, 0)
    ut = synth.normal_field(prob.M, synth.CFG_GRAD, 1, 1)
    plan = Plan(n, K, X, a, c, precision=precision)
    loss, gf, ga, gc = _grads(plan, f, ut, a, c)
    u = osolve.solve(prob, f)
    of, oa, oc = osolve.grad(prob, f, 2 * (u - ut))
    assert np.linalg.norm(gf - of) / np.linalg.norm(of) <= 1e-10
    np.testing.assert_allclose(ga, oa, rtol=1e-9)
    np.testing.assert_allclose(gc, oc, rtol=1e-9)
    # FP64 central differences (step 1e-6) of the loss evaluated by the GPU
    # float64 solve
    p64 = Plan(n, K, X, a, c, precision="fp64")
    utg = torch.from_numpy(ut).cuda()

    def L(aa, cc, ff):
        p64.set_coefficients(aa, cc)
        return float(torch.sum((p64.solve(ff) - utg) ** 2))

    fg = torch.from_numpy(f).cuda()
    h = 1e-6
    for i in range(3):
        ap, am = list(a), list(a)
        ap[i] += h
        am[i] -= h
        fd = (L(ap, c, fg) - L(am, c, fg)) / (2 * h)
        assert abs(fd - ga[i]) <= 1e-6 * max(1.0, abs(fd))
    fd = (L(a, c + h, fg) - L(a, c - h, fg)) / (2 * h)
    assert abs(fd - gc) <= 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0, 0), (7, 3, 11), (14, 14, 14)]:
        e = torch.zeros_like(fg)
        e[idx] = h
        fd = (L(a, c, fg + e) - L(a, c, fg - e)) / (2 * h)
        assert abs(fd - gf[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_gradients_fullsize_3d_n5_K64_mixed():
    """3D n=5, K=64^3 (319^3 = 32.5 M DOF), a = (1,1,1), c = 0, mixed precision."""
    from paper_1701_03967_gb300 import Plan
    n, K, X, a, c = 5, (64, 64, 64), (1.0, 1.0, 1.0), (1.0, 1.0, 1.0), 0.0
    prob = osolve.Problem(n, K, X, a, c)
    f = synth.normal_field(prob.M, synth.CFG_GRAD, 0, 0)
    ut = synth.normal_field(prob.M, synth.CFG_GRAD, 0, 1)
    plan = Plan(n, K, X, a, c, precision="mixed")
    loss, gf, ga, gc = _grads(plan, f, ut, a, c)
    u = osolve.solve(prob, f)
    of, oa, oc = osolve.grad(prob, f, 2 * (u - ut))
    rel_f = np.linalg.norm(gf - of) / np.linalg.norm(of)
    print(f"grad_f rel {rel_f:.3e}  grad_a {ga} vs {oa}  grad_c {gc} vs {oc}")
    assert rel_f <= 1e-10
    np.testing.assert_allclose(ga, oa, rtol=1e-9)
    np.testing.assert_allclose(gc, oc, rtol=1e-9)
