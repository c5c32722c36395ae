"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  This module draws random numbers only; it holds none of the solver's
arithmetic.

Every stream is ``numpy.random.default_rng([170103967, config_id, problem_id,
rhs_id])`` so that the GPU path and the FP64 oracle see the same bytes.
"""

import numpy as np

SEED = 170103967

# workload identifiers (used only as seed components)
CFG_SMALL_2D = 1      # 2D n=2 K=16x16, 5 right-hand sides
CFG_LARGE_2D = 2      # 2D n=9 K=1024x1024 on [0,1]x[0,2], a=(1,2.5), c=1
CFG_3D = 3            # 3D n=9 K=64^3 and n=4 K=128^3
CFG_BATCHED = 4       # 256 mixed problems
CFG_GRAD = 5          # 3D n=5 K=64^3 gradients
CFG_TEST = 99         # ad-hoc test problems


def rng(config_id, problem_id=0, rhs_id=0):
    return np.random.default_rng([SEED, int(config_id), int(problem_id), int(rhs_id)])


def normal_field(shape, config_id, problem_id=0, rhs_id=0):
    """float64 array of i.i.d. N(0,1) entries."""
    return rng(config_id, problem_id, rhs_id).standard_normal(shape)


def normal_batch(nrhs, shape, config_id, problem_id=0, first_rhs=0):
    """(nrhs,) + shape float64 array; right-hand side r uses stream rhs_id=r."""
    out = np.empty((nrhs,) + tuple(shape))
    for r in range(nrhs):
        out[r] = normal_field(shape, config_id, problem_id, first_rhs + r)
    return out


BATCHED_K_CHOICES = (16, 32, 48, 96, 128, 384, 512)


def batched_problems(count=256, max_work=1 << 25, config_id=CFG_BATCHED):
    """Problem specs of the batched workload: N in {2,3} with p=1/2, n uniform
    in {2..8}, K_i drawn independently per axis from BATCHED_K_CHOICES,
    a_i ~ U[0.5, 4], c ~ U[0, 2], X_i = 1, nrhs uniform in {1..8}.  A problem
    whose DOF * nrhs exceeds ``max_work`` is redrawn from the same stream.
    Returns a list of dicts with keys N, n, K, X, a, c, nrhs."""
    specs = []
    for pid in range(count):
        g = rng(config_id, pid, 0)
        while True:
            N = 2 if g.random() < 0.5 else 3
            n = int(g.integers(2, 9))
            K = tuple(int(g.choice(BATCHED_K_CHOICES)) for _ in range(N))
            a = tuple(float(x) for x in g.uniform(0.5, 4.0, size=N))
            c = float(g.uniform(0.0, 2.0))
            nrhs = int(g.integers(1, 9))
            dof = 1
            for k in K:
                dof *= n * k - 1
            if dof * nrhs <= max_work:
                break
        specs.append(dict(N=N, n=n, K=K, X=(1.0,) * N, a=a, c=c, nrhs=nrhs))
    return specs
