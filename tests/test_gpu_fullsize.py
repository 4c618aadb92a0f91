"""Full-size checks of the benchmarked workloads, on outputs the oracle computes
one by one from its local matrices (no global matrix at these sizes).

- the FP64 apply at 64^3 cells for every degree of the operator sweep
  (k = 3 is in test_gpu_apply.py), in the launch configuration bench.py times;
- the mixed-precision solve on 96^3 cells at k = 3 (226.9 M DoF): the
  residual b - A x at sampled rows, with A x evaluated by the oracle, is
  bounded by the solver's 1e-8 relative tolerance, and the pressure has zero
  mean.
"""
import numpy as np
import pytest

from oracle.discretization import Discretization
from seeded_inputs import manufactured_coefficients, random_vector

pytestmark = pytest.mark.gpu


def _rows(N, seed, count=600):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, N, count), np.arange(0, 100), N - 1 - np.arange(100)]))


@pytest.mark.parametrize("k", [1, 2, 4, 5])
def test_sweep_apply_full_size_sampled_rows(stk, k):
    import torch

    n = 64
    d = Discretization(n, k)
    x = random_vector(2000 + k, d.N)
    P = stk.StokesMG(n, k, 1.0)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    P.apply(xd, yd)
    rows = _rows(d.N, k)
    y = yd[torch.from_numpy(rows).cuda()].cpu().numpy()
    ref = d.apply_rows(x, rows)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    P.close()


def test_mixed_solve_full_size_sampled_residual(stk):
    import torch

    n, k = 96, 3
    d = Discretization(n, k)
    P = stk.StokesMG(n, k, 1.0, precision=stk.PREC_MIXED)
    b = torch.empty(d.N, dtype=torch.float64, device="cuda")
    P.rhs(manufactured_coefficients(3000), b)
    x = torch.zeros_like(b)
    info = P.solve(b, x, rtol=1e-8)
    assert info["converged"] and info["relres"] <= 1e-8
    bnorm = float(torch.linalg.vector_norm(b))
    # the library's own FP64 residual
    r = torch.empty_like(b)
    P.residual(x, b, r)
    assert float(torch.linalg.vector_norm(r)) <= 1.01e-8 * bnorm
    # the oracle's rows of A x at sampled DoFs: every |r_i| <= ||r||_2 <= 1e-8 ||b||_2
    rows = _rows(d.N, 7)
    xs = x.cpu().numpy()
    ref = d.apply_rows(xs, rows)
    r_rows = b.cpu().numpy()[rows] - ref
    free = d.free_mask()[rows]
    assert np.abs(r_rows[free]).max() <= 1.01e-8 * bnorm
    # pressure of zero mean (tensor Gauss weights x cell volume)
    w = d.pressure_weights()
    p = xs[d.offsets[3]:]
    assert abs(float(w @ p)) <= 1e-10 * np.abs(p).max()
    P.close()
