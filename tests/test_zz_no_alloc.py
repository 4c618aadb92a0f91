"""stk_smooth_static: the smoother variant that allocates no device memory.

Callers that may not allocate (a framework whose memory pool owns every
device allocation, a real-time loop that cannot absorb a cudaMalloc stall) use
it in place of stk_smooth.  It must give the same result
as stk_smooth, call after call, although every call reuses the same static
residual array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle.discretization import Discretization
from seeded_inputs import random_vector

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("n,k", [(4, 2), (8, 3)])
def test_static_smoother_matches_allocating_smoother_twice(stk, n, k):
    import torch

    d = Discretization(n, k)
    P = stk.StokesMG(n, k, local_cg_mode=stk.CG_FIXED, local_cg_iters=15)
    x0 = random_vector(2100 + n + k, d.N) * d.free_mask()
    b = torch.from_numpy(random_vector(2200 + n + k, d.N) * d.free_mask()).cuda()
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        xa = torch.from_numpy(x0).to(dtype).cuda()
        xs = xa.clone()
        bb = b.to(dtype)
        for _ in range(2):  # two calls in a row: the second reuses the static array
            P.smooth(xa, bb)
            P.smooth_static(xs, bb)
            torch.cuda.synchronize()
            ya, ys = xa.cpu().double().numpy(), xs.cpu().double().numpy()
            assert _relerr(ys, ya) <= tol
    P.close()


def test_static_smoother_allocates_nothing_on_a_fresh_problem(stk, monkeypatch):
    """With every library allocation made to fail (the host-side injector,
    STK_FAIL_ALLOC_AFTER=0), stk_smooth_static still runs on a problem that no
    other smoothing call has touched (no workspace exists yet), twice in a row,
    and matches stk_smooth run afterwards on a second problem built the same way."""
    import torch

    n, k = 4, 3
    d = Discretization(n, k)
    x0 = random_vector(2300, d.N) * d.free_mask()
    b = torch.from_numpy(random_vector(2301, d.N) * d.free_mask()).cuda()
    fresh = stk.StokesMG(n, k, local_cg_mode=stk.CG_FIXED, local_cg_iters=15)
    xs = torch.from_numpy(x0).cuda()
    monkeypatch.setenv("STK_FAIL_ALLOC_AFTER", "0")
    fresh.smooth_static(xs, b)
    fresh.smooth_static(xs, b)
    torch.cuda.synchronize()
    # the injector is live: an allocating call on the same problem fails
    with pytest.raises(stk.StokesError) as err:
        fresh.smooth(xs.clone(), b)
    assert err.value.code == -3
    monkeypatch.delenv("STK_FAIL_ALLOC_AFTER")
    other = stk.StokesMG(n, k, local_cg_mode=stk.CG_FIXED, local_cg_iters=15)
    xa = torch.from_numpy(x0).cuda()
    other.smooth(xa, b)
    other.smooth(xa, b)
    torch.cuda.synchronize()
    assert _relerr(xs.cpu().numpy(), xa.cpu().numpy()) <= 1e-12
    fresh.close()
    other.close()


def test_static_smoother_rejects_levels_beyond_its_array(stk):
    import torch

    P = stk.StokesMG(32, 3)  # 8.5 M DoF: 68 MB of FP64 residual > 32 MiB
    N = P.layout()["n_total"]
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(x)
    with pytest.raises(stk.StokesError) as err:
        P.smooth_static(x, b)
    assert err.value.code == -1 and "too large" in str(err.value)
    # a coarser level of the same problem fits
    x1 = torch.zeros(P.layout(1)["n_total"], dtype=torch.float64, device="cuda")
    P.smooth_static(x1, torch.zeros_like(x1), level=1)
    P.close()
