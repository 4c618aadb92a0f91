"""GPU parity of the matrix-free operator (Algorithm 1) against the oracle's
assembled matrix, element by element, through the C ABI.

FP64 bar: relative max-norm error 1e-12.  FP32 bar: 1e-5, with the oracle fed
the float32-rounded input so that only the kernel's arithmetic differs.
"""
import numpy as np
import pytest

from oracle.discretization import Discretization
from seeded_inputs import random_vector

from _parity import check

pytestmark = pytest.mark.gpu

# (n, k): several tiles, ragged tails, runs that start inside a column or span
# several (the default grid gives CTAs ~4 cells each on small meshes) and every degree
CASES = [(2, 1), (6, 1), (12, 1), (3, 2), (8, 2), (4, 3), (6, 3), (3, 4), (6, 4), (2, 5), (4, 5)]


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("n,k", CASES)
def test_apply_matches_assembled_operator(stk, n, k):
    import torch

    d = Discretization(n, k, nu=1.0)
    A = d.assemble()
    x = random_vector(1000 + 10 * n + k, d.N)
    x_used = x * d.free_mask()
    y_ref = A @ x_used
    P = stk.StokesMG(n, k, 1.0)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    P.apply(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert np.isfinite(y).all()
    check(_relerr(y, y_ref), 1e-12)
    assert np.all(y[~d.free_mask()] == 0.0)
    # FP32
    x32 = x.astype(np.float32)
    y_ref32 = A @ (x32.astype(np.float64) * d.free_mask())
    y32 = torch.full((d.N,), float("nan"), dtype=torch.float32, device="cuda")
    P.apply(torch.from_numpy(x32).cuda(), y32)
    torch.cuda.synchronize()
    check(_relerr(y32.cpu().numpy().astype(np.float64), y_ref32), 1e-5)
    P.close()


@pytest.mark.parametrize("n,k,nu", [(4, 2, 0.37), (6, 3, 2.5)])
def test_residual_and_viscosity(stk, n, k, nu):
    import torch

    d = Discretization(n, k, nu=nu)
    A = d.assemble()
    x = random_vector(77, d.N)
    b = random_vector(78, d.N)
    r_ref = b - A @ (x * d.free_mask())
    P = stk.StokesMG(n, k, nu)
    xd, bd = torch.from_numpy(x).cuda(), torch.from_numpy(b).cuda()
    rd = torch.empty_like(xd)
    P.residual(xd, bd, rd)
    r = rd.cpu().numpy()
    f = d.free_mask()
    check(_relerr(r[f], r_ref[f]), 1e-12)
    # residual in place of b
    P.residual(xd, bd, bd)
    assert np.array_equal(bd.cpu().numpy(), r)
    P.close()


def test_coarser_levels(stk):
    import torch

    P = stk.StokesMG(8, 2, 1.0)
    for level, n in enumerate([2, 4, 8]):
        assert P.layout(level)["n"] == n
        d = Discretization(n, 2)
        x = random_vector(5 + level, d.N)
        y = torch.empty(d.N, dtype=torch.float64, device="cuda")
        P.apply(torch.from_numpy(x).cuda(), y, level=level)
        check(_relerr(y.cpu().numpy(), d.assemble() @ (x * d.free_mask())), 1e-12)
    P.close()


def test_full_size_sampled_rows(stk):
    """The benchmarked workload (64^3 cells, k = 3, 67.3 M DoF) at 2000 sampled
    outputs, computed one by one by the oracle from its local matrices."""
    import torch

    n, k = 64, 3
    d = Discretization(n, k)
    x = random_vector(1001, d.N)
    P = stk.StokesMG(n, k, 1.0)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    P.apply(xd, yd)
    y = yd.cpu().numpy()
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.integers(0, d.N, 1500), np.arange(0, 300), d.N - 1 - np.arange(200)])
    ref = d.apply_rows(x, rows)
    check(np.abs(y[rows] - ref).max() / np.abs(ref).max(), 1e-12)
    P.close()


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_autotuned_apply_keeps_parity(stk, dtype_name):
    import torch

    n, k = 8, 2
    d = Discretization(n, k)
    A = d.assemble()
    P = stk.StokesMG(n, k, 1.0)
    dt = stk.F64 if dtype_name == "f64" else stk.F32
    tuned = P.autotune(dt)
    # run length of the persistent velocity march: n, halved down to 2
    assert all(2 <= v <= P.layout(level)["n"] for level, v in tuned.items())
    x = random_vector(4242, d.N)
    tdt = torch.float64 if dtype_name == "f64" else torch.float32
    xd = torch.from_numpy(x).to(tdt).cuda()
    yd = torch.empty_like(xd)
    P.apply(xd, yd)
    ref = A @ (xd.cpu().double().numpy() * d.free_mask())
    assert _relerr(yd.cpu().double().numpy(), ref) <= (1e-12 if dtype_name == "f64" else 1e-5)
    P.close()


@pytest.mark.parametrize("n,k,blk", [(12, 2, 5), (12, 3, 1), (6, 4, 4), (16, 1, 3), (4, 5, 3)])
def test_set_tuning_run_lengths_keep_parity(stk, n, k, blk):
    """Every run length of the persistent march (ragged last runs, runs of one
    cell, remainders split across CTAs) gives the assembled operator's
    product; 0 restores the built-in choice."""
    import torch

    d = Discretization(n, k)
    A = d.assemble()
    P = stk.StokesMG(n, k, 1.0)
    x = random_vector(4343 + n + k, d.N)
    ref = A @ (x * d.free_mask())
    for dt, tdt, bar in ((stk.F64, torch.float64, 1e-12), (stk.F32, torch.float32, 1e-5)):
        P.set_tuning(-1, dt, blk)
        xd = torch.from_numpy(x).to(tdt).cuda()
        yd = torch.full_like(xd, float("nan"))
        P.apply(xd, yd)
        r = A @ (xd.cpu().double().numpy() * d.free_mask())
        check(_relerr(yd.cpu().double().numpy(), r), bar, f"blk={blk} {tdt}")
        P.set_tuning(-1, dt, 0)
    with pytest.raises(stk.StokesError):
        P.set_tuning(0, stk.F64, -1)
    P.close()
