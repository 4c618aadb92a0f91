"""GPU parity of the multigrid pieces against the CPU oracle, through the C ABI.

transfers (Sec. 3), one smoothing step of Algorithm 2 with the Schur-CG local
solver (fixed step count, as the oracle's restatement) and with a converged
CG against the Direct (dense LU) local solver, the exact coarse solve, one
V-cycle, and the FGMRES solve in FP64 and mixed precision.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.discretization import Discretization
from oracle.manufactured import Manufactured, rhs
from oracle.multigrid import Hierarchy
from oracle.transfer import prolongation
from seeded_inputs import manufactured_coefficients, random_vector

from _parity import check

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def dev(x, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return t.to(dtype) if dtype is not None else t


@pytest.mark.parametrize("k,nf", [(1, 4), (1, 8), (2, 4), (3, 8), (4, 4), (5, 4)])
def test_transfers(stk, k, nf):
    import torch

    C, F = Discretization(nf // 2, k), Discretization(nf, k)
    Pm = prolongation(C, F)
    P = stk.StokesMG(nf, k)
    L = P.num_levels - 1
    xc = random_vector(300 + k, C.N) * C.free_mask()
    xf0 = random_vector(400 + k, F.N) * F.free_mask()
    out = dev(xf0.copy())
    P.prolongate_add(dev(xc), out)
    check(relerr(out.cpu().numpy(), xf0 + Pm @ xc), 1e-12)
    rf = random_vector(500 + k, F.N)
    rc = torch.full((C.N,), float("nan"), dtype=torch.float64, device="cuda")
    P.restrict(dev(rf), rc)
    check(relerr(rc.cpu().numpy(), Pm.T @ (rf * F.free_mask())), 1e-12)
    # FP32
    out32 = dev(xf0.astype(np.float32))
    P.prolongate_add(dev(xc.astype(np.float32)), out32)
    ref = xf0.astype(np.float32).astype(float) + Pm @ xc.astype(np.float32).astype(float)
    check(relerr(out32.cpu().numpy().astype(float), ref), 1e-5)
    rc32 = torch.empty(C.N, dtype=torch.float32, device="cuda")
    P.restrict(dev(rf.astype(np.float32)), rc32)
    check(relerr(rc32.cpu().numpy().astype(float), Pm.T @ (rf.astype(np.float32).astype(float) * F.free_mask())), 1e-5)
    P.close()


@pytest.mark.parametrize("n,k,iters", [(4, 1, 15), (4, 2, 15), (6, 2, 15), (4, 3, 15), (4, 4, 8), (8, 2, 5), (4, 5, 8)])
def test_smooth_fixed_cg_matches_oracle(stk, n, k, iters):
    H = Hierarchy(n, k, local=("schur", iters))
    d = H.levels[-1].disc
    x0 = random_vector(600 + n + k, d.N) * d.free_mask()
    b = random_vector(700 + n + k, d.N) * d.free_mask()
    ref = H.smooth(len(H.levels) - 1, x0, b)
    P = stk.StokesMG(n, k, local_cg_mode=stk.CG_FIXED, local_cg_iters=iters)
    x = dev(x0.copy())
    P.smooth(x, dev(b))
    check(relerr(x.cpu().numpy(), ref), 1e-12)
    # FP32 smoother against the same FP64 reference
    x32 = dev(x0.astype(np.float32))
    P.smooth(x32, dev(b.astype(np.float32)))
    check(relerr(x32.cpu().numpy().astype(float), ref), 1e-5)
    P.close()


@pytest.mark.parametrize("n,k", [(3, 2), (4, 3), (6, 1)])
def test_smooth_converged_cg_equals_direct(stk, n, k):
    H = Hierarchy(n, k, local="lu")
    d = H.levels[-1].disc
    x0 = random_vector(800 + n + k, d.N) * d.free_mask()
    b = random_vector(900 + n + k, d.N) * d.free_mask()
    ref = H.smooth(len(H.levels) - 1, x0, b)
    P = stk.StokesMG(n, k, local_cg_mode=stk.CG_TOL, local_cg_iters=2000, local_cg_tol=1e-14)
    x = dev(x0.copy())
    P.smooth(x, dev(b))
    check(relerr(x.cpu().numpy(), ref), 1e-12)
    P.close()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_coarse_solve_is_pseudo_inverse(stk, k):
    H = Hierarchy(2, k)
    d = H.levels[0].disc
    b = random_vector(1100 + k, d.N) * d.free_mask()
    ref = H.coarse_solve(b)
    P = stk.StokesMG(2, k)
    x = dev(np.full(d.N, np.nan))
    P.coarse_solve(dev(b), x)
    xs = x.cpu().numpy()
    # both are mean-free in the pressure coefficients; compare directly
    check(relerr(xs, ref), 1e-12)
    P.close()


@pytest.mark.parametrize("n,k", [(4, 2), (8, 1), (4, 3), (8, 2)])
def test_vcycle_matches_oracle(stk, n, k):
    H = Hierarchy(n, k, local=("schur", 15))
    d = H.levels[-1].disc
    b = random_vector(1200 + n + k, d.N) * d.free_mask()
    ref = H.vcycle(b)
    P = stk.StokesMG(n, k, local_cg_mode=stk.CG_FIXED, local_cg_iters=15)
    x = dev(np.full(d.N, np.nan))
    P.vcycle(dev(b), x)
    check(relerr(x.cpu().numpy(), ref), 1e-12)
    x32 = dev(np.full(d.N, np.nan, dtype=np.float32))
    P.vcycle(dev(b.astype(np.float32)), x32)
    check(relerr(x32.cpu().numpy().astype(float), ref), 1e-5)
    P.close()


@pytest.mark.parametrize("n,k", [(4, 2), (8, 2), (4, 3)])
def test_solve_matches_oracle(stk, n, k):
    man = Manufactured(manufactured_coefficients(0))
    H = Hierarchy(n, k, local=("schur", 15))
    d = H.levels[-1].disc
    b = rhs(d, man)
    ref, info_ref = H.solve(b, tol=1e-8)
    for prec in (stk.PREC_FP64, stk.PREC_MIXED):
        P = stk.StokesMG(n, k, precision=prec, local_cg_mode=stk.CG_FIXED, local_cg_iters=15)
        x = dev(np.zeros(d.N))
        info = P.solve(dev(b), x, rtol=1e-8)
        xs = x.cpu().numpy()
        A = H.levels[-1].A
        true_rel = np.linalg.norm(b - A @ xs) / np.linalg.norm(b)
        assert info["converged"] and true_rel <= 1e-8
        if prec == stk.PREC_FP64:
            assert info["iterations"] == info_ref["iterations"]
            check(relerr(xs, ref), 1e-12)
        else:
            assert abs(info["iterations"] - info_ref["iterations"]) <= 1
            check(relerr(xs, ref), 1e-6)
        P.close()


@pytest.mark.parametrize("n,k,nu", [(2, 1, 1.0), (4, 2, 1.0), (4, 3, 0.6), (3, 4, 1.0), (2, 5, 1.0)])
def test_rhs_matches_oracle(stk, n, k, nu):
    import torch

    coef = manufactured_coefficients(17)
    d = Discretization(n, k, nu=nu)
    ref = rhs(d, Manufactured(coef, nu=nu))
    P = stk.StokesMG(n, k, nu)
    b = torch.full((d.N,), float("nan"), dtype=torch.float64, device="cuda")
    P.rhs(coef, b)
    check(relerr(b.cpu().numpy(), ref), 1e-12)
    P.close()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_coarse_solve_on_3cube(stk, k):
    """n = 3 * 2^L hierarchies end on a 3^3 mesh, solved exactly by block
    elimination (dense velocity-block inverses and Schur complement)."""
    H = Hierarchy(3, k)
    d = H.levels[0].disc
    b = random_vector(1300 + k, d.N) * d.free_mask()
    ref = H.coarse_solve(b)  # bordered dense LU: the pressure-row mean goes to the multiplier
    P = stk.StokesMG(3, k)
    x = dev(np.full(d.N, np.nan))
    P.coarse_solve(dev(b), x)
    check(relerr(x.cpu().numpy(), ref), 1e-12)
    # consistent right-hand side, FP32 in and out (the solve itself runs in FP64)
    b[d.offsets[3]:] -= b[d.offsets[3]:].mean()
    ref = H.coarse_solve(b)
    x32 = dev(np.full(d.N, np.nan, dtype=np.float32))
    P.coarse_solve(dev(b.astype(np.float32)), x32)
    check(relerr(x32.cpu().numpy().astype(np.float64), ref), 1e-5)
    P.close()


def test_coarse_factors_shared_and_keyed(stk):
    """The 3^3 factors are shared by problems with the same (k, nu, penalty)
    and rebuilt for another nu; each problem still solves its own system."""
    k = 2
    results = {}
    for nu, pf in ((1.0, 1.0), (0.37, 1.0), (1.0, 2.5)):
        H = Hierarchy(3, k, nu=nu, penalty_factor=pf)
        d = H.levels[0].disc
        b = random_vector(1350, d.N) * d.free_mask()
        ref = H.coarse_solve(b)
        Ps = [stk.StokesMG(3, k, nu, penalty_factor=pf), stk.StokesMG(6, k, nu, penalty_factor=pf)]
        xs = []
        for P in Ps:
            x = dev(np.full(d.N, np.nan))
            P.coarse_solve(dev(b), x)
            xs.append(x.cpu().numpy())
        assert np.array_equal(xs[0], xs[1])  # same factors, same kernels
        check(relerr(xs[0], ref), 1e-12)
        results[(nu, pf)] = xs[0]
        for P in Ps:
            P.close()
    assert not np.allclose(results[(1.0, 1.0)], results[(0.37, 1.0)])


@pytest.mark.parametrize("n,k", [(6, 2), (12, 1)])
def test_vcycle_and_solve_on_3cube_hierarchy(stk, n, k):
    man = Manufactured(manufactured_coefficients(5))
    H = Hierarchy(n, k, local=("schur", 15))
    d = H.levels[-1].disc
    b = rhs(d, man)
    ref = H.vcycle(b)
    P = stk.StokesMG(n, k, local_cg_mode=stk.CG_FIXED, local_cg_iters=15)
    x = dev(np.full(d.N, np.nan))
    P.vcycle(dev(b), x)
    check(relerr(x.cpu().numpy(), ref), 1e-12)
    xs = dev(np.zeros(d.N))
    info = P.solve(dev(b), xs, rtol=1e-8)
    _, info_ref = H.solve(b, tol=1e-8)
    assert info["converged"] and abs(info["iterations"] - info_ref["iterations"]) <= 1
    P.close()


def test_non_convergence_and_bad_arguments_report_status(stk):
    """Failure paths on the host side of the ABI: an iteration limit that is
    too small returns STK_ENOCONV with the info filled and the last iterate in
    x; malformed calls return STK_EINVAL with a message and leave the problem
    usable."""
    import torch

    man = Manufactured(manufactured_coefficients(0))
    d = Discretization(4, 2)
    b = rhs(d, man)
    P = stk.StokesMG(4, 2, max_iter=1)
    x = dev(np.zeros(d.N))
    info = P.solve(dev(b), x, rtol=1e-12, check=False)
    assert info["status"] == -4 and not info["converged"] and info["iterations"] == 1
    assert 0 < info["relres"] < 1 and np.isfinite(x.cpu().numpy()).all()
    with pytest.raises(stk.StokesError) as err:
        P.solve(dev(b), x, rtol=1e-12)
    assert err.value.code == -4
    # wrong level / dtype / length are rejected before any launch
    with pytest.raises((stk.StokesError, ValueError)):
        P.apply(dev(b), x, level=7)
    with pytest.raises(ValueError):
        P.apply(dev(b[:-1].copy()), x)
    y = torch.empty_like(x)
    P.apply(dev(b), y)  # still usable
    assert np.isfinite(y.cpu().numpy()).all()
    P.close()


def test_tight_local_tolerance_in_fp32_still_converges(stk):
    """A TOL-mode local CG tighter than FP32 can reach (1e-10) is floored at
    1e-6 in the FP32 smoother, so the mixed-precision solve converges as with
    the default fixed step count."""
    import torch

    s = torch.cuda.Stream()
    P = stk.StokesMG(32, 3, 1.0, precision=stk.PREC_MIXED, stream=s, local_cg_mode=stk.CG_TOL,
                     local_cg_iters=200, local_cg_tol=1e-10)
    b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        P.rhs(manufactured_coefficients(3000), b)
    x = torch.zeros_like(b)
    info = P.solve(b, x, rtol=1e-8)
    assert info["converged"] and info["iterations"] <= 6
    P.close()


@pytest.mark.parametrize("n,k", [(3, 2), (4, 3), (6, 1), (4, 2)])
def test_smooth_direct_equals_oracle_lu(stk, n, k):
    """The Direct local solver (Sec. 3.2: the exact patch solve, here the
    precomputed inverse of each patch type's Schur complement) against the
    oracle's bordered dense LU of every patch."""
    H = Hierarchy(n, k, local="lu")
    d = H.levels[-1].disc
    x0 = random_vector(1500 + n + k, d.N) * d.free_mask()
    b = random_vector(1600 + n + k, d.N) * d.free_mask()
    ref = H.smooth(len(H.levels) - 1, x0, b)
    P = stk.StokesMG(n, k, local_cg_mode=stk.LOCAL_DIRECT)
    x = dev(x0.copy())
    P.smooth(x, dev(b))
    check(relerr(x.cpu().numpy(), ref), 1e-12)
    x32 = dev(x0.astype(np.float32))
    P.smooth(x32, dev(b.astype(np.float32)))
    check(relerr(x32.cpu().numpy().astype(float), ref), 1e-5)
    P.close()


def test_direct_local_solver_solve(stk):
    """With exact local solves the V-cycle contracts at least as well as with
    15 CG steps; the solve reaches 1e-8 and matches the oracle's solution."""
    import torch

    n, k = 8, 3
    man = Manufactured(manufactured_coefficients(21))
    H = Hierarchy(n, k, local="lu")
    d = H.levels[-1].disc
    b = rhs(d, man)
    x_ref, info_ref = H.solve(b, tol=1e-8)
    its = {}
    for mode in (stk.LOCAL_DIRECT, stk.CG_FIXED):
        P = stk.StokesMG(n, k, precision=stk.PREC_MIXED, local_cg_mode=mode)
        x = torch.zeros(d.N, dtype=torch.float64, device="cuda")
        info = P.solve(dev(b), x, rtol=1e-8)
        assert info["converged"]
        its[mode] = info["iterations"]
        if mode == stk.LOCAL_DIRECT:
            nv = d.offsets[3]
            xs = x.cpu().numpy()
            assert np.abs(xs[:nv] - x_ref[:nv]).max() <= 1e-6 * np.abs(x_ref[:nv]).max()
            assert abs(info["iterations"] - info_ref["iterations"]) <= 1
        P.close()
    assert its[stk.LOCAL_DIRECT] <= its[stk.CG_FIXED]


def test_autotuned_smoother_keeps_parity(stk):
    """stk_autotune also picks the smoother's form per smoothed level (split or
    fused, the faster) and whether the interior patches get their own launch;
    the smoothing step it then runs still matches the oracle's."""
    n, k = 8, 2
    H = Hierarchy(n, k, local=("schur", 15))
    d = H.levels[-1].disc
    x0 = random_vector(1700, d.N) * d.free_mask()
    b = random_vector(1701, d.N) * d.free_mask()
    ref = H.smooth(len(H.levels) - 1, x0, b)
    P = stk.StokesMG(n, k, local_cg_mode=stk.CG_FIXED, local_cg_iters=15)
    tuned = P.autotune(stk.F64, with_smoother=True)
    assert tuned[0][1] == -1 and all(tuned[level][1] in (0, 1) for level in range(1, P.num_levels))
    assert tuned[0][2] == -1 and all(tuned[level][2] in (0, 1) for level in range(1, P.num_levels))
    x = dev(x0.copy())
    P.smooth(x, dev(b))
    check(relerr(x.cpu().numpy(), ref), 1e-12)
    P.close()


@pytest.mark.parametrize("n,k", [(32, 2), (32, 3), (16, 4)])
def test_direct_gemm_equals_per_patch_product(stk, n, k):
    """The FP32 Direct smoother with the interior patches' products of a
    colour as one GEMM (tensor cores with the FP32 emulation, or plain FP32)
    equals the per-patch product in the patch kernel to FP32 rounding; FP64 is
    unaffected (always the per-patch product)."""
    import torch

    x0 = None
    out = {}
    for mode in (0, 1, 2):
        P = stk.StokesMG(n, k, local_cg_mode=stk.LOCAL_DIRECT, direct_gemm=mode)
        N = P.layout()["n_total"]
        if x0 is None:
            x0 = random_vector(1800 + n + k, N)
            b = random_vector(1900 + n + k, N)
        x = dev(x0.astype(np.float32))
        P.smooth(x, dev(b.astype(np.float32)))
        out[mode] = x.cpu().numpy().astype(float)
        P.close()
    check(relerr(out[1], out[0]), 1e-5, "fp32 gemm")
    check(relerr(out[2], out[0]), 1e-5, "bf16x9 gemm")
