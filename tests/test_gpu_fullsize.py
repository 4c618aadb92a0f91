"""Full-size checks of the benchmarked workloads, on outputs the oracle computes
one by one from its local matrices (no global matrix at these sizes).

- the FP64 apply at 64^3 cells for every degree of the operator sweep
  (k = 3 is in test_gpu_apply.py), in the launch configuration bench.py times;
- the FP32 apply at 64^3 cells for every degree;
- one colour of the smoother at 64^3, k = 3 (the interior-patch kernel and
  the boundary patches) against the oracle's patch solves;
- the mixed-precision solve on 96^3 cells at k = 3 (226.9 M DoF): the
  residual b - A x at sampled rows, with A x evaluated by the oracle, is
  bounded by the solver's 1e-8 relative tolerance, and the pressure has zero
  mean.
"""
import numpy as np
import pytest

from oracle.discretization import Discretization
from seeded_inputs import manufactured_coefficients, random_vector

from _parity import check

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
    check(np.abs(y - ref).max() / np.abs(ref).max(), 1e-12, "f64")
    P.close()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_fp32_apply_full_size_sampled_rows(stk, k):
    """The FP32 apply of the V-cycle (its own register pipeline for k <= 3) at
    64^3 cells, every degree, against the oracle's rows of the float32-rounded
    input evaluated in FP64."""
    import torch

    n = 64
    d = Discretization(n, k)
    x = random_vector(2050 + k, d.N).astype(np.float32)
    P = stk.StokesMG(n, k, 1.0)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    P.apply(xd, yd)
    rows = _rows(d.N, 10 + k, count=400)
    y = yd[torch.from_numpy(rows).cuda()].cpu().double().numpy()
    ref = d.apply_rows(x.astype(np.float64), rows)
    check(np.abs(y - ref).max() / np.abs(ref).max(), 1e-5, "f32")
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


def _patch_problem(d, vertex, x, b):
    """Patch matrix A_j = R_j A R_j^T and local residual R_j (b - A x) of the
    patch at `vertex`, from the oracle's local pieces of the patch's 8 cells."""
    from oracle.multigrid import patch_dofs

    cells = [(vertex[0] - 1 + a, vertex[1] - 1 + bb, vertex[2] - 1 + c) for c in (0, 1) for bb in (0, 1) for a in (0, 1)]
    cols, K = d.local_rows(cells)
    J = patch_dofs(d, vertex)
    pos = np.searchsorted(cols, J)
    rows = K[pos]
    Aj = rows[:, pos].toarray()
    r = b[J] - rows @ x[cols]
    return J, Aj, r


def _colour_sample(n, colour, count, seed):
    from oracle.multigrid import colour_vertices

    verts = colour_vertices(n, colour)
    rng = np.random.default_rng(seed)
    pick = [verts[i] for i in rng.choice(len(verts), count, replace=False)]
    # the corners of the colour's vertex grid: patches on the boundary in up to three directions
    lo = [min(v[d] for v in verts) for d in range(3)]
    hi = [max(v[d] for v in verts) for d in range(3)]
    corners = [(a, b, c) for a in (lo[0], hi[0]) for b in (lo[1], hi[1]) for c in (lo[2], hi[2])]
    return list(dict.fromkeys(corners + pick))


@pytest.mark.parametrize("colour", [0, 7])
def test_smoother_colour_full_size_against_oracle(stk, colour):
    """One colour of Algorithm 2 on the 64^3, k = 3 level of the benchmarked
    smoother, in the launch configuration of stk_smooth: at this size the
    interior patches of a colour run in their own kernel (colour 0 of an even
    mesh has only interior patches; colour 7 also has every boundary type).
    Sampled patches are compared with the oracle's local solve of the patch
    problem R_j A R_j^T built from its own local matrices and the residual
    R_j (b - A x) of the same seeded x and b: the fixed 15-step Schur CG
    against the oracle's Schur CG, the Direct local solver against the dense
    LU of the bordered patch system, in FP64 and FP32."""
    import torch

    from oracle.multigrid import LocalSolver

    n, k = 64, 3
    d = Discretization(n, k)
    free = d.free_mask()
    npress = (2 * k + 2) ** 3
    x0 = random_vector(2500 + colour, d.N) * free
    b0 = random_vector(2600 + colour, d.N) * free
    verts = _colour_sample(n, colour, 6, 2700 + colour)
    for mode, ref_solver in ((stk.CG_FIXED, LocalSolver(("schur", 15))), (stk.LOCAL_DIRECT, LocalSolver("lu"))):
        P = stk.StokesMG(n, k, 1.0, local_cg_mode=mode, local_cg_iters=15)
        for dt, bar in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            xin = x0.astype(np.float32).astype(np.float64) if dt == torch.float32 else x0
            bin_ = b0.astype(np.float32).astype(np.float64) if dt == torch.float32 else b0
            x = torch.from_numpy(xin).to(dt).cuda()
            bd = torch.from_numpy(bin_).to(dt).cuda()
            P.smooth_colour(colour, x, bd)
            xh = x.cpu().double().numpy()
            worst = 0.0
            for v in verts:
                J, Aj, r = _patch_problem(d, v, xin, bin_)
                ref = ref_solver(Aj, npress, r)
                got = xh[J] - xin[J]
                worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
            check(worst, bar, f"mode={mode} {dt}")
            del x, bd
        P.close()
