"""Batched solves and the captured V-cycle (the batching row of the hot path).

stk_solve_batch advances many independent problems of uneven sizes and
degrees together, each on its own stream; every problem runs the same kernels
in the same order as a solve of its own, so the results are bitwise those of
one-by-one solves.  The V-cycle replayed from a CUDA graph likewise equals the
directly launched one bitwise.  One batched problem is checked against the
oracle's solve.
"""
import numpy as np
import pytest

from oracle.manufactured import Manufactured, rhs
from oracle.multigrid import Hierarchy
from seeded_inputs import manufactured_coefficients

from _parity import check

pytestmark = pytest.mark.gpu

# 2^3- and 3^3-based hierarchies, k = 1..3
PROBLEMS = [(4, 2), (6, 1), (3, 3), (8, 2), (12, 2), (4, 3)]


def _setup(stk, precision):
    import torch

    probs, bs = [], []
    for i, (n, k) in enumerate(PROBLEMS):
        s = torch.cuda.Stream()
        P = stk.StokesMG(n, k, 1.0, precision=precision, stream=s)
        b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
        with torch.cuda.stream(s):
            P.rhs(manufactured_coefficients(500 + i), b)
        probs.append(P)
        bs.append(b)
    torch.cuda.synchronize()
    return probs, bs


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_equals_one_by_one(stk, precision):
    import torch

    prec = stk.PREC_MIXED if precision == "mixed" else stk.PREC_FP64
    probs, bs = _setup(stk, prec)
    xs = [torch.zeros_like(b) for b in bs]
    infos = stk.solve_batch(probs, bs, xs, 1e-8)
    assert all(i["converged"] and i["relres"] <= 1e-8 for i in infos)
    for P, b, x, info in zip(probs, bs, xs, infos):
        x1 = torch.zeros_like(b)
        one = P.solve(b, x1, rtol=1e-8)
        assert one["iterations"] == info["iterations"]
        assert torch.equal(x1, x)
        P.close()


def test_batch_against_oracle(stk):
    import torch

    n, k = 4, 2
    man = Manufactured(manufactured_coefficients(500))
    H = Hierarchy(n, k, local=("schur", 15))
    d = H.levels[-1].disc
    b = rhs(d, man)
    x_ref, info_ref = H.solve(b, tol=1e-8)
    probs, bs = _setup(stk, stk.PREC_FP64)
    assert np.abs(bs[0].cpu().numpy() - b).max() <= 1e-12 * np.abs(b).max()
    xs = [torch.zeros_like(bb) for bb in bs]
    infos = stk.solve_batch(probs, bs, xs, 1e-8)
    assert abs(infos[0]["iterations"] - info_ref["iterations"]) <= 1
    x = xs[0].cpu().numpy()
    # both solve to a relative residual of 1e-8: compare the velocities
    nv = d.offsets[3]
    assert np.abs(x[:nv] - x_ref[:nv]).max() <= 1e-6 * np.abs(x_ref[:nv]).max()
    for P in probs:
        P.close()


def test_graph_replay_equals_direct_launches(stk):
    import torch

    out = []
    for graphs in (True, False):
        s = torch.cuda.Stream()
        P = stk.StokesMG(8, 2, 1.0, precision=stk.PREC_MIXED, stream=s, use_graphs=graphs)
        b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
        with torch.cuda.stream(s):
            P.rhs(manufactured_coefficients(900), b)
        x = torch.zeros_like(b)
        info = P.solve(b, x, rtol=1e-10)
        assert info["converged"] and info["iterations"] >= 3  # the graph is captured and replayed
        out.append(x.cpu().numpy())
        P.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_smooth_batch_equals_separate_smoothing(stk, dtype_name):
    """One smoothing step of several problems of the same degree with one patch
    launch per colour equals separate smoothing steps bitwise, on the finest
    and on coarser levels."""
    import torch

    from seeded_inputs import random_vector

    dt = torch.float64 if dtype_name == "f64" else torch.float32
    sizes = [(4, -1), (6, -1), (8, -1), (3, -1), (8, 1), (12, 1)]
    s = torch.cuda.Stream()
    # the merged launches run the split form of the smoother (residual apply, then patch kernel)
    probs = [stk.StokesMG(n, 2, 1.0, stream=s, fused_smoother=False) for n, _ in sizes]
    levels = [P._lvl(l) for P, (_, l) in zip(probs, sizes)]
    xs, bs = [], []
    for i, (P, l) in enumerate(zip(probs, levels)):
        N = P.layout(l)["n_total"]
        xs.append(torch.from_numpy(random_vector(700 + i, N)).to(dt).cuda())
        bs.append(torch.from_numpy(random_vector(800 + i, N)).to(dt).cuda())
    ref = [x.clone() for x in xs]
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for P, x, b, l in zip(probs, ref, bs, levels):
            P.smooth(x, b, level=l)
        stk.smooth_batch(probs, xs, bs, levels)
    s.synchronize()
    for a, r in zip(xs, ref):
        assert torch.equal(a, r)
    for P in probs:
        P.close()


@pytest.mark.parametrize("dtype_name", ["f64", "f32"])
def test_interior_launch_matches_single_kernel(stk, dtype_name):
    """On a 64^3 level the interior patches of a colour run in their own
    kernel (no dense transforms) and the boundary ones in a second launch;
    the multi-problem path runs every patch in the general kernel.  Both give
    the same smoothing step to rounding."""
    import torch

    from seeded_inputs import random_vector

    dt = torch.float64 if dtype_name == "f64" else torch.float32
    s = torch.cuda.Stream()
    P = stk.StokesMG(64, 2, 1.0, stream=s, fused_smoother=False)
    N = P.layout()["n_total"]
    b = torch.from_numpy(random_vector(950, N)).to(dt).cuda()
    x1 = torch.from_numpy(random_vector(951, N)).to(dt).cuda()
    x2 = x1.clone()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        P.smooth(x1, b)
        stk.smooth_batch([P], [x2], [b])
    s.synchronize()
    err = float((x1 - x2).abs().max() / x2.abs().max())
    assert err <= (1e-13 if dtype_name == "f64" else 1e-6)
    P.close()


@pytest.mark.parametrize("n,k", [(2, 3), (3, 2), (4, 1), (6, 4), (8, 2), (6, 5), (64, 3)])
def test_fused_smoother_equals_split_smoother(stk, n, k):
    """The fused colour step (patch residual computed inside the patch kernel
    from the x of before the colour, colours alternating between two buffers,
    unowned entries copied across) equals the split form (a residual apply
    of the whole level per colour, then the patch kernel) to rounding, for
    2^3- and 3^3-based meshes, every degree and the 64^3 level whose
    interior patches run in their own launch; also the Direct local solver."""
    import torch

    from seeded_inputs import random_vector

    for mode in (stk.CG_FIXED, stk.LOCAL_DIRECT) if n <= 8 else (stk.CG_FIXED,):
        fused = stk.StokesMG(n, k, 1.0, local_cg_mode=mode)
        split = stk.StokesMG(n, k, 1.0, local_cg_mode=mode, fused_smoother=False)
        N = fused.layout()["n_total"]
        for dt, bar in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            # constrained entries carry garbage: both forms must leave them as they are
            x0 = torch.from_numpy(random_vector(3100 + n + k, N)).to(dt).cuda()
            b = torch.from_numpy(random_vector(3200 + n + k, N)).to(dt).cuda()
            xa, xb = x0.clone(), x0.clone()
            fused.smooth(xa, b)
            split.smooth(xb, b)
            torch.cuda.synchronize()
            check(float((xa - xb).abs().max() / xb.abs().max()), bar, f"mode={mode} {dt}")
            # one colour alone (the entry point copies x to its input buffer)
            ya, yb = x0.clone(), x0.clone()
            fused.smooth_colour(5, ya, b)
            split.smooth_colour(5, yb, b)
            torch.cuda.synchronize()
            check(float((ya - yb).abs().max() / yb.abs().max()), bar, f"colour 5 mode={mode} {dt}")
        fused.close()
        split.close()


@pytest.mark.parametrize("n,k,mode,prec", [(24, 3, "direct", "mixed"), (12, 2, "direct", "fp64"), (16, 2, "cg", "mixed")])
def test_stream_solves_direct_and_cg(stk, n, k, mode, prec):
    """Solves on a stream of their own (the whole solve as one graph, or, for
    the FP32 Direct smoother with its cuBLAS GEMM, host-driven with the
    V-cycle graph) converge, and equal the solve with graphs off bitwise."""
    import torch

    from seeded_inputs import manufactured_coefficients

    local = stk.LOCAL_DIRECT if mode == "direct" else stk.CG_FIXED
    precision = stk.PREC_MIXED if prec == "mixed" else stk.PREC_FP64
    out = []
    for graphs in (True, False):
        s = torch.cuda.Stream()
        P = stk.StokesMG(n, k, 1.0, precision=precision, stream=s, local_cg_mode=local, use_graphs=graphs)
        b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
        with torch.cuda.stream(s):
            P.rhs(manufactured_coefficients(950), b)
        x = torch.zeros_like(b)
        for _ in range(2):  # the second solve replays what the first built
            info = P.solve(b, x, rtol=1e-8)
        assert info["converged"] and info["relres"] <= 1e-8
        out.append(x.cpu().numpy())
        P.close()
    assert np.array_equal(out[0], out[1])
