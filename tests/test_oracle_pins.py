"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle through a route it does not use itself: closed
forms, an independently built Kronecker form (Sec. 2.3), printed numbers of the
paper (tests/golden), nestedness of the spaces (Sec. 3), exactness of the
Direct local solver (Sec. 3.3) and the 3D iteration-count claim (Sec. 3.3).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.basis import gauss_legendre, gauss_lobatto, lagrange
from oracle.discretization import Discretization
from oracle.manufactured import Manufactured, interpolate, l2_errors, rhs
from oracle.multigrid import Hierarchy, LocalSolver, colour_vertices, patch_dofs, schur_cg
from oracle.transfer import prolongation
from seeded_inputs import manufactured_coefficients, random_vector

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


# ------------------------------------------------------------ seeded inputs
def test_splitmix64_reference_outputs():
    """splitmix64 (Steele, Lea, Flood 2014) from state 0: the first outputs of
    the published generator are e220a8397b1dcdaf, 6e789e6aa1b965f4,
    06c45d188009454f; uniform draws use the top 53 bits."""
    from seeded_inputs import splitmix64_stream, uniform_pm1

    z = splitmix64_stream(0, 3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = uniform_pm1(0, 1)[0]
    assert u == 2.0 * ((0xE220A8397B1DCDAF >> 11) / 2.0 ** 53) - 1.0


# ----------------------------------------------------------------- 1D pieces
def test_quadrature_closed_forms():
    x, w = gauss_lobatto(3)
    assert np.allclose(x, [0, 0.5, 1], atol=1e-15) and np.allclose(w, [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    x, w = gauss_lobatto(4)
    s = 1 / math.sqrt(5)
    assert np.allclose(x, [0, (1 - s) / 2, (1 + s) / 2, 1], atol=1e-15)
    assert np.allclose(w, [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-15)
    x, w = gauss_legendre(2)
    assert np.allclose(x, [(1 - 1 / math.sqrt(3)) / 2, (1 + 1 / math.sqrt(3)) / 2], atol=1e-15)
    for npts in range(2, 9):
        xg, wg = gauss_legendre(npts)
        xl, wl = gauss_lobatto(npts)
        for p in range(2 * npts):
            assert abs(wg @ xg ** p - 1 / (p + 1)) < 1e-14
        for p in range(2 * npts - 2):
            assert abs(wl @ xl ** p - 1 / (p + 1)) < 1e-14


def test_lagrange_basis():
    z = gauss_lobatto(5)[0]
    V, D = lagrange(z, z)
    assert np.allclose(V, np.eye(5), atol=1e-14)
    t = np.linspace(0, 1, 11)
    V, D = lagrange(z, t)
    # partition of unity and exact reproduction of t^3 and its derivative
    assert np.allclose(V.sum(0), 1, atol=1e-13) and np.allclose(D.sum(0), 0, atol=1e-11)
    assert np.allclose((z ** 3) @ V, t ** 3, atol=1e-13)
    assert np.allclose((z ** 3) @ D, 3 * t ** 2, atol=1e-11)


# --------------------------------------------------------------- DoF counts
@pytest.mark.parametrize("k", [2, 4])
def test_dof_counts_match_paper(k):
    # a vertex patch is 2x2x2 cells; Table 2 counts its DoFs including boundary normals
    assert Discretization(2, k).N == GOLDEN["dofs_per_patch"][str(k)]
    # 64^3 mesh: "between 28 and 131 million DoFs" (Sec. 4.2)
    assert round(Discretization(64, k).N / 1e6) == GOLDEN["dofs_64_cubed_millions"][str(k)]


def test_patch_subspace_size():
    for k in range(1, 6):
        d = Discretization(4, k)
        J = patch_dofs(d, (2, 2, 2))
        assert len(J) == 3 * (2 * k + 1) * (2 * k + 2) ** 2 + (2 * k + 2) ** 3
        assert d.free_mask()[J].all()
    # the patches of one colour share no DoF (Sec. 3.1: they can run in parallel)
    d = Discretization(6, 2)
    for colour in range(8):
        seen = np.zeros(d.N, dtype=int)
        for v in colour_vertices(6, colour):
            seen[patch_dofs(d, v)] += 1
        assert seen.max() == 1


# ------------------------------------------------- Kronecker form (Sec. 2.3)
def _one_d(n, k, nu, gamma):
    """Global 1D matrices by 1D Gauss quadrature, written independently of the oracle."""
    h = 1.0 / n
    m = n * (k + 1)
    zc = gauss_lobatto(k + 2)[0]
    zd = gauss_legendre(k + 1)[0]
    xq, wq = gauss_legendre(k + 4)
    Vc, Dc = lagrange(zc, xq)
    Vd, Dd = lagrange(zd, xq)
    LC = np.zeros((m + 1, m + 1))
    MC = np.zeros((m + 1, m + 1))
    Dv = np.zeros((m, m + 1))
    LD = np.zeros((m, m))
    MD = np.zeros((m, m))
    for c in range(n):
        ic = c * (k + 1) + np.arange(k + 2)
        idd = c * (k + 1) + np.arange(k + 1)
        LC[np.ix_(ic, ic)] += (Dc * wq) @ Dc.T / h
        MC[np.ix_(ic, ic)] += (Vc * wq) @ Vc.T * h
        Dv[np.ix_(idd, ic)] += (Vd * wq) @ Dc.T
        LD[np.ix_(idd, idd)] += (Dd * wq) @ Dd.T / h
        MD[np.ix_(idd, idd)] += (Vd * wq) @ Vd.T * h
    # traces of the discontinuous basis at both ends of a cell (physical derivatives)
    V0, D0 = lagrange(zd, [0.0])
    V1, D1 = lagrange(zd, [1.0])
    v0, v1, d0, d1 = V0[:, 0], V1[:, 0], D0[:, 0] / h, D1[:, 0] / h
    for f in range(1, n):  # interior point between cells f-1 (-) and f (+), n = +1
        im = (f - 1) * (k + 1) + np.arange(k + 1)
        ip = f * (k + 1) + np.arange(k + 1)
        jump = np.zeros(m)  # [[phi]] = phi^- - phi^+
        avg = np.zeros(m)  # {{phi'}}
        jump[im] += v1
        jump[ip] -= v0
        avg[im] += 0.5 * d1
        avg[ip] += 0.5 * d0
        LD += gamma * np.outer(jump, jump) - np.outer(jump, avg) - np.outer(avg, jump)
    for side in (0, 1):
        idx = (0 if side == 0 else n - 1) * (k + 1) + np.arange(k + 1)
        val = np.zeros(m)
        dn = np.zeros(m)
        val[idx] = v0 if side == 0 else v1
        dn[idx] = -d0 if side == 0 else d1
        LD += 2 * gamma * np.outer(val, val) - np.outer(val, dn) - np.outer(dn, val)
    return LC, MC, Dv, LD, MD


def kron_stokes(n, k, nu=1.0, penalty_factor=1.0):
    gamma = penalty_factor * (k + 1) * (k + 2) * n
    LC, MC, Dv, LD, MD = _one_d(n, k, nu, gamma)
    kr = lambda a, b, c: sp.kron(sp.kron(sp.csr_matrix(a), sp.csr_matrix(b)), sp.csr_matrix(c))
    # kron(z, y, x): x is the fastest index
    Ax = nu * (kr(MD, MD, LC) + kr(MD, LD, MC) + kr(LD, MD, MC))
    Ay = nu * (kr(MD, LC, MD) + kr(MD, MC, LD) + kr(LD, MC, MD))
    Az = nu * (kr(LC, MD, MD) + kr(MC, MD, LD) + kr(MC, LD, MD))
    Bx = kr(MD, MD, Dv)
    By = kr(MD, Dv, MD)
    Bz = kr(Dv, MD, MD)
    B = sp.hstack([Bx, By, Bz])
    A = sp.bmat([[sp.block_diag([Ax, Ay, Az]), B.T], [B, None]]).tocsr()
    return A


@pytest.mark.parametrize("n,k,nu,pf", [(2, 1, 1.0, 1.0), (3, 2, 0.7, 1.0), (2, 3, 1.0, 2.5), (4, 1, 2.0, 1.0), (2, 5, 1.0, 1.0)])
def test_assembly_equals_kronecker_form(n, k, nu, pf):
    d = Discretization(n, k, nu, pf)
    A = d.assemble()
    K = kron_stokes(n, k, nu, pf)
    f = sp.diags(d.free_mask().astype(float))
    K = (f @ K @ f).tocsr()
    diff = abs(A - K).max()
    assert diff <= 1e-13 * abs(K).max(), diff


def test_symmetry_nullspace_coercivity():
    for n, k in [(2, 2), (3, 1), (2, 4)]:
        d = Discretization(n, k)
        A = d.assemble()
        assert abs(A - A.T).max() < 1e-13 * abs(A).max()
        one = np.zeros(d.N)
        one[d.offsets[3]:] = 1
        assert np.abs(A @ one).max() < 1e-13 * abs(A).max()  # B^T 1 = 0
        f = d.free_mask().copy()
        f[d.offsets[3]:] = False
        ev = np.linalg.eigvalsh(A[f][:, f].toarray())
        assert ev.min() > 0  # SIPG velocity block is coercive with this penalty


@pytest.mark.parametrize("n,k", [(2, 2), (3, 2), (2, 3)])
def test_smooth_field_energy_and_divergence(n, k):
    """u_c = b(x)b(y)b(z), b = s(1-s), lies in V_h and H^1_0: a_h(u,u) = |grad u|^2 = 1/300;
    with q = x:  (q, div u) = -int u_x = -1/216 (integration by parts)."""
    d = Discretization(n, k)
    A = d.assemble()
    u = np.zeros(d.N)
    h, k1 = d.h, k + 1
    for c in range(4):
        E = d.ext[c]
        g = np.arange(E[0] * E[1] * E[2])
        idx = [g % E[0], (g // E[0]) % E[1], g // (E[0] * E[1])]
        X = []
        for dd in range(3):
            if c == dd:
                cell = np.minimum(idx[dd] // k1, n - 1)
                X.append((cell + d.zC[idx[dd] - cell * k1]) * h)
            else:
                X.append((idx[dd] // k1 + d.zD[idx[dd] % k1]) * h)
        if c < 3:
            u[d.offsets[c] + g] = X[0] * (1 - X[0]) * X[1] * (1 - X[1]) * X[2] * (1 - X[2])
        else:
            q = np.zeros(d.N)
            q[d.offsets[3] + g] = X[0]
    assert abs(u @ (A @ u) - 1.0 / 300.0) < 1e-12
    assert abs(q @ (A @ u) - (-1.0 / 216.0)) < 1e-13


@pytest.mark.parametrize("n,k,pf", [(2, 1, 1.0), (3, 2, 1.7)])
def test_boundary_penalty_closed_form(n, k, pf):
    """u = (b(x), 0, 0), b = s(1-s), has zero normal trace but tangential
    trace b(x) on the four faces y, z in {0, 1}, where d_n u = 0; the Nitsche
    terms of eq. `bilinear` add 2 gamma int b^2 = 2 gamma / 30 per face:
    a_h(u, u) = 1/3 + 8 gamma / 30."""
    d = Discretization(n, k, 1.0, pf)
    E = d.ext[0]
    g = np.arange(E[0] * E[1] * E[2])
    i0 = g % E[0]
    cell = np.minimum(i0 // (k + 1), n - 1)
    x = (cell + d.zC[i0 - cell * (k + 1)]) * d.h
    u = np.zeros(d.N)
    u[g] = x * (1 - x)
    assert abs(u @ (d.assemble() @ u) - (1.0 / 3.0 + 8.0 * d.gamma / 30.0)) < 1e-12 * d.gamma


def test_pressure_weights_integrate_polynomials():
    """The weights of the zero-mean pressure projection are int psi_i: they
    integrate every field of the pressure space exactly, e.g. x^a y^b z^c with
    a, b, c <= k (integral 1 / ((a+1)(b+1)(c+1)))."""
    for n, k in [(2, 1), (3, 2)]:
        d = Discretization(n, k)
        W = d.pressure_weights()
        m = d.m
        g = np.arange(m)
        x = (g // (k + 1) + d.zD[g % (k + 1)]) * d.h
        X = [np.kron(np.ones(m * m), x), np.kron(np.kron(np.ones(m), x), np.ones(m)), np.kron(x, np.ones(m * m))]
        for a, b, c in [(0, 0, 0), (k, 0, 0), (0, k, 1), (1, 1, k)]:
            assert abs(W @ (X[0] ** a * X[1] ** b * X[2] ** c) - 1.0 / ((a + 1) * (b + 1) * (c + 1))) < 1e-14


def test_apply_rows_matches_assembly():
    d = Discretization(3, 2)
    A = d.assemble()
    x = random_vector(7, d.N) * d.free_mask()
    rows = np.arange(0, d.N, 37)
    assert np.abs(d.apply_rows(x, rows) - (A @ x)[rows]).max() < 1e-13 * np.abs(A @ x).max()


@pytest.mark.parametrize("n,k,vertex", [(4, 2, (2, 2, 2)), (4, 2, (1, 2, 3)), (5, 1, (4, 1, 2)), (4, 3, (3, 3, 1))])
def test_local_rows_of_a_patch_match_assembly(n, k, vertex):
    """The rows of the patch DoFs built from the patch's eight cells and their
    faces alone equal those rows of the globally assembled matrix, for an
    interior patch and for patches touching the boundary: the route the
    full-size smoother checks take, pinned against the global assembly."""
    d = Discretization(n, k)
    A = d.assemble()
    J = patch_dofs(d, vertex)
    cells = [(vertex[0] - 1 + a, vertex[1] - 1 + b, vertex[2] - 1 + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    cols, K = d.local_rows(cells)
    pos = np.searchsorted(cols, J)
    assert np.array_equal(cols[pos], J)
    ref = A[J][:, cols].toarray()
    got = K[pos].toarray()
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    # and nothing outside cols couples to the patch rows
    outside = np.setdiff1d(np.arange(d.N), cols)
    assert A[J][:, outside].nnz == 0


# ---------------------------------------------------- manufactured solution
def test_manufactured_solution_properties():
    man = Manufactured(manufactured_coefficients(0), nu=1.3)
    rng = np.random.default_rng(3)
    X = rng.uniform(0.05, 0.95, (20, 3))
    x, y, z = X.T
    e = 1e-4
    # divergence free (central differences of u)
    div = 0.0
    for c in range(3):
        dp = X.copy()
        dm = X.copy()
        dp[:, c] += e
        dm[:, c] -= e
        div = div + (man.velocity(*dp.T)[:, c] - man.velocity(*dm.T)[:, c]) / (2 * e)
    assert np.abs(div).max() < 1e-6
    # forcing = -nu Lap u + grad p against finite differences
    lap = np.zeros((20, 3))
    for c in range(3):
        dp = X.copy()
        dm = X.copy()
        dp[:, c] += e
        dm[:, c] -= e
        lap += (man.velocity(*dp.T) - 2 * man.velocity(*X.T) + man.velocity(*dm.T)) / e ** 2
    gp = np.stack([(man.pressure(*(X + e * np.eye(3)[c]).T) - man.pressure(*(X - e * np.eye(3)[c]).T)) / (2 * e) for c in range(3)], 1)
    assert np.abs(man.forcing(x, y, z) - (-1.3 * lap + gp)).max() < 1e-4 * (1 + np.abs(lap).max())
    # no-slip boundary
    B = rng.uniform(0, 1, (10, 3))
    for c in range(3):
        for v in (0.0, 1.0):
            P = B.copy()
            P[:, c] = v
            assert np.abs(man.velocity(*P.T)).max() < 1e-14


# -------------------------------------------------------------- transfers
@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_is_the_embedding(k):
    C, F = Discretization(2, k), Discretization(4, k)
    P = prolongation(C, F)
    xc = random_vector(11, C.N) * C.free_mask()
    pts = np.random.default_rng(5).uniform(0, 1, (25, 3))
    uc, pc = C.evaluate(xc, pts)
    uf, pf = F.evaluate(P @ xc, pts)
    assert np.abs(uc - uf).max() < 1e-13 and np.abs(pc - pf).max() < 1e-13
    # interpolants of a coarse-space function match node by node
    man = Manufactured(manufactured_coefficients(1))
    Ic = interpolate(C, man)
    If_from_c = P @ Ic
    uu, pp = C.evaluate(Ic, pts)
    uu2, pp2 = F.evaluate(If_from_c, pts)
    assert np.abs(uu - uu2).max() < 1e-13


@pytest.mark.parametrize("n,k,nu,pf", [(2, 1, 1.0, 1.0), (2, 2, 0.7, 1.3), (3, 2, 1.0, 1.0), (2, 3, 1.0, 1.0)])
def test_galerkin_product_is_the_coarse_matrix_with_doubled_penalty(n, k, nu, pf):
    """The spaces are nested (Sec. 3), so for coarse functions the fine form
    differs from the coarse one only through the penalty gamma_e ~ 1/h, twice
    as large on the fine mesh; jumps across fine faces inside a coarse cell
    vanish.  Hence P^T A_fine P is the coarse matrix assembled with twice the
    penalty factor, and its divergence blocks are the coarse ones."""
    C, F = Discretization(n, k, nu, pf), Discretization(2 * n, k, nu, pf)
    P = prolongation(C, F)
    G = (P.T @ F.assemble() @ P).tocsr()
    A2 = Discretization(n, k, nu, 2 * pf).assemble()
    assert abs(G - A2).max() <= 1e-13 * abs(A2).max()
    A1 = C.assemble()
    p0 = C.offsets[3]
    assert abs(G[p0:] - A1[p0:]).max() <= 1e-13 * abs(A1).max()
    # the velocity block does depend on the penalty: the identity is not vacuous
    assert abs(G - A1).max() > 0.1 * abs(A1).max()


# ---------------------------------------------------------- local solvers
def test_direct_local_solver_is_exact_on_one_patch():
    """On the 2^3 mesh the single vertex patch holds every free DoF: one
    smoothing step with the Direct solver solves the system exactly."""
    H = Hierarchy(2, 2)
    d = H.levels[0].disc
    b = rhs(d, Manufactured(manufactured_coefficients(2)))
    x = H.smooth(0, np.zeros(d.N), b)
    assert np.linalg.norm(H.levels[0].A @ x - b) < 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("k", [1, 2])
def test_each_colour_leaves_its_patch_in_equilibrium(k):
    """On the 3^3 mesh every colour holds one vertex patch.  After a colour's
    update (Algorithm 2, exact local solver) the residual on that patch's DoFs
    is zero in the velocity and a constant in the pressure (the local kernel).
    After a whole step only the last colour's patch is in equilibrium, which
    pins the ascending colour order."""
    H = Hierarchy(3, k)
    d = H.levels[0].disc
    A = H.levels[0].A
    npress = (2 * k + 2) ** 3
    b = random_vector(19, d.N) * d.free_mask()
    x0 = random_vector(20, d.N) * d.free_mask()

    def imbalance(x, colour):
        (v,) = colour_vertices(3, colour)
        res = (b - A @ x)[patch_dofs(d, v)]
        return max(np.abs(res[:-npress]).max(), np.ptp(res[-npress:])) / np.abs(b).max()

    x = x0.copy()
    for colour in range(8):
        H.smooth_colour(0, colour, x, b)
        assert imbalance(x, colour) < 1e-12
    assert np.array_equal(x, H.smooth(0, x0, b))
    assert imbalance(x, 7) < 1e-12 and imbalance(x, 0) > 1e-3


@pytest.mark.parametrize("k", [1, 2])
def test_schur_cg_minimises_the_energy_error(k):
    """Sec. 3.2: the pressure after j CG steps on S P = g (S = B A^-1 B^T,
    g = B A^-1 F - G made mean-free) is the S-energy-best approximation of
    the exact P in the Krylov space span{g, S g, ..., S^(j-1) g}; the velocity
    is then A^-1 (F - B^T P).  Brute force by the Galerkin condition on an
    orthonormal basis of the explicit Krylov vectors."""
    n = 3
    d = Discretization(n, k)
    A = d.assemble()
    (v,) = colour_vertices(n, 5)
    J = patch_dofs(d, v)
    Aj = A[J][:, J].toarray()
    npress = (2 * k + 2) ** 3
    nv = len(J) - npress
    r = random_vector(29, d.N)[J]
    F, G = r[:nv], r[nv:]
    Av = Aj[:nv, :nv]
    B = Aj[nv:, :nv]
    S = B @ np.linalg.solve(Av, B.T)
    g = B @ np.linalg.solve(Av, F) - G
    g = g - g.mean()
    Pstar = np.linalg.lstsq(S, g, rcond=None)[0]
    Pstar = Pstar - Pstar.mean()
    Ainv = lambda w: np.linalg.solve(Av, w)
    for j in range(1, 6):
        K = [g]
        for _ in range(j - 1):
            K.append(S @ K[-1])
        Q = np.linalg.qr(np.stack(K, 1))[0]
        Pj = Q @ np.linalg.solve(Q.T @ S @ Q, Q.T @ g)
        out = schur_cg(Ainv, B, F, G, "schur", j)
        assert np.abs(out[nv:] - Pj).max() <= 1e-9 * np.abs(Pj).max(), j
        assert np.abs(out[:nv] - Ainv(F - B.T @ Pj)).max() <= 1e-9 * np.abs(out[:nv]).max()
        # the energy error decreases strictly along the iteration
        e = Pj - Pstar
        err = e @ S @ e
        if j > 1:
            assert err < prev
        prev = err


def test_coarse_solve_is_exact():
    """Sec. 3: the coarsest level (2^3 or 3^3 cells) is solved exactly: for a
    consistent b = A x the solve returns x up to a constant pressure, and the
    bordered system fixes that constant to a zero coefficient sum."""
    for n, k in [(2, 1), (2, 3), (3, 1), (3, 2)]:
        H = Hierarchy(n, k)
        d = H.levels[0].disc
        A = H.levels[0].A
        xt = random_vector(21, d.N) * d.free_mask()
        x = H.coarse_solve(A @ xt)
        p0 = d.offsets[3]
        assert np.abs(x[:p0] - xt[:p0]).max() < 1e-10 * np.abs(xt).max()
        dp = x[p0:] - xt[p0:]
        assert np.ptp(dp) < 1e-10 * np.abs(xt).max()
        assert abs(x[p0:].sum()) < 1e-10 * np.abs(xt).max() * len(dp)


@pytest.mark.parametrize("n,k", [(3, 1), (4, 2), (3, 3)])
def test_schur_cg_equals_direct(n, k):
    d = Discretization(n, k)
    A = d.assemble()
    r = random_vector(13, d.N) * d.free_mask()
    npress = (2 * k + 2) ** 3
    lu, sc = LocalSolver("lu"), LocalSolver(("schur_tol", 1e-15))
    for v in colour_vertices(n, 0) + colour_vertices(n, 7):
        J = patch_dofs(d, v)
        Aj = A[J][:, J].toarray()
        x1 = lu(Aj, npress, r[J])
        x2 = sc(Aj, npress, r[J])
        assert np.abs(x1 - x2).max() < 1e-10 * np.abs(x1).max()
        # the corrected local residual is the constant-pressure component only
        res = r[J] - Aj @ x1
        assert np.abs(res[:-npress]).max() < 1e-11 * np.abs(r[J]).max()
        assert np.ptp(res[-npress:]) < 1e-11 * np.abs(r[J]).max()


# ------------------------------------------------ solver and discretization
@pytest.mark.slow
def test_convergence_divergence_and_flat_iterations():
    """k = 2 on n = 4, 8: optimal L2 rates (k+1) for velocity and pressure,
    pointwise divergence-free velocity, GMRES steps flat under refinement."""
    man = Manufactured(manufactured_coefficients(0))
    errs, its = [], []
    for n in (4, 8):
        H = Hierarchy(n, 2)
        d = H.levels[-1].disc
        x, info = H.solve(rhs(d, man), tol=1e-11)
        assert info["converged"]
        errs.append(l2_errors(d, man, x))
        its.append(info["iterations"])
        pts = np.random.default_rng(9).uniform(0, 1, (30, 3))
        assert np.abs(d.divergence(x, pts)).max() < 1e-9
    ru = math.log2(errs[0][0] / errs[1][0])
    rp = math.log2(errs[0][1] / errs[1][1])
    assert ru > 2.7 and rp > 2.7, (ru, rp)
    assert abs(its[1] - its[0]) <= 2


@pytest.mark.slow
def test_optimal_rates_k3():
    """k = 3 on n = 4, 8 (about 80 s): L2 rates near k+1 = 4 for velocity and
    pressure (observed 3.7 and 4.0; the 2 -> 4 step is still pre-asymptotic
    for the pressure)."""
    man = Manufactured(manufactured_coefficients(0))
    errs = []
    for n in (4, 8):
        H = Hierarchy(n, 3)
        d = H.levels[-1].disc
        x, info = H.solve(rhs(d, man), tol=1e-12)
        assert info["converged"]
        errs.append(l2_errors(d, man, x))
    ru = math.log2(errs[0][0] / errs[1][0])
    rp = math.log2(errs[0][1] / errs[1][1])
    assert ru > 3.4 and rp > 3.6, (ru, rp)


def test_three_steps_for_k3():
    """Sec. 3.3: from k = 3 on, no more than three GMRES steps to 1e-8."""
    H = Hierarchy(4, 3)
    d = H.levels[-1].disc
    _, info = H.solve(rhs(d, Manufactured(manufactured_coefficients(0))), tol=1e-8)
    assert info["iterations"] <= GOLDEN["max_gmres_steps_k_ge_3"]["value"]
    assert info["nu"] <= 3.0


@pytest.mark.parametrize("restart", [20, 2])
def test_fgmres_minimises_the_residual(restart):
    """The V-cycle from x0 = 0 is a fixed linear map M, so flexible GMRES is
    right-preconditioned GMRES: within a restart cycle from residual r its
    j-th residual is min_c ||r - [A M w_0, ..., A M w_{j-1}] c|| over the
    Krylov vectors w_0 = r, w_{i+1} = A M w_i.  Brute force by least squares
    on those vectors, restart by restart."""
    H = Hierarchy(4, 1)
    d = H.levels[-1].disc
    A = H.levels[-1].A
    b = A @ (random_vector(23, d.N) * d.free_mask())
    steps = 4
    _, info = H.solve(b, tol=1e-30, restart=restart, maxit=steps)
    bnorm = np.linalg.norm(b)
    x = np.zeros(d.N)
    hist = [1.0]
    while len(hist) <= steps:
        r = b - A @ x
        W, Z = [r / np.linalg.norm(r)], []
        for _ in range(min(restart, steps + 1 - len(hist))):
            Z.append(H.vcycle(W[-1]))
            w = A @ Z[-1]
            W.append(w / np.linalg.norm(w))
            K = np.stack(W[1:], 1)
            c = np.linalg.lstsq(K, r, rcond=None)[0]
            hist.append(np.linalg.norm(r - K @ c) / bnorm)
        for zi, ci, wn in zip(Z, c, [np.linalg.norm(A @ z) for z in Z]):
            x = x + (ci / wn) * zi
    got = np.array(info["residuals"])
    ref = np.array(hist)
    assert len(got) == steps + 1
    assert np.all(np.abs(got - ref) <= 1e-10 + 1e-6 * ref), (got, ref)
    assert ref[-1] < 1e-3  # the V-cycle preconditioner is doing its job


@pytest.mark.parametrize("k,local", [(2, "lu"), (2, ("schur", 15)), (4, "lu")])
def test_table2_three_steps_to_1e6(k, local):
    """Table 2: three GMRES steps reach a relative residual of 1e-6 for RT_2
    and RT_4 (quoted on 32^3 cells; the counts are flat under refinement,
    Sec. 3.3, so the 4^3 mesh stands in), with the Direct (exact) and the
    Schur-complement local solver."""
    H = Hierarchy(4, k, local=local)
    d = H.levels[-1].disc
    _, info = H.solve(rhs(d, Manufactured(manufactured_coefficients(0))), tol=1e-6)
    assert info["converged"]
    assert info["iterations"] <= GOLDEN["table2_iterations_tol_1e-6"][str(k)]


def test_fractional_iteration_count_definition():
    # reduction of exactly 1e-8 in n steps gives nu = n (Sec. 3.3, read with a division)
    n = 3
    rbar = (1e-8) ** (1.0 / n)
    assert abs(-8.0 / math.log10(rbar) - n) < 1e-12
