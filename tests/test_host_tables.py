"""Host logic of the library, checked without a GPU: the 1D fast-diagonalization
eigenpairs that stk_setup builds for the vertex-patch local solver (Sec. 3.2,
eq. `inverse2d`, eq. `fast_inverse`), read through stk_patch_eigen, the 1D
cell matrices of the operator apply (Sec. 2.3), read through stk_cell_tables,
and the 1D child matrices of the level transfers (Sec. 3), read through
stk_transfer_tables.

The 1D patch operators are taken as principal submatrices of global 1D
matrices assembled independently in tests/test_oracle_pins.py (its Kronecker
check builds them by 1D Gauss quadrature); the library's tables must satisfy
K S = M S diag(lambda), S^T M S = I, lambda > 0, and, where it reports the
even-odd order, have reflection-symmetric columns first and antisymmetric ones
after.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from test_oracle_pins import _one_d


@pytest.fixture(scope="module")
def binding():
    from paper_2410_09497_gb300 import build

    build.build()
    import paper_2410_09497_gb300 as m

    return m


def _patch_operators(n, k, pf, direction):
    """(K, M) of one 1D patch operator from the global 1D matrices (nu removed)."""
    gamma = pf * (k + 1) * (k + 2) * n
    LC, MC, _, LD, MD = _one_d(n, k, 1.0, gamma)
    k1 = k + 1
    if direction == 0:  # vertex 2 of a 4-cell line: the interior nodes of cells 1 and 2
        idx = np.arange(k1 + 1, 3 * k1)
        return LC[np.ix_(idx, idx)], MC[np.ix_(idx, idx)]
    first = {1: 1, 2: 0, 3: n - 2, 4: 0}[direction]  # lower cell of the patch
    idx = np.arange(first * k1, (first + 2) * k1)
    return LD[np.ix_(idx, idx)], MD[np.ix_(idx, idx)]


CASES = [(4, 0), (4, 1), (4, 2), (4, 3), (2, 4)]  # direction 4 (both boundaries) needs n = 2


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,direction", CASES)
def test_fdm_eigenpairs(binding, k, n, direction):
    nu, pf = (2.5, 1.5) if k == 3 else (1.0, 1.0)
    S, lam, eo = binding.patch_eigen(n, k, direction, nu=nu, penalty_factor=pf)
    K, M = _patch_operators(n, k, pf, direction)
    dim = 2 * k + 1 if direction == 0 else 2 * k + 2
    assert S.shape == (dim, dim) and K.shape == (dim, dim)
    scale = np.abs(K).max()
    assert np.abs(K @ S - M @ S * lam).max() <= 1e-11 * scale * np.abs(S).max()
    assert np.abs(S.T @ M @ S - np.eye(dim)).max() <= 1e-12
    assert lam.min() > 0  # continuous stiffness with both end nodes removed / coercive SIPG
    # the operators of direction 0, 1 (interior) and 4 (both boundaries) are
    # symmetric under the reflection of the patch, those of 2 and 3 are not
    assert eo == (direction in (0, 1, 4))
    if eo:
        R = S[::-1]
        ne = (dim + 1) // 2
        assert np.abs(R[:, :ne] - S[:, :ne]).max() <= 1e-10 * np.abs(S).max()
        assert np.abs(R[:, ne:] + S[:, ne:]).max() <= 1e-10 * np.abs(S).max()


def test_patch_eigen_rejects_invalid_arguments(binding):
    lib = binding.load_library()
    S = np.zeros(144)
    lam = np.zeros(12)
    import ctypes

    d, e = ctypes.c_int(), ctypes.c_int()
    args = lambda n, k, nu, pf, dirn: lib.stk_patch_eigen(n, k, nu, pf, dirn, S.ctypes.data, lam.ctypes.data, ctypes.byref(d), ctypes.byref(e))
    assert args(4, 0, 1.0, 1.0, 0) == -1
    assert args(4, 6, 1.0, 1.0, 0) == -1
    assert args(1, 2, 1.0, 1.0, 0) == -1
    assert args(4, 2, 0.0, 1.0, 0) == -1
    assert args(4, 2, 1.0, -1.0, 0) == -1
    assert args(4, 2, 1.0, 1.0, 5) == -1
    assert b"direction" in lib.stk_last_error(None)
    assert lib.stk_patch_eigen(4, 2, 1.0, 1.0, 0, None, lam.ctypes.data, ctypes.byref(d), ctypes.byref(e)) == -1
    assert args(4, 2, 1.0, 1.0, 1) == 0 and d.value == 6


def _type_direction(vertex_index, n):
    """stk_patch_eigen direction of a discontinuous direction from the patch's
    position: 1 + (lower cell on the mesh boundary) + 2 (upper cell on it)."""
    return 1 + (1 if vertex_index == 1 else 0) + (2 if vertex_index == n - 1 else 0)


@pytest.mark.parametrize("n,k,vertex,nu", [(4, 1, (2, 2, 2), 1.0), (4, 2, (3, 1, 2), 1.0), (4, 3, (2, 1, 3), 2.5), (2, 2, (1, 1, 1), 1.0), (3, 2, (1, 2, 1), 0.7)])
def test_fdm_inverse_equals_the_oracle_patch_block(binding, n, k, vertex, nu):
    """Sec. 3.2, eq. `fast_inverse`: for each velocity component c, with the
    library's 1D eigenpairs (the continuous direction c, and the patch's
    boundary types in the other two), (S_z (x) S_y (x) S_x)
    diag(1 / nu (l_z + l_y + l_x)) (S_z (x) S_y (x) S_x)^T is the inverse of
    the u_c block of the patch matrix that the oracle assembles by quadrature."""
    from oracle.discretization import Discretization
    from oracle.multigrid import patch_dofs

    d = Discretization(n, k, nu)
    A = d.assemble()
    J = patch_dofs(d, vertex)
    n0 = (2 * k + 1) * (2 * k + 2) ** 2
    rng = np.random.default_rng(41)
    for c in range(3):
        Jc = J[c * n0:(c + 1) * n0]
        Au = A[Jc][:, Jc].toarray()
        S1, l1 = [], []
        for dirn in range(3):  # x, y, z
            S_d, l_d, _ = binding.patch_eigen(n, k, 0 if dirn == c else _type_direction(vertex[dirn], n), nu=nu)
            S1.append(S_d)
            l1.append(l_d)
        S = np.kron(S1[2], np.kron(S1[1], S1[0]))
        lam = nu * np.add.outer(np.add.outer(l1[2], l1[1]), l1[0]).reshape(-1)
        r = rng.standard_normal(n0)
        fdm = S @ ((S.T @ r) / lam)
        ref = np.linalg.solve(Au, r)
        assert np.abs(fdm - ref).max() <= 1e-11 * np.abs(ref).max(), c


# ------------------------------------------------------------ operator tables
# The 1D cell matrices of the operator apply (Sec. 2.3), read through
# stk_cell_tables, assembled into global 1D matrices and compared with the
# independent 1D assembly of tests/test_oracle_pins.py (whose Kronecker sum
# equals the oracle's literal assembly of eq. `bilinear`).


def _assemble_from_cells(t, n, k):
    nc, nd = k + 2, k + 1
    m = n * nd
    KC = np.zeros((m + 1, m + 1))
    MC = np.zeros((m + 1, m + 1))
    D = np.zeros((m, m + 1))
    L = np.zeros((m, m))
    for c in range(n):
        ic = c * nd + np.arange(nc)
        idd = c * nd + np.arange(nd)
        KC[np.ix_(ic, ic)] += t["KC"]
        MC[np.ix_(ic, ic)] += t["MC"]
        D[np.ix_(idd, ic)] += t["D"]
        L[np.ix_(idd, idd)] += t["LS"][1 if c == 0 else (2 if c == n - 1 else 0)]
        if c > 0:
            L[np.ix_(idd, idd - nd)] += t["LLO"]
        if c < n - 1:
            L[np.ix_(idd, idd + nd)] += t["LHI"]
    return KC, MC, D, L, np.diag(np.tile(t["S"], n))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,nu,pf", [(2, 1.0, 1.0), (3, 0.5, 2.0), (5, 2.0, 1.0)])
def test_cell_tables_assemble_to_the_global_1d_operators(binding, n, k, nu, pf):
    # n = 2 has no interior cell; LS[0] is checked by n = 3 and 5
    t = binding.cell_tables(n, k, nu=nu, penalty_factor=pf)
    gamma = pf * (k + 1) * (k + 2) * n
    LC, MC, Dv, LD, MD = _one_d(n, k, 1.0, gamma)
    KCg, MCg, Dg, Lg, Sg = _assemble_from_cells(t, n, k)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(KCg, nu * LC) < 1e-12
    assert rel(MCg, MC) < 1e-12
    assert rel(Dg, Dv) < 1e-12
    assert rel(Lg, nu * LD) < 1e-12
    assert rel(Sg, MD) < 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_cell_tables_reflection_symmetry(binding, k):
    """The node sets are symmetric under the cell's reflection, so KC, MC and
    the interior penalty block are centro-symmetric, D is antisymmetric, the
    two boundary blocks and the two coupling blocks are each other's
    reflections, and the Gauss mass is symmetric: the structure an even-odd
    evaluation of the apply uses."""
    t = binding.cell_tables(4, k, nu=1.3, penalty_factor=1.0)
    R = lambda a: a[::-1, ::-1]
    close = lambda a, b: np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert close(R(t["KC"]), t["KC"]) and close(R(t["MC"]), t["MC"])
    assert close(R(t["LS"][0]), t["LS"][0]) and close(R(t["LS"][1]), t["LS"][2])
    assert close(R(t["LLO"]), t["LHI"])
    assert close(R(t["D"]), -t["D"])
    assert close(t["S"][::-1], t["S"])


def test_cell_tables_rejects_invalid_arguments(binding):
    import ctypes

    lib = binding.load_library()
    buf = np.zeros(1024)
    assert lib.stk_cell_tables(4, 0, 1.0, 1.0, buf.ctypes.data) == -1
    assert lib.stk_cell_tables(4, 6, 1.0, 1.0, buf.ctypes.data) == -1
    assert lib.stk_cell_tables(1, 2, 1.0, 1.0, buf.ctypes.data) == -1
    assert lib.stk_cell_tables(4, 2, 0.0, 1.0, buf.ctypes.data) == -1
    assert lib.stk_cell_tables(4, 2, 1.0, -1.0, buf.ctypes.data) == -1
    assert lib.stk_cell_tables(4, 2, 1.0, 1.0, None) == -1
    assert b"cell_tables" in lib.stk_last_error(None)
    assert lib.stk_cell_tables(4, 2, 1.0, 1.0, ctypes.c_void_p(buf.ctypes.data)) == 0


# ------------------------------------------------------------ transfer tables
# The 1D child matrices of the level transfers (Sec. 3), read through
# stk_transfer_tables, put together the way the transfer kernels use them (a
# fine node is the lower k+1 nodes of a child along every direction; the
# upper end node of the continuous direction is a constrained boundary node)
# must give the oracle's prolongation matrix, built by evaluating the coarse
# basis at every fine support point.


def _prolongation_from_tables(PC, PD, nc_cells, k):
    nd = k + 1
    mc, mf = nc_cells * nd, 2 * nc_cells * nd
    P1 = {}
    for cont, T, ext_c, ext_f in ((True, PC, mc + 1, mf + 1), (False, PD, mc, mf)):
        M = np.zeros((ext_f, ext_c))
        nb = T.shape[2]
        for c in range(nc_cells):
            for ch in range(2):
                for a in range(nd):
                    M[(2 * c + ch) * nd + a, c * nd + np.arange(nb)] = T[ch, a]
        P1[cont] = M
    blocks = []
    for comp in range(4):
        f = [P1[d == comp] for d in range(3)]
        blocks.append(sp.kron(sp.kron(sp.csr_matrix(f[2]), sp.csr_matrix(f[1])), sp.csr_matrix(f[0])))
    return sp.block_diag(blocks).tocsr()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("nc_cells", [1, 2, 3])
def test_transfer_tables_give_the_oracle_embedding(binding, nc_cells, k):
    from oracle.discretization import Discretization
    from oracle.transfer import prolongation

    PC, PD = binding.transfer_tables(k)
    coarse, fine = Discretization(nc_cells, k), Discretization(2 * nc_cells, k)
    Po = prolongation(coarse, fine).tocsr()
    Pt = _prolongation_from_tables(PC, PD, nc_cells, k)
    ff, fc = fine.free_mask(), coarse.free_mask()
    diff = (Pt - Po)[ff][:, fc]
    assert diff.nnz == 0 or np.abs(diff.data).max() < 1e-13 * np.abs(Po.data).max()
    # the oracle's rows and columns of constrained DoFs are zero
    assert Po[~ff].nnz == 0 or not Po[~ff].data.any()
    assert Po[:, ~fc].nnz == 0 or not Po[:, ~fc].data.any()


def test_transfer_tables_reject_invalid_arguments(binding):
    lib = binding.load_library()
    buf = np.zeros(512)
    assert lib.stk_transfer_tables(0, buf.ctypes.data) == -1
    assert lib.stk_transfer_tables(6, buf.ctypes.data) == -1
    assert lib.stk_transfer_tables(3, None) == -1
    assert b"transfer_tables" in lib.stk_last_error(None)
