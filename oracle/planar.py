"""The method on the unit square, for the two-dimensional results of Table 1 (test infrastructure only).

Sec. 4.1 reports fractional GMRES iteration counts of the method in two
dimensions (Table 1).  This module sets up the same discretization and solver
on n x n cells:

  * spaces (Sec. 2.1): velocity component c is continuous of degree k+1 in
    direction c (Gauss-Lobatto nodes) and discontinuous of degree k in the
    other direction (Gauss nodes); pressure DGQ_k.  Layout [u_x | u_y | p],
    x fastest; u_x on (m+1) x m nodes, u_y on m x (m+1), p on m x m,
    m = n (k+1); boundary normal entries are constrained to zero.
  * operator (eq. `weak_form`, eq. `bilinear`) in the Kronecker form the
    paper notes for Cartesian meshes (Sec. 2.3), written with x as the fast
    factor:
        A_x = nu (M_D (x) L_C + L_D (x) M_C),   A_y = nu (L_C (x) M_D + M_C (x) L_D),
        B_x = M_D (x) D,   B_y = D (x) M_D,    A = [[diag(A_x, A_y), B^T], [B, 0]].
    L_C, M_C: stiffness and mass of the continuous 1D basis; M_D: the
    (diagonal) Gauss mass; D_qa = (psi_q, phi_a'); L_D: the 1D
    interior-penalty operator, i.e. the cell stiffness plus, at every interior
    point, gamma [[u]][[v]] - {{u'}}[[v]] - [[u]]{{v'}} and, at the two ends,
    2 gamma u v - d_n u v - u d_n v (the terms of eq. `bilinear` along one
    direction).  gamma = penalty_factor (k+1)(k+2)/h as in three dimensions.
    All 1D integrals by the (k+3)-point Gauss rule of each cell (exact).
  * vertex patches of 2 x 2 cells around the interior vertices, in four
    colours (i mod 2) + 2 (j mod 2) (Sec. 3.1, Algorithm 2); the embedding as
    prolongation (Kronecker product of the 1D embeddings of each field) and
    its transpose as restriction; exact coarse solve on 2 x 2 (or 3 x 3)
    cells; V-cycle and FGMRES(20) as in three dimensions (`Hierarchy`).
  * right-hand side: the paper's 2D reference solution u = (d_y psi, -d_x psi),
    p = cos(2 pi x) cos(2 pi y), psi = phi(x) phi(y).  Its phi uses constants
    sigma, mu that the paper does not give; phi(s) = s^2 (1-s)^2 sin(pi s), a
    bump of the same shape centred at 1/2, replaces it (a reading).
    b_i = (f, phi_i) with f = -nu Laplace(u) + grad p, by the (k+3)-point
    Gauss rule per cell; pressure rows 0.

The 3D counterpart of the Kronecker identity is pinned against literal
quadrature; this module is pinned by closed forms, by the Galerkin identity of
the nested spaces and by Table 1 (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .basis import continuous_nodes, discontinuous_nodes, gauss_legendre, lagrange
from .manufactured import G
from .multigrid import Hierarchy


def one_d_matrices(n: int, k: int, gamma: float):
    """Global 1D matrices (L_C, M_C, D, L_D, M_D) on n cells of [0, 1]."""
    h = 1.0 / n
    m = n * (k + 1)
    zc, zd = continuous_nodes(k), discontinuous_nodes(k)
    xq, wq = gauss_legendre(k + 3)
    Vc, Dc = lagrange(zc, xq)
    Vd, Dd = lagrange(zd, xq)
    LC = np.zeros((m + 1, m + 1))
    MC = np.zeros((m + 1, m + 1))
    D = np.zeros((m, m + 1))
    LD = np.zeros((m, m))
    MD = np.zeros((m, m))
    for c in range(n):
        ic = c * (k + 1) + np.arange(k + 2)
        idd = c * (k + 1) + np.arange(k + 1)
        LC[np.ix_(ic, ic)] += (Dc * wq) @ Dc.T / h
        MC[np.ix_(ic, ic)] += (Vc * wq) @ Vc.T * h
        D[np.ix_(idd, ic)] += (Vd * wq) @ Dc.T
        LD[np.ix_(idd, idd)] += (Dd * wq) @ Dd.T / h
        MD[np.ix_(idd, idd)] += (Vd * wq) @ Vd.T * h
    V0, D0 = lagrange(zd, [0.0])
    V1, D1 = lagrange(zd, [1.0])
    lo_v, hi_v, lo_d, hi_d = V0[:, 0], V1[:, 0], D0[:, 0] / h, D1[:, 0] / h
    for f in range(1, n):  # the point between cell f-1 (minus side) and cell f (plus side)
        minus = (f - 1) * (k + 1) + np.arange(k + 1)
        plus = f * (k + 1) + np.arange(k + 1)
        jump = np.zeros(m)
        mean_d = np.zeros(m)
        jump[minus] += hi_v
        jump[plus] -= lo_v
        mean_d[minus] += 0.5 * hi_d
        mean_d[plus] += 0.5 * lo_d
        LD += gamma * np.outer(jump, jump) - np.outer(mean_d, jump) - np.outer(jump, mean_d)
    for end in (0, 1):
        cell = 0 if end == 0 else n - 1
        idx = cell * (k + 1) + np.arange(k + 1)
        val = np.zeros(m)
        dn = np.zeros(m)
        val[idx] = lo_v if end == 0 else hi_v
        dn[idx] = -lo_d if end == 0 else hi_d
        LD += 2 * gamma * np.outer(val, val) - np.outer(dn, val) - np.outer(val, dn)
    return LC, MC, D, LD, MD


def _load_1d(n: int, k: int, fn, continuous: bool) -> np.ndarray:
    """(g, phi_i) for the global continuous or discontinuous 1D basis."""
    h = 1.0 / n
    z = continuous_nodes(k) if continuous else discontinuous_nodes(k)
    xq, wq = gauss_legendre(k + 3)
    V, _ = lagrange(z, xq)
    m = n * (k + 1)
    out = np.zeros(m + 1 if continuous else m)
    for c in range(n):
        idx = c * (k + 1) + np.arange(len(z))
        out[idx] += V @ (wq * fn((c + xq) * h)) * h
    return out


class PlanarDiscretization:
    """DoF numbering and the Stokes matrix of one uniform n x n mesh at degree k."""

    def __init__(self, n: int, k: int, nu: float = 1.0, penalty_factor: float = 1.0):
        self.n, self.k, self.nu = int(n), int(k), float(nu)
        self.h = 1.0 / n
        self.m = n * (k + 1)
        self.gamma = penalty_factor * (k + 1) * (k + 2) / self.h
        m = self.m
        nv = (m + 1) * m
        self.ext = [(m + 1, m), (m, m + 1), (m, m)]
        self.offsets = [0, nv, 2 * nv]
        self.pressure_start = 2 * nv
        self.N = 2 * nv + m * m
        self._free = None

    def index(self, comp: int, i0, i1):
        return self.offsets[comp] + np.asarray(i0) + self.ext[comp][0] * np.asarray(i1)

    def free_mask(self) -> np.ndarray:
        if self._free is None:
            free = np.ones(self.N, dtype=bool)
            m = self.m
            for c in range(2):
                E = self.ext[c]
                g = np.arange(E[0] * E[1])
                i = (g % E[0]) if c == 0 else (g // E[0])
                free[self.offsets[c] + g[(i == 0) | (i == m)]] = False
            self._free = free
        return self._free

    def assemble(self) -> sp.csr_matrix:
        LC, MC, D, LD, MD = (sp.csr_matrix(a) for a in one_d_matrices(self.n, self.k, self.gamma))
        kr = sp.kron
        Ax = self.nu * (kr(MD, LC) + kr(LD, MC))
        Ay = self.nu * (kr(LC, MD) + kr(MC, LD))
        B = sp.hstack([kr(MD, D), kr(D, MD)])
        A = sp.bmat([[sp.block_diag([Ax, Ay]), B.T], [B, None]]).tocsr()
        f = sp.diags(self.free_mask().astype(np.float64))
        A = (f @ A @ f).tocsr()
        A.eliminate_zeros()
        return A

    def pressure_weights(self) -> np.ndarray:
        """int_Omega psi_i for every pressure DoF (Gauss weights x h^2)."""
        _, w = gauss_legendre(self.k + 1)
        g = np.arange(self.m)
        w1 = w[g % (self.k + 1)] * self.h
        return np.outer(w1, w1).reshape(-1)

    def rhs(self) -> np.ndarray:
        """Load vector of the reference solution (module docstring)."""
        n, k, nu = self.n, self.k, self.nu
        w = 2 * math.pi
        Gs = lambda j: (lambda s: G(1, s, j))
        b = np.zeros(self.N)
        # f_x = -nu (phi'' phi' + phi phi''')(x, y) - 2 pi sin(2 pi x) cos(2 pi y)
        terms_x = [(-nu, Gs(2), Gs(1)), (-nu, Gs(0), Gs(3)),
                   (-w, lambda s: np.sin(w * s), lambda s: np.cos(w * s))]
        # f_y = nu (phi''' phi + phi' phi'')(x, y) - 2 pi cos(2 pi x) sin(2 pi y)
        terms_y = [(nu, Gs(3), Gs(0)), (nu, Gs(1), Gs(2)),
                   (-w, lambda s: np.cos(w * s), lambda s: np.sin(w * s))]
        for c, terms in ((0, terms_x), (1, terms_y)):
            v = 0.0
            for a, gx, gy in terms:
                lx = _load_1d(n, k, gx, continuous=(c == 0))
                ly = _load_1d(n, k, gy, continuous=(c == 1))
                v = v + a * np.kron(ly, lx)
            b[self.offsets[c]:self.offsets[c] + v.size] = v
        return b * self.free_mask()


def planar_patch_dofs(disc: PlanarDiscretization, vertex) -> np.ndarray:
    """DoFs of the patch of the 2 x 2 cells around interior vertex (i, j):
    u_x, u_y without the normal DoFs on the patch boundary, then the pressure."""
    k1 = disc.k + 1
    out = []
    for c in range(3):
        rng = []
        for d in range(2):
            lo = (vertex[d] - 1) * k1
            rng.append(np.arange(lo + 1, lo + 2 * k1) if c == d else np.arange(lo, lo + 2 * k1))
        i1, i0 = np.meshgrid(rng[1], rng[0], indexing="ij")
        out.append(disc.index(c, i0, i1).reshape(-1))
    return np.concatenate(out)


def planar_colour_vertices(n: int, colour: int):
    bits = [(colour >> d) & 1 for d in range(2)]
    rng = [[i for i in range(1, n) if i % 2 == bits[d]] for d in range(2)]
    return [(i, j) for j in rng[1] for i in rng[0]]


def _embedding_1d(nc: int, k: int, continuous: bool) -> np.ndarray:
    """Values of the coarse 1D basis (nc cells) at the fine nodes (2 nc cells)."""
    z = continuous_nodes(k) if continuous else discontinuous_nodes(k)
    k1 = k + 1
    nf = 2 * nc
    size_f = nf * k1 + (1 if continuous else 0)
    size_c = nc * k1 + (1 if continuous else 0)
    E = np.zeros((size_f, size_c))
    for i in range(size_f):
        cell = min(i // k1, nf - 1) if continuous else i // k1
        x = (cell + z[i - cell * k1]) / nf  # fine node position
        parent = min(int(x * nc), nc - 1) if continuous else cell // 2
        V, _ = lagrange(z, [x * nc - parent])
        E[i, parent * k1 + np.arange(len(z))] = V[:, 0]
    return E


def planar_prolongation(coarse: PlanarDiscretization, fine: PlanarDiscretization) -> sp.csr_matrix:
    """N_fine x N_coarse embedding, Kronecker products of the 1D embeddings
    (rows and columns of constrained DoFs zero)."""
    Ec = sp.csr_matrix(_embedding_1d(coarse.n, coarse.k, True))
    Ed = sp.csr_matrix(_embedding_1d(coarse.n, coarse.k, False))
    P = sp.block_diag([sp.kron(Ed, Ec), sp.kron(Ec, Ed), sp.kron(Ed, Ed)]).tocsr()
    P.data[np.abs(P.data) < 1e-14] = 0.0
    Df = sp.diags(fine.free_mask().astype(np.float64))
    Dc = sp.diags(coarse.free_mask().astype(np.float64))
    P = (Df @ P @ Dc).tocsr()
    P.eliminate_zeros()
    return P


class PlanarHierarchy(Hierarchy):
    """The 3D solver's hierarchy, smoother, V-cycle and FGMRES with the planar pieces."""

    n_colours = 4

    def _discretization(self, n, k, nu, penalty_factor):
        return PlanarDiscretization(n, k, nu, penalty_factor)

    def _prolongation(self, coarse, fine):
        return planar_prolongation(coarse, fine)

    def _patches(self, disc, colour):
        return [planar_patch_dofs(disc, v) for v in planar_colour_vertices(disc.n, colour)]

    def _npress(self, disc):
        return (2 * disc.k + 2) ** 2


def planar_reference_solution(x, y):
    """The 2D reference solution of the module docstring: u = (d_y psi, -d_x psi),
    psi = phi(x) phi(y) with phi = G_1, and p = cos(2 pi x) cos(2 pi y)."""
    ux = G(1, x, 0) * G(1, y, 1)
    uy = -G(1, x, 1) * G(1, y, 0)
    p = np.cos(2 * math.pi * x) * np.cos(2 * math.pi * y)
    return ux, uy, p


def planar_l2_errors(disc: PlanarDiscretization, vec: np.ndarray):
    """(||u - u_h||, ||(-p) - p_h||) over the unit square for the reference
    solution, by the (k+3)^2-point Gauss rule of every cell (the discrete
    pressure approximates -p: the velocity rows carry +(p, div v))."""
    k, n, h, m = disc.k, disc.n, disc.h, disc.m
    xq, wq = gauss_legendre(k + 3)
    Vc, _ = lagrange(continuous_nodes(k), xq)  # [node, point]
    Vd, _ = lagrange(discontinuous_nodes(k), xq)
    W = np.outer(wq, wq) * h * h  # [qy, qx]
    ux_all = vec[:disc.offsets[1]].reshape(m, m + 1)   # [iy, ix]
    uy_all = vec[disc.offsets[1]:disc.offsets[2]].reshape(m + 1, m)
    p_all = vec[disc.offsets[2]:].reshape(m, m)
    eu = ep = 0.0
    for cy in range(n):
        for cx in range(n):
            X = (cx + xq) * h
            Y = (cy + xq) * h
            XX, YY = np.meshgrid(X, Y)  # [qy, qx]
            ux_c = ux_all[cy * (k + 1):(cy + 1) * (k + 1), cx * (k + 1):cx * (k + 1) + k + 2]  # [b, a]
            uy_c = uy_all[cy * (k + 1):cy * (k + 1) + k + 2, cx * (k + 1):(cx + 1) * (k + 1)]  # [a, b]
            p_c = p_all[cy * (k + 1):(cy + 1) * (k + 1), cx * (k + 1):(cx + 1) * (k + 1)]
            uxh = Vd.T @ ux_c @ Vc       # [qy, qx]
            uyh = Vc.T @ uy_c @ Vd
            ph = Vd.T @ p_c @ Vd
            ux, uy, p = planar_reference_solution(XX, YY)
            eu += np.sum(W * ((uxh - ux) ** 2 + (uyh - uy) ** 2))
            ep += np.sum(W * (ph + p) ** 2)
    return math.sqrt(eu), math.sqrt(ep)
