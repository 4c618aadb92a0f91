"""Vertex-patch multiplicative Schwarz smoother, V-cycle and flexible GMRES (test infrastructure only).

  * Vertex patches (Sec. 3.1, Fig. 2): one patch per interior vertex, the
    2x2x2 cells around it.  Its subspace X_j holds every DoF supported in the
    patch except the normal velocity DoFs on the patch boundary.
  * Colouring (Sec. 3.1, Fig. 3): colour (i mod 2) + 2 (j mod 2) + 4 (l mod 2)
    of the vertex (i, j, l); colours run in ascending order.
  * Algorithm 2: for each colour, r = b - A x once, then for every patch of
    the colour x += R_j^T A_j^{-1} R_j r.  The patches of one colour share no
    DoF, so their corrections are independent.
  * Local solvers (Sec. 3.2, Sec. 3.3):
      - "lu": the pseudo-inverse of the patch matrix A_j = R_j A R_j^T, computed
        as the dense LU of the bordered system [[A_j, e], [e^T, 0]], e = the
        patch pressure ones-vector (the "Direct solver").  The extracted
        matrices are cached by their exact bytes, so each patch type is
        factored once.
      - ("schur", iters) / ("schur_tol", tol): the Schur-complement method:
        S P = B A^{-1} F - G by conjugate gradients on the mean-free subspace,
        S = B A^{-1} B^T, then U = A^{-1} (F - B^T P), with A^{-1} by a dense
        Cholesky factorisation of the velocity block (the fast diagonalization
        of the paper is an evaluation of the same A^{-1}).
  * V-cycle (Sec. 3): one pre- and one post-smoothing step, residual
    restriction by the transpose of the embedding, exact coarse solve.
  * Outer solver (Sec. 3.3): flexible GMRES with restart 20, right
    preconditioned by one V-cycle, x0 = 0, modified Gram-Schmidt, Givens
    rotations, stop at ||b - A x|| <= tol ||b||.  The returned pressure has
    zero L2 mean.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .discretization import Discretization
from .transfer import prolongation


def patch_dofs(disc: Discretization, vertex) -> np.ndarray:
    """Global DoFs of the subspace X_j of the patch at interior vertex (i, j, l).

    Velocity component c: the 2k+1 nodes strictly inside the two cells in
    direction c, all 2k+2 nodes of the two cells in the other directions;
    pressure: all (2k+2)^3 nodes.  Ordered u_x, u_y, u_z, p, x fastest.
    """
    k1 = disc.k + 1
    out = []
    for c in range(4):
        rng = []
        for d in range(3):
            lo = (vertex[d] - 1) * k1
            if c == d:
                rng.append(np.arange(lo + 1, lo + 2 * k1))
            else:
                rng.append(np.arange(lo, lo + 2 * k1))
        i2, i1, i0 = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
        out.append(disc.index(c, i0, i1, i2).reshape(-1))
    return np.concatenate(out)


def colour_vertices(n: int, colour: int):
    """Interior vertices (i, j, l) in [1, n-1]^3 of one colour."""
    bits = [(colour >> d) & 1 for d in range(3)]
    rng = [np.arange(1, n)[np.arange(1, n) % 2 == bits[d]] for d in range(3)]
    return [(i, j, l) for l in rng[2] for j in rng[1] for i in rng[0]]


class LocalSolver:
    def __init__(self, mode="lu"):
        self.mode = mode
        self._lu = {}
        self._chol = {}

    def __call__(self, Aj: np.ndarray, npress: int, r: np.ndarray) -> np.ndarray:
        if self.mode == "lu":
            return self._direct(Aj, npress, r)
        kind, param = self.mode
        return self._schur(Aj, npress, r, kind, param)

    def _direct(self, Aj, npress, r):
        key = Aj.tobytes()
        f = self._lu.get(key)
        if f is None:
            nl = Aj.shape[0]
            K = np.zeros((nl + 1, nl + 1))
            K[:nl, :nl] = Aj
            K[nl - npress:nl, nl] = 1.0
            K[nl, nl - npress:nl] = 1.0
            f = sla.lu_factor(K)
            self._lu[key] = f
        return sla.lu_solve(f, np.concatenate([r, [0.0]]))[:-1]

    def _schur(self, Aj, npress, r, kind, param):
        nv = Aj.shape[0] - npress
        key = Aj.tobytes()
        f = self._chol.get(key)
        if f is None:
            f = sla.cho_factor(Aj[:nv, :nv])
            self._chol[key] = f
        B = Aj[nv:, :nv]
        F, G = r[:nv], r[nv:]
        Ainv = lambda v: sla.cho_solve(f, v)
        return schur_cg(Ainv, B, F, G, kind, param)


def schur_cg(Ainv, B, F, G, kind, param):
    """Schur-complement local solve (Sec. 3.2, reading of its equations).

    S P = B A^{-1} F - G on the subspace of mean-free pressures, by conjugate
    gradients from P = 0: a fixed number of steps (kind "schur") or until the
    residual drops below param times its initial norm (kind "schur_tol").
    Then U = A^{-1} (F - B^T P).  Returns [U, P].
    """
    rhs = B @ Ainv(F) - G
    rhs = rhs - rhs.mean()
    P = np.zeros_like(rhs)
    res = rhs.copy()
    d = res.copy()
    rr = res @ res
    r0 = np.sqrt(rr)
    maxit = param if kind == "schur" else 10 * len(G)
    it = 0
    while it < maxit:
        if kind == "schur_tol" and np.sqrt(rr) <= param * r0:
            break
        if rr == 0.0:
            break
        Sd = B @ Ainv(B.T @ d)
        alpha = rr / (d @ Sd)
        P = P + alpha * d
        res = res - alpha * Sd
        res = res - res.mean()
        rr_new = res @ res
        d = res + (rr_new / rr) * d
        rr = rr_new
        it += 1
    U = Ainv(F - B.T @ P)
    return np.concatenate([U, P])


class Level:
    def __init__(self, disc: Discretization):
        self.disc = disc
        self.A = disc.assemble()
        self.free = disc.free_mask()
        self.P = None  # embedding from the next coarser level


class Hierarchy:
    """Mesh hierarchy n_L = n, n_{l-1} = n_l / 2, down to the coarsest mesh (2 or 3 cells per side)."""

    n_colours = 8

    def __init__(self, n: int, k: int, nu: float = 1.0, penalty_factor: float = 1.0, local="lu"):
        sizes = [n]
        while sizes[-1] % 2 == 0 and sizes[-1] > 3:
            sizes.append(sizes[-1] // 2)
        if sizes[-1] not in (2, 3):
            raise ValueError("mesh size must be 2 or 3 times a power of two")
        sizes = sizes[::-1]
        self.levels = [Level(self._discretization(s, k, nu, penalty_factor)) for s in sizes]
        for l in range(1, len(self.levels)):
            self.levels[l].P = self._prolongation(self.levels[l - 1].disc, self.levels[l].disc)
        self.local = LocalSolver(local)
        self._coarse = None

    # the pieces that depend on the space dimension
    def _discretization(self, n, k, nu, penalty_factor):
        return Discretization(n, k, nu, penalty_factor)

    def _prolongation(self, coarse, fine):
        return prolongation(coarse, fine)

    def _patches(self, disc, colour):
        return [patch_dofs(disc, v) for v in colour_vertices(disc.n, colour)]

    def _npress(self, disc):
        return (2 * disc.k + 2) ** 3

    # ---------------------------------------------------------------- smoother
    def smooth(self, l: int, x: np.ndarray, b: np.ndarray) -> np.ndarray:
        """One step of Algorithm 2 on level l (colours in ascending order)."""
        x = x.copy()
        for colour in range(self.n_colours):
            self.smooth_colour(l, colour, x, b)
        return x

    def smooth_colour(self, l: int, colour: int, x: np.ndarray, b: np.ndarray) -> np.ndarray:
        """One colour of Algorithm 2 on level l, in place: the residual of the
        current x, then every patch of the colour adds its local solve into x."""
        lev = self.levels[l]
        disc, A = lev.disc, lev.A
        npress = self._npress(disc)
        r = b - A @ x
        r[~lev.free] = 0.0
        for J in self._patches(disc, colour):
            Aj = A[J][:, J].toarray()
            x[J] += self.local(Aj, npress, r[J])
        return x

    # ------------------------------------------------------------ coarse solve
    def coarse_solve(self, b: np.ndarray) -> np.ndarray:
        """Exact coarse solve: dense LU of the bordered free system (pseudo-inverse)."""
        lev = self.levels[0]
        disc = lev.disc
        f = lev.free
        if self._coarse is None:
            Af = lev.A[f][:, f].toarray()
            nf = Af.shape[0]
            e = np.zeros(disc.N)
            e[disc.pressure_start:] = 1.0
            e = e[f]
            K = np.zeros((nf + 1, nf + 1))
            K[:nf, :nf] = Af
            K[:nf, nf] = e
            K[nf, :nf] = e
            self._coarse = sla.lu_factor(K)
        x = np.zeros(disc.N)
        x[f] = sla.lu_solve(self._coarse, np.concatenate([b[f], [0.0]]))[:-1]
        return x

    # ----------------------------------------------------------------- V-cycle
    def vcycle(self, b: np.ndarray, l: int | None = None) -> np.ndarray:
        """x = P_l^{-1} b with x0 = 0 (Sec. 3: pre-smooth, coarse correction, post-smooth)."""
        if l is None:
            l = len(self.levels) - 1
        if l == 0:
            return self.coarse_solve(b)
        lev = self.levels[l]
        x = self.smooth(l, np.zeros_like(b), b)
        r = b - lev.A @ x
        r[~lev.free] = 0.0
        xc = self.vcycle(lev.P.T @ r, l - 1)
        x = x + lev.P @ xc
        x = self.smooth(l, x, b)
        return x

    # ------------------------------------------------------------------ FGMRES
    def solve(self, b: np.ndarray, tol: float = 1e-8, restart: int = 20, maxit: int = 200):
        """Right-preconditioned flexible GMRES(restart), x0 = 0.

        Returns (x, info) with info["iterations"], info["residuals"] (relative
        Euclidean residual after each iteration, starting with 1.0) and the
        fractional iteration count info["nu"] = -8 / log10(rbar),
        rbar = (||r_n|| / ||r_0||)^(1/n) (Sec. 3.3, read with a division).
        """
        fine = self.levels[-1]
        A = fine.A
        bnorm = np.linalg.norm(b)
        x = np.zeros_like(b)
        hist = [1.0]
        its = 0
        converged = bnorm == 0.0
        r = b.copy()
        while not converged and its < maxit:
            beta = np.linalg.norm(r)
            V = [r / beta]
            Z = []
            H = np.zeros((restart + 1, restart))
            cs = np.zeros(restart)
            sn = np.zeros(restart)
            g = np.zeros(restart + 1)
            g[0] = beta
            j_done = 0
            for j in range(restart):
                z = self.vcycle(V[j])
                Z.append(z)
                w = A @ z
                for i in range(j + 1):
                    H[i, j] = w @ V[i]
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(w)
                V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
                for i in range(j):
                    t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                    H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                    H[i, j] = t
                den = np.hypot(H[j, j], H[j + 1, j])
                cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
                H[j, j] = den
                H[j + 1, j] = 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                its += 1
                j_done = j + 1
                hist.append(abs(g[j + 1]) / bnorm)
                if abs(g[j + 1]) <= tol * bnorm or its >= maxit:
                    break
            y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
            for i in range(j_done):
                x = x + y[i] * Z[i]
            r = b - A @ x
            r[~fine.free] = 0.0
            converged = np.linalg.norm(r) <= tol * bnorm
        x = project_pressure_mean(fine.disc, x)
        rel = np.linalg.norm(b - A @ x) / bnorm if bnorm else 0.0
        n_it = len(hist) - 1
        nu_frac = float("nan")
        if n_it > 0 and hist[-1] > 0:
            rbar = hist[-1] ** (1.0 / n_it)
            nu_frac = -8.0 / np.log10(rbar)
        return x, {"iterations": n_it, "residuals": hist, "nu": nu_frac, "relres": rel, "converged": converged}


def project_pressure_mean(disc: Discretization, x: np.ndarray) -> np.ndarray:
    """Shift the pressure so that its L2 mean is zero: sum_i W_i p_i = 0."""
    x = x.copy()
    W = disc.pressure_weights()
    p0 = disc.pressure_start
    p = x[p0:]
    x[p0:] = p - (W @ p) / W.sum()
    return x
