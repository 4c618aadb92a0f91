"""Literal assembly of the RT_k x DGQ_k Stokes matrix (test infrastructure only).

Follows Sec. 2.1 of the paper:
  * spaces (Sec. 2.1): velocity component c is Q_{k+1} in direction c
    (continuous, its normal trace) and Q_k in the two other directions
    (discontinuous); pressure is DGQ_k.  On the affine Cartesian mesh of
    Sec. 2.2 (Jacobian diag(1/h)) the contravariant Piola map only scales each
    component by a constant, which the nodal definition absorbs.
  * viscous form a_h: eq. `bilinear`, evaluated literally with 3x3 tensors at
    quadrature points: cell term (grad u, grad v), interior faces
    4 gamma <{{u (x) n}}, {{v (x) n}}> - 2 <{{grad u}}, {{v (x) n}}>
    - 2 <{{grad v}}, {{u (x) n}}>, boundary faces
    2 gamma <u, v> - <d_n u, v> - <u, d_n v>; {{.}} is the average of eq.
    `average`.  The whole viscous form is multiplied by the viscosity nu.
  * divergence blocks: eq. `weak_form` together with the divergence term of
    Algorithm 1 and the symmetric block form of eq. `block_A`: velocity rows get
    +(p, div v), pressure rows get +(q, div u) (a reading: two of the three
    passages use the symmetric form; the discrete pressure then approximates -p).
  * penalty: gamma = penalty_factor * (k+1)(k+2) / h (the paper leaves
    gamma_e undefined; a reading).
  * quadrature: (k+3)-point Gauss rule per direction, exact for every
    integrand of the bilinear form.

Vector layout (the same contract the library exposes): [u_x | u_y | u_z | p].
Component c is stored on an (E0, E1, E2) grid, x fastest, with E_d = m+1 in
direction c and m otherwise (m = n (k+1)); p on (m, m, m).  Node a of cell j
in a direction has global 1D index j (k+1) + a.  Normal velocity entries on
the domain boundary (index 0 or m in direction c) are constrained to zero:
the operator ignores them on input and returns 0 there.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import continuous_nodes, discontinuous_nodes, gauss_legendre, lagrange

_DROP = 1e-12  # relative size below which an assembled entry is roundoff of a structural zero


class Discretization:
    """DoF numbering and local matrices of one uniform n^3 mesh at degree k."""

    def __init__(self, n: int, k: int, nu: float = 1.0, penalty_factor: float = 1.0):
        if n < 1 or k < 0:
            raise ValueError("need n >= 1 and k >= 0")
        self.n, self.k, self.nu = int(n), int(k), float(nu)
        self.h = 1.0 / n
        self.m = n * (k + 1)
        self.gamma = penalty_factor * (k + 1) * (k + 2) / self.h
        m = self.m
        self.ext = [tuple(m + 1 if d == c else m for d in range(3)) for c in range(3)] + [(m, m, m)]
        nv = (m + 1) * m * m
        self.offsets = [0, nv, 2 * nv, 3 * nv]
        self.pressure_start = 3 * nv
        self.n_vel_component = nv
        self.n_pressure = m ** 3
        self.N = 3 * nv + m ** 3
        self.zC = continuous_nodes(k)
        self.zD = discontinuous_nodes(k)
        self._local = None
        self._free = None

    # ------------------------------------------------------------------ numbering
    def index(self, comp: int, i0, i1, i2):
        """Global index of node (i0, i1, i2) of component comp (3 = pressure)."""
        E0, E1, _ = self.ext[comp]
        return self.offsets[comp] + np.asarray(i0) + E0 * (np.asarray(i1) + E1 * np.asarray(i2))

    def free_mask(self) -> np.ndarray:
        """True for every DoF that is not a boundary normal velocity entry."""
        if self._free is None:
            free = np.ones(self.N, dtype=bool)
            m = self.m
            for c in range(3):
                E = self.ext[c]
                g = np.arange(E[0] * E[1] * E[2])
                idx = [g % E[0], (g // E[0]) % E[1], g // (E[0] * E[1])]
                bnd = (idx[c] == 0) | (idx[c] == m)
                free[self.offsets[c] + g[bnd]] = False
            self._free = free
        return self._free

    def local_layout(self):
        """Per local DoF of a cell: (kind, a0, a1, a2), kind 0..2 velocity, 3 pressure.

        Ordering: u_x nodes (a0 fastest), then u_y, u_z, then pressure.
        """
        if self._local is None:
            k = self.k
            rows = []
            for c in range(4):
                e = [k + 2 if d == c else k + 1 for d in range(3)]
                for a2 in range(e[2]):
                    for a1 in range(e[1]):
                        for a0 in range(e[0]):
                            rows.append((c, a0, a1, a2))
            self._local = np.array(rows, dtype=np.int64)
        return self._local

    def n_local_velocity(self) -> int:
        k = self.k
        return 3 * (k + 2) * (k + 1) ** 2

    def cell_dofs(self, cells: np.ndarray) -> np.ndarray:
        """Global indices (ncell, nloc) of the local DoFs of the given cells (ncell, 3)."""
        cells = np.atleast_2d(np.asarray(cells, dtype=np.int64))
        lay = self.local_layout()
        k1 = self.k + 1
        out = np.empty((cells.shape[0], lay.shape[0]), dtype=np.int64)
        for c in range(4):
            sel = lay[:, 0] == c
            a = lay[sel, 1:]
            i0 = cells[:, 0:1] * k1 + a[None, :, 0]
            i1 = cells[:, 1:2] * k1 + a[None, :, 1]
            i2 = cells[:, 2:3] * k1 + a[None, :, 2]
            out[:, sel] = self.index(c, i0, i1, i2)
        return out

    # ------------------------------------------------------------ basis on a cell
    def eval_velocity(self, p0, p1, p2):
        """Velocity basis of one cell on the tensor grid p0 x p1 x p2 (reference coords).

        Returns val[nv, P, 3] and grad[nv, P, 3, 3] with grad[..., i, j] = d_j u_i
        in physical coordinates; P runs over the grid with p0 fastest.
        """
        h = self.h
        pts = [np.atleast_1d(np.asarray(p, dtype=np.float64)) for p in (p0, p1, p2)]
        P = len(pts[0]) * len(pts[1]) * len(pts[2])
        vals, grads = [], []
        for c in range(3):
            tabs = []
            for d in range(3):
                z = self.zC if d == c else self.zD
                V, D = lagrange(z, pts[d])
                tabs.append((V, D / h))
            na = [tabs[d][0].shape[0] for d in range(3)]

            def outer(f0, f1, f2):
                t = np.einsum("zr,yq,xp->zyxrqp", f2, f1, f0)
                return t.reshape(na[0] * na[1] * na[2], P)

            v = outer(tabs[0][0], tabs[1][0], tabs[2][0])
            val = np.zeros((v.shape[0], P, 3))
            val[:, :, c] = v
            grad = np.zeros((v.shape[0], P, 3, 3))
            grad[:, :, c, 0] = outer(tabs[0][1], tabs[1][0], tabs[2][0])
            grad[:, :, c, 1] = outer(tabs[0][0], tabs[1][1], tabs[2][0])
            grad[:, :, c, 2] = outer(tabs[0][0], tabs[1][0], tabs[2][1])
            vals.append(val)
            grads.append(grad)
        return np.concatenate(vals), np.concatenate(grads)

    def eval_pressure(self, p0, p1, p2):
        """Pressure basis of one cell on a tensor grid: psi[np, P]."""
        pts = [np.atleast_1d(np.asarray(p, dtype=np.float64)) for p in (p0, p1, p2)]
        V = [lagrange(self.zD, pts[d])[0] for d in range(3)]
        t = np.einsum("zr,yq,xp->zyxrqp", V[2], V[1], V[0])
        return t.reshape(V[0].shape[0] * V[1].shape[0] * V[2].shape[0], -1)

    # ------------------------------------------------------------ local matrices
    def cell_matrix(self) -> np.ndarray:
        """Cell matrix [[nu A_K, B_K^T], [B_K, 0]] by (k+3)^3-point Gauss quadrature."""
        k, h = self.k, self.h
        xq, wq = gauss_legendre(k + 3)
        val, grad = self.eval_velocity(xq, xq, xq)
        psi = self.eval_pressure(xq, xq, xq)
        W = np.einsum("r,q,p->rqp", wq, wq, wq).reshape(-1) * h ** 3
        A = self.nu * np.einsum("apij,bpij,p->ab", grad, grad, W, optimize=True)
        div = np.einsum("apii->ap", grad)
        B = np.einsum("qp,vp,p->qv", psi, div, W, optimize=True)
        nv, npr = A.shape[0], B.shape[0]
        K = np.zeros((nv + npr, nv + npr))
        K[:nv, :nv] = A
        K[:nv, nv:] = B.T
        K[nv:, :nv] = B
        return K

    def _face_grid(self, d: int, xi_d: float):
        xq, wq = gauss_legendre(self.k + 3)
        pts = [xq, xq, xq]
        pts[d] = np.array([xi_d])
        tang = [e for e in range(3) if e != d]
        W = np.einsum("q,p->qp", wq, wq).reshape(-1) * self.h ** 2
        return pts, W

    def interior_face_matrix(self, d: int) -> np.ndarray:
        """Viscous face matrix of an interior face normal to direction d.

        Local DoFs: the velocity DoFs of the lower cell K- (reference coordinate
        1 on the face) followed by those of the upper cell K+ (coordinate 0).
        The normal n = n^- = e_d.  Returns nu times the interior-face terms of
        eq. `bilinear` (test index first).
        """
        g = self.gamma
        pts_m, W = self._face_grid(d, 1.0)
        pts_p, _ = self._face_grid(d, 0.0)
        vm, gm = self.eval_velocity(*pts_m)
        vp, gp = self.eval_velocity(*pts_p)
        nvl, P = vm.shape[0], vm.shape[1]
        z = np.zeros_like(vm)
        zg = np.zeros_like(gm)
        u_minus = np.concatenate([vm, z])
        u_plus = np.concatenate([z, vp])
        g_minus = np.concatenate([gm, zg])
        g_plus = np.concatenate([zg, gp])
        nvec = np.zeros(3)
        nvec[d] = 1.0
        # {{u (x) n}} = (u^- (x) n^- + u^+ (x) n^+) / 2, n^+ = -n^-
        avg_un = 0.5 * (np.einsum("api,j->apij", u_minus, nvec) + np.einsum("api,j->apij", u_plus, -nvec))
        avg_grad = 0.5 * (g_minus + g_plus)
        t1 = 4.0 * g * np.einsum("apij,bpij,p->ab", avg_un, avg_un, W, optimize=True)
        t2 = -2.0 * np.einsum("bpij,apij,p->ab", avg_grad, avg_un, W, optimize=True)
        t3 = -2.0 * np.einsum("apij,bpij,p->ab", avg_grad, avg_un, W, optimize=True)
        return self.nu * (t1 + t2 + t3)

    def boundary_face_matrix(self, d: int, side: int) -> np.ndarray:
        """Viscous boundary-face matrix (Nitsche terms of eq. `bilinear`).

        side 0: face x_d = 0 of a cell with index 0 in direction d, outward
        normal -e_d; side 1: face x_d = 1, outward normal +e_d.  Local DoFs are
        the velocity DoFs of that cell.
        """
        g = self.gamma
        pts, W = self._face_grid(d, float(side))
        v, gr = self.eval_velocity(*pts)
        nvec = np.zeros(3)
        nvec[d] = 1.0 if side == 1 else -1.0
        dn = np.einsum("apij,j->api", gr, nvec)
        t1 = 2.0 * g * np.einsum("bpi,api,p->ab", v, v, W, optimize=True)
        t2 = -np.einsum("bpi,api,p->ab", dn, v, W, optimize=True)
        t3 = -np.einsum("bpi,api,p->ab", v, dn, W, optimize=True)
        return self.nu * (t1 + t2 + t3)

    # ------------------------------------------------------------------ assembly
    def _all_cells(self):
        n = self.n
        c = np.arange(n ** 3)
        return np.stack([c % n, (c // n) % n, c // (n * n)], axis=1)

    def assemble(self, chunk: int = 256) -> sp.csr_matrix:
        """Global N x N Stokes matrix with the boundary normal DoFs removed.

        Rows and columns of constrained DoFs are zero.  Entries below 1e-12 of
        the largest entry are dropped: they are the roundoff left by quadrature
        of structurally zero integrals (Gauss-point orthogonality) and by the
        cancellation of the two cell pieces of a shared normal DoF.
        """
        N = self.N
        itype = np.int64
        total = sp.csr_matrix((N, N))

        def add_local(Kloc, G):
            nonlocal total
            scale = np.abs(Kloc).max()
            ia, ib = np.nonzero(np.abs(Kloc) > 1e-15 * scale)
            vals = Kloc[ia, ib]
            for s in range(0, G.shape[0], chunk):
                g = G[s:s + chunk]
                r = g[:, ia].reshape(-1).astype(itype)
                c = g[:, ib].reshape(-1).astype(itype)
                v = np.broadcast_to(vals, (g.shape[0], len(vals))).reshape(-1)
                total = total + sp.csr_matrix((v, (r, c)), shape=(N, N))

        cells = self._all_cells()
        G = self.cell_dofs(cells)
        add_local(self.cell_matrix(), G)
        nvl = self.n_local_velocity()
        n = self.n
        for d in range(3):
            lower = cells[cells[:, d] < n - 1]
            upper = lower.copy()
            upper[:, d] += 1
            if lower.shape[0]:
                Gf = np.concatenate([self.cell_dofs(lower)[:, :nvl], self.cell_dofs(upper)[:, :nvl]], axis=1)
                add_local(self.interior_face_matrix(d), Gf)
            for side in (0, 1):
                sel = cells[:, d] == (0 if side == 0 else n - 1)
                add_local(self.boundary_face_matrix(d, side), self.cell_dofs(cells[sel])[:, :nvl])
        A = total.tocsr()
        A.sum_duplicates()
        scale = np.abs(A.data).max()
        A.data[np.abs(A.data) < _DROP * scale] = 0.0
        A.eliminate_zeros()
        f = self.free_mask().astype(np.float64)
        Dm = sp.diags(f)
        A = (Dm @ A @ Dm).tocsr()
        A.eliminate_zeros()
        return A

    # --------------------------------------------------- rows from a cell subset
    def local_rows(self, cells):
        """The global matrix restricted to the DoFs of a set of cells, built
        from the same local pieces as `assemble` without a global matrix.

        Sums the cell matrices of `cells` (array (ncell, 3)), the interior-face
        matrices of every face of those cells (whether or not the cell on the
        other side is in the set) and the boundary-face matrices of their faces
        on the domain boundary.  Returns (cols, K): cols the sorted global DoFs
        these pieces touch, K a CSR matrix over cols.  A row of K equals the
        global matrix's row (over cols) for every DoF whose cells all belong
        to `cells`: then every cell and face contributing to that row is
        included.  Constrained DoFs have zero rows and columns; entries below
        1e-12 of the largest are dropped, as in `assemble`.
        """
        cells = np.atleast_2d(np.asarray(cells, dtype=np.int64))
        n = self.n
        nvl = self.n_local_velocity()
        pieces = [(self.cell_dofs(cells), self.cell_matrix())]
        inner = {d: set() for d in range(3)}
        bnd = {(d, s): set() for d in range(3) for s in (0, 1)}
        for cell in map(tuple, cells):
            for d in range(3):
                if cell[d] > 0:
                    lo = list(cell)
                    lo[d] -= 1
                    inner[d].add(tuple(lo))
                else:
                    bnd[(d, 0)].add(cell)
                if cell[d] < n - 1:
                    inner[d].add(cell)
                else:
                    bnd[(d, 1)].add(cell)
        for d in range(3):
            if inner[d]:
                lower = np.array(sorted(inner[d]), dtype=np.int64)
                upper = lower.copy()
                upper[:, d] += 1
                Gf = np.concatenate([self.cell_dofs(lower)[:, :nvl], self.cell_dofs(upper)[:, :nvl]], axis=1)
                pieces.append((Gf, self.interior_face_matrix(d)))
            for s in (0, 1):
                if bnd[(d, s)]:
                    sel = np.array(sorted(bnd[(d, s)]), dtype=np.int64)
                    pieces.append((self.cell_dofs(sel)[:, :nvl], self.boundary_face_matrix(d, s)))
        cols = np.unique(np.concatenate([G.reshape(-1) for G, _ in pieces]))
        rows_l, cols_l, vals = [], [], []
        for G, Kloc in pieces:
            scale = np.abs(Kloc).max()
            ia, ib = np.nonzero(np.abs(Kloc) > 1e-15 * scale)
            Gl = np.searchsorted(cols, G)
            rows_l.append(Gl[:, ia].reshape(-1))
            cols_l.append(Gl[:, ib].reshape(-1))
            vals.append(np.broadcast_to(Kloc[ia, ib], (G.shape[0], len(ia))).reshape(-1))
        nc = len(cols)
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows_l), np.concatenate(cols_l))), shape=(nc, nc))
        K.sum_duplicates()
        scale = np.abs(K.data).max()
        K.data[np.abs(K.data) < _DROP * scale] = 0.0
        K.eliminate_zeros()
        f = sp.diags(self.free_mask()[cols].astype(np.float64))
        K = (f @ K @ f).tocsr()
        K.eliminate_zeros()
        return cols, K

    # ------------------------------------------------------- sampled row products
    def apply_rows(self, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
        """(A x)[rows] from the local matrices, without a global matrix.

        For each requested DoF the contributions of every cell and every face
        that carries it are summed, exactly as the assembly does; used to check
        very large meshes at sampled outputs.  Entries are not thresholded, so
        results agree with `assemble` to roundoff.
        """
        x = np.where(self.free_mask(), x, 0.0)
        free = self.free_mask()
        Kc = self.cell_matrix()
        Fi = [self.interior_face_matrix(d) for d in range(3)]
        Fb = [[self.boundary_face_matrix(d, s) for s in (0, 1)] for d in range(3)]
        nvl = self.n_local_velocity()
        n, k1 = self.n, self.k + 1
        out = np.zeros(len(rows))
        for r_i, g in enumerate(np.asarray(rows, dtype=np.int64)):
            if not free[g]:
                continue
            comp = int(np.searchsorted(self.offsets, g, side="right") - 1) if g < self.offsets[3] else 3
            loc = g - self.offsets[comp]
            E = self.ext[comp]
            idx = [loc % E[0], (loc // E[0]) % E[1], loc // (E[0] * E[1])]
            cand = []
            for d in range(3):
                cs = {min(idx[d] // k1, n - 1)}
                if comp == d and idx[d] % k1 == 0 and idx[d] > 0:
                    cs.add(idx[d] // k1 - 1)
                cand.append(sorted(c for c in cs if 0 <= c < n))
            cells = [(a, b, c) for c in cand[2] for b in cand[1] for a in cand[0]]
            acc = 0.0
            faces = set()
            for cell in cells:
                G = self.cell_dofs(np.array([cell]))[0]
                for pos in np.nonzero(G == g)[0]:
                    acc += Kc[pos] @ x[G]
                for d in range(3):
                    for s in (0, 1):
                        nb = list(cell)
                        nb[d] += 1 if s == 1 else -1
                        if 0 <= nb[d] < n:
                            lo = cell if s == 1 else tuple(nb)
                            faces.add(("i", d, tuple(lo)))
                        else:
                            faces.add(("b", d, s, tuple(cell)))
            for f in faces:
                if f[0] == "i":
                    _, d, lo = f
                    up = list(lo)
                    up[d] += 1
                    Gf = np.concatenate([self.cell_dofs(np.array([lo]))[0, :nvl], self.cell_dofs(np.array([up]))[0, :nvl]])
                    M = Fi[d]
                else:
                    _, d, s, cell = f
                    Gf = self.cell_dofs(np.array([cell]))[0, :nvl]
                    M = Fb[d][s]
                for pos in np.nonzero(Gf == g)[0]:
                    acc += M[pos] @ x[Gf]
            out[r_i] = acc
        return out

    # ------------------------------------------------------------- FE evaluation
    def evaluate(self, vec: np.ndarray, points: np.ndarray):
        """Velocity (P, 3) and pressure (P,) of the FE function `vec` at physical points.

        Each point is evaluated in the cell that contains it (the upper cell
        on a cell boundary); used by transfer and divergence pins.
        """
        pts = np.atleast_2d(points)
        n, h = self.n, self.h
        uvals = np.zeros((pts.shape[0], 3))
        pvals = np.zeros(pts.shape[0])
        for i, x in enumerate(pts):
            cell = np.minimum((x / h).astype(np.int64), n - 1)
            xi = x / h - cell
            G = self.cell_dofs(cell[None])[0]
            val, _ = self.eval_velocity([xi[0]], [xi[1]], [xi[2]])
            psi = self.eval_pressure([xi[0]], [xi[1]], [xi[2]])
            nvl = val.shape[0]
            uvals[i] = np.einsum("a,ai->i", vec[G[:nvl]], val[:, 0, :])
            pvals[i] = vec[G[nvl:]] @ psi[:, 0]
        return uvals, pvals

    def divergence(self, vec: np.ndarray, points: np.ndarray) -> np.ndarray:
        """div u_h of the FE velocity at physical points."""
        pts = np.atleast_2d(points)
        n, h = self.n, self.h
        out = np.zeros(pts.shape[0])
        for i, x in enumerate(pts):
            cell = np.minimum((x / h).astype(np.int64), n - 1)
            xi = x / h - cell
            G = self.cell_dofs(cell[None])[0]
            _, gr = self.eval_velocity([xi[0]], [xi[1]], [xi[2]])
            nvl = gr.shape[0]
            out[i] = vec[G[:nvl]] @ np.einsum("aii->a", gr[:, 0])
        return out

    def pressure_weights(self) -> np.ndarray:
        """Quadrature weight of each pressure DoF: int_Omega psi_i = W_i (Gauss weights x h^3)."""
        _, w = gauss_legendre(self.k + 1)
        m, k1 = self.m, self.k + 1
        g = np.arange(m)
        w1 = w[g % k1] * self.h
        return np.einsum("z,y,x->zyx", w1, w1, w1).reshape(-1)
