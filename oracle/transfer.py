"""Level transfers of the oracle (test infrastructure only).

Sec. 3: prolongation I^up from X_{l} to X_{l+1} is the canonical embedding of
the nested spaces; restriction I^down is read as its transpose (the paper calls
it an l2-projection; a reading).  In the nodal bases the embedding has entries
phi^coarse_j(x_i) for every fine support point x_i: the coarse function is
interpolated at the fine nodes.  Built here by evaluating the coarse basis of
the parent cell at every fine support point.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import lagrange


def prolongation(coarse, fine) -> sp.csr_matrix:
    """N_fine x N_coarse embedding matrix (fine mesh = coarse mesh refined once).

    Rows and columns of constrained (boundary normal) DoFs are zero.
    """
    if fine.n != 2 * coarse.n or fine.k != coarse.k:
        raise ValueError("fine mesh must be the coarse mesh refined once, same degree")
    k1 = fine.k + 1
    rows, cols, vals = [], [], []
    for c in range(4):
        Ef, Ec = fine.ext[c], coarse.ext[c]
        tabs, cidx = [], []
        for d in range(3):
            i = np.arange(Ef[d])
            cont = c == d
            fc = np.minimum(i // k1, fine.n - 1) if cont else i // k1
            a = i - fc * k1
            z = fine.zC if cont else fine.zD
            # position in units of coarse cells: (fc + z_a) / 2
            parent = fc // 2
            xi = ((fc - 2 * parent) + z[a]) / 2.0
            zc = coarse.zC if cont else coarse.zD
            V, _ = lagrange(zc, xi)  # (na, E_f)
            tabs.append(V.T)  # (E_f, na)
            cidx.append(parent[:, None] * k1 + np.arange(V.shape[0])[None, :])  # coarse 1D node
        val = np.einsum("za,yb,xc->zyxabc", tabs[2], tabs[1], tabs[0])  # fine z,y,x ; coarse a2,a1,a0
        # fine global index in (z, y, x) order
        gi0 = np.arange(Ef[0])[None, None, :]
        gi1 = np.arange(Ef[1])[None, :, None]
        gi2 = np.arange(Ef[2])[:, None, None]
        fglob = fine.index(c, gi0, gi1, gi2)  # (z, y, x)
        cglob = coarse.index(
            c,
            cidx[0][None, None, :, None, None, :],
            cidx[1][None, :, None, None, :, None],
            cidx[2][:, None, None, :, None, None],
        )  # (z, y, x, a2, a1, a0)
        r = np.broadcast_to(fglob[..., None, None, None], val.shape).reshape(-1)
        cc = np.broadcast_to(cglob, val.shape).reshape(-1)
        v = val.reshape(-1)
        keep = np.abs(v) > 1e-14
        rows.append(r[keep])
        cols.append(cc[keep])
        vals.append(v[keep])
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(fine.N, coarse.N))
    P.sum_duplicates()
    Df = sp.diags(fine.free_mask().astype(np.float64))
    Dc = sp.diags(coarse.free_mask().astype(np.float64))
    P = (Df @ P @ Dc).tocsr()
    P.eliminate_zeros()
    return P


def restriction(coarse, fine) -> sp.csr_matrix:
    """Residual restriction: transpose of the embedding."""
    return prolongation(coarse, fine).T.tocsr()
