"""1D quadrature and Lagrange bases for the oracle (test infrastructure only).

Node choice (a reading: the paper shows support points in Fig. 1 and in the
index-storage figure of Sec. 4 but never names them): the continuous
("parallel") direction of a Raviart-Thomas component uses degree k+1 Lagrange
polynomials on the k+2 Gauss-Lobatto points of a cell; the discontinuous
("orthogonal") directions and the DGQ_k pressure use degree k Lagrange
polynomials on the k+1 Gauss points.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(nq: int):
    """Gauss-Legendre nodes and weights mapped to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto(npts: int):
    """Gauss-Lobatto-Legendre nodes and weights on [0, 1] (npts >= 2).

    Interior nodes are the roots of P'_{N}, N = npts - 1, polished by Newton
    steps on P'_N; weights are 2 / (N (N+1) P_N(x)^2) on [-1, 1].
    """
    N = npts - 1
    cN = np.zeros(N + 1)
    cN[N] = 1.0
    dcN = np.polynomial.legendre.legder(cN)
    if N >= 2:
        r = np.sort(np.real(np.polynomial.legendre.legroots(dcN)))
        d2 = np.polynomial.legendre.legder(dcN)
        for _ in range(4):
            r = r - np.polynomial.legendre.legval(r, dcN) / np.polynomial.legendre.legval(r, d2)
        x = np.concatenate([[-1.0], r, [1.0]])
    else:
        x = np.array([-1.0, 1.0])
    PN = np.polynomial.legendre.legval(x, cN)
    w = 2.0 / (N * (N + 1) * PN ** 2)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange(z, t):
    """Lagrange basis on nodes z evaluated at points t.

    Returns (V, D) with V[i, q] = l_i(t_q) and D[i, q] = l_i'(t_q), from the
    product formula and its derivative by the product rule.
    """
    z = np.asarray(z, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    p = len(z)
    V = np.ones((p, len(t)))
    D = np.zeros((p, len(t)))
    for i in range(p):
        for j in range(p):
            if j != i:
                V[i] *= (t - z[j]) / (z[i] - z[j])
        for l in range(p):
            if l == i:
                continue
            term = np.full(len(t), 1.0 / (z[i] - z[l]))
            for j in range(p):
                if j != i and j != l:
                    term *= (t - z[j]) / (z[i] - z[j])
            D[i] += term
    return V, D


def continuous_nodes(k: int):
    """Support points of the continuous direction: k+2 Gauss-Lobatto points."""
    return gauss_lobatto(k + 2)[0]


def discontinuous_nodes(k: int):
    """Support points of the discontinuous directions and the pressure: k+1 Gauss points."""
    return gauss_legendre(k + 1)[0]
