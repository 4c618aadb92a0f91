"""Seeded manufactured Stokes solution, right-hand side and L2 errors (test infrastructure only).

Sec. 3.3 manufactures the right-hand side from a divergence-free velocity
u = curl(psi) and a cosine pressure.  The paper's psi uses constants sigma and
mu that it never states, so the seeded family drawn by `seeded_inputs`
replaces it (a reading; the paper's exact solution stays unpinned):
    psi_c = sum_t alpha[c,t] G_a(x) G_b(y) G_c(z),  G_a(s) = s^2 (1-s)^2 sin(a pi s),
    u = curl(psi_x, psi_y, psi_z),   p = sum_t beta[t] cos(a pi x) cos(b pi y) cos(c pi z),
    f = -nu Laplace(u) + grad p       (eq. `model`).
u vanishes on the boundary because psi and grad psi do, and div u = 0.

Right-hand side: b_i = (f, phi_i) by the (k+3)-point Gauss rule of every cell
(a fixed rule, so that any two implementations agree to roundoff); pressure
rows are 0.  Because the velocity rows of eq. `weak_form` carry +(p, div v),
the discrete pressure approximates -p (see `l2_errors`).
"""
from __future__ import annotations

import math

import numpy as np

from .basis import gauss_legendre


def _P(s, j):
    """j-th derivative of s^2 (1-s)^2."""
    if j == 0:
        return s * s - 2 * s ** 3 + s ** 4
    if j == 1:
        return 2 * s - 6 * s * s + 4 * s ** 3
    if j == 2:
        return 2 - 12 * s + 12 * s * s
    if j == 3:
        return -12 + 24 * s
    if j == 4:
        return np.full_like(s, 24.0)
    return np.zeros_like(s)


def G(a: int, s, n: int):
    """n-th derivative of G_a(s) = s^2 (1-s)^2 sin(a pi s) by the Leibniz rule."""
    s = np.asarray(s, dtype=np.float64)
    w = a * math.pi
    out = np.zeros_like(s)
    for j in range(n + 1):
        out += math.comb(n, j) * _P(s, j) * w ** (n - j) * np.sin(w * s + (n - j) * math.pi / 2)
    return out


class Manufactured:
    def __init__(self, coeffs: dict, nu: float = 1.0):
        self.pf = np.asarray(coeffs["psi_freq"])
        self.pa = np.asarray(coeffs["psi_amp"])
        self.qf = np.asarray(coeffs["p_freq"])
        self.qa = np.asarray(coeffs["p_amp"])
        self.nu = float(nu)

    def psi(self, c, dx, dy, dz, x, y, z):
        """Partial derivative (dx, dy, dz) of psi_c."""
        out = np.zeros_like(np.asarray(x, dtype=np.float64))
        for t in range(3):
            a, b, cc = self.pf[c, t]
            out += self.pa[c, t] * G(a, x, dx) * G(b, y, dy) * G(cc, z, dz)
        return out

    def _curl(self, fn, x, y, z):
        # curl of the vector field (fn(0, .), fn(1, .), fn(2, .)); fn(c, e) = d_e of component c
        return np.stack([fn(2, 1) - fn(1, 2), fn(0, 2) - fn(2, 0), fn(1, 0) - fn(0, 1)], axis=-1)

    def velocity(self, x, y, z):
        def d(c, e):
            o = [0, 0, 0]
            o[e] = 1
            return self.psi(c, *o, x, y, z)
        return self._curl(d, x, y, z)

    def velocity_laplacian(self, x, y, z):
        def d(c, e):
            acc = 0.0
            for l in range(3):
                o = [0, 0, 0]
                o[e] += 1
                o[l] += 2
                acc = acc + self.psi(c, *o, x, y, z)
            return acc
        return self._curl(d, x, y, z)

    def pressure(self, x, y, z):
        out = np.zeros_like(np.asarray(x, dtype=np.float64))
        for t in range(3):
            a, b, c = self.qf[t]
            out += self.qa[t] * np.cos(a * math.pi * x) * np.cos(b * math.pi * y) * np.cos(c * math.pi * z)
        return out

    def pressure_gradient(self, x, y, z):
        gx = np.zeros_like(np.asarray(x, dtype=np.float64))
        gy = np.zeros_like(gx)
        gz = np.zeros_like(gx)
        pi = math.pi
        for t in range(3):
            a, b, c = self.qf[t]
            A = self.qa[t]
            cx, cy, cz = np.cos(a * pi * x), np.cos(b * pi * y), np.cos(c * pi * z)
            sx, sy, sz = np.sin(a * pi * x), np.sin(b * pi * y), np.sin(c * pi * z)
            gx += -A * a * pi * sx * cy * cz
            gy += -A * b * pi * cx * sy * cz
            gz += -A * c * pi * cx * cy * sz
        return np.stack([gx, gy, gz], axis=-1)

    def forcing(self, x, y, z):
        """f = -nu Laplace(u) + grad p (eq. `model`)."""
        return -self.nu * self.velocity_laplacian(x, y, z) + self.pressure_gradient(x, y, z)


def _cell_points(disc, nq):
    """Physical quadrature points (ncell, P, 3) and weights (P,) of the nq^3 Gauss rule."""
    xq, wq = gauss_legendre(nq)
    h = disc.h
    cells = disc._all_cells()
    g = np.stack(np.meshgrid(xq, xq, xq, indexing="ij"), axis=-1)  # [x, y, z] index order
    g = np.transpose(g, (2, 1, 0, 3)).reshape(-1, 3)  # x fastest
    pts = (cells[:, None, :] + g[None, :, :]) * h
    W = np.einsum("r,q,p->rqp", wq, wq, wq).reshape(-1) * h ** 3
    return cells, pts, W, xq


def rhs(disc, man: Manufactured) -> np.ndarray:
    """b_i = (f, phi_i) with the (k+3)^3 Gauss rule per cell; pressure rows and constrained rows 0."""
    cells, pts, W, xq = _cell_points(disc, disc.k + 3)
    val, _ = disc.eval_velocity(xq, xq, xq)
    f = man.forcing(pts[..., 0], pts[..., 1], pts[..., 2])  # (ncell, P, 3)
    loc = np.einsum("api,cpi,p->ca", val, f, W, optimize=True)
    G = disc.cell_dofs(cells)[:, : val.shape[0]]
    b = np.zeros(disc.N)
    np.add.at(b, G.reshape(-1), loc.reshape(-1))
    b[~disc.free_mask()] = 0.0
    return b


def interpolate(disc, man: Manufactured, pressure_sign: float = -1.0) -> np.ndarray:
    """Nodal interpolant of (u, pressure_sign * p): each DoF is the value at its support point."""
    vec = np.zeros(disc.N)
    h, k1 = disc.h, disc.k + 1
    for c in range(4):
        E = disc.ext[c]
        g = np.arange(E[0] * E[1] * E[2])
        idx = [g % E[0], (g // E[0]) % E[1], g // (E[0] * E[1])]
        coords = []
        for d in range(3):
            if c == d:
                cell = np.minimum(idx[d] // k1, disc.n - 1)
                a = idx[d] - cell * k1
                coords.append((cell + disc.zC[a]) * h)
            else:
                coords.append((idx[d] // k1 + disc.zD[idx[d] % k1]) * h)
        if c < 3:
            vec[disc.offsets[c] + g] = man.velocity(*coords)[:, c]
        else:
            vec[disc.offsets[3] + g] = pressure_sign * man.pressure(*coords)
    vec[~disc.free_mask()] = 0.0
    return vec


def l2_errors(disc, man: Manufactured, vec: np.ndarray, pressure_sign: float = -1.0):
    """(||u - u_h||_L2, ||pressure_sign * p - p_h||_L2) with (k+3)^3 Gauss points.

    The discrete pressure is compared after removing its L2 mean (the exact
    pressure has zero mean).
    """
    cells, pts, W, xq = _cell_points(disc, disc.k + 3)
    val, _ = disc.eval_velocity(xq, xq, xq)
    psi = disc.eval_pressure(xq, xq, xq)
    G = disc.cell_dofs(cells)
    nvl = val.shape[0]
    uh = np.einsum("ca,api->cpi", vec[G[:, :nvl]], val, optimize=True)
    ph = np.einsum("ca,ap->cp", vec[G[:, nvl:]], psi, optimize=True)
    u = man.velocity(pts[..., 0], pts[..., 1], pts[..., 2])
    p = pressure_sign * man.pressure(pts[..., 0], pts[..., 1], pts[..., 2])
    vol = W.sum() * len(cells)
    ph = ph - (ph * W).sum() / vol
    eu = np.sqrt(np.einsum("cpi,p->", (u - uh) ** 2, W))
    ep = np.sqrt(np.einsum("cp,p->", (p - ph) ** 2, W))
    return eu, ep
