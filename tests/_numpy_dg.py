"""Independent numpy evaluation of piecewise Legendre states, used by the pins.

Written without the oracle: numpy.polynomial.legendre does the basis, numpy's
leggauss the quadrature, and cells are located here from the geometry of the
two meshes (dual = primal shifted by half a cell).  Periodic meshes only.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def leg(n, x, d=0):
    c = np.zeros(n + 1)
    c[n] = 1.0
    if d:
        c = npleg.legder(c, d)
    return npleg.legval(x, c)


def modes(dim, k, basis_q=True):
    if dim == 1:
        return [(a, 0) for a in range(k + 1)]
    if basis_q:
        return [(a, b) for b in range(k + 1) for a in range(k + 1)]
    return [(a, s - a) for s in range(k + 1) for a in range(s, -1, -1)]


def eval_mesh(u, mesh, pts, dim, k, L, n, basis_q=True):
    """Values of mesh `mesh` of state u [2,F,M,ny,nx] at physical points pts [n,dim]
    on the periodic box [0,L)^dim with n cells per direction.  Returns [npts, F]."""
    h = L / n
    md = modes(dim, k, basis_q)
    F = u.shape[1]
    out = np.zeros((len(pts), F))
    s = 0.5 * mesh
    ix = np.floor(pts[:, 0] / h - s).astype(int)
    xi = (pts[:, 0] - (ix + 0.5 + s) * h) / (0.5 * h)
    ix = np.mod(ix, n)
    if dim == 2:
        iy = np.floor(pts[:, 1] / h - s).astype(int)
        eta = (pts[:, 1] - (iy + 0.5 + s) * h) / (0.5 * h)
        iy = np.mod(iy, n)
    else:
        iy = np.zeros_like(ix)
        eta = np.zeros_like(xi)
    for m, (a, b) in enumerate(md):
        ph = leg(a, xi) * (leg(b, eta) if dim == 2 else 1.0)
        out += u[mesh][:, m][:, iy, ix].T * ph[:, None]
    return out


def subcell_rule(dim, k, L, n):
    """Composite Gauss rule on the cells cut by both meshes (quarter / half cells):
    exact for the piecewise polynomials of both meshes.  Returns (points, weights)."""
    g, w = np.polynomial.legendre.leggauss(k + 2)
    hs = L / (2 * n)
    x1 = (np.arange(2 * n)[:, None] + 0.5 + 0.5 * g[None, :]) * hs
    w1 = np.broadcast_to(0.5 * w[None, :] * hs, x1.shape)
    x1, w1 = x1.ravel(), w1.ravel()
    if dim == 1:
        return x1[:, None], w1
    X, Y = np.meshgrid(x1, x1, indexing="xy")
    WX, WY = np.meshgrid(w1, w1, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1), (WX * WY).ravel()
