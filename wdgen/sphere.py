"""Cubed-sphere Haar workload (seeded synthetic input, no solver arithmetic).

The unit sphere is covered by six patches, the faces of the cube [-1, 1]^3
projected radially (equiangular gnomonic charts: parameters alpha, beta in
[-pi/4, pi/4], cube point with tangent coordinates tan(alpha), tan(beta)).
Each patch carries a 2^J x 2^J grid of panels and, in parameter space, the
isotropic 2D Haar basis of the unit square (same levelwise order as
``haar_basis(2, J)``); the global index is patch * 4^J + local index.

Discretisation (the same one-point rule as the flat workloads): a panel c has
the point x_c = the cube point of its parameter midpoint, normalised, and the
area |c| = the spherical area of the quadrilateral through its four (unit)
corners, split into two spherical triangles whose excess E satisfies
tan(E / 2) = |a . (b x c)| / (1 + a.b + b.c + c.a).  K_ss[c, c'] =
sqrt(|c| |c'|) k(|x_c - x_c'|), k on the chordal distance; the normalised
panel indicators are orthonormal in L2(S^2), so the wavelets are too (mass
matrix I) and A = mask(T K_ss T^T) + nugget I.

Compression: keep (lambda, lambda') iff dist(supp, supp') <= 2 * 2^-min(j, j')
on the unit sphere, with a conservative support distance
max(0, |m - m'| - r - r'): m is the mean of the unit corner points of the
panels in the support, r the largest distance from m to those points.

Patches are numbered 0:+x, 1:+y, 2:-x, 3:+z, 4:-y, 5:-z, so that the pairs
(0, 1), (2, 3), (4, 5) share an edge; the dissection of the patch set then
cuts {0, 1} from the rest, {2, 3} from {4, 5}, and each pair along its edge.
"""
from __future__ import annotations

import math

import numpy as np

from .haar import Basis, Kernel, fwt, haar_basis, rhs

NPATCH = 6


def cube_point(face: int, ta, tb, xp=np):
    """Point on the cube surface of face `face` with tangent coordinates
    (ta, tb) in [-1, 1]^2; returns (x, y, z)."""
    one = xp.ones_like(ta)
    if face == 0:
        return one, ta, tb
    if face == 1:
        return -ta, one, tb
    if face == 2:
        return -one, -ta, tb
    if face == 3:
        return -tb, ta, one
    if face == 4:
        return ta, -one, tb
    if face == 5:
        return tb, ta, -one
    raise ValueError(face)


def _unit(x, y, z, xp=np):
    r = xp.sqrt(x * x + y * y + z * z)
    return xp.stack([x / r, y / r, z / r], -1)


def panel_grid(J: int, xp=np, device=None):
    """(points [6, n, n, 3], areas [6, n, n], corners [6, n+1, n+1, 3]) of the
    panels, arrays indexed [patch, iy, ix]."""
    n = 1 << J
    h = (math.pi / 2) / n
    kw = {} if xp is np else dict(device=device)
    mid = -math.pi / 4 + (xp.arange(n, dtype=xp.float64, **kw) + 0.5) * h
    edge = -math.pi / 4 + xp.arange(n + 1, dtype=xp.float64, **kw) * h
    pts, areas, corners = [], [], []
    for f in range(NPATCH):
        tb, ta = xp.meshgrid(xp.tan(mid), xp.tan(mid), indexing="ij")     # [iy, ix]
        pts.append(_unit(*cube_point(f, ta, tb, xp), xp))
        cb, ca = xp.meshgrid(xp.tan(edge), xp.tan(edge), indexing="ij")
        g = _unit(*cube_point(f, ca, cb, xp), xp)                            # [n+1, n+1, 3]
        corners.append(g)
        a, b, c, d = g[:-1, :-1], g[:-1, 1:], g[1:, 1:], g[1:, :-1]
        areas.append(_tri_area(a, b, c, xp) + _tri_area(a, c, d, xp))
    return xp.stack(pts), xp.stack(areas), xp.stack(corners)


def _tri_area(a, b, c, xp=np):
    """Spherical excess of the triangle with unit vertices a, b, c."""
    cr = xp.stack([b[..., 1] * c[..., 2] - b[..., 2] * c[..., 1],
                   b[..., 2] * c[..., 0] - b[..., 0] * c[..., 2],
                   b[..., 0] * c[..., 1] - b[..., 1] * c[..., 0]], -1)
    num = xp.abs((a * cr).sum(-1))
    den = 1.0 + (a * b).sum(-1) + (b * c).sum(-1) + (c * a).sum(-1)
    return 2.0 * xp.arctan2(num, den) if xp is np else 2.0 * xp.atan2(num, den)


def sphere_basis(J: int) -> Basis:
    """Six copies of the 2D Haar basis of a 2^J x 2^J patch, with patch ids."""
    b = haar_basis(2, J)
    N = b.N
    return Basis(2, J, np.tile(b.level, NPATCH), np.tile(b.box_lo, (NPATCH, 1)),
                 np.tile(b.box_side, NPATCH), np.repeat(np.arange(NPATCH, dtype=np.int32), N))


def support_spheres(basis: Basis):
    """(m [N, 3], r [N]): bounding sphere of every support from the unit corner
    points of its panels."""
    J = basis.J
    _, _, corners = panel_grid(J)
    N = basis.N
    m = np.empty((N, 3))
    r = np.empty(N)
    lo = basis.box_lo.astype(np.int64)
    side = basis.box_side.astype(np.int64)
    for s in np.unique(side):
        idx = np.nonzero(side == s)[0]
        k = np.arange(s + 1)
        for q0 in range(0, idx.size, 4096):
            sel = idx[q0:q0 + 4096]
            ys = lo[sel, 1][:, None, None] + k[None, :, None]
            xs = lo[sel, 0][:, None, None] + k[None, None, :]
            g = corners[basis.patch[sel][:, None, None], ys, xs]          # [cnt, s+1, s+1, 3]
            g = g.reshape(sel.size, -1, 3)
            mm = g.mean(1)
            m[sel] = mm
            r[sel] = np.sqrt(((g - mm[:, None, :]) ** 2).sum(-1)).max(1)
    return m, r


def sphere_pattern(basis: Basis, device: str = "cpu", block: int = 2048):
    """Lower CSC (colptr int64, rowidx int32, diagonal first, rows sorted) of
    the compressed pattern."""
    import torch
    m, r = support_spheres(basis)
    N = basis.N
    dev = torch.device(device)
    M = torch.tensor(m, device=dev)
    R = torch.tensor(r, device=dev)
    lev = torch.tensor(basis.level.astype(np.int64), device=dev)
    cols, rows = [], []
    for c0 in range(0, N, block):
        c1 = min(N, c0 + block)
        Mi, Ri, Li = M[c0:], R[c0:], lev[c0:]                                 # rows >= c0
        d = torch.cdist(Mi, M[c0:c1], compute_mode="donot_use_mm_for_euclid_dist") - Ri[:, None] - R[None, c0:c1]
        d = torch.clamp(d, min=0.0)
        jmin = torch.minimum(Li[:, None], lev[None, c0:c1])
        thr = 2.0 * torch.pow(2.0, -jmin.to(torch.float64))
        keep = d <= thr
        ii = torch.arange(c0, N, device=dev)[:, None]
        jj = torch.arange(c0, c1, device=dev)[None, :]
        keep &= ii >= jj
        nz = torch.nonzero(keep.T)                                           # (col, row) sorted by col, row
        cols.append((nz[:, 0] + c0).cpu().numpy())
        rows.append((nz[:, 1] + c0).cpu().numpy())
    col = np.concatenate(cols)
    row = np.concatenate(rows).astype(np.int32)
    colptr = np.zeros(N + 1, np.int64)
    np.add.at(colptr, col + 1, 1)
    colptr = np.cumsum(colptr)
    return colptr, row


def sphere_values(basis: Basis, colptr, rowidx, kernel: Kernel, nugget: float, device: str = "cpu"):
    """Values of the compressed matrix on its lower pattern (float64 numpy),
    computed block by block over patch pairs."""
    import torch
    J = basis.J
    n = 1 << J
    Np = n * n
    dev = torch.device(device)
    pts, areas, _ = panel_grid(J, torch, dev)
    X = pts.reshape(NPATCH, Np, 3)
    W = torch.sqrt(areas.reshape(NPATCH, Np))
    cp = np.asarray(colptr)
    ri = np.asarray(rowidx).astype(np.int64)
    col = np.repeat(np.arange(cp.size - 1), np.diff(cp))
    pr, pc = ri // Np, col // Np
    vals = np.empty(ri.size, np.float64)
    for p in range(NPATCH):
        for q in range(p + 1):
            sel = np.nonzero((pr == p) & (pc == q))[0]
            if sel.size == 0:
                continue
            K = kernel(torch.cdist(X[p], X[q], compute_mode="donot_use_mm_for_euclid_dist"), torch) * W[p][:, None] * W[q][None, :]
            Y = fwt(K.reshape(Np, n, n), 2, J, torch)            # [cells p, wavelets q]
            del K
            Y = Y.T.contiguous()                                   # [wavelets q, cells p]
            C = fwt(Y.reshape(Np, n, n), 2, J, torch)            # [wavelets q, wavelets p]
            del Y
            li = torch.tensor(ri[sel] - p * Np, device=dev)
            lj = torch.tensor(col[sel] - q * Np, device=dev)
            vals[sel] = C[lj, li].cpu().numpy()
            del C
    vals[cp[:-1]] += nugget
    return vals


def sphere_workload(J: int = 7, ell: float = 0.3, nugget: float = 1e-3, nsamples: int = 128,
                    seed: int = 0, device: str = "cpu"):
    """The cubed-sphere configuration: 6 x 2^J x 2^J panels (J = 7: N = 98,304),
    exponential kernel on the chordal distance, nugget 1e-3; Z = nsamples
    standard normal vectors (rhs(N, nsamples, seed))."""
    b = sphere_basis(J)
    cp, ri = sphere_pattern(b, device)
    v = sphere_values(b, cp, ri, Kernel("exponential", ell), nugget, device)
    return b, cp, ri, v, rhs(b.N, nsamples, seed)
