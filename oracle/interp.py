"""Oracle of the potential interpolation step of arXiv 2401.07416, Sec. 2.3 / 3.2.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, FP64.

The paper computes the potential of one periodic cell (DFT) and then expands and
interpolates it onto the simulation mesh (the step it reports as dominant).
Reading: the cell's potential is given on a regular cnx x cny x cnz lattice,
Vc[k][j][i] at origin + (i Lx / cnx, j Ly / cny, k Lz / cnz), periodic with the
cell lengths (Lx, Ly, Lz) in every axis (the expansion tiles the cell); V at a
simulation node r = (i hx, j hy, k hz) (Sec. 2.1) is the trilinear interpolation
of that periodic lattice at r.
"""
from __future__ import annotations

import math

import numpy as np


def trilinear_periodic(Vc: np.ndarray, cell, origin, shape, h) -> np.ndarray:
    """V[nz][ny][nx] on the simulation nodes (i hx, j hy, k hz) from the periodic
    coarse lattice Vc[cnz][cny][cnx] of cell lengths `cell` starting at `origin`."""
    Vc = np.asarray(Vc, dtype=np.float64)
    cnz, cny, cnx = Vc.shape
    nz, ny, nx = shape
    out = np.empty((nz, ny, nx))

    def locate(pos, o, L, n):
        u = (pos - o) / L * n            # lattice coordinate
        i0 = math.floor(u)
        f = u - i0
        return i0 % n, (i0 + 1) % n, f

    xs = [locate(i * h[0], origin[0], cell[0], cnx) for i in range(nx)]
    ys = [locate(j * h[1], origin[1], cell[1], cny) for j in range(ny)]
    zs = [locate(k * h[2], origin[2], cell[2], cnz) for k in range(nz)]
    for k, (z0, z1, fz) in enumerate(zs):
        for j, (y0, y1, fy) in enumerate(ys):
            for i, (x0, x1, fx) in enumerate(xs):
                c00 = Vc[z0, y0, x0] * (1 - fx) + Vc[z0, y0, x1] * fx
                c01 = Vc[z0, y1, x0] * (1 - fx) + Vc[z0, y1, x1] * fx
                c10 = Vc[z1, y0, x0] * (1 - fx) + Vc[z1, y0, x1] * fx
                c11 = Vc[z1, y1, x0] * (1 - fx) + Vc[z1, y1, x1] * fx
                c0 = c00 * (1 - fy) + c01 * fy
                c1 = c10 * (1 - fy) + c11 * fy
                out[k, j, i] = c0 * (1 - fz) + c1 * fz
    return out
