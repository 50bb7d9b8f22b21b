"""Oracle runs on a window of a grid that is periodic in x and y (test helper).

The full 512 x 512 x 1024 grid is beyond what the oracle can run in a test, so its
GPU state is checked on columns: a window of width x width nodes starting at
node (x0, y0) (any integers; the window may wrap across the periodic seams),
all nz planes, with walls on the window's x and y faces.  The window's potential
and packet are those of the full grid at the same positions (the oracle's
window forms, with the full grid's periods for the minimum image).  The leapfrog
reads one neighbour per half step and the half-step start applies A once, so a
wall's influence moves in by at most 2N + 1 cells in N steps: nodes farther
than that from the window's faces hold the full grid's values.  These facts are
pinned on the CPU in test_oracle_pins.py against full-grid oracle runs.
"""
import math

import numpy as np

import oracle
from paper_2401_07416_gb300 import workloads as W


def margin(steps: int) -> int:
    """Cells from a window face beyond which the window equals the full grid."""
    return 2 * steps + 2


def window_grid(g, width: int):
    return W.Grid(nx=width, ny=width, nz=g.nz, hx=g.hx, hy=g.hy, hz=g.hz, dt=g.dt,
                  bc=(W.DIRICHLET, W.DIRICHLET, g.bc[2]), mask_lo=g.mask_lo,
                  mask_hi=g.mask_hi, mask_eta=g.mask_eta, det_k=-1,
                  mask_kind=getattr(g, "mask_kind", 0))


def window_start(g, atoms, packet, x0: int, y0: int, width: int):
    """(window grid, V, R^0, Im psi0) of the window at node (x0, y0) of grid g.
    The packet must be a plane wave along x and y (sigma <= 0 there, k0 a
    multiple of 2 pi / L on each axis): its per-column norm is then the same in
    every column, so the full grid's normalisation is the window's times
    sqrt(window area / grid area)."""
    assert packet.sigma[0] <= 0 and packet.sigma[1] <= 0
    sub = window_grid(g, width)
    origin = (x0 * g.hx, y0 * g.hy, 0.0)
    L = g.lengths
    period = [l if b == W.PERIODIC else 0.0 for l, b in zip(L, g.bc)]
    V = oracle.potential_atoms_window(sub, origin, period, atoms, rc=oracle.default_cutoff(g))
    R0, I0 = oracle.wavepacket_window(sub, origin, packet.r0, packet.sigma, packet.k0)
    s = math.sqrt((width * width) / (g.nx * g.ny))
    return sub, V, R0 * s, I0 * s


def window_run(g, atoms, packet, x0: int, y0: int, width: int, steps: int):
    """Oracle (R^N, I^{N-1/2}) on the window after `steps` steps."""
    sub, V, R0, I0 = window_start(g, atoms, packet, x0, y0, width)
    R, I, _, _ = oracle.run(sub, V, R0, oracle.init_half(sub, V, R0, I0), steps, flux=False)
    return R, I


def full_slice(a, g, x0: int, y0: int, width: int):
    """The window's nodes of a full-grid array [nz][ny][nx] (wrapping in x, y)."""
    xs = np.arange(x0, x0 + width) % g.nx
    ys = np.arange(y0, y0 + width) % g.ny
    return a[:, ys][:, :, xs]
