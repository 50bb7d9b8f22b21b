"""Dense-matrix statements of the discrete problem, for pinning the oracle.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

On small grids (up to ~10^3 nodes) the finite-difference Hamiltonian of Eq. 2,
H = -(hbar^2 / 2m) (Lx + Ly + Lz) + diag(V), is built here as a dense matrix from
Kronecker products of 1-D second-difference matrices (a construction independent
of the stencil loops in ``tdse_oracle.c``) and diagonalised with
``numpy.linalg.eigh``.  Two exact results follow:

* The leapfrog of Eqs. 8-9 acts on each eigenmode of A = -(dt/hbar) H (eigenvalue a)
  as the 2x2 map  (r, i) -> ((1 - a^2) r - a i, a r + i)  on (R^n, I^{n-1/2}).  Its
  N-th power is the exact discrete result after N steps, up to rounding.
* exp(-i H t / hbar) psi0 is the exact solution of the semi-discrete equation; the
  leapfrog must approach it at second order in dt.
"""
from __future__ import annotations

import numpy as np


def second_difference(n: int, h: float, periodic: bool) -> np.ndarray:
    """(f[i+1] - 2 f[i] + f[i-1]) / h^2 with wrap-around (Eqs. 13-14) or zero walls."""
    L = np.zeros((n, n))
    for i in range(n):
        L[i, i] = -2.0
        if i + 1 < n:
            L[i, i + 1] = 1.0
        elif periodic:
            L[i, (i + 1) % n] += 1.0
        if i - 1 >= 0:
            L[i, i - 1] = 1.0
        elif periodic:
            L[i, (i - 1) % n] += 1.0
    return L / (h * h)


def hamiltonian(g, V=None) -> np.ndarray:
    """Dense H for the [nz][ny][nx] (x fastest) ordering."""
    Ix, Iy, Iz = np.eye(g.nx), np.eye(g.ny), np.eye(g.nz)
    Lx = second_difference(g.nx, g.hx, g.bc[0] == 0)
    Ly = second_difference(g.ny, g.hy, g.bc[1] == 0)
    Lz = second_difference(g.nz, g.hz, g.bc[2] == 0)
    lap = (np.kron(Iz, np.kron(Iy, Lx)) + np.kron(Iz, np.kron(Ly, Ix))
           + np.kron(Lz, np.kron(Iy, Ix)))
    H = -(g.hbar ** 2) / (2.0 * g.mass) * lap
    if V is not None:
        H = H + np.diag(np.asarray(V, dtype=np.float64).ravel())
    return H


def leapfrog_exact(g, V, R0, Ihalf, nsteps: int):
    """(R^N, I^{N-1/2}) of the unmasked leapfrog, from the eigen-decomposition of A."""
    A = -(g.dt / g.hbar) * hamiltonian(g, V)
    a, U = np.linalg.eigh(A)
    r = U.T @ np.asarray(R0, dtype=np.float64).ravel()
    i = U.T @ np.asarray(Ihalf, dtype=np.float64).ravel()
    # 2x2 per-mode map raised to the N-th power by repeated squaring
    m11, m12, m21, m22 = 1.0 - a * a, -a, a, np.ones_like(a)
    p11, p12, p21, p22 = np.ones_like(a), np.zeros_like(a), np.zeros_like(a), np.ones_like(a)
    n = int(nsteps)
    while n:
        if n & 1:
            p11, p12, p21, p22 = (m11 * p11 + m12 * p21, m11 * p12 + m12 * p22,
                                  m21 * p11 + m22 * p21, m21 * p12 + m22 * p22)
        m11, m12, m21, m22 = (m11 * m11 + m12 * m21, m11 * m12 + m12 * m22,
                              m21 * m11 + m22 * m21, m21 * m12 + m22 * m22)
        n >>= 1
    rN = p11 * r + p12 * i
    iN = p21 * r + p22 * i
    shp = (g.nz, g.ny, g.nx)
    return (U @ rN).reshape(shp), (U @ iN).reshape(shp)


def schrodinger_exact(g, V, psi0: np.ndarray, t: float) -> np.ndarray:
    """exp(-i H t / hbar) psi0 for the dense H."""
    E, U = np.linalg.eigh(hamiltonian(g, V))
    c = U.T @ np.asarray(psi0, dtype=np.complex128).ravel()
    return (U @ (np.exp(-1j * E * t / g.hbar) * c)).reshape((g.nz, g.ny, g.nx))


def spectral_radius_A(g, V=None) -> float:
    """max |a| over the eigenvalues a of A = -(dt/hbar) H (the leapfrog is stable
    for max |a| < 2)."""
    a = np.linalg.eigvalsh(-(g.dt / g.hbar) * hamiltonian(g, V))
    return float(np.max(np.abs(a)))
