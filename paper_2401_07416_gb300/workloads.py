"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmarks.

This module holds geometry and parameters only: grid shapes, spacings, time steps,
boundary flags, absorbing-layer widths, detector-plane indices, wave-packet
parameters, atom positions and charges, and seeded random test arrays.  It holds
none of the method's arithmetic: the potential, the wave packet, the stencil, the
mask profile and every observable are computed separately by the CUDA library and
by the oracle.

Units are atomic units throughout (hbar = m = 1, lengths in bohr, time in a.u.).

The five workloads stand in for the paper's electron-diffraction runs (Sec. 2.3):
an electron Gaussian packet (Eq. 3) moving toward -z onto a slab of softened-Coulomb
atoms, with periodic x, y (Sec. 2.1) and an absorbing layer along z (Eq. 10 is
replaced by a multiplicative cos^2 layer).  The paper's DFT potentials and its
C6-SAM structures are not available; synthetic slabs with the same shape of
problem replace them.

Geometry conventions (the paper leaves them open):
  * nodes sit at r = (i hx, j hy, k hz), i, j, k >= 0 (Sec. 2.1, Eqs. 6-7);
  * the top atomic layer is at z_t = 0.40 Lz, further layers one lattice constant
    below it;
  * the packet centre is 2.5 bohr above the top layer;
  * the detector face lies 1.0 bohr below the lowest layer (transmission);
  * seeds: member m of workload c uses numpy default_rng(1000 c + m).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

PERIODIC = 0
DIRICHLET = 1

MASK_COS2 = 0
MASK_CAP = 1
FP64 = 0
FP32 = 1
FP32_KAHAN = 2


@dataclasses.dataclass
class Grid:
    """Uniform grid, time step and boundary treatment of one simulation."""

    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float
    dt: float
    hbar: float = 1.0
    mass: float = 1.0
    bc: Tuple[int, int, int] = (PERIODIC, PERIODIC, DIRICHLET)
    mask_lo: int = 0          # absorbing cells at the z = 0 end
    mask_hi: int = 0          # absorbing cells at the z = nz-1 end
    mask_eta: float = 0.1     # absorbing-layer strength (cos^2: eta; CAP: W at the outer plane)
    det_k: int = -1           # detector face between planes det_k and det_k+1 (-1: off)
    obs_every: int = 20       # period of the norm/energy reductions (Sec. 2.3: h = 20)
    mask_kind: int = 0        # MASK_COS2, or MASK_CAP: Eq. 10's quadratic potential, split

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def lengths(self) -> Tuple[float, float, float]:
        return (self.nx * self.hx, self.ny * self.hy, self.nz * self.hz)


@dataclasses.dataclass
class Packet:
    """Gaussian packet parameters (Eq. 3 with a vector wave number).

    sigma[a] <= 0 marks a plane-wave axis (no Gaussian factor along a).
    """

    r0: Tuple[float, float, float]
    sigma: Tuple[float, float, float]
    k0: Tuple[float, float, float]


@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    packet: Packet
    atoms: Optional[np.ndarray]     # [n, 4] rows (x, y, z, Z), or None for V = 0
    soft_a2: float = 0.25           # softening a^2 in -Z / sqrt(r^2 + a^2)
    steps: int = 0
    precision: int = FP64


def rng_for(config: int, member: int = 0) -> np.random.Generator:
    return np.random.default_rng(1000 * config + member)


def square_slab(n_side: int, layers: int, spacing: float, z_top: float,
                lx: float, ly: float, rng: np.random.Generator,
                jitter: float, charges=(6.0, 8.0)) -> np.ndarray:
    """Atoms of a square-lattice slab, layer l at z_top - l*spacing.

    Sites are ((i + 1/2) ax, (j + 1/2) ay) with ax = lx / n_side, so the lattice
    tiles the periodic cell; each position gets an isotropic Gaussian jitter and
    each atom a charge drawn uniformly from `charges`.
    """
    ax, ay = lx / n_side, ly / n_side
    rows = []
    for layer in range(layers):
        for j in range(n_side):
            for i in range(n_side):
                rows.append(((i + 0.5) * ax, (j + 0.5) * ay, z_top - layer * spacing))
    pos = np.asarray(rows, dtype=np.float64)
    pos += rng.normal(0.0, jitter, size=pos.shape)
    z = rng.choice(np.asarray(charges, dtype=np.float64), size=(pos.shape[0], 1))
    return np.hstack([pos, z])


def benzene_like(center: Tuple[float, float, float], angle: float) -> np.ndarray:
    """Rigid 12-atom ring molecule in the xy plane: 6 C on a 2.65-bohr ring and
    6 H on a 4.7-bohr ring at the same angles, rotated by `angle`."""
    rows = []
    for radius, charge in ((2.65, 6.0), (4.7, 1.0)):
        for s in range(6):
            a = angle + s * math.pi / 3.0
            rows.append((center[0] + radius * math.cos(a),
                         center[1] + radius * math.sin(a),
                         center[2], charge))
    return np.asarray(rows, dtype=np.float64)


def _diffraction_grid(nx, ny, nz, h, dt, bottom_z) -> Grid:
    det_z = bottom_z - 1.0
    return Grid(nx=nx, ny=ny, nz=nz, hx=h, hy=h, hz=h, dt=dt,
                bc=(PERIODIC, PERIODIC, DIRICHLET), mask_lo=20, mask_hi=20,
                mask_eta=0.1, det_k=int(math.floor(det_z / h)), obs_every=20)


def _incident_packet(grid: Grid, z_top: float) -> Packet:
    lx, ly, _ = grid.lengths
    return Packet(r0=(0.5 * lx, 0.5 * ly, z_top + 2.5), sigma=(0.0, 0.0, 2.0),
                  k0=(0.0, 0.0, -1.9))


def config1() -> Workload:
    """64^3 free packet, h = 0.2, dt = 0.002, V = 0, zero Dirichlet walls, 500 steps."""
    n, h = 64, 0.2
    g = Grid(nx=n, ny=n, nz=n, hx=h, hy=h, hz=h, dt=0.002,
             bc=(DIRICHLET, DIRICHLET, DIRICHLET), det_k=-1, obs_every=20)
    c = 0.5 * (n - 1) * h
    return Workload("free-packet 64^3 FP64", g,
                    Packet(r0=(c, c, c), sigma=(1.5, 1.5, 1.5), k0=(0.0, 0.0, 2.0)),
                    atoms=None, steps=500, precision=FP64)


def config2(precision: int = FP32_KAHAN) -> Workload:
    """128x128x256 diffraction run: 2 layers x 4x4 atoms, spacing 3.2, 4000 steps."""
    nx, ny, nz, h = 128, 128, 256, 0.1
    lz = nz * h
    z_top = 0.40 * lz
    atoms = square_slab(4, 2, 3.2, z_top, nx * h, ny * h, rng_for(2), 0.05)
    g = _diffraction_grid(nx, ny, nz, h, 5e-4, z_top - 3.2)
    return Workload("diffraction 128x128x256", g, _incident_packet(g, z_top), atoms,
                    steps=4000, precision=precision)


def config3(members: int = 48, precision: int = FP32_KAHAN) -> List[Workload]:
    """Batch of organic-film members on uneven grids (x, y in {96,128,160}, z in {192,256})."""
    out = []
    for m in range(members):
        rng = rng_for(3, m)
        nx = int(rng.choice([96, 128, 160]))
        ny = int(rng.choice([96, 128, 160]))
        nz = int(rng.choice([192, 256]))
        h = 0.1
        lx, ly, lz = nx * h, ny * h, nz * h
        z_top = 0.40 * lz
        centre = np.array([0.5 * lx, 0.5 * ly, z_top]) + rng.normal(0.0, 0.3, size=3)
        atoms = benzene_like(tuple(centre), float(rng.uniform(0.0, 2.0 * math.pi)))
        g = _diffraction_grid(nx, ny, nz, h, 5e-4, float(centre[2]))
        out.append(Workload(f"film member {m} ({nx}x{ny}x{nz})", g,
                            _incident_packet(g, float(centre[2])), atoms,
                            steps=2000, precision=precision))
    return out


def config4(precision: int = FP32_KAHAN) -> Workload:
    """96x96x192 adjoint case: 2 layers x 4x4 atoms (spacing 2.4), 3000 steps."""
    nx, ny, nz, h = 96, 96, 192, 0.1
    lz = nz * h
    z_top = 0.40 * lz
    a = nx * h / 4
    atoms = square_slab(4, 2, a, z_top, nx * h, ny * h, rng_for(4), 0.05)
    g = _diffraction_grid(nx, ny, nz, h, 5e-4, z_top - a)
    return Workload("adjoint 96x96x192", g, _incident_packet(g, z_top), atoms,
                    steps=3000, precision=precision)


def config4_target_atoms(atoms: np.ndarray) -> np.ndarray:
    """Target structure of the adjoint loss: every position perturbed by N(0, 0.1^2)."""
    rng = rng_for(4, 1)
    out = atoms.copy()
    out[:, :3] += rng.normal(0.0, 0.1, size=(atoms.shape[0], 3))
    return out


def config5(precision: int = FP32_KAHAN) -> Workload:
    """512x512x1024 throughput run: 4 layers x 16x16 atoms (spacing 1.6), 1000 steps."""
    nx, ny, nz, h = 512, 512, 1024, 0.05
    lz = nz * h
    z_top = 0.40 * lz
    a = nx * h / 16
    atoms = square_slab(16, 4, a, z_top, nx * h, ny * h, rng_for(5), 0.05)
    g = _diffraction_grid(nx, ny, nz, h, 5e-4, z_top - 3 * a)
    return Workload("throughput 512x512x1024", g, _incident_packet(g, z_top), atoms,
                    steps=1000, precision=precision)


# Atomic-unit conversions for the paper's SI / eV / angstrom settings.
BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
HARTREE_PER_EV = 1.0 / 27.211386245988


def wavevector_from_energy(E: float, hbar: float = 1.0, mass: float = 1.0) -> float:
    """Eq. 4: lambda = sqrt(2 hbar^2 pi^2 / (m E)), so |k| = 2 pi / lambda = sqrt(2 m E) / hbar."""
    lam = math.sqrt(2.0 * hbar * hbar * math.pi * math.pi / (mass * E))
    return 2.0 * math.pi / lam


def cu111(precision: int = FP32_KAHAN, nx: int = 240, ny: int = 240, nz: int = 420,
          cap_planes: int = 100, cap_strength: float = 2.0) -> Workload:
    """The paper's Cu(111) electron-diffraction geometry (Sec. 2.1 and Sec. 3.1) with a
    synthetic potential.

    Mesh: 240 x 240 x 420 nodes over 35.4 x 35.4 x 70 angstrom (anisotropic: h_x =
    h_y = 0.1475 A, h_z = 0.1667 A; the 35.4 A extent is the one that reproduces
    Eq. 11's 0.38 as), plus `cap_planes` absorbing planes appended at the bottom of
    a z-periodic domain (Eq. 10's set-up, here as the quadratic split-step layer of
    strength `cap_strength` Ha).  dt from Eq. 11.  Packet (Eqs. 3-4): sigma = 1.8 A,
    E = 60 eV, centred in x, y at r_z0 = 42 A above the appended region, moving -z.
    Slab (synthetic stand-in for the DFT potential): four Cu(111)-like layers of
    15 x 15 atoms, 2.087 A apart with the top layer at 30 A, each layer's square
    lattice shifted by a third of a site from the one above (ABC stacking), charge
    11 (the 3d10 4s1 valence shell) in the softened Coulomb form.  The detector
    plane sits at 37.6 A (Sec. 2.3).  Smaller nx, ny keep the spacings and the atom
    density (15 atoms per 240 nodes; a narrow window of the same geometry for tests)."""
    A = BOHR_PER_ANGSTROM
    hx = hy = 35.4 / 240 * A
    hz = 70.0 / 420 * A
    z0 = cap_planes * hz                       # the physical domain starts above the layer
    lx, ly = nx * hx, ny * hy
    g = Grid(nx=nx, ny=ny, nz=nz + cap_planes, hx=hx, hy=hy, hz=hz, dt=0.0,
             bc=(PERIODIC, PERIODIC, PERIODIC), mask_lo=cap_planes, mask_hi=0,
             mask_eta=cap_strength, mask_kind=MASK_CAP,
             det_k=min(nz + cap_planes - 2, int(round(z0 / hz + 37.6 * A / hz))), obs_every=20)
    n_side = max(1, round(15 * nx / 240))
    ax, ay = lx / n_side, ly / n_side
    rows = []
    for layer in range(4):
        z = z0 + (30.0 - 2.087 * layer) * A
        shift = (layer % 3) / 3.0
        for j in range(n_side):
            for i in range(n_side):
                rows.append(((i + 0.5 + shift) * ax % lx, (j + 0.5 + shift) * ay % ly, z, 11.0))
    atoms = np.array(rows)
    k = wavevector_from_energy(60.0 * HARTREE_PER_EV)
    packet = Packet((0.5 * lx, 0.5 * ly, z0 + 42.0 * A), (1.8 * A, 1.8 * A, 1.8 * A), (0.0, 0.0, -k))
    return Workload("Cu(111) 240x240x420 + 100 CAP planes", g, packet, atoms, steps=8000,
                    precision=precision)


def random_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded standard-normal test array (FP64)."""
    return np.random.default_rng(seed).normal(0.0, scale, size=shape)


def random_potential(grid: Grid, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded smooth-free random potential V[nz][ny][nx] for operator tests."""
    return random_field((grid.nz, grid.ny, grid.nx), seed, scale)


def small_grid(nx, ny, nz, h=(0.2, 0.25, 0.3), dt=2e-3, bc=(DIRICHLET,) * 3,
               mask=0, det_k=-1, eta=0.1) -> Grid:
    """Small anisotropic grid for unit and parity tests."""
    return Grid(nx=nx, ny=ny, nz=nz, hx=h[0], hy=h[1], hz=h[2], dt=dt, bc=tuple(bc),
                mask_lo=mask, mask_hi=mask, mask_eta=eta, det_k=det_k, obs_every=20)
