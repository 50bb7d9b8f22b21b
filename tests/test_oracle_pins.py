"""Pins of the FP64 oracle against results fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a number the
paper prints, a closed form, the exact discrete result from a dense
eigendecomposition, an invariant, a convergence order, or finite differences.
A plausible mistake anywhere in the oracle (a dropped term, a wrong sign or
index, a transposed axis, a wrong coefficient) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2401_07416_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")
BOHR_A = 0.529177210903
HARTREE_EV = 27.211386245988
AU_TIME_AS = 24.188843265857


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------------------- paper values

def test_eq11_time_step_matches_paper_cu111():
    """Eq. 11 on the Cu(111) grid gives the 0.38 as printed after it (Sec. 2.1)."""
    gv = golden()["dt_cu111"]
    h = [e / n / BOHR_A for e, n in zip(gv["extent_angstrom"], gv["nodes"])]
    dt_as = oracle.default_dt(*h) * AU_TIME_AS
    assert round(dt_as, gv["printed_digits"]) == pytest.approx(gv["dt_attoseconds"])
    # the other printed extent (40.9 angstrom along x) would give 0.48 as instead
    h_alt = [40.9 / 240 / BOHR_A, 40.9 / 240 / BOHR_A, 70.0 / 420 / BOHR_A]
    assert oracle.default_dt(*h_alt) * AU_TIME_AS > 0.45


def test_eq4_wavelength_matches_de_broglie():
    """Eq. 4 in atomic units vs the textbook electron de Broglie relation."""
    gv = golden()["electron_wavelength"]
    for e_ev in gv["energies_eV"]:
        lam_bohr = oracle.wavelength(e_ev / HARTREE_EV)
        ref = gv["debroglie_constant_angstrom_sqrt_eV"] / math.sqrt(e_ev)
        assert lam_bohr * BOHR_A == pytest.approx(ref, rel=2e-5)


def test_mesh_point_counts():
    """Sec. 3.1 mesh counts (grid plus 100 CAP planes); the second printed value
    drops a digit, the product is 29,952,000."""
    gv = golden()["mesh_points"]
    counts = [nx * ny * (nz + gv["cap_planes"]) for nx, ny, nz in gv["grids"]]
    assert counts[0] == gv["printed"][0]
    assert counts[1] == 10 * gv["printed"][1]


# --------------------------------------------------------------------------- exact discrete map

@pytest.mark.parametrize("bc", [(1, 1, 1), (0, 0, 1), (0, 0, 0), (1, 0, 0)])
def test_leapfrog_equals_dense_eigen_map(bc):
    """N oracle steps equal the N-th power of the per-mode 2x2 leapfrog map of
    the dense Hamiltonian (Eqs. 8-9), on an anisotropic non-cubic grid."""
    g = W.small_grid(5, 6, 7, h=(0.21, 0.26, 0.33), bc=bc)
    V = W.random_potential(g, 11, 3.0)
    g.dt = 1.0
    g.dt = 1.5 / dense.spectral_radius_A(g, V)   # max |a| = 1.5 (stable, far from 0)
    R0 = W.random_field((g.nz, g.ny, g.nx), 1)
    I0 = W.random_field((g.nz, g.ny, g.nx), 2)
    R, I, _, _ = oracle.run(g, V, R0, I0, 60, use_mask=False, flux=False)
    Re, Ie = dense.leapfrog_exact(g, V, R0, I0, 60)
    scale = max(np.abs(Re).max(), np.abs(Ie).max())
    assert np.abs(R - Re).max() / scale < 1e-12
    assert np.abs(I - Ie).max() / scale < 1e-12


def test_apply_A_equals_dense_operator():
    """A f from the stencil loops equals -(dt/hbar) H f with the Kronecker H."""
    g = W.small_grid(4, 5, 6, h=(0.3, 0.2, 0.25), bc=(0, 1, 0))
    V = W.random_potential(g, 5)
    f = W.random_field((g.nz, g.ny, g.nx), 6)
    A = -(g.dt / g.hbar) * dense.hamiltonian(g, V)
    np.testing.assert_allclose(oracle.apply_A(g, V, f).ravel(), A @ f.ravel(), rtol=0,
                               atol=1e-14 * np.abs(A).max() * np.abs(f).max() * 10)


def _second_order_errors(naive):
    g = W.small_grid(7, 7, 7, h=(0.35, 0.35, 0.35), bc=(1, 1, 1))
    V = W.random_potential(g, 21, 0.5)
    packet = W.Packet(r0=(1.05, 1.05, 1.05), sigma=(0.6, 0.6, 0.6), k0=(0.0, 0.0, 1.5))
    R0, Ipsi = oracle.wavepacket(g, packet.r0, packet.sigma, packet.k0)
    T = 0.4
    errs = []
    for nsteps in (40, 80, 160):
        g.dt = T / nsteps
        I = oracle.init_half(g, V, R0, Ipsi, naive=naive)
        R, Ih, _, _ = oracle.run(g, V, R0, I, nsteps, use_mask=False, flux=False)
        psi0 = R0 + 1j * Ipsi
        ex_R = dense.schrodinger_exact(g, V, psi0, T).real
        ex_I = dense.schrodinger_exact(g, V, psi0, T - 0.5 * g.dt).imag
        errs.append(np.sqrt(np.sum((R - ex_R) ** 2 + (Ih - ex_I) ** 2)))
    return errs


def test_second_order_in_dt_against_exp_iHt():
    """Leapfrog vs exp(-iHt/hbar) psi0 from the dense H: error ratio 4 per dt halving
    (second order), which also fixes the signs of Eqs. 8 and 9."""
    e = _second_order_errors(naive=False)
    assert e[0] / e[1] == pytest.approx(4.0, abs=0.2)
    assert e[1] / e[2] == pytest.approx(4.0, abs=0.2)


def test_naive_half_step_start_is_first_order():
    """Starting with I = Im psi0 (no half step) loses an order: ratio ~2."""
    e = _second_order_errors(naive=True)
    assert e[1] / e[2] == pytest.approx(2.0, abs=0.3)


def test_stability_threshold():
    """Bounded at dt * max|eig(H)|/hbar = 1.98, divergent at 2.02."""
    g = W.small_grid(6, 6, 6, h=(0.3, 0.3, 0.3), bc=(0, 0, 0))
    V = W.random_potential(g, 3, 0.5)
    g.dt = 1.0
    lam = dense.spectral_radius_A(g, V)
    R0 = W.random_field((6, 6, 6), 4)
    I0 = W.random_field((6, 6, 6), 5)
    amp = {}
    for ratio in (1.98, 2.02):
        g.dt = ratio / lam
        R, I, _, _ = oracle.run(g, V, R0, I0, 600, use_mask=False, flux=False)
        amp[ratio] = np.abs(R).max() / np.abs(R0).max()
    assert amp[1.98] < 50
    assert amp[2.02] > 1e20


# --------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("bc", [(0, 0, 1), (1, 1, 1), (0, 0, 0)])
def test_Q_and_energy_conserved(bc):
    g = W.small_grid(10, 9, 12, h=(0.2, 0.2, 0.2), dt=0.004, bc=bc)
    V = W.random_potential(g, 8, 2.0)
    p = W.Packet((1.0, 0.9, 1.2), (0.5, 0.6, 0.5), (0.5, -0.3, 1.0))
    R, I = oracle.initial_state(g, p, V)
    o0 = oracle.observables(g, V, R, I)
    R2, I2, _, _ = oracle.run(g, V, R, I, 300, use_mask=False, flux=False)
    o1 = oracle.observables(g, V, R2, I2)
    assert abs(o1["Q"] / o0["Q"] - 1) < 1e-13
    assert abs(o1["energy"] / o0["energy"] - 1) < 1e-12
    # the paper's density R^2 + I^{n-1/2}^2 is not conserved exactly but stays O(dt)-close
    assert abs(o1["norm_paper"] / o0["Q"] - 1) < 1e-2


def test_mask_makes_Q_non_increasing():
    g = W.small_grid(8, 8, 40, h=(0.2, 0.2, 0.2), dt=0.004, bc=(0, 0, 1), mask=8, eta=0.5)
    p = W.Packet((0.8, 0.8, 1.5), (0.0, 0.0, 0.5), (0.0, 0.0, -3.0))
    R, I = oracle.initial_state(g, p)
    q_prev = oracle.observables(g, None, R, I)["Q"]
    for _ in range(30):
        R, I, _, _ = oracle.run(g, None, R, I, 5, use_mask=True, flux=False)
        q = oracle.observables(g, None, R, I)["Q"]
        assert q <= q_prev * (1 + 1e-14)
        q_prev = q
    assert q_prev < 0.9


def test_energy_of_discrete_plane_wave():
    """E of a lattice plane wave on a periodic grid is its closed-form eigenvalue
    sum_a (hbar^2 / (m h_a^2)) (1 - cos k_a h_a)."""
    g = W.small_grid(8, 10, 12, h=(0.3, 0.25, 0.2), dt=0.003, bc=(0, 0, 0))
    k = [2 * math.pi * m / (n * h) for m, n, h in ((1, g.nx, g.hx), (2, g.ny, g.hy),
                                                     (3, g.nz, g.hz))]
    z, y, x = np.meshgrid(np.arange(g.nz) * g.hz, np.arange(g.ny) * g.hy,
                          np.arange(g.nx) * g.hx, indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    R0 = np.cos(ph)
    I = oracle.init_half(g, None, R0, np.sin(ph))
    e_ref = sum((1 - math.cos(ka * ha)) / (ha * ha) for ka, ha in zip(k, (g.hx, g.hy, g.hz)))
    assert oracle.observables(g, None, R0, I)["energy"] == pytest.approx(e_ref, rel=1e-12)


def test_mask_profile_values():
    """cos^2 layer: interior 1, deepest cell cos^2(eta pi/2), innermost cos^2(eta pi/(2W))."""
    g = W.small_grid(4, 4, 60, mask=20, eta=0.1)
    M = oracle.mask(g)
    assert np.all(M[20:40] == 1.0)
    assert M[0] == pytest.approx(0.97552825814757682, rel=1e-14)  # cos^2(0.05 pi)
    assert M[-1] == pytest.approx(M[0], rel=1e-15)
    assert M[19] == pytest.approx(math.cos(0.1 * math.pi / 40) ** 2, rel=1e-15)
    assert np.all(np.diff(M[:20]) > 0) and np.all(np.diff(M[40:]) < 0)


# --------------------------------------------------------------------------- closed-form dynamics

def _free_packet_continuum(g, p, t):
    """Textbook free Gaussian packet, product over axes (hbar = m = 1)."""
    coords = np.meshgrid(np.arange(g.nz) * g.hz, np.arange(g.ny) * g.hy,
                         np.arange(g.nx) * g.hx, indexing="ij")
    coords = coords[::-1]  # x, y, z
    psi = np.ones((g.nz, g.ny, g.nx), dtype=complex)
    for a in range(3):
        s2, k = p.sigma[a] ** 2, p.k0[a]
        alpha = 1 + 1j * t / s2
        d = coords[a] - p.r0[a]
        psi *= alpha ** -0.5 * np.exp(-(d - k * t) ** 2 / (2 * s2 * alpha)
                                      + 1j * k * d - 0.5j * k * k * t)
    return psi


def test_free_packet_centroid_and_width():
    """Config-1 packet after t = 1: the centroid moves at the lattice group velocity
    (hbar/(m h)) sin(k h) averaged over the packet's momenta; widths follow
    sigma_t = sigma sqrt(1 + (hbar t cos(k0 h)/(m sigma^2))^2)."""
    wl = W.config1()
    g, p = wl.grid, wl.packet
    R, I = oracle.initial_state(g, p)
    o0 = oracle.observables(g, None, R, I)
    R, I, _, _ = oracle.run(g, None, R, I, wl.steps, use_mask=False, flux=False)
    o = oracle.observables(g, None, R, I)
    t = wl.steps * g.dt
    h, s, k0 = g.hz, p.sigma[2], p.k0[2]
    vbar = math.sin(k0 * h) / h * math.exp(-h * h / (4 * s * s))
    assert o["mean"][2] - o0["mean"][2] == pytest.approx(vbar * t, abs=0.02)
    assert abs(o["mean"][0] - p.r0[0]) < 1e-9
    var = o["second"] - o["mean"] ** 2
    sx = s * math.sqrt(1 + (t / s ** 2) ** 2)
    sz = s * math.sqrt(1 + (t * math.cos(k0 * h) / s ** 2) ** 2)
    assert var[0] == pytest.approx(sx * sx / 2, rel=0.01)
    assert var[1] == pytest.approx(sx * sx / 2, rel=0.01)
    assert var[2] == pytest.approx(sz * sz / 2, rel=0.02)
    assert o["Q"] == pytest.approx(o0["Q"], rel=1e-12)


@pytest.mark.slow
def test_free_packet_second_order_in_h():
    """Pointwise error vs the continuum packet, interior |z - <z>| < 3 sigma_t:
    ratio ~4 per halving of h at fixed box length and t."""
    errs = []
    for n, h in ((24, 0.5), (48, 0.25), (96, 0.125)):
        nz = n * 4 // 3
        g = W.Grid(nx=n, ny=n, nz=nz, hx=h, hy=h, hz=h, dt=0.0025,
                   bc=(W.DIRICHLET,) * 3)
        c = 0.5 * (n - 1) * h
        cz = 0.5 * (nz - 1) * h - 1.0
        p = W.Packet((c, c, cz), (1.5, 1.5, 1.5), (0.0, 0.0, 1.5))
        R, I = oracle.initial_state(g, p)
        nsteps = 400
        R, I, _, _ = oracle.run(g, None, R, I, nsteps, use_mask=False, flux=False)
        t = nsteps * g.dt
        ref0 = _free_packet_continuum(g, p, 0.0)
        scale = 1 / math.sqrt(np.sum(np.abs(ref0) ** 2) * h ** 3)
        ref = _free_packet_continuum(g, p, t) * scale
        refI = _free_packet_continuum(g, p, t - 0.5 * g.dt) * scale
        st = 1.5 * math.sqrt(1 + (t / 2.25) ** 2)
        z, y, x = np.meshgrid(np.arange(nz) * h, np.arange(n) * h, np.arange(n) * h,
                              indexing="ij")
        sel = ((np.abs(z - cz - p.k0[2] * t) < 2.5 * st) & (np.abs(y - c) < 2.5 * st)
               & (np.abs(x - c) < 2.5 * st))
        e = np.sqrt(np.sum((R - ref.real)[sel] ** 2 + (I - refI.imag)[sel] ** 2) * h ** 3)
        errs.append(e)
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.1)


def test_harmonic_coherent_state():
    """V = r^2/2: a displaced ground state oscillates as <x> = x0 cos t with
    constant width (variance 1/2)."""
    n, h = 40, 0.25
    c = 0.5 * (n - 1) * h
    g = W.Grid(nx=n, ny=n, nz=n, hx=h, hy=h, hz=h, dt=0.002, bc=(W.DIRICHLET,) * 3)
    z, y, x = np.meshgrid(*(np.arange(n) * h - c,) * 3, indexing="ij")
    V = 0.5 * (x * x + y * y + z * z)
    p = W.Packet((c + 1.0, c, c), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    R, I = oracle.initial_state(g, p, V)
    total = 0
    for target in (math.pi / 2, math.pi):
        nsteps = int(round(target / g.dt)) - total
        R, I, _, _ = oracle.run(g, V, R, I, nsteps, use_mask=False, flux=False)
        total += nsteps
        o = oracle.observables(g, V, R, I)
        t = total * g.dt
        assert o["mean"][0] - c == pytest.approx(math.cos(t), abs=0.03)
        var = o["second"] - o["mean"] ** 2
        # the lattice changes the width by O(h^2) ~ (0.25)^2 / 2
        assert var[0] == pytest.approx(0.5, rel=0.05)
        assert var[2] == pytest.approx(0.5, rel=0.05)


# --------------------------------------------------------------------------- flux

def test_flux_equals_probability_crossing_the_face():
    """Integrated detector flux equals the growth of Q on the +z side of the face,
    to O(dt) (the exact discrete identity uses (R^n + R^{n+1})/2)."""
    g = W.small_grid(8, 8, 60, h=(0.2, 0.2, 0.2), dt=0.002, bc=(0, 0, 1), det_k=30)
    p = W.Packet((0.8, 0.8, 4.0), (0.0, 0.0, 0.8), (0.0, 0.0, 2.0))
    V = W.random_potential(g, 9, 0.2)
    R, I = oracle.initial_state(g, p, V)

    def q_up(R, I):
        Ip = I + oracle.apply_A(g, V, R)
        return np.sum((R * R + Ip * I)[g.det_k + 1:]) * g.hx * g.hy * g.hz

    q0 = q_up(R, I)
    R2, I2, F, _ = oracle.run(g, V, R, I, 600, use_mask=False, flux=True)
    phi = F.sum() * g.hx * g.hy
    dq = q_up(R2, I2) - q0
    assert dq > 0.2
    assert phi == pytest.approx(dq, rel=2e-3)


def test_plane_wave_is_exact_and_its_flux_has_a_closed_form():
    """With V = 0 on a periodic z axis, the mode e^{ikz} is an eigenvector of A with
    eigenvalue -lam, lam = 4 c_z sin^2(kh/2), and Eqs. 8-9 are solved exactly by the
    unit plane wave R^n = cos(kz - n phi), I^{n+1/2} = sin(kz - (n+1/2) phi) with
    2 sin(phi/2) = lam (substituting gives that condition and unit amplitudes for
    both parts).  The face flux j = hbar/(m h)(R_k I_k+1 - R_k+1 I_k) of that
    solution is hbar sin(kh) cos(phi/2) / (m h) at every pixel and step."""
    h, dt, nz, mode, N = 0.2, 0.004, 32, 3, 37
    g = W.small_grid(4, 4, nz, h=(0.3, 0.25, h), dt=dt, bc=(0, 0, 0), det_k=10)
    k = 2.0 * math.pi * mode / (nz * h)
    lam = 4.0 * (g.hbar * dt / (2.0 * g.mass * h * h)) * math.sin(0.5 * k * h) ** 2
    phi = 2.0 * math.asin(0.5 * lam)
    kz = np.broadcast_to((k * h * np.arange(nz))[:, None, None], (nz, g.ny, g.nx))
    R, I, F, jl = oracle.run(g, None, np.cos(kz), np.sin(kz + 0.5 * phi), N,
                             use_mask=False, flux=True)
    assert np.abs(R - np.cos(kz - N * phi)).max() < 1e-12
    assert np.abs(I - np.sin(kz - (N - 0.5) * phi)).max() < 1e-12
    j = g.hbar * math.sin(k * h) * math.cos(0.5 * phi) / (g.mass * h)
    assert np.abs(jl - j).max() < 1e-12 * j
    assert np.abs(F - N * dt * j).max() < 1e-12 * N * dt * j


# --------------------------------------------------------------------------- potential

def test_single_atom_potential_closed_form():
    """No periodic axis: V = -Z / sqrt(r^2 + a^2) (softened Coulomb)."""
    g = W.small_grid(9, 10, 11, h=(0.3, 0.3, 0.3), bc=(1, 1, 1))
    atom = np.array([[1.1, 1.3, 1.7, 6.0]])
    V = oracle.potential_atoms(g, atom, a2=0.25)
    for (k, j, i) in [(0, 0, 0), (5, 4, 3), (10, 9, 8), (6, 4, 4)]:
        r2 = (i * 0.3 - 1.1) ** 2 + (j * 0.3 - 1.3) ** 2 + (k * 0.3 - 1.7) ** 2
        assert V[k, j, i] == pytest.approx(-6.0 / math.sqrt(r2 + 0.25), rel=1e-14)


def test_periodic_potential_cutoff_is_c1_and_minimum_image():
    g = W.small_grid(40, 40, 8, h=(0.1, 0.1, 0.1), bc=(0, 0, 1))
    rc = oracle.default_cutoff(g)
    assert rc == pytest.approx(2.0)
    atom = np.array([[0.05, 2.0, 0.3, 1.0]])
    V = oracle.potential_atoms(g, atom)
    # minimum image: x = 3.9 is 0.15 from the atom's image at 4.05, as is x = 0.2
    assert V[3, 20, 39] == pytest.approx(V[3, 20, 2], rel=1e-14)
    assert V[3, 20, 0] == pytest.approx(V[3, 20, 1], rel=1e-14)
    # zero beyond the cut-off; value, slope and curvature -> 0 at r_c (C2)
    line = np.array([[0.0, 0.0, 0.0, 1.0]])
    g1 = W.small_grid(4000, 1, 1, h=(0.001, 1.0, 1.0), bc=(0, 1, 1))
    v = oracle.potential_atoms(g1, line, rc=1.5)[0, 0]
    r = np.minimum(np.arange(4000), 4000 - np.arange(4000)) * 0.001
    assert np.all(v[r >= 1.5] == 0.0)
    i = 1499                                   # r = 1.499, next to r_c
    d1 = (v[i + 1] - v[i - 1]) / 0.002
    d2 = (v[i + 1] - 2 * v[i] + v[i - 1]) / 1e-6
    assert abs(v[i]) < 1e-8 and abs(d1) < 1e-5 and abs(d2) < 2e-2
    assert abs(v[500] - v[499]) / 0.001 > 0.1  # but not flat inside
    # with no cut-off the profile is the textbook softened Coulomb
    v_nc = oracle.potential_atoms(g1, line, rc=0.0)[0, 0]
    np.testing.assert_allclose(v_nc[:1000], -1 / np.sqrt(r[:1000] ** 2 + 0.25), rtol=1e-14)


def test_superposition_and_atom_gradient_by_finite_differences():
    g = W.small_grid(12, 12, 10, h=(0.25, 0.25, 0.25), bc=(0, 0, 1))
    atoms = np.array([[1.0, 1.2, 1.1, 6.0], [2.1, 0.4, 1.4, 8.0]])
    V = oracle.potential_atoms(g, atoms)
    V0 = oracle.potential_atoms(g, atoms[:1])
    V1 = oracle.potential_atoms(g, atoms[1:])
    np.testing.assert_allclose(V, V0 + V1, rtol=1e-13, atol=1e-14)
    w = W.random_potential(g, 33)
    grad = oracle.atom_gradient(g, atoms, w)
    eps = 1e-5
    for a in range(2):
        for p in range(4):
            ap, am = atoms.copy(), atoms.copy()
            ap[a, p] += eps
            am[a, p] -= eps
            fd = np.sum(w * (oracle.potential_atoms(g, ap) - oracle.potential_atoms(g, am))) / (2 * eps)
            assert grad[a, p] == pytest.approx(fd, rel=1e-6, abs=1e-8)


# --------------------------------------------------------------------------- packet

def test_wavepacket_normalised_and_shaped():
    g = W.small_grid(16, 16, 16, h=(0.2, 0.2, 0.2), bc=(1, 1, 1))
    p = W.Packet((1.5, 1.6, 1.4), (0.5, 0.6, 0.0), (0.3, 0.0, -2.0))
    R, I = oracle.wavepacket(g, p.r0, p.sigma, p.k0)
    assert np.sum(R * R + I * I) * 0.2 ** 3 == pytest.approx(1.0, rel=1e-14)
    amp = np.sqrt(R * R + I * I)
    # plane-wave axis z: |psi| constant along z
    np.testing.assert_allclose(amp[:, 5, 7], amp[0, 5, 7], rtol=1e-13)
    # Gaussian along x with sigma 0.5: amplitude ratio at distance 0.2 from r0 ...
    # ... vs distance 0: node x = 1.4 and 1.6 straddle r0 = 1.5
    a14, a16 = amp[3, 8, 7], amp[3, 8, 8]
    assert a14 == pytest.approx(a16, rel=1e-13)
    a12 = amp[3, 8, 6]
    assert a12 / a14 == pytest.approx(math.exp(-(0.3 ** 2 - 0.1 ** 2) / (2 * 0.25)), rel=1e-12)
    # phase advances by k0 . dr
    ph = np.angle(R + 1j * I)
    dz = np.angle(np.exp(1j * (ph[1, 5, 7] - ph[0, 5, 7])))
    assert dz == pytest.approx(-2.0 * 0.2, abs=1e-12)


# --------------------------------------------------------------------------- adjoint

def _loss(g, V, R0, I0, nsteps, target):
    R, I = R0, oracle.init_half(g, V, R0, I0)
    _, _, F, _ = oracle.run(g, V, R, I, nsteps, use_mask=True, flux=True)
    return float(np.sum((F - target) ** 2)), F


def _adjoint_case():
    g = W.small_grid(8, 8, 24, h=(0.25, 0.25, 0.25), dt=0.004, bc=(0, 0, 1), det_k=6,
                     mask=4, eta=0.5)
    atoms = np.array([[1.0, 1.0, 2.5, 6.0], [0.2, 1.5, 2.2, 8.0]])
    p = W.Packet((1.0, 1.0, 4.2), (0.0, 0.0, 0.7), (0.0, 0.0, -2.5))
    R0, I0 = oracle.wavepacket(g, p.r0, p.sigma, p.k0)
    return g, atoms, R0, I0


def test_adjoint_matches_finite_differences_in_V():
    g, atoms, R0, I0 = _adjoint_case()
    V = oracle.potential_atoms(g, atoms)
    nsteps = 160
    target = np.zeros((g.ny, g.nx))
    L0, F = _loss(g, V, R0, I0, nsteps, target)
    target = F * 0.5 + 0.01
    L0, F = _loss(g, V, R0, I0, nsteps, target)
    gV = oracle.adjoint(g, V, R0, I0, nsteps, 2 * (F - target))
    rng = np.random.default_rng(0)
    eps = 1e-4
    for trial in range(4):
        dV = rng.normal(size=V.shape)
        if trial == 0:           # a direction concentrated near the detector face
            dV[:g.det_k - 2] = 0
            dV[g.det_k + 4:] = 0
        lp, _ = _loss(g, V + eps * dV, R0, I0, nsteps, target)
        lm, _ = _loss(g, V - eps * dV, R0, I0, nsteps, target)
        fd = (lp - lm) / (2 * eps)
        assert np.sum(gV * dV) == pytest.approx(fd, rel=1e-6)


def test_adjoint_chain_rule_to_atoms_matches_finite_differences():
    g, atoms, R0, I0 = _adjoint_case()
    nsteps = 120
    V = oracle.potential_atoms(g, atoms)
    _, F = _loss(g, V, R0, I0, nsteps, np.zeros((g.ny, g.nx)))
    target = 0.7 * F
    _, F = _loss(g, V, R0, I0, nsteps, target)
    gatoms = oracle.atom_gradient(g, atoms, oracle.adjoint(g, V, R0, I0, nsteps, 2 * (F - target)))
    eps = 1e-4
    for a in range(2):
        for p in range(4):
            ap, am = atoms.copy(), atoms.copy()
            ap[a, p] += eps
            am[a, p] -= eps
            lp, _ = _loss(g, oracle.potential_atoms(g, ap), R0, I0, nsteps, target)
            lm, _ = _loss(g, oracle.potential_atoms(g, am), R0, I0, nsteps, target)
            assert gatoms[a, p] == pytest.approx((lp - lm) / (2 * eps), rel=1e-6)


# ---------------------------------------------------------------- Eqs. 15-16

def test_detector_frame_is_the_density_on_the_plane():
    """Eq. 15: the frame is R^2 + I^2 of the detector plane, nothing else."""
    from oracle import detector as D
    rng = np.random.default_rng(11)
    R = rng.normal(size=(6, 5, 4))
    I = rng.normal(size=(6, 5, 4))
    f = D.detector_frame(R, I, 3)
    assert f.shape == (5, 4)
    for y in range(5):
        for x in range(4):
            assert f[y, x] == R[3, y, x] ** 2 + I[3, y, x] ** 2


def test_dissimilarity_closed_forms():
    """Eq. 16 on inputs with a known answer.  (i) Trajectories that differ by a
    constant c on every pixel and frame: d = |c| sqrt(P dA).  (ii) A difference
    growing linearly in time, c t: the trapezoidal rule is exact for a linear
    integrand, so d = |c| sqrt(P dA) (t0 + t1) / 2 on [t0, t1] covered by frames."""
    from oracle import detector as D
    P, M, dA = 30, 7, 0.04
    t = np.linspace(0.0, 1.2, M)
    base = np.random.default_rng(3).uniform(0.0, 1.0, size=(M, P))
    c = 0.37
    frames = np.stack([base, base + c])
    d = D.dissimilarity(frames, t, 0.0, 1.2, dA)
    assert d[0, 1] == pytest.approx(c * np.sqrt(P * dA), rel=1e-13)
    lin = np.stack([base, base + c * t[:, None]])
    d = D.dissimilarity(lin, t, 0.0, 1.2, dA)
    assert d[0, 1] == pytest.approx(c * np.sqrt(P * dA) * 0.6, rel=1e-13)
    # window of frames 2..5: t0 = t[2], t1 = t[5]
    d = D.dissimilarity(lin, t, t[2], t[5], dA)
    assert d[0, 1] == pytest.approx(c * np.sqrt(P * dA) * 0.5 * (t[2] + t[5]), rel=1e-13)


def test_dissimilarity_is_a_metric():
    """Each frame's term is an L2 distance and the time sum has non-negative
    weights, so d is symmetric, zero on the diagonal, and obeys the triangle
    inequality."""
    from oracle import detector as D
    rng = np.random.default_rng(5)
    frames = rng.uniform(0.0, 1.0, size=(6, 5, 40))
    t = np.array([0.0, 0.1, 0.25, 0.3, 0.5])
    d = D.dissimilarity(frames, t, 0.05, 0.5, 0.01)
    assert np.all(np.diag(d) == 0.0)
    assert np.allclose(d, d.T, rtol=0, atol=0)
    for a in range(6):
        for b in range(6):
            for c in range(6):
                assert d[a, c] <= d[a, b] + d[b, c] + 1e-15
    # frame 0 lies outside the window: changing it changes nothing
    g = frames.copy()
    g[:, 0] += 5.0
    assert np.array_equal(D.dissimilarity(g, t, 0.05, 0.5, 0.01), d)


def test_dissimilarity_single_frame_window():
    """One frame inside [t0, t1] stands for the whole window: d = its L2 distance."""
    from oracle import detector as D
    rng = np.random.default_rng(8)
    frames = rng.uniform(size=(2, 3, 10))
    t = np.array([0.0, 1.0, 2.0])
    d = D.dissimilarity(frames, t, 0.5, 1.5, 0.3)
    expect = np.sqrt(0.3 * np.sum((frames[0, 1] - frames[1, 1]) ** 2))
    assert d[0, 1] == pytest.approx(expect, rel=1e-14)
    with pytest.raises(ValueError):
        D.dissimilarity(frames, t, 2.5, 3.0, 0.3)


# ---------------------------------------------------------------- Eq. 10 absorbing potential

def test_cap_mask_is_the_split_step_of_eq10():
    """MASK_CAP: each layer plane's factor is what the absorbing term alone,
    d psi/dt = -W psi / hbar, does over one step (checked by an ODE solve, not the
    closed form), with Eq. 10's W growing as the square of the depth into the layer
    and equal to mask_eta at the outermost plane."""
    import dataclasses
    from scipy.integrate import solve_ivp
    g = W.small_grid(4, 4, 40, dt=0.01, bc=(0, 0, 0))
    g = dataclasses.replace(g, mask_lo=12, mask_hi=0, mask_eta=30.0, mask_kind=W.MASK_CAP,
                            hbar=1.0)
    M = oracle.mask(g)
    assert np.all(M[12:] == 1.0)
    for k in range(12):
        depth = 12 - k                                  # 12 at the outermost plane k = 0
        Wk = 30.0 * (depth / 12.0) ** 2                 # Eq. 10: quadratic in the depth
        sol = solve_ivp(lambda t, y: -Wk * y, (0.0, g.dt), [1.0], rtol=1e-12, atol=1e-14)
        assert M[k] == pytest.approx(sol.y[0, -1], rel=1e-9)
    # quadratic profile: ln M is proportional to depth^2
    ratios = np.log(M[:12]) / np.log(M[0])
    assert np.allclose(ratios, ((12 - np.arange(12)) / 12.0) ** 2, rtol=1e-12)


def test_cap_absorbs_and_vanishes_at_zero_strength():
    """With the CAP the invariant Q never grows; with zero strength the layer is
    transparent (Q conserved as without any mask)."""
    import dataclasses
    g = W.small_grid(8, 8, 60, h=(0.3, 0.3, 0.2), dt=0.004, bc=(0, 0, 0))
    p = W.Packet((1.2, 1.2, 4.0), (0.0, 0.0, 1.0), (0.0, 0.0, -3.0))
    cap = dataclasses.replace(g, mask_lo=15, mask_kind=W.MASK_CAP, mask_eta=20.0)
    R, I = oracle.initial_state(cap, p, None)
    q = [oracle.observables(cap, None, R, I)["Q"]]
    for _ in range(30):
        R, I, _, _ = oracle.run(cap, None, R, I, 20, flux=False)
        q.append(oracle.observables(cap, None, R, I)["Q"])
    assert all(b <= a * (1 + 1e-13) for a, b in zip(q, q[1:]))
    assert q[-1] < 0.5 * q[0]                      # the packet ran into the layer
    off = dataclasses.replace(cap, mask_eta=0.0)
    R, I = oracle.initial_state(off, p, None)
    q0 = oracle.observables(off, None, R, I)["Q"]
    R, I, _, _ = oracle.run(off, None, R, I, 600, flux=False)
    assert oracle.observables(off, None, R, I)["Q"] == pytest.approx(q0, rel=1e-12)


# ---------------------------------------------------------------- potential interpolation

def test_interpolation_reproduces_lattice_values_and_tensor_products():
    """Trilinear interpolation of the periodic cell: (i) nodes that coincide with
    lattice points take the lattice value; (ii) a tensor product f(x) g(y) q(z) of
    periodic piecewise-linear functions with knots on the lattice is reproduced
    exactly everywhere (trilinear interpolation is exact on that space)."""
    from oracle import interp as OI
    cnx, cny, cnz = 6, 5, 7
    cell = (3.0, 2.5, 3.5)
    rng = np.random.default_rng(2)
    Vc = rng.normal(size=(cnz, cny, cnx))
    # (i) simulation spacing = lattice spacing, origin on the lattice
    h = (cell[0] / cnx, cell[1] / cny, cell[2] / cnz)
    V = OI.trilinear_periodic(Vc, cell, (0.0, 0.0, 0.0), (2 * cnz, cny, 3 * cnx), h)
    for k in range(2 * cnz):
        for i in range(3 * cnx):
            assert V[k, 2, i] == pytest.approx(Vc[k % cnz, 2, i % cnx], abs=1e-12)
    # (ii) tensor products of knot-wise linear periodic functions, off-lattice nodes
    fx, fy, fz = rng.normal(size=cnx), rng.normal(size=cny), rng.normal(size=cnz)
    Vt = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    origin = (0.31, -0.7, 1.9)

    def pl(vals, L, n, o, pos):                       # periodic piecewise-linear
        u = (pos - o) / L * n
        i0 = int(np.floor(u))
        t = u - i0
        return vals[i0 % n] * (1 - t) + vals[(i0 + 1) % n] * t

    hh = (0.37, 0.29, 0.41)
    V = OI.trilinear_periodic(Vt, cell, origin, (9, 8, 11), hh)
    for k in range(9):
        for j in range(8):
            for i in range(11):
                expect = (pl(fz, cell[2], cnz, origin[2], k * hh[2]) *
                          pl(fy, cell[1], cny, origin[1], j * hh[1]) *
                          pl(fx, cell[0], cnx, origin[0], i * hh[0]))
                assert V[k, j, i] == pytest.approx(expect, rel=1e-12, abs=1e-12)


def test_interpolation_matches_scipy_on_a_padded_lattice():
    """Independent check: scipy's RegularGridInterpolator on the lattice padded by
    one periodic image gives the same values."""
    from scipy.interpolate import RegularGridInterpolator
    from oracle import interp as OI
    cnx, cny, cnz = 7, 4, 9
    cell = (2.1, 1.3, 4.4)
    Vc = np.random.default_rng(9).normal(size=(cnz, cny, cnx))
    pad = np.pad(Vc, ((0, 1), (0, 1), (0, 1)), mode="wrap")
    axes = [np.arange(n + 1) * L / n for n, L in ((cnz, cell[2]), (cny, cell[1]), (cnx, cell[0]))]
    f = RegularGridInterpolator(axes, pad)
    h, origin = (0.23, 0.17, 0.31), (0.05, 0.4, -1.0)
    V = OI.trilinear_periodic(Vc, cell, origin, (10, 7, 12), h)
    pts = []
    for k in range(10):
        for j in range(7):
            for i in range(12):
                pts.append([((k * h[2] - origin[2]) % cell[2]), ((j * h[1] - origin[1]) % cell[1]),
                            ((i * h[0] - origin[0]) % cell[0])])
    ref = f(np.array(pts)).reshape(10, 7, 12)
    assert np.abs(V - ref).max() < 1e-12


def test_oracle_steps_independent_of_thread_count():
    """The step, packet and flux loops write per node: one thread and several give
    bit-identical results (so the serial and all-core timings run the same program)."""
    g = W.small_grid(12, 10, 16, h=(0.3, 0.35, 0.25), dt=0.01, bc=(0, 0, 1), mask=3, det_k=7)
    V = W.random_potential(g, 11, 1.5)
    p = W.Packet((1.8, 1.7, 2.0), (0.8, 0.9, 0.7), (0.4, -0.3, 1.1))
    n = oracle.max_threads()
    out = []
    try:
        for threads in (1, max(2, n)):
            oracle.set_threads(threads)
            R, I = oracle.initial_state(g, p, V)
            out.append(oracle.run(g, V, R, I, 9, use_mask=True, flux=True))
    finally:
        oracle.set_threads(n)
    for a, b in zip(out[0], out[1]):
        if isinstance(a, np.ndarray):
            assert np.array_equal(a, b)


# --------------------------------------------------------------------------- window forms

def _periodic_slab_case():
    """A 36 x 28 x 22 grid, periodic in x and y (Eqs. 13-14), walls and absorbing
    layers in z, a small seeded slab, and a packet that is a plane wave along x
    (one period of the box) and y (k = 0), Gaussian along z."""
    g = W.Grid(nx=36, ny=28, nz=22, hx=0.21, hy=0.19, hz=0.23, dt=0.004,
               bc=(W.PERIODIC, W.PERIODIC, W.DIRICHLET), mask_lo=3, mask_hi=3,
               mask_eta=0.4, det_k=-1)
    atoms = W.square_slab(3, 2, 2.1, 0.55 * g.lengths[2], 0.3, 0.7, W.rng_for(77), 0.05)
    kx = 2 * math.pi / g.lengths[0]
    packet = W.Packet((1.0, 1.0, 0.5 * g.lengths[2]), (0.0, 0.0, 0.8), (kx, 0.0, -1.2))
    return g, atoms, packet


WINDOWS = [(-5, -3), (20, 15), (0, 0), (29, 25), (-12, 17)]


def test_window_potential_equals_full_grid_slices():
    """The oracle's window form of the atom potential (node (0,0,0) at a non-zero
    origin, minimum image with the full grid's periods) equals the full-grid
    potential at the same nodes, including windows that cross the periodic seams
    or start at negative indices.  The full-grid form is pinned above (closed
    form, images, cut-off); this pins the window branch to it."""
    import light_cone as LC
    g, atoms, packet = _periodic_slab_case()
    V = oracle.potential_atoms(g, atoms)
    for x0, y0 in WINDOWS:
        sub, Vw, _, _ = LC.window_start(g, atoms, packet, x0, y0, 12)
        ref = LC.full_slice(V, g, x0, y0, 12)
        assert np.abs(Vw - ref).max() <= 1e-12 * np.abs(ref).max(), (x0, y0)


def test_window_packet_equals_full_grid_slices():
    """The window form of the Eq. 3 packet, rescaled by sqrt(window area / grid
    area) for a packet that is a plane wave along x and y, equals the full grid's
    normalised packet on the window's nodes; with a Gaussian along every axis
    and a window inside the grid, the window packet is the full one times a
    single constant (its own normalisation)."""
    import light_cone as LC
    g, atoms, packet = _periodic_slab_case()
    R, I = oracle.wavepacket(g, packet.r0, packet.sigma, packet.k0)
    for x0, y0 in WINDOWS:
        _, _, Rw, Iw = LC.window_start(g, atoms, packet, x0, y0, 12)
        Rr, Ir = LC.full_slice(R, g, x0, y0, 12), LC.full_slice(I, g, x0, y0, 12)
        scale = max(np.abs(Rr).max(), np.abs(Ir).max())
        assert max(np.abs(Rw - Rr).max(), np.abs(Iw - Ir).max()) <= 1e-12 * scale, (x0, y0)
    # Gaussian in x and y too: the window's origin enters each factor exactly once
    r0, sig = (3.5, 2.9, 2.6), (1.1, 0.9, 0.8)
    R, I = oracle.wavepacket(g, r0, sig, packet.k0)
    sub = LC.window_grid(g, 12)
    Rw, Iw = oracle.wavepacket_window(sub, (10 * g.hx, 7 * g.hy, 0.0), r0, sig, packet.k0)
    Rr, Ir = R[:, 7:19, 10:22], I[:, 7:19, 10:22]
    c = np.sqrt(np.sum(Rw ** 2 + Iw ** 2) / np.sum(Rr ** 2 + Ir ** 2))
    assert np.abs(Rw - c * Rr).max() <= 1e-12 * np.abs(Rw).max()
    assert np.abs(Iw - c * Ir).max() <= 1e-12 * np.abs(Iw).max()


@pytest.mark.parametrize("steps", [1, 3])
def test_light_cone_window_equals_full_periodic_run(steps):
    """After N steps, window nodes more than 2N + 1 cells inside the window's walls
    hold the full periodic run's values (the claim the 512 x 512 x 1024 GPU check
    rests on), while nodes next to the walls do not (the check can fail)."""
    import light_cone as LC
    g, atoms, packet = _periodic_slab_case()
    V = oracle.potential_atoms(g, atoms)
    R0, I0 = oracle.wavepacket(g, packet.r0, packet.sigma, packet.k0)
    Rf, If, _, _ = oracle.run(g, V, R0, oracle.init_half(g, V, R0, I0), steps, flux=False)
    width = 2 * LC.margin(steps) + 6
    m = LC.margin(steps)
    inner = (slice(None), slice(m, width - m), slice(m, width - m))
    for x0, y0 in WINDOWS:
        Rw, Iw = LC.window_run(g, atoms, packet, x0, y0, width, steps)
        Rr, Ir = LC.full_slice(Rf, g, x0, y0, width), LC.full_slice(If, g, x0, y0, width)
        scale = max(np.abs(Rr).max(), np.abs(Ir).max())
        err = max(np.abs(Rw - Rr)[inner].max(), np.abs(Iw - Ir)[inner].max())
        assert err <= 1e-12 * scale, (x0, y0, err / scale)
        edge = max(np.abs(Rw - Rr)[:, :, 0].max(), np.abs(Iw - Ir)[:, :, 0].max())
        assert edge > 1e-6 * scale, (x0, y0)
