"""Adjoint (reverse-time leapfrog with FP64 checkpoints) through the C ABI.

Pins: (1) the GPU FP64 adjoint equals the oracle's stored-state adjoint on a small
case (dL/dV and the atom chain rule), max |diff| / max |ref| <= 1e-9; (2) the
FP32 and FP32+Kahan adjoints agree with the FP64 adjoint to 2e-3 (relative L2 of
dL/dV); (3) at the 96x96x192, 3000-step size, the FP64 adjoint gradient through
the torch.autograd wrappers agrees with central finite differences of the GPU
forward (eps = 1e-4) to 1e-6 relative, component by component: all 128 atom
parameters (32 positions and charges) and dL/dV along 16 seeded directions
(whole grid, around the slab, in the absorbing layers).  Each derivative is held
to 1e-6 of max(|fd|, 1e-3 x the largest |fd| of its kind): components far below
the largest of their kind are held to that absolute floor.
"""
import numpy as np
import pytest

import oracle
from paper_2401_07416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_07416_gb300 import build
    build.build()
    from paper_2401_07416_gb300 import tdse
    return tdse


def small_case():
    g = W.small_grid(8, 8, 24, h=(0.25, 0.25, 0.25), dt=0.004, bc=(0, 0, 1), det_k=6,
                     mask=4, eta=0.5)
    atoms = np.array([[1.0, 1.0, 2.5, 6.0], [0.2, 1.5, 2.2, 8.0]])
    p = W.Packet((1.0, 1.0, 4.2), (0.0, 0.0, 0.7), (0.0, 0.0, -2.5))
    return g, atoms, p


def gpu_gradients(T, g, atoms, p, nsteps, target, precision, ckpt=10):
    from paper_2401_07416_gb300.sim import Sim
    with Sim(g, precision=precision, ckpt_every=ckpt) as s:
        s.set_atoms(0, atoms)
        s.set_packet(0, p)
        s.step(nsteps)
        F = s.flux_map(0)
        gF = 2 * (F - target)
        gV = np.zeros((g.nz, g.ny, g.nx))
        ga = np.zeros_like(atoms)
        T.tdse_adjoint(s.ctx, 0, gF, gV, ga)
    return F, gV, ga


def test_fp64_adjoint_matches_oracle(T):
    g, atoms, p = small_case()
    n = 160
    V = oracle.potential_atoms(g, atoms)
    R0, I0 = oracle.wavepacket(g, p.r0, p.sigma, p.k0)
    _, _, F0, _ = oracle.run(g, V, R0, oracle.init_half(g, V, R0, I0), n)
    target = 0.5 * F0 + 0.01
    F, gV, ga = gpu_gradients(T, g, atoms, p, n, target, T.FP64)
    assert np.abs(F - F0).max() <= 1e-11 * np.abs(F0).max()
    gV_o = oracle.adjoint(g, V, R0, I0, n, 2 * (F0 - target))
    ga_o = oracle.atom_gradient(g, atoms, gV_o)
    assert np.abs(gV - gV_o).max() <= 1e-9 * np.abs(gV_o).max()
    assert np.abs(ga - ga_o).max() <= 1e-9 * np.abs(ga_o).max()


ADJ_CASES = {
    # (nx, ny, nz, bc, mask, det_k, atoms): ragged 32 x 8 tiles, several z-chunks, the
    # detector faces at a chunk boundary and at the top plane, a periodic z axis
    "walls": (8, 8, 24, (0, 0, 1), 4, 6),
    "chunks": (36, 20, 48, (0, 0, 1), 5, 15),
    "zper": (12, 10, 40, (1, 0, 0), 0, 38),
    "wallxy": (20, 12, 36, (1, 1, 1), 3, 16),
}


@pytest.mark.parametrize("precision", ["FP64", "FP32", "FP32_KAHAN"])
@pytest.mark.parametrize("name", list(ADJ_CASES))
def test_fused_adjoint_step_equals_three_passes(T, name, precision):
    """The fused backward step (one z-march over tiles, two buffer sets) and the
    three in-place passes share their per-cell arithmetic: dL/dV and the atom
    gradient agree bit for bit, and the FP64 form matches the oracle."""
    from paper_2401_07416_gb300.sim import Sim
    nx, ny, nz, bc, mask, kd = ADJ_CASES[name]
    g = W.small_grid(nx, ny, nz, h=(0.25, 0.22, 0.24), dt=0.004, bc=bc, det_k=kd, mask=mask, eta=0.5)
    L = g.lengths
    atoms = np.array([[0.3 * L[0], 0.4 * L[1], 0.5 * L[2], 6.0], [0.7 * L[0], 0.2 * L[1], 0.45 * L[2], 8.0]])
    p = W.Packet((0.5 * L[0], 0.5 * L[1], 0.6 * L[2]), (0.0, 0.0, 0.7), (0.0, 0.0, -2.5))
    prec = getattr(T, precision)
    n = 37
    rng = np.random.default_rng(7)
    out = {}
    for fused in (True, False):
        with Sim(g, precision=prec, ckpt_every=10) as s:
            s.set_atoms(0, atoms)
            s.set_packet(0, p)
            s.step(n)
            gF = rng.normal(size=(ny, nx)) if not out else out["gF"]
            gV = np.zeros((nz, ny, nx))
            ga = np.zeros_like(atoms)
            T.tdse_set_adjoint_fused(s.ctx, fused)
            T.tdse_adjoint(s.ctx, 0, gF, gV, ga)
        out.setdefault("gF", gF)
        out[fused] = (gV, ga)
    assert np.array_equal(out[True][0], out[False][0]), name
    assert np.array_equal(out[True][1], out[False][1]), name
    assert np.abs(out[True][0]).max() > 0
    if prec == T.FP64:
        V = oracle.potential_atoms(g, atoms)
        R0, I0 = oracle.wavepacket(g, p.r0, p.sigma, p.k0)
        gV_o = oracle.adjoint(g, V, R0, I0, n, out["gF"])
        assert np.abs(out[True][0] - gV_o).max() <= 1e-9 * np.abs(gV_o).max()


@pytest.mark.parametrize("precision", ["FP32", "FP32_KAHAN"])
def test_fp32_adjoint_close_to_fp64(T, precision):
    g, atoms, p = small_case()
    n = 160
    F0, gV64, ga64 = gpu_gradients(T, g, atoms, p, n, 0.0, T.FP64)
    target = 0.5 * F0 + 0.01
    _, gV64, ga64 = gpu_gradients(T, g, atoms, p, n, target, T.FP64)
    _, gV32, ga32 = gpu_gradients(T, g, atoms, p, n, target, getattr(T, precision))
    assert np.linalg.norm(gV32 - gV64) <= 2e-3 * np.linalg.norm(gV64)
    assert np.linalg.norm(ga32 - ga64) <= 2e-3 * np.linalg.norm(ga64)


FD_EPS = 1e-4      # central differences (forward runs in FP64)
FD_REL = 1e-6      # relative agreement asked of every derivative
FD_FLOOR = 1e-3    # ... measured against max(|fd|, FD_FLOOR * the largest |fd| of its kind)


def fd_agrees(ad, fd, kinds):
    """Per-component check: |ad - fd| <= FD_REL * max(|fd|, FD_FLOOR * max |fd| of the
    same kind).  Returns the worst ratio of error to allowance."""
    ad, fd = np.asarray(ad, dtype=float), np.asarray(fd, dtype=float)
    worst = 0.0
    for k in set(kinds):
        sel = np.array([kk == k for kk in kinds])
        ref = np.maximum(np.abs(fd[sel]), FD_FLOOR * np.abs(fd[sel]).max())
        worst = max(worst, float((np.abs(ad[sel] - fd[sel]) / (FD_REL * ref)).max()))
    return worst


def test_config4_atom_gradient_vs_finite_differences_all_128(T):
    """96x96x192, 3000 FP64 steps, checkpoints every 100: the adjoint gradient of
    the detector-flux loss w.r.t. every position and charge of the 32 atoms
    (through the torch.autograd wrapper) against central finite differences of
    the GPU forward, component by component."""
    import torch
    from paper_2401_07416_gb300.sim import Sim, diffraction_loss, flux_from_atoms
    wl = W.config4(W.FP64)
    g, atoms, p, n = wl.grid, wl.atoms, wl.packet, wl.steps
    assert atoms.shape == (32, 4)
    with Sim(g, precision=T.FP64, ckpt_every=100) as s:
        s.set_atoms(0, W.config4_target_atoms(atoms))
        s.set_packet(0, p)
        s.step(n)
        target = s.flux_map(0)

        def loss(a):
            s.set_atoms(0, a)
            s.set_packet(0, p)
            s.step(n)
            return float(np.sum((s.flux_map(0) - target) ** 2))

        a_t = torch.tensor(atoms, requires_grad=True)
        L = diffraction_loss(flux_from_atoms(a_t, s, 0, p, n), torch.from_numpy(target))
        L.backward()
        grad = a_t.grad.numpy()
        fd = np.zeros_like(atoms)
        for a in range(atoms.shape[0]):
            for k in range(4):
                ap, am = atoms.copy(), atoms.copy()
                ap[a, k] += FD_EPS
                am[a, k] -= FD_EPS
                fd[a, k] = (loss(ap) - loss(am)) / (2 * FD_EPS)
    kinds = ["position"] * 3 + ["charge"]
    worst = fd_agrees(grad.ravel(), fd.ravel(), [kinds[i % 4] for i in range(fd.size)])
    print(f"config4 atom gradient vs FD (128 parameters): worst error / allowance {worst:.3f}")
    assert worst <= 1.0


def test_config4_potential_gradient_vs_finite_differences(T):
    """Same case, dL/dV from the torch.autograd wrapper of the gridded potential
    (flux_from_potential) against central finite differences along 16 seeded
    directions: 12 spanning the whole grid, 2 confined to a box around the slab and
    2 to the absorbing layers at the z ends."""
    import torch
    from paper_2401_07416_gb300.sim import Sim, diffraction_loss, flux_from_potential
    wl = W.config4(W.FP64)
    g, atoms, p, n = wl.grid, wl.atoms, wl.packet, wl.steps
    rng = np.random.default_rng(4016)
    shape = (g.nz, g.ny, g.nx)
    z_slab = int(round(atoms[:, 2].mean() / g.hz))
    dirs, kinds = [], []
    for i in range(16):
        u = rng.normal(size=shape)
        if 12 <= i < 14:
            box = np.zeros(shape)
            box[z_slab - 16:z_slab + 16, 20:52, 30:62] = 1.0
            u *= box
            kinds.append("slab")
        elif i >= 14:
            lay = np.zeros(shape)
            lay[:g.mask_lo] = 1.0
            lay[g.nz - g.mask_hi:] = 1.0
            u *= lay
            kinds.append("layer")
        else:
            kinds.append("grid")
        dirs.append(u)
    with Sim(g, precision=T.FP64, ckpt_every=100) as s:
        s.set_atoms(0, W.config4_target_atoms(atoms))
        s.set_packet(0, p)
        s.step(n)
        target = s.flux_map(0)
        s.set_atoms(0, atoms)
        V0 = s.potential(0)

        def loss(V):
            s.set_potential(0, V)
            s.set_packet(0, p)
            s.step(n)
            return float(np.sum((s.flux_map(0) - target) ** 2))

        V_t = torch.tensor(V0, requires_grad=True)
        L = diffraction_loss(flux_from_potential(V_t, s, 0, p, n), torch.from_numpy(target))
        L.backward()
        gV = V_t.grad.numpy()
        ad = [float(np.sum(gV * u)) for u in dirs]
        fd = [(loss(V0 + FD_EPS * u) - loss(V0 - FD_EPS * u)) / (2 * FD_EPS) for u in dirs]
    # the layer directions see little of the packet: their scale is the grid's
    floor_kind = ["grid" if k == "layer" else k for k in kinds]
    worst = fd_agrees(ad, fd, floor_kind)
    print(f"config4 dL/dV vs FD along 16 directions: worst error / allowance {worst:.3f}")
    assert worst <= 1.0


def test_adjoint_rejects_a_zero_absorbing_factor(T):
    """A CAP layer so strong that exp(-W dt / hbar) underflows to 0 on its outer planes:
    the forward runs, the adjoint cannot divide the factor out and reports EINVAL."""
    import dataclasses
    from paper_2401_07416_gb300.sim import Sim
    g = W.small_grid(16, 12, 24, h=(0.2, 0.2, 0.2), dt=0.004, bc=(0, 0, 1), mask=4, det_k=10)
    g = dataclasses.replace(g, obs_every=5, mask_kind=W.MASK_CAP, mask_eta=1e6)
    with Sim(g, precision=T.FP64, ckpt_every=5) as s:
        s.set_potential(0, W.random_potential(g, 3, 1.0))
        s.set_packet(0, W.Packet((1.6, 1.2, 2.4), (0.6, 0.6, 0.6), (0.0, 0.0, 1.0)))
        s.step(10)
        with pytest.raises(T.TdseError) as e:
            T.tdse_adjoint(s.ctx, 0, np.ones((g.ny, g.nx)), None, None)
        assert e.value.status == T.EINVAL
