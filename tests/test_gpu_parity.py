"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written here, used by every case):
  FP64 GPU:        max |gpu - oracle| / max |oracle| <= 1e-11 for R, I, the flux map
                   and the observables;
  FP32 / Kahan:    ||psi_gpu - psi_oracle||_2 / ||psi_oracle||_2 <= 1e-4 and
                   |Q_gpu - Q_oracle| / Q_oracle <= 1e-5;
  fused vs unfused and batched vs solo: bitwise equal (same arithmetic, same order).
Small grids span several tiles with ragged tails in x, y and z (default tiles are
56 x 20 in FP32 T=1, 24 x 24 in FP32 and Kahan T=2, 60 x 12 in FP64;
z-chunks are chosen per launch), and the degenerate cases: the smallest legal grid
(4 x 1 x 3, walls) and a grid whose periodic z axis (3 planes) is shorter than the
z halo of a two-step launch.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2401_07416_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32_L2 = 1e-4
TOL32_Q = 1e-5


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_07416_gb300 import build
    build.build()
    from paper_2401_07416_gb300 import tdse
    return tdse


def make_sim(grids, precision, tblock=0, ckpt_every=0):
    from paper_2401_07416_gb300.sim import Sim
    return Sim(grids, precision=precision, tblock=tblock, ckpt_every=ckpt_every)


def maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def l2rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2)) / np.sqrt(np.sum(b ** 2)))


CASES = {
    # name: (nx, ny, nz, bc, mask, det_k)
    "walls": (20, 37, 41, (1, 1, 1), 5, 12),
    "slab": (132, 44, 50, (0, 0, 1), 6, 20),
    "periodic": (24, 24, 30, (0, 0, 0), 0, 5),
    "mixed": (36, 28, 33, (0, 1, 0), 4, 9),
    # periodic axes shorter than twice the ghost width: both ghost zones are copies
    "short": (12, 9, 26, (0, 0, 1), 3, 8),
    # the smallest legal grid (nx >= 4, ny >= 1, nz >= 3), walls everywhere
    "minimal": (4, 1, 3, (1, 1, 1), 0, -1),
    # periodic everywhere at the shortest periodic lengths, 3 z planes (the z halo
    # of a two-step launch wraps around the axis more than once)
    "thin": (8, 8, 3, (0, 0, 0), 0, 0),
}


def case(name, seed=0):
    nx, ny, nz, bc, mask, det = CASES[name]
    g = W.small_grid(nx, ny, nz, h=(0.21, 0.19, 0.23), dt=0.004, bc=bc, mask=mask, det_k=det,
                     eta=0.5)
    V = W.random_potential(g, 100 + seed, 2.0)
    L = g.lengths
    p = W.Packet((0.5 * L[0], 0.45 * L[1], 0.55 * L[2]), (0.9, 1.1, 0.8), (0.4, -0.3, -1.8))
    return g, V, p


def oracle_run(g, V, p, nsteps):
    R0, I0 = oracle.initial_state(g, p, V)
    R, I, F, jl = oracle.run(g, V, R0, I0, nsteps, use_mask=True, flux=g.det_k >= 0)
    return (R0, I0), (R, I, F, jl), oracle.observables(g, V, R, I)


def gpu_run(g, V, p, nsteps, precision, tblock=0):
    s = make_sim(g, precision, tblock)
    s.set_potential(0, V)
    s.set_packet(0, p)
    init = s.state(0)
    s.step(nsteps)
    R, I = s.state(0)
    F = s.flux_map(0)
    obs = s.observables(0)
    s.close()
    return init, (R, I, F), obs


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_matches_oracle(T, name):
    g, V, p = case(name)
    n = 23
    (R0, I0), (Ro, Io, Fo, _), oo = oracle_run(g, V, p, n)
    (Rg0, Ig0), (Rg, Ig, Fg), og = gpu_run(g, V, p, n, T.FP64)
    assert maxrel(Rg0, R0) < 1e-13 and maxrel(Ig0, I0) < 1e-13
    scale = max(np.abs(Ro).max(), np.abs(Io).max())
    assert np.abs(Rg - Ro).max() / scale < TOL64
    assert np.abs(Ig - Io).max() / scale < TOL64
    if g.det_k >= 0:
        assert maxrel(Fg, Fo) < TOL64
    assert og["Q"] == pytest.approx(oo["Q"], rel=TOL64)
    assert og["energy"] == pytest.approx(oo["energy"], rel=TOL64)
    assert og["norm_paper"] == pytest.approx(oo["norm_paper"], rel=TOL64)


@pytest.mark.parametrize("precision", ["FP32", "FP32_KAHAN"])
@pytest.mark.parametrize("tblock", [1, 2, 3, 4])
@pytest.mark.parametrize("name", list(CASES))
def test_fp32_matches_oracle(T, name, precision, tblock):
    g, V, p = case(name, seed=1)
    n = 23
    (R0, I0), (Ro, Io, Fo, _), oo = oracle_run(g, V, p, n)
    (Rg0, Ig0), (Rg, Ig, Fg), og = gpu_run(g, V, p, n, getattr(T, precision), tblock)
    # the packet start is computed in FP64; Kahan keeps value + compensation (~48
    # bits), plain FP32 rounds each value once (2^-24 relative)
    tol0 = 1e-13 if precision == "FP32_KAHAN" else 1e-7
    assert maxrel(Rg0, R0) < tol0 and maxrel(Ig0, I0) < tol0
    psi_err = math.sqrt(np.sum((Rg - Ro) ** 2 + (Ig - Io) ** 2) / np.sum(Ro ** 2 + Io ** 2))
    assert psi_err < TOL32_L2
    assert abs(og["Q"] - oo["Q"]) / oo["Q"] < TOL32_Q
    if g.det_k >= 0 and np.abs(Fo).max() > 0:
        assert l2rel(Fg, Fo) < 1e-3


@pytest.mark.parametrize("precision", ["FP32", "FP32_KAHAN"])
@pytest.mark.parametrize("tblock", [2, 3, 4])
@pytest.mark.parametrize("name", ["slab", "mixed"])
def test_fused_steps_bitwise_equal_to_one_step_launches(T, name, precision, tblock):
    g, V, p = case(name, seed=2)
    a = gpu_run(g, V, p, 18, getattr(T, precision), tblock=tblock)
    b = gpu_run(g, V, p, 18, getattr(T, precision), tblock=1)
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["FP64", "FP32_KAHAN"])
def test_zero_steps_leave_the_state(T, precision):
    g, V, p = case("slab")
    s = make_sim(g, getattr(T, precision))
    s.set_potential(0, V)
    s.set_packet(0, p)
    R0, I0 = s.state(0)
    q0 = s.observables(0)
    s.step(0)
    R1, I1 = s.state(0)
    q1 = s.observables(0)
    s.close()
    assert np.array_equal(R0, R1) and np.array_equal(I0, I1)
    assert q1["step"] == q0["step"] and q1["Q"] == q0["Q"]


def test_potential_from_atoms_matches_oracle(T):
    g = W.small_grid(40, 36, 30, h=(0.2, 0.22, 0.25), bc=(0, 0, 1))
    rng = np.random.default_rng(5)
    atoms = np.column_stack([rng.uniform(0, 8, 12), rng.uniform(0, 7.9, 12),
                             rng.uniform(1, 6, 12), rng.choice([1.0, 6.0, 8.0], 12)])
    s = make_sim(g, T.FP64)
    s.set_atoms(0, atoms)
    Vg = s.potential(0)
    s.close()
    Vo = oracle.potential_atoms(g, atoms)
    assert maxrel(Vg, Vo) < 1e-14


def test_set_state_roundtrip_and_kahan_exactness(T):
    g, V, p = case("slab")
    R = W.random_field((g.nz, g.ny, g.nx), 7)
    I = W.random_field((g.nz, g.ny, g.nx), 8)
    for prec in (T.FP64, T.FP32_KAHAN):
        s = make_sim(g, prec)
        s.set_potential(0, V)
        s.set_state(0, R, I)
        Rg, Ig = s.state(0)
        s.close()
        # FP64 exact; Kahan stores value + compensation, recovering ~48 bits
        tol = 0.0 if prec == T.FP64 else 1e-13
        assert np.abs(Rg - R).max() <= tol * np.abs(R).max()
        assert np.abs(Ig - I).max() <= tol * np.abs(I).max()


def test_batched_members_equal_solo_runs(T):
    names = ["walls", "slab", "mixed"]
    cs = [case(n, seed=3) for n in names]
    # the same precision and depth for the batch and the solo runs; walls/mixed
    # differ in shape so the work list interleaves uneven members
    for prec in (T.FP32_KAHAN, T.FP64):
        s = make_sim([c[0] for c in cs], prec)
        for i, (g, V, p) in enumerate(cs):
            s.set_potential(i, V)
            s.set_packet(i, p)
        s.step(14)
        batch = [(s.state(i), s.flux_map(i)) for i in range(len(cs))]
        s.close()
        for i, (g, V, p) in enumerate(cs):
            _, (R, I, F), _ = gpu_run(g, V, p, 14, prec)
            assert np.array_equal(batch[i][0][0], R)
            assert np.array_equal(batch[i][0][1], I)
            assert np.array_equal(batch[i][1], F)


@pytest.mark.parametrize("precision", ["FP32_KAHAN", "FP32", "FP64"])
def test_batch_graph_replay_equals_direct_launches(T, precision):
    """Uneven members in one context: step sequences replayed from captured CUDA
    graphs (the default) give the same states, flux maps and observation records,
    bit for bit, as the same launches issued one by one."""
    prec = getattr(T, precision)
    cs = [case(n, seed=6) for n in ["walls", "slab", "mixed"]]
    out = []
    for graphs in (True, False):
        s = make_sim([c[0] for c in cs], prec)
        if not graphs:
            T.tdse_set_graphs(s.ctx, False)
        for i, (g, V, p) in enumerate(cs):
            s.set_potential(i, V)
            s.set_packet(i, p)
        s.step(45)   # segments of 20, 20 and 5 steps between observation points
        s.step(35)   # the 20-step segment again (a replay of its captured graph)
        out.append([(*s.state(i), s.flux_map(i), s.history(i)) for i in range(len(cs))])
        s.close()
    for i in range(len(cs)):
        for a, b in zip(out[0][i], out[1][i]):
            assert np.array_equal(a, b), i


@pytest.mark.parametrize("precision", ["FP32_KAHAN", "FP64"])
def test_batched_reductions_equal_solo_reductions(T, precision):
    """A context with several members reduces all of them in one launch: every
    member's recorded Q, paper norm and energy equal, bit for bit, those of the
    same member run alone (same blocks, same items, same order)."""
    prec = getattr(T, precision)
    cs = [case(n, seed=4) for n in ["walls", "slab", "mixed", "periodic"]]
    s = make_sim([c[0] for c in cs], prec)
    for i, (g, V, p) in enumerate(cs):
        s.set_potential(i, V)
        s.set_packet(i, p)
    s.step(45)
    hist = [s.history(i) for i in range(len(cs))]
    s.close()
    for i, (g, V, p) in enumerate(cs):
        solo = make_sim(g, prec)
        solo.set_potential(0, V)
        solo.set_packet(0, p)
        solo.step(45)
        h = solo.history(0)
        solo.close()
        assert h.shape == hist[i].shape == (3, 4)
        assert np.array_equal(h, hist[i]), i


def test_config1_free_packet_full_size(T):
    """64^3 FP64, 500 steps: GPU = oracle to 1e-11, and the oracle-pinned closed-form
    drift of the centroid holds for the GPU result too."""
    wl = W.config1()
    g = wl.grid
    (R0, I0), (Ro, Io, _, _), oo = oracle_run(g, None, wl.packet, wl.steps)
    s = make_sim(g, T.FP64)
    s.set_packet(0, wl.packet)
    s.step(wl.steps)
    Rg, Ig = s.state(0)
    og = s.observables(0)
    hist = s.history(0)
    s.close()
    scale = np.abs(Ro).max()
    assert np.abs(Rg - Ro).max() / scale < TOL64
    assert np.abs(Ig - Io).max() / scale < TOL64
    assert og["Q"] == pytest.approx(oo["Q"], rel=TOL64)
    # Q conserved along the run (no absorbing layer), every 20 steps
    assert hist.shape[0] == wl.steps // g.obs_every + 1
    assert np.abs(hist[:, 1] / hist[0, 1] - 1).max() < 1e-12


def test_observation_history_and_eq11_default_dt(T):
    g = W.small_grid(16, 16, 16, h=(0.2, 0.2, 0.2), dt=0.0, bc=(1, 1, 1))
    s = make_sim(g, T.FP64)
    s.set_packet(0, W.Packet((1.5, 1.5, 1.5), (0.5, 0.5, 0.5), (0, 0, 1)))
    s.step(45)
    h = s.history(0)
    o = s.observables(0)
    s.close()
    assert list(h[:, 0]) == [0, 20, 40]
    assert o["step"] == 45
    assert o["t"] == pytest.approx(45 * 0.2 ** 2 / 5)


def test_unstable_run_reports_status(T):
    """A potential that makes the scheme unstable (dt |V| far above 2) grows the
    invariant; tdse_step must report TDSE_EUNSTABLE instead of returning garbage."""
    g = W.small_grid(16, 16, 16, h=(0.2, 0.2, 0.2), dt=0.004, bc=(1, 1, 1))
    V = np.full((16, 16, 16), 3000.0)   # dt * V = 12 >> 2
    s = make_sim(g, T.FP64)
    s.set_potential(0, V)
    s.set_packet(0, W.Packet((1.5, 1.5, 1.5), (0.5, 0.5, 0.5), (0, 0, 1)))
    with pytest.raises(T.TdseError) as e:
        s.step(200)
    s.close()
    assert e.value.status == T.EUNSTABLE


@pytest.mark.parametrize("precision", ["FP32", "FP32_KAHAN"])
@pytest.mark.parametrize("name", ["walls", "mixed", "short", "minimal", "thin"])
def test_every_fused_variant_bitwise_equal(T, name, precision):
    """Register-window and tensor-memory-window kernels, with a CTA barrier per
    plane or a producer warp and neighbour barriers, every tile shape and fused
    depth: the same arithmetic in the same order, so states and flux maps agree bit
    for bit with one-step launches."""
    g, V, p = case(name, seed=5)
    prec = getattr(T, precision)
    ref = None
    runs = [(1, 0)] + [(tb, v) for tb in (2, 3, 4) for v in range(T.tdse_variant_count(prec, tb))]
    for tb, v in runs:
        s = make_sim(g, prec, tb)
        T.tdse_set_variant(s.ctx, tb, v)
        s.set_potential(0, V)
        s.set_packet(0, p)
        s.step(14)
        got = (*s.state(0), s.flux_map(0))
        s.close()
        if ref is None:
            ref = got
            continue
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), (name, precision, tb, v)


@pytest.mark.parametrize("precision", ["FP64", "FP32_KAHAN"])
def test_potential_from_pinned_pageable_and_device_buffers(T, precision):
    """tdse_set_potential takes V from pageable host memory (copied first), from
    page-locked host memory (read directly by the d kernel; also at an offset of one
    element, so not 16-byte aligned) and from the device: the resident V and the
    states after 10 steps are the same bits."""
    import torch
    g, V, p = case("mixed", seed=7)
    prec = getattr(T, precision)
    n = V.size
    big = torch.empty(n + 1, dtype=torch.float64, pin_memory=True)
    big[1:] = torch.from_numpy(V.ravel())
    pinned = torch.empty(V.shape, dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.from_numpy(V))
    sources = {"pageable": V, "pinned": pinned, "pinned+8B": big[1:].view(V.shape),
               "device": torch.from_numpy(V).cuda()}
    ref = None
    for name, src in sources.items():
        s = make_sim(g, prec, 0)
        T.tdse_set_potential(s.ctx, 0, src)
        back = np.zeros(V.shape)
        T.tdse_get_potential(s.ctx, 0, back)
        assert np.array_equal(back, V), name
        s.set_packet(0, p)
        s.step(10)
        got = (*s.state(0), s.flux_map(0))
        s.close()
        if ref is None:
            ref = got
            continue
        for a_, b_ in zip(got, ref):
            assert np.array_equal(a_, b_), name


@pytest.mark.parametrize("precision", ["FP32", "FP32_KAHAN"])
def test_z_chunk_lengths_bitwise_equal(T, precision):
    """Any z-chunk length (short, ragged against nz, longer than the column) hands
    each output node to exactly one work item that computes it the same way: states
    and flux maps equal bit for bit."""
    g = W.small_grid(76, 100, 40, h=(0.21, 0.19, 0.23), dt=0.004, bc=(0, 1, 1), mask=4,
                     det_k=11, eta=0.5)                 # several tiles along x and y
    V = W.random_potential(g, 106, 2.0)
    L = g.lengths
    p = W.Packet((0.5 * L[0], 0.45 * L[1], 0.55 * L[2]), (0.9, 1.1, 0.8), (0.4, -0.3, -1.8))
    prec = getattr(T, precision)
    ref = None
    for chunk in (0, 9, 13, 17, 50, 1000):
        s = make_sim(g, prec, 2)
        T.tdse_set_chunk(s.ctx, 2, chunk)
        s.set_potential(0, V)
        s.set_packet(0, p)
        s.step(14)
        got = (*s.state(0), s.flux_map(0))
        s.close()
        if ref is None:
            ref = got
            continue
        for a_, b_ in zip(got, ref):
            assert np.array_equal(a_, b_), (precision, chunk)


@pytest.mark.parametrize("precision", ["FP64", "FP32_KAHAN"])
def test_eq10_absorbing_layer_matches_oracle(T, precision):
    """The paper's set-up of Eq. 10: one quadratic absorbing layer at the bottom of a
    z-periodic domain (MASK_CAP, operator split), fused kernel vs oracle."""
    import dataclasses
    g = W.small_grid(24, 20, 64, h=(0.21, 0.19, 0.23), dt=0.004, bc=(0, 0, 0), det_k=30)
    g = dataclasses.replace(g, mask_lo=22, mask_hi=0, mask_kind=W.MASK_CAP, mask_eta=15.0)
    V = W.random_potential(g, 300, 2.0)
    L = g.lengths
    p = W.Packet((0.5 * L[0], 0.5 * L[1], 0.40 * L[2]), (1.0, 1.0, 0.9), (0.2, 0.1, -2.5))
    n = 41
    _, (Ro, Io, Fo, _), oo = oracle_run(g, V, p, n)
    _, (Rg, Ig, Fg), og = gpu_run(g, V, p, n, getattr(T, precision))
    if precision == "FP64":
        scale = max(np.abs(Ro).max(), np.abs(Io).max())
        assert max(np.abs(Rg - Ro).max(), np.abs(Ig - Io).max()) / scale < TOL64
        assert maxrel(Fg, Fo) < TOL64
        assert og["Q"] == pytest.approx(oo["Q"], rel=TOL64)
    else:
        assert l2rel(np.concatenate([Rg, Ig]), np.concatenate([Ro, Io])) < TOL32_L2
        assert abs(og["Q"] - oo["Q"]) / oo["Q"] < TOL32_Q
    assert oo["Q"] < 0.999   # the layer absorbed part of the packet


@pytest.mark.parametrize("on_device", [False, True])
def test_potential_interpolated_from_a_periodic_cell(T, on_device):
    """Sec. 2.3's expansion + interpolation of a cell potential, on the GPU, against
    the oracle's trilinear interpolation (FP64, lattice incommensurate with the grid,
    origin off the grid, ragged sizes)."""
    import torch
    from oracle import interp as OI
    g = W.small_grid(36, 22, 31, h=(0.21, 0.19, 0.23), bc=(0, 0, 1))
    rng = np.random.default_rng(14)
    Vc = rng.normal(scale=3.0, size=(29, 11, 13))
    cell, origin = (2.73, 1.91, 6.05), (0.37, -0.52, 0.8)
    Vo = OI.trilinear_periodic(Vc, cell, origin, (g.nz, g.ny, g.nx), (g.hx, g.hy, g.hz))
    s = make_sim(g, T.FP64)
    src = torch.from_numpy(Vc).cuda() if on_device else Vc
    s.set_potential_grid(0, src, cell, origin)
    Vg = s.potential(0)
    s.close()
    assert np.abs(Vg - Vo).max() <= 1e-14 * np.abs(Vo).max()
    with pytest.raises(T.TdseError) as e:
        s2 = make_sim(g, T.FP64)
        try:
            s2.set_potential_grid(0, Vc, (2.73, 0.0, 6.05), origin)
        finally:
            s2.close()
    assert e.value.status == T.EINVAL


@pytest.mark.parametrize("precision", ["FP64", "FP32_KAHAN"])
def test_paper_cu111_geometry_window(T, precision):
    """The paper's Cu(111) run set-up (anisotropic 35.4 x 35.4 x 70 A mesh spacing,
    100 appended Eq. 10 absorbing planes on a z-periodic domain, Eq. 11 time step,
    Eq. 4 packet at 60 eV) on a 32 x 32 window in x, y, against the oracle."""
    import dataclasses
    wl = W.cu111(nx=32, ny=32)
    g = wl.grid                                   # dt = 0: the library applies Eq. 11
    go = dataclasses.replace(g, dt=oracle.default_dt(g.hx, g.hy, g.hz))   # the oracle, explicitly
    V = oracle.potential_atoms(go, wl.atoms)
    R0, I0 = oracle.initial_state(go, wl.packet, V)
    n = 30
    Ro, Io, Fo, _ = oracle.run(go, V, R0, I0, n)
    oo = oracle.observables(go, V, Ro, Io)
    from paper_2401_07416_gb300.sim import Sim
    with Sim(g, precision=getattr(T, precision)) as s:
        s.set_atoms(0, wl.atoms)
        s.set_packet(0, wl.packet)
        s.step(n)
        Rg, Ig = s.state(0)
        og = s.observables(0)
        assert og["t"] == pytest.approx(n * go.dt, rel=1e-15)
    if precision == "FP64":
        scale = max(np.abs(Ro).max(), np.abs(Io).max())
        assert max(np.abs(Rg - Ro).max(), np.abs(Ig - Io).max()) / scale < TOL64
        assert og["Q"] == pytest.approx(oo["Q"], rel=TOL64)
    else:
        assert l2rel(np.concatenate([Rg, Ig]), np.concatenate([Ro, Io])) < TOL32_L2
        assert abs(og["Q"] - oo["Q"]) / oo["Q"] < TOL32_Q
