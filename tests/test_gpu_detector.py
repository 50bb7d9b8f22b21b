"""Detector-plane density frames (Eq. 15) and the Eq. 16 dissimilarity on the GPU,
through the C ABI, against the FP64 oracle (oracle/detector.py).

Tolerances: frames FP64 max |gpu - oracle| / max |oracle| <= 1e-11, FP32+Kahan
relative L2 <= 2e-4 (the density is quadratic in psi, whose tolerance is 1e-4);
dissimilarity of given frames (FP64 arithmetic on both sides, different summation
order) relative 1e-12; dissimilarity of simulated trajectories 1e-9 (FP64 runs).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from oracle import detector as OD
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


def slab_case(seed, obs_every=5):
    g = W.small_grid(40, 36, 44, h=(0.21, 0.19, 0.23), dt=0.004, bc=(0, 0, 1), mask=5, det_k=12,
                     eta=0.5)
    g = dataclasses.replace(g, obs_every=obs_every)
    V = W.random_potential(g, 200 + seed, 2.0)
    L = g.lengths
    p = W.Packet((0.5 * L[0], 0.5 * L[1], 0.6 * L[2]), (0.9, 1.0, 0.8), (0.3, -0.2, -2.2))
    return g, V, p


def oracle_frames(g, V, p, nsteps, every):
    R, I = oracle.initial_state(g, p, V)
    frames = [OD.detector_frame(R, I, g.det_k)]
    for _ in range(nsteps // every):
        R, I, _, _ = oracle.run(g, V, R, I, every, use_mask=True, flux=False)
        frames.append(OD.detector_frame(R, I, g.det_k))
    return np.array(frames)


def gpu_frames(T, g, V, p, nsteps, precision, capacity=16):
    from paper_2401_07416_gb300.sim import Sim
    with Sim(g, precision=precision) as s:
        s.set_frames(capacity)
        s.set_potential(0, V)
        s.set_packet(0, p)
        s.step(nsteps)
        return s.frames(0)


@pytest.mark.parametrize("precision", ["FP64", "FP32_KAHAN"])
def test_frames_match_oracle(T, precision):
    g, V, p = slab_case(0)
    n = 30
    fo = oracle_frames(g, V, p, n, g.obs_every)
    fg, steps = gpu_frames(T, g, V, p, n, getattr(T, precision))
    assert list(steps) == list(range(0, n + 1, g.obs_every))
    assert fg.shape == fo.shape
    if precision == "FP64":
        assert np.abs(fg - fo).max() <= 1e-11 * np.abs(fo).max()
    else:
        for a, b in zip(fg, fo):
            assert np.linalg.norm(a - b) <= 2e-4 * np.linalg.norm(b)


def test_frame_capacity_and_reset(T):
    g, V, p = slab_case(1)
    from paper_2401_07416_gb300.sim import Sim
    with Sim(g, precision=T.FP64) as s:
        s.set_frames(3)
        s.set_potential(0, V)
        s.set_packet(0, p)
        s.step(40)                       # observation points 0, 5, ..., 40: only 3 kept
        f, steps = s.frames(0)
        assert list(steps) == [0, 5, 10]
        s.set_packet(0, p)               # a new run (at the context's step 40) starts a new recording
        f2, steps2 = s.frames(0)
        assert list(steps2) == [40] and np.array_equal(f2[0], f[0])
        s.set_frames(0)
        assert s.frames(0)[0].shape[0] == 0
    gw = W.small_grid(8, 8, 8)            # no detector plane
    with Sim(gw, precision=T.FP64) as s:
        with pytest.raises(T.TdseError) as e:
            s.set_frames(2)
        assert e.value.status == T.EINVAL


@pytest.mark.parametrize("on_device", [False, True])
def test_dissimilarity_matches_oracle(T, on_device):
    import torch
    rng = np.random.default_rng(21)
    K, M, P = 37, 9, 1000             # ragged against the 32 x 32 tiles and 32-pixel chunks
    frames = rng.uniform(0.0, 1.0, size=(K, M, P))
    frames[5] = frames[4]             # an identical pair
    t = np.cumsum(rng.uniform(0.05, 0.2, size=M))
    t0, t1, dA = t[1], t[7], 0.013
    do = OD.dissimilarity(frames, t, t0, t1, dA)
    if on_device:
        dg = T.tdse_dissimilarity(torch.from_numpy(frames).cuda(), t, t0, t1, dA).cpu().numpy()
    else:
        dg = T.tdse_dissimilarity(frames, t, t0, t1, dA)
    assert np.all(np.diag(dg) == 0.0) and np.array_equal(dg, dg.T)
    assert dg[4, 5] == 0.0
    assert np.abs(dg - do).max() <= 1e-12 * np.abs(do).max()


def test_dissimilarity_invalid_arguments(T):
    f = np.zeros((2, 3, 4))
    t = np.array([0.0, 1.0, 2.0])
    for args in [(f, t, 1.0, 1.0, 0.1), (f, t, 0.0, 1.0, 0.0), (f, t, 2.5, 3.0, 0.1)]:
        with pytest.raises(T.TdseError) as e:
            T.tdse_dissimilarity(*args)
        assert e.value.status == T.EINVAL


def test_batch_trajectories_dissimilarity(T):
    """Three films in one batch record their frames; their Eq. 16 matrix matches the
    oracle's for the same three trajectories."""
    cases = [slab_case(s, obs_every=4) for s in range(3)]
    n = 24
    from paper_2401_07416_gb300.sim import Sim
    with Sim([c[0] for c in cases], precision=T.FP64) as s:
        for i, (g, V, p) in enumerate(cases):
            s.set_frames(16, i)
            s.set_potential(i, V)
            s.set_packet(i, p)
        s.step(n)
        fg = np.array([s.frames(i)[0] for i in range(3)])
    fo = np.array([oracle_frames(g, V, p, n, 4) for g, V, p in cases])
    g = cases[0][0]
    t = np.arange(fg.shape[1]) * 4 * g.dt
    dA = g.hx * g.hy
    dg = T.tdse_dissimilarity(fg, t, t[1], t[-1], dA)
    do = OD.dissimilarity(fo, t, t[1], t[-1], dA)
    assert np.abs(dg - do).max() <= 1e-9 * np.abs(do).max()
    assert do[0, 1] > 0 and do[1, 2] > 0
