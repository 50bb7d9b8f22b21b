"""Failure paths of the step, made on the host with every device access valid.

- Allocation failure: an allocator callback that returns NULL on its k-th call
  gives TDSE_ENOMEM, and the context is still destroyed cleanly.
- Expired waits: tdse_set_wait_limit(ctx, 0) makes every wait of the step kernels
  for a tile's data test its data once, so waits for loads still in flight
  expire while every load stays valid.  The kernels then stop, wait for their
  own loads, release tensor memory and leave; tdse_step returns TDSE_ETIMEOUT and
  the context refuses further steps.  A fresh context on the same kernels then
  runs normally (nothing was left held on the device).
- Divergence: an unstable run ends tdse_step at the observation point that saw
  it (within two observation intervals), not after all requested steps.
"""
import ctypes

import numpy as np
import pytest

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
    g = W.small_grid(40, 36, 48, h=(0.2, 0.2, 0.2), dt=0.004, bc=(0, 0, 1), mask=6, det_k=20,
                     eta=0.3)
    p = W.Packet((4.0, 3.6, 5.0), (1.0, 1.0, 1.0), (0.0, 0.0, -1.5))
    return g, p


class CountingAllocator:
    """Device memory from torch's caching allocator; returns NULL on call `fail_at`
    (1-based; 0: never)."""

    def __init__(self, T, fail_at=0):
        import torch
        self.calls = 0
        self.live = set()
        self.fail_at = fail_at
        dev = torch.cuda.current_device()
        stream = torch.cuda.current_stream()

        def alloc(nbytes, user):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            self.live.add(ptr)
            return ptr

        def free(ptr, user):
            self.live.discard(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.cbs = (T.ALLOC_FN(alloc), T.FREE_FN(free))


def run_with_allocator(T, prec, tblock, alloc):
    g, p = small_case()
    ctx = T.tdse_create([T.params_from_grid(g, prec, tblock)])
    try:
        T.tdse_set_allocator(ctx, *alloc.cbs)
        T.tdse_set_wavepacket(ctx, 0, p.r0, p.sigma, p.k0)
        T.tdse_step(ctx, 4)
        return T.OK
    except T.TdseError as e:
        return e.status
    finally:
        T.tdse_destroy(ctx)


@pytest.mark.parametrize("prec,tblock", [("FP64", 1), ("FP32_KAHAN", 2)])
def test_allocator_null_gives_enomem(T, prec, tblock):
    prec = getattr(T, prec)
    full = CountingAllocator(T)
    assert run_with_allocator(T, prec, tblock, full) == T.OK
    n = full.calls
    assert n > 10 and not full.live        # every allocation was freed by tdse_destroy
    # the first, a middle and the last allocation of the run fail in turn
    for k in sorted({1, 2, n // 3, n // 2, n - 1, n}):
        a = CountingAllocator(T, fail_at=k)
        assert run_with_allocator(T, prec, tblock, a) == T.ENOMEM, k
        assert not a.live, k               # destroyed cleanly after the failure
    # the device is still fine afterwards
    assert run_with_allocator(T, prec, tblock, CountingAllocator(T)) == T.OK


def variant_index(T, prec, tblock, name):
    for v in range(T.tdse_variant_count(prec, tblock)):
        g, _ = small_case()
        ctx = T.tdse_create([T.params_from_grid(g, prec, tblock)])
        try:
            T.tdse_set_variant(ctx, tblock, v)
            if T.tdse_get_tuning(ctx)["name"][tblock] == name:
                return v
        finally:
            T.tdse_destroy(ctx)
    raise LookupError(name)


@pytest.mark.parametrize("prec,tblock,variant", [
    ("FP64", 1, None), ("FP32", 1, None), ("FP32", 2, None), ("FP32_KAHAN", 2, None),
    # split plane barrier: every warp waits for its loads and for the other warps itself
    ("FP32", 2, "f32_t2_split_w32_r32x1_pf2_b2"), ("FP32_KAHAN", 2, "k32_t2_split_w32_r32x1_pf2_b2"),
    ("FP32_KAHAN", 2, "k32_t2_split_r32x1_pf3")])
def test_expired_wait_gives_etimeout_and_fails_the_context(T, prec, tblock, variant):
    from paper_2401_07416_gb300.sim import Sim
    prec = getattr(T, prec)
    v = None if variant is None else variant_index(T, prec, tblock, variant)
    g, p = small_case()
    s = Sim(g, precision=prec, tblock=tblock)
    if v is not None:
        T.tdse_set_variant(s.ctx, tblock, v)
    s.set_packet(0, p)
    s.step(tblock)                        # a normal launch first
    T.tdse_set_wait_limit(s.ctx, 0)
    with pytest.raises(T.TdseError) as e:
        s.step(40)
    assert e.value.status == T.ETIMEOUT, str(e.value)
    with pytest.raises(T.TdseError) as e2:
        s.step(2)
    assert e2.value.status == T.ESTATE
    s.state(0)                            # reading the (meaningless) state still works
    s.close()
    # the same kernels run normally in a new context: no wait, tensor memory or load
    # was left behind, and the result equals a run that never saw a timeout
    ref = None
    for _ in range(2):
        with Sim(g, precision=prec, tblock=tblock) as s2:
            if v is not None:
                T.tdse_set_variant(s2.ctx, tblock, v)
            s2.set_packet(0, p)
            s2.step(20)
            got = s2.state(0)
        if ref is not None:
            assert all(np.array_equal(a, b) for a, b in zip(got, ref))
        ref = got


def test_wait_limit_rejects_negative(T):
    g, _ = small_case()
    ctx = T.tdse_create([T.params_from_grid(g, T.FP64, 1)])
    try:
        with pytest.raises(T.TdseError) as e:
            T.tdse_set_wait_limit(ctx, -1)
        assert e.value.status == T.EINVAL
    finally:
        T.tdse_destroy(ctx)


def test_divergence_ends_the_call_at_the_failing_observation(T):
    """dt |V| = 12, far beyond the leapfrog's bound of 2: the state grows without
    bound.  A request of a million steps ends at most two observation intervals
    after the first observation point that fails the reduction's check (Q or E not
    finite, or Q above (1 + 1e-3) Q0 when Q0 > 0; here Q0 < 0, so the run is caught
    when it overflows), the point the message names, not after all requested steps."""
    import re
    from paper_2401_07416_gb300.sim import Sim
    g = W.small_grid(16, 16, 16, h=(0.2, 0.2, 0.2), dt=0.004, bc=(1, 1, 1))
    with Sim(g, precision=T.FP64) as s:
        s.set_potential(0, np.full((16, 16, 16), 3000.0))
        s.set_packet(0, W.Packet((1.5, 1.5, 1.5), (0.5, 0.5, 0.5), (0, 0, 1)))
        with pytest.raises(T.TdseError) as e:
            s.step(10 ** 6)
        assert e.value.status == T.EUNSTABLE
        named = int(re.search(r"observation of step (\d+)", str(e.value)).group(1))
        hist = s.history(0)                      # rows (step, Q, paper norm, energy)
        q0 = hist[0, 1]
        bad = [int(r[0]) for r in hist
               if not (np.isfinite(r[1]) and np.isfinite(r[3])) or (q0 > 0 and r[1] > (1 + 1e-3) * q0)]
        assert bad and bad[0] == named, (bad[:3], named)
        end = s.observables(0)["step"]
        assert named <= end <= named + 2 * g.obs_every, (named, end)
        with pytest.raises(T.TdseError) as e2:
            s.step(1)
        assert e2.value.status == T.ESTATE
