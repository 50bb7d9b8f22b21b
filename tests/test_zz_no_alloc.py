"""The allocation-free observables entry point.

tdse_observables_static computes Q, the paper norm and the energy of a
device-resident state using a static device array as scratch, for callers that
cannot allocate device memory (for instance a host program whose device memory
belongs to another allocator).  Its results must match the FP64 oracle's
reduction of the same state and those of the context path, tdse_observables,
within the FP64 tolerance of the parity tests, on two calls in a row (the second
call reuses the scratch left by the first), and for two geometries of different
nz.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2401_07416_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-11


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_07416_gb300 import build
    build.build()
    from paper_2401_07416_gb300 import tdse
    return tdse


def context_observables(T, g, V, R, I):
    p = T.params_from_grid(g, T.FP64)
    ctx = T.tdse_create([p])
    try:
        T.tdse_set_potential(ctx, 0, V)
        T.tdse_set_state(ctx, 0, R, I)
        return T.tdse_observables(ctx, 0)
    finally:
        T.tdse_destroy(ctx)


@pytest.mark.parametrize("shape,bc", [((36, 28, 40), (0, 0, 1)), ((20, 17, 9), (1, 0, 0))])
def test_static_scratch_matches_context_path(T, shape, bc):
    import torch
    nx, ny, nz = shape
    g = W.small_grid(nx, ny, nz, h=(0.2, 0.23, 0.19), dt=0.003, bc=bc)
    R = W.random_field((nz, ny, nx), 41)
    I = W.random_field((nz, ny, nx), 42)
    V = W.random_potential(g, 43, 2.0)
    ref = context_observables(T, g, V, R, I)
    orc = oracle.observables(g, V, R, I)
    Rd, Id, Vd = (torch.from_numpy(a).cuda() for a in (R, I, V))
    p = T.params_from_grid(g, T.FP64)
    for _ in range(2):
        got = T.tdse_observables_static(p, Rd, Id, Vd,
                                        torch.cuda.current_stream().cuda_stream)
        for k in ("Q", "norm_paper", "energy"):
            assert got[k] == pytest.approx(orc[k], rel=TOL64), k
            assert got[k] == pytest.approx(ref[k], rel=TOL64), k


def test_static_scratch_rejects_short_arrays(T):
    """The binding refuses arrays that hold fewer values than the grid (the
    kernels would read past them) before anything reaches the library."""
    import torch
    g = W.small_grid(8, 6, 10, h=(0.2, 0.2, 0.2), dt=0.003)
    p = T.params_from_grid(g, T.FP64)
    full = torch.zeros(10 * 6 * 8, device="cuda", dtype=torch.float64)
    short = torch.zeros(10 * 6 * 8 - 1, device="cuda", dtype=torch.float64)
    for args in ((short, full, None), (full, short, None), (full, full, short)):
        with pytest.raises(ValueError):
            T.tdse_observables_static(p, *args)


def test_static_scratch_rejects_too_many_planes(T):
    import torch
    g = W.small_grid(4, 1, 8193, h=(0.2, 0.2, 0.2), dt=0.003)
    p = T.params_from_grid(g, T.FP64)
    x = torch.zeros(4 * 1 * 8193, device="cuda", dtype=torch.float64)   # a full grid's worth
    with pytest.raises(T.TdseError) as e:
        T.tdse_observables_static(p, x, x, None)
    assert e.value.status == T.EINVAL
