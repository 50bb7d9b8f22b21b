"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every function declared in include/tdse.h; the ctypes structures match
the C layout; parameter validation and call-order errors come back as status
codes; with no GPU the library fails loudly instead of falling back to the CPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2401_07416_gb300 import build as B
from paper_2401_07416_gb300 import tdse as T
from paper_2401_07416_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tdse.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return T.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"TDSE_API\s+[\w\s\*]+?\b(tdse_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", T.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(tdse_\w+)", out))
    assert set(names) <= exported, set(names) - exported
    for n in names:
        assert hasattr(lib, n)
    assert set(names) == set(T.SIGNATURES)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stdio.h>
#include <stddef.h>
#include "tdse.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %d\n", sizeof(tdse_params),
         offsetof(tdse_params, hx), offsetof(tdse_params, bc), offsetof(tdse_params, mask_eta),
         offsetof(tdse_params, det_k), offsetof(tdse_params, tblock), sizeof(tdse_obs),
         sizeof(tdse_profile), offsetof(tdse_profile, launches_at_depth),
         offsetof(tdse_profile, ms_at_depth), sizeof(tdse_tuning), offsetof(tdse_tuning, ms_per_step),
         offsetof(tdse_tuning, name), TDSE_MAX_TBLOCK);
  printf("%zu %zu\n", offsetof(tdse_profile, adjoint_ms), offsetof(tdse_tuning, chunk));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    P, Pr, Tu = T.Params, T.Profile, T.Tuning
    assert vals == [ctypes.sizeof(P), P.hx.offset, P.bc.offset, P.mask_eta.offset,
                    P.det_k.offset, P.tblock.offset, ctypes.sizeof(T.Obs), ctypes.sizeof(Pr),
                    Pr.launches_at_depth.offset, Pr.ms_at_depth.offset, ctypes.sizeof(Tu),
                    Tu.ms_per_step.offset, Tu.name.offset, T.MAX_TBLOCK, Pr.adjoint_ms.offset,
                    Tu.chunk.offset]


def _params(**kw):
    g = W.small_grid(16, 12, 20, bc=(0, 0, 1))
    p = T.params_from_grid(g, precision=kw.pop("precision", T.FP32))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("field,value", [
    ("nx", 18),            # not a multiple of 4
    ("nz", 2),
    ("hx", 0.0),
    ("dt", 10.0),          # far above the leapfrog stability bound
    ("det_k", 19),         # needs det_k <= nz-2
    ("mask_lo", 30),
    ("precision", 7),
    ("tblock", 5),
    ("mask_kind", 2),      # neither cos^2 nor the Eq. 10 absorbing potential
    ("ny", 1 << 25),       # xy plane above 2^30 nodes (32-bit per-plane indices)
])
def test_create_rejects_bad_parameters(lib, field, value):
    with pytest.raises(T.TdseError) as e:
        T.tdse_create([_params(**{field: value})])
    assert e.value.status == T.EINVAL


def test_create_rejects_mixed_precision_batch(lib):
    with pytest.raises(T.TdseError):
        T.tdse_create([_params(), _params(precision=T.FP64)])


def test_default_dt_is_eq11(lib):
    p = _params(dt=0.0)
    ctx = T.tdse_create([p])
    T.tdse_destroy(ctx)   # accepted: dt <= 0 selects m min(h)^2 / (5 hbar)


def test_call_order_and_no_gpu_errors(lib):
    ctx = T.tdse_create([_params()])
    try:
        with pytest.raises(T.TdseError) as e:
            T.tdse_step(ctx, 1)
        assert e.value.status == T.ESTATE
        with pytest.raises(T.TdseError) as e:
            T.tdse_observables(ctx, 3)
        assert e.value.status == T.EINVAL
        import torch
        if not torch.cuda.is_available():
            # no CPU fallback: device work fails with a CUDA status
            with pytest.raises(T.TdseError) as e:
                T.tdse_set_wavepacket(ctx, 0, (1, 1, 1), (0.5, 0.5, 0.5), (0, 0, 1))
            assert e.value.status in (T.ECUDA, T.ENOMEM)
    finally:
        T.tdse_destroy(ctx)


def test_new_entry_points_validate_before_device_work(lib):
    """Argument checks of the frame buffer, the cell-potential interpolation and the
    Eq. 16 dissimilarity answer EINVAL without touching a GPU."""
    import numpy as np
    ctx = T.tdse_create([_params(det_k=-1)])
    try:
        with pytest.raises(T.TdseError) as e:
            T.tdse_set_frame_capacity(ctx, 0, 4)            # no detector plane
        assert e.value.status == T.EINVAL
        with pytest.raises(T.TdseError) as e:
            T.tdse_set_potential_grid(ctx, 0, np.zeros((3, 3, 3)), (1.0, -1.0, 1.0))
        assert e.value.status == T.EINVAL
        with pytest.raises(T.TdseError) as e:
            T.tdse_set_potential_grid(ctx, 0, np.zeros((3, 3, 3)), (1.0, 1.0, 1.0),
                                      (0.0, float("nan"), 0.0))
        assert e.value.status == T.EINVAL
    finally:
        T.tdse_destroy(ctx)
    f = np.zeros((2, 3, 4))
    t = np.array([0.0, 1.0, 2.0])
    for args in [(f, t, 1.0, 1.0, 0.1), (f, t, 0.0, 1.0, -1.0), (f, t, 5.0, 6.0, 0.1)]:
        with pytest.raises(T.TdseError) as e:
            T.tdse_dissimilarity(*args)
        assert e.value.status == T.EINVAL


def test_static_observables_validate_before_device_work(lib):
    """tdse_observables_static rejects a bad geometry with EINVAL before any CUDA
    call: the dummy host pointers below are never dereferenced."""
    import numpy as np
    buf = np.zeros(4)
    out = np.zeros(3)
    ptr = buf.ctypes.data_as(ctypes.c_void_p)
    optr = out.ctypes.data_as(ctypes.c_void_p)
    for field, value in (("nz", 8193), ("ny", 1 << 27), ("hz", 0.0)):
        p = _params(**{field: value})
        assert T.lib().tdse_observables_static(ctypes.byref(p), ptr, ptr, None, optr, None) == T.EINVAL
    for axis in range(3):               # boundary flags tdse_create would reject
        p = _params()
        p.bc[axis] = 2
        assert T.lib().tdse_observables_static(ctypes.byref(p), ptr, ptr, None, optr, None) == T.EINVAL
    p = _params()
    assert T.lib().tdse_observables_static(ctypes.byref(p), None, ptr, None, optr, None) == T.EINVAL


def test_version_string(lib):
    assert "sm_103a" in T.tdse_version()


def test_build_is_stale_when_flags_change(lib, monkeypatch):
    """The library is rebuilt when the compiler flags differ from those recorded
    at its build, not only when a source is newer."""
    from paper_2401_07416_gb300 import build as B
    assert not B._stale()
    monkeypatch.setattr(B, "FLAGS", B.FLAGS + ["-DTDSE_FLAG_PROBE"])
    assert B._stale()
    monkeypatch.setattr(B, "ARCH", ["-gencode", "arch=compute_100a,code=sm_100a"])
    assert B._stale()
