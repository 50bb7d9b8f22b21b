"""Thin ctypes binding of libtdse (include/tdse.h), function for function.

Only argument marshalling happens here: every computation runs in the CUDA
kernels of ``libtdse.so``.  Arrays may be numpy arrays (host memory) or torch
CUDA tensors (device memory, float64, contiguous); the ``on_device`` flag of the
C call is derived from the argument.  Every non-zero status raises ``TdseError``
with the library's message.  There is no fallback: if ``libtdse.so`` is missing
or no GPU is present the calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdse.so")

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "TDSE_OK", -1: "TDSE_EINVAL", -2: "TDSE_ENOMEM", -3: "TDSE_ECUDA",
                -4: "TDSE_EUNSTABLE", -5: "TDSE_ETIMEOUT", -6: "TDSE_ESTATE"}
FP64, FP32, FP32_KAHAN = W.FP64, W.FP32, W.FP32_KAHAN


class TdseError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("dt", ctypes.c_double), ("hbar", ctypes.c_double), ("mass", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("mask_lo", ctypes.c_int), ("mask_hi", ctypes.c_int),
                ("mask_eta", ctypes.c_double), ("det_k", ctypes.c_int),
                ("obs_every", ctypes.c_int), ("ckpt_every", ctypes.c_int),
                ("precision", ctypes.c_int), ("tblock", ctypes.c_int),
                ("mask_kind", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class Obs(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_double), ("norm_paper", ctypes.c_double),
                ("energy", ctypes.c_double), ("flux", ctypes.c_double),
                ("flux_integrated", ctypes.c_double), ("t", ctypes.c_double),
                ("step", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


MAX_TBLOCK = 4   # TDSE_MAX_TBLOCK


class Profile(ctypes.Structure):
    _fields_ = [("step_launches", ctypes.c_longlong), ("step_ms", ctypes.c_double),
                ("reduce_launches", ctypes.c_longlong), ("reduce_ms", ctypes.c_double),
                ("cells_per_launch", ctypes.c_longlong), ("steps_per_launch", ctypes.c_int),
                ("reserved", ctypes.c_int),
                ("launches_at_depth", ctypes.c_longlong * (MAX_TBLOCK + 1)),
                ("ms_at_depth", ctypes.c_double * (MAX_TBLOCK + 1)),
                ("adjoint_steps", ctypes.c_longlong), ("adjoint_ms", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("tblock", ctypes.c_int), ("variant", ctypes.c_int * (MAX_TBLOCK + 1)),
                ("ms_per_step", ctypes.c_double * (MAX_TBLOCK + 1)),
                ("name", (ctypes.c_char * 48) * (MAX_TBLOCK + 1)),
                ("chunk", ctypes.c_int * (MAX_TBLOCK + 1))]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# C signatures: name -> (restype, argtypes)
_VP, _I, _D, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
SIGNATURES = {
    "tdse_create": (_I, [ctypes.POINTER(Params), _I, ctypes.POINTER(_VP)]),
    "tdse_set_allocator": (_I, [_VP, ALLOC_FN, FREE_FN, _VP]),
    "tdse_set_stream": (_I, [_VP, _VP]),
    "tdse_set_potential": (_I, [_VP, _I, _VP, _I]),
    "tdse_set_atoms": (_I, [_VP, _I, _I, _VP, _D, _D]),
    "tdse_get_potential": (_I, [_VP, _I, _VP, _I]),
    "tdse_set_wavepacket": (_I, [_VP, _I, _VP, _VP, _VP]),
    "tdse_set_state": (_I, [_VP, _I, _VP, _VP, _I]),
    "tdse_step": (_I, [_VP, _LL]),
    "tdse_observables": (_I, [_VP, _I, ctypes.POINTER(Obs)]),
    "tdse_get_obs_history": (_I, [_VP, _I, _VP, _I, ctypes.POINTER(_I)]),
    "tdse_get_state": (_I, [_VP, _I, _VP, _VP, _I]),
    "tdse_get_flux_map": (_I, [_VP, _I, _VP, _I]),
    "tdse_set_frame_capacity": (_I, [_VP, _I, _I]),
    "tdse_set_potential_grid": (_I, [_VP, _I, _VP, _I, _I, _I, _VP, _VP, _I]),
    "tdse_get_frames": (_I, [_VP, _I, _VP, _VP, _I, ctypes.POINTER(_I), _I]),
    "tdse_dissimilarity": (_I, [_VP, _I, _I, ctypes.c_longlong, _VP, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, _VP, _I, _VP]),
    "tdse_adjoint": (_I, [_VP, _I, _VP, _VP, _VP, _I]),
    "tdse_save_state": (_I, [_VP, ctypes.c_char_p]),
    "tdse_load_state": (_I, [_VP, ctypes.c_char_p]),
    "tdse_variant_count": (_I, [_I, _I]),
    "tdse_set_variant": (_I, [_VP, _I, _I]),
    "tdse_autotune": (_I, [_VP, _I]),
    "tdse_get_tuning": (_I, [_VP, ctypes.POINTER(Tuning)]),
    "tdse_set_graphs": (_I, [_VP, _I]),
    "tdse_set_wait_limit": (_I, [_VP, _LL]),
    "tdse_set_adjoint_fused": (_I, [_VP, _I]),
    "tdse_set_chunk": (_I, [_VP, _I, _I]),
    "tdse_set_profiling": (_I, [_VP, _I]),
    "tdse_get_profile": (_I, [_VP, ctypes.POINTER(Profile)]),
    "tdse_observables_static": (_I, [ctypes.POINTER(Params), _VP, _VP, _VP, _VP, _VP]),
    "tdse_last_error": (ctypes.c_char_p, [_VP]),
    "tdse_version": (ctypes.c_char_p, []),
    "tdse_destroy": (_I, [_VP]),
}

_lib = None


def lib():
    """Open libtdse.so (built by ``paper_2401_07416_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2401_07416_gb300.build` (needs nvcc)")
        _lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _check(ctx, status: int):
    if status != OK:
        msg = lib().tdse_last_error(ctx)
        raise TdseError(status, msg.decode() if msg else "")


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _arg(a, writable=False):
    """(pointer, on_device, keepalive) for a numpy array or a torch CUDA tensor."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("torch tensors passed to libtdse must be contiguous float64")
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0, a
    arr = np.asarray(a)
    if arr.dtype != np.float64 or not arr.flags.c_contiguous or (writable and not arr.flags.writeable):
        if writable:
            raise TypeError("output arrays must be writable C-contiguous float64")
        arr = np.ascontiguousarray(arr, dtype=np.float64)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


def params_from_grid(g: W.Grid, precision: int = FP64, tblock: int = 0,
                     ckpt_every: int = 0) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = g.nx, g.ny, g.nz
    p.hx, p.hy, p.hz = g.hx, g.hy, g.hz
    p.dt, p.hbar, p.mass = g.dt, g.hbar, g.mass
    p.bc[:] = list(g.bc)
    p.mask_lo, p.mask_hi, p.mask_eta = g.mask_lo, g.mask_hi, g.mask_eta
    p.det_k = g.det_k
    p.obs_every = g.obs_every
    p.ckpt_every = ckpt_every
    p.precision = precision
    p.tblock = tblock
    p.mask_kind = getattr(g, "mask_kind", 0)
    return p


# ------------------------------------------------------------------ C calls, same names

def tdse_version() -> str:
    return lib().tdse_version().decode()


def tdse_create(params: Sequence[Params]):
    arr = (Params * len(params))(*params)
    ctx = ctypes.c_void_p()
    st = lib().tdse_create(arr, len(params), ctypes.byref(ctx))
    if st != OK:
        raise TdseError(st, "tdse_create rejected the parameters")
    return ctx


def tdse_set_allocator(ctx, alloc_fn, free_fn, user=None):
    _check(ctx, lib().tdse_set_allocator(ctx, alloc_fn, free_fn, user))


def tdse_set_stream(ctx, stream_ptr: int):
    _check(ctx, lib().tdse_set_stream(ctx, ctypes.c_void_p(stream_ptr)))


def tdse_set_potential(ctx, member: int, V):
    p, dev, keep = _arg(V)
    _check(ctx, lib().tdse_set_potential(ctx, member, p, dev))


def tdse_set_atoms(ctx, member: int, atoms, soft_a2: float = 0.25, r_cut: float = 0.0):
    a = np.ascontiguousarray(atoms, dtype=np.float64).reshape(-1, 4)
    _check(ctx, lib().tdse_set_atoms(ctx, member, a.shape[0], a.ctypes.data_as(ctypes.c_void_p),
                                     soft_a2, r_cut))


def tdse_get_potential(ctx, member: int, V):
    p, dev, _ = _arg(V, writable=True)
    _check(ctx, lib().tdse_get_potential(ctx, member, p, dev))
    return V


def tdse_set_wavepacket(ctx, member: int, r0, sigma, k0):
    r0, sigma, k0 = (np.ascontiguousarray(v, dtype=np.float64) for v in (r0, sigma, k0))
    _check(ctx, lib().tdse_set_wavepacket(ctx, member, r0.ctypes.data_as(ctypes.c_void_p),
                                          sigma.ctypes.data_as(ctypes.c_void_p),
                                          k0.ctypes.data_as(ctypes.c_void_p)))


def tdse_set_state(ctx, member: int, R, I):
    pr, dr, kr = _arg(R)
    pi, di, ki = _arg(I)
    if dr != di:
        raise TypeError("R and I must both be host or both be device arrays")
    _check(ctx, lib().tdse_set_state(ctx, member, pr, pi, dr))


def tdse_step(ctx, nsteps: int):
    _check(ctx, lib().tdse_step(ctx, int(nsteps)))


def tdse_observables(ctx, member: int) -> dict:
    o = Obs()
    _check(ctx, lib().tdse_observables(ctx, member, ctypes.byref(o)))
    return o.as_dict()


def tdse_get_obs_history(ctx, member: int) -> np.ndarray:
    n = ctypes.c_int()
    _check(ctx, lib().tdse_get_obs_history(ctx, member, None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, 4))
    _check(ctx, lib().tdse_get_obs_history(ctx, member, out.ctypes.data_as(ctypes.c_void_p),
                                           n.value, ctypes.byref(n)))
    return out


def tdse_get_state(ctx, member: int, R=None, I=None):
    """Fill R and I (numpy or torch float64 of shape (nz, ny, nx)); returns them."""
    pr, dr, _ = _arg(R, writable=True)
    pi, di, _ = _arg(I, writable=True)
    dev = dr if R is not None else di
    _check(ctx, lib().tdse_get_state(ctx, member, pr, pi, dev))
    return R, I


def tdse_get_flux_map(ctx, member: int, F):
    p, dev, _ = _arg(F, writable=True)
    _check(ctx, lib().tdse_get_flux_map(ctx, member, p, dev))
    return F


def tdse_set_potential_grid(ctx, member: int, Vc, cell, origin=(0.0, 0.0, 0.0)):
    """Potential interpolated from one periodic cell Vc[cnz][cny][cnx] of lengths
    `cell` whose lattice starts at `origin` (numpy or torch CUDA float64)."""
    pv, dev, keep = _arg(Vc)
    cnz, cny, cnx = tuple(Vc.shape)
    c = (ctypes.c_double * 3)(*cell)
    o = (ctypes.c_double * 3)(*origin)
    _check(ctx, lib().tdse_set_potential_grid(ctx, member, pv, cnx, cny, cnz, c, o, dev))


def tdse_set_frame_capacity(ctx, member: int, capacity: int):
    _check(ctx, lib().tdse_set_frame_capacity(ctx, member, capacity))


def tdse_get_frames(ctx, member: int, ny: int, nx: int):
    """(frames [count][ny][nx], steps [count]) recorded for member m (Eq. 15)."""
    n = ctypes.c_int()
    _check(ctx, lib().tdse_get_frames(ctx, member, None, None, 0, ctypes.byref(n), 0))
    frames = np.zeros((n.value, ny, nx))
    steps = np.zeros(n.value, dtype=np.int64)
    _check(ctx, lib().tdse_get_frames(ctx, member, frames.ctypes.data_as(ctypes.c_void_p),
                                      steps.ctypes.data_as(ctypes.c_void_p), n.value,
                                      ctypes.byref(n), 0))
    return frames, steps


def tdse_dissimilarity(frames, t, t0: float, t1: float, dA: float, d=None, stream_ptr: int = 0):
    """Eq. 16 for frames [K][M][P...] (numpy, or torch CUDA float64); returns d [K][K]
    (numpy for numpy input, else the given or a new torch tensor)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    shape = tuple(frames.shape)
    K, M = shape[0], shape[1]
    P = int(np.prod(shape[2:])) if len(shape) > 2 else 1
    pf, dev, keep = _arg(frames)
    if d is None:
        if dev:
            import torch
            d = torch.empty((K, K), dtype=torch.float64, device=frames.device)
        else:
            d = np.zeros((K, K))
    pd, ddev, _ = _arg(d, writable=True)
    if ddev != dev:
        raise TypeError("frames and d must both be on the device or both on the host")
    st = lib().tdse_dissimilarity(pf, K, M, P, t.ctypes.data_as(ctypes.c_void_p), t0, t1, dA,
                                  pd, dev, ctypes.c_void_p(stream_ptr))
    if st != OK:
        raise TdseError(st, "tdse_dissimilarity failed")
    return d


def tdse_adjoint(ctx, member: int, dL_dF, dL_dV=None, dL_datoms=None):
    pf, df, kf = _arg(dL_dF)
    pv, dv, _ = _arg(dL_dV, writable=True)
    pa, da, _ = _arg(dL_datoms, writable=True)
    devs = {d for d, a in ((df, dL_dF), (dv, dL_dV), (da, dL_datoms)) if a is not None}
    if len(devs) > 1:
        raise TypeError("adjoint arrays must all be host or all be device arrays")
    _check(ctx, lib().tdse_adjoint(ctx, member, pf, pv, pa, devs.pop() if devs else 0))


def tdse_save_state(ctx, path: str):
    _check(ctx, lib().tdse_save_state(ctx, os.fsencode(path)))


def tdse_load_state(ctx, path: str):
    _check(ctx, lib().tdse_load_state(ctx, os.fsencode(path)))


def tdse_variant_count(precision: int, tsteps: int) -> int:
    return lib().tdse_variant_count(precision, tsteps)


def tdse_set_variant(ctx, tsteps: int, variant: int):
    _check(ctx, lib().tdse_set_variant(ctx, tsteps, variant))


def tdse_autotune(ctx, launches: int = 4):
    _check(ctx, lib().tdse_autotune(ctx, launches))


def tdse_get_tuning(ctx) -> dict:
    t = Tuning()
    _check(ctx, lib().tdse_get_tuning(ctx, ctypes.byref(t)))
    depths = [T for T in range(1, MAX_TBLOCK + 1) if t.name[T].value]
    return {"tblock": t.tblock,
            "variant": {T: t.variant[T] for T in depths},
            "ms_per_step": {T: t.ms_per_step[T] for T in depths},
            "name": {T: t.name[T].value.decode() for T in depths},
            "chunk": {T: t.chunk[T] for T in depths}}


def tdse_set_graphs(ctx, enable: bool):
    _check(ctx, lib().tdse_set_graphs(ctx, int(bool(enable))))


def tdse_set_chunk(ctx, tsteps: int, planes: int):
    _check(ctx, lib().tdse_set_chunk(ctx, tsteps, planes))


def tdse_set_adjoint_fused(ctx, enable: bool):
    _check(ctx, lib().tdse_set_adjoint_fused(ctx, int(bool(enable))))


def tdse_set_wait_limit(ctx, ns: int):
    _check(ctx, lib().tdse_set_wait_limit(ctx, int(ns)))


def tdse_set_profiling(ctx, enable: bool):
    _check(ctx, lib().tdse_set_profiling(ctx, int(bool(enable))))


def tdse_get_profile(ctx) -> dict:
    p = Profile()
    _check(ctx, lib().tdse_get_profile(ctx, ctypes.byref(p)))
    out = {k: getattr(p, k) for k, _ in p._fields_ if k not in ("reserved", "launches_at_depth",
                                                                 "ms_at_depth")}
    out["launches_at_depth"] = {T: p.launches_at_depth[T] for T in range(1, MAX_TBLOCK + 1)}
    out["ms_at_depth"] = {T: p.ms_at_depth[T] for T in range(1, MAX_TBLOCK + 1)}
    return out


def tdse_observables_static(params: Params, R, I, V=None, stream_ptr: int = 0) -> dict:
    """Q, paper norm and energy of a device-resident FP64 state, computed without
    any device allocation (for callers that cannot allocate)."""
    import torch
    pr, dr, _ = _arg(R)
    pi, di, _ = _arg(I)
    pv, dv, _ = _arg(V)
    if not (dr and di and (V is None or dv)):
        raise TypeError("R, I and V must be CUDA tensors")
    # the kernels read nx*ny*nz values of each array (and their neighbours) on the
    # current device: anything shorter, or elsewhere, is refused here
    n = params.nx * params.ny * params.nz
    dev = torch.cuda.current_device()
    for name, a in (("R", R), ("I", I), ("V", V)):
        if a is None:
            continue
        if a.numel() != n:
            raise ValueError(f"{name} holds {a.numel()} values, the grid has {n}")
        if a.device.index != dev:
            raise ValueError(f"{name} is on cuda:{a.device.index}, the current device is cuda:{dev}")
    out = np.zeros(3)
    st = lib().tdse_observables_static(ctypes.byref(params), pr, pi, pv,
                                       out.ctypes.data_as(ctypes.c_void_p),
                                       ctypes.c_void_p(stream_ptr))
    if st != OK:
        raise TdseError(st, "tdse_observables_static failed (nz > 8192, bad geometry or CUDA error)")
    return {"Q": out[0], "norm_paper": out[1], "energy": out[2]}


def tdse_last_error(ctx) -> str:
    m = lib().tdse_last_error(ctx)
    return m.decode() if m else ""


def tdse_destroy(ctx):
    if ctx:
        lib().tdse_destroy(ctx)
