"""Oracle: a plain FP64 CPU implementation of the FDTD leapfrog for the 3-D TDSE.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only callers.
The CUDA library never imports, links or executes anything here, and this package
never imports the CUDA library: the two share no code.

``tdse_oracle.c`` is compiled with gcc (``-O2 -fopenmp -ffp-contract=off``, no
fused multiply-adds so that x86 and Arm give the same bits) into
``liboracle.so`` next to it; this module marshals numpy arrays to it.

Every function follows the paper (arXiv 2401.07416) as cited in ``tdse_oracle.c``:
Eqs. 8-9 (update), Eq. 3 (packet), Eq. 4 (wavelength), Eq. 11 (time step),
Eqs. 13-14 (periodic neighbours).  Readings where the paper is silent are listed
in that file's header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdse_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


class OrcGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("dt", ctypes.c_double), ("hbar", ctypes.c_double), ("mass", ctypes.c_double),
                ("bc", ctypes.c_int * 3), ("mask_lo", ctypes.c_int), ("mask_hi", ctypes.c_int),
                ("mask_eta", ctypes.c_double), ("det_k", ctypes.c_int),
                ("mask_kind", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc if it is missing or older than its source."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                           "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        g = ctypes.POINTER(OrcGrid)
        sig = {
            "orc_coefficients": (None, [g, p]),
            "orc_default_dt": (d, [d, d, d, d, d]),
            "orc_wavelength": (d, [d, d, d]),
            "orc_apply_A": (None, [g, p, p, p]),
            "orc_mask": (None, [g, p]),
            "orc_potential_atoms": (None, [g, i, p, d, d, p]),
            "orc_potential_atoms_at": (None, [g, p, p, i, p, d, d, p]),
            "orc_wavepacket_at": (None, [g, p, p, p, p, p, p]),
            "orc_atom_gradient": (None, [g, i, p, d, d, p, p]),
            "orc_wavepacket": (None, [g, p, p, p, p, p]),
            "orc_init_half": (None, [g, p, p, p, i]),
            "orc_step": (None, [g, p, p, p, p, p]),
            "orc_run": (None, [g, p, i, p, p, ctypes.c_long, p, p]),
            "orc_observables": (None, [g, p, p, p, p]),
            "orc_adjoint": (None, [g, p, i, p, p, ctypes.c_long, p, p]),
            "orc_set_threads": (None, [i]),
            "orc_max_threads": (i, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's loops (timing only)."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def _grid(g) -> OrcGrid:
    return OrcGrid(g.nx, g.ny, g.nz, g.hx, g.hy, g.hz, g.dt, g.hbar, g.mass,
                   (ctypes.c_int * 3)(*g.bc), g.mask_lo, g.mask_hi, g.mask_eta, g.det_k,
                   getattr(g, "mask_kind", 0))


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def shape(g):
    return (g.nz, g.ny, g.nx)


def coefficients(g) -> np.ndarray:
    out = np.zeros(4)
    lib().orc_coefficients(ctypes.byref(_grid(g)), _ptr(out))
    return out


def default_dt(hx, hy, hz, hbar=1.0, mass=1.0) -> float:
    return lib().orc_default_dt(hx, hy, hz, hbar, mass)


def wavelength(energy, hbar=1.0, mass=1.0) -> float:
    return lib().orc_wavelength(energy, hbar, mass)


def apply_A(g, V, f) -> np.ndarray:
    f = _f64(f)
    out = np.empty_like(f)
    lib().orc_apply_A(ctypes.byref(_grid(g)), _ptr(None if V is None else _f64(V)), _ptr(f),
                      _ptr(out))
    return out


def mask(g) -> np.ndarray:
    out = np.empty(g.nz)
    lib().orc_mask(ctypes.byref(_grid(g)), _ptr(out))
    return out


def potential_atoms(g, atoms, a2=0.25, rc=None) -> np.ndarray:
    """Softened-Coulomb potential; rc=None picks min(periodic lengths)/2 (no cut-off
    if no axis is periodic)."""
    atoms = _f64(atoms)
    if rc is None:
        rc = default_cutoff(g)
    V = np.empty(shape(g))
    lib().orc_potential_atoms(ctypes.byref(_grid(g)), atoms.shape[0], _ptr(atoms), a2, rc,
                              _ptr(V))
    return V


def potential_atoms_window(g, origin, period, atoms, a2=0.25, rc=0.0) -> np.ndarray:
    """Potential on the window grid g whose node (0,0,0) sits at `origin` of a larger
    grid; period[a] > 0 gives the larger grid's period along a (minimum image),
    period[a] <= 0 no images.  rc must be given: the larger grid's cut-off."""
    atoms = _f64(atoms)
    V = np.empty(shape(g))
    lib().orc_potential_atoms_at(ctypes.byref(_grid(g)), _ptr(_f64(origin)), _ptr(_f64(period)),
                                 atoms.shape[0], _ptr(atoms), a2, rc, _ptr(V))
    return V


def wavepacket_window(g, origin, r0, sigma, k0):
    """Eq. 3 packet on the window grid g at `origin`, normalised on the window."""
    R = np.empty(shape(g))
    I = np.empty(shape(g))
    lib().orc_wavepacket_at(ctypes.byref(_grid(g)), _ptr(_f64(origin)), _ptr(_f64(r0)),
                            _ptr(_f64(sigma)), _ptr(_f64(k0)), _ptr(R), _ptr(I))
    return R, I


def default_cutoff(g) -> float:
    lens = [n * h for n, h, b in ((g.nx, g.hx, g.bc[0]), (g.ny, g.hy, g.bc[1]),
                                   (g.nz, g.hz, g.bc[2])) if b == 0]
    return 0.5 * min(lens) if lens else 0.0


def atom_gradient(g, atoms, dLdV, a2=0.25, rc=None) -> np.ndarray:
    atoms = _f64(atoms)
    if rc is None:
        rc = default_cutoff(g)
    out = np.zeros_like(atoms)
    lib().orc_atom_gradient(ctypes.byref(_grid(g)), atoms.shape[0], _ptr(atoms), a2, rc,
                            _ptr(_f64(dLdV)), _ptr(out))
    return out


def wavepacket(g, r0, sigma, k0):
    R = np.empty(shape(g))
    I = np.empty(shape(g))
    lib().orc_wavepacket(ctypes.byref(_grid(g)), _ptr(_f64(r0)), _ptr(_f64(sigma)),
                         _ptr(_f64(k0)), _ptr(R), _ptr(I))
    return R, I


def init_half(g, V, R, I0, naive=False) -> np.ndarray:
    I = _f64(I0).copy()
    lib().orc_init_half(ctypes.byref(_grid(g)), _ptr(None if V is None else _f64(V)),
                        _ptr(_f64(R)), _ptr(I), int(naive))
    return I


def initial_state(g, packet, V=None, naive=False):
    """(R^0, I^{-1/2}) for a packet: Eq. 3 then the half-step start."""
    R, I0 = wavepacket(g, packet.r0, packet.sigma, packet.k0)
    return R, init_half(g, V, R, I0, naive)


def step(g, V, R, I, use_mask=True, want_flux=False):
    """One leapfrog step in place on copies; returns (R, I, j or None)."""
    R = _f64(R).copy()
    I = _f64(I).copy()
    M = mask(g) if use_mask else None
    j = np.zeros((g.ny, g.nx)) if want_flux else None
    lib().orc_step(ctypes.byref(_grid(g)), _ptr(None if V is None else _f64(V)), _ptr(M),
                   _ptr(R), _ptr(I), _ptr(j))
    return R, I, j


def run(g, V, R, I, nsteps, use_mask=True, flux=True):
    """nsteps leapfrog steps on copies; returns (R, I, F, jlast)."""
    R = _f64(R).copy()
    I = _f64(I).copy()
    F = np.zeros((g.ny, g.nx)) if flux else None
    jl = np.zeros((g.ny, g.nx)) if flux else None
    lib().orc_run(ctypes.byref(_grid(g)), _ptr(None if V is None else _f64(V)), int(use_mask),
                  _ptr(R), _ptr(I), int(nsteps), _ptr(F), _ptr(jl))
    return R, I, F, jl


def observables(g, V, R, I) -> dict:
    out = np.zeros(9)
    lib().orc_observables(ctypes.byref(_grid(g)), _ptr(None if V is None else _f64(V)),
                          _ptr(_f64(R)), _ptr(_f64(I)), _ptr(out))
    q = out[0]
    return {"Q": q, "norm_paper": out[1], "energy": out[2],
            "mean": out[3:6] / q, "second": out[6:9] / q}


def adjoint(g, V, R0, I0, nsteps, gF, use_mask=True) -> np.ndarray:
    """dL/dV for a loss L(F) of the integrated flux, given gF = dL/dF.
    (R0, I0) = Re/Im psi0 before the half-step start."""
    gV = np.zeros(shape(g))
    lib().orc_adjoint(ctypes.byref(_grid(g)), _ptr(None if V is None else _f64(V)),
                      int(use_mask), _ptr(_f64(R0)), _ptr(_f64(I0)), int(nsteps),
                      _ptr(_f64(gF)), _ptr(gV))
    return gV
