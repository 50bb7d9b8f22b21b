"""PyTorch-facing wrapper of libtdse: device memory from torch's caching
allocator, work on torch's current CUDA stream, results as numpy or torch.

Every computation runs in libtdse's CUDA kernels through the C ABI.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Union

import numpy as np

from . import tdse as T
from . import workloads as W


class Sim:
    """One context holding `len(grids)` independent simulations (a batch)."""

    def __init__(self, grids: Union[W.Grid, Sequence[W.Grid]], precision: int = T.FP32_KAHAN,
                 tblock: int = 0, ckpt_every: int = 0, torch_memory: bool = True):
        if isinstance(grids, W.Grid):
            grids = [grids]
        self.grids: List[W.Grid] = list(grids)
        self.precision = precision
        self.ctx = T.tdse_create([T.params_from_grid(g, precision, tblock, ckpt_every)
                                  for g in self.grids])
        self._callbacks = None
        if torch_memory:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("libtdse needs a CUDA device; none is available")
            stream = torch.cuda.current_stream()
            dev = torch.cuda.current_device()

            def _alloc(nbytes, user):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._callbacks = (T.ALLOC_FN(_alloc), T.FREE_FN(_free))
            T.tdse_set_allocator(self.ctx, self._callbacks[0], self._callbacks[1])
            T.tdse_set_stream(self.ctx, stream.cuda_stream)

    # -- set-up
    def set_atoms(self, member: int, atoms: np.ndarray, soft_a2: float = 0.25, r_cut: float = 0.0):
        T.tdse_set_atoms(self.ctx, member, atoms, soft_a2, r_cut)

    def set_potential(self, member: int, V):
        T.tdse_set_potential(self.ctx, member, V)

    def set_potential_grid(self, member: int, Vc, cell, origin=(0.0, 0.0, 0.0)):
        """Potential interpolated from one periodic cell (Sec. 2.3)."""
        T.tdse_set_potential_grid(self.ctx, member, Vc, cell, origin)

    def potential(self, member: int = 0) -> np.ndarray:
        g = self.grids[member]
        V = np.zeros((g.nz, g.ny, g.nx))
        T.tdse_get_potential(self.ctx, member, V)
        return V

    def set_packet(self, member: int, packet: W.Packet):
        T.tdse_set_wavepacket(self.ctx, member, packet.r0, packet.sigma, packet.k0)

    def set_state(self, member: int, R, I):
        T.tdse_set_state(self.ctx, member, R, I)

    def autotune(self, launches: int = 4) -> dict:
        """Time every kernel variant on this batch and keep the fastest."""
        T.tdse_autotune(self.ctx, launches)
        return T.tdse_get_tuning(self.ctx)

    def tuning(self) -> dict:
        return T.tdse_get_tuning(self.ctx)

    # -- stepping and results
    def step(self, n: int):
        T.tdse_step(self.ctx, n)

    def observables(self, member: int = 0) -> dict:
        return T.tdse_observables(self.ctx, member)

    def history(self, member: int = 0) -> np.ndarray:
        return T.tdse_get_obs_history(self.ctx, member)

    def state(self, member: int = 0):
        g = self.grids[member]
        R = np.zeros((g.nz, g.ny, g.nx))
        I = np.zeros((g.nz, g.ny, g.nx))
        T.tdse_get_state(self.ctx, member, R, I)
        return R, I

    def set_frames(self, capacity: int, member: int = 0):
        """Record up to `capacity` detector density frames (Eq. 15) of member m."""
        T.tdse_set_frame_capacity(self.ctx, member, capacity)

    def frames(self, member: int = 0):
        """(frames [count][ny][nx], steps [count]) recorded so far."""
        g = self.grids[member]
        return T.tdse_get_frames(self.ctx, member, g.ny, g.nx)

    def flux_map(self, member: int = 0) -> np.ndarray:
        g = self.grids[member]
        F = np.zeros((g.ny, g.nx))
        T.tdse_get_flux_map(self.ctx, member, F)
        return F

    def save(self, path: str):
        T.tdse_save_state(self.ctx, path)

    def load(self, path: str):
        T.tdse_load_state(self.ctx, path)

    def close(self):
        if self.ctx:
            T.tdse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _torch():
    import torch
    return torch


def flux_from_atoms(atoms, sim: "Sim", member: int, packet: W.Packet, nsteps: int,
                    soft_a2: float = 0.25, r_cut: float = 0.0):
    """Differentiable map atoms [n, 4] (x, y, z, Z) -> time-integrated detector flux
    F [ny, nx].  forward builds V from the atoms, sets the packet and runs `nsteps`
    (every member of `sim` advances: use a one-member Sim); backward calls
    tdse_adjoint.  `sim` must have been created with ckpt_every > 0."""
    torch = _torch()

    class Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a):
            sim.set_atoms(member, a.detach().cpu().double().numpy(), soft_a2, r_cut)
            sim.set_packet(member, packet)
            sim.step(nsteps)
            return torch.from_numpy(sim.flux_map(member)).to(a.device)

        @staticmethod
        def backward(ctx, gF):
            g = np.zeros(tuple(atoms.shape))
            T.tdse_adjoint(sim.ctx, member, gF.detach().cpu().double().numpy(), None, g)
            return torch.from_numpy(g).to(gF.device)

    return Fn.apply(atoms)


def flux_from_potential(V, sim: "Sim", member: int, packet: W.Packet, nsteps: int):
    """Differentiable map V [nz, ny, nx] -> F [ny, nx] (same contract as flux_from_atoms)."""
    torch = _torch()

    class Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v):
            sim.set_potential(member, v.detach().double().contiguous())
            sim.set_packet(member, packet)
            sim.step(nsteps)
            return torch.from_numpy(sim.flux_map(member)).to(v.device)

        @staticmethod
        def backward(ctx, gF):
            g = np.zeros(tuple(V.shape))
            T.tdse_adjoint(sim.ctx, member, gF.detach().cpu().double().numpy(), g, None)
            return torch.from_numpy(g).to(gF.device)

    return Fn.apply(V)


def diffraction_loss(F, F_target):
    """L = sum over detector pixels of (F - F*)^2 (no area weight)."""
    return ((F - F_target) ** 2).sum()
