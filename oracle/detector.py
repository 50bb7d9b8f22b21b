"""Oracle of the detector-plane data of arXiv 2401.07416, Sec. 2.3 and Sec. 3.2.

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, FP64, written
from the paper's definitions with nothing blocked, fused or reordered.

* Eq. 15: the detector-plane density frame rho = psi_R^2 + psi_I^2 on the plane
  D = {z = z_det}.  With psi_R at integer and psi_I at half-integer time levels,
  the density at step n is R^n^2 + I^{n-1/2}^2 (Sec. 2.1, the sentence after
  Eq. 9); the detector plane is the grid plane det_k.
* Eq. 16: the dissimilarity of two trajectories k, j,
      d_kj = 1/(t1 - t0) * int_{t0}^{t1} ( int_D (rho_k - rho_j)^2 dr )^{1/2} dt.
  Reading (the paper gives the integral only): frames are kept every h-th step,
  so the time integral is the trapezoidal rule over the frames whose time lies
  in [t0, t1]; a single such frame stands for the whole window.  The plane
  integral is dA times the sum over the pixels (dA = h_x h_y).
"""
from __future__ import annotations

import numpy as np


def detector_frame(R: np.ndarray, I: np.ndarray, det_k: int) -> np.ndarray:
    """Eq. 15 at one time level: R[det_k]^2 + I[det_k]^2 for [nz][ny][nx] arrays."""
    r = np.asarray(R, dtype=np.float64)[det_k]
    i = np.asarray(I, dtype=np.float64)[det_k]
    return r * r + i * i


def window_weights(t: np.ndarray, t0: float, t1: float) -> np.ndarray:
    """Trapezoidal weights of the frame times inside [t0, t1] (zero outside), so that
    sum_m w_m f(t_m) approximates int f dt over the frames in the window."""
    t = np.asarray(t, dtype=np.float64)
    inside = np.nonzero((t >= t0) & (t <= t1))[0]
    w = np.zeros(t.shape[0])
    if inside.size == 0:
        raise ValueError("no frame time in [t0, t1]")
    if inside.size == 1:
        w[inside[0]] = t1 - t0
        return w
    for a, b in zip(inside[:-1], inside[1:]):
        half = 0.5 * (t[b] - t[a])
        w[a] += half
        w[b] += half
    return w


def dissimilarity(frames: np.ndarray, t: np.ndarray, t0: float, t1: float, dA: float) -> np.ndarray:
    """Eq. 16 for every pair of K trajectories: frames is [K][M][P] (M frames of P
    pixels at the common times t[M]); returns d[K][K]."""
    F = np.asarray(frames, dtype=np.float64)
    K, M = F.shape[0], F.shape[1]
    F = F.reshape(K, M, -1)
    w = window_weights(t, t0, t1)
    d = np.zeros((K, K))
    for k in range(K):
        for j in range(K):
            total = 0.0
            for m in range(M):
                if w[m] == 0.0:
                    continue
                diff = F[k, m] - F[j, m]
                total += w[m] * np.sqrt(dA * np.sum(diff * diff))
            d[k, j] = total / (t1 - t0)
    return d
