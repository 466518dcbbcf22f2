"""FNO surrogate oracle (TEST INFRASTRUCTURE ONLY): the network of the
library's surrogate, written from its definition in float64 numpy, with
numpy's real FFTs as the transform step, plus central finite differences.

Parameter vector layout (flat, in this order):
  W_lift [C][NP+3], b_lift [C],
  per layer l: R_l [2][mode][C][C] (real, imaginary parts; mode = (kz, ky, kx)
               over kz, ky in S = {0..m-1, P-m..P-1}, kx in 0..m-1),
               W_l [C][C], b_l [C],
  W_q1 [H][C], b_q1 [H], W_q2 [NO][H], b_q2 [NO].
Inputs: params [B][NP]; the features add x, y, z = -1 + 2 i / P.
Fields are [B][channels][z][y][x].
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

__all__ = ["FnoConfig", "num_params", "unpack", "forward", "loss", "finite_difference_grad"]


class FnoConfig:
    def __init__(self, in_params, width, layers, patch, modes, hidden, out_channels):
        self.NP, self.C, self.L, self.P, self.m, self.H, self.NO = (in_params, width, layers, patch, modes,
                                                                    hidden, out_channels)
        self.NT = 2 * modes
        self.MODES = modes * self.NT * self.NT


def num_params(c: FnoConfig) -> int:
    FI = c.NP + 3
    n = c.C * FI + c.C
    n += c.L * (2 * c.MODES * c.C * c.C + c.C * c.C + c.C)
    n += c.H * c.C + c.H + c.NO * c.H + c.NO
    return n


def unpack(theta: np.ndarray, c: FnoConfig) -> dict:
    FI = c.NP + 3
    o = 0
    out = {}

    def take(name, shape):
        nonlocal o
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n

    take("Wl", (c.C, FI))
    take("bl", (c.C,))
    for l in range(c.L):
        take("R%d" % l, (2, c.NT, c.NT, c.m, c.C, c.C))
        take("W%d" % l, (c.C, c.C))
        take("b%d" % l, (c.C,))
    take("Wq1", (c.H, c.C))
    take("bq1", (c.H,))
    take("Wq2", (c.NO, c.H))
    take("bq2", (c.NO,))
    assert o == theta.size
    return out


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _features(prm, c: FnoConfig):
    B = prm.shape[0]
    P = c.P
    q = -1.0 + 2.0 * np.arange(P) / P
    feat = np.empty((B, c.NP + 3, P, P, P))
    feat[:, :c.NP] = prm[:, :, None, None, None]
    feat[:, c.NP] = q[None, None, None, :]            # x (last axis)
    feat[:, c.NP + 1] = q[None, None, :, None]        # y
    feat[:, c.NP + 2] = q[None, :, None, None]        # z
    return feat


def forward(theta: np.ndarray, prm: np.ndarray, c: FnoConfig) -> np.ndarray:
    """Network output [B][NO][P][P][P]."""
    w = unpack(np.asarray(theta, dtype=np.float64), c)
    P, m = c.P, c.m
    S = np.concatenate([np.arange(m), np.arange(P - m, P)])
    v = np.einsum("of,bfzyx->bozyx", w["Wl"], _features(np.asarray(prm, np.float64), c)) \
        + w["bl"][None, :, None, None, None]
    for l in range(c.L):
        V = np.fft.rfftn(v, axes=(-3, -2, -1))[:, :, S][:, :, :, S][..., :m]      # [B, C, NT, NT, m]
        R = w["R%d" % l][0] + 1j * w["R%d" % l][1]                                 # [NT, NT, m, C, C]
        U = np.einsum("bizyx,zyxio->bozyx", V, R)
        full = np.zeros(v.shape[:2] + (P, P, P // 2 + 1), dtype=np.complex128)
        full[:, :, S[:, None], S[None, :], :m] = U
        spec = np.fft.irfftn(full, s=(P, P, P), axes=(-3, -2, -1))
        z = spec + np.einsum("oc,bczyx->bozyx", w["W%d" % l], v) + w["b%d" % l][None, :, None, None, None]
        v = _gelu(z) if l + 1 < c.L else z
    h = _gelu(np.einsum("hc,bczyx->bhzyx", w["Wq1"], v) + w["bq1"][None, :, None, None, None])
    return np.einsum("oh,bhzyx->bozyx", w["Wq2"], h) + w["bq2"][None, :, None, None, None]


def loss(theta, prm, target, c: FnoConfig) -> float:
    """Mean squared error over all outputs."""
    d = forward(theta, prm, c) - target
    return float(np.mean(d * d))


def finite_difference_grad(theta, prm, target, c: FnoConfig, idx, h=1e-5) -> np.ndarray:
    """Central differences of the loss at the parameter indices idx."""
    theta = np.array(theta, dtype=np.float64, copy=True)
    g = np.empty(len(idx))
    for n, i in enumerate(idx):
        t0 = theta[i]
        theta[i] = t0 + h
        lp = loss(theta, prm, target, c)
        theta[i] = t0 - h
        lm = loss(theta, prm, target, c)
        theta[i] = t0
        g[n] = (lp - lm) / (2 * h)
    return g
