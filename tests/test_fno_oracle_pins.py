"""Pins of the surrogate-network oracle against independent definitions."""
import math

import numpy as np

from oracle import fno_oracle as F


def _zero_spectral(theta, c):
    w = F.unpack(theta, c)
    for l in range(c.L):
        w["R%d" % l][...] = 0.0
    return theta


def test_without_spectral_weights_the_net_is_a_pointwise_mlp():
    c = F.FnoConfig(2, 3, 2, 4, 1, 5, 2)
    rng = np.random.default_rng(0)
    theta = _zero_spectral(rng.standard_normal(F.num_params(c)) * 0.5, c)
    prm = rng.standard_normal((1, 2))
    out = F.forward(theta, prm, c)
    w = F.unpack(theta, c)
    gelu = lambda x: 0.5 * x * (1 + math.erf(x / math.sqrt(2)))
    q = lambda i: -1 + 2 * i / c.P
    for (z, y, x) in [(0, 0, 0), (1, 2, 3), (3, 1, 2)]:
        feat = [prm[0, 0], prm[0, 1], q(x), q(y), q(z)]
        v = [sum(w["Wl"][o][f] * feat[f] for f in range(5)) + w["bl"][o] for o in range(c.C)]
        for l in range(c.L):
            zz = [sum(w["W%d" % l][o][i] * v[i] for i in range(c.C)) + w["b%d" % l][o] for o in range(c.C)]
            v = [gelu(t) for t in zz] if l + 1 < c.L else zz
        h = [gelu(sum(w["Wq1"][k][i] * v[i] for i in range(c.C)) + w["bq1"][k]) for k in range(c.H)]
        o = [sum(w["Wq2"][j][k] * h[k] for k in range(c.H)) + w["bq2"][j] for j in range(c.NO)]
        assert np.allclose(out[0, :, z, y, x], o, atol=1e-12)


def _spectral_bruteforce(v, R, P, m):
    """Truncated spectral convolution by explicit sums: forward DFT at kept
    modes, complex channel mixing, real inverse with kx > 0 counted twice."""
    C = v.shape[0]
    S = list(range(m)) + list(range(P - m, P))
    out = np.zeros_like(v)
    grid = np.arange(P)
    for a, kz in enumerate(S):
        for b, ky in enumerate(S):
            for kx in range(m):
                ph = np.exp(-2j * np.pi * (kz * grid[:, None, None] + ky * grid[None, :, None] + kx * grid[None, None, :]) / P)
                Vk = np.array([np.sum(v[i] * ph) for i in range(C)])
                Uk = Vk @ R[a, b, kx]
                wgt = 1.0 if kx == 0 else 2.0
                for o in range(C):
                    out[o] += wgt * np.real(Uk[o] * np.conj(ph)) / P ** 3
    return out


def test_spectral_layer_equals_explicit_sums():
    c = F.FnoConfig(1, 2, 1, 6, 2, 2, 1)
    rng = np.random.default_rng(3)
    theta = rng.standard_normal(F.num_params(c)) * 0.3
    w = F.unpack(theta, c)
    # isolate the spectral layer: identity lift on channel 0/1 of the features is awkward,
    # so compare the layer's pre-activation through a one-layer net with W = 0, b = 0
    w["W0"][...] = 0.0
    w["b0"][...] = 0.0
    prm = rng.standard_normal((1, 1))
    # reconstruct v0 and the layer output via the oracle internals
    feat = F._features(prm, c)
    v0 = np.einsum("of,bfzyx->bozyx", w["Wl"], feat)[0] + w["bl"][:, None, None, None]
    R = w["R0"][0] + 1j * w["R0"][1]
    want = _spectral_bruteforce(v0, R, c.P, c.m)
    # one-layer net output = Wq2 gelu(Wq1 z + bq1) + bq2 with z the spectral output
    z = want
    pre = np.einsum("hc,czyx->hzyx", w["Wq1"], z) + w["bq1"][:, None, None, None]
    from scipy.special import erf
    h = 0.5 * pre * (1 + erf(pre / np.sqrt(2)))
    expect = np.einsum("oh,hzyx->ozyx", w["Wq2"], h) + w["bq2"][:, None, None, None]
    got = F.forward(theta, prm, c)[0]
    assert np.max(np.abs(got - expect)) < 1e-12


def test_identity_spectral_weights_keep_kept_modes_and_drop_others():
    c = F.FnoConfig(0, 1, 1, 8, 2, 1, 1)
    P, m = c.P, c.m
    x = np.arange(P)
    kept = np.cos(2 * np.pi * (1 * x[None, None, :] + 1 * x[None, :, None] - 1 * x[:, None, None]) / P)
    dropped = np.cos(2 * np.pi * 3 * x / P)[None, None, :] * np.ones((P, P, 1))
    R = np.zeros((2, c.NT, c.NT, m, 1, 1))
    R[0] = 1.0
    for field, expect in ((kept, kept), (dropped, 0 * dropped)):
        V = np.fft.rfftn(field, axes=(0, 1, 2))
        S = np.concatenate([np.arange(m), np.arange(P - m, P)])
        full = np.zeros_like(V)
        full[S[:, None], S[None, :], :m] = V[S[:, None], S[None, :], :m] * (R[0, :, :, :, 0, 0] + 1j * R[1, :, :, :, 0, 0])
        out = np.fft.irfftn(full, s=(P, P, P), axes=(0, 1, 2))
        assert np.max(np.abs(out - expect)) < 1e-12
