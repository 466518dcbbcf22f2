"""Pins of the surrogate-network oracle against independent definitions."""
import math

import numpy as np
import pytest

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


def _ramp_filter_net(axis):
    """One-channel net whose trunk output is the low-pass filtered coordinate
    ramp along `axis` (0 = z, 2 = x): lift = that coordinate, spectral weights
    = identity on every kept mode, W = 0, b = 0, projection gelu(z)."""
    c = F.FnoConfig(0, 1, 1, 8, 2, 1, 1)
    theta = np.zeros(F.num_params(c))
    w = F.unpack(theta, c)
    w["Wl"][0, {2: 0, 1: 1, 0: 2}[axis]] = 1.0          # features are (x, y, z)
    w["R0"][0][...] = 1.0
    w["Wq1"][...] = 1.0
    w["Wq2"][...] = 1.0
    return c, theta


def _ramp_partial_sum(P, kept):
    """Re (1/P) sum_{k in kept} R_k e^{2 pi i k n / P} for the ramp
    r_n = -1 + 2 n / P, with its DFT in closed form: R_0 = -1 and, for k != 0,
    R_k = (2/P) sum_n n w^n = 2 / (w - 1), w = e^{-2 pi i k / P}."""
    n = np.arange(P)
    out = np.zeros(P, dtype=complex)
    for k in kept:
        Rk = -1.0 if k % P == 0 else 2.0 / (np.exp(-2j * np.pi * k / P) - 1.0)
        out += Rk * np.exp(2j * np.pi * k * n / P)
    return out.real / P


@pytest.mark.parametrize("axis", [2, 0])
def test_identity_spectral_weights_low_pass_the_lifted_ramp(axis):
    """The spectral layer with identity weights keeps exactly the corner modes:
    kx in 0..m-1 (counted with its mirror, the last axis is the real-FFT axis)
    and kz, ky in {0..m-1} U {P-m..P-1}."""
    c, theta = _ramp_filter_net(axis)
    P, m = c.P, c.m
    if axis == 2:
        kept = [0] + [s * k for k in range(1, m) for s in (1, -1)]
    else:
        kept = list(range(m)) + list(range(-m, 0))
    f = _ramp_partial_sum(P, kept)
    gelu = np.vectorize(lambda t: 0.5 * t * (1.0 + math.erf(t / math.sqrt(2.0))))
    expect = gelu(f)
    out = F.forward(theta, np.zeros((1, 0)), c)[0, 0]
    got = out[0, 0, :] if axis == 2 else out[:, 0, 0]
    assert np.max(np.abs(got - expect)) < 1e-13
    other = out - (got[None, None, :] if axis == 2 else got[:, None, None])
    assert np.max(np.abs(other)) < 1e-13                 # constant along the other axes


# ------------------------------------------------------------- loss and gradients
def _constant_net(B, NO, value):
    """All weights zero except b_q2: the output is `value` at every point."""
    c = F.FnoConfig(1, 2, 1, 2, 1, 2, NO)
    theta = np.zeros(F.num_params(c))
    F.unpack(theta, c)["bq2"][...] = value
    return c, theta, np.zeros((B, 1))


def _loss_pin_holds():
    # outputs 0.5 everywhere on a 2 x 1 x 2^3 array; target differences are
    # 0 except -1, +1, -2 in batch 0 and +3 in batch 1: sum of squares 15 over 16
    c, theta, prm = _constant_net(2, 1, 0.5)
    t = np.full((2, 1, 2, 2, 2), 0.5)
    t[0, 0, 0, 0, 1] = 1.5
    t[0, 0, 0, 1, 0] = -0.5
    t[0, 0, 1, 1, 0] = 2.5
    t[1, 0, 1, 0, 1] = -2.5
    return abs(F.loss(theta, prm, t, c) - 15.0 / 16.0) < 1e-15


def test_loss_is_the_mean_of_squared_differences():
    assert _loss_pin_holds()


def _linear_param_case():
    """A random net; the output is affine in W_q2 and b_q2, so the loss is a
    quadratic in them with the closed-form gradient
    dL/db_q2[o] = 2/N sum d[:, o],  dL/dW_q2[o, k] = 2/N sum d[:, o] h[:, k],
    N = number of outputs, d = output - target, h = hidden activations."""
    c = F.FnoConfig(2, 3, 2, 4, 1, 3, 2)
    rng = np.random.default_rng(11)
    theta = rng.standard_normal(F.num_params(c)) * 0.4
    prm = rng.standard_normal((2, 2))
    target = rng.standard_normal((2, c.NO, c.P, c.P, c.P))
    w = F.unpack(theta, c)
    d = F.forward(theta, prm, c) - target
    N = d.size
    # the hidden activations, read through the same network with W_q2 = unit row, b_q2 = 0
    h = np.empty((2, c.H) + d.shape[2:])
    for k in range(c.H):
        th = theta.copy()
        wk = F.unpack(th, c)
        wk["Wq2"][...] = 0.0
        wk["Wq2"][0, k] = 1.0
        wk["bq2"][...] = 0.0
        h[:, k] = F.forward(th, prm, c)[:, 0]
    g_b = 2.0 / N * d.sum(axis=(0, 2, 3, 4))
    g_W = 2.0 / N * np.einsum("bozyx,bkzyx->ok", d, h)
    off_W = int(w["Wq2"].ctypes.data - theta.ctypes.data) // 8
    off_b = int(w["bq2"].ctypes.data - theta.ctypes.data) // 8
    idx = [off_b + o for o in range(c.NO)] + [off_W + o * c.H + k for o in range(c.NO) for k in range(c.H)]
    exact = np.concatenate([g_b, g_W.ravel()])
    return c, theta, prm, target, idx, exact


def _fd_pin_holds(fd):
    c, theta, prm, target, idx, exact = _linear_param_case()
    got = fd(theta, prm, target, c, idx)
    return np.max(np.abs(got - exact)) <= 1e-8 * np.max(np.abs(exact))


def test_finite_differences_exact_on_a_quadratic():
    """Central differences are exact (up to rounding) for a quadratic."""
    assert _fd_pin_holds(F.finite_difference_grad)


def test_loss_and_gradient_pins_catch_planted_mistakes(monkeypatch):
    good_loss = F.loss

    def loss_sum(theta, prm, target, c):                 # sum instead of mean
        d = F.forward(theta, prm, c) - target
        return float(np.sum(d * d))

    def loss_abs(theta, prm, target, c):                 # mean |d|
        return float(np.mean(np.abs(F.forward(theta, prm, c) - target)))

    def loss_batch_mean(theta, prm, target, c):         # mean over the batch only
        d = F.forward(theta, prm, c) - target
        return float(np.sum(d * d) / d.shape[0])

    for bad in (loss_sum, loss_abs, loss_batch_mean):
        monkeypatch.setattr(F, "loss", bad)
        assert not _loss_pin_holds(), bad.__name__
    monkeypatch.setattr(F, "loss", good_loss)

    def fd_one_sided(theta, prm, target, c, idx, h=1e-5):
        theta = np.array(theta, dtype=np.float64, copy=True)
        l0 = F.loss(theta, prm, target, c)
        g = np.empty(len(idx))
        for n, i in enumerate(idx):
            t0 = theta[i]
            theta[i] = t0 + h
            g[n] = (F.loss(theta, prm, target, c) - l0) / h
            theta[i] = t0
        return g

    def fd_no_half(theta, prm, target, c, idx, h=1e-5):  # divides by h, not 2h
        return 2.0 * F.finite_difference_grad(theta, prm, target, c, idx, h)

    for bad in (fd_one_sided, fd_no_half):
        assert not _fd_pin_holds(bad), bad.__name__
