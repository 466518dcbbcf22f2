"""Method-level check of the mapping (Sec. 3.1, Fig. 4a): the focal field from
the periodic layer of period D against a direct computation on the full
domain x, y, z in [-20, 20) lambda, for the flat-top case f = 0.3, R0 = 16
lambda, L = 2 lambda, eps = 0.1 at 12 points per wavelength, one exact step to
t = R0/c.  The paper reports a peak-field error of at most 0.9 % near
D_min/L ~ 1.9 and below 0.1 % at D/L ~ 3.5; the bounds here allow a factor 2.
"""
import json
import math

import numpy as np
import pytest

from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LAM, R0, L, PPW, HALF = 1.0, 16.0, 2.0, 12, 20.0


def focal_region(lib, g, m, p, T):
    """Ex, Ey, Ez on three planes x = -0.3, 0, 0.3 over |y|, |z| < 0.6 lambda
    (inside R < 1 lambda, where the cut-out is 1 at t = R0/c)."""
    out = []
    with lib.Context(g, m, T, 32) as ctx:
        for xp in (-0.3, 0.0, 0.3):
            out.append(ctx.focal_one_shot(p, T, xp, 48, 48, -0.6, 0.6, -0.6, 0.6, comps=(0, 1, 2)))
    return np.stack(out)


def test_mapped_vs_direct_error_against_D(lib):
    theta = math.atan(1.0 / (2 * 0.3))
    p = W.PulseSpec(kind=W.FLAT_TOP, lam=LAM, theta=theta, eps=0.1, P0=1.0, div_project=0)
    m = W.MappingSpec(R0=R0, L=L)
    c = 1.0
    T = R0 / c
    N = int(2 * HALF * PPW)                                     # 480
    d = 2 * HALF / N
    direct = W.GridSpec(N, N, N, d, d, d, -HALF, -HALF, -HALF, c)
    ref = focal_region(lib, direct, m, p, T)
    peak = np.max(np.abs(ref))
    errs = {}
    for ratio in (1.875, 2.0, 2.5, 3.0, 3.75):
        D = ratio * L
        Nx = int(round(D * PPW / LAM))
        g = W.GridSpec(Nx, N, N, D / Nx, d, d, -(R0 - L / 2) - D, -HALF, -HALF, c)
        got = focal_region(lib, g, m, p, T)
        errs[ratio] = float(np.max(np.abs(got - ref)) / peak)
    print("relative peak-field error vs D/L:", json.dumps(errs))
    assert errs[1.875] <= 2 * 0.009
    assert errs[3.75] <= 2 * 0.001
    assert errs[3.75] < errs[2.0] < errs[1.875] * 1.5
