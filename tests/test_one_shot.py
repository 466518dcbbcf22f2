"""One-shot focal field (one exact step of T, sampled from the spectrum)
against the oracle's exact step, plus its state rules."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ogrid(g):
    return O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def opulse(p):
    return O.Pulse(p.kind, p.lam, p.theta, p.eps, p.P0, p.n_cycles, p.cep, p.ellipticity, p.pol_angle,
                   p.div_project)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("N,project", [(64, 1), (64, 0), (48, 1)])
@pytest.mark.parametrize("path", ["auto", "generic"])
def test_one_shot_matches_oracle(lib, prec, N, project, path):
    g, m, p, n_steps, plane = W.tight_focus_workload(N=N)
    p.div_project = project
    T = m.R0 / g.c
    ys, zs = W.plane_points(plane)
    with lib.Context(g, m, T / n_steps, prec) as ctx:
        if path == "generic":
            ctx.set_kernel_path(lib.PATH_GENERIC)
        got = ctx.focal_one_shot(p, T, plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"],
                                 plane["z0"], plane["z1"], comps=(0, 1, 2))
        assert abs(ctx.time - T) == 0.0
        with pytest.raises(lib.PsatdError):
            ctx.advance(1)                         # storage holds the spectrum now
        again = ctx.sample_focal_plane(plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"],
                                       plane["z0"], plane["z1"], comps=(0, 1, 2))
        assert np.array_equal(again, got)          # sampled from the held spectrum
        ctx.init_pulse(p)
        ctx.advance(0)
    og, om = ogrid(g), O.Mapping(m.R0, m.L)
    f0 = O.init_fields(og, om, opulse(p))
    ref = O.sample_plane(O.advance_exact(f0, og, T), og, om, plane["x_p"], ys, zs, T, comps=(0, 1, 2))
    assert np.max(np.abs(ref)) > 0
    assert rel(got, ref) <= (1e-12 if prec == 64 else 1e-5)


@pytest.mark.parametrize("prec", [64, 32])
def test_one_shot_equals_many_steps(lib, prec):
    """Semigroup at the API level: one step of T and n steps of T/n give the
    same focal plane (Sec. 2.1)."""
    g, m, p, n_steps, plane = W.tight_focus_workload(N=64)
    T = m.R0 / g.c
    args = (plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
    with lib.Context(g, m, T / n_steps, prec) as ctx:
        one = ctx.focal_one_shot(p, T, *args)
        ctx.init_pulse(p)
        ctx.advance(n_steps)
        many = ctx.sample_focal_plane(*args)
    assert rel(one, many) <= (1e-11 if prec == 64 else 2e-5)
