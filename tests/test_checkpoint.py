"""Checkpoint / resume: the whole state of a run is the six fields and the time
t = steps * dt, read with get_field / time and restored with set_field /
set_time.  A run of n1 + n2 steps and a run of n1 steps, saved, restored into a
new context and continued for n2 steps give bit-identical fields and the same
focal plane (the window I_S depends on t)."""
import numpy as np
import pytest

from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [64, 32])
def test_resume_is_bit_identical_mapped_pulse(lib, prec):
    g, m, p, n_steps, plane = W.tight_focus_workload(N=32)
    dt = (m.R0 / g.c) / n_steps
    n1, n2 = 5, 7
    args = (plane["x_p"], 16, 12, plane["y0"], plane["y1"], plane["z0"], plane["z1"])
    with lib.Context(g, m, dt, prec) as a:
        a.init_pulse(p)
        a.advance(n1 + n2)
        want, t_want = a.get_field(-1), a.time
        s_want = a.sample_focal_plane(*args)
    with lib.Context(g, m, dt, prec) as b:
        b.init_pulse(p)
        b.advance(n1)
        saved, t_saved = b.get_field(-1), b.time
    with lib.Context(g, m, dt, prec) as c:
        c.set_fields(saved)
        c.set_time(t_saved)
        c.advance(n2)
        got, t_got = c.get_field(-1), c.time
        s_got = c.sample_focal_plane(*args)
    assert t_saved == pytest.approx(n1 * dt, rel=1e-15)
    assert t_got == t_want          # the same additions of dt in the same order
    assert np.array_equal(got, want)
    assert np.array_equal(s_got, s_want)


def test_resume_is_bit_identical_real_fields(lib):
    g = W.GridSpec(256, 256, 64, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    f0 = np.random.default_rng(11).standard_normal((6, 64, 256, 256)).astype(np.float32)
    dt = 0.29
    with lib.Context(g, None, dt, 32, real=True) as a:
        a.set_fields(f0)
        a.advance(4)
        want = a.get_field(-1)
    with lib.Context(g, None, dt, 32, real=True) as b:
        b.set_fields(f0)
        b.advance(1)
        saved = b.get_field(-1)
    with lib.Context(g, None, dt, 32, real=True) as c:
        c.set_fields(saved)
        c.advance(3)
        got = c.get_field(-1)
    assert got.dtype == np.float32
    assert np.array_equal(got, want)
