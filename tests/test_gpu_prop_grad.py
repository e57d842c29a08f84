"""GPU propagation adjoint (srp_prop_grad, through the C ABI) against the
oracle's central differences of the frozen-hit RK4 arc.

Bar, per entry (tests/_gradbar.py): |g - r| <= 1e-3 |r| + 1e-5 max|r| of the
entry's group (initial state, coefficients, joint parameters, attitude
quaternion).
The oracle's parameter step is h = 1e-3: L = lam . y1 carries the rounding of
a ~4e7 m state through hundreds of steps (~1e-8 absolute), which h = 1e-6
would turn into 1e-2 errors in gradients of order 1; F_H is smooth, so the
truncation error at h = 1e-3 is ~h^2 relative.  The
two sides propagate and record hit sets independently (FP32 + FP64 hand-off
on the GPU, FP64 brute force in the oracle); stage states agree to far below
a pixel, so the recorded hit sets agree except on rays at an edge.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

from _gradbar import check_group

pytestmark = pytest.mark.gpu

MU_E = 3.986004418e14
MU_S = 1.32712440018e20
AU = 1.495978707e11


@pytest.fixture(scope="module")
def ctx():
    from paper_2608_07307_gb300 import srp
    c = srp.Context(0)
    yield c
    c.close()


def geo_state(phase=0.3, inc=0.02):
    a = 42164e3
    v = math.sqrt(MU_E / a)
    c, s = math.cos(phase), math.sin(phase)
    return np.array([a * c, a * s, 0.0, -v * s * math.cos(inc), v * c * math.cos(inc), v * math.sin(inc)])


def compare(ctx, m, y0, t1, lam, off, ckpt, pp_kw, gpu_kw, h=1e-3):
    from paper_2608_07307_gb300 import srp
    mid = ctx.load_mesh(m)
    ctx.set_panel_angles(mid, off)
    g = ctx.prop_grad(mid, y0[None], [[0.0, t1]], lam[None], ckpt_every=ckpt, panel_mode=srp.PANELS_TRACK_OFFSET,
                      **gpu_kw)
    pp = O.prop_params(method=1, mass=m.mass, **pp_kw)
    r = O.arc_frozen_grad(m, pp, 0.0, t1, y0, lam, offsets=off, h=h)
    assert np.max(np.abs(g["y1"][0, :3] - r["y1"][:3])) < 1e-2, (g["y1"][0], r["y1"])
    check_group("y0", g["y0"][0], r["y0"])
    check_group("mat", g["mat"], r["mat"])
    check_group("angle", g["angle"], r["angle"])
    check_group("q", g["q"], r["q"])
    return g, r


def test_geo_lvlh_quaternion_j2_sun(ctx):
    m = I.box_wing().with_materials([[0.3, 0.2], [0.25, 0.15], [0.4, 0.1]])
    m.mass = 20.0
    q = (0.96, 0.1, -0.2, 0.15)
    lam = np.array([1.0, -0.5, 0.3, 400.0, 200.0, -100.0])
    common = dict(j2=True, sun3=True, N=32, bounces=1, h0=60.0, q=q)
    compare(ctx, m, geo_state(), 200 * 60.0, lam, np.array([0.0, 0.05, -0.03]), 50,
            dict(srp=True, attitude=0, **common), dict(srp_on=True, attitude=0, **common))


def test_heliocentric_inertial_two_bounces(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.box_wing().with_materials([[0.3, 0.2], [0.25, 0.15], [0.4, 0.1]])
    m.mass = 5.0
    v = math.sqrt(MU_S / AU)
    y0 = np.array([AU, 0.0, 0.0, 0.0, v * 0.8, v * 0.6])
    q = (0.8, -0.3, 0.4, 0.33)
    lam = np.array([0.2, 1.0, -0.4, 1e4, -2e4, 5e3])
    common = dict(N=32, bounces=2, h0=3600.0, q=q, central=1, attitude=1)
    compare(ctx, m, y0, 40 * 3600.0, lam, np.array([0.0, -0.1, 0.08]), 16, dict(srp=True, **common),
            dict(srp_on=True, **common))


def test_spacecraft_small_tracking(ctx):
    m = I.spacecraft(0.25)
    m.mass = 8.0
    lam = np.array([0.0, 1.0, 0.0, 0.0, 300.0, 0.0])
    common = dict(j2=True, sun3=False, N=48, bounces=1, h0=60.0)
    compare(ctx, m, geo_state(1.1), 60 * 60.0, lam, np.zeros(4), 25,
            dict(srp=True, attitude=0, **common), dict(srp_on=True, attitude=0, **common))


def test_without_srp_only_the_state_gradient_is_left(ctx):
    m = I.box_wing()
    lam = np.array([1.0, 2.0, -1.0, 10.0, 0.0, 5.0])
    common = dict(j2=True, sun3=True, N=16, bounces=0, h0=120.0)
    g, r = compare(ctx, m, geo_state(2.0), 100 * 120.0, lam, np.zeros(3), 30,
                   dict(srp=False, **common), dict(srp_on=False, **common))
    assert np.all(g["mat"] == 0) and np.all(g["angle"] == 0) and np.all(g["q"] == 0)


def test_checkpoint_interval_does_not_change_the_result(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.box_wing()
    m.mass = 20.0
    mid = ctx.load_mesh(m)
    y0 = np.stack([geo_state(0.1), geo_state(0.7, 0.05)])
    lam = np.array([[1.0, 0, 0, 0, 0, 0], [0, 1.0, 0, 0, 0, 100.0]])
    kw = dict(j2=True, sun3=True, N=24, bounces=1, h0=60.0, q=(0.9, 0.0, 0.3, 0.1),
              panel_mode=srp.PANELS_TRACK_OFFSET)
    ctx.set_panel_angles(mid, np.array([0.0, 0.02, 0.04]))
    outs = [ctx.prop_grad(mid, y0, [[0.0, 37 * 60.0]] * 2, lam, ckpt_every=c, **kw) for c in (1, 7, 100)]
    for o in outs[1:]:
        for k in ("y1", "y0", "mat", "angle", "q"):
            assert np.array_equal(o[k], outs[0][k]), k
    # the final state equals srp_propagate's RK4 arc
    y1, st, _ = ctx.propagate(mid, y0, [[0.0, 37 * 60.0]] * 2, method=srp.RK4, j2=True, sun3=True, N=24, bounces=1,
                              h0=60.0, q=(0.9, 0.0, 0.3, 0.1), panel_mode=srp.PANELS_TRACK_OFFSET)
    assert np.array_equal(y1, outs[0]["y1"])
    with pytest.raises(srp.SrpError):
        ctx.prop_grad(mid, y0, [[0.0, 37 * 60.0], [0.0, 38 * 60.0]], lam, **kw)
