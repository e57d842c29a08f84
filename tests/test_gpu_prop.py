"""GPU parity of srp_propagate (device RKF7(8) / RK4 with the ray-traced SRP
force in every stage, graph-captured) against the oracle's propagation.

Bars: the 30-day propagated position within 10 m of the oracle.  When the GPU
replays the oracle's accepted steps, the only difference left is the SRP force,
which may differ by 1e-4 relative, so the position may differ by at most 1e-4 of
the displacement that SRP itself causes over the arc.  Free-running arcs also
differ by the two integrators' step choices (each within rtol)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MU = 3.986004418e14


def kepler_state(a, e, i, raan, argp, M, mu=MU):
    E = M
    for _ in range(50):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    nu = 2 * math.atan2(math.sqrt(1 + e) * math.sin(E / 2), math.sqrt(1 - e) * math.cos(E / 2))
    p = a * (1 - e * e)
    r = p / (1 + e * math.cos(nu))
    rp = np.array([r * math.cos(nu), r * math.sin(nu), 0.0])
    vp = np.array([-math.sin(nu), e + math.cos(nu), 0.0]) * math.sqrt(mu / p)
    cO, sO, ci, si, cw, sw = (math.cos(raan), math.sin(raan), math.cos(i), math.sin(i), math.cos(argp),
                              math.sin(argp))
    Q = np.array([[cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci, sO * si],
                  [sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci, -cO * si],
                  [sw * si, cw * si, ci]])
    return np.concatenate([Q @ rp, Q @ vp])


@pytest.fixture(scope="module")
def ctx():
    from paper_2608_07307_gb300 import srp
    c = srp.Context(0)
    yield c
    c.close()


GEO = kepler_state(42164e3, 0.001, math.radians(0.1), 0.0, 0.0, 0.0)


def test_two_body_and_j2_without_srp(ctx):
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    y0 = kepler_state(7000e3, 0.01, 0.9, 0.3, 0.2, 0.1)
    y1, st, _ = ctx.propagate(mid, y0, [0.0, 20000.0], j2=True, srp_on=False)
    yo, so, _ = O.propagate(None, O.prop_params(central=0, j2=True), 0.0, 20000.0, y0)
    assert st[0]["steps"] == so[0] and st[0]["rejects"] == so[1]
    assert np.linalg.norm(y1[0, :3] - yo[:3]) < 1e-4


def test_geo_with_srp_one_day(ctx):
    """Free-running: both integrators meet rtol 1e-12 with slightly different step
    sequences (the embedded error estimate sees the ~1e-7 relative FP32-sum
    differences of the SRP force); replaying the oracle's steps isolates the SRP
    force difference, which must leave the state essentially unchanged."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    kw = dict(j2=True, sun3=True, N=32, bounces=1)
    y1, st, hl = ctx.propagate(mid, GEO, [0.0, 86400.0], h_cap=512, **kw)
    pp = O.prop_params(central=0, j2=True, sun3=True, srp=True, mass=m.mass, N=32, bounces=1)
    yo, so, ho = O.propagate(m, pp, 0.0, 86400.0, GEO)
    assert abs(st[0]["steps"] - so[0]) <= 3 and st[0]["t"] == 86400.0
    assert np.linalg.norm(y1[0, :3] - yo[:3]) < 0.5
    yn, _, hn = O.propagate(None, O.prop_params(central=0, j2=True, sun3=True), 0.0, 86400.0, GEO)
    srp_effect = np.linalg.norm(yo[:3] - yn[:3])
    assert srp_effect > 1.0          # the SRP term is really there
    yr, sr, _ = ctx.propagate(mid, GEO, [0.0, 86400.0], h_replay=ho[None, :], **kw)
    assert sr[0]["steps"] == so[0] and abs(sr[0]["t"] - ho.sum()) < 1e-9
    assert np.linalg.norm(yr[0, :3] - yo[:3]) <= 1e-4 * srp_effect + 1e-6


def test_rk4_fixed_step_with_srp(ctx):
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    from paper_2608_07307_gb300 import srp
    y1, st, _ = ctx.propagate(mid, GEO, [0.0, 200 * 60.0], method=srp.RK4, h0=60.0, N=32, bounces=1)
    pp = O.prop_params(central=0, srp=True, mass=m.mass, N=32, bounces=1, method=1, h0=60.0)
    yo, so, _ = O.propagate(m, pp, 0.0, 200 * 60.0, GEO)
    assert st[0]["steps"] == so[0] == 200
    assert np.linalg.norm(y1[0, :3] - yo[:3]) < 1e-4


def test_heliocentric_inertial_attitude(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.spacecraft(0.5)
    mid = ctx.load_mesh(m)
    AU = 1.495978707e11
    y0 = kepler_state(0.557 * AU, 0.682, 0.0, 0.0, 0.0, 0.3, mu=1.32712440018e20)
    q = (math.cos(0.2), 0.0, 0.0, math.sin(0.2))
    T = 5 * 86400.0
    pp = O.prop_params(central=1, srp=True, mass=m.mass, N=48, bounces=2, attitude=1, q=q, h0=3600.0, rtol=1e-11,
                       atol_pos=1.0, atol_vel=1e-6)
    yo, so, ho = O.propagate(m, pp, 0.0, T, y0)
    y1, st, _ = ctx.propagate(mid, y0, [0.0, T], central=srp.CENTRAL_SUN, attitude=srp.ATT_INERTIAL, q=q,
                              N=48, bounces=2, h_replay=ho[None, :])
    assert st[0]["steps"] == so[0]
    yn, _, _ = O.propagate(None, O.prop_params(central=1, h0=3600.0, rtol=1e-11, atol_pos=1.0, atol_vel=1e-6), 0.0,
                           T, y0, h_replay=ho)
    srp_effect = np.linalg.norm(yo[:3] - yn[:3])
    assert srp_effect > 1e3
    assert np.linalg.norm(y1[0, :3] - yo[:3]) <= 1e-4 * srp_effect


def test_several_trajectories_of_uneven_length(ctx):
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    y0 = np.stack([GEO, kepler_state(42164e3, 0.01, 0.05, 1.0, 0.5, 2.0), kepler_state(30000e3, 0.2, 0.3, 0, 0, 1)])
    t01 = np.array([[0.0, 40000.0], [0.0, 10000.0], [1000.0, 30000.0]])
    y1, st, _ = ctx.propagate(mid, y0, t01, j2=True, sun3=True, N=24, bounces=1)
    pp = O.prop_params(central=0, j2=True, sun3=True, srp=True, mass=m.mass, N=24, bounces=1)
    for k in range(3):
        yo, so, _ = O.propagate(m, pp, t01[k, 0], t01[k, 1], y0[k])
        assert abs(st[k]["steps"] - so[0]) <= 3 and st[k]["t"] == t01[k, 1]
        assert np.linalg.norm(y1[k, :3] - yo[:3]) < 0.5


def test_thirty_day_geo_within_ten_metres(ctx):
    """Box-wing in GEO, tracking panels, two-body + J2 + Sun + SRP (128 x 128 rays,
    1 bounce), RKF7(8) rtol 1e-12 over 30 days: GPU vs oracle."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    T = 30 * 86400.0
    y1, st, _ = ctx.propagate(mid, GEO, [0.0, T], j2=True, sun3=True, N=128, bounces=1)
    pp = O.prop_params(central=0, j2=True, sun3=True, srp=True, mass=m.mass, N=128, bounces=1)
    yo, so, _ = O.propagate(m, pp, 0.0, T, GEO)
    assert np.linalg.norm(y1[0, :3] - yo[:3]) < 10.0
    assert abs(st[0]["steps"] - so[0]) <= 0.05 * so[0]


def test_host_loop_matches_graph_bitwise(ctx):
    """The host-driven mode issues the same kernels in the same order."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    a, sa, _ = ctx.propagate(mid, GEO, [0.0, 20000.0], j2=True, sun3=True, N=32, bounces=1)
    b, sb, _ = ctx.propagate(mid, GEO, [0.0, 20000.0], j2=True, sun3=True, N=32, bounces=1, host_loop=True)
    assert np.array_equal(a, b) and sa[0]["steps"] == sb[0]["steps"]


def test_propagate_argument_errors(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    with pytest.raises(srp.SrpError) as e:
        ctx.propagate(mid, GEO, [0.0, 100.0], h0=0.0)
    assert e.value.code == -1
    with pytest.raises(srp.SrpError) as e:
        ctx.propagate(mid, GEO, [0.0, 1e6], max_steps=3, srp_on=False)
    assert e.value.code == -7


def test_resume_a_fixed_step_arc_exactly(ctx):
    """Checkpoint / resume: an RK4 arc split at a step boundary, the second half
    started from the first half's state, equals the whole arc bit for bit."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    kw = dict(method=1, h0=60.0, j2=True, sun3=True, N=32, bounces=1)
    y_all, s_all, _ = ctx.propagate(mid, GEO, [0.0, 7200.0], **kw)
    y_a, s_a, _ = ctx.propagate(mid, GEO, [0.0, 3600.0], **kw)
    y_b, s_b, _ = ctx.propagate(mid, y_a[0], [3600.0, 7200.0], **kw)
    assert s_a[0]["steps"] + s_b[0]["steps"] == s_all[0]["steps"] == 120
    assert np.array_equal(y_b, y_all)


def test_resume_an_adaptive_arc_with_the_proposed_step(ctx):
    """RKF7(8): split at the end of an accepted step of the whole arc and resume
    with h0 = the first half's h_next: the same steps, the same end state
    (up to the rounding of the shortened last step of the first half)."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    kw = dict(j2=True, sun3=True, N=32, bounces=1)
    y_all, s_all, hl = ctx.propagate(mid, GEO, [0.0, 43200.0], h_cap=256, **kw)
    t_m = 0.0
    for h in hl[0, :12]:
        t_m += h
    y_a, s_a, _ = ctx.propagate(mid, GEO, [0.0, t_m], **kw)
    assert s_a[0]["steps"] == 12 and s_a[0]["t"] == t_m
    assert abs(s_a[0]["h_next"] / hl[0, 12] - 1.0) < 1e-6 or s_a[0]["h_next"] >= hl[0, 12]
    y_b, s_b, _ = ctx.propagate(mid, y_a[0], [t_m, 43200.0], h0=s_a[0]["h_next"], **kw)
    assert s_a[0]["steps"] + s_b[0]["steps"] == s_all[0]["steps"]
    assert np.linalg.norm(y_b[0, :3] - y_all[0, :3]) < 1e-4
