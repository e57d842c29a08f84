"""GPU parity of the diffuse secondary rays (Sec. 6.1; srp_eval_params
n_diffuse) against the oracle, which draws the same SplitMix64 samples.

The diffuse part is computed in FP64 on both sides from the same sample
stream, so the increment it adds to force and torque must agree far below the
evaluation bar: within 1e-6 of the increment itself (unless a primary or
specular segment met an edge differently, which these scenes avoid), and the
totals within the evaluation bar of 1e-4."""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P0 = 4.56e-6


@pytest.fixture(scope="module")
def ctx():
    from paper_2608_07307_gb300 import srp
    c = srp.Context(0)
    yield c
    c.close()


def _both(ctx, mid, m, dirs, N, B, K, seed, procs=1):
    Fg0, Tg0 = ctx.eval_batch(mid, dirs, N=N, bounces=B)
    Fg, Tg = ctx.eval_batch(mid, dirs, N=N, bounces=B, n_diffuse=K, diffuse_seed=seed)
    out = []
    for k, s in enumerate(dirs):
        a = O.evaluate(m, s, N, B, P0=P0, procs=procs)
        b = O.evaluate(m, s, N, B, P0=P0, n_diffuse=K, diffuse_seed=seed, procs=procs)
        out.append((Fg[k], Tg[k], Fg[k] - Fg0[k], Tg[k] - Tg0[k], b["F"], b["T"], b["F"] - a["F"], b["T"] - a["T"]))
    return out


def _check(rows, rel=1e-6):
    for k, (Fg, Tg, dFg, dTg, Fo, To, dFo, dTo) in enumerate(rows):
        fn = np.linalg.norm(Fo)
        assert np.linalg.norm(Fg - Fo) <= 1e-4 * fn, k
        assert np.linalg.norm(Tg - To) <= 1e-4 * max(np.linalg.norm(To), fn), k
        dn = np.linalg.norm(dFo)
        assert np.linalg.norm(dFg - dFo) <= rel * dn + 1e-12 * fn, (k, dFg, dFo)
        assert np.linalg.norm(dTg - dTo) <= rel * max(np.linalg.norm(dTo), dn) + 1e-12 * fn, (k, dTg, dTo)


def test_box_wing_two_levels_16_rays(ctx):
    """The paper's setting (two levels, 16 diffuse rays) on the box-wing."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    dirs = I.sun_dirs_uniform(8, seed=11)
    rows = _both(ctx, mid, m, dirs, 64, 2, 16, 3)
    _check(rows)
    assert sum(np.linalg.norm(r[6]) > 0 for r in rows) >= 4  # the diffuse light does reach other parts


def test_two_plate_transfer(ctx):
    """A Lambertian floor lighting an absorbing wall: nearly all of the diffuse
    increment is the floor's light on the wall."""
    floor = I.flat_plate(1.0, 1.0, center=(0.5, 0.5), mat=((0.0, 1.0), (0.0, 1.0)))
    w = I.flat_plate(1.0, 1.0, center=(0.5, 0.5), mat=((0.0, 0.0), (0.0, 0.0)))
    xyz = np.asarray(w.xyz, np.float64).copy()
    w.xyz = np.stack([1.2 - xyz[:, 2], xyz[:, 1], xyz[:, 0]], axis=1)
    m = I.merge([floor, w])
    mid = ctx.load_mesh(m)
    th = math.radians(30.0)
    dirs = np.array([[-math.sin(th), 0.0, math.cos(th)], [-0.5, 0.3, 0.81]])
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rows = _both(ctx, mid, m, dirs, 80, 1, 32, 17)
    _check(rows)
    assert rows[0][6][0] > 0.02 * np.linalg.norm(rows[0][4])


def test_spacecraft_with_the_bvh(ctx):
    """The 12k-triangle spacecraft: diffuse rays through the 4-wide BVH."""
    m = I.spacecraft(0.1)
    mid = ctx.load_mesh(m)
    dirs = I.sun_dirs_fibonacci(4096)[[700, 2900]]
    rows = _both(ctx, mid, m, dirs, 64, 1, 8, 5, procs=8)
    _check(rows)


def test_zero_rays_or_no_level_change_nothing(ctx):
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    dirs = I.sun_dirs_uniform(4, seed=2)
    F0, T0 = ctx.eval_batch(mid, dirs, N=48, bounces=2)
    F1, T1 = ctx.eval_batch(mid, dirs, N=48, bounces=2, n_diffuse=0, diffuse_seed=99)
    assert np.array_equal(F0, F1) and np.array_equal(T0, T1)
    G0, _ = ctx.eval_batch(mid, dirs, N=48, bounces=0)
    G1, _ = ctx.eval_batch(mid, dirs, N=48, bounces=0, n_diffuse=16)
    assert np.array_equal(G0, G1)
    # deterministic
    H1, _ = ctx.eval_batch(mid, dirs, N=48, bounces=2, n_diffuse=16, diffuse_seed=4)
    H2, _ = ctx.eval_batch(mid, dirs, N=48, bounces=2, n_diffuse=16, diffuse_seed=4)
    assert np.array_equal(H1, H2)


def test_arguments_and_unsupported_forms(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    d = I.sun_dirs_uniform(2, seed=1)
    for bad in (-1, 257):
        with pytest.raises(srp.SrpError) as e:
            ctx.eval_batch(mid, d, N=16, bounces=1, n_diffuse=bad)
        assert e.value.code == srp.SRP_ERR_ARG
    p = srp.PropParams()
    p.method, p.h0, p.max_steps, p.rtol, p.atol_pos, p.atol_vel = srp.RKF78, 60.0, 1000, 1e-12, 1e-6, 1e-9
    p.eval = srp.EvalParams(16, 1, P0, 1e-9, 0, 0, 4, 0)
    tr = (srp.Traj * 1)()
    tr[0].mesh_id = mid
    y1 = np.zeros(6)
    assert ctx.lib.srp_propagate_batch(ctx.h, C.byref(p), 1, tr, y1.ctypes.data, None) == srp.SRP_ERR_ARG


def test_propagation_with_diffuse_rays(ctx):
    """A GEO hour with diffuse rays runs, and moves the state by a tiny amount
    against the same arc without them."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    a, inc = 42164e3, math.radians(0.1)
    v = math.sqrt(3.986004418e14 / a)
    y0 = np.array([a, 0.0, 0.0, 0.0, v * math.cos(inc), v * math.sin(inc)])
    kw = dict(j2=True, sun3=True, N=48, bounces=2)
    y0a, s0, _ = ctx.propagate(mid, y0, [0.0, 3600.0], **kw)
    y1a, s1, _ = ctx.propagate(mid, y0, [0.0, 3600.0], n_diffuse=8, **kw)
    assert s0[0]["status"] == 0 and s1[0]["status"] == 0
    dy = np.linalg.norm(y1a[0, :3] - y0a[0, :3])
    assert 0.0 < dy < 1.0


def test_sum_modes_with_diffuse_rays(ctx):
    """The precision report's FP32 sums above the tile take the diffuse blocks'
    sums too: with compensated FP32 the evaluation stays within 1e-6 of the FP64
    sums, with plain FP32 (a few hundred tile values per evaluation) within 1e-4."""
    from paper_2608_07307_gb300 import srp
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    dirs = I.sun_dirs_uniform(4, seed=5)
    kw = dict(N=128, bounces=2, n_diffuse=16, diffuse_seed=3)
    F64, T64 = ctx.eval_batch(mid, dirs, **kw)
    for flag, bar in ((srp.EVAL_SUM_COMP32, 1e-6), (srp.EVAL_SUM_FP32, 1e-4)):
        F, T = ctx.eval_batch(mid, dirs, flags=flag, **kw)
        for k in range(len(dirs)):
            fn = np.linalg.norm(F64[k])
            assert np.linalg.norm(F[k] - F64[k]) <= bar * fn, (flag, k)
            assert np.linalg.norm(T[k] - T64[k]) <= bar * max(np.linalg.norm(T64[k]), fn), (flag, k)
    ctx.free_mesh(mid)
