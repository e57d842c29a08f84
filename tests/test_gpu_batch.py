"""Batched heterogeneous propagation (srp_propagate_batch) and the trace-shape
autotuner (srp_autotune), through the C ABI.

A batch mixes meshes, ray grids, bounce counts, joint laws, central bodies and
attitudes in one pipeline per integrator stage.  Each trajectory's result must
equal srp_propagate's for that trajectory alone, bit for bit (the same kernels
and per-slot sums; the batch only changes which slot a trajectory sits in),
including after the batch compacts its finished trajectories away.  The tile
shape changes no hit decision; forces change only by the rounding of the
32-ray FP32 tile sums (at most 31 x 2^-24 ~ 2e-6 relative).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MU_E = 3.986004418e14
MU_S = 1.32712440018e20
AU = 1.495978707e11


def geo(phase, inc=0.001):
    a = 42164e3
    v = math.sqrt(MU_E / a)
    c, s = math.cos(phase), math.sin(phase)
    return [a * c, a * s, 0.0, -v * s * math.cos(inc), v * c * math.cos(inc), v * math.sin(inc)]


def helio(r_au, phase):
    r = r_au * AU
    v = math.sqrt(MU_S / r)
    c, s = math.cos(phase), math.sin(phase)
    return [r * c, r * s, 0.0, -v * s, v * c, 0.0]


def mixed(ctx):
    from paper_2608_07307_gb300 import srp
    bw, sc5, sc25 = I.box_wing(), I.spacecraft(0.5), I.spacecraft(0.25)
    ids = {k: ctx.load_mesh(m) for k, m in (("bw", bw), ("sc5", sc5), ("sc25", sc25))}
    T = srp.PANELS_TRACK
    trajs = [
        dict(mesh_id=ids["bw"], N=64, bounces=1, panel_mode=T, central=0, attitude=0, y0=geo(0.1), t0=0.0,
             t1=3 * 3600.0),
        dict(mesh_id=ids["bw"], N=48, bounces=2, panel_mode=srp.PANELS_TRACK_OFFSET, angles=[0.0, 0.1, -0.2],
             central=0, attitude=0, q=(0.9, 0.1, 0.3, 0.2), y0=geo(1.3, 0.01), t0=0.0, t1=3600.0),
        dict(mesh_id=ids["sc5"], N=96, bounces=1, panel_mode=srp.PANELS_SET, angles=[0.0, 0.0, 0.5, -0.4],
             central=1, attitude=1, q=(0.7, -0.2, 0.5, 0.4), y0=helio(1.0, 0.3), t0=0.0, t1=2 * 86400.0),
        dict(mesh_id=ids["sc25"], N=128, bounces=0, panel_mode=T, central=0, attitude=0, y0=geo(2.2), t0=0.0,
             t1=6 * 3600.0),
        dict(mesh_id=ids["bw"], N=32, bounces=0, panel_mode=T, central=1, attitude=1, q=(1.0, 0.0, 0.0, 0.0),
             y0=helio(0.8, 1.0), t0=0.0, t1=5 * 86400.0),
        dict(mesh_id=ids["sc5"], N=64, bounces=2, panel_mode=T, central=0, attitude=0, y0=geo(4.0), t0=600.0,
             t1=2400.0),
    ]
    return trajs


def alone(ctx, t, kw):
    from paper_2608_07307_gb300 import srp
    mid = t["mesh_id"]
    if t.get("angles") is not None:
        ctx.set_panel_angles(mid, np.asarray(t["angles"]))
    y1, st, _ = ctx.propagate(mid, np.asarray(t["y0"]), [t["t0"], t["t1"]], central=t["central"],
                              attitude=t["attitude"], q=t.get("q", (1.0, 0.0, 0.0, 0.0)), N=t["N"],
                              bounces=t["bounces"], panel_mode=t["panel_mode"], **kw)
    if t.get("angles") is not None:
        ctx.set_panel_angles(mid, np.zeros(len(t["angles"])))
    return y1[0], st[0]


def test_batch_equals_each_trajectory_alone():
    from paper_2608_07307_gb300 import srp
    with srp.Context(0) as ctx:
        trajs = mixed(ctx)
        kw = dict(j2=True, sun3=True, rtol=1e-12, h0=60.0)
        y1, st = ctx.propagate_batch(trajs, **kw)
        for k, t in enumerate(trajs):
            ya, sa = alone(ctx, t, kw)
            assert sa["steps"] == st[k]["steps"] and sa["rejects"] == st[k]["rejects"], (k, sa, st[k])
            assert np.array_equal(ya, y1[k]), (k, ya, y1[k])
        assert all(s["status"] == 0 for s in st)


def test_batch_compacts_and_matches_rk4():
    """Many short and a few long arcs: most slots finish early and the batch
    compacts several times; RK4 fixed steps."""
    from paper_2608_07307_gb300 import srp
    with srp.Context(0) as ctx:
        bw = ctx.load_mesh(I.box_wing())
        trajs = [dict(mesh_id=bw, N=32 + 8 * (k % 3), bounces=k % 2, panel_mode=srp.PANELS_TRACK, central=0,
                      attitude=0, y0=geo(0.3 * k), t0=0.0, t1=(2 + (k * 7) % 13) * 60.0 * (10 if k % 5 == 0 else 1))
                 for k in range(12)]
        kw = dict(method=srp.RK4, j2=True, sun3=False, h0=60.0)
        y1, st = ctx.propagate_batch(trajs, **kw)
        for k, t in enumerate(trajs):
            ya, sa = alone(ctx, t, kw)
            assert np.array_equal(ya, y1[k]) and sa["steps"] == st[k]["steps"], k


def test_autotune_and_tile_shapes_keep_decisions():
    from paper_2608_07307_gb300 import srp
    with srp.Context(0) as ctx:
        m = I.spacecraft(0.25)
        mid = ctx.load_mesh(m)
        w, ms = ctx.autotune(mid, 128, 2)
        assert w in (4, 8, 16, 32) and all(x > 0 for x in ms)
        assert ms[(4, 8, 16, 32).index(w)] == min(ms)
        dirs = I.sun_dirs_fibonacci(8)
        ref = None
        for tw in (4, 8, 16, 32):
            ctx.set_tile_shape(mid, 100, 2, tw)
            F, T, H = ctx.eval_batch(mid, dirs, N=100, bounces=2, hits=True)
            if ref is None:
                ref = (F, T, H)
                continue
            assert np.array_equal(H, ref[2]), tw
            for k in range(len(dirs)):
                fn = np.linalg.norm(ref[0][k])
                assert np.linalg.norm(F[k] - ref[0][k]) <= 2e-6 * fn, (tw, k)
                assert np.linalg.norm(T[k] - ref[1][k]) <= 2e-6 * max(np.linalg.norm(ref[1][k]), fn), (tw, k)
        # and against the oracle for one direction, with the narrowest tiles
        ctx.set_tile_shape(mid, 100, 2, 4)
        F, T, H = ctx.eval_batch(mid, dirs[:1], N=100, bounces=2, hits=True)
        r = O.evaluate(m, dirs[0], 100, 2, want_hits=True, want_edge=True, procs=4)
        fn = np.linalg.norm(r["F"])
        assert np.linalg.norm(F[0] - r["F"]) <= 1e-4 * fn
        diff = np.nonzero((np.asarray(H[0]) != r["hits"]).any(axis=1))[0]
        assert len(diff) <= 1e-5 * 100 * 100 + 1
        for ray in diff:
            k = int(np.argmax(H[0][ray] != r["hits"][ray]))
            assert r["edge"][ray, k] < 1e-6 * r["win"][6]


def test_batch_with_autotune_and_errors():
    from paper_2608_07307_gb300 import srp
    with srp.Context(0) as ctx:
        trajs = mixed(ctx)[:4]
        kw = dict(j2=True, sun3=True, rtol=1e-12, h0=60.0)
        y_ref, _ = ctx.propagate_batch(trajs, **kw)
        y_tun, st = ctx.propagate_batch(trajs, autotune=True, **kw)
        assert np.max(np.abs(y_tun[:, :3] - y_ref[:, :3])) < 1e-3
        bad = dict(trajs[0], N=0)
        with pytest.raises(srp.SrpError) as e:
            ctx.propagate_batch([trajs[1], bad], **kw)
        assert e.value.code == -1
