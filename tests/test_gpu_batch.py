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
        # Another tile shape moves the forces by the rounding of the FP32 tile
        # sums, which can flip an accept/reject decision of the adaptive step;
        # a different step sequence moves the result by up to the local error
        # the integrator admits per step (rtol |r|).
        for k in range(len(trajs)):
            bound = 4.0 * st[k]["steps"] * kw["rtol"] * np.linalg.norm(y_ref[k, :3])
            assert np.linalg.norm(y_tun[k, :3] - y_ref[k, :3]) <= bound, (k, bound)
        bad = dict(trajs[0], N=0)
        with pytest.raises(srp.SrpError) as e:
            ctx.propagate_batch([trajs[1], bad], **kw)
        assert e.value.code == -1


def _oracle_traj(args):
    """The oracle's arc with SRP, its step count and accepted steps, and the
    length of the displacement SRP causes (the same arc without SRP)."""
    mesh, pp_kw, t0, t1, y0 = args
    y1, st, hlog = O.propagate(mesh, O.prop_params(srp=True, **pp_kw), t0, t1, y0)
    yn, _, _ = O.propagate(None, O.prop_params(srp=False, **pp_kw), t0, t1, y0)
    return y1, int(st[0]), hlog, float(np.linalg.norm(y1[:3] - yn[:3]))


def test_batch_against_the_oracle():
    """srp_propagate_batch on eight heterogeneous trajectories against the
    oracle's own propagation of each (RKF7(8), rtol 1e-12, two-body + J2 + Sun
    + SRP around the Earth, Sun + SRP around the Sun): box-wing, two-axis
    box-wing and a 583-triangle spacecraft; N 32-64; 0-2 bounces; tracking,
    tracking with offsets and commanded joints; LVLH and inertial attitudes.

    Two checks per trajectory.  (1) Replay: the same trajectory through
    srp_propagate (whose result the batch equals bit for bit, see the test
    above) on the oracle's accepted steps must land within 1e-6 of the SRP
    displacement plus 1 mm of the oracle: this isolates the force evaluation
    and the integrator arithmetic.  (2) Free running: the batch's own adaptive
    steps must be within 5% (at least 2) of the oracle's count and its final
    position within the largest of the 30-day 10 m bar scaled to the arc,
    4 / N^2 of the SRP displacement, 4 x steps x rtol |r| and 1 cm.  The
    force of an N x N grid jumps by about one pixel's share whenever a pixel
    changes its hit as the Sun moves in the body frame, so two integrators
    whose steps fall at different times (one accept/reject decision is enough)
    sample those jumps differently; the integrator's error estimate does not
    see them."""
    import multiprocessing as mp
    import os
    from paper_2608_07307_gb300 import srp
    bw, bw2, sc = I.box_wing(), I.box_wing_two_axis(), I.spacecraft(0.5)
    bw.mass = bw2.mass = sc.mass = 40.0  # light craft: SRP moves these arcs by hundreds of metres or more
    meshes = dict(bw=bw, bw2=bw2, sc=sc)
    T, S, O_ = srp.PANELS_TRACK, srp.PANELS_SET, srp.PANELS_TRACK_OFFSET
    day = 86400.0
    spec = [
        ("bw", 32, 1, T, None, 0, 0, (1.0, 0, 0, 0), geo(0.1), 0.0, 0.5 * day),
        ("bw", 48, 2, S, [0.0, 0.4, -0.3], 0, 0, (0.9, 0.1, 0.3, 0.2), geo(1.3, 0.01), 0.0, 0.4 * day),
        ("bw", 64, 0, O_, [0.0, 0.1, -0.2], 1, 1, (0.8, -0.3, 0.4, 0.33), helio(1.0, 0.3), 0.0, 3 * day),
        ("sc", 32, 1, T, None, 0, 0, (1.0, 0, 0, 0), geo(2.2), 600.0, 0.3 * day),
        ("sc", 48, 2, S, [0.0, 0.0, 0.5, -0.4], 1, 1, (0.7, -0.2, 0.5, 0.4), helio(0.8, 1.0), 0.0, 2 * day),
        ("bw2", 48, 1, T, None, 0, 0, (1.0, 0, 0, 0), geo(4.0, 0.02), 0.0, 0.5 * day),
        ("sc", 64, 0, O_, [0.0, 0.05, 0.0, 0.1], 0, 0, (0.96, 0.1, -0.2, 0.15), geo(5.1), 0.0, 0.25 * day),
        ("bw2", 32, 2, S, [0.0, 0.3, 0.6, -0.5, 0.2], 1, 1, (1.0, 0, 0, 0), helio(1.15, 2.0), 0.0, 4 * day),
    ]
    common = dict(j2=True, sun3=True, rtol=1e-12, h0=60.0)
    jobs = []
    for mk, N, B, mode, ang, central, att, q, y0, t0, t1 in spec:
        pp_kw = dict(central=central, j2=central == 0, sun3=central == 0, attitude=att, q=q,
                     mass=meshes[mk].mass, N=N, bounces=B, rtol=1e-12, h0=60.0)
        if mode == S:
            pp_kw["angles"] = ang
        elif mode == O_:
            pp_kw["offsets"] = ang
        jobs.append((meshes[mk], pp_kw, t0, t1, np.asarray(y0)))
    # the oracle first (spawn-started processes), then the GPU
    procs = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        ref = pool.map(_oracle_traj, jobs)
    with srp.Context(0) as ctx:
        ids = {k: ctx.load_mesh(m) for k, m in meshes.items()}
        trajs = [dict(mesh_id=ids[mk], N=N, bounces=B, panel_mode=mode, angles=ang, central=central, attitude=att,
                      q=q, y0=y0, t0=t0, t1=t1)
                 for mk, N, B, mode, ang, central, att, q, y0, t0, t1 in spec]
        y1, st = ctx.propagate_batch(trajs, **common)
        for k, ((yo, so, ho, d_srp), t) in enumerate(zip(ref, trajs)):
            # (1) the oracle's steps replayed
            if t["angles"] is not None:
                ctx.set_panel_angles(t["mesh_id"], np.asarray(t["angles"]))
            yr, sr, _ = ctx.propagate(t["mesh_id"], np.asarray(t["y0"]), [t["t0"], t["t1"]], central=t["central"],
                                      attitude=t["attitude"], q=t["q"], N=t["N"], bounces=t["bounces"],
                                      panel_mode=t["panel_mode"], h_replay=ho[None, :], **common)
            if t["angles"] is not None:
                ctx.set_panel_angles(t["mesh_id"], np.zeros(len(t["angles"])))
            err_r = np.linalg.norm(yr[0, :3] - yo[:3])
            assert sr[0]["steps"] == so and err_r <= 1e-6 * d_srp + 1e-3, (k, err_r, d_srp)
            # (2) free running
            N = t["N"]
            arc = t["t1"] - t["t0"]
            bar = max(10.0 * arc / (30 * day), 4.0 * d_srp / N ** 2, 4.0 * so * 1e-12 * np.linalg.norm(yo[:3]), 1e-2)
            assert d_srp > 10.0 * bar, (k, d_srp, bar)   # SRP matters well beyond the bar
            assert st[k]["status"] == 0
            err = np.linalg.norm(y1[k, :3] - yo[:3])
            assert err <= bar, (k, err, bar)
            assert abs(st[k]["steps"] - so) <= max(2, 0.05 * so), (k, st[k]["steps"], so)
