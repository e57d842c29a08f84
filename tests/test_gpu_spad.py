"""GPU parity of the SPAD interpolation model (Sec. 4.2, Sec. 6.1) against the
oracle: the table built by the evaluation pipeline, the interpolant at
arbitrary directions, and propagation with the interpolated force.

Bars: table entries within 1e-4 of the largest entry (the evaluation bar);
the interpolant (FP64 on both sides, the same definition) within 1e-12 of
the table's scale; a propagated GEO day within 1 mm of the oracle's with the
same step count."""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MU = 3.986004418e14


@pytest.fixture(scope="module")
def ctx():
    from paper_2608_07307_gb300 import srp
    c = srp.Context(0)
    yield c
    c.close()


def _geo():
    a, inc = 42164e3, math.radians(0.1)
    v = math.sqrt(MU / a)
    return np.array([a, 0.0, 0.0, 0.0, v * math.cos(inc), v * math.sin(inc)])


def _rand_dirs(n, seed):
    q = np.random.default_rng(seed).normal(size=(n, 3))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


@pytest.mark.parametrize("grid", [I.SPAD_20x10, I.SPAD_20x10S], ids=["20x10", "20x10S"])
def test_table_matches_the_oracle(ctx, grid):
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    tab = ctx.spad_build(mid, grid, N=64, bounces=1)
    ref = O.spad_table(m, grid, N=64, bounces=1)
    assert tab.shape == (10, 20, 6)
    fs = np.abs(ref[..., :3]).max()
    ts = np.abs(ref[..., 3:]).max()
    assert np.abs(tab[..., :3] - ref[..., :3]).max() <= 1e-4 * fs
    assert np.abs(tab[..., 3:] - ref[..., 3:]).max() <= 1e-4 * ts + 1e-4 * fs
    # the device-table form equals the host one
    tab_d = ctx.spad_build(mid, grid, N=64, bounces=1, device=True)
    assert np.array_equal(tab_d.cpu().numpy(), tab)


def test_table_of_a_larger_mesh_against_the_oracle(ctx):
    """The 12k-triangle spacecraft, two bounces, a coarse grid (oracle cost)."""
    m = I.spacecraft(0.1)
    mid = ctx.load_mesh(m)
    g = I.spad_grid(5, 3, -170.0, -60.0, 55.0)
    tab = ctx.spad_build(mid, g, N=96, bounces=2)
    ref = O.spad_table(m, g, N=96, bounces=2, procs=8)
    fs = np.abs(ref[..., :3]).max()
    assert np.abs(tab[..., :3] - ref[..., :3]).max() <= 1e-4 * fs


@pytest.mark.parametrize("grid", [I.SPAD_20x10, I.SPAD_20x10S, I.spad_grid(7, 5, 13.0, -70.0, 31.0),
                                  I.spad_grid(1, 1, 0.0, 0.0, 1.0)], ids=["20x10", "20x10S", "odd", "single"])
def test_interpolant_matches_the_oracle(ctx, grid):
    rng = np.random.default_rng(1)
    tab = rng.normal(size=(grid["n_el"], grid["n_az"], 6))
    dirs = np.concatenate([_rand_dirs(3000, 2), O.spad_dirs(grid).reshape(-1, 3),
                           [[0, 0, 1.0], [0, 0, -1.0], [-1.0, 0, 0], [-1.0, -1e-300, 0], [1e-3, 0, 1]]])
    dist = rng.uniform(0.3, 2.0, size=len(dirs))
    dist[::17] = -1.0
    F, T = ctx.spad_eval(grid, tab, dirs, dist)
    ref = np.array([O.spad_interp(grid, tab, s, d) for s, d in zip(dirs, dist)])
    scale = np.abs(tab).max() / 0.3 ** 2
    assert np.abs(F - ref[:, :3]).max() <= 1e-12 * scale
    assert np.abs(T - ref[:, 3:]).max() <= 1e-12 * scale
    assert np.all(F[::17] == 0.0) and np.all(T[::17] == 0.0)
    # without distances: 1 AU
    F1, _ = ctx.spad_eval(grid, tab, dirs[:50])
    ref1 = np.array([O.spad_interp(grid, tab, s, 1.0)[:3] for s in dirs[:50]])
    assert np.abs(F1 - ref1).max() <= 1e-12 * np.abs(tab).max()


def test_interpolant_device_tensors(ctx):
    import torch
    g = I.SPAD_20x10S
    tab = np.random.default_rng(3).normal(size=(10, 20, 6))
    dirs = _rand_dirs(1000, 4)
    dist = np.random.default_rng(5).uniform(0.5, 1.5, size=1000)
    F, T = ctx.spad_eval(g, tab, dirs, dist)
    Fd, Td = ctx.spad_eval(g, torch.tensor(tab, device="cuda"), torch.tensor(dirs, device="cuda"),
                           torch.tensor(dist, device="cuda"))
    assert Fd.is_cuda and np.array_equal(Fd.cpu().numpy(), F) and np.array_equal(Td.cpu().numpy(), T)


def test_bad_grids_are_rejected(ctx):
    from paper_2608_07307_gb300 import srp
    tab = np.zeros((10, 20, 6))
    for bad in (dict(I.SPAD_20x10, n_az=0), dict(I.SPAD_20x10, n_el=0), dict(I.SPAD_20x10, d_el=0.0),
                dict(I.SPAD_20x10, d_el=-0.1), dict(I.SPAD_20x10, az0=float("nan")),
                dict(I.SPAD_20x10, n_az=1 << 21), dict(I.SPAD_20x10, n_az=1 << 13, n_el=1 << 12)):
        with pytest.raises(srp.SrpError) as e:
            ctx.spad_eval(bad, tab, [[1.0, 0, 0]])
        assert e.value.code == srp.SRP_ERR_ARG


def test_propagation_matches_the_oracle(ctx):
    """GEO day, RKF7(8) rtol 1e-12, J2 + Sun + SPAD force from the oracle's table."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    g = I.SPAD_20x10S
    tab = O.spad_table(m, g, N=32, bounces=1)
    y0 = _geo()
    y1, st, _ = ctx.propagate(mid, y0, [0.0, 86400.0], j2=True, sun3=True, spad=(g, tab))
    pp = O.prop_params(central=0, j2=True, sun3=True, srp=True, mass=m.mass, spad=(g, tab))
    yo, so, _ = O.propagate(None, pp, 0.0, 86400.0, y0)
    assert st[0]["steps"] == so[0] and st[0]["rejects"] == so[1] and st[0]["t"] == 86400.0
    assert np.linalg.norm(y1[0, :3] - yo[:3]) < 1e-3
    yn, _, _ = O.propagate(None, O.prop_params(central=0, j2=True, sun3=True), 0.0, 86400.0, y0)
    assert np.linalg.norm(yo[:3] - yn[:3]) > 1.0  # the interpolated SRP term is really there
    # the host-driven loop takes the same steps
    yh, sh, _ = ctx.propagate(mid, y0, [0.0, 86400.0], j2=True, sun3=True, spad=(g, tab), host_loop=True)
    assert sh[0]["steps"] == st[0]["steps"] and np.array_equal(yh, y1)


def test_propagation_zero_table_is_srp_off(ctx):
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    y0 = _geo()
    y_off, s_off, _ = ctx.propagate(mid, y0, [0.0, 6 * 3600.0], j2=True, sun3=True, srp_on=False)
    y_z, s_z, _ = ctx.propagate(mid, y0, [0.0, 6 * 3600.0], j2=True, sun3=True,
                                spad=(I.SPAD_20x10, np.zeros((10, 20, 6))))
    assert np.array_equal(y_off, y_z) and s_off[0]["steps"] == s_z[0]["steps"]


def test_denser_tables_track_the_direct_propagation_closer(ctx):
    """The paper's RQ1 comparison in miniature (Sec. 7): GEO day with
    tracking panels, direct ray tracing against SPAD tables of three
    densities built from the same evaluations; the position gap to the
    direct arc shrinks as the grid refines and stays a small part of the
    displacement SRP causes."""
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    y0 = _geo()
    kw = dict(j2=True, sun3=True, N=128, bounces=1)
    yd, _, _ = ctx.propagate(mid, y0, [0.0, 86400.0], **kw)
    yn, _, _ = ctx.propagate(mid, y0, [0.0, 86400.0], j2=True, sun3=True, srp_on=False)
    effect = np.linalg.norm(yd[0, :3] - yn[0, :3])
    gaps = []
    for g in (I.SPAD_20x10S, I.spad_grid(40, 20, -175.0, -85.0), I.spad_grid(160, 80, -175.0, -85.0)):
        tab = ctx.spad_build(mid, g, N=128, bounces=1)
        ys, _, _ = ctx.propagate(mid, y0, [0.0, 86400.0], j2=True, sun3=True, spad=(g, tab))
        gaps.append(np.linalg.norm(ys[0, :3] - yd[0, :3]))
    assert effect > 1.0
    assert gaps[2] < gaps[1] < gaps[0] < 0.2 * effect, (gaps, effect)


def test_batch_and_adjoint_reject_a_table(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    tab = np.zeros((10, 20, 6))
    p = srp.PropParams()
    p.method, p.h0, p.max_steps, p.rtol, p.atol_pos, p.atol_vel = srp.RKF78, 60.0, 1000, 1e-12, 1e-6, 1e-9
    p.spad_table = tab.ctypes.data
    p.spad_grid = srp.spad_grid_struct(I.SPAD_20x10)
    tr = (srp.Traj * 1)()
    tr[0].mesh_id = mid
    y1 = np.zeros(6)
    rc = ctx.lib.srp_propagate_batch(ctx.h, C.byref(p), 1, tr, y1.ctypes.data, None)
    assert rc == srp.SRP_ERR_ARG
    p.method = srp.RK4
    y0, t01, g1 = _geo(), np.array([0.0, 600.0]), np.zeros(6)
    rc = ctx.lib.srp_prop_grad(ctx.h, mid, C.byref(p), 1, y0.ctypes.data, t01.ctypes.data, g1.ctypes.data, 100,
                               None, None, None, None, None, None)
    assert rc == srp.SRP_ERR_ARG
