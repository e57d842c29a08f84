"""Rasterised primary visibility against BVH traversal of every primary ray.

All primary rays of an evaluation are parallel, so the default path projects
each triangle into the window and applies the traversal's own FP32 test to the
pixel centres it covers.  Hits must be identical to the traversal's (both are
exact: certain FP32 decisions, the rest settled in FP64), forces equal up to
the FP32 rounding of the hit points (the traversal can settle a pixel in FP64
that the raster settles in FP32 when the two meet different candidates): 2e-6
relative.  Covers small triangles (spacecraft), window-sized ones (box-wing,
chunked), a one-part scene reflecting onto itself, a fan whose hub pixel has
too many candidates (that pixel traverses), and a stack of window-sized plates
whose list of large triangles overflows (every pixel of the evaluation
traverses)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2608_07307_gb300 import srp
    c = srp.Context(0)
    yield c
    c.close()


def _fan(k=16):
    ang = np.arange(k) * 2 * math.pi / k
    verts = np.concatenate([[[0.0, 0.0, 0.0]], np.stack([np.cos(ang), np.sin(ang), np.zeros(k)], 1)])
    tri = np.array([[0, 1 + i, 1 + (i + 1) % k] for i in range(k)], np.int32)
    return I.Mesh(verts, tri, np.zeros(k, np.int32), np.zeros((k, 2), np.int32), np.array([[0.3, 0.2]]),
                  **I._parts(1, [-1]), name="fan")


def _stack(n=600):
    b = I._Builder()
    for k in range(n):
        v = np.array([[-1.0, -1.0, 0.01 * k], [1.0, -1.0, 0.01 * k], [1.0, 1.0, 0.01 * k], [-1.0, 1.0, 0.01 * k]])
        b.add(v, np.array([[0, 1, 2], [0, 2, 3]]), 0, 0, 0)
    return I._single_part(b, ((0.5, 0.1),), "stack")


def _plane():
    from test_gpu_parity import _plane_scene
    return _plane_scene()


CASES = {
    "spacecraft": (lambda: I.spacecraft(0.1), I.sun_dirs_fibonacci(6), 192, 2),
    "box_wing": (I.box_wing, I.sun_dirs_uniform(6, seed=3), 160, 1),
    "plane": (_plane, np.array([[-0.6, 0.1, 0.8], [-0.8, 0.3, 0.5]]), 128, 2),
    "fan": (_fan, np.array([[0.0, 0.0, 1.0]]), 63, 1),
    "stack": (_stack, np.array([[0.1, 0.2, 1.0]]), 256, 1),
}


@pytest.mark.parametrize("name", list(CASES))
def test_raster_equals_traversal(ctx, name):
    make, dirs, N, B = CASES[name]
    m = make()
    dirs = np.asarray(dirs, np.float64)
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    mid = ctx.load_mesh(m)
    F1, T1, H1 = ctx.eval_batch(mid, dirs, N=N, bounces=B, hits=True)
    F2, T2, H2 = ctx.eval_batch(mid, dirs, N=N, bounces=B, hits=True, traverse=True)
    assert np.array_equal(H1, H2), name
    for k in range(len(dirs)):
        fn = np.linalg.norm(F2[k])
        assert np.linalg.norm(F1[k] - F2[k]) <= 2e-6 * fn, (name, k)
        assert np.linalg.norm(T1[k] - T2[k]) <= 2e-6 * max(np.linalg.norm(T2[k]), fn), (name, k)
    # the raster really replaced the primary traversal (or, for the stack, fell back to it)
    ctx.eval_batch(mid, dirs[:1], N=N, bounces=0, count=True)
    rast = ctx.eval_stats()["nodes_visited"] / (N * N)
    ctx.eval_batch(mid, dirs[:1], N=N, bounces=0, count=True, traverse=True)
    trav = ctx.eval_stats()["nodes_visited"] / (N * N)
    if name == "stack":
        assert rast == trav > 0
    elif name == "fan":
        assert 0 < rast < trav
    else:
        assert rast < 0.05 * trav, (rast, trav)
    ctx.free_mesh(mid)


def test_raster_against_oracle_spacecraft(ctx):
    m = I.spacecraft(0.1)
    mid = ctx.load_mesh(m)
    s = I.sun_dirs_fibonacci(6)[4]
    N = 150
    F, T, H = ctx.eval_batch(mid, s[None], N=N, bounces=1, hits=True)
    r = O.evaluate(m, s, N, 1, want_hits=True, want_edge=True, procs=4)
    fn = np.linalg.norm(r["F"])
    assert np.linalg.norm(F[0] - r["F"]) <= 1e-4 * fn
    diff = np.nonzero((np.asarray(H[0]) != r["hits"]).any(axis=1))[0]
    assert len(diff) <= 1e-5 * N * N + 1
    for ray in diff:
        k = int(np.argmax(H[0][ray] != r["hits"][ray]))
        assert r["edge"][ray, k] < 1e-6 * r["win"][6]


@pytest.mark.parametrize("name", ["spacecraft", "fan", "stack"])
def test_launch_shapes_give_the_same_evaluation(ctx, name):
    """A launch of fewer than four evaluations clears the pixel keys in the frame
    kernel, runs the second raster pass as one launch and poses one vertex a
    thread; larger launches use a clear kernel, two second-pass launches and
    four vertices a thread.  Each evaluation's hits, force and torque are the
    same bits either way (every decision and every sum is per slot, in a fixed
    order)."""
    make, dirs, N, B = CASES[name]
    m = make()
    dirs = np.asarray(dirs, np.float64)
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    many = np.concatenate([dirs] * (8 // len(dirs) + 1))[:8]
    mid = ctx.load_mesh(m)
    Fm, Tm, Hm = ctx.eval_batch(mid, many, N=N, bounces=B, hits=True)
    for k in range(len(dirs)):
        F1, T1, H1 = ctx.eval_batch(mid, many[k:k + 1], N=N, bounces=B, hits=True)
        assert np.array_equal(H1[0], Hm[k]), (name, k)
        assert np.array_equal(F1[0], Fm[k]) and np.array_equal(T1[0], Tm[k]), (name, k)
    ctx.free_mesh(mid)
