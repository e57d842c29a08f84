"""The work-queue schedule (SRP_EVAL_QUEUE): the raster's second pass and the
trace of a chunk as one persistent launch whose trace items wait, with a
bound, for their slot's second pass.

The queue changes the order in which work runs, not what is computed: force,
torque and hit ids must equal the separate-launch schedule's bit for bit, for
single meshes, for a grid whose list of large-triangle chunks overflows, and
for a heterogeneous batch of trajectories.  The bounded wait's error path is
tested by making every wait target a count that is never reached (a flag that
nothing sets): the call returns SRP_ERR_TIMEOUT after the bound and the
context stays usable."""
import math

import numpy as np
import pytest

from paper_2608_07307_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2608_07307_gb300 import srp
    c = srp.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("mesh_fn, N, B, n", [(I.box_wing, 128, 2, 12), (lambda: I.spacecraft(0.25), 256, 2, 40),
                                              (lambda: I.spacecraft(0.05), 1024, 2, 16),
                                              (I.box_wing_two_axis, 96, 1, 9)])
def test_queue_equals_separate_launches(ctx, mesh_fn, N, B, n):
    from paper_2608_07307_gb300 import srp
    m = mesh_fn()
    mid = ctx.load_mesh(m)
    dirs = I.sun_dirs_fibonacci(4096)[::4096 // n][:n]
    F0, T0, H0 = ctx.eval_batch(mid, dirs, N=N, bounces=B, hits=True)
    F1, T1, H1 = ctx.eval_batch(mid, dirs, N=N, bounces=B, hits=True, flags=srp.EVAL_QUEUE)
    assert np.array_equal(F0, F1) and np.array_equal(T0, T1)
    assert np.array_equal(np.asarray(H0), np.asarray(H1))
    F2, T2 = ctx.eval_batch(mid, dirs, N=N, bounces=B, flags=srp.EVAL_QUEUE)
    assert np.array_equal(F0, F2) and np.array_equal(T0, T2)
    ctx.free_mesh(mid)


def test_queue_with_a_full_chunk_list(ctx):
    """At the largest grid the flat plate's four triangles list more chunks
    than the list holds: the slot's pixels traverse, both schedules agree and
    match the closed form."""
    from paper_2608_07307_gb300 import srp
    mat = ((0.3, 0.2), (0.1, 0.4))
    m = I.flat_plate(2.0, 1.0, mat=mat)
    mid = ctx.load_mesh(m)
    th = 0.7
    s = np.array([[math.sin(th), 0, math.cos(th)]])
    F0, T0 = ctx.eval_batch(mid, s, N=srp.MAX_N, bounces=0)
    F1, T1 = ctx.eval_batch(mid, s, N=srp.MAX_N, bounces=0, flags=srp.EVAL_QUEUE)
    assert np.array_equal(F0, F1) and np.array_equal(T0, T1)
    c = math.cos(th)
    Fcf = -4.56e-6 * 2.0 * c * ((1 - 0.3) * s[0] + 2 * (0.3 * c + 0.2 / 3) * np.array([0, 0, 1.0]))
    assert np.linalg.norm(F1[0] - Fcf) < 1e-6 * np.linalg.norm(Fcf)
    ctx.free_mesh(mid)


def test_queue_in_the_batched_propagation(ctx):
    from paper_2608_07307_gb300 import srp
    from test_gpu_batch import mixed
    trajs = mixed(ctx)
    kw = dict(j2=True, sun3=True, rtol=1e-12, h0=60.0)
    y0, s0 = ctx.propagate_batch(trajs, **kw)
    y1, s1 = ctx.propagate_batch(trajs, flags=srp.EVAL_QUEUE, **kw)
    assert np.array_equal(y0, y1)
    assert [x["steps"] for x in s0] == [x["steps"] for x in s1]


def test_wait_that_runs_out_reports_timeout(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.spacecraft(0.25)
    mid = ctx.load_mesh(m)
    dirs = I.sun_dirs_fibonacci(8)
    F0, T0 = ctx.eval_batch(mid, dirs, N=128, bounces=1)
    with pytest.raises(srp.SrpError) as e:
        ctx.eval_batch(mid, dirs, N=128, bounces=1, flags=srp.EVAL_TEST_WAIT_TIMEOUT)
    assert e.value.code == srp.SRP_ERR_TIMEOUT
    # the context is usable afterwards, with and without the queue
    F1, T1 = ctx.eval_batch(mid, dirs, N=128, bounces=1, flags=srp.EVAL_QUEUE)
    F2, T2 = ctx.eval_batch(mid, dirs, N=128, bounces=1)
    assert np.array_equal(F0, F1) and np.array_equal(F0, F2) and np.array_equal(T0, T2)
    ctx.free_mesh(mid)
