"""Structural checks of the library's building blocks and its error paths on
the GPU (nothing here faults, traps or waits):

  * the BVH build's radix sort against numpy's stable sort;
  * the 4-wide trees as evaluations use them: every triangle in exactly one
    leaf, every child box inside its parent's, every posed triangle inside its
    leaf box, at rest and after the panels turned (refit);
  * a traversal bound that runs out reports SRP_ERR_STACK and the context
    stays usable;
  * an allocation beyond the memory cap reports SRP_ERR_OOM and the context
    stays usable.
"""
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


@pytest.mark.parametrize("n,bits", [(1000, 64), (70001, 56), (300000, 17), (5, 8)])
def test_radix_sort_is_numpys_stable_sort(ctx, n, bits):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2**63, size=n, dtype=np.uint64) | (rng.integers(0, 2, size=n, dtype=np.uint64) << np.uint64(63))
    keys[::7] = keys[3]  # ties: input order must survive
    vals = np.arange(n, dtype=np.int32)
    k, v = ctx.sort_pairs(keys, vals, bits)
    used = (bits + 7) // 8 * 8  # whole bytes, as documented
    mask = np.uint64((1 << used) - 1) if used < 64 else np.uint64(2**64 - 1)
    order = np.argsort(keys & mask, kind="stable")
    assert np.array_equal(v, vals[order]) and np.array_equal(k, keys[order])


@pytest.mark.parametrize("mesh", ["box_wing", "box_wing_two_axis", "spacecraft_0.1", "spacecraft_0.05"])
def test_trees_at_rest_and_after_the_panels_turn(ctx, mesh):
    m = I.spacecraft(float(mesh.split("_")[1])) if mesh.startswith("spacecraft") else getattr(I, mesh)()
    mid = ctx.load_mesh(m)
    for s in [None] + list(I.sun_dirs_uniform(4, seed=8)):
        r = ctx.mesh_check(mid, s)
        assert r["n_tris"] == m.n_tris and r["n_parts"] == len(m.parent)
        assert r["leaf_refs"] == m.n_tris and r["tris_not_once"] == 0, r
        assert r["boxes_outside_parent"] == 0 and r["tris_outside_leaf"] == 0 and r["walk_bound"] == 0, r
        assert r["nodes"] > 0


def test_walk_bound_reports_and_the_context_recovers(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.spacecraft(0.1)
    mid = ctx.load_mesh(m)
    d = I.sun_dirs_uniform(3, seed=1)
    F0, _ = ctx.eval_batch(mid, d, N=64, bounces=1)
    with pytest.raises(srp.SrpError) as e:
        ctx.eval_batch(mid, d, N=64, bounces=1, flags=srp.EVAL_TEST_WALK_BOUND)
    assert e.value.code == srp.SRP_ERR_STACK
    F1, _ = ctx.eval_batch(mid, d, N=64, bounces=1)
    assert np.array_equal(F0, F1)


def test_memory_cap_reports_oom_and_the_context_recovers(ctx):
    from paper_2608_07307_gb300 import srp
    m = I.box_wing()
    mid = ctx.load_mesh(m)
    d = I.sun_dirs_uniform(2, seed=2)
    F0, _ = ctx.eval_batch(mid, d, N=64, bounces=1)
    used, cap = ctx.memory_usage()
    assert used > 0 and cap == 0
    try:
        ctx.set_memory_limit(used + 1024)
        with pytest.raises(srp.SrpError) as e:
            ctx.eval_batch(mid, d, N=2048, bounces=2)  # needs far more than 1 KiB of new buffers
        assert e.value.code == srp.SRP_ERR_OOM
        assert ctx.memory_usage()[0] <= used + 1024
    finally:
        ctx.set_memory_limit(0)
    F1, _ = ctx.eval_batch(mid, d, N=64, bounces=1)
    assert np.array_equal(F0, F1)
    F2, _ = ctx.eval_batch(mid, d, N=2048, bounces=2)
    assert np.all(np.isfinite(F2))
