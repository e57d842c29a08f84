"""srp_eval_noalloc, the entry point that allocates nothing, against srp_eval_batch.

Some callers cannot allocate device memory while they run: flight or real-time
software with a memory budget fixed at start-up (an allocation could fail or
stall in mid-mission), hosts that hand out memory only from their own pool.  They use
srp_eval_noalloc, whose only scratch is a fixed device array inside the
library.  These checks call it through the C ABI and compare its force and
torque with srp_eval_batch on the same rigid mesh, within the 1e-4 relative
tolerance the other parity tests use, on two calls in a row (the shared scratch
must carry nothing from one call into the next).  This file is collected last
so that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2608_07307_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P0 = 4.56e-6
TOL = 1e-4


def rigid(mesh):
    mesh.axis = np.zeros_like(mesh.axis)   # no joints: the rest pose is the posed mesh
    return mesh


def close(F, T, Fr, Tr):
    fn = np.linalg.norm(Fr)
    assert np.linalg.norm(F - Fr) <= TOL * fn, (F, Fr)
    assert np.linalg.norm(T - Tr) <= TOL * max(np.linalg.norm(Tr), fn), (T, Tr)


@pytest.mark.parametrize("mesh_fn, N, bounces", [(I.box_wing, 256, 1), (lambda: I.spacecraft(0.5), 128, 2)])
def test_noalloc_matches_eval_batch_twice(mesh_fn, N, bounces):
    import torch
    from paper_2608_07307_gb300 import srp

    m = rigid(mesh_fn())
    m.c_ref = np.array([0.1, -0.2, 0.3])
    dirs = I.sun_dirs_uniform(2, seed=7)
    with srp.Context(0) as ctx:
        mid = ctx.load_mesh(m)
        Fb, Tb = ctx.eval_batch(mid, dirs, N=N, bounces=bounces, P0=P0)
    xyz = torch.tensor(np.asarray(m.xyz, np.float64)[m.tri].reshape(-1, 9), device="cuda")
    tmat = torch.tensor(m.tri_mat, dtype=torch.int32, device="cuda")
    mat = torch.tensor(m.mat, dtype=torch.float64, device="cuda")
    for k in range(2):
        F = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        T = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        srp.eval_noalloc(xyz, tmat, mat, dirs[k], 1.0, m.c_ref, N, bounces, P0, 1e-9, F, T)
        torch.cuda.synchronize()
        close(F.cpu().numpy(), T.cpu().numpy(), Fb[k], Tb[k])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2608_07307_gb300 import srp

    m = rigid(I.box_wing())
    xyz = torch.tensor(m.xyz[m.tri].reshape(-1, 9), device="cuda")
    tmat = torch.tensor(m.tri_mat, dtype=torch.int32, device="cuda")
    mat = torch.tensor(m.mat, dtype=torch.float64, device="cuda")
    F = torch.zeros(3, dtype=torch.float64, device="cuda")
    T = torch.zeros_like(F)
    with pytest.raises(srp.SrpError) as e:
        srp.eval_noalloc(xyz, tmat, mat, (0, 0, 1.0), 1.0, (0, 0, 0), 2048, 1, P0, 1e-9, F, T)
    assert e.value.code == -1


def test_noalloc_out_of_range_material_gives_nan():
    """A material index outside [0, n_mats) is never used to read the table:
    the result comes out NaN instead; the next valid call is clean again."""
    import torch
    from paper_2608_07307_gb300 import srp

    m = rigid(I.box_wing())
    xyz = torch.tensor(m.xyz[m.tri].reshape(-1, 9), device="cuda")
    mat = torch.tensor(m.mat, dtype=torch.float64, device="cuda")
    good = torch.tensor(m.tri_mat, dtype=torch.int32, device="cuda")
    bad = good.clone()
    bad[:, :] = len(m.mat) + 5        # every side out of range
    bad2 = good.clone()
    bad2[:, :] = -1
    F = torch.zeros(3, dtype=torch.float64, device="cuda")
    T = torch.zeros_like(F)
    for b in (bad, bad2):
        srp.eval_noalloc(xyz, b, mat, (0.3, 0.2, 0.9), 1.0, (0, 0, 0), 64, 1, P0, 1e-9, F, T)
        torch.cuda.synchronize()
        assert torch.isnan(F).all() and torch.isnan(T).all()
    srp.eval_noalloc(xyz, good, mat, (0.3, 0.2, 0.9), 1.0, (0, 0, 0), 64, 1, P0, 1e-9, F, T)
    torch.cuda.synchronize()
    assert torch.isfinite(F).all() and torch.isfinite(T).all() and F.abs().max() > 0


def test_noalloc_binding_rejects_bad_tensors():
    """The binding checks dtype, shape, contiguity and device before the call."""
    import torch
    from paper_2608_07307_gb300 import srp

    m = rigid(I.box_wing())
    xyz = torch.tensor(m.xyz[m.tri].reshape(-1, 9), device="cuda")
    tmat = torch.tensor(m.tri_mat, dtype=torch.int32, device="cuda")
    mat = torch.tensor(m.mat, dtype=torch.float64, device="cuda")
    F = torch.zeros(3, dtype=torch.float64, device="cuda")
    T = torch.zeros_like(F)
    cases = [
        (xyz.float(), tmat, mat, F),                                  # FP32 vertices
        (xyz, tmat.long(), mat, F),                                   # int64 materials
        (xyz.reshape(-1, 3, 3), tmat, mat, F),                        # [n, 3, 3]
        (xyz.t().contiguous().t(), tmat, mat, F),                     # not contiguous
        (xyz.cpu(), tmat, mat, F),                                    # host memory
        (xyz, tmat, mat, torch.zeros(4, dtype=torch.float64, device="cuda")),
    ]
    for x, tm, mt, f in cases:
        with pytest.raises(srp.SrpError) as e:
            srp.eval_noalloc(x, tm, mt, (0, 0, 1.0), 1.0, (0, 0, 0), 64, 1, P0, 1e-9, f, T)
        assert e.value.code == srp.SRP_ERR_ARG
