"""Python binding of libsrp (include/srp.h): argument marshalling only.

Every computation happens in the CUDA kernels behind the C ABI.  Arrays may be
numpy arrays (host memory) or torch tensors (CUDA tensors are passed as device
pointers, on the context's stream).  There is no fallback: if libsrp.so cannot
be loaded, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SRP_OK = 0
ERRORS = {-1: "SRP_ERR_ARG", -2: "SRP_ERR_OOM", -3: "SRP_ERR_CUDA", -4: "SRP_ERR_MESH", -5: "SRP_ERR_STACK",
          -6: "SRP_ERR_TIMEOUT", -7: "SRP_ERR_STEP", -8: "SRP_ERR_STATE"}
globals().update({name: code for code, name in ERRORS.items()})
SRP_F32, SRP_F64 = 0, 1
PANELS_TRACK, PANELS_SET, PANELS_TRACK_OFFSET = 0, 1, 2
EVAL_COUNT = 1
EVAL_TIMING = 2
EVAL_TRAVERSE = 8  # primary hits by BVH traversal instead of rasterisation (same results)
EVAL_TEST_WALK_BOUND = 16  # tests of the walk bound's error path: every BVH walk stops after one step
EVAL_AUTOTUNE = 4
EVAL_SERIAL = 32  # one pipeline lane: with timing, each phase's time is its own kernels' GPU time
EVAL_QUEUE = 64  # second raster pass and trace as one persistent launch over a work queue
EVAL_TEST_WAIT_TIMEOUT = 128  # tests of the work queue's bounded wait (SRP_ERR_TIMEOUT)
EVAL_SUM_COMP32 = 256  # sums above the tile in compensated FP32 instead of FP64 (precision report)
EVAL_SUM_FP32 = 512  # sums above the tile in plain FP32 (precision report)
MAX_BOUNCES = 4
MAX_N = 8192  # SRP_MAX_N: rays per window side
MAX_DIFFUSE = 256  # diffuse secondary rays per hit (srp_eval_params.n_diffuse)

# Symbols declared in include/srp.h (checked by the tests against the library).
EXPORTS = ["srp_create", "srp_destroy", "srp_last_error", "srp_mesh_load", "srp_mesh_free", "srp_set_panel_angles",
           "srp_eval_batch", "srp_eval_stats_get", "srp_propagate", "srp_eval_noalloc", "srp_set_materials",
           "srp_grad", "srp_prop_grad", "srp_propagate_batch", "srp_autotune", "srp_set_tile_shape",
           "srp_spad_build", "srp_spad_eval", "srp_set_memory_limit", "srp_memory_usage", "srp_sort_pairs",
           "srp_mesh_check"]


class Traj(C.Structure):
    """One trajectory of srp_propagate_batch (layout of srp_traj)."""
    _fields_ = [("mesh_id", C.c_int32), ("N", C.c_int32), ("bounces", C.c_int32), ("panel_mode", C.c_int32),
                ("angles", C.c_void_p), ("central", C.c_int32), ("attitude", C.c_int32), ("q", C.c_double * 4),
                ("y0", C.c_double * 6), ("t0", C.c_double), ("t1", C.c_double)]


class SrpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [
        ("n_verts", C.c_int32), ("vertex_dtype", C.c_int32), ("xyz", C.c_void_p),
        ("n_tris", C.c_int32), ("tri", C.c_void_p), ("tri_part", C.c_void_p), ("tri_mat", C.c_void_p),
        ("n_mats", C.c_int32), ("mat", C.c_void_p),
        ("n_parts", C.c_int32), ("parent", C.c_void_p), ("pivot", C.c_void_p), ("axis", C.c_void_p),
        ("limits", C.c_void_p), ("normal0", C.c_void_p),
        ("c_ref", C.c_double * 3), ("mass", C.c_double),
    ]


class EvalParams(C.Structure):
    _fields_ = [("N", C.c_int32), ("bounces", C.c_int32), ("P0", C.c_double), ("eps_rel", C.c_double),
                ("panel_mode", C.c_int32), ("flags", C.c_int32), ("n_diffuse", C.c_int32),
                ("diffuse_seed", C.c_uint32)]


class EvalStats(C.Structure):
    _fields_ = [("evals", C.c_int64), ("rays", C.c_int64), ("segments", C.c_int64),
                ("hits", C.c_int64 * (MAX_BOUNCES + 1)), ("refined", C.c_int64), ("nodes_visited", C.c_int64),
                ("tris_tested", C.c_int64), ("box_tests", C.c_int64), ("handoff_cause", C.c_int64 * 4),
                ("launches", C.c_int64),
                ("trace_launches", C.c_int64), ("ms_geometry", C.c_double), ("ms_trace", C.c_double),
                ("ms_refine", C.c_double), ("ms_reduce", C.c_double), ("ms_transfer", C.c_double),
                ("ms_raster", C.c_double)]


RKF78, RK4 = 0, 1
CENTRAL_EARTH, CENTRAL_SUN = 0, 1
ATT_LVLH, ATT_INERTIAL = 0, 1


class SpadGrid(C.Structure):
    _fields_ = [("n_az", C.c_int32), ("n_el", C.c_int32), ("az0", C.c_double), ("el0", C.c_double),
                ("d_el", C.c_double)]


def spad_grid_struct(g) -> SpadGrid:
    """srp_spad_grid from a dict with n_az, n_el, az0, el0, d_el (radians)."""
    if isinstance(g, SpadGrid):
        return g
    return SpadGrid(int(g["n_az"]), int(g["n_el"]), float(g["az0"]), float(g["el0"]), float(g["d_el"]))


class PropParams(C.Structure):
    _fields_ = [("method", C.c_int32), ("central", C.c_int32), ("j2", C.c_int32), ("sun3", C.c_int32),
                ("srp", C.c_int32), ("attitude", C.c_int32), ("q", C.c_double * 4), ("epoch_mjd_tt", C.c_double),
                ("rtol", C.c_double), ("atol_pos", C.c_double), ("atol_vel", C.c_double), ("h0", C.c_double),
                ("h_min", C.c_double), ("h_max", C.c_double), ("max_steps", C.c_int64), ("poll", C.c_int32),
                ("host_loop", C.c_int32), ("eval", EvalParams), ("h_replay", C.c_void_p), ("n_replay", C.c_int64),
                ("spad_table", C.c_void_p), ("spad_grid", SpadGrid)]


class PropStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rejects", C.c_int64), ("evals", C.c_int64), ("t", C.c_double),
                ("status", C.c_int32), ("reserved", C.c_int32), ("h_next", C.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libsrp.so (building it first when sources changed)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsrp.so not found at {path}")
        lib = C.CDLL(path)
        lib.srp_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p]
        lib.srp_destroy.argtypes = [C.c_void_p]
        lib.srp_destroy.restype = None
        lib.srp_last_error.argtypes = [C.c_void_p]
        lib.srp_last_error.restype = C.c_char_p
        lib.srp_mesh_load.argtypes = [C.c_void_p, C.POINTER(MeshDesc), C.POINTER(C.c_int32)]
        lib.srp_mesh_free.argtypes = [C.c_void_p, C.c_int32]
        lib.srp_set_panel_angles.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
        lib.srp_eval_batch.argtypes = [C.c_void_p, C.c_int32, C.POINTER(EvalParams), C.c_int32, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.srp_eval_stats_get.argtypes = [C.c_void_p, C.POINTER(EvalStats)]
        lib.srp_set_materials.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
        lib.srp_grad.argtypes = [C.c_void_p, C.c_int32, C.POINTER(EvalParams), C.c_int32] + [C.c_void_p] * 12
        lib.srp_propagate_batch.argtypes = [C.c_void_p, C.POINTER(PropParams), C.c_int32, C.POINTER(Traj),
                                            C.c_void_p, C.POINTER(PropStats)]
        lib.srp_autotune.argtypes = [C.c_void_p, C.c_int32, C.POINTER(EvalParams), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double)]
        lib.srp_set_tile_shape.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32]
        lib.srp_prop_grad.argtypes = [C.c_void_p, C.c_int32, C.POINTER(PropParams), C.c_int32, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.POINTER(PropStats)]
        lib.srp_propagate.argtypes = [C.c_void_p, C.c_int32, C.POINTER(PropParams), C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(PropStats), C.c_void_p, C.c_int64]
        lib.srp_spad_build.argtypes = [C.c_void_p, C.c_int32, C.POINTER(EvalParams), C.POINTER(SpadGrid), C.c_void_p]
        lib.srp_spad_eval.argtypes = [C.c_void_p, C.POINTER(SpadGrid), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]
        lib.srp_set_memory_limit.argtypes = [C.c_void_p, C.c_uint64]
        lib.srp_memory_usage.argtypes = [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        lib.srp_sort_pairs.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]
        lib.srp_mesh_check.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int64)]
        lib.srp_eval_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                         C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_double), C.c_int32,
                                         C.c_int32, C.c_double, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
        _lib = lib
    return _lib


def eval_noalloc(tri_xyz, tri_mat, mat, sun_dir, sun_dist_au, c_ref, N, bounces, P0, eps_rel, force, torque,
                 stream=None):
    """srp_eval_noalloc: one evaluation that allocates nothing.  tri_xyz
    [n_tris, 9] float64, tri_mat [n_tris, 2] int32, mat [n_mats, 2] float64,
    force / torque [3] float64 are CUDA tensors the caller owns; sun_dir and
    c_ref are 3-sequences.  Asynchronous on `stream` (default: torch's current
    stream); raises SrpError on a non-zero status."""
    import torch
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream()
    n = int(tri_xyz.shape[0]) if tri_xyz.dim() >= 1 else 0
    m = int(mat.shape[0]) if mat.dim() >= 1 else 0
    want = ((tri_xyz, torch.float64, (n, 9)), (tri_mat, torch.int32, (n, 2)), (mat, torch.float64, (m, 2)),
            (force, torch.float64, (3,)), (torque, torch.float64, (3,)))
    for k, (t, dt, shape) in enumerate(want):
        if not isinstance(t, torch.Tensor) or t.dtype != dt or tuple(t.shape) != shape or not t.is_contiguous():
            raise SrpError(SRP_ERR_ARG, f"srp_eval_noalloc: argument {k} must be a contiguous {dt} tensor of "
                                        f"shape {shape}")
        if t.device.type != "cuda" or t.device != st.device:
            raise SrpError(SRP_ERR_ARG, f"srp_eval_noalloc: argument {k} must live on the stream's device {st.device}")
    s = (C.c_double * 3)(*[float(x) for x in sun_dir])
    c = (C.c_double * 3)(*[float(x) for x in c_ref])
    rc = lib.srp_eval_noalloc(tri_xyz.data_ptr(), tri_mat.data_ptr(), int(tri_xyz.shape[0]), mat.data_ptr(),
                              int(mat.shape[0]), s, float(sun_dist_au), c, int(N), int(bounces), float(P0),
                              float(eps_rel), force.data_ptr(), torque.data_ptr(), st.cuda_stream)
    if rc != SRP_OK:
        raise SrpError(rc, "srp_eval_noalloc failed")


def _ptr(x):
    """(pointer, keepalive) of a numpy array or torch tensor (C-contiguous)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, x
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x
    raise TypeError(f"unsupported array type {type(x)}")


def _maker(like):
    """Allocator of float64 outputs placed like `like` (CUDA tensor or numpy)."""
    if _is_cuda(like):
        import torch
        return lambda shape: torch.empty(shape, dtype=torch.float64, device=like.device)
    return lambda shape: np.empty(shape)


def _is_cuda(x):
    try:
        import torch
        return isinstance(x, torch.Tensor) and x.is_cuda
    except ImportError:
        return False


class Context:
    """One srp_ctx: a CUDA device, a stream, the loaded meshes."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = C.c_void_p()
        st = None
        if stream is not None:
            st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = self.lib.srp_create(C.byref(h), device, st)
        if rc != SRP_OK:
            raise SrpError(rc, f"srp_create(device={device}) failed")
        self.h = h
        self.device = device
        self.meshes = {}
        self.mesh_info = {}

    def _check(self, rc):
        if rc != SRP_OK:
            raise SrpError(rc, self.lib.srp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.srp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load_mesh(self, mesh) -> int:
        """Load a mesh given as paper_2608_07307_gb300.inputs.Mesh (or any object
        with the same array attributes)."""
        xyz = np.ascontiguousarray(mesh.xyz)
        dt = SRP_F64 if xyz.dtype == np.float64 else SRP_F32
        if xyz.dtype not in (np.float32, np.float64):
            xyz = np.ascontiguousarray(xyz, np.float64)
            dt = SRP_F64
        keep = dict(
            xyz=xyz, tri=np.ascontiguousarray(mesh.tri, np.int32), tri_part=np.ascontiguousarray(mesh.tri_part, np.int32),
            tri_mat=np.ascontiguousarray(mesh.tri_mat, np.int32), mat=np.ascontiguousarray(mesh.mat, np.float64),
            parent=np.ascontiguousarray(mesh.parent, np.int32), pivot=np.ascontiguousarray(mesh.pivot, np.float64),
            axis=np.ascontiguousarray(mesh.axis, np.float64), limits=np.ascontiguousarray(mesh.limits, np.float64),
            normal0=np.ascontiguousarray(mesh.normal0, np.float64))
        d = MeshDesc(len(xyz), dt, keep["xyz"].ctypes.data, len(keep["tri"]), keep["tri"].ctypes.data,
                     keep["tri_part"].ctypes.data, keep["tri_mat"].ctypes.data, len(keep["mat"]),
                     keep["mat"].ctypes.data, len(keep["parent"]), keep["parent"].ctypes.data,
                     keep["pivot"].ctypes.data, keep["axis"].ctypes.data, keep["limits"].ctypes.data,
                     keep["normal0"].ctypes.data, (C.c_double * 3)(*np.asarray(mesh.c_ref, np.float64)),
                     float(getattr(mesh, "mass", 1.0)))
        mid = C.c_int32(-1)
        self._check(self.lib.srp_mesh_load(self.h, C.byref(d), C.byref(mid)))
        self.meshes[mid.value] = len(keep["parent"])
        self.mesh_info[mid.value] = dict(n_parts=len(keep["parent"]), n_mats=len(keep["mat"]))
        return mid.value

    def free_mesh(self, mesh_id: int):
        self._check(self.lib.srp_mesh_free(self.h, mesh_id))
        self.meshes.pop(mesh_id, None)

    def set_panel_angles(self, mesh_id: int, angles):
        """srp_set_panel_angles: commanded angles / tracking offsets [n_parts]
        (numpy, sequence, or torch tensor on the host or the device)."""
        if _is_cuda(angles):
            a = angles.detach().to(dtype=__import__("torch").float64).contiguous()
        else:
            a = angles.detach().cpu().numpy() if hasattr(angles, "detach") else angles
            a = np.ascontiguousarray(np.asarray(a, np.float64))
        pa, k = _ptr(a)
        self._check(self.lib.srp_set_panel_angles(self.h, mesh_id, int(a.shape[0]), pa))

    def eval_batch(self, mesh_id: int, sun_dirs, sun_dist=None, N: int = 256, bounces: int = 1, P0: float = 4.56e-6,
                   eps_rel: float = 1e-9, panel_mode: int = PANELS_TRACK, hits: bool = False, count: bool = False,
                   timing: bool = False, out=None, traverse: bool = False, n_diffuse: int = 0,
                   diffuse_seed: int = 0, flags: int = 0, quat=None):
        """Force [n,3] (N) and torque [n,3] (N m); with hits=True also the per-ray
        hit triangle ids [n, N*N, bounces+1].  Outputs live where the input lives
        (CUDA tensor in, CUDA tensors out; numpy in, numpy out) unless `out`
        = (force, torque[, hits]) is given.  n_diffuse: diffuse secondary rays
        per hit (srp_eval_params).  quat [n,4] (body -> inertial, scalar
        first): sun_dirs are then inertial and the first output is the SRP
        acceleration R(q) F / mass (m/s^2, inertial frame)."""
        n = int(sun_dirs.shape[0])
        cuda = _is_cuda(sun_dirs)
        conv = lambda x: None if x is None else (np.ascontiguousarray(x, np.float64) if isinstance(x, np.ndarray)  # noqa: E731
                                                 else x.contiguous())
        sun_dirs, sun_dist, quat = conv(sun_dirs), conv(sun_dist), conv(quat)
        nseg = bounces + 1
        if out is not None:
            force, torque = out[0], out[1]
            hit = out[2] if len(out) > 2 else None
        elif cuda:
            import torch
            force = torch.empty((n, 3), dtype=torch.float64, device=sun_dirs.device)
            torque = torch.empty_like(force)
            hit = torch.empty((n, N * N, nseg), dtype=torch.int32, device=sun_dirs.device) if hits else None
        else:
            force, torque = np.empty((n, 3)), np.empty((n, 3))
            hit = np.empty((n, N * N, nseg), np.int32) if hits else None
        p = EvalParams(N, bounces, P0, eps_rel, panel_mode, (EVAL_COUNT if count else 0) | (EVAL_TIMING if timing else 0)
                       | (EVAL_TRAVERSE if traverse else 0) | flags, n_diffuse, diffuse_seed)
        ps, k1 = _ptr(sun_dirs)
        pq, k0 = _ptr(quat)
        pd, k2 = _ptr(sun_dist)
        pf, k3 = _ptr(force)
        pt, k4 = _ptr(torque)
        ph, k5 = _ptr(hit)
        self._check(self.lib.srp_eval_batch(self.h, mesh_id, C.byref(p), n, ps, pq, pd, pf, pt, ph))
        return (force, torque, hit) if hits else (force, torque)

    def propagate(self, mesh_id: int, y0, t0_t1, method: int = RKF78, central: int = CENTRAL_EARTH, j2=False,
                  sun3=False, srp_on=True, attitude: int = ATT_LVLH, q=(1.0, 0.0, 0.0, 0.0),
                  epoch_mjd_tt: float = 61041.0, rtol: float = 1e-12, atol_pos: float = 1e-6,
                  atol_vel: float = 1e-9, h0: float = 60.0, h_min: float = 1e-6, h_max: float = 0.0,
                  max_steps: int = 10_000_000, poll: int = 16, N: int = 64, bounces: int = 1, P0: float = 4.56e-6,
                  eps_rel: float = 1e-9, panel_mode: int = PANELS_TRACK, h_cap: int = 0, h_replay=None,
                  host_loop: bool = False, traverse: bool = False, spad=None, n_diffuse: int = 0,
                  diffuse_seed: int = 0):
        """srp_propagate: y1 [n, 6], per-trajectory stats (list of dicts) and,
        with h_cap > 0, the accepted step sizes [n, h_cap] (NaN padded).
        h_replay [n, k]: take exactly these RKF7(8) steps (replay).
        spad = (grid, table): the SRP force is the SPAD interpolant of the
        table (spad_build) instead of a ray-traced evaluation."""
        y0 = np.ascontiguousarray(np.asarray(y0, np.float64).reshape(-1, 6))
        n = len(y0)
        t01 = np.ascontiguousarray(np.asarray(t0_t1, np.float64).reshape(n, 2))
        hr = None if h_replay is None else np.ascontiguousarray(np.asarray(h_replay, np.float64).reshape(n, -1))
        p = PropParams(method, central, int(j2), int(sun3), int(srp_on), attitude, (C.c_double * 4)(*q),
                       epoch_mjd_tt, rtol, atol_pos, atol_vel, h0, h_min, h_max, max_steps, poll, int(host_loop),
                       EvalParams(N, bounces, P0, eps_rel, panel_mode, EVAL_TRAVERSE if traverse else 0, n_diffuse,
                                  diffuse_seed),
                       hr.ctypes.data if hr is not None else None, 0 if hr is None else hr.shape[1])
        keep = None
        if spad is not None:
            grid, table = spad
            table = self._spad_table_arg(table)
            p.spad_table, keep = _ptr(table)
            p.spad_grid = spad_grid_struct(grid)
        y1 = np.empty((n, 6))
        st = (PropStats * n)()
        hl = np.full((n, h_cap), np.nan) if h_cap > 0 else None
        self._check(self.lib.srp_propagate(self.h, mesh_id, C.byref(p), n, y0.ctypes.data, t01.ctypes.data,
                                           y1.ctypes.data, st, hl.ctypes.data if hl is not None else None,
                                           h_cap))
        stats = [dict(steps=s.steps, rejects=s.rejects, evals=s.evals, t=s.t, status=s.status, h_next=s.h_next) for s in st]
        if hl is not None:
            for i, s in enumerate(stats):
                hl[i, min(s["steps"], h_cap):] = np.nan
        return y1, stats, hl

    @staticmethod
    def _spad_table_arg(table):
        if _is_cuda(table):
            return table.detach().to(dtype=__import__("torch").float64).contiguous()
        if hasattr(table, "detach"):
            table = table.detach().cpu().numpy()
        return np.ascontiguousarray(np.asarray(table, np.float64))

    def spad_build(self, mesh_id: int, grid, N: int = 256, bounces: int = 1, P0: float = 4.56e-6,
                   eps_rel: float = 1e-9, panel_mode: int = PANELS_TRACK, traverse: bool = False, device=False):
        """srp_spad_build: the SPAD table [n_el, n_az, 6] (F, T at 1 AU) of the
        grid (a dict with n_az, n_el, az0, el0, d_el in radians); a CUDA
        tensor when device=True, else a numpy array."""
        g = spad_grid_struct(grid)
        if device:
            import torch
            table = torch.empty((g.n_el, g.n_az, 6), dtype=torch.float64, device=f"cuda:{self.device}")
        else:
            table = np.empty((g.n_el, g.n_az, 6))
        p = EvalParams(N, bounces, P0, eps_rel, panel_mode, EVAL_TRAVERSE if traverse else 0)
        pt, k = _ptr(table)
        self._check(self.lib.srp_spad_build(self.h, mesh_id, C.byref(p), C.byref(g), pt))
        return table

    def spad_eval(self, grid, table, sun_dirs, sun_dist=None):
        """srp_spad_eval: (force [n, 3], torque [n, 3]) of the SPAD interpolant;
        CUDA tensors in give CUDA tensors out."""
        g = spad_grid_struct(grid)
        table = self._spad_table_arg(table)
        if _is_cuda(sun_dirs):
            import torch
            sun_dirs = sun_dirs.detach().to(dtype=torch.float64).contiguous()
            if sun_dist is not None:
                sun_dist = sun_dist.detach().to(device=sun_dirs.device, dtype=torch.float64).contiguous()
            n = sun_dirs.shape[0]
            force = torch.empty((n, 3), dtype=torch.float64, device=sun_dirs.device)
            torque = torch.empty_like(force)
        else:
            sun_dirs = np.ascontiguousarray(np.asarray(sun_dirs, np.float64).reshape(-1, 3))
            if sun_dist is not None:
                sun_dist = np.ascontiguousarray(np.asarray(sun_dist, np.float64).reshape(-1))
            n = sun_dirs.shape[0]
            force, torque = np.empty((n, 3)), np.empty((n, 3))
        pg, k0 = _ptr(table)
        ps, k1 = _ptr(sun_dirs)
        pd, k2 = _ptr(sun_dist)
        pf, k3 = _ptr(force)
        pt, k4 = _ptr(torque)
        self._check(self.lib.srp_spad_eval(self.h, C.byref(g), pg, n, ps, pd, pf, pt))
        return force, torque

    def set_memory_limit(self, nbytes: int):
        """srp_set_memory_limit: cap on the library's device memory (0: none)."""
        self._check(self.lib.srp_set_memory_limit(self.h, int(nbytes)))

    def memory_usage(self):
        """srp_memory_usage: (bytes held, cap)."""
        u, l = C.c_uint64(), C.c_uint64()
        self._check(self.lib.srp_memory_usage(self.h, C.byref(u), C.byref(l)))
        return int(u.value), int(l.value)

    def sort_pairs(self, keys, vals, key_bits: int = 64):
        """srp_sort_pairs: the build's stable radix sort, on copies; returns
        (keys, vals) sorted by key bits [0, key_bits)."""
        k = np.ascontiguousarray(np.asarray(keys, np.uint64)).copy()
        v = np.ascontiguousarray(np.asarray(vals, np.int32)).copy()
        if len(k) != len(v):
            raise ValueError("keys and vals differ in length")
        self._check(self.lib.srp_sort_pairs(self.h, len(k), k.ctypes.data, v.ctypes.data, int(key_bits)))
        return k, v

    def mesh_check(self, mesh_id: int, sun_dir=None):
        """srp_mesh_check: dict of the BVH structure counts after posing."""
        rep = (C.c_int64 * 8)()
        s = None if sun_dir is None else np.ascontiguousarray(np.asarray(sun_dir, np.float64).reshape(3))
        self._check(self.lib.srp_mesh_check(self.h, mesh_id, s.ctypes.data if s is not None else None, rep))
        names = ["leaf_refs", "tris_not_once", "boxes_outside_parent", "tris_outside_leaf", "nodes", "walk_bound",
                 "n_tris", "n_parts"]
        return dict(zip(names, [int(x) for x in rep]))

    def set_materials(self, mesh_id: int, mat):
        """srp_set_materials: new (rho_s, rho_d) per material, [n_mats, 2]."""
        if _is_cuda(mat):
            mat = mat.detach().to(dtype=__import__("torch").float64).contiguous()
        else:
            mat = mat.detach().cpu().numpy() if hasattr(mat, "detach") else mat
            mat = np.ascontiguousarray(np.asarray(mat, np.float64))
        pm, k = _ptr(mat)
        self._check(self.lib.srp_set_materials(self.h, mesh_id, int(mat.shape[0]), pm))

    def grad(self, mesh_id: int, sun_dirs, g_force, g_torque, sun_dist=None, N: int = 256, bounces: int = 1,
             P0: float = 4.56e-6, eps_rel: float = 1e-9, panel_mode: int = PANELS_TRACK, n_mats=None,
             n_parts=None, quat=None):
        """srp_grad: force, torque and the frozen-hit gradients of
        L = sum g_force . F + g_torque . T.  Returns a dict with F, T [n,3],
        sun [n,3], dist [n] (when sun_dist is given), mat [n_mats,2],
        angle [n_parts] and, with quat [n,4], quat [n,4] (F is then the
        inertial SRP acceleration R(q) F / mass and sun_dirs are inertial).
        CUDA tensors in, CUDA tensors out; numpy otherwise."""
        n = int(sun_dirs.shape[0])
        cuda = _is_cuda(sun_dirs)
        mk = _maker(sun_dirs)
        conv = lambda x: None if x is None else (np.ascontiguousarray(x, np.float64) if isinstance(x, np.ndarray)  # noqa: E731
                                                 else x.contiguous())
        sun_dirs, g_force, g_torque, sun_dist, quat = map(conv, (sun_dirs, g_force, g_torque, sun_dist, quat))
        M = self.mesh_info[mesh_id]["n_mats"] if n_mats is None else n_mats
        P = self.mesh_info[mesh_id]["n_parts"] if n_parts is None else n_parts
        out = dict(F=mk((n, 3)), T=mk((n, 3)), sun=mk((n, 3)), mat=mk((M, 2)), angle=mk((P,)))
        if sun_dist is not None:
            out["dist"] = mk((n,))
        if quat is not None:
            out["quat"] = mk((n, 4))
        p = EvalParams(N, bounces, P0, eps_rel, panel_mode, 0)
        args = [sun_dirs, quat, sun_dist, g_force, g_torque, out["F"], out["T"], out["sun"], out.get("dist"),
                out["mat"], out["angle"], out.get("quat")]
        ptrs = [_ptr(x) for x in args]
        self._check(self.lib.srp_grad(self.h, mesh_id, C.byref(p), n, *[q[0] for q in ptrs]))
        return out

    def prop_grad(self, mesh_id: int, y0, t0_t1, g_y1, ckpt_every: int = 100, central: int = CENTRAL_EARTH,
                  j2=False, sun3=False, srp_on=True, attitude: int = ATT_LVLH, q=(1.0, 0.0, 0.0, 0.0),
                  epoch_mjd_tt: float = 61041.0, h0: float = 60.0, max_steps: int = 10_000_000, N: int = 64,
                  bounces: int = 1, P0: float = 4.56e-6, eps_rel: float = 1e-9, panel_mode: int = PANELS_TRACK):
        """srp_prop_grad: RK4 arc and the gradients of sum g_y1 . y1.  Returns
        a dict with y1 [n,6], y0 [n,6] (gradient), mat [M,2], angle [P], q [4]
        and the per-trajectory stats."""
        y0 = np.ascontiguousarray(np.asarray(y0, np.float64).reshape(-1, 6))
        n = len(y0)
        t01 = np.ascontiguousarray(np.asarray(t0_t1, np.float64).reshape(n, 2))
        g1 = np.ascontiguousarray(np.asarray(g_y1, np.float64).reshape(n, 6))
        p = PropParams(RK4, central, int(j2), int(sun3), int(srp_on), attitude, (C.c_double * 4)(*q), epoch_mjd_tt,
                       0.0, 0.0, 0.0, h0, 0.0, 0.0, max_steps, 0, 0, EvalParams(N, bounces, P0, eps_rel, panel_mode, 0),
                       None, 0)
        info = self.mesh_info[mesh_id]
        out = dict(y1=np.empty((n, 6)), y0=np.empty((n, 6)), mat=np.empty((info["n_mats"], 2)),
                   angle=np.empty(info["n_parts"]), q=np.empty(4))
        st = (PropStats * n)()
        self._check(self.lib.srp_prop_grad(self.h, mesh_id, C.byref(p), n, y0.ctypes.data, t01.ctypes.data,
                                           g1.ctypes.data, int(ckpt_every), out["y1"].ctypes.data,
                                           out["y0"].ctypes.data, out["mat"].ctypes.data, out["angle"].ctypes.data,
                                           out["q"].ctypes.data, st))
        out["stats"] = [dict(steps=s.steps, rejects=s.rejects, evals=s.evals, t=s.t, status=s.status, h_next=s.h_next) for s in st]
        return out

    def propagate_batch(self, trajs, method: int = RKF78, j2=False, sun3=False, srp_on=True,
                        epoch_mjd_tt: float = 61041.0, rtol: float = 1e-12, atol_pos: float = 1e-6,
                        atol_vel: float = 1e-9, h0: float = 60.0, h_min: float = 1e-6, h_max: float = 0.0,
                        max_steps: int = 10_000_000, poll: int = 16, P0: float = 4.56e-6, eps_rel: float = 1e-9,
                        autotune: bool = False, traverse: bool = False, flags: int = 0):
        """srp_propagate_batch over a list of trajectory dicts with keys mesh_id,
        N, bounces, panel_mode, angles (or None), central, attitude, q, y0, t0,
        t1.  Returns (y1 [n, 6], stats list)."""
        n = len(trajs)
        arr = (Traj * n)()
        keep = []
        for i, t in enumerate(trajs):
            ang = t.get("angles")
            a = None if ang is None else np.ascontiguousarray(np.asarray(ang, np.float64))
            keep.append(a)
            arr[i] = Traj(int(t["mesh_id"]), int(t["N"]), int(t["bounces"]), int(t.get("panel_mode", PANELS_TRACK)),
                          a.ctypes.data if a is not None else None, int(t.get("central", CENTRAL_EARTH)),
                          int(t.get("attitude", ATT_LVLH)), (C.c_double * 4)(*t.get("q", (1.0, 0.0, 0.0, 0.0))),
                          (C.c_double * 6)(*[float(x) for x in t["y0"]]), float(t["t0"]), float(t["t1"]))
        p = PropParams(method, 0, int(j2), int(sun3), int(srp_on), 0, (C.c_double * 4)(1.0, 0.0, 0.0, 0.0),
                       epoch_mjd_tt, rtol, atol_pos, atol_vel, h0, h_min, h_max, max_steps, poll, 0,
                       EvalParams(1, 0, P0, eps_rel, 0, (EVAL_AUTOTUNE if autotune else 0)
                                  | (EVAL_TRAVERSE if traverse else 0) | flags), None, 0)
        y1 = np.empty((n, 6))
        st = (PropStats * n)()
        self._check(self.lib.srp_propagate_batch(self.h, C.byref(p), n, arr, y1.ctypes.data, st))
        return y1, [dict(steps=s.steps, rejects=s.rejects, evals=s.evals, t=s.t, status=s.status, h_next=s.h_next) for s in st]

    def autotune(self, mesh_id: int, N: int, bounces: int, P0: float = 4.56e-6, eps_rel: float = 1e-9,
                 panel_mode: int = PANELS_TRACK):
        """srp_autotune: (chosen tile width, ms per evaluation of widths 4, 8, 16, 32)."""
        p = EvalParams(N, bounces, P0, eps_rel, panel_mode, 0)
        w = C.c_int32(0)
        ms = (C.c_double * 4)()
        self._check(self.lib.srp_autotune(self.h, mesh_id, C.byref(p), C.byref(w), ms))
        return int(w.value), list(ms)

    def set_tile_shape(self, mesh_id: int, N: int, bounces: int, tile_w: int):
        """srp_set_tile_shape: trace tiles tile_w pixels wide for (mesh, N, bounces)."""
        self._check(self.lib.srp_set_tile_shape(self.h, mesh_id, N, bounces, tile_w))

    def eval_stats(self) -> dict:
        s = EvalStats()
        self._check(self.lib.srp_eval_stats_get(self.h, C.byref(s)))
        return dict(evals=s.evals, rays=s.rays, segments=s.segments, hits=list(s.hits), refined=s.refined,
                    nodes_visited=s.nodes_visited, tris_tested=s.tris_tested, box_tests=s.box_tests,
                    handoff_cause=list(s.handoff_cause), launches=s.launches, trace_launches=s.trace_launches, ms_geometry=s.ms_geometry,
                    ms_trace=s.ms_trace, ms_refine=s.ms_refine, ms_reduce=s.ms_reduce, ms_transfer=s.ms_transfer,
                    ms_raster=s.ms_raster)
