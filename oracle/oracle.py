"""Python harness for the FP64 brute-force oracle (``srp_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs.  The library under
``paper_2608_07307_gb300/`` never imports this module, and this module never
imports that library (it reads meshes produced by the shared input generators
as plain numpy arrays).

The C code is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/liboracle.so`` with floating-point contraction disabled, so
x86 and Arm hosts round identically.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SOURCES = ["srp_oracle.c", "frozen_oracle.c", "prop_oracle.c", "spad_oracle.c"]
HEADERS = ["srp_oracle.h"]
LIB = os.path.join(BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FP contraction, no fast-math)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    deps = srcs + [os.path.join(HERE, h) for h in HEADERS]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in deps):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class _Mesh(C.Structure):
    _fields_ = [
        ("n_verts", C.c_int32), ("xyz", C.POINTER(C.c_double)),
        ("n_tris", C.c_int32), ("tri", C.POINTER(C.c_int32)),
        ("tri_part", C.POINTER(C.c_int32)), ("tri_mat", C.POINTER(C.c_int32)),
        ("n_mats", C.c_int32), ("mat", C.POINTER(C.c_double)),
        ("n_parts", C.c_int32), ("parent", C.POINTER(C.c_int32)),
        ("pivot", C.POINTER(C.c_double)), ("axis", C.POINTER(C.c_double)),
        ("limits", C.POINTER(C.c_double)), ("normal0", C.POINTER(C.c_double)),
        ("c_ref", C.c_double * 3),
    ]


class _Params(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("bounces", C.c_int32), ("P0", C.c_double), ("dist_au", C.c_double),
        ("eps_rel", C.c_double), ("track", C.c_int32), ("angles", C.POINTER(C.c_double)),
        ("n_diffuse", C.c_int32), ("diffuse_seed", C.c_uint32),
    ]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_eval_range.restype = C.c_int
        _lib.orc_eval_rays.restype = C.c_int
        _lib.orc_pose.restype = C.c_int
        _lib.orc_window_ids.restype = C.c_int
        _lib.orc_eval_frozen.restype = C.c_int
        _lib.orc_rk4_arc.restype = C.c_int
        _lib.orc_splitmix64.restype = C.c_uint64
        _lib.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class OMesh:
    """A mesh held in the C layout (FP32 vertices promoted exactly to FP64)."""

    def __init__(self, mesh):
        self.keep = dict(
            xyz=np.ascontiguousarray(np.asarray(mesh.xyz).astype(np.float64)),
            tri=np.ascontiguousarray(mesh.tri.astype(np.int32)),
            tri_part=np.ascontiguousarray(mesh.tri_part.astype(np.int32)),
            tri_mat=np.ascontiguousarray(mesh.tri_mat.astype(np.int32)),
            mat=np.ascontiguousarray(np.asarray(mesh.mat, np.float64)),
            parent=np.ascontiguousarray(mesh.parent.astype(np.int32)),
            pivot=np.ascontiguousarray(np.asarray(mesh.pivot, np.float64)),
            axis=np.ascontiguousarray(np.asarray(mesh.axis, np.float64)),
            limits=np.ascontiguousarray(np.asarray(mesh.limits, np.float64)),
            normal0=np.ascontiguousarray(np.asarray(mesh.normal0, np.float64)),
        )
        k = self.keep
        self.n_parts = len(k["parent"])
        self.s = _Mesh(len(k["xyz"]), _dp(k["xyz"]), len(k["tri"]), _ip(k["tri"]), _ip(k["tri_part"]),
                       _ip(k["tri_mat"]), len(k["mat"]), _dp(k["mat"]), self.n_parts, _ip(k["parent"]),
                       _dp(k["pivot"]), _dp(k["axis"]), _dp(k["limits"]), _dp(k["normal0"]),
                       (C.c_double * 3)(*np.asarray(mesh.c_ref, np.float64)))


def _params(N, bounces, P0, dist_au, eps_rel, angles, n_parts, offsets=None, n_diffuse=0, diffuse_seed=0):
    """Sun tracking (no angles), commanded angles, or tracking + offsets."""
    if angles is not None and offsets is not None:
        raise ValueError("give commanded angles or tracking offsets, not both")
    if angles is None and offsets is None:
        return _Params(N, bounces, P0, dist_au, eps_rel, 1, None, n_diffuse, diffuse_seed), None
    a = np.ascontiguousarray(np.asarray(angles if offsets is None else offsets, np.float64).reshape(n_parts))
    return _Params(N, bounces, P0, dist_au, eps_rel, 0 if offsets is None else 2, _dp(a), n_diffuse,
                   diffuse_seed), a


def pose(mesh, s, angles=None, offsets=None):
    """(joint angles [P], posed vertices [V,3]) for Sun direction s (Sec. 4.4.2):
    tracking, commanded `angles`, or tracking plus `offsets`."""
    om = OMesh(mesh)
    s = np.ascontiguousarray(np.asarray(s, np.float64))
    ang = np.zeros(om.n_parts)
    xyz = np.zeros_like(om.keep["xyz"])
    p, a_in = _params(1, 0, 0.0, 1.0, 0.0, angles, om.n_parts, offsets)
    rc = lib().orc_pose(C.byref(om.s), _dp(s), C.c_int32(p.track), _dp(a_in) if a_in is not None else None,
                        _dp(ang), _dp(xyz))
    if rc != 0:
        raise ValueError(f"orc_pose failed: {rc}")
    return ang, xyz


def eval_range(mesh, s, N, bounces=1, P0=4.56e-6, dist_au=1.0, eps_rel=1e-9, angles=None, r0=0, r1=None,
               want_hits=False, want_edge=False, _om=None, offsets=None, n_diffuse=0, diffuse_seed=0):
    """Trace rays [r0, r1) of one direction.  Returns a dict with the unscaled
    sums `acc` (6), the `scale` P dA, the window `win` (8), joint `angles`,
    per-segment hit counts `nhit`, and optionally `hits` / `edge` per ray."""
    om = _om or OMesh(mesh)
    r1 = N * N if r1 is None else r1
    p, keep = _params(N, bounces, P0, dist_au, eps_rel, angles, om.n_parts, offsets, n_diffuse, diffuse_seed)
    s = np.ascontiguousarray(np.asarray(s, np.float64))
    acc = np.zeros(6)
    scale = np.zeros(1)
    win = np.zeros(8)
    ang = np.zeros(om.n_parts)
    nseg = bounces + 1
    hits = np.empty((r1 - r0, nseg), np.int32) if want_hits else None
    edge = np.empty((r1 - r0, nseg), np.float64) if want_edge else None
    nhit = np.zeros(nseg, np.int64)
    rc = lib().orc_eval_range(C.byref(om.s), C.byref(p), _dp(s), C.c_int64(r0), C.c_int64(r1), _dp(acc),
                              _dp(scale), _dp(win), _dp(ang), _ip(hits) if hits is not None else None,
                              _dp(edge) if edge is not None else None,
                              nhit.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc != 0:
        raise ValueError(f"orc_eval_range failed: {rc}")
    return dict(acc=acc, scale=float(scale[0]), win=win, angles=ang, nhit=nhit, hits=hits, edge=edge)


def _worker(args):
    mesh, s, kw, r0, r1 = args
    return eval_range(mesh, s, r0=r0, r1=r1, **kw)


def evaluate(mesh, s, N, bounces=1, P0=4.56e-6, dist_au=1.0, eps_rel=1e-9, angles=None, want_hits=False,
             want_edge=False, procs=1, chunks=None, offsets=None, n_diffuse=0, diffuse_seed=0):
    """Force F (N) and torque T (N m) about c_ref for one Sun direction.

    With procs > 1 the ray range is split into contiguous chunks traced by
    spawn-started worker processes (each single-threaded); the partial sums
    are added in chunk order, so the result does not depend on scheduling."""
    kw = dict(N=N, bounces=bounces, P0=P0, dist_au=dist_au, eps_rel=eps_rel, angles=angles,
              want_hits=want_hits, want_edge=want_edge, offsets=offsets, n_diffuse=n_diffuse,
              diffuse_seed=diffuse_seed)
    R = N * N
    if procs <= 1:
        parts = [eval_range(mesh, s, **kw)]
    else:
        import multiprocessing as mp
        n = chunks or procs * 4
        bounds = [R * k // n for k in range(n + 1)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs) as pool:
            parts = pool.map(_worker, [(mesh, s, kw, bounds[k], bounds[k + 1]) for k in range(n)])
    acc = np.zeros(6)
    for q in parts:
        acc = acc + q["acc"]
    out = dict(parts[0])
    out["acc"] = acc
    out["nhit"] = sum(q["nhit"] for q in parts)
    if want_hits:
        out["hits"] = np.concatenate([q["hits"] for q in parts])
    if want_edge:
        out["edge"] = np.concatenate([q["edge"] for q in parts])
    out["F"] = acc[:3] * out["scale"]
    out["T"] = acc[3:] * out["scale"]
    return out


def _rays_worker(args):
    mesh, s, rays, N, kw = args
    return eval_rays(mesh, s, rays, N, **kw)


def eval_rays(mesh, s, rays, N, bounces=1, P0=4.56e-6, dist_au=1.0, eps_rel=1e-9, angles=None, n_diffuse=0,
              diffuse_seed=0, procs=1):
    """Per-ray unscaled contributions [n, 6], hits [n, nseg] and edge proximity
    [n, nseg] for an explicit list of primary ray indices (sampled checks).
    With procs > 1 the list is split into contiguous pieces traced by
    spawn-started worker processes and the results are concatenated in order."""
    if procs > 1 and len(rays) > 1:
        import multiprocessing as mp
        kw = dict(bounces=bounces, P0=P0, dist_au=dist_au, eps_rel=eps_rel, angles=angles, n_diffuse=n_diffuse,
                  diffuse_seed=diffuse_seed)
        rays = np.asarray(rays, np.int64)
        n = min(len(rays), procs * 4)
        bounds = [len(rays) * k // n for k in range(n + 1)]
        with mp.get_context("spawn").Pool(procs) as pool:
            parts = pool.map(_rays_worker, [(mesh, s, rays[bounds[k]:bounds[k + 1]], N, kw) for k in range(n)])
        return {key: np.concatenate([q[key] for q in parts]) for key in ("contrib", "hits", "edge")}
    om = OMesh(mesh)
    p, keep = _params(N, bounces, P0, dist_au, eps_rel, angles, om.n_parts, None, n_diffuse, diffuse_seed)
    rays = np.ascontiguousarray(np.asarray(rays, np.int64))
    n = len(rays)
    nseg = bounces + 1
    contrib = np.zeros((n, 6))
    hits = np.empty((n, nseg), np.int32)
    edge = np.empty((n, nseg))
    s = np.ascontiguousarray(np.asarray(s, np.float64))
    rc = lib().orc_eval_rays(C.byref(om.s), C.byref(p), _dp(s), C.c_int64(n),
                             rays.ctypes.data_as(C.POINTER(C.c_int64)), _dp(contrib), _ip(hits), _dp(edge))
    if rc != 0:
        raise ValueError(f"orc_eval_rays failed: {rc}")
    return dict(contrib=contrib, hits=hits, edge=edge)


def timed_rays(mesh, s, N, bounces, n_rays, seed=0, P0=4.56e-6, dist_au=1.0, eps_rel=1e-9, angles=None):
    """Time the oracle, as it stands, on n_rays sampled primary rays of one
    direction (single thread, force sums only).  Returns (seconds, rays)."""
    om = OMesh(mesh)
    p, keep = _params(N, bounces, P0, dist_au, eps_rel, angles, om.n_parts)
    rng = np.random.default_rng(seed)
    rays = np.ascontiguousarray(rng.choice(N * N, size=min(n_rays, N * N), replace=False).astype(np.int64))
    contrib = np.zeros((len(rays), 6))
    s = np.ascontiguousarray(np.asarray(s, np.float64))
    t0 = time.perf_counter()
    rc = lib().orc_eval_rays(C.byref(om.s), C.byref(p), _dp(s), C.c_int64(len(rays)),
                             rays.ctypes.data_as(C.POINTER(C.c_int64)), _dp(contrib), None, None)
    dt = time.perf_counter() - t0
    if rc != 0:
        raise ValueError(f"orc_eval_rays failed: {rc}")
    return dt, len(rays)


# ------------------------------------------------------- frozen-hit gradients
def window_ids(mesh, s, angles=None, offsets=None):
    """The four posed vertices extreme along u and v for unit Sun direction s
    (argmin u, argmax u, argmin v, argmax v; lowest index among equals)."""
    om = OMesh(mesh)
    p, keep = _params(1, 0, 0.0, 1.0, 0.0, angles, om.n_parts, offsets)
    ids = np.zeros(4, np.int32)
    s = np.ascontiguousarray(np.asarray(s, np.float64))
    rc = lib().orc_window_ids(C.byref(om.s), C.byref(p), _dp(s), _ip(ids))
    if rc != 0:
        raise ValueError(f"orc_window_ids failed: {rc}")
    return ids


def eval_frozen(mesh, s, hits, ids, N, bounces=1, P0=4.56e-6, dist_au=1.0, angles=None, offsets=None, mat=None,
                _om=None):
    """Force and torque of the frozen-hit function F_H (frozen_oracle.c) at Sun
    direction s (any length), with optical coefficients `mat` [M, 2] in place
    of the mesh's when given.  hits: [N*N, bounces+1] recorded ids."""
    om = _om or OMesh(mesh)
    ms = om.s
    keepm = None
    if mat is not None:
        keepm = np.ascontiguousarray(np.asarray(mat, np.float64).reshape(-1, 2))
        ms = _Mesh.from_buffer_copy(om.s)
        ms.mat = _dp(keepm)
    p, keep = _params(N, bounces, P0, dist_au, 0.0, angles, om.n_parts, offsets)
    hits = np.ascontiguousarray(np.asarray(hits, np.int32).reshape(N * N, bounces + 1))
    ids = np.ascontiguousarray(np.asarray(ids, np.int32))
    s = np.ascontiguousarray(np.asarray(s, np.float64))
    acc, scale = np.zeros(6), np.zeros(1)
    rc = lib().orc_eval_frozen(C.byref(ms), C.byref(p), _dp(s), C.c_int64(0), C.c_int64(N * N), _ip(hits), _ip(ids),
                               _dp(acc), _dp(scale))
    if rc != 0:
        raise ValueError(f"orc_eval_frozen failed: {rc}")
    return acc[:3] * scale[0], acc[3:] * scale[0]


def frozen_grad(mesh, s, N, bounces, gF, gT, dist_au=1.0, P0=4.56e-6, eps_rel=1e-9, angles=None, offsets=None,
                h=1e-6, procs=1):
    """Reference gradient: central differences, step h, of the scalar
    L = gF . F_H + gT . T_H with respect to every optical coefficient, every
    joint angle parameter (commanded angle, or offset from the tracking angle;
    tracking alone is read as offsets of zero), the three components of the
    Sun direction s and the Sun distance.  The hit set and window vertices are
    recorded by the traced oracle at the base point.
    Returns dict(mat [M, 2], angle [P], sun [3], dist, F, T, hits, ids)."""
    om = OMesh(mesh)
    P = om.n_parts
    if angles is None and offsets is None:
        offsets = np.zeros(P)
    s = np.asarray(s, np.float64)
    s_unit = s / np.linalg.norm(s)  # the traced oracle takes a unit vector; F_H normalises itself
    base = evaluate(mesh, s_unit, N, bounces, P0=P0, dist_au=dist_au, eps_rel=eps_rel, angles=angles,
                    offsets=offsets, want_hits=True, procs=procs)
    hits = base["hits"]
    ids = window_ids(mesh, s_unit, angles=angles, offsets=offsets)
    gF, gT = np.asarray(gF, np.float64), np.asarray(gT, np.float64)
    mat0 = np.asarray(mesh.mat, np.float64).reshape(-1, 2)

    def L(s_=s, dist=dist_au, ang=angles, off=offsets, mat=None):
        F, T = eval_frozen(mesh, s_, hits, ids, N, bounces, P0, dist, angles=ang, offsets=off, mat=mat, _om=om)
        return float(gF @ F + gT @ T)

    g_mat = np.zeros_like(mat0)
    for i in range(mat0.shape[0]):
        for c in range(2):
            mp, mm = mat0.copy(), mat0.copy()
            mp[i, c] += h
            mm[i, c] -= h
            g_mat[i, c] = (L(mat=mp) - L(mat=mm)) / (2 * h)
    g_ang = np.zeros(P)
    for q in range(P):
        if angles is not None:
            ap, am = np.array(angles, np.float64), np.array(angles, np.float64)
            ap[q] += h
            am[q] -= h
            g_ang[q] = (L(ang=ap) - L(ang=am)) / (2 * h)
        else:
            op, omn = np.array(offsets, np.float64), np.array(offsets, np.float64)
            op[q] += h
            omn[q] -= h
            g_ang[q] = (L(off=op) - L(off=omn)) / (2 * h)
    g_sun = np.zeros(3)
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        g_sun[k] = (L(s_=s + e) - L(s_=s - e)) / (2 * h)
    g_dist = (L(dist=dist_au + h) - L(dist=dist_au - h)) / (2 * h)
    return dict(mat=g_mat, angle=g_ang, sun=g_sun, dist=g_dist, F=base["F"], T=base["T"], hits=hits, ids=ids)


# --------------------------------------------------------------- propagation
class Prop(C.Structure):
    """Propagation settings (layout of orc_prop in prop_oracle.c)."""
    _fields_ = [
        ("central", C.c_int32), ("j2", C.c_int32), ("sun3", C.c_int32), ("srp", C.c_int32),
        ("attitude", C.c_int32), ("q", C.c_double * 4), ("epoch_mjd_tt", C.c_double), ("mass", C.c_double),
        ("N", C.c_int32), ("bounces", C.c_int32), ("P0", C.c_double), ("eps_rel", C.c_double),
        ("method", C.c_int32), ("rtol", C.c_double), ("atol_pos", C.c_double), ("atol_vel", C.c_double),
        ("h0", C.c_double), ("h_min", C.c_double), ("h_max", C.c_double), ("max_steps", C.c_int64),
        ("spad_table", C.POINTER(C.c_double)), ("spad_n_az", C.c_int32), ("spad_n_el", C.c_int32),
        ("spad_az0", C.c_double), ("spad_el0", C.c_double), ("spad_d_el", C.c_double),
        ("track", C.c_int32), ("angles", C.POINTER(C.c_double)),
    ]


def prop_params(central=0, j2=False, sun3=False, srp=False, attitude=0, q=(1.0, 0.0, 0.0, 0.0),
                epoch_mjd_tt=61041.0, mass=1000.0, N=64, bounces=1, P0=4.56e-6, eps_rel=1e-9, method=0,
                rtol=1e-12, atol_pos=1e-6, atol_vel=1e-9, h0=60.0, h_min=1e-6, h_max=0.0, max_steps=10_000_000,
                spad=None, angles=None, offsets=None):
    """spad = (grid, table): the SRP force comes from the SPAD interpolant
    (spad_interp) of `table` instead of the ray tracer.  Joints track the Sun
    unless commanded `angles` or tracking `offsets` (one per part) are given."""
    pp = Prop(central, int(j2), int(sun3), int(srp), attitude, (C.c_double * 4)(*q), epoch_mjd_tt, mass, N,
              bounces, P0, eps_rel, method, rtol, atol_pos, atol_vel, h0, h_min, h_max, max_steps)
    pp.track = 1
    if angles is not None or offsets is not None:
        if angles is not None and offsets is not None:
            raise ValueError("give commanded angles or tracking offsets, not both")
        a = np.ascontiguousarray(np.asarray(angles if offsets is None else offsets, np.float64).ravel())
        pp._angles_keep = a
        pp.angles = _dp(a)
        pp.track = 0 if offsets is None else 2
    if spad is not None:
        g, tab = spad
        tab = np.ascontiguousarray(np.asarray(tab, np.float64).reshape(g["n_el"], g["n_az"], 6))
        pp._spad_keep = tab
        pp.spad_table = _dp(tab)
        pp.spad_n_az, pp.spad_n_el = g["n_az"], g["n_el"]
        pp.spad_az0, pp.spad_el0, pp.spad_d_el = g["az0"], g["el0"], g["d_el"]
    return pp


def rkf78_tableau():
    c, a, b7, b8 = np.zeros(13), np.zeros(169), np.zeros(13), np.zeros(13)
    lib().orc_rkf78_tableau(_dp(c), _dp(a), _dp(b7), _dp(b8))
    return c, a.reshape(13, 13), b7, b8


def sun_position(mjd_tt):
    r = np.zeros(3)
    lib().orc_sun_position(C.c_double(mjd_tt), _dp(r))
    return r


def attitude(pp, y):
    R = np.zeros(9)
    y = np.ascontiguousarray(np.asarray(y, np.float64))
    lib().orc_attitude(C.byref(pp), _dp(y), _dp(R))
    return R.reshape(3, 3)


def accel(mesh, pp, t, y):
    """(a [3], aux [8]) with aux = Sun dir body, Sun distance AU, shadow flag, F_body."""
    om = OMesh(mesh) if mesh is not None else None
    y = np.ascontiguousarray(np.asarray(y, np.float64))
    a, aux = np.zeros(3), np.zeros(8)
    rc = lib().orc_accel(C.byref(om.s) if om else None, C.byref(pp), C.c_double(t), _dp(y), _dp(a), _dp(aux))
    if rc != 0:
        raise ValueError(f"orc_accel failed: {rc}")
    return a, aux


def propagate(mesh, pp, t0, t1, y0, h_cap=1_000_000, h_replay=None):
    """Propagate y0 over [t0, t1].  Returns (y1, stats[acc, rej, evals], h_log)."""
    om = OMesh(mesh) if mesh is not None else None
    y0 = np.ascontiguousarray(np.asarray(y0, np.float64))
    y1 = np.zeros(6)
    stats = np.zeros(3, np.int64)
    hlog = np.zeros(h_cap)
    hr = None if h_replay is None else np.ascontiguousarray(np.asarray(h_replay, np.float64))
    rc = lib().orc_propagate(C.byref(om.s) if om else None, C.byref(pp), C.c_double(t0), C.c_double(t1), _dp(y0),
                             _dp(y1), stats.ctypes.data_as(C.POINTER(C.c_int64)), _dp(hlog), C.c_int64(h_cap),
                             _dp(hr) if hr is not None else None, C.c_int64(0 if hr is None else len(hr)))
    if rc != 0:
        raise ValueError(f"orc_propagate failed: {rc}")
    return y1, stats, hlog[: min(int(stats[0]), h_cap)]


# ------------------------------------------------ frozen-hit RK4 arc gradients
def _arc(mesh, pp, t0, t1, y0, record, rec, track, angles, om=None):
    om = om or (OMesh(mesh) if mesh is not None else None)
    y0 = np.ascontiguousarray(np.asarray(y0, np.float64))
    y1 = np.zeros(6)
    nst = np.zeros(1, np.int64)
    a = None if angles is None else np.ascontiguousarray(np.asarray(angles, np.float64))
    hits, ids, lit = rec["hits"], rec["ids"], rec["lit"]
    rc = lib().orc_rk4_arc(C.byref(om.s) if om else None, C.byref(pp), C.c_int32(track), _dp(a) if a is not None else None,
                           C.c_double(t0), C.c_double(t1), _dp(y0), C.c_int32(record), _ip(hits), _ip(ids), _ip(lit),
                           C.c_int64(len(lit)), _dp(y1), nst.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc != 0:
        raise ValueError(f"orc_rk4_arc failed: {rc}")
    return y1, int(nst[0])


def _arc_mode(offsets, angles):
    if offsets is not None and angles is not None:
        raise ValueError("give commanded angles or tracking offsets, not both")
    if angles is not None:
        return 0, angles
    if offsets is not None:
        return 2, offsets
    return 1, None


def rk4_arc_record(mesh, pp, t0, t1, y0, offsets=None, angles=None):
    """Fixed-step RK4 arc (pp.method must be 1) with the traced SRP in every
    stage, recording each stage's hit set, window vertices and lit flag.
    Returns (y1, record)."""
    n_steps = int(math.ceil((t1 - t0) / pp.h0 - 1e-9))
    cap = 4 * max(n_steps, 1) + 4
    rays = pp.N * pp.N
    rec = dict(hits=np.full((cap, rays, pp.bounces + 1), -1, np.int32), ids=np.zeros((cap, 4), np.int32),
               lit=np.zeros(cap, np.int32))
    track, a = _arc_mode(offsets, angles)
    y1, _ = _arc(mesh, pp, t0, t1, y0, 1, rec, track, a)
    return y1, rec


def rk4_arc_frozen(mesh, pp, t0, t1, y0, rec, offsets=None, angles=None, mat=None, _om=None):
    """The same arc with every SRP evaluation replaced by F_H on the record;
    `mat` [M, 2] replaces the optical coefficients when given."""
    om = _om or OMesh(mesh)
    if mat is not None:
        keepm = np.ascontiguousarray(np.asarray(mat, np.float64).reshape(-1, 2))
        om2 = OMesh.__new__(OMesh)
        om2.keep = dict(om.keep, mat=keepm)
        om2.n_parts = om.n_parts
        om2.s = _Mesh.from_buffer_copy(om.s)
        om2.s.mat = _dp(keepm)
        om = om2
    track, a = _arc_mode(offsets, angles)
    return _arc(mesh, pp, t0, t1, y0, 0, rec, track, a, om=om)[0]


def arc_frozen_grad(mesh, pp, t0, t1, y0, lam, offsets=None, angles=None, h=1e-6, h_pos=1.0, h_vel=1e-3):
    """Reference gradient of L = lam . y1 for an RK4 arc with every SRP
    evaluation frozen at the hit sets of the base arc: central differences
    with step h in each optical coefficient, joint parameter and quaternion
    component (pp.q), and steps h_pos (m) / h_vel (m/s) in the initial state.
    Returns dict(y0 [6], mat [M, 2], angle [P], q [4], y1 [6], record)."""
    om = OMesh(mesh)
    P = om.n_parts
    if offsets is None and angles is None:
        offsets = np.zeros(P)
    lam = np.asarray(lam, np.float64)
    y0 = np.asarray(y0, np.float64)
    y1, rec = rk4_arc_record(mesh, pp, t0, t1, y0, offsets=offsets, angles=angles)

    def L(y0_=y0, pp_=pp, off=offsets, ang=angles, mat=None):
        return float(lam @ rk4_arc_frozen(mesh, pp_, t0, t1, y0_, rec, offsets=off, angles=ang, mat=mat, _om=om))

    g_y0 = np.zeros(6)
    for i in range(6):
        e = np.zeros(6)
        e[i] = h_pos if i < 3 else h_vel
        g_y0[i] = (L(y0_=y0 + e) - L(y0_=y0 - e)) / (2 * e[i])
    mat0 = np.asarray(mesh.mat, np.float64).reshape(-1, 2)
    g_mat = np.zeros_like(mat0)
    for i in range(mat0.shape[0]):
        for c in range(2):
            mp, mm = mat0.copy(), mat0.copy()
            mp[i, c] += h
            mm[i, c] -= h
            g_mat[i, c] = (L(mat=mp) - L(mat=mm)) / (2 * h)
    g_ang = np.zeros(P)
    for q in range(P):
        base = np.array(angles if angles is not None else offsets, np.float64)
        bp, bm = base.copy(), base.copy()
        bp[q] += h
        bm[q] -= h
        if angles is not None:
            g_ang[q] = (L(ang=bp) - L(ang=bm)) / (2 * h)
        else:
            g_ang[q] = (L(off=bp) - L(off=bm)) / (2 * h)
    g_q = np.zeros(4)
    for c in range(4):
        qp, qm = Prop.from_buffer_copy(pp), Prop.from_buffer_copy(pp)
        qp.q[c] += h
        qm.q[c] -= h
        g_q[c] = (L(pp_=qp) - L(pp_=qm)) / (2 * h)
    return dict(y0=g_y0, mat=g_mat, angle=g_ang, q=g_q, y1=y1, record=rec)


# ---------------------------------------------- SPAD interpolation (Sec. 4.2)
def spad_dirs(grid):
    """Body-frame Sun directions of the SPAD samples, [n_el][n_az][3]."""
    n_az, n_el = grid["n_az"], grid["n_el"]
    out = np.zeros((n_el, n_az, 3))
    for j in range(n_el):
        for i in range(n_az):
            s = np.zeros(3)
            lib().orc_spad_dir(C.c_int32(n_az), C.c_double(grid["az0"]), C.c_double(grid["el0"]),
                               C.c_double(grid["d_el"]), C.c_int32(i), C.c_int32(j), _dp(s))
            out[j, i] = s
    return out


def spad_table(mesh, grid, N, bounces=1, P0=4.56e-6, eps_rel=1e-9, procs=1):
    """The SPAD table: force and torque of `evaluate` at 1 AU for every
    sample direction, [n_el][n_az][6]."""
    d = spad_dirs(grid)
    tab = np.zeros(d.shape[:2] + (6,))
    for j in range(d.shape[0]):
        for i in range(d.shape[1]):
            r = evaluate(mesh, d[j, i], N, bounces, P0=P0, dist_au=1.0, eps_rel=eps_rel, procs=procs)
            tab[j, i, :3], tab[j, i, 3:] = r["F"], r["T"]
    return tab


def spad_interp(grid, table, s, dist_au=1.0):
    """Bilinear SPAD interpolant at body-frame direction s: [F (3), T (3)]."""
    tab = np.ascontiguousarray(np.asarray(table, np.float64).reshape(grid["n_el"], grid["n_az"], 6))
    s = np.ascontiguousarray(np.asarray(s, np.float64))
    out = np.zeros(6)
    rc = lib().orc_spad_interp(C.c_int32(grid["n_az"]), C.c_int32(grid["n_el"]), C.c_double(grid["az0"]),
                               C.c_double(grid["el0"]), C.c_double(grid["d_el"]), _dp(tab), _dp(s),
                               C.c_double(dist_au), _dp(out))
    if rc != 0:
        raise ValueError(f"orc_spad_interp failed: {rc}")
    return out


# ------------------------------------------- diffuse secondary rays (Sec. 6.1)
def splitmix64(seed, c):
    """Output number c (from 0) of the oracle's SplitMix64 stream for `seed`."""
    return int(lib().orc_splitmix64(C.c_uint64(seed), C.c_uint64(c)))


def diffuse_dir(seed, c, nf):
    """The oracle's cosine-weighted diffuse direction for sample counter c
    about unit normal nf."""
    nf = np.ascontiguousarray(np.asarray(nf, np.float64))
    w = np.zeros(3)
    lib().orc_diffuse_dir(C.c_uint64(seed), C.c_uint64(c), _dp(nf), _dp(w))
    return w
