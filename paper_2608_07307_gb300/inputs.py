"""Seeded synthetic inputs: spacecraft meshes, Sun directions, test scenes.

This module is the one piece shared by the oracle harness (``oracle/``), the
tests and ``bench.py``.  It only lays out geometry and draws numbers; it holds
none of the method's arithmetic (no posing, no ray tracing, no force law).

The paper's own meshes (Parker Solar Probe, 39 257 triangles, and a GPS-like
BoxWing, 212 triangles; Sec. 5.1, Table 1) are not available, so the
spacecraft here are procedural stand-ins of the same kind: a bus, a dish and
two articulated solar-array wings with front/back materials.

Mesh conventions (the C ABI's ``srp_mesh_desc`` uses the same arrays):
  xyz       (V, 3) float64 or float32  rest pose, body frame, metres
  tri       (T, 3) int32               counter-clockwise seen from the front
  tri_part  (T,)   int32               rigid part of each triangle
  tri_mat   (T, 2) int32               material of the front / back side
  mat       (M, 2) float64             rho_s, rho_d per material
  parent    (P,)   int32               kinematic tree (Sec. 4.4.1); -1 = root
  pivot     (P, 3) float64             joint pivot, rest body frame
  axis      (P, 3) float64             unit joint axis, zero for a rigid link
  limits    (P, 2) float64             admissible joint interval (rad)
  normal0   (P, 3) float64             rest front normal of a panel part
  c_ref     (3,)   float64             torque reference point
  mass      float                      kg
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "splitmix64", "uniform01", "sun_dirs_uniform", "sun_dirs_fibonacci",
    "box_wing", "box_wing_two_axis", "spacecraft", "flat_plate", "two_plates", "box", "icosphere",
    "v_trough", "random_soup", "merge", "spad_grid", "SPAD_20x10", "SPAD_20x10S",
]

_MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) from `seed`."""
    out = np.empty(n, dtype=np.uint64)
    x = seed & _MASK
    for k in range(n):
        x = (x + 0x9E3779B97F4A7C15) & _MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out[k] = z ^ (z >> 31)
    return out


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of SplitMix64 outputs."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sun_dirs_uniform(n: int, seed: int = 0) -> np.ndarray:
    """n unit vectors uniform on the sphere: z = 2 u1 - 1, phi = 2 pi u2."""
    u = uniform01(seed, 2 * n).reshape(n, 2)
    z = 2.0 * u[:, 0] - 1.0
    phi = 2.0 * math.pi * u[:, 1]
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def spad_grid(n_az: int, n_el: int, az0_deg: float, el0_deg: float, d_el_deg: float | None = None) -> dict:
    """A SPAD sampling grid (Sec. 4.2, Sec. 6.1): n_az azimuths from az0, spaced
    360/n_az degrees around the circle, and n_el elevations from el0, spaced
    d_el (default 180/n_el) degrees.  Angles in radians in the result."""
    d_el = 180.0 / n_el if d_el_deg is None else d_el_deg
    return {"n_az": int(n_az), "n_el": int(n_el), "az0": math.radians(az0_deg), "el0": math.radians(el0_deg),
            "d_el": math.radians(d_el)}


# the two tables of the paper's comparison: from (-180, -90) degrees, and
# shifted by 5 degrees on both axes (no sample at 0 degrees elevation)
SPAD_20x10 = spad_grid(20, 10, -180.0, -90.0)
SPAD_20x10S = spad_grid(20, 10, -175.0, -85.0)


def sun_dirs_fibonacci(n: int) -> np.ndarray:
    """Fibonacci sphere: z_i = 1 - (2i+1)/n, phi_i = i pi (3 - sqrt 5)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


@dataclass
class Mesh:
    xyz: np.ndarray
    tri: np.ndarray
    tri_part: np.ndarray
    tri_mat: np.ndarray
    mat: np.ndarray
    parent: np.ndarray
    pivot: np.ndarray
    axis: np.ndarray
    limits: np.ndarray
    normal0: np.ndarray
    c_ref: np.ndarray = field(default_factory=lambda: np.zeros(3))
    mass: float = 1.0
    name: str = "mesh"

    @property
    def n_tris(self) -> int:
        return int(self.tri.shape[0])

    def with_materials(self, mat) -> "Mesh":
        m = Mesh(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        m.mat = np.ascontiguousarray(np.asarray(mat, dtype=np.float64).reshape(-1, 2))
        return m

    def as_float32(self) -> "Mesh":
        m = Mesh(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        m.xyz = np.ascontiguousarray(self.xyz.astype(np.float32))
        return m


# ------------------------------------------------------------------ builders
class _Builder:
    """Accumulates triangles part by part; vertices are never shared by parts."""

    def __init__(self):
        self.v, self.t, self.tp, self.tm = [], [], [], []
        self.nv = 0

    def add(self, verts, tris, part, mat_front, mat_back):
        verts = np.asarray(verts, dtype=np.float64).reshape(-1, 3)
        tris = np.asarray(tris, dtype=np.int64).reshape(-1, 3) + self.nv
        self.v.append(verts)
        self.t.append(tris)
        self.tp.append(np.full(len(tris), part, np.int32))
        self.tm.append(np.tile(np.array([[mat_front, mat_back]], np.int32), (len(tris), 1)))
        self.nv += len(verts)

    def arrays(self):
        return (np.ascontiguousarray(np.concatenate(self.v)),
                np.ascontiguousarray(np.concatenate(self.t).astype(np.int32)),
                np.ascontiguousarray(np.concatenate(self.tp)),
                np.ascontiguousarray(np.concatenate(self.tm)))


def _grid(origin, eu, ev, nu, nv):
    """Quad grid origin + a eu/nu + b ev/nv, two triangles per cell, front = eu x ev."""
    origin, eu, ev = (np.asarray(x, np.float64) for x in (origin, eu, ev))
    a = np.arange(nu + 1) / nu
    b = np.arange(nv + 1) / nv
    verts = origin + a[:, None, None] * eu + b[None, :, None] * ev
    verts = verts.reshape(-1, 3)
    idx = lambda i, j: i * (nv + 1) + j  # noqa: E731
    tris = []
    for i in range(nu):
        for j in range(nv):
            p00, p10, p11, p01 = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris.append((p00, p10, p11))
            tris.append((p00, p11, p01))
    return verts, np.array(tris, np.int64)


def _box_faces(lo, hi, h):
    """Six outward-facing subdivided faces of the box [lo, hi] with facet ~h."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    ext = hi - lo
    n = lambda L: max(1, int(round(L / h))) if h else 1  # noqa: E731
    X, Y, Z = np.eye(3)
    faces = [
        ((hi[0], lo[1], lo[2]), Y * ext[1], Z * ext[2], n(ext[1]), n(ext[2])),   # +x
        ((lo[0], lo[1], lo[2]), Z * ext[2], Y * ext[1], n(ext[2]), n(ext[1])),   # -x
        ((lo[0], hi[1], lo[2]), Z * ext[2], X * ext[0], n(ext[2]), n(ext[0])),   # +y
        ((lo[0], lo[1], lo[2]), X * ext[0], Z * ext[2], n(ext[0]), n(ext[2])),   # -y
        ((lo[0], lo[1], hi[2]), X * ext[0], Y * ext[1], n(ext[0]), n(ext[1])),   # +z
        ((lo[0], lo[1], lo[2]), Y * ext[1], X * ext[0], n(ext[1]), n(ext[0])),   # -z
    ]
    out = []
    for o, eu, ev, nu, nv in faces:
        out.append(_grid(o, eu, ev, nu, nv))
    return out


def _add_box(b: _Builder, lo, hi, h, part, mf, mb):
    for verts, tris in _box_faces(lo, hi, h):
        b.add(verts, tris, part, mf, mb)


def _parts(n, parent, pivot=None, axis=None, limits=None, normal0=None):
    pv = np.zeros((n, 3)) if pivot is None else np.asarray(pivot, np.float64).reshape(n, 3)
    ax = np.zeros((n, 3)) if axis is None else np.asarray(axis, np.float64).reshape(n, 3)
    lm = np.tile([[-math.pi, math.pi]], (n, 1)) if limits is None else np.asarray(limits, np.float64).reshape(n, 2)
    n0 = np.tile([[0.0, 0.0, 1.0]], (n, 1)) if normal0 is None else np.asarray(normal0, np.float64).reshape(n, 3)
    return dict(parent=np.asarray(parent, np.int32), pivot=np.ascontiguousarray(pv), axis=np.ascontiguousarray(ax),
                limits=np.ascontiguousarray(lm), normal0=np.ascontiguousarray(n0))


# -------------------------------------------------------------- spacecraft
def box_wing() -> Mesh:
    """Small box-wing spacecraft, FP64 vertices, 16 triangles.

    Bus: 1 m cube centred at the origin, one quad per face (12 triangles),
    rho_s = 0.1, rho_d = 0.2 on both sides.  Two 2 x 1 m flat panels (2
    triangles each) along +y and -y, inner edge at |y| = 0.75 m, rest front
    normal +z; front rho_s = rho_d = 0.05, back rho_s = 0, rho_d = 0.1.  Each
    panel turns about the body y axis through its inner-edge pivot with an
    unrestricted interval (-pi, pi].  Mass 2269 kg (the paper's BoxWing dry
    mass, Sec. 5.1).
    """
    b = _Builder()
    _add_box(b, (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), None, 0, 0, 0)
    b.add(*_grid((-0.5, 0.75, 0.0), (1.0, 0, 0), (0, 2.0, 0), 1, 1), 1, 1, 2)
    b.add(*_grid((-0.5, -2.75, 0.0), (1.0, 0, 0), (0, 2.0, 0), 1, 1), 2, 1, 2)
    xyz, tri, tp, tm = b.arrays()
    mat = np.array([[0.1, 0.2], [0.05, 0.05], [0.0, 0.1]])
    parts = _parts(3, [-1, 0, 0], pivot=[[0, 0, 0], [0, 0.75, 0], [0, -0.75, 0]],
                   axis=[[0, 0, 0], [0, 1, 0], [0, 1, 0]])
    return Mesh(xyz, tri, tp, tm, mat, c_ref=np.zeros(3), mass=2269.0, name="box_wing", **parts)


def box_wing_two_axis() -> Mesh:
    """The box-wing with a two-axis array drive per wing (Sec. 9): a yoke
    (a 0.1 m square strut, bus material, from y = 0.51 to 0.74 m) turns about
    the body y axis within +-90 degrees and carries the 2 x 1 m panel, which
    folds about the x axis through its inner edge (|y| = 0.75 m) within +-45
    degrees.  Both joints track the Sun with reference normal +z.  Parts: bus,
    yoke +y, yoke -y, panel +y, panel -y; 40 triangles; mass 2269 kg.
    """
    b = _Builder()
    _add_box(b, (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), None, 0, 0, 0)
    _add_box(b, (-0.05, 0.51, -0.05), (0.05, 0.74, 0.05), None, 1, 0, 0)
    _add_box(b, (-0.05, -0.74, -0.05), (0.05, -0.51, 0.05), None, 2, 0, 0)
    b.add(*_grid((-0.5, 0.75, 0.0), (1.0, 0, 0), (0, 2.0, 0), 1, 1), 3, 1, 2)
    b.add(*_grid((-0.5, -2.75, 0.0), (1.0, 0, 0), (0, 2.0, 0), 1, 1), 4, 1, 2)
    xyz, tri, tp, tm = b.arrays()
    mat = np.array([[0.1, 0.2], [0.05, 0.05], [0.0, 0.1]])
    half, quarter = math.pi / 2, math.pi / 4
    parts = _parts(5, [-1, 0, 0, 1, 2],
                   pivot=[[0, 0, 0], [0, 0.5, 0], [0, -0.5, 0], [0, 0.75, 0], [0, -0.75, 0]],
                   axis=[[0, 0, 0], [0, 1, 0], [0, 1, 0], [1, 0, 0], [1, 0, 0]],
                   limits=[[-math.pi, math.pi], [-half, half], [-half, half], [-quarter, quarter],
                           [-quarter, quarter]])
    return Mesh(xyz, tri, tp, tm, mat, c_ref=np.zeros(3), mass=2269.0, name="box_wing_two_axis", **parts)


def spacecraft(h: float = 0.05, seed: int = 0) -> Mesh:
    """Procedural complex spacecraft, FP32 vertices.

    At h = 0.05 m: bus 2 x 2 x 3 m box in 0.05 m facets (25 600 triangles); a
    3 m paraboloid dish, f/D = 0.4, 128 azimuth x 64 radial rings (16 256);
    two 8 x 2.5 m wings meshed as a 0.1 m cell lattice (4 000 each) with four
    perimeter frame struts and a yoke (12 triangles each, not subdivided).
    About 50k triangles; h = 0.025 gives about 200k.  Four materials with
    rho_s, rho_d drawn from SplitMix64(seed) in [0, 0.5]: 0 bus/struts/dish
    back, 1 dish front, 2 wing front, 3 wing back.  Parts: 0 bus (root),
    1 dish (rigid link), 2 / 3 wings turning about body y through (0, +-1, 0).
    Mass 555 kg (the paper's Parker Solar Probe dry mass, Sec. 5.1).
    """
    b = _Builder()
    _add_box(b, (-1.0, -1.0, -1.5), (1.0, 1.0, 1.5), h, 0, 0, 0)
    # dish: z = z0 + rho^2 / (4 f), concave (front) side facing +z
    n_az = max(8, int(round(128 * 0.05 / h)))
    n_rad = max(2, int(round(64 * 0.05 / h)))
    f, R, z0 = 1.2, 1.5, 1.6
    verts = [(0.0, 0.0, z0)]
    for k in range(1, n_rad + 1):
        rho = R * k / n_rad
        for a in range(n_az):
            phi = 2.0 * math.pi * a / n_az
            verts.append((rho * math.cos(phi), rho * math.sin(phi), z0 + rho * rho / (4.0 * f)))
    ring = lambda k, a: 1 + (k - 1) * n_az + (a % n_az)  # noqa: E731
    tris = [(0, ring(1, a), ring(1, a + 1)) for a in range(n_az)]
    for k in range(1, n_rad):
        for a in range(n_az):
            tris.append((ring(k, a), ring(k + 1, a), ring(k + 1, a + 1)))
            tris.append((ring(k, a), ring(k + 1, a + 1), ring(k, a + 1)))
    b.add(np.array(verts), np.array(tris), 1, 1, 0)
    # wings
    cell = 2.0 * h
    for part, sgn in ((2, 1.0), (3, -1.0)):
        y0, y1 = (1.5, 9.5) if sgn > 0 else (-9.5, -1.5)
        nu, nv = max(1, int(round(2.5 / cell))), max(1, int(round(8.0 / cell)))
        b.add(*_grid((-1.25, y0, 0.0), (2.5, 0, 0), (0, 8.0, 0), nu, nv), part, 2, 3)
        s1, s2 = 0.02, 0.015
        _add_box(b, (-1.25 - s1, y0 - s1, -s1), (-1.25 + s1, y1 + s1, s1), None, part, 0, 0)
        _add_box(b, (1.25 - s1, y0 - s1, -s1), (1.25 + s1, y1 + s1, s1), None, part, 0, 0)
        _add_box(b, (-1.25, y0 - s2, -s2), (1.25, y0 + s2, s2), None, part, 0, 0)
        _add_box(b, (-1.25, y1 - s2, -s2), (1.25, y1 + s2, s2), None, part, 0, 0)
        ylo, yhi = (0.98, 1.5) if sgn > 0 else (-1.5, -0.98)
        _add_box(b, (-0.03, ylo, -0.03), (0.03, yhi, 0.03), None, part, 0, 0)
    xyz, tri, tp, tm = b.arrays()
    mat = (0.5 * uniform01(seed, 8)).reshape(4, 2)
    parts = _parts(4, [-1, 0, 0, 0], pivot=[[0, 0, 0], [0, 0, 0], [0, 1.0, 0], [0, -1.0, 0]],
                   axis=[[0, 0, 0], [0, 0, 0], [0, 1, 0], [0, 1, 0]])
    return Mesh(xyz.astype(np.float32), tri, tp, tm, mat, c_ref=np.zeros(3), mass=555.0,
                name=f"spacecraft_h{h:g}", **parts)


# ------------------------------------------------------------- test scenes
def _single_part(b: _Builder, mat, name, c_ref=(0, 0, 0)) -> Mesh:
    xyz, tri, tp, tm = b.arrays()
    return Mesh(xyz, tri, tp, tm, np.asarray(mat, np.float64).reshape(-1, 2), c_ref=np.asarray(c_ref, np.float64),
                name=name, **_parts(1, [-1]))


def _fan_rect(origin, eu, ev, centre=(0.4637, 0.5811)):
    """Rectangle origin + [0,1] eu + [0,1] ev as four triangles around an
    off-centre interior point, front = eu x ev.  The interior point is generic
    so that no pixel centre of a window aligned with eu, ev lies on a diagonal."""
    o, eu, ev = (np.asarray(x, np.float64) for x in (origin, eu, ev))
    c = o + centre[0] * eu + centre[1] * ev
    verts = np.array([o, o + eu, o + eu + ev, o + ev, c])
    tris = np.array([(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)])
    return verts, tris


def flat_plate(lx=2.0, ly=1.0, z=0.0, mat=((0.3, 0.2), (0.1, 0.4)), center=(0.0, 0.0)) -> Mesh:
    """Rectangle |x - cx| <= lx/2, |y - cy| <= ly/2 at height z, front normal +z,
    four triangles around a generic interior point; material 0 on the front,
    1 on the back."""
    b = _Builder()
    cx, cy = center
    b.add(*_fan_rect((cx - lx / 2, cy - ly / 2, z), (lx, 0, 0), (0, ly, 0)), 0, 0, 1)
    return _single_part(b, mat, "flat_plate")


def two_plates(lx=2.0, ly=1.0, gap=0.5, mat=((0.3, 0.2), (0.1, 0.4))) -> Mesh:
    """Two identical parallel plates, front normals +z, at z = 0 and z = -gap."""
    b = _Builder()
    b.add(*_fan_rect((-lx / 2, -ly / 2, 0.0), (lx, 0, 0), (0, ly, 0)), 0, 0, 1)
    b.add(*_fan_rect((-lx / 2, -ly / 2, -gap), (lx, 0, 0), (0, ly, 0)), 0, 0, 1)
    return _single_part(b, mat, "two_plates")


def box(lo=(-0.5, -0.5, -0.5), hi=(0.5, 0.5, 0.5), h=None, mat=((0.0, 0.0),)) -> Mesh:
    b = _Builder()
    _add_box(b, lo, hi, h, 0, 0, 0)
    return _single_part(b, mat, "box")


def icosphere(level: int = 2, radius: float = 1.0, mat=((0.0, 0.0),)) -> Mesh:
    """Icosahedron refined `level` times (each triangle split in four, new
    vertices pushed to the sphere), outward counter-clockwise faces."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b_):
            key = (min(a, b_), max(a, b_))
            if key not in cache:
                p = v[a] + v[b_]
                v.append(p / np.linalg.norm(p))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for a, b_, c in f:
            ab, bc, ca = mid(a, b_), mid(b_, c), mid(c, a)
            nf += [(a, ab, ca), (b_, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    bld = _Builder()
    bld.add(np.array(v) * radius, np.array(f), 0, 0, 0)
    return _single_part(bld, mat, f"icosphere{level}")


def v_trough(a=1.0, w=1.5, mat=((1.0, 0.0),)) -> Mesh:
    """Two plates at 90 degrees sharing the edge along y at the origin:
    z = -x for x in [-a, 0] and z = x for x in [0, a], y in [0, w], inner
    (upward) sides as fronts.  Light arriving along -z is retroreflected."""
    bld = _Builder()
    bld.add(*_fan_rect((-a, 0.0, a), (a, 0, -a), (0, w, 0)), 0, 0, 0)
    bld.add(*_fan_rect((0.0, 0.0, 0.0), (a, 0, a), (0, w, 0)), 0, 0, 0)
    return _single_part(bld, mat, "v_trough")


def random_soup(n: int, seed: int, scale=1.0, size=0.4, n_mats=3) -> Mesh:
    """n random triangles in a cube of side 2*scale (single rigid part)."""
    u = uniform01(seed, n * 9 + 2 * n_mats + 2 * n)
    c = (u[: 3 * n].reshape(n, 3) * 2.0 - 1.0) * scale
    off = (u[3 * n: 9 * n].reshape(n, 2, 3) * 2.0 - 1.0) * size * scale
    verts = np.concatenate([c[:, None, :], c[:, None, :] + off], axis=1).reshape(-1, 3)
    tris = np.arange(3 * n).reshape(n, 3)
    mats = (0.5 * u[9 * n: 9 * n + 2 * n_mats]).reshape(n_mats, 2)
    side = (u[9 * n + 2 * n_mats:] * n_mats).astype(np.int32).reshape(n, 2) % n_mats
    bld = _Builder()
    bld.add(verts, tris, 0, 0, 0)
    xyz, tri, tp, _ = bld.arrays()
    return Mesh(xyz, tri, tp, np.ascontiguousarray(side), mats, name=f"soup{n}", **_parts(1, [-1]))


def merge(meshes, joints=None) -> Mesh:
    """Concatenate single-part meshes into one multi-part mesh.  `joints` is a
    list of dicts (parent, pivot, axis, limits, normal0) per mesh, the first
    being the root; materials are concatenated."""
    bld = _Builder()
    mats = []
    moff = 0
    for k, m in enumerate(meshes):
        bld.v.append(m.xyz.astype(np.float64))
        bld.t.append(m.tri.astype(np.int64) + bld.nv)
        bld.tp.append(np.full(m.n_tris, k, np.int32))
        bld.tm.append((m.tri_mat + moff).astype(np.int32))
        bld.nv += len(m.xyz)
        mats.append(m.mat)
        moff += len(m.mat)
    xyz, tri, tp, tm = bld.arrays()
    n = len(meshes)
    joints = joints or [dict(parent=-1)] + [dict(parent=0)] * (n - 1)
    get = lambda key, dflt: [j.get(key, dflt) for j in joints]  # noqa: E731
    parts = _parts(n, get("parent", 0), get("pivot", (0, 0, 0)), get("axis", (0, 0, 0)),
                   get("limits", (-math.pi, math.pi)), get("normal0", (0, 0, 1)))
    return Mesh(xyz, tri, tp, tm, np.concatenate(mats), name="merged", **parts)
