"""Pins of the oracle's edge-proximity output against closed forms.

The parity tests forgive a GPU/oracle hit-id mismatch only on rays whose
oracle edge proximity is below 1e-6 of the window diagonal (the north-star
bar "within 1e-6 relative of an edge", read as: the distance, in the plane
normal to the ray, from the ray to the boundary of any triangle it reaches no
later than its hit).  Those distances are checked here against geometry worked
out without the oracle's code:

* a right triangle seen face-on: the distance from a pixel centre to its
  boundary is min(x, y, (1 - x/a - y/b) a b / sqrt(a^2 + b^2)) in the legs'
  frame, inside and outside the triangle;
* the same triangle tilted by alpha about a leg: the distance is measured in
  the plane normal to the ray, so the other leg shrinks to b cos(alpha) (a
  distance measured in the triangle's own plane would not);
* triangles beyond the hit do not count, triangles before it do (the t window);
* a second triangle at the hit's depth within the tolerance makes the
  distance zero (a tie), one farther than the tolerance does not.

The pixel centres come from the window definition (tight bounds on the basis
of Duff et al. 2017 around d, centres at (i + 1/2) / N of the extent).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

S_UP = np.array([0.0, 0.0, 1.0])  # photons travel along -z


def mesh_of(tris, mats=((0.2, 0.1),)):
    """Single rigid part; every triangle its own three vertices."""
    xyz = np.asarray(tris, np.float64).reshape(-1, 3)
    n = len(xyz) // 3
    return I.Mesh(xyz, np.arange(3 * n, dtype=np.int32).reshape(n, 3), np.zeros(n, np.int32),
                  np.zeros((n, 2), np.int32), np.asarray(mats, np.float64), **I._parts(1, [-1]))


def onb(n):
    """The window's basis convention (Duff et al., JCGT 6(1), 2017)."""
    sg = math.copysign(1.0, n[2])
    a = -1.0 / (sg + n[2])
    b = n[0] * n[1] * a
    return (np.array([1.0 + sg * n[0] ** 2 * a, sg * b, -sg * n[0]]),
            np.array([b, sg + n[1] ** 2 * a, -n[1]]))


def pixel_xy(win, N, s):
    """World (x, y) of every pixel centre, ray order r = i N + j (s along z, so
    the plane normal to the ray is the xy plane)."""
    u, v = onb(-np.asarray(s))
    c = (np.arange(N) + 0.5) / N
    uc = win[0] + c * (win[1] - win[0])
    vc = win[2] + c * (win[3] - win[2])
    P = uc[:, None, None] * u + vc[None, :, None] * v
    return P[..., 0].reshape(-1), P[..., 1].reshape(-1)


def right_tri_dist(x, y, a, b):
    """Distance from (x, y), inside the box [0, a] x [0, b], to the boundary of
    the right triangle (0, 0), (a, 0), (0, b): the legs' feet and the
    hypotenuse's foot all fall on the segments there."""
    hyp = np.abs(x / a + y / b - 1.0) * a * b / math.hypot(a, b)
    return np.minimum(np.minimum(np.abs(x), np.abs(y)), hyp)


def seg_dist(px, py, ax, ay, bx, by):
    """Point-segment distance by rotating the segment onto the x axis."""
    L = math.hypot(bx - ax, by - ay)
    c, s = (bx - ax) / L, (by - ay) / L
    qx = (px - ax) * c + (py - ay) * s       # along the segment
    qy = -(px - ax) * s + (py - ay) * c      # across it
    inside = (qx >= 0.0) & (qx <= L)
    return np.where(inside, np.abs(qy), np.minimum(np.hypot(qx, qy), np.hypot(qx - L, qy)))


def tri_boundary_dist(px, py, t):
    (ax, ay), (bx, by), (cx, cy) = t
    return np.minimum(np.minimum(seg_dist(px, py, ax, ay, bx, by), seg_dist(px, py, bx, by, cx, cy)),
                      seg_dist(px, py, cx, cy, ax, ay))


def edges(mesh, N, s=S_UP):
    r = O.evaluate(mesh, s, N, bounces=0, want_hits=True, want_edge=True)
    return r, r["edge"][:, 0], r["hits"][:, 0]


@pytest.mark.parametrize("a,b", [(1.0, 1.0), (2.0, 0.7)])
def test_face_on_right_triangle(a, b):
    m = mesh_of([[0, 0, 0], [a, 0, 0], [0, b, 0]])
    N = 37
    r, e, h = edges(m, N)
    x, y = pixel_xy(r["win"], N, S_UP)
    want = right_tri_dist(x, y, a, b)
    assert np.max(np.abs(e - want)) < 1e-12 * (a + b)
    inside = x / a + y / b < 1.0
    assert inside.any() and (~inside).any()          # both kinds of pixel are covered
    clear = want > 1e-9                              # centres on an edge count as inside (R6)
    assert np.array_equal((h >= 0)[clear], inside[clear])


@pytest.mark.parametrize("alpha", [0.3, 1.0, 1.3])
def test_distance_is_measured_normal_to_the_ray(alpha):
    a, b = 1.5, 1.0
    m = mesh_of([[0, 0, 0], [a, 0, 0], [0, b * math.cos(alpha), b * math.sin(alpha)]])
    N = 41
    r, e, _ = edges(m, N)
    x, y = pixel_xy(r["win"], N, S_UP)
    want = right_tri_dist(x, y, a, b * math.cos(alpha))
    assert np.max(np.abs(e - want)) < 1e-12 * (a + b)
    # the in-plane distance differs: a reading in the triangle's plane fails here
    in_plane = right_tri_dist(x, y / math.cos(alpha), a, b)
    assert np.max(np.abs(in_plane - want)) > 1e-2


def test_triangles_beyond_the_hit_do_not_count():
    a, b = 2.0, 1.6
    big = [[0, 0, 0], [a, 0, 0], [0, b, 0]]
    front = [(0.15 * a, 0.1 * b), (0.55 * a, 0.1 * b), (0.15 * a, 0.45 * b)]   # z = +0.3, before
    back = [(0.2 * a, 0.5 * b), (0.45 * a, 0.5 * b), (0.2 * a, 0.75 * b)]     # z = -0.3, beyond
    m = mesh_of(big + [[x, y, 0.3] for x, y in front] + [[x, y, -0.3] for x, y in back])
    N = 64
    r, e, h = edges(m, N)
    x, y = pixel_xy(r["win"], N, S_UP)
    d_big = right_tri_dist(x, y, a, b)
    d_front = tri_boundary_dist(x, y, front)
    d_back = tri_boundary_dist(x, y, back)
    want = np.where(h == 1, d_front,                                  # the small front triangle is hit
           np.where(h == 0, np.minimum(d_big, d_front),               # big plate hit: the front one is before it
                    np.minimum(np.minimum(d_big, d_front), d_back)))  # a miss: everything ahead counts
    assert (h == 0).any() and (h == 1).any() and (h == -1).any() and not (h == 2).any()
    assert np.max(np.abs(e - want)) < 1e-12 * (a + b)
    # the back triangle's edges are near many rays that stop on the big plate first
    on_big = h == 0
    assert (d_back[on_big] < want[on_big] - 1e-3).sum() > 20


def test_tie_within_tolerance_is_zero():
    a, b = 1.2, 1.0
    N = 33
    base = [[0, 0, 0], [a, 0, 0], [0, b, 0]]
    # the window's diagonal of the face-on scene (flat: no depth extent)
    L = math.hypot(a, b)
    for dz, tie in ((0.0, True), (-0.4e-6 * L, True), (-5e-6 * L, False)):
        m = mesh_of(base + [[x, y, dz] for x, y, _ in base])
        r, e, h = edges(m, N)
        x, y = pixel_xy(r["win"], N, S_UP)
        d = right_tri_dist(x, y, a, b)
        hit = h >= 0
        assert hit.any() and (~hit).any()
        assert np.array_equal(h[hit], np.zeros(hit.sum(), np.int32))   # ties go to the lower id
        if tie:
            assert np.all(e[hit] == 0.0)
        else:
            assert np.max(np.abs(e[hit] - d[hit])) < 1e-12          # farther than tol: beyond the hit
        # a ray that misses both still sees the nearer boundary
        assert np.max(np.abs(e[~hit] - d[~hit])) < 1e-12


def test_flagged_rays_are_a_thin_band():
    # On a face-on plate the rays flagged by the 1e-6 L test are exactly the
    # pixel centres within 1e-6 L of an edge (here: none unless placed there).
    a, b = 1.0, 1.0
    N = 40   # centres at (k + 1/2) / 40: the hypotenuse x + y = 1 holds no centre
    m = mesh_of([[0, 0, 0], [a, 0, 0], [0, b, 0]])
    r, e, _ = edges(m, N)
    L = r["win"][6]
    x, y = pixel_xy(r["win"], N, S_UP)
    assert np.array_equal(e < 1e-6 * L, right_tri_dist(x, y, a, b) < 1e-6 * L)
    # N odd puts centres exactly on the hypotenuse ((k + 1/2)/N + (N - k - 1/2)/N = 1)
    N = 41
    r, e, h = edges(m, N)
    x, y = pixel_xy(r["win"], N, S_UP)
    on = np.abs(x + y - 1.0) < 1e-12
    assert on.sum() >= N - 1
    assert np.all(e[on] < 1e-6 * r["win"][6])
