"""Pins of the oracle's frozen-hit function F_H and of its finite-difference
gradient (the reference for the adjoint), each against something other than
F_H itself:

  * at the base point F_H equals the traced oracle (a different code path:
    Moller-Trumbore distances, search over every triangle);
  * the optical coefficients never change which triangle a ray hits (when every
    rho_s > 0), so F_H in the coefficients equals the traced oracle there; it is
    affine in rho_d and a polynomial of degree bounces + 1 in each rho_s, so a
    wide five-point stencil of traced evaluations gives the exact derivative;
  * a hinged plate that tracks the Sun has a closed form for force and torque
    (every pixel lands on the plate), so F_H's gradient in the joint offset,
    the in-plane Sun direction, the distance and the coefficients equals the
    closed form's.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

P0 = 4.56e-6


def rel(a, b, scale):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) / scale


@pytest.mark.parametrize("bounces", [0, 2])
def test_frozen_equals_traced_at_base_point(bounces):
    m = I.box_wing()
    for k, s in enumerate(I.sun_dirs_uniform(6, seed=21)):
        off = np.array([0.0, 0.13, -0.21]) if k % 2 else None
        r = O.evaluate(m, s, 48, bounces, offsets=off, want_hits=True)
        ids = O.window_ids(m, s, offsets=off)
        F, T = O.eval_frozen(m, s * 2.5, r["hits"], ids, 48, bounces, offsets=off)  # length of s is irrelevant
        fn = np.linalg.norm(r["F"])
        assert rel(F, r["F"], fn) < 1e-12
        assert rel(T, r["T"], max(np.linalg.norm(r["T"]), fn)) < 1e-12


def test_frozen_equals_traced_spacecraft():
    m = I.spacecraft(0.5)
    s = I.sun_dirs_fibonacci(7)[3]
    r = O.evaluate(m, s, 40, 2, want_hits=True)
    F, T = O.eval_frozen(m, s, r["hits"], O.window_ids(m, s), 40, 2)
    fn = np.linalg.norm(r["F"])
    assert rel(F, r["F"], fn) < 1e-12 and rel(T, r["T"], max(np.linalg.norm(r["T"]), fn)) < 1e-12


@pytest.mark.parametrize("bounces", [0, 2])
def test_material_gradient_matches_traced_polynomial(bounces):
    mat = np.array([[0.3, 0.2], [0.25, 0.15], [0.4, 0.1]])
    m = I.box_wing().with_materials(mat)
    s = I.sun_dirs_uniform(5, seed=2)[3]
    N = 40
    rng = np.random.default_rng(5)
    gF, gT = rng.normal(size=3), rng.normal(size=3)
    g = O.frozen_grad(m, s, N, bounces, gF, gT)

    def L(mm):
        r = O.evaluate(m.with_materials(mm), s, N, bounces)
        return gF @ r["F"] + gT @ r["T"]

    D = 0.05
    ref = np.zeros_like(mat)
    for i in range(mat.shape[0]):
        for c in range(2):
            f = []
            for k in (-2, -1, 1, 2):
                mm = mat.copy()
                mm[i, c] += k * D
                f.append(L(mm))
            ref[i, c] = (f[0] - 8 * f[1] + 8 * f[2] - f[3]) / (12 * D)  # exact for degree <= 4
    scale = np.max(np.abs(ref))
    assert scale > 0
    assert rel(g["mat"], ref, scale) < 1e-7, (g["mat"], ref)


def hinged_plate(w=2.0, h=1.0, y0=1.3, z0=0.4, mat=((0.35, 0.25), (0.1, 0.3))):
    """A w x h plate (front +z at rest) centred at (0, y0, 0) on a joint about
    the body y axis through (0, 0, z0); the root part holds no triangle."""
    verts, tris = I._fan_rect((-w / 2, y0 - h / 2, 0.0), (w, 0, 0), (0, h, 0))
    tri = np.ascontiguousarray(np.asarray(tris, np.int32))
    return I.Mesh(np.ascontiguousarray(verts), tri, np.ones(len(tri), np.int32),
                  np.tile(np.array([[0, 1]], np.int32), (len(tri), 1)), np.asarray(mat, np.float64),
                  **I._parts(2, [-1, 0], pivot=[[0, 0, 0], [0, 0, z0]], axis=[[0, 0, 0], [0, 1, 0]]),
                  c_ref=np.zeros(3), name="hinged_plate")


def hinged_closed_form(s, delta, dist, mat, w=2.0, h=1.0, y0=1.3, z0=0.4):
    """Force and torque on the tracking hinged plate: the joint angle is
    phi + delta (phi the Sun's azimuth about y), the lit area A cos(delta), the
    centre of pressure the plate centre rotated about the pivot."""
    s = np.asarray(s, np.float64)
    sh = s / np.linalg.norm(s)
    th = math.atan2(sh[0], sh[2]) + delta
    n = np.array([math.sin(th), 0.0, math.cos(th)])
    c = float(n @ sh)
    rs, rd = mat[0]
    F = P0 / dist ** 2 * w * h * c * ((1 - rs) * (-sh) - 2 * (rs * c + rd / 3) * n)
    p = np.array([0.0, 0.0, z0])
    q = np.array([0.0, y0, 0.0]) - p
    Rq = np.array([math.cos(th) * q[0] + math.sin(th) * q[2], q[1], -math.sin(th) * q[0] + math.cos(th) * q[2]])
    return F, np.cross(p + Rq, F)


def test_hinged_plate_gradient_matches_closed_form():
    m = hinged_plate()
    mat = np.asarray(m.mat)
    phi, delta, dist = 0.6, 0.15, 0.9
    s = np.array([math.sin(phi), 0.0, math.cos(phi)])
    N = 24
    # F_H itself equals the closed form (every pixel centre lands on the plate)
    off = np.array([0.0, delta])
    r = O.evaluate(m, s, N, 1, dist_au=dist, offsets=off, want_hits=True)
    Fc, Tc = hinged_closed_form(s, delta, dist, mat)
    assert np.all(r["hits"][:, 0] >= 0) and np.all(r["hits"][:, 1] < 0)
    assert rel(r["F"], Fc, np.linalg.norm(Fc)) < 1e-12 and rel(r["T"], Tc, np.linalg.norm(Fc)) < 1e-12
    rng = np.random.default_rng(11)
    gF, gT = rng.normal(size=3), rng.normal(size=3)
    g = O.frozen_grad(m, s, N, 1, gF, gT, dist_au=dist, offsets=off)
    h = 1e-6

    def L(s_=s, de=delta, di=dist, mm=mat):
        F, T = hinged_closed_form(s_, de, di, mm)
        return gF @ F + gT @ T

    ref_angle = (L(de=delta + h) - L(de=delta - h)) / (2 * h)
    ref_sun = [(L(s_=s + h * e) - L(s_=s - h * e)) / (2 * h) for e in np.eye(3)]
    ref_dist = (L(di=dist + h) - L(di=dist - h)) / (2 * h)
    ref_mat = np.zeros_like(mat)
    for c in range(2):
        mp, mm_ = mat.copy(), mat.copy()
        mp[0, c] += h
        mm_[0, c] -= h
        ref_mat[0, c] = (L(mm=mp) - L(mm=mm_)) / (2 * h)
    sc = max(abs(ref_angle), *map(abs, ref_sun), abs(ref_dist))
    assert abs(g["angle"][1] - ref_angle) < 1e-7 * sc
    assert g["angle"][0] == 0.0  # the root has no joint
    assert abs(g["sun"][0] - ref_sun[0]) < 1e-7 * sc and abs(g["sun"][2] - ref_sun[2]) < 1e-7 * sc
    assert abs(g["dist"] - ref_dist) < 1e-7 * sc
    assert rel(g["mat"], ref_mat, np.max(np.abs(ref_mat))) < 1e-7
    # the distance derivative of an inverse-square law
    assert abs(g["dist"] + 2 * (gF @ r["F"] + gT @ r["T"]) / dist) < 1e-7 * abs(g["dist"])


def test_clamped_joint_has_no_offset_gradient():
    m = hinged_plate()
    m.limits = np.array([[-math.pi, math.pi], [-0.2, 0.2]])
    s = np.array([math.sin(0.9), 0.0, math.cos(0.9)])  # tracking wants 0.9 rad: clamped at 0.2
    g = O.frozen_grad(m, s, 16, 1, np.array([1.0, 0.5, -0.3]), np.array([0.2, -0.1, 0.4]))
    assert g["angle"][1] == 0.0


def test_sun_direction_length_is_irrelevant():
    """F_H(lambda s) = F_H(s): the gradient in s at lambda s is the gradient at
    s divided by lambda, and every other gradient is unchanged."""
    m = I.box_wing()
    s = I.sun_dirs_uniform(4, seed=6)[2]
    gF, gT = np.array([0.3, -1.0, 0.4]), np.array([0.5, 0.2, -0.7])
    off = np.array([0.0, 0.1, -0.05])
    g1 = O.frozen_grad(m, s, 24, 1, gF, gT, offsets=off)
    g2 = O.frozen_grad(m, 2.5 * s, 24, 1, gF, gT, offsets=off)
    sc = np.max(np.abs(g1["sun"]))
    assert rel(g2["sun"] * 2.5, g1["sun"], sc) < 1e-8
    assert rel(g2["angle"], g1["angle"], np.max(np.abs(g1["angle"]))) < 1e-8
    assert rel(g2["mat"], g1["mat"], np.max(np.abs(g1["mat"]))) < 1e-8
    # the radial component of the direction gradient vanishes
    assert abs(g1["sun"] @ s) < 1e-6 * sc
