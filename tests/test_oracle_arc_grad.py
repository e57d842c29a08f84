"""Pins of the oracle's frozen-hit RK4 arc and of its finite-difference
gradient (the reference for the propagation adjoint):

  * the frozen arc equals the traced arc at the base point;
  * without SRP the gradient in the initial state is the state transition
    matrix of the linearised motion about a circular orbit, known in closed
    form (Clohessy-Wiltshire / Hill equations), and no parameter gradient is
    left;
  * a Sun-tracking hinged plate on a heliocentric arc, inertially fixed:
    every pixel always lands on the plate, so the traced arc is itself smooth
    in the coefficients, the joint offset and the quaternion components that
    turn the body about its y axis, and a wide five-point stencil of traced
    arcs gives the reference for the frozen arc's gradient.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

MU_E = 3.986004418e14
MU_S = 1.32712440018e20
AU = 1.495978707e11


def hinged_plate(mass=1.0):
    verts, tris = I._fan_rect((-1.0, 0.8, 0.0), (2.0, 0, 0), (0, 1.0, 0))
    tri = np.ascontiguousarray(np.asarray(tris, np.int32))
    return I.Mesh(np.ascontiguousarray(verts), tri, np.ones(len(tri), np.int32),
                  np.tile(np.array([[0, 1]], np.int32), (len(tri), 1)), np.array([[0.35, 0.25], [0.1, 0.3]]),
                  **I._parts(2, [-1, 0], pivot=[[0, 0, 0], [0, 0, 0.4]], axis=[[0, 0, 0], [0, 1, 0]]),
                  c_ref=np.zeros(3), mass=mass, name="hinged_plate")


def test_frozen_arc_equals_traced_arc():
    m = I.box_wing()
    pp = O.prop_params(srp=True, j2=True, sun3=True, mass=20.0, N=24, bounces=1, method=1, h0=60.0,
                       q=(0.96, 0.1, -0.2, 0.15))
    a = 42164e3
    v = math.sqrt(MU_E / a)
    y0 = np.array([a, 0, 0, 0, v * math.cos(0.02), v * math.sin(0.02)])
    yt, st, _ = O.propagate(m, pp, 0.0, 3000.0, y0)
    y1, rec = O.rk4_arc_record(m, pp, 0.0, 3000.0, y0)
    yf = O.rk4_arc_frozen(m, pp, 0.0, 3000.0, y0, rec)
    assert np.max(np.abs(y1[:3] - yt[:3])) < 1e-6 and np.max(np.abs(yf[:3] - yt[:3])) < 1e-6
    assert rec["lit"][: 4 * st[0]].all()


def test_initial_state_gradient_is_the_hill_transition_matrix():
    a = 7.0e6
    n = math.sqrt(MU_E / a ** 3)
    y0 = np.array([a, 0.0, 0.0, 0.0, n * a, 0.0])
    T = 1500.0
    pp = O.prop_params(srp=False, method=1, h0=15.0)
    m = I.box_wing()
    rows = [O.arc_frozen_grad(m, pp, 0.0, T, y0, e) for e in np.eye(6)]
    J = np.array([r["y0"] for r in rows])
    for r in rows:
        assert np.all(r["mat"] == 0) and np.all(r["angle"] == 0) and np.all(r["q"] == 0)
    c, s, nt = math.cos(n * T), math.sin(n * T), n * T
    Phi = np.array([
        [4 - 3 * c, 0, 0, s / n, 2 * (1 - c) / n, 0],
        [6 * (s - nt), 1, 0, -2 * (1 - c) / n, (4 * s - 3 * nt) / n, 0],
        [0, 0, c, 0, 0, s / n],
        [3 * n * s, 0, 0, c, 2 * s, 0],
        [-6 * n * (1 - c), 0, 0, -2 * s, 4 * c - 3, 0],
        [0, 0, -n * s, 0, 0, c]])

    def frame(t):
        C = np.array([[math.cos(n * t), -math.sin(n * t), 0], [math.sin(n * t), math.cos(n * t), 0], [0, 0, 1]])
        W = np.array([[0, -n, 0], [n, 0, 0], [0, 0, 0]])  # omega x
        Tm = np.zeros((6, 6))
        Tm[:3, :3] = C
        Tm[3:, :3] = C @ W
        Tm[3:, 3:] = C
        return Tm

    Jref = frame(T) @ Phi @ np.linalg.inv(frame(0.0))
    for k in range(6):
        assert np.max(np.abs(J[k] - Jref[k])) <= 1e-6 * np.max(np.abs(Jref[k])), (k, J[k], Jref[k])


def test_hinged_plate_arc_gradient_matches_traced_arcs():
    m = hinged_plate(mass=1.0)
    r = AU
    v = math.sqrt(MU_S / r)
    y0 = np.array([r, 0.0, 0.0, 0.0, 0.0, v])  # orbit in the inertial x-z plane
    pp = O.prop_params(central=1, srp=True, mass=m.mass, N=8, bounces=1, method=1, h0=3600.0, attitude=1,
                       q=(1.0, 0.0, 0.0, 0.0))
    t1 = 48 * 3600.0
    off = np.array([0.0, 0.12])
    lam = np.array([0.3, 0.0, -1.0, 200.0, 0.0, 50.0])
    g = O.arc_frozen_grad(m, pp, 0.0, t1, y0, lam, offsets=off, h=1e-4)  # |y| ~ 1 AU: a wider step
    rec = g["record"]
    assert rec["lit"][:4 * 48].all() and np.all(rec["hits"][:4 * 48, :, 0] >= 0)

    def L(mm=None, of=off, qq=None):
        mesh = m if mm is None else m.with_materials(mm)
        p2 = O.Prop.from_buffer_copy(pp)
        if qq is not None:
            for k in range(4):
                p2.q[k] = qq[k]
        y1, _ = O.rk4_arc_record(mesh, p2, 0.0, t1, y0, offsets=of)  # traced arc
        return lam @ y1

    D = 1e-3
    stencil = lambda f: (f(-2) - 8 * f(-1) + 8 * f(1) - f(2)) / (12 * D)  # noqa: E731
    mat0 = np.asarray(m.mat)
    ref_mat = np.zeros_like(mat0)
    for c in range(2):
        def fm(k, c=c):
            mm = mat0.copy()
            mm[0, c] += k * D
            return L(mm=mm)
        ref_mat[0, c] = stencil(fm)
    ref_off = stencil(lambda k: L(of=off + np.array([0.0, k * D])))
    assert np.max(np.abs(g["mat"] - ref_mat)) <= 1e-5 * np.max(np.abs(ref_mat))
    assert abs(g["angle"][1] - ref_off) <= 1e-5 * abs(ref_off)


def test_hinged_plate_arc_attitude_gradient_matches_traced_arcs():
    """A commanded (not tracking) plate on a body turned 0.3 rad about y: the
    quaternion components (q0, q2) keep the turn about y, so every pixel still
    lands on the plate while the incidence angle changes."""
    m = hinged_plate(mass=1.0)
    v = math.sqrt(MU_S / AU)
    y0 = np.array([AU, 0.0, 0.0, 0.0, 0.0, v])
    qb = np.array([math.cos(0.15), 0.0, math.sin(0.15), 0.0])
    pp = O.prop_params(central=1, srp=True, mass=m.mass, N=8, bounces=1, method=1, h0=3600.0, attitude=1, q=tuple(qb))
    t1 = 48 * 3600.0
    ang = np.array([0.0, -2.0])
    lam = np.array([0.3, 0.0, -1.0, 200.0, 0.0, 50.0])
    g = O.arc_frozen_grad(m, pp, 0.0, t1, y0, lam, angles=ang, h=1e-4)
    assert np.all(g["record"]["hits"][:4 * 48, :, 0] >= 0)

    def L(qq=qb, an=ang):
        p2 = O.Prop.from_buffer_copy(pp)
        for k in range(4):
            p2.q[k] = qq[k]
        y1, _ = O.rk4_arc_record(m, p2, 0.0, t1, y0, angles=an)  # traced arc
        return lam @ y1

    D = 1e-3
    stencil = lambda f: (f(-2) - 8 * f(-1) + 8 * f(1) - f(2)) / (12 * D)  # noqa: E731
    ref_q = [stencil(lambda k, c=c: L(qq=qb + k * D * np.eye(4)[c])) for c in (0, 2)]
    ref_a = stencil(lambda k: L(an=ang + np.array([0.0, k * D])))
    sc = max(abs(ref_q[0]), abs(ref_q[1]))
    assert abs(g["q"][0] - ref_q[0]) <= 1e-5 * sc and abs(g["q"][2] - ref_q[1]) <= 1e-5 * sc
    assert abs(g["angle"][1] - ref_a) <= 1e-5 * abs(ref_a)
    # a turn of the body by d(beta) about y and the opposite turn of the joint
    # leave the plate, hence the arc, unchanged: g_angle = g_q . dq/dbeta
    dq = np.array([-qb[2] / 2, 0.0, qb[0] / 2, 0.0])
    assert abs(ref_a) > 0 and abs(g["angle"][1] - g["q"] @ dq) <= 1e-5 * abs(ref_a)
