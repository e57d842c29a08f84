"""Pins of the oracle's orbit propagation (Sec. 3, Eqs. 1-3) against
mathematics and independent references: the RK 7(8) order conditions and
numerical order, Kepler's closed-form two-body motion, RK4 convergence order,
conservation laws, the J2 secular node rate, an independent solar ephemeris
(Astronomical Almanac low-precision formula), attitude-frame properties, the
cylindrical shadow, and bitwise step replay."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

MU = 3.986004418e14
RE = 6378137.0
J2 = 1.08262668e-3
AU = 1.495978707e11


def kepler_state(a, e, i, raan, argp, M, mu=MU):
    """Position/velocity from classical elements (Newton on Kepler's equation)."""
    E = M if e < 0.8 else math.pi
    for _ in range(50):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    nu = 2 * math.atan2(math.sqrt(1 + e) * math.sin(E / 2), math.sqrt(1 - e) * math.cos(E / 2))
    p = a * (1 - e * e)
    r = p / (1 + e * math.cos(nu))
    rp = np.array([r * math.cos(nu), r * math.sin(nu), 0.0])
    vp = np.array([-math.sin(nu), e + math.cos(nu), 0.0]) * math.sqrt(mu / p)
    cO, sO, ci, si, cw, sw = (math.cos(raan), math.sin(raan), math.cos(i), math.sin(i), math.cos(argp),
                              math.sin(argp))
    Q = np.array([[cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci, sO * si],
                  [sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci, -cO * si],
                  [sw * si, cw * si, ci]])
    return np.concatenate([Q @ rp, Q @ vp])


def test_rkf78_order_conditions():
    c, A, b7, b8 = O.rkf78_tableau()
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    for k in range(7):
        assert abs(b7 @ c ** k - 1 / (k + 1)) < 1e-14
    for k in range(8):
        assert abs(b8 @ c ** k - 1 / (k + 1)) < 1e-14
    for b in (b7, b8):
        assert abs(b @ (A @ c) - 1 / 6) < 1e-14
        assert abs(b @ (c * (A @ c)) - 1 / 8) < 1e-14
        assert abs(b @ (A @ (A @ c)) - 1 / 24) < 1e-14
        assert abs(b @ (A @ c ** 2) - 1 / 12) < 1e-14
        assert abs(b @ (c ** 2 * (A @ c)) - 1 / 10) < 1e-14
        assert abs(b @ (A @ (c * (A @ c))) - 1 / 40) < 1e-14


def test_rkf78_numerical_order():
    """Local error of the 7th / 8th-order weights falls by ~2^8 / 2^9 per halving."""
    c, A, b7, b8 = O.rkf78_tableau()

    def f(t, y):
        return np.array([y[1], -math.sin(y[0]) + 0.3 * math.cos(t)])

    def step(t, y, h, b):
        k = np.zeros((13, 2))
        for s in range(13):
            k[s] = f(t + c[s] * h, y + h * (A[s, :s] @ k[:s]))
        return y + h * (b @ k)

    def ref(h):
        y = y0.copy()
        for j in range(256):
            y = step(j * h / 256, y, h / 256, b8)
        return y

    y0 = np.array([1.1, 0.2])
    for b, lo, hi in ((b7, 150, 450), (b8, 300, 900)):
        e = [np.linalg.norm(step(0.0, y0, h, b) - ref(h)) for h in (0.4, 0.2)]
        assert lo < e[0] / e[1] < hi


def test_two_body_matches_kepler():
    a, e = 42164e3 * 0.9, 0.12
    y0 = kepler_state(a, e, 0.3, 0.2, 0.7, 0.4)
    n = math.sqrt(MU / a ** 3)
    T = 86400.0
    pp = O.prop_params(central=0, rtol=1e-13, atol_pos=1e-7, atol_vel=1e-10)
    y1, stats, _ = O.propagate(None, pp, 0.0, T, y0)
    want = kepler_state(a, e, 0.3, 0.2, 0.7, 0.4 + n * T)
    assert np.linalg.norm(y1[:3] - want[:3]) < 1e-3
    assert stats[0] > 10 and stats[2] == 13 * (stats[0] + stats[1])


def test_rk4_fourth_order():
    y0 = kepler_state(7000e3, 0.01, 0.5, 0.0, 0.0, 0.0)
    a = 7000e3
    T = 6000.0
    want = kepler_state(7000e3, 0.01, 0.5, 0.0, 0.0, math.sqrt(MU / a ** 3) * T)
    errs = []
    for h in (60.0, 30.0):
        pp = O.prop_params(method=1, h0=h)
        y1, stats, _ = O.propagate(None, pp, 0.0, T, y0)
        assert stats[0] == round(T / h)
        errs.append(np.linalg.norm(y1[:3] - want[:3]))
    assert 12 < errs[0] / errs[1] < 20


def test_j2_acceleration_is_gradient_of_potential():
    pp = O.prop_params(central=0, j2=True)
    pp0 = O.prop_params(central=0)
    r = np.array([5.1e6, -3.2e6, 4.4e6])

    def V(x):
        rr = np.linalg.norm(x)
        return -MU / rr + MU * J2 * RE ** 2 / rr ** 3 * (3 * x[2] ** 2 / rr ** 2 - 1) / 2

    g = np.zeros(3)
    for k in range(3):
        dx = np.zeros(3); dx[k] = 1.0
        g[k] = -(V(r + dx) - V(r - dx)) / 2.0
    a, _ = O.accel(None, pp, 0.0, np.concatenate([r, np.zeros(3)]))
    a0, _ = O.accel(None, pp0, 0.0, np.concatenate([r, np.zeros(3)]))
    assert np.linalg.norm(a - g) < 1e-6 * np.linalg.norm(a - a0)


def test_j2_conservation_and_node_rate():
    a, e, i = 7000e3, 0.001, math.radians(50.0)
    y0 = kepler_state(a, e, i, 0.0, 0.0, 0.0)
    pp = O.prop_params(central=0, j2=True, rtol=1e-12)
    T = 2 * 86400.0

    def energy(y):
        r = np.linalg.norm(y[:3])
        return 0.5 * y[3:] @ y[3:] - MU / r + MU * J2 * RE ** 2 / r ** 3 * (3 * y[2] ** 2 / r ** 2 - 1) / 2

    y1, _, _ = O.propagate(None, pp, 0.0, T, y0)
    assert abs(energy(y1) - energy(y0)) < 1e-9 * abs(energy(y0))
    hz = lambda y: np.cross(y[:3], y[3:])[2]  # noqa: E731
    assert abs(hz(y1) - hz(y0)) < 1e-9 * abs(hz(y0))
    h1 = np.cross(y1[:3], y1[3:])
    raan = math.atan2(h1[0], -h1[1])
    n = math.sqrt(MU / a ** 3)
    rate = -1.5 * n * J2 * (RE / (a * (1 - e * e))) ** 2 * math.cos(i)
    assert abs(raan / (rate * T) - 1) < 0.02


def almanac_sun(mjd):
    """Astronomical Almanac low-precision Sun (independent of Montenbruck & Gill's series)."""
    n = mjd - 51544.5
    L = math.radians((280.460 + 0.9856474 * n) % 360)
    g = math.radians((357.528 + 0.9856003 * n) % 360)
    lam = L + math.radians(1.915 * math.sin(g) + 0.020 * math.sin(2 * g))
    eps = math.radians(23.439 - 4e-7 * n)
    R = (1.00014 - 0.01671 * math.cos(g) - 0.00014 * math.cos(2 * g)) * AU
    return R * np.array([math.cos(lam), math.cos(eps) * math.sin(lam), math.sin(eps) * math.sin(lam)])


def test_sun_ephemeris_against_almanac():
    """Ecliptic longitude: the series refers to the J2000 equinox, the Almanac
    formula to the equinox of date (precession 1.3972 deg per century); the
    series keeps the perihelion fixed, so agreement is to ~0.1 deg."""
    eps0 = math.radians(23.43929111)
    for mjd in np.linspace(61041.0, 61041.0 + 365.0, 37):
        r = O.sun_position(mjd)
        w = almanac_sun(mjd)
        T = (mjd - 51544.5) / 36525.0
        ey = r[1] * math.cos(eps0) + r[2] * math.sin(eps0)
        ez = -r[1] * math.sin(eps0) + r[2] * math.cos(eps0)
        assert abs(ez) < 1e-6 * np.linalg.norm(r)           # in the ecliptic plane
        lam = math.degrees(math.atan2(ey, r[0])) + 1.3972 * T
        eps = math.radians(23.439 - 4e-7 * (mjd - 51544.5))
        lam_w = math.degrees(math.atan2(w[1] * math.cos(eps) + w[2] * math.sin(eps), w[0]))
        assert abs((lam - lam_w + 180) % 360 - 180) < 0.1
        assert abs(np.linalg.norm(r) / np.linalg.norm(w) - 1) < 2e-4


def test_lvlh_attitude_frame():
    y = kepler_state(42164e3, 0.001, 0.1, 0.3, 0.2, 1.0)
    pp = O.prop_params(attitude=0)
    R = O.attitude(pp, y)
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-14) and abs(np.linalg.det(R) - 1) < 1e-14
    assert np.allclose(R[:, 2], -y[:3] / np.linalg.norm(y[:3]), atol=1e-15)
    h = np.cross(y[:3], y[3:])
    assert np.allclose(R[:, 1], -h / np.linalg.norm(h), atol=1e-15)
    q = (math.cos(0.35), 0.0, math.sin(0.35), 0.0)   # 0.7 rad about y
    R2 = O.attitude(O.prop_params(attitude=1, q=q), y)
    from scipy.spatial.transform import Rotation
    assert np.allclose(R2, Rotation.from_rotvec([0, 0.7, 0]).as_matrix(), atol=1e-15)


def test_srp_acceleration_and_shadow():
    m = I.box_wing()
    pp = O.prop_params(central=0, srp=True, mass=m.mass, N=32, bounces=1)
    rs = O.sun_position(61041.0)
    e = rs / np.linalg.norm(rs)
    side = np.cross(e, [0, 0, 1.0]); side /= np.linalg.norm(side)
    r_lit = 42164e3 * side
    v = np.cross([0, 0, 1.0], r_lit) / np.linalg.norm(r_lit) * 3074.0
    y = np.concatenate([r_lit, v])
    a_srp, aux = O.accel(m, pp, 0.0, y)
    a_g, _ = O.accel(None, O.prop_params(central=0), 0.0, y)
    R = O.attitude(pp, y)
    sb = R.T @ ((rs - r_lit) / np.linalg.norm(rs - r_lit))
    assert np.allclose(aux[:3], sb, atol=1e-15) and aux[4] == 0.0
    ev = O.evaluate(m, aux[:3].copy(), 32, bounces=1, dist_au=aux[3])
    assert np.allclose(aux[5:], ev["F"], rtol=1e-13, atol=0)
    assert np.linalg.norm((a_srp - a_g) - R @ ev["F"] / m.mass) < 1e-15 * np.linalg.norm(a_g)
    assert 1e-9 < np.linalg.norm(a_srp - a_g) < 1e-7
    y_sh = np.concatenate([-42164e3 * e, v])
    a2, aux2 = O.accel(m, pp, 0.0, y_sh)
    a2g, _ = O.accel(None, O.prop_params(central=0), 0.0, y_sh)
    assert aux2[4] == 1.0 and np.array_equal(a2, a2g)


def test_step_replay_is_bitwise():
    m = I.box_wing()
    y0 = kepler_state(42164e3, 0.001, math.radians(0.1), 0.0, 0.0, 0.0)
    pp = O.prop_params(central=0, j2=True, sun3=True, srp=True, mass=m.mass, N=16, bounces=1)
    y1, stats, hlog = O.propagate(m, pp, 0.0, 7200.0, y0)
    y2, _, _ = O.propagate(m, pp, 0.0, 7200.0, y0, h_replay=hlog)
    assert np.array_equal(y1, y2)
    assert abs(hlog.sum() - 7200.0) < 1e-9


def test_sun_third_body_is_tidal():
    """For |r| << |r_sun| the third-body term is the tidal field
    (mu_S / |r_S|^3) (3 (r . e) e - r), to relative order |r| / |r_S|."""
    pp_s = O.prop_params(central=0, sun3=True)
    pp_0 = O.prop_params(central=0)
    rs = O.sun_position(61041.0 + 3.7)
    e = rs / np.linalg.norm(rs)
    for r in (np.array([42164e3, 0, 0]), np.array([1e7, -3e7, 2e7]), 42164e3 * e):
        y = np.concatenate([r, np.zeros(3)])
        a = O.accel(None, pp_s, 3.7 * 86400.0, y)[0] - O.accel(None, pp_0, 3.7 * 86400.0, y)[0]
        tidal = 1.32712440018e20 / np.linalg.norm(rs) ** 3 * (3 * (r @ e) * e - r)
        assert np.linalg.norm(a - tidal) < 2e-3 * np.linalg.norm(tidal)
