"""Pins of the oracle's SPAD interpolation model (Sec. 4.2, Sec. 6.1).

The interpolant is pinned by what bilinear interpolation on an azimuth /
elevation grid must do, whatever the code: reproduce the samples, be exact
for functions bilinear in (azimuth, elevation), wrap around in azimuth, clamp
beyond the outer elevation rows, scale as 1/r^2, and converge at second
order on a smooth field.  The table builder is pinned by an absorbing box,
whose force is exactly along the photon direction with the projected area as
magnitude up to the pixel quadrature; the propagation hook by a zero table
(no SRP) and by a state whose Sun direction is a sample direction.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I

GRIDS = [I.SPAD_20x10, I.SPAD_20x10S, I.spad_grid(7, 5, 13.0, -70.0, 31.0)]


def _dir(az, el):
    return np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])


def _daz(g):
    return 2 * math.pi / g["n_az"]


def _bilinear_table(g, coef):
    """Entry (j, i) = a + b i + c j + d i j per component (coef [4][6])."""
    j, i = np.meshgrid(np.arange(g["n_el"]), np.arange(g["n_az"]), indexing="ij")
    a, b, c, d = coef
    return a + b * i[..., None] + c * j[..., None] + d * (i * j)[..., None]


def test_grid_directions_of_the_paper_sets():
    """20 x 10 from (-180, -90) degrees has a row at 0 degrees elevation and
    the shifted set does not (Sec. 6.1); every direction is a unit vector with
    the stated azimuth and elevation."""
    for g, has_zero in ((I.SPAD_20x10, True), (I.SPAD_20x10S, False)):
        d = O.spad_dirs(g)
        assert d.shape == (10, 20, 3)
        assert np.allclose(np.linalg.norm(d, axis=2), 1.0, atol=1e-15)
        el = np.degrees(np.arcsin(np.clip(d[:, 0, 2], -1, 1)))
        assert np.any(np.abs(el) < 1e-9) == has_zero
        assert np.allclose(np.diff(el), 18.0, atol=1e-9)
        az = np.degrees(np.arctan2(d[5, :, 1], d[5, :, 0]))
        steps = np.mod(np.diff(az), 360.0)
        assert np.allclose(steps, 18.0, atol=1e-9)
    assert np.allclose(O.spad_dirs(I.SPAD_20x10)[5, 0], [-1.0, 0.0, 0.0], atol=1e-15)
    assert np.allclose(O.spad_dirs(I.SPAD_20x10S)[0, 0], _dir(math.radians(-175), math.radians(-85)), atol=1e-15)


@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_samples_are_reproduced(gi):
    g = GRIDS[gi]
    tab = np.random.default_rng(gi).normal(size=(g["n_el"], g["n_az"], 6))
    d = O.spad_dirs(g)
    for j in range(g["n_el"]):
        for i in range(g["n_az"]):
            if abs(abs(g["el0"] + j * g["d_el"]) - math.pi / 2) < 1e-12:
                continue  # a pole: every azimuth is the same direction
            assert np.allclose(O.spad_interp(g, tab, d[j, i]), tab[j, i], rtol=0, atol=1e-12), (j, i)


@pytest.mark.parametrize("gi", range(len(GRIDS)))
def test_exact_for_bilinear_fields(gi):
    """Inside the grid (no wrap, no clamp) the interpolant of a field
    bilinear in (azimuth, elevation) is that field; distinct coefficients on
    the two axes catch swapped weights or a transposed table."""
    g = GRIDS[gi]
    rng = np.random.default_rng(10 + gi)
    coef = rng.normal(size=(4, 6))
    tab = _bilinear_table(g, coef)
    a, b, c, d = coef
    for _ in range(200):
        u = rng.uniform(0, g["n_az"] - 1)
        v = rng.uniform(0, g["n_el"] - 1)
        el = g["el0"] + v * g["d_el"]
        if abs(el) > math.pi / 2 - 1e-6:
            continue
        got = O.spad_interp(g, tab, _dir(g["az0"] + u * _daz(g), el))
        assert np.allclose(got, a + b * u + c * v + d * u * v, rtol=0, atol=1e-11)


def test_azimuth_wraps_to_the_first_column():
    g = I.SPAD_20x10S
    tab = np.zeros((10, 20, 6))
    tab[:, 0, :] = 1.0
    el = g["el0"] + 4.5 * g["d_el"]
    for u, want in ((0.25, 0.75), (19.25, 0.25), (19.75, 0.75), (19.5, 0.5), (-0.25, 0.75), (1.5, 0.0)):
        got = O.spad_interp(g, tab, _dir(g["az0"] + u * _daz(g), el))
        assert np.allclose(got, want, atol=1e-12), u


def test_elevation_clamps_beyond_the_outer_rows():
    rng = np.random.default_rng(3)
    coef = rng.normal(size=(4, 6))
    a, b, c, d = coef
    for g, el_deg, row in ((I.SPAD_20x10, 85.0, 9), (I.SPAD_20x10, 72.0 + 1e-7, 9),
                           (I.SPAD_20x10S, -89.0, 0), (I.SPAD_20x10S, 80.0, 9)):
        tab = _bilinear_table(g, coef)
        u = 3.3
        got = O.spad_interp(g, tab, _dir(g["az0"] + u * _daz(g), math.radians(el_deg)))
        assert np.allclose(got, a + b * u + c * row + d * u * row, atol=1e-11), (el_deg, row)


def test_distance_scaling_and_skip():
    g = I.SPAD_20x10
    tab = np.random.default_rng(4).normal(size=(10, 20, 6))
    s = _dir(0.3, 0.2)
    base = O.spad_interp(g, tab, s, 1.0)
    assert np.allclose(O.spad_interp(g, tab, s, 2.0), base / 4.0, rtol=1e-15, atol=0)
    assert np.allclose(O.spad_interp(g, tab, s, 0.5), base * 4.0, rtol=1e-15, atol=0)
    assert np.all(O.spad_interp(g, tab, s, -1.0) == 0.0)
    # only the direction of s matters
    assert np.allclose(O.spad_interp(g, tab, 7.5 * s), base, rtol=1e-14, atol=1e-15)


def test_second_order_convergence_on_a_smooth_field():
    """The cannonball law F = -C s sampled on grids of spacing h and h/2:
    the largest interpolation error (away from the clamped polar caps)
    falls by ~4 (bilinear), not ~2 (nearest sample or a wrong weight)."""
    rng = np.random.default_rng(5)
    q = rng.normal(size=(4000, 3))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q = q[np.abs(q[:, 2]) < math.sin(math.radians(60))]
    errs = []
    for n in (20, 40, 80):
        g = I.spad_grid(n, n // 2, -180.0, -90.0)
        d = O.spad_dirs(g)
        tab = np.concatenate([-d, np.zeros_like(d)], axis=2)
        e = max(np.abs(O.spad_interp(g, tab, s)[:3] + s).max() for s in q)
        errs.append(e)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.3 < r2 < 4.7, errs


def test_table_of_an_absorbing_box():
    """All-absorbing unit cube: every pixel's momentum is along d = -s, so
    each entry's force is exactly antiparallel to its sample direction, with
    magnitude P0 times the projected area |s_x| + |s_y| + |s_z| up to the
    pixel quadrature; torque about the centre vanishes by symmetry up to it."""
    g = I.spad_grid(6, 4, -180.0, -80.0, 40.0)
    mesh = I.box(mat=((0.0, 0.0),))
    P0 = 4.56e-6
    tab = O.spad_table(mesh, g, N=48, bounces=0, P0=P0)
    d = O.spad_dirs(g)
    for j in range(g["n_el"]):
        for i in range(g["n_az"]):
            s, F = d[j, i], tab[j, i, :3]
            Fn = np.linalg.norm(F)
            assert np.linalg.norm(np.cross(F / Fn, -s)) < 1e-12 and np.dot(F, s) < 0, (j, i)
            assert abs(Fn / (P0 * np.abs(s).sum()) - 1.0) < 0.05, (j, i, Fn)
            assert np.linalg.norm(tab[j, i, 3:]) < 0.05 * Fn


def _helio_state(s_body, dist_au):
    """Heliocentric position whose Sun direction (body = inertial) is s_body."""
    r = -dist_au * 1.495978707e11 * np.asarray(s_body)
    v = np.cross([0.0, 0.0, 1.0], r)
    v = v / np.linalg.norm(v) * 30e3
    return np.concatenate([r, v])


def test_propagation_zero_table_is_no_srp():
    g = I.SPAD_20x10
    y0 = np.array([42164e3, 0.0, 0.0, 0.0, 3074.66, 5.0])
    off = O.prop_params(j2=True, sun3=True, srp=False, mass=800.0)
    zero = O.prop_params(j2=True, sun3=True, srp=True, mass=800.0, spad=(g, np.zeros((10, 20, 6))))
    y_off, st_off, _ = O.propagate(None, off, 0.0, 6 * 3600.0, y0)
    y_zero, st_zero, _ = O.propagate(None, zero, 0.0, 6 * 3600.0, y0)
    assert np.array_equal(y_off, y_zero) and np.array_equal(st_off[:2], st_zero[:2])


def test_propagation_acceleration_at_a_sample_direction():
    """With the Sun along sample (j, i) in the body frame, the SRP
    acceleration is R F_ji / (m r^2); here R = I (inertial attitude q = 1),
    so a_SRP = F_ji / (m r_AU^2)."""
    g = I.SPAD_20x10S
    tab = np.random.default_rng(6).normal(size=(10, 20, 6)) * 1e-5
    s = O.spad_dirs(g)[3, 11]
    y = _helio_state(s, 0.8)
    m = 555.0
    kw = dict(central=1, attitude=1, mass=m)
    a_on, aux = O.accel(None, O.prop_params(srp=True, spad=(g, tab), **kw), 0.0, y)
    a_off, _ = O.accel(None, O.prop_params(srp=False, **kw), 0.0, y)
    want = tab[3, 11, :3] / (m * 0.8 ** 2)
    assert np.allclose(aux[:3], s, atol=1e-15) and abs(aux[3] - 0.8) < 1e-15
    assert np.allclose(a_on - a_off, want, rtol=1e-9, atol=0)
