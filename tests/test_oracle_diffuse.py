"""Pins of the oracle's diffuse secondary rays (Sec. 6.1's diffuse rays; the
reading: K cosine-distributed rays of weight w rho_d / K per hit of a segment
that has a next level, each traced once, depositing the full per-hit law).

What fixes them, independently of the oracle: the published SplitMix64
stream; the moments of the cosine-weighted hemisphere (mean (2/3) n, second
moment of the cosine 1/2, where a uniform hemisphere gives 1/2 and 1/3); K = 0
and bounces = 0 leave the specular model unchanged; a convex body's diffuse
light escapes; and the momentum that a Lambertian plate sends to an absorbing
plate equals the radiative-transfer integral over both plates, computed here
by quadrature without rays.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2608_07307_gb300 import inputs as I


def test_generator_is_splitmix64():
    assert O.splitmix64(0, 0) == 0xE220A8397B1DCDAF  # published first output for seed 0
    for seed in (0, 12345, 2**32 - 1):
        ref = I.splitmix64(seed, 64)
        for c in (0, 1, 7, 63):
            assert O.splitmix64(seed, c) == int(ref[c])


@pytest.mark.parametrize("nf", [(0, 0, 1.0), (0, 0, -1.0), (0.6, -0.48, 0.64), (1.0, 0, 0)])
def test_samples_are_cosine_weighted(nf):
    nf = np.asarray(nf) / np.linalg.norm(nf)
    w = np.array([O.diffuse_dir(7, c, nf) for c in range(20000)])
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-14)
    cos = w @ nf
    assert cos.min() > 0.0
    assert np.linalg.norm(w.mean(axis=0) - 2.0 / 3.0 * nf) < 0.012
    assert abs((cos ** 2).mean() - 0.5) < 0.01
    # tangential directions are isotropic: no preferred azimuth
    t = w - np.outer(cos, nf)
    assert np.linalg.norm(t.mean(axis=0)) < 0.012


def test_no_diffuse_or_no_level_is_the_specular_model():
    m = I.box_wing()
    s = np.array([0.3, 0.5, 0.8]) / np.linalg.norm([0.3, 0.5, 0.8])
    base = O.evaluate(m, s, 48, 2)
    assert np.array_equal(O.evaluate(m, s, 48, 2, n_diffuse=0, diffuse_seed=9)["acc"], base["acc"])
    b0 = O.evaluate(m, s, 48, 0)
    assert np.array_equal(O.evaluate(m, s, 48, 0, n_diffuse=16)["acc"], b0["acc"])
    # with a level left, the diffuse light of the panels reaches the bus
    assert not np.array_equal(O.evaluate(m, s, 48, 2, n_diffuse=16)["acc"], base["acc"])


def test_diffuse_light_of_a_convex_body_escapes():
    m = I.icosphere(2, mat=((0.2, 0.5),))
    for s in I.sun_dirs_uniform(3, seed=4):
        a = O.evaluate(m, s, 40, 2)
        b = O.evaluate(m, s, 40, 2, n_diffuse=32)
        assert np.array_equal(a["acc"], b["acc"])


def _wall(x0, rho=(0.0, 0.0)):
    """Unit square in the plane x = x0 (y, z in [0, 1]), front face towards -x."""
    w = I.flat_plate(1.0, 1.0, center=(0.5, 0.5), mat=(rho, rho))
    xyz = np.asarray(w.xyz, np.float64).copy()
    # (x, y, z) -> (x0 - z, y, x): the plate's +z front normal turns to -x
    w.xyz = np.stack([x0 - xyz[:, 2], xyz[:, 1], xyz[:, 0]], axis=1)
    return w


def _transfer_quadrature(gap, n=36):
    """Momentum per unit incident power density that a Lambertian unit square
    A (z = 0, x, y in [0, 1], normal +z) sends to the absorbing unit square B
    (x = 1 + gap, y, z in [0, 1]): the double area integral of
    cos_A cos_B / (pi r^2) times the unit direction, midpoint rule."""
    g = (np.arange(n) + 0.5) / n
    px, py = np.meshgrid(g, g, indexing="ij")
    qy, qz = np.meshgrid(g, g, indexing="ij")
    P = np.stack([px.ravel(), py.ravel(), np.zeros(n * n)], axis=1)
    Q = np.stack([np.full(n * n, 1.0 + gap), qy.ravel(), qz.ravel()], axis=1)
    D = Q[None, :, :] - P[:, None, :]
    r2 = (D ** 2).sum(axis=2)
    r = np.sqrt(r2)
    cos_a = D[:, :, 2] / r
    cos_b = D[:, :, 0] / r
    k = cos_a * cos_b / (math.pi * r2) / (n * n) / (n * n)
    return (k[:, :, None] * D / r[:, :, None]).sum(axis=(0, 1))


def test_lambertian_transfer_between_two_plates():
    """A white Lambertian floor (rho_d = 1, rho_s = 0) lit at 30 degrees and an
    absorbing wall beyond a 0.2 m gap: the extra force that the diffuse rays
    add is the momentum the floor's diffuse light brings to the wall,
    P cos(theta_sun) rho_d x (transfer integral), within the Monte Carlo
    error of the rays."""
    gap = 0.2
    floor = I.flat_plate(1.0, 1.0, center=(0.5, 0.5), mat=((0.0, 1.0), (0.0, 1.0)))
    m = I.merge([floor, _wall(1.0 + gap)])
    th = math.radians(30.0)
    s = np.array([-math.sin(th), 0.0, math.cos(th)])  # photons travel towards +x and down
    P0 = 4.56e-6
    a = O.evaluate(m, s, 64, 1, P0=P0)
    b = O.evaluate(m, s, 64, 1, P0=P0, n_diffuse=64, diffuse_seed=3)
    dF = b["F"] - a["F"]
    want = P0 * math.cos(th) * 1.0 * _transfer_quadrature(gap)
    assert want[0] > 0 and abs(want[1]) < 1e-3 * want[0]
    assert abs(dF[0] / want[0] - 1.0) < 0.03, (dF, want)
    assert abs(dF[2] / want[2] - 1.0) < 0.05, (dF, want)
    assert abs(dF[1]) < 0.05 * want[0]
