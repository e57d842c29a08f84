"""The gradient bar shared by the adjoint parity tests.

Per entry: |g_i - r_i| <= 1e-3 |r_i| + floor, with floor = 1e-5 of the
group's largest oracle entry.  The floor is the FP32 rounding of the GPU's
per-ray adjoint terms (each carries a relative error of a few dozen units of
2^-24 ~ 6e-8; they are summed in FP64, so an entry built from terms of both
signs keeps an absolute error of order 1e-6 of the terms' scale, which the
group's largest entry bounds within a factor of a few) and, on arcs, the
oracle's central-difference rounding.  An entry the frozen hit set makes
exactly zero (a material no ray reaches) must come out zero on both sides.
"""
import numpy as np

GTOL = 1e-3
FLOOR = 1e-5


def check_group(name, g, r, tol=GTOL, floor=FLOOR):
    g, r = np.asarray(g, np.float64), np.asarray(r, np.float64)
    sc = np.max(np.abs(r))
    if sc == 0.0:
        assert np.max(np.abs(g)) <= 1e-12, (name, g)
        return
    bound = tol * np.abs(r) + floor * sc
    err = np.abs(g - r)
    bad = err > bound
    worst = float(np.max(err / np.maximum(np.abs(r), floor * sc)))
    assert not bad.any(), (f"{name}: entries {np.nonzero(bad.ravel())[0].tolist()} off; "
                           f"worst |g - r| / max(|r|, floor) {worst:.3g}\n gpu {g}\n fd  {r}")
    return worst
