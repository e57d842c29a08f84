"""Propagate the GEO arc of the propagation workload from the command line.

    python -m paper_2608_07307_gb300.geo_arc [--days D] [--facet H] [--N N]
        [--bounces B] [--spad 20x10|20x10S] [--host-loop]

Spacecraft `inputs.spacecraft(H)` (Sun-tracking panels), orbit a = 42164 km,
e = 0, i = 0.1 deg, two-body + J2 + Sun + SRP (ray-traced with N^2 rays and B
bounces, or interpolated from a SPAD table built first), RKF7(8) rtol 1e-12.
The arc runs twice (the first run builds the workspace and the step graph)
and the second is timed; prints the steps, the time per step and the final
state.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import inputs as I
from . import srp


def main(argv=None):
    p = argparse.ArgumentParser(prog="python -m paper_2608_07307_gb300.geo_arc")
    p.add_argument("--days", type=float, default=1.0)
    p.add_argument("--facet", type=float, default=0.025)
    p.add_argument("--N", type=int, default=512)
    p.add_argument("--bounces", type=int, default=1)
    p.add_argument("--spad", choices=["20x10", "20x10S"], default=None)
    p.add_argument("--host-loop", action="store_true")
    a = p.parse_args(argv)
    ctx = srp.Context(0)
    mesh = I.spacecraft(a.facet)
    mid = ctx.load_mesh(mesh)
    a_geo, inc = 42164e3, math.radians(0.1)
    v = math.sqrt(3.986004418e14 / a_geo)
    y0 = np.array([a_geo, 0.0, 0.0, 0.0, v * math.cos(inc), v * math.sin(inc)])
    kw = dict(j2=True, sun3=True, N=a.N, bounces=a.bounces, rtol=1e-12, host_loop=a.host_loop)
    if a.spad:
        g = I.SPAD_20x10 if a.spad == "20x10" else I.SPAD_20x10S
        kw["spad"] = (g, ctx.spad_build(mid, g, N=a.N, bounces=a.bounces))
    arc = [0.0, a.days * 86400.0]
    ctx.propagate(mid, y0, arc, **kw)
    t0 = time.perf_counter()
    y1, st, _ = ctx.propagate(mid, y0, arc, **kw)
    dt = time.perf_counter() - t0
    n = max(st[0]["steps"], 1)
    print(f"{mesh.n_tris} triangles, {a.days:g} days: {st[0]['steps']} steps, {st[0]['rejects']} rejected, "
          f"{dt:.3f} s, {dt / n * 1e3:.3f} ms/step")
    print("y1", " ".join(repr(float(x)) for x in y1[0]))
    ctx.close()


if __name__ == "__main__":
    main()
