"""Writes boxwing_forces.txt: the oracle's force and torque for the plain
method's box-wing workload (16 triangles with Sun-tracking panels, 256 x 256
rays, 1 specular bounce, P0 = 4.56e-6 N/m^2 at 1 AU) at the 256 Sun directions
drawn uniformly on the sphere from seed 0.

Each line: direction index k, then Fx Fy Fz (N) and Tx Ty Tz (N m), FP64 as
written by repr().  Every value is computed by oracle.evaluate alone.

    python tests/golden/make_boxwing.py [procs]
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N, BOUNCES, N_DIRS = 256, 1, 256


def _one(k):
    from oracle import oracle as O
    from paper_2608_07307_gb300 import inputs as I
    r = O.evaluate(I.box_wing(), I.sun_dirs_uniform(N_DIRS, seed=0)[k], N, BOUNCES)
    return k, list(r["F"]) + list(r["T"])


def main():
    import multiprocessing as mp
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        rows = sorted(pool.map(_one, range(N_DIRS)))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "boxwing_forces.txt")
    with open(out, "w") as f:
        f.write("# oracle force and torque, box-wing, N = 256, 1 bounce, 256 uniform directions (seed 0)\n")
        f.write("# (tests/golden/make_boxwing.py)\n# k Fx Fy Fz Tx Ty Tz\n")
        for k, v in rows:
            f.write(f"{k} " + " ".join(repr(float(x)) for x in v) + "\n")


if __name__ == "__main__":
    main()
