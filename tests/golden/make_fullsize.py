"""Writes fullsize_forces.txt: the oracle's force and torque for whole
evaluations at the benchmark sizes, which no GPU test can afford to trace with
the oracle at run time.

Each line: mesh facet h, N, bounces, index k of the 4096-point Fibonacci
direction table, then Fx Fy Fz (N) and Tx Ty Tz (N m), FP64 as written by
repr().  Meshes come from paper_2608_07307_gb300.inputs.spacecraft(h); every
value is computed by oracle.evaluate (ray-sharded over spawn-started
processes, partial sums added in a fixed order), nothing else.

    python tests/golden/make_fullsize.py [procs]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

CASES = [
    # the precision form: ~50k triangles, 1024^2 rays, 2 bounces
    (0.05, 1024, 2, 0), (0.05, 1024, 2, 1365), (0.05, 1024, 2, 2730),
    # the headline: ~200k triangles, 1024^2 rays, 2 bounces
    (0.025, 1024, 2, 0), (0.025, 1024, 2, 17),
]


def main():
    from oracle import oracle as O
    from paper_2608_07307_gb300 import inputs as I

    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    dirs = I.sun_dirs_fibonacci(4096)
    meshes = {}
    lines = []
    for h, N, B, k in CASES:
        if h not in meshes:
            meshes[h] = I.spacecraft(h)
        t0 = time.perf_counter()
        r = O.evaluate(meshes[h], dirs[k], N, B, procs=procs)
        vals = " ".join(repr(float(x)) for x in list(r["F"]) + list(r["T"]))
        lines.append(f"{h!r} {N} {B} {k} {vals}")
        print(f"h={h} N={N} B={B} k={k}: {time.perf_counter() - t0:.0f} s", flush=True)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_forces.txt")
    with open(out, "w") as f:
        f.write("# oracle force and torque, whole evaluations (tests/golden/make_fullsize.py)\n")
        f.write("# h N bounces k Fx Fy Fz Tx Ty Tz\n")
        for ln in lines:
            f.write(ln + "\n")


if __name__ == "__main__":
    main()
