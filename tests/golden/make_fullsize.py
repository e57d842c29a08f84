"""Writes fullsize_forces.txt: the oracle's force and torque for whole
evaluations at the benchmark sizes, which no GPU test can afford to trace with
the oracle at run time.

Each line: mesh facet h, N, bounces, index k of the 4096-point Fibonacci
direction table, then Fx Fy Fz (N) and Tx Ty Tz (N m), FP64 as written by
repr().  Cases: three directions of the ~50k-triangle precision form and two
of the ~200k-triangle headline used by the parity tests, and 16 seeded
directions of the precision form for the benchmark's per-direction error
report; lines already in the file are kept, only missing cases are traced.  Meshes come from paper_2608_07307_gb300.inputs.spacecraft(h); every
value is computed by oracle.evaluate (ray-sharded over spawn-started
processes, partial sums added in a fixed order), nothing else.

    python tests/golden/make_fullsize.py [procs]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def seeded_precision_directions():
    """The 16 directions of the 4096-point table on which the precision form
    (~50k triangles, 1024^2 rays, 2 bounces) is compared whole with the
    oracle: distinct indices from the seeded uniform stream (seed 16)."""
    from paper_2608_07307_gb300 import inputs as I
    u = I.uniform01(16, 64)
    ks = []
    for x in u:
        k = int(x * 4096)
        if k not in ks:
            ks.append(k)
        if len(ks) == 16:
            break
    return sorted(ks)


def cases():
    c = [
        # the precision form: ~50k triangles, 1024^2 rays, 2 bounces
        (0.05, 1024, 2, 0), (0.05, 1024, 2, 1365), (0.05, 1024, 2, 2730),
        # the headline: ~200k triangles, 1024^2 rays, 2 bounces
        (0.025, 1024, 2, 0), (0.025, 1024, 2, 17),
    ]
    c += [(0.05, 1024, 2, k) for k in seeded_precision_directions() if (0.05, 1024, 2, k) not in c]
    return c


def main():
    from oracle import oracle as O
    from paper_2608_07307_gb300 import inputs as I

    procs = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    dirs = I.sun_dirs_fibonacci(4096)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_forces.txt")
    # lines this script wrote before are kept (the oracle is deterministic)
    have = {}
    if os.path.exists(out):
        for ln in open(out):
            if ln.startswith("#") or not ln.strip():
                continue
            v = ln.split()
            have[(float(v[0]), int(v[1]), int(v[2]), int(v[3]))] = ln.rstrip("\n")
    meshes = {}
    lines = []
    for h, N, B, k in cases():
        if (h, N, B, k) in have:
            lines.append(have[(h, N, B, k)])
            continue
        if h not in meshes:
            meshes[h] = I.spacecraft(h)
        t0 = time.perf_counter()
        r = O.evaluate(meshes[h], dirs[k], N, B, procs=procs)
        vals = " ".join(repr(float(x)) for x in list(r["F"]) + list(r["T"]))
        lines.append(f"{h!r} {N} {B} {k} {vals}")
        print(f"h={h} N={N} B={B} k={k}: {time.perf_counter() - t0:.0f} s", flush=True)
        _write(out, lines + [have[c] for c in have if have[c] not in lines])
    _write(out, lines)


def _write(out, lines):
    with open(out, "w") as f:
        f.write("# oracle force and torque, whole evaluations (tests/golden/make_fullsize.py)\n")
        f.write("# h N bounces k Fx Fy Fz Tx Ty Tz\n")
        for ln in lines:
            f.write(ln + "\n")


if __name__ == "__main__":
    main()
