"""The C-ABI library builds, loads and exports every function include/*.h declares.
No compute call runs here (CPU only)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \t\*]*?\b(srp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("srp_create", "srp_destroy", "srp_last_error", "srp_mesh_load", "srp_set_panel_angles",
              "srp_eval_batch"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2608_07307_gb300 import build, srp
    path = build.build()
    lib = C.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert sorted(srp.EXPORTS) == declared_functions()


def test_create_fails_loudly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2608_07307_gb300 import srp
    with pytest.raises(srp.SrpError) as e:
        srp.Context(0)
    assert e.value.code == -3


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror of an include/srp.h struct has the C size and the C
    offset for each field (gcc compiles a probe of the header here)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_2608_07307_gb300 import srp
    pairs = {"srp_mesh_desc": srp.MeshDesc, "srp_eval_params": srp.EvalParams, "srp_eval_stats": srp.EvalStats,
             "srp_spad_grid": srp.SpadGrid, "srp_prop_params": srp.PropParams, "srp_prop_stats": srp.PropStats,
             "srp_traj": srp.Traj}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "srp.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])


def test_binding_constants_match_the_header():
    """Every #define of include/srp.h that the binding mirrors (under its own
    name or without the SRP_ prefix) has the header's value."""
    from paper_2608_07307_gb300 import srp
    text = open(os.path.join(ROOT, "include", "srp.h")).read()
    defs = dict(re.findall(r"^#define\s+(SRP_\w+)\s+\(?(-?\d+)\)?", text, flags=re.M))
    checked = 0
    for name, val in defs.items():
        for py in (name, name[len("SRP_"):]):
            if hasattr(srp, py) and isinstance(getattr(srp, py), int):
                assert getattr(srp, py) == int(val), (name, py, getattr(srp, py), val)
                checked += 1
                break
    assert checked >= 15, checked
