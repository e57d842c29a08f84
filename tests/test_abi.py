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
