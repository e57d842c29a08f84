"""Host-side pieces of bench.py that need no GPU: the parity record's reading
of the stored oracle forces and its error arithmetic."""
import os
import sys
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _FakeCtx:
    """Returns the stored oracle values for the directions asked (by index in
    the Fibonacci table), optionally perturbed."""

    def __init__(self, rows, rel=0.0):
        from paper_2608_07307_gb300 import inputs as I
        self.dirs = I.sun_dirs_fibonacci(4096)
        self.rows = rows
        self.rel = rel

    def eval_batch(self, mid, dirs, N, bounces):
        F, T = [], []
        for d in dirs:
            k = int(np.argmin(np.abs(self.dirs - d).sum(axis=1)))
            r = next(r for r in self.rows if int(r[3]) == k and int(r[1]) == N and int(r[2]) == bounces)
            F.append([float(x) * (1 + self.rel) for x in r[4:7]])
            T.append([float(x) for x in r[7:10]])
        return np.array(F), np.array(T)


def _rows(facet=0.025):
    path = os.path.join(ROOT, "tests", "golden", "fullsize_forces.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return [r for r in rows if float(r[0]) == facet]


def test_parity_record_reads_the_stored_oracle_forces():
    sys.path.insert(0, ROOT)
    import bench
    a = SimpleNamespace(facet=0.025, N=1024, bounces=2)
    rec = bench.parity_record(_FakeCtx(_rows()), 0, a)
    assert rec["directions"] == [0, 17]
    assert rec["force_rel_err_max"] == 0.0 and rec["torque_rel_err_max"] == 0.0
    rec = bench.parity_record(_FakeCtx(_rows(), rel=2e-5), 0, a)
    assert abs(rec["force_rel_err_max"] - 2e-5) < 1e-12
    # sizes the file holds no oracle values for
    assert bench.parity_record(_FakeCtx(_rows()), 0, SimpleNamespace(facet=0.025, N=512, bounces=1)) is None


def test_relative_errors_and_golden_rows():
    """The per-direction error the bench reports: force relative to the oracle
    force's norm, torque relative to the larger of the oracle's torque and force
    norms (a torque near zero is judged against the force's scale); and the
    stored rows it compares with."""
    sys.path.insert(0, ROOT)
    import bench
    Fo = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 2.0]])
    To = np.array([[0.0, 0.0, 10.0], [0.0, 0.0, 0.0]])
    F = Fo + np.array([[0.0, 0.0, 5e-5], [1e-4, 0.0, 0.0]])
    T = To + np.array([[0.0, 1e-3, 0.0], [0.0, 2e-4, 0.0]])
    rf, rt = bench._rel_errors(F, T, Fo, To)
    assert np.allclose(rf, [1e-5, 5e-5]) and np.allclose(rt, [1e-4, 1e-4])
    rows = bench._golden_rows("boxwing_forces.txt")
    assert len(rows) == 256 and all(len(r) == 7 for r in rows)
    assert bench._golden_rows("no_such_file.txt") == []
