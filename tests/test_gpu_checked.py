"""The bounds-checked debug build (-DQG_CHECKED) on small and ragged grids.

In that build every shared-memory and global access of the generic row and column passes and of their FFT checks
its index against the array's extent; an index outside it sets a status bit (QG_ERR_BOUNDS at the next sync) and
the access is skipped, so a wrong index is reported instead of touching memory outside the array.  The grids
N = 16, 18, 24 and 54 run those kernels with partial column tiles (6, 7, 8 and 18 kept k_x columns against tiles of
4 or 2) and radix-3 passes.  Every closure, both schemes and both precisions step here through the checked library,
loaded in a child process (the binding keeps one library per process), and must report no bad index and match
the oracle.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2508_06678_gb300 as qg
import oracle as O
import synth as S

def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))

count = 0
for n in (16, 18, 24, 54):
    for kind in (S.NONE, S.SMAG, S.LEITH, S.DSMAG, S.DLEITH):
        for scheme in (O.RK3_EXACT, O.AB2CN):
            dt, eta = (2e-3, 1e-3) if scheme == O.RK3_EXACT else (5e-4, 2e-3)
            wl = S.Workload("chk", n, "island", beta=5.0, U=0.5, closure=kind, c=0.2, radius=0.9, seed=n + kind,
                            dt=dt, eta=eta)
            w0 = S.init_field(n + kind, n, k_peak=n / 5)
            ref = O.QGOracle(n, wl.L, wl.beta, wl.U, wl.mask(), wl.sponge_field(), O.Closure(kind, c=0.2),
                             O.Params(dt=dt, eta=eta, scheme=scheme))
            ref.set_state(w0)
            ref.step(3)
            for prec, tol in ((qg.QG_FP64, 1e-12), (qg.QG_FP32, 1e-4)):
                with qg.QGSolver.from_workload(wl, precision=prec, scheme=scheme) as s:
                    s.set_state(w0)
                    s.step(3)
                    s.sync()  # raises QGError(QG_ERR_BOUNDS) if any checked access was out of range
                    got = s.get_state()
                    s.diagnostics()
                err = rel(got, ref.get_state())
                assert err < tol, (n, kind, scheme, prec, err)
                count += 1
print("checked runs", count)
"""


@pytest.fixture(scope="module")
def checked_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_06678_gb300.build import CHECKED_DIR, build_checked
    path = os.path.join(CHECKED_DIR, "libqg.so")
    if not os.path.exists(path):
        build_checked()
    return path


def test_checked_build_small_and_ragged_grids(checked_lib):
    env = dict(os.environ, QG_LIB=checked_lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked runs 80" in r.stdout
