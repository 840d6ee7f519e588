"""The index-checked build of the library (-DJXF_DEBUG: every computed
stencil and face index is checked against its array and clamped, a
violation reported as JXF_ERR_BOUNDS) on small runs of every kernel family,
in a process of its own: no index leaves its array, and the results agree
with the release build (to round-off: the checks may change how the compiler
schedules and contracts the arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def test_checked_build_finds_no_index_outside_its_array(tmp_path):
    from paper_2402_05193_gb300 import build
    lib = build.build_checked()
    out_c, out_r = str(tmp_path / "checked.npz"), str(tmp_path / "release.npz")
    env = dict(os.environ, JXF_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_runs.py"), out_c], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    sys.path.insert(0, HERE)
    import checked_runs
    checked_runs.run(out_r)  # this process's (release) library
    a, b = np.load(out_c), np.load(out_r)
    assert sorted(a.files) == sorted(b.files)
    worst = {}
    for k in a.files:
        x, y = a[k], b[k]
        scale = np.maximum(np.abs(y).reshape(y.shape[0], -1).max(axis=1), 1e-300)
        err = (np.abs(x - y).reshape(y.shape[0], -1).max(axis=1) / scale).max()
        worst[k] = float(err)
        tol = 1e-5 if ("fp32" in k or k.startswith("batch")) else 1e-10
        assert err <= tol, (k, err)
    print("checked vs release build, per run max rel difference:", worst)
