"""The bounds-checked debug build (libbgk_debug.so: every neighbour and point index a
kernel loads is checked against the point range, a bad one recorded as BGK_E_BOUNDS and
its access skipped) steps the cavities as the regular build does: no index is out of
range, and f and the moments agree bit for bit (the checks touch no arithmetic).  It runs
in a subprocess, since a process loads one of the two libraries."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bgk_inputs as bi

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CASES = [("cavity2d_n41_v16_f64", {"storage": "f32"}, 20),
          ("cavity2d_ale_n201_v32_f32", {"n": 31, "nv": 12}, 10),
          ("cavity3d_n41_v16_f32", {"n": 9, "nv": 8}, 5),
          ("cavity2d_n41_v16_f64", {"n": 21, "nv": 8}, 10)]

_SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
import bgk_inputs as bi
import paper_2408_02350_gb300 as g
out = {}
for k, (name, over, steps) in enumerate(json.loads(sys.argv[1])):
    p = bi.config(name, **over)
    s = g.Solver([p], [bi.cloud_for(p)])
    s.set_maxwellian()
    s.step(steps)
    s.sync()
    np.save(sys.argv[2] + "/f%%d.npy" %% k, s.get_f())
    rho, u, T = s.moments()
    np.save(sys.argv[2] + "/m%%d.npy" %% k, np.concatenate([rho, u.ravel(), T]))
    s.close()
print(g.LIB_PATH)
"""


def _run(tmp, debug):
    env = dict(os.environ)
    env.pop("BGK_LIBRARY", None)
    if debug:
        env["BGK_LIBRARY"] = "debug"
    os.makedirs(tmp, exist_ok=True)
    r = subprocess.run([sys.executable, "-c", _SCRIPT % {"root": ROOT}, json.dumps(_CASES), tmp], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()[-1]


def test_debug_build_steps_like_the_regular_build(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_02350_gb300 import _build
    _build.build()
    _build.build(debug=True)
    a, b = str(tmp_path / "regular"), str(tmp_path / "debug")
    assert _run(a, False).endswith("libbgk.so")
    assert _run(b, True).endswith("libbgk_debug.so")
    for k in range(len(_CASES)):
        for stem in ("f", "m"):
            x = np.load(os.path.join(a, "%s%d.npy" % (stem, k)))
            y = np.load(os.path.join(b, "%s%d.npy" % (stem, k)))
            assert np.array_equal(x, y), (k, stem, np.abs(x - y).max())
