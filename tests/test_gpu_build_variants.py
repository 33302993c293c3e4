"""The build variants step the cavities as the regular build does, f and the moments bit
for bit:
- debug (libbgk_debug.so): every neighbour and point index a kernel loads is checked
  against the point range, a bad one recorded as BGK_E_BOUNDS and its access skipped; no
  index is out of range here and the checks touch no arithmetic;
- staged (libbgk_staged.so): the 2D FP32 transport takes its neighbour rows through
  per-warp rings of bulk copies into shared memory, completion counted on mbarriers,
  instead of through L1; the same sums in the same order (the last velocity slice of the
  12^2 and 20^2 grids is ragged: 4 of its 32 lanes carry velocities).
Each runs in a subprocess, since a process loads one of the libraries."""
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
          ("cavity2d_n41_v16_f64", {"n": 21, "nv": 8}, 10),
          ("body2d_ale_n201_v32_f32", {"n": 61, "nv": 20}, 10)]

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


def _run(tmp, variant):
    env = dict(os.environ)
    env.pop("BGK_LIBRARY", None)
    if variant:
        env["BGK_LIBRARY"] = variant
    os.makedirs(tmp, exist_ok=True)
    r = subprocess.run([sys.executable, "-c", _SCRIPT % {"root": ROOT}, json.dumps(_CASES), tmp], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()[-1]


@pytest.mark.parametrize("variant", ["debug", "staged"])
def test_build_variant_steps_like_the_regular_build(tmp_path, variant):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_02350_gb300 import _build
    _build.build()
    _build.build(variant=variant)
    a, b = str(tmp_path / "regular"), str(tmp_path / variant)
    assert _run(a, None).endswith("libbgk.so")
    assert _run(b, variant).endswith("libbgk_%s.so" % variant)
    for k in range(len(_CASES)):
        for stem in ("f", "m"):
            x = np.load(os.path.join(a, "%s%d.npy" % (stem, k)))
            y = np.load(os.path.join(b, "%s%d.npy" % (stem, k)))
            assert np.array_equal(x, y), (k, stem, np.abs(x - y).max())
