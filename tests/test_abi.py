"""The C-ABI library builds, loads and exports every symbol include/bgk.h declares (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import bgk_inputs as bi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_02350_gb300 import _build
    _build.build()
    import paper_2408_02350_gb300 as g
    return g


def _declared():
    src = open(os.path.join(ROOT, "include", "bgk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bgk_[a-z_]+)\s*\(", src)))


def test_header_declares_the_expected_entry_points():
    names = _declared()
    for must in ("bgk_init", "bgk_neighbours", "bgk_step", "bgk_moments", "bgk_free", "bgk_sync"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    h = C.CDLL(lib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(h, n)]
    assert not missing, missing
    assert set(_declared()) <= set(lib.exported_symbols()) | {"bgk_version"}
    assert lib.bgk_version() == 9


def test_error_codes_match_header(lib):
    src = open(os.path.join(ROOT, "include", "bgk.h")).read()
    codes = {name: int(v) for name, v in re.findall(r"\b(BGK_(?:OK|E_[A-Z_]+))\s*=\s*(\d+)", src)}
    assert codes["BGK_E_BOUNDS"] == 9
    for name, v in codes.items():
        assert getattr(lib, name) == v, name


def test_build_variants_are_selected_by_name(tmp_path):
    # each variant builds into a library of its own, and BGK_LIBRARY picks it at import
    import subprocess
    import sys
    from paper_2408_02350_gb300 import _build
    assert set(_build.VARIANTS) == {"debug", "staged"}
    assert _build.lib_path(None) == _build.LIB
    for v in _build.VARIANTS:
        assert _build.lib_path(v).endswith("libbgk_%s.so" % v)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for v, want in (("staged", "libbgk_staged.so"), ("debug", "libbgk_debug.so"), ("other", "libbgk.so")):
        env = dict(os.environ, BGK_LIBRARY=v)
        r = subprocess.run([sys.executable, "-c", "import paper_2408_02350_gb300 as g; print(g.LIB_PATH)"],
                           cwd=root, env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-1000:]
        assert r.stdout.strip().endswith(want), (v, r.stdout)


def test_bounds_checked_debug_build_exports_every_symbol():
    # the debug build (every list index a kernel loads checked against the point range)
    # compiles for sm_103a and exports the same ABI
    from paper_2408_02350_gb300 import _build
    path = _build.build(debug=True)
    h = C.CDLL(path)
    missing = [n for n in _declared() if not hasattr(h, n)]
    assert not missing, missing
    assert h.bgk_version() == 9


@pytest.mark.parametrize("struct", ["bgk_params", "bgk_stats"])
def test_struct_layout_matches_header(lib, struct, tmp_path):
    # sizes and field offsets of the ctypes mirrors against a C compiler's view of include/bgk.h
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    q = getattr(lib, struct)
    names = [f[0] for f in q._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {n}));\n' for n in names)
    src.write_text(f'#include <stddef.h>\n#include <stdio.h>\n#include "bgk.h"\nint main(void) {{\n'
                   f'  printf("%zu\\n", sizeof({struct}));\n{body}  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == C.sizeof(q)
    assert out[1:] == [getattr(q, n).offset for n in names]


@pytest.mark.parametrize("field,value", [("dim", 4), ("nv", 1), ("nv", 65), ("storage", 3), ("max_nbrs", 0),
                                         ("dt", 0.0), ("h", -1.0), ("tau_mode", 5), ("kn", 0.0)])
def test_init_rejects_bad_parameters_before_touching_the_device(lib, field, value):
    p = bi.config("cavity2d_n41_v16_f64", n=5)
    cl = bi.cloud_for(p)
    q = lib.params_from(p)
    setattr(q, field, value)
    with pytest.raises(lib.BGKError) as e:
        lib.bgk_init([q], [len(cl["kind"])], cl["x"], cl["kind"], cl["normal"])
    assert e.value.code == lib.BGK_E_INVAL
    assert "bgk_init" in lib.bgk_last_error(None)


@pytest.mark.parametrize("what,value", [("x", float("nan")), ("x", 1.5), ("x", -0.1), ("kind", -1),
                                        ("normal", float("inf"))])
def test_init_rejects_corrupt_geometry_before_touching_the_device(lib, what, value):
    # a corrupted position, kind or normal of one point of the second case
    p = bi.config("cavity2d_n41_v16_f64", n=5)
    cl = bi.cloud_for(p)
    n = len(cl["kind"])
    x = np.concatenate([cl["x"], cl["x"]])
    kind = np.concatenate([cl["kind"], cl["kind"]])
    normal = np.concatenate([cl["normal"], cl["normal"]])
    i = n + 7
    if what == "x":
        x[i, 1] = value
    elif what == "kind":
        kind[i] = value
    else:
        normal[i, 0] = value
    q = lib.params_from(p)
    with pytest.raises(lib.BGKError) as e:
        lib.bgk_init([q, q], [n, n], x, kind, normal)
    assert e.value.code == lib.BGK_E_INVAL
    msg = lib.bgk_last_error(None)
    assert "case 1" in msg and "point 7" in msg, msg


@pytest.mark.parametrize("change", ["moving_without_ale", "lid_id", "negative_radius", "negative_id"])
def test_init_rejects_bad_body_parameters(lib, change):
    p = bi.config("body2d_ale_n201_v32_f32", n=11, nv=4, storage="f64", body_radius=0.2, body_centre=[0.5, 0.5, 0.0])
    cl = bi.cloud_for(p)
    q = lib.params_from(p)
    if change == "moving_without_ale":
        q.ale = 0
    elif change == "lid_id":
        q.body_wall = q.lid_wall
    elif change == "negative_radius":
        q.body_radius = -0.1
    else:
        q.body_wall = -1
    with pytest.raises(lib.BGKError) as e:
        lib.bgk_init([q], [len(cl["kind"])], cl["x"], cl["kind"], cl["normal"])
    assert e.value.code == lib.BGK_E_INVAL
    assert "body" in lib.bgk_last_error(None)


@pytest.mark.parametrize("order,ale", [(3, 0), (-1, 0), (2, 1)])
def test_init_rejects_bad_time_orders(lib, order, ale):
    p = bi.config("cavity2d_n41_v16_f64", n=5, time_order=order, ale=ale)
    cl = bi.cloud_for(p)
    with pytest.raises(lib.BGKError) as e:
        lib.bgk_init([lib.params_from(p)], [len(cl["kind"])], cl["x"], cl["kind"], cl["normal"])
    assert e.value.code == lib.BGK_E_INVAL
    assert "time_order" in lib.bgk_last_error(None)


@pytest.mark.parametrize("lo,hi", [(2, 8), (8, 8), (12, 8), (0, 300), (-4, 8), (4, 0)])
def test_init_rejects_bad_velocity_slabs(lib, lo, hi):
    # nv = 16 in 2D: 256 velocities; starts must be multiples of 4, 0 <= lo < hi <= 256
    p = bi.config("cavity2d_n41_v16_f64", n=5, vk_lo=lo, vk_hi=hi)
    cl = bi.cloud_for(p)
    with pytest.raises(lib.BGKError) as e:
        lib.bgk_init([lib.params_from(p)], [len(cl["kind"])], cl["x"], cl["kind"], cl["normal"])
    assert e.value.code == lib.BGK_E_INVAL
    assert "slab" in lib.bgk_last_error(None)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2408_02350_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"(#|//).*", "", text).lower() or f.endswith(".md"), f
