"""The C ABI without a GPU: the library builds, loads, exports every function
declared in include/dcem.h, and validates arguments before any device work
(an invalid call returns a status code, never crashes)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2112_07115_gb300 import build
    build.build()
    from paper_2112_07115_gb300 import dcem
    return dcem


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dcem.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dcem_[a-z_]+)\s*\(", txt)))


def test_header_declares_expected_calls():
    names = declared_functions()
    for must in ["dcem_scene_create", "dcem_scene_update_transforms", "dcem_trace_frame",
                 "dcem_scene_reset_cache", "dcem_scene_destroy", "dcem_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(L.EXPORTED)


def test_struct_sizes_match_header(L):
    assert C.sizeof(L.Path) == 224
    assert C.sizeof(L.Params) == 64
    assert L.PATH_DTYPE.itemsize == 224


def test_status_strings(L):
    for st in range(0, -9, -1):
        s = L.status_string(st)
        assert s and s != "unknown status"
    assert L.status_string(-99) == "unknown status"


def test_params_default(L):
    p = L.default_params()
    assert p.freq_hz == 28e9 and p.tx_power_w == 5.0 and p.max_refl == 3
    assert p.mode == L.MODE_FULL and abs(p.rx_radius_scale - 1.35) < 1e-6
    assert list(p.pol) == [0.0, 0.0, 1.0]


def _create(L, tris, mats_idx, mats, tri_obj=None, nobj=0):
    lib = L.lib()
    h = C.c_void_p()
    tris = np.ascontiguousarray(tris, np.float32)
    mi = np.ascontiguousarray(mats_idx, np.int32)
    marr = (L.Material * max(1, len(mats)))()
    for i, (e, s, p) in enumerate(mats):
        marr[i].eps_r, marr[i].sigma, marr[i].pec = e, s, p
    to = None if tri_obj is None else np.ascontiguousarray(tri_obj, np.int32)
    rc = lib.dcem_scene_create(tris.ctypes.data if tris.size else None, tris.size // 9,
                               mi.ctypes.data if mi.size else None, marr, len(mats),
                               to.ctypes.data if to is not None else None, nobj, None, C.byref(h))
    return rc, h


def test_create_argument_errors(L):
    tri = np.zeros((1, 9), np.float32)
    conc = [(5.31, 0.0326, 0)]
    assert L.lib().dcem_scene_create(None, 0, None, None, 0, None, 0, None, None) == L.ERR_ARG
    assert _create(L, tri, [1], conc)[0] == L.ERR_ARG                 # material out of range
    assert _create(L, tri, [0], conc, tri_obj=[2], nobj=1)[0] == L.ERR_ARG  # object out of range
    assert _create(L, tri, [0], [])[0] == L.ERR_ARG                   # no materials
    assert _create(L, tri, [0], [(5.0, -1.0, 0)])[0] == L.ERR_ARG     # negative conductivity
    bad = tri.copy()
    bad[0, 4] = np.nan
    assert _create(L, bad, [0], conc)[0] == L.ERR_NONFINITE


def test_null_scene_calls(L):
    lib = L.lib()
    p = L.default_params()
    r = L.Result()
    tx = (C.c_float * 3)(0, 0, 0)
    assert lib.dcem_trace_frame(None, tx, None, 0, 0, C.byref(p), C.byref(r)) == L.ERR_ARG
    assert lib.dcem_scene_set_rays(None, None, 0) == L.ERR_ARG
    assert lib.dcem_scene_update_transforms(None, None, 0) == L.ERR_ARG
    assert lib.dcem_scene_reset_cache(None) == L.ERR_ARG
    assert lib.dcem_scene_set_graph_replay(None, 1) == L.ERR_ARG
    assert lib.dcem_scene_set_trace_config(None, -1, 256, 24) == L.ERR_ARG
    assert lib.dcem_batch_create(None, 1, None, None) == L.ERR_ARG
    assert lib.dcem_batch_update_transforms(None, None, 0) == L.ERR_ARG
    assert lib.dcem_batch_trace(None, None, None, None, None, 0, C.byref(p), None, None) == L.ERR_ARG
    lib.dcem_batch_destroy(None)
    assert lib.dcem_scene_set_transmission(None, None, 0, 1) == L.ERR_ARG
    assert lib.dcem_scene_set_diffraction(None, 1, None) == L.ERR_ARG
    assert lib.dcem_scene_autotune(None, tx, 1, None, 0, 0, C.byref(p), 1, None, None, None) == L.ERR_ARG
    n = (C.c_int32 * 1)(4)
    assert lib.dcem_scene_set_ray_sets(None, None, n, 1) == L.ERR_ARG
    assert lib.dcem_trace_links(None, tx, 1, None, 0, 0, C.byref(p), C.byref(r)) == L.ERR_ARG
    assert lib.dcem_scene_info(None, None, None, None, None, None) == L.ERR_ARG
    n = C.c_int32(0)
    assert lib.dcem_scene_gradient_size(None, C.byref(n)) == L.ERR_ARG
    assert lib.dcem_path_gradients(None, tx, None, 0, 0, None, 0, C.byref(p), 0, None, None, None) == L.ERR_ARG
    lib.dcem_scene_destroy(None)  # no-op


def test_valid_create_without_gpu_reports_cuda_error(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("this machine has a GPU")
    rc, h = _create(L, np.zeros((1, 9), np.float32), [0], [(5.31, 0.0326, 0)])
    assert rc == L.ERR_CUDA and not h.value


def _c_layout(tmp_path, structs):
    """sizeof and field offsets of the header's structs, as a C compiler lays
    them out (gcc, the header alone)."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dcem.h"', "int main(void) {"]
    for cname, fields in structs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        a, b, c = ln.split()
        got[(a, b)] = int(c)
    return got


def test_ctypes_layout_matches_header(L, tmp_path):
    pairs = [("dcem_material", L.Material), ("dcem_params", L.Params), ("dcem_path", L.Path),
             ("dcem_stats", L.Stats), ("dcem_result", L.Result)]
    structs = [(c, [f for f, _ in py._fields_]) for c, py in pairs]
    got = _c_layout(tmp_path, structs)
    for cname, py in pairs:
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
