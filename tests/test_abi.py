"""The C-ABI library loads and exports every entry point that include/lbl.h
declares; argument checks that run before any device work reject bad input.
No kernel is launched here (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

import paper_1810_02612_gb300 as L
from paper_1810_02612_gb300 import lbl as B


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbl_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbl_roadmap_upload", "lbl_frame_transform", "lbl_label", "lbl_monitor_step"):
        assert required in names
    assert sorted(B.EXPORTS) == names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.library_path() if os.path.exists(B.library_path()) else B._build.build())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_python_binding_has_the_same_names():
    for name in declared_functions():
        assert callable(getattr(L, name)), name


def test_struct_layouts_match_the_header():
    assert ctypes.sizeof(B.lbl_grid) == 56
    assert B.lbl_grid.res.offset == 8 and B.lbl_grid.order.offset == 32
    assert B.lbl_grid.d.offset == 36 and B.lbl_grid.tres.offset == 40 and B.lbl_grid.t0.offset == 48
    assert ctypes.sizeof(B.lbl_pose) == 32
    assert ctypes.sizeof(B.lbl_config) == 24
    assert ctypes.sizeof(B.lbl_batch_tuning) == 28 and B.lbl_batch_tuning.ms.offset == 20


def test_version_and_empty_error():
    assert L.lbl_version() == 10100  # 1.1.0: the transform building the pyramid, labels from it
    assert L.lbl_last_error() == ""


@pytest.mark.parametrize("args", [
    (0, 1, [0], [[0, 0]], -1),        # no states
    (17, 0, [], [[0]] * 17, -1),       # too many states
    (2, 9, list(range(9)), np.zeros((2, 512)), -1),  # too many letter bits
    (2, 1, [64], [[0, 0], [0, 0]], -1),  # label bit out of range
    (2, 1, [3], [[0, 2], [0, 0]], -1),   # delta names a missing state
    (2, 1, [3], [[0, 1], [0, 0]], 2),    # reject is not a state
])
def test_monitor_create_rejects_bad_tables(args):
    n, m, rel, delta, rej = args
    with pytest.raises(L.LblError) as ei:
        L.lbl_monitor_create(n, m, rel, delta, rej)
    assert ei.value.code == L.LBL_EINVAL
    assert L.lbl_last_error() != ""


@pytest.mark.parametrize("grid", [
    dict(w=0, h=4, res=1.0, x0=0.0, y0=0.0, order=0),
    dict(w=4, h=4, res=0.0, x0=0.0, y0=0.0, order=0),
    dict(w=6, h=6, res=1.0, x0=0.0, y0=0.0, order=1),   # z-order needs a power of two
    dict(w=8, h=4, res=1.0, x0=0.0, y0=0.0, order=1),   # and a square
    dict(w=8, h=8, res=1.0, x0=0.0, y0=0.0, order=7),
    dict(w=8, h=8, res=1.0, x0=0.0, y0=0.0, order=1, d=4, tres=0.1, t0=0.0),  # z-order cube needs d == w
    dict(w=8, h=8, res=1.0, x0=0.0, y0=0.0, order=0, d=4, tres=0.0, t0=0.0),  # slabs need a length
    dict(w=32768, h=32768, res=1.0, x0=0.0, y0=0.0, order=0, d=4, tres=1.0, t0=0.0),  # too many cells
])
def test_roadmap_upload_rejects_bad_grids_before_device_work(grid):
    g = B.lbl_grid(**grid)
    with pytest.raises(L.LblError) as ei:
        L.lbl_roadmap_upload(g, np.zeros(1, np.int64), np.zeros(0, np.int32), stream=0)
    assert ei.value.code == L.LBL_EINVAL


def test_null_handles_are_rejected_or_ignored():
    L.lbl_roadmap_free(None)
    L.lbl_monitor_free(None)
    L.lbl_session_free(None)
    with pytest.raises(L.LblError):
        L.lbl_roadmap_info(None)
    with pytest.raises(L.LblError):
        L.lbl_label(None, 0, 1, 0, stream=0)


def test_pyramid_entry_points_refuse_a_null_roadmap():
    """The transform that builds the pyramid and the labels from it need a
    roadmap; both refuse NULL with LBL_EINVAL before any device work."""
    world = B.lbl_grid(4, 4, 0.3, 0.0, 0.0, 0)
    for call in (lambda: L.lbl_frame_transform_pyramid(None, world, 8192, 4, (0.0, 0.0, 0.0), 4096, stream=0),
                 lambda: L.lbl_label_pyramid(None, 4, 8192, stream=0)):
        with pytest.raises(L.LblError) as ei:
            call()
        assert ei.value.code == L.LBL_EINVAL and "NULL roadmap" in L.lbl_last_error()


def test_binding_refuses_host_arrays_for_device_arguments():
    g = B.lbl_grid(8, 8, 1.0, 0.0, 0.0, 0)
    with pytest.raises(TypeError):
        L.lbl_frame_transform(g, np.zeros((1, 8, 8), np.uint8), 1, (0, 0, 0), g, np.zeros(64, np.uint64), stream=0)


def header_constants():
    """Integer #defines of include/lbl.h (function-like macros excluded)."""
    out = {}
    for m in re.finditer(r"^#define\s+(LBL_[A-Z0-9_]+)\s+\(?(-?\d+)u?\)?", open(os.path.join(ROOT, "include", "lbl.h")).read(),
                         flags=re.M):
        out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_equal_the_header():
    consts = header_constants()
    assert {"LBL_OK", "LBL_EINVAL", "LBL_ALGO_QUAD", "LBL_UPLOAD_QUAD", "LBL_UPLOAD_KEEP_ORDER"} <= set(consts)
    for name, value in consts.items():
        if hasattr(B, name):
            assert getattr(B, name) == value, name
    for name in ("LBL_ALGO_AUTO", "LBL_ALGO_CSR", "LBL_ALGO_BITTILE", "LBL_ALGO_SECTOR", "LBL_ALGO_QUAD",
                 "LBL_UPLOAD_DEVICE_PTRS", "LBL_UPLOAD_BITTILE", "LBL_UPLOAD_SECTOR", "LBL_UPLOAD_QUAD",
                 "LBL_UPLOAD_KEEP_ORDER", "LBL_STAGE_TRANSFORM", "LBL_STAGE_LABEL", "LBL_ORDER_MORTON"):
        assert getattr(B, name) == consts[name], name


def test_packed_word_width_follows_the_header_macro():
    src = open(os.path.join(ROOT, "include", "lbl.h")).read()
    m = re.search(r"#define LBL_PACKED_WORD_BYTES\(n_props\)\s*(.+)", src)
    expr = m.group(1).replace("(n_props)", "P")
    # the C conditional chain ((P) <= 8 ? 1 : ...) read as nested Python conditionals
    py = re.sub(r"\(?P <= (\d+) \? (\d+) : ", r"(\2 if P <= \1 else ", expr).rstrip(")") + ")" * expr.count("?")
    for P in range(0, 65):
        assert L.packed_word_bytes(P) == eval(py, {"P": P}), P  # noqa: S307
    assert [L.packed_word_bytes(P) for P in (0, 8, 9, 16, 17, 32, 33, 64)] == [1, 1, 2, 2, 4, 4, 8, 8]


def test_transform_and_packing_refuse_bad_arguments_before_device_work():
    """Grids past 32768 cells a side, and packed words off their width's
    alignment, are refused by the host checks (the pointers here are never
    dereferenced)."""
    world = B.lbl_grid(4, 4, 0.3, 0.0, 0.0, 0)
    tall = B.lbl_grid(3, 40_000, 0.01, 0.0, 0.0, 0)
    with pytest.raises(L.LblError) as ei:
        L.lbl_frame_transform(world, 4096, 1, (0.0, 0.0, 0.0), tall, 8192, stream=0)
    assert ei.value.code == L.LBL_EINVAL
    with pytest.raises(L.LblError) as ei:
        L.lbl_pack_planes(world, 4096, 9, 8193, stream=0)  # 16-bit words at an odd address
    assert ei.value.code == L.LBL_EINVAL and "aligned" in L.lbl_last_error()
    with pytest.raises(L.LblError) as ei:
        L.lbl_frame_transform_words(world, 8194, 33, (0.0, 0.0, 0.0), world, 8192, stream=0)  # 32-bit words
    assert ei.value.code == L.LBL_EINVAL


def test_binding_refuses_to_run_without_the_library():
    """No fallback: with the CUDA library absent, loading it raises."""
    import subprocess
    import sys
    missing = os.path.join(ROOT, "_no_such_liblbl.so")
    code = ("import paper_1810_02612_gb300.lbl as B, paper_1810_02612_gb300.build as Bd\n"
            f"B._lib = None\nBd.LIB = {missing!r}\n"
            "try:\n    B.load(build_if_needed=False)\nexcept ImportError as e:\n    print('refused:', e)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "refused:" in r.stdout, r.stdout + r.stderr
