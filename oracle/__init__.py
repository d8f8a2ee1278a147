"""ORACLE — test infrastructure only.

Python access to the plain C oracle in ``lbl_oracle.c`` (the CPU definition of
the labeling path of arXiv 1810.02612).  Only ``tests/``, the smoke check and
the benchmark's CPU-baseline leg import this package; the product library never
does, and the two share no code.

Every function takes and returns numpy arrays in the same layouts as the
C-ABI of the product library:

* ``planes``  uint8[P][h][w]  world-frame occupancy, one plane per proposition
* ``O``       uint64[cells]   proposition word per agent cell (bit p = prop p)
* ``rowptr``  int64[E+1], ``colidx`` int32[nnz]  CSR rows of the trajectory
  matrix M (eq. 11)
* ``L``       uint64[E]       label word per edge (eq. 10)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbl_oracle.c")
_LIB = os.path.join(_HERE, "_liblbl_oracle.so")

ROWMAJOR = 0
MORTON = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library (gcc, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.orc_morton.restype = ctypes.c_uint64
        lib.orc_morton.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        lib.orc_cell_index.restype = i64
        lib.orc_cell_index.argtypes = [i32, i32, i32, i32]
        lib.orc_frame_coeffs.restype = None
        lib.orc_frame_coeffs.argtypes = [f64] * 9 + [p]
        lib.orc_frame_transform.restype = ctypes.c_int
        lib.orc_frame_transform.argtypes = [i32, i32, f64, f64, f64, p, i32, f64, f64, f64,
                                            i32, i32, f64, f64, f64, i32, p]
        lib.orc_label.restype = None
        lib.orc_label.argtypes = [i64, p, p, p, i32, p, i32]
        lib.orc_label_rows.restype = None
        lib.orc_label_rows.argtypes = [i64, p, p, p, p, i32, p]
        lib.orc_monitor.restype = ctypes.c_int
        lib.orc_monitor.argtypes = [i32, i32, p, p, i32, p, i64, p, p]
        lib.orc_arc_geometry.restype = None
        lib.orc_arc_geometry.argtypes = [p, p]
        lib.orc_arc_dist.restype = f64
        lib.orc_arc_dist.argtypes = [p, p, f64, f64]
        lib.orc_sweep.restype = i64
        lib.orc_sweep.argtypes = [i64, p, f64, i32, i32, f64, f64, f64, i32, p, p]
        lib.orc_morton3.restype = ctypes.c_uint64
        lib.orc_morton3.argtypes = [ctypes.c_uint32] * 3
        lib.orc_cell_index3.restype = i64
        lib.orc_cell_index3.argtypes = [i32] * 6
        lib.orc_time_coeffs.restype = None
        lib.orc_time_coeffs.argtypes = [f64] * 5 + [p]
        lib.orc_frame_transform3.restype = ctypes.c_int
        lib.orc_frame_transform3.argtypes = ([i32, i32, i32] + [f64] * 5 + [p, i32] + [f64] * 4 + [i32, i32, i32]
                                             + [f64] * 5 + [i32, p])
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def morton(ix: int, iy: int) -> int:
    """z-order index of cell (ix, iy) (Sec. 4.1)."""
    return int(_load().orc_morton(ix, iy))


def cell_index(order: int, w: int, ix: int, iy: int) -> int:
    return int(_load().orc_cell_index(order, w, ix, iy))


def frame_coeffs(world, agent, pose) -> np.ndarray:
    """Q32.32 coefficients {A00, A01, B0, A10, A11, B1} of the agent-cell ->
    world-cell map at ``pose`` = (X, Y, theta)."""
    out = np.zeros(6, np.int64)
    _load().orc_frame_coeffs(world.res, world.x0, world.y0, agent.res, agent.x0, agent.y0,
                             float(pose[0]), float(pose[1]), float(pose[2]), _ptr(out))
    return out


def frame_transform(world, planes: np.ndarray, pose, agent) -> np.ndarray:
    """Agent-frame proposition words O at ``pose`` (Sec. 5, eq. 13)."""
    planes = np.ascontiguousarray(planes, dtype=np.uint8)
    P = planes.shape[0]
    assert planes.shape[1:] == (world.h, world.w)
    O = np.zeros(agent.w * agent.h, np.uint64)
    rc = _load().orc_frame_transform(world.w, world.h, world.res, world.x0, world.y0, _ptr(planes), P,
                                     float(pose[0]), float(pose[1]), float(pose[2]),
                                     agent.w, agent.h, agent.res, agent.x0, agent.y0, agent.order, _ptr(O))
    if rc != 0:
        raise ValueError("oracle frame transform rejected its arguments")
    return O


def label(rowptr: np.ndarray, colidx: np.ndarray, O: np.ndarray, P: int, threads: int = 1) -> np.ndarray:
    """L = (M.O > 0) packed as one word per edge (eq. 10 over the CSR rows of eq. 11)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colidx = np.ascontiguousarray(colidx, np.int32)
    O = np.ascontiguousarray(O, np.uint64)
    E = rowptr.shape[0] - 1
    L = np.zeros(max(E, 0), np.uint64)
    if E > 0:
        _load().orc_label(E, _ptr(rowptr), _ptr(colidx), _ptr(O), P, _ptr(L), threads)
    return L


def label_rows(rows: np.ndarray, rowptr: np.ndarray, colidx: np.ndarray, O: np.ndarray, P: int) -> np.ndarray:
    """Labels of the listed rows only."""
    rows = np.ascontiguousarray(rows, np.int64)
    L = np.zeros(rows.shape[0], np.uint64)
    if rows.shape[0]:
        _load().orc_label_rows(rows.shape[0], _ptr(rows), _ptr(np.ascontiguousarray(rowptr, np.int64)),
                               _ptr(np.ascontiguousarray(colidx, np.int32)),
                               _ptr(np.ascontiguousarray(O, np.uint64)), P, _ptr(L))
    return L


def monitor(n_states: int, m: int, relbits, delta, reject: int, L: np.ndarray):
    """Per-edge next-state word and violation mask of a safety monitor (Sec. 3.2)."""
    relbits = np.ascontiguousarray(relbits, np.uint8)
    delta = np.ascontiguousarray(delta, np.uint8)
    L = np.ascontiguousarray(L, np.uint64)
    n = L.shape[0]
    nxt = np.zeros(n, np.uint64)
    viol = np.zeros(n, np.uint16)
    rc = _load().orc_monitor(n_states, m, _ptr(relbits), _ptr(delta), reject, _ptr(L), n, _ptr(nxt), _ptr(viol))
    if rc != 0:
        raise ValueError("oracle monitor rejected its arguments")
    return nxt, viol


def morton3(ix: int, iy: int, it: int) -> int:
    """3-D z-order index of cell (ix, iy, it) of the (x, y, tau) workspace."""
    return int(_load().orc_morton3(ix, iy, it))


def cell_index3(order: int, w: int, h: int, ix: int, iy: int, it: int) -> int:
    return int(_load().orc_cell_index3(order, w, h, ix, iy, it))


def frame_transform3(world, vols: np.ndarray, pose, agent) -> np.ndarray:
    """Agent-frame words of a time-augmented workspace: vols uint8[P][d][h][w],
    pose (X, Y, theta, T); grids carry d, tres, t0 (Sec. 5, eq. 13)."""
    vols = np.ascontiguousarray(vols, dtype=np.uint8)
    P = vols.shape[0]
    assert vols.shape[1:] == (world.d, world.h, world.w)
    O = np.zeros(agent.w * agent.h * agent.d, np.uint64)
    rc = _load().orc_frame_transform3(world.w, world.h, world.d, world.res, world.x0, world.y0, world.tres,
                                      world.t0, _ptr(vols), P, float(pose[0]), float(pose[1]), float(pose[2]),
                                      float(pose[3]), agent.w, agent.h, agent.d, agent.res, agent.x0, agent.y0,
                                      agent.tres, agent.t0, agent.order, _ptr(O))
    if rc != 0:
        raise ValueError("oracle 3-D frame transform rejected its arguments")
    return O


def sweep(arcs: np.ndarray, radius: float, grid):
    """Swept-cell rows (rowptr, colidx) of arcs (x, y, heading, curvature,
    length) over every cell of a 2-D grid: eq. 7 with a disc footprint,
    discretised by cell centres."""
    arcs = np.ascontiguousarray(arcs, np.float64).reshape(-1, 5)
    n = arcs.shape[0]
    counts = np.zeros(max(n, 1), np.int64)
    total = _load().orc_sweep(n, _ptr(arcs), float(radius), grid.w, grid.h, grid.res, grid.x0, grid.y0,
                              grid.order, _ptr(counts), None)
    keys = np.zeros(max(total, 1), np.int32)
    _load().orc_sweep(n, _ptr(arcs), float(radius), grid.w, grid.h, grid.res, grid.x0, grid.y0, grid.order,
                      _ptr(counts), _ptr(keys))
    rowptr = np.zeros(n + 1, np.int64)
    rowptr[1:] = np.cumsum(counts[:n])
    return rowptr, keys[:total]
