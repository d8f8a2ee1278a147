"""Python binding of liblbl (include/lbl.h): argument marshalling only.

Every function carries the C name and forwards to the shared library; all
computation happens in the CUDA kernels behind it.  Device buffers are torch
CUDA tensors (or raw integer device pointers), host buffers numpy arrays or CPU
tensors.  A non-zero status raises :class:`LblError` with the library's
message.  There is no CPU fallback: if ``liblbl.so`` cannot be built or loaded
the import of the first call fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBL_OK = 0
LBL_EINVAL = -1
LBL_ENOMEM = -2
LBL_ECUDA = -3
LBL_ETIMEOUT = -4
LBL_EUNSUPPORTED = -5

LBL_ORDER_ROWMAJOR = 0
LBL_ORDER_MORTON = 1

LBL_ALGO_AUTO = 0
LBL_ALGO_CSR = 1
LBL_ALGO_BITTILE = 2
LBL_ALGO_SECTOR = 3
LBL_ALGO_QUAD = 4
LBL_ALGO_MMA = 5

LBL_PIPE_REGISTERS = 1
LBL_PIPE_BULK = 2
LBL_PIPE_ASYNC = 3
LBL_PIPE_FRONT = 4

LBL_NOALLOC_MAX_PLANE_WORDS = 524288

LBL_STAGE_TRANSFORM = 1
LBL_STAGE_LABEL = 2

LBL_UPLOAD_DEVICE_PTRS = 1
LBL_UPLOAD_BITTILE = 2
LBL_UPLOAD_SECTOR = 4
LBL_UPLOAD_QUAD = 8
LBL_UPLOAD_KEEP_ORDER = 16
LBL_UPLOAD_MMA = 32

# every entry point declared in include/lbl.h
EXPORTS = (
    "lbl_last_error", "lbl_version",
    "lbl_roadmap_upload", "lbl_roadmap_rasterize", "lbl_roadmap_rows", "lbl_roadmap_free", "lbl_roadmap_info",
    "lbl_roadmap_form_info", "lbl_roadmap_set_wait_limit",
    "lbl_roadmap_status",
    "lbl_frame_transform", "lbl_pack_planes", "lbl_frame_transform_words",
    "lbl_monitor_create", "lbl_monitor_free", "lbl_monitor_step",
    "lbl_label", "lbl_frame_transform_pyramid", "lbl_label_pyramid", "lbl_label_blocks_noalloc",
    "lbl_roadmap_autotune", "lbl_mma_probe",
    "lbl_session_create", "lbl_session_run", "lbl_session_free",
    "lbl_batch_create", "lbl_batch_set_frames", "lbl_batch_launch", "lbl_batch_free", "lbl_batch_autotune",
    "lbl_server_create", "lbl_server_submit", "lbl_server_wait", "lbl_server_stats", "lbl_server_free",
)


class LblError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class lbl_grid(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("res", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("order", ctypes.c_int32),
                ("d", ctypes.c_int32), ("tres", ctypes.c_double), ("t0", ctypes.c_double)]


class lbl_pose(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double), ("y", ctypes.c_double), ("theta", ctypes.c_double),
                ("t", ctypes.c_double)]


class lbl_frame(ctypes.Structure):
    _fields_ = [("world", lbl_grid), ("d_planes", ctypes.c_void_p), ("pose", lbl_pose), ("d_O", ctypes.c_void_p),
                ("d_L", ctypes.c_void_p), ("d_next", ctypes.c_void_p), ("d_viol", ctypes.c_void_p)]


LBL_BATCH_CLASSES = 4


class lbl_batch_tuning(ctypes.Structure):
    _fields_ = [("word_bytes", ctypes.c_int32), ("items", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("units_per_warp", ctypes.c_int32), ("ms", ctypes.c_float),
                ("ms_default", ctypes.c_float)]


class lbl_config(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("lanes_per_edge", ctypes.c_int32),
                ("early_exit", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("pipeline", ctypes.c_int32),
                ("depth", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load liblbl.so (building it first when sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"liblbl.so is not built ({_build.LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    p, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    G = ctypes.POINTER(lbl_grid)
    sig = {
        "lbl_last_error": (ctypes.c_char_p, []),
        "lbl_version": (ctypes.c_int, []),
        "lbl_roadmap_upload": (ctypes.c_int, [G, p, p, i64, i64, u32, p, ctypes.POINTER(p)]),
        "lbl_roadmap_rasterize": (ctypes.c_int, [G, p, i64, ctypes.c_double, u32, p, ctypes.POINTER(p)]),
        "lbl_roadmap_rows": (ctypes.c_int, [p, p, p, p]),
        "lbl_roadmap_free": (ctypes.c_int, [p]),
        "lbl_roadmap_info": (ctypes.c_int, [p, p, p, p, p, p, p]),
        "lbl_roadmap_form_info": (ctypes.c_int, [p, i32, p, p]),
        "lbl_roadmap_set_wait_limit": (ctypes.c_int, [p, i64]),
        "lbl_roadmap_status": (ctypes.c_int, [p, p]),
        "lbl_frame_transform": (ctypes.c_int, [G, p, i32, lbl_pose, G, p, p]),
        "lbl_pack_planes": (ctypes.c_int, [G, p, i32, p, p]),
        "lbl_frame_transform_words": (ctypes.c_int, [G, p, i32, lbl_pose, G, p, p]),
        "lbl_monitor_create": (ctypes.c_int, [i32, i32, p, p, i32, ctypes.POINTER(p)]),
        "lbl_monitor_free": (ctypes.c_int, [p]),
        "lbl_monitor_step": (ctypes.c_int, [p, p, i64, p, p, p]),
        "lbl_label": (ctypes.c_int, [p, p, i32, p, p, p, p, ctypes.POINTER(lbl_config), p]),
        "lbl_frame_transform_pyramid": (ctypes.c_int, [p, G, p, i32, lbl_pose, p, p]),
        "lbl_label_pyramid": (ctypes.c_int, [p, i32, p, p, p, p, ctypes.POINTER(lbl_config), p]),
        "lbl_label_blocks_noalloc": (ctypes.c_int, [p, p, p, i64, p, i64, i32, p, p]),
        "lbl_roadmap_autotune": (ctypes.c_int, [p, p, i32, p, p, p, p, i32, ctypes.POINTER(lbl_config), p]),
        "lbl_mma_probe": (ctypes.c_int, [i32, i32, i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]),
        "lbl_session_create": (ctypes.c_int, [p, G, i32, p, ctypes.POINTER(lbl_config), ctypes.POINTER(p)]),
        "lbl_session_run": (ctypes.c_int, [p, p, lbl_pose, p, p, p, p]),
        "lbl_session_free": (ctypes.c_int, [p]),
        "lbl_batch_create": (ctypes.c_int, [i32, p, p, p, i32, ctypes.POINTER(p)]),
        "lbl_batch_set_frames": (ctypes.c_int, [p, ctypes.POINTER(lbl_frame)]),
        "lbl_batch_launch": (ctypes.c_int, [p, u32, p]),
        "lbl_batch_free": (ctypes.c_int, [p]),
        "lbl_batch_autotune": (ctypes.c_int, [p, i32, p, ctypes.POINTER(lbl_batch_tuning)]),
        "lbl_server_create": (ctypes.c_int, [i32, p, p, p, i32, i32, i64, ctypes.POINTER(p)]),
        "lbl_server_submit": (ctypes.c_int, [p, i32, G, p, lbl_pose, p, p, p, i64, ctypes.POINTER(i64)]),
        "lbl_server_wait": (ctypes.c_int, [p, i64, i64, ctypes.POINTER(i64)]),
        "lbl_server_stats": (ctypes.c_int, [p, p, p, p, p]),
        "lbl_server_free": (ctypes.c_int, [p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ------------------------------------------------------------- marshalling

def _grid(g) -> lbl_grid:
    if isinstance(g, lbl_grid):
        return g
    return lbl_grid(int(g.w), int(g.h), float(g.res), float(g.x0), float(g.y0), int(getattr(g, "order", 0)),
                    int(getattr(g, "d", 1)), float(getattr(g, "tres", 1.0)), float(getattr(g, "t0", 0.0)))


def _pose(p) -> lbl_pose:
    """(x, y, theta) or (x, y, theta, t)."""
    if isinstance(p, lbl_pose):
        return p
    return lbl_pose(float(p[0]), float(p[1]), float(p[2]), float(p[3]) if len(p) > 3 else 0.0)


def _cfg(cfg):
    if cfg is None:
        return None
    if isinstance(cfg, lbl_config):
        return ctypes.byref(cfg)
    c = lbl_config(int(cfg.get("algo", 0)), int(cfg.get("lanes_per_edge", 0)), int(cfg.get("early_exit", -1)),
                   int(cfg.get("ctas_per_sm", 0)), int(cfg.get("pipeline", 0)), int(cfg.get("depth", 0)))
    return ctypes.byref(c)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _dev(x, dtype_name: str, what: str):
    """Device pointer of a CUDA tensor (contiguous, given dtype) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not _is_torch(x) or not x.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    if str(x.dtype) != "torch." + dtype_name:
        raise TypeError(f"{what}: expected torch.{dtype_name}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    return x.data_ptr()


def _host(x, np_dtype, what: str):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if _is_torch(x):
        if x.is_cuda:
            raise TypeError(f"{what}: expected host memory")
        if not x.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        return x.data_ptr()
    a = x
    if not isinstance(a, np.ndarray) or a.dtype != np_dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{what}: expected a contiguous numpy {np.dtype(np_dtype).name} array")
    return a.ctypes.data


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc: int):
    if rc != LBL_OK:
        msg = load().lbl_last_error()
        raise LblError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------- entry points

def lbl_version() -> int:
    return load().lbl_version()


def lbl_last_error() -> str:
    return load().lbl_last_error().decode()


def lbl_roadmap_upload(agent, rowptr, colidx, flags: int = 0, stream=None) -> int:
    """Make a roadmap resident on the device; returns the handle.
    rowptr int64[E+1] / colidx int32[nnz]: numpy/CPU tensors, or CUDA tensors
    (then LBL_UPLOAD_DEVICE_PTRS is set)."""
    lib = load()
    E = int(rowptr.shape[0]) - 1
    nnz = int(colidx.shape[0])
    if _is_torch(rowptr) and rowptr.is_cuda:
        flags |= LBL_UPLOAD_DEVICE_PTRS
        rp, ci = _dev(rowptr, "int64", "rowptr"), _dev(colidx, "int32", "colidx")
    else:
        rp, ci = _host(rowptr, np.int64, "rowptr"), _host(colidx, np.int32, "colidx")
    out = ctypes.c_void_p()
    g = _grid(agent)
    _check(lib.lbl_roadmap_upload(ctypes.byref(g), rp, ci, E, nnz, flags, _stream(stream), ctypes.byref(out)))
    return out.value


def lbl_roadmap_rasterize(agent, arcs, radius: float, flags: int = 0, stream=None) -> int:
    """Build a roadmap on the device from arcs float64[E][5] (x, y, heading,
    curvature, length) with a disc footprint of `radius`; returns the handle."""
    a = np.ascontiguousarray(arcs, np.float64).reshape(-1, 5)
    out = ctypes.c_void_p()
    g = _grid(agent)
    _check(load().lbl_roadmap_rasterize(ctypes.byref(g), a.ctypes.data if a.size else None, a.shape[0],
                                        float(radius), int(flags), _stream(stream), ctypes.byref(out)))
    return out.value


def lbl_roadmap_rows(rm, d_rowptr, d_colidx, stream=None) -> None:
    """Copy a roadmap's rows into device tensors int64[E+1] / int32[nnz]."""
    _check(load().lbl_roadmap_rows(rm, _dev(d_rowptr, "int64", "rowptr"), _dev(d_colidx, "int32", "colidx"),
                                   _stream(stream)))


def lbl_roadmap_free(rm) -> None:
    _check(load().lbl_roadmap_free(rm))


def lbl_roadmap_info(rm):
    """(n_edges, nnz, n_block_entries, n_sector_entries, n_qdadic_entries, device_bytes) of a roadmap."""
    v = [ctypes.c_int64() for _ in range(6)]
    _check(load().lbl_roadmap_info(rm, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lbl_roadmap_form_info(rm, algo: int):
    """(entries, tiles) of one labeling form of the roadmap."""
    n, t = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().lbl_roadmap_form_info(rm, int(algo), ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def lbl_roadmap_set_wait_limit(rm, limit_ns: int) -> None:
    _check(load().lbl_roadmap_set_wait_limit(rm, int(limit_ns)))


def lbl_roadmap_status(rm, stream=None) -> None:
    """Synchronise the stream; raise LblError(LBL_ETIMEOUT) if a labeling kernel
    on this roadmap gave up a bounded wait since the last check."""
    _check(load().lbl_roadmap_status(rm, _stream(stream)))


def lbl_frame_transform(world, d_planes, n_props: int, pose, agent, d_O, stream=None) -> None:
    w, a = _grid(world), _grid(agent)
    _check(load().lbl_frame_transform(ctypes.byref(w), _dev(d_planes, "uint8", "planes"), int(n_props),
                                      _pose(pose), ctypes.byref(a), _dev(d_O, "uint64", "O"), _stream(stream)))


def packed_word_bytes(n_props: int) -> int:
    """Bytes of one packed world word (LBL_PACKED_WORD_BYTES)."""
    return 1 if n_props <= 8 else 2 if n_props <= 16 else 4 if n_props <= 32 else 8


_PACKED_DTYPES = {1: "uint8", 2: "int16", 4: "int32", 8: "uint64"}


def packed_word_dtype(n_props: int) -> str:
    """torch dtype name for a buffer of packed world words (the bits are what
    count: 16- and 32-bit words use the signed types torch supports everywhere)."""
    return _PACKED_DTYPES[packed_word_bytes(n_props)]


def _words(x, n_props: int, what: str):
    if isinstance(x, int) or x is None:
        return x
    wb = packed_word_bytes(n_props)
    if not _is_torch(x) or not x.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    if x.element_size() != wb or x.is_floating_point() or x.is_complex() or str(x.dtype) == "torch.bool":
        raise TypeError(f"{what}: expected {wb}-byte integer words for {n_props} propositions, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    return x.data_ptr()


def lbl_pack_planes(world, d_planes, n_props: int, d_words, stream=None) -> None:
    w = _grid(world)
    _check(load().lbl_pack_planes(ctypes.byref(w), _dev(d_planes, "uint8", "planes"), int(n_props),
                                  _words(d_words, n_props, "words"), _stream(stream)))


def lbl_frame_transform_words(world, d_words, n_props: int, pose, agent, d_O, stream=None) -> None:
    w, a = _grid(world), _grid(agent)
    _check(load().lbl_frame_transform_words(ctypes.byref(w), _words(d_words, n_props, "words"), int(n_props),
                                            _pose(pose), ctypes.byref(a), _dev(d_O, "uint64", "O"),
                                            _stream(stream)))


def lbl_monitor_create(n_states: int, m: int, relbits, delta, reject: int) -> int:
    rel = np.ascontiguousarray(relbits, np.uint8)
    dl = np.ascontiguousarray(delta, np.uint8).ravel()
    out = ctypes.c_void_p()
    _check(load().lbl_monitor_create(int(n_states), int(m), rel.ctypes.data if rel.size else None,
                                     dl.ctypes.data, int(reject), ctypes.byref(out)))
    return out.value


def lbl_monitor_free(mon) -> None:
    _check(load().lbl_monitor_free(mon))


def lbl_monitor_step(mon, d_L, n: int, d_next, d_viol, stream=None) -> None:
    _check(load().lbl_monitor_step(mon, _dev(d_L, "uint64", "L"), int(n), _dev(d_next, "uint64", "next"),
                                   _dev(d_viol, "uint16", "viol"), _stream(stream)))


def lbl_label(rm, d_O, n_props: int, d_L, mon=None, d_next=None, d_viol=None, cfg=None, stream=None) -> None:
    _check(load().lbl_label(rm, _dev(d_O, "uint64", "O"), int(n_props), _dev(d_L, "uint64", "L"), mon,
                            _dev(d_next, "uint64", "next"), _dev(d_viol, "uint16", "viol"), _cfg(cfg),
                            _stream(stream)))


def lbl_frame_transform_pyramid(rm, world, d_words, n_props: int, pose, d_O=None, stream=None) -> None:
    """The packed-word frame transform that also builds the roadmap's quadtree
    pyramid of its words (d_O may be None on z-order agent grids)."""
    w = _grid(world)
    _check(load().lbl_frame_transform_pyramid(rm, ctypes.byref(w), _words(d_words, n_props, "words"), int(n_props),
                                              _pose(pose), _dev(d_O, "uint64", "O"), _stream(stream)))


def lbl_label_pyramid(rm, n_props: int, d_L, mon=None, d_next=None, d_viol=None, cfg=None, stream=None) -> None:
    """Quadtree-form labels from the pyramid lbl_frame_transform_pyramid built."""
    _check(load().lbl_label_pyramid(rm, int(n_props), _dev(d_L, "uint64", "L"), mon, _dev(d_next, "uint64", "next"),
                                    _dev(d_viol, "uint16", "viol"), _cfg(cfg), _stream(stream)))


def lbl_label_blocks_noalloc(d_block_rowptr, d_block_id, d_block_mask, n_edges: int, d_O, n_cells: int,
                             n_props: int, d_L, stream=None) -> None:
    """Block-form labels from caller memory only; the working copy of O lives in
    the library's fixed device array (no allocation in the call)."""
    _check(load().lbl_label_blocks_noalloc(_dev(d_block_rowptr, "int64", "block_rowptr"),
                                           _dev(d_block_id, "uint32", "block_id"),
                                           _dev(d_block_mask, "uint64", "block_mask"), int(n_edges),
                                           _dev(d_O, "uint64", "O"), int(n_cells), int(n_props),
                                           _dev(d_L, "uint64", "L"), _stream(stream)))


def lbl_mma_probe(kind: int = 0, n: int = 64, reps: int = 4000, ctas_per_sm: int = 4):
    """Measured tcgen05 rate (TFLOP/s) and exactness of the accumulated counts."""
    t, ex = ctypes.c_double(0.0), ctypes.c_int32(0)
    _check(load().lbl_mma_probe(int(kind), int(n), int(reps), int(ctas_per_sm), ctypes.byref(t), ctypes.byref(ex)))
    return {"tflops": t.value, "exact": bool(ex.value)}


def lbl_roadmap_autotune(rm, d_O, n_props: int, d_L, mon=None, d_next=None, d_viol=None, reps: int = 5,
                         stream=None) -> dict:
    """Time every labeling variant on this frame; the fastest becomes the
    roadmap's AUTO choice for n_props.  Returns the chosen configuration."""
    c = lbl_config()
    _check(load().lbl_roadmap_autotune(rm, _dev(d_O, "uint64", "O"), int(n_props), mon, _dev(d_L, "uint64", "L"),
                                       _dev(d_next, "uint64", "next"), _dev(d_viol, "uint16", "viol"), int(reps),
                                       ctypes.byref(c), _stream(stream)))
    return {f: getattr(c, f) for f, _ in lbl_config._fields_}


def lbl_session_create(rm, world, n_props: int, mon=None, cfg=None) -> int:
    out = ctypes.c_void_p()
    w = _grid(world)
    _check(load().lbl_session_create(rm, ctypes.byref(w), int(n_props), mon, _cfg(cfg), ctypes.byref(out)))
    return out.value


def lbl_session_run(ss, h_planes, pose, h_L, h_next=None, h_viol=None, stream=None) -> None:
    _check(load().lbl_session_run(ss, _host(h_planes, np.uint8, "planes"), _pose(pose),
                                  _host(h_L, np.uint64, "L"), _host(h_next, np.uint64, "next"),
                                  _host(h_viol, np.uint16, "viol"), _stream(stream)))


def lbl_session_free(ss) -> None:
    _check(load().lbl_session_free(ss))


def lbl_batch_create(rms, n_props, mons=None, ctas_per_sm: int = 0) -> int:
    """Plan one batched launch over these roadmaps (one frame each)."""
    n = len(rms)
    R = (ctypes.c_void_p * n)(*rms)
    Pn = (ctypes.c_int32 * n)(*[int(p) for p in n_props])
    M = (ctypes.c_void_p * n)(*(mons if mons is not None else [None] * n))
    out = ctypes.c_void_p()
    _check(load().lbl_batch_create(n, R, Pn, M, int(ctas_per_sm), ctypes.byref(out)))
    return out.value


def lbl_batch_set_frames(b, frames) -> None:
    """frames: list of dicts with world, d_planes, pose, d_O, d_L[, d_next, d_viol]."""
    arr = (lbl_frame * len(frames))()
    for i, f in enumerate(frames):
        arr[i].world = _grid(f["world"])
        arr[i].d_planes = _dev(f["d_planes"], "uint8", "planes")
        arr[i].pose = _pose(f["pose"])
        arr[i].d_O = _dev(f["d_O"], "uint64", "O")
        arr[i].d_L = _dev(f["d_L"], "uint64", "L")
        arr[i].d_next = _dev(f.get("d_next"), "uint64", "next")
        arr[i].d_viol = _dev(f.get("d_viol"), "uint16", "viol")
    _check(load().lbl_batch_set_frames(b, arr))


def lbl_batch_launch(b, stages: int = 3, stream=None) -> None:
    """stages: LBL_STAGE_TRANSFORM | LBL_STAGE_LABEL (default both)."""
    _check(load().lbl_batch_launch(b, int(stages), _stream(stream)))


def lbl_batch_autotune(b, reps: int = 5, stream=None) -> list:
    """Per word-width class (1, 2, 4, 8 bytes): the chosen plan and its time."""
    out = (lbl_batch_tuning * LBL_BATCH_CLASSES)()
    _check(load().lbl_batch_autotune(b, int(reps), _stream(stream), out))
    return [{f: getattr(t, f) for f, _ in lbl_batch_tuning._fields_} for t in out]


def lbl_batch_free(b) -> None:
    _check(load().lbl_batch_free(b))


def lbl_server_create(rms, n_props, mons=None, lanes: int = 2, mem_budget: int = 1 << 30, max_batch: int = 128) -> int:
    """Start a serving loop over these resident roadmaps."""
    n = len(rms)
    R = (ctypes.c_void_p * n)(*rms)
    Pn = (ctypes.c_int32 * n)(*[int(p) for p in n_props])
    M = (ctypes.c_void_p * n)(*(mons if mons is not None else [None] * n))
    out = ctypes.c_void_p()
    _check(load().lbl_server_create(n, R, Pn, M, int(lanes), int(max_batch), int(mem_budget), ctypes.byref(out)))
    return out.value


def lbl_server_submit(srv, roadmap: int, world, h_planes, pose, h_L, h_next=None, h_viol=None,
                      arrival_ns: int = 0) -> int:
    """Queue one request; returns its ticket.  Host buffers must outlive it."""
    t = ctypes.c_int64()
    w = _grid(world)
    _check(load().lbl_server_submit(srv, int(roadmap), ctypes.byref(w), _host(h_planes, np.uint8, "planes"),
                                    _pose(pose), _host(h_L, np.uint64, "L"), _host(h_next, np.uint64, "next"),
                                    _host(h_viol, np.uint16, "viol"), int(arrival_ns), ctypes.byref(t)))
    return t.value


def lbl_server_wait(srv, ticket: int, timeout_ms: int = 10000) -> int:
    """Wait for a ticket; returns its latency in ns (arrival to host-visible)."""
    lat = ctypes.c_int64()
    _check(load().lbl_server_wait(srv, int(ticket), int(timeout_ms), ctypes.byref(lat)))
    return lat.value


def lbl_server_stats(srv) -> dict:
    v = [ctypes.c_int64() for _ in range(4)]
    _check(load().lbl_server_stats(srv, *[ctypes.byref(x) for x in v]))
    return dict(zip(("batches", "completed", "max_batch", "arena_used"), [x.value for x in v]))


def lbl_server_free(srv) -> None:
    _check(load().lbl_server_free(srv))
