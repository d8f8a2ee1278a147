"""Seeded synthetic inputs for the labeling path (tests and benchmark only).

This module draws random shape parameters with numpy and rasterises them with
the small C helper ``lbl_synth.c``.  It produces inputs only: roadmaps as CSR
rows of swept cells (the trajectory matrix M of eq. 10, stored as in eq. 11),
world-frame proposition planes, poses and monitor tables.  It holds none of the
labeling arithmetic, and both the oracle and the CUDA library consume what it
makes.

Workload recipes (the paper's own scenario, Sec. 5, is not public; these stand
in for it with the shapes it reports):

``plain``    64x64 agent grid at 0.5 m, 4 propositions of random discs
             (radius U[1,4] m) filled to >= 10 % each; 2,000 arcs with
             curvature U[-0.2,0.2] 1/m, length U[5,30] m, disc footprint 1 m.
``driving``  256x256 at 0.25 m, 32 propositions mixing lane bands (3.5 m wide),
             discs and convex polygons with fill U[2,20] %; 100,000 arcs with
             curvature U[-0.3,0.3], length U[5,40] m, footprint 1.2 m; the world
             grid is resampled at a random agent pose.
``large``    512x512 at 0.2 m, 64 propositions (mix as driving), 1,000,000 arcs
             (driving arc law), a 16-state safety monitor over 8 label bits.
``paper``    2048x1024 row-major at 0.1 m (2^21 cells, as in Sec. 5), two
             propositions: small moving discs at ~1 % fill and the outside of a
             circular lane loop at ~90 % fill; 1,097,702 short arcs whose mean
             sweep is ~0.0223 % of the cells (Table 1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbl_synth.c")
_LIB = os.path.join(_HERE, "_liblbl_synth.so")

ROWMAJOR = 0
MORTON = 1

_lib = None


def build(force: bool = False) -> str:
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
        lib.synth_sweep_build.restype = p
        lib.synth_sweep_build.argtypes = [i64, p, f64, i32, i32, f64, f64, f64, i32, i32, p]
        lib.synth_sweep_take.restype = ctypes.c_int
        lib.synth_sweep_take.argtypes = [p, p, p]
        lib.synth_free_build.restype = None
        lib.synth_free_build.argtypes = [p]
        lib.synth_arc_dist.restype = None
        lib.synth_arc_dist.argtypes = [p, i64, p, p]
        lib.synth_plane_disc.restype = i64
        lib.synth_plane_disc.argtypes = [p, i32, i32, f64, f64, f64, f64, f64, f64]
        lib.synth_plane_band.restype = i64
        lib.synth_plane_band.argtypes = [p, i32, i32, f64, f64, f64, p, f64]
        lib.synth_plane_polygon.restype = i64
        lib.synth_plane_polygon.argtypes = [p, i32, i32, f64, f64, f64, p, p, i32]
        lib.synth_sweep3_build.restype = p
        lib.synth_sweep3_build.argtypes = [i64, p, f64, i32, i32, i32, f64, f64, f64, f64, f64, i32, i32, p]
        lib.synth_volume_moving_disc.restype = i64
        lib.synth_volume_moving_disc.argtypes = [p, i32, i32, i32] + [f64] * 10
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass(frozen=True)
class Grid:
    """Occupancy-grid descriptor: ``w`` x ``h`` cells of side ``res`` metres whose
    cell (0,0) has its lower-left corner at (x0, y0) in the grid's own frame;
    ``order`` is the cell numbering (ROWMAJOR or MORTON).  A time-augmented grid
    (Sec. 5) has ``d`` > 1 time slabs of ``tres`` seconds starting at ``t0``."""
    w: int
    h: int
    res: float
    x0: float
    y0: float
    order: int = ROWMAJOR
    d: int = 1
    tres: float = 1.0
    t0: float = 0.0

    @property
    def cells(self) -> int:
        return self.w * self.h * self.d


def agent_grid(w: int, res: float, order: int = MORTON, h: int | None = None) -> Grid:
    """Agent-frame grid centred on the agent (agent at the centre, facing +x)."""
    h = w if h is None else h
    return Grid(w, h, float(res), -w * res / 2.0, -h * res / 2.0, order)


def world_grid(w: int, h: int, res: float) -> Grid:
    """World-frame grid with its corner at the world origin, row-major planes."""
    return Grid(w, h, float(res), 0.0, 0.0, ROWMAJOR)


# ------------------------------------------------------------------ roadmaps

def sample_arcs(rng: np.random.Generator, n: int, grid: Grid, kappa=(-0.2, 0.2), length=(5.0, 30.0)) -> np.ndarray:
    """n constant-curvature arcs (x, y, heading, curvature, length) with start
    points uniform over the grid's extent."""
    arcs = np.empty((n, 5), np.float64)
    arcs[:, 0] = grid.x0 + rng.random(n) * grid.w * grid.res
    arcs[:, 1] = grid.y0 + rng.random(n) * grid.h * grid.res
    arcs[:, 2] = rng.random(n) * 2.0 * math.pi
    arcs[:, 3] = kappa[0] + rng.random(n) * (kappa[1] - kappa[0])
    arcs[:, 4] = length[0] + rng.random(n) * (length[1] - length[0])
    return arcs


def sweep_csr(arcs: np.ndarray, radius: float, grid: Grid, threads: int = 0):
    """CSR rows (rowptr int64[E+1], colidx int32[nnz]) of the cells whose centre
    lies within ``radius`` of each arc; each row sorted ascending in the grid's
    cell order, no duplicates."""
    arcs = np.ascontiguousarray(arcs, np.float64)
    E = arcs.shape[0]
    nnz = ctypes.c_int64(0)
    h = _load().synth_sweep_build(E, _ptr(arcs), float(radius), grid.w, grid.h, grid.res, grid.x0, grid.y0,
                                  grid.order, int(threads), ctypes.byref(nnz))
    if not h:
        raise MemoryError("sweep rasterisation failed")
    rowptr = np.empty(E + 1, np.int64)
    colidx = np.empty(nnz.value, np.int32)
    if _load().synth_sweep_take(h, _ptr(rowptr), _ptr(colidx)) != 0:
        raise MemoryError("sweep copy failed")
    return rowptr, colidx


def sweep3_csr(arcs6: np.ndarray, radius: float, grid: Grid, threads: int = 0):
    """CSR rows of the time-augmented cells swept by arcs travelled at constant
    speed: arcs6[n] = (x, y, heading, curvature, length, speed); cell
    (ix, iy, it) is in the row iff a point reached during time slab it (closed)
    lies within ``radius`` of the cell's (x, y) centre."""
    arcs6 = np.ascontiguousarray(arcs6, np.float64)
    E = arcs6.shape[0]
    nnz = ctypes.c_int64(0)
    h = _load().synth_sweep3_build(E, _ptr(arcs6), float(radius), grid.w, grid.h, grid.d, grid.res, grid.x0,
                                   grid.y0, grid.tres, grid.t0, grid.order, int(threads), ctypes.byref(nnz))
    if not h:
        raise MemoryError("3-D sweep rasterisation failed")
    rowptr = np.empty(E + 1, np.int64)
    colidx = np.empty(nnz.value, np.int32)
    if _load().synth_sweep_take(h, _ptr(rowptr), _ptr(colidx)) != 0:
        raise MemoryError("sweep copy failed")
    return rowptr, colidx


def arc_distance(arc5, xy: np.ndarray) -> np.ndarray:
    """Distance from points xy[n,2] to one arc (the generator's closed form)."""
    arc5 = np.ascontiguousarray(arc5, np.float64)
    xy = np.ascontiguousarray(xy, np.float64)
    out = np.empty(xy.shape[0], np.float64)
    _load().synth_arc_dist(_ptr(arc5), xy.shape[0], _ptr(xy), _ptr(out))
    return out


# ------------------------------------------------------------ world planes

def _add_disc(plane, g: Grid, cx, cy, r):
    return _load().synth_plane_disc(_ptr(plane), g.w, g.h, g.res, g.x0, g.y0, cx, cy, r)


def _add_band(plane, g: Grid, arc5, half_width):
    a = np.ascontiguousarray(arc5, np.float64)
    return _load().synth_plane_band(_ptr(plane), g.w, g.h, g.res, g.x0, g.y0, _ptr(a), half_width)


def _add_polygon(plane, g: Grid, xs, ys):
    xs = np.ascontiguousarray(xs, np.float64)
    ys = np.ascontiguousarray(ys, np.float64)
    return _load().synth_plane_polygon(_ptr(plane), g.w, g.h, g.res, g.x0, g.y0, _ptr(xs), _ptr(ys), xs.shape[0])


def _fill_plane(rng, plane, g: Grid, kind: str, target: float, max_shapes: int = 20000):
    ext_x, ext_y = g.w * g.res, g.h * g.res
    filled = int(np.count_nonzero(plane))
    goal = target * g.cells
    shapes = 0
    while filled < goal and shapes < max_shapes:
        cx = g.x0 + rng.random() * ext_x
        cy = g.y0 + rng.random() * ext_y
        if kind == "disc":
            filled += _add_disc(plane, g, cx, cy, 1.0 + 3.0 * rng.random())
        elif kind == "band":
            th = rng.random() * 2.0 * math.pi
            length = 2.0 * math.hypot(ext_x, ext_y)
            kap = -0.01 + 0.02 * rng.random()
            arc = (cx - 0.5 * length * math.cos(th), cy - 0.5 * length * math.sin(th), th, kap, length)
            filled += _add_band(plane, g, arc, 1.75)
        elif kind == "poly":
            k = int(rng.integers(5, 9))
            ang = np.sort(rng.random(k) * 2.0 * math.pi)
            rad = 1.5 + 3.5 * rng.random()
            filled += _add_polygon(plane, g, cx + rad * np.cos(ang), cy + rad * np.sin(ang))
        else:
            raise ValueError(kind)
        shapes += 1
    return filled


def planes_discs(rng, P: int, g: Grid, fill: float = 0.10) -> np.ndarray:
    planes = np.zeros((P, g.h, g.w), np.uint8)
    for p in range(P):
        _fill_plane(rng, planes[p], g, "disc", fill)
    return planes


def planes_mixed(rng, P: int, g: Grid, fill=(0.02, 0.20)) -> np.ndarray:
    """Lane bands, discs and convex polygons; per-proposition fill U[fill]."""
    planes = np.zeros((P, g.h, g.w), np.uint8)
    kinds = ("band", "disc", "poly")
    for p in range(P):
        kind = kinds[int(rng.integers(0, 3))]
        target = fill[0] + (fill[1] - fill[0]) * rng.random()
        _fill_plane(rng, planes[p], g, kind, target)
    return planes


def planes_paper(rng, g: Grid) -> np.ndarray:
    """Two propositions shaped like Sec. 5's: moving vehicles (~1 % fill) and the
    outside of a circular nominal lane loop (~90 % fill)."""
    planes = np.zeros((2, g.h, g.w), np.uint8)
    _fill_plane(rng, planes[0], g, "disc", 0.01)
    cx, cy = g.x0 + g.w * g.res / 2, g.y0 + g.h * g.res / 2
    R = 0.39 * min(g.w, g.h) * g.res
    half = 0.05 * g.cells * g.res * g.res / (2 * math.pi * R)
    lane = np.zeros((g.h, g.w), np.uint8)
    _add_band(lane, g, (cx + R, cy, math.pi / 2, 1.0 / R, 2 * math.pi * R * 1.01), half)
    planes[1] = 1 - lane
    return planes


# ------------------------------------------------------------------ monitor

@dataclass
class Monitor:
    """Deterministic safety monitor: ``delta[q][letter]`` over letters formed
    from label bits ``relbits``; ``reject`` is the violation sink."""
    n_states: int
    m: int
    relbits: np.ndarray
    delta: np.ndarray
    reject: int


def random_monitor(rng, n_states: int, m: int, P: int, p_reject: float = 0.05) -> Monitor:
    relbits = rng.choice(P, size=m, replace=False).astype(np.uint8) if m else np.zeros(0, np.uint8)
    reject = n_states - 1
    delta = rng.integers(0, n_states - 1, size=(n_states, 1 << m)).astype(np.uint8)
    delta[rng.random((n_states, 1 << m)) < p_reject] = reject
    delta[reject, :] = reject
    return Monitor(n_states, m, relbits, delta, reject)


# ---------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    agent: Grid
    world: Grid
    P: int
    arcs: np.ndarray
    radius: float
    rowptr: np.ndarray
    colidx: np.ndarray
    planes: np.ndarray
    pose: tuple
    monitor: Monitor | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return self.rowptr.shape[0] - 1

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


RECIPES = {
    "plain": dict(n=64, res=0.5, P=4, edges=2000, kappa=(-0.2, 0.2), length=(5.0, 30.0), radius=1.0,
                  planes="discs", order=MORTON, pose="identity", monitor=None),
    "driving": dict(n=256, res=0.25, P=32, edges=100_000, kappa=(-0.3, 0.3), length=(5.0, 40.0), radius=1.2,
                    planes="mixed", order=MORTON, pose="random", monitor=None),
    "large": dict(n=512, res=0.2, P=64, edges=1_000_000, kappa=(-0.3, 0.3), length=(5.0, 40.0), radius=1.2,
                  planes="mixed", order=MORTON, pose="random", monitor=(16, 8)),
    "paper": dict(n=2048, h=1024, res=0.1, P=2, edges=1_097_702, kappa=(-0.3, 0.3), length=(2.0, 5.8),
                  radius=0.5, planes="paper", order=ROWMAJOR, pose="random", monitor=None),
}


def random_pose(rng, world: Grid):
    ext_x, ext_y = world.w * world.res, world.h * world.res
    return (world.x0 + ext_x * (0.25 + 0.5 * rng.random()),
            world.y0 + ext_y * (0.25 + 0.5 * rng.random()),
            2.0 * math.pi * rng.random())


def make(name: str, seed: int = 0, edges: int | None = None, threads: int = 0, **over) -> Workload:
    """Build one workload from its recipe; ``edges`` and keyword overrides
    shrink it for tests."""
    r = dict(RECIPES[name])
    r.update(over)
    if edges is not None:
        r["edges"] = edges
    rng = np.random.default_rng(seed)
    n, h = r["n"], r.get("h", r["n"])
    agent = agent_grid(n, r["res"], r["order"], h=h)
    world = world_grid(n, h, r["res"])
    P = r["P"]
    if r["planes"] == "discs":
        planes = planes_discs(rng, P, world)
    elif r["planes"] == "mixed":
        planes = planes_mixed(rng, P, world)
    else:
        planes = planes_paper(rng, world)
    if r["pose"] == "identity":
        pose = (world.x0 + world.w * world.res / 2, world.y0 + world.h * world.res / 2, 0.0)
    else:
        pose = random_pose(rng, world)
    arcs = sample_arcs(rng, r["edges"], agent, r["kappa"], r["length"])
    rowptr, colidx = sweep_csr(arcs, r["radius"], agent, threads)
    mon = None
    if r["monitor"]:
        mon = random_monitor(rng, r["monitor"][0], r["monitor"][1], P)
    return Workload(name, agent, world, P, arcs, r["radius"], rowptr, colidx, planes, pose, mon,
                    meta=dict(seed=seed, recipe=r))


# ------------------------------------------------------------- batched frames

@dataclass
class BatchFrame:
    """One frame of a batch: a roadmap (rows of a master pool), its world planes
    (the first P planes of the pool's), P and a pose."""
    agent: Grid
    world: Grid
    P: int
    rowptr: np.ndarray
    colidx: np.ndarray
    planes: np.ndarray
    pose: tuple
    grid_key: int

    @property
    def n_edges(self) -> int:
        return self.rowptr.shape[0] - 1

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def make_batch(seed: int = 0, frames: int = 64, edges=(10_000, 500_000), grids=(128, 256, 512), res: float = 0.25,
               props=(8, 64), threads: int = 0):
    """`frames` agents/frames with roadmaps of log-uniform size in `edges`, grids
    from `grids` at `res` (z-order), propositions U{props}; driving arc law.
    Roadmaps are the first rows of one master pool per grid size, planes the
    first P of one 64-proposition set per grid size."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(edges[0]), np.log(edges[1]), size=frames)).astype(np.int64)
    keys = rng.integers(0, len(grids), size=frames)
    Ps = rng.integers(props[0], props[1] + 1, size=frames)
    pools = {}
    for k in sorted(set(int(x) for x in keys)):
        n = grids[k]
        agent = agent_grid(n, res, MORTON)
        world = world_grid(n, n, res)
        n_max = int(sizes[keys == k].max())
        arcs = sample_arcs(rng, n_max, agent, (-0.3, 0.3), (5.0, 40.0))
        rowptr, colidx = sweep_csr(arcs, 1.2, agent, threads)
        planes = planes_mixed(rng, props[1], world)
        pools[k] = (agent, world, rowptr, colidx, planes)
    out = []
    for i in range(frames):
        agent, world, rowptr, colidx, planes = pools[int(keys[i])]
        E = int(sizes[i])
        rp = rowptr[: E + 1]
        out.append(BatchFrame(agent, world, int(Ps[i]), rp, colidx[: int(rp[-1])], planes[: int(Ps[i])],
                              random_pose(rng, world), int(keys[i])))
    return out


# ------------------------------------------------ time-augmented workspace

def agent_grid3(n: int, res: float, d: int, tres: float, order: int = MORTON) -> Grid:
    """Agent-frame (x, y, tau) grid: n x n cells centred on the agent, d time
    slabs of tres seconds from the query time 0."""
    return Grid(n, n, float(res), -n * res / 2.0, -n * res / 2.0, order, d, float(tres), 0.0)


def world_grid3(w: int, h: int, res: float, d: int, tres: float) -> Grid:
    return Grid(w, h, float(res), 0.0, 0.0, ROWMAJOR, d, float(tres), 0.0)


def volumes_paper3d(rng, g: Grid) -> np.ndarray:
    """Two time-augmented propositions shaped like Sec. 5's: moving vehicles
    (discs of 1-2.5 m moving at 5-15 m/s, ~1 % of the volume) and the outside of
    a circular lane loop (static, ~90 %)."""
    vols = np.zeros((2, g.d, g.h, g.w), np.uint8)
    goal = 0.01 * g.cells
    filled, shapes = 0, 0
    while filled < goal and shapes < 10000:
        cx = g.x0 + rng.random() * g.w * g.res
        cy = g.y0 + rng.random() * g.h * g.res
        sp = 5.0 + 10.0 * rng.random()
        hd = 2 * math.pi * rng.random()
        filled += _load().synth_volume_moving_disc(_ptr(vols[0]), g.w, g.h, g.d, g.res, g.x0, g.y0, g.tres, g.t0,
                                                   cx, cy, sp * math.cos(hd), sp * math.sin(hd),
                                                   1.0 + 1.5 * rng.random())
        shapes += 1
    cx, cy = g.x0 + g.w * g.res / 2, g.y0 + g.h * g.res / 2
    R = 0.39 * min(g.w, g.h) * g.res
    half = 0.05 * g.w * g.h * g.res * g.res / (2 * math.pi * R)
    lane = np.zeros((g.h, g.w), np.uint8)
    _add_band(lane, g, (cx + R, cy, math.pi / 2, 1.0 / R, 2 * math.pi * R * 1.01), half)
    vols[1] = (1 - lane)[None, :, :]
    return vols


def sample_arcs3(rng, n: int, grid: Grid, kappa=(-0.3, 0.3), length=(5.0, 30.0), speed=(8.0, 15.0)) -> np.ndarray:
    a = np.empty((n, 6), np.float64)
    a[:, :5] = sample_arcs(rng, n, grid, kappa, length)
    a[:, 5] = speed[0] + rng.random(n) * (speed[1] - speed[0])
    return a


def make_paper3d(seed: int = 0, edges: int = 1_097_702, n: int = 128, d: int = 128, threads: int = 0,
                 res: float = 0.4, tres: float = 0.05, radius: float = 0.8, order: int = MORTON) -> Workload:
    """The paper's time-augmented workspace (Sec. 5): 128 x 128 x 128 = 2^21
    cells of 0.4 m x 0.4 m x 0.05 s, two propositions, arcs travelled at
    8-15 m/s with a 0.8 m disc footprint."""
    rng = np.random.default_rng(seed)
    agent = agent_grid3(n, res, d, tres, order)
    world = world_grid3(n, n, res, d, tres)
    vols = volumes_paper3d(rng, world)
    pose = random_pose(rng, world) + (0.0,)
    arcs = sample_arcs3(rng, edges, agent)
    rowptr, colidx = sweep3_csr(arcs, radius, agent, threads)
    return Workload("paper3d", agent, world, 2, arcs, radius, rowptr, colidx, vols, pose, None,
                    meta=dict(seed=seed))
