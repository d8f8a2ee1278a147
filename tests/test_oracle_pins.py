"""Pins for the oracle: each test checks it against something other than itself
(values the paper prints, closed forms, invariants, brute force on continuous
geometry, the semantics of the LTL formula).  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from conftest import GOLDEN

U64 = np.uint64


def bits(word, P):
    return [(int(word) >> p) & 1 for p in range(P)]


def pack_rows(boolmat):
    """bool[n][P] -> uint64[n] (bit p = column p)."""
    n, P = boolmat.shape
    out = np.zeros(n, np.uint64)
    for p in range(P):
        out |= boolmat[:, p].astype(np.uint64) << U64(p)
    return out


def dense_from_csr(rowptr, colidx, n_cols):
    E = rowptr.shape[0] - 1
    A = np.zeros((E, n_cols), np.int64)
    for e in range(E):
        A[e, colidx[rowptr[e]:rowptr[e + 1]]] = 1
    return A


# ----------------------------------------------------------- eq. 11 example

def _read_csr_demo():
    rows, r, c = [], None, None
    with open(os.path.join(GOLDEN, "csr_demo.txt")) as f:
        mode = None
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line == "matrix":
                mode = "m"
                continue
            if line.startswith("r "):
                r = np.array([int(x) for x in line.split()[1:]], np.int64)
            elif line.startswith("c "):
                c = np.array([int(x) for x in line.split()[1:]], np.int32)
            elif mode == "m":
                rows.append([int(x) for x in line.split()])
    return np.array(rows, np.int64), r, c


def test_csr_demo_each_unit_proposition_reads_one_matrix_column():
    M, r, c = _read_csr_demo()
    # the printed CSR arrays describe the printed matrix
    assert (dense_from_csr(r, c, 5) == M).all()
    # P = e_j (one proposition occupying only cell j): L = column j of M
    for j in range(5):
        O = np.zeros(5, np.uint64)
        O[j] = 1
        L = oracle.label(r, c, O, 1)
        assert [int(x) for x in L] == list(M[:, j]), j
    # the example pairing in the paper's notation: P = e_3 gives L = (0,0,0,1,1)
    O = np.zeros(5, np.uint64)
    O[3] = 1
    assert [int(x) for x in oracle.label(r, c, O, 1)] == [0, 0, 0, 1, 1]


def test_csr_demo_multi_proposition_is_boolean_matmul():
    M, r, c = _read_csr_demo()
    rng = np.random.default_rng(3)
    Pm = rng.integers(0, 2, size=(5, 7))
    O = pack_rows(Pm)
    L = oracle.label(r, c, O, 7)
    expect = pack_rows((M @ Pm) > 0)
    assert (L == expect).all()
    assert (oracle.label_rows(np.array([4, 0, 2]), r, c, O, 7) == expect[[4, 0, 2]]).all()


# ------------------------------------------------- eq. 10 as an int matmul

@pytest.mark.parametrize("P", [1, 5, 64])
def test_label_equals_dense_integer_matmul(P):
    rng = np.random.default_rng(P)
    n_cells, E = 300, 120
    rowptr = [0]
    cols = []
    for e in range(E):
        k = int(rng.integers(0, 40)) if e % 17 else 0  # some empty rows
        cs = np.sort(rng.choice(n_cells, size=k, replace=False))
        cols.extend(cs.tolist())
        rowptr.append(len(cols))
    rowptr = np.array(rowptr, np.int64)
    colidx = np.array(cols, np.int32)
    Pm = (rng.random((n_cells, P)) < 0.03).astype(np.int64)
    O = pack_rows(Pm)
    A = dense_from_csr(rowptr, colidx, n_cells)
    expect = pack_rows((A @ Pm) > 0)
    assert (oracle.label(rowptr, colidx, O, P) == expect).all()
    assert (oracle.label(rowptr, colidx, O, P, threads=4) == expect).all()
    rows = rng.integers(0, E, 50)
    assert (oracle.label_rows(rows, rowptr, colidx, O, P) == expect[rows]).all()


def test_label_bits_at_or_above_P_are_zero():
    rowptr = np.array([0, 2], np.int64)
    colidx = np.array([0, 1], np.int32)
    O = np.array([0xFFFFFFFFFFFFFFFF, 0xF0], np.uint64)
    assert int(oracle.label(rowptr, colidx, O, 3)[0]) == 0b111
    assert int(oracle.label(rowptr, colidx, O, 64)[0]) == 0xFFFFFFFFFFFFFFFF
    assert int(oracle.label(rowptr, colidx, O, 0)[0]) == 0
    assert int(oracle.label(rowptr, colidx, O, 5, threads=3)[0]) == 0b11111


# ------------------------------------------------------ Algorithm 1 z-order

def alg1_index(x, lo, hi, d):
    """Sec. 4.1, Algorithm 1 (descend the space-partitioning tree), with the
    pivot step read as 0.5**(floor((i-1)/k)+2), the axis taken modulo k and
    the test read as 'query on the high side'."""
    k = len(x)
    z = [(x[i] - lo[i]) / (hi[i] - lo[i]) for i in range(k)]
    p = [0.5] * k
    n, j = 0, 0
    for i in range(1, d + 1):
        step = 0.5 ** ((i - 1) // k + 2)
        if z[j] >= p[j]:
            p[j] += step
            n += 2 ** (d - i)
        else:
            p[j] -= step
        j = (j + 1) % k
    return n


@pytest.mark.parametrize("N", [2, 8, 32])
def test_morton_matches_algorithm1_tree_descent(N):
    d = 2 * int(math.log2(N))
    seen = set()
    for iy in range(N):
        for ix in range(N):
            centre = ((ix + 0.5) / N, (iy + 0.5) / N)
            n = alg1_index(centre, (0, 0), (1, 1), d)
            assert oracle.morton(ix, iy) == n
            assert oracle.cell_index(oracle.MORTON, N, ix, iy) == n
            seen.add(n)
    assert seen == set(range(N * N))  # a bijection onto [0, N^2)


def test_morton_large_coordinates():
    # x bit i at 2i+1, y bit i at 2i, up to 16-bit coordinates
    assert oracle.morton(0xFFFF, 0) == int("10" * 16, 2)
    assert oracle.morton(0, 0xFFFF) == int("01" * 16, 2)
    assert oracle.morton(1 << 15, 1 << 15) == 3 << 30


def test_rowmajor_index():
    assert oracle.cell_index(oracle.ROWMAJOR, 37, 5, 3) == 3 * 37 + 5


# -------------------------------------------------------- frame transform

def _morton_ref(ix, iy, N):
    return alg1_index(((ix + 0.5) / N, (iy + 0.5) / N), (0, 0), (1, 1), 2 * int(math.log2(N)))


def _expect_from_map(planes, agent, mapper):
    """Expected O from a hand-derived map (ix,iy) -> world cell (wx,wy)."""
    P, Hw, Ww = planes.shape
    O = np.zeros(agent.w * agent.h, np.uint64)
    for iy in range(agent.h):
        for ix in range(agent.w):
            wx, wy = mapper(ix, iy)
            word = 0
            if 0 <= wx < Ww and 0 <= wy < Hw:
                for p in range(P):
                    if planes[p, wy, wx]:
                        word |= 1 << p
            idx = _morton_ref(ix, iy, agent.w) if agent.order == oracle.MORTON else iy * agent.w + ix
            O[idx] = word
    return O


@pytest.mark.parametrize("order", [oracle.ROWMAJOR, oracle.MORTON])
@pytest.mark.parametrize("quarter", [0, 1, 2, 3])
def test_frame_transform_quarter_turns_are_exact_permutations(order, quarter):
    N, res = 16, 0.5
    rng = np.random.default_rng(quarter)
    planes = (rng.random((5, N, N)) < 0.3).astype(np.uint8)
    world = synth.world_grid(N, N, res)
    agent = synth.agent_grid(N, res, order)
    pose = (N * res / 2, N * res / 2, quarter * math.pi / 2)
    # world point = pose + R(theta) * agent centre, worked out per quarter turn
    maps = [lambda ix, iy: (ix, iy),
            lambda ix, iy: (N - 1 - iy, ix),
            lambda ix, iy: (N - 1 - ix, N - 1 - iy),
            lambda ix, iy: (iy, N - 1 - ix)]
    O = oracle.frame_transform(world, planes, pose, agent)
    assert (O == _expect_from_map(planes, agent, maps[quarter])).all()


def test_frame_transform_whole_cell_translation_is_a_shift():
    N, res = 16, 0.25
    rng = np.random.default_rng(7)
    planes = (rng.random((3, 24, 20)) < 0.4).astype(np.uint8)  # non-square world
    world = synth.world_grid(20, 24, res)
    agent = synth.agent_grid(N, res, oracle.ROWMAJOR)
    for dx, dy in [(0, 0), (3, -2), (-5, 7), (12, 12)]:
        pose = (N * res / 2 + dx * res, N * res / 2 + dy * res, 0.0)
        O = oracle.frame_transform(world, planes, pose, agent)
        assert (O == _expect_from_map(planes, agent, lambda ix, iy: (ix + dx, iy + dy))).all()


def test_frame_transform_random_pose_matches_double_geometry():
    """General pose: compare with the world point computed in double from the
    rotation of each agent-cell centre; cells whose world coordinate lies within
    1e-6 cell of a boundary are skipped (the fixed-point reading may round
    either way there)."""
    rng = np.random.default_rng(11)
    world = synth.world_grid(40, 30, 0.3)
    planes = (rng.random((7, 30, 40)) < 0.5).astype(np.uint8)
    for order, N in [(oracle.MORTON, 32), (oracle.ROWMAJOR, 24)]:
        agent = synth.agent_grid(N, 0.2, order)
        for _ in range(6):
            pose = (rng.random() * 14 - 1, rng.random() * 11 - 1, rng.random() * 2 * math.pi)
            O = oracle.frame_transform(world, planes, pose, agent)
            ix, iy = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
            cx = agent.x0 + (ix + 0.5) * agent.res
            cy = agent.y0 + (iy + 0.5) * agent.res
            c, s = math.cos(pose[2]), math.sin(pose[2])
            px = pose[0] + c * cx - s * cy
            py = pose[1] + s * cx + c * cy
            u = (px - world.x0) / world.res
            v = (py - world.y0) / world.res
            wx, wy = np.floor(u).astype(int), np.floor(v).astype(int)
            amb = (np.abs(u - np.round(u)) < 1e-6) | (np.abs(v - np.round(v)) < 1e-6)
            checked = 0
            for y in range(N):
                for x in range(N):
                    if amb[y, x]:
                        continue
                    word = 0
                    if 0 <= wx[y, x] < world.w and 0 <= wy[y, x] < world.h:
                        for p in range(7):
                            if planes[p, wy[y, x], wx[y, x]]:
                                word |= 1 << p
                    idx = _morton_ref(x, y, N) if order == oracle.MORTON else y * N + x
                    assert int(O[idx]) == word, (pose, x, y)
                    checked += 1
            assert checked > 0.99 * N * N


def test_frame_transform_out_of_bounds_reads_zero():
    world = synth.world_grid(8, 8, 1.0)
    planes = np.ones((4, 8, 8), np.uint8)
    agent = synth.agent_grid(8, 1.0, oracle.ROWMAJOR)
    O = oracle.frame_transform(world, planes, (-100.0, -100.0, 0.3), agent)
    assert (O == 0).all()
    O = oracle.frame_transform(world, planes, (4.0, 4.0, 0.0), agent)
    assert (O == 0xF).all()
    # half off the negative side: agent x in [-4,4) maps to world x in [-4,4)
    O = oracle.frame_transform(world, planes, (0.0, 4.0, 0.0), agent).reshape(8, 8)
    assert (O[:, :4] == 0).all() and (O[:, 4:] == 0xF).all()


def test_frame_coeffs_quarter_turn_are_exact():
    world = synth.world_grid(16, 16, 0.5)
    agent = synth.agent_grid(16, 0.5, oracle.ROWMAJOR)
    q = oracle.frame_coeffs(world, agent, (4.0, 4.0, math.pi / 2))
    one = 1 << 32
    assert list(q[[0, 1, 3, 4]]) == [0, -one, one, 0]


# --------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def plain():
    return synth.make("plain", seed=1)


def _labels(wl, planes=None, pose=None):
    O = oracle.frame_transform(wl.world, wl.planes if planes is None else planes,
                               wl.pose if pose is None else pose, wl.agent)
    return O, oracle.label(wl.rowptr, wl.colidx, O, wl.P)


def test_invariant_empty_and_full_grids(plain):
    _, L0 = _labels(plain, planes=np.zeros_like(plain.planes))
    assert (L0 == 0).all()
    _, L1 = _labels(plain, planes=np.ones_like(plain.planes))
    nonempty = np.diff(plain.rowptr) > 0
    assert (L1[nonempty] == (1 << plain.P) - 1).all()
    assert (L1[~nonempty] == 0).all()


def test_invariant_monotone_in_occupancy(plain):
    rng = np.random.default_rng(5)
    more = plain.planes | (rng.random(plain.planes.shape) < 0.05).astype(np.uint8)
    _, L = _labels(plain)
    _, L2 = _labels(plain, planes=more)
    assert ((L & ~L2) == 0).all()
    assert (L2 != L).any()


def test_invariant_cell_permutation(plain):
    O, L = _labels(plain)
    rng = np.random.default_rng(9)
    perm = rng.permutation(O.shape[0])  # new index of old cell i is perm[i]
    O2 = np.zeros_like(O)
    O2[perm] = O
    col2 = perm[plain.colidx].astype(np.int32)
    rowptr = plain.rowptr
    for e in range(plain.n_edges):  # keep rows sorted, as the format requires
        col2[rowptr[e]:rowptr[e + 1]].sort()
    assert (oracle.label(rowptr, col2, O2, plain.P) == L).all()
    # and z-order vs row-major numbering of the same roadmap and world
    wl_rm = synth.make("plain", seed=1, order=synth.ROWMAJOR)
    _, L_rm = _labels(wl_rm)
    assert (L_rm == L).all()


@pytest.mark.parametrize("quarter", [1, 2, 3])
def test_invariant_quarter_turn_of_the_whole_scene(quarter):
    """Rotate every arc and the world by k*90 degrees about the grid centre:
    the swept-cell sets and the occupancy rotate cell-for-cell, so the labels
    are unchanged."""
    wl = synth.make("plain", seed=2, edges=400)
    N, res = wl.agent.w, wl.agent.res
    _, L = _labels(wl)
    ang = quarter * math.pi / 2
    c, s = round(math.cos(ang)), round(math.sin(ang))
    arcs = wl.arcs.copy()
    arcs[:, 0] = c * wl.arcs[:, 0] - s * wl.arcs[:, 1]
    arcs[:, 1] = s * wl.arcs[:, 0] + c * wl.arcs[:, 1]
    arcs[:, 2] = wl.arcs[:, 2] + ang
    rowptr, colidx = synth.sweep_csr(arcs, wl.radius, wl.agent)
    # planes are indexed [y][x] with y up: a counter-clockwise quarter turn about
    # the centre sends cell (x, y) to (N-1-y, x), i.e. new[y][x] = old[N-1-x][y]
    planes = np.stack([np.rot90(p, k=-quarter) for p in wl.planes])
    assert wl.pose[2] == 0.0  # the plain scene is seen at the identity pose
    O = oracle.frame_transform(wl.world, np.ascontiguousarray(planes), wl.pose, wl.agent)
    assert (oracle.label(rowptr, colidx, O, wl.P) == L).all()
    # the same rotation as a change of heading only (eq. 13): the world stays,
    # the agent turns by -90k degrees
    O3 = oracle.frame_transform(wl.world, wl.planes, (wl.pose[0], wl.pose[1], -ang), wl.agent)
    assert (oracle.label(rowptr, colidx, O3, wl.P) == L).all()
    assert N * res > 0


# ------------------------------------------- eq. 7 continuous brute force

def _arc_points(arc, n=10000):
    x, y, th, k, s = arc
    t = np.linspace(0.0, s, n)
    if abs(k) < 1e-9:
        return np.stack([x + t * math.cos(th), y + t * math.sin(th)], 1)
    return np.stack([x + (np.sin(th + k * t) - math.sin(th)) / k,
                     y - (np.cos(th + k * t) - math.cos(th)) / k], 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_labels_match_continuous_geometry(seed):
    """eq. 7: prop p labels edge e iff some agent cell whose centre is within the
    footprint radius of the arc lies over a world cell whose centre is inside one
    of p's discs.  Evaluated here from the shapes by dense arc sampling and
    direct rotation, and compared with generator + oracle as lower/upper bounds
    that differ only at numerical ties."""
    rng = np.random.default_rng(100 + seed)
    N, res = 16, 0.5
    agent = synth.agent_grid(N, res, synth.MORTON if seed != 1 else synth.ROWMAJOR)
    world = synth.world_grid(20, 18, 0.45)
    P = 3
    discs = [[(rng.random() * 9, rng.random() * 8, 0.4 + rng.random() * 1.5) for _ in range(4)] for _ in range(P)]
    planes = np.zeros((P, world.h, world.w), np.uint8)
    for p in range(P):
        for (cx, cy, r) in discs[p]:
            synth._add_disc(planes[p], world, cx, cy, r)
    pose = (4.5 + rng.random(), 4.0 + rng.random(), rng.random() * 2 * math.pi)
    E, radius = 48, 0.6
    arcs = synth.sample_arcs(rng, E, agent, kappa=(-0.6, 0.6), length=(0.5, 9.0))
    arcs[0, 3] = 0.0  # one straight edge
    rowptr, colidx = synth.sweep_csr(arcs, radius, agent)
    O = oracle.frame_transform(world, planes, pose, agent)
    L = oracle.label(rowptr, colidx, O, P)

    ix, iy = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    cx = (agent.x0 + (ix + 0.5) * res).ravel()
    cy = (agent.y0 + (iy + 0.5) * res).ravel()
    c, s = math.cos(pose[2]), math.sin(pose[2])
    u = (pose[0] + c * cx - s * cy - world.x0) / world.res
    v = (pose[1] + s * cx + c * cy - world.y0) / world.res

    def occupied(wx, wy, p):
        if not (0 <= wx < world.w and 0 <= wy < world.h):
            return False
        px, py = world.x0 + (wx + 0.5) * world.res, world.y0 + (wy + 0.5) * world.res
        return any((px - dx) ** 2 + (py - dy) ** 2 <= r * r for (dx, dy, r) in discs[p])

    # per agent cell: props surely / possibly present under it
    sure = np.zeros((N * N, P), bool)
    maybe = np.zeros((N * N, P), bool)
    for i in range(N * N):
        cands_x = {math.floor(u[i])} | ({math.floor(u[i] + 1e-9), math.floor(u[i] - 1e-9)})
        cands_y = {math.floor(v[i])} | ({math.floor(v[i] + 1e-9), math.floor(v[i] - 1e-9)})
        for p in range(P):
            vals = [occupied(a, b, p) for a in cands_x for b in cands_y]
            sure[i, p] = all(vals)
            maybe[i, p] = any(vals)
    tight = 0
    for e in range(E):
        pts = _arc_points(arcs[e])
        h = arcs[e, 4] / (pts.shape[0] - 1)
        d = np.sqrt(((cx[:, None] - pts[None, :, 0]) ** 2 + (cy[:, None] - pts[None, :, 1]) ** 2).min(1))
        inside = d <= radius - 1e-9
        possible = d <= radius + h / 2 + 1e-9
        lo = np.any(sure[inside], axis=0) if inside.any() else np.zeros(P, bool)
        hi = np.any(maybe[possible], axis=0) if possible.any() else np.zeros(P, bool)
        got = np.array(bits(L[e], P), bool)
        assert (lo <= got).all() and (got <= hi).all(), (e, lo, got, hi)
        tight += (lo == hi).all()
    assert tight >= E - 2  # the bounds pin almost every edge exactly


def test_generator_rows_match_brute_force_cell_test():
    """Swept rows equal the set of in-grid cell centres within the radius of the
    densely sampled arc (ties within the sampling error excluded)."""
    rng = np.random.default_rng(21)
    agent = synth.agent_grid(32, 0.25, synth.MORTON)
    arcs = synth.sample_arcs(rng, 40, agent, kappa=(-1.5, 1.5), length=(0.2, 25.0))
    rowptr, colidx = synth.sweep_csr(arcs, 0.3, agent)
    N = agent.w
    ix, iy = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    cx = (agent.x0 + (ix + 0.5) * agent.res).ravel()
    cy = (agent.y0 + (iy + 0.5) * agent.res).ravel()
    keys = np.array([_morton_ref(x, y, N) for y in range(N) for x in range(N)])
    for e in range(40):
        pts = _arc_points(arcs[e], 20000)
        h = arcs[e, 4] / (pts.shape[0] - 1)
        d = np.sqrt(((cx[:, None] - pts[None, :, 0]) ** 2 + (cy[:, None] - pts[None, :, 1]) ** 2).min(1))
        row = set(colidx[rowptr[e]:rowptr[e + 1]].tolist())
        assert set(keys[d <= 0.3 - 1e-9].tolist()) <= row
        assert row <= set(keys[d <= 0.3 + h / 2 + 1e-9].tolist())
        assert list(colidx[rowptr[e]:rowptr[e + 1]]) == sorted(row)


# ------------------------------------------------------------------ monitor

def _read_split_lane():
    delta, traces, n_states, reject = {}, [], None, None
    with open(os.path.join(GOLDEN, "split_lane.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t = line.split()
            if t[0] == "states":
                n_states = int(t[1])
            elif t[0] == "reject":
                reject = int(t[1])
            elif t[0] == "delta":
                delta[int(t[1])] = [int(t[2]), int(t[3])]
            elif t[0] == "trace":
                arrow = t.index("->")
                traces.append(([int(x) for x in t[1:arrow]], [int(x) for x in t[arrow + 1:]]))
    table = np.array([delta[q] for q in range(n_states)], np.uint8)
    return n_states, reject, table, traces


def _run(nxt_word, q):
    return (int(nxt_word) >> (4 * q)) & 15


def test_split_lane_monitor_table_and_fig1_trace():
    n_states, reject, table, traces = _read_split_lane()
    bit = 5  # split_lane is proposition 5 of an 8-proposition label word
    relbits = np.array([bit], np.uint8)
    for labels, states in traces:
        L = np.array([(1 << bit) if x else 0 for x in labels], np.uint64)
        nxt, viol = oracle.monitor(n_states, 1, relbits, table, reject, L)
        q, seen = 0, []
        for e in range(len(labels)):
            q = _run(nxt[e], q)
            seen.append(q)
        assert seen == states
    # every (state, letter) pair of the hand-derived table
    for q in range(n_states):
        for letter in range(2):
            L = np.array([(letter << bit) | 0b10000001], np.uint64)  # other bits must not matter
            nxt, viol = oracle.monitor(n_states, 1, relbits, table, reject, L)
            assert _run(nxt[0], q) == table[q, letter]
            assert bool(int(viol[0]) >> q & 1) == (table[q, letter] == reject)


def test_split_lane_monitor_rejects_exactly_the_bad_prefixes():
    """phi = always(split_lane -> next not split_lane): a finite label sequence is
    a bad prefix iff two consecutive labels both contain split_lane."""
    n_states, reject, table, _ = _read_split_lane()
    rng = np.random.default_rng(0)
    bit = 17
    for _ in range(300):
        n = int(rng.integers(1, 12))
        seq = rng.random(n) < 0.35
        L = np.array([(rng.integers(0, 1 << 16) & ~(1 << bit)) | (int(x) << bit) for x in seq], np.uint64)
        nxt, viol = oracle.monitor(n_states, 1, np.array([bit], np.uint8), table, reject, L)
        q, rejected = 0, False
        for e in range(n):
            rejected |= bool(int(viol[e]) >> q & 1)
            q = _run(nxt[e], q)
        bad = any(seq[i] and seq[i + 1] for i in range(n - 1))
        assert rejected == bad == (q == reject)


def test_two_proposition_monitor_letter_order():
    """phi = always(a -> next b) over label bits a=9, b=2: the table is built from
    the letter as a set (bit j of the letter <-> relbits[j]); the monitor rejects
    exactly when some label with a is followed by a label without b."""
    a, b = 9, 2
    relbits = np.array([a, b], np.uint8)
    # states: 0 no obligation, 1 'next label must contain b', 2 reject
    table = np.zeros((3, 4), np.uint8)
    for letter in range(4):
        has = {relbits[j] for j in range(2) if letter >> j & 1}
        table[0, letter] = 1 if a in has else 0
        table[1, letter] = 2 if b not in has else (1 if a in has else 0)
        table[2, letter] = 2
    rng = np.random.default_rng(1)
    for _ in range(300):
        n = int(rng.integers(1, 10))
        A = rng.random(n) < 0.4
        B = rng.random(n) < 0.6
        L = np.array([(int(x) << a) | (int(y) << b) | (1 << 40) for x, y in zip(A, B)], np.uint64)
        nxt, viol = oracle.monitor(3, 2, relbits, table, 2, L)
        q = 0
        for e in range(n):
            q = _run(nxt[e], q)
        bad = any(A[i] and not B[i + 1] for i in range(n - 1))
        assert (q == 2) == bad


def test_monitor_unused_state_fields_are_zero():
    rng = np.random.default_rng(4)
    table = rng.integers(0, 5, size=(5, 8)).astype(np.uint8)
    L = rng.integers(0, 2**62, size=100, dtype=np.uint64)
    nxt, viol = oracle.monitor(5, 3, np.array([0, 61, 33], np.uint8), table, 4, L)
    assert ((nxt >> U64(20)) == 0).all()
    assert ((viol >> np.uint16(5)) == 0).all()


# ------------------------------------------------ swept-cell rasteriser

def _centres(grid):
    N = grid.w
    ix, iy = np.meshgrid(np.arange(N), np.arange(grid.h), indexing="xy")
    cx = (grid.x0 + (ix + 0.5) * grid.res).ravel()
    cy = (grid.y0 + (iy + 0.5) * grid.res).ravel()
    if grid.order == synth.MORTON:
        keys = np.array([_morton_ref(x, y, N) for y in range(grid.h) for x in range(N)])
    else:
        keys = (iy * N + ix).ravel()
    return cx, cy, keys


@pytest.mark.parametrize("order", [synth.MORTON, synth.ROWMAJOR])
def test_oracle_sweep_matches_dense_arc_sampling(order):
    """eq. 7 with a disc footprint: a cell is in row e iff its centre is within
    the radius of some point of the arc (dense sampling bounds the distance
    from both sides; only ties are left undecided)."""
    rng = np.random.default_rng(50 + order)
    grid = synth.agent_grid(32, 0.25, order)
    arcs = synth.sample_arcs(rng, 50, grid, kappa=(-1.5, 1.5), length=(0.1, 30.0))
    arcs[0, 3] = 0.0          # straight
    arcs[1, 3:5] = (1.2, 12.0)  # more than a full turn
    arcs[2, 0:2] = (-20.0, 0.0)  # starts outside the grid
    rowptr, colidx = oracle.sweep(arcs, 0.4, grid)
    cx, cy, keys = _centres(grid)
    for e in range(50):
        pts = _arc_points(arcs[e], 20000)
        h = arcs[e, 4] / (pts.shape[0] - 1)
        d = np.sqrt(((cx[:, None] - pts[None, :, 0]) ** 2 + (cy[:, None] - pts[None, :, 1]) ** 2).min(1))
        row = colidx[rowptr[e]:rowptr[e + 1]]
        assert set(keys[d <= 0.4 - 1e-9].tolist()) <= set(row.tolist()) <= set(keys[d <= 0.4 + h / 2 + 1e-9].tolist())
        assert (np.diff(row) > 0).all()


def test_oracle_sweep_full_turn_is_an_annulus():
    grid = synth.agent_grid(64, 0.2, synth.ROWMAJOR)
    k, r = 0.4, 0.5
    arc = np.array([[0.0, -2.5, 0.0, k, 2 * math.pi / k + 0.3]])  # circle of radius 2.5 centred at the origin
    rowptr, colidx = oracle.sweep(arc, r, grid)
    cx, cy, keys = _centres(grid)
    ring = np.abs(np.hypot(cx, cy) - 1 / k) <= r
    tie = np.abs(np.abs(np.hypot(cx, cy) - 1 / k) - r) < 1e-9
    got = np.zeros(grid.cells, bool)
    got[colidx] = True
    assert (got[~tie] == ring[~tie]).all()


def test_oracle_sweep_zero_length_arc_is_its_start_point():
    grid = synth.agent_grid(32, 0.25, synth.ROWMAJOR)
    cx, cy, keys = _centres(grid)
    for k in (0.0, 0.7, -2.0):
        arc = np.array([[0.3, -0.6, 1.0, k, 0.0]])
        rowptr, colidx = oracle.sweep(arc, 0.5, grid)
        d = np.hypot(cx - 0.3, cy + 0.6)
        assert set(colidx.tolist()) == set(keys[d <= 0.5].tolist())


def test_oracle_sweep_agrees_with_the_generator_away_from_ties():
    rng = np.random.default_rng(77)
    grid = synth.agent_grid(64, 0.5, synth.MORTON)
    arcs = synth.sample_arcs(rng, 200, grid)
    r1, c1 = oracle.sweep(arcs, 1.0, grid)
    r2, c2 = synth.sweep_csr(arcs, 1.0, grid)
    assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
