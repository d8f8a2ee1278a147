"""Pins for the oracle's time-augmented (x, y, tau) workspace (Sec. 5): 3-D
z-order from Algorithm 1's tree descent, closed forms of the 3-D frame
transform (identity, time shift of eq. 13, quarter turns), double geometry at
random poses, reduction to the 2-D labels for a static world, and a continuous
brute force with moving objects.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import alg1_index


def _m3(ix, iy, it, n):
    return alg1_index(((ix + 0.5) / n, (iy + 0.5) / n, (it + 0.5) / n), (0, 0, 0), (1, 1, 1), 3 * int(math.log2(n)))


@pytest.mark.parametrize("n", [2, 4, 8])
def test_morton3_matches_algorithm1_with_three_axes(n):
    seen = set()
    for it in range(n):
        for iy in range(n):
            for ix in range(n):
                m = oracle.morton3(ix, iy, it)
                assert m == _m3(ix, iy, it, n)
                assert oracle.cell_index3(oracle.MORTON, n, n, ix, iy, it) == m
                seen.add(m)
    assert seen == set(range(n ** 3))


def test_rowmajor_index3():
    assert oracle.cell_index3(oracle.ROWMAJOR, 7, 5, 2, 3, 4) == (4 * 5 + 3) * 7 + 2


def _pack(vols, wx, wy, wt):
    P, D, H, W = vols.shape
    if not (0 <= wx < W and 0 <= wy < H and 0 <= wt < D):
        return 0
    word = 0
    for p in range(P):
        if vols[p, wt, wy, wx]:
            word |= 1 << p
    return word


def _expect3(vols, agent, mapper):
    O = np.zeros(agent.cells, np.uint64)
    for it in range(agent.d):
        for iy in range(agent.h):
            for ix in range(agent.w):
                wx, wy, wt = mapper(ix, iy, it)
                idx = (_m3(ix, iy, it, agent.w) if agent.order == oracle.MORTON
                       else (it * agent.h + iy) * agent.w + ix)
                O[idx] = _pack(vols, wx, wy, wt)
    return O


@pytest.mark.parametrize("order", [oracle.ROWMAJOR, oracle.MORTON])
@pytest.mark.parametrize("shift", [0, 3, -2, 9])
def test_frame3_time_shift_is_a_slab_shift(order, shift):
    """eq. 13 in t: querying at T = k * tres reads world slab it + k."""
    n, res, tres = 8, 0.5, 0.1
    rng = np.random.default_rng(shift + 10)
    vols = (rng.random((3, n, n, n)) < 0.3).astype(np.uint8)
    world = synth.world_grid3(n, n, res, n, tres)
    agent = synth.agent_grid3(n, res, n, tres, order)
    pose = (n * res / 2, n * res / 2, 0.0, shift * tres)
    O = oracle.frame_transform3(world, vols, pose, agent)
    assert np.array_equal(O, _expect3(vols, agent, lambda ix, iy, it: (ix, iy, it + shift)))


@pytest.mark.parametrize("quarter", [1, 2, 3])
def test_frame3_quarter_turns_permute_every_slab(quarter):
    n, res, tres = 8, 0.5, 0.2
    rng = np.random.default_rng(quarter)
    vols = (rng.random((2, n, n, n)) < 0.4).astype(np.uint8)
    world = synth.world_grid3(n, n, res, n, tres)
    agent = synth.agent_grid3(n, res, n, tres, oracle.MORTON)
    maps = [None,
            lambda ix, iy, it: (n - 1 - iy, ix, it),
            lambda ix, iy, it: (n - 1 - ix, n - 1 - iy, it),
            lambda ix, iy, it: (iy, n - 1 - ix, it)]
    O = oracle.frame_transform3(world, vols, (n * res / 2, n * res / 2, quarter * math.pi / 2, 0.0), agent)
    assert np.array_equal(O, _expect3(vols, agent, maps[quarter]))


def test_frame3_random_pose_matches_double_geometry():
    rng = np.random.default_rng(31)
    world = synth.Grid(20, 17, 0.3, 0.0, 0.0, synth.ROWMAJOR, 12, 0.07, -0.1)
    vols = (rng.random((4, 12, 17, 20)) < 0.5).astype(np.uint8)
    agent = synth.agent_grid3(8, 0.25, 8, 0.05, oracle.MORTON)
    for _ in range(5):
        pose = (2 + 2 * rng.random(), 2 + 2 * rng.random(), 2 * math.pi * rng.random(), 0.3 * rng.random() - 0.1)
        O = oracle.frame_transform3(world, vols, pose, agent)
        c, s = math.cos(pose[2]), math.sin(pose[2])
        checked = 0
        for it in range(agent.d):
            vt = (pose[3] + agent.t0 + (it + 0.5) * agent.tres - world.t0) / world.tres
            for iy in range(agent.h):
                for ix in range(agent.w):
                    cx = agent.x0 + (ix + 0.5) * agent.res
                    cy = agent.y0 + (iy + 0.5) * agent.res
                    u = (pose[0] + c * cx - s * cy - world.x0) / world.res
                    v = (pose[1] + s * cx + c * cy - world.y0) / world.res
                    if min(abs(u - round(u)), abs(v - round(v)), abs(vt - round(vt))) < 1e-6:
                        continue
                    assert int(O[_m3(ix, iy, it, 8)]) == _pack(vols, math.floor(u), math.floor(v), math.floor(vt))
                    checked += 1
        assert checked > 0.99 * agent.cells


def test_static_world_reduces_to_the_2d_labels():
    """With the same occupancy in every time slab and arcs that end within the
    horizon, an edge meets a proposition in (x, y, tau) iff its 2-D sweep does."""
    rng = np.random.default_rng(4)
    n, res, d, tres = 16, 0.5, 16, 0.25
    agent3 = synth.agent_grid3(n, res, d, tres, synth.MORTON)
    agent2 = synth.agent_grid(n, res, synth.MORTON)
    world3 = synth.world_grid3(n, n, res, d, tres)
    world2 = synth.world_grid(n, n, res)
    planes = synth.planes_discs(rng, 3, world2, fill=0.08)
    vols = np.repeat(planes[:, None, :, :], d, axis=1)
    arcs6 = synth.sample_arcs3(rng, 300, agent2, kappa=(-0.5, 0.5), length=(0.5, 6.0), speed=(2.0, 3.0))
    assert (arcs6[:, 4] / arcs6[:, 5] < d * tres).all()  # every arc ends within the horizon
    r3, c3 = synth.sweep3_csr(arcs6, 0.6, agent3)
    r2, c2 = synth.sweep_csr(arcs6[:, :5], 0.6, agent2)
    pose = (n * res / 2 + 0.3, n * res / 2 - 0.2, 0.4)
    L3 = oracle.label(r3, c3, oracle.frame_transform3(world3, vols, pose + (0.0,), agent3), 3)
    L2 = oracle.label(r2, c2, oracle.frame_transform(world2, planes, pose, agent2), 3)
    assert np.array_equal(L3, L2)
    assert (L2 != 0).any() and (L2 == 0).any()


def _arc_point(a, s):
    x, y, th, k = a[0], a[1], a[2], a[3]
    if abs(k) < 1e-9:
        return x + s * math.cos(th), y + s * math.sin(th)
    return x + (math.sin(th + k * s) - math.sin(th)) / k, y - (math.cos(th + k * s) - math.cos(th)) / k


def test_moving_objects_match_continuous_geometry():
    """eq. 7 in (x, y, tau): prop p labels edge e iff for some arc point reached
    during time slab it, an agent cell of that slab within the footprint radius
    lies over a world cell occupied by one of p's moving discs at the slab's
    mid time.  Lower/upper bounds from dense sampling; they differ only at ties."""
    rng = np.random.default_rng(8)
    n, res, d, tres = 8, 0.5, 8, 0.25
    agent = synth.agent_grid3(n, res, d, tres, synth.MORTON)
    world = synth.world_grid3(n, n, res, d, tres)
    discs = []
    vols = np.zeros((2, d, n, n), np.uint8)
    for p in range(2):
        for _ in range(3):
            prm = (rng.random() * 4, rng.random() * 4, 2 * rng.random() - 1, 2 * rng.random() - 1,
                   0.4 + 0.6 * rng.random())
            discs.append((p,) + prm)
            synth._load().synth_volume_moving_disc(synth._ptr(vols[p]), n, n, d, res, 0.0, 0.0, tres, 0.0, *prm)
    pose = (2.0, 2.0, 0.0, 0.0)  # agent grid = world grid, at T = 0
    arcs6 = synth.sample_arcs3(rng, 40, agent, kappa=(-0.6, 0.6), length=(0.5, 4.0), speed=(1.0, 3.0))
    radius = 0.55
    rp, ci = synth.sweep3_csr(arcs6, radius, agent)
    L = oracle.label(rp, ci, oracle.frame_transform3(world, vols, pose, agent), 2)

    def occupied(p, ix, iy, it):
        t = (it + 0.5) * tres
        cx, cy = (ix + 0.5) * res, (iy + 0.5) * res
        return any(q == p and (cx - (x + vx * t)) ** 2 + (cy - (y + vy * t)) ** 2 <= r * r
                   for (q, x, y, vx, vy, r) in discs)

    tight = 0
    for e in range(40):
        a = arcs6[e]
        lo, hi = np.zeros(2, bool), np.zeros(2, bool)
        for it in range(d):
            sa, sb = max(0.0, a[5] * it * tres), min(a[4], a[5] * (it + 1) * tres)
            if sa > sb:
                continue
            ss = np.linspace(sa, sb, 400)
            h = (sb - sa) / 399 if sb > sa else 0.0
            pts = np.array([_arc_point(a, s) for s in ss])
            for iy in range(n):
                for ix in range(n):
                    cx, cy = agent.x0 + (ix + 0.5) * res, agent.y0 + (iy + 0.5) * res
                    dist = np.sqrt(((pts - (cx, cy)) ** 2).sum(1)).min()
                    for p in range(2):
                        if occupied(p, ix, iy, it):
                            lo[p] |= dist <= radius - 1e-9
                            hi[p] |= dist <= radius + h / 2 + 1e-9
        got = np.array([(int(L[e]) >> p) & 1 for p in range(2)], bool)
        assert (lo <= got).all() and (got <= hi).all(), e
        tight += (lo == hi).all()
    assert tight >= 38
