"""Roadmaps built on the device (lbl_roadmap_rasterize) have exactly the
oracle's rows, and label exactly like uploaded ones."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_02612_gb300 as L  # noqa: E402


def _rows(rm):
    E, nnz = L.lbl_roadmap_info(rm)[:2]
    rp = torch.empty(E + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    L.lbl_roadmap_rows(rm, rp, ci)
    torch.cuda.synchronize()
    return rp.cpu().numpy(), ci.cpu().numpy()[:nnz]


def _arcs(rng, grid, n):
    arcs = synth.sample_arcs(rng, n, grid, kappa=(-0.8, 0.8), length=(0.0, 25.0))
    arcs[0, 3] = 0.0                       # straight
    arcs[1, 3:5] = (0.6, 2 * math.pi / 0.6 + 1)  # more than a full turn
    arcs[2, 3:5] = (-0.6, 1.2 * math.pi / 0.6)   # more than half a turn
    arcs[3, 0:2] = (grid.x0 - 15.0, grid.y0 + 3.0)  # starts outside, runs in
    arcs[4, 0:2] = (grid.x0 - 80.0, grid.y0 - 80.0)  # never meets the grid
    arcs[5, 3] = 1e-7                      # radius of curvature 10,000 km: fp64 only
    arcs[6, 4] = 0.0                       # a point
    return arcs


@pytest.mark.parametrize("order", [synth.MORTON, synth.ROWMAJOR])
@pytest.mark.parametrize("radius", [0.4, 1.3])
def test_rasterized_rows_within_dense_arc_sampling_bounds(order, radius):
    """eq. 7 without the oracle's closed form: the device rows lie between the
    cells whose centres are within the radius of densely sampled arc points
    (lower set) and those within radius + half the sampling step (upper set),
    so a mistake the rasteriser shared with the oracle's geometry would still
    show.  Rows are strictly increasing."""
    from test_oracle_pins import _arc_points, _centres
    rng = np.random.default_rng(70 + order + int(radius * 10))
    grid = synth.agent_grid(32, 0.25, order)
    arcs = _arcs(rng, grid, 60)
    arcs[7:, 3] = rng.uniform(-1.5, 1.5, size=arcs.shape[0] - 7)  # tighter turns than _arcs draws
    rm = L.lbl_roadmap_rasterize(grid, arcs, radius)
    try:
        rp, ci = _rows(rm)
    finally:
        L.lbl_roadmap_free(rm)
    cx, cy, keys = _centres(grid)
    for e in range(arcs.shape[0]):
        pts = _arc_points(arcs[e], 20000)
        h = arcs[e, 4] / (pts.shape[0] - 1)
        d = np.sqrt(((cx[:, None] - pts[None, :, 0]) ** 2 + (cy[:, None] - pts[None, :, 1]) ** 2).min(1))
        row = ci[rp[e]:rp[e + 1]]
        lower = set(keys[d <= radius - 1e-9].tolist())
        upper = set(keys[d <= radius + h / 2 + 1e-9].tolist())
        assert lower <= set(row.tolist()) <= upper, e
        assert (np.diff(row) > 0).all(), e


@pytest.mark.parametrize("order", [synth.MORTON, synth.ROWMAJOR])
@pytest.mark.parametrize("radius", [0.3, 1.0, 2.7])
def test_rasterized_rows_equal_the_oracle(order, radius):
    rng = np.random.default_rng(int(radius * 10) + order)
    grid = synth.agent_grid(64, 0.25, order)
    arcs = _arcs(rng, grid, 400)
    rm = L.lbl_roadmap_rasterize(grid, arcs, radius)
    try:
        rp, ci = _rows(rm)
        want_rp, want_ci = oracle.sweep(arcs, radius, grid)
        assert np.array_equal(rp, want_rp)
        assert np.array_equal(ci, want_ci)
    finally:
        L.lbl_roadmap_free(rm)


def test_rasterized_non_square_and_odd_grid():
    rng = np.random.default_rng(3)
    grid = synth.Grid(77, 41, 0.3, -9.0, -4.0, synth.ROWMAJOR)
    arcs = _arcs(rng, grid, 300)
    rm = L.lbl_roadmap_rasterize(grid, arcs, 0.9)
    try:
        rp, ci = _rows(rm)
        want_rp, want_ci = oracle.sweep(arcs, 0.9, grid)
        assert np.array_equal(rp, want_rp) and np.array_equal(ci, want_ci)
    finally:
        L.lbl_roadmap_free(rm)


def test_rasterized_full_size_rows_sampled_and_labels():
    """The 512x512 grid of the 1M-edge workload (200k arcs here): sampled rows
    equal the oracle's, and every label equals the uploaded roadmap's."""
    wl = synth.make("large", seed=13, edges=200_000)
    rm = L.lbl_roadmap_rasterize(wl.agent, wl.arcs, wl.radius, flags=L.LBL_UPLOAD_SECTOR)
    up = L.lbl_roadmap_upload(wl.agent, wl.rowptr, wl.colidx)
    try:
        rp, ci = _rows(rm)
        rows = np.random.default_rng(0).choice(wl.n_edges, 60, replace=False)
        for e in rows:
            orp, oci = oracle.sweep(wl.arcs[e:e + 1], wl.radius, wl.agent)
            assert np.array_equal(ci[rp[e]:rp[e + 1]], oci), e
        O = torch.empty(wl.agent.cells, dtype=torch.uint64, device="cuda")
        L.lbl_frame_transform(wl.world, torch.from_numpy(wl.planes).cuda(), wl.P, wl.pose, wl.agent, O)
        a = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
        b = torch.empty(wl.n_edges, dtype=torch.uint64, device="cuda")
        L.lbl_label(rm, O, wl.P, a, cfg=dict(algo=L.LBL_ALGO_SECTOR))
        L.lbl_label(up, O, wl.P, b)
        torch.cuda.synchronize()
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    finally:
        L.lbl_roadmap_free(rm)
        L.lbl_roadmap_free(up)


def test_rasterize_rejects_bad_arguments():
    grid = synth.agent_grid(16, 0.5, synth.MORTON)
    with pytest.raises(L.LblError):
        L.lbl_roadmap_rasterize(grid, np.array([[0.0, 0.0, 0.0, 0.1, -1.0]]), 1.0)
    with pytest.raises(L.LblError):
        L.lbl_roadmap_rasterize(grid, np.array([[0.0, 0.0, 0.0, 0.1, 1.0]]), 0.0)
    with pytest.raises(L.LblError) as ei:
        L.lbl_roadmap_rasterize(synth.agent_grid3(8, 0.5, 8, 0.1), np.zeros((1, 5)), 1.0)
    assert ei.value.code == L.LBL_EUNSUPPORTED
